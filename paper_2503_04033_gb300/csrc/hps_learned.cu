// Learned low-rank correction of the leaf DtN map (an extension beyond the
// paper, whose DtN maps are always computed exactly).
//
// A three-layer MLP maps the sampled coefficient b of a box (all p^3 grid
// values, input x = 2 (b - 1)) to factors U, V in R^{m x r}; the predicted map
// is T_hat = T0 + s U V^T, with T0 the DtN map of the same box for b = 1 and s
// a fixed target scale.  Training minimises L = mean over boxes and entries of
// (U V^T - (T - T0)/s)^2.
//
// Layers (row-major, weights [in][out]):
//   a1 = relu(x W0 + c0),  a2 = relu(a1 W1 + c1),  y = a2 W2 + c2,
//   U = y[:, 0 : m r] as [m][r],  V = y[:, m r : 2 m r] as [m][r].
//
// Every product runs on the tensor cores (tcgen05 kind::f16, BF16 operands,
// FP32 accumulation in TMEM; tc_gemm_bf16 computes C = -A B^T with both
// operands K-major).  Weights are kept in FP32 (master copy, Adam moments)
// with two BF16 copies holding -W^T (forward products) and -W (back
// propagation), so that C = -A B^T gives +A W.  Each product's other operand
// is rounded to BF16 where it is made: by k_act, which adds the bias, applies
// ReLU or the ReLU mask and writes the BF16 copies (row-major, and transposed
// with the batch as the K index for the weight gradients).  Every BF16 buffer
// has its K extent padded to a multiple of 8 with zeros (16-byte TMA rows).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hps_internal.h"

namespace {
inline int pad8(int v) { return (v + 7) & ~7; }
}

struct hps_mlp {
    int device = 0;
    int dims[4] = {0, 0, 0, 0};        // n_in, h1, h2, n_out
    int kp[4] = {0, 0, 0, 0};          // dims padded to multiples of 8 (BF16 K extents)
    int m = 0, rank = 0, rp = 0, mp = 0;   // rank, m padded to multiples of 8
    float* W[3] = {};                  // FP32 master weights [in][out]
    float* c[3] = {};                  // biases [out]
    __nv_bfloat16* WnT[3] = {};        // -W^T [out][kp(in)] (forward products)
    __nv_bfloat16* Wn[3] = {};         // -W [in][kp(out)] (back propagation; layers 1, 2)
    float* gW[3] = {};
    float* gc[3] = {};
    float* mW[3] = {};
    float* vW[3] = {};
    float* mc[3] = {};
    float* vc[3] = {};
    long long adam_t = 0;
    // forward buffers (capacity cap_f boxes)
    int cap_f = 0;
    __nv_bfloat16 *xb = nullptr, *a1b = nullptr, *a2b = nullptr;   // [B][kp]
    float *z = nullptr, *y = nullptr;                            // [B][max(h1, h2)], [B][n_out]
    // training buffers (capacity cap_t boxes; transposed copies [F][pad8(cap_t)])
    int cap_t = 0;
    __nv_bfloat16 *xT = nullptr, *a1T = nullptr, *a2T = nullptr;
    __nv_bfloat16 *Un = nullptr, *Vb = nullptr, *UT = nullptr, *VT = nullptr;   // [B][m][rp], [B][r][mp]
    float* E = nullptr;                                                        // [B][m][m]
    __nv_bfloat16 *Gn = nullptr, *GnT = nullptr;                               // [B][m][mp]
    float *dy = nullptr, *d2 = nullptr, *d1 = nullptr;                         // [B][F]
    __nv_bfloat16 *dyb = nullptr, *d2b = nullptr;                              // [B][kp]
    __nv_bfloat16 *dyTn = nullptr, *d2Tn = nullptr, *d1Tn = nullptr;           // -transposes [F][pad8(B)]
    double* loss = nullptr;
    double* lpart = nullptr;           // per (box, 32-row tile) sums of e^2 [cap_t][ceil(m / 32)]
    float* part = nullptr;             // split-K partial products
    long long part_cap = 0;
    float* dtarget = nullptr;          // hps_mlp_grad's FP32 targets (T - T0)/s
    size_t dcap = 0;
};

namespace {

// Elementwise stage after a product, on 32 x 32 tiles of an R x C matrix
// (batch entry blockIdx.z): v = Z (in_kind 0) or float(2 (Z - 1)) (in_kind
// 1, the network input from b), then + bias[c], relu, and zero where
// mask[r][c] (BF16) is not positive.  Writes v to Zo (FP32, may alias Z),
// sN * bf16(v) to Nb [R][ldn] (columns C..ldn-1 zero) and sT * bf16(v) to
// Tb [C][ldt] transposed (columns R..ldt-1 zero); each output optional.
template <typename TI>
__global__ void __launch_bounds__(256)
k_act(int R, int C, const TI* __restrict__ Z, long long ldz, long long sZ, int in_kind,
      const float* __restrict__ bias, int relu, const __nv_bfloat16* __restrict__ mask, long long ldmask,
      long long sMask, float* Zo, long long ldzo, long long sZo, __nv_bfloat16* __restrict__ Nb, long long ldn,
      long long sN_, float sgnN, __nv_bfloat16* __restrict__ Tb, long long ldt, long long sT_, float sgnT)
{
    __shared__ float tile[32][33];
    const long long z = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int cc = c0 + tx;
    // all loads first (Zo may alias Z), then the stores
    float v[4];
    bool in[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 8 * i;
        in[i] = r < R && cc < C;
        v[i] = 0.0f;
        if (in[i]) {
            const TI zin = Z[z * sZ + (long long)r * ldz + cc];
            v[i] = in_kind == 1 ? float(2.0 * ((double)zin - 1.0)) : float(zin);
            if (bias) v[i] += bias[cc];
            if (relu) v[i] = fmaxf(v[i], 0.0f);
            if (mask && !(__bfloat162float(mask[z * sMask + (long long)r * ldmask + cc]) > 0.0f)) v[i] = 0.0f;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int rr = ty + 8 * i, r = r0 + rr;
        if (in[i] && Zo) Zo[z * sZo + (long long)r * ldzo + cc] = v[i];
        tile[rr][tx] = v[i];
        if (Nb && r < R && cc < ldn) Nb[z * sN_ + (long long)r * ldn + cc] = __float2bfloat16_rn(sgnN * v[i]);
    }
    if (!Tb) return;
    __syncthreads();
    for (int cr = ty; cr < 32; cr += 8) {
        const int tc = c0 + cr, r = r0 + tx;
        if (tc < C && r < ldt) Tb[z * sT_ + (long long)tc * ldt + r] = __float2bfloat16_rn(sgnT * tile[tx][cr]);
    }
}

template <typename TI>
void act(int R, int C, const TI* Z, long long ldz, long long sZ, int in_kind, const float* bias, int relu,
         const __nv_bfloat16* mask, long long ldmask, long long sMask, float* Zo, long long ldzo, long long sZo,
         __nv_bfloat16* Nb, long long ldn, long long sN_, float sgnN, __nv_bfloat16* Tb, long long ldt, long long sT_,
         float sgnT, int batch, cudaStream_t st)
{
    // the tiles cover the padded extents of both outputs
    const long long rows = std::max<long long>(R, Tb ? ldt : R), cols = std::max<long long>(C, Nb ? ldn : C);
    dim3 grd((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)batch);
    k_act<TI><<<grd, dim3(32, 8), 0, st>>>(R, C, Z, ldz, sZ, in_kind, bias, relu, mask, ldmask, sMask, Zo, ldzo, sZo,
                                           Nb, ldn, sN_, sgnN, Tb, ldt, sT_, sgnT);
}

// Loss stage of box blockIdx.y, tile row blockIdx.x (32 rows), walking the
// tile columns: e = E - D (FP32, D the box's target (T - T0)/s), the block's
// sum of e^2 to part[box][tile row] (FP32 per thread, FP64 across them),
// and G = g e written as -bf16(G) to Gn [m][ldg] and -bf16(G^T) to GnT
// [m][ldg] (columns m..ldg-1 zero).
__global__ void __launch_bounds__(256)
k_loss(int m, const float* __restrict__ E, const float* __restrict__ D, float g, __nv_bfloat16* __restrict__ Gn,
       __nv_bfloat16* __restrict__ GnT, int ldg, double* __restrict__ part)
{
    __shared__ float tile[32][33];
    __shared__ double red[8];
    const long long z = blockIdx.y, mm2 = (long long)m * m, gpl = (long long)m * ldg;
    const int r0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float acc = 0.0f;
    for (int c0 = 0; c0 < ldg; c0 += 32) {
        const int cc = c0 + tx;
        float e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = r0 + ty + 8 * i;
            e[i] = 0.0f;
            if (r < m && cc < m) {
                const long long ix = z * mm2 + (long long)r * m + cc;
                e[i] = E[ix] - D[ix];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int rr = ty + 8 * i, r = r0 + rr;
            acc = fmaf(e[i], e[i], acc);
            const float gv = g * e[i];
            tile[rr][tx] = gv;
            if (r < m && cc < ldg) Gn[z * gpl + (long long)r * ldg + cc] = __float2bfloat16_rn(-gv);
        }
        __syncthreads();
        for (int cr = ty; cr < 32; cr += 8) {
            const int tc = c0 + cr, r = r0 + tx;
            if (tc < m && r < ldg) GnT[z * gpl + (long long)tc * ldg + r] = __float2bfloat16_rn(-tile[tx][cr]);
        }
        __syncthreads();
    }
    double dacc = acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, off);
    if (tx == 0) red[ty] = dacc;
    __syncthreads();
    if (tx == 0 && ty == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[z * gridDim.x + blockIdx.x] = t;
    }
}

// D = float((T - T0) / s) for every box (T0 [m][m] shared).
__global__ void k_target(long long n, long long mm2, const double* __restrict__ T, const double* __restrict__ T0,
                         double inv_s, float* __restrict__ D)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        D[i] = float((T[i] - T0[i % mm2]) * inv_s);
}

// *out = sum of part[0..n) in a fixed order (one CTA).
__global__ void k_sum(int n, const double* __restrict__ part, double* __restrict__ out)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// C[i] = sum over s < S of P[s][i] (split-K partial products), i < n.
__global__ void k_reduce_splits(long long n, int S, const float* __restrict__ P, float* __restrict__ C)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int q = 0; q < S; ++q) acc += P[q * n + i];
        C[i] = acc;
    }
}

// g[j] = sum over rows of d[r][j]
__global__ void k_colsum(int rows, int cols, const float* __restrict__ d, float* __restrict__ g)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float acc = 0.0f;
    for (int r = 0; r < rows; ++r) acc += d[(long long)r * cols + j];
    g[j] = acc;
}

__global__ void k_adam(long long n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ mo,
                       float* __restrict__ ve, float lr, float b1, float b2, float eps, float bc1, float bc2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float m = b1 * mo[i] + (1.0f - b1) * gi;
        const float v = b2 * ve[i] + (1.0f - b2) * gi * gi;
        mo[i] = m;
        ve[i] = v;
        w[i] = w[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    }
}

__global__ void k_split_uv(int B, int mr, const float* __restrict__ y, int ldy, double* __restrict__ U,
                           double* __restrict__ V)
{
    const long long total = (long long)B * mr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / mr, e = i - b * mr;
        U[i] = y[b * ldy + e];
        V[i] = y[b * ldy + mr + e];
    }
}

// T[b] = T0 + s U[b] V[b]^T (FP64)
__global__ void k_lowrank(int m, int r, const double* __restrict__ T0, double s, const double* __restrict__ U,
                          const double* __restrict__ V, double* __restrict__ T)
{
    const int b = blockIdx.z;
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const double* u = U + ((long long)b * m + i) * r;
    const double* v = V + ((long long)b * m + j) * r;
    double acc = 0.0;
    for (int k = 0; k < r; ++k) acc += u[k] * v[k];
    T[((long long)b * m + i) * m + j] = T0[(long long)i * m + j] + s * acc;
}

// splitmix64 -> uniform in [-a, a)
unsigned long long splitmix(unsigned long long& s)
{
    unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

template <typename T>
void free_all(T*& p) { cudaFree(p); p = nullptr; }

template <typename T>
bool alloc_n(T*& p, size_t n) { return cudaMalloc(&p, sizeof(T) * std::max<size_t>(n, 1)) == cudaSuccess; }

void free_fwd(hps_mlp* net)
{
    free_all(net->xb); free_all(net->a1b); free_all(net->a2b); free_all(net->z); free_all(net->y);
    net->cap_f = 0;
}

void free_train(hps_mlp* net)
{
    free_all(net->xT); free_all(net->a1T); free_all(net->a2T);
    free_all(net->Un); free_all(net->Vb); free_all(net->UT); free_all(net->VT);
    free_all(net->E); free_all(net->Gn); free_all(net->GnT);
    free_all(net->dy); free_all(net->d2); free_all(net->d1); free_all(net->dyb); free_all(net->d2b);
    free_all(net->dyTn); free_all(net->d2Tn); free_all(net->d1Tn); free_all(net->lpart);
    net->cap_t = 0;
}

void free_mlp(hps_mlp* net)
{
    for (int l = 0; l < 3; ++l) {
        free_all(net->W[l]); free_all(net->c[l]); free_all(net->WnT[l]); free_all(net->Wn[l]);
        free_all(net->gW[l]); free_all(net->gc[l]);
        free_all(net->mW[l]); free_all(net->vW[l]); free_all(net->mc[l]); free_all(net->vc[l]);
    }
    free_fwd(net);
    free_train(net);
    free_all(net->loss);
    free_all(net->part);
    net->part_cap = 0;
    free_all(net->dtarget);
    net->dcap = 0;
}

long long split_need(const hps_mlp* net, int B);

// The split-K partial buffer for batches of up to B boxes.
hps_status ensure_part(hps_mlp* net, int B)
{
    const long long need = split_need(net, B);
    if (need <= net->part_cap) return HPS_OK;
    cudaDeviceSynchronize();
    free_all(net->part);
    net->part_cap = 0;
    if (!alloc_n(net->part, (size_t)need)) { cudaGetLastError(); return HPS_ENOMEM; }
    net->part_cap = need;
    return HPS_OK;
}

hps_status ensure_fwd(hps_mlp* net, int B)
{
    if (B <= net->cap_f) return HPS_OK;
    cudaDeviceSynchronize();
    free_fwd(net);
    const int* d = net->dims;
    const int* k = net->kp;
    const size_t Bz = (size_t)B;
    if (!alloc_n(net->xb, Bz * k[0]) || !alloc_n(net->a1b, Bz * k[1]) || !alloc_n(net->a2b, Bz * k[2]) ||
        !alloc_n(net->z, Bz * std::max(d[1], d[2])) || !alloc_n(net->y, Bz * d[3])) {
        cudaGetLastError();
        free_fwd(net);
        return HPS_ENOMEM;
    }
    net->cap_f = B;
    return HPS_OK;
}

hps_status ensure_train(hps_mlp* net, int B)
{
    if (B <= net->cap_t) return HPS_OK;
    cudaDeviceSynchronize();
    free_train(net);
    const int* d = net->dims;
    const int* k = net->kp;
    const size_t Bz = (size_t)B, Bp = (size_t)pad8(B), m = net->m, r = net->rank, rp = net->rp, mp = net->mp;
    if (!alloc_n(net->xT, d[0] * Bp) || !alloc_n(net->a1T, d[1] * Bp) || !alloc_n(net->a2T, d[2] * Bp) ||
        !alloc_n(net->Un, Bz * m * rp) || !alloc_n(net->Vb, Bz * m * rp) || !alloc_n(net->UT, Bz * r * mp) ||
        !alloc_n(net->VT, Bz * r * mp) || !alloc_n(net->E, Bz * m * m) || !alloc_n(net->Gn, Bz * m * mp) ||
        !alloc_n(net->GnT, Bz * m * mp) || !alloc_n(net->dy, Bz * d[3]) || !alloc_n(net->d2, Bz * d[2]) ||
        !alloc_n(net->d1, Bz * d[1]) || !alloc_n(net->dyb, Bz * k[3]) || !alloc_n(net->d2b, Bz * k[2]) ||
        !alloc_n(net->dyTn, d[3] * Bp) || !alloc_n(net->d2Tn, d[2] * Bp) || !alloc_n(net->d1Tn, d[1] * Bp) ||
        !alloc_n(net->lpart, Bz * ((m + 31) / 32))) {
        cudaGetLastError();
        free_train(net);
        return HPS_ENOMEM;
    }
    net->cap_t = B;
    return HPS_OK;
}

// The BF16 copies -W^T and -W of layer l's FP32 weights.
void refresh_copies(hps_mlp* net, int l, cudaStream_t st)
{
    const int* d = net->dims;
    const int* k = net->kp;
    act<float>(d[l], d[l + 1], net->W[l], d[l + 1], 0, 0, nullptr, 0, nullptr, 0, 0, nullptr, 0, 0, net->Wn[l],
               k[l + 1], 0, -1.0f, net->WnT[l], k[l], 0, -1.0f, 1, st);
}

// Split-K partial products: a product of one batch entry with fewer output
// tiles than half the SMs and K >= 256 runs as S products over K ranges of
// Ks (a multiple of 32) into partial buffers, summed by k_reduce_splits.
constexpr int kSplitMaxTiles = 76, kSplitMinK = 128;

int split_count(int M, int N, int K, int batch, long long ldc)
{
    const int bn = N > 128 ? 256 : (N > 64 ? 128 : 64);
    const long long tiles = (long long)((M + 127) / 128) * ((N + bn - 1) / bn) * batch;
    if (batch != 1 || ldc != N || tiles >= kSplitMaxTiles || K < 2 * kSplitMinK) return 1;
    return (int)std::min<long long>((152 + tiles - 1) / tiles, K / kSplitMinK);
}

// C [M][N] = A B^T for BF16 operands with a negated side (see the header);
// A [M][lda], B [N][ldb], K the used extent.  Batch strides of 0 for one
// entry are given a valid value for the tensor maps.
bool gemm(hps_mlp* net, int M, int N, int K, const __nv_bfloat16* A, long long lda, long long sA,
          const __nv_bfloat16* B, long long ldb, long long sB, float* C, long long ldc, long long sC, int batch,
          cudaStream_t st)
{
    if (batch == 1) {
        sA = (long long)M * lda;
        sB = (long long)N * ldb;
        sC = (long long)M * ldc;
    }
    int S = split_count(M, N, K, batch, ldc);
    if (S <= 1 || !net->part) return hps::tc_gemm_bf16(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, false, batch, st);
    const int Ks = ((K + S - 1) / S + 31) / 32 * 32;
    S = (K + Ks - 1) / Ks;
    const long long mn = (long long)M * N;
    if ((long long)S * mn > net->part_cap) return hps::tc_gemm_bf16(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, false,
                                                                     batch, st);
    // S - 1 full ranges as batch entries (operand batch stride Ks), then the
    // last range; the plain product if the ranges cannot be described to TMA
    // (nothing is launched then)
    if (!hps::tc_gemm_bf16(M, N, Ks, A, lda, Ks, B, ldb, Ks, net->part, N, mn, false, S - 1, st))
        return hps::tc_gemm_bf16(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, false, batch, st);
    const long long k0 = (long long)(S - 1) * Ks;
    if (!hps::tc_gemm_bf16(M, N, (int)(K - k0), A + k0, lda, sA, B + k0, ldb, sB, net->part + (S - 1) * mn, N, mn,
                           false, 1, st))
        return false;
    k_reduce_splits<<<blocks_for(mn), 256, 0, st>>>(mn, S, net->part, C);
    return true;
}

// Largest split-K partial buffer (floats) any product of the network needs
// for a batch of B boxes.
long long split_need(const hps_mlp* net, int B)
{
    const int* d = net->dims;
    const int* k = net->kp;
    const int Bp = pad8(B);
    const int shapes[8][3] = {{B, d[1], k[0]},  {B, d[2], k[1]},  {B, d[3], k[2]},  {d[2], d[3], Bp},
                              {B, d[2], k[3]}, {d[1], d[2], Bp}, {B, d[1], k[2]}, {d[0], d[1], Bp}};
    long long need = 0;
    for (const auto& sh : shapes) {
        int S = split_count(sh[0], sh[1], sh[2], 1, sh[1]);
        if (S > 1) {
            const int Ks = ((sh[2] + S - 1) / S + 31) / 32 * 32;
            S = (sh[2] + Ks - 1) / Ks;
            need = std::max(need, (long long)S * sh[0] * sh[1]);
        }
    }
    return need;
}

// Forward pass of B boxes into net->y (bias included); with `train`, the
// transposed BF16 activations for the weight gradients as well.
bool forward(hps_mlp* net, int B, const double* b_in, bool train, cudaStream_t st)
{
    const int* d = net->dims;
    const int* k = net->kp;
    const int Bp = pad8(B);
    act<double>(B, d[0], b_in, d[0], 0, 1, nullptr, 0, nullptr, 0, 0, nullptr, 0, 0, net->xb, k[0], 0, 1.0f,
                train ? net->xT : nullptr, Bp, 0, 1.0f, 1, st);
    if (!gemm(net, B, d[1], k[0], net->xb, k[0], 0, net->WnT[0], k[0], 0, net->z, d[1], 0, 1, st)) return false;
    act<float>(B, d[1], net->z, d[1], 0, 0, net->c[0], 1, nullptr, 0, 0, nullptr, 0, 0, net->a1b, k[1], 0, 1.0f,
               train ? net->a1T : nullptr, Bp, 0, 1.0f, 1, st);
    if (!gemm(net, B, d[2], k[1], net->a1b, k[1], 0, net->WnT[1], k[1], 0, net->z, d[2], 0, 1, st)) return false;
    act<float>(B, d[2], net->z, d[2], 0, 0, net->c[1], 1, nullptr, 0, 0, nullptr, 0, 0, net->a2b, k[2], 0, 1.0f,
               train ? net->a2T : nullptr, Bp, 0, 1.0f, 1, st);
    if (!gemm(net, B, d[3], k[2], net->a2b, k[2], 0, net->WnT[2], k[2], 0, net->y, d[3], 0, 1, st)) return false;
    act<float>(B, d[3], net->y, d[3], 0, 0, net->c[2], 0, nullptr, 0, 0, net->y, d[3], 0, nullptr, 0, 0, 1.0f,
               nullptr, 0, 0, 1.0f, 1, st);
    return true;
}

}  // namespace

using namespace hps;

extern "C" {

hps_status hps_mlp_create(int device, int n_in, int n_h1, int n_h2, int m, int rank, unsigned long long seed,
                          hps_mlp** out)
{
    if (!out || n_in < 1 || n_h1 < 1 || n_h2 < 1 || m < 1 || rank < 1) return HPS_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return HPS_ECUDA; }
    hps_mlp* net = new (std::nothrow) hps_mlp();
    if (!net) return HPS_ENOMEM;
    net->device = device;
    net->dims[0] = n_in; net->dims[1] = n_h1; net->dims[2] = n_h2; net->dims[3] = 2 * m * rank;
    for (int l = 0; l < 4; ++l) net->kp[l] = pad8(net->dims[l]);
    net->m = m;
    net->rank = rank;
    net->rp = pad8(rank);
    net->mp = pad8(m);
    unsigned long long s = seed;
    for (int l = 0; l < 3; ++l) {
        const size_t nw = (size_t)net->dims[l] * net->dims[l + 1], nc = net->dims[l + 1];
        bool ok = alloc_n(net->W[l], nw) && alloc_n(net->c[l], nc) &&
                  alloc_n(net->WnT[l], (size_t)net->dims[l + 1] * net->kp[l]) &&
                  alloc_n(net->Wn[l], (size_t)net->dims[l] * net->kp[l + 1]) && alloc_n(net->gW[l], nw) &&
                  alloc_n(net->gc[l], nc) && alloc_n(net->mW[l], nw) && alloc_n(net->vW[l], nw) &&
                  alloc_n(net->mc[l], nc) && alloc_n(net->vc[l], nc);
        if (!ok) { cudaGetLastError(); free_mlp(net); delete net; return HPS_ENOMEM; }
        // He-uniform weights (scaled down on the output layer), zero biases.
        std::vector<float> w(nw);
        const double a = std::sqrt(6.0 / net->dims[l]) * (l == 2 ? 0.1 : 1.0);
        for (size_t i = 0; i < nw; ++i) w[i] = float(a * (2.0 * ((splitmix(s) >> 11) * 0x1.0p-53) - 1.0));
        cudaMemcpy(net->W[l], w.data(), nw * 4, cudaMemcpyHostToDevice);
        cudaMemset(net->c[l], 0, nc * 4);
        cudaMemset(net->mW[l], 0, nw * 4); cudaMemset(net->vW[l], 0, nw * 4);
        cudaMemset(net->mc[l], 0, nc * 4); cudaMemset(net->vc[l], 0, nc * 4);
        refresh_copies(net, l, nullptr);
    }
    if (!alloc_n(net->loss, 1)) { cudaGetLastError(); free_mlp(net); delete net; return HPS_ENOMEM; }
    if (cudaDeviceSynchronize() != cudaSuccess) { free_mlp(net); delete net; return HPS_ECUDA; }
    *out = net;
    return HPS_OK;
}

void hps_mlp_destroy(hps_mlp* net)
{
    if (!net) return;
    cudaSetDevice(net->device);
    cudaDeviceSynchronize();
    free_mlp(net);
    delete net;
}

size_t hps_mlp_num_params(const hps_mlp* net)
{
    if (!net) return 0;
    size_t n = 0;
    for (int l = 0; l < 3; ++l) n += (size_t)net->dims[l] * net->dims[l + 1] + net->dims[l + 1];
    return n;
}

// Parameters (or gradients, which = 1) as one host array: W0, c0, W1, c1, W2, c2.
hps_status hps_mlp_copy_params(hps_mlp* net, int which, float* host, int to_device)
{
    if (!net || !host || which < 0 || which > 1) return HPS_EINVAL;
    if (to_device && which) return HPS_EINVAL;
    if (cudaSetDevice(net->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return HPS_ECUDA;
    size_t off = 0;
    for (int l = 0; l < 3; ++l) {
        const size_t nw = (size_t)net->dims[l] * net->dims[l + 1], nc = net->dims[l + 1];
        float* w = which ? net->gW[l] : net->W[l];
        float* c = which ? net->gc[l] : net->c[l];
        cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
        if (cudaMemcpy(to_device ? (void*)w : (void*)(host + off), to_device ? (void*)(host + off) : (void*)w, nw * 4,
                       kind) != cudaSuccess)
            return HPS_ECUDA;
        off += nw;
        if (cudaMemcpy(to_device ? (void*)c : (void*)(host + off), to_device ? (void*)(host + off) : (void*)c, nc * 4,
                       kind) != cudaSuccess)
            return HPS_ECUDA;
        off += nc;
        if (to_device) refresh_copies(net, l, nullptr);
    }
    return cudaDeviceSynchronize() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_forward(hps_mlp* net, int B, const double* b_in, double* U, double* V, void* stream)
{
    if (!net || B < 0 || (B > 0 && (!b_in || !U || !V))) return HPS_EINVAL;
    if (B == 0) return HPS_OK;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    hps_status rc = ensure_fwd(net, B);
    if (rc == HPS_OK) rc = ensure_part(net, B);
    if (rc != HPS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!forward(net, B, b_in, false, st)) return HPS_ECUDA;
    const int mr = net->m * net->rank;
    k_split_uv<<<blocks_for((long long)B * mr), 256, 0, st>>>(B, mr, net->y, net->dims[3], U, V);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_target(int nbox, int m, const double* T, const double* T0, double scale, float* D, void* stream)
{
    if (nbox < 0 || m < 1 || !(scale > 0) || (nbox > 0 && (!T || !T0 || !D))) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    const long long mm2 = (long long)m * m, n = (long long)nbox * mm2;
    k_target<<<blocks_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, mm2, T, T0, 1.0 / scale, D);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_grad_target(hps_mlp* net, int B, const double* b_in, const float* D, double* loss_out, void* stream)
{
    if (!net || B < 1 || !b_in || !D) return HPS_EINVAL;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    hps_status rc = ensure_fwd(net, B);
    if (rc == HPS_OK) rc = ensure_train(net, B);
    if (rc == HPS_OK) rc = ensure_part(net, B);
    if (rc != HPS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int* d = net->dims;
    const int* k = net->kp;
    const int m = net->m, r = net->rank, mr = m * r, rp = net->rp, mp = net->mp, Bp = pad8(B);
    const long long mm2 = (long long)m * m;
    bool ok = forward(net, B, b_in, true, st);
    // BF16 factors: -U and V [m][rp] for E = U V^T, U^T and V^T [r][mp] for E^T U and E V
    act<float>(m, r, net->y, r, d[3], 0, nullptr, 0, nullptr, 0, 0, nullptr, 0, 0, net->Un, rp, (long long)m * rp,
               -1.0f, net->UT, mp, (long long)r * mp, 1.0f, B, st);
    act<float>(m, r, net->y + mr, r, d[3], 0, nullptr, 0, nullptr, 0, 0, nullptr, 0, 0, net->Vb, rp,
               (long long)m * rp, 1.0f, net->VT, mp, (long long)r * mp, 1.0f, B, st);
    ok = ok && gemm(net, m, m, rp, net->Un, rp, (long long)m * rp, net->Vb, rp, (long long)m * rp, net->E, m, mm2, B, st);
    // e = U V^T - D, loss = mean e^2, G = (2 / (B m^2)) e
    {
        const int rt = (m + 31) / 32;
        k_loss<<<dim3((unsigned)rt, (unsigned)B), dim3(32, 8), 0, st>>>(m, net->E, D, 2.0f / float((double)B * mm2),
                                                                       net->Gn, net->GnT, mp, net->lpart);
        k_sum<<<1, 256, 0, st>>>(rt * B, net->lpart, net->loss);
    }
    // dU = G V, dV = G^T U into dy
    ok = ok && gemm(net, m, r, mp, net->Gn, mp, (long long)m * mp, net->VT, mp, (long long)r * mp, net->dy, r, d[3], B, st);
    ok = ok && gemm(net, m, r, mp, net->GnT, mp, (long long)m * mp, net->UT, mp, (long long)r * mp, net->dy + mr, r, d[3],
                    B, st);
    // layer 3: gc2 from dy, gW2 = a2^T dy, d2 = (dy W2^T) * [a2 > 0]
    k_colsum<<<(d[3] + 255) / 256, 256, 0, st>>>(B, d[3], net->dy, net->gc[2]);
    act<float>(B, d[3], net->dy, d[3], 0, 0, nullptr, 0, nullptr, 0, 0, nullptr, 0, 0, net->dyb, k[3], 0, 1.0f,
               net->dyTn, Bp, 0, -1.0f, 1, st);
    ok = ok && gemm(net, d[2], d[3], Bp, net->a2T, Bp, 0, net->dyTn, Bp, 0, net->gW[2], d[3], 0, 1, st);
    ok = ok && gemm(net, B, d[2], k[3], net->dyb, k[3], 0, net->Wn[2], k[3], 0, net->d2, d[2], 0, 1, st);
    act<float>(B, d[2], net->d2, d[2], 0, 0, nullptr, 0, net->a2b, k[2], 0, net->d2, d[2], 0, net->d2b, k[2], 0, 1.0f,
               net->d2Tn, Bp, 0, -1.0f, 1, st);
    // layer 2
    k_colsum<<<(d[2] + 255) / 256, 256, 0, st>>>(B, d[2], net->d2, net->gc[1]);
    ok = ok && gemm(net, d[1], d[2], Bp, net->a1T, Bp, 0, net->d2Tn, Bp, 0, net->gW[1], d[2], 0, 1, st);
    ok = ok && gemm(net, B, d[1], k[2], net->d2b, k[2], 0, net->Wn[1], k[2], 0, net->d1, d[1], 0, 1, st);
    act<float>(B, d[1], net->d1, d[1], 0, 0, nullptr, 0, net->a1b, k[1], 0, net->d1, d[1], 0, nullptr, 0, 0, 1.0f,
               net->d1Tn, Bp, 0, -1.0f, 1, st);
    // layer 1
    k_colsum<<<(d[1] + 255) / 256, 256, 0, st>>>(B, d[1], net->d1, net->gc[0]);
    ok = ok && gemm(net, d[0], d[1], Bp, net->xT, Bp, 0, net->d1Tn, Bp, 0, net->gW[0], d[1], 0, 1, st);
    if (!ok) return HPS_ECUDA;
    if (loss_out) {
        double l = 0.0;
        if (cudaMemcpyAsync(&l, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return HPS_ECUDA;
        *loss_out = l / ((double)B * mm2);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_grad(hps_mlp* net, int B, const double* b_in, const double* T, const double* T0, double scale,
                        double* loss_out, void* stream)
{
    if (!net || B < 1 || !b_in || !T || !T0 || !(scale > 0)) return HPS_EINVAL;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    const size_t need = (size_t)B * net->m * net->m;
    if (need > net->dcap) {
        cudaDeviceSynchronize();
        free_all(net->dtarget);
        net->dcap = 0;
        if (!alloc_n(net->dtarget, need)) { cudaGetLastError(); return HPS_ENOMEM; }
        net->dcap = need;
    }
    hps_status rc = hps_mlp_target(B, net->m, T, T0, scale, net->dtarget, stream);
    if (rc != HPS_OK) return rc;
    return hps_mlp_grad_target(net, B, b_in, net->dtarget, loss_out, stream);
}

hps_status hps_mlp_adam_step(hps_mlp* net, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!net || !(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) return HPS_EINVAL;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    net->adam_t += 1;
    const float bc1 = 1.0f - std::pow(beta1, (float)net->adam_t);
    const float bc2 = 1.0f - std::pow(beta2, (float)net->adam_t);
    for (int l = 0; l < 3; ++l) {
        const long long nw = (long long)net->dims[l] * net->dims[l + 1], nc = net->dims[l + 1];
        k_adam<<<blocks_for(nw), 256, 0, st>>>(nw, net->W[l], net->gW[l], net->mW[l], net->vW[l], lr, beta1, beta2, eps,
                                              bc1, bc2);
        k_adam<<<blocks_for(nc), 256, 0, st>>>(nc, net->c[l], net->gc[l], net->mc[l], net->vc[l], lr, beta1, beta2, eps,
                                              bc1, bc2);
        refresh_copies(net, l, st);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_lowrank_dtn(int nbox, int m, int rank, const double* T0, double scale, const double* U,
                           const double* V, double* T, void* stream)
{
    if (nbox < 0 || m < 1 || rank < 1 || (nbox > 0 && (!T0 || !U || !V || !T))) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    dim3 grd((unsigned)((m + 127) / 128), (unsigned)m, (unsigned)nbox);
    k_lowrank<<<grd, 128, 0, static_cast<cudaStream_t>(stream)>>>(m, rank, T0, scale, U, V, T);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // extern "C"
