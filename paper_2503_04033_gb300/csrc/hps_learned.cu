// Learned low-rank correction of the leaf DtN map (an extension beyond the
// paper, whose DtN maps are always computed exactly).
//
// A three-layer MLP maps the sampled coefficient b of a box (all p^3 grid
// values, input x = 2 (b - 1)) to factors U, V in R^{m x r}; the predicted map
// is T_hat = T0 + s U V^T, with T0 the DtN map of the same box for b = 1 and s
// a fixed target scale.  Weights are kept in FP32 (master copy, Adam moments)
// and used in BF16 by every product, which accumulates in FP32.  Training
// minimises L = mean over boxes and entries of (U V^T - (T - T0)/s)^2.
//
// Layers (row-major, weights [in][out]):
//   a1 = relu(x W0 + c0),  a2 = relu(a1 W1 + c1),  y = a2 W2 + c2,
//   U = y[:, 0 : m r] as [m][r],  V = y[:, m r : 2 m r] as [m][r].
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hps_internal.h"

struct hps_mlp {
    int device = 0;
    int dims[4] = {0, 0, 0, 0};        // n_in, h1, h2, n_out
    int m = 0, rank = 0;
    float* W[3] = {};                  // FP32 master weights [in][out]
    float* c[3] = {};                  // biases [out]
    __nv_bfloat16* Wb[3] = {};         // BF16 copies used by the products
    float* gW[3] = {};
    float* gc[3] = {};
    float* mW[3] = {};
    float* vW[3] = {};
    float* mc[3] = {};
    float* vc[3] = {};
    long long adam_t = 0;
    int cap = 0;                       // batch capacity of the activation buffers
    float *x = nullptr, *a1 = nullptr, *a2 = nullptr, *y = nullptr, *dy = nullptr, *d2 = nullptr,
          *d1 = nullptr, *E = nullptr;
    double* loss = nullptr;
};

namespace {

// C[b] = alpha opA(A[b]) opB(B[b]) + beta C[b] (+ bias[j]) (relu) (* [mask > 0])
// opA(i, k) = tA ? A[k lda + i] : A[i lda + k];  opB(k, j) = tB ? B[j ldb + k] : B[k ldb + j].
template <typename TB>
__global__ void __launch_bounds__(256)
k_mm(int M, int N, int K, const float* __restrict__ A, long long sA, int lda, int tA, const TB* __restrict__ B,
     long long sB, int ldb, int tB, float* __restrict__ C, long long sC, int ldc, float alpha, float beta,
     const float* __restrict__ bias, int relu, const float* __restrict__ mask, int ldmask)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM + 1];
    __shared__ float Bs[BK][BN + 1];
    const int z = blockIdx.z;
    A += z * sA;
    B += z * sB;
    C += z * sC;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += 256) {
            int i, kk;
            if (tA) { i = idx % BM; kk = idx / BM; } else { kk = idx % BK; i = idx / BK; }
            const int r = m0 + i, kc = k0 + kk;
            float v = 0.0f;
            if (r < M && kc < K) v = tA ? A[(long long)kc * lda + r] : A[(long long)r * lda + kc];
            As[kk][i] = v;
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += 256) {
            int jj, kk;
            if (tB) { kk = idx % BK; jj = idx / BK; } else { jj = idx % BN; kk = idx / BN; }
            const int c = n0 + jj, kc = k0 + kk;
            float v = 0.0f;
            if (c < N && kc < K) v = float(tB ? B[(long long)c * ldb + kc] : B[(long long)kc * ldb + c]);
            Bs[kk][jj] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int bq = 0; bq < 4; ++bq) bv[bq] = Bs[kk][tx * 4 + bq];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int bq = 0; bq < 4; ++bq) acc[a][bq] += av[a] * bv[bq];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = m0 + ty * 4 + a;
        if (r >= M) continue;
#pragma unroll
        for (int bq = 0; bq < 4; ++bq) {
            const int c = n0 + tx * 4 + bq;
            if (c >= N) continue;
            float v = alpha * acc[a][bq];
            if (beta != 0.0f) v += beta * C[(long long)r * ldc + c];
            if (bias) v += bias[c];
            if (relu) v = fmaxf(v, 0.0f);
            if (mask && !(mask[(long long)r * ldmask + c] > 0.0f)) v = 0.0f;
            C[(long long)r * ldc + c] = v;
        }
    }
}

template <typename TB>
void mm(int M, int N, int K, const float* A, long long sA, int lda, int tA, const TB* B, long long sB, int ldb,
        int tB, float* C, long long sC, int ldc, float alpha, float beta, const float* bias, int relu,
        const float* mask, int ldmask, int batch, cudaStream_t st)
{
    dim3 grd((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)batch);
    k_mm<TB><<<grd, 256, 0, st>>>(M, N, K, A, sA, lda, tA, B, sB, ldb, tB, C, sC, ldc, alpha, beta, bias, relu,
                                   mask, ldmask);
}

__global__ void k_input(int n, const double* __restrict__ b, float* __restrict__ x)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = float(2.0 * (b[i] - 1.0));
}

// E = E - (T - T0) / s (E holds U V^T, T0 shared by the batch); accumulates sum E^2.
__global__ void k_residual_target(long long n, long long mm2, float* __restrict__ E, const double* __restrict__ T,
                                  const double* __restrict__ T0, double inv_s, double* loss)
{
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float e = E[i] - float((T[i] - T0[i % mm2]) * inv_s);
        E[i] = e;
        acc += (double)e * e;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
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
                       float* __restrict__ ve, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2, float eps,
                       float bc1, float bc2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float m = b1 * mo[i] + (1.0f - b1) * gi;
        const float v = b2 * ve[i] + (1.0f - b2) * gi * gi;
        mo[i] = m;
        ve[i] = v;
        const float wi = w[i] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        wb[i] = __float2bfloat16(w[i]);
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

void free_mlp(hps_mlp* net)
{
    for (int l = 0; l < 3; ++l) {
        cudaFree(net->W[l]); cudaFree(net->c[l]); cudaFree(net->Wb[l]); cudaFree(net->gW[l]); cudaFree(net->gc[l]);
        cudaFree(net->mW[l]); cudaFree(net->vW[l]); cudaFree(net->mc[l]); cudaFree(net->vc[l]);
    }
    cudaFree(net->x); cudaFree(net->a1); cudaFree(net->a2); cudaFree(net->y); cudaFree(net->dy);
    cudaFree(net->d2); cudaFree(net->d1); cudaFree(net->E); cudaFree(net->loss);
}

hps_status ensure_batch(hps_mlp* net, int B)
{
    if (B <= net->cap) return HPS_OK;
    cudaDeviceSynchronize();
    cudaFree(net->x); cudaFree(net->a1); cudaFree(net->a2); cudaFree(net->y); cudaFree(net->dy);
    cudaFree(net->d2); cudaFree(net->d1); cudaFree(net->E);
    const int* d = net->dims;
    const size_t mm2 = (size_t)net->m * net->m;
    if (cudaMalloc(&net->x, sizeof(float) * (size_t)B * d[0]) != cudaSuccess ||
        cudaMalloc(&net->a1, sizeof(float) * (size_t)B * d[1]) != cudaSuccess ||
        cudaMalloc(&net->a2, sizeof(float) * (size_t)B * d[2]) != cudaSuccess ||
        cudaMalloc(&net->y, sizeof(float) * (size_t)B * d[3]) != cudaSuccess ||
        cudaMalloc(&net->dy, sizeof(float) * (size_t)B * d[3]) != cudaSuccess ||
        cudaMalloc(&net->d2, sizeof(float) * (size_t)B * d[2]) != cudaSuccess ||
        cudaMalloc(&net->d1, sizeof(float) * (size_t)B * d[1]) != cudaSuccess ||
        cudaMalloc(&net->E, sizeof(float) * (size_t)B * mm2) != cudaSuccess) {
        cudaGetLastError();
        net->cap = 0;
        return HPS_ENOMEM;
    }
    net->cap = B;
    return HPS_OK;
}

void forward(hps_mlp* net, int B, const double* b_in, cudaStream_t st)
{
    const int* d = net->dims;
    k_input<<<blocks_for((long long)B * d[0]), 256, 0, st>>>(B * d[0], b_in, net->x);
    mm<__nv_bfloat16>(B, d[1], d[0], net->x, 0, d[0], 0, net->Wb[0], 0, d[1], 0, net->a1, 0, d[1], 1.f, 0.f, net->c[0],
                      1, nullptr, 0, 1, st);
    mm<__nv_bfloat16>(B, d[2], d[1], net->a1, 0, d[1], 0, net->Wb[1], 0, d[2], 0, net->a2, 0, d[2], 1.f, 0.f, net->c[1],
                      1, nullptr, 0, 1, st);
    mm<__nv_bfloat16>(B, d[3], d[2], net->a2, 0, d[2], 0, net->Wb[2], 0, d[3], 0, net->y, 0, d[3], 1.f, 0.f, net->c[2],
                      0, nullptr, 0, 1, st);
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
    net->m = m;
    net->rank = rank;
    unsigned long long s = seed;
    for (int l = 0; l < 3; ++l) {
        const size_t nw = (size_t)net->dims[l] * net->dims[l + 1], nc = net->dims[l + 1];
        bool ok = cudaMalloc(&net->W[l], nw * 4) == cudaSuccess && cudaMalloc(&net->c[l], nc * 4) == cudaSuccess &&
                  cudaMalloc(&net->Wb[l], nw * 2) == cudaSuccess && cudaMalloc(&net->gW[l], nw * 4) == cudaSuccess &&
                  cudaMalloc(&net->gc[l], nc * 4) == cudaSuccess && cudaMalloc(&net->mW[l], nw * 4) == cudaSuccess &&
                  cudaMalloc(&net->vW[l], nw * 4) == cudaSuccess && cudaMalloc(&net->mc[l], nc * 4) == cudaSuccess &&
                  cudaMalloc(&net->vc[l], nc * 4) == cudaSuccess;
        if (!ok) { cudaGetLastError(); free_mlp(net); delete net; return HPS_ENOMEM; }
        // He-uniform weights (scaled down on the output layer), zero biases.
        std::vector<float> w(nw);
        const double a = std::sqrt(6.0 / net->dims[l]) * (l == 2 ? 0.1 : 1.0);
        for (size_t i = 0; i < nw; ++i) w[i] = float(a * (2.0 * ((splitmix(s) >> 11) * 0x1.0p-53) - 1.0));
        cudaMemcpy(net->W[l], w.data(), nw * 4, cudaMemcpyHostToDevice);
        cudaMemset(net->c[l], 0, nc * 4);
        cudaMemset(net->mW[l], 0, nw * 4); cudaMemset(net->vW[l], 0, nw * 4);
        cudaMemset(net->mc[l], 0, nc * 4); cudaMemset(net->vc[l], 0, nc * 4);
        k_to_bf16<<<blocks_for(nw), 256>>>((long long)nw, net->W[l], net->Wb[l]);
    }
    if (cudaMalloc(&net->loss, sizeof(double)) != cudaSuccess) { cudaGetLastError(); free_mlp(net); delete net; return HPS_ENOMEM; }
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
    if (cudaSetDevice(net->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return HPS_ECUDA;
    size_t off = 0;
    for (int l = 0; l < 3; ++l) {
        const size_t nw = (size_t)net->dims[l] * net->dims[l + 1], nc = net->dims[l + 1];
        float* w = which ? net->gW[l] : net->W[l];
        float* c = which ? net->gc[l] : net->c[l];
        cudaMemcpyKind kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
        if (to_device && which) return HPS_EINVAL;
        if (cudaMemcpy(to_device ? (void*)w : (void*)(host + off), to_device ? (void*)(host + off) : (void*)w, nw * 4,
                       kind) != cudaSuccess)
            return HPS_ECUDA;
        off += nw;
        if (cudaMemcpy(to_device ? (void*)c : (void*)(host + off), to_device ? (void*)(host + off) : (void*)c, nc * 4,
                       kind) != cudaSuccess)
            return HPS_ECUDA;
        off += nc;
        if (to_device) k_to_bf16<<<blocks_for(nw), 256>>>((long long)nw, net->W[l], net->Wb[l]);
    }
    return cudaDeviceSynchronize() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_forward(hps_mlp* net, int B, const double* b_in, double* U, double* V, void* stream)
{
    if (!net || B < 0 || (B > 0 && (!b_in || !U || !V))) return HPS_EINVAL;
    if (B == 0) return HPS_OK;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    hps_status rc = ensure_batch(net, B);
    if (rc != HPS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    forward(net, B, b_in, st);
    const int mr = net->m * net->rank;
    k_split_uv<<<blocks_for((long long)B * mr), 256, 0, st>>>(B, mr, net->y, net->dims[3], U, V);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_mlp_grad(hps_mlp* net, int B, const double* b_in, const double* T, const double* T0, double scale,
                        double* loss_out, void* stream)
{
    if (!net || B < 1 || !b_in || !T || !T0 || !(scale > 0)) return HPS_EINVAL;
    if (cudaSetDevice(net->device) != cudaSuccess) return HPS_ECUDA;
    hps_status rc = ensure_batch(net, B);
    if (rc != HPS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int* d = net->dims;
    const int m = net->m, r = net->rank, mr = m * r;
    const long long mm2 = (long long)m * m;
    forward(net, B, b_in, st);
    // E = U V^T - (T - T0) / s ; loss = mean E^2
    mm<float>(m, m, r, net->y, d[3], r, 0, net->y + mr, d[3], r, 1, net->E, mm2, m, 1.f, 0.f, nullptr, 0, nullptr, 0, B,
              st);
    cudaMemsetAsync(net->loss, 0, sizeof(double), st);
    k_residual_target<<<blocks_for(B * mm2), 256, 0, st>>>(B * mm2, mm2, net->E, T, T0, 1.0 / scale, net->loss);
    // dU = (2 / (B m^2)) E V ; dV = (2 / (B m^2)) E^T U
    const float g = 2.0f / float((double)B * mm2);
    mm<float>(m, r, m, net->E, mm2, m, 0, net->y + mr, d[3], r, 0, net->dy, d[3], r, g, 0.f, nullptr, 0, nullptr, 0, B,
              st);
    mm<float>(m, r, m, net->E, mm2, m, 1, net->y, d[3], r, 0, net->dy + mr, d[3], r, g, 0.f, nullptr, 0, nullptr, 0, B,
              st);
    // layer 3
    mm<float>(d[2], d[3], B, net->a2, 0, d[2], 1, net->dy, 0, d[3], 0, net->gW[2], 0, d[3], 1.f, 0.f, nullptr, 0,
              nullptr, 0, 1, st);
    k_colsum<<<(d[3] + 255) / 256, 256, 0, st>>>(B, d[3], net->dy, net->gc[2]);
    mm<__nv_bfloat16>(B, d[2], d[3], net->dy, 0, d[3], 0, net->Wb[2], 0, d[3], 1, net->d2, 0, d[2], 1.f, 0.f, nullptr, 0,
                      net->a2, d[2], 1, st);
    // layer 2
    mm<float>(d[1], d[2], B, net->a1, 0, d[1], 1, net->d2, 0, d[2], 0, net->gW[1], 0, d[2], 1.f, 0.f, nullptr, 0,
              nullptr, 0, 1, st);
    k_colsum<<<(d[2] + 255) / 256, 256, 0, st>>>(B, d[2], net->d2, net->gc[1]);
    mm<__nv_bfloat16>(B, d[1], d[2], net->d2, 0, d[2], 0, net->Wb[1], 0, d[2], 1, net->d1, 0, d[1], 1.f, 0.f, nullptr, 0,
                      net->a1, d[1], 1, st);
    // layer 1
    mm<float>(d[0], d[1], B, net->x, 0, d[0], 1, net->d1, 0, d[1], 0, net->gW[0], 0, d[1], 1.f, 0.f, nullptr, 0,
              nullptr, 0, 1, st);
    k_colsum<<<(d[1] + 255) / 256, 256, 0, st>>>(B, d[1], net->d1, net->gc[0]);
    if (loss_out) {
        double l = 0.0;
        if (cudaMemcpyAsync(&l, net->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return HPS_ECUDA;
        *loss_out = l / ((double)B * mm2);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
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
        k_adam<<<blocks_for(nw), 256, 0, st>>>(nw, net->W[l], net->gW[l], net->mW[l], net->vW[l], net->Wb[l], lr, beta1,
                                              beta2, eps, bc1, bc2);
        k_adam<<<blocks_for(nc), 256, 0, st>>>(nc, net->c[l], net->gc[l], net->mc[l], net->vc[l], nullptr, lr, beta1,
                                              beta2, eps, bc1, bc2);
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
