// Interface solve on the GPU: nested dissection of the interface system over
// the box grid, factored and solved level by level with batched FP64 kernels.
//
// The interface system (Sec. 3.1; Eq. 4 with f_b = 0 at shared faces) asks
// that at every shared face node the outward fluxes T^tau u_b^tau + h^tau of
// the boxes that share it add up to zero, with u = g known on the outer
// boundary.  Sec. 3 recalls how the original HPS method eliminates it: boxes
// are merged in pairs and the nodes of the face between the two halves are
// eliminated, so that each merged box carries a DtN map of its own boundary.
// For a merge of a and b, with 1 and 2 the outer slots of a and b and 3 the
// face nodes between them,
//     W = T^a_33 + T^b_33,
//     u_3 = S [u_1; u_2] - W^{-1} (h^a_3 + h^b_3),    S = -W^{-1} [T^a_31  T^b_32],
//     T = diag(T^a_11, T^b_22) + E S,                   E = [T^a_13; T^b_23],
//     h = [h^a_1; h^b_2] - E W^{-1} (h^a_3 + h^b_3).
// The paper factors the same system with a host multifrontal solver (MUMPS,
// Sec. 3.2), which orders it by nested dissection as well; here every merge
// of a level is one batch of the library's FP64 LU with partial pivoting
// (W carrying [T^a_31 T^b_32 | I] as right-hand sides), and the solve is two
// sweeps of batched matrix-vector products: up the tree for h, down for u.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "hps_iface.h"
#include "hps_internal.h"

namespace hps {
int ctx_device(const hps_ctx* ctx);
}

namespace {

using hps::IfNode;
using hps::IfPlan;

// Per-merge descriptor read by the kernels of one level.
struct IfDesc {
    const double* Ta;   // factorisation: the children's DtN maps (leaf: T + box m^2; merge: its T)
    const double* Tb;
    long long lda, ldb; // their row pitch
    double* va;         // solve: the children's level flux buffers hv (NULL for a leaf child)
    double* vb;
    double* wa;         // solve: the children's level boundary-value buffers uv (NULL for a leaf child)
    double* wb;
    long long oa, ob;   // first row of the child's block there (index in level x e_pad of that level)
    int leafa, leafb;   // box index of a leaf child, else -1
    int na1, nsep, nb2, loff;   // face counts; lists a1, a3, b2, b3 start at loff (face slots)
};

struct IfLevel {
    int nn = 0, s_pad = 0, e_pad = 0;
    std::vector<int> ids;
    std::vector<IfDesc> desc;
    std::vector<int> lists;
    IfDesc* d_desc = nullptr;
    int* d_lists = nullptr;
    double* Winv = nullptr;   // [nn][s_pad][s_pad]
    double* S = nullptr;      // [nn][s_pad][e_pad]
    double* E = nullptr;      // [nn][e_pad][s_pad]
    double* Tn = nullptr;     // factorisation only: merged maps [nn][e_pad][e_pad]
    double* hv = nullptr;     // solve: merged fluxes [nn][e_pad][nrhs]
    double* uv = nullptr;     // solve: boundary values [nn][e_pad][nrhs]
    double* t3 = nullptr;     // solve: h^a_3 + h^b_3, then reused for S [u_1; u_2] [nn][s_pad][nrhs]
    double* y = nullptr;      // solve: W^{-1} (h^a_3 + h^b_3) [nn][s_pad][nrhs]
};

constexpr int kMaxSeparator = 14000;   // the panel keeps a column of W in shared memory

}  // namespace

struct hps_interface {
    int device = 0;
    int p = 0, q = 0, qq = 0, m = 0, nbox = 0, nrhs_max = 0;
    IfPlan plan;
    std::vector<IfLevel> levels;
    // Dirichlet faces of the leaves: per box, the columns of T on its outer faces
    double* TD = nullptr;          // [ndface][m][qq]
    int* d_dinfo = nullptr;        // [nbox][8]: count, first block, then the local faces
    std::vector<int> dinfo;
    int ndface = 0;
    double* hl = nullptr;          // [nbox][nrhs][m]: leaf fluxes with the Dirichlet term
    size_t bytes = 0;
};

namespace {

__device__ __forceinline__ int slot_pos(const int* list, int i, int qq)
{
    const int f = i / qq;
    return list[f] * qq + (i - f * qq);
}

// M = [W | T^a_31 T^b_32 | I] of each merge, rows of pitch ldm, padded rows
// and columns of W an identity so the LU stays regular.
__global__ void k_if_gather_lu(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad,
                               int e_pad, double* __restrict__ M, long long ldm, long long sM)
{
    const IfDesc d = desc[blockIdx.y];
    const int i = blockIdx.x;
    double* row = M + (long long)blockIdx.y * sM + (long long)i * ldm;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    const double* Ra = nullptr;
    const double* Rb = nullptr;
    if (i < s) {
        Ra = d.Ta + (long long)slot_pos(a3, i, qq) * d.lda;
        Rb = d.Tb + (long long)slot_pos(b3, i, qq) * d.ldb;
    }
    const int c_rhs = s_pad, c_id = s_pad + e_pad, c_end = s_pad + e_pad + s_pad;
    for (int j = threadIdx.x; j < ldm; j += blockDim.x) {
        double v = 0.0;
        if (j < c_rhs) {
            if (i < s) {
                if (j < s) v = Ra[slot_pos(a3, j, qq)] + Rb[slot_pos(b3, j, qq)];
            } else if (j == i) {
                v = 1.0;
            }
        } else if (j < c_id) {
            const int jj = j - c_rhs;
            if (i < s) {
                if (jj < ea) v = Ra[slot_pos(a1, jj, qq)];
                else if (jj < ea + eb) v = Rb[slot_pos(b2, jj - ea, qq)];
            }
        } else if (j < c_end) {
            v = (j - c_id == i) ? 1.0 : 0.0;
        }
        row[j] = v;
    }
}

// E = [T^a_13; T^b_23] and the block diagonal diag(T^a_11, T^b_22) that the
// merged map starts from.
__global__ void k_if_gather_et(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad,
                               int e_pad, double* __restrict__ E, double* __restrict__ Tn)
{
    const IfDesc d = desc[blockIdx.y];
    const int i = blockIdx.x;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    double* Er = E + (long long)blockIdx.y * e_pad * s_pad + (long long)i * s_pad;
    double* Tr = Tn + (long long)blockIdx.y * e_pad * e_pad + (long long)i * e_pad;
    const double* R = nullptr;
    const int* sep = nullptr;
    const int* own = nullptr;
    int c0 = 0, c1 = 0;
    if (i < ea) {
        R = d.Ta + (long long)slot_pos(a1, i, qq) * d.lda;
        sep = a3; own = a1; c0 = 0; c1 = ea;
    } else if (i < ea + eb) {
        R = d.Tb + (long long)slot_pos(b2, i - ea, qq) * d.ldb;
        sep = b3; own = b2; c0 = ea; c1 = ea + eb;
    }
    for (int j = threadIdx.x; j < s_pad; j += blockDim.x)
        Er[j] = (R && j < s) ? R[slot_pos(sep, j, qq)] : 0.0;
    for (int j = threadIdx.x; j < e_pad; j += blockDim.x)
        Tr[j] = (R && j >= c0 && j < c1) ? R[slot_pos(own, j - c0, qq)] : 0.0;
}

// S = -X[:, 0:e_pad] and W^{-1} = X[:, e_pad:e_pad+s_pad] from the solved
// right-hand-side columns of M.
__global__ void k_if_extract(const double* __restrict__ M, long long ldm, long long sM, int s_pad, int e_pad,
                             double* __restrict__ S, double* __restrict__ Winv)
{
    const int i = blockIdx.x, node = blockIdx.y;
    const double* X = M + (long long)node * sM + (long long)i * ldm + s_pad;
    double* Sr = S + ((long long)node * s_pad + i) * e_pad;
    double* Wr = Winv + ((long long)node * s_pad + i) * s_pad;
    for (int j = threadIdx.x; j < e_pad; j += blockDim.x) Sr[j] = -X[j];
    for (int j = threadIdx.x; j < s_pad; j += blockDim.x) Wr[j] = X[e_pad + j];
}

// Leaf fluxes with the known outer values moved over: hl = h + T[:, D] g_D,
// and u_b = g on the outer faces (0 without g).  One thread per (box, load, row).
__global__ void k_if_leaf_dirichlet(int nbox, int nrhs, int m, int qq, const int* __restrict__ dinfo,
                                    const double* __restrict__ TD, const double* __restrict__ h,
                                    const double* __restrict__ g, double* __restrict__ hl, double* __restrict__ ub)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)nbox * nrhs * m;
    if (t >= total) return;
    const int r = (int)(t % m);
    const long long bc = t / m;
    const int box = (int)(bc / nrhs);
    const int* di = dinfo + 8 * box;
    const int nd = di[0];
    const double* gb = g ? g + bc * m : nullptr;
    if (hl) {
        double acc = h[t];
        if (gb)
            for (int k = 0; k < nd; ++k) {
                const double* Tk = TD + ((long long)(di[1] + k) * m + r) * qq;
                const double* gk = gb + di[2 + k] * qq;
                for (int l = 0; l < qq; ++l) acc += Tk[l] * gk[l];
            }
        hl[t] = acc;
    }
    const int f = r / qq;
    for (int k = 0; k < nd; ++k)
        if (di[2 + k] == f) ub[t] = gb ? gb[r] : 0.0;
}

// Upward gather of one level: t3 = h^a_3 + h^b_3, hv = [h^a_1; h^b_2].
// A leaf child's fluxes come from hsrc [nbox][nrhs][m].
__global__ void k_if_up(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad, int e_pad,
                        int nrhs, int m, const double* __restrict__ hsrc, double* __restrict__ t3,
                        double* __restrict__ hv)
{
    const IfDesc d = desc[blockIdx.y];
    const int rows = s_pad > e_pad ? s_pad : e_pad;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * nrhs) return;
    const int i = idx / nrhs, c = idx - i * nrhs;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    auto va = [&](int pos) {
        return d.leafa >= 0 ? hsrc[((long long)d.leafa * nrhs + c) * m + pos] : d.va[(d.oa + pos) * nrhs + c];
    };
    auto vb = [&](int pos) {
        return d.leafb >= 0 ? hsrc[((long long)d.leafb * nrhs + c) * m + pos] : d.vb[(d.ob + pos) * nrhs + c];
    };
    if (i < s_pad)
        t3[((long long)blockIdx.y * s_pad + i) * nrhs + c] =
            i < s ? va(slot_pos(a3, i, qq)) + vb(slot_pos(b3, i, qq)) : 0.0;
    if (i < e_pad) {
        double v = 0.0;
        if (i < ea) v = va(slot_pos(a1, i, qq));
        else if (i < ea + eb) v = vb(slot_pos(b2, i - ea, qq));
        hv[((long long)blockIdx.y * e_pad + i) * nrhs + c] = v;
    }
}

// Downward scatter of one level: each child receives its outer values from
// the parent's boundary values uv and its separator values u_3 = t3 - y
// (t3 holding S [u_1; u_2]).  A leaf child writes u_b [nbox][nrhs][m].
__global__ void k_if_down(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad,
                          int e_pad, int nrhs, int m, const double* __restrict__ uv, const double* __restrict__ t3,
                          const double* __restrict__ y, double* __restrict__ ub)
{
    const IfDesc d = desc[blockIdx.y];
    const int rows = s_pad > e_pad ? s_pad : e_pad;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * nrhs) return;
    const int i = idx / nrhs, c = idx - i * nrhs;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    auto put_a = [&](int pos, double v) {
        if (d.leafa >= 0) ub[((long long)d.leafa * nrhs + c) * m + pos] = v;
        else d.wa[(d.oa + pos) * nrhs + c] = v;
    };
    auto put_b = [&](int pos, double v) {
        if (d.leafb >= 0) ub[((long long)d.leafb * nrhs + c) * m + pos] = v;
        else d.wb[(d.ob + pos) * nrhs + c] = v;
    };
    if (i < s) {
        const long long o = ((long long)blockIdx.y * s_pad + i) * nrhs + c;
        const double u3 = t3[o] - y[o];
        put_a(slot_pos(a3, i, qq), u3);
        put_b(slot_pos(b3, i, qq), u3);
    }
    if (i < ea + eb) {
        const double v = uv[((long long)blockIdx.y * e_pad + i) * nrhs + c];
        if (i < ea) put_a(slot_pos(a1, i, qq), v);
        else put_b(slot_pos(b2, i - ea, qq), v);
    }
}

// O = [acc] O + alpha A B for a batch of small-N products (N = nrhs <= 16,
// NC columns per pass).  TPR threads share one output row (32 .. 256, sized
// to K so that each thread reads a few elements of it) and a CTA of 256
// threads takes 256 / TPR rows: rows of A are read once, coalesced, with
// enough loads in flight per SM whether a level has one merge or hundreds.
// Partial sums are joined by warp shuffles, across warps through shared
// memory.  A [M][K] (pitch lda), B [K][N], O [M][N].
template <int NC, int TPR>
__global__ void __launch_bounds__(256) k_if_mv(int Mr, int K, int N, const double* __restrict__ A, long long lda,
                                               long long sA, const double* __restrict__ B, long long sB,
                                               double* __restrict__ O, long long sO, double alpha, int acc)
{
    constexpr int RPC = 256 / TPR, WPR = TPR / 32;
    __shared__ double red[8][NC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = threadIdx.x % TPR, rloc = threadIdx.x / TPR;
    const int row = blockIdx.x * RPC + rloc;
    const bool live = row < Mr;
    const double* Ar = A + (long long)blockIdx.y * sA + (long long)(live ? row : 0) * lda;
    const double* Bb = B + (long long)blockIdx.y * sB;
    double* Or = O + (long long)blockIdx.y * sO + (long long)row * N;
    for (int c0 = 0; c0 < N; c0 += NC) {
        double s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = 0.0;
        if (live) {
#pragma unroll 4
            for (int k = t; k < K; k += TPR) {
                const double a = Ar[k];
                const double* Bk = Bb + (long long)k * N + c0;
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (c0 + c < N) s[c] += a * Bk[c];
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        }
        if (WPR == 1) {
            if (live) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (lane == c && c0 + c < N) Or[c0 + c] = (acc ? Or[c0 + c] : 0.0) + alpha * s[c];
            }
        } else {
            if (lane == 0) {
#pragma unroll
                for (int c = 0; c < NC; ++c) red[warp][c] = s[c];
            }
            __syncthreads();
            if (live && t < NC && c0 + t < N) {
                double v = 0.0;
#pragma unroll
                for (int w = 0; w < WPR; ++w) v += red[rloc * WPR + w][t];
                Or[c0 + t] = (acc ? Or[c0 + t] : 0.0) + alpha * v;
            }
            __syncthreads();
        }
    }
}

template <int NC>
void launch_mv(int nn, int Mr, int N, int K, const double* A, long long lda, long long sA, const double* B,
               long long sB, double* O, long long sO, double alpha, int acc, cudaStream_t st)
{
    // threads per row: about K / 8 elements each, 32 .. 256
    int tpr = 32;
    while (tpr < 256 && tpr * 8 < K) tpr *= 2;
    const unsigned rows_per_cta = 256 / tpr;
    dim3 grd((unsigned)((Mr + rows_per_cta - 1) / rows_per_cta), (unsigned)nn);
    if (tpr == 32) k_if_mv<NC, 32><<<grd, 256, 0, st>>>(Mr, K, N, A, lda, sA, B, sB, O, sO, alpha, acc);
    else if (tpr == 64) k_if_mv<NC, 64><<<grd, 256, 0, st>>>(Mr, K, N, A, lda, sA, B, sB, O, sO, alpha, acc);
    else if (tpr == 128) k_if_mv<NC, 128><<<grd, 256, 0, st>>>(Mr, K, N, A, lda, sA, B, sB, O, sO, alpha, acc);
    else k_if_mv<NC, 256><<<grd, 256, 0, st>>>(Mr, K, N, A, lda, sA, B, sB, O, sO, alpha, acc);
}

// O = [acc] O + alpha A B over the merges of a level: row-split products
// for few columns, the register-tiled CUDA-core product otherwise.
void if_product(int nn, int Mr, int N, int K, const double* A, long long lda, long long sA, const double* B,
                long long sB, double* O, long long sO, double alpha, bool acc, cudaStream_t st)
{
    if (Mr <= 0 || N <= 0 || nn <= 0) return;
    if (N <= 16) {
        hps::prof_begin(hps::KC_MISC, st);
        if (N <= 2) launch_mv<2>(nn, Mr, N, K, A, lda, sA, B, sB, O, sO, alpha, acc ? 1 : 0, st);
        else launch_mv<8>(nn, Mr, N, K, A, lda, sA, B, sB, O, sO, alpha, acc ? 1 : 0, st);
        hps::prof_end(hps::KC_MISC, st, 2.0 * nn * Mr * (double)N * K, 8.0 * nn * ((double)Mr * K + (double)Mr * N));
        return;
    }
    hps::GemmArgs<double> a{};
    a.A = A; a.lda = lda; a.sA = sA;
    a.B = B; a.ldb = N; a.sB = sB;
    a.O = O; a.ldo = N; a.sO = sO;
    a.M = Mr; a.N = N; a.K = K;
    a.alpha = alpha;
    a.mode = acc ? hps::GM_ACC : hps::GM_SET;
    hps::launch_gemm<double>(a, nn, st);
}

void free_interface(hps_interface* F)
{
    for (IfLevel& L : F->levels) {
        cudaFree(L.d_desc); cudaFree(L.d_lists); cudaFree(L.Winv); cudaFree(L.S); cudaFree(L.E);
        cudaFree(L.Tn); cudaFree(L.hv); cudaFree(L.uv); cudaFree(L.t3); cudaFree(L.y);
    }
    cudaFree(F->TD);
    cudaFree(F->d_dinfo);
    cudaFree(F->hl);
}

#define IF_TRY(expr)                                         \
    do {                                                     \
        if ((expr) != cudaSuccess) { cudaGetLastError(); rc = HPS_ENOMEM; goto fail; } \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count, size_t* total)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    *total += sizeof(T) * count;
    return cudaMalloc(p, sizeof(T) * count);
}

}  // namespace

extern "C" {

hps_status hps_interface_factor(hps_ctx* ctx, int p, const int nb[3], const double* T, int nrhs_max, void* stream,
                                hps_interface** out)
{
    if (!out) return HPS_EINVAL;
    *out = nullptr;
    if (!ctx || !T || nrhs_max < 1 || nrhs_max > 256) return HPS_EINVAL;
    hps_interface* F = new (std::nothrow) hps_interface();
    if (!F) return HPS_ENOMEM;
    if (!hps::build_iface_plan(p, nb, &F->plan)) { delete F; return HPS_EINVAL; }
    F->device = hps::ctx_device(ctx);
    if (cudaSetDevice(F->device) != cudaSuccess) { delete F; return HPS_ECUDA; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const IfPlan& P = F->plan;
    F->p = p;
    F->q = p - 2;
    F->qq = F->q * F->q;
    F->m = 6 * F->qq;
    F->nbox = P.nbox;
    F->nrhs_max = nrhs_max;
    const int qq = F->qq, m = F->m, R = nrhs_max;
    hps_status rc = HPS_OK;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int* d_status = nullptr;
    size_t status_cap = 0;
    std::vector<int> level_of(P.nodes.size(), -1), index_in(P.nodes.size(), -1);

    // Outer faces of the leaves: copy T's columns there.
    F->dinfo.assign((size_t)8 * P.nbox, 0);
    for (int box = 0; box < P.nbox; ++box) {
        int* di = &F->dinfo[(size_t)8 * box];
        di[1] = F->ndface;
        for (int f = 0; f < 6; ++f)
            if (!P.nodes[box].leaf_iface[f]) di[2 + di[0]++] = f;
        F->ndface += di[0];
    }
    IF_TRY(dalloc(&F->TD, (size_t)F->ndface * m * qq, &F->bytes));
    IF_TRY(dalloc(&F->d_dinfo, F->dinfo.size(), &F->bytes));
    IF_TRY(cudaMemcpy(F->d_dinfo, F->dinfo.data(), sizeof(int) * F->dinfo.size(), cudaMemcpyHostToDevice));
    IF_TRY(dalloc(&F->hl, (size_t)P.nbox * R * m, &F->bytes));
    for (int box = 0; box < P.nbox; ++box) {
        const int* di = &F->dinfo[(size_t)8 * box];
        for (int k = 0; k < di[0]; ++k)
            IF_TRY(cudaMemcpy2DAsync(F->TD + (size_t)(di[1] + k) * m * qq, sizeof(double) * qq,
                                     T + (size_t)box * m * m + (size_t)di[2 + k] * qq, sizeof(double) * m,
                                     sizeof(double) * qq, m, cudaMemcpyDeviceToDevice, st));
    }

    // Level sizes and buffers.
    F->levels.resize(P.levels.size());
    for (size_t lv = 0; lv < P.levels.size(); ++lv) {
        IfLevel& L = F->levels[lv];
        L.ids = P.levels[lv];
        L.nn = (int)L.ids.size();
        for (int k = 0; k < L.nn; ++k) {
            const IfNode& N = P.nodes[L.ids[k]];
            L.s_pad = std::max(L.s_pad, (int)N.a3.size() * qq);
            L.e_pad = std::max(L.e_pad, (int)(N.a1.size() + N.b2.size()) * qq);
            level_of[L.ids[k]] = (int)lv;
            index_in[L.ids[k]] = k;
        }
        if (L.s_pad > kMaxSeparator) { rc = HPS_ENOMEM; goto fail; }
        const size_t nn = L.nn, s = L.s_pad, e = L.e_pad;
        IF_TRY(dalloc(&L.Winv, nn * s * s, &F->bytes));
        IF_TRY(dalloc(&L.S, nn * s * e, &F->bytes));
        IF_TRY(dalloc(&L.E, nn * e * s, &F->bytes));
        IF_TRY(dalloc(&L.hv, nn * e * R, &F->bytes));
        IF_TRY(dalloc(&L.uv, nn * e * R, &F->bytes));
        // rows of uv beyond a merge's own boundary stay zero: S has zero columns there
        if (L.uv) IF_TRY(cudaMemsetAsync(L.uv, 0, sizeof(double) * nn * e * R, st));
        IF_TRY(dalloc(&L.t3, nn * s * R, &F->bytes));
        IF_TRY(dalloc(&L.y, nn * s * R, &F->bytes));
        size_t tmp = 0;
        IF_TRY(dalloc(&L.Tn, nn * e * e, &tmp));
    }
    // Descriptors (children's maps and vectors now have addresses).
    for (size_t lv = 0; lv < F->levels.size(); ++lv) {
        IfLevel& L = F->levels[lv];
        L.desc.resize(L.nn);
        L.lists.clear();
        for (int k = 0; k < L.nn; ++k) {
            const IfNode& N = P.nodes[L.ids[k]];
            IfDesc& d = L.desc[k];
            std::memset(&d, 0, sizeof(d));
            for (int side = 0; side < 2; ++side) {
                const int c = N.child[side];
                const double* Tc;
                long long ld;
                double *vc = nullptr, *wc = nullptr;
                long long oc = 0;
                int leaf = -1;
                if (c < P.nbox) {
                    Tc = T + (size_t)c * m * m;
                    ld = m;
                    leaf = c;
                } else {
                    const IfLevel& C = F->levels[level_of[c]];
                    const size_t ci = index_in[c];
                    Tc = C.Tn + ci * C.e_pad * C.e_pad;
                    ld = C.e_pad;
                    vc = C.hv;
                    wc = C.uv;
                    oc = (long long)ci * C.e_pad;
                }
                if (side == 0) { d.Ta = Tc; d.lda = ld; d.va = vc; d.wa = wc; d.oa = oc; d.leafa = leaf; }
                else { d.Tb = Tc; d.ldb = ld; d.vb = vc; d.wb = wc; d.ob = oc; d.leafb = leaf; }
            }
            d.na1 = (int)N.a1.size();
            d.nsep = (int)N.a3.size();
            d.nb2 = (int)N.b2.size();
            d.loff = (int)L.lists.size();
            for (int v : N.a1) L.lists.push_back(v);
            for (int v : N.a3) L.lists.push_back(v);
            for (int v : N.b2) L.lists.push_back(v);
            for (int v : N.b3) L.lists.push_back(v);
        }
        IF_TRY(dalloc(&L.d_desc, L.desc.size(), &F->bytes));
        IF_TRY(dalloc(&L.d_lists, std::max<size_t>(L.lists.size(), 1), &F->bytes));
        IF_TRY(cudaMemcpy(L.d_desc, L.desc.data(), sizeof(IfDesc) * L.desc.size(), cudaMemcpyHostToDevice));
        if (!L.lists.empty())
            IF_TRY(cudaMemcpy(L.d_lists, L.lists.data(), sizeof(int) * L.lists.size(), cudaMemcpyHostToDevice));
    }

    // Factorisation, level by level.
    for (size_t lv = 0; lv < F->levels.size(); ++lv) {
        IfLevel& L = F->levels[lv];
        const int s = L.s_pad, e = L.e_pad;
        hps::Plan PL = hps::make_plan(s, e + s, HPS_FP64, 64, false, false);
        const size_t need = PL.per_box * (size_t)L.nn;
        if (need > ws_bytes) {
            if (ws) { cudaStreamSynchronize(st); cudaFree(ws); ws = nullptr; ws_bytes = 0; }
            IF_TRY(cudaMalloc(&ws, need));
            ws_bytes = need;
        }
        if ((size_t)L.nn > status_cap) {
            if (d_status) { cudaStreamSynchronize(st); cudaFree(d_status); d_status = nullptr; }
            IF_TRY(cudaMalloc(&d_status, sizeof(int) * L.nn));
            status_cap = L.nn;
        }
        hps::Work<double> w = hps::carve<double>(PL, ws, L.nn);
        IF_TRY(cudaMemsetAsync(d_status, 0, sizeof(int) * L.nn, st));
        k_if_gather_lu<<<dim3((unsigned)s, (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e, w.M, PL.ldm,
                                                                           w.sM);
        if (e > 0)
            k_if_gather_et<<<dim3((unsigned)e, (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e, L.E,
                                                                              L.Tn);
        hps::lu_factor<double>(PL, w, L.nn, d_status, st);
        hps::lu_backward<double>(PL, w, L.nn, s, e + s, nullptr, st);
        k_if_extract<<<dim3((unsigned)s, (unsigned)L.nn), 256, 0, st>>>(w.M, PL.ldm, w.sM, s, e, L.S, L.Winv);
        if (e > 0) if_product(L.nn, e, e, s, L.E, s, (long long)e * s, L.S, (long long)s * e, L.Tn,
                              (long long)e * e, 1.0, true, st);
        if (cudaGetLastError() != cudaSuccess) { rc = HPS_ECUDA; goto fail; }
        std::vector<int> hs(L.nn);
        if (cudaMemcpyAsync(hs.data(), d_status, sizeof(int) * L.nn, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { rc = HPS_ECUDA; goto fail; }
        for (int v : hs)
            if (v != 0) { rc = (hps_status)v; goto fail; }
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) { rc = HPS_ECUDA; goto fail; }
    for (IfLevel& L : F->levels) { cudaFree(L.Tn); L.Tn = nullptr; }
    cudaFree(ws);
    cudaFree(d_status);
    *out = F;
    return HPS_OK;
fail:
    cudaStreamSynchronize(st);
    cudaFree(ws);
    cudaFree(d_status);
    free_interface(F);
    delete F;
    return rc;
}

hps_status hps_interface_solve(hps_interface* F, int nrhs, const double* h, const double* g, double* ub,
                               void* stream)
{
    if (!F || nrhs < 1 || nrhs > F->nrhs_max || !h || !ub) return HPS_EINVAL;
    if (cudaSetDevice(F->device) != cudaSuccess) return HPS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int qq = F->qq, m = F->m, R = nrhs;
    {
        const long long total = (long long)F->nbox * R * m;
        hps::prof_begin(hps::KC_MISC, st);
        k_if_leaf_dirichlet<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            F->nbox, R, m, qq, F->d_dinfo, F->TD, h, g, g ? F->hl : nullptr, ub);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * (double)total * (g ? 4 : 1));
    }
    const double* hsrc = g ? F->hl : h;
    // Upward: fluxes of every merged box.
    for (IfLevel& L : F->levels) {
        const int s = L.s_pad, e = L.e_pad, rows = std::max(s, e);
        const long long n = (long long)rows * R;
        hps::prof_begin(hps::KC_MISC, st);
        k_if_up<<<dim3((unsigned)((n + 255) / 256), (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e, R,
                                                                                    m, hsrc, L.t3, L.hv);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * L.nn * (double)n * 3);
        if_product(L.nn, s, R, s, L.Winv, s, (long long)s * s, L.t3, (long long)s * R, L.y, (long long)s * R, 1.0,
                   false, st);
        if (e > 0) if_product(L.nn, e, R, s, L.E, s, (long long)e * s, L.y, (long long)s * R, L.hv,
                              (long long)e * R, -1.0, true, st);
    }
    // Downward: separator values, then every child's boundary values.
    for (size_t lv = F->levels.size(); lv-- > 0;) {
        IfLevel& L = F->levels[lv];
        const int s = L.s_pad, e = L.e_pad, rows = std::max(s, e);
        const long long n = (long long)rows * R;
        if (e > 0) if_product(L.nn, s, R, e, L.S, e, (long long)s * e, L.uv, (long long)e * R, L.t3,
                              (long long)s * R, 1.0, false, st);
        else if (cudaMemsetAsync(L.t3, 0, sizeof(double) * (size_t)L.nn * s * R, st) != cudaSuccess) return HPS_ECUDA;
        hps::prof_begin(hps::KC_MISC, st);
        k_if_down<<<dim3((unsigned)((n + 255) / 256), (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e,
                                                                                      R, m, L.uv, L.t3, L.y, ub);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * L.nn * (double)n * 4);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status hps_interface_info(const hps_interface* F, int* n_merge, int* n_levels, int* max_separator, size_t* bytes)
{
    if (!F) return HPS_EINVAL;
    int nm = 0, ms = 0;
    for (const IfLevel& L : F->levels) {
        nm += L.nn;
        ms = std::max(ms, L.s_pad);
    }
    if (n_merge) *n_merge = nm;
    if (n_levels) *n_levels = (int)F->levels.size();
    if (max_separator) *max_separator = ms;
    if (bytes) *bytes = F->bytes;
    return HPS_OK;
}

void hps_interface_destroy(hps_interface* F)
{
    if (!F) return;
    cudaSetDevice(F->device);
    cudaDeviceSynchronize();
    free_interface(F);
    delete F;
}

}  // extern "C"
