// Interface solve on the GPU: nested dissection of the interface system over
// the box grid, factored and solved level by level with batched kernels.
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
// of a level is one batch of the library's blocked LU with partial pivoting
// (W carrying [T^a_31 T^b_32 | I] as right-hand sides), and the solve is two
// sweeps of batched matrix-vector products: up the tree for h, down for u.
//
// Two precisions.  HPS_FP64 keeps every factor in FP64.  HPS_FP32_IR factors
// and stores in FP32 (CUDA-core FP32 LU and products, 64 times the FP64 issue
// rate on this part, half the bytes per solve) and recovers FP64 accuracy in
// each solve by iterative refinement on the interface system itself: with
// u_k the current face values, each box's flux T^tau u_k^tau + h^tau (FP64,
// the caller's maps kept as a copy) sums, over the boxes sharing a node, to
// the residual of the interface equations, so solving the same system with
// those fluxes as loads gives the correction.  Corrections stop on the
// device once they are below 1e-14 relative or stop shrinking.
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
    const double* Ta;   // factorisation: a leaf child's DtN map (T + box m^2, FP64), else NULL
    const double* Tb;
    const void* Ma;     // factorisation: a merge child's map (its level's storage type), else NULL
    const void* Mb;
    long long lda, ldb; // row pitch of the child's map
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
    void* Winv = nullptr;     // [nn][s_pad][s_pad]   (storage type: double or float)
    void* S = nullptr;        // [nn][s_pad][e_pad]
    void* E = nullptr;        // [nn][e_pad][s_pad]
    void* Tn = nullptr;       // factorisation only: merged maps [nn][e_pad][e_pad]
    double* hv = nullptr;     // solve: merged fluxes [nn][e_pad][nrhs]
    double* uv = nullptr;     // solve: boundary values [nn][e_pad][nrhs]
    double* t3 = nullptr;     // solve: h^a_3 + h^b_3, then reused for S [u_1; u_2] [nn][s_pad][nrhs]
    double* y = nullptr;      // solve: W^{-1} (h^a_3 + h^b_3) [nn][s_pad][nrhs]
};

constexpr int kMaxSeparator = 14000;   // the panel keeps a column of W in shared memory
constexpr int kRefineMax = 10;         // FP32_IR: most corrections per solve
constexpr double kRefineTol = 1e-14;   // FP32_IR: stop when ||du|| <= tol ||u||

}  // namespace

struct hps_interface {
    int device = 0;
    int p = 0, q = 0, qq = 0, m = 0, nbox = 0, nrhs_max = 0;
    bool fp32 = false;                 // HPS_FP32_IR: FP32 factors, FP64 refinement in each solve
    IfPlan plan;
    std::vector<IfLevel> levels;
    // Dirichlet faces of the leaves: per box, the columns of T on its outer faces
    double* TD = nullptr;          // [ndface][m][qq]
    int* d_dinfo = nullptr;        // [nbox][8]: count, first block, then the local faces
    std::vector<int> dinfo;
    int ndface = 0;
    double* hl = nullptr;          // [nbox][nrhs][m]: leaf fluxes with the Dirichlet term
    // FP32_IR refinement
    double* Tcopy = nullptr;       // [nbox][m][m]: the leaf maps (FP64)
    double* hcur = nullptr;        // [nbox][nrhs][m]: fluxes of the current face values
    double* du = nullptr;          // [nbox][nrhs][m]: the correction
    double* rstat = nullptr;       // [4]: ||du||^2, ||u||^2, previous ||du||^2, last relative correction
    int* rflag = nullptr;          // [2]: converged, corrections taken
    size_t bytes = 0;
};

namespace {

__device__ __forceinline__ int slot_pos(const int* list, int i, int qq)
{
    const int f = i / qq;
    return list[f] * qq + (i - f * qq);
}

// Row r of a child's map (leaf: FP64 map of the box; merge: its stored map).
template <typename MT>
struct MapRow {
    const double* d;
    const MT* f;
    __device__ double operator[](int j) const { return d ? d[j] : (double)f[j]; }
};

template <typename MT>
__device__ __forceinline__ MapRow<MT> map_row(const double* T, const void* M, long long ld, int r)
{
    MapRow<MT> R;
    R.d = T ? T + (long long)r * ld : nullptr;
    R.f = T ? nullptr : static_cast<const MT*>(M) + (long long)r * ld;
    return R;
}

// M = [W | T^a_31 T^b_32 | I] of each merge, rows of pitch ldm, padded rows
// and columns of W an identity so the LU stays regular.
template <typename MT>
__global__ void k_if_gather_lu(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad,
                               int e_pad, MT* __restrict__ M, long long ldm, long long sM)
{
    const IfDesc d = desc[blockIdx.y];
    const int i = blockIdx.x;
    MT* row = M + (long long)blockIdx.y * sM + (long long)i * ldm;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    MapRow<MT> Ra{nullptr, nullptr}, Rb{nullptr, nullptr};
    if (i < s) {
        Ra = map_row<MT>(d.Ta, d.Ma, d.lda, slot_pos(a3, i, qq));
        Rb = map_row<MT>(d.Tb, d.Mb, d.ldb, slot_pos(b3, i, qq));
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
        row[j] = (MT)v;
    }
}

// E = [T^a_13; T^b_23] and the block diagonal diag(T^a_11, T^b_22) that the
// merged map starts from.
template <typename MT>
__global__ void k_if_gather_et(const IfDesc* __restrict__ desc, const int* __restrict__ lists, int qq, int s_pad,
                               int e_pad, MT* __restrict__ E, MT* __restrict__ Tn)
{
    const IfDesc d = desc[blockIdx.y];
    const int i = blockIdx.x;
    const int* a1 = lists + d.loff;
    const int* a3 = a1 + d.na1;
    const int* b2 = a3 + d.nsep;
    const int* b3 = b2 + d.nb2;
    const int s = d.nsep * qq, ea = d.na1 * qq, eb = d.nb2 * qq;
    MT* Er = E + (long long)blockIdx.y * e_pad * s_pad + (long long)i * s_pad;
    MT* Tr = Tn + (long long)blockIdx.y * e_pad * e_pad + (long long)i * e_pad;
    MapRow<MT> R{nullptr, nullptr};
    bool have = false;
    const int* sep = nullptr;
    const int* own = nullptr;
    int c0 = 0, c1 = 0;
    if (i < ea) {
        R = map_row<MT>(d.Ta, d.Ma, d.lda, slot_pos(a1, i, qq));
        have = true; sep = a3; own = a1; c0 = 0; c1 = ea;
    } else if (i < ea + eb) {
        R = map_row<MT>(d.Tb, d.Mb, d.ldb, slot_pos(b2, i - ea, qq));
        have = true; sep = b3; own = b2; c0 = ea; c1 = ea + eb;
    }
    for (int j = threadIdx.x; j < s_pad; j += blockDim.x)
        Er[j] = (MT)((have && j < s) ? R[slot_pos(sep, j, qq)] : 0.0);
    for (int j = threadIdx.x; j < e_pad; j += blockDim.x)
        Tr[j] = (MT)((have && j >= c0 && j < c1) ? R[slot_pos(own, j - c0, qq)] : 0.0);
}

// S = -X[:, 0:e_pad] and W^{-1} = X[:, e_pad:e_pad+s_pad] from the solved
// right-hand-side columns of M.
template <typename MT>
__global__ void k_if_extract(const MT* __restrict__ M, long long ldm, long long sM, int s_pad, int e_pad,
                             MT* __restrict__ S, MT* __restrict__ Winv)
{
    const int i = blockIdx.x, node = blockIdx.y;
    const MT* X = M + (long long)node * sM + (long long)i * ldm + s_pad;
    MT* Sr = S + ((long long)node * s_pad + i) * e_pad;
    MT* Wr = Winv + ((long long)node * s_pad + i) * s_pad;
    for (int j = threadIdx.x; j < e_pad; j += blockDim.x) Sr[j] = -X[j];
    for (int j = threadIdx.x; j < s_pad; j += blockDim.x) Wr[j] = X[e_pad + j];
}

// Leaf fluxes with the known outer values moved over: hl = h + T[:, D] g_D,
// and u_b = g on the outer faces (0 without g).  One thread per (box, load, row).
__global__ void k_if_leaf_dirichlet(int nbox, int nrhs, int m, int qq, const int* __restrict__ dinfo,
                                    const double* __restrict__ TD, const double* __restrict__ h,
                                    const double* __restrict__ g, double* __restrict__ hl, double* __restrict__ ub,
                                    const int* __restrict__ skip)
{
    if (skip && *skip) return;
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
                        double* __restrict__ hv, const int* __restrict__ skip)
{
    if (skip && *skip) return;
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
                          const double* __restrict__ y, double* __restrict__ ub, const int* __restrict__ skip)
{
    if (skip && *skip) return;
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
// NC columns per pass), A in the storage type MT, B and O in FP64, sums in
// FP64.  TPR threads share one output row (32 .. 256, sized to K so that each
// thread reads a few elements of it) and a CTA of 256 threads takes 256 / TPR
// rows: rows of A are read once, coalesced, with enough loads in flight per
// SM whether a level has one merge or hundreds.  Partial sums are joined by
// warp shuffles, across warps through shared memory.  A [M][K] (pitch lda);
// B element (k, c) at k bk + c bc; O element (r, c) at r ok + c oc.
template <int NC, int TPR, typename MT>
__global__ void __launch_bounds__(256) k_if_mv(int Mr, int K, int N, const MT* __restrict__ A, long long lda,
                                               long long sA, const double* __restrict__ B, long long sB,
                                               long long bk, long long bc, double* __restrict__ O, long long sO,
                                               long long ok, long long oc, double alpha, int acc,
                                               const int* __restrict__ skip)
{
    constexpr int RPC = 256 / TPR, WPR = TPR / 32;
    if (skip && *skip) return;
    __shared__ double red[8][NC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t = threadIdx.x % TPR, rloc = threadIdx.x / TPR;
    const int row = blockIdx.x * RPC + rloc;
    const bool live = row < Mr;
    const MT* Ar = A + (long long)blockIdx.y * sA + (long long)(live ? row : 0) * lda;
    const double* Bb = B + (long long)blockIdx.y * sB;
    double* Or = O + (long long)blockIdx.y * sO + (long long)row * ok;
    for (int c0 = 0; c0 < N; c0 += NC) {
        double s[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = 0.0;
        if (live) {
#pragma unroll 4
            for (int k = t; k < K; k += TPR) {
                const double a = (double)Ar[k];
                const double* Bk = Bb + (long long)k * bk + (long long)c0 * bc;
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (c0 + c < N) s[c] += a * Bk[c * bc];
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
                    if (lane == c && c0 + c < N) {
                        double* o = Or + (long long)(c0 + c) * oc;
                        *o = (acc ? *o : 0.0) + alpha * s[c];
                    }
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
                double* o = Or + (long long)(c0 + t) * oc;
                *o = (acc ? *o : 0.0) + alpha * v;
            }
            __syncthreads();
        }
    }
}

template <int NC, typename MT>
void launch_mv(int nn, int Mr, int N, int K, const MT* A, long long lda, long long sA, const double* B, long long sB,
               long long bk, long long bc, double* O, long long sO, long long ok, long long oc, double alpha, int acc,
               const int* skip, cudaStream_t st)
{
    // threads per row: about K / 8 elements each, 32 .. 256
    int tpr = 32;
    while (tpr < 256 && tpr * 8 < K) tpr *= 2;
    const unsigned rows_per_cta = 256 / tpr;
    dim3 grd((unsigned)((Mr + rows_per_cta - 1) / rows_per_cta), (unsigned)nn);
#define IF_MV(TP) \
    k_if_mv<NC, TP, MT><<<grd, 256, 0, st>>>(Mr, K, N, A, lda, sA, B, sB, bk, bc, O, sO, ok, oc, alpha, acc, skip)
    if (tpr == 32) IF_MV(32);
    else if (tpr == 64) IF_MV(64);
    else if (tpr == 128) IF_MV(128);
    else IF_MV(256);
#undef IF_MV
}

// O = [acc] O + alpha A B over the merges of a level (B [K][N], O [M][N]):
// row-split products, A in the storage type MT.
template <typename MT>
void if_product(int nn, int Mr, int N, int K, const MT* A, long long lda, long long sA, const double* B, long long sB,
                double* O, long long sO, double alpha, bool acc, const int* skip, cudaStream_t st)
{
    if (Mr <= 0 || N <= 0 || nn <= 0) return;
    if (sizeof(MT) == sizeof(double) && N > 16 && !skip) {
        // many loads: the register-tiled CUDA-core product reads A once per 64 columns
        hps::GemmArgs<double> a{};
        a.A = reinterpret_cast<const double*>(A); a.lda = lda; a.sA = sA;
        a.B = B; a.ldb = N; a.sB = sB;
        a.O = O; a.ldo = N; a.sO = sO;
        a.M = Mr; a.N = N; a.K = K;
        a.alpha = alpha;
        a.mode = acc ? hps::GM_ACC : hps::GM_SET;
        hps::launch_gemm<double>(a, nn, st);
        return;
    }
    hps::prof_begin(hps::KC_MISC, st);
    if (N <= 2) launch_mv<2, MT>(nn, Mr, N, K, A, lda, sA, B, sB, N, 1, O, sO, N, 1, alpha, acc ? 1 : 0, skip, st);
    else launch_mv<8, MT>(nn, Mr, N, K, A, lda, sA, B, sB, N, 1, O, sO, N, 1, alpha, acc ? 1 : 0, skip, st);
    hps::prof_end(hps::KC_MISC, st, 2.0 * nn * Mr * (double)N * K,
                  (double)nn * ((double)Mr * K * sizeof(MT) + 8.0 * (double)Mr * N));
}

// Merged maps of a level in the factorisation: Tn += E S (E [e][s], S [s][e]).
template <typename MT>
void if_merge_product(int nn, int e, int s, const MT* E, const MT* S, MT* Tn, cudaStream_t st)
{
    hps::GemmArgs<MT> a{};
    a.A = E; a.lda = s; a.sA = (long long)e * s;
    a.B = S; a.ldb = e; a.sB = (long long)s * e;
    a.O = Tn; a.ldo = e; a.sO = (long long)e * e;
    a.M = e; a.N = e; a.K = s;
    a.alpha = (MT)1;
    a.mode = hps::GM_ACC;
    hps::launch_gemm<MT>(a, nn, st);
}

// FP32_IR refinement: u += du over all face values, ||du||^2 and ||u||^2.
__global__ void k_if_update(long long total, const double* __restrict__ du, double* __restrict__ ub,
                            double* __restrict__ rstat, const int* __restrict__ skip)
{
    if (*skip) return;
    double a = 0.0, b = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const double d = du[t];
        const double u = ub[t] + d;
        ub[t] = u;
        a += d * d;
        b += u * u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(rstat + 0, a);
        atomicAdd(rstat + 1, b);
    }
}

// Stop once the correction is below tol relative or no longer shrinks by half.
__global__ void k_if_check(double* rstat, int* flag, double tol)
{
    if (flag[0]) return;
    const double d2 = rstat[0], u2 = rstat[1], prev = rstat[2];
    const double rel = u2 > 0.0 ? sqrt(d2 / u2) : 0.0;
    flag[1] += 1;
    rstat[3] = rel;
    if (!(rel > tol) || (prev >= 0.0 && d2 > 0.25 * prev)) flag[0] = 1;
    rstat[2] = d2;
    rstat[0] = 0.0;
    rstat[1] = 0.0;
}

__global__ void k_if_check_reset(double* rstat, int* flag)
{
    rstat[0] = 0.0;
    rstat[1] = 0.0;
    rstat[2] = -1.0;
    rstat[3] = 0.0;
    flag[0] = 0;
    flag[1] = 0;
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
    cudaFree(F->Tcopy);
    cudaFree(F->hcur);
    cudaFree(F->du);
    cudaFree(F->rstat);
    cudaFree(F->rflag);
}

#define IF_TRY(expr)                                         \
    do {                                                     \
        if ((expr) != cudaSuccess) { cudaGetLastError(); rc = HPS_ENOMEM; goto fail; } \
    } while (0)

cudaError_t dalloc_bytes(void** p, size_t bytes, size_t* total)
{
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    *total += bytes;
    return cudaMalloc(p, bytes);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count, size_t* total)
{
    void* v = nullptr;
    cudaError_t e = dalloc_bytes(&v, sizeof(T) * count, total);
    *p = static_cast<T*>(v);
    return e;
}

// One level of the factorisation in storage type MT; the LU workspace grows
// as needed.  Returns the first nonzero status of the level's LUs.
template <typename MT>
hps_status factor_level(IfLevel& L, int qq, void** ws, size_t* ws_bytes, int** d_status, size_t* status_cap,
                        cudaStream_t st)
{
    const int s = L.s_pad, e = L.e_pad;
    const hps_precision prec = sizeof(MT) == 8 ? HPS_FP64 : HPS_FP32_IR;
    // FP32 factors: the leaf path's tensor-core LU with 3 x BF16 operands and
    // FP32 accumulation (FP32's 24 bits: the interface systems are less well
    // conditioned than the leaves, and the scaled 2 x FP16 form's 22 bits
    // leave the refinement of some of them without contraction); the solve's
    // FP64 refinement recovers the digits
    const bool tc = sizeof(MT) == 4 && s >= 256;
    hps::Plan PL = hps::make_plan(s, e + s, tc ? HPS_BF16_IR : prec, 0, tc, false);
    const size_t need = PL.per_box * (size_t)L.nn;
    if (need > *ws_bytes) {
        if (*ws) { cudaStreamSynchronize(st); cudaFree(*ws); *ws = nullptr; *ws_bytes = 0; }
        if (cudaMalloc(ws, need) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
        *ws_bytes = need;
    }
    if ((size_t)L.nn > *status_cap) {
        if (*d_status) { cudaStreamSynchronize(st); cudaFree(*d_status); *d_status = nullptr; }
        if (cudaMalloc(d_status, sizeof(int) * L.nn) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
        *status_cap = L.nn;
    }
    hps::Work<MT> w = hps::carve<MT>(PL, *ws, L.nn);
    if (cudaMemsetAsync(*d_status, 0, sizeof(int) * L.nn, st) != cudaSuccess) return HPS_ECUDA;
    k_if_gather_lu<MT><<<dim3((unsigned)s, (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e, w.M, PL.ldm,
                                                                           w.sM);
    if (e > 0)
        k_if_gather_et<MT><<<dim3((unsigned)e, (unsigned)L.nn), 256, 0, st>>>(
            L.d_desc, L.d_lists, qq, s, e, static_cast<MT*>(L.E), static_cast<MT*>(L.Tn));
    bool tc_done = false;
    if constexpr (sizeof(MT) == 4) {
        if (PL.tc) {
            hps::tc_reset_abort(st);
            if (!hps::tc_lu_factor(PL, w, L.nn, *d_status, st) ||
                !hps::tc_lu_backward(PL, w, L.nn, s, e + s, nullptr, st))
                return HPS_ECUDA;
            tc_done = true;
        }
    }
    if (!tc_done) {
        hps::lu_factor<MT>(PL, w, L.nn, *d_status, st);
        hps::lu_backward<MT>(PL, w, L.nn, s, e + s, nullptr, st);
    }
    k_if_extract<MT><<<dim3((unsigned)s, (unsigned)L.nn), 256, 0, st>>>(w.M, PL.ldm, w.sM, s, e,
                                                                         static_cast<MT*>(L.S),
                                                                         static_cast<MT*>(L.Winv));
    if (e > 0)
        if_merge_product<MT>(L.nn, e, s, static_cast<const MT*>(L.E), static_cast<const MT*>(L.S),
                             static_cast<MT*>(L.Tn), st);
    if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
    std::vector<int> hs(L.nn);
    if (cudaMemcpyAsync(hs.data(), *d_status, sizeof(int) * L.nn, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return HPS_ECUDA;
    for (int v : hs)
        if (v != 0) return (hps_status)v;
    return HPS_OK;
}

// The elimination sweeps of one solve: u_b from the leaf fluxes h (and g).
template <typename MT>
void solve_sweeps(hps_interface* F, int R, const double* h, const double* g, double* ub, const int* skip,
                  cudaStream_t st)
{
    const int qq = F->qq, m = F->m;
    {
        const long long total = (long long)F->nbox * R * m;
        hps::prof_begin(hps::KC_MISC, st);
        k_if_leaf_dirichlet<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            F->nbox, R, m, qq, F->d_dinfo, F->TD, h, g, g ? F->hl : nullptr, ub, skip);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * (double)total * (g ? 4 : 1));
    }
    const double* hsrc = g ? F->hl : h;
    // Upward: fluxes of every merged box.
    for (IfLevel& L : F->levels) {
        const int s = L.s_pad, e = L.e_pad, rows = std::max(s, e);
        const long long n = (long long)rows * R;
        hps::prof_begin(hps::KC_MISC, st);
        k_if_up<<<dim3((unsigned)((n + 255) / 256), (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e, R,
                                                                                    m, hsrc, L.t3, L.hv, skip);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * L.nn * (double)n * 3);
        if_product<MT>(L.nn, s, R, s, static_cast<const MT*>(L.Winv), s, (long long)s * s, L.t3, (long long)s * R,
                       L.y, (long long)s * R, 1.0, false, skip, st);
        if (e > 0)
            if_product<MT>(L.nn, e, R, s, static_cast<const MT*>(L.E), s, (long long)e * s, L.y, (long long)s * R,
                           L.hv, (long long)e * R, -1.0, true, skip, st);
    }
    // Downward: separator values, then every child's boundary values.
    for (size_t lv = F->levels.size(); lv-- > 0;) {
        IfLevel& L = F->levels[lv];
        const int s = L.s_pad, e = L.e_pad, rows = std::max(s, e);
        const long long n = (long long)rows * R;
        // e = 0 (the root): S [u_1; u_2] is empty and the product writes zeros
        if_product<MT>(L.nn, s, R, e, static_cast<const MT*>(L.S), e, (long long)s * e, L.uv, (long long)e * R, L.t3,
                       (long long)s * R, 1.0, false, skip, st);
        hps::prof_begin(hps::KC_MISC, st);
        k_if_down<<<dim3((unsigned)((n + 255) / 256), (unsigned)L.nn), 256, 0, st>>>(L.d_desc, L.d_lists, qq, s, e,
                                                                                      R, m, L.uv, L.t3, L.y, ub, skip);
        hps::prof_end(hps::KC_MISC, st, 0.0, 8.0 * L.nn * (double)n * 4);
    }
}

// The factorisation for a grid of 3-D boxes (nfaces = 6, q^2 nodes per face)
// or of 2-D boxes (nfaces = 4, q nodes per edge, nb[2] = 1).
hps_status interface_factor(hps_ctx* ctx, int p, const int nb[3], int nfaces, const double* T, int nrhs_max,
                            hps_precision precision, void* stream, hps_interface** out)
{
    if (!out) return HPS_EINVAL;
    *out = nullptr;
    if (!ctx || !T || nrhs_max < 1 || nrhs_max > 256) return HPS_EINVAL;
    if (precision != HPS_FP64 && precision != HPS_FP32_IR) return HPS_EINVAL;
    hps_interface* F = new (std::nothrow) hps_interface();
    if (!F) return HPS_ENOMEM;
    if (!hps::build_iface_plan(p, nb, &F->plan, nfaces)) { delete F; return HPS_EINVAL; }
    F->device = hps::ctx_device(ctx);
    if (cudaSetDevice(F->device) != cudaSuccess) { delete F; return HPS_ECUDA; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const IfPlan& P = F->plan;
    F->p = p;
    F->q = p - 2;
    F->qq = nfaces == 6 ? F->q * F->q : F->q;   // nodes per face slot
    F->m = nfaces * F->qq;
    F->nbox = P.nbox;
    F->nrhs_max = nrhs_max;
    F->fp32 = precision == HPS_FP32_IR;
    const size_t elt = F->fp32 ? sizeof(float) : sizeof(double);
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
        for (int f = 0; f < nfaces; ++f)
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
    if (F->fp32) {
        IF_TRY(dalloc(&F->Tcopy, (size_t)P.nbox * m * m, &F->bytes));
        IF_TRY(cudaMemcpyAsync(F->Tcopy, T, sizeof(double) * (size_t)P.nbox * m * m, cudaMemcpyDeviceToDevice, st));
        IF_TRY(dalloc(&F->hcur, (size_t)P.nbox * R * m, &F->bytes));
        IF_TRY(dalloc(&F->du, (size_t)P.nbox * R * m, &F->bytes));
        IF_TRY(dalloc(&F->rstat, 4, &F->bytes));
        IF_TRY(dalloc(&F->rflag, 2, &F->bytes));
        IF_TRY(cudaMemsetAsync(F->rflag, 0, sizeof(int) * 2, st));
        IF_TRY(cudaMemsetAsync(F->rstat, 0, sizeof(double) * 4, st));
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
        IF_TRY(dalloc_bytes(&L.Winv, nn * s * s * elt, &F->bytes));
        IF_TRY(dalloc_bytes(&L.S, nn * s * e * elt, &F->bytes));
        IF_TRY(dalloc_bytes(&L.E, nn * e * s * elt, &F->bytes));
        IF_TRY(dalloc(&L.hv, nn * e * R, &F->bytes));
        IF_TRY(dalloc(&L.uv, nn * e * R, &F->bytes));
        // rows of uv beyond a merge's own boundary stay zero: S has zero columns there
        if (L.uv) IF_TRY(cudaMemsetAsync(L.uv, 0, sizeof(double) * nn * e * R, st));
        IF_TRY(dalloc(&L.t3, nn * s * R, &F->bytes));
        IF_TRY(dalloc(&L.y, nn * s * R, &F->bytes));
        size_t tmp = 0;
        IF_TRY(dalloc_bytes(&L.Tn, nn * e * e * elt, &tmp));
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
                const double* Tc = nullptr;
                const void* Mc = nullptr;
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
                    Mc = static_cast<const char*>(C.Tn) + ci * C.e_pad * C.e_pad * elt;
                    ld = C.e_pad;
                    vc = C.hv;
                    wc = C.uv;
                    oc = (long long)ci * C.e_pad;
                }
                if (side == 0) { d.Ta = Tc; d.Ma = Mc; d.lda = ld; d.va = vc; d.wa = wc; d.oa = oc; d.leafa = leaf; }
                else { d.Tb = Tc; d.Mb = Mc; d.ldb = ld; d.vb = vc; d.wb = wc; d.ob = oc; d.leafb = leaf; }
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
        rc = F->fp32 ? factor_level<float>(F->levels[lv], qq, &ws, &ws_bytes, &d_status, &status_cap, st)
                     : factor_level<double>(F->levels[lv], qq, &ws, &ws_bytes, &d_status, &status_cap, st);
        if (rc != HPS_OK) goto fail;
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

}  // namespace

extern "C" {

hps_status hps_interface_factor(hps_ctx* ctx, int p, const int nb[3], const double* T, int nrhs_max,
                                hps_precision precision, void* stream, hps_interface** out)
{
    return interface_factor(ctx, p, nb, 6, T, nrhs_max, precision, stream, out);
}

hps_status hps_interface2d_factor(hps_ctx* ctx, int p, const int nb[2], const double* T, int nrhs_max,
                                  hps_precision precision, void* stream, hps_interface** out)
{
    if (out) *out = nullptr;
    if (!nb) return HPS_EINVAL;
    const int nb3[3] = {nb[0], nb[1], 1};
    return interface_factor(ctx, p, nb3, 4, T, nrhs_max, precision, stream, out);
}

hps_status hps_interface_solve(hps_interface* F, int nrhs, const double* h, const double* g, double* ub,
                               void* stream)
{
    if (!F || nrhs < 1 || nrhs > F->nrhs_max || !h || !ub) return HPS_EINVAL;
    if (cudaSetDevice(F->device) != cudaSuccess) return HPS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int m = F->m, R = nrhs;
    if (!F->fp32) {
        solve_sweeps<double>(F, R, h, g, ub, nullptr, st);
        return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
    }
    // FP32 factors: first solve, then corrections from the FP64 flux residual
    // (each box's T u + h, summed over the boxes sharing a node, is the
    // residual of the interface equations; g stays fixed, so corrections
    // vanish on the outer faces).
    const long long total = (long long)F->nbox * R * m;
    k_if_check_reset<<<1, 1, 0, st>>>(F->rstat, F->rflag);
    solve_sweeps<float>(F, R, h, g, ub, nullptr, st);
    for (int it = 0; it < kRefineMax; ++it) {
        if (cudaMemcpyAsync(F->hcur, h, sizeof(double) * total, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return HPS_ECUDA;
        // hcur[box][c][r] += sum_j T[box][r][j] ub[box][c][j]
        hps::prof_begin(hps::KC_MISC, st);
        if (R <= 2)
            launch_mv<2, double>(F->nbox, m, R, m, F->Tcopy, m, (long long)m * m, ub, (long long)R * m, 1, m, F->hcur,
                                 (long long)R * m, 1, m, 1.0, 1, F->rflag, st);
        else
            launch_mv<8, double>(F->nbox, m, R, m, F->Tcopy, m, (long long)m * m, ub, (long long)R * m, 1, m, F->hcur,
                                 (long long)R * m, 1, m, 1.0, 1, F->rflag, st);
        hps::prof_end(hps::KC_MISC, st, 2.0 * F->nbox * (double)m * m * R, 8.0 * F->nbox * (double)m * m);
        solve_sweeps<float>(F, R, F->hcur, nullptr, F->du, F->rflag, st);
        k_if_update<<<(unsigned)std::min<long long>((total + 255) / 256, 4096), 256, 0, st>>>(total, F->du, ub,
                                                                                             F->rstat, F->rflag);
        k_if_check<<<1, 1, 0, st>>>(F->rstat, F->rflag, kRefineTol);
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

hps_status hps_interface_last_refinement(hps_interface* F, int* corrections, double* rel_correction)
{
    if (!F) return HPS_EINVAL;
    if (!F->fp32) {
        if (corrections) *corrections = 0;
        if (rel_correction) *rel_correction = 0.0;
        return HPS_OK;
    }
    if (cudaSetDevice(F->device) != cudaSuccess) return HPS_ECUDA;
    int fl[2] = {0, 0};
    double rs[4] = {0, 0, 0, 0};
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(fl, F->rflag, sizeof(fl), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(rs, F->rstat, sizeof(rs), cudaMemcpyDeviceToHost) != cudaSuccess)
        return HPS_ECUDA;
    if (corrections) *corrections = fl[1];
    if (rel_correction) *rel_correction = rs[3];
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
