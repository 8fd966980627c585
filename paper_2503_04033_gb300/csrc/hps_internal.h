// Internal declarations of the HPS leaf library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <algorithm>
#include <vector>

#include "../../include/hps.h"

namespace hps {

constexpr int kMaxP = 24;
constexpr int kMaxNB = 128;          // largest LU block (K of every update product)
constexpr int kPanelThreads = 512;   // threads of the panel-factorisation CTA

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

enum RhsKind { RHS_DTN = 0, RHS_LOAD = 1, RHS_TRACE = 2, RHS_DTN_LOAD = 3 };

// Update-product epilogue modes (see gemm description in hps_kernels.cuh).
enum GemmMode { GM_SET = 0, GM_ACC = 1, GM_FWD = 2, GM_BWD = 3 };

// Per-(p, h) device tables: physical first and second derivative matrices,
// [3][p][p] each (axis-major), FP64.
struct Geometry {
    int p = 0, q = 0, n = 0, m = 0;
    double h[3] = {0, 0, 0};
    double* dD = nullptr;
    double* dD2 = nullptr;
    float* dDF = nullptr;   // double-float line tables of the first correction's residual, [3][df_tab_f4(q)] float4
};

// float4 entries of one axis's double-float line table: the (E, O) pairs of
// the even/odd split [h][h], for odd q the middle column, middle row and
// diagonal (2h + 1 float2, padded to h + 1 float4), then the two boundary
// couplings D2[i][0], D2[i][p-1] of each interior row [q]; every value as a
// (hi, lo) float pair.
inline int df_tab_f4(int q)
{
    const int h = q / 2;
    return h * h + ((q & 1) ? h + 1 : 0) + q;
}

// Rounded FP64 product and sum, never contracted into a fused multiply-add, so
// host and device code that use them give the same bits.
__host__ __device__ inline double mul_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
__host__ __device__ inline double add_rn(double a, double b)
{
#ifdef __CUDA_ARCH__
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}

// Physical 1-D operators of every axis from the reference Chebyshev matrix
// Dhat (p x p on [-1, 1], Sec. 2.1): D = (2 / h_a) Dhat and D2 = D D, each
// [3][p][p] row-major.  D2 of the Chebyshev-Lobatto nodes is centro-symmetric
// (D2[i][j] = D2[p-1-i][p-1-j]); the product holds that only up to rounding,
// so each entry is averaged with its mirror to hold it exactly (the FP64
// residual's even/odd line split relies on it).  Run by one thread, on the
// host or the device, with the same bits either way.
__host__ __device__ inline void geometry_tables(int p, const double* Dhat, const double* h, double* D, double* D2)
{
    const int pp = p * p;
    for (int a = 0; a < 3; ++a) {
        const double s = 2.0 / h[a];
        double* Da = D + a * pp;
        double* D2a = D2 + a * pp;
        for (int e = 0; e < pp; ++e) Da[e] = mul_rn(s, Dhat[e]);
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int l = 0; l < p; ++l) acc = add_rn(acc, mul_rn(Da[i * p + l], Da[l * p + j]));
                D2a[i * p + j] = acc;
            }
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                const int e = i * p + j, f = (p - 1 - i) * p + (p - 1 - j);
                if (e < f) {
                    const double v = mul_rn(0.5, add_rn(D2a[e], D2a[f]));
                    D2a[e] = v;
                    D2a[f] = v;
                }
            }
    }
}

// Batched O = src + alpha * A * B over boxes (blockIdx.z), all row-major.
template <typename T>
struct GemmArgs {
    const T* A; long long lda, sA;
    const T* B; long long ldb, sB;
    T* O;       long long ldo, sO;
    int M, N, K;
    T alpha;
    int mode, split;
    const int* perm; long long sP;   // GM_FWD: source row of local row r (relative)
    const T* W; long long ldw, sW;   // GM_FWD: saved rows of the panel
    const int* skip;                 // per box: nonzero = leave untouched
};

// ---------------------------------------------------------------- LU plans

struct Plan {
    int n = 0, r = 0, NB = 0, ib = 0, nsteps = 0;
    long long ldm = 0;
    size_t elt = 0;                  // bytes per LU element
    bool tc = false;                 // FP32 products on the tensor cores
    bool tma_epi = true;             // tcgen05 epilogue through TMA where O is 16-byte aligned
    int unit_max = 1;                // tcgen05 path: up to this many consecutive LU steps joined into one unit
    int KG = 0;                      // K extent of the gathered right operand (unit_max x NB)
    int bn_max = 256;                // widest tensor-core tile (128 or 256 columns)
    int fmt = 0;                     // tcgen05 operand format: 0 = 3 x TF32, 1 = 3 x BF16, 2 = scaled 2 x FP16
    bool fuse_fwd = false;           // forward solves: next G written by the epilogue (scattered stores)
    bool fuse_bwd = false;           // backward solves: next G written by the epilogue
    std::vector<int> k0, nbs;
    std::vector<long long> fw_off, bw_off, perm_off;
    long long fw_elems = 0, bw_elems = 0, perm_elems = 0;
    // per-box byte sizes of the workspace pieces
    size_t bM = 0, bF = 0, bB = 0, bW = 0, bG = 0, bP = 0, bX = 0, bFp = 0, bBp = 0, bGp = 0;
    size_t bInv = 0, bGp2 = 0, bW2 = 0;   // tensor-core solves: inverse permutations, second G and W buffers
    size_t bKB = 0;                       // refinement: kappa^2 b at the interior nodes (FP64 and split)
    size_t bRC = 0, bIT = 0;              // format 2: K scales of the F and B packs, column scales of a G
    size_t per_box = 0;
};

inline Plan make_plan(int n, int r, hps_precision prec, int nb_opt, bool use_tc, bool need_x, int lu_unit = 4,
                      bool fp16_ops = false)
{
    Plan P;
    P.n = n;
    P.r = r;
    const bool fp64 = (prec == HPS_FP64);
    P.elt = fp64 ? 8 : 4;
    P.tc = !fp64 && use_tc;
    P.fmt = !P.tc ? 0 : (prec == HPS_BF16_IR ? 1 : (fp16_ops ? 2 : 0));
    P.fuse_bwd = P.tc && P.fmt == 0;
    int NB = nb_opt > 0 ? nb_opt : (fp64 ? 64 : 128);
    if (fp64 && NB > 64) NB = 64;
    if (NB > kMaxNB) NB = kMaxNB;
    P.NB = NB;
    P.ldm = (long long)align_up((size_t)(n + r), 8);
    // panel inner-block width: the block column of the panel lives in shared memory
    const size_t static_smem = 32 * kMaxNB * P.elt + 2048;
    const size_t budget = 227 * 1024 - static_smem;
    int ib = 32;
    while (ib > 1 && (size_t)ib * n * P.elt + (size_t)n * 5 > budget) ib >>= 1;
    if (ib > NB) ib = NB;
    P.ib = ib;
    for (int k = 0; k < n; k += NB) {
        const int nb = std::min(NB, n - k);
        P.k0.push_back(k);
        P.nbs.push_back(nb);
        P.fw_off.push_back(P.fw_elems);
        P.bw_off.push_back(P.bw_elems);
        P.perm_off.push_back(P.perm_elems);
        P.fw_elems += (long long)(n - k) * NB;
        P.bw_elems += (long long)(k + nb) * NB;
        P.perm_elems += (n - k);
    }
    P.nsteps = (int)P.k0.size();
    P.unit_max = 1;
    if (P.tc)
        while (2 * P.unit_max <= lu_unit && 2 * P.unit_max <= P.nsteps && 2 * P.unit_max <= 8) P.unit_max *= 2;
    P.KG = P.unit_max * NB;
    const size_t A = 256;
    P.bM = align_up((size_t)n * P.ldm * P.elt, A);
    P.bF = align_up((size_t)P.fw_elems * P.elt, A);
    P.bB = align_up((size_t)P.bw_elems * P.elt, A);
    P.bW = align_up((size_t)P.KG * P.ldm * P.elt, A);
    P.bG = P.bW;
    P.bP = align_up((size_t)P.perm_elems * sizeof(int), A);
    P.bX = need_x ? align_up((size_t)n * r * sizeof(double), A) : 0;
    P.bKB = need_x ? align_up((size_t)n * (sizeof(double) + 2 * sizeof(float)), A) : 0;
    if (P.tc) {
        // split (hi, lo) K-major copies of F, B and G for the tensor-core products
        // (3 x TF32: two FP32 planes; 3 x BF16: three 2-byte planes)
        const size_t pk = P.fmt == 1 ? 3 * 2 : (P.fmt == 2 ? 2 * 2 : 2 * sizeof(float));
        P.bFp = align_up((size_t)P.fw_elems * pk, A);
        P.bBp = align_up((size_t)P.bw_elems * pk, A);
        P.bGp = align_up((size_t)P.ldm * P.KG * pk, A);
        P.bInv = P.fuse_fwd ? P.bP : 0;
        P.bGp2 = P.bGp;
        P.bW2 = P.bW;
        if (P.fmt == 2) {
            P.bRC = align_up((size_t)P.nsteps * NB * sizeof(float), A);
            P.bIT = align_up((size_t)(P.ldm + 64) * sizeof(float), A);
        }
    }
    P.per_box = P.bM + P.bF + P.bB + P.bW + P.bG + P.bP + P.bX + P.bFp + P.bBp + P.bGp + P.bInv + P.bGp2 + P.bW2 + P.bKB +
                2 * P.bRC + 2 * P.bIT + 64;
    return P;
}

// Pointers of one chunk's workspace.
template <typename T>
struct Work {
    T *M, *F, *B, *W, *G;
    int* perm;
    double* X;
    float *Fp, *Bp, *Gp;
    int* inv;
    float *Gp2, *W2;
    double* kb;
    float2* kbs;   // kappa^2 b as (hi, lo) float pairs, [nbox][n] after kb's [nbox][n]
    float *rcF, *rcB;   // format 2: 1 / (power-of-two scale) of each K column of F_s, B_s ([step][NB] per box)
    float *it1, *it2;   // format 2: 1 / (power-of-two scale) of each column of the G in Gp, Gp2
    double* norms;
    int* skip;
    long long sM, sF, sB, sG, sP, sX, sFp, sBp, sGp, sRC, sIT;
};

template <typename T>
inline Work<T> carve(const Plan& P, void* base, int nbox)
{
    Work<T> w{};
    char* c = static_cast<char*>(base);
    auto take = [&](size_t per_box) { char* r = c; c += per_box * (size_t)nbox; return r; };
    w.M = reinterpret_cast<T*>(take(P.bM));
    w.F = reinterpret_cast<T*>(take(P.bF));
    w.B = reinterpret_cast<T*>(take(P.bB));
    w.W = reinterpret_cast<T*>(take(P.bW));
    w.G = reinterpret_cast<T*>(take(P.bG));
    w.perm = reinterpret_cast<int*>(take(P.bP));
    w.X = P.bX ? reinterpret_cast<double*>(take(P.bX)) : nullptr;
    w.Fp = P.bFp ? reinterpret_cast<float*>(take(P.bFp)) : nullptr;
    w.Bp = P.bBp ? reinterpret_cast<float*>(take(P.bBp)) : nullptr;
    w.Gp = P.bGp ? reinterpret_cast<float*>(take(P.bGp)) : nullptr;
    w.inv = P.bInv ? reinterpret_cast<int*>(take(P.bInv)) : nullptr;
    w.Gp2 = P.bGp2 ? reinterpret_cast<float*>(take(P.bGp2)) : nullptr;
    w.W2 = P.bW2 ? reinterpret_cast<float*>(take(P.bW2)) : nullptr;
    w.kb = P.bKB ? reinterpret_cast<double*>(take(P.bKB)) : nullptr;
    w.kbs = w.kb ? reinterpret_cast<float2*>(w.kb + (size_t)nbox * P.n) : nullptr;
    w.rcF = P.bRC ? reinterpret_cast<float*>(take(P.bRC)) : nullptr;
    w.rcB = P.bRC ? reinterpret_cast<float*>(take(P.bRC)) : nullptr;
    w.it1 = P.bIT ? reinterpret_cast<float*>(take(P.bIT)) : nullptr;
    w.it2 = P.bIT ? reinterpret_cast<float*>(take(P.bIT)) : nullptr;
    w.sRC = (long long)(P.bRC / sizeof(float));
    w.sIT = (long long)(P.bIT / sizeof(float));
    w.norms = reinterpret_cast<double*>(take(align_up(2 * sizeof(double), 16)));
    w.skip = reinterpret_cast<int*>(take(align_up(sizeof(int), 16)));
    w.sM = (long long)(P.bM / P.elt);
    w.sF = (long long)(P.bF / P.elt);
    w.sB = (long long)(P.bB / P.elt);
    w.sG = (long long)(P.bG / P.elt);
    w.sP = (long long)(P.bP / sizeof(int));
    w.sX = (long long)(P.bX / sizeof(double));
    const size_t pke = P.fmt ? 2 : sizeof(float);   // strides of the split operands in their elements
    w.sFp = (long long)(P.bFp / pke);
    w.sBp = (long long)(P.bBp / pke);
    w.sGp = (long long)(P.bGp / pke);
    return w;
}


// ---------------------------------------------------------------- profiling

// Kernel classes timed by the optional event profiler (HPS_OPT_PROFILE).
enum KernelClass {
    KC_BUILD = 0, KC_PANEL, KC_UPDATE_CUDACORE, KC_UPDATE_TC, KC_GATHER, KC_RESIDUAL, KC_REFINE, KC_DN,
    KC_UPDATE_TC_REFINE, KC_PACK, KC_RESIDUAL_DF, KC_MISC, KC_RESIDUAL_DF64, KC_COUNT
};

// When profiling is on for the calling thread, prof_begin/prof_end bracket a
// launch with CUDA events on its stream and record its algorithmic flops and
// bytes; otherwise they do nothing.
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double flops, double bytes);

// Host launchers (hps_lu.cu).
template <typename T>
void launch_build_aug(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b,
                      long long sb, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                      T* M, long long ldm, long long sM, int* status, int zero_row_box, cudaStream_t st,
                      const double* beta = nullptr);

template <typename T>
void launch_panel(T* M, long long ldm, long long sM, int n, int k, int nb, int ib,
                  int* perm, long long sP, T* Ftop, long long ldf, long long sF,
                  T* Btop, long long ldb, long long sB, int* status, const int* skip,
                  int nbox, cudaStream_t st);

template <typename T>
void launch_gather(const T* M, long long ldm, long long sM, int k, int nb, int c0, int ncols,
                   const int* perm, long long sP, T* W, T* G, long long ldg, long long sG,
                   const int* skip, int nbox, cudaStream_t st);

template <typename T>
void launch_gemm(const GemmArgs<T>& a, int nbox, cudaStream_t st);

void launch_dn(const Geometry& g, int nbox, const double* X, long long ldx, long long sX,
               int ncols, double* out, long long sOut, int transposed_out, int add_abb,
               cudaStream_t st);

template <typename TS>
void launch_extract(const TS* src, long long lds, long long sS, int n, int ncols,
                    double* X, long long ldx, long long sX, int nbox, cudaStream_t st, double* xnorm = nullptr);

// out = A u at the interior nodes of full nodal fields (zero at the others).
void launch_apply_op(const Geometry& g, double kappa, int nbox, int nfield, const double* b, const double* u,
                     double* out, cudaStream_t st, const double* beta = nullptr);

// M's right-hand-side columns n .. n + nrhs (LOAD: f_i, TRACE: -A_ib u_b), the
// factors in M's first n columns left as they are.
template <typename T>
void launch_load_rhs(const Geometry& g, int nbox, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                     T* M, long long ldm, long long sM, int* status, cudaStream_t st, const double* beta = nullptr);

void launch_residual(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b, long long sb,
                     int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                     const double* X, long long ldx, long long sX,
                     float* R, long long ldr, long long sR, const int* skip, cudaStream_t st,
                     const double* kb = nullptr, const double* beta = nullptr);
void selftest_conversions(long long n, unsigned long long seed, unsigned long long* mism_dev, cudaStream_t st);
void launch_kappa_b(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b, long long sb,
                    double* kb, float2* kbs, cudaStream_t st);

// Residual of the first solution X0 (FP32, rows of pitch ld, box stride sbx),
// written over X0 in place as FP32: R = B - A_ii X0 in double-float
// arithmetic.  Needs g.dDF and the split kappa^2 b (launch_kappa_b).
// Whether the double-float residual's per-CTA tables and line buffers fit in
// shared memory at this order (x64: the form that reads an FP64 X).
bool residual_df_fits(const Geometry& g, bool x64);
// With X64 (FP64 [n][ldx] per box, stride sX64) the residual is of that
// solution instead, each entry split into two floats (about 2^-46 relative to
// the terms' magnitudes as well), and X0R only receives R.
void launch_residual_df(const Geometry& g, int nbox, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                        float* X0R, long long ld, long long sbx, const float2* kbs, const int* skip,
                        cudaStream_t st, const double* X64 = nullptr, long long ldx = 0, long long sX64 = 0);

void launch_ir_update(const float* D, long long ldd, long long sD, int n, int ncols,
                      double* X, long long ldx, long long sX, double* norms /*[nbox][2]*/,
                      const int* skip, int nbox, cudaStream_t st, bool want_xn = false);

void launch_ir_check(int nbox, double* norms, double tol, int last, int* skip,
                     int* iters, double* relcorr, int* status, cudaStream_t st, bool hold = false,
                     double floor_coef = 0.0, double dfgate = 0.0, int* route = nullptr, int* skip_df = nullptr,
                     int* skip_64 = nullptr);

// Error floor of a correction computed from the double-float residual,
// relative to that correction's own size.  The residual of X0 is formed with
// relative error about 2^-46 of the terms' magnitudes |A_ii||X0| + |B|; the
// LU that produced X0 has a backward error of about 2^-22 relative to the
// same magnitudes (22-bit split operands, FP32 storage and accumulation).
// Both pass through the same A_ii^{-1}, so the correction's error is about
// 2^-24 times X0's error, which the correction itself measures: the floor is
// taken as 100 * 2^-24 * ||dX_1||, a factor 100 of margin.
constexpr double kDfFloor = 100.0 / 16777216.0;

// Routing of the later residuals (HPS_OPT_RESIDUAL_DF = 3).  A residual of
// an FP64 X split into two floats is formed with relative error about 2^-46
// of the terms' magnitudes, against 2^-53 in FP64; A_ii^{-1} amplifies that
// error by about rel_1 / 2^-22, where rel_1 = ||dX_1|| / ||X|| is the first
// correction's size (it measures X0's error, which the same amplification
// made from the LU's 2^-22).  A box whose rel_1 is at most kDfGate therefore
// has a double-float residual floor below about kDfGate 2^-24 ~ 2e-11 of X,
// a factor 5 under the 1e-10 target; its later residuals run in
// double-float, every other box's in FP64.
constexpr double kDfGate = 3.0e-4;

void launch_transpose_add(const double* X, long long ldx, long long sX, int n, int ncols,
                          const double* v, double* out, int nbox, cudaStream_t st);

void launch_recon_stored(const double* S, int n, int m, int nrhs, const double* v,
                         const double* ub, double* ui, int nbox, cudaStream_t st);

void launch_fill_int(int* p, int value, long long count, cudaStream_t st);

// Residual gate of the learned DtN correction (hps_lu.cu).
void launch_probes(long long total, unsigned long long seed, double* phi, cudaStream_t st);
void launch_abb_add(const Geometry& g, int nbox, int k, const double* phi, double* out, cudaStream_t st);
void launch_apply_probes(int m, int k, int nbox, const double* That, const double* phi, double* tp, cudaStream_t st);
void launch_gate_decide(int m, int k, int nbox, const double* tp_hat, const double* tp, const double* norms,
                        double tol, int* accept, double* err, cudaStream_t st);
void launch_identity_loads(int p, int n, double* f, cudaStream_t st);
void launch_transpose_f32(int n, const double* in, float* out, cudaStream_t st);

// Host-side 1-D operators (hps_abi.cu): Chebyshev-Lobatto nodes on [-1,1] and
// the spectral differentiation matrix (row-major p x p).
void cheb_nodes(int p, double* t);
void cheb_diff(int p, double* D);

// CUDA-core LU sequences (hps_abi.cu): factorisation carrying the RHS block,
// forward replay and backward substitution of RHS columns [c0, c0 + nc).
template <typename T>
void lu_factor(const Plan& P, Work<T>& w, int nbox, int* status, cudaStream_t st);
template <typename T>
void lu_forward(const Plan& P, Work<T>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st);
template <typename T>
void lu_backward(const Plan& P, Work<T>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st);

// Tensor-core (tcgen05, 3-term TF32 split) versions of the LU sequences (hps_tc.cu).
// They return false when a TMA descriptor cannot be encoded.  A tensor-core
// launch whose bounded wait gave up raises a device-wide abort flag (checked
// with tc_abort_raised, cleared by tc_reset_abort) and marks its box
// HPS_ETIMEOUT.
// C = (accumulate ? C : 0) - A B^T on tcgen05 with BF16 A [M][K], B [N][K]
// (K-major, row pitches lda, ldb multiples of 8) and FP32 C [M][N] (pitch
// ldc), batch strides sA, sB, sC.  False when the operands cannot be
// described to TMA.
bool tc_gemm_bf16(int M, int N, int K, const void* A, long long lda, long long sA, const void* B, long long ldb,
                  long long sB, float* C, long long ldc, long long sC, bool accumulate, int batch, cudaStream_t st);
void tc_reset_abort(cudaStream_t st);

// Test hook: the next tensor-core launch of a call that writes box status
// makes its first mbarrier wait run out (nothing is issued to fill it); that
// launch and the rest of the call end with HPS_ETIMEOUT in box_status.
void tc_test_stall_next(int on);
bool tc_test_stall_armed();
bool tc_abort_raised();
bool tc_lu_factor(const Plan& P, Work<float>& w, int nbox, int* status, cudaStream_t st);
bool tc_lu_forward(const Plan& P, Work<float>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st);
bool tc_lu_backward(const Plan& P, Work<float>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st);

}  // namespace hps
