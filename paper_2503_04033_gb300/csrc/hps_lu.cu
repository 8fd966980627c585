// CUDA-core kernels of the leaf reduction: operator assembly, the blocked LU
// with partial pivoting (panel factorisation with warp-shuffle pivot search),
// the row-gather and update products that carry the triangular solves, the
// FP64 refinement residual, and the D_n / flux products.
//
// Storage of one box's working matrix M (row-major, leading dimension ldm):
//   M = [ A_ii | RHS ]   n rows, n + r used columns,
// where RHS is -A_ib (DtN build, Sec. 2.2: S = -A_ii^{-1} A_ib), the body loads
// f_i (particular solution) or -A_ib u_b (recomputed reconstruction).
//
// Blocked right-looking LU, step s covers columns [k, k + nb):
//   panel:  P_s [A11; A21] = [L11; L21] U11 (partial pivoting), with
//           F_s = [-L11^{-1}; L21 L11^{-1}]  and  B_s top = -U11^{-1}.
//   update: for all columns right of the panel (remaining A_ii columns and RHS)
//           G = (P_s M)[k:k+nb],  W = M[k:k+nb] (rows before the swaps), then
//           M[r] <- src(r) - F_s[r-k] G   for r >= k,
//           src(r) = 0 for r < k + nb (so the rows become U12 = L11^{-1} G),
//           src(r) = old row pi_s(r) otherwise (from W when it sat in the panel).
//   The row interchanges are therefore never applied as a separate pass; the
//   permutation rides in the update's epilogue.
// Backward substitution (U x = y) runs the same product with
//   B_s = [U[0:k, k:k+nb] U11^{-1}; -U11^{-1}], src(r) = M[r] for r < k, 0 after.
// (On the tensor-core path two consecutive steps are joined into one product
// of depth 2 NB; see the LU sequences in hps_tc.cu.)
// Forward substitution of new right-hand sides replays the stored (pi_s, F_s).
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include <type_traits>

#include "hps_internal.h"

namespace hps {

namespace {

__device__ __forceinline__ int imin(int a, int b) { return a < b ? a : b; }

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Conversions between FP64 and FP32 on the integer pipe (on GB300 the FP64
// pipe that executes the conversion instructions is the residual's and the
// refinement update's bottleneck).  Both follow the IEEE-754 binary64 /
// binary32 encodings; anything outside the normal range goes to the hardware
// conversion.  hps_selftest_conversions checks them bit for bit against it.
//
// double -> float, round to nearest even: the 52-bit significand is rounded
// to 23 bits by adding 0x0FFFFFFF plus the kept part's last bit before the
// 29-bit shift (a carry into the exponent is the correct result, up to
// infinity), and the exponent is rebiased from 1023 to 127.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned long long a = u & 0x7FFFFFFFFFFFFFFFull;
    const unsigned e = (unsigned)(a >> 52);
    if (e - 897u > 253u) return __double2float_rn(x);   // zero, float subnormal or overflow, inf, NaN
    const unsigned long long r = (a + 0x0FFFFFFFull + ((a >> 29) & 1ull)) >> 29;
    const unsigned f = (unsigned)(r - (896ull << 23)) | (unsigned)((u >> 32) & 0x80000000u);
    return __uint_as_float(f);
}

// float -> double (exact): the significand moves up 29 bits and the exponent
// is rebiased from 127 to 1023; zero keeps its sign.
__device__ __forceinline__ double f2d(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
    if (e - 1u > 253u) {
        if ((u << 1) == 0u) return __longlong_as_double((long long)sgn);
        return (double)x;                                  // subnormal, inf, NaN
    }
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x7FFFFFFFu) << 29) + (896ull << 52) | sgn));
}

// ---------------------------------------------------------------- assembly

// Rows per CTA of the operator build.
constexpr int kBuildRows = 4;

// Builds [A_ii | B] for a batch of boxes straight into the LU workspace
// (Eq. 2's collocation restricted to the interior rows, Kronecker form:
// A = -(D2x (x) I (x) I + I (x) D2y (x) I + I (x) I (x) D2z) - kappa^2 diag(b)).
// A_ii has 3q - 2 nonzeros per row (the three grid lines through the node) and
// the DtN block -A_ib six (the face nodes at the ends of those lines), so a CTA
// first clears its kBuildRows rows with 16-byte stores and then writes the
// nonzeros and the dense load / trace columns; every value is formed in FP64
// and rounded once to T.  B is -A_ib (DTN), f_i (LOAD), -A_ib u_b (TRACE) or
// [-A_ib | f_i] (DTN_LOAD).  With beta (per box [3][p^3]) the operator gains
// the first-order term div(beta u): + D_a[i][l] beta_a(l) on every entry of
// the a-line (the product rule of collocation differentiation), couplings
// included; the pattern of nonzeros is the same.
template <typename T>
__global__ void __launch_bounds__(256)
k_build_aug(int p, int n, int nrhs, int ldm_cols, const double* __restrict__ D2, double kappa2,
            const double* __restrict__ kappa_box, const double* __restrict__ b, long long sb, int rhs_kind,
            const double* __restrict__ rhs, long long s_rhs, T* __restrict__ M, long long ldm, long long sM,
            int* status, int zero_row_box, const double* __restrict__ D1, const double* __restrict__ beta,
            long long sbeta)
{
    const int box = blockIdx.y;
    const int r0 = blockIdx.x * kBuildRows;
    const int rows = imin(kBuildRows, n - r0);
    T* Mb = M + box * sM + (long long)r0 * ldm;
    // 1. clear the rows (ldm and the row starts are multiples of 16 bytes)
    {
        using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
        constexpr int per = 16 / sizeof(T);
        const int nv = (int)(ldm / per);
        V* Mv = reinterpret_cast<V*>(Mb);
        V z;
        memset(&z, 0, sizeof(z));
        for (int idx = threadIdx.x; idx < rows * nv; idx += blockDim.x) {
            const int rr = idx / nv, cv = idx - rr * nv;
            Mv[(long long)rr * (ldm / per) + cv] = z;
        }
    }
    __syncthreads();
    // 2. the nonzeros of A_ii and of the DtN block, and the dense columns
    const int q = p - 2, qq = q * q, pp = p * p;
    const double* D2x = D2;
    const double* D2y = D2 + pp;
    const double* D2z = D2 + 2 * pp;
    const double k2 = kappa_box ? kappa_box[box] * kappa_box[box] : kappa2;
    const int p3 = pp * p;
    const double* bt = beta ? beta + box * sbeta : nullptr;   // [3][p^3] of this box
    // first-order coefficient of node (ii, jj, kk) on its a-line at position l
    auto c1 = [&](int a, int own, int l, int ii, int jj, int kk) -> double {
        return bt ? __ldg(D1 + a * pp + own * p + l) * __ldg(bt + a * p3 + ii + p * jj + pp * kk) : 0.0;
    };
    const bool dtn = rhs_kind == RHS_DTN || rhs_kind == RHS_DTN_LOAD;
    const int ndtn = dtn ? 6 : 0;
    const int dense0 = rhs_kind == RHS_DTN_LOAD ? 6 * qq : 0;   // first dense column within B
    const int ndense = rhs_kind == RHS_DTN ? 0 : nrhs - dense0;
    const int dkind = rhs_kind == RHS_DTN_LOAD ? RHS_LOAD : rhs_kind;
    const int per_row = 3 * q - 2 + ndtn + ndense;
    for (int idx = threadIdx.x; idx < rows * per_row; idx += blockDim.x) {
        const int rr = idx / per_row, e = idx - rr * per_row;
        const int r = r0 + rr;
        const int i = r % q + 1, j = (r / q) % q + 1, k = r / qq + 1;
        T* row = Mb + (long long)rr * ldm;
        if (e < 3 * q - 2) {
            if (box == zero_row_box && r == 0) continue;   // test hook: exactly singular A_ii
            int c;
            double v;
            if (e < q) {                                   // x line, with the diagonal
                const int i2 = e + 1;
                c = (i2 - 1) + q * (j - 1) + qq * (k - 1);
                v = 0.0 - __ldg(D2x + i * p + i2) + c1(0, i, i2, i2, j, k);
                if (i2 == i) {
                    v -= __ldg(D2y + j * p + j);
                    v -= __ldg(D2z + k * p + k);
                    v += c1(1, j, j, i, j, k) + c1(2, k, k, i, j, k);
                    const double bv = __ldg(b + box * sb + i + p * j + pp * k);
                    if (!isfinite(bv)) status[box] = HPS_EINVAL;
                    v -= k2 * bv;
                }
            } else if (e < 2 * q - 1) {                    // y line off the diagonal
                int j2 = e - q + 1;
                if (j2 >= j) ++j2;
                c = (i - 1) + q * (j2 - 1) + qq * (k - 1);
                v = 0.0 - __ldg(D2y + j * p + j2) + c1(1, j, j2, i, j2, k);
            } else {                                       // z line off the diagonal
                int k2i = e - (2 * q - 1) + 1;
                if (k2i >= k) ++k2i;
                c = (i - 1) + q * (j - 1) + qq * (k2i - 1);
                v = 0.0 - __ldg(D2z + k * p + k2i) + c1(2, k, k2i, i, j, k2i);
            }
            row[c] = T(v);
        } else if (e < 3 * q - 2 + ndtn) {
            // -A_ib: the face node at the end of one of the row's grid lines
            const int f = e - (3 * q - 2), axis = f >> 1, ep = (f & 1) ? p - 1 : 0;
            int a, bb;
            double v;
            if (axis == 0) { a = j; bb = k; v = __ldg(D2x + i * p + ep) - c1(0, i, ep, ep, j, k); }
            else if (axis == 1) { a = i; bb = k; v = __ldg(D2y + j * p + ep) - c1(1, j, ep, i, ep, k); }
            else { a = i; bb = j; v = __ldg(D2z + k * p + ep) - c1(2, k, ep, i, j, ep); }
            row[n + f * qq + (a - 1) + q * (bb - 1)] = T(v);
        } else {
            const int cf = e - (3 * q - 2 + ndtn);
            double v;
            if (dkind == RHS_LOAD) {
                v = __ldg(rhs + box * s_rhs + (long long)cf * p * pp + i + p * j + pp * k);
            } else {
                // -A_ib u_b: the six face nodes on this row's three grid lines.
                const double* ub = rhs + box * s_rhs + (long long)cf * 6 * qq;
                const int sx = (j - 1) + q * (k - 1), sy = (i - 1) + q * (k - 1), sz = (i - 1) + q * (j - 1);
                const int e1 = p - 1;
                v = (__ldg(D2x + i * p) - c1(0, i, 0, 0, j, k)) * ub[0 * qq + sx]
                  + (__ldg(D2x + i * p + e1) - c1(0, i, e1, e1, j, k)) * ub[1 * qq + sx]
                  + (__ldg(D2y + j * p) - c1(1, j, 0, i, 0, k)) * ub[2 * qq + sy]
                  + (__ldg(D2y + j * p + e1) - c1(1, j, e1, i, e1, k)) * ub[3 * qq + sy]
                  + (__ldg(D2z + k * p) - c1(2, k, 0, i, j, 0)) * ub[4 * qq + sz]
                  + (__ldg(D2z + k * p + e1) - c1(2, k, e1, i, j, e1)) * ub[5 * qq + sz];
            }
            if (!isfinite(v)) status[box] = HPS_EINVAL;
            row[n + dense0 + cf] = T(v);
        }
    }
}

// The right-hand-side columns n .. n + nrhs of M alone, for solves with a
// stored factorisation: f_i (LOAD) or -A_ib u_b (TRACE) per column, the rest
// of M (the factors) untouched.  Thread per (row, column), rows over the grid.
template <typename T>
__global__ void k_load_rhs(int p, int n, int nrhs, const double* __restrict__ D2, int rhs_kind,
                           const double* __restrict__ rhs, long long s_rhs, T* __restrict__ M, long long ldm,
                           long long sM, int* status, const double* __restrict__ D1, const double* __restrict__ beta)
{
    const int box = blockIdx.y;
    const int q = p - 2, qq = q * q, pp = p * p;
    const double* D2x = D2;
    const double* D2y = D2 + pp;
    const double* D2z = D2 + 2 * pp;
    const long long total = (long long)n * nrhs;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / nrhs), cf = (int)(idx - (long long)r * nrhs);
        const int i = r % q + 1, j = (r / q) % q + 1, k = r / qq + 1;
        double v;
        if (rhs_kind == RHS_LOAD) {
            v = __ldg(rhs + box * s_rhs + (long long)cf * p * pp + i + p * j + pp * k);
        } else {
            const double* ub = rhs + box * s_rhs + (long long)cf * 6 * qq;
            const int sx = (j - 1) + q * (k - 1), sy = (i - 1) + q * (k - 1), sz = (i - 1) + q * (j - 1);
            double cx0 = __ldg(D2x + i * p), cx1 = __ldg(D2x + i * p + p - 1);
            double cy0 = __ldg(D2y + j * p), cy1 = __ldg(D2y + j * p + p - 1);
            double cz0 = __ldg(D2z + k * p), cz1 = __ldg(D2z + k * p + p - 1);
            if (beta) {   // minus the first-order couplings D_a[i][e] beta_a(face node)
                const int p3 = pp * p, e1 = p - 1;
                const double* bt = beta + box * 3LL * p3;
                cx0 -= __ldg(D1 + i * p) * bt[0 + p * j + pp * k];
                cx1 -= __ldg(D1 + i * p + e1) * bt[e1 + p * j + pp * k];
                cy0 -= __ldg(D1 + pp + j * p) * bt[p3 + i + pp * k];
                cy1 -= __ldg(D1 + pp + j * p + e1) * bt[p3 + i + p * e1 + pp * k];
                cz0 -= __ldg(D1 + 2 * pp + k * p) * bt[2 * p3 + i + p * j];
                cz1 -= __ldg(D1 + 2 * pp + k * p + e1) * bt[2 * p3 + i + p * j + pp * e1];
            }
            v = cx0 * ub[0 * qq + sx] + cx1 * ub[1 * qq + sx] + cy0 * ub[2 * qq + sy] + cy1 * ub[3 * qq + sy] +
                cz0 * ub[4 * qq + sz] + cz1 * ub[5 * qq + sz];
        }
        if (!isfinite(v)) status[box] = HPS_EINVAL;
        M[box * sM + (long long)r * ldm + n + cf] = T(v);
    }
}

// out = A u at the interior nodes of full nodal fields u (all p^3 values of a
// box): the interior rows of Eq. 2's collocation, -(D2x + D2y + D2z) along the
// three grid lines through each node, minus kappa^2 b u; zero at the other
// nodes.  One CTA per (field, box), the field staged in shared memory.
__global__ void k_apply_op(int p, int nfield, const double* __restrict__ D2, double kappa2,
                           const double* __restrict__ b, long long sb, const double* __restrict__ u,
                           double* __restrict__ out, const double* __restrict__ D1, const double* __restrict__ beta)
{
    extern __shared__ double us[];
    const int c = blockIdx.x, box = blockIdx.y;
    const int pp = p * p, p3 = pp * p;
    const double* ub = u + ((long long)box * nfield + c) * p3;
    double* ob = out + ((long long)box * nfield + c) * p3;
    for (int idx = threadIdx.x; idx < p3; idx += blockDim.x) us[idx] = ub[idx];
    __syncthreads();
    const double* D2x = D2;
    const double* D2y = D2 + pp;
    const double* D2z = D2 + 2 * pp;
    for (int idx = threadIdx.x; idx < p3; idx += blockDim.x) {
        const int i = idx % p, j = (idx / p) % p, k = idx / pp;
        if (i == 0 || j == 0 || k == 0 || i == p - 1 || j == p - 1 || k == p - 1) {
            ob[idx] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int l = 0; l < p; ++l)
            acc += __ldg(D2x + i * p + l) * us[l + p * j + pp * k] + __ldg(D2y + j * p + l) * us[i + p * l + pp * k] +
                   __ldg(D2z + k * p + l) * us[i + p * j + pp * l];
        double conv = 0.0;   // div(beta u): D_a applied to beta_a u along the three lines
        if (beta) {
            const double* bt = beta + box * 3LL * p3;
            for (int l = 0; l < p; ++l) {
                const int nx = l + p * j + pp * k, ny = i + p * l + pp * k, nz = i + p * j + pp * l;
                conv += __ldg(D1 + i * p + l) * __ldg(bt + nx) * us[nx] +
                        __ldg(D1 + pp + j * p + l) * __ldg(bt + p3 + ny) * us[ny] +
                        __ldg(D1 + 2 * pp + k * p + l) * __ldg(bt + 2 * p3 + nz) * us[nz];
            }
        }
        ob[idx] = -acc + conv - kappa2 * __ldg(b + box * sb + idx) * us[idx];
    }
}

// ---------------------------------------------------------------- panel

// Arg-max of |value| over the CTA with ties to the lowest index.
template <typename T>
__device__ __forceinline__ void argmax_merge(T& v, int& i, T ov, int oi)
{
    if (ov > v || (ov == v && oi < i)) { v = ov; i = oi; }
}

// Inverse of a triangle held in A (P x P, row-major, P a power of two >= 16,
// padded with the identity): the unit lower triangle below A's diagonal
// (lower) or the upper triangle with its diagonal.  The 16 x 16 diagonal
// blocks are inverted by substitution (a column per thread), then blocks of
// doubling size b are joined: for [[A1, 0], [C, D]] the off-diagonal block
// of the inverse is -D^{-1} (C A1^{-1}); for [[A1, B], [0, D]] it is
// -A1^{-1} (B D^{-1}).  The middle product is parked in the free triangle of
// A.  X must be zero on entry and receives the inverse.  A zero diagonal
// entry is read as 1 (the box is already flagged singular).
template <typename T>
__device__ void tri_inverse(T* A, T* X, int P, bool lower, int tid)
{
    if (tid < P) {
        const int q0 = (tid >> 4) << 4, c = tid;
        if (lower) {
            X[c * P + c] = T(1);
            for (int r = c + 1; r < q0 + 16; ++r) {
                T acc = T(0);
                for (int t = c; t < r; ++t) acc -= A[r * P + t] * X[t * P + c];
                X[r * P + c] = acc;
            }
        } else {
            T d = A[c * P + c];
            if (d == T(0)) d = T(1);
            X[c * P + c] = T(1) / d;
            for (int r = c - 1; r >= q0; --r) {
                T acc = T(0);
                for (int t = r + 1; t <= c; ++t) acc -= A[r * P + t] * X[t * P + c];
                T dr = A[r * P + r];
                if (dr == T(0)) dr = T(1);
                X[r * P + c] = acc / dr;
            }
        }
    }
    __syncthreads();
    for (int b = 16; b < P; b *= 2) {
        const int items = (P / (2 * b)) * b * b;
        // middle products into the free triangle of A
        for (int it = tid; it < items; it += kPanelThreads) {
            const int pr = it / (b * b), e = it - pr * b * b, r = e / b, c = e - r * b, i0 = 2 * b * pr;
            T acc = T(0);
            if (lower) {   // C A1^{-1}: C = A[i0+b+r][i0+t], A1^{-1} lower
                for (int t = c; t < b; ++t) acc += A[(i0 + b + r) * P + i0 + t] * X[(i0 + t) * P + i0 + c];
                A[(i0 + r) * P + i0 + b + c] = acc;
            } else {       // B D^{-1}: B = A[i0+r][i0+b+t], D^{-1} upper
                for (int t = 0; t <= c; ++t) acc += A[(i0 + r) * P + i0 + b + t] * X[(i0 + b + t) * P + i0 + b + c];
                A[(i0 + b + r) * P + i0 + c] = acc;
            }
        }
        __syncthreads();
        for (int it = tid; it < items; it += kPanelThreads) {
            const int pr = it / (b * b), e = it - pr * b * b, r = e / b, c = e - r * b, i0 = 2 * b * pr;
            T acc = T(0);
            if (lower) {   // -D^{-1} (C A1^{-1}), D^{-1} lower
                for (int t = 0; t <= r; ++t) acc -= X[(i0 + b + r) * P + i0 + b + t] * A[(i0 + t) * P + i0 + b + c];
                X[(i0 + b + r) * P + i0 + c] = acc;
            } else {       // -A1^{-1} (B D^{-1}), A1^{-1} upper
                for (int t = r; t < b; ++t) acc -= X[(i0 + r) * P + i0 + t] * A[(i0 + b + t) * P + i0 + c];
                X[(i0 + r) * P + i0 + b + c] = acc;
            }
        }
        __syncthreads();
    }
}

// One CTA factors one box's panel M[k:n, k:k+nb] (Algorithm 1's batched LU,
// P A_ii = L U with partial pivoting).  The panel is processed in inner blocks
// of ib columns that live in shared memory (column-major, R rows, in the order
// the rows were loaded; pos2row maps a pivot position to its loaded row); the
// pivot search is a warp-shuffle arg-max followed by a cross-warp pass.  After the
// panel: the step's row permutation perm[r] (source row of local row r),
// F top = -L11^{-1} and B top = -U11^{-1}.
constexpr int kSwapPer = (64 * kMaxNB + kPanelThreads - 1) / kPanelThreads;

template <typename T>
__global__ void __launch_bounds__(kPanelThreads)
k_panel(T* __restrict__ M, long long ldm, long long sM, int n, int k, int nb, int ib,
        int* __restrict__ perm, long long sP, T* __restrict__ Ftop, long long ldf, long long sF,
        T* __restrict__ Btop, long long ldb, long long sB, int* status, const int* skip)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Sb = reinterpret_cast<T*>(smem_raw);
    const int R0 = n - k;
    unsigned short* pos2row = reinterpret_cast<unsigned short*>(smem_raw + (size_t)ib * R0 * sizeof(T));
    unsigned short* row2pos = pos2row + R0;
    unsigned char* active = reinterpret_cast<unsigned char*>(row2pos + R0);
    __shared__ int swp[kMaxNB];
    __shared__ T red_v[2][kPanelThreads / 32];
    __shared__ int red_i[2][kPanelThreads / 32];
    __shared__ int s_sing, s_nmv;
    __shared__ unsigned short mv[64];
    __shared__ T Xs[32 * kMaxNB];

    const int box = blockIdx.x;
    if (skip && skip[box]) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kPanelThreads / 32;
    T* Mb = M + box * sM;
    if (tid == 0) s_sing = 0;

    for (int jb = 0; jb < nb; jb += ib) {
        const int w = imin(ib, nb - jb);
        const int R = R0 - jb;
        T* base = Mb + (long long)(k + jb) * ldm + (k + jb);
        for (int idx = tid; idx < R * w; idx += kPanelThreads) {
            const int r = idx / w, c = idx - r * w;
            Sb[c * R + r] = base[(long long)r * ldm + c];
        }
        for (int r = tid; r < R; r += kPanelThreads) {
            pos2row[r] = (unsigned short)r;
            row2pos[r] = (unsigned short)r;
            active[r] = 1;
        }
        __syncthreads();
        // Rows stay where they were loaded; interchanges are tracked in
        // pos2row/row2pos and applied when the block is written back.  Each
        // thread owns rows tid, tid + 512, ...; the arg-max candidates of the
        // next column are formed during this column's update, so every pivot
        // column costs one barrier.  Ties go to the lowest loaded row.
        {
            T bv = T(-1);
            int bi = INT_MAX;
            for (int r = tid; r < R; r += kPanelThreads) argmax_merge(bv, bi, tabs(Sb[r]), r);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                argmax_merge(bv, bi, ov, oi);
            }
            if (lane == 0) { red_v[0][warp] = bv; red_i[0][warp] = bi; }
        }
        __syncthreads();
        for (int c = 0; c < w; ++c) {
            const int cur = c & 1;
            T bv = red_v[cur][0];
            int bi = red_i[cur][0];
#pragma unroll
            for (int q = 1; q < NW; ++q) argmax_merge(bv, bi, red_v[cur][q], red_i[cur][q]);
            // Candidates come from rows still active, so a valid index needs no
            // further test; none (every |value| NaN) keeps the row in place.
            int pr = bi;
            if (pr < 0 || pr >= R) pr = pos2row[c];
            if (tid == 0) {
                const int pp = row2pos[pr], qr = pos2row[c];
                pos2row[c] = (unsigned short)pr;
                pos2row[pp] = (unsigned short)qr;
                row2pos[pr] = (unsigned short)c;
                row2pos[qr] = (unsigned short)pp;
                swp[jb + c] = jb + pp;
                active[pr] = 0;
            }
            T piv = Sb[c * R + pr];
            if (piv == T(0)) {
                // Exactly singular: record it and keep the arithmetic finite.
                if (tid == 0) s_sing = 1;
                piv = T(1);
            }
            const T rinv = T(1) / piv;
            T nv = T(-1);
            int ni = INT_MAX;
            for (int r = tid; r < R; r += kPanelThreads) {
                if (r == pr || !active[r]) continue;
                const T l = Sb[c * R + r] * rinv;
                Sb[c * R + r] = l;
                for (int cc = c + 1; cc < w; ++cc) Sb[cc * R + r] -= l * Sb[cc * R + pr];
                if (c + 1 < w) argmax_merge(nv, ni, tabs(Sb[(c + 1) * R + r]), r);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, nv, off);
                const int oi = __shfl_xor_sync(0xffffffffu, ni, off);
                argmax_merge(nv, ni, ov, oi);
            }
            if (lane == 0) { red_v[cur ^ 1][warp] = nv; red_i[cur ^ 1][warp] = ni; }
            __syncthreads();
        }
        for (int idx = tid; idx < R * w; idx += kPanelThreads) {
            const int r = idx / w, c = idx - r * w;
            base[(long long)r * ldm + c] = Sb[c * R + pos2row[r]];
        }
        __syncthreads();
        // This block's interchanges on the panel's other columns: at most 2w
        // positions moved (pos2row[r] != r); their values are all read before
        // any is written.
        if (tid == 0) s_nmv = 0;
        __syncthreads();
        for (int r = tid; r < R; r += kPanelThreads)
            if (pos2row[r] != r) mv[atomicAdd(&s_nmv, 1)] = (unsigned short)r;
        __syncthreads();
        {
            const int nmv = s_nmv, nother = nb - w;
            T val[kSwapPer];
#pragma unroll
            for (int u = 0; u < kSwapPer; ++u) {
                const int idx = tid + u * kPanelThreads;
                if (idx < nmv * nother) {
                    const int q = idx / nother, oc = idx - q * nother;
                    const int col = oc < jb ? oc : oc + w;
                    val[u] = Mb[(long long)(k + jb + pos2row[mv[q]]) * ldm + k + col];
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kSwapPer; ++u) {
                const int idx = tid + u * kPanelThreads;
                if (idx < nmv * nother) {
                    const int q = idx / nother, oc = idx - q * nother;
                    const int col = oc < jb ? oc : oc + w;
                    Mb[(long long)(k + jb + mv[q]) * ldm + k + col] = val[u];
                }
            }
        }
        __syncthreads();
        // Right-looking update of the panel columns [jb+w, nb): U12 rows by a
        // forward substitution, then the trailing rows, each thread taking a
        // 4 x 4 tile (per pivot column: 4 loads of L, one 4-wide load of U12,
        // 16 multiply-adds); consecutive threads take consecutive column
        // groups of the same rows, so the global accesses are contiguous.
        const int ncr = nb - jb - w;
        if (ncr > 0) {
            T* rb = Mb + (long long)(k + jb) * ldm + (k + jb + w);
            for (int col = tid; col < ncr; col += kPanelThreads) {
                for (int c = 0; c < w; ++c) {
                    T x = rb[(long long)c * ldm + col];
                    const int pc = pos2row[c];
                    for (int c2 = 0; c2 < c; ++c2) x -= Sb[c2 * R + pc] * Xs[c2 * kMaxNB + col];
                    Xs[c * kMaxNB + col] = x;
                    rb[(long long)c * ldm + col] = x;
                }
            }
            __syncthreads();
            const int rg = (R - w + 3) >> 2, cg = (ncr + 3) >> 2;
            const bool vec = sizeof(T) == 4 && ((reinterpret_cast<uintptr_t>(rb) & 15) == 0) && (ldm & 3) == 0;
            for (int item = tid; item < rg * cg; item += kPanelThreads) {
                const int gi = item / cg, gc = item - gi * cg;
                const int r0 = w + 4 * gi, c0 = 4 * gc;
                int src[4];
                T acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r0 + u;
                    src[u] = pos2row[r < R ? r : w];
                    T* rowp = rb + (long long)r * ldm + c0;
                    if (r < R && vec && c0 + 3 < ncr) {
                        const float4 v4 = *reinterpret_cast<const float4*>(rowp);
                        acc[u][0] = T(v4.x); acc[u][1] = T(v4.y); acc[u][2] = T(v4.z); acc[u][3] = T(v4.w);
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = (r < R && c0 + v < ncr) ? rowp[v] : T(0);
                    }
                }
                for (int c = 0; c < w; ++c) {
                    T a[4], bv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) a[u] = Sb[c * R + src[u]];
#pragma unroll
                    for (int v = 0; v < 4; ++v) bv[v] = Xs[c * kMaxNB + c0 + v];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] -= a[u] * bv[v];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r0 + u;
                    if (r >= R) break;
                    T* rowp = rb + (long long)r * ldm + c0;
                    if (vec && c0 + 3 < ncr) {
                        *reinterpret_cast<float4*>(rowp) =
                            make_float4(float(acc[u][0]), float(acc[u][1]), float(acc[u][2]), float(acc[u][3]));
                    } else {
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (c0 + v < ncr) rowp[v] = acc[u][v];
                    }
                }
            }
            __syncthreads();
        }
    }

    // Row permutation of the step: position r holds the old row perm[r].
    int* pb = perm + box * sP;
    for (int r = tid; r < R0; r += kPanelThreads) pb[r] = r;
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < nb; ++i) {
            const int a = i, bb = swp[i];
            if (a != bb) { const int t = pb[a]; pb[a] = pb[bb]; pb[bb] = t; }
        }
    if (tid == 0 && s_sing && status[box] == 0) status[box] = HPS_ESINGULAR;

    // Inverses of the diagonal blocks, L11^{-1} and U11^{-1}, by blocks.
    int Pd = 16;
    while (Pd < nb) Pd *= 2;
    T* Ap = Sb;                 // Pd x Pd, padded with the identity
    T* X = Sb + Pd * Pd;        // the inverse
    for (int idx = tid; idx < Pd * Pd; idx += kPanelThreads) {
        const int r = idx / Pd, c = idx - r * Pd;
        Ap[idx] = (r < nb && c < r) ? Mb[(long long)(k + r) * ldm + k + c] : T(0);
        X[idx] = T(0);
    }
    __syncthreads();
    tri_inverse<T>(Ap, X, Pd, true, tid);
    T* Fb = Ftop + box * sF;
    for (int idx = tid; idx < nb * nb; idx += kPanelThreads) {
        const int r = idx / nb, c = idx - r * nb;
        Fb[r * ldf + c] = -X[r * Pd + c];
    }
    __syncthreads();
    for (int idx = tid; idx < Pd * Pd; idx += kPanelThreads) {
        const int r = idx / Pd, c = idx - r * Pd;
        Ap[idx] = (r < nb && c >= r && c < nb) ? Mb[(long long)(k + r) * ldm + k + c] : (r == c && r >= nb ? T(1) : T(0));
        X[idx] = T(0);
    }
    __syncthreads();
    tri_inverse<T>(Ap, X, Pd, false, tid);
    T* Bb = Btop + box * sB;
    for (int idx = tid; idx < nb * nb; idx += kPanelThreads) {
        const int r = idx / nb, c = idx - r * nb;
        Bb[r * ldb + c] = -X[r * Pd + c];
    }
}

// ---------------------------------------------------------------- gather

// W = M[k:k+nb, c0:c0+ncols] and G = M[k + perm[i], c0:c0+ncols] (perm NULL:
// identity, W skipped when NULL).
template <typename T>
__global__ void k_gather(const T* __restrict__ M, long long ldm, long long sM, int k, int nb, int c0,
                         int ncols, const int* __restrict__ perm, long long sP, T* __restrict__ W,
                         T* __restrict__ G, long long ldg, long long sG, const int* skip)
{
    const int box = blockIdx.z;
    if (skip && skip[box]) return;
    const int i = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncols || i >= nb) return;
    const T* Mb = M + box * sM;
    const int src = perm ? k + perm[box * sP + i] : k + i;
    G[box * sG + (long long)i * ldg + c] = Mb[(long long)src * ldm + c0 + c];
    if (W) W[box * sG + (long long)i * ldg + c] = Mb[(long long)(k + i) * ldm + c0 + c];
}

// ---------------------------------------------------------------- update product

// O = src + alpha * A B, register-tiled on the CUDA cores (TM x TN outputs per
// thread).  Modes: GM_SET src = 0; GM_ACC src = O; GM_FWD rows < split take
// 0 and the others their permuted source row (in place or from W); GM_BWD
// rows < split keep O, the others take 0.
template <typename T, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
k_gemm(GemmArgs<T> g)
{
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN];
    const int box = blockIdx.z;
    if (g.skip && g.skip[box]) return;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const T* A = g.A + box * g.sA;
    const T* B = g.B + box * g.sB;
    T* O = g.O + box * g.sO;
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    T acc[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[a][c] = T(0);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        for (int idx = threadIdx.x; idx < BM * BK; idx += NT) {
            const int i = idx / BK, kk = idx - i * BK;
            const int r = m0 + i, kc = k0 + kk;
            As[kk][i] = (r < g.M && kc < g.K) ? A[(long long)r * g.lda + kc] : T(0);
        }
        for (int idx = threadIdx.x; idx < BK * BN; idx += NT) {
            const int kk = idx / BN, jj = idx - kk * BN;
            const int kc = k0 + kk, c = n0 + jj;
            Bs[kk][jj] = (kc < g.K && c < g.N) ? B[(long long)kc * g.ldb + c] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T av[TM], bv[TN];
#pragma unroll
            for (int a = 0; a < TM; ++a) av[a] = As[kk][ty * TM + a];
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx * TN + c];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int c = 0; c < TN; ++c) acc[a][c] += av[a] * bv[c];
        }
        __syncthreads();
    }
    const T* Wb = g.W ? g.W + box * g.sW : nullptr;
    const int* Pb = g.perm ? g.perm + box * g.sP : nullptr;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int r = m0 + ty * TM + a;
        if (r >= g.M) continue;
        const T* srow = nullptr;
        bool zero = false;
        if (g.mode == GM_SET) zero = true;
        else if (g.mode == GM_ACC) srow = O + (long long)r * g.ldo;
        else if (g.mode == GM_FWD) {
            if (r < g.split) zero = true;
            else {
                const int pr = Pb[r];
                srow = (pr >= g.split) ? O + (long long)r * g.ldo : Wb + (long long)pr * g.ldw;
            }
        } else {
            if (r < g.split) srow = O + (long long)r * g.ldo;
            else zero = true;
        }
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int cc = n0 + tx * TN + c;
            if (cc >= g.N) continue;
            const T s = zero ? T(0) : srow[cc];
            O[(long long)r * g.ldo + cc] = s + g.alpha * acc[a][c];
        }
    }
}

// ---------------------------------------------------------------- D_n products

// out(row r, column c) = sign_f ( sum_{l interior} D_a[e, l] X[line(r, l), c]
//                                 + [add_abb] (D_a[e, e] [c = r] + D_a[e, e'] [c = opp(r)]) )
// for face row r on face f (axis a, own index e, opposite e').  With X = S this
// is T = A_bb + A_bi S (Eq. 8); with X = v and no A_bb it is h = A_bi v.
// One thread forms the outputs of both faces of an axis at the same face
// position (rows f qq + s and (f + 1) qq + s), which read the same grid line
// of X: the line is loaded once.
__global__ void k_dn(int p, int n, int m, int ncols, const double* __restrict__ D,
                     const double* __restrict__ X, long long ldx, long long sX, double* __restrict__ out,
                     long long sOut, int transposed_out, int add_abb)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r2 = blockIdx.y;   // axis * qq + s
    const int box = blockIdx.z;
    if (c >= ncols) return;
    const int q = p - 2, qq = q * q;
    const int axis = r2 / qq, s = r2 - axis * qq, a = s % q + 1, bb = s / q + 1;
    const int r0 = 2 * axis * qq + s, r1 = r0 + qq;   // face 2 axis (node index 0), face 2 axis + 1 (p - 1)
    const double* D0 = D + axis * p * p;               // row 0 of D_axis
    const double* D1 = D0 + (p - 1) * p;               // row p - 1
    const double* Xb = X + box * sX;
    long long base, stride;
    if (axis == 0) { base = q * (a - 1) + qq * (bb - 1) - 1; stride = 1; }
    else if (axis == 1) { base = (a - 1) + qq * (bb - 1) - q; stride = q; }
    else { base = (a - 1) + q * (bb - 1) - qq; stride = qq; }
    double acc0 = 0.0, acc1 = 0.0;
    for (int l = 1; l <= q; ++l) {
        const double x = Xb[(base + l * stride) * ldx + c];
        acc0 += __ldg(D0 + l) * x;
        acc1 += __ldg(D1 + l) * x;
    }
    if (add_abb) {
        if (c == r0) { acc0 += __ldg(D0); acc1 += __ldg(D1); }
        if (c == r1) { acc0 += __ldg(D0 + p - 1); acc1 += __ldg(D1 + p - 1); }
    }
    acc0 = -acc0;   // outward normal of the low face is -axis
    double* ob = out + box * sOut;
    if (transposed_out) {
        ob[(long long)c * m + r0] = acc0;
        ob[(long long)c * m + r1] = acc1;
    } else {
        ob[(long long)r0 * m + c] = acc0;
        ob[(long long)r1 * m + c] = acc1;
    }
}

// ---------------------------------------------------------------- refinement

// Sum of v over the CTA added to *out (one atomic per CTA).
template <typename V>
__device__ __forceinline__ void block_sum_add(V v, double* out)
{
    __shared__ V part[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) part[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += (double)part[i];
        atomicAdd(out, t);
    }
}

// X = src in FP64 (the first solution of the refinement); with xnorm, also
// ||X||^2 per box into xnorm[2 box + 1] (FP32 partial sums: the stopping rule
// needs the size of X, not its digits).  CTAs loop over rows, threads over
// columns.
template <typename TS>
__global__ void __launch_bounds__(256)
k_extract(const TS* __restrict__ src, long long lds, long long sS, int n, int ncols, double* __restrict__ X,
          long long ldx, long long sX, double* xnorm)
{
    const int box = blockIdx.y;
    float xn = 0.0f;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const TS* srow = src + box * sS + (long long)r * lds;
        double* xrow = X + box * sX + (long long)r * ldx;
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
            const TS v = srow[c];
            if constexpr (sizeof(TS) == 4) xrow[c] = f2d(v);
            else xrow[c] = double(v);
            if (xnorm) xn = fmaf((float)v, (float)v, xn);
        }
    }
    if (xnorm) block_sum_add(xn, xnorm + 2 * box + 1);
}

// Shared-memory loads of the line tables kept in the loop: the tables are
// invariant across a CTA's lines, and hoisting them would take ~2h^2 registers.
__device__ __forceinline__ double2 lds_f64x2(const double* p)
{
    double2 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ double lds_f64(const double* p)
{
    double v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
    return v;
}

// One line of q interior values along an axis through the interior block of
// D^2 (centro-symmetric: D2[i][l] = D2[q+1-i][q+1-l], held exactly so on the
// host).  With e_l = x_l + x_{q+1-l} and o_l = x_l - x_{q+1-l}, the outputs
// i and q+1-i are (sum_l E[i][l] e_l) +- (sum_l O[i][l] o_l), with
// E = (D2[i][l] + D2[i][q+1-l]) / 2 and O = (D2[i][l] - D2[i][q+1-l]) / 2, so
// a pair costs 2h multiply-adds instead of 2q (h = q/2; an odd q adds the
// middle column).  tab holds (E, O) pairs [h][h], then for odd q the middle
// column [h], the middle row's E part [h] and its diagonal entry.
template <int Q, class Emit>
__device__ __forceinline__ void eo_line(const double* __restrict__ src, int stride, const double* tab, Emit&& emit)
{
    constexpr int H = Q / 2;
    double x[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) x[l] = src[l * stride];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        const double a = x[l], z = x[Q - 1 - l];
        x[l] = a + z;
        x[Q - 1 - l] = a - z;
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        double2 eo = lds_f64x2(tab + 2 * (i * H));
        double se = eo.x * x[0];
        double so = eo.y * x[Q - 1];
#pragma unroll
        for (int l = 1; l < H; ++l) {
            eo = lds_f64x2(tab + 2 * (i * H + l));
            se = fma(eo.x, x[l], se);
            so = fma(eo.y, x[Q - 1 - l], so);
        }
        if constexpr ((Q & 1) != 0) se = fma(lds_f64(tab + 2 * H * H + i), x[H], se);
        emit(i, se + so);
        emit(Q - 1 - i, se - so);
    }
    if constexpr ((Q & 1) != 0) {
        const double* Em = tab + 2 * H * H + H;
        double sm = lds_f64(Em + H) * x[H];
#pragma unroll
        for (int l = 0; l < H; ++l) sm = fma(lds_f64(Em + l), x[l], sm);
        emit(H, sm);
    }
}

// Doubles per axis table (even, so every axis table stays 16-byte aligned).
template <int Q>
__host__ __device__ constexpr int eo_tab_size()
{
    return (2 * (Q / 2) * (Q / 2) + ((Q & 1) ? 2 * (Q / 2) + 1 : 0) + 1) & ~1;
}

// Threads of the residual CTA (one per grid line of a pass) and the CTAs per
// SM the register cap allows for (about 96 registers a thread).
template <int Q>
__host__ __device__ constexpr int res_threads() { return ((Q * Q + 31) / 32) * 32; }
template <int Q>
__host__ __device__ constexpr int res_min_blocks()
{
    return 65536 / (res_threads<Q>() * 96) > 1 ? 65536 / (res_threads<Q>() * 96) : 1;
}

// R = B - A_ii X in FP64, matrix-free: A_ii X applies the 1-D second-derivative
// matrices along the three grid lines through each interior node plus the
// kappa^2 b diagonal (the Kronecker structure of Eq. 2's collocation); B is
// -A_ib (DTN), f_i (LOAD) or -A_ib u_b (TRACE).  One CTA takes one column of
// X for one box, staged in shared memory, with one thread per grid line; the
// three axes are applied line by line (eo_line) into an accumulator, the z
// pass finishing each point.  R is written in FP32 for the correction solve.
// CONV: the operator also has the first-order term div(beta u) (beta per box
// [3][p^3]): each pass subtracts D_a (beta_a X) along its lines (the interior
// part; the face part is in B), by a plain q-term sum per output.
template <int Q, bool CONV>
__global__ void __launch_bounds__(res_threads<Q>(), res_min_blocks<Q>())
k_residual(int p, int n, int nrhs, const double* __restrict__ D2, double kappa2,
           const double* __restrict__ kappa_box, const double* __restrict__ b, long long sb, int rhs_kind,
           const double* __restrict__ rhs, long long s_rhs, const double* __restrict__ X, long long ldx,
           long long sX, float* __restrict__ R, long long ldr, long long sR, const int* skip,
           const double* __restrict__ kb, const double* __restrict__ D1, const double* __restrict__ beta)
{
    constexpr int H = Q / 2, TA = eo_tab_size<Q>();
    constexpr int q = Q, qq = Q * Q;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int box = blockIdx.y;
    if (skip && skip[box]) return;
    const int cw = blockIdx.x;                               // column of X and R
    const int pp = p * p;
    double* Xs = reinterpret_cast<double*>(smem_raw);       // [n]
    double* Ac = Xs + n;                                     // [n]
    double* D2s = Ac + n;                                    // [3][p][p]
    double* tab = D2s + ((3 * pp + 1) & ~1);                 // [3][TA]
    double* D1s = tab + 3 * TA;                              // CONV: [3][p][p]
    const int p3 = pp * p;
    const double* bt = CONV ? beta + (long long)box * 3 * p3 : nullptr;
    if constexpr (CONV)
        for (int idx = threadIdx.x; idx < 3 * pp; idx += blockDim.x) D1s[idx] = D1[idx];
    // CONV: sum_l D_a[o][l] beta_a(node l) X(node l) over the interior nodes l of a line
    auto conv_line = [&](int a, int o, const double* xline, int xstride, const double* bline, int bstride) {
        double cv = 0.0;
#pragma unroll 2
        for (int l = 1; l <= Q; ++l)
            cv = fma(D1s[a * pp + o * p + l], __ldg(bline + l * bstride) * xline[(l - 1) * xstride], cv);
        return cv;
    };
    const double* Xb = X + box * sX + cw;
    for (int r = threadIdx.x; r < n; r += blockDim.x) Xs[r] = Xb[(long long)r * ldx];
    for (int idx = threadIdx.x; idx < 3 * pp; idx += blockDim.x) D2s[idx] = D2[idx];
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * TA; idx += blockDim.x) {
        const int a = idx / TA, t = idx - a * TA;
        const double* D = D2s + a * pp;
        double v;
        if (t < 2 * H * H) {
            constexpr int Hd = H > 0 ? H : 1;   // q = 1 has no pairs
            const int tt = t >> 1, i = tt / Hd + 1, l = tt - (tt / Hd) * Hd + 1;
            const double u = D[i * p + l], w = D[i * p + (p - 1 - l)];
            v = (t & 1) ? 0.5 * (u - w) : 0.5 * (u + w);
        } else if (t >= 2 * H * H + ((Q & 1) ? 2 * H + 1 : 0)) {
            v = 0.0;                            // padding
        } else {
            const int t2 = t - 2 * H * H, mid = H + 1;
            if (t2 < H) v = D[(t2 + 1) * p + mid];
            else if (t2 < 2 * H) {
                const int l = t2 - H + 1;
                v = 0.5 * (D[mid * p + l] + D[mid * p + (p - 1 - l)]);
            } else v = D[mid * p + mid];
        }
        tab[idx] = v;
    }
    __syncthreads();
    const int ln = threadIdx.x;
    // x lines (ln = j0 + q k0): Ac = D2x X
    if (ln < qq) {
        const int base = ln * q;
        eo_line<Q>(Xs + base, 1, tab, [&](int i, double v) { Ac[base + i] = v; });
        if constexpr (CONV) {
            const int j = ln % q + 1, k = ln / q + 1;
            const double* bl = bt + p * j + pp * k;   // beta_x along this line (node index l)
            for (int i = 0; i < q; ++i) Ac[base + i] -= conv_line(0, i + 1, Xs + base, 1, bl, 1);
        }
    }
    __syncthreads();
    // y lines (ln = i0 + q k0): Ac += D2y X
    if (ln < qq) {
        const int base = ln % q + qq * (ln / q);
        eo_line<Q>(Xs + base, q, tab + TA, [&](int j, double v) { Ac[base + q * j] += v; });
        if constexpr (CONV) {
            const int i = ln % q + 1, k = ln / q + 1;
            const double* bl = bt + p3 + i + pp * k;   // beta_y along this line
            for (int j = 0; j < q; ++j) Ac[base + q * j] -= conv_line(1, j + 1, Xs + base, q, bl, p);
        }
    }
    __syncthreads();
    // z lines (ln = i0 + q j0), then every point of the line is finished.
    if (ln < qq) {
        const double* bb = b + box * sb;
        const double k2 = kappa_box ? kappa_box[box] * kappa_box[box] : kappa2;
        const int i = ln % q + 1, j = ln / q + 1;
        int cg = cw, kind = rhs_kind;
        if (kind == RHS_DTN_LOAD) {
            if (cg < 6 * qq) kind = RHS_DTN;
            else { kind = RHS_LOAD; cg -= 6 * qq; }
        }
        const double* rx = D2s + i * p;
        const double* ry = D2s + pp + j * p;
        float* Rb = R + box * sR + cw;
        const double* kbb = kb ? kb + (long long)box * n : nullptr;
        // CONV: the first-order coupling of interior node (i, j, k) to face node
        // e of axis a is D_a[own][e] beta_a(face node); B = -A_ib carries minus it
        auto c1 = [&](int a, int own, int e, int ii, int jj, int kk) -> double {
            if constexpr (CONV) return D1s[a * pp + own * p + e] * __ldg(bt + a * p3 + ii + p * jj + pp * kk);
            else return 0.0;
        };
        eo_line<Q>(Xs + ln, qq, tab + 2 * TA, [&](int k0, double v) {
            const int k = k0 + 1, r = ln + qq * k0;
            const double* rz = D2s + 2 * pp + k * p;
            const int gi = i + p * j + pp * k;
            // R = B - A_ii x = B + (D2 sums) x + kappa^2 b x (- div(beta x) with CONV)
            double res = fma(kbb ? kbb[r] : k2 * bb[gi], Xs[r], Ac[r] + v);
            if constexpr (CONV) res -= conv_line(2, k, Xs + ln, qq, bt + 2 * p3 + i + p * j, pp);
            if (kind == RHS_DTN) {   // -A_ib e_f: nonzero only next to face node f
                const int f = cg / qq, s2 = cg % qq, a = s2 % q + 1, b2 = s2 / q + 1;
                const int axis = f >> 1, e = (f & 1) ? p - 1 : 0;
                if (axis == 0 && j == a && k == b2) res += rx[e] - c1(0, i, e, e, j, k);
                else if (axis == 1 && i == a && k == b2) res += ry[e] - c1(1, j, e, i, e, k);
                else if (axis == 2 && i == a && j == b2) res += rz[e] - c1(2, k, e, i, j, e);
            } else if (kind == RHS_LOAD) {
                res += rhs[box * s_rhs + (long long)cg * p * pp + gi];
            } else {
                const double* ub = rhs + box * s_rhs + (long long)cg * 6 * qq;
                const int sx = (j - 1) + q * (k - 1), sy = (i - 1) + q * (k - 1), sz = (i - 1) + q * (j - 1);
                const int e1 = p - 1;
                res += (rx[0] - c1(0, i, 0, 0, j, k)) * ub[sx] + (rx[e1] - c1(0, i, e1, e1, j, k)) * ub[qq + sx] +
                       (ry[0] - c1(1, j, 0, i, 0, k)) * ub[2 * qq + sy] +
                       (ry[e1] - c1(1, j, e1, i, e1, k)) * ub[3 * qq + sy] +
                       (rz[0] - c1(2, k, 0, i, j, 0)) * ub[4 * qq + sz] +
                       (rz[e1] - c1(2, k, e1, i, j, e1)) * ub[5 * qq + sz];
            }
            Rb[(long long)r * ldr] = d2f_rn(res);
        });
    }
}

// ------------------------------------------- double-float first residual
// The first correction starts from the FP32 solution X0, whose error (about
// the LU's precision times the conditioning) leaves room for a residual less
// accurate than FP64: with about 2^-46 relative to sum |terms| it adds an
// error near cond(A_ii) 2^-46 to X1, far below X0's.  That residual runs on
// the FP32 pipes as double-float ("hi + lo" float pairs): each X0 entry is
// exactly one float, a line's even/odd butterfly is exact (TwoSum), the
// products take their leading part exactly (TwoProduct by FMA) and sums carry
// their rounding error (TwoSum, Knuth).  The _rn intrinsics keep the compiler
// from contracting or reassociating these steps.

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (h, l) = (ah + al)(bh + bl), al bl dropped (2^-48 relative)
__device__ __forceinline__ void df_mul(float& h, float& l, float ah, float al, float bh, float bl)
{
    h = __fmul_rn(ah, bh);
    l = __fmaf_rn(ah, bh, -h);
    l = __fmaf_rn(ah, bl, l);
    l = __fmaf_rn(al, bh, l);
}
// (h, l) += (ah + al)(bh + bl)
__device__ __forceinline__ void df_mac(float& h, float& l, float ah, float al, float bh, float bl)
{
    float p, e, s, c;
    df_mul(p, e, ah, al, bh, bl);
    two_sum(h, p, s, c);
    h = s;
    l = __fadd_rn(l, __fadd_rn(c, e));
}
// (h, l) += (ah + al) b for a float b
__device__ __forceinline__ void df_mac1(float& h, float& l, float ah, float al, float b)
{
    const float p = __fmul_rn(ah, b);
    float e = __fmaf_rn(ah, b, -p);
    e = __fmaf_rn(al, b, e);
    float s, c;
    two_sum(h, p, s, c);
    h = s;
    l = __fadd_rn(l, __fadd_rn(c, e));
}
// (h, l) += (bh, bl)
__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl)
{
    float s, c;
    two_sum(h, bh, s, c);
    h = s;
    l = __fadd_rn(l, __fadd_rn(c, bl));
}
__device__ __forceinline__ float4 lds_f32x4(const float4* p)
{
    float4 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds_f32x2(const float2* p)
{
    float2 v;
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

template <int Q>
__host__ __device__ constexpr int df_tab_q() { return (Q / 2) * (Q / 2) + ((Q & 1) ? Q / 2 + 1 : 0) + Q; }

// eo_line in double-float: one line of FP32 values through the split tables
// (E, O as (hi, lo) pairs); emit(i, hi, lo).
template <int Q, class Emit>
__device__ __forceinline__ void eo_line_df(const float* __restrict__ src, int stride, const float4* tab, Emit&& emit)
{
    constexpr int H = Q / 2;
    float x[Q], y[Q];   // after the butterfly: (x, y)[l] = e_l and (x, y)[Q-1-l] = o_l, exactly
#pragma unroll
    for (int l = 0; l < Q; ++l) x[l] = src[l * stride];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        const float a = x[l], z = x[Q - 1 - l];
        two_sum(a, z, x[l], y[l]);
        two_sum(a, -z, x[Q - 1 - l], y[Q - 1 - l]);
    }
    const float2* t2 = reinterpret_cast<const float2*>(tab + H * H);   // odd q: middle column, row, diagonal
    // The pair loop stays rolled (x and y are indexed by l only): unrolled, the
    // three passes outgrow the instruction cache.
#pragma unroll 1
    for (int i = 0; i < H; ++i) {
        float4 t = lds_f32x4(tab + i * H);
        float seh, sel, soh, sol;
        df_mul(seh, sel, t.x, t.y, x[0], y[0]);
        df_mul(soh, sol, t.z, t.w, x[Q - 1], y[Q - 1]);
#pragma unroll
        for (int l = 1; l < H; ++l) {
            t = lds_f32x4(tab + i * H + l);
            df_mac(seh, sel, t.x, t.y, x[l], y[l]);
            df_mac(soh, sol, t.z, t.w, x[Q - 1 - l], y[Q - 1 - l]);
        }
        if constexpr ((Q & 1) != 0) {
            const float2 mc = lds_f32x2(t2 + i);
            df_mac1(seh, sel, mc.x, mc.y, x[H]);
        }
        float ph = seh, pl = sel;
        df_add(ph, pl, soh, sol);
        emit(i, ph, pl);
        df_add(seh, sel, -soh, -sol);
        emit(Q - 1 - i, seh, sel);
    }
    if constexpr ((Q & 1) != 0) {
        const float2 dg = lds_f32x2(t2 + 2 * H);
        float smh = __fmul_rn(dg.x, x[H]), sml = __fmaf_rn(dg.x, x[H], -smh);
        sml = __fmaf_rn(dg.y, x[H], sml);
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const float2 em = lds_f32x2(t2 + H + l);
            df_mac(smh, sml, em.x, em.y, x[l], y[l]);
        }
        emit(H, smh, sml);
    }
}

// The same line in plain FP32 with the leading (hi) parts of the tables:
// the contribution of the low part of a split FP64 X, itself 2^-24 of X, so
// FP32 rounding here is 2^-48 of the terms.  emit(i, value).
template <int Q, class Emit>
__device__ __forceinline__ void eo_line_f32(const float* __restrict__ src, int stride, const float4* tab, Emit&& emit)
{
    constexpr int H = Q / 2;
    float x[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) x[l] = src[l * stride];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        const float a = x[l], z = x[Q - 1 - l];
        x[l] = a + z;
        x[Q - 1 - l] = a - z;
    }
    const float2* t2 = reinterpret_cast<const float2*>(tab + H * H);
#pragma unroll 1
    for (int i = 0; i < H; ++i) {
        float se = 0.0f, so = 0.0f;
#pragma unroll
        for (int l = 0; l < H; ++l) {
            const float4 t = lds_f32x4(tab + i * H + l);
            se = fmaf(t.x, x[l], se);
            so = fmaf(t.z, x[Q - 1 - l], so);
        }
        if constexpr ((Q & 1) != 0) se = fmaf(lds_f32x2(t2 + i).x, x[H], se);
        emit(i, se + so);
        emit(Q - 1 - i, se - so);
    }
    if constexpr ((Q & 1) != 0) {
        float sm = lds_f32x2(t2 + 2 * H).x * x[H];
#pragma unroll
        for (int l = 0; l < H; ++l) sm = fmaf(lds_f32x2(t2 + H + l).x, x[l], sm);
        emit(H, sm);
    }
}

// R = B - A_ii X0 for the FP32 first solution X0, in double-float, written
// over X0 (each CTA reads its whole column before it writes).  Same passes
// and CTA shape as k_residual; DTN right-hand sides are added in
// double-float, LOAD and TRACE ones in FP64 at the end.
// X64: X is an FP64 solution (X64 [n][ldx] per box, stride sX64) split per
// entry into hi = float(x) and lo = float(x - hi) (x - hi is exact in FP64,
// lo rounds at 2^-48 of x): A_ii hi in double-float as above, A_ii lo in FP32
// (eo_line_f32, added to the pairs' low parts), R written to X0R (which is
// then output only).  Otherwise X0R holds X0 and receives R.
// CTAs per SM the double-float residual is built for up to q = 16: shared
// memory (the column, its low parts and the accumulator) and registers (72 a
// thread) both allow four at q = 14; larger q keep the FP64 kernel's bound
// (a tighter one spills there).
template <int Q>
__host__ __device__ constexpr int res_df_min_blocks()
{
    return Q > 16 ? res_min_blocks<Q>()
                  : (65536 / (res_threads<Q>() * 72) > 1 ? 65536 / (res_threads<Q>() * 72) : 1);
}

template <int Q, bool X64>
__global__ void __launch_bounds__(res_threads<Q>(), res_df_min_blocks<Q>())
k_residual_df(int p, int n, const float4* __restrict__ DF, const float2* __restrict__ kbs, int rhs_kind,
              const double* __restrict__ rhs, long long s_rhs, float* X0R, long long ld, long long sbx,
              const int* skip, const double* __restrict__ Xin, long long ldx, long long sX64)
{
    constexpr int TF = df_tab_q<Q>(), q = Q, qq = Q * Q;
    constexpr int BO = TF - Q;   // boundary couplings within an axis table
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int box = blockIdx.y;
    if (skip && skip[box]) return;
    const int cw = blockIdx.x;
    float4* tab = reinterpret_cast<float4*>(smem_raw);       // [3][TF]
    float2* Ac = reinterpret_cast<float2*>(tab + 3 * TF);   // [n]
    float* Xs = reinterpret_cast<float*>(Ac + n);           // [n]
    float* Xl = Xs + n;                                      // [n] low parts (X64 only)
    float* col = X0R + box * sbx + cw;
    const float2* kbb = kbs + (long long)box * n;            // kappa^2 b (hi, lo), read where used
    // The column (one entry per row, rows ld apart): every load of a thread
    // issued before its stores, so one memory latency covers the column.
    if constexpr (X64) {
        const double* xc = Xin + box * sX64 + cw;
        constexpr int LU = 8;
        for (int r0 = threadIdx.x; r0 < n; r0 += LU * blockDim.x) {
            double v[LU];
#pragma unroll
            for (int u = 0; u < LU; ++u) {
                const int r = r0 + u * blockDim.x;
                v[u] = r < n ? xc[(long long)r * ldx] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < LU; ++u) {
                const int r = r0 + u * blockDim.x;
                if (r < n) {
                    const float hi = d2f_rn(v[u]);
                    Xs[r] = hi;
                    Xl[r] = d2f_rn(v[u] - f2d(hi));
                }
            }
        }
    } else {
        constexpr int LU = 16;
        for (int r0 = threadIdx.x; r0 < n; r0 += LU * blockDim.x) {
            float v[LU];
#pragma unroll
            for (int u = 0; u < LU; ++u) {
                const int r = r0 + u * blockDim.x;
                v[u] = r < n ? col[(long long)r * ld] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < LU; ++u) {
                const int r = r0 + u * blockDim.x;
                if (r < n) Xs[r] = v[u];
            }
        }
    }
    for (int idx = threadIdx.x; idx < 3 * TF; idx += blockDim.x) tab[idx] = DF[idx];
    __syncthreads();
    const int ln = threadIdx.x;
    if (ln < qq) {
        const int base = ln * q;
        eo_line_df<Q>(Xs + base, 1, tab, [&](int i, float h, float l) { Ac[base + i] = make_float2(h, l); });
        if constexpr (X64) eo_line_f32<Q>(Xl + base, 1, tab, [&](int i, float v) { Ac[base + i].y += v; });
    }
    __syncthreads();
    if (ln < qq) {
        const int base = ln % q + qq * (ln / q);
        eo_line_df<Q>(Xs + base, q, tab + TF, [&](int j, float h, float l) {
            float2 a = Ac[base + q * j];
            df_add(a.x, a.y, h, l);
            Ac[base + q * j] = a;
        });
        if constexpr (X64) eo_line_f32<Q>(Xl + base, q, tab + TF, [&](int j, float v) { Ac[base + q * j].y += v; });
    }
    __syncthreads();
    if (ln < qq) {
        const int i = ln % q + 1, j = ln / q + 1;
        int cg = cw, kind = rhs_kind;
        if (kind == RHS_DTN_LOAD) {
            if (cg < 6 * qq) kind = RHS_DTN;
            else { kind = RHS_LOAD; cg -= 6 * qq; }
        }
        if constexpr (X64) eo_line_f32<Q>(Xl + ln, qq, tab + 2 * TF, [&](int k0, float v) { Ac[ln + qq * k0].y += v; });
        eo_line_df<Q>(Xs + ln, qq, tab + 2 * TF, [&](int k0, float h, float l) {
            const int k = k0 + 1, r = ln + qq * k0;
            float2 a = Ac[r];
            df_add(a.x, a.y, h, l);
            const float2 kk = __ldg(kbb + r);
            df_mac1(a.x, a.y, kk.x, kk.y, Xs[r]);
            if constexpr (X64) a.y = fmaf(kk.x, Xl[r], a.y);
            float out;
            if (kind == RHS_DTN) {   // -A_ib e_f: D2[.][0] or D2[.][p-1] next to face node f
                const int f = cg / qq, s2 = cg % qq, u = s2 % q + 1, v = s2 / q + 1;
                const int axis = f >> 1;
                const bool hit = (axis == 0 && j == u && k == v) || (axis == 1 && i == u && k == v) ||
                                 (axis == 2 && i == u && j == v);
                if (hit) {
                    const int row = axis == 0 ? i : (axis == 1 ? j : k);
                    const float4 c = tab[axis * TF + BO + row - 1];
                    if (f & 1) df_add(a.x, a.y, c.z, c.w);
                    else df_add(a.x, a.y, c.x, c.y);
                }
                out = __fadd_rn(a.x, a.y);
            } else {
                double res = f2d(a.x) + f2d(a.y);
                const int gi = i + p * j + p * p * k;
                if (kind == RHS_LOAD) {
                    res += rhs[box * s_rhs + (long long)cg * p * p * p + gi];
                } else {
                    const double* ub = rhs + box * s_rhs + (long long)cg * 6 * qq;
                    const int sx = (j - 1) + q * (k - 1), sy = (i - 1) + q * (k - 1), sz = (i - 1) + q * (j - 1);
                    const float4 cx = tab[BO + i - 1], cy = tab[TF + BO + j - 1], cz = tab[2 * TF + BO + k - 1];
                    res += (f2d(cx.x) + f2d(cx.y)) * ub[sx] + (f2d(cx.z) + f2d(cx.w)) * ub[qq + sx] +
                           (f2d(cy.x) + f2d(cy.y)) * ub[2 * qq + sy] + (f2d(cy.z) + f2d(cy.w)) * ub[3 * qq + sy] +
                           (f2d(cz.x) + f2d(cz.y)) * ub[4 * qq + sz] + (f2d(cz.z) + f2d(cz.w)) * ub[5 * qq + sz];
                }
                out = d2f_rn(res);
            }
            col[(long long)r * ld] = out;
        });
    }
}

// X += D (the FP32 correction) in FP64.  ||D||^2 per box goes to norms[2 box]
// (FP32 partial sums, as for ||X|| in k_extract); with want_xn also ||X||^2
// after the update, in FP64, to norms[2 box + 1].
__global__ void __launch_bounds__(256)
k_ir_update(const float* __restrict__ D, long long ldd, long long sD, int n, int ncols, double* __restrict__ X,
            long long ldx, long long sX, double* norms, const int* skip, int want_xn)
{
    const int box = blockIdx.y;
    if (skip && skip[box]) return;
    float dn = 0.0f;
    double xn = 0.0;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const float* drow = D + box * sD + (long long)r * ldd;
        double* xrow = X + box * sX + (long long)r * ldx;
        for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
            const float d = drow[c];
            const double x = xrow[c] + f2d(d);
            xrow[c] = x;
            dn = fmaf(d, d, dn);
            if (want_xn) xn = fma(x, x, xn);
        }
    }
    block_sum_add(dn, norms + 2 * box);
    if (want_xn) {
        __syncthreads();
        block_sum_add(xn, norms + 2 * box + 1);
    }
}

// Per-box stopping rule of the refinement.  After correction k >= 2
// (relative size rel_k = ||dX_k|| / ||X||) the remaining error is about
// rho * rel_k, with the contraction rho estimated by rel_k / rel_{k-1}; a box
// stops when that prediction, with a factor 10 of margin, plus
// floor_coef * rel_k (the error the correction's own residual may carry, see
// kDfFloor) is below tol, or when the correction has stopped shrinking (less
// than a halving) while already below stag_tol, i.e. X sits at the
// residual's noise floor.  The first correction gives no rate (X0's error and
// the contraction need not match, e.g. for smooth right-hand sides), so it
// ends the refinement only when it is itself below tol.
//
// With dfgate > 0 the check also routes each box's later residuals: at the
// first correction it records whether rel_1 <= dfgate (split[box]: the
// double-float residual is accurate enough for this box, see kDfGate), and
// after every correction it writes the skip flags of the two residual
// kernels, skip_df (boxes done or routed to FP64) and skip_64 (boxes done or
// routed to double-float).
__global__ void k_ir_check(int nbox, double* norms, double tol, double stag_tol, int last, int* skip, int* iters,
                           double* relcorr, int* status, int hold, double floor_coef, double dfgate, int* route,
                           int* skip_df, int* skip_64)
{
    const int box = blockIdx.x * blockDim.x + threadIdx.x;
    if (box >= nbox || skip[box]) return;
    const double dn = norms[2 * box], xn = norms[2 * box + 1];
    const double rel = xn > 0.0 ? sqrt(dn / xn) : sqrt(dn);
    iters[box] += 1;
    const double prev = iters[box] == 1 ? 0.0 : relcorr[box];   // no rate estimate from the first correction
    relcorr[box] = rel;
    norms[2 * box] = 0.0;   // ||X||^2 (from the first solution) is kept
    bool done = false;
    if (prev > 0.0) {
        const double rho = rel / prev;
        done = rel * fmin(1.0, 10.0 * rho) + floor_coef * rel <= tol || (rel <= stag_tol && rho > 0.5);
    } else {
        done = rel <= tol;
    }
    if (hold) done = false;   // this correction came from the double-float residual: one more in FP64
    if (done) skip[box] = 1;
    else if (last && status[box] == 0) status[box] = isfinite(rel) ? HPS_ENOCONV : HPS_EINVAL;
    if (dfgate > 0.0) {
        if (iters[box] == 1) route[box] = rel <= dfgate ? 1 : 0;
        skip_df[box] = done || !route[box];
        skip_64[box] = done || route[box];
    }
}

// out[c][r] = X[r][c] (+ v[c][r]) for the [nrhs][n] output layouts.
__global__ void k_transpose_add(const double* __restrict__ X, long long ldx, long long sX, int n, int ncols,
                                const double* __restrict__ v, double* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    const int box = blockIdx.z;
    if (r >= n) return;
    const long long o = ((long long)box * ncols + c) * n + r;
    double x = X[box * sX + (long long)r * ldx + c];
    if (v) x += v[o];
    out[o] = x;
}

// u_i = v + S u_b with a stored S (one warp per interior row).
__global__ void k_recon_stored(const double* __restrict__ S, int n, int m, int nrhs,
                               const double* __restrict__ v, const double* __restrict__ ub,
                               double* __restrict__ ui)
{
    const int warps = blockDim.x >> 5;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int box = blockIdx.y;
    if (r >= n) return;
    const double* Srow = S + ((long long)box * n + r) * m;
    for (int c = 0; c < nrhs; ++c) {
        const double* u = ub + ((long long)box * nrhs + c) * m;
        double acc = 0.0;
        for (int l = lane; l < m; l += 32) acc += Srow[l] * u[l];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            const long long o = ((long long)box * nrhs + c) * n + r;
            ui[o] = acc + (v ? v[o] : 0.0);
        }
    }
}


// ---------------------------------------------------------------- residual gate

// Seeded Gaussian probe traces phi[box][j][r] (counter-based: splitmix64 of
// (seed, box, j, r), Box-Muller), so any caller can regenerate them.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_probes(long long total, unsigned long long seed, double* __restrict__ phi)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = mix64(seed ^ mix64(2 * (unsigned long long)i));
        const unsigned long long b = mix64(seed ^ mix64(2 * (unsigned long long)i + 1));
        const double u1 = ((a >> 11) + 1) * 0x1.0p-53, u2 = (b >> 11) * 0x1.0p-53;
        phi[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
}

// out[box][j][r] += (A_bb phi)[r]: the face row's own and opposite face node.
__global__ void k_abb_add(int p, int m, int k, const double* __restrict__ D, const double* __restrict__ phi,
                          double* __restrict__ out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, box = blockIdx.z;
    if (r >= m) return;
    const int q = p - 2, qq = q * q;
    const int f = r / qq, s = r - f * qq, axis = f >> 1;
    const int e = (f & 1) ? p - 1 : 0, eo = (f & 1) ? 0 : p - 1;
    const double sg = (f & 1) ? 1.0 : -1.0;
    const double* Da = D + axis * p * p + e * p;
    const double* ph = phi + ((long long)box * k + j) * m;
    out[((long long)box * k + j) * m + r] += sg * (Da[e] * ph[r] + Da[eo] * ph[(f ^ 1) * qq + s]);
}

// tp[box][j][r] = sum_c That[box][r][c] phi[box][j][c]  (one warp per row r)
__global__ void k_apply_probes(int m, int k, const double* __restrict__ That, const double* __restrict__ phi,
                               double* __restrict__ tp)
{
    const int warps = blockDim.x >> 5;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    const int box = blockIdx.y;
    if (r >= m) return;
    const double* row = That + ((long long)box * m + r) * m;
    for (int j = 0; j < k; ++j) {
        const double* ph = phi + ((long long)box * k + j) * m;
        double acc = 0.0;
        for (int c = lane; c < m; c += 32) acc += row[c] * ph[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) tp[((long long)box * k + j) * m + r] = acc;
    }
}

// err = ||T_hat phi - T phi|| / ||T phi|| over the probes; accept when err <= tol
// and the Richardson iteration for T phi has converged (last relative step <= 1e-8).
__global__ void k_gate_decide(int m, int k, const double* __restrict__ tp_hat, const double* __restrict__ tp,
                              const double* __restrict__ norms, double tol, int* __restrict__ accept,
                              double* __restrict__ err)
{
    __shared__ double sd[32], sn[32];
    const int box = blockIdx.x;
    double d = 0.0, nn = 0.0;
    for (int i = threadIdx.x; i < m * k; i += blockDim.x) {
        const double a = tp_hat[(long long)box * m * k + i], b = tp[(long long)box * m * k + i];
        d += (a - b) * (a - b);
        nn += b * b;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, off);
        nn += __shfl_xor_sync(0xffffffffu, nn, off);
    }
    if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = d; sn[threadIdx.x >> 5] = nn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double D2 = 0.0, N2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { D2 += sd[w]; N2 += sn[w]; }
        const double e = N2 > 0.0 ? sqrt(D2 / N2) : INFINITY;
        const double step = norms[2 * box + 1] > 0.0 ? sqrt(norms[2 * box] / norms[2 * box + 1]) : INFINITY;
        err[box] = e;
        accept[box] = (e <= tol && step <= 1e-8) ? 1 : 0;
    }
}

// f[c][grid node of interior node c] = 1: the identity as n loads.
__global__ void k_identity_loads(int p, int n, double* __restrict__ f)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int q = p - 2, i = c % q + 1, j = (c / q) % q + 1, k = c / (q * q) + 1;
    f[(long long)c * p * p * p + i + p * j + p * p * k] = 1.0;
}

// out[r][c] = float(in[c][r]) (n x n)
__global__ void k_transpose_f32(int n, const double* __restrict__ in, float* __restrict__ out)
{
    __shared__ double t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < n && c < n) t[y][threadIdx.x] = in[(long long)r * n + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = bx + y, c = by + threadIdx.x;
        if (r < n && c < n) out[(long long)r * n + c] = float(t[threadIdx.x][y]);
    }
}

__global__ void k_fill_int(int* p, int value, long long count)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = value;
}

}  // namespace

// ---------------------------------------------------------------- launchers

template <typename T>
void launch_build_aug(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b,
                      long long sb, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                      T* M, long long ldm, long long sM, int* status, int zero_row_box, cudaStream_t st,
                      const double* beta)
{
    dim3 grd((unsigned)((g.n + kBuildRows - 1) / kBuildRows), (unsigned)nbox);
    prof_begin(KC_BUILD, st);
    k_build_aug<T><<<grd, 256, 0, st>>>(g.p, g.n, nrhs, (int)ldm, g.dD2, kappa * kappa, kappa_box, b, sb, rhs_kind,
                                        rhs_src, s_rhs, M, ldm, sM, status, zero_row_box, g.dD, beta,
                                        3LL * g.p * g.p * g.p);
    prof_end(KC_BUILD, st, 0.0, (double)nbox * g.n * ldm * sizeof(T));
}

void launch_apply_op(const Geometry& g, double kappa, int nbox, int nfield, const double* b, const double* u,
                     double* out, cudaStream_t st, const double* beta)
{
    const size_t smem = (size_t)g.p * g.p * g.p * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_apply_op, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    dim3 grd((unsigned)nfield, (unsigned)nbox);
    prof_begin(KC_MISC, st);
    k_apply_op<<<grd, 256, smem, st>>>(g.p, nfield, g.dD2, kappa * kappa, b, (long long)g.p * g.p * g.p, u, out,
                                       g.dD, beta);
    prof_end(KC_MISC, st, (double)nbox * nfield * g.n * (6.0 * g.p + 3.0),
             (double)nbox * nfield * g.p * g.p * g.p * 24.0);
}

template <typename T>
void launch_load_rhs(const Geometry& g, int nbox, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                     T* M, long long ldm, long long sM, int* status, cudaStream_t st, const double* beta)
{
    const long long total = (long long)g.n * nrhs;
    dim3 grd((unsigned)std::min<long long>((total + 255) / 256, 256), (unsigned)nbox);
    prof_begin(KC_BUILD, st);
    k_load_rhs<T><<<grd, 256, 0, st>>>(g.p, g.n, nrhs, g.dD2, rhs_kind, rhs_src, s_rhs, M, ldm, sM, status, g.dD,
                                       beta);
    prof_end(KC_BUILD, st, 0.0, (double)nbox * total * (8.0 + sizeof(T)));
}

template <typename T>
void launch_panel(T* M, long long ldm, long long sM, int n, int k, int nb, int ib,
                  int* perm, long long sP, T* Ftop, long long ldf, long long sF,
                  T* Btop, long long ldb, long long sB, int* status, const int* skip,
                  int nbox, cudaStream_t st)
{
    static size_t dyn_max = 0;
    if (!dyn_max) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_panel<T>);
        dyn_max = 227 * 1024 - fa.sharedSizeBytes;
        cudaFuncSetAttribute(k_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    }
    // Widest inner block (<= 32 columns, power of two) whose rows fit in what
    // is left of shared memory; the panel shrinks as k grows, so later steps
    // take wider blocks.  The plan's ib is the width of the first step.
    const size_t R0 = (size_t)(n - k);
    ib = 32;
    while (ib > 1 && (size_t)ib * R0 * sizeof(T) + R0 * 5 > dyn_max) ib >>= 1;
    if (ib > nb) ib = nb;
    const size_t s1 = (size_t)ib * R0 * sizeof(T) + R0 * 5;
    int Pd = 16;
    while (Pd < nb) Pd *= 2;
    const size_t s2 = (size_t)2 * Pd * Pd * sizeof(T);   // the padded triangle and its inverse
    const size_t smem = s1 > s2 ? s1 : s2;
    prof_begin(KC_PANEL, st);
    k_panel<T><<<nbox, kPanelThreads, smem, st>>>(M, ldm, sM, n, k, nb, ib, perm, sP, Ftop, ldf, sF,
                                                  Btop, ldb, sB, status, skip);
    prof_end(KC_PANEL, st, (double)nbox * (n - k) * (double)nb * nb, (double)nbox * 2.0 * (n - k) * nb * sizeof(T));
}

template <typename T>
void launch_gather(const T* M, long long ldm, long long sM, int k, int nb, int c0, int ncols,
                   const int* perm, long long sP, T* W, T* G, long long ldg, long long sG,
                   const int* skip, int nbox, cudaStream_t st)
{
    dim3 grd((unsigned)((ncols + 127) / 128), (unsigned)nb, (unsigned)nbox);
    prof_begin(KC_GATHER, st);
    k_gather<T><<<grd, 128, 0, st>>>(M, ldm, sM, k, nb, c0, ncols, perm, sP, W, G, ldg, sG, skip);
    prof_end(KC_GATHER, st, 0.0, (double)nbox * nb * (double)ncols * sizeof(T) * (W ? 3 : 2));
}

template <>
void launch_gemm<double>(const GemmArgs<double>& a, int nbox, cudaStream_t st)
{
    constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
    dim3 grd((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM), (unsigned)nbox);
    if (a.M <= 0 || a.N <= 0) return;
    prof_begin(KC_UPDATE_CUDACORE, st);
    k_gemm<double, BM, BN, BK, TM, TN><<<grd, (BM / TM) * (BN / TN), 0, st>>>(a);
    prof_end(KC_UPDATE_CUDACORE, st, 2.0 * nbox * a.M * (double)a.N * a.K, (double)nbox * ((double)a.M * a.K + (double)a.K * a.N + 2.0 * a.M * a.N) * 8);
}

template <>
void launch_gemm<float>(const GemmArgs<float>& a, int nbox, cudaStream_t st)
{
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 grd((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM), (unsigned)nbox);
    if (a.M <= 0 || a.N <= 0) return;
    prof_begin(KC_UPDATE_CUDACORE, st);
    k_gemm<float, BM, BN, BK, TM, TN><<<grd, (BM / TM) * (BN / TN), 0, st>>>(a);
    prof_end(KC_UPDATE_CUDACORE, st, 2.0 * nbox * a.M * (double)a.N * a.K, (double)nbox * ((double)a.M * a.K + (double)a.K * a.N + 2.0 * a.M * a.N) * 4);
}

void launch_dn(const Geometry& g, int nbox, const double* X, long long ldx, long long sX,
               int ncols, double* out, long long sOut, int transposed_out, int add_abb,
               cudaStream_t st)
{
    dim3 grd((unsigned)((ncols + 127) / 128), (unsigned)(g.m / 2), (unsigned)nbox);
    prof_begin(KC_DN, st);
    k_dn<<<grd, 128, 0, st>>>(g.p, g.n, g.m, ncols, g.dD, X, ldx, sX, out, sOut, transposed_out, add_abb);
    prof_end(KC_DN, st, 2.0 * nbox * g.m * (double)ncols * g.q, (double)nbox * ((double)g.n + g.m) * ncols * 8);
}

template <typename TS>
void launch_extract(const TS* src, long long lds, long long sS, int n, int ncols,
                    double* X, long long ldx, long long sX, int nbox, cudaStream_t st, double* xnorm)
{
    dim3 grd((unsigned)std::min(n, 96), (unsigned)nbox);
    prof_begin(KC_REFINE, st);
    k_extract<TS><<<grd, 256, 0, st>>>(src, lds, sS, n, ncols, X, ldx, sX, xnorm);
    prof_end(KC_REFINE, st, 0.0, (double)nbox * n * (double)ncols * (sizeof(TS) + 8));
}

// kb[box][r] = kappa^2 b at interior node r (the residual's diagonal term,
// the same for every column of a box).
__global__ void k_kappa_b(int p, int n, const double* __restrict__ b, long long sb, double kappa2,
                          const double* __restrict__ kappa_box, double* __restrict__ kb, float2* __restrict__ kbs)
{
    const int box = blockIdx.y;
    const int q = p - 2, qq = q * q, pp = p * p;
    const double k2 = kappa_box ? kappa_box[box] * kappa_box[box] : kappa2;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int i = r % q + 1, j = (r / q) % q + 1, k = r / qq + 1;
        const double v = k2 * b[box * sb + i + p * j + pp * k];
        kb[(long long)box * n + r] = v;
        if (kbs) {
            const float hi = __double2float_rn(v);
            kbs[(long long)box * n + r] = make_float2(hi, __double2float_rn(v - (double)hi));
        }
    }
}

// Self-test of d2f_rn and f2d against the hardware conversions over n
// values: splitmix64 bit patterns (all exponents), values near the float
// range limits and rounding ties.  mism[0] counts double -> float
// mismatches, mism[1] float -> double (bitwise; NaN against NaN).
__global__ void k_selftest_conv(long long n, unsigned long long seed, unsigned long long* mism)
{
    unsigned long long bad_d = 0, bad_f = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        unsigned long long bits = z;
        const int kind = (int)(i & 7);
        if (kind == 1) bits = (z & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(1023 + (int)((z >> 52) % 40) - 20) << 52);
        if (kind == 2) bits = (z & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(896 + (int)((z >> 52) % 4)) << 52);
        if (kind == 3) bits = (z & 0x800FFFFFFFFFFFFFull) | ((unsigned long long)(1148 + (int)((z >> 52) % 4)) << 52);
        if (kind == 4) bits = (z & 0xFFFFFFFFE0000000ull) | 0x10000000ull;   // exact ties at the 23-bit boundary
        if (kind == 5) bits = (z & 0xFFFFFFFFE0000000ull) | 0x0FFFFFFFull;
        const double x = __longlong_as_double((long long)bits);
        const float a = d2f_rn(x), b = __double2float_rn(x);
        if (!((a != a && b != b) || __float_as_uint(a) == __float_as_uint(b))) ++bad_d;
        const float y = __uint_as_float((unsigned)(z >> 7));
        const double c = f2d(y), d = (double)y;
        if (!((c != c && d != d) || __double_as_longlong(c) == __double_as_longlong(d))) ++bad_f;
    }
    if (bad_d) atomicAdd(mism, bad_d);
    if (bad_f) atomicAdd(mism + 1, bad_f);
}

void selftest_conversions(long long n, unsigned long long seed, unsigned long long* mism_dev, cudaStream_t st)
{
    k_selftest_conv<<<1024, 256, 0, st>>>(n, seed, mism_dev);
}

void launch_kappa_b(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b, long long sb,
                    double* kb, float2* kbs, cudaStream_t st)
{
    dim3 grd((unsigned)((g.n + 255) / 256), (unsigned)nbox);
    prof_begin(KC_MISC, st);
    k_kappa_b<<<grd, 256, 0, st>>>(g.p, g.n, b, sb, kappa * kappa, kappa_box, kb, kbs);
    prof_end(KC_MISC, st, 0.0, (double)nbox * g.n * 24.0);
}

namespace {
template <int Q, bool CONV>
void residual_q(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b, long long sb,
                int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs, const double* X, long long ldx,
                long long sX, float* R, long long ldr, long long sR, const int* skip, cudaStream_t st,
                const double* kb, const double* beta)
{
    const size_t tables = (size_t)((3 * g.p * g.p + 1) & ~1) + 3 * eo_tab_size<Q>() + (CONV ? 3 * g.p * g.p : 0);
    const size_t smem = ((size_t)2 * g.n + tables) * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_residual<Q, CONV>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    dim3 grd((unsigned)nrhs, (unsigned)nbox);
    // FP64 operations per entry: three line passes (butterfly 1, pairs h + 1
    // (odd q: + 1 for the middle column), accumulate 1) and the finish (3);
    // the first-order term adds q + 1 per line pass.
    const double per = 3.0 * (2.0 + 2.0 * (Q / 2) + ((Q & 1) ? 2.0 : 0.0)) + 3.0 + (CONV ? 3.0 * (Q + 1) : 0.0);
    prof_begin(KC_RESIDUAL, st);
    k_residual<Q, CONV><<<grd, res_threads<Q>(), smem, st>>>(g.p, g.n, nrhs, g.dD2, kappa * kappa, kappa_box, b, sb,
                                                              rhs_kind, rhs_src, s_rhs, X, ldx, sX, R, ldr, sR, skip,
                                                              kb, g.dD, beta);
    prof_end(KC_RESIDUAL, st, (double)nbox * g.n * (double)nrhs * per, (double)nbox * g.n * (double)nrhs * 12.0);
}
}  // namespace

void launch_residual(const Geometry& g, double kappa, const double* kappa_box, int nbox, const double* b, long long sb,
                     int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                     const double* X, long long ldx, long long sX,
                     float* R, long long ldr, long long sR, const int* skip, cudaStream_t st, const double* kb,
                     const double* beta)
{
    static_assert(kMaxP - 2 == 22, "one residual instantiation per interior line length");
#define HPS_RES_CASE(QV)                                                                                         \
    case QV:                                                                                                     \
        if (beta)                                                                                                \
            residual_q<QV, true>(g, kappa, kappa_box, nbox, b, sb, rhs_kind, nrhs, rhs_src, s_rhs, X, ldx, sX, R, \
                                 ldr, sR, skip, st, kb, beta);                                                   \
        else                                                                                                     \
            residual_q<QV, false>(g, kappa, kappa_box, nbox, b, sb, rhs_kind, nrhs, rhs_src, s_rhs, X, ldx, sX,   \
                                  R, ldr, sR, skip, st, kb, nullptr);                                            \
        break;
    switch (g.q) {
        HPS_RES_CASE(1) HPS_RES_CASE(2) HPS_RES_CASE(3) HPS_RES_CASE(4) HPS_RES_CASE(5) HPS_RES_CASE(6)
        HPS_RES_CASE(7) HPS_RES_CASE(8) HPS_RES_CASE(9) HPS_RES_CASE(10) HPS_RES_CASE(11) HPS_RES_CASE(12)
        HPS_RES_CASE(13) HPS_RES_CASE(14) HPS_RES_CASE(15) HPS_RES_CASE(16) HPS_RES_CASE(17) HPS_RES_CASE(18)
        HPS_RES_CASE(19) HPS_RES_CASE(20) HPS_RES_CASE(21) HPS_RES_CASE(22)
        default: break;
    }
#undef HPS_RES_CASE
}

namespace {
template <int Q>
void residual_df_q(const Geometry& g, int nbox, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                   float* X0R, long long ld, long long sbx, const float2* kbs, const int* skip, cudaStream_t st,
                   const double* X64, long long ldx, long long sX64)
{
    const size_t smem = (size_t)3 * df_tab_q<Q>() * sizeof(float4) +
                        (size_t)g.n * (sizeof(float2) + (X64 ? 2 : 1) * sizeof(float));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_residual_df<Q, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        cudaFuncSetAttribute(k_residual_df<Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    dim3 grd((unsigned)nrhs, (unsigned)nbox);
    prof_begin(X64 ? KC_RESIDUAL_DF64 : KC_RESIDUAL_DF, st);
    if (X64)
        k_residual_df<Q, true><<<grd, res_threads<Q>(), smem, st>>>(g.p, g.n, reinterpret_cast<const float4*>(g.dDF),
                                                                     kbs, rhs_kind, rhs_src, s_rhs, X0R, ld, sbx, skip,
                                                                     X64, ldx, sX64);
    else
        k_residual_df<Q, false><<<grd, res_threads<Q>(), smem, st>>>(g.p, g.n, reinterpret_cast<const float4*>(g.dDF),
                                                                      kbs, rhs_kind, rhs_src, s_rhs, X0R, ld, sbx,
                                                                      skip, nullptr, 0, 0);
    // work counted as for the FP64 residual (its operations per entry); bytes:
    // X (FP32, or FP64 for X64) and R in FP32, the split kappa^2 b
    const double per = 3.0 * (2.0 + 2.0 * (Q / 2) + ((Q & 1) ? 2.0 : 0.0)) + 3.0;
    prof_end(X64 ? KC_RESIDUAL_DF64 : KC_RESIDUAL_DF, st, (double)nbox * g.n * (double)nrhs * per,
             (double)nbox * g.n * (double)nrhs * (X64 ? 12.0 : 8.0));
}
}  // namespace

bool residual_df_fits(const Geometry& g, bool x64)
{
    const size_t smem = (size_t)3 * df_tab_f4(g.q) * sizeof(float4) +
                        (size_t)g.n * (sizeof(float2) + (x64 ? 2 : 1) * sizeof(float));
    return smem <= 227 * 1024;
}

void launch_residual_df(const Geometry& g, int nbox, int rhs_kind, int nrhs, const double* rhs_src, long long s_rhs,
                        float* X0R, long long ld, long long sbx, const float2* kbs, const int* skip, cudaStream_t st,
                        const double* X64, long long ldx, long long sX64)
{
#define HPS_RES_CASE(QV)                                                                                          \
    case QV:                                                                                                      \
        residual_df_q<QV>(g, nbox, rhs_kind, nrhs, rhs_src, s_rhs, X0R, ld, sbx, kbs, skip, st, X64, ldx, sX64); \
        break;
    switch (g.q) {
        HPS_RES_CASE(1) HPS_RES_CASE(2) HPS_RES_CASE(3) HPS_RES_CASE(4) HPS_RES_CASE(5) HPS_RES_CASE(6)
        HPS_RES_CASE(7) HPS_RES_CASE(8) HPS_RES_CASE(9) HPS_RES_CASE(10) HPS_RES_CASE(11) HPS_RES_CASE(12)
        HPS_RES_CASE(13) HPS_RES_CASE(14) HPS_RES_CASE(15) HPS_RES_CASE(16) HPS_RES_CASE(17) HPS_RES_CASE(18)
        HPS_RES_CASE(19) HPS_RES_CASE(20) HPS_RES_CASE(21) HPS_RES_CASE(22)
        default: break;
    }
#undef HPS_RES_CASE
}

void launch_ir_update(const float* D, long long ldd, long long sD, int n, int ncols,
                      double* X, long long ldx, long long sX, double* norms,
                      const int* skip, int nbox, cudaStream_t st, bool want_xn)
{
    dim3 grd((unsigned)std::min(n, 96), (unsigned)nbox);
    prof_begin(KC_REFINE, st);
    k_ir_update<<<grd, 256, 0, st>>>(D, ldd, sD, n, ncols, X, ldx, sX, norms, skip, want_xn ? 1 : 0);
    prof_end(KC_REFINE, st, 0.0, (double)nbox * n * (double)ncols * 20.0);
}

void launch_ir_check(int nbox, double* norms, double tol, int last, int* skip,
                     int* iters, double* relcorr, int* status, cudaStream_t st, bool hold, double floor_coef,
                     double dfgate, int* route, int* skip_df, int* skip_64)
{
    prof_begin(KC_MISC, st);
    k_ir_check<<<(nbox + 127) / 128, 128, 0, st>>>(nbox, norms, tol, 1e-11, last, skip, iters, relcorr, status,
                                                    hold ? 1 : 0, floor_coef, dfgate, route, skip_df, skip_64);
    prof_end(KC_MISC, st, 0.0, (double)nbox * 40.0);
}

void launch_transpose_add(const double* X, long long ldx, long long sX, int n, int ncols,
                          const double* v, double* out, int nbox, cudaStream_t st)
{
    dim3 grd((unsigned)((n + 127) / 128), (unsigned)ncols, (unsigned)nbox);
    prof_begin(KC_MISC, st);
    k_transpose_add<<<grd, 128, 0, st>>>(X, ldx, sX, n, ncols, v, out);
    prof_end(KC_MISC, st, 0.0, (double)nbox * n * (double)ncols * (v ? 24.0 : 16.0));
}

void launch_recon_stored(const double* S, int n, int m, int nrhs, const double* v,
                         const double* ub, double* ui, int nbox, cudaStream_t st)
{
    dim3 grd((unsigned)((n + 7) / 8), (unsigned)nbox);
    prof_begin(KC_MISC, st);
    k_recon_stored<<<grd, 256, 0, st>>>(S, n, m, nrhs, v, ub, ui);
    prof_end(KC_MISC, st, 2.0 * nbox * n * (double)m * nrhs, (double)nbox * n * (double)m * 8.0);
}


void launch_probes(long long total, unsigned long long seed, double* phi, cudaStream_t st)
{
    k_probes<<<(int)std::min<long long>((total + 255) / 256, 4096), 256, 0, st>>>(total, seed, phi);
}

void launch_abb_add(const Geometry& g, int nbox, int k, const double* phi, double* out, cudaStream_t st)
{
    dim3 grd((unsigned)((g.m + 127) / 128), (unsigned)k, (unsigned)nbox);
    k_abb_add<<<grd, 128, 0, st>>>(g.p, g.m, k, g.dD, phi, out);
}

void launch_apply_probes(int m, int k, int nbox, const double* That, const double* phi, double* tp, cudaStream_t st)
{
    dim3 grd((unsigned)((m + 7) / 8), (unsigned)nbox);
    k_apply_probes<<<grd, 256, 0, st>>>(m, k, That, phi, tp);
}

void launch_gate_decide(int m, int k, int nbox, const double* tp_hat, const double* tp, const double* norms,
                        double tol, int* accept, double* err, cudaStream_t st)
{
    k_gate_decide<<<nbox, 256, 0, st>>>(m, k, tp_hat, tp, norms, tol, accept, err);
}

void launch_identity_loads(int p, int n, double* f, cudaStream_t st)
{
    k_identity_loads<<<(n + 255) / 256, 256, 0, st>>>(p, n, f);
}

void launch_transpose_f32(int n, const double* in, float* out, cudaStream_t st)
{
    dim3 grd((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32));
    k_transpose_f32<<<grd, dim3(32, 8), 0, st>>>(n, in, out);
}

void launch_fill_int(int* p, int value, long long count, cudaStream_t st)
{
    if (count <= 0) return;
    int blocks = (int)((count + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_fill_int<<<blocks, 256, 0, st>>>(p, value, count);
}

template void launch_build_aug<float>(const Geometry&, double, const double*, int, const double*, long long, int,
                                      int, const double*, long long, float*, long long, long long, int*, int,
                                      cudaStream_t, const double*);
template void launch_build_aug<double>(const Geometry&, double, const double*, int, const double*, long long, int,
                                       int, const double*, long long, double*, long long, long long, int*, int,
                                       cudaStream_t, const double*);
template void launch_load_rhs<float>(const Geometry&, int, int, int, const double*, long long, float*, long long,
                                     long long, int*, cudaStream_t, const double*);
template void launch_load_rhs<double>(const Geometry&, int, int, int, const double*, long long, double*, long long,
                                      long long, int*, cudaStream_t, const double*);
template void launch_panel<float>(float*, long long, long long, int, int, int, int, int*, long long, float*,
                                  long long, long long, float*, long long, long long, int*, const int*, int,
                                  cudaStream_t);
template void launch_panel<double>(double*, long long, long long, int, int, int, int, int*, long long, double*,
                                   long long, long long, double*, long long, long long, int*, const int*, int,
                                   cudaStream_t);
template void launch_gather<float>(const float*, long long, long long, int, int, int, int, const int*, long long,
                                   float*, float*, long long, long long, const int*, int, cudaStream_t);
template void launch_gather<double>(const double*, long long, long long, int, int, int, int, const int*,
                                    long long, double*, double*, long long, long long, const int*, int,
                                    cudaStream_t);
template void launch_extract<float>(const float*, long long, long long, int, int, double*, long long, long long,
                                    int, cudaStream_t, double*);
template void launch_extract<double>(const double*, long long, long long, int, int, double*, long long,
                                     long long, int, cudaStream_t, double*);

}  // namespace hps
