// Leaf impedance-to-impedance (ItI) maps, FP64.
//
// The two-level scheme adapts to HPS built on ItI maps (Sec. 6); on this
// library's leaf collocation (Sec. 2.1: interior and face nodes, Eq. 2's
// rows) the ItI map R of a box takes impedance data f = du/dn + i eta u on the
// face nodes to g = du/dn - i eta u for the solution of the homogeneous
// equation in the box:
//
//     [ A_ii   A_ib           ] [u_i]   [0]
//     [ A_bi   A_bb + i eta I ] [u_b] = [f],     R f = f - 2 i eta u_b.
//
// The system never needs A_ii alone, so R exists where kappa^2 is a
// Dirichlet eigenvalue of the box (where T = A_bb - A_bi A_ii^{-1} A_ib does
// not).  It is complex; each box's system is factored in its real form
//
//     [ A   -eta E ] [x_r]   [F]
//     [ eta E   A  ] [x_i] = [0],      E = diag(0_n, I_m),  F = [0; I_m],
//
// (size 2N, N = n + m, m real right-hand sides: the unit impedance data) by
// the library's batched FP64 LU with partial pivoting, and
// R = I - 2 i eta (x_r + i x_i)_b, i.e. Re R = I + 2 eta x_i,b and
// Im R = -2 eta x_r,b.
#include <algorithm>
#include <cmath>

#include "hps_internal.h"

namespace {

constexpr int kItiMaxP = 16;
constexpr int kItiRows = 4;   // rows per CTA of the build

// The reference Chebyshev matrix and the box size by value: the D and D2
// tables are formed on the device (the helper of the context path), so the
// call makes no host-to-device copy and stays stream-ordered.
struct ItiTables {
    int p;
    double h[3];
    double Dhat[kItiMaxP * kItiMaxP];
};

__global__ void k_iti_tables(const ItiTables a, double* D, double* D2)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) hps::geometry_tables(a.p, a.Dhat, a.h, D, D2);
}

// Writes rows [r0, r0 + kItiRows) of box blockIdx.y's augmented real system
// [K | F] (2N x (2N + m), row pitch ldm).  Row layout of each half: the n
// interior rows (Eq. 2: -sum D2 along the three grid lines - kappa^2 b), then
// the m face rows (outward normal derivative along the face's axis); the
// columns of a half are the n interior then m face unknowns.  D and D2 are
// [3][p][p] (axis-major), b [nbox][p^3].
__global__ void __launch_bounds__(256)
k_build_iti(int p, int n, int m, const double* __restrict__ D, const double* __restrict__ D2, double kappa2,
            double eta, const double* __restrict__ b, int nrhs, const double* __restrict__ f, double* __restrict__ M,
            long long ldm, long long sM, int* status)
{
    const int box = blockIdx.y;
    const int N = n + m, N2 = 2 * N;
    const int r0 = blockIdx.x * kItiRows;
    const int rows = min(kItiRows, N2 - r0);
    double* Mb = M + box * sM + (long long)r0 * ldm;
    {
        const int nv = (int)(ldm / 2);
        double2* Mv = reinterpret_cast<double2*>(Mb);
        for (int idx = threadIdx.x; idx < rows * nv; idx += blockDim.x) {
            const int rr = idx / nv, cv = idx - rr * nv;
            Mv[(long long)rr * nv + cv] = make_double2(0.0, 0.0);
        }
    }
    __syncthreads();
    const int q = p - 2, qq = q * q, pp = p * p;
    // column of grid node (i, j, k) (interior or face, never an edge) within a half
    auto col = [&](int i, int j, int k) -> int {
        if (i >= 1 && i <= q && j >= 1 && j <= q && k >= 1 && k <= q) return (i - 1) + q * (j - 1) + qq * (k - 1);
        int f, a, c;
        if (i == 0 || i == p - 1) { f = i ? 1 : 0; a = j; c = k; }
        else if (j == 0 || j == p - 1) { f = j ? 3 : 2; a = i; c = k; }
        else { f = k ? 5 : 4; a = i; c = j; }
        return n + f * qq + (a - 1) + q * (c - 1);
    };
    for (int rr = 0; rr < rows; ++rr) {
        const int R = r0 + rr, half = R / N, lr = R - half * N, off = half * N;
        double* row = Mb + (long long)rr * ldm;
        if (lr < n) {
            const int i = lr % q + 1, j = (lr / q) % q + 1, k = lr / qq + 1;
            // the three grid lines through (i, j, k): p entries each, the
            // diagonal shared
            for (int e = threadIdx.x; e < 3 * p; e += blockDim.x) {
                const int a = e / p, l = e - a * p;
                int ii = i, jj = j, kk = k, own;
                if (a == 0) { ii = l; own = i; }
                else if (a == 1) { jj = l; own = j; }
                else { kk = l; own = k; }
                if (l == own && a > 0) continue;   // the diagonal is written once, by the x line
                double v = -__ldg(D2 + a * pp + own * p + l);
                if (l == own) {
                    v -= __ldg(D2 + pp + j * p + j) + __ldg(D2 + 2 * pp + k * p + k);
                    const double bv = __ldg(b + (long long)box * p * pp + i + p * j + pp * k);
                    if (!isfinite(bv)) status[box] = HPS_EINVAL;
                    v -= kappa2 * bv;
                }
                row[off + col(ii, jj, kk)] = v;
            }
            if (half == 0) {   // the loads' interior values: right-hand sides m .. m + nrhs - 1
                const long long gi = i + p * j + (long long)pp * k;
                for (int c = threadIdx.x; c < nrhs; c += blockDim.x) {
                    const double fv = __ldg(f + ((long long)box * nrhs + c) * p * pp + gi);
                    if (!isfinite(fv)) status[box] = HPS_EINVAL;
                    row[N2 + m + c] = fv;
                }
            }
        } else {
            const int r = lr - n, f = r / qq, s = r - f * qq, axis = f >> 1;
            const int a = s % q + 1, c = s / q + 1, e = (f & 1) ? p - 1 : 0;
            const double sg = (f & 1) ? 1.0 : -1.0;
            for (int l = threadIdx.x; l < p; l += blockDim.x) {
                int ii, jj, kk;
                if (axis == 0) { ii = l; jj = a; kk = c; }
                else if (axis == 1) { ii = a; jj = l; kk = c; }
                else { ii = a; jj = c; kk = l; }
                row[off + col(ii, jj, kk)] = sg * __ldg(D + axis * pp + e * p + l);
            }
            if (threadIdx.x == 0) {
                // the impedance coupling between the halves, and F
                if (half == 0) {
                    row[N + n + r] = -eta;
                    row[N2 + r] = 1.0;
                } else {
                    row[n + r] = eta;
                }
            }
        }
    }
}

// R[box][r][c] = (delta_rc + 2 eta x_i[n + r][c], -2 eta x_r[n + r][c]) from
// the solved right-hand-side columns (interleaved real and imaginary parts).
__global__ void k_extract_iti(int n, int m, const double* __restrict__ M, long long ldm, long long sM, double eta,
                              double* __restrict__ R)
{
    const int box = blockIdx.y;
    const int N = n + m;
    const long long mm = (long long)m * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < mm; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / m), c = (int)(e - (long long)r * m);
        const double* X = M + box * sM + 2 * N;
        const double xr = X[(long long)(n + r) * ldm + c], xi = X[(long long)(N + n + r) * ldm + c];
        double* o = R + 2 * (box * mm + e);
        o[0] = (r == c ? 1.0 : 0.0) + 2.0 * eta * xi;
        o[1] = -2.0 * eta * xr;
    }
}

// S[box][i][c] = x_r[i][c] + i x_i[i][c] (interior rows, unit impedance data).
__global__ void k_extract_iti_s(int n, int m, const double* __restrict__ M, long long ldm, long long sM,
                                double* __restrict__ S)
{
    const int box = blockIdx.y;
    const int N = n + m;
    const long long nm = (long long)n * m;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nm; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / m), c = (int)(e - (long long)i * m);
        const double* X = M + box * sM + 2 * N;
        double* o = S + 2 * (box * nm + e);
        o[0] = X[(long long)i * ldm + c];
        o[1] = X[(long long)(N + i) * ldm + c];
    }
}

// Loads: v[box][c][i] = x[i][m + c] (interior) and hout[box][c][r] =
// -2 i eta x[n + r][m + c] (the outgoing impedance with zero incoming data).
__global__ void k_extract_iti_loads(int n, int m, int nrhs, const double* __restrict__ M, long long ldm, long long sM,
                                    double eta, double* __restrict__ v, double* __restrict__ hout)
{
    const int box = blockIdx.y;
    const int N = n + m;
    const long long tot = (long long)nrhs * (n + m);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / (n + m)), r = (int)(e - (long long)c * (n + m));
        const double* X = M + box * sM + 2 * N + m + c;
        const double xr = X[(long long)r * ldm], xi = X[(long long)(N + r) * ldm];
        if (r < n) {
            if (v) {
                double* o = v + 2 * (((long long)box * nrhs + c) * n + r);
                o[0] = xr;
                o[1] = xi;
            }
        } else if (hout) {
            double* o = hout + 2 * (((long long)box * nrhs + c) * m + (r - n));
            o[0] = 2.0 * eta * xi;
            o[1] = -2.0 * eta * xr;
        }
    }
}

// Box solution from incoming impedance data fin [box][c][m] (complex): the
// interior u_i = S fin + v and the face values u_b = (fin - g) / (2 i eta),
// g = R fin + hout.  One CTA per (row block, load, box); rows 0..n-1 interior,
// n..n+m-1 face (complex arithmetic written out on (re, im) pairs).
__global__ void __launch_bounds__(256)
k_iti_reconstruct(int n, int m, int nrhs, double eta, const double* __restrict__ R, const double* __restrict__ S,
                  const double* __restrict__ v, const double* __restrict__ hout, const double* __restrict__ fin,
                  double* __restrict__ ui, double* __restrict__ ub)
{
    const int c = blockIdx.y, box = blockIdx.z;
    const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * warps + (threadIdx.x >> 5);
    if (row >= n + m) return;
    const bool face = row >= n;
    if (face ? !ub : !ui) return;
    const int r = face ? row - n : row;
    const double* A = face ? R + 2 * (((long long)box * m + r) * m) : S + 2 * (((long long)box * n + r) * m);
    const double* x = fin + 2 * (((long long)box * nrhs + c) * m);
    double ar = 0.0, ai = 0.0;
    for (int l = lane; l < m; l += 32) {
        const double a0 = A[2 * l], a1 = A[2 * l + 1], x0 = x[2 * l], x1 = x[2 * l + 1];
        ar = fma(a0, x0, fma(-a1, x1, ar));
        ai = fma(a0, x1, fma(a1, x0, ai));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, off);
        ai += __shfl_xor_sync(0xffffffffu, ai, off);
    }
    if (lane != 0) return;
    if (!face) {
        double* o = ui + 2 * (((long long)box * nrhs + c) * n + r);
        const double* vv = v ? v + 2 * (((long long)box * nrhs + c) * n + r) : nullptr;
        o[0] = ar + (vv ? vv[0] : 0.0);
        o[1] = ai + (vv ? vv[1] : 0.0);
    } else {
        // g = R fin + hout; u_b = (fin - g) / (2 i eta) = -i (fin - g) / (2 eta)
        const double* hh = hout ? hout + 2 * (((long long)box * nrhs + c) * m + r) : nullptr;
        const double gr = ar + (hh ? hh[0] : 0.0), gim = ai + (hh ? hh[1] : 0.0);
        const double dr = x[2 * r] - gr, di = x[2 * r + 1] - gim;
        double* o = ub + 2 * (((long long)box * nrhs + c) * m + r);
        o[0] = di / (2.0 * eta);
        o[1] = -dr / (2.0 * eta);
    }
}

}  // namespace

extern "C" {

hps_status hps_leaf_iti_solve(const hps_leaf_kind* kind, double eta, int nbox, const double* b, int nrhs,
                              const double* f, double* R, double* S, double* v, double* hout, int* box_status,
                              void* stream)
{
    if (!kind || kind->p < 4 || kind->p > kItiMaxP || !std::isfinite(kind->kappa) || !std::isfinite(eta) ||
        !(eta != 0.0) || nbox < 0 || nrhs < 0 || nrhs > 256 || kind->beta)
        return HPS_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(kind->h[a] > 0.0) || !std::isfinite(kind->h[a])) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || (!R && !S && nrhs == 0) || (nrhs > 0 && (!f || (!v && !hout)))) return HPS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int p = kind->p, q = p - 2, n = q * q * q, m = 6 * q * q, N2 = 2 * (n + m), pp = p * p;
    ItiTables ta;
    ta.p = p;
    for (int a = 0; a < 3; ++a) ta.h[a] = kind->h[a];
    hps::cheb_diff(p, ta.Dhat);
    hps::Plan PL = hps::make_plan(N2, m + nrhs, HPS_FP64, 0, false, false);
    const size_t tab_bytes = hps::align_up(sizeof(double) * 6 * pp, 256);
    const size_t st_bytes = hps::align_up(sizeof(int) * (size_t)nbox, 256);
    const size_t bytes = tab_bytes + st_bytes + PL.per_box * (size_t)nbox;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, bytes, st) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
    char* base = static_cast<char*>(ws);
    double* dtab = reinterpret_cast<double*>(base);
    int* status = box_status ? box_status : reinterpret_cast<int*>(base + tab_bytes);
    hps::Work<double> w = hps::carve<double>(PL, base + tab_bytes + st_bytes, nbox);
    hps_status rc = HPS_OK;
    k_iti_tables<<<1, 1, 0, st>>>(ta, dtab, dtab + 3 * pp);
    if (cudaMemsetAsync(status, 0, sizeof(int) * (size_t)nbox, st) != cudaSuccess) rc = HPS_ECUDA;
    if (rc == HPS_OK) {
        k_build_iti<<<dim3((unsigned)((N2 + kItiRows - 1) / kItiRows), (unsigned)nbox), 256, 0, st>>>(
            p, n, m, dtab, dtab + 3 * pp, kind->kappa * kind->kappa, eta, b, nrhs, f, w.M, PL.ldm, w.sM, status);
        hps::lu_factor<double>(PL, w, nbox, status, st);
        hps::lu_backward<double>(PL, w, nbox, N2, m + nrhs, nullptr, st);
        const long long mm = (long long)m * m, nm = (long long)n * m;
        if (R)
            k_extract_iti<<<dim3((unsigned)std::min<long long>((mm + 255) / 256, 1024), (unsigned)nbox), 256, 0, st>>>(
                n, m, w.M, PL.ldm, w.sM, eta, R);
        if (S)
            k_extract_iti_s<<<dim3((unsigned)std::min<long long>((nm + 255) / 256, 1024), (unsigned)nbox), 256, 0,
                              st>>>(n, m, w.M, PL.ldm, w.sM, S);
        if (nrhs > 0) {
            const long long tot = (long long)nrhs * (n + m);
            k_extract_iti_loads<<<dim3((unsigned)std::min<long long>((tot + 255) / 256, 1024), (unsigned)nbox), 256, 0,
                                  st>>>(n, m, nrhs, w.M, PL.ldm, w.sM, eta, v, hout);
        }
        if (cudaGetLastError() != cudaSuccess) rc = HPS_ECUDA;
    }
    if (cudaFreeAsync(ws, st) != cudaSuccess && rc == HPS_OK) rc = HPS_ECUDA;
    return rc;
}

hps_status hps_leaf_iti(const hps_leaf_kind* kind, double eta, int nbox, const double* b, double* R, int* box_status,
                        void* stream)
{
    if (!R && nbox > 0) return HPS_EINVAL;
    return hps_leaf_iti_solve(kind, eta, nbox, b, 0, nullptr, R, nullptr, nullptr, nullptr, box_status, stream);
}

hps_status hps_leaf_iti_reconstruct(int p, double eta, int nbox, int nrhs, const double* R, const double* S,
                                    const double* v, const double* hout, const double* fin, double* ui, double* ub,
                                    void* stream)
{
    if (p < 4 || p > kItiMaxP || !std::isfinite(eta) || !(eta != 0.0) || nbox < 0 || nrhs < 1 || nrhs > 256)
        return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!fin || (!ui && !ub) || (ui && !S) || (ub && !R)) return HPS_EINVAL;
    const int q = p - 2, n = q * q * q, m = 6 * q * q;
    const int warps = 8;
    dim3 grd((unsigned)((n + m + warps - 1) / warps), (unsigned)nrhs, (unsigned)nbox);
    k_iti_reconstruct<<<grd, 32 * warps, 0, static_cast<cudaStream_t>(stream)>>>(n, m, nrhs, eta, R, S, v, hout, fin,
                                                                                  ui, ub);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // extern "C"
