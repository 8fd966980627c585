// The 2-D leaf reduction on the GPU (FP64).
//
// The method is the same in two dimensions (Sec. 1; Sec. 3.2 sizes the 2-D
// DtN maps at about 4p x 4p): a p x p Chebyshev-Lobatto grid per box, the
// four corners dropped (Remark 1), n = (p-2)^2 interior and m = 4 (p-2) edge
// nodes.  Per box, one FP64 LU with partial pivoting of A_ii carries the
// right-hand sides [-A_ib | f_i] (the library's blocked LU: panel kernel and
// CUDA-core update products), giving S = -A_ii^{-1} A_ib and v = A_ii^{-1} f_i
// in one factorisation; T = A_bb + A_bi S and h = A_bi v are the structured
// D_n products (q terms per entry).  Reconstruction u_i = v + S u_b reuses the
// stored-S kernel of the 3-D path.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hps_internal.h"

namespace {

// The per-axis D and D^2 tables by value: one small kernel writes them to the
// workspace, so the call makes no host-to-device copy and stays
// stream-ordered (kernel parameters are captured at launch).
struct Tables2d {
    double t[4 * hps::kMaxP * hps::kMaxP];
};
static_assert(sizeof(Tables2d) <= 32000, "kernel parameter space");

__global__ void k_tables2d(const Tables2d a, int count, double* __restrict__ out)
{
    for (int k = threadIdx.x; k < count; k += blockDim.x) out[k] = a.t[k];
}

// M = [A_ii | -A_ib | f_i] of each box (row r = interior node (i, j)).
//   A_ii(r, c) = -D2x[i][i'] [j' = j] - D2y[j][j'] [i' = i] - kappa^2 b(i, j) [c = r]
//   A_ib(r, e) for edge node e at grid (gi, gj): the same two terms.
__global__ void k_build2d(int p, const double* __restrict__ D2, double kappa, const double* __restrict__ b,
                          int nrhs, const double* __restrict__ f, double* __restrict__ M, long long ldm,
                          long long sM, int* __restrict__ status)
{
    const int q = p - 2, n = q * q, m = 4 * q, e = p - 1;
    const int r = blockIdx.x, box = blockIdx.y;
    const int i = r % q + 1, j = r / q + 1;
    const double* D2x = D2;
    const double* D2y = D2 + p * p;
    const double bv = b[(long long)box * p * p + i + p * j];
    if (threadIdx.x == 0 && !isfinite(bv)) status[box] = HPS_EINVAL;
    double* row = M + (long long)box * sM + (long long)r * ldm;
    for (int c = threadIdx.x; c < ldm; c += blockDim.x) {
        double v = 0.0;
        if (c < n) {
            const int i2 = c % q + 1, j2 = c / q + 1;
            if (j2 == j) v -= D2x[i * p + i2];
            if (i2 == i) v -= D2y[j * p + j2];
            if (c == r) v -= kappa * kappa * bv;
        } else if (c < n + m) {
            const int ed = c - n, fe = ed / q, a = ed % q + 1;
            const int side = (fe % 2 == 0) ? 0 : e;
            const int gi = (fe / 2 == 0) ? side : a, gj = (fe / 2 == 0) ? a : side;
            double aib = 0.0;
            if (gj == j) aib -= D2x[i * p + gi];
            if (gi == i) aib -= D2y[j * p + gj];
            v = -aib;
        } else if (c < n + m + nrhs) {
            v = f[((long long)box * nrhs + (c - n - m)) * p * p + i + p * j];
        }
        row[c] = v;
    }
}

// Outward normal derivative of [X; edge values] on edge row r (edge f, free
// index a): sgn_f (sum_{l=1..q} D_a[own][l] X(interior (l, a)) + A_bb terms).
// With X the S columns and A_bb this is T = A_bb + A_bi S; with X the v
// columns and no A_bb it is h = A_bi v.  out_T: [nbox][m][m]; out_h:
// [nbox][nrhs][m] (transposed).
__global__ void k_dn2d(int p, const double* __restrict__ D, const double* __restrict__ M, long long ldm,
                       long long sM, int col0, int ncols, int add_abb, double* __restrict__ out, int transposed)
{
    const int q = p - 2, m = 4 * q, e = p - 1;
    const int r = blockIdx.x, box = blockIdx.y;
    const int f = r / q, a = r % q + 1, axis = f / 2;
    const int own = (f % 2 == 0) ? 0 : e, opp = e - own;
    const double sgn = (f % 2 == 0) ? -1.0 : 1.0;
    const double* Da = D + axis * p * p + own * p;
    const double* Mb = M + (long long)box * sM;
    const int ropp = (f ^ 1) * q + (a - 1);
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        double acc = 0.0;
        for (int l = 1; l <= q; ++l) {
            const int row = axis == 0 ? (l - 1) + q * (a - 1) : (a - 1) + q * (l - 1);
            acc += Da[l] * Mb[(long long)row * ldm + col0 + c];
        }
        if (add_abb) {
            if (c == r) acc += Da[own];
            if (c == ropp) acc += Da[opp];
        }
        const double v = sgn * acc;
        if (transposed) out[((long long)box * ncols + c) * m + r] = v;
        else out[((long long)box * m + r) * ncols + c] = v;
    }
}

// Copies of the solved columns: S [nbox][n][m] and v [nbox][nrhs][n].
__global__ void k_extract2d(int n, int m, int nrhs, const double* __restrict__ M, long long ldm, long long sM,
                            double* __restrict__ S, double* __restrict__ v)
{
    const int r = blockIdx.x, box = blockIdx.y;
    const double* Mr = M + (long long)box * sM + (long long)r * ldm + n;
    for (int c = threadIdx.x; c < m + nrhs; c += blockDim.x) {
        if (c < m) {
            if (S) S[((long long)box * n + r) * m + c] = Mr[c];
        } else if (v) {
            v[((long long)box * nrhs + (c - m)) * n + r] = Mr[c];
        }
    }
}

}  // namespace

extern "C" {

hps_status hps_leaf2d_solve(int p, const double h[2], double kappa, int nbox, const double* b, int nrhs,
                            const double* f, double* T, double* S, double* v, double* hflux, int* box_status,
                            void* stream)
{
    if (p < 3 || p > hps::kMaxP || !h || !(h[0] > 0.0) || !(h[1] > 0.0) || !std::isfinite(kappa) || nbox < 0 ||
        nrhs < 0 || nrhs > 256)
        return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || (nrhs > 0 && (!f || !v || !hflux)) || (!T && !S && nrhs == 0)) return HPS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int q = p - 2, n = q * q, m = 4 * q;
    // physical D and D^2 per axis, [2][p][p]
    std::vector<double> Dhat((size_t)p * p);
    Tables2d tab;
    const int ntab = 4 * p * p;
    hps::cheb_diff(p, Dhat.data());
    for (int a = 0; a < 2; ++a) {
        double* Da = tab.t + (size_t)a * p * p;
        double* D2a = tab.t + (size_t)(2 + a) * p * p;
        const double s = 2.0 / h[a];
        for (int k = 0; k < p * p; ++k) Da[k] = s * Dhat[k];
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int l = 0; l < p; ++l) acc += Da[i * p + l] * Da[l * p + j];
                D2a[i * p + j] = acc;
            }
    }
    hps::Plan PL = hps::make_plan(n, m + nrhs, HPS_FP64, 0, false, false);
    const size_t tab_bytes = hps::align_up(sizeof(double) * (size_t)ntab, 256);
    const size_t st_bytes = hps::align_up(sizeof(int) * (size_t)nbox, 256);
    const size_t bytes = tab_bytes + st_bytes + PL.per_box * (size_t)nbox;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, bytes, st) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
    char* base = static_cast<char*>(ws);
    double* dtab = reinterpret_cast<double*>(base);
    int* status = box_status ? box_status : reinterpret_cast<int*>(base + tab_bytes);
    hps::Work<double> w = hps::carve<double>(PL, base + tab_bytes + st_bytes, nbox);
    hps_status rc = HPS_OK;
    k_tables2d<<<1, 256, 0, st>>>(tab, ntab, dtab);
    if (cudaMemsetAsync(status, 0, sizeof(int) * (size_t)nbox, st) != cudaSuccess) rc = HPS_ECUDA;
    if (rc == HPS_OK) {
        const double* dD = dtab;
        const double* dD2 = dtab + 2 * p * p;
        k_build2d<<<dim3((unsigned)n, (unsigned)nbox), 128, 0, st>>>(p, dD2, kappa, b, nrhs, f, w.M, PL.ldm, w.sM,
                                                                      status);
        hps::lu_factor<double>(PL, w, nbox, status, st);
        hps::lu_backward<double>(PL, w, nbox, n, m + nrhs, nullptr, st);
        if (T) k_dn2d<<<dim3((unsigned)m, (unsigned)nbox), 128, 0, st>>>(p, dD, w.M, PL.ldm, w.sM, n, m, 1, T, 0);
        if (nrhs > 0)
            k_dn2d<<<dim3((unsigned)m, (unsigned)nbox), 128, 0, st>>>(p, dD, w.M, PL.ldm, w.sM, n + m, nrhs, 0,
                                                                       hflux, 1);
        if (S || nrhs > 0)
            k_extract2d<<<dim3((unsigned)n, (unsigned)nbox), 128, 0, st>>>(n, m, nrhs, w.M, PL.ldm, w.sM, S,
                                                                            nrhs > 0 ? v : nullptr);
        if (cudaGetLastError() != cudaSuccess) rc = HPS_ECUDA;
    }
    if (cudaFreeAsync(ws, st) != cudaSuccess && rc == HPS_OK) rc = HPS_ECUDA;
    return rc;
}

hps_status hps_leaf2d_reconstruct(int p, int nbox, int nrhs, const double* S, const double* v, const double* ub,
                                  double* ui, void* stream)
{
    if (p < 3 || p > hps::kMaxP || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!S || !ub || !ui) return HPS_EINVAL;
    const int q = p - 2;
    hps::launch_recon_stored(S, q * q, 4 * q, nrhs, v, ub, ui, nbox, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // extern "C"
