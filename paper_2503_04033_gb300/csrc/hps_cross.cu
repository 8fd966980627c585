// Leaf reduction for operators with cross terms on Legendre face grids (FP64).
//
// Remark 1 of Sec. 2.1: the edge and corner nodes of a box can be dropped only
// when the operator has no cross terms d_a d_b u (a != b); with cross terms
// each face's data lives on a (p-1) x (p-1) grid of Gauss-Legendre nodes
// instead of the p x p Chebyshev grid.  Sec. 4.3 needs it: the parameter map
// of a curved domain brings variable coefficients and a cross term.  The
// operator is
//     A u = -sum_{a,b} C_ab(x) d_a d_b u + sum_a d_a(x) d_a u - kappa^2 b(x) u
// with C symmetric.  Per box, on the p^3 Chebyshev-Lobatto grid:
//  * the boundary Chebyshev nodes (faces, edges, corners) take their values
//    from the faces' Legendre data: a node on one face the face's
//    interpolant (degree p-2 per coordinate, the p x (p-1) matrix G on each
//    face coordinate), a node on several faces the average over them;
//  * one FP64 LU with partial pivoting of A_II (interior rows and columns)
//    carries [-A_IE P | f_I]: S = -A_II^{-1} A_IE P and v = A_II^{-1} f_I;
//  * T = T_E + Q N_I S and h = Q N_I v, with N_I the outward normal
//    derivative at the faces' interior Chebyshev nodes from interior values
//    and Q the (p-1) x p Chebyshev-to-Legendre interpolation on both face
//    coordinates; T_E = Q N P, the part of the DtN map that comes straight
//    from the face data, is the same for every box of a size and is built on
//    the host.
// An interior row couples to boundary nodes only along its three grid lines
// (second and first derivatives) and the borders of its three coordinate
// planes (cross terms), so its part of -A_IE P on each face is three tensor
// terms in G (k_build_cross).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "hps_internal.h"

namespace {

constexpr int kCrossMaxP = 16;

// Gauss-Legendre nodes (roots of P_N, ascending) by Newton's method on the
// three-term recurrence, from the asymptotic first guesses.
void legendre_roots(int N, double* x)
{
    for (int i = 0; i < N; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (N + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < N; ++k) {
                const double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            const double dp = N * (z * p1 - p0) / (z * z - 1.0);
            const double dz = N == 1 ? z : p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[N - 1 - i] = z;   // the guesses run from +1 down
    }
}

// L[i][j] = l_j(dst_i) for the Lagrange basis of the nodes src (ns of them).
void lagrange(const double* src, int ns, const double* dst, int nd, double* L)
{
    for (int i = 0; i < nd; ++i)
        for (int j = 0; j < ns; ++j) {
            double v = 1.0;
            for (int k = 0; k < ns; ++k)
                if (k != j) v *= (dst[i] - src[k]) / (src[j] - src[k]);
            L[i * ns + j] = v;
        }
}

struct CrossTables {
    int p = 0;
    std::vector<double> D, D2;   // [3][p][p] physical first and second derivative
    std::vector<double> G;       // [p][p-1]: Legendre values to Chebyshev nodes
    std::vector<double> Q;       // [p-1][p]: Chebyshev values to Legendre nodes
    std::vector<double> TE;      // [m][m]: Q N P, the DtN part straight from the face data
};

__host__ __device__ inline int fidx(int p, int i, int j, int k) { return i + p * (j + p * k); }

// Face f: normal axis a = f / 2, side f % 2, free axes u < v.
__host__ __device__ inline void face_axes(int f, int& a, int& u, int& v)
{
    a = f / 2;
    u = a == 0 ? 1 : 0;
    v = a == 2 ? 1 : 2;
}

void cross_tables(int p, const double h[3], CrossTables& t)
{
    const int pl = p - 1, ml = pl * pl, m = 6 * ml, pp = p * p, e = p - 1;
    t.p = p;
    std::vector<double> Dh(pp), tn(p), gn(pl);
    hps::cheb_diff(p, Dh.data());
    hps::cheb_nodes(p, tn.data());
    legendre_roots(pl, gn.data());
    t.D.assign(3 * pp, 0.0);
    t.D2.assign(3 * pp, 0.0);
    for (int a = 0; a < 3; ++a) {
        const double s = 2.0 / h[a];
        for (int k = 0; k < pp; ++k) t.D[a * pp + k] = s * Dh[k];
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int l = 0; l < p; ++l) acc += t.D[a * pp + i * p + l] * t.D[a * pp + l * p + j];
                t.D2[a * pp + i * p + j] = acc;
            }
    }
    t.G.assign((size_t)p * pl, 0.0);
    t.Q.assign((size_t)pl * p, 0.0);
    lagrange(gn.data(), pl, tn.data(), p, t.G.data());
    lagrange(tn.data(), p, gn.data(), pl, t.Q.data());
    // faces sharing each grid node (boundary nodes: 1, 2 or 3)
    std::vector<int> cnt((size_t)pp * p, 0);
    for (int f = 0; f < 6; ++f) {
        int a, u, v;
        face_axes(f, a, u, v);
        for (int iv = 0; iv < p; ++iv)
            for (int iu = 0; iu < p; ++iu) {
                int c[3];
                c[a] = (f & 1) ? e : 0;
                c[u] = iu;
                c[v] = iv;
                ++cnt[fidx(p, c[0], c[1], c[2])];
            }
    }
    // T_E, one column (a unit datum at Legendre node (fc, sc, tc)) at a time
    t.TE.assign((size_t)m * m, 0.0);
    std::vector<double> U((size_t)pp * p), dn(pp), zq((size_t)pl * p);
    for (int col = 0; col < m; ++col) {
        const int fc = col / ml, sc = col % pl, tcl = (col % ml) / pl;
        int ac, uc, vc;
        face_axes(fc, ac, uc, vc);
        std::fill(U.begin(), U.end(), 0.0);
        for (int iv = 0; iv < p; ++iv)
            for (int iu = 0; iu < p; ++iu) {
                int c[3];
                c[ac] = (fc & 1) ? e : 0;
                c[uc] = iu;
                c[vc] = iv;
                const int r = fidx(p, c[0], c[1], c[2]);
                U[r] = t.G[iu * pl + sc] * t.G[iv * pl + tcl] / cnt[r];
            }
        for (int f = 0; f < 6; ++f) {
            int a, u, v;
            face_axes(f, a, u, v);
            const double sgn = (f & 1) ? 1.0 : -1.0;
            const double* Da = t.D.data() + a * pp + ((f & 1) ? e : 0) * p;
            for (int iv = 0; iv < p; ++iv)
                for (int iu = 0; iu < p; ++iu) {
                    double acc = 0.0;
                    for (int l = 0; l < p; ++l) {
                        int c[3];
                        c[a] = l;
                        c[u] = iu;
                        c[v] = iv;
                        acc += Da[l] * U[fidx(p, c[0], c[1], c[2])];
                    }
                    dn[iu + p * iv] = sgn * acc;
                }
            for (int ss = 0; ss < pl; ++ss)          // Q along u, then along v
                for (int iv = 0; iv < p; ++iv) {
                    double acc = 0.0;
                    for (int iu = 0; iu < p; ++iu) acc += t.Q[ss * p + iu] * dn[iu + p * iv];
                    zq[ss * p + iv] = acc;
                }
            for (int tt = 0; tt < pl; ++tt)
                for (int ss = 0; ss < pl; ++ss) {
                    double acc = 0.0;
                    for (int iv = 0; iv < p; ++iv) acc += t.Q[tt * p + iv] * zq[ss * p + iv];
                    t.TE[(size_t)(f * ml + ss + pl * tt) * m + col] = acc;
                }
        }
    }
}

// Device view of the tables: D, D2 [3][p][p], G [p][p-1], Q [p-1][p].
struct CrossDev {
    const double *D, *D2, *G, *Q;
};

// Row r (interior node (i0, i1, i2)) of M = [A_II | -A_IE P | f_I] for one
// box.  C [nbox][6][p^3] (C11, C22, C33, C12, C13, C23), d [nbox][3][p^3] or
// null, b [nbox][p^3], f [nbox][nrhs][p^3].
__global__ void __launch_bounds__(128) k_build_cross(int p, CrossDev tb, double kappa, const double* __restrict__ C,
                                                     const double* __restrict__ d, const double* __restrict__ b,
                                                     int nrhs, const double* __restrict__ f, double* __restrict__ M,
                                                     long long ldm, long long sM, int* __restrict__ status)
{
    __shared__ double coef[10];                  // C (6), d (3), kappa^2 b
    __shared__ double lin[6][2][kCrossMaxP];     // per face: sums over the u-line and the v-line, per Legendre index
    __shared__ double pt[6];                     // per face: the coefficient of the node on the row's normal line
    const int q = p - 2, n = q * q * q, pl = p - 1, ml = pl * pl, m = 6 * ml, pp = p * p, e = p - 1;
    const int r = blockIdx.x, box = blockIdx.y;
    const int idx[3] = {r % q + 1, (r / q) % q + 1, r / (q * q) + 1};
    const int g = fidx(p, idx[0], idx[1], idx[2]);
    const long long p3 = (long long)pp * p;
    if (threadIdx.x < 6) coef[threadIdx.x] = C[((long long)box * 6 + threadIdx.x) * p3 + g];
    else if (threadIdx.x < 9) coef[threadIdx.x] = d ? d[((long long)box * 3 + threadIdx.x - 6) * p3 + g] : 0.0;
    else if (threadIdx.x == 9) {
        const double bv = b[(long long)box * p3 + g];
        if (!isfinite(bv)) status[box] = HPS_EINVAL;
        coef[9] = kappa * kappa * bv;
    }
    __syncthreads();
    const int ci[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};   // C_ab in coef[]
    auto Dm = [&](int a, int i, int j) { return tb.D[a * pp + i * p + j]; };
    auto D2m = [&](int a, int i, int j) { return tb.D2[a * pp + i * p + j]; };
    // per-face tensor terms of -A_IE P
    for (int w = threadIdx.x; w < 6 * 2 * pl; w += blockDim.x) {
        const int fc = w / (2 * pl), which = (w / pl) % 2, s = w % pl;
        int a, u, v;
        face_axes(fc, a, u, v);
        const int la = (fc & 1) ? e : 0, o = which ? v : u;   // o: the axis the line runs along
        const double base = -2.0 * coef[ci[a][o]] * Dm(a, idx[a], la);
        double acc = 0.0;
        for (int l = 0; l < p; ++l) {
            const double wgt = (l == 0 || l == e) ? 0.5 : 1.0;   // edge nodes: shared by two faces
            acc += base * Dm(o, idx[o], l) * wgt * tb.G[l * pl + s];
        }
        lin[fc][which][s] = acc;
    }
    if (threadIdx.x < 6) {
        const int fc = threadIdx.x, a = fc / 2, la = (fc & 1) ? e : 0;
        pt[fc] = -coef[ci[a][a]] * D2m(a, idx[a], la) + coef[6 + a] * Dm(a, idx[a], la);
    }
    __syncthreads();
    double* row = M + (long long)box * sM + (long long)r * ldm;
    for (int c = threadIdx.x; c < ldm; c += blockDim.x) {
        double val = 0.0;
        if (c < n) {
            const int cc[3] = {c % q + 1, (c / q) % q + 1, c / (q * q) + 1};
            int ndiff = 0, ax0 = -1, ax1 = -1;
            for (int a = 0; a < 3; ++a)
                if (cc[a] != idx[a]) {
                    if (ndiff == 0) ax0 = a;
                    else ax1 = a;
                    ++ndiff;
                }
            if (ndiff == 0) {
                for (int a = 0; a < 3; ++a) {
                    val += -coef[ci[a][a]] * D2m(a, idx[a], idx[a]) + coef[6 + a] * Dm(a, idx[a], idx[a]);
                    for (int bb = a + 1; bb < 3; ++bb)
                        val -= 2.0 * coef[ci[a][bb]] * Dm(a, idx[a], idx[a]) * Dm(bb, idx[bb], idx[bb]);
                }
                val -= coef[9];
            } else if (ndiff == 1) {
                const int a = ax0;
                val = -coef[ci[a][a]] * D2m(a, idx[a], cc[a]) + coef[6 + a] * Dm(a, idx[a], cc[a]);
                for (int bb = 0; bb < 3; ++bb)
                    if (bb != a) val -= 2.0 * coef[ci[a][bb]] * Dm(a, idx[a], cc[a]) * Dm(bb, idx[bb], idx[bb]);
            } else if (ndiff == 2) {
                val = -2.0 * coef[ci[ax0][ax1]] * Dm(ax0, idx[ax0], cc[ax0]) * Dm(ax1, idx[ax1], cc[ax1]);
            }
        } else if (c < n + m) {
            const int k = c - n, fc = k / ml, s = k % pl, t = (k % ml) / pl;
            int a, u, v;
            face_axes(fc, a, u, v);
            const double gu = tb.G[idx[u] * pl + s], gv = tb.G[idx[v] * pl + t];
            val = -(pt[fc] * gu * gv + lin[fc][0][s] * gv + gu * lin[fc][1][t]);
        } else if (c < n + m + nrhs) {
            val = f[((long long)box * nrhs + (c - n - m)) * p3 + g];
        }
        row[c] = val;
    }
}

// T = T_E + Q N_I S (add_te) or h = Q N_I v on face fc for 32 columns of the
// solved block (columns col0 + c of M's rows): the normal derivative at the
// face's q x q interior Chebyshev nodes from the q interior values of each
// normal line, then Q on both face coordinates.  out: T [nbox][m][m] rows
// (fc, s, t), or h transposed [nbox][ncols][m].
__global__ void __launch_bounds__(256) k_dn_cross(int p, CrossDev tb, const double* __restrict__ M, long long ldm,
                                                  long long sM, int col0, int ncols, const double* __restrict__ TE,
                                                  double* __restrict__ out, int transposed)
{
    extern __shared__ double sh[];
    const int q = p - 2, pl = p - 1, ml = pl * pl, m = 6 * ml, pp = p * p, e = p - 1;
    const int fc = blockIdx.x % 6, cb = (blockIdx.x / 6) * 32, box = blockIdx.y;
    double* Y = sh;                 // [q*q][32]: normal derivatives at interior face nodes (iu, iv)
    double* Z = sh + q * q * 32;    // [q][pl][32]: Q applied along v
    int a, u, v;
    face_axes(fc, a, u, v);
    const double sgn = (fc & 1) ? 1.0 : -1.0;
    const double* Da = tb.D + a * pp + ((fc & 1) ? e : 0) * p;
    const double* Mb = M + (long long)box * sM + col0;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;   // 8 groups share the face nodes
    const int c = cb + lane;
    const bool live = c < ncols;
    for (int node = grp; node < q * q; node += 8) {
        const int iu = node % q + 1, iv = node / q + 1;
        double acc = 0.0;
        if (live)
            for (int l = 1; l <= q; ++l) {
                int cc[3];
                cc[a] = l;
                cc[u] = iu;
                cc[v] = iv;
                const int rr = (cc[0] - 1) + q * ((cc[1] - 1) + q * (cc[2] - 1));
                acc += Da[l] * Mb[(long long)rr * ldm + c];
            }
        Y[node * 32 + lane] = sgn * acc;
    }
    __syncthreads();
    for (int w = grp; w < q * pl; w += 8) {
        const int iu = w % q, t = w / q;
        double acc = 0.0;
        for (int iv = 0; iv < q; ++iv) acc += tb.Q[t * p + iv + 1] * Y[(iu + q * iv) * 32 + lane];
        Z[(iu + q * t) * 32 + lane] = acc;
    }
    __syncthreads();
    for (int w = grp; w < ml; w += 8) {
        const int s = w % pl, t = w / pl;
        double acc = 0.0;
        for (int iu = 0; iu < q; ++iu) acc += tb.Q[s * p + iu + 1] * Z[(iu + q * t) * 32 + lane];
        if (!live) continue;
        const int rowo = fc * ml + s + pl * t;
        if (transposed) {
            out[((long long)box * ncols + c) * m + rowo] = acc;
        } else {
            if (TE) acc += TE[(long long)rowo * m + c];
            out[((long long)box * m + rowo) * ncols + c] = acc;
        }
    }
}

// S [nbox][n][m] and v [nbox][nrhs][n] out of the solved columns.
__global__ void k_extract_cross(int n, int m, int nrhs, const double* __restrict__ M, long long ldm, long long sM,
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

hps_status hps_leaf_cross_sizes(int p, int* n, int* m)
{
    if (p < 3 || p > kCrossMaxP) return HPS_EINVAL;
    if (n) *n = (p - 2) * (p - 2) * (p - 2);
    if (m) *m = 6 * (p - 1) * (p - 1);
    return HPS_OK;
}

hps_status hps_leaf_cross_nodes(int p, const double lo[3], const double h[3], double* xyz)
{
    if (p < 3 || p > kCrossMaxP || !lo || !h || !xyz) return HPS_EINVAL;
    const int pl = p - 1, ml = pl * pl;
    std::vector<double> g(pl);
    legendre_roots(pl, g.data());
    for (int f = 0; f < 6; ++f) {
        int a, u, v;
        face_axes(f, a, u, v);
        for (int t = 0; t < pl; ++t)
            for (int s = 0; s < pl; ++s) {
                double* x = xyz + 3 * (f * ml + s + pl * t);
                x[a] = lo[a] + ((f & 1) ? h[a] : 0.0);
                x[u] = lo[u] + 0.5 * h[u] * (g[s] + 1.0);
                x[v] = lo[v] + 0.5 * h[v] * (g[t] + 1.0);
            }
    }
    return HPS_OK;
}

hps_status hps_leaf_cross_solve(int p, const double h[3], double kappa, int nbox, const double* C, const double* d,
                                const double* b, int nrhs, const double* f, double* T, double* S, double* v,
                                double* hflux, int* box_status, void* stream)
{
    if (p < 4 || p > kCrossMaxP || !h || !std::isfinite(kappa) || nbox < 0 || nrhs < 0 || nrhs > 256)
        return HPS_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(h[a] > 0.0) || !std::isfinite(h[a])) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!C || !b || (nrhs > 0 && (!f || !v || !hflux)) || (!T && !S && nrhs == 0)) return HPS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int q = p - 2, n = q * q * q, m = 6 * (p - 1) * (p - 1), pp = p * p;
    CrossTables tab;
    cross_tables(p, h, tab);
    // device tables: D, D2, G, Q, then T_E
    std::vector<double> small;
    small.insert(small.end(), tab.D.begin(), tab.D.end());
    small.insert(small.end(), tab.D2.begin(), tab.D2.end());
    small.insert(small.end(), tab.G.begin(), tab.G.end());
    small.insert(small.end(), tab.Q.begin(), tab.Q.end());
    hps::Plan PL = hps::make_plan(n, m + nrhs, HPS_FP64, 0, false, false);
    const size_t small_bytes = hps::align_up(sizeof(double) * small.size(), 256);
    const size_t te_bytes = hps::align_up(sizeof(double) * tab.TE.size(), 256);
    const size_t st_bytes = hps::align_up(sizeof(int) * (size_t)nbox, 256);
    const size_t bytes = small_bytes + te_bytes + st_bytes + PL.per_box * (size_t)nbox;
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, bytes, st) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
    char* base = static_cast<char*>(ws);
    double* dsmall = reinterpret_cast<double*>(base);
    double* dte = reinterpret_cast<double*>(base + small_bytes);
    int* status = box_status ? box_status : reinterpret_cast<int*>(base + small_bytes + te_bytes);
    hps::Work<double> w = hps::carve<double>(PL, base + small_bytes + te_bytes + st_bytes, nbox);
    hps_status rc = HPS_OK;
    // pageable sources: the copies are staged before the call returns
    if (cudaMemcpyAsync(dsmall, small.data(), sizeof(double) * small.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dte, tab.TE.data(), sizeof(double) * tab.TE.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(int) * (size_t)nbox, st) != cudaSuccess)
        rc = HPS_ECUDA;
    if (rc == HPS_OK) {
        CrossDev tb;
        tb.D = dsmall;
        tb.D2 = dsmall + 3 * pp;
        tb.G = dsmall + 6 * pp;
        tb.Q = dsmall + 6 * pp + p * (p - 1);
        k_build_cross<<<dim3((unsigned)n, (unsigned)nbox), 128, 0, st>>>(p, tb, kappa, C, d, b, nrhs, f, w.M, PL.ldm,
                                                                         w.sM, status);
        hps::lu_factor<double>(PL, w, nbox, status, st);
        hps::lu_backward<double>(PL, w, nbox, n, m + nrhs, nullptr, st);
        const size_t smem = (size_t)(q * q + q * (p - 1)) * 32 * sizeof(double);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_dn_cross, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
        if (T)
            k_dn_cross<<<dim3((unsigned)(6 * ((m + 31) / 32)), (unsigned)nbox), 256, smem, st>>>(
                p, tb, w.M, PL.ldm, w.sM, n, m, dte, T, 0);
        if (nrhs > 0)
            k_dn_cross<<<dim3((unsigned)(6 * ((nrhs + 31) / 32)), (unsigned)nbox), 256, smem, st>>>(
                p, tb, w.M, PL.ldm, w.sM, n + m, nrhs, nullptr, hflux, 1);
        if (S || nrhs > 0)
            k_extract_cross<<<dim3((unsigned)n, (unsigned)nbox), 128, 0, st>>>(n, m, nrhs, w.M, PL.ldm, w.sM, S,
                                                                                nrhs > 0 ? v : nullptr);
        if (cudaGetLastError() != cudaSuccess) rc = HPS_ECUDA;
    }
    if (cudaFreeAsync(ws, st) != cudaSuccess && rc == HPS_OK) rc = HPS_ECUDA;
    return rc;
}

hps_status hps_leaf_cross_reconstruct(int p, int nbox, int nrhs, const double* S, const double* v, const double* ub,
                                      double* ui, void* stream)
{
    if (p < 4 || p > kCrossMaxP || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!S || !ub || !ui) return HPS_EINVAL;
    const int q = p - 2;
    hps::launch_recon_stored(S, q * q * q, 6 * (p - 1) * (p - 1), nrhs, v, ub, ui, nbox,
                             static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

}  // extern "C"
