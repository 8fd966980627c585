/*
 * hps_oracle.c -- plain FP64 CPU oracle for the leaf-box reduction of the
 * two-level HPS solver (Kump, Yesypenko, Martinsson, arXiv:2503.04033).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously correct reference
 * that the CUDA library is checked against.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the library never
 * does, and it shares no code with the CUDA path.
 *
 * Every routine is the direct definition, in FP64, row-major:
 *   - Chebyshev-Lobatto nodes and the 1-D spectral differentiation matrix
 *     (Sec. 2.1: tensor Chebyshev grid per box, collocation as in Trefethen's
 *     "Spectral Methods in MATLAB");
 *   - the local equilibrium matrix A^tau (Algorithm 1, first step): interior
 *     rows apply the Helmholtz operator -Lap u - kappa^2 b u (Eq. 2), face rows
 *     take the outward normal derivative (Eq. 4, one box's half of the
 *     flux-continuity row), edge and corner nodes dropped (Remark 1);
 *   - the partition into A_ii, A_ib, A_bi, A_bb (Eq. 5);
 *   - S = -A_ii^{-1} A_ib and T = A_bb + A_bi S (Sec. 2.2 and Eq. 8), by a plain
 *     LU with partial pivoting (ties go to the lowest row);
 *   - v = A_ii^{-1} f_i, h = A_bi v and u_i = v + S u_b (the four solve steps of
 *     Sec. 2.2; Algorithm 2).
 *
 * Index conventions (shared by the library's C ABI, written out here on
 * their own):
 *   grid node (i,j,k), 0 <= i,j,k < p, has index i + p*j + p*p*k;
 *   interior node (i,j,k), 1 <= i,j,k <= q = p-2, has index (i-1) + q(j-1) + q^2(k-1);
 *   face f in order x-, x+, y-, y+, z-, z+; face node (a,b) with a the lower
 *   free axis has index n + f q^2 + (a-1) + q(b-1) in the kept list.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ sizes */

int oc_sizes(int p, int* n, int* m)
{
    if (p < 3) return -1;
    int q = p - 2;
    *n = q * q * q;
    *m = 6 * q * q;
    return 0;
}

/* ------------------------------------------------ 1-D nodes and D (Sec. 2.1) */

/* Chebyshev-Lobatto points on [-1,1] in ascending order,
 * t_j = -cos(pi j/(p-1)), written as sin(pi (2j-N)/(2N)) so that the set is
 * exactly symmetric about 0. */
void oc_nodes(int p, double* t)
{
    int N = p - 1;
    for (int j = 0; j < p; ++j)
        t[j] = sin(M_PI * (double)(2 * j - N) / (2.0 * N));
}

/* Spectral differentiation matrix on the nodes above (Trefethen, Spectral
 * Methods in MATLAB, ch. 6): D_ij = (c_i/c_j) (-1)^(i+j) / (t_i - t_j) for
 * i != j with c_0 = c_N = 2 and c_j = 1 otherwise; the diagonal from the
 * negative-sum rule D_ii = -sum_{j!=i} D_ij.  The node differences use
 * t_i - t_j = 2 sin((th_i+th_j)/2) sin((th_i-th_j)/2), th_j = pi j/N, which
 * keeps them accurate when the nodes cluster.  Row-major p x p. */
void oc_diff(int p, double* D)
{
    int N = p - 1;
    for (int i = 0; i < p; ++i) {
        double ci = (i == 0 || i == N) ? 2.0 : 1.0;
        double rowsum = 0.0;
        for (int j = 0; j < p; ++j) {
            if (i == j) continue;
            double cj = (j == 0 || j == N) ? 2.0 : 1.0;
            double thi = M_PI * i / N, thj = M_PI * j / N;
            double diff = 2.0 * sin(0.5 * (thi + thj)) * sin(0.5 * (thi - thj));
            double sgn = ((i + j) % 2 == 0) ? 1.0 : -1.0;
            double v = (ci / cj) * sgn / diff;
            D[i * p + j] = v;
            rowsum += v;
        }
        D[i * p + i] = -rowsum;
    }
}

/* Physical coordinates of the p^3 nodes of a box [lo, lo+h]:
 * x = lo + h (t+1)/2 per axis; xyz is [p^3][3] in grid-node order. */
void oc_node_coords(int p, const double* lo, const double* h, double* xyz)
{
    double* t = (double*)malloc(sizeof(double) * p);
    oc_nodes(p, t);
    for (int k = 0; k < p; ++k)
        for (int j = 0; j < p; ++j)
            for (int i = 0; i < p; ++i) {
                int g = i + p * j + p * p * k;
                xyz[3 * g + 0] = lo[0] + 0.5 * h[0] * (t[i] + 1.0);
                xyz[3 * g + 1] = lo[1] + 0.5 * h[1] * (t[j] + 1.0);
                xyz[3 * g + 2] = lo[2] + 0.5 * h[2] * (t[k] + 1.0);
            }
    free(t);
}

/* ------------------------------------------------ node classification */

/* Position of grid node (i,j,k) in the kept list (interior first, then the
 * six faces), or -1 for edge and corner nodes, which Remark 1 drops. */
int oc_kept_index(int p, int i, int j, int k)
{
    int q = p - 2, n = q * q * q, e = p - 1;
    int bi = (i == 0 || i == e), bj = (j == 0 || j == e), bk = (k == 0 || k == e);
    int nb = bi + bj + bk;
    if (nb == 0) return (i - 1) + q * (j - 1) + q * q * (k - 1);
    if (nb > 1) return -1;
    int f, a, b;
    if (bi)      { f = (i == 0) ? 0 : 1; a = j; b = k; }
    else if (bj) { f = (j == 0) ? 2 : 3; a = i; b = k; }
    else         { f = (k == 0) ? 4 : 5; a = i; b = j; }
    return n + f * q * q + (a - 1) + q * (b - 1);
}

/* Inverse map: kept index -> grid indices. */
void oc_kept_to_grid(int p, int idx, int* gi, int* gj, int* gk)
{
    int q = p - 2, n = q * q * q, e = p - 1;
    if (idx < n) {
        *gi = idx % q + 1; *gj = (idx / q) % q + 1; *gk = idx / (q * q) + 1;
        return;
    }
    int r = idx - n, f = r / (q * q), s = r % (q * q);
    int a = s % q + 1, b = s / q + 1;
    int side = (f % 2 == 0) ? 0 : e;
    switch (f / 2) {
    case 0: *gi = side; *gj = a; *gk = b; break;
    case 1: *gi = a; *gj = side; *gk = b; break;
    default: *gi = a; *gj = b; *gk = side; break;
    }
}

/* ------------------------------------------------ local matrix A^tau */

static void physical_d(int p, double h, const double* Dhat, double* D, double* D2)
{
    double s = 2.0 / h;
    for (int i = 0; i < p * p; ++i) D[i] = s * Dhat[i];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            double acc = 0.0;
            for (int l = 0; l < p; ++l) acc += D[i * p + l] * D[l * p + j];
            D2[i * p + j] = acc;
        }
}

/* Full local matrix over the kept nodes, (n+m) x (n+m) row-major.
 *   interior row (i,j,k):  -sum_i' D2x[i,i'] u(i',j,k) - sum_j' D2y[j,j'] u(i,j',k)
 *                          -sum_k' D2z[k,k'] u(i,j,k') - kappa^2 b(i,j,k) u(i,j,k)
 *   face row on side s of axis a (outward normal n = -e_a on the low side,
 *   +e_a on the high side):  (n . e_a) sum_l D_a[e,l] u(... l ...),
 *   e the face's own grid index along a.
 * b holds all p^3 node values; only interior ones enter.  beta (NULL, or
 * [3][p^3] node values of a velocity-like field) adds the divergence-form
 * first-order term div(beta u) to the interior rows:
 *   + sum_i' Dx[i,i'] beta_x(i',j,k) u(i',j,k) + (the same along y and z),
 * the product rule of collocation differentiation applied to beta_a u. */
void oc_leaf_matrix(int p, const double* h, double kappa, const double* b, const double* beta, double* A)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q, N = n + m, e = p - 1;
    double* Dhat = (double*)malloc(sizeof(double) * p * p);
    double* D = (double*)malloc(sizeof(double) * 3 * p * p);
    double* D2 = (double*)malloc(sizeof(double) * 3 * p * p);
    oc_diff(p, Dhat);
    for (int a = 0; a < 3; ++a) physical_d(p, h[a], Dhat, D + a * p * p, D2 + a * p * p);
    memset(A, 0, sizeof(double) * (size_t)N * N);
    for (int row = 0; row < N; ++row) {
        int i, j, k;
        oc_kept_to_grid(p, row, &i, &j, &k);
        double* Ar = A + (size_t)row * N;
        if (row < n) {
            for (int l = 0; l < p; ++l) {
                Ar[oc_kept_index(p, l, j, k)] -= D2[0 * p * p + i * p + l];
                Ar[oc_kept_index(p, i, l, k)] -= D2[1 * p * p + j * p + l];
                Ar[oc_kept_index(p, i, j, l)] -= D2[2 * p * p + k * p + l];
            }
            Ar[row] -= kappa * kappa * b[i + p * j + p * p * k];
            if (beta) {
                const int P3 = p * p * p;
                for (int l = 0; l < p; ++l) {
                    Ar[oc_kept_index(p, l, j, k)] += D[0 * p * p + i * p + l] * beta[0 * P3 + l + p * j + p * p * k];
                    Ar[oc_kept_index(p, i, l, k)] += D[1 * p * p + j * p + l] * beta[1 * P3 + i + p * l + p * p * k];
                    Ar[oc_kept_index(p, i, j, l)] += D[2 * p * p + k * p + l] * beta[2 * P3 + i + p * j + p * p * l];
                }
            }
        } else {
            int f = (row - n) / (q * q), axis = f / 2;
            double sgn = (f % 2 == 0) ? -1.0 : 1.0;
            int own = (f % 2 == 0) ? 0 : e;
            const double* Da = D + axis * p * p + own * p;
            for (int l = 0; l < p; ++l) {
                int col = axis == 0 ? oc_kept_index(p, l, j, k)
                        : axis == 1 ? oc_kept_index(p, i, l, k)
                                    : oc_kept_index(p, i, j, l);
                Ar[col] += sgn * Da[l];
            }
        }
    }
    free(Dhat); free(D); free(D2);
}

/* Split the local matrix into the four blocks of Eq. 5 (all row-major). */
void oc_split_blocks(int p, const double* A, double* Aii, double* Aib, double* Abi, double* Abb)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q, N = n + m;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            double v = A[(size_t)r * N + c];
            if (r < n && c < n) { if (Aii) Aii[(size_t)r * n + c] = v; }
            else if (r < n)     { if (Aib) Aib[(size_t)r * m + (c - n)] = v; }
            else if (c < n)     { if (Abi) Abi[(size_t)(r - n) * n + c] = v; }
            else                { if (Abb) Abb[(size_t)(r - n) * m + (c - n)] = v; }
        }
}

/* ------------------------------------------------ dense LU (partial pivoting) */

/* In-place LU with partial pivoting of a row-major n x n matrix, kji order.
 * piv[k] is the row swapped with row k at step k (ties go to the lowest row).
 * Returns 0, or k+1 if the k-th pivot is exactly zero (the matrix is singular). */
int oc_lu(int n, double* A, int* piv)
{
    int info = 0;
    for (int k = 0; k < n; ++k) {
        int pr = k;
        double best = fabs(A[(size_t)k * n + k]);
        for (int r = k + 1; r < n; ++r) {
            double v = fabs(A[(size_t)r * n + k]);
            if (v > best) { best = v; pr = r; }
        }
        piv[k] = pr;
        if (pr != k)
            for (int c = 0; c < n; ++c) {
                double tmp = A[(size_t)k * n + c];
                A[(size_t)k * n + c] = A[(size_t)pr * n + c];
                A[(size_t)pr * n + c] = tmp;
            }
        double pivot = A[(size_t)k * n + k];
        if (pivot == 0.0) { if (!info) info = k + 1; continue; }
        const double* Ak = A + (size_t)k * n;
#pragma omp parallel for schedule(static) if (n - k > 256)
        for (int r = k + 1; r < n; ++r) {
            double* Arow = A + (size_t)r * n;
            double l = Arow[k] / pivot;
            Arow[k] = l;
            for (int c = k + 1; c < n; ++c) Arow[c] -= l * Ak[c];
        }
    }
    return info;
}

/* Solve A X = B in place with the factors from oc_lu; X is n x nrhs row-major.
 * Row swaps in factorisation order, then L (unit lower), then U. */
void oc_lu_solve(int n, const double* LU, const int* piv, int nrhs, double* X)
{
    for (int k = 0; k < n; ++k)
        if (piv[k] != k)
            for (int c = 0; c < nrhs; ++c) {
                double tmp = X[(size_t)k * nrhs + c];
                X[(size_t)k * nrhs + c] = X[(size_t)piv[k] * nrhs + c];
                X[(size_t)piv[k] * nrhs + c] = tmp;
            }
    const int CB = 64;
#pragma omp parallel for schedule(dynamic) if (nrhs > CB && n > 256)
    for (int c0 = 0; c0 < nrhs; c0 += CB) {
        int c1 = c0 + CB < nrhs ? c0 + CB : nrhs;
        for (int i = 0; i < n; ++i) {
            double* Xi = X + (size_t)i * nrhs;
            for (int k = 0; k < i; ++k) {
                double l = LU[(size_t)i * n + k];
                if (l == 0.0) continue;
                const double* Xk = X + (size_t)k * nrhs;
                for (int c = c0; c < c1; ++c) Xi[c] -= l * Xk[c];
            }
        }
        for (int i = n - 1; i >= 0; --i) {
            double* Xi = X + (size_t)i * nrhs;
            for (int k = i + 1; k < n; ++k) {
                double u = LU[(size_t)i * n + k];
                if (u == 0.0) continue;
                const double* Xk = X + (size_t)k * nrhs;
                for (int c = c0; c < c1; ++c) Xi[c] -= u * Xk[c];
            }
            double d = LU[(size_t)i * n + i];
            for (int c = c0; c < c1; ++c) Xi[c] /= d;
        }
    }
}

/* C = A B + C0 (plain triple loop); A is r x s, B is s x t, all row-major.
 * C0 may be NULL (treated as zero). */
static void matmul_add(int r, int s, int t, const double* A, const double* B, const double* C0, double* C)
{
#pragma omp parallel for schedule(static) if ((long)r * s * t > 20000000L)
    for (int i = 0; i < r; ++i) {
        double* Ci = C + (size_t)i * t;
        for (int c = 0; c < t; ++c) Ci[c] = C0 ? C0[(size_t)i * t + c] : 0.0;
        for (int l = 0; l < s; ++l) {
            double a = A[(size_t)i * s + l];
            if (a == 0.0) continue;
            const double* Bl = B + (size_t)l * t;
            for (int c = 0; c < t; ++c) Ci[c] += a * Bl[c];
        }
    }
}

/* ------------------------------------------------ leaf reduction (Sec. 2.2) */

/* Builds A^tau, factors A_ii, and returns
 *   S = -A_ii^{-1} A_ib      (n x m, row-major; may be NULL),
 *   T = A_bb + A_bi S        (m x m, row-major; may be NULL).
 * Returns 0, or the 1-based zero-pivot position if A_ii is singular. */
int oc_leaf_dtn(int p, const double* h, double kappa, const double* b, const double* beta, double* T, double* S)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q, N = n + m;
    double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* Aii = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* X = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* Abi = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* Abb = (double*)malloc(sizeof(double) * (size_t)m * m);
    int* piv = (int*)malloc(sizeof(int) * n);
    oc_leaf_matrix(p, h, kappa, b, beta, A);
    oc_split_blocks(p, A, Aii, X, Abi, Abb);           /* X <- A_ib */
    free(A);
    for (size_t e = 0; e < (size_t)n * m; ++e) X[e] = -X[e];   /* X <- -A_ib */
    int info = oc_lu(n, Aii, piv);
    if (info == 0) {
        oc_lu_solve(n, Aii, piv, m, X);                /* X = S */
        if (S) memcpy(S, X, sizeof(double) * (size_t)n * m);
        if (T) matmul_add(m, n, m, Abi, X, Abb, T);
    }
    free(Aii); free(X); free(Abi); free(Abb); free(piv);
    return info;
}

/* Particular solution and its flux for nrhs body loads (Sec. 2.2 steps 1-2;
 * Algorithm 2, first loop):  v = A_ii^{-1} f_i,  h = A_bi v.
 * f is [nrhs][p^3] (grid order; only interior values enter), v is [nrhs][n],
 * hflux is [nrhs][m]. */
int oc_leaf_particular(int p, const double* h, double kappa, const double* b, const double* beta, int nrhs,
                       const double* f, double* v, double* hflux)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q, N = n + m;
    double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* Aii = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* Abi = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* X = (double*)malloc(sizeof(double) * (size_t)n * nrhs);
    int* piv = (int*)malloc(sizeof(int) * n);
    oc_leaf_matrix(p, h, kappa, b, beta, A);
    oc_split_blocks(p, A, Aii, NULL, Abi, NULL);
    free(A);
    for (int r = 0; r < n; ++r) {                      /* X[r][c] = f_c(interior node r) */
        int i, j, k;
        oc_kept_to_grid(p, r, &i, &j, &k);
        for (int c = 0; c < nrhs; ++c)
            X[(size_t)r * nrhs + c] = f[(size_t)c * p * p * p + i + p * j + p * p * k];
    }
    int info = oc_lu(n, Aii, piv);
    if (info == 0) {
        oc_lu_solve(n, Aii, piv, nrhs, X);
        for (int c = 0; c < nrhs; ++c)
            for (int r = 0; r < n; ++r) v[(size_t)c * n + r] = X[(size_t)r * nrhs + c];
        for (int c = 0; c < nrhs; ++c)
            for (int r = 0; r < m; ++r) {
                double acc = 0.0;
                for (int l = 0; l < n; ++l) acc += Abi[(size_t)r * n + l] * X[(size_t)l * nrhs + c];
                hflux[(size_t)c * m + r] = acc;
            }
    }
    free(Aii); free(Abi); free(X); free(piv);
    return info;
}

/* Interior reconstruction (Sec. 2.2 step 4; Algorithm 2, last loop):
 * u_i = v + S u_b with S recomputed as in oc_leaf_dtn.  v, ui are [nrhs][n],
 * ub is [nrhs][m]. */
int oc_leaf_reconstruct(int p, const double* h, double kappa, const double* b, const double* beta, int nrhs,
                        const double* v, const double* ub, double* ui)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q;
    double* S = (double*)malloc(sizeof(double) * (size_t)n * m);
    int info = oc_leaf_dtn(p, h, kappa, b, beta, NULL, S);
    if (info == 0)
        for (int c = 0; c < nrhs; ++c)
            for (int r = 0; r < n; ++r) {
                double acc = v[(size_t)c * n + r];
                for (int l = 0; l < m; ++l) acc += S[(size_t)r * m + l] * ub[(size_t)c * m + l];
                ui[(size_t)c * n + r] = acc;
            }
    free(S);
    return info;
}

/* ------------------------------------------------ batches ("for all boxes in parallel") */

/* Algorithm 1's loop over boxes, boxes spread over threads.  b is [nbox][p^3],
 * T is [nbox][m][m], S is [nbox][n][m] or NULL, status[nbox] gets each box's
 * return code.  nthreads <= 0 uses the OpenMP default. */
void oc_batch_dtn(int p, const double* h, double kappa, int nbox, const double* b,
                  double* T, double* S, int* status, int nthreads)
{
    int q = p - 2, n = q * q * q, m = 6 * q * q;
    size_t P3 = (size_t)p * p * p;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic) num_threads(nthreads)
#endif
    for (int bx = 0; bx < nbox; ++bx)
        status[bx] = oc_leaf_dtn(p, h, kappa, b + bx * P3, NULL,
                                 T ? T + (size_t)bx * m * m : NULL,
                                 S ? S + (size_t)bx * n * m : NULL);
    (void)nthreads;
}

int oc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ================================================================== 2-D
 *
 * The two-dimensional form of the same reduction (Sec. 1 and Sec. 3.2 treat
 * 2-D and 3-D alike: a p x p Chebyshev grid per box, corners dropped as in
 * Remark 1, DtN maps of size about 4p x 4p).
 *
 * Index conventions:
 *   grid node (i,j), 0 <= i,j < p, has index i + p*j;
 *   interior node (i,j), 1 <= i,j <= q = p-2, has index (i-1) + q(j-1);
 *   edge f in order x-, x+, y-, y+; edge node a (the free index, 1..q) has
 *   index n + f q + (a-1) in the kept list;  n = q^2, m = 4q.
 */

int oc2_sizes(int p, int* n, int* m)
{
    if (p < 3) return -1;
    int q = p - 2;
    *n = q * q;
    *m = 4 * q;
    return 0;
}

/* Coordinates [p^2][2] of a box [lo, lo+h] in grid-node order. */
void oc2_node_coords(int p, const double* lo, const double* h, double* xy)
{
    double* t = (double*)malloc(sizeof(double) * p);
    oc_nodes(p, t);
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) {
            int g = i + p * j;
            xy[2 * g + 0] = lo[0] + 0.5 * h[0] * (t[i] + 1.0);
            xy[2 * g + 1] = lo[1] + 0.5 * h[1] * (t[j] + 1.0);
        }
    free(t);
}

/* Kept index of grid node (i,j) (interior first, then the four edges), or
 * -1 for a corner. */
int oc2_kept_index(int p, int i, int j)
{
    int q = p - 2, n = q * q, e = p - 1;
    int bi = (i == 0 || i == e), bj = (j == 0 || j == e);
    if (!bi && !bj) return (i - 1) + q * (j - 1);
    if (bi && bj) return -1;
    if (bi) return n + ((i == 0) ? 0 : 1) * q + (j - 1);
    return n + ((j == 0) ? 2 : 3) * q + (i - 1);
}

void oc2_kept_to_grid(int p, int idx, int* gi, int* gj)
{
    int q = p - 2, n = q * q, e = p - 1;
    if (idx < n) { *gi = idx % q + 1; *gj = idx / q + 1; return; }
    int r = idx - n, f = r / q, a = r % q + 1;
    int side = (f % 2 == 0) ? 0 : e;
    if (f / 2 == 0) { *gi = side; *gj = a; }
    else            { *gi = a; *gj = side; }
}

/* Local matrix over the kept nodes, (n+m) x (n+m) row-major:
 *   interior row (i,j): -sum_i' D2x[i,i'] u(i',j) - sum_j' D2y[j,j'] u(i,j') - kappa^2 b(i,j) u(i,j);
 *   edge row on side s of axis a: (n . e_a) sum_l D_a[e,l] u(... l ...), the
 *   outward normal derivative, e the edge's own grid index along a.
 * b holds all p^2 node values. */
void oc2_leaf_matrix(int p, const double* h, double kappa, const double* b, double* A)
{
    int q = p - 2, n = q * q, m = 4 * q, N = n + m, e = p - 1;
    double* Dhat = (double*)malloc(sizeof(double) * p * p);
    double* D = (double*)malloc(sizeof(double) * 2 * p * p);
    double* D2 = (double*)malloc(sizeof(double) * 2 * p * p);
    oc_diff(p, Dhat);
    for (int a = 0; a < 2; ++a) physical_d(p, h[a], Dhat, D + a * p * p, D2 + a * p * p);
    memset(A, 0, sizeof(double) * (size_t)N * N);
    for (int row = 0; row < N; ++row) {
        int i, j;
        oc2_kept_to_grid(p, row, &i, &j);
        double* Ar = A + (size_t)row * N;
        if (row < n) {
            for (int l = 0; l < p; ++l) {
                Ar[oc2_kept_index(p, l, j)] -= D2[0 * p * p + i * p + l];
                Ar[oc2_kept_index(p, i, l)] -= D2[1 * p * p + j * p + l];
            }
            Ar[row] -= kappa * kappa * b[i + p * j];
        } else {
            int f = (row - n) / q, axis = f / 2;
            double sgn = (f % 2 == 0) ? -1.0 : 1.0;
            int own = (f % 2 == 0) ? 0 : e;
            const double* Da = D + axis * p * p + own * p;
            for (int l = 0; l < p; ++l) {
                int col = axis == 0 ? oc2_kept_index(p, l, j) : oc2_kept_index(p, i, l);
                Ar[col] += sgn * Da[l];
            }
        }
    }
    free(Dhat); free(D); free(D2);
}

/* S = -A_ii^{-1} A_ib (n x m) and T = A_bb + A_bi S (m x m), either NULL. */
int oc2_leaf_dtn(int p, const double* h, double kappa, const double* b, double* T, double* S)
{
    int q = p - 2, n = q * q, m = 4 * q, N = n + m;
    double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* Aii = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* X = (double*)malloc(sizeof(double) * (size_t)n * m);
    double* Abi = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* Abb = (double*)malloc(sizeof(double) * (size_t)m * m);
    int* piv = (int*)malloc(sizeof(int) * n);
    oc2_leaf_matrix(p, h, kappa, b, A);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            double v = A[(size_t)r * N + c];
            if (r < n && c < n) Aii[(size_t)r * n + c] = v;
            else if (r < n)     X[(size_t)r * m + (c - n)] = -v;     /* -A_ib */
            else if (c < n)     Abi[(size_t)(r - n) * n + c] = v;
            else                Abb[(size_t)(r - n) * m + (c - n)] = v;
        }
    free(A);
    int info = oc_lu(n, Aii, piv);
    if (info == 0) {
        oc_lu_solve(n, Aii, piv, m, X);
        if (S) memcpy(S, X, sizeof(double) * (size_t)n * m);
        if (T) matmul_add(m, n, m, Abi, X, Abb, T);
    }
    free(Aii); free(X); free(Abi); free(Abb); free(piv);
    return info;
}

/* v = A_ii^{-1} f_i and h = A_bi v for nrhs loads f [nrhs][p^2] (grid
 * order); v [nrhs][n], hflux [nrhs][m]. */
int oc2_leaf_particular(int p, const double* h, double kappa, const double* b, int nrhs, const double* f,
                        double* v, double* hflux)
{
    int q = p - 2, n = q * q, m = 4 * q, N = n + m;
    double* A = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* Aii = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* Abi = (double*)malloc(sizeof(double) * (size_t)m * n);
    double* X = (double*)malloc(sizeof(double) * (size_t)n * nrhs);
    int* piv = (int*)malloc(sizeof(int) * n);
    oc2_leaf_matrix(p, h, kappa, b, A);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < n; ++c) {
            if (r < n) Aii[(size_t)r * n + c] = A[(size_t)r * N + c];
            else       Abi[(size_t)(r - n) * n + c] = A[(size_t)r * N + c];
        }
    free(A);
    for (int r = 0; r < n; ++r) {
        int i, j;
        oc2_kept_to_grid(p, r, &i, &j);
        for (int c = 0; c < nrhs; ++c) X[(size_t)r * nrhs + c] = f[(size_t)c * p * p + i + p * j];
    }
    int info = oc_lu(n, Aii, piv);
    if (info == 0) {
        oc_lu_solve(n, Aii, piv, nrhs, X);
        for (int c = 0; c < nrhs; ++c)
            for (int r = 0; r < n; ++r) v[(size_t)c * n + r] = X[(size_t)r * nrhs + c];
        for (int c = 0; c < nrhs; ++c)
            for (int r = 0; r < m; ++r) {
                double acc = 0.0;
                for (int l = 0; l < n; ++l) acc += Abi[(size_t)r * n + l] * X[(size_t)l * nrhs + c];
                hflux[(size_t)c * m + r] = acc;
            }
    }
    free(Aii); free(Abi); free(X); free(piv);
    return info;
}
