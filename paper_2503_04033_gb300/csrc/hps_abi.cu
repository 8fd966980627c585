// C ABI of the HPS leaf library: context, workspace, per-(p, h) operator
// tables, LU plans, and the launch sequences of the build and solve stages.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "hps_internal.h"

using namespace hps;

namespace hps {

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
};

struct Profiler {
    std::vector<ProfRec> recs;
    size_t used = 0;
    long long launches[KC_COUNT] = {};
    double ms[KC_COUNT] = {}, flops[KC_COUNT] = {}, bytes[KC_COUNT] = {};
};

thread_local Profiler* t_prof = nullptr;

void prof_begin(int cls, cudaStream_t st)
{
    Profiler* p = t_prof;
    if (!p) return;
    if (p->used == p->recs.size()) {
        ProfRec r{};
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
        p->recs.push_back(r);
    }
    ProfRec& r = p->recs[p->used];
    r.cls = cls;
    cudaEventRecord(r.a, st);
}

void prof_end(int cls, cudaStream_t st, double flops, double bytes)
{
    Profiler* p = t_prof;
    if (!p) return;
    ProfRec& r = p->recs[p->used++];
    r.cls = cls;
    r.flops = flops;
    r.bytes = bytes;
    cudaEventRecord(r.b, st);
}

static void prof_resolve(Profiler* p)
{
    for (size_t i = 0; i < p->used; ++i) {
        ProfRec& r = p->recs[i];
        float ms = 0.0f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        p->launches[r.cls] += 1;
        p->ms[r.cls] += ms;
        p->flops[r.cls] += r.flops;
        p->bytes[r.cls] += r.bytes;
    }
    p->used = 0;
}

}  // namespace hps

struct hps_ctx {
    int device = 0;
    size_t ws_max = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::map<std::tuple<int, double, double, double>, Geometry> geoms;
    int ir_iters = 8;
    double ir_tol = 1e-12;
    int nb_opt = 0;
    int use_tc = 1;
    int sync = 0;
    int zero_row_box = -1;
    bool prof_on = false;
    hps::Profiler prof;
    int* d_iters = nullptr;
    double* d_relcorr = nullptr;
    size_t diag_cap = 0;
    int last_nbox = 0;
    cudaStream_t last_stream = nullptr;
    std::mutex mu;
};

namespace hps {

// ------------------------------------------------------------ 1-D operators

// Chebyshev-Lobatto nodes on [-1,1], ascending, t_j = -cos(pi j / N), N = p-1
// (Sec. 2.1), evaluated as sin(pi (2j - N) / (2N)) for exact symmetry.
void cheb_nodes(int p, double* t)
{
    const int N = p - 1;
    for (int j = 0; j < p; ++j) t[j] = std::sin(M_PI * double(2 * j - N) / (2.0 * N));
}

// Spectral differentiation matrix for those nodes (Trefethen, Spectral Methods
// in MATLAB, ch. 6), off-diagonal (c_i/c_j)(-1)^{i+j}/(t_i - t_j), node
// differences through 2 sin((a+b)/2) sin((a-b)/2), diagonal by negative row
// sums.
void cheb_diff(int p, double* D)
{
    const int N = p - 1;
    for (int i = 0; i < p; ++i) {
        double s = 0.0;
        const double ci = (i == 0 || i == N) ? 2.0 : 1.0;
        for (int j = 0; j < p; ++j) {
            if (j == i) continue;
            const double cj = (j == 0 || j == N) ? 2.0 : 1.0;
            const double a = M_PI * i / N, bth = M_PI * j / N;
            const double d = 2.0 * std::sin(0.5 * (a + bth)) * std::sin(0.5 * (a - bth));
            const double v = (ci / cj) * (((i + j) & 1) ? -1.0 : 1.0) / d;
            D[i * p + j] = v;
            s += v;
        }
        D[i * p + i] = -s;
    }
}

// ------------------------------------------------------------ LU sequences

template <typename T>
GemmArgs<T> gargs()
{
    GemmArgs<T> a{};
    a.alpha = T(-1);
    return a;
}

// Right-looking blocked LU of M's first n columns, carrying the update over
// all n + r used columns (so the RHS block receives L^{-1} P B).
template <typename T>
void lu_factor(const Plan& P, Work<T>& w, int nbox, int* status, cudaStream_t st)
{
    const int n = P.n, NB = P.NB;
    const long long ldm = P.ldm;
    for (int s = 0; s < P.nsteps; ++s) {
        const int k = P.k0[s], nb = P.nbs[s];
        T* Fs = w.F + P.fw_off[s];
        T* Bs = w.B + P.bw_off[s];
        int* Ps = w.perm + P.perm_off[s];
        launch_panel<T>(w.M, ldm, w.sM, n, k, nb, P.ib, Ps, w.sP, Fs, NB, w.sF, Bs + (long long)k * NB, NB, w.sB,
                        status, nullptr, nbox, st);
        if (n - k - nb > 0) {
            GemmArgs<T> a = gargs<T>();
            a.A = w.M + (long long)(k + nb) * ldm + k; a.lda = ldm; a.sA = w.sM;
            a.B = Fs; a.ldb = NB; a.sB = w.sF;
            a.O = Fs + (long long)nb * NB; a.ldo = NB; a.sO = w.sF;
            a.M = n - k - nb; a.N = nb; a.K = nb; a.mode = GM_SET;
            launch_gemm<T>(a, nbox, st);
        }
        if (k > 0) {
            GemmArgs<T> a = gargs<T>();
            a.A = w.M + k; a.lda = ldm; a.sA = w.sM;
            a.B = Bs + (long long)k * NB; a.ldb = NB; a.sB = w.sB;
            a.O = Bs; a.ldo = NB; a.sO = w.sB;
            a.M = k; a.N = nb; a.K = nb; a.mode = GM_SET;
            launch_gemm<T>(a, nbox, st);
        }
        const int c0 = k + nb, nc = n + P.r - c0;
        if (nc > 0) {
            launch_gather<T>(w.M, ldm, w.sM, k, nb, c0, nc, Ps, w.sP, w.W, w.G, ldm, w.sG, nullptr, nbox, st);
            GemmArgs<T> a = gargs<T>();
            a.A = Fs; a.lda = NB; a.sA = w.sF;
            a.B = w.G; a.ldb = ldm; a.sB = w.sG;
            a.O = w.M + (long long)k * ldm + c0; a.ldo = ldm; a.sO = w.sM;
            a.M = n - k; a.N = nc; a.K = nb; a.mode = GM_FWD; a.split = nb;
            a.perm = Ps; a.sP = w.sP; a.W = w.W; a.ldw = ldm; a.sW = w.sG;
            launch_gemm<T>(a, nbox, st);
        }
    }
}

// Forward substitution L y = P b of RHS columns [c0, c0 + nc) with the stored steps.
template <typename T>
void lu_forward(const Plan& P, Work<T>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st)
{
    const int n = P.n, NB = P.NB;
    const long long ldm = P.ldm;
    for (int s = 0; s < P.nsteps; ++s) {
        const int k = P.k0[s], nb = P.nbs[s];
        T* Fs = w.F + P.fw_off[s];
        int* Ps = w.perm + P.perm_off[s];
        launch_gather<T>(w.M, ldm, w.sM, k, nb, c0, nc, Ps, w.sP, w.W, w.G, ldm, w.sG, skip, nbox, st);
        GemmArgs<T> a = gargs<T>();
        a.A = Fs; a.lda = NB; a.sA = w.sF;
        a.B = w.G; a.ldb = ldm; a.sB = w.sG;
        a.O = w.M + (long long)k * ldm + c0; a.ldo = ldm; a.sO = w.sM;
        a.M = n - k; a.N = nc; a.K = nb; a.mode = GM_FWD; a.split = nb;
        a.perm = Ps; a.sP = w.sP; a.W = w.W; a.ldw = ldm; a.sW = w.sG; a.skip = skip;
        launch_gemm<T>(a, nbox, st);
    }
}

// Backward substitution U x = y of RHS columns [c0, c0 + nc).
template <typename T>
void lu_backward(const Plan& P, Work<T>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st)
{
    const int NB = P.NB;
    const long long ldm = P.ldm;
    for (int s = P.nsteps - 1; s >= 0; --s) {
        const int k = P.k0[s], nb = P.nbs[s];
        T* Bs = w.B + P.bw_off[s];
        launch_gather<T>(w.M, ldm, w.sM, k, nb, c0, nc, nullptr, 0, nullptr, w.G, ldm, w.sG, skip, nbox, st);
        GemmArgs<T> a = gargs<T>();
        a.A = Bs; a.lda = NB; a.sA = w.sB;
        a.B = w.G; a.ldb = ldm; a.sB = w.sG;
        a.O = w.M + c0; a.ldo = ldm; a.sO = w.sM;
        a.M = k + nb; a.N = nc; a.K = nb; a.mode = GM_BWD; a.split = k; a.skip = skip;
        launch_gemm<T>(a, nbox, st);
    }
}

template void lu_factor<double>(const Plan&, Work<double>&, int, int*, cudaStream_t);
template void lu_factor<float>(const Plan&, Work<float>&, int, int*, cudaStream_t);
template void lu_forward<float>(const Plan&, Work<float>&, int, int, int, const int*, cudaStream_t);
template void lu_backward<double>(const Plan&, Work<double>&, int, int, int, const int*, cudaStream_t);
template void lu_backward<float>(const Plan&, Work<float>&, int, int, int, const int*, cudaStream_t);

}  // namespace hps

namespace {

#define HPS_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return HPS_ECUDA;             \
    } while (0)

bool valid_p(int p) { return p >= 3 && p <= kMaxP; }

hps_status get_geometry(hps_ctx* ctx, const hps_leaf_kind* kind, Geometry** out)
{
    auto key = std::make_tuple(kind->p, kind->h[0], kind->h[1], kind->h[2]);
    auto it = ctx->geoms.find(key);
    if (it != ctx->geoms.end()) { *out = &it->second; return HPS_OK; }
    Geometry g;
    g.p = kind->p;
    g.q = g.p - 2;
    g.n = g.q * g.q * g.q;
    g.m = 6 * g.q * g.q;
    const int p = g.p, pp = p * p;
    std::vector<double> Dhat(pp), D(3 * pp), D2(3 * pp);
    cheb_diff(p, Dhat.data());
    for (int a = 0; a < 3; ++a) {
        g.h[a] = kind->h[a];
        const double s = 2.0 / kind->h[a];
        for (int e = 0; e < pp; ++e) D[a * pp + e] = s * Dhat[e];
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                double acc = 0.0;
                for (int l = 0; l < p; ++l) acc += D[a * pp + i * p + l] * D[a * pp + l * p + j];
                D2[a * pp + i * p + j] = acc;
            }
    }
    HPS_CUDA_TRY(cudaMalloc(&g.dD, sizeof(double) * 3 * pp));
    HPS_CUDA_TRY(cudaMalloc(&g.dD2, sizeof(double) * 3 * pp));
    HPS_CUDA_TRY(cudaMemcpy(g.dD, D.data(), sizeof(double) * 3 * pp, cudaMemcpyHostToDevice));
    HPS_CUDA_TRY(cudaMemcpy(g.dD2, D2.data(), sizeof(double) * 3 * pp, cudaMemcpyHostToDevice));
    auto res = ctx->geoms.emplace(key, g);
    *out = &res.first->second;
    return HPS_OK;
}

hps_status ensure_workspace(hps_ctx* ctx, const Plan& P, int nbox, int* chunk)
{
    size_t limit = ctx->ws_max;
    if (limit == 0) {
        size_t fr = 0, tot = 0;
        HPS_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        limit = ctx->ws_bytes + (size_t)(0.85 * (double)fr);
    }
    if (P.per_box > limit) return HPS_ENOMEM;
    int c = (int)std::min<size_t>((size_t)nbox, limit / P.per_box);
    const size_t need = P.per_box * (size_t)c;
    if (need > ctx->ws_bytes) {
        if (ctx->ws) { cudaDeviceSynchronize(); cudaFree(ctx->ws); ctx->ws = nullptr; ctx->ws_bytes = 0; }
        if (cudaMalloc(&ctx->ws, need) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
        ctx->ws_bytes = need;
    }
    *chunk = c;
    return HPS_OK;
}

hps_status ensure_diag(hps_ctx* ctx, int nbox, cudaStream_t st)
{
    if ((size_t)nbox > ctx->diag_cap) {
        if (ctx->d_iters) { cudaFree(ctx->d_iters); cudaFree(ctx->d_relcorr); }
        HPS_CUDA_TRY(cudaMalloc(&ctx->d_iters, sizeof(int) * nbox));
        HPS_CUDA_TRY(cudaMalloc(&ctx->d_relcorr, sizeof(double) * nbox));
        ctx->diag_cap = nbox;
    }
    HPS_CUDA_TRY(cudaMemsetAsync(ctx->d_iters, 0, sizeof(int) * nbox, st));
    HPS_CUDA_TRY(cudaMemsetAsync(ctx->d_relcorr, 0, sizeof(double) * nbox, st));
    return HPS_OK;
}

// ------------------------------------------------------------ one chunk of a leaf call

struct CallSpec {
    int rhs_kind;        // RhsKind
    int r;               // RHS columns
    const double* rhs;   // f or u_b (chunk base), NULL for DTN
    long long s_rhs;     // per-box stride of rhs
    int zero_row_box;    // test hook: chunk-local box whose A_ii gets a zero row (-1: none)
};

// Solves A_ii X = B for one chunk; the FP64 solution ends in X (ld = ldx,
// per-box stride sX), in the caller's buffer or the workspace.
template <typename T>
hps_status solve_chunk(hps_ctx* ctx, const Geometry& g, const hps_leaf_kind* kind, const Plan& P,
                       Work<T>& w, int nbox, const double* b, const CallSpec& cs, double* X, long long ldx,
                       long long sX, int* status, int* iters, double* relcorr, cudaStream_t st);

template <>
hps_status solve_chunk<double>(hps_ctx*, const Geometry& g, const hps_leaf_kind* kind, const Plan& P,
                               Work<double>& w, int nbox, const double* b, const CallSpec& cs, double* X,
                               long long ldx, long long sX, int* status, int*, double*, cudaStream_t st)
{
    const long long p3 = (long long)g.p * g.p * g.p;
    launch_build_aug<double>(g, kind->kappa, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M, P.ldm, w.sM,
                             status, cs.zero_row_box, st);
    lu_factor<double>(P, w, nbox, status, st);
    lu_backward<double>(P, w, nbox, g.n, cs.r, nullptr, st);
    if (X) launch_extract<double>(w.M + g.n, P.ldm, w.sM, g.n, cs.r, X, ldx, sX, nbox, st);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

template <>
hps_status solve_chunk<float>(hps_ctx* ctx, const Geometry& g, const hps_leaf_kind* kind, const Plan& P,
                              Work<float>& w, int nbox, const double* b, const CallSpec& cs, double* X,
                              long long ldx, long long sX, int* status, int* iters, double* relcorr,
                              cudaStream_t st)
{
    const long long p3 = (long long)g.p * g.p * g.p;
    launch_build_aug<float>(g, kind->kappa, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M, P.ldm, w.sM,
                            status, cs.zero_row_box, st);
    if (P.tc) {
        tc_reset_abort(st);
        if (!tc_lu_factor(P, w, nbox, status, st)) return HPS_ECUDA;
        if (!tc_lu_backward(P, w, nbox, g.n, cs.r, nullptr, st)) return HPS_ECUDA;
    } else {
        lu_factor<float>(P, w, nbox, status, st);
        lu_backward<float>(P, w, nbox, g.n, cs.r, nullptr, st);
    }
    launch_extract<float>(w.M + g.n, P.ldm, w.sM, g.n, cs.r, X, ldx, sX, nbox, st);
    // FP64 iterative refinement: R = B - A_ii X (FP64, matrix-free), solve with
    // the FP32 factors, X += correction (FP64).
    HPS_CUDA_TRY(cudaMemsetAsync(w.skip, 0, sizeof(int) * nbox, st));
    HPS_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(double) * 2 * nbox, st));
    const int its = ctx->ir_iters;
    for (int it = 0; it < its; ++it) {
        launch_residual(g, kind->kappa, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, X, ldx, sX,
                        w.M + g.n, P.ldm, w.sM, w.skip, st);
        if (P.tc) {
            if (!tc_lu_forward(P, w, nbox, g.n, cs.r, w.skip, st)) return HPS_ECUDA;
            if (!tc_lu_backward(P, w, nbox, g.n, cs.r, w.skip, st)) return HPS_ECUDA;
        } else {
            lu_forward<float>(P, w, nbox, g.n, cs.r, w.skip, st);
            lu_backward<float>(P, w, nbox, g.n, cs.r, w.skip, st);
        }
        launch_ir_update(w.M + g.n, P.ldm, w.sM, g.n, cs.r, X, ldx, sX, w.norms, w.skip, nbox, st);
        launch_ir_check(nbox, w.norms, ctx->ir_tol, it == its - 1, w.skip, iters, relcorr, status, st);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status check_kind(const hps_leaf_kind* kind)
{
    if (!kind || !valid_p(kind->p)) return HPS_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(kind->h[a] > 0.0) || !std::isfinite(kind->h[a])) return HPS_EINVAL;
    if (!std::isfinite(kind->kappa)) return HPS_EINVAL;
    return HPS_OK;
}

hps_status finish(hps_ctx* ctx, int nbox, int* box_status, cudaStream_t st)
{
    if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
    ctx->last_nbox = nbox;
    ctx->last_stream = st;
    if (!ctx->sync) return HPS_OK;
    HPS_CUDA_TRY(cudaStreamSynchronize(st));
    if (box_status && nbox > 0) {
        std::vector<int> h(nbox);
        HPS_CUDA_TRY(cudaMemcpy(h.data(), box_status, sizeof(int) * nbox, cudaMemcpyDeviceToHost));
        for (int v : h)
            if (v) return (hps_status)v;
    }
    return HPS_OK;
}

// Generic driver: chunks the batch and runs solve_chunk, then `post` per chunk.
template <typename T, typename Post>
hps_status run_solve(hps_ctx* ctx, const Geometry& g, const hps_leaf_kind* kind, hps_precision prec, int nbox,
                     const double* b, int rhs_kind, int r, const double* rhs, long long s_rhs, double* Xuser,
                     long long ldx_user, long long sX_user, int* box_status, cudaStream_t st, Post post)
{
    const bool need_x = (prec != HPS_FP64) && !Xuser;
    Plan P = make_plan(g.n, r, prec, ctx->nb_opt, ctx->use_tc != 0, need_x || prec == HPS_FP64);
    int chunk = 0;
    hps_status rc = ensure_workspace(ctx, P, nbox, &chunk);
    if (rc != HPS_OK) return rc;
    rc = ensure_diag(ctx, nbox, st);
    if (rc != HPS_OK) return rc;
    int* status = box_status;
    const long long p3 = (long long)g.p * g.p * g.p;
    for (int b0 = 0; b0 < nbox; b0 += chunk) {
        const int nc = std::min(chunk, nbox - b0);
        Work<T> w = carve<T>(P, ctx->ws, nc);
        int* stc = status + b0;
        double* X;
        long long ldx, sX;
        if (Xuser) { X = Xuser + (long long)b0 * sX_user; ldx = ldx_user; sX = sX_user; }
        else { X = w.X; ldx = r; sX = w.sX; }
        const int zr = (ctx->zero_row_box >= b0 && ctx->zero_row_box < b0 + nc) ? ctx->zero_row_box - b0 : -1;
        CallSpec cs{rhs_kind, r, rhs ? rhs + (long long)b0 * s_rhs : nullptr, s_rhs, zr};
        rc = solve_chunk<T>(ctx, g, kind, P, w, nc, b + (long long)b0 * p3, cs, X, ldx, sX, stc,
                            ctx->d_iters + b0, ctx->d_relcorr + b0, st);
        if (rc != HPS_OK) return rc;
        post(b0, nc, X, ldx, sX);
        if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
    }
    return HPS_OK;
}

struct ProfScope {
    explicit ProfScope(hps_ctx* c) { hps::t_prof = c->prof_on ? &c->prof : nullptr; }
    ~ProfScope() { hps::t_prof = nullptr; }
};

struct StatusBuf {
    int* ptr = nullptr;
    bool owned = false;
    ~StatusBuf() { if (owned) cudaFree(ptr); }
};

hps_status prepare_status(int* user, int nbox, cudaStream_t st, StatusBuf& sb)
{
    if (user) sb.ptr = user;
    else {
        HPS_CUDA_TRY(cudaMalloc(&sb.ptr, sizeof(int) * (nbox > 0 ? nbox : 1)));
        sb.owned = true;
    }
    HPS_CUDA_TRY(cudaMemsetAsync(sb.ptr, 0, sizeof(int) * nbox, st));
    return HPS_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

const char* hps_status_string(hps_status s)
{
    switch (s) {
    case HPS_OK: return "ok";
    case HPS_EINVAL: return "invalid argument or non-finite input";
    case HPS_ENOMEM: return "workspace limit too small or device allocation failed";
    case HPS_ESINGULAR: return "zero pivot: A_ii is singular";
    case HPS_ENOCONV: return "iterative refinement did not converge";
    case HPS_ECUDA: return "CUDA runtime error";
    case HPS_ETIMEOUT: return "bounded device wait gave up";
    }
    return "unknown status";
}

hps_status hps_leaf_sizes(int p, int* n, int* m)
{
    if (!valid_p(p) || !n || !m) return HPS_EINVAL;
    const int q = p - 2;
    *n = q * q * q;
    *m = 6 * q * q;
    return HPS_OK;
}

hps_status hps_leaf_nodes(int p, const double lo[3], const double h[3], double* xyz)
{
    if (!valid_p(p) || !lo || !h || !xyz) return HPS_EINVAL;
    double t[kMaxP];
    cheb_nodes(p, t);
    for (int k = 0; k < p; ++k)
        for (int j = 0; j < p; ++j)
            for (int i = 0; i < p; ++i) {
                const int gi = i + p * j + p * p * k;
                xyz[3 * gi + 0] = lo[0] + 0.5 * h[0] * (t[i] + 1.0);
                xyz[3 * gi + 1] = lo[1] + 0.5 * h[1] * (t[j] + 1.0);
                xyz[3 * gi + 2] = lo[2] + 0.5 * h[2] * (t[k] + 1.0);
            }
    return HPS_OK;
}

size_t hps_workspace_per_box(int p, hps_precision prec)
{
    if (!valid_p(p)) return 0;
    const int q = p - 2, n = q * q * q, m = 6 * q * q;
    return make_plan(n, m, prec, 0, true, prec != HPS_FP64).per_box;
}

hps_status hps_create(hps_ctx** out, int device, size_t workspace_bytes_max)
{
    if (!out) return HPS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return HPS_ECUDA; }
    if (device < 0 || device >= ndev) return HPS_EINVAL;
    HPS_CUDA_TRY(cudaSetDevice(device));
    hps_ctx* c = new (std::nothrow) hps_ctx();
    if (!c) return HPS_ENOMEM;
    c->device = device;
    c->ws_max = workspace_bytes_max;
    if (const char* e = std::getenv("HPS_TENSOR_CORES")) c->use_tc = std::atoi(e) != 0;
    *out = c;
    return HPS_OK;
}

void hps_destroy(hps_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    for (auto& kv : ctx->geoms) { cudaFree(kv.second.dD); cudaFree(kv.second.dD2); }
    if (ctx->d_iters) cudaFree(ctx->d_iters);
    if (ctx->d_relcorr) cudaFree(ctx->d_relcorr);
    for (auto& r : ctx->prof.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    delete ctx;
}

hps_status hps_set_option(hps_ctx* ctx, int option, double value)
{
    if (!ctx || !std::isfinite(value)) return HPS_EINVAL;
    switch (option) {
    case HPS_OPT_IR_MAX_ITERS:
        if (value < 0 || value > 20) return HPS_EINVAL;
        ctx->ir_iters = (int)value;
        return HPS_OK;
    case HPS_OPT_IR_TOL:
        if (!(value > 0)) return HPS_EINVAL;
        ctx->ir_tol = value;
        return HPS_OK;
    case HPS_OPT_BLOCK:
        if (!(value == 0 || value == 32 || value == 64 || value == 128)) return HPS_EINVAL;
        ctx->nb_opt = (int)value;
        return HPS_OK;
    case HPS_OPT_TENSOR_CORES:
        ctx->use_tc = value != 0;
        return HPS_OK;
    case HPS_OPT_SYNC:
        ctx->sync = value != 0;
        return HPS_OK;
    case HPS_OPT_TEST_SINGULAR_BOX:
        ctx->zero_row_box = (int)value;
        return HPS_OK;
    }
    return HPS_EINVAL;
}

hps_status hps_leaf_build_dtn(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, const double* b, double* T,
                              double* S, hps_precision prec, int* box_status, void* stream)
{
    if (!ctx || nbox < 0) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || !T) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    rc = get_geometry(ctx, kind, &g);
    if (rc != HPS_OK) return rc;
    StatusBuf sbuf;
    rc = prepare_status(box_status, nbox, st, sbuf);
    if (rc != HPS_OK) return rc;
    const int n = g->n, m = g->m;
    auto post = [&](int b0, int nc, double* X, long long ldx, long long sX) {
        launch_dn(*g, nc, X, ldx, sX, m, T + (long long)b0 * m * m, (long long)m * m, 0, 1, st);
    };
    if (prec == HPS_FP64) {
        // FP64: the solution stays in the working matrix; S (if wanted) is copied out.
        rc = run_solve<double>(ctx, *g, kind, prec, nbox, b, RHS_DTN, m, nullptr, 0, S, m, (long long)n * m,
                               sbuf.ptr, st, post);
    } else {
        rc = run_solve<float>(ctx, *g, kind, prec, nbox, b, RHS_DTN, m, nullptr, 0, S, m, (long long)n * m,
                              sbuf.ptr, st, post);
    }
    if (rc != HPS_OK) return rc;
    return finish(ctx, nbox, box_status, st);
}

hps_status hps_leaf_particular(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs, const double* b,
                               const double* f, double* v, double* h, hps_precision prec, int* box_status,
                               void* stream)
{
    if (!ctx || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || !f || !v || !h) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    rc = get_geometry(ctx, kind, &g);
    if (rc != HPS_OK) return rc;
    StatusBuf sbuf;
    rc = prepare_status(box_status, nbox, st, sbuf);
    if (rc != HPS_OK) return rc;
    const int n = g->n, m = g->m;
    const long long p3 = (long long)g->p * g->p * g->p;
    auto post = [&](int b0, int nc, double* X, long long ldx, long long sX) {
        launch_transpose_add(X, ldx, sX, n, nrhs, nullptr, v + (long long)b0 * nrhs * n, nc, st);
        launch_dn(*g, nc, X, ldx, sX, nrhs, h + (long long)b0 * nrhs * m, (long long)nrhs * m, 1, 0, st);
    };
    if (prec == HPS_FP64)
        rc = run_solve<double>(ctx, *g, kind, prec, nbox, b, RHS_LOAD, nrhs, f, nrhs * p3, nullptr, 0, 0, sbuf.ptr,
                               st, post);
    else
        rc = run_solve<float>(ctx, *g, kind, prec, nbox, b, RHS_LOAD, nrhs, f, nrhs * p3, nullptr, 0, 0, sbuf.ptr,
                              st, post);
    if (rc != HPS_OK) return rc;
    return finish(ctx, nbox, box_status, st);
}

hps_status hps_leaf_reconstruct(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs, const double* b,
                                const double* S, const double* v, const double* ub, double* ui,
                                hps_precision prec, int* box_status, void* stream)
{
    if (!ctx || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!ub || !ui || (!S && !b)) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    rc = get_geometry(ctx, kind, &g);
    if (rc != HPS_OK) return rc;
    StatusBuf sbuf;
    rc = prepare_status(box_status, nbox, st, sbuf);
    if (rc != HPS_OK) return rc;
    const int n = g->n, m = g->m;
    if (S) {
        launch_recon_stored(S, n, m, nrhs, v, ub, ui, nbox, st);
        return finish(ctx, nbox, box_status, st);
    }
    auto post = [&](int b0, int nc, double* X, long long ldx, long long sX) {
        launch_transpose_add(X, ldx, sX, n, nrhs, v ? v + (long long)b0 * nrhs * n : nullptr,
                             ui + (long long)b0 * nrhs * n, nc, st);
    };
    if (prec == HPS_FP64)
        rc = run_solve<double>(ctx, *g, kind, prec, nbox, b, RHS_TRACE, nrhs, ub, (long long)nrhs * m, nullptr, 0,
                               0, sbuf.ptr, st, post);
    else
        rc = run_solve<float>(ctx, *g, kind, prec, nbox, b, RHS_TRACE, nrhs, ub, (long long)nrhs * m, nullptr, 0,
                              0, sbuf.ptr, st, post);
    if (rc != HPS_OK) return rc;
    return finish(ctx, nbox, box_status, st);
}

hps_status hps_profile_enable(hps_ctx* ctx, int on)
{
    if (!ctx) return HPS_EINVAL;
    ctx->prof_on = on != 0;
    return HPS_OK;
}

hps_status hps_profile_reset(hps_ctx* ctx)
{
    if (!ctx) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    hps::prof_resolve(&ctx->prof);
    for (int c = 0; c < KC_COUNT; ++c) {
        ctx->prof.launches[c] = 0;
        ctx->prof.ms[c] = ctx->prof.flops[c] = ctx->prof.bytes[c] = 0.0;
    }
    return HPS_OK;
}

hps_status hps_profile_get(hps_ctx* ctx, int cls, long long* launches, double* ms, double* flops, double* bytes)
{
    if (!ctx || cls < 0 || cls >= KC_COUNT) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    hps::prof_resolve(&ctx->prof);
    if (launches) *launches = ctx->prof.launches[cls];
    if (ms) *ms = ctx->prof.ms[cls];
    if (flops) *flops = ctx->prof.flops[cls];
    if (bytes) *bytes = ctx->prof.bytes[cls];
    return HPS_OK;
}

hps_status hps_last_refinement(hps_ctx* ctx, int nbox, int* iters, double* rel_correction)
{
    if (!ctx || nbox < 0 || nbox > ctx->last_nbox) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    HPS_CUDA_TRY(cudaStreamSynchronize(ctx->last_stream));
    if (iters) HPS_CUDA_TRY(cudaMemcpy(iters, ctx->d_iters, sizeof(int) * nbox, cudaMemcpyDeviceToHost));
    if (rel_correction)
        HPS_CUDA_TRY(cudaMemcpy(rel_correction, ctx->d_relcorr, sizeof(double) * nbox, cudaMemcpyDeviceToHost));
    return HPS_OK;
}

}  // extern "C"
