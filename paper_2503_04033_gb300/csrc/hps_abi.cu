// C ABI of the HPS leaf library: context, workspace, per-(p, h) operator
// tables, LU plans, and the launch sequences of the build and solve stages.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
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

// One tuned LU schedule: block NB, unit length, widest tensor-core tile.
struct TuneChoice {
    int nb = 0, unit = 0, bn = 0;
};

struct hps_ctx {
    int device = 0;
    size_t ws_max = 0;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::map<std::tuple<int, double, double, double>, Geometry> geoms;
    int ir_iters = 8;
    double ir_tol = 1e-11;
    int nb_opt = 0;
    int tc_epi_cp = 0;          // 1: tcgen05 epilogue always in the cp.async form
    int lu_unit = 4;            // tcgen05 path: LU steps joined into units of up to this many (1, 2, 4, 8)
    int tc_fuse = -1;           // -1: fused gathers where they measured faster, 0: never, 1: backward sweeps
    int res_df = 3;             // residual precision (HPS_OPT_RESIDUAL_DF): double-float, routed per box
    int fp16_ops = 1;           // FP32_IR tensor-core products on scaled 2 x FP16 operands (format 2)
    int concurrent = 1;         // HPS_OPT_GROUPS_CONCURRENT: the groups of a mixed batch on their own streams
    std::vector<cudaStream_t> side;   // one stream per group of a concurrent mixed batch
    std::vector<cudaEvent_t> side_done;
    cudaEvent_t side_fork = nullptr;
    std::vector<size_t> ws_off;       // workspace offset of each job of the current call (concurrent layout)
    int use_tc = 1;
    int sync = 0;
    int zero_row_box = -1;
    bool prof_on = false;
    hps::Profiler prof;
    int autotune = 0;
    int graphs = 0;
    std::map<std::tuple<int, int, int>, TuneChoice> tuned;  // (p, precision, tensor cores) -> schedule
    std::map<std::string, cudaGraphExec_t> graph_cache;     // captured calls
    int* d_iters = nullptr;
    double* d_relcorr = nullptr;
    size_t diag_cap = 0;
    double* d_kappa = nullptr;
    size_t kappa_cap = 0;
    int* d_status = nullptr;
    size_t status_cap = 0;
    cudaStream_t cap_stream = nullptr;     // stream used only for graph capture
    std::map<std::tuple<int, double, double, double, double>, float*> a0inv;   // gate preconditioners
    void* gate_buf = nullptr;
    size_t gate_cap = 0;
    int last_nbox = 0;
    cudaStream_t last_stream = nullptr;
    std::mutex mu;
};

// A stored factorisation of every box's A_ii (hps_leaf_factor): the workspace
// of one chunk holding all the boxes, kept between calls.
struct hps_leaf_factors {
    hps_ctx* ctx = nullptr;
    hps::Geometry* g = nullptr;
    hps::Plan P;
    hps_precision prec = HPS_FP64;
    int nbox = 0, nrhs_max = 0;
    double kappa = 0.0;
    void* buf = nullptr;            // the chunk workspace (factors, operator copies, kappa^2 b, solve buffers)
    int* d_fstatus = nullptr;       // per box: status of the factorisation
    int* d_status = nullptr;        // per box: status of the last solve when the caller passes none
    int* d_iters = nullptr;         // refinement diagnostics of the last solve
    double* d_relcorr = nullptr;
    double* beta = nullptr;         // copy of the first-order field [nbox][3][p^3], or NULL
    std::map<std::string, cudaGraphExec_t> graphs;   // captured solves (HPS_OPT_GRAPHS)
};

namespace hps {

int ctx_device(const hps_ctx* ctx) { return ctx->device; }

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
template void lu_forward<double>(const Plan&, Work<double>&, int, int, int, const int*, cudaStream_t);
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

hps_status get_geometry(hps_ctx* ctx, int p, const double h[3], Geometry** out)
{
    auto key = std::make_tuple(p, h[0], h[1], h[2]);
    auto it = ctx->geoms.find(key);
    if (it != ctx->geoms.end()) { *out = &it->second; return HPS_OK; }
    Geometry g;
    g.p = p;
    g.q = g.p - 2;
    g.n = g.q * g.q * g.q;
    g.m = 6 * g.q * g.q;
    const int pp = p * p;
    std::vector<double> Dhat(pp), D(3 * pp), D2(3 * pp);
    cheb_diff(p, Dhat.data());
    for (int a = 0; a < 3; ++a) g.h[a] = h[a];
    geometry_tables(p, Dhat.data(), g.h, D.data(), D2.data());
    HPS_CUDA_TRY(cudaMalloc(&g.dD, sizeof(double) * 3 * pp));
    HPS_CUDA_TRY(cudaMalloc(&g.dD2, sizeof(double) * 3 * pp));
    HPS_CUDA_TRY(cudaMemcpy(g.dD, D.data(), sizeof(double) * 3 * pp, cudaMemcpyHostToDevice));
    HPS_CUDA_TRY(cudaMemcpy(g.dD2, D2.data(), sizeof(double) * 3 * pp, cudaMemcpyHostToDevice));
    // Double-float line tables of the first residual: the even/odd (E, O)
    // pairs, the odd-q middle entries and the boundary couplings of each axis,
    // every value split as hi = float(v), lo = float(v - hi).
    {
        const int q = g.q, H = q / 2, TF = df_tab_f4(q);
        std::vector<float> DF((size_t)3 * TF * 4, 0.0f);
        auto split = [](double v, float* o) {
            o[0] = (float)v;
            o[1] = (float)(v - (double)o[0]);
        };
        for (int a = 0; a < 3; ++a) {
            const double* Dm = D2.data() + (size_t)a * pp;
            float* t = DF.data() + (size_t)a * TF * 4;
            for (int i = 0; i < H; ++i)
                for (int l = 0; l < H; ++l) {
                    const double u = Dm[(i + 1) * p + (l + 1)], w = Dm[(i + 1) * p + (p - 2 - l)];
                    split(0.5 * (u + w), t + 4 * (i * H + l));
                    split(0.5 * (u - w), t + 4 * (i * H + l) + 2);
                }
            int off = 4 * H * H;
            if (q & 1) {
                const int mid = H + 1;
                for (int i = 0; i < H; ++i) split(Dm[(i + 1) * p + mid], t + off + 2 * i);
                for (int l = 0; l < H; ++l)
                    split(0.5 * (Dm[mid * p + (l + 1)] + Dm[mid * p + (p - 2 - l)]), t + off + 2 * H + 2 * l);
                split(Dm[mid * p + mid], t + off + 4 * H);
                off += 4 * (H + 1);
            }
            for (int i = 1; i <= q; ++i) {
                split(Dm[i * p], t + off + 4 * (i - 1));
                split(Dm[i * p + p - 1], t + off + 4 * (i - 1) + 2);
            }
        }
        HPS_CUDA_TRY(cudaMalloc(&g.dDF, sizeof(float) * DF.size()));
        HPS_CUDA_TRY(cudaMemcpy(g.dDF, DF.data(), sizeof(float) * DF.size(), cudaMemcpyHostToDevice));
    }
    auto res = ctx->geoms.emplace(key, g);
    *out = &res.first->second;
    return HPS_OK;
}

void clear_graphs(hps_ctx* ctx)
{
    for (auto& kv : ctx->graph_cache) cudaGraphExecDestroy(kv.second);
    ctx->graph_cache.clear();
}

// ------------------------------------------------------------ jobs

// One homogeneous batch of a call: boxes of one order p and size h, with a
// common wavenumber or one per box, and one kind of right-hand side.
struct Job {
    const Geometry* g = nullptr;
    int nbox = 0;
    double kappa = 0.0;
    const double* kappa_dev = nullptr;   // device [nbox]: per-box wavenumber (NULL: kappa)
    const double* b = nullptr;
    int rhs_kind = RHS_DTN;
    int nload = 0;                       // load columns (LOAD, DTN_LOAD) or trace columns (TRACE)
    const double* rhs = nullptr;         // f [nbox][nload][p^3] or u_b [nbox][nload][m]
    double* T = nullptr;
    double* S = nullptr;
    double* v = nullptr;
    double* hf = nullptr;
    double* ui = nullptr;
    const double* vadd = nullptr;
    int* status = nullptr;               // device [nbox]
    int diag_off = 0;                    // offset into the refinement diagnostics
    int nb = 0;                          // LU block (0: context default)
    int unit = 0;                        // LU unit length (0: context default)
    int bn = 0;                          // widest tensor-core tile (0: 256)
    int zero_row_box = -1;               // test hook
    const double* beta = nullptr;        // device [nbox][3][p^3]: first-order term div(beta u), or NULL
};

int job_cols(const Job& j)
{
    if (j.rhs_kind == RHS_DTN) return j.g->m;
    if (j.rhs_kind == RHS_DTN_LOAD) return j.g->m + j.nload;
    return j.nload;
}

long long job_srhs(const Job& j)
{
    const long long p3 = (long long)j.g->p * j.g->p * j.g->p;
    if (j.rhs_kind == RHS_LOAD || j.rhs_kind == RHS_DTN_LOAD) return j.nload * p3;
    if (j.rhs_kind == RHS_TRACE) return (long long)j.nload * j.g->m;
    return 0;
}

Plan job_plan(const hps_ctx* ctx, const Job& j, hps_precision prec)
{
    Plan P = make_plan(j.g->n, job_cols(j), prec, j.nb ? j.nb : ctx->nb_opt, ctx->use_tc != 0, prec != HPS_FP64,
                       j.unit ? j.unit : ctx->lu_unit, ctx->fp16_ops != 0);
    P.bn_max = j.bn ? j.bn : 256;
    P.tma_epi = ctx->tc_epi_cp == 0;
    if (ctx->tc_fuse >= 0) P.fuse_bwd = P.tc && ctx->tc_fuse != 0;
    if (P.fmt == 2) P.fuse_bwd = false;   // the fused gather writes unscaled operands
    return P;
}

// Sizes the workspace for the largest chunk any job will run; all device
// allocation of a call happens here, before any launch is enqueued.
hps_status ensure_workspace(hps_ctx* ctx, const std::vector<Plan>& plans, const std::vector<Job>& jobs,
                            std::vector<int>& chunk)
{
    size_t limit = ctx->ws_max;
    if (limit == 0) {
        size_t fr = 0, tot = 0;
        HPS_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        limit = ctx->ws_bytes + (size_t)(0.85 * (double)fr);
    }
    size_t need = 0;
    chunk.assign(jobs.size(), 0);
    ctx->ws_off.assign(jobs.size(), 0);
    // Concurrent layout (several groups): every job whole, in its own slice,
    // when all of them fit at once; else one slice reused job after job.
    if (ctx->concurrent && jobs.size() > 1) {
        size_t sum = 0;
        for (size_t i = 0; i < jobs.size(); ++i) {
            ctx->ws_off[i] = sum;
            sum += align_up(plans[i].per_box * (size_t)jobs[i].nbox, 256);
        }
        if (sum <= limit) {
            for (size_t i = 0; i < jobs.size(); ++i) chunk[i] = jobs[i].nbox;
            need = sum;
        } else {
            ctx->ws_off.assign(jobs.size(), 0);
        }
    }
    if (need == 0)
        for (size_t i = 0; i < jobs.size(); ++i) {
            if (plans[i].per_box > limit) return HPS_ENOMEM;
            chunk[i] = (int)std::min<size_t>((size_t)jobs[i].nbox, limit / plans[i].per_box);
            need = std::max(need, plans[i].per_box * (size_t)chunk[i]);
        }
    // streams and events of a concurrent call (created before any capture)
    const bool conc = jobs.size() > 1 && ctx->ws_off.back() > 0;
    if (conc) {
        if (!ctx->side_fork) HPS_CUDA_TRY(cudaEventCreateWithFlags(&ctx->side_fork, cudaEventDisableTiming));
        while (ctx->side.size() < jobs.size()) {
            cudaStream_t sst = nullptr;
            cudaEvent_t ev = nullptr;
            HPS_CUDA_TRY(cudaStreamCreateWithFlags(&sst, cudaStreamNonBlocking));
            ctx->side.push_back(sst);
            HPS_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            ctx->side_done.push_back(ev);
        }
    }
    if (need > ctx->ws_bytes) {
        if (ctx->ws) {
            cudaDeviceSynchronize();
            cudaFree(ctx->ws);
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
            clear_graphs(ctx);
        }
        if (cudaMalloc(&ctx->ws, need) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
        ctx->ws_bytes = need;
    }
    return HPS_OK;
}

template <typename T>
hps_status grow(T** p, size_t* cap, size_t count)
{
    if (count <= *cap) return HPS_OK;
    if (*p) { cudaDeviceSynchronize(); cudaFree(*p); *p = nullptr; *cap = 0; }
    HPS_CUDA_TRY(cudaMalloc(p, sizeof(T) * count));
    *cap = count;
    return HPS_OK;
}

// ------------------------------------------------------------ one chunk of a job

struct CallSpec {
    int rhs_kind;               // RhsKind
    int r;                      // RHS columns
    const double* rhs;          // f or u_b (chunk base), NULL for DTN
    long long s_rhs;            // per-box stride of rhs
    int zero_row_box;           // test hook: chunk-local box whose A_ii gets a zero row (-1: none)
    const double* kappa_dev;    // chunk base of the per-box wavenumbers, or NULL
    double kappa;
    const double* beta = nullptr;   // chunk base of the first-order field [box][3][p^3], or NULL
};

// Solves A_ii X = B for one chunk.  FP64: the solution stays in M's RHS
// columns.  FP32 + refinement: the FP64 solution is written to X.
template <typename T>
hps_status solve_chunk(hps_ctx* ctx, const Geometry& g, const CallSpec& cs, const Plan& P, Work<T>& w, int nbox,
                       const double* b, double* X, long long ldx, long long sX, int* status, int* iters,
                       double* relcorr, cudaStream_t st);

template <>
hps_status solve_chunk<double>(hps_ctx*, const Geometry& g, const CallSpec& cs, const Plan& P, Work<double>& w,
                               int nbox, const double* b, double*, long long, long long, int* status, int*, double*,
                               cudaStream_t st)
{
    const long long p3 = (long long)g.p * g.p * g.p;
    launch_build_aug<double>(g, cs.kappa, cs.kappa_dev, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M, P.ldm,
                             w.sM, status, cs.zero_row_box, st, cs.beta);
    lu_factor<double>(P, w, nbox, status, st);
    lu_backward<double>(P, w, nbox, g.n, cs.r, nullptr, st);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status refine_chunk(hps_ctx* ctx, const Geometry& g, const CallSpec& cs, const Plan& P, Work<float>& w, int nbox,
                        const double* b, double* X, long long ldx, long long sX, int* status, int* iters,
                        double* relcorr, cudaStream_t st, bool have_kb);

template <>
hps_status solve_chunk<float>(hps_ctx* ctx, const Geometry& g, const CallSpec& cs, const Plan& P, Work<float>& w,
                              int nbox, const double* b, double* X, long long ldx, long long sX, int* status,
                              int* iters, double* relcorr, cudaStream_t st)
{
    const long long p3 = (long long)g.p * g.p * g.p;
    launch_build_aug<float>(g, cs.kappa, cs.kappa_dev, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M, P.ldm,
                            w.sM, status, cs.zero_row_box, st, cs.beta);
    if (P.tc) {
        tc_reset_abort(st);
        if (!tc_lu_factor(P, w, nbox, status, st)) return HPS_ECUDA;
        if (!tc_lu_backward(P, w, nbox, g.n, cs.r, nullptr, st)) return HPS_ECUDA;
    } else {
        lu_factor<float>(P, w, nbox, status, st);
        lu_backward<float>(P, w, nbox, g.n, cs.r, nullptr, st);
    }
    return refine_chunk(ctx, g, cs, P, w, nbox, b, X, ldx, sX, status, iters, relcorr, st, false);
}

// FP64 iterative refinement of the first solution in M's right-hand-side
// columns: R = B - A_ii X (FP64, matrix-free), solve with the FP32 factors,
// X += correction (FP64).  ||X|| for the stopping rule is taken once, from
// the first solution.  have_kb: kappa^2 b (and its split) is already in w.kb
// (a stored factorisation), b is then not read.
hps_status refine_chunk(hps_ctx* ctx, const Geometry& g, const CallSpec& cs, const Plan& P, Work<float>& w, int nbox,
                        const double* b, double* X, long long ldx, long long sX, int* status, int* iters,
                        double* relcorr, cudaStream_t st, bool have_kb)
{
    const long long p3 = (long long)g.p * g.p * g.p;
    HPS_CUDA_TRY(cudaMemsetAsync(w.skip, 0, sizeof(int) * nbox, st));
    HPS_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(double) * 2 * nbox, st));
    launch_extract<float>(w.M + g.n, P.ldm, w.sM, g.n, cs.r, X, ldx, sX, nbox, st, w.norms);
    const int its = ctx->ir_iters;
    // The first residual, of the FP32 solution itself, may run in double-float:
    // with res_df = 1 when at least one FP64-residual correction follows it
    // (which then ends the refinement), with res_df = 2 always, the stopping
    // rule then counting the double-float floor (kDfFloor) in its prediction.
    const bool df = ctx->res_df && its >= (ctx->res_df >= 2 ? 1 : 2) && g.dDF && residual_df_fits(g, false) &&
                    !cs.beta;   // the double-float form has no first-order term
    if (its > 0 && !have_kb) launch_kappa_b(g, cs.kappa, cs.kappa_dev, nbox, b, p3, w.kb, df ? w.kbs : nullptr, st);
    // With res_df = 3 the workspace's per-box flag area (four ints per box)
    // holds, after skip, the residual route and the two kernels' skip flags.
    const bool df3 = df && ctx->res_df == 3 && residual_df_fits(g, true);   // else every later one in FP64
    int* route = w.skip + nbox;
    int* skip_df = w.skip + 2 * nbox;
    int* skip_64 = w.skip + 3 * nbox;
    for (int it = 0; it < its; ++it) {
        if (df && it == 0)
            launch_residual_df(g, nbox, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M + g.n, P.ldm, w.sM, w.kbs, w.skip,
                               st);
        else if (df3) {   // routed by k_ir_check: double-float for well-conditioned boxes, FP64 for the rest
            launch_residual_df(g, nbox, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, w.M + g.n, P.ldm, w.sM, w.kbs, skip_df,
                               st, X, ldx, sX);
            launch_residual(g, cs.kappa, cs.kappa_dev, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, X, ldx, sX,
                            w.M + g.n, P.ldm, w.sM, skip_64, st, w.kb, cs.beta);
        } else
            launch_residual(g, cs.kappa, cs.kappa_dev, nbox, b, p3, cs.rhs_kind, cs.r, cs.rhs, cs.s_rhs, X, ldx, sX,
                            w.M + g.n, P.ldm, w.sM, w.skip, st, w.kb, cs.beta);
        if (P.tc) {
            if (!tc_lu_forward(P, w, nbox, g.n, cs.r, w.skip, st)) return HPS_ECUDA;
            if (!tc_lu_backward(P, w, nbox, g.n, cs.r, w.skip, st)) return HPS_ECUDA;
        } else {
            lu_forward<float>(P, w, nbox, g.n, cs.r, w.skip, st);
            lu_backward<float>(P, w, nbox, g.n, cs.r, w.skip, st);
        }
        launch_ir_update(w.M + g.n, P.ldm, w.sM, g.n, cs.r, X, ldx, sX, w.norms, w.skip, nbox, st);
        const bool df_it = df && it == 0;
        launch_ir_check(nbox, w.norms, ctx->ir_tol, it == its - 1, w.skip, iters, relcorr, status, st,
                        df_it && ctx->res_df == 1, df_it && ctx->res_df >= 2 ? kDfFloor : 0.0, df3 ? kDfGate : 0.0,
                        route, skip_df, skip_64);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// Everything a job enqueues: per chunk, the solve and the products that turn
// the solution X into the requested outputs (T, S, v, h, u_i).
template <typename T>
hps_status enqueue_job(hps_ctx* ctx, const Job& j, const Plan& P, int chunk, cudaStream_t st, void* ws)
{
    const Geometry& g = *j.g;
    const int n = g.n, m = g.m, r = job_cols(j);
    const long long p3 = (long long)g.p * g.p * g.p, s_rhs = job_srhs(j);
    for (int b0 = 0; b0 < j.nbox; b0 += chunk) {
        const int nc = std::min(chunk, j.nbox - b0);
        Work<T> w = carve<T>(P, ws, nc);
        CallSpec cs;
        cs.rhs_kind = j.rhs_kind;
        cs.r = r;
        cs.rhs = j.rhs ? j.rhs + (long long)b0 * s_rhs : nullptr;
        cs.s_rhs = s_rhs;
        cs.zero_row_box = (j.zero_row_box >= b0 && j.zero_row_box < b0 + nc) ? j.zero_row_box - b0 : -1;
        cs.kappa_dev = j.kappa_dev ? j.kappa_dev + b0 : nullptr;
        cs.kappa = j.kappa;
        cs.beta = j.beta ? j.beta + (long long)b0 * 3 * p3 : nullptr;
        double* X;
        long long ldx, sX;
        if (P.elt == 8) {
            X = reinterpret_cast<double*>(w.M) + n;
            ldx = P.ldm;
            sX = w.sM;
        } else {
            X = w.X;
            ldx = r;
            sX = w.sX;
        }
        hps_status rc = solve_chunk<T>(ctx, g, cs, P, w, nc, j.b + (long long)b0 * p3, X, ldx, sX, j.status + b0,
                                       ctx->d_iters + j.diag_off + b0, ctx->d_relcorr + j.diag_off + b0, st);
        if (rc != HPS_OK) return rc;
        if (j.rhs_kind == RHS_DTN || j.rhs_kind == RHS_DTN_LOAD) {
            launch_dn(g, nc, X, ldx, sX, m, j.T + (long long)b0 * m * m, (long long)m * m, 0, 1, st);
            if (j.S) launch_extract<double>(X, ldx, sX, n, m, j.S + (long long)b0 * n * m, m, (long long)n * m, nc, st);
        }
        if (j.rhs_kind == RHS_LOAD || j.rhs_kind == RHS_DTN_LOAD) {
            const int off = j.rhs_kind == RHS_DTN_LOAD ? m : 0;
            launch_transpose_add(X + off, ldx, sX, n, j.nload, nullptr, j.v + (long long)b0 * j.nload * n, nc, st);
            launch_dn(g, nc, X + off, ldx, sX, j.nload, j.hf + (long long)b0 * j.nload * m, (long long)j.nload * m, 1,
                      0, st);
        }
        if (j.rhs_kind == RHS_TRACE)
            launch_transpose_add(X, ldx, sX, n, j.nload, j.vadd ? j.vadd + (long long)b0 * j.nload * n : nullptr,
                                 j.ui + (long long)b0 * j.nload * n, nc, st);
        if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
    }
    return HPS_OK;
}

hps_status enqueue_all(hps_ctx* ctx, const std::vector<Job>& jobs, const std::vector<Plan>& plans,
                       const std::vector<int>& chunk, hps_precision prec, int total, cudaStream_t st)
{
    HPS_CUDA_TRY(cudaMemsetAsync(ctx->d_iters, 0, sizeof(int) * total, st));
    HPS_CUDA_TRY(cudaMemsetAsync(ctx->d_relcorr, 0, sizeof(double) * total, st));
    for (const Job& j : jobs) HPS_CUDA_TRY(cudaMemsetAsync(j.status, 0, sizeof(int) * j.nbox, st));
    // Groups of a mixed batch run concurrently, each on its own stream and
    // workspace slice (ensure_workspace chose the layout), joined back to st.
    const bool conc = jobs.size() > 1 && ctx->ws_off.size() == jobs.size() && ctx->ws_off.back() > 0 &&
                      ctx->side.size() >= jobs.size();
    if (conc) HPS_CUDA_TRY(cudaEventRecord(ctx->side_fork, st));
    for (size_t i = 0; i < jobs.size(); ++i) {
        cudaStream_t js = conc ? ctx->side[i] : st;
        void* ws = static_cast<char*>(ctx->ws) + (conc ? ctx->ws_off[i] : 0);
        if (conc) HPS_CUDA_TRY(cudaStreamWaitEvent(js, ctx->side_fork, 0));
        hps_status rc = prec == HPS_FP64 ? enqueue_job<double>(ctx, jobs[i], plans[i], chunk[i], js, ws)
                                         : enqueue_job<float>(ctx, jobs[i], plans[i], chunk[i], js, ws);
        if (rc != HPS_OK) return rc;
        if (conc) {
            HPS_CUDA_TRY(cudaEventRecord(ctx->side_done[i], js));
            HPS_CUDA_TRY(cudaStreamWaitEvent(st, ctx->side_done[i], 0));
        }
    }
    return HPS_OK;
}

// ------------------------------------------------------------ autotuning of the LU schedule

std::string tune_file() { const char* e = std::getenv("HPS_TUNE_CACHE"); return e ? e : ""; }

// Cache file: one line per (p, precision, tensor cores): "p prec tc nb unit bn".
void load_tuning(hps_ctx* ctx)
{
    const std::string f = tune_file();
    if (f.empty()) return;
    FILE* fp = std::fopen(f.c_str(), "r");
    if (!fp) return;
    char line[256];
    while (std::fgets(line, sizeof line, fp)) {
        int p, prec, tc;
        TuneChoice c;
        if (std::sscanf(line, "%d %d %d %d %d %d", &p, &prec, &tc, &c.nb, &c.unit, &c.bn) == 6)
            ctx->tuned[std::make_tuple(p, prec, tc)] = c;
    }
    std::fclose(fp);
}

void save_tuning(const hps_ctx* ctx)
{
    const std::string f = tune_file();
    if (f.empty()) return;
    FILE* fp = std::fopen(f.c_str(), "w");
    if (!fp) return;
    for (const auto& kv : ctx->tuned)
        std::fprintf(fp, "%d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                     kv.second.nb, kv.second.unit, kv.second.bn);
    std::fclose(fp);
}

// Schedule candidates of a (precision, tensor cores) combination: the LU
// block NB, the LU unit length (steps joined per product; NB x unit <= 512)
// and the widest tensor-core tile (products narrower than it use 64- or
// 128-column tiles anyway).
std::vector<TuneChoice> tune_candidates(hps_precision prec, bool tc)
{
    if (prec == HPS_FP64 || !tc) return {{32, 1, 256}, {64, 1, 256}};
    return {{128, 4, 256}, {128, 2, 256}, {64, 8, 256}, {64, 4, 256}, {128, 4, 128}, {64, 8, 128}};
}

// Picks the LU schedule for (p, precision, tensor cores) by timing each
// candidate on up to 8 of the job's own boxes (their outputs are rewritten by
// the real run).  Synchronises the stream; never runs inside a capture.
hps_status tune_job(hps_ctx* ctx, Job& j, hps_precision prec, cudaStream_t st)
{
    const auto key = std::make_tuple(j.g->p, (int)prec, ctx->use_tc);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
        j.nb = it->second.nb; j.unit = it->second.unit; j.bn = it->second.bn;
        return HPS_OK;
    }
    const std::vector<TuneChoice> cands = tune_candidates(prec, ctx->use_tc != 0);
    Job trial = j;
    trial.nbox = std::min(j.nbox, 8);
    trial.zero_row_box = -1;
    float best = 1e30f;
    TuneChoice best_c = cands.front();
    cudaEvent_t e0, e1;
    HPS_CUDA_TRY(cudaEventCreate(&e0));
    HPS_CUDA_TRY(cudaEventCreate(&e1));
    for (const TuneChoice& c : cands) {
        trial.nb = c.nb; trial.unit = c.unit; trial.bn = c.bn;
        std::vector<Job> jobs{trial};
        std::vector<Plan> plans{job_plan(ctx, trial, prec)};
        std::vector<int> chunk;
        hps_status rc = ensure_workspace(ctx, plans, jobs, chunk);
        if (rc != HPS_OK) continue;
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {   // the first run warms the code paths
            cudaEventRecord(e0, st);
            rc = enqueue_all(ctx, jobs, plans, chunk, prec, trial.nbox, st);
            cudaEventRecord(e1, st);
            if (rc != HPS_OK) break;
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rc == HPS_OK && ms < best) { best = ms; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned[key] = best_c;
    save_tuning(ctx);
    j.nb = best_c.nb; j.unit = best_c.unit; j.bn = best_c.bn;
    return HPS_OK;
}

// ------------------------------------------------------------ running a call

// Plan phase (geometry, tuning, workspace, diagnostics: every allocation),
// then the enqueue phase, optionally through a cached CUDA graph.
hps_status run_jobs(hps_ctx* ctx, std::vector<Job>& jobs, hps_precision prec, cudaStream_t st)
{
    int total = 0;
    for (Job& j : jobs) {
        j.diag_off = total;
        total += j.nbox;
    }
    size_t cap_i = ctx->diag_cap, cap_d = ctx->diag_cap;
    hps_status rc = grow(&ctx->d_iters, &cap_i, (size_t)total);
    if (rc != HPS_OK) return rc;
    rc = grow(&ctx->d_relcorr, &cap_d, (size_t)total);
    if (rc != HPS_OK) return rc;
    ctx->diag_cap = std::min(cap_i, cap_d);
    if (ctx->autotune)
        for (Job& j : jobs) {
            rc = tune_job(ctx, j, prec, st);
            if (rc != HPS_OK) return rc;
        }
    std::vector<Plan> plans;
    for (const Job& j : jobs) plans.push_back(job_plan(ctx, j, prec));
    std::vector<int> chunk;
    rc = ensure_workspace(ctx, plans, jobs, chunk);
    if (rc != HPS_OK) return rc;
    const bool use_graph = ctx->graphs && !ctx->prof_on && !tc_test_stall_armed();
    if (!use_graph) return enqueue_all(ctx, jobs, plans, chunk, prec, total, st);
    std::ostringstream key;
    key << (int)prec << ' ' << ctx->ir_iters << ' ' << ctx->ir_tol << ' ' << ctx->use_tc << ' ' << ctx->tc_epi_cp << ' ' << ctx->lu_unit << ' ' << ctx->tc_fuse << ' ' << ctx->res_df << ' ' << ctx->fp16_ops << ' ' << ctx->concurrent << ' ' << ctx->ws << ' '
        << ctx->d_iters << ' ' << ctx->d_relcorr;
    for (size_t i = 0; i < jobs.size(); ++i) {
        const Job& j = jobs[i];
        key << " | " << j.g->p << ' ' << j.g->h[0] << ' ' << j.g->h[1] << ' ' << j.g->h[2] << ' ' << j.nbox << ' '
            << j.kappa << ' ' << j.kappa_dev << ' ' << j.b << ' ' << j.rhs_kind << ' ' << j.nload << ' ' << j.rhs
            << ' ' << j.T << ' ' << j.S << ' ' << j.v << ' ' << j.hf << ' ' << j.ui << ' ' << j.vadd << ' '
            << j.status << ' ' << plans[i].NB << ' ' << plans[i].unit_max << ' ' << plans[i].bn_max << ' ' << chunk[i] << ' ' << j.zero_row_box << ' ' << j.beta;
    }
    auto hit = ctx->graph_cache.find(key.str());
    if (hit == ctx->graph_cache.end()) {
        // Capture on the context's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); launch on the caller's.
        if (!ctx->cap_stream) HPS_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        HPS_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_all(ctx, jobs, plans, chunk, prec, total, ctx->cap_stream);
        cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (rc != HPS_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (ce != cudaSuccess) return HPS_ECUDA;
        cudaGraphExec_t exec = nullptr;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return HPS_ECUDA;
        hit = ctx->graph_cache.emplace(key.str(), exec).first;
    }
    HPS_CUDA_TRY(cudaGraphLaunch(hit->second, st));
    return HPS_OK;
}

hps_status check_kind(const hps_leaf_kind* kind)
{
    if (!kind || !valid_p(kind->p)) return HPS_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(kind->h[a] > 0.0) || !std::isfinite(kind->h[a])) return HPS_EINVAL;
    if (!std::isfinite(kind->kappa)) return HPS_EINVAL;
    return HPS_OK;
}

hps_status finish(hps_ctx* ctx, const std::vector<Job>& jobs, cudaStream_t st)
{
    if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
    int total = 0;
    for (const Job& j : jobs) total += j.nbox;
    ctx->last_nbox = total;
    ctx->last_stream = st;
    if (!ctx->sync) return HPS_OK;
    HPS_CUDA_TRY(cudaStreamSynchronize(st));
    for (const Job& j : jobs) {
        std::vector<int> h(j.nbox);
        HPS_CUDA_TRY(cudaMemcpy(h.data(), j.status, sizeof(int) * j.nbox, cudaMemcpyDeviceToHost));
        for (int v : h)
            if (v) return (hps_status)v;
    }
    return HPS_OK;
}

struct ProfScope {
    explicit ProfScope(hps_ctx* c) { hps::t_prof = c->prof_on ? &c->prof : nullptr; }
    ~ProfScope() { hps::t_prof = nullptr; }
};

// Status words: the caller's array, or a slice of the context's own.
hps_status status_ptrs(hps_ctx* ctx, std::vector<Job>& jobs, const std::vector<int*>& user)
{
    size_t need = 0;
    for (size_t i = 0; i < jobs.size(); ++i)
        if (!user[i]) need += jobs[i].nbox;
    hps_status rc = grow(&ctx->d_status, &ctx->status_cap, need > 0 ? need : 1);
    if (rc != HPS_OK) return rc;
    size_t off = 0;
    for (size_t i = 0; i < jobs.size(); ++i) {
        if (user[i]) jobs[i].status = user[i];
        else { jobs[i].status = ctx->d_status + off; off += jobs[i].nbox; }
    }
    return HPS_OK;
}

// Runs a single-kind call (the three leaf entry points).
hps_status run_single(hps_ctx* ctx, Job j, const hps_leaf_kind* kind, hps_precision prec, int* box_status,
                      void* stream)
{
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    hps_status rc = get_geometry(ctx, kind->p, kind->h, &g);
    if (rc != HPS_OK) return rc;
    j.g = g;
    j.kappa = kind->kappa;
    j.beta = kind->beta;
    j.zero_row_box = ctx->zero_row_box;
    std::vector<Job> jobs{j};
    rc = status_ptrs(ctx, jobs, {box_status});
    if (rc != HPS_OK) return rc;
    rc = run_jobs(ctx, jobs, prec, st);
    if (rc != HPS_OK) return rc;
    return finish(ctx, jobs, st);
}

// ------------------------------------------------------------ stored factorisations

template <typename T>
hps_status factors_factor(hps_leaf_factors* F, const double* b, cudaStream_t st)
{
    const Geometry& g = *F->g;
    const long long p3 = (long long)g.p * g.p * g.p;
    Work<T> w = carve<T>(F->P, F->buf, F->nbox);
    HPS_CUDA_TRY(cudaMemsetAsync(F->d_fstatus, 0, sizeof(int) * F->nbox, st));
    launch_build_aug<T>(g, F->kappa, nullptr, F->nbox, b, p3, RHS_LOAD, 0, nullptr, 0, w.M, F->P.ldm, w.sM,
                        F->d_fstatus, F->ctx->zero_row_box, st, F->beta);
    if constexpr (sizeof(T) == 8) {
        lu_factor<double>(F->P, w, F->nbox, F->d_fstatus, st);
    } else {
        if (F->P.tc) {
            tc_reset_abort(st);
            if (!tc_lu_factor(F->P, w, F->nbox, F->d_fstatus, st)) return HPS_ECUDA;
        } else {
            lu_factor<float>(F->P, w, F->nbox, F->d_fstatus, st);
        }
        launch_kappa_b(g, F->kappa, nullptr, F->nbox, b, p3, w.kb, w.kbs, st);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

// X = A_ii^{-1} B for B = f_i (LOAD) or -A_ib u_b (TRACE), nrhs columns, with
// the stored factors (and the FP64 refinement of the mixed path); then the
// outputs: v and h = A_bi v (LOAD) or u_i = X + v (TRACE).
template <typename T>
hps_status factors_solve(hps_leaf_factors* F, int rhs_kind, int nrhs, const double* rhs, const double* vadd,
                         double* out0, double* out1, int* status, cudaStream_t st)
{
    const Geometry& g = *F->g;
    const int n = g.n, m = g.m, nbox = F->nbox;
    const long long p3 = (long long)g.p * g.p * g.p;
    const long long s_rhs = rhs_kind == RHS_LOAD ? nrhs * p3 : (long long)nrhs * m;
    Work<T> w = carve<T>(F->P, F->buf, nbox);
    HPS_CUDA_TRY(cudaMemcpyAsync(status, F->d_fstatus, sizeof(int) * nbox, cudaMemcpyDeviceToDevice, st));
    launch_load_rhs<T>(g, nbox, rhs_kind, nrhs, rhs, s_rhs, w.M, F->P.ldm, w.sM, status, st, F->beta);
    double* X;
    long long ldx, sX;
    if constexpr (sizeof(T) == 8) {
        lu_forward<double>(F->P, w, nbox, n, nrhs, nullptr, st);
        lu_backward<double>(F->P, w, nbox, n, nrhs, nullptr, st);
        X = reinterpret_cast<double*>(w.M) + n;
        ldx = F->P.ldm;
        sX = w.sM;
    } else {
        if (F->P.tc) {
            tc_reset_abort(st);
            if (!tc_lu_forward(F->P, w, nbox, n, nrhs, nullptr, st)) return HPS_ECUDA;
            if (!tc_lu_backward(F->P, w, nbox, n, nrhs, nullptr, st)) return HPS_ECUDA;
        } else {
            lu_forward<float>(F->P, w, nbox, n, nrhs, nullptr, st);
            lu_backward<float>(F->P, w, nbox, n, nrhs, nullptr, st);
        }
        X = w.X;
        ldx = nrhs;
        sX = w.sX;
        CallSpec cs;
        cs.rhs_kind = rhs_kind;
        cs.r = nrhs;
        cs.rhs = rhs;
        cs.s_rhs = s_rhs;
        cs.zero_row_box = -1;
        cs.kappa_dev = nullptr;
        cs.kappa = F->kappa;
        cs.beta = F->beta;
        HPS_CUDA_TRY(cudaMemsetAsync(F->d_iters, 0, sizeof(int) * nbox, st));
        HPS_CUDA_TRY(cudaMemsetAsync(F->d_relcorr, 0, sizeof(double) * nbox, st));
        hps_status rc = refine_chunk(F->ctx, g, cs, F->P, w, nbox, nullptr, X, ldx, sX, status, F->d_iters,
                                     F->d_relcorr, st, true);
        if (rc != HPS_OK) return rc;
    }
    if (rhs_kind == RHS_LOAD) {
        launch_transpose_add(X, ldx, sX, n, nrhs, nullptr, out0, nbox, st);
        launch_dn(g, nbox, X, ldx, sX, nrhs, out1, (long long)nrhs * m, 1, 0, st);
    } else {
        launch_transpose_add(X, ldx, sX, n, nrhs, vadd, out0, nbox, st);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

hps_status factors_run(hps_leaf_factors* F, int rhs_kind, int nrhs, const double* rhs, const double* vadd,
                       double* out0, double* out1, int* box_status, void* stream)
{
    hps_ctx* ctx = F->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    int* status = box_status ? box_status : F->d_status;
    auto enqueue = [&](cudaStream_t s) {
        return F->prec == HPS_FP64 ? factors_solve<double>(F, rhs_kind, nrhs, rhs, vadd, out0, out1, status, s)
                                   : factors_solve<float>(F, rhs_kind, nrhs, rhs, vadd, out0, out1, status, s);
    };
    hps_status rc = HPS_OK;
    if (ctx->graphs && !ctx->prof_on) {
        // one captured graph per distinct solve (same buffers and options), as
        // for the one-shot calls; time steps replay it
        std::ostringstream key;
        key << rhs_kind << ' ' << nrhs << ' ' << rhs << ' ' << vadd << ' ' << out0 << ' ' << out1 << ' ' << status
            << ' ' << ctx->ir_iters << ' ' << ctx->ir_tol << ' ' << ctx->res_df;
        auto hit = F->graphs.find(key.str());
        if (hit == F->graphs.end()) {
            if (!ctx->cap_stream) HPS_CUDA_TRY(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            HPS_CUDA_TRY(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue(ctx->cap_stream);
            cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (rc != HPS_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
            if (ce != cudaSuccess) return HPS_ECUDA;
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return HPS_ECUDA;
            hit = F->graphs.emplace(key.str(), exec).first;
        }
        HPS_CUDA_TRY(cudaGraphLaunch(hit->second, st));
    } else {
        rc = enqueue(st);
    }
    if (rc != HPS_OK) return rc;
    if (!ctx->sync) return HPS_OK;
    HPS_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> h(F->nbox);
    HPS_CUDA_TRY(cudaMemcpy(h.data(), status, sizeof(int) * F->nbox, cudaMemcpyDeviceToHost));
    for (int v : h)
        if (v) return (hps_status)v;
    return HPS_OK;
}

}  // namespace

// ================================================================ C ABI

extern "C" {

hps_status hps_selftest_conversions(int device, long long n, unsigned long long seed, long long* mismatches)
{
    if (n < 0 || !mismatches) return HPS_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return HPS_ECUDA;
    unsigned long long* d = nullptr;
    unsigned long long h[2] = {0, 0};
    hps_status rc = HPS_OK;
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) rc = HPS_ENOMEM;
    if (rc == HPS_OK && cudaMemset(d, 0, sizeof(h)) != cudaSuccess) rc = HPS_ECUDA;
    if (rc == HPS_OK) {
        hps::selftest_conversions(n, seed, d, 0);
        if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HPS_ECUDA;
    }
    if (d) cudaFree(d);
    cudaSetDevice(prev);
    mismatches[0] = (long long)h[0];
    mismatches[1] = (long long)h[1];
    return rc;
}

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
    return make_plan(n, m, prec, 0, true, prec != HPS_FP64, 4, true).per_box;
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
    load_tuning(c);
    *out = c;
    return HPS_OK;
}

void hps_destroy(hps_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    clear_graphs(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    for (auto& kv : ctx->geoms) { cudaFree(kv.second.dD); cudaFree(kv.second.dD2); cudaFree(kv.second.dDF); }
    if (ctx->d_iters) cudaFree(ctx->d_iters);
    if (ctx->d_relcorr) cudaFree(ctx->d_relcorr);
    if (ctx->d_kappa) cudaFree(ctx->d_kappa);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (auto& kv : ctx->a0inv) cudaFree(kv.second);
    if (ctx->gate_buf) cudaFree(ctx->gate_buf);
    for (cudaStream_t sst : ctx->side) cudaStreamDestroy(sst);
    for (cudaEvent_t ev : ctx->side_done) cudaEventDestroy(ev);
    if (ctx->side_fork) cudaEventDestroy(ctx->side_fork);
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
    case HPS_OPT_AUTOTUNE:
        ctx->autotune = value != 0;
        return HPS_OK;
    case HPS_OPT_GRAPHS:
        ctx->graphs = value != 0;
        return HPS_OK;
    case HPS_OPT_TC_EPILOGUE:
        if (!(value == 0 || value == 1)) return HPS_EINVAL;
        ctx->tc_epi_cp = (int)value;
        return HPS_OK;
    case HPS_OPT_LU_UNIT:
        if (!(value == 1 || value == 2 || value == 4 || value == 8)) return HPS_EINVAL;
        ctx->lu_unit = (int)value;
        return HPS_OK;
    case HPS_OPT_TC_FUSE:
        if (!(value == -1 || value == 0 || value == 1)) return HPS_EINVAL;
        ctx->tc_fuse = (int)value;
        return HPS_OK;
    case HPS_OPT_RESIDUAL_DF:
        if (!(value == 0 || value == 1 || value == 2 || value == 3)) return HPS_EINVAL;
        ctx->res_df = (int)value;
        return HPS_OK;
    case HPS_OPT_FP16_OPERANDS:
        if (!(value == 0 || value == 1)) return HPS_EINVAL;
        ctx->fp16_ops = (int)value;
        return HPS_OK;
    case HPS_OPT_GROUPS_CONCURRENT:
        if (!(value == 0 || value == 1)) return HPS_EINVAL;
        ctx->concurrent = (int)value;
        return HPS_OK;
    case HPS_OPT_TEST_SINGULAR_BOX:
        ctx->zero_row_box = (int)value;
        return HPS_OK;
    case HPS_OPT_TEST_TC_TIMEOUT:
        if (!(value == 0 || value == 1)) return HPS_EINVAL;
        tc_test_stall_next((int)value);
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
    if (prec != HPS_FP64 && prec != HPS_FP32_IR && prec != HPS_BF16_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || !T) return HPS_EINVAL;
    Job j;
    j.nbox = nbox;
    j.b = b;
    j.rhs_kind = RHS_DTN;
    j.T = T;
    j.S = S;
    return run_single(ctx, j, kind, prec, box_status, stream);
}

hps_status hps_leaf_particular(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs, const double* b,
                               const double* f, double* v, double* h, hps_precision prec, int* box_status,
                               void* stream)
{
    if (!ctx || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR && prec != HPS_BF16_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || !f || !v || !h) return HPS_EINVAL;
    Job j;
    j.nbox = nbox;
    j.b = b;
    j.rhs_kind = RHS_LOAD;
    j.nload = nrhs;
    j.rhs = f;
    j.v = v;
    j.hf = h;
    return run_single(ctx, j, kind, prec, box_status, stream);
}

hps_status hps_leaf_reconstruct(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nrhs, const double* b,
                                const double* S, const double* v, const double* ub, double* ui,
                                hps_precision prec, int* box_status, void* stream)
{
    if (!ctx || nbox < 0 || nrhs < 1 || nrhs > 256) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR && prec != HPS_BF16_IR) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!ub || !ui || (!S && !b)) return HPS_EINVAL;
    if (S) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        HPS_CUDA_TRY(cudaSetDevice(ctx->device));
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        ProfScope prof_scope(ctx);
        const int q = kind->p - 2, n = q * q * q, m = 6 * q * q;
        if (box_status) HPS_CUDA_TRY(cudaMemsetAsync(box_status, 0, sizeof(int) * nbox, st));
        launch_recon_stored(S, n, m, nrhs, v, ub, ui, nbox, st);
        if (cudaGetLastError() != cudaSuccess) return HPS_ECUDA;
        ctx->last_nbox = 0;
        ctx->last_stream = st;
        return HPS_OK;
    }
    Job j;
    j.nbox = nbox;
    j.b = b;
    j.rhs_kind = RHS_TRACE;
    j.nload = nrhs;
    j.rhs = ub;
    j.ui = ui;
    j.vadd = v;
    return run_single(ctx, j, kind, prec, box_status, stream);
}


hps_status hps_leaf_factor(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, const double* b, int nrhs_max,
                           hps_precision prec, int* box_status, void* stream, hps_leaf_factors** out)
{
    if (!out) return HPS_EINVAL;
    *out = nullptr;
    if (!ctx || nbox < 1 || nrhs_max < 1 || nrhs_max > 256 || !b) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR && prec != HPS_BF16_IR) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    hps::Geometry* g = nullptr;
    rc = get_geometry(ctx, kind->p, kind->h, &g);
    if (rc != HPS_OK) return rc;
    Job j;
    j.g = g;
    j.nbox = nbox;
    j.rhs_kind = RHS_LOAD;
    j.nload = nrhs_max;
    hps_leaf_factors* F = new hps_leaf_factors;
    F->ctx = ctx;
    F->g = g;
    F->P = job_plan(ctx, j, prec);
    F->prec = prec;
    F->nbox = nbox;
    F->nrhs_max = nrhs_max;
    F->kappa = kind->kappa;
    const size_t bytes = F->P.per_box * (size_t)nbox;
    if (cudaMalloc(&F->buf, bytes) != cudaSuccess || cudaMalloc(&F->d_fstatus, sizeof(int) * nbox) != cudaSuccess ||
        cudaMalloc(&F->d_status, sizeof(int) * nbox) != cudaSuccess ||
        cudaMalloc(&F->d_iters, sizeof(int) * nbox) != cudaSuccess ||
        cudaMalloc(&F->d_relcorr, sizeof(double) * nbox) != cudaSuccess ||
        (kind->beta && cudaMalloc(&F->beta, sizeof(double) * 3 * (size_t)g->p * g->p * g->p * nbox) != cudaSuccess)) {
        cudaGetLastError();
        hps_leaf_factors_destroy(F);
        return HPS_ENOMEM;
    }
    if (F->beta &&
        cudaMemcpyAsync(F->beta, kind->beta, sizeof(double) * 3 * (size_t)g->p * g->p * g->p * nbox,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        hps_leaf_factors_destroy(F);
        return HPS_ECUDA;
    }
    rc = prec == HPS_FP64 ? factors_factor<double>(F, b, st) : factors_factor<float>(F, b, st);
    if (rc == HPS_OK && box_status)
        rc = cudaMemcpyAsync(box_status, F->d_fstatus, sizeof(int) * nbox, cudaMemcpyDeviceToDevice, st) ==
                     cudaSuccess
                 ? HPS_OK
                 : HPS_ECUDA;
    if (rc == HPS_OK && ctx->sync) {
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = HPS_ECUDA;
        else {
            std::vector<int> h(nbox);
            if (cudaMemcpy(h.data(), F->d_fstatus, sizeof(int) * nbox, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = HPS_ECUDA;
            for (int v : h)
                if (rc == HPS_OK && v) rc = (hps_status)v;
            if (rc != HPS_OK && rc != HPS_ECUDA) {   // a box failed: the factors still exist
                *out = F;
                return rc;
            }
        }
    }
    if (rc != HPS_OK) {
        hps_leaf_factors_destroy(F);
        return rc;
    }
    *out = F;
    return HPS_OK;
}

hps_status hps_leaf_solve_factored(hps_leaf_factors* F, int nrhs, const double* f, double* v, double* h,
                                   int* box_status, void* stream)
{
    if (!F || nrhs < 1 || nrhs > F->nrhs_max || !f || !v || !h) return HPS_EINVAL;
    return factors_run(F, RHS_LOAD, nrhs, f, nullptr, v, h, box_status, stream);
}

hps_status hps_leaf_reconstruct_factored(hps_leaf_factors* F, int nrhs, const double* v, const double* ub,
                                         double* ui, int* box_status, void* stream)
{
    if (!F || nrhs < 1 || nrhs > F->nrhs_max || !ub || !ui) return HPS_EINVAL;
    return factors_run(F, RHS_TRACE, nrhs, ub, v, ui, nullptr, box_status, stream);
}

hps_status hps_leaf_apply(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, int nfield, const double* b,
                          const double* u, double* out, void* stream)
{
    if (!ctx || nbox < 0 || nfield < 1) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (nbox == 0) return HPS_OK;
    if (!b || !u || !out) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    rc = get_geometry(ctx, kind->p, kind->h, &g);
    if (rc != HPS_OK) return rc;
    launch_apply_op(*g, kind->kappa, nbox, nfield, b, u, out, st, kind->beta);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}

void hps_leaf_factors_destroy(hps_leaf_factors* F)
{
    if (!F) return;
    if (F->ctx) cudaSetDevice(F->ctx->device);
    cudaFree(F->buf);
    cudaFree(F->d_fstatus);
    cudaFree(F->d_status);
    cudaFree(F->d_iters);
    cudaFree(F->d_relcorr);
    cudaFree(F->beta);
    for (auto& kv : F->graphs) cudaGraphExecDestroy(kv.second);
    delete F;
}

hps_status hps_leaf_groups(hps_ctx* ctx, int ngroups, const hps_leaf_group* groups, hps_precision prec,
                           void* stream)
{
    if (!ctx || ngroups < 0 || (ngroups > 0 && !groups)) return HPS_EINVAL;
    if (prec != HPS_FP64 && prec != HPS_FP32_IR && prec != HPS_BF16_IR) return HPS_EINVAL;
    size_t nk = 0;
    for (int i = 0; i < ngroups; ++i) {
        const hps_leaf_group& G = groups[i];
        if (!valid_p(G.p) || G.nbox < 0 || G.nrhs < 0 || G.nrhs > 256) return HPS_EINVAL;
        for (int a = 0; a < 3; ++a)
            if (!(G.h[a] > 0.0) || !std::isfinite(G.h[a])) return HPS_EINVAL;
        if (G.nbox == 0) continue;
        if (!G.b || !G.kappa || (!G.T && G.nrhs == 0)) return HPS_EINVAL;
        if (G.nrhs > 0 && (!G.f || !G.v || !G.hflux)) return HPS_EINVAL;
        for (int bx = 0; bx < G.nbox; ++bx)
            if (!std::isfinite(G.kappa[bx])) return HPS_EINVAL;
        nk += G.nbox;
    }
    if (nk == 0) return HPS_OK;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    hps_status rc = grow(&ctx->d_kappa, &ctx->kappa_cap, nk);
    if (rc != HPS_OK) return rc;
    std::vector<double> kap;
    kap.reserve(nk);
    std::vector<Job> jobs;
    std::vector<int*> user;
    for (int i = 0; i < ngroups; ++i) {
        const hps_leaf_group& G = groups[i];
        if (G.nbox == 0) continue;
        Geometry* g = nullptr;
        rc = get_geometry(ctx, G.p, G.h, &g);
        if (rc != HPS_OK) return rc;
        Job j;
        j.g = g;
        j.nbox = G.nbox;
        j.kappa_dev = ctx->d_kappa + kap.size();
        kap.insert(kap.end(), G.kappa, G.kappa + G.nbox);
        j.b = G.b;
        j.T = G.T;
        j.S = G.T ? G.S : nullptr;
        if (G.T && G.nrhs > 0) j.rhs_kind = RHS_DTN_LOAD;
        else if (G.T) j.rhs_kind = RHS_DTN;
        else j.rhs_kind = RHS_LOAD;
        j.nload = G.nrhs;
        j.rhs = G.nrhs ? G.f : nullptr;
        j.v = G.v;
        j.hf = G.hflux;
        jobs.push_back(j);
        user.push_back(G.box_status);
    }
    // Per-box wavenumbers go to the device outside any captured graph.
    HPS_CUDA_TRY(cudaMemcpyAsync(ctx->d_kappa, kap.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, st));
    rc = status_ptrs(ctx, jobs, user);
    if (rc != HPS_OK) return rc;
    rc = run_jobs(ctx, jobs, prec, st);
    if (rc != HPS_OK) return rc;
    return finish(ctx, jobs, st);
}


// The residual gate of a predicted DtN map (for the learned correction; the
// paper has no counterpart).  For k seeded probe traces phi per box it forms
// T phi = A_bb phi + A_bi w with A_ii w = -A_ib phi, solving for w by
// Richardson iteration preconditioned with A0^{-1}, the interior block of the
// same box with b = 1 (computed once per (p, h, kappa) with the FP64 LU and
// kept in FP32); residuals are FP64 and matrix-free.  A box is accepted when
// ||T_hat phi - T phi|| <= tol ||T phi|| and the iteration has converged.
hps_status hps_dtn_gate(hps_ctx* ctx, const hps_leaf_kind* kind, int nbox, const double* b, const double* T_hat,
                        int nprobe, unsigned long long seed, int iters, double tol, int* accept, double* err,
                        void* stream)
{
    if (!ctx || nbox < 0 || nprobe < 1 || nprobe > 64 || iters < 1 || iters > 200 || !(tol > 0)) return HPS_EINVAL;
    hps_status rc = check_kind(kind);
    if (rc != HPS_OK) return rc;
    if (kind->beta) return HPS_EINVAL;   // the gate's preconditioner has no first-order term
    if (nbox == 0) return HPS_OK;
    if (!b || !T_hat || !accept || !err) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->mu);
    HPS_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ProfScope prof_scope(ctx);
    Geometry* g = nullptr;
    rc = get_geometry(ctx, kind->p, kind->h, &g);
    if (rc != HPS_OK) return rc;
    const int p = g->p, n = g->n, m = g->m, k = nprobe;
    const long long p3 = (long long)p * p * p;
    const auto key = std::make_tuple(p, kind->h[0], kind->h[1], kind->h[2], kind->kappa);
    auto it = ctx->a0inv.find(key);
    if (it == ctx->a0inv.end()) {
        // A0^{-1}: the FP64 LU of the b = 1 block applied to the identity (n loads).
        double *ones = nullptr, *f = nullptr, *v = nullptr, *hf = nullptr;
        float* inv = nullptr;
        int* stt = nullptr;
        bool ok = cudaMalloc(&ones, sizeof(double) * p3) == cudaSuccess &&
                  cudaMalloc(&f, sizeof(double) * n * p3) == cudaSuccess &&
                  cudaMalloc(&v, sizeof(double) * (size_t)n * n) == cudaSuccess &&
                  cudaMalloc(&hf, sizeof(double) * (size_t)n * m) == cudaSuccess &&
                  cudaMalloc(&inv, sizeof(float) * (size_t)n * n) == cudaSuccess &&
                  cudaMalloc(&stt, sizeof(int)) == cudaSuccess;
        if (ok) {
            std::vector<double> h1(p3, 1.0);
            cudaMemcpy(ones, h1.data(), sizeof(double) * p3, cudaMemcpyHostToDevice);
            cudaMemsetAsync(f, 0, sizeof(double) * n * p3, st);
            launch_identity_loads(p, n, f, st);
            Job j;
            j.g = g; j.nbox = 1; j.kappa = kind->kappa; j.b = ones; j.rhs_kind = RHS_LOAD; j.nload = n; j.rhs = f;
            j.v = v; j.hf = hf; j.status = stt;
            std::vector<Job> jobs{j};
            const int gsave = ctx->graphs, tsave = ctx->autotune;
            ctx->graphs = 0;
            ctx->autotune = 0;
            rc = run_jobs(ctx, jobs, HPS_FP64, st);
            ctx->graphs = gsave;
            ctx->autotune = tsave;
            if (rc == HPS_OK) launch_transpose_f32(n, v, inv, st);
            int hs = 0;
            if (rc == HPS_OK && (cudaMemcpyAsync(&hs, stt, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                                 cudaStreamSynchronize(st) != cudaSuccess))
                rc = HPS_ECUDA;
            if (rc == HPS_OK && hs != 0) rc = (hps_status)hs;
        } else {
            cudaGetLastError();
            rc = HPS_ENOMEM;
        }
        cudaFree(ones); cudaFree(f); cudaFree(v); cudaFree(hf); cudaFree(stt);
        if (rc != HPS_OK) { cudaFree(inv); return rc; }
        it = ctx->a0inv.emplace(key, inv).first;
    }
    // Workspace: probes, w (FP64) and R, delta (FP32) laid out [n][nbox k], probe products.
    const size_t nk = (size_t)nbox * k;
    const size_t b_phi = align_up(sizeof(double) * nk * m, 256), b_w = align_up(sizeof(double) * nk * n, 256);
    const size_t b_r = align_up(sizeof(float) * nk * n, 256), b_tp = b_phi;
    const size_t b_norm = align_up(sizeof(double) * 2 * nbox, 256);
    const size_t need = b_phi + b_w + 2 * b_r + 2 * b_tp + b_norm;
    if (need > ctx->gate_cap) {
        if (ctx->gate_buf) { cudaDeviceSynchronize(); cudaFree(ctx->gate_buf); ctx->gate_buf = nullptr; ctx->gate_cap = 0; }
        if (cudaMalloc(&ctx->gate_buf, need) != cudaSuccess) { cudaGetLastError(); return HPS_ENOMEM; }
        ctx->gate_cap = need;
    }
    char* c = static_cast<char*>(ctx->gate_buf);
    double* phi = reinterpret_cast<double*>(c); c += b_phi;
    double* w = reinterpret_cast<double*>(c); c += b_w;
    float* R = reinterpret_cast<float*>(c); c += b_r;
    float* D = reinterpret_cast<float*>(c); c += b_r;
    double* tp = reinterpret_cast<double*>(c); c += b_tp;
    double* tph = reinterpret_cast<double*>(c); c += b_tp;
    double* norms = reinterpret_cast<double*>(c);
    launch_probes((long long)nk * m, seed, phi, st);
    HPS_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(double) * nk * n, st));
    const long long ld = (long long)nk;   // row pitch of w, R, D: all boxes' probes side by side
    for (int i = 0; i < iters; ++i) {
        if (i == iters - 1) HPS_CUDA_TRY(cudaMemsetAsync(norms, 0, sizeof(double) * 2 * nbox, st));
        launch_residual(*g, kind->kappa, nullptr, nbox, b, p3, RHS_TRACE, k, phi, (long long)k * m, w, ld, k, R, ld, k,
                        nullptr, st);
        GemmArgs<float> a{};
        a.A = it->second; a.lda = n; a.sA = 0;
        a.B = R; a.ldb = ld; a.sB = 0;
        a.O = D; a.ldo = ld; a.sO = 0;
        a.M = n; a.N = (int)nk; a.K = n; a.alpha = 1.0f; a.mode = GM_SET;
        launch_gemm<float>(a, 1, st);
        launch_ir_update(D, ld, k, n, k, w, ld, k, norms, nullptr, nbox, st, true);
    }
    launch_dn(*g, nbox, w, ld, k, k, tp, (long long)k * m, 1, 0, st);
    launch_abb_add(*g, nbox, k, phi, tp, st);
    launch_apply_probes(m, k, nbox, T_hat, phi, tph, st);
    launch_gate_decide(m, k, nbox, tph, tp, norms, tol, accept, err, st);
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
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
