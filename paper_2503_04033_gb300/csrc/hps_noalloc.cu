// hps_leaf_build_dtn_noalloc: the FP64 DtN build with no device allocation.
//
// Some callers cannot call cudaMalloc: a host application whose device
// memory is owned by another allocator (for example a framework's caching
// allocator that has already reserved the GPU), or a latency-critical loop in
// which cudaMalloc/cudaFree would stall on an implicit device synchronisation.
// This entry point serves them.  Its scratch memory (operator tables, status
// words and the LU workspace) lives in one file-scope __device__ array of
// kScratchBytes, which every GPU that loads this library holds until the
// process exits.  The caller still passes b and T; nothing else is allocated.
#include <cstring>
#include <mutex>

#include "hps_internal.h"

namespace {

constexpr size_t kScratchBytes = 64ull << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxNoallocP = 14;                 // the largest order whose one-box workspace fits the scratch

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// The reference Chebyshev matrix and the box size, passed by value as a kernel
// parameter: the tables need no host-to-device copy.
struct TableArgs {
    int p;
    double h[3];
    double Dhat[kMaxNoallocP * kMaxNoallocP];
};

// D and D2 of every axis written into the scratch by one thread, with the
// helper (and so the bits) of the context path's tables.
__global__ void k_noalloc_tables(const TableArgs a, double* D, double* D2)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) hps::geometry_tables(a.p, a.Dhat, a.h, D, D2);
}

hps_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return HPS_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HPS_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return HPS_OK;
}

}  // namespace

using namespace hps;

extern "C" hps_status hps_leaf_build_dtn_noalloc(const hps_leaf_kind* kind, int nbox, const double* b, double* T,
                                                 int* box_status, void* stream)
{
    if (!kind || kind->p < 3 || kind->p > kMaxP || nbox < 0 || kind->beta) return HPS_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(kind->h[a] > 0.0)) return HPS_EINVAL;
    if (nbox == 0) return HPS_OK;
    if (!b || !T) return HPS_EINVAL;
    const int p = kind->p, q = p - 2, n = q * q * q, m = 6 * q * q, pp = p * p;
    const long long p3 = (long long)pp * p;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Scratch layout: [D | D2 | status words | per-box LU workspace x chunk].
    const Plan P = make_plan(n, m, HPS_FP64, 0, false, false);
    const size_t tables = align_up(2 * 3 * (size_t)pp * sizeof(double), 256);
    const size_t fixed = tables + (box_status ? 0 : align_up((size_t)nbox * sizeof(int), 256));
    if (p > kMaxNoallocP || fixed + P.per_box > kScratchBytes) return HPS_ENOMEM;   // one box does not fit
    const int chunk = (int)std::min<size_t>((size_t)nbox, (kScratchBytes - fixed) / P.per_box);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HPS_ECUDA;
    unsigned char* base = nullptr;
    hps_status rc = scratch_address(dev, &base);
    if (rc != HPS_OK) return rc;

    // Operator tables, built on the device from the reference matrix (host
    // arithmetic only for Dhat, which travels as a kernel parameter).
    TableArgs ta{};
    ta.p = p;
    for (int a = 0; a < 3; ++a) ta.h[a] = kind->h[a];
    cheb_diff(p, ta.Dhat);
    Geometry g;
    g.p = p; g.q = q; g.n = n; g.m = m;
    for (int a = 0; a < 3; ++a) g.h[a] = kind->h[a];
    g.dD = reinterpret_cast<double*>(base);
    g.dD2 = g.dD + 3 * pp;
    k_noalloc_tables<<<1, 32, 0, st>>>(ta, g.dD, g.dD2);

    // Status words must start at zero (the array keeps the previous call's contents).
    int* status = box_status ? box_status : reinterpret_cast<int*>(base + tables);
    if (cudaMemsetAsync(status, 0, sizeof(int) * nbox, st) != cudaSuccess) return HPS_ECUDA;

    unsigned char* wbase = base + fixed;
    for (int b0 = 0; b0 < nbox; b0 += chunk) {
        const int nc = std::min(chunk, nbox - b0);
        Work<double> w = carve<double>(P, wbase, nc);
        launch_build_aug<double>(g, kind->kappa, nullptr, nc, b + b0 * p3, p3, RHS_DTN, m, nullptr, 0, w.M, P.ldm, w.sM,
                                 status + b0, -1, st);
        lu_factor<double>(P, w, nc, status + b0, st);
        lu_backward<double>(P, w, nc, n, m, nullptr, st);
        launch_dn(g, nc, w.M + n, P.ldm, w.sM, m, T + (long long)b0 * m * m, (long long)m * m, 0, 1, st);
    }
    return cudaGetLastError() == cudaSuccess ? HPS_OK : HPS_ECUDA;
}
