// Tensor-core update products of the FP32 LU (sm_103a, tcgen05 + TMA).
//
// Every trailing update and triangular-solve step of the blocked LU is a
// product O <- src - A G with A = F_s or B_s (rows x NB, or rows x 2 NB for a
// pair of steps) and G the step's gathered rows; see hps_lu.cu for the scheme
// and the LU sequences at the end of this file for the pairs.  Here that
// product runs on the 5th-generation tensor cores with FP32 accuracy from
// split operands (TcFmt): 3 x TF32 (x = hi + lo, three kind::tf32 products)
// or 3 x BF16 (x = hi + mid + lo, six kind::f16 products), FP32 accumulation
// in TMEM.  The split operands are packed K-major (A as [plane][row][k], G
// transposed to [plane][col][k]) so that TMA brings 64-byte rows of K into
// shared memory in the 64B-swizzled layout that tcgen05.mma reads directly.
//
// A persistent CTA per SM walks output tiles (128 x 256 for TF32, 128 x 128
// for BF16): warp 0 issues the TMA loads (3-stage ring of 48 KiB K chunks;
// the left operand may come from two tensor maps), warp 1 owns two TMEM
// accumulators and issues the MMAs (one elected lane), warps 2-5 drain TMEM
// with tcgen05.ld and apply the epilogue (source rows: zero, in place, or
// saved pivot rows; by TMA in and out where O is 16-byte aligned, cp.async
// otherwise) while the next tile accumulates.  At K = 2 NB the product sits
// at the 3 x TF32 ridge: tensor work and operand plus O traffic both matter.
// All mbarrier waits are bounded; a wait that gives up marks the box
// HPS_ETIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <utility>
#include <vector>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int TC_BM = 128;                                  // tile rows = TMEM lanes
constexpr uint32_t ROWB = 64;                               // bytes of an operand row in one K chunk (64B swizzle)
constexpr uint32_t A_TILE = TC_BM * ROWB;                   // 8 KiB per plane
constexpr int TC_STAGES = 3;
constexpr int TC_EPI_WARPS = 4;                             // one per TMEM lane quarter
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;          // warp 0 TMA, warp 1 MMA, warps 2.. epilogue

// Operand formats of the update product.  FMT 0: each operand x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi) (2 planes of FP32 containers, kind::tf32,
// products hi*hi + hi*lo + lo*hi).  FMT 1: x = hi + mid + lo, three BF16
// roundings of the successive remainders (3 planes, kind::f16 with BF16 A
// and B, products hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi).  Both
// drop only terms below FP32 rounding and accumulate in FP32.  FMT 2: x = hi
// + lo, two FP16 roundings (2 planes, kind::f16 with FP16 A and B, products
// hi*hi + hi*lo + lo*hi): the same 22 bits as FMT 0 in half the bytes, with
// twice the MMA rate.  FP16's range is kept by power-of-two scales: each K
// column of the left operand is scaled to a maximum below 2^15 and the
// matching row of the right operand by the inverse (the product is
// unchanged), then each column of the right operand is scaled to a maximum
// below 2^15 and the epilogue multiplies the accumulator column by the
// inverse.  Values far below their column's maximum lose bits only at 2^-39
// of that maximum.  A K chunk is one 64-byte row: 16 TF32 or 32 BF16 / FP16
// values.
template <int FMT>
struct TcFmt;
template <>
struct TcFmt<0> {
    static constexpr int NPL = 2, EB = 4, KPC = 16, BN = 256;
};
template <>
struct TcFmt<1> {
    static constexpr int NPL = 3, EB = 2, KPC = 32, BN = 128;
};
template <>
struct TcFmt<2> {
    static constexpr int NPL = 2, EB = 2, KPC = 32, BN = 256;
};
template <int FMT>
__host__ __device__ constexpr uint32_t b_tile() { return (uint32_t)TcFmt<FMT>::BN * ROWB; }
template <int FMT>
__host__ __device__ constexpr uint32_t stage_bytes() { return (uint32_t)TcFmt<FMT>::NPL * (A_TILE + b_tile<FMT>()); }
constexpr uint32_t STAGE_BYTES = 48 * 1024;
constexpr int TC_BN_NARROW = 64;                            // tile width for products of at most 64 columns
static_assert(stage_bytes<0>() == STAGE_BYTES && stage_bytes<1>() == STAGE_BYTES && stage_bytes<2>() == STAGE_BYTES,
              "one shared-memory layout");
constexpr uint32_t TBUF_FLOATS = 32 * 32;                   // per-epilogue-warp transpose buffer (XOR-swizzled)
constexpr int TC_PRE = 3;                                   // source chunks in flight per epilogue warp
constexpr uint32_t EPI_FLOATS = TBUF_FLOATS * (1 + TC_PRE) + 64;   // transpose + source ring + row pointers
constexpr int TE_PRE = 5;                                  // TMA epilogue: 32 x 32 chunk buffers per warp
constexpr int TE_LA = 3;                                   // chunks fetched ahead (one store may still read)
constexpr uint32_t TE_CHUNK = 32 * 32 * 4;                 // 4 KiB, 128-byte rows, 128B swizzle
constexpr size_t EPI_BYTES_CP = (size_t)TC_EPI_WARPS * EPI_FLOATS * 4;
constexpr size_t EPI_BYTES_TMA = (size_t)TC_EPI_WARPS * TE_PRE * TE_CHUNK;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * STAGE_BYTES + (EPI_BYTES_CP > EPI_BYTES_TMA ? EPI_BYTES_CP : EPI_BYTES_TMA) +
                           1024;
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s per wait

struct TcArgs {
    float* O; long long ldo, sO;
    int M, N, kch;
    int kch1, a2_off;                // K chunks from the first A map; row offset of the second map
    int tiles_m, tiles_n, tiles;
    int nbox;
    int cl;                          // CTA pairs (cluster of 2) sharing B by TMA multicast
    int units, units_per_box;        // work units: tiles, or row-tile pairs x column tiles when cl
    int vec;                         // rows of O and W are 16-byte aligned: float4 epilogue
    int tma_epi;                     // O is 16-byte aligned: source tiles in and results out by TMA
    int mode, split;
    const int* perm; long long sP;
    const float* W; long long ldw, sW;
    const int* skip;
    int* status;
    const float* invt; long long sInvt;   // format 2: 1 / scale of each column of the right operand
    // fused gather of the next product (TMA epilogue only): output row r goes
    // to the next split right operand nG at K index ninv[r - ng_off] (or
    // r - ng_off without ninv) when that lies in [0, ng_len) and is >= 0, and
    // rows [nw_off, nw_off + nw_len) are saved to nW
    void* nG; long long ng_plane, nsG; int ngK;
    const int* ninv; long long nsInv; int ng_off, ng_len;
    float* nW; long long nsW, nldw; int nw_off, nw_len;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Set by the first CTA whose wait gives up; every other wait then returns at
// once, so a broken launch ends in about WAIT_NS instead of spinning per CTA.
__device__ int g_tc_abort;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase; false when it gave up.  The epilogue
// warps back off (spinning warps steal issue slots); the single-thread TMA
// and MMA roles poll (try_wait already suspends in hardware for a while).
template <bool kBackoff = true>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (kBackoff && it >= 8) __nanosleep(it < 64 ? 32 : 128);
        if ((it & 255u) == 255u) {
            if (*reinterpret_cast<volatile int*>(&g_tc_abort)) return false;
            if (global_ns() - t0 > WAIT_NS) {
                atomicExch(&g_tc_abort, 1);
                return false;
            }
        }
    }
}

// Bounded wait used only to let copies already in flight land before a CTA
// that gave up exits (it does not return early on the abort flag).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return;
        __nanosleep(128);
        if ((it & 63u) == 63u && global_ns() - t0 > WAIT_NS / 4) return;
    }
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1,
                                            int c2, int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// TMA load delivered to the same shared-memory offset in every CTA of the
// cluster named in mask, each CTA's mbarrier at bar receiving the bytes.
__device__ __forceinline__ void tma_load_4d_mc(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1,
                                               int c2, int c3, uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%3, %4, %5, %6}], [%2], %7;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "h"(mask)
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t nclusters_x()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, uint32_t bar, int c0, int c1, int c2)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, uint32_t src, int c0, int c1, int c2)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(tm)),
                 "r"(src), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D(tmem) (+)= A(smem) * B(smem)^T, M = 128, N = TC_BN, K = 8, TF32 in, FP32 accumulate.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Arrive, once the MMAs issued so far complete, on the mbarrier at bar in every
// CTA of the cluster named in mask.
__device__ __forceinline__ void mma_commit_mc(uint32_t bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::
                     "r"(bar),
                 "h"(mask)
                 : "memory");
}

// The CTA's sequence of work units.  Alone, a CTA takes tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... (box-major, so a box's A and G stay in L2 while
// its tiles run).  In a pair, both CTAs of cluster c take units c, c + nclusters,
// ...; a unit is a pair of vertically adjacent row tiles at one column tile,
// the CTA of rank r taking row tile 2 i + r.
struct TcSched {
    int u0, ustep, units, upb, tiles_n, rank, cl, bn;
    __device__ bool skipped(int u, const int* skip) const { return skip && skip[u / upb]; }
    __device__ int first_from(int u, const int* skip) const
    {
        while (u < units && skipped(u, skip)) u += ustep;
        return u;
    }
    __device__ void decode(int u, int& box, int& m0, int& n0) const
    {
        box = u / upb;
        const int rem = u - box * upb, mi = rem / tiles_n;
        n0 = (rem - mi * tiles_n) * bn;
        m0 = (cl ? 2 * mi + rank : mi) * TC_BM;
    }
};

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 64-byte swizzle, rows of
// 64 bytes (16 FP32 values), 8-row core groups 512 bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
    d |= (uint64_t)(512 >> 4) << 32;            // stride byte offset
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)4 << 61;                     // 64-byte swizzle
    return d;
}

// D(tmem) (+)= A(smem) * B(smem)^T, M = 128, N = BN, K = 16, BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// The split pieces of x in operand format FMT, written to plane pl of a
// buffer of FP32 containers (FMT 0: tf32(x), tf32(x - hi)) or BF16 bits
// (FMT 1: successive BF16 roundings; FMT 2: FP16 roundings of x and x - hi,
// x already scaled; every remainder is exact in FP32).
template <int FMT>
__device__ __forceinline__ void split_store(void* dst, long long idx, long long plane, float x)
{
    if constexpr (FMT == 0) {
        float* d = static_cast<float*>(dst);
        const float hi = to_tf32(x);
        d[idx] = hi;
        d[plane + idx] = to_tf32(x - hi);
    } else if constexpr (FMT == 2) {
        __half* d = static_cast<__half*>(dst);
        const __half h = __float2half_rn(x);
        d[idx] = h;
        d[plane + idx] = __float2half_rn(x - __half2float(h));
    } else {
        unsigned short* d = static_cast<unsigned short*>(dst);
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h);
        const __nv_bfloat16 m = __float2bfloat16_rn(r1);
        const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
        d[idx] = __bfloat16_as_ushort(h);
        d[plane + idx] = __bfloat16_as_ushort(m);
        d[2 * plane + idx] = __bfloat16_as_ushort(l);
    }
}

// Format 2: the accumulator chunk's 32 columns times 1 / their right-operand
// scale.  Lane l holds the scales of columns l, l + 32, ... of the tile in
// its8 (loaded once per tile); each chunk takes its8[0] by shuffles and
// shifts the rest down.
__device__ __forceinline__ void scale_chunk(uint32_t (&v)[32], float (&its8)[8])
{
    const float sl = its8[0];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __float_as_uint(__uint_as_float(v[c]) * __shfl_sync(0xffffffffu, sl, c));
#pragma unroll
    for (int c8 = 0; c8 < 7; ++c8) its8[c8] = its8[c8 + 1];
}
__device__ __forceinline__ void load_tile_scales(float (&its8)[8], const float* ib, int nch, int lane)
{
#pragma unroll
    for (int c8 = 0; c8 < 8; ++c8) its8[c8] = c8 < nch ? __ldg(ib + 32 * c8 + lane) : 1.0f;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent update product O <- src - A G over (box, row tile, column tile),
// in the work-unit order of TcSched.  TMEM holds two 128 x BN FP32
// accumulators: the epilogue drains one while the MMAs fill the other.  BN
// is the format's tile width, or TC_BN_NARROW for products with few columns
// (the solves of a few right-hand sides), which would otherwise spend most
// of each MMA on padding.
template <int FMT, int BNT>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_update(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
            const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmO, TcArgs a)
{
    using Fm = TcFmt<FMT>;
    constexpr int BN = BNT, KPC = Fm::KPC, NPL = Fm::NPL;
    constexpr uint32_t B_TILE = (uint32_t)BN * ROWB;
    constexpr uint32_t STAGE_TX = (uint32_t)NPL * (A_TILE + B_TILE);   // bytes a stage receives
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t ld_bar[TC_EPI_WARPS][TE_PRE];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];
    __shared__ __align__(8) uint64_t tempty_bar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* sbase_ptr = smem_raw + (sbase - smem_u32(smem_raw));
    TcSched sc;
    sc.bn = BN;
    sc.cl = a.cl;
    sc.tiles_n = a.tiles_n;
    sc.units = a.units;
    sc.upb = a.units_per_box;
    if (a.cl) {
        sc.u0 = (int)cluster_id_x();
        sc.ustep = (int)nclusters_x();
        sc.rank = (int)cluster_ctarank();
    } else {
        sc.u0 = blockIdx.x;
        sc.ustep = gridDim.x;
        sc.rank = 0;
    }
    float* tbuf_all = reinterpret_cast<float*>(sbase_ptr + TC_STAGES * STAGE_BYTES);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), a.cl ? 2 : 1);   // a pair: both CTAs' MMAs release a stage
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), TC_EPI_WARPS);
        }
        for (int w = 0; w < TC_EPI_WARPS; ++w)
            for (int q = 0; q < TE_PRE; ++q) mbar_init(smem_u32(&ld_bar[w][q]), 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), 2 * BN);
    tc_fence_before();
    __syncthreads();
    if (a.cl) cluster_sync_all();   // the partner's barriers exist before any multicast reaches them
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA2)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            uint32_t g = 0;
            bool ok = true;
            for (int u = sc.u0; u < sc.units && ok; u += sc.ustep) {
                if (sc.skipped(u, a.skip)) continue;
                int box, m0, n0;
                sc.decode(u, box, m0, n0);
                for (int ch = 0; ch < a.kch; ++ch, ++g) {
                    const int s = g % TC_STAGES;
                    const uint32_t use = g / TC_STAGES;
                    if (g >= TC_STAGES && !mbar_wait<false>(smem_u32(&empty_bar[s]), (use - 1) & 1)) {
                        fail_sh = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    mbar_expect_tx(fb, STAGE_TX);
                    // A's K chunks past kch1 come from the second map, whose row 0 is
                    // row a2_off of the product (rows above it load as zeros)
                    const bool second = ch >= a.kch1;
                    const CUtensorMap* ma = second ? &tmA2 : &tmA;
                    const int ka = (second ? ch - a.kch1 : ch) * KPC, ra = second ? m0 - a.a2_off : m0;
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) tma_load_4d(st + pl * A_TILE, ma, fb, ka, ra, pl, box);
                    const uint32_t sb0 = st + NPL * A_TILE;
                    if (a.cl) {
                        // this CTA's half of B's rows, into both CTAs of the pair
                        const uint32_t off = (uint32_t)sc.rank * (B_TILE / 2);
                        const int nr = n0 + sc.rank * (BN / 2);
#pragma unroll
                        for (int pl = 0; pl < NPL; ++pl)
                            tma_load_4d_mc(sb0 + pl * B_TILE + off, &tmB, fb, ch * KPC, nr, pl, box, 0x3);
                    } else {
#pragma unroll
                        for (int pl = 0; pl < NPL; ++pl) tma_load_4d(sb0 + pl * B_TILE, &tmB, fb, ch * KPC, n0, pl, box);
                    }
                }
            }
            // Drain: the last loads issued into each stage have landed, and
            // (in a pair) both MMAs have released every stage, so no arrival
            // from the partner is still on its way when this CTA exits.
            for (uint32_t h = (g > TC_STAGES ? g - TC_STAGES : 0); h < g; ++h) {
                if (!mbar_wait<false>(smem_u32(&full_bar[h % TC_STAGES]), (h / TC_STAGES) & 1)) fail_sh = 1;
                if (!mbar_wait<false>(smem_u32(&empty_bar[h % TC_STAGES]), (h / TC_STAGES) & 1)) fail_sh = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc =
                FMT == 0 ? tf32_idesc(TC_BM, BN) : (FMT == 1 ? bf16_idesc(TC_BM, BN) : f16_idesc(TC_BM, BN));
            uint32_t g = 0, j = 0;
            bool ok = true;
            for (int u = sc.u0; u < sc.units && ok; u += sc.ustep) {
                if (sc.skipped(u, a.skip)) continue;
                const int b = j & 1;
                const uint32_t uj = j >> 1;
                if (j >= 2 && !mbar_wait<false>(smem_u32(&tempty_bar[b]), (uj - 1) & 1)) { fail_sh = 1; break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int ch = 0; ch < a.kch; ++ch, ++g) {
                    const int s = g % TC_STAGES;
                    if (!mbar_wait<false>(smem_u32(&full_bar[s]), (g / TC_STAGES) & 1)) { fail_sh = 1; ok = false; break; }
                    tc_fence_after();
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    uint64_t ad[NPL], bd[NPL];
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) {
                        ad[pl] = sw64_desc(st + pl * A_TILE);
                        bd[pl] = sw64_desc(st + NPL * A_TILE + pl * B_TILE);
                    }
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t o = (uint64_t)((kk * 32) >> 4);   // one MMA's K: 32 bytes of the row
                        const uint32_t acc0 = (ch | kk) != 0;
                        if constexpr (FMT == 0) {
                            mma_tf32(d, ad[0] + o, bd[0] + o, idesc, acc0);
                            mma_tf32(d, ad[0] + o, bd[1] + o, idesc, 1);
                            mma_tf32(d, ad[1] + o, bd[0] + o, idesc, 1);
                        } else if constexpr (FMT == 2) {
                            mma_bf16(d, ad[1] + o, bd[0] + o, idesc, acc0);
                            mma_bf16(d, ad[0] + o, bd[1] + o, idesc, 1);
                            mma_bf16(d, ad[0] + o, bd[0] + o, idesc, 1);
                        } else {
                            // smallest terms first
                            mma_bf16(d, ad[2] + o, bd[0] + o, idesc, acc0);
                            mma_bf16(d, ad[1] + o, bd[1] + o, idesc, 1);
                            mma_bf16(d, ad[0] + o, bd[2] + o, idesc, 1);
                            mma_bf16(d, ad[1] + o, bd[0] + o, idesc, 1);
                            mma_bf16(d, ad[0] + o, bd[1] + o, idesc, 1);
                            mma_bf16(d, ad[0] + o, bd[0] + o, idesc, 1);
                        }
                    }
                    if (a.cl) mma_commit_mc(smem_u32(&empty_bar[s]), 0x3);
                    else mma_commit(smem_u32(&empty_bar[s]));
                }
                mma_commit(smem_u32(&tfull_bar[b]));
                ++j;
            }
        }
    } else if (a.tma_epi) {
        // Epilogue warps 2..5, TMA form: warp w owns TMEM lane quarter qd = w % 4
        // (tile rows 32 qd .. +31) and a ring of TE_PRE 32 x 32 buffers.  Lane 0
        // fetches each chunk's source rows from O by TMA TE_LA chunks ahead
        // (across tiles; rows and columns past O's edge arrive as zeros); each
        // lane then owns one row: it reads the accumulator row from TMEM,
        // replaces the staged row by src - acc in place (128B swizzle: 16-byte
        // unit u of row r sits at u ^ (r % 8), so a quarter-warp touches 8
        // distinct bank groups) and lane 0 stores the chunk back by TMA, which
        // clips at O's edge.  Rows whose source is zero (SET, the pivot block
        // in FWD, below the split in BWD) or a saved row W (FWD rows whose
        // pivot source lies above the split) ignore the staged row.
        const int qd = warp & 3, ew = warp - 2;
        const uint32_t ring = sbase + TC_STAGES * STAGE_BYTES + (uint32_t)ew * (TE_PRE * TE_CHUNK);
        unsigned char* ring_p = sbase_ptr + TC_STAGES * STAGE_BYTES + (size_t)ew * (TE_PRE * TE_CHUNK);
        const uint32_t lbar0 = smem_u32(&ld_bar[ew][0]);
        const bool need_src = a.mode != GM_SET;
        if (lane == 0) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmO)) : "memory");
        auto first_from = [&](int u) { return sc.first_from(u, a.skip); };
        auto geom = [&](int u, int& box, int& m0, int& n0, int& nch) {
            sc.decode(u, box, m0, n0);
            nch = (min(BN, a.N - n0) + 31) / 32;
        };
        // load cursor (lane 0): next chunk to fetch is number lg, chunk lcc of unit lt
        int lt = first_from(sc.u0), lcc = 0;
        uint32_t lg = 0;
        auto issue = [&]() {
            int box, m0, n0, nch;
            geom(lt, box, m0, n0, nch);
            const uint32_t buf = lg % TE_PRE;
            mbar_expect_tx(lbar0 + 8 * buf, TE_CHUNK);
            tma_load_3d(ring + buf * TE_CHUNK, &tmO, lbar0 + 8 * buf, n0 + 32 * lcc, m0 + 32 * qd, box);
            ++lg;
            if (++lcc == nch) {
                lcc = 0;
                lt = first_from(lt + sc.ustep);
            }
        };
        if (lane == 0 && need_src)
            for (int i = 0; i < TE_LA && lt < sc.units; ++i) issue();
        uint32_t g = 0, j = 0;
        bool ok = true;
        for (int t = first_from(sc.u0); t < sc.units && ok; t = first_from(t + sc.ustep), ++j) {
            int box, m0, n0, nch;
            geom(t, box, m0, n0, nch);
            const int b = j & 1;
            float its8[8];   // format 2 column scales (the loads overlap the wait)
            if constexpr (FMT == 2) load_tile_scales(its8, a.invt + box * a.sInvt + n0, nch, lane);
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[b]), (j >> 1) & 1);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            // this lane's row: source 0 = zero, 1 = staged O row, 2 = saved row of W
            const int myr = m0 + qd * 32 + lane;
            int ngi = -1, nwr = -1;   // the row's K index in the next product's G, its row in the next W
            if (a.nG && myr < a.M) {
                const int rr = myr - a.ng_off;
                if (rr >= 0 && rr < a.ng_len) ngi = a.ninv ? a.ninv[box * a.nsInv + rr] : rr;
                const int wr = myr - a.nw_off;
                if (a.nW && wr >= 0 && wr < a.nw_len) nwr = wr;
            }
            void* nGb = nullptr;
            if (ngi >= 0)
                nGb = FMT == 0 ? (void*)(static_cast<float*>(a.nG) + box * a.nsG)
                               : (void*)(static_cast<unsigned short*>(a.nG) + box * a.nsG);   // not with FMT 2
            int srck = 0;
            const float* wrow = nullptr;
            if (myr < a.M) {
                if (a.mode == GM_FWD) {
                    if (myr >= a.split) {
                        const int pr = a.perm[box * a.sP + myr];
                        if (pr >= a.split) srck = 1;
                        else {
                            srck = 2;
                            wrow = a.W + box * a.sW + (long long)pr * a.ldw;
                        }
                    }
                } else if (a.mode == GM_BWD) {
                    srck = myr < a.split ? 1 : 0;
                } else if (a.mode == GM_ACC) {
                    srck = 1;
                }
            }
            for (int cc = 0; cc < nch; ++cc, ++g) {
                const uint32_t buf = g % TE_PRE;
                if (lane == 0) {
                    if (need_src) {
                        if (lt < sc.units) {
                            bulk_wait_read<TE_PRE - TE_LA - 1>();   // the buffer's last store has read it
                            issue();
                        }
                    } else {
                        bulk_wait_read<TE_PRE - 1>();
                    }
                }
                __syncwarp();
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * BN + cc * 32), v);
                if (cc == nch - 1) {
                    // the accumulator is in registers: hand the TMEM buffer back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
                }
                if (need_src && !mbar_wait(lbar0 + 8 * buf, (g / TE_PRE) & 1)) ok = false;
                if (!__all_sync(0xffffffffu, ok ? 1 : 0)) {
                    ok = false;
                    break;
                }
                float4* rowp = reinterpret_cast<float4*>(ring_p + buf * TE_CHUNK + lane * 128);
                const int cb = n0 + cc * 32;
                if constexpr (FMT == 2) scale_chunk(v, its8);
                // all eight source reads first, then the eight results
                float4 sv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    sv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (srck == 1) {
                        sv[u] = rowp[u ^ (lane & 7)];
                    } else if (srck == 2) {
                        const int c = cb + 4 * u;
                        sv[u].x = c < a.N ? wrow[c] : 0.f;
                        sv[u].y = c + 1 < a.N ? wrow[c + 1] : 0.f;
                        sv[u].z = c + 2 < a.N ? wrow[c + 2] : 0.f;
                        sv[u].w = c + 3 < a.N ? wrow[c + 3] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float4* p4 = rowp + (u ^ (lane & 7));
                    const float4 o = make_float4(sv[u].x - __uint_as_float(v[4 * u]), sv[u].y - __uint_as_float(v[4 * u + 1]),
                                                 sv[u].z - __uint_as_float(v[4 * u + 2]), sv[u].w - __uint_as_float(v[4 * u + 3]));
                    *p4 = o;
                    if (ngi >= 0 || nwr >= 0) {
                        const int c = cb + 4 * u;
                        const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            if (c + j >= a.N) break;
                            if (ngi >= 0) split_store<FMT>(nGb, (long long)(c + j) * a.ngK + ngi, a.ng_plane, ov[j]);
                            if (nwr >= 0) a.nW[box * a.nsW + (long long)nwr * a.nldw + c + j] = ov[j];
                        }
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tma_store_3d(&tmO, ring + buf * TE_CHUNK, cb, m0 + qd * 32, box);
                    bulk_commit();
                }
            }
        }
        if (lane == 0) {
            if (!ok) {
                fail_sh = 1;
                for (uint32_t h = g; h < lg; ++h) mbar_drain(lbar0 + 8 * (h % TE_PRE), (h / TE_PRE) & 1);
            }
            bulk_wait_all();
        }
        __syncwarp();
    } else {
        // Epilogue warps 2..5: warp w owns TMEM lane quarter qd = w % 4 (tile
        // rows 32 qd .. 32 qd + 31).  The source rows of each 32 x 32 chunk are
        // brought into shared memory with cp.async TC_PRE chunks ahead (absent
        // rows and columns are zero-filled); the accumulator chunk (thread =
        // row) is transposed through shared memory; then the chunk is written
        // out row by row with coalesced stores.  When rows are 16-byte aligned
        // (a.vec) every copy, shared access and store moves 16 bytes: lane l
        // covers columns 4 (l % 8) .. +3 of rows l / 8 + 4 i.
        const int qd = warp & 3;
        float* eb = tbuf_all + (warp - 2) * EPI_FLOATS;
        float* tb = eb;                                       // transpose buffer [32][32], 16-byte XOR swizzle
        float* sb = eb + TBUF_FLOATS;                         // TC_PRE source chunks [32][32]
        const float** sp = reinterpret_cast<const float**>(eb + TBUF_FLOATS * (1 + TC_PRE));
        const uint32_t sb_u32 = smem_u32(sb);
        const int l8 = lane & 7, l3 = lane >> 3;
        uint32_t j = 0;
        for (int u = sc.u0; u < sc.units; u += sc.ustep) {
            if (sc.skipped(u, a.skip)) continue;
            int box, m0, n0;
            sc.decode(u, box, m0, n0);
            const int row0 = m0 + qd * 32;
            const int rows_here = max(0, min(32, a.M - row0));
            float* Ob = a.O + box * a.sO;
            {
                const int myr = row0 + lane;
                const float* srow = nullptr;
                if (lane < rows_here) {
                    if (a.mode == GM_FWD) {
                        if (myr >= a.split) {
                            const int pr = a.perm[box * a.sP + myr];
                            srow = (pr >= a.split) ? Ob + (long long)myr * a.ldo
                                                   : a.W + box * a.sW + (long long)pr * a.ldw;
                        }
                    } else if (a.mode == GM_BWD) {
                        if (myr < a.split) srow = Ob + (long long)myr * a.ldo;
                    } else if (a.mode == GM_ACC) {
                        srow = Ob + (long long)myr * a.ldo;
                    }
                }
                sp[lane] = srow;
            }
            __syncwarp();
            const int nchunks = (min(BN, a.N - n0) + 31) / 32;
            float its8[8];   // format 2 column scales
            if constexpr (FMT == 2) load_tile_scales(its8, a.invt + box * a.sInvt + n0, nchunks, lane);
            auto prefetch = [&](int cc) {
                const int cb = n0 + cc * 32;
                const uint32_t buf = sb_u32 + (uint32_t)((cc % TC_PRE) * 4096);
                if (a.vec) {
                    const int col = cb + 4 * l8;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int rr = l3 + 4 * i;
                        const float* q = sp[rr];
                        const bool have = q != nullptr && col < a.N;   // N % 4 == 0 when a.vec
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(buf + (rr * 32 + 4 * l8) * 4),
                                     "l"(have ? q + col : Ob), "r"(have ? 16 : 0)
                                     : "memory");
                    }
                } else {
                    const int col = cb + lane;
#pragma unroll 8
                    for (int rr = 0; rr < 32; ++rr) {
                        const float* q = sp[rr];
                        const bool have = q != nullptr && col < a.N;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(buf + (rr * 32 + lane) * 4),
                                     "l"(have ? q + col : Ob), "r"(have ? 4 : 0)
                                     : "memory");
                    }
                }
            };
            for (int cc = 0; cc < TC_PRE - 1; ++cc) {
                if (cc < nchunks) prefetch(cc);
                asm volatile("cp.async.commit_group;" ::: "memory");
            }
            const int b = j & 1;
            bool ok = true;
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[b]), (j >> 1) & 1);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                asm volatile("cp.async.wait_all;" ::: "memory");
                if (lane == 0) fail_sh = 1;
                break;
            }
            tc_fence_after();
            float* orow0 = Ob + (long long)row0 * a.ldo;
#pragma unroll 1
            for (int cc = 0; cc < nchunks; ++cc) {
                if (cc + TC_PRE - 1 < nchunks) prefetch(cc + TC_PRE - 1);
                asm volatile("cp.async.commit_group;" ::: "memory");
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * BN + cc * 32), v);
                if constexpr (FMT == 2) scale_chunk(v, its8);
                // row = lane; 16-byte group g of the row goes to slot g ^ (lane & 7)
#pragma unroll
                for (int g = 0; g < 8; ++g)
                    *reinterpret_cast<float4*>(tb + lane * 32 + 4 * (g ^ (lane & 7))) =
                        make_float4(__uint_as_float(v[4 * g]), __uint_as_float(v[4 * g + 1]),
                                    __uint_as_float(v[4 * g + 2]), __uint_as_float(v[4 * g + 3]));
                asm volatile("cp.async.wait_group %0;" ::"n"(TC_PRE - 1) : "memory");
                __syncwarp();
                const float* sc = sb + (cc % TC_PRE) * 1024;
                const int cb = n0 + cc * 32;
                if (a.vec) {
                    const int col = cb + 4 * l8;
                    if (col < a.N) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int rr = l3 + 4 * i;
                            if (rr < rows_here) {
                                const float4 s4 = *reinterpret_cast<const float4*>(sc + rr * 32 + 4 * l8);
                                const float4 t4 = *reinterpret_cast<const float4*>(tb + rr * 32 + 4 * (l8 ^ (rr & 7)));
                                *reinterpret_cast<float4*>(orow0 + (long long)rr * a.ldo + col) =
                                    make_float4(s4.x - t4.x, s4.y - t4.y, s4.z - t4.z, s4.w - t4.w);
                            }
                        }
                    }
                } else {
                    const int col = cb + lane;
                    if (col < a.N) {
#pragma unroll 8
                        for (int rr = 0; rr < rows_here; ++rr)
                            orow0[(long long)rr * a.ldo + col] =
                                sc[rr * 32 + lane] - tb[rr * 32 + 4 * ((lane >> 2) ^ (rr & 7)) + (lane & 3)];
                    }
                }
                __syncwarp();
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
            ++j;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (a.cl) cluster_sync_all();   // neither CTA of a pair leaves while the other may still reach it
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
    if (threadIdx.x == 0 && fail_sh && a.status)
        for (int bx = 0; bx < a.nbox; ++bx) atomicCAS(a.status + bx, 0, HPS_ETIMEOUT);
}

// dst = the split planes (rows x NB each, zero beyond nb) of the first nb
// columns of src (rows of pitch lds).
template <int FMT>
__global__ void k_pack_split(const float* __restrict__ src, long long lds, long long sS, int rows, int NB, int nb,
                             void* __restrict__ dst, long long sD)
{
    const int box = blockIdx.y;
    const long long total = (long long)rows * NB;
    void* db = FMT == 0 ? (void*)(static_cast<float*>(dst) + box * sD) : (void*)(static_cast<unsigned short*>(dst) + box * sD);
    const float* sb = src + box * sS;
    // rows over the grid, columns over the threads (no index division)
    for (int r = blockIdx.x * blockDim.y + threadIdx.y; r < rows; r += gridDim.x * blockDim.y) {
        const float* srow = sb + (long long)r * lds;
        for (int c = threadIdx.x; c < NB; c += blockDim.x)
            split_store<FMT>(db, (long long)r * NB + c, total, c < nb ? srow[c] : 0.0f);
    }
}

// Gather the step's rows (through perm), save the unpermuted rows to W, and
// write the split, transposed G: Gp[plane][c][i] for i < NB (zero for i >= nb).
template <int FMT>
__global__ void k_gather_pack(const float* __restrict__ M, long long ldm, long long sM, int k, int nb, int NB,
                              int c0, int nc, const int* __restrict__ perm, long long sP, float* __restrict__ W,
                              long long ldw, long long sW, void* __restrict__ Gp, long long plane, long long sGp,
                              const int* skip)
{
    __shared__ float tile[32][33];
    const int box = blockIdx.z;
    if (skip && skip[box]) return;
    const int i0 = blockIdx.y * 32, cb = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float* Mb = M + box * sM;
    for (int ii = ty; ii < 32; ii += 8) {
        const int i = i0 + ii, c = cb + tx;
        float v = 0.0f;
        if (i < nb && c < nc) {
            const int src = k + (perm ? perm[box * sP + i] : i);
            v = Mb[(long long)src * ldm + c0 + c];
            if (W) W[box * sW + (long long)i * ldw + c] = Mb[(long long)(k + i) * ldm + c0 + c];
        }
        tile[ii][tx] = v;
    }
    __syncthreads();
    void* G = FMT == 0 ? (void*)(static_cast<float*>(Gp) + box * sGp) : (void*)(static_cast<unsigned short*>(Gp) + box * sGp);
    for (int cc = ty; cc < 32; cc += 8) {
        const int c = cb + cc, i = i0 + tx;
        if (c < nc) split_store<FMT>(G, (long long)c * NB + i, plane, tile[tx][cc]);
    }
}

// Format 2 scales: 2^(15 - e) for a column maximum mx < 2^e (so every scaled
// value stays below 2^15, inside FP16's range after rounding), 1 for an empty
// or all-zero column; exponents are clamped to +-100.  Built from the
// exponent field, so both the scale and its inverse are exact powers of two.
__device__ __forceinline__ int scale_exp(float mx)
{
    if (!(mx > 0.0f)) return 0;
    const int eb = (int)((__float_as_uint(mx) >> 23) & 0xffu);   // mx < 2^(eb - 126) (subnormals: 2^-126)
    if (eb == 0xff) return 0;                                     // inf: left unscaled, it shows in the result
    int e = 15 - (eb == 0 ? -126 : eb - 126);
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}
__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }

// Format 2 left operand: dst = the split planes (rows x NB, zero beyond nb)
// of src's first nb columns, each column k scaled by 2^s_k (scale_exp of its
// maximum over the rows); rc[k] = 2^-s_k, the factor the right operand's row
// k takes.  One CTA per box and 32 columns: a pass for the maxima, a pass
// for the values.
__global__ void k_pack_f16(const float* __restrict__ src, long long lds, long long sS, int rows, int NB, int nb,
                           __half* __restrict__ dst, long long sD, float* __restrict__ rc, long long sC)
{
    __shared__ float red[8][33];
    __shared__ float scl[32];
    const int box = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
    const int c = blockIdx.x * 32 + tx;
    const float* sb = src + box * sS;
    float mx = 0.0f;
    if (c < nb)
        for (int r = ty; r < rows; r += 8) mx = fmaxf(mx, fabsf(sb[(long long)r * lds + c]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0) {
        float m = red[0][tx];
#pragma unroll
        for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i][tx]);
        const int e = scale_exp(m);
        scl[tx] = pow2f(e);
        if (c < NB) rc[box * sC + c] = pow2f(-e);
    }
    __syncthreads();
    if (c >= NB) return;
    const float sc = scl[tx];
    const long long total = (long long)rows * NB;
    __half* db = dst + box * sD;
    for (int r = ty; r < rows; r += 8)
        split_store<2>(db, (long long)r * NB + c, total, c < nb ? sb[(long long)r * lds + c] * sc : 0.0f);
}

// Format 2 right operand: as k_gather_pack, with row i of the gathered block
// multiplied by rc[i] (the left operand's K scale inverse) and then each
// column c scaled by 2^t_c (scale_exp of its maximum); invt[c] = 2^-t_c for
// the epilogue.  One CTA per box and 32 columns, the whole K extent (gK rows)
// in shared memory.
__global__ void k_gather_pack_f16(const float* __restrict__ M, long long ldm, long long sM, int k, int nb, int gK,
                                  int c0, int nc, const int* __restrict__ perm, long long sP, float* __restrict__ W,
                                  long long ldw, long long sW, __half* __restrict__ Gp, long long plane, long long sGp,
                                  const float* __restrict__ rc, long long sC, float* __restrict__ invt,
                                  long long sIt, const int* skip)
{
    extern __shared__ float gt[];   // [gK][33]
    __shared__ float red[8][33];
    __shared__ float scl[32];
    const int box = blockIdx.y;
    if (skip && skip[box]) return;
    const int cb = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y;
    const float* Mb = M + box * sM;
    const float* rcb = rc + box * sC;
    const int c = cb + tx;
    const int ncc = min(32, nc - cb);   // columns of this chunk (uniform over the CTA)
    if (ncc == 32) {
        float mx = 0.0f;
        for (int i = ty; i < gK; i += 8) {
            float v = 0.0f;
            if (i < nb) {
                const int srcr = k + (perm ? perm[box * sP + i] : i);
                v = Mb[(long long)srcr * ldm + c0 + c] * rcb[i];
                if (W) W[box * sW + (long long)i * ldw + c] = Mb[(long long)(k + i) * ldm + c0 + c];
                mx = fmaxf(mx, fabsf(v));
            }
            gt[i * 33 + tx] = v;
        }
        red[ty][tx] = mx;
    } else {
        // a narrow chunk (few right-hand sides, or the last columns): the 256
        // threads split into ncc groups of tpc, one group per column, each
        // thread taking every tpc-th row, so the scattered pivot-row loads of
        // a column are issued together; column maxima through shared memory.
        __shared__ float colmax[256];
        const int tid = ty * 32 + tx;
        const int tpc = 256 / ncc;               // threads per column, >= 8 (ncc <= 31)
        const int cc = tid / tpc, r0 = tid - cc * tpc;
        float mx = 0.0f;
        if (cc < ncc) {
            for (int i = r0; i < gK; i += tpc) {
                float v = 0.0f;
                if (i < nb) {
                    const int srcr = k + (perm ? perm[box * sP + i] : i);
                    v = Mb[(long long)srcr * ldm + c0 + cb + cc] * rcb[i];
                    if (W) W[box * sW + (long long)i * ldw + cb + cc] = Mb[(long long)(k + i) * ldm + c0 + cb + cc];
                    mx = fmaxf(mx, fabsf(v));
                }
                gt[i * 33 + cc] = v;
            }
        }
        colmax[tid] = mx;
        __syncthreads();
        if (tid < 32) {
            float m = 0.0f;
            if (tid < ncc)
                for (int t = tid * tpc; t < (tid + 1) * tpc; ++t) m = fmaxf(m, colmax[t]);
            red[0][tid] = m;
#pragma unroll
            for (int r = 1; r < 8; ++r) red[r][tid] = 0.0f;
        }
    }
    __syncthreads();
    if (ty == 0) {
        float m = red[0][tx];
#pragma unroll
        for (int i = 1; i < 8; ++i) m = fmaxf(m, red[i][tx]);
        const int e = scale_exp(m);
        scl[tx] = pow2f(e);
        invt[box * sIt + c] = pow2f(-e);
    }
    __syncthreads();
    __half* G = Gp + box * sGp;
    for (int cc = ty; cc < 32; cc += 8) {
        const int col = cb + cc;
        if (col >= nc) break;
        const float sc = scl[cc];
        for (int i = tx; i < gK; i += 32) split_store<2>(G, (long long)col * gK + i, plane, gt[i * 33 + cc] * sc);
    }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 4-D map over split K-major operands: (k, row, plane, box); K, strides and
// the box in elements of format FMT, one 64-byte row of K per box row.
template <int FMT>
bool make_map(CUtensorMap* tm, const void* base, int K, long long rows, long long plane_elems, long long box_elems,
              int nbox, int box_rows)
{
    using Fm = TcFmt<FMT>;
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)Fm::NPL, (cuuint64_t)nbox};
    cuuint64_t strides[3] = {(cuuint64_t)K * Fm::EB, (cuuint64_t)plane_elems * Fm::EB, (cuuint64_t)box_elems * Fm::EB};
    cuuint32_t boxd[4] = {(cuuint32_t)Fm::KPC, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = FMT == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                            : (FMT == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    CUresult r = fn(tm, dt, 4,
                    const_cast<void*>(base), dims, strides, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Left operand of an update product: split rows of NB values (K-major), a_rows
// rows per box; a second part (rows offset by a2_off, K2 further values of K)
// joins a pair of LU steps into one product.  Pointers and strides are in
// elements of the plan's operand format.
struct TcLeft {
    const void* A; long long rows, sA;
    const void* A2; long long rows2, sA2;
    int K1, K2, a2_off;
};

TcLeft left1(const void* A, long long rows, long long sA, int K)
{
    TcLeft l{};
    l.A = A; l.rows = rows; l.sA = sA; l.K1 = K;
    return l;
}

template <int FMT, int BNT>
bool launch_tc_update_w(const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                        const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, bool allow_pairs, bool* fused)
{
    using Fm = TcFmt<FMT>;
    const int K = L.K1 + L.K2;
    if (args.M <= 0 || args.N <= 0) return true;
    static int num_sms = 0, max_pairs = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_tc_update<FMT, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        if (num_sms <= 0) num_sms = 1;
        // how many CTA pairs fit at once (an SM whose cluster partner is
        // missing stays idle in pair mode)
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(num_sms & ~1));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = TC_SMEM;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, (void*)k_tc_update<FMT, BNT>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            nc = 0;
        }
        max_pairs = nc;
    }
    TcArgs a = args;
    a.kch = (K + Fm::KPC - 1) / Fm::KPC;
    a.kch1 = L.K2 ? L.K1 / Fm::KPC : a.kch;   // L.K1 is a whole block when a second part follows
    a.a2_off = L.a2_off;
    a.tiles_m = (a.M + TC_BM - 1) / TC_BM;
    a.tiles_n = (a.N + BNT - 1) / BNT;
    a.tiles = a.tiles_m * a.tiles_n * nbox;
    a.nbox = nbox;
    a.cl = (allow_pairs && max_pairs > 0 && a.tiles_m >= 2) ? 1 : 0;
    a.units_per_box = (a.cl ? (a.tiles_m + 1) / 2 : a.tiles_m) * a.tiles_n;
    a.units = a.units_per_box * nbox;
    CUtensorMap ta, ta2, tb;
    if (!make_map<FMT>(&ta, L.A, NB, L.rows, L.rows * NB, L.sA, nbox, TC_BM) ||
        !make_map<FMT>(&tb, Gp, gK, args.N, g_plane, sGp, nbox, a.cl ? BNT / 2 : BNT))
        return false;
    if (L.K2) {
        if (!make_map<FMT>(&ta2, L.A2, NB, L.rows2, L.rows2 * NB, L.sA2, nbox, TC_BM)) return false;
    } else {
        ta2 = ta;
    }
    const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    a.vec = al16(a.O) && (a.ldo % 4 == 0) && (a.sO % 4 == 0) && (a.N % 4 == 0) &&
            (!a.W || (al16(a.W) && a.ldw % 4 == 0 && a.sW % 4 == 0));
    CUtensorMap to{};
    a.tma_epi = 0;
    if (al16(a.O) && a.ldo % 4 == 0 && a.sO % 4 == 0 && allow_tma) {
        auto fn = encode_fn();
        cuuint64_t dims[3] = {(cuuint64_t)a.N, (cuuint64_t)a.M, (cuuint64_t)nbox};
        cuuint64_t strides[2] = {(cuuint64_t)a.ldo * 4, (cuuint64_t)a.sO * 4};
        cuuint32_t boxd[3] = {32, 32, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (fn && fn(&to, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.O, dims, strides, boxd, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            a.tma_epi = 1;
    }
    if (!a.tma_epi) {   // the next product's gather is fused into the TMA epilogue only
        a.nG = nullptr;
        a.nW = nullptr;
    }
    if (fused) *fused = a.nG != nullptr;
    // Refinement replays (skip flags set) are timed apart: their boxes drop out
    // as they converge, so their flop counts are upper bounds.
    const int cls = a.skip ? KC_UPDATE_TC_REFINE : KC_UPDATE_TC;
    prof_begin(cls, st);
    if (a.cl) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(2 * std::min(a.units, max_pairs)));
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = TC_SMEM;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, k_tc_update<FMT, BNT>, ta, ta2, tb, to, a) != cudaSuccess) return false;
    } else {
        dim3 grd((unsigned)std::min(a.units, num_sms));
        k_tc_update<FMT, BNT><<<grd, TC_THREADS, TC_SMEM, st>>>(ta, ta2, tb, to, a);
    }
    const double kk = (double)K;
    prof_end(cls, st, 2.0 * nbox * a.M * (double)a.N * kk,
             (double)nbox * ((a.M + (double)a.N) * kk * Fm::NPL * Fm::EB + 2.0 * a.M * (double)a.N * 4));
    return true;
}

template <int FMT>
bool launch_tc_update_f(const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                        const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, bool allow_pairs, bool* fused)
{
    if (args.N <= TC_BN_NARROW && TcFmt<FMT>::BN > TC_BN_NARROW)
        return launch_tc_update_w<FMT, TC_BN_NARROW>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma,
                                                     allow_pairs, fused);
    return launch_tc_update_w<FMT, TcFmt<FMT>::BN>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma,
                                                   allow_pairs, fused);
}

bool launch_tc_update(int fmt, const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                      const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, bool allow_pairs,
                      bool* fused = nullptr)
{
    if (fmt == 2) return launch_tc_update_f<2>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, allow_pairs, fused);
    return fmt ? launch_tc_update_f<1>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, allow_pairs, fused)
               : launch_tc_update_f<0>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, allow_pairs, fused);
}

// Element `off` of a split-operand buffer of format fmt.
void* pk_at(void* base, long long off, int fmt)
{
    return fmt ? (void*)(static_cast<unsigned short*>(base) + off) : (void*)(static_cast<float*>(base) + off);
}

// rc (format 2 only): the K scales' inverses of this pack, per box stride sC.
void launch_pack_split(int fmt, const float* src, long long lds, long long sS, int rows, int NB, int nb, void* dst,
                       long long sD, int nbox, cudaStream_t st, float* rc = nullptr, long long sC = 0)
{
    const long long total = (long long)rows * NB;
    const dim3 blk(32, 8);   // 8 rows of 32-column strips per CTA
    prof_begin(KC_PACK, st);
    if (fmt == 2) {
        k_pack_f16<<<dim3((unsigned)((NB + 31) / 32), (unsigned)nbox), blk, 0, st>>>(
            src, lds, sS, rows, NB, nb, static_cast<__half*>(dst), sD, rc, sC);
        prof_end(KC_PACK, st, 0.0, (double)nbox * total * (4.0 + 4.0));
        return;
    }
    dim3 grd((unsigned)std::max(1, std::min((rows + 7) / 8, 128)), (unsigned)nbox);
    if (fmt) k_pack_split<1><<<grd, blk, 0, st>>>(src, lds, sS, rows, NB, nb, dst, sD);
    else k_pack_split<0><<<grd, blk, 0, st>>>(src, lds, sS, rows, NB, nb, dst, sD);
    prof_end(KC_PACK, st, 0.0, (double)nbox * total * (4.0 + (fmt ? 6.0 : 8.0)));
}

// rc, sC (format 2 only): the left operand's K scale inverses for the
// gathered rows; invt, sIt: where the column scale inverses go.
void gather_pack_raw(int fmt, const float* M, long long ldm, long long sM, int k, int nb, int gK, int c0, int nc,
                     const int* perm, long long sP, float* W, long long ldw, long long sW, void* Gp, long long plane,
                     long long sGp, const int* skip, int nbox, cudaStream_t st, const float* rc = nullptr,
                     long long sC = 0, float* invt = nullptr, long long sIt = 0)
{
    prof_begin(KC_GATHER, st);
    if (fmt == 2) {
        const dim3 grd((unsigned)((nc + 31) / 32), (unsigned)nbox), blk(32, 8);
        k_gather_pack_f16<<<grd, blk, (size_t)gK * 33 * sizeof(float), st>>>(
            M, ldm, sM, k, nb, gK, c0, nc, perm, sP, W, ldw, sW, static_cast<__half*>(Gp), plane, sGp, rc, sC, invt,
            sIt, skip);
        prof_end(KC_GATHER, st, 0.0, (double)nbox * nb * (double)nc * (4.0 + (W ? 4.0 : 0.0) + 4.0));
        return;
    }
    const dim3 grd((unsigned)((nc + 31) / 32), (unsigned)(gK / 32), (unsigned)nbox), blk(32, 8);
    if (fmt)
        k_gather_pack<1><<<grd, blk, 0, st>>>(M, ldm, sM, k, nb, gK, c0, nc, perm, sP, W, ldw, sW, Gp, plane, sGp, skip);
    else
        k_gather_pack<0><<<grd, blk, 0, st>>>(M, ldm, sM, k, nb, gK, c0, nc, perm, sP, W, ldw, sW, Gp, plane, sGp, skip);
    prof_end(KC_GATHER, st, 0.0, (double)nbox * nb * (double)nc * (4.0 + (W ? 4.0 : 0.0) + (fmt ? 6.0 : 8.0)));
}

void launch_gather_pack(const Plan& P, Work<float>& w, int k, int nb, int c0, int nc, const int* perm, bool save_w,
                        const int* skip, int nbox, cudaStream_t st, const float* rc)
{
    gather_pack_raw(P.fmt, w.M, P.ldm, w.sM, k, nb, P.KG, c0, nc, perm, w.sP, save_w ? w.W : nullptr, P.ldm, w.sG,
                    w.Gp, P.ldm * P.KG, w.sGp, skip, nbox, st, rc, w.sRC, w.it1, w.sIT);
}

TcArgs targs(float* O, long long ldo, long long sO, int M, int N, int mode, int split)
{
    TcArgs a{};
    a.O = O; a.ldo = ldo; a.sO = sO; a.M = M; a.N = N; a.mode = mode; a.split = split;
    return a;
}

}  // namespace

void tc_reset_abort(cudaStream_t st)
{
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_abort) == cudaSuccess) cudaMemsetAsync(p, 0, sizeof(int), st);
}

bool tc_abort_raised()
{
    int v = 0;
    cudaMemcpyFromSymbol(&v, g_tc_abort, sizeof(int));
    return v != 0;
}

// ---------------------------------------------------------------- LU sequences
//
// With step pairs (P.step_pairs), two consecutive LU steps s, s+1 act as one
// step of 2 NB rows wherever they apply to many columns.  Step s+1 applied to
// the columns of F_s, and step s applied (backwards) to the columns of
// B_{s+1}, give the pair's operators:
//   forward  [F_s' | F_{s+1}] (F_{s+1}'s rows start NB rows lower),
//   backward [B_s | B_{s+1}'],
// with the composed row permutation pi_c(i) = pi_s(i) for i < nb_s, else
// pi_s(nb_s + pi_{s+1}(i - nb_s)).  A row below the pair's block still either
// stays in place or receives a block row, so the update epilogue is the same
// with split = 2 NB.  The factorisation updates only the next block's columns
// with step s (look-ahead), factors that panel, then updates everything else
// once with the pair; the solves run one product per pair.  Each pass over the
// trailing rows and right-hand sides then serves two steps.

namespace {

// pi_s <- pi_c (both arrays in shared memory first; one CTA per box).
__global__ void k_perm_compose(int* __restrict__ perm0, const int* __restrict__ perm1, long long sP, int R, int nb0)
{
    extern __shared__ int psh[];
    int* a = psh;
    int* b = psh + R;
    const int box = blockIdx.x;
    int* p0 = perm0 + box * sP;
    const int* p1 = perm1 + box * sP;
    for (int i = threadIdx.x; i < R; i += blockDim.x) a[i] = p0[i];
    for (int i = threadIdx.x; i < R - nb0; i += blockDim.x) b[i] = p1[i];
    __syncthreads();
    for (int i = threadIdx.x; i < R; i += blockDim.x) p0[i] = i < nb0 ? a[i] : a[nb0 + b[i - nb0]];
}

void launch_perm_compose(int* perm0, const int* perm1, long long sP, int R, int nb0, int nbox, cudaStream_t st)
{
    const size_t smem = (size_t)(2 * R - nb0) * sizeof(int);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_perm_compose, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    prof_begin(KC_MISC, st);
    k_perm_compose<<<nbox, 256, smem, st>>>(perm0, perm1, sP, R, nb0);
    prof_end(KC_MISC, st, 0.0, (double)nbox * (3.0 * R - nb0) * 4.0);
}

// inv[r] = i where perm[i] = r for i < w, -1 for the other rows r < R (one
// CTA per box): the K index in a product's G of each row it gathers.
__global__ void k_perm_inverse(const int* __restrict__ perm, int* __restrict__ inv, long long sP, int R, int w)
{
    const int box = blockIdx.x;
    for (int r = threadIdx.x; r < R; r += blockDim.x) inv[box * sP + r] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < w; i += blockDim.x) inv[box * sP + perm[box * sP + i]] = i;
}

// Start of step s's split F_s / B_s in the operand format of the plan.
int npl(const Plan& P) { return P.fmt == 1 ? 3 : 2; }
// Format 2: K scale inverses of F_s and B_s (null otherwise).
const float* rcf(const Plan& P, const Work<float>& w, int s) { return w.rcF ? w.rcF + (long long)s * P.NB : nullptr; }
const float* rcb(const Plan& P, const Work<float>& w, int s) { return w.rcB ? w.rcB + (long long)s * P.NB : nullptr; }
float* rcf_w(const Plan& P, Work<float>& w, int s) { return w.rcF ? w.rcF + (long long)s * P.NB : nullptr; }
float* rcb_w(const Plan& P, Work<float>& w, int s) { return w.rcB ? w.rcB + (long long)s * P.NB : nullptr; }
void* fpk(const Plan& P, const Work<float>& w, int s) { return pk_at(w.Fp, (long long)npl(P) * P.fw_off[s], P.fmt); }
void* bpk(const Plan& P, const Work<float>& w, int s) { return pk_at(w.Bp, (long long)npl(P) * P.bw_off[s], P.fmt); }

// Left operands of the pair (s, s+1).
TcLeft left_fwd_pair(const Plan& P, const Work<float>& w, int s)
{
    TcLeft l{};
    l.A = fpk(P, w, s);
    l.rows = P.n - P.k0[s];
    l.sA = w.sFp;
    l.K1 = P.nbs[s];
    l.A2 = fpk(P, w, s + 1);
    l.rows2 = P.n - P.k0[s + 1];
    l.sA2 = w.sFp;
    l.K2 = P.nbs[s + 1];
    l.a2_off = P.nbs[s];
    return l;
}

TcLeft left_bwd_pair(const Plan& P, const Work<float>& w, int s)
{
    TcLeft l{};
    l.A = bpk(P, w, s);
    l.rows = P.k0[s] + P.nbs[s];
    l.sA = w.sBp;
    l.K1 = P.nbs[s];
    l.A2 = bpk(P, w, s + 1);
    l.rows2 = P.k0[s + 1] + P.nbs[s + 1];
    l.sA2 = w.sBp;
    l.K2 = P.nbs[s + 1];
    l.a2_off = 0;
    return l;
}

// Units of the solves: (first step, 1 or 2 steps).
std::vector<std::pair<int, int>> solve_units(const Plan& P)
{
    std::vector<std::pair<int, int>> u;
    for (int s = 0; s < P.nsteps;) {
        const int len = (P.step_pairs && s + 1 < P.nsteps) ? 2 : 1;
        u.emplace_back(s, len);
        s += len;
    }
    return u;
}

}  // namespace

bool tc_lu_factor(const Plan& P, Work<float>& w, int nbox, int* status, cudaStream_t st)
{
    const int n = P.n, NB = P.NB, KG = P.KG;
    const long long ldm = P.ldm, gplane = ldm * KG;
    auto up = [&](const TcLeft& L, TcArgs a) {
        a.invt = w.it1;
        a.sInvt = w.sIT;
        return launch_tc_update(P.fmt, L, w.Gp, gplane, w.sGp, KG, NB, a, nbox, st, P.tma_epi, P.tc_pairs);
    };
    // Panel of step s, its operators F_s and B_s (FP32 and split copies).
    auto panel_ops = [&](int s, bool pack_b) -> bool {
        const int k = P.k0[s], nb = P.nbs[s];
        float* Fs = w.F + P.fw_off[s];
        float* Bs = w.B + P.bw_off[s];
        int* Ps = w.perm + P.perm_off[s];
        launch_panel<float>(w.M, ldm, w.sM, n, k, nb, P.ib, Ps, w.sP, Fs, NB, w.sF, Bs + (long long)k * NB, NB,
                            w.sB, status, nullptr, nbox, st);
        // F rows below the panel, L21 L11^{-1} = -(L21 * F_top), and B rows above
        // it, U01 U11^{-1} = -(U01 * B_top), as tensor-core products: the left
        // operand is split into the step's own (not yet filled) pack region,
        // the right one, transposed, into the G pack.
        if (n - k - nb > 0) {
            void* Fp = fpk(P, w, s);
            launch_pack_split(P.fmt, w.M + (long long)(k + nb) * ldm + k, ldm, w.sM, n - k - nb, NB, nb, Fp, w.sFp,
                              nbox, st, rcf_w(P, w, s), w.sRC);
            gather_pack_raw(P.fmt, Fs, NB, w.sF, 0, nb, KG, 0, nb, nullptr, 0, nullptr, 0, 0, w.Gp, gplane, w.sGp, nullptr,
                            nbox, st, rcf(P, w, s), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(Fs + (long long)nb * NB, NB, w.sF, n - k - nb, nb, GM_SET, 0);
            if (!up(left1(Fp, n - k - nb, w.sFp, nb), a)) return false;
        }
        if (k > 0) {
            void* Bp = bpk(P, w, s);
            launch_pack_split(P.fmt, w.M + k, ldm, w.sM, k, NB, nb, Bp, w.sBp, nbox, st, rcb_w(P, w, s), w.sRC);
            gather_pack_raw(P.fmt, Bs + (long long)k * NB, NB, w.sB, 0, nb, KG, 0, nb, nullptr, 0, nullptr, 0, 0, w.Gp,
                            gplane, w.sGp, nullptr, nbox, st, rcb(P, w, s), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(Bs, NB, w.sB, k, nb, GM_SET, 0);
            if (!up(left1(Bp, k, w.sBp, nb), a)) return false;
        }
        launch_pack_split(P.fmt, Fs, NB, w.sF, n - k, NB, nb, fpk(P, w, s), w.sFp, nbox, st, rcf_w(P, w, s), w.sRC);
        if (pack_b)
            launch_pack_split(P.fmt, Bs, NB, w.sB, k + nb, NB, nb, bpk(P, w, s), w.sBp, nbox, st, rcb_w(P, w, s), w.sRC);
        return true;
    };
    // Step s's update of M's columns [c0, c0 + nc).
    auto update1 = [&](int s, int c0, int nc) -> bool {
        if (nc <= 0) return true;
        const int k = P.k0[s], nb = P.nbs[s];
        int* Ps = w.perm + P.perm_off[s];
        launch_gather_pack(P, w, k, nb, c0, nc, Ps, true, nullptr, nbox, st, rcf(P, w, s));
        TcArgs a = targs(w.M + (long long)k * ldm + c0, ldm, w.sM, n - k, nc, GM_FWD, nb);
        a.perm = Ps; a.sP = w.sP; a.W = w.W; a.ldw = ldm; a.sW = w.sG; a.status = status;
        return up(left1(fpk(P, w, s), n - k, w.sFp, nb), a);
    };
    // The pair's operators and permutation from those of its two steps.
    auto combine = [&](int s) -> bool {
        const int k = P.k0[s], nb0 = P.nbs[s], k1 = P.k0[s + 1], nb1 = P.nbs[s + 1];
        float* F0 = w.F + P.fw_off[s];
        float* B1 = w.B + P.bw_off[s + 1];
        int* P0 = w.perm + P.perm_off[s];
        const int* P1 = w.perm + P.perm_off[s + 1];
        {   // F_s' = forward step s+1 on F_s's rows [nb0, n - k)
            gather_pack_raw(P.fmt, F0, NB, w.sF, nb0, nb1, KG, 0, nb0, P1, w.sP, w.W, NB, w.sG, w.Gp, gplane, w.sGp, nullptr,
                            nbox, st, rcf(P, w, s + 1), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(F0 + (long long)nb0 * NB, NB, w.sF, n - k1, nb0, GM_FWD, nb1);
            a.perm = P1; a.sP = w.sP; a.W = w.W; a.ldw = NB; a.sW = w.sG; a.status = status;
            if (!up(left1(fpk(P, w, s + 1), n - k1, w.sFp, nb1), a)) return false;
            launch_pack_split(P.fmt, F0, NB, w.sF, n - k, NB, nb0, fpk(P, w, s), w.sFp, nbox, st, rcf_w(P, w, s),
                              w.sRC);
        }
        {   // B_{s+1}' = backward step s on B_{s+1}'s rows [0, k + nb0)
            gather_pack_raw(P.fmt, B1, NB, w.sB, k, nb0, KG, 0, nb1, nullptr, 0, nullptr, 0, 0, w.Gp, gplane, w.sGp,
                            nullptr, nbox, st, rcb(P, w, s), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(B1, NB, w.sB, k + nb0, nb1, GM_BWD, k);
            a.status = status;
            if (!up(left1(bpk(P, w, s), k + nb0, w.sBp, nb0), a)) return false;
            launch_pack_split(P.fmt, B1, NB, w.sB, k1 + nb1, NB, nb1, bpk(P, w, s + 1), w.sBp, nbox, st,
                              rcb_w(P, w, s + 1), w.sRC);
        }
        launch_perm_compose(P0, P1, w.sP, n - k, nb0, nbox, st);
        return true;
    };
    for (const auto& u : solve_units(P)) {
        const int s = u.first, k = P.k0[s];
        if (u.second == 1) {
            if (!panel_ops(s, true)) return false;
            if (!update1(s, k + P.nbs[s], n + P.r - k - P.nbs[s])) return false;
            continue;
        }
        const int nb0 = P.nbs[s], wp = nb0 + P.nbs[s + 1];
        if (!panel_ops(s, true)) return false;
        if (!update1(s, k + nb0, P.nbs[s + 1])) return false;   // look-ahead: the next panel's columns
        if (!panel_ops(s + 1, false)) return false;             // B_{s+1} is split once combined
        if (!combine(s)) return false;
        const int c0 = k + wp, nc = n + P.r - c0;
        if (nc > 0) {
            int* Pc = w.perm + P.perm_off[s];
            launch_gather_pack(P, w, k, wp, c0, nc, Pc, true, nullptr, nbox, st, rcf(P, w, s));
            TcArgs a = targs(w.M + (long long)k * ldm + c0, ldm, w.sM, n - k, nc, GM_FWD, wp);
            a.perm = Pc; a.sP = w.sP; a.W = w.W; a.ldw = ldm; a.sW = w.sG; a.status = status;
            if (!up(left_fwd_pair(P, w, s), a)) return false;
        }
    }
    // Inverse permutations of the solve units, for gathers fused into the
    // forward solves.
    if (P.fuse_fwd)
        for (const auto& u : solve_units(P)) {
            const int s = u.first, wp = u.second == 2 ? P.nbs[s] + P.nbs[s + 1] : P.nbs[s];
            prof_begin(KC_MISC, st);
            k_perm_inverse<<<nbox, 256, 0, st>>>(w.perm + P.perm_off[s], w.inv + P.perm_off[s], w.sP, n - P.k0[s],
                                                 wp);
            prof_end(KC_MISC, st, 0.0, (double)nbox * (n - P.k0[s]) * 8.0);
        }
    return true;
}

// The solves alternate between two (G, W) buffers.  In the backward sweep
// the next unit's G is the block of rows just above the current one, so the
// current product's epilogue writes it (contiguous K indices, coalesced
// stores) straight from its results; only the first product of a sweep, a
// ragged next unit, or an output that is not 16-byte aligned (cp.async
// epilogue) gathers on its own.  Measured on the p = 16 workload this pays
// with the 3 x TF32 operands and not with the 3 x BF16 ones (three 2-byte
// stores per element), hence P.fuse_bwd.
bool tc_lu_forward(const Plan& P, Work<float>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st)
{
    const int n = P.n;
    const long long ldm = P.ldm, gplane = ldm * P.KG;
    void* Gb[2] = {w.Gp, w.Gp2};
    float* Wb[2] = {w.W, w.W2};
    float* Ib[2] = {w.it1, w.it2};
    const auto units = solve_units(P);
    auto width = [&](size_t u) { const int s = units[u].first; return units[u].second == 2 ? P.nbs[s] + P.nbs[s + 1] : P.nbs[s]; };
    bool have = false;   // the current unit's G and W are in buffer cur
    for (size_t u = 0; u < units.size(); ++u) {
        const int s = units[u].first, k = P.k0[s], wp = width(u), cur = (int)(u & 1);
        int* Ps = w.perm + P.perm_off[s];
        if (!have)
            gather_pack_raw(P.fmt, w.M, ldm, w.sM, k, wp, P.KG, c0, nc, Ps, w.sP, Wb[cur], ldm, w.sG, Gb[cur], gplane,
                            w.sGp, skip, nbox, st, rcf(P, w, s), w.sRC, Ib[cur], w.sIT);
        TcArgs a = targs(w.M + (long long)k * ldm + c0, ldm, w.sM, n - k, nc, GM_FWD, wp);
        a.perm = Ps; a.sP = w.sP; a.W = Wb[cur]; a.ldw = ldm; a.sW = w.sG; a.skip = skip;
        a.invt = Ib[cur]; a.sInvt = w.sIT;
        // The next unit's G is gathered through its pivot permutation, whose
        // source rows scatter over the rows this product writes: stores from
        // the epilogue would not coalesce, so the forward sweep gathers on
        // its own (the machinery is in place: P.fuse_fwd).
        if (P.fuse_fwd && u + 1 < units.size() && width(u + 1) % (P.fmt ? 32 : 16) == 0) {
            const int s1 = units[u + 1].first;
            a.nG = Gb[cur ^ 1]; a.ng_plane = gplane; a.nsG = w.sGp; a.ngK = P.KG;
            a.ninv = w.inv + P.perm_off[s1]; a.nsInv = w.sP; a.ng_off = wp; a.ng_len = n - P.k0[s1];
            a.nW = Wb[cur ^ 1]; a.nsW = w.sG; a.nldw = ldm; a.nw_off = wp; a.nw_len = width(u + 1);
        }
        const TcLeft L = units[u].second == 2 ? left_fwd_pair(P, w, s) : left1(fpk(P, w, s), n - k, w.sFp, wp);
        if (!launch_tc_update(P.fmt, L, Gb[cur], gplane, w.sGp, P.KG, P.NB, a, nbox, st, P.tma_epi, P.tc_pairs, &have))
            return false;
    }
    return true;
}

bool tc_lu_backward(const Plan& P, Work<float>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st)
{
    const long long ldm = P.ldm, gplane = ldm * P.KG;
    void* Gb[2] = {w.Gp, w.Gp2};
    float* Ib[2] = {w.it1, w.it2};
    const auto units = solve_units(P);
    auto width = [&](size_t u) { const int s = units[u].first; return units[u].second == 2 ? P.nbs[s] + P.nbs[s + 1] : P.nbs[s]; };
    bool have = false;
    int cur = 0;
    for (size_t q = units.size(); q-- > 0; cur ^= 1) {
        const int s = units[q].first, k = P.k0[s], wp = width(q);
        if (!have)
            gather_pack_raw(P.fmt, w.M, ldm, w.sM, k, wp, P.KG, c0, nc, nullptr, 0, nullptr, 0, 0, Gb[cur], gplane,
                            w.sGp, skip, nbox, st, rcb(P, w, s), w.sRC, Ib[cur], w.sIT);
        TcArgs a = targs(w.M + c0, ldm, w.sM, k + wp, nc, GM_BWD, k);
        a.skip = skip;
        a.invt = Ib[cur]; a.sInvt = w.sIT;
        if (P.fuse_bwd && q > 0 && width(q - 1) % (P.fmt ? 32 : 16) == 0) {
            const int wq = width(q - 1);
            a.nG = Gb[cur ^ 1]; a.ng_plane = gplane; a.nsG = w.sGp; a.ngK = P.KG;
            a.ninv = nullptr; a.ng_off = k - wq; a.ng_len = wq;
        }
        const TcLeft L = units[q].second == 2 ? left_bwd_pair(P, w, s) : left1(bpk(P, w, s), k + wp, w.sBp, wp);
        if (!launch_tc_update(P.fmt, L, Gb[cur], gplane, w.sGp, P.KG, P.NB, a, nbox, st, P.tma_epi, P.tc_pairs, &have))
            return false;
    }
    return true;
}

}  // namespace hps
