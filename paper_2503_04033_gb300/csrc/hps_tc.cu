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
#include <functional>
#include <utility>
#include <vector>

#include "hps_internal.h"

namespace hps {

namespace {

constexpr int TC_BM = 128;                                  // tile rows = TMEM lanes
constexpr uint32_t ROWB = 64;                               // bytes of an operand row in one K chunk (64B swizzle)
constexpr uint32_t A_TILE = TC_BM * ROWB;                   // 8 KiB per plane
#ifndef HPS_TC_STAGES
#define HPS_TC_STAGES 3
#endif
#ifndef HPS_TE_WARPS
#define HPS_TE_WARPS 8
#endif
#ifndef HPS_TE_PRE
#define HPS_TE_PRE 2
#endif
#ifndef HPS_TE_LA
#define HPS_TE_LA 1
#endif
#ifndef HPS_TC_PRE
#define HPS_TC_PRE 3
#endif
constexpr int TC_STAGES = HPS_TC_STAGES;   // operand stages of the TMA -> MMA ring
constexpr int TC_EPI_WARPS = 4;                             // cp.async epilogue: one per TMEM lane quarter
constexpr int TE_WARPS = HPS_TE_WARPS;                      // TMA epilogue: 4 or 8 (two per lane quarter)
static_assert(TE_WARPS == 4 || TE_WARPS == 8, "the TMA epilogue takes one or two warps per TMEM lane quarter");
constexpr int TC_THREADS = 64 + 32 * TE_WARPS;              // warp 0 TMA, warp 1 MMA, warps 2.. epilogue

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
// FMT 3: plain BF16 operands, one plane, one kind::f16 product per K step
// (the learned correction's network: BF16 weights and activations, FP32
// accumulation).
template <>
struct TcFmt<3> {
    static constexpr int NPL = 1, EB = 2, KPC = 32, BN = 256;
};
template <int FMT>
__host__ __device__ constexpr uint32_t b_tile() { return (uint32_t)TcFmt<FMT>::BN * ROWB; }
template <int FMT>
__host__ __device__ constexpr uint32_t stage_bytes() { return (uint32_t)TcFmt<FMT>::NPL * (A_TILE + b_tile<FMT>()); }
constexpr uint32_t STAGE_BYTES = 48 * 1024;
constexpr int TC_BN_NARROW = 64;                            // tile width for products of at most 64 columns
static_assert(stage_bytes<0>() == STAGE_BYTES && stage_bytes<1>() == STAGE_BYTES && stage_bytes<2>() == STAGE_BYTES &&
                  stage_bytes<3>() <= STAGE_BYTES,
              "one shared-memory layout");
constexpr uint32_t TBUF_FLOATS = 32 * 32;                   // per-epilogue-warp transpose buffer (XOR-swizzled)
constexpr int TC_PRE = HPS_TC_PRE;                          // source chunks in flight per epilogue warp
constexpr uint32_t EPI_FLOATS = TBUF_FLOATS * (1 + TC_PRE) + 64;   // transpose + source ring + row pointers
constexpr int TE_PRE = HPS_TE_PRE;                         // TMA epilogue: 32 x 32 chunk buffers per warp
constexpr int TE_LA = HPS_TE_LA;                           // chunks fetched ahead (TE_PRE - TE_LA - 1 stores may still read)
static_assert(TE_LA >= 1 && TE_LA < TE_PRE, "the epilogue ring needs a buffer beyond the fetched-ahead chunks");
constexpr uint32_t TE_CHUNK = 32 * 32 * 4;                 // 4 KiB, 128-byte rows, 128B swizzle
constexpr size_t EPI_BYTES_CP = (size_t)TC_EPI_WARPS * EPI_FLOATS * 4;
constexpr size_t EPI_BYTES_TMA = (size_t)TE_WARPS * TE_PRE * TE_CHUNK;
constexpr size_t TC_SMEM = (size_t)TC_STAGES * STAGE_BYTES + (EPI_BYTES_CP > EPI_BYTES_TMA ? EPI_BYTES_CP : EPI_BYTES_TMA) +
                           1024;
static_assert(TC_SMEM <= 227 * 1024, "operand stages and epilogue buffers exceed a CTA's shared memory");
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s per wait (TcArgs.wait_ns)

// Tensor maps of one update product: up to eight parts of the left operand
// (the steps of an LU unit), the right operand G and the output O.
constexpr int kMaxParts = 8;
struct TcMaps {
    CUtensorMap A[kMaxParts];
    CUtensorMap B;
    CUtensorMap O;
};

struct TcArgs {
    float* O; long long ldo, sO;
    int M, N, kch;
    int nparts;                      // parts of the left operand (one tensor map each)
    int kch_end[kMaxParts];          // K chunk where part i ends (parts follow each other along K)
    int a_off[kMaxParts];            // row of the product where part i's row 0 sits (rows above load as zeros)
    int tiles_m, tiles_n, tiles;
    int nbox;
    int units, units_per_box;        // work units (output tiles) in all, and per box
    int vec;                         // rows of O and W are 16-byte aligned: float4 epilogue
    int tma_epi;                     // O is 16-byte aligned: source tiles in and results out by TMA
    int mode, split;
    unsigned long long wait_ns;      // limit of every mbarrier wait
    int test_stall;                  // test hook: the TMA role issues nothing, so the first wait runs out
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

// Bounded wait on an mbarrier phase (limit in ns); false when it gave up.  The
// epilogue warps back off (spinning warps steal issue slots); the
// single-thread TMA and MMA roles poll (try_wait already suspends in hardware
// for a while).
template <bool kBackoff = true>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (kBackoff && it >= 8) __nanosleep(it < 64 ? 32 : 128);
        if ((it & 255u) == 255u) {
            if (*reinterpret_cast<volatile int*>(&g_tc_abort)) return false;
            if (global_ns() - t0 > limit) {
                atomicExch(&g_tc_abort, 1);
                return false;
            }
        }
    }
}

// Bounded wait used only to let asynchronous work already in flight (TMA
// copies, MMAs) finish before a CTA that gave up exits; it does not return
// early on the abort flag.  Such work completes by itself, so in practice this
// returns at once.
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, uint64_t limit)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return;
        __nanosleep(128);
        if ((it & 63u) == 63u && global_ns() - t0 > limit) return;
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

// The CTA's sequence of work units (output tiles): blockIdx.x, blockIdx.x +
// gridDim.x, ... (box-major, so a box's A and G stay in L2 while its tiles
// run).
struct TcSched {
    int u0, ustep, units, upb, tiles_n, bn;
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
        m0 = mi * TC_BM;
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
    } else if constexpr (FMT == 3) {
        static_cast<__nv_bfloat16*>(dst)[idx] = __float2bfloat16_rn(x);
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
__device__ __forceinline__ void shift_scales(float (&its8)[8])
{
#pragma unroll
    for (int c8 = 0; c8 < 7; ++c8) its8[c8] = its8[c8 + 1];
}
__device__ __forceinline__ void scale_chunk(uint32_t (&v)[32], float (&its8)[8])
{
    const float sl = its8[0];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __float_as_uint(__uint_as_float(v[c]) * __shfl_sync(0xffffffffu, sl, c));
    shift_scales(its8);
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
k_tc_update(const __grid_constant__ TcMaps tm, TcArgs a)
{
    const CUtensorMap& tmB = tm.B;
    const CUtensorMap& tmO = tm.O;
    using Fm = TcFmt<FMT>;
    constexpr int BN = BNT, KPC = Fm::KPC, NPL = Fm::NPL;
    constexpr uint32_t B_TILE = (uint32_t)BN * ROWB;
    constexpr uint32_t STAGE_TX = (uint32_t)NPL * (A_TILE + B_TILE);   // bytes a stage receives
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t ld_bar[TE_WARPS][TE_PRE];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[TC_STAGES];
    __shared__ __align__(8) uint64_t tfull_bar[2];
    __shared__ __align__(8) uint64_t tempty_bar[2];
    __shared__ __align__(8) uint64_t mdrain_bar;   // the MMA role's last commit when it gives up
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    unsigned char* sbase_ptr = smem_raw + (sbase - smem_u32(smem_raw));
    TcSched sc;
    sc.bn = BN;
    sc.tiles_n = a.tiles_n;
    sc.units = a.units;
    sc.upb = a.units_per_box;
    sc.u0 = blockIdx.x;
    sc.ustep = gridDim.x;
    float* tbuf_all = reinterpret_cast<float*>(sbase_ptr + TC_STAGES * STAGE_BYTES);

    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull_bar[b]), 1);
            mbar_init(smem_u32(&tempty_bar[b]), a.tma_epi ? TE_WARPS : TC_EPI_WARPS);
        }
        for (int w = 0; w < TE_WARPS; ++w)
            for (int q = 0; q < TE_PRE; ++q) mbar_init(smem_u32(&ld_bar[w][q]), 1);
        mbar_init(smem_u32(&mdrain_bar), 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(&tmem_base_sh), 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        if (lane == 0) {
            for (int pi = 0; pi < a.nparts; ++pi)
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tm.A[pi])) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
            uint32_t g = 0;
            bool ok = !a.test_stall;
            for (int u = sc.u0; u < sc.units && ok; u += sc.ustep) {
                if (sc.skipped(u, a.skip)) continue;
                int box, m0, n0;
                sc.decode(u, box, m0, n0);
                for (int ch = 0; ch < a.kch; ++ch, ++g) {
                    const int s = g % TC_STAGES;
                    const uint32_t use = g / TC_STAGES;
                    if (g >= TC_STAGES && !mbar_wait<false>(smem_u32(&empty_bar[s]), (use - 1) & 1, a.wait_ns)) {
                        fail_sh = 1;
                        ok = false;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    const uint32_t st = sbase + s * STAGE_BYTES;
                    mbar_expect_tx(fb, STAGE_TX);
                    // A's K chunks come from the part whose range holds ch; part
                    // i's row 0 is row a_off[i] of the product (rows above it
                    // load as zeros)
                    int pi = 0;
                    while (pi + 1 < a.nparts && ch >= a.kch_end[pi]) ++pi;
                    const CUtensorMap* ma = &tm.A[pi];
                    const int ka = (ch - (pi ? a.kch_end[pi - 1] : 0)) * KPC, ra = m0 - a.a_off[pi];
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) tma_load_4d(st + pl * A_TILE, ma, fb, ka, ra, pl, box);
                    const uint32_t sb0 = st + NPL * A_TILE;
#pragma unroll
                    for (int pl = 0; pl < NPL; ++pl) tma_load_4d(sb0 + pl * B_TILE, &tmB, fb, ch * KPC, n0, pl, box);
                }
            }
            // Drain: the last loads issued into each stage have landed before
            // this CTA exits (the MMA role waits for its own MMAs).
            for (uint32_t h = (g > TC_STAGES ? g - TC_STAGES : 0); h < g; ++h)
                mbar_drain(smem_u32(&full_bar[h % TC_STAGES]), (h / TC_STAGES) & 1, a.wait_ns / 4);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc =
                FMT == 0 ? tf32_idesc(TC_BM, BN) : ((FMT == 1 || FMT == 3) ? bf16_idesc(TC_BM, BN) : f16_idesc(TC_BM, BN));
            uint32_t g = 0, j = 0;
            bool ok = true;
            for (int u = sc.u0; u < sc.units && ok; u += sc.ustep) {
                if (sc.skipped(u, a.skip)) continue;
                const int b = j & 1;
                const uint32_t uj = j >> 1;
                if (j >= 2 && !mbar_wait<false>(smem_u32(&tempty_bar[b]), (uj - 1) & 1, a.wait_ns)) {
                    fail_sh = 1;
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * BN);
                for (int ch = 0; ch < a.kch; ++ch, ++g) {
                    const int s = g % TC_STAGES;
                    if (!mbar_wait<false>(smem_u32(&full_bar[s]), (g / TC_STAGES) & 1, a.wait_ns)) {
                        fail_sh = 1;
                        ok = false;
                        break;
                    }
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
                        } else if constexpr (FMT == 3) {
                            mma_bf16(d, ad[0] + o, bd[0] + o, idesc, acc0);
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
                    mma_commit(smem_u32(&empty_bar[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&tfull_bar[b]));
                ++j;
            }
            if (!ok) {
                // every MMA issued so far completes before TMEM is released
                mma_commit(smem_u32(&mdrain_bar));
                mbar_drain(smem_u32(&mdrain_bar), 0, a.wait_ns / 4);
            }
        }
    } else if (a.tma_epi) {
        // Epilogue warps 2.., TMA form: warp w owns TMEM lane quarter qd = w % 4
        // (tile rows 32 qd .. +31) and a ring of TE_PRE 32 x 32 buffers; with
        // eight warps two share a quarter and take alternate 32-column chunks
        // of each tile (warp w the chunks h, h + 2, .. with h = (w - 2) / 4),
        // so that two chains of TMEM loads, staging and stores overlap.  Lane 0
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
        constexpr int CST = TE_WARPS / 4;   // chunk stride of a warp within a tile
        const int h = ew / 4;               // its first chunk
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
        int lt = first_from(sc.u0), lcc = h;
        uint32_t lg = 0;
        auto settle = [&]() {   // past the tiles that hold no chunk of this warp
            while (lt < sc.units) {
                int box, m0, n0, nch;
                geom(lt, box, m0, n0, nch);
                if (lcc < nch) return;
                lt = first_from(lt + sc.ustep);
                lcc = h;
            }
        };
        settle();
        auto issue = [&]() {
            int box, m0, n0, nch;
            geom(lt, box, m0, n0, nch);
            const uint32_t buf = lg % TE_PRE;
            mbar_expect_tx(lbar0 + 8 * buf, TE_CHUNK);
            tma_load_3d(ring + buf * TE_CHUNK, &tmO, lbar0 + 8 * buf, n0 + 32 * lcc, m0 + 32 * qd, box);
            ++lg;
            lcc += CST;
            settle();
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
            if constexpr (FMT == 2) {
                load_tile_scales(its8, a.invt + box * a.sInvt + n0, nch, lane);
                if (h) shift_scales(its8);
            }
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[b]), (j >> 1) & 1, a.wait_ns);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            if (h >= nch) {   // no chunk of this tile for this warp: hand the buffer back at once
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
                continue;
            }
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
            for (int cc = h; cc < nch; cc += CST, ++g) {
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
                if (cc + CST >= nch) {
                    // the accumulator is in registers: hand the TMEM buffer back
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&tempty_bar[b]));
                }
                if (need_src && !mbar_wait(lbar0 + 8 * buf, (g / TE_PRE) & 1, a.wait_ns)) ok = false;
                if (!__all_sync(0xffffffffu, ok ? 1 : 0)) {
                    ok = false;
                    break;
                }
                float4* rowp = reinterpret_cast<float4*>(ring_p + buf * TE_CHUNK + lane * 128);
                const int cb = n0 + cc * 32;
                if constexpr (FMT == 2) {
                    scale_chunk(v, its8);
                    if (CST == 2) shift_scales(its8);
                }
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
                for (uint32_t h = g; h < lg; ++h) mbar_drain(lbar0 + 8 * (h % TE_PRE), (h / TE_PRE) & 1, a.wait_ns / 4);
            }
            bulk_wait_all();
        }
        __syncwarp();
    } else if (warp < 2 + TC_EPI_WARPS) {
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
            if (lane == 0) ok = mbar_wait(smem_u32(&tfull_bar[b]), (j >> 1) & 1, a.wait_ns);
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

// The same pack reading src once: a cluster of kPackCl CTAs per 32-column
// strip, each CTA holding a contiguous share of the rows in shared memory.
// Each CTA forms its share's column maxima, the cluster exchanges them
// through distributed shared memory, and every CTA scales and splits its
// rows from shared memory.  The maxima are over the same entries as
// k_pack_f16's, so the planes and rc are the same bit for bit.
constexpr int kPackCl = 8;

__global__ void __cluster_dims__(kPackCl, 1, 1) __launch_bounds__(256)
k_pack_f16_cl(const float* __restrict__ src, long long lds, long long sS, int rows, int NB, int nb,
              __half* __restrict__ dst, long long sD, float* __restrict__ rc, long long sC, int chunk)
{
    extern __shared__ float4 tile[];   // [chunk][8] float4: this CTA's rows of the strip
    __shared__ float red[32][33];
    __shared__ float part[32];         // this CTA's column maxima (read by the cluster)
    __shared__ float scl[32];
    unsigned rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const int box = blockIdx.y, strip = blockIdx.x / kPackCl;
    const int tid = threadIdx.x, tq = tid & 7, tr = tid >> 3;   // 4 columns 4 tq.., rows tr, tr + 32, ..
    const int c0 = strip * 32, cq = c0 + 4 * tq;
    const int r0 = (int)rank * chunk, r1 = min(rows, r0 + chunk);
    const float* sb = src + box * sS;
    const bool vec = cq + 4 <= nb && ((reinterpret_cast<uintptr_t>(sb + cq) & 15) == 0) && (lds & 3) == 0;
    float mx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    constexpr int U = 4;   // rows per thread in flight
    for (int rb = r0 + tr; rb < r1; rb += 32 * U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = rb + 32 * u;
            v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < r1) {
                const float* rp = sb + (long long)r * lds + cq;
                if (vec) v[u] = __ldg(reinterpret_cast<const float4*>(rp));
                else {
                    if (cq + 0 < nb) v[u].x = rp[0];
                    if (cq + 1 < nb) v[u].y = rp[1];
                    if (cq + 2 < nb) v[u].z = rp[2];
                    if (cq + 3 < nb) v[u].w = rp[3];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = rb + 32 * u;
            if (r < r1) {
                tile[(r - r0) * 8 + tq] = v[u];
                mx[0] = fmaxf(mx[0], fabsf(v[u].x));
                mx[1] = fmaxf(mx[1], fabsf(v[u].y));
                mx[2] = fmaxf(mx[2], fabsf(v[u].z));
                mx[3] = fmaxf(mx[3], fabsf(v[u].w));
            }
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) red[tr][4 * tq + u] = mx[u];
    __syncthreads();
    if (tid < 32) {
        float m = red[0][tid];
        for (int i = 1; i < 32; ++i) m = fmaxf(m, red[i][tid]);
        part[tid] = m;
    }
    // every CTA's maxima written and visible to the cluster
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if (tid < 32) {
        const unsigned local = (unsigned)__cvta_generic_to_shared(&part[tid]);
        float m = 0.0f;
        for (unsigned q = 0; q < (unsigned)kPackCl; ++q) {
            unsigned remote;
            float v;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(q));
            asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(remote) : "memory");
            m = fmaxf(m, v);
        }
        const int e = scale_exp(m);
        scl[tid] = pow2f(e);
        if (rank == 0 && c0 + tid < NB) rc[box * sC + c0 + tid] = pow2f(-e);
    }
    // the peers' maxima are read: a CTA may leave once every CTA has arrived
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    __syncthreads();
    if (cq < NB) {
        const float s0 = scl[4 * tq], s1 = scl[4 * tq + 1], s2 = scl[4 * tq + 2], s3 = scl[4 * tq + 3];
        const long long total = (long long)rows * NB;
        __half* db = dst + box * sD;
        const bool vst = cq + 4 <= NB && (NB & 3) == 0 && (sD & 3) == 0 &&
                         ((reinterpret_cast<uintptr_t>(dst) & 7) == 0);
        for (int r = r0 + tr; r < r1; r += 32) {
            const float4 v = tile[(r - r0) * 8 + tq];
            const float x[4] = {v.x * s0, v.y * s1, v.z * s2, v.w * s3};
            __half hi[4], lo[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                hi[u] = __float2half_rn(x[u]);
                lo[u] = __float2half_rn(x[u] - __half2float(hi[u]));
            }
            const long long idx = (long long)r * NB + cq;
            if (vst) {
                uint2 ph, pl;
                ph.x = (uint32_t)__half_as_ushort(hi[0]) | ((uint32_t)__half_as_ushort(hi[1]) << 16);
                ph.y = (uint32_t)__half_as_ushort(hi[2]) | ((uint32_t)__half_as_ushort(hi[3]) << 16);
                pl.x = (uint32_t)__half_as_ushort(lo[0]) | ((uint32_t)__half_as_ushort(lo[1]) << 16);
                pl.y = (uint32_t)__half_as_ushort(lo[2]) | ((uint32_t)__half_as_ushort(lo[3]) << 16);
                *reinterpret_cast<uint2*>(db + idx) = ph;
                *reinterpret_cast<uint2*>(db + total + idx) = pl;
            } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (cq + u < NB) {
                        db[idx + u] = hi[u];
                        db[total + idx + u] = lo[u];
                    }
            }
        }
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
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
    const bool vec4 = ncc == 32 && ((reinterpret_cast<uintptr_t>(Mb + c0 + cb) & 15) == 0) && (ldm & 3) == 0 &&
                      (!W || (((reinterpret_cast<uintptr_t>(W + box * sW + cb) & 15) == 0) && (ldw & 3) == 0));
    if (vec4) {
        // 16-byte loads: thread (tr, tq) takes columns 4 tq .. 4 tq + 3 of
        // rows tr, tr + 32, ...; GU rows per thread in flight (row indices
        // first, then every load, then the stores)
        constexpr int GU = 4;
        const int tid = ty * 32 + tx, tq = tid & 7, tr = tid >> 3;
        float mx4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int i0 = tr; i0 < gK; i0 += 32 * GU) {
            int srcr[GU];
            float4 v[GU], wv[GU];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int i = i0 + 32 * u;
                srcr[u] = i < nb ? k + (perm ? perm[box * sP + i] : i) : -1;
            }
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int i = i0 + 32 * u;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                wv[u] = v[u];
                if (srcr[u] >= 0) {
                    v[u] = *reinterpret_cast<const float4*>(Mb + (long long)srcr[u] * ldm + c0 + cb + 4 * tq);
                    if (W) wv[u] = *reinterpret_cast<const float4*>(Mb + (long long)(k + i) * ldm + c0 + cb + 4 * tq);
                }
            }
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int i = i0 + 32 * u;
                if (i >= gK) break;
                float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
                if (srcr[u] >= 0) {
                    if (W) *reinterpret_cast<float4*>(W + box * sW + (long long)i * ldw + cb + 4 * tq) = wv[u];
                    const float r = rcb[i];
#pragma unroll
                    for (int j2 = 0; j2 < 4; ++j2) {
                        e[j2] *= r;
                        mx4[j2] = fmaxf(mx4[j2], fabsf(e[j2]));
                    }
                }
#pragma unroll
                for (int j2 = 0; j2 < 4; ++j2) gt[i * 33 + 4 * tq + j2] = e[j2];
            }
        }
        // column maxima: the 32 row groups of each column through shared memory
        __shared__ float cm[32][33];
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) cm[tr][4 * tq + j2] = mx4[j2];
        __syncthreads();
        if (ty == 0) {
            float m = 0.0f;
            for (int r = 0; r < 32; ++r) m = fmaxf(m, cm[r][tx]);
            red[0][tx] = m;
        }
        if (ty < 8 && ty > 0) red[ty][tx] = 0.0f;
    } else if (ncc == 32) {
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

// Test hook (HPS_OPT_TEST_TC_TIMEOUT): the next product launch that carries
// box status words stalls on purpose (host-side flag, read on the host only).
int g_test_stall_next = 0;

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
              int nbox, int box_rows, long long pitch = 0)
{
    using Fm = TcFmt<FMT>;
    auto fn = encode_fn();
    if (!fn) return false;
    if (pitch <= 0) pitch = K;
    cuuint64_t dims[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)Fm::NPL, (cuuint64_t)nbox};
    cuuint64_t strides[3] = {(cuuint64_t)pitch * Fm::EB, (cuuint64_t)plane_elems * Fm::EB,
                             (cuuint64_t)box_elems * Fm::EB};
    cuuint32_t boxd[4] = {(cuuint32_t)Fm::KPC, (cuuint32_t)box_rows, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = FMT == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                            : ((FMT == 1 || FMT == 3) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    CUresult r = fn(tm, dt, 4,
                    const_cast<void*>(base), dims, strides, boxd, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Left operand of an update product: the split K-major packs of up to eight
// LU steps (a unit), part i with rows[i] rows per box of NB values, K[i] of
// them used (only the last part may be ragged), its row 0 at row off[i] of
// the product.  Pointers and strides are in elements of the plan's operand
// format; ld[i] is part i's row pitch (0: NB).
struct TcLeft {
    int nparts;
    const void* A[kMaxParts];
    long long rows[kMaxParts], sA[kMaxParts];
    int K[kMaxParts], off[kMaxParts];
    long long ld[kMaxParts];
};

TcLeft left1(const void* A, long long rows, long long sA, int K)
{
    TcLeft l{};
    l.nparts = 1;
    l.A[0] = A; l.rows[0] = rows; l.sA[0] = sA; l.K[0] = K;
    return l;
}

template <int FMT, int BNT>
bool launch_tc_update_w(const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                        const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, bool* fused, long long ldg = 0)
{
    using Fm = TcFmt<FMT>;
    int K = 0;
    for (int i = 0; i < L.nparts; ++i) K += L.K[i];
    if (args.M <= 0 || args.N <= 0) return true;
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(k_tc_update<FMT, BNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
        if (num_sms <= 0) num_sms = 1;
    }
    TcArgs a = args;
    a.wait_ns = WAIT_NS;
    a.test_stall = 0;
    if (g_test_stall_next && a.status) {
        // test hook: this launch's TMA role issues nothing, so its first
        // wait runs out after 2 ms and the launch ends with HPS_ETIMEOUT
        g_test_stall_next = 0;
        a.test_stall = 1;
        a.wait_ns = 2000000ull;
    }
    a.kch = (K + Fm::KPC - 1) / Fm::KPC;
    a.nparts = L.nparts;
    {
        int ce = 0;
        for (int i = 0; i < L.nparts; ++i) {   // every part but the last is a whole number of chunks
            ce += (L.K[i] + Fm::KPC - 1) / Fm::KPC;
            a.kch_end[i] = ce;
            a.a_off[i] = L.off[i];
        }
    }
    a.tiles_m = (a.M + TC_BM - 1) / TC_BM;
    a.tiles_n = (a.N + BNT - 1) / BNT;
    a.tiles = a.tiles_m * a.tiles_n * nbox;
    a.nbox = nbox;
    a.units_per_box = a.tiles_m * a.tiles_n;
    a.units = a.units_per_box * nbox;
    TcMaps maps{};
    for (int i = 0; i < L.nparts; ++i)
        if (!make_map<FMT>(&maps.A[i], L.A[i], NB, L.rows[i], L.rows[i] * NB, L.sA[i], nbox, TC_BM, L.ld[i]))
            return false;
    for (int i = L.nparts; i < kMaxParts; ++i) maps.A[i] = maps.A[0];
    if (!make_map<FMT>(&maps.B, Gp, gK, args.N, g_plane, sGp, nbox, BNT, ldg)) return false;
    const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    a.vec = al16(a.O) && (a.ldo % 4 == 0) && (a.sO % 4 == 0) && (a.N % 4 == 0) &&
            (!a.W || (al16(a.W) && a.ldw % 4 == 0 && a.sW % 4 == 0));
    a.tma_epi = 0;
    if (al16(a.O) && a.ldo % 4 == 0 && a.sO % 4 == 0 && allow_tma) {
        auto fn = encode_fn();
        cuuint64_t dims[3] = {(cuuint64_t)a.N, (cuuint64_t)a.M, (cuuint64_t)nbox};
        cuuint64_t strides[2] = {(cuuint64_t)a.ldo * 4, (cuuint64_t)a.sO * 4};
        cuuint32_t boxd[3] = {32, 32, 1};
        cuuint32_t es[3] = {1, 1, 1};
        if (fn && fn(&maps.O, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.O, dims, strides, boxd, es,
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
    {
        dim3 grd((unsigned)std::min(a.units, num_sms));
        k_tc_update<FMT, BNT><<<grd, TC_THREADS, TC_SMEM, st>>>(maps, a);
    }
    const double kk = (double)K;
    prof_end(cls, st, 2.0 * nbox * a.M * (double)a.N * kk,
             (double)nbox * ((a.M + (double)a.N) * kk * Fm::NPL * Fm::EB + 2.0 * a.M * (double)a.N * 4));
    return true;
}

template <int FMT>
bool launch_tc_update_f(const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                        const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, int bn_max, bool* fused,
                        long long ldg = 0)
{
    if (args.N <= TC_BN_NARROW && TcFmt<FMT>::BN > TC_BN_NARROW)
        return launch_tc_update_w<FMT, TC_BN_NARROW>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma,
                                                     fused, ldg);
    if ((args.N <= 2 * TC_BN_NARROW || bn_max <= 2 * TC_BN_NARROW) && TcFmt<FMT>::BN > 2 * TC_BN_NARROW)
        return launch_tc_update_w<FMT, 2 * TC_BN_NARROW>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma,
                                                         fused, ldg);
    return launch_tc_update_w<FMT, TcFmt<FMT>::BN>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma,
                                                   fused, ldg);
}

bool launch_tc_update(int fmt, const TcLeft& L, const void* Gp, long long g_plane, long long sGp, int gK, int NB,
                      const TcArgs& args, int nbox, cudaStream_t st, bool allow_tma, int bn_max,
                      bool* fused = nullptr)
{
    if (fmt == 2) return launch_tc_update_f<2>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, bn_max, fused);
    return fmt ? launch_tc_update_f<1>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, bn_max, fused)
               : launch_tc_update_f<0>(L, Gp, g_plane, sGp, gK, NB, args, nbox, st, allow_tma, bn_max, fused);
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
        // one read of src when a cluster's shares fit in shared memory
        constexpr size_t kClSmemMax = 192 * 1024;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_pack_f16_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmemMax);
            attr = true;
        }
        const int chunk = (rows + kPackCl - 1) / kPackCl;
        const size_t smem = (size_t)chunk * 32 * sizeof(float);
        if (smem <= kClSmemMax && chunk > 0) {
            k_pack_f16_cl<<<dim3((unsigned)(((NB + 31) / 32) * kPackCl), (unsigned)nbox), 256, smem, st>>>(
                src, lds, sS, rows, NB, nb, static_cast<__half*>(dst), sD, rc, sC, chunk);
        } else {
            k_pack_f16<<<dim3((unsigned)((NB + 31) / 32), (unsigned)nbox), blk, 0, st>>>(
                src, lds, sS, rows, NB, nb, static_cast<__half*>(dst), sD, rc, sC);
        }
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
        static bool attr = false;   // a unit of 4 steps holds 512 x 33 floats of K
        if (!attr) {
            cudaFuncSetAttribute(k_gather_pack_f16, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            attr = true;
        }
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

// C = (accumulate ? C : 0) - A B^T per batch entry on tcgen05 with BF16
// operands (format 3) and FP32 accumulation: A [M][K] and B [N][K] BF16,
// K-major with row pitches lda, ldb (multiples of 8: 16-byte TMA rows) and
// batch strides sA, sB; C [M][N] FP32 with row pitch ldc, batch stride sC.
// K chunks past K read as zeros.  False when a tensor map cannot be encoded.
bool tc_gemm_bf16(int M, int N, int K, const void* A, long long lda, long long sA, const void* B, long long ldb,
                  long long sB, float* C, long long ldc, long long sC, bool accumulate, int batch, cudaStream_t st)
{
    if (K <= 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K) return false;
    if (M <= 0 || N <= 0 || batch <= 0) return true;
    TcLeft L = left1(A, M, sA, K);
    L.ld[0] = lda;
    TcArgs a = targs(C, ldc, sC, M, N, accumulate ? GM_ACC : GM_SET, 0);
    return launch_tc_update_f<3>(L, B, (long long)N * ldb, sB, K, K, a, batch, st, true, 256, nullptr, ldb);
}

void tc_test_stall_next(int on) { g_test_stall_next = on ? 1 : 0; }
bool tc_test_stall_armed() { return g_test_stall_next != 0; }

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
// LU steps are joined into units of up to eight (P.unit_max) wherever they
// apply to many columns.  Two adjacent units A (steps s..) and B (the next
// ones) become one: B applied forward to the columns of A's F parts, and A
// applied backward to the columns of B's B parts, give the joined unit's
// operators
//   forward  [F_A' | F_B] (each part's rows start at its own step),
//   backward [B_A | B_B'],
// with the composed row permutation pi_c(i) = pi_A(i) for i < w_A, else
// pi_A(w_A + pi_B(i - w_A)) (w_A = A's width).  A row below the unit's block
// still either stays in place or receives a block row, so the update epilogue
// is the same with split = the unit's width.  A unit of 2h steps is factored
// as: its first h steps (recursively), their update of the other h steps'
// columns, those h steps (recursively), the join; then it updates every
// later column once, with K = its width.  The solves run one product per
// unit.  Each pass over the trailing rows and right-hand sides then serves up
// to eight steps.

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
// Format 2: K scales of F_s and B_s (null otherwise); those of consecutive
// steps are contiguous, so a unit's scales start at its first step's.
const float* rcf(const Plan& P, const Work<float>& w, int s) { return w.rcF ? w.rcF + (long long)s * P.NB : nullptr; }
const float* rcb(const Plan& P, const Work<float>& w, int s) { return w.rcB ? w.rcB + (long long)s * P.NB : nullptr; }
float* rcf_w(const Plan& P, Work<float>& w, int s) { return w.rcF ? w.rcF + (long long)s * P.NB : nullptr; }
float* rcb_w(const Plan& P, Work<float>& w, int s) { return w.rcB ? w.rcB + (long long)s * P.NB : nullptr; }
void* fpk(const Plan& P, const Work<float>& w, int s) { return pk_at(w.Fp, (long long)npl(P) * P.fw_off[s], P.fmt); }
void* bpk(const Plan& P, const Work<float>& w, int s) { return pk_at(w.Bp, (long long)npl(P) * P.bw_off[s], P.fmt); }

// Columns (K) of the steps [s, s + len).
int unit_width(const Plan& P, int s, int len)
{
    int wd = 0;
    for (int i = 0; i < len; ++i) wd += P.nbs[s + i];
    return wd;
}

// Left operands of the unit (s, len): forward parts F_{s+i} (rows from step
// s+i's start), backward parts B_{s+i} (rows from 0).
TcLeft left_fwd(const Plan& P, const Work<float>& w, int s, int len)
{
    TcLeft l{};
    l.nparts = len;
    for (int i = 0; i < len; ++i) {
        l.A[i] = fpk(P, w, s + i);
        l.rows[i] = P.n - P.k0[s + i];
        l.sA[i] = w.sFp;
        l.K[i] = P.nbs[s + i];
        l.off[i] = P.k0[s + i] - P.k0[s];
    }
    return l;
}

TcLeft left_bwd(const Plan& P, const Work<float>& w, int s, int len)
{
    TcLeft l{};
    l.nparts = len;
    for (int i = 0; i < len; ++i) {
        l.A[i] = bpk(P, w, s + i);
        l.rows[i] = P.k0[s + i] + P.nbs[s + i];
        l.sA[i] = w.sBp;
        l.K[i] = P.nbs[s + i];
        l.off[i] = 0;
    }
    return l;
}

}  // namespace

// Units of the LU: (first step, steps), each a power of two up to P.unit_max.
std::vector<std::pair<int, int>> lu_units(const Plan& P)
{
    std::vector<std::pair<int, int>> u;
    for (int s = 0; s < P.nsteps;) {
        int len = 1;
        while (2 * len <= P.unit_max && s + 2 * len <= P.nsteps) len *= 2;
        u.emplace_back(s, len);
        s += len;
    }
    return u;
}

bool tc_lu_factor(const Plan& P, Work<float>& w, int nbox, int* status, cudaStream_t st)
{
    const int n = P.n, NB = P.NB, KG = P.KG;
    const long long ldm = P.ldm, gplane = ldm * KG;
    auto up = [&](const TcLeft& L, TcArgs a) {
        a.invt = w.it1;
        a.sInvt = w.sIT;
        return launch_tc_update(P.fmt, L, w.Gp, gplane, w.sGp, KG, NB, a, nbox, st, P.tma_epi, P.bn_max);
    };
    // Panel of step s, its operators F_s and B_s (FP32 and split copies; B_s's
    // split only when pack_b: a B part that a join rewrites before any
    // product reads it is split after that join).
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
    // The unit (s, len) applied to M's columns [c0, c0 + nc).
    auto update = [&](int s, int len, int c0, int nc) -> bool {
        if (nc <= 0) return true;
        const int k = P.k0[s], wp = unit_width(P, s, len);
        int* Ps = w.perm + P.perm_off[s];
        launch_gather_pack(P, w, k, wp, c0, nc, Ps, true, nullptr, nbox, st, rcf(P, w, s));
        TcArgs a = targs(w.M + (long long)k * ldm + c0, ldm, w.sM, n - k, nc, GM_FWD, wp);
        a.perm = Ps; a.sP = w.sP; a.W = w.W; a.ldw = ldm; a.sW = w.sG; a.status = status;
        return up(left_fwd(P, w, s, len), a);
    };
    // Join the units A = (s, h) and B = (s + h, h) into (s, 2 h).
    auto join = [&](int s, int h) -> bool {
        const int kA = P.k0[s], kB = P.k0[s + h], wA = unit_width(P, s, h), wB = unit_width(P, s + h, h);
        int* PA = w.perm + P.perm_off[s];
        const int* PB = w.perm + P.perm_off[s + h];
        for (int i = 0; i < h; ++i) {   // F_{s+i}' = B forward on F_{s+i}'s rows from B's start
            const int t = s + i, off = kB - P.k0[t];
            float* Ft = w.F + P.fw_off[t];
            gather_pack_raw(P.fmt, Ft, NB, w.sF, off, wB, KG, 0, P.nbs[t], PB, w.sP, w.W, NB, w.sG, w.Gp, gplane,
                            w.sGp, nullptr, nbox, st, rcf(P, w, s + h), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(Ft + (long long)off * NB, NB, w.sF, n - kB, P.nbs[t], GM_FWD, wB);
            a.perm = PB; a.sP = w.sP; a.W = w.W; a.ldw = NB; a.sW = w.sG; a.status = status;
            if (!up(left_fwd(P, w, s + h, h), a)) return false;
            launch_pack_split(P.fmt, Ft, NB, w.sF, n - P.k0[t], NB, P.nbs[t], fpk(P, w, t), w.sFp, nbox, st,
                              rcf_w(P, w, t), w.sRC);
        }
        for (int i = 0; i < h; ++i) {   // B_{s+h+i}' = A backward on B_{s+h+i}'s rows up to A's end
            const int t = s + h + i;
            float* Bt = w.B + P.bw_off[t];
            gather_pack_raw(P.fmt, Bt, NB, w.sB, kA, wA, KG, 0, P.nbs[t], nullptr, 0, nullptr, 0, 0, w.Gp, gplane,
                            w.sGp, nullptr, nbox, st, rcb(P, w, s), w.sRC, w.it1, w.sIT);
            TcArgs a = targs(Bt, NB, w.sB, kA + wA, P.nbs[t], GM_BWD, kA);
            a.status = status;
            if (!up(left_bwd(P, w, s, h), a)) return false;
            launch_pack_split(P.fmt, Bt, NB, w.sB, P.k0[t] + P.nbs[t], NB, P.nbs[t], bpk(P, w, t), w.sBp, nbox, st,
                              rcb_w(P, w, t), w.sRC);
        }
        launch_perm_compose(PA, PB, w.sP, n - kA, wA, nbox, st);
        return true;
    };
    // Factor the unit (s, len) whose columns are up to date with every earlier
    // unit; a B part is split at its panel only if it is the first step of a
    // pair (the join of that pair reads it; every other B part is rewritten
    // and split by a join first).
    std::function<bool(int, int, int)> factor_unit = [&](int s, int len, int top) -> bool {
        if (len == 1) return panel_ops(s, ((s - top) & 1) == 0);
        const int h = len / 2;
        if (!factor_unit(s, h, top)) return false;
        const int c0 = P.k0[s + h];
        if (!update(s, h, c0, unit_width(P, s + h, h))) return false;   // look-ahead on the second half's panels
        if (!factor_unit(s + h, h, top)) return false;
        return join(s, h);
    };
    for (const auto& u : lu_units(P)) {
        const int s = u.first, len = u.second;
        if (!factor_unit(s, len, s)) return false;
        const int c0 = P.k0[s] + unit_width(P, s, len);
        if (!update(s, len, c0, n + P.r - c0)) return false;
    }
    // Inverse permutations of the units, for gathers fused into the forward
    // solves.
    if (P.fuse_fwd)
        for (const auto& u : lu_units(P)) {
            const int s = u.first, wp = unit_width(P, s, u.second);
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
    const auto units = lu_units(P);
    auto width = [&](size_t u) { return unit_width(P, units[u].first, units[u].second); };
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
        if (!launch_tc_update(P.fmt, left_fwd(P, w, s, units[u].second), Gb[cur], gplane, w.sGp, P.KG, P.NB, a, nbox,
                              st, P.tma_epi, P.bn_max, &have))
            return false;
    }
    return true;
}

bool tc_lu_backward(const Plan& P, Work<float>& w, int nbox, int c0, int nc, const int* skip, cudaStream_t st)
{
    const long long ldm = P.ldm, gplane = ldm * P.KG;
    void* Gb[2] = {w.Gp, w.Gp2};
    float* Ib[2] = {w.it1, w.it2};
    const auto units = lu_units(P);
    auto width = [&](size_t u) { return unit_width(P, units[u].first, units[u].second); };
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
        if (!launch_tc_update(P.fmt, left_bwd(P, w, s, units[q].second), Gb[cur], gplane, w.sGp, P.KG, P.NB, a, nbox,
                              st, P.tma_epi, P.bn_max, &have))
            return false;
    }
    return true;
}

}  // namespace hps
