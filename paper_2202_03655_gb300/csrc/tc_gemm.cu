// Tensor-core GEMMs of the factored matvec K~V = U (S (U^T V)) for FP32 factors (sm_103a):
// tcgen05.mma (kind::tf32, accumulators in TMEM), operand tiles staged by TMA
// (cp.async.bulk.tensor) through an mbarrier pipeline, warp-specialised CTAs.
//
// Accuracy: one TF32 product keeps about 11 bits, far from what tol = 1e-6 needs, so every
// product is split three ways, A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi, with
// A_hi = A rounded to TF32 (cvt.rna.tf32.f32, exactly representable) and A_lo = A - A_hi.
// The dropped A_lo B_lo term is ~2^-22 relative.  The high and low parts of W and V are
// formed once per call by small preparation kernels; those of the U tiles on the fly.
//
//   k_tc_uw  : Y = alpha U W + beta B.  M = 128 rows of U (points), N = BN >= c, K = rank.
//   k_tc_utv : partial W = U^T V over a chunk of rows.  M = 128 columns of U, N = BN, K = rows.
//
// Data path of one K step (64 values of K): a U-producer warp brings the raw FP32 U tile
// (128 x 64, 32 KB) into a 4-deep ring; converter warps (thread = MMA row) read it, release the
// slot at once, split it into hi / lo and write both into TMEM with tcgen05.st.  A B-producer
// warp brings the K-major SW128 tiles of B_hi and B_lo, stacked into one 2 BN-row operand, into
// their own ring.  The MMA warp then issues, per 8 values of K, A_hi x [B_hi; B_lo] (N = 2 BN)
// and A_lo x B_hi (N = BN), both with A from TMEM.  HBM loads of U therefore wait only for the
// converters, never for MMA completion, and the issuing warp spends its time on 16 MMAs and one
// commit per 32 KB of U.
//
// The tensor core's FP32 accumulation is not rounded to nearest, and its error grows with
// the number of MMAs summed into one accumulator (about 1.7e-5 relative after 400 32-deep
// steps).  So each K step starts a fresh TMEM accumulator and the promotion warps add it
// (both N halves) into FP32 registers (round to nearest); two TMEM accumulators alternate so
// that the MMAs of the next step run while the last one is promoted.
//
// TMEM (512 columns, one CTA per SM): accumulators (2 BN columns) at 128 b, b < 2; A buffers
// (hi in 64 columns, lo in the next 64) at 256 + 128 b, b < 2.
//
// CTA roles (11 warps): warp 0 U producer, warp 1 MMA issuer and TMEM owner, warps 2-5
// converters, warps 6-9 promotion and epilogue, warp 10 B producer.  A warp w reads and
// writes TMEM lanes 32 (w mod 4) .. +31, so converter and promotion warps each cover the 128
// lanes once.  Every wait on an mbarrier is bounded by a clock limit; on expiry the kernel
// records an error, drains its own copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace hdf {
namespace tc {

constexpr int BM = 128;                 // MMA M
constexpr int BK = 64;                  // K elements per step: two 128-byte swizzle rows of FP32
constexpr int KH = 32;                  // K elements per 128-byte swizzle row (one TMA box)
constexpr int NTHREADS = 352;
constexpr int S_U = 4;                  // U ring depth (32 KB per stage)
constexpr int NACC = 2;                 // TMEM accumulators
constexpr int NA = 2;                   // TMEM A buffers (hi + lo)
constexpr int NDONE = 8;                // ring of "MMAs of step it complete" barriers
constexpr int IR = 16;                  // ring of work items handed from the U producer to the other roles
constexpr int NCONS = 10;               // item consumers: B producer, MMA warp, 4 converter and 4 promotion warps
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAcol = 256;         // first TMEM column of the A buffers
// Bounded waits.  A wait on work (a tile, a buffer, an accumulator, a work item) gives up after
// d_wait_cycles clock cycles of this device (about 2 s by default; hdf_set_wait_limit changes it,
// so that tests can make a wait run out).  The drains at exit -- every copy a producer issued
// has landed, every MMA the issuing warp committed has completed -- keep kDrainCycles whatever
// the work limit, so a CTA never frees its TMEM or leaves while its own copies are in flight.
constexpr long long kDefaultWaitCycles = 4000000000ll;   // about 2 s at 2 GHz
constexpr long long kDrainCycles = 4000000000ll;
__device__ long long d_wait_cycles = kDefaultWaitCycles;

// B ring depth (2 BN rows x 64 K per stage, hi and lo stacked): the B tiles come mostly from L2
// but with ~2000 cycles of latency, so the ring takes what shared memory leaves beside the U
// ring (at most 224 KB in all).  At most 7, which the done-ring parity argument needs.
template <int BN>
__host__ __device__ constexpr int b_stages() { return BN >= 64 ? 3 : 6; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
// The work-wait limit of this device (read on the slow path of a wait only).
__device__ __forceinline__ long long wait_limit() { return *reinterpret_cast<volatile long long*>(&d_wait_cycles); }
// Waits for the completion of the phase with the given parity; false once `limit` cycles pass.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long limit) {
    const uint32_t a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (mbar_try(a, parity)) return true;
        if (clock64() - t0 > limit) return false;
    }
}
// A wait on work: the device's work-wait limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    return mbar_wait_for(bar, parity, wait_limit());
}
// True in exactly one lane of a converged warp.
__device__ __forceinline__ bool elect_one() {
    uint32_t pred;
    asm volatile("{\n .reg .pred p;\n elect.sync _|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n" : "=r"(pred));
    return pred != 0;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout: rows of
// 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
    const uint32_t a = smem_u32(p);
    uint64_t d = 0;
    d |= (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = N_.
template <int N_>
__host__ __device__ constexpr uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N_ >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// D (TMEM) (+)= A (TMEM, 128 lanes x 8 columns) * B (shared memory descriptor).
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                            uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane -> registers (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// 16 consecutive TMEM columns of this thread's lane -> registers (no wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// registers -> 32 consecutive TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// The TF32 value nearest to x, ties away from zero, on the integer pipe: adding half a unit of
// the 13 dropped mantissa bits to the bit pattern and clearing them rounds the magnitude to
// nearest with ties away from zero (a carry into the exponent is the correct rounding up).  Equal
// to the conversion instruction cvt.rna.tf32.f32 for every finite x (hdf_check_tf32_rounding
// compares the two over all 2^32 bit patterns), at two integer operations instead of one
// conversion, which the operand converters and generators issue once per element.
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& h, uint32_t& l) {
    const float hf = tf32_hi(x);
    h = __float_as_uint(hf);
    l = __float_as_uint(x - hf);
}

// Asynchronous global -> shared copies (per thread; bytes beyond src_bytes are zero-filled), one
// commit group per pipeline step, and the wait for all but the newest N groups.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory carve-up common to both kernels: S_U raw U tiles (32 KB, 1024-aligned), SB
// stacked B tiles (per 32-K half: BN hi rows then BN lo rows of 128 bytes, K-major SW128),
// then the mbarriers.
template <int BN>
struct Smem {
    static constexpr int SB = b_stages<BN>();
    static constexpr uint32_t UBYTES = BM * BK * 4;             // one U stage
    static constexpr uint32_t BHALF = 2 * BN * KH * 4;          // stacked hi/lo rows of one 32-K half
    static constexpr uint32_t BBYTES = 2 * BHALF;               // one B stage
    unsigned char* U;
    unsigned char* B;
    uint64_t *ufull, *uempty, *bfull, *afull, *done, *acce, *drain, *itfull, *itempty;
    int64_t* items;
    uint32_t* slot;
    __device__ explicit Smem(unsigned char* raw) {
        // 1024-byte alignment by an offset from the shared-memory pointer itself, so that the
        // compiler still sees shared-memory accesses (a round trip through an integer would
        // leave generic ones)
        unsigned char* base = raw + ((1024u - (smem_u32(raw) & 1023u)) & 1023u);
        U = base;
        B = U + S_U * UBYTES;
        ufull = reinterpret_cast<uint64_t*>(B + SB * BBYTES);
        uempty = ufull + S_U;
        bfull = uempty + S_U;
        afull = bfull + SB;
        done = afull + NA;
        acce = done + NDONE;
        drain = acce + NACC;
        itfull = drain + 1;
        itempty = itfull + IR;
        items = reinterpret_cast<int64_t*>(itempty + IR);
        slot = reinterpret_cast<uint32_t*>(items + IR);
    }
    static constexpr size_t bytes() {
        return 1024 + (size_t)S_U * UBYTES + (size_t)SB * BBYTES + (2 * S_U + SB + NA + NDONE + NACC + 1 + 3 * IR) * 8 +
               16;
    }
};

// Barrier set-up and TMEM allocation (warp 1 owns the TMEM); returns the TMEM base address.
// ncons: item consumers (warps and threads that release an item slot); bcount: arrivals that
// complete a B stage (1 for a TMA producer, the warp count for B-generator warps).
template <int BN>
__device__ __forceinline__ uint32_t cta_setup(Smem<BN>& sm, int warp, int ncons = NCONS, int bcount = 1) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < S_U; ++s) { mbar_init(&sm.ufull[s], 1); mbar_init(&sm.uempty[s], 4); }
        for (int s = 0; s < Smem<BN>::SB; ++s) mbar_init(&sm.bfull[s], bcount);
        for (int b = 0; b < NA; ++b) mbar_init(&sm.afull[b], 4);
        for (int j = 0; j < NDONE; ++j) mbar_init(&sm.done[j], 1);
        for (int b = 0; b < NACC; ++b) mbar_init(&sm.acce[b], 4);
        mbar_init(sm.drain, 1);
        for (int j = 0; j < IR; ++j) { mbar_init(&sm.itfull[j], 1); mbar_init(&sm.itempty[j], ncons); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sm.slot)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *sm.slot;
}

template <int BN>
__device__ __forceinline__ void cta_teardown(uint32_t tmem, int warp) {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Waits until the MMAs of step j are complete (one tcgen05.commit per step on done[j mod 8]).
// Every waiter has already seen step j - 8 complete, and step j + 8 cannot be issued before the
// waiter moves on (the B producer runs at most SB <= 7 steps ahead of the MMAs, the converters
// NA = 2, and the MMAs at most NACC = 2 steps ahead of the promotion), so the parity is
// unambiguous.
template <int BN>
__device__ __forceinline__ bool wait_done(Smem<BN>& sm, uint32_t j) {
    return mbar_wait(&sm.done[j % NDONE], (j / NDONE) & 1);
}

// The MMA warp waits on three barriers at once: lane 0 the accumulator, lane 1 the B stage,
// the other lanes the A buffer, so one try_wait instruction covers all three.
__device__ __forceinline__ bool mbar_wait_lanes(uint32_t a, uint32_t parity) {
    bool mine = mbar_try(a, parity);
    if (__all_sync(0xffffffffu, mine)) return true;
    const long long lim = wait_limit();
    const long long t0 = clock64();
    for (;;) {
        if (!mine) mine = mbar_try(a, parity);
        if (__all_sync(0xffffffffu, mine)) return true;
        if (__any_sync(0xffffffffu, clock64() - t0 > lim)) return false;
    }
}

// MMA issuer (whole warp converged; one elected lane issues): per K step, 8 x (A_hi x [B_hi;
// B_lo], A_lo x B_hi) from the A buffer in TMEM and the stacked B stage, then one commit that
// frees the B stage and the A buffer and publishes the accumulator.
template <int BN>
__device__ __forceinline__ bool mma_step(Smem<BN>& sm, uint32_t tmem, uint32_t it, int lane) {
    constexpr int SB = Smem<BN>::SB;
    constexpr uint32_t id2 = idesc_tf32<2 * BN>(), id1 = idesc_tf32<BN>();
    const uint32_t sb = it % SB, b = it % NA, buf = it % NACC;
    const uint32_t a = lane == 0 ? smem_u32(&sm.acce[buf]) : lane == 1 ? smem_u32(&sm.bfull[sb]) : smem_u32(&sm.afull[b]);
    const uint32_t par = lane == 0 ? ((it / NACC) & 1) ^ 1 : lane == 1 ? (it / SB) & 1 : (it / NA) & 1;
    if (!mbar_wait_lanes(a, par)) return false;
    tc_fence_after();
    const uint32_t d = tmem + buf * 2 * BN;
    const uint32_t ahi = tmem + kAcol + 128 * b, alo = ahi + 64;
    const uint64_t b0 = sw128_desc(sm.B + sb * Smem<BN>::BBYTES);
    constexpr uint64_t halfstep = Smem<BN>::BHALF >> 4;
    if (elect_one()) {
#pragma unroll
        for (int kk = 0; kk < BK / 8; ++kk) {
            const uint64_t db = b0 + (kk >> 2) * halfstep + (uint64_t)(((kk & 3) * 32) >> 4);
            mma_tf32_ts(d, ahi + 8 * kk, db, id2, kk > 0 ? 1u : 0u);     // [hi.hi | hi.lo]
            mma_tf32_ts(d, alo + 8 * kk, db, id1, 1u);                  // lo.hi into the first half
        }
        mma_commit(&sm.done[it % NDONE]);
    }
    __syncwarp();
    return true;
}

// Converter tail: 64 raw values of this thread's row -> hi / lo in A buffer of step `it`.
template <int BN>
__device__ __forceinline__ void convert_publish(Smem<BN>& sm, uint32_t tmem, uint32_t it, int q, int lane,
                                                const float* x) {
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + kAcol + 128 * (it % NA);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t hi[32], lo[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) split_tf32(x[32 * h + k], hi[k], lo[k]);
        tmem_st32(ta + 32 * h, hi);
        tmem_st32(ta + 64 + 32 * h, lo);
    }
    tmem_st_wait();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.afull[it % NA]);
}

// Converter head: wait for the U stage of step `it` and for the A buffer, then (after the caller
// has read the stage) release the stage.
template <int BN>
__device__ __forceinline__ bool convert_wait(Smem<BN>& sm, uint32_t it) {
    if (!mbar_wait(&sm.ufull[it % S_U], (it / S_U) & 1)) return false;
    if (it >= (uint32_t)NA && !wait_done<BN>(sm, it - NA)) return false;
    tc_fence_after();
    return true;
}
template <int BN>
__device__ __forceinline__ void convert_release(Smem<BN>& sm, uint32_t it, int lane) {
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.uempty[it % S_U]);
}

// Promotion of the accumulator of step `it` (both N halves) into FP32 registers.
template <int BN>
__device__ __forceinline__ bool promote(Smem<BN>& sm, uint32_t tmem, uint32_t it, int q, int lane, float* acc) {
    const uint32_t buf = it % NACC;
    if (!wait_done<BN>(sm, it)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + buf * 2 * BN;
    uint32_t v[2 * BN];
    if constexpr (BN == 16) {
        tmem_ld32(ta, v);
    } else {
#pragma unroll
        for (int j0 = 0; j0 < 2 * BN; j0 += 32) tmem_ld32(ta + j0, v + j0);
    }
    tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] += __uint_as_float(v[j]) + __uint_as_float(v[BN + j]);
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.acce[buf]);
    return true;
}

// The same promotion 32 accumulator columns at a time (half the registers of promote), for
// kernels whose promotion warps keep more state beside the sums.
template <int BN>
__device__ __forceinline__ bool promote_lean(Smem<BN>& sm, uint32_t tmem, uint32_t it, int q, int lane, float* acc) {
    const uint32_t buf = it % NACC;
    if (!wait_done<BN>(sm, it)) return false;
    tc_fence_after();
    const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + buf * 2 * BN;
    if constexpr (BN == 16) {
        uint32_t v[32];
        tmem_ld32(ta, v);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] += __uint_as_float(v[j]) + __uint_as_float(v[16 + j]);
    } else {
#pragma unroll
        for (int j0 = 0; j0 < BN; j0 += 32) {
            uint32_t a[32], b[32];
            tmem_ld32(ta + j0, a);
            tmem_ld32(ta + BN + j0, b);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j0 + j] += __uint_as_float(a[j]) + __uint_as_float(b[j]);
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.acce[buf]);
    return true;
}

// MMA warp exit: every MMA it issued is complete before the CTA frees its TMEM.
template <int BN>
__device__ __forceinline__ void mma_drain(Smem<BN>& sm, bool ok, int* err) {
    if (elect_one()) mma_commit(sm.drain);
    __syncwarp();
    if (!mbar_wait_for(sm.drain, 0, kDrainCycles)) ok = false;
    if (!ok && (threadIdx.x & 31) == 0) atomicExch(err, 1);
}

// Producer drain: every copy this thread issued on `full` (a ring of `depth`) has landed.
__device__ __forceinline__ bool producer_drain(uint64_t* full, int depth, uint32_t it) {
    bool ok = true;
    for (uint32_t q = (it > (uint32_t)depth ? it - depth : 0); q < it; ++q)
        if (!mbar_wait_for(&full[q % depth], (q / depth) & 1, kDrainCycles)) ok = false;
    return ok;
}

// B producer, one step: stacked hi / lo tiles of K rows [k0, k0 + 64) (two 32-K halves) and
// operand rows [y0, y0 + BN).
template <int BN>
__device__ __forceinline__ bool load_b(Smem<BN>& sm, uint32_t it, const CUtensorMap* mhi, const CUtensorMap* mlo,
                                       int k0, int y0 = 0) {
    constexpr int SB = Smem<BN>::SB;
    const uint32_t sb = it % SB;
    if (it >= (uint32_t)SB && !wait_done<BN>(sm, it - SB)) return false;
    mbar_expect_tx(&sm.bfull[sb], Smem<BN>::BBYTES);
    unsigned char* dst = sm.B + sb * Smem<BN>::BBYTES;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        tma_load_2d(dst + h * Smem<BN>::BHALF, mhi, k0 + KH * h, y0, &sm.bfull[sb]);
        tma_load_2d(dst + h * Smem<BN>::BHALF + BN * KH * 4, mlo, k0 + KH * h, y0, &sm.bfull[sb]);
    }
    return true;
}

// Work-item hand-off (dynamic scheduling).  The U producer takes item k of this CTA (its block
// index first, then from a global counter), publishes it in slot k mod 16 and moves on; every
// other role reads the slot once and releases it.  A value >= nitems ends the sequence.
template <int BN>
__device__ __forceinline__ bool publish_item(Smem<BN>& sm, uint32_t k, int64_t item) {
    const uint32_t j = k % IR;
    if (!mbar_wait(&sm.itempty[j], ((k / IR) & 1) ^ 1)) return false;
    sm.items[j] = item;
    mbar_arrive(&sm.itfull[j]);
    return true;
}
// Called by one thread (whole_warp false) or by a whole converged warp; -1 on a timeout.
template <int BN>
__device__ __forceinline__ int64_t take_item(Smem<BN>& sm, uint32_t k, bool whole_warp) {
    const uint32_t j = k % IR;
    bool ok = mbar_wait(&sm.itfull[j], (k / IR) & 1);
    if (whole_warp) ok = __all_sync(0xffffffffu, ok);
    if (!ok) return -1;
    const int64_t item = sm.items[j];
    if (whole_warp) __syncwarp();
    if (!whole_warp || (threadIdx.x & 31) == 0) mbar_arrive(&sm.itempty[j]);
    return item;
}

struct UwArgs {
    int64_t n;          // rows of U
    int nkt;            // K steps (ceil(rank / 64))
    int c;              // columns of W, Y
    float alpha, beta;
    const float* B; int64_t ldb;
    float* Y; int64_t ldy;
    int* err;
};

// Y = alpha U W + beta B for 128-row tiles of U (persistent over tiles).
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_uw(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mW,
            const __grid_constant__ CUtensorMap mWlo, UwArgs p) {
    using SM = Smem<BN>;
    extern __shared__ unsigned char raw[];
    SM sm(raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = cta_setup<BN>(sm, warp);
    const int64_t ntiles = (p.n + BM - 1) / BM;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int kt = 0; kt < p.nkt; ++kt, ++it) {
                    const uint32_t s = it % S_U;
                    if (!mbar_wait(&sm.uempty[s], ((it / S_U) & 1) ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&sm.ufull[s], SM::UBYTES);
                    unsigned char* dst = sm.U + s * SM::UBYTES;
                    tma_load_2d(dst, &mU, kt * BK, (int)(tile * BM), &sm.ufull[s]);
                    tma_load_2d(dst + SM::UBYTES / 2, &mU, kt * BK + KH, (int)(tile * BM), &sm.ufull[s]);
                }
            }
            if (!producer_drain(sm.ufull, S_U, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
                for (int kt = 0; kt < p.nkt && ok; ++kt, ++it) ok = load_b<BN>(sm, it, &mW, &mWlo, kt * BK);
            if (!producer_drain(sm.bfull, SM::SB, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 1) {
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
            for (int kt = 0; kt < p.nkt && ok; ++kt, ++it) ok = mma_step<BN>(sm, tmem, it, lane);
        mma_drain(sm, ok, p.err);
    } else if (warp < 6) {
        // thread = row m of the U tile; each 32-K half is SW128 (16-byte chunk j of row m at chunk
        // position j ^ (m mod 8)), so the eight threads of a load phase hit distinct banks
        const int q = warp & 3, m = 32 * q + lane;
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int kt = 0; kt < p.nkt; ++kt, ++it) {
                if (!convert_wait<BN>(sm, it)) { ok = false; break; }
                const unsigned char* R = sm.U + (it % S_U) * SM::UBYTES + m * 128;
                float x[64];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 v = *reinterpret_cast<const float4*>(R + h * (SM::UBYTES / 2) + ((j ^ (m & 7)) << 4));
                        x[32 * h + 4 * j + 0] = v.x; x[32 * h + 4 * j + 1] = v.y;
                        x[32 * h + 4 * j + 2] = v.z; x[32 * h + 4 * j + 3] = v.w;
                    }
                convert_release<BN>(sm, it, lane);
                convert_publish<BN>(sm, tmem, it, q, lane, x);
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            for (int kt = 0; kt < p.nkt && ok; ++kt, ++it) ok = promote<BN>(sm, tmem, it, q, lane, acc);
            if (!ok) break;
            const int64_t row = tile * BM + 32 * q + lane;
            if (row < p.n) {
#pragma unroll
                for (int j = 0; j < BN; ++j) {
                    if (j < p.c) {
                        float out = p.alpha * acc[j];
                        if (p.B) out += p.beta * p.B[row + (int64_t)j * p.ldb];
                        p.Y[row + (int64_t)j * p.ldy] = out;
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    }
    cta_teardown<BN>(tmem, warp);
}

struct UtvArgs {
    int64_t r;          // columns of U (M extent)
    int64_t n;          // rows of U
    int64_t chunk;      // rows per K chunk (a multiple of 64)
    int nchunk;
    int mblocks;        // ceil(r / 128)
    int c;
    double* part;       // part[(chunk * c + j) * r + a]
    float* part32;      // the same partial sums in FP32 (each is an FP32 register sum) when not null
    int* err;
    int* next;          // work-item counter, zero at launch
};

// Partial U^T V: items (column block of U, chunk of rows), persistent over items.
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_utv(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mV,
             const __grid_constant__ CUtensorMap mVlo, UtvArgs p) {
    using SM = Smem<BN>;
    extern __shared__ unsigned char raw_[];
    SM sm(raw_);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = cta_setup<BN>(sm, warp);
    const int64_t nitems = (int64_t)p.mblocks * p.nchunk;
    bool ok = true;
    auto ksteps = [&](int64_t item) -> int {
        const int64_t ch = item / p.mblocks;
        const int64_t i0 = ch * p.chunk, i1 = min(p.n, i0 + p.chunk);
        return (int)((i1 - i0 + BK - 1) / BK);
    };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0, k = 0;
            int64_t item = blockIdx.x;
            while (ok) {
                if (!publish_item<BN>(sm, k++, item)) { ok = false; break; }
                if (item >= nitems) break;
                const int64_t mb = item % p.mblocks, ch = item / p.mblocks;
                const int64_t i0 = ch * p.chunk;
                const int nk = ksteps(item);
                // the next item is claimed 8 steps before the end of this one, so that the
                // atomic's latency overlaps the copies still to be issued
                const int claim_at = nk > 8 ? nk - 8 : 0;
                int64_t nxt = nitems;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    if (kt == claim_at) nxt = (int64_t)gridDim.x + atomicAdd(p.next, 1);
                    const uint32_t s = it % S_U;
                    if (!mbar_wait(&sm.uempty[s], ((it / S_U) & 1) ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&sm.ufull[s], SM::UBYTES);
                    tma_load_2d(sm.U + s * SM::UBYTES, &mU, (int)(mb * BM), (int)(i0 + (int64_t)kt * BK), &sm.ufull[s]);
                }
                item = nxt;
            }
            if (!producer_drain(sm.ufull, S_U, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            uint32_t it = 0;
            for (uint32_t k = 0; ok; ++k) {
                const int64_t item = take_item<BN>(sm, k, false);
                if (item < 0) { ok = false; break; }
                if (item >= nitems) break;
                const int64_t i0 = (item / p.mblocks) * p.chunk;
                const int nk = ksteps(item);
                for (int kt = 0; kt < nk && ok; ++kt, ++it)
                    ok = load_b<BN>(sm, it, &mV, &mVlo, (int)(i0 + (int64_t)kt * BK));
            }
            if (!producer_drain(sm.bfull, SM::SB, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 1) {
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk && ok; ++kt, ++it) ok = mma_step<BN>(sm, tmem, it, lane);
        }
        mma_drain(sm, ok, p.err);
    } else if (warp < 6) {
        // thread = column m of the U block (row m of A = U^T); the stored tile is [64 rows][128
        // columns], so each load of the warp reads 32 consecutive floats of one row
        const int q = warp & 3, m = 32 * q + lane;
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                if (!convert_wait<BN>(sm, it)) { ok = false; break; }
                const float* R = reinterpret_cast<const float*>(sm.U + (it % S_U) * SM::UBYTES) + m;
                float x[64];
#pragma unroll
                for (int k2 = 0; k2 < BK; ++k2) x[k2] = R[k2 * BM];
                convert_release<BN>(sm, it, lane);
                convert_publish<BN>(sm, tmem, it, q, lane, x);
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk && ok; ++kt, ++it) ok = promote_lean<BN>(sm, tmem, it, q, lane, acc);
            if (!ok) break;
            const int64_t mb = item % p.mblocks, ch = item / p.mblocks;
            const int64_t a = mb * BM + 32 * q + lane;
            if (a < p.r) {
                if (p.part32) {
#pragma unroll
                    for (int j = 0; j < BN; ++j)
                        if (j < p.c) p.part32[((int64_t)ch * p.c + j) * p.r + a] = acc[j];
                } else {
#pragma unroll
                    for (int j = 0; j < BN; ++j)
                        if (j < p.c) p.part[((int64_t)ch * p.c + j) * p.r + a] = (double)acc[j];
                }
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    }
    cta_teardown<BN>(tmem, warp);
}

// ------------------------------------------------ matrix-free products on the tensor cores
// The products of a matrix-free factor (mfree.cu): the stored Z rows are the A operand, brought
// by TMA exactly like the U tiles of k_tc_utv / k_tc_uw; only the small second operand changes.
//   k_tc_mf_utv: W[(k,s,m,j), c] = sum_i Z[i, zoff_m + j] (A0F[i, aoff_m + q] V[i, c]).
//     M = 128 rows j of the tails of degree m, N = BN columns n = (q, c), K = points.  The B
//     tiles A0F (.) V are formed in shared memory by two generator warps (10, 11), in the
//     K-major 128-byte-swizzle layout the TMA would write, TF32 hi / lo stacked.  For the small
//     degrees (few tails j, many pairs q) a tile takes the transposed roles: M = 128 pairs q (the
//     A0F block of m by TMA), N = BN columns n = (j, c), B = Z (.) V.
//   k_tc_mf_uw: Y[i, c] = sum over phases (m, n0) of sum_q A0F[i, aoff_m + q] Q[i, (q, c)],
//     Q = Z[:, zoff_m + j] W_m[j, (q, c)]: M = 128 points, N = BN columns, K = the tails of m.
//     The B tiles come by TMA from W gathered per phase (k_prep_mf_w); the promotion warps
//     contract each phase's accumulator with A0F into y and write Y once per tile.
constexpr int NGEN = 2;                 // B-generator warps (10, 11)
constexpr int NTHREADS_MF = 32 * (10 + NGEN);   // the roles of k_tc_utv, the generators in place of the B producer
constexpr int NCONS_MF = NGEN + 9;      // item consumers: generators, MMA, 4 converters, 4 promotion

struct MfUtvTcArgs {
    int64_t n, chunk;                   // points, points per K chunk (a multiple of 64)
    int nchunk, ntiles;
    const int4* tiles;                  // (m, y0, n0, flag), see k_tc_mf_utv
    const float* A0F; int ldA;
    const float* Z; int ldZ;
    const float* V; int64_t ldv; int c;
    const int* zoff; const int* zcnt; const int* aoff; const int* acnt; const int64_t* wcol;
    double* part; int64_t r;            // part[(chunk * c + cc) * r + a]
    int* err; int* next;
};

// CP: c padded to 16, 32 or 64 (a divisor of BN).  Tile (m, y0, n0, flag): with flag 0 rows
// y0.. are the tails j of degree m (A = Z columns zoff_m + j, map mZ) and column n is
// (q, cc) = (n / CP, n mod CP) (B = A0F (.) V); with flag 1 rows y0.. are the pairs q of m
// (A = A0F columns aoff_m + q, map mA) and column n is (j, cc) (B = Z (.) V).  Columns with
// cc >= c are zero.
template <int BN, int CP>
__global__ void __launch_bounds__(NTHREADS_MF, 1)
    k_tc_mf_utv(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mA, MfUtvTcArgs p) {
    using SM = Smem<BN>;
    static_assert(BN % CP == 0, "column groups must not straddle a tile");
    constexpr int SB = SM::SB;
    // with CP = 16 the last U stage holds the generators' staging ring and Z takes the others
    constexpr bool STG = CP == 16;
    constexpr int SU = STG ? S_U - 1 : S_U;
    extern __shared__ unsigned char raw_[];
    SM sm(raw_);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = cta_setup<BN>(sm, warp, NCONS_MF, NGEN);
    const int64_t nitems = (int64_t)p.ntiles * p.nchunk;
    bool ok = true;
    auto ksteps = [&](int64_t item) -> int {
        const int64_t ch = item / p.ntiles;
        const int64_t i0 = ch * p.chunk, i1 = min(p.n, i0 + p.chunk);
        return (int)((i1 - i0 + BK - 1) / BK);
    };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0, k = 0;
            int64_t item = blockIdx.x;
            while (ok) {
                if (!publish_item<BN>(sm, k++, item)) { ok = false; break; }
                if (item >= nitems) break;
                const int4 tl = p.tiles[item % p.ntiles];
                const int64_t i0 = (item / p.ntiles) * p.chunk;
                const CUtensorMap* map = tl.w ? &mA : &mZ;
                const int zx = (tl.w ? p.aoff[tl.x] : p.zoff[tl.x]) + tl.y;
                const int nk = ksteps(item);
                const int claim_at = nk > 8 ? nk - 8 : 0;
                int64_t nxt = nitems;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    if (kt == claim_at) nxt = (int64_t)gridDim.x + atomicAdd(p.next, 1);
                    const uint32_t s = it % SU;
                    if (!mbar_wait(&sm.uempty[s], ((it / SU) & 1) ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&sm.ufull[s], SM::UBYTES);
                    tma_load_2d(sm.U + s * SM::UBYTES, map, zx, (int)(i0 + (int64_t)kt * BK), &sm.ufull[s]);
                }
                item = nxt;
            }
            if (!producer_drain(sm.ufull, SU, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp >= 10) {
        // B generators: warp 10 forms points 0..31 of a step, warp 11 points 32..63 (the two
        // 32-K halves of the stage).  A thread owns four consecutive points 4 pg .. 4 pg + 3 (one
        // 16-byte chunk of a K-major row; pg = 8 (warp - 10) + lane mod 8) and the 16 rows
        // n = g CP + rs CP / 4 + u of the stage (rs = lane / 8, g < BN / CP, u < CP / 4).  Per step
        // it takes the BN / CP values of A0F of each point (one aligned 16-byte piece: A0F blocks
        // start on 16-byte boundaries and q0 is a multiple of BN / CP) and four values of V per
        // column, and writes each row's hi and lo chunk with one 16-byte store.  With CP = 16 the
        // values come through a cp.async ring DS - 1 steps ahead, otherwise as register loads one
        // step ahead.
        static_assert(NGEN * 32 == BK && BN == 64, "two generator warps, 8 chunks x 4 row sets each");
        constexpr int NQ = BN / CP, NU = CP / 4;
        const int pg = (warp - 10) * 8 + (lane & 7), rs = lane >> 3;
        const int h = warp - 10, jc = lane & 7;
        const bool vec = ((reinterpret_cast<uintptr_t>(p.V) | (uintptr_t)p.ldv * 4u) & 15u) == 0;
        if constexpr (STG) {
            // values of DS steps staged by cp.async, DS - 1 steps ahead (A0F rows come mostly from
            // DRAM, far beyond one step's time).  Slot: the 4 x 16 chunks of the generated factor
            // (chunk [e][pg]: the 16 bytes of point 4 pg + e, copied by the lane with rs = e and
            // read by the four lanes of pg after the warp's barrier), then the 4 x 64 chunks of V
            // (chunk [u][t]: the four points of column 4 rs + u, copied and read by thread t).
            constexpr int DS = 4, SLOT = (4 * 16 + 4 * 64) * 4;     // floats per slot
            static_assert(NQ == 4 && NU == 4 && DS * SLOT * 4 <= (int)SM::UBYTES, "the ring fits one U stage");
            float* stg = reinterpret_cast<float*>(sm.U + (S_U - 1) * SM::UBYTES);
            const int t = (warp - 10) * 32 + lane;
            uint32_t it = 0;
            for (uint32_t k = 0; ok; ++k) {
                const int64_t item = take_item<BN>(sm, k, true);
                if (item < 0) { ok = false; break; }
                if (item >= nitems) break;
                const int4 tl = p.tiles[item % p.ntiles];
                // the generated operand's factor: A0F columns aoff_m + q (flag 0) or Z columns
                // zoff_m + j (flag 1), from column q0 of the block of nq
                const int m = tl.x, q0 = tl.z / CP;
                const float* gsrc = tl.w ? p.Z : p.A0F;
                const int64_t gld = tl.w ? (int64_t)p.ldZ : (int64_t)p.ldA;
                const int ao = tl.w ? p.zoff[m] : p.aoff[m], nq = tl.w ? p.zcnt[m] : p.acnt[m];
                const int64_t i0 = (item / p.ntiles) * p.chunk, i1 = min(p.n, i0 + p.chunk);
                const int nk = ksteps(item);
                const uint32_t abytes = 4u * (uint32_t)max(0, min(NQ, nq - q0));
                // per-item bases, advanced by one step of BK points per copy
                const int64_t ib = i0 + 4 * pg;
                const float* g_first = gsrc + ao + q0;                       // row 0: a valid address
                const float* a_base = g_first + (ib + rs) * gld;
                const int64_t a_step = (int64_t)BK * gld;
                // the copies of step kt2 (zero-filled outside the item; an empty group past its end)
                auto issue = [&](int kt2) {
                    if (kt2 < nk) {
                        float* slot = stg + (kt2 % DS) * SLOT;
                        const int64_t i4 = ib + (int64_t)kt2 * BK;
                        const bool pe = i4 + rs < i1;
                        cp_async16(slot + (rs * 16 + pg) * 4, pe ? a_base + kt2 * a_step : g_first, pe ? abytes : 0u);
                        const int cnt = (int)max((int64_t)0, min((int64_t)4, i1 - i4));
#pragma unroll
                        for (int u = 0; u < NU; ++u) {
                            const int cc = rs * NU + u;
                            const int nv = cc < p.c ? cnt : 0;
                            float* dst = slot + 4 * 16 * 4 + (u * 64 + t) * 4;
                            const float* vp = nv > 0 ? p.V + i4 + (int64_t)cc * p.ldv : p.V;
                            if (vec) {
                                cp_async16(dst, vp, 4u * (uint32_t)nv);
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e) cp_async4(dst + e, e < nv ? vp + e : p.V, e < nv ? 4u : 0u);
                            }
                        }
                    }
                    cp_commit();
                };
#pragma unroll
                for (int kt2 = 0; kt2 < DS - 1; ++kt2) issue(kt2);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const uint32_t sb = it % SB;
                    issue(kt + DS - 1);
                    cp_wait<DS - 1>();
                    __syncwarp();            // the factor chunks of the other lanes of this warp
                    const float* slot = stg + (kt % DS) * SLOT;
                    float av[NQ][4], vv[NU][4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float4 w = *reinterpret_cast<const float4*>(slot + (e * 16 + pg) * 4);
                        av[0][e] = w.x; av[1][e] = w.y; av[2][e] = w.z; av[3][e] = w.w;
                    }
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        const float4 w = *reinterpret_cast<const float4*>(slot + 4 * 16 * 4 + (u * 64 + t) * 4);
                        vv[u][0] = w.x; vv[u][1] = w.y; vv[u][2] = w.z; vv[u][3] = w.w;
                    }
                    bool free_ = (it < (uint32_t)SB) || wait_done<BN>(sm, it - SB);
                    free_ = __all_sync(0xffffffffu, free_);
                    if (!free_) { ok = false; break; }
                    unsigned char* stage = sm.B + sb * SM::BBYTES + h * SM::BHALF;
#pragma unroll
                    for (int g = 0; g < NQ; ++g)
#pragma unroll
                        for (int u = 0; u < NU; ++u) {
                            const int nrow = g * CP + rs * NU + u;
                            uint32_t hi[4], lo[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) split_tf32(av[g][e] * vv[u][e], hi[e], lo[e]);
                            const uint32_t off = (uint32_t)nrow * 128u + ((uint32_t)(jc ^ (nrow & 7)) << 4);
                            *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                            *reinterpret_cast<uint4*>(stage + BN * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                        }
                    // the tensor core reads the stage through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.bfull[sb]);
                }
                cp_wait<0>();      // no copy of this thread is in flight past its item
                if (!ok) break;
            }
        } else {
            uint32_t it = 0;
            for (uint32_t k = 0; ok; ++k) {
                const int64_t item = take_item<BN>(sm, k, true);
                if (item < 0) { ok = false; break; }
                if (item >= nitems) break;
                const int4 tl = p.tiles[item % p.ntiles];
                // the generated operand's factor: A0F columns aoff_m + q (flag 0) or Z columns
                // zoff_m + j (flag 1), from column q0 of the block of nq
                const int m = tl.x, q0 = tl.z / CP;
                const float* gsrc = tl.w ? p.Z : p.A0F;
                const int64_t gld = tl.w ? (int64_t)p.ldZ : (int64_t)p.ldA;
                const int ao = tl.w ? p.zoff[m] : p.aoff[m], nq = tl.w ? p.zcnt[m] : p.acnt[m];
                const int64_t i0 = (item / p.ntiles) * p.chunk, i1 = min(p.n, i0 + p.chunk);
                const int nk = ksteps(item);
                // the thread's values for step kt; with CP <= 32 the next step's are loaded while this
                // step's products are formed
                constexpr bool PF = CP <= 32;
                float av[NQ][4], vv[NU][4], an[NQ][4], vn[NU][4];
                auto load = [&](int kt2, float (&a_)[NQ][4], float (&v_)[NU][4]) {
                    const int64_t i4 = i0 + (int64_t)kt2 * BK + 4 * pg;
                    const bool on = kt2 < nk;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const bool pe = on && i4 + e < i1;
                        const float* ap = gsrc + (i4 + e) * gld + ao + q0;
                        float w[NQ];
                        if constexpr (NQ == 4) {
                            const float4 t = pe ? __ldg(reinterpret_cast<const float4*>(ap)) : make_float4(0.f, 0.f, 0.f, 0.f);
                            w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
                        } else if constexpr (NQ == 2) {
                            const float2 t = pe ? __ldg(reinterpret_cast<const float2*>(ap)) : make_float2(0.f, 0.f);
                            w[0] = t.x; w[1] = t.y;
                        } else {
                            w[0] = pe ? __ldg(ap) : 0.f;
                        }
#pragma unroll
                        for (int g = 0; g < NQ; ++g) a_[g][e] = q0 + g < nq ? w[g] : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < NU; ++u) {
                        const int cc = rs * NU + u;
                        const float* vp = p.V + i4 + (int64_t)cc * p.ldv;
                        if (on && cc < p.c && vec && i4 + 3 < i1) {
                            const float4 w = __ldg(reinterpret_cast<const float4*>(vp));
                            v_[u][0] = w.x; v_[u][1] = w.y; v_[u][2] = w.z; v_[u][3] = w.w;
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) v_[u][e] = (on && cc < p.c && i4 + e < i1) ? __ldg(vp + e) : 0.f;
                        }
                    }
                };
                if (PF) load(0, av, vv);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const uint32_t sb = it % SB;
                    if (PF) {
                        load(kt + 1, an, vn);
                    } else {
                        load(kt, av, vv);
                    }
                    bool free_ = (it < (uint32_t)SB) || wait_done<BN>(sm, it - SB);
                    free_ = __all_sync(0xffffffffu, free_);
                    if (!free_) { ok = false; break; }
                    unsigned char* stage = sm.B + sb * SM::BBYTES + h * SM::BHALF;
#pragma unroll
                    for (int g = 0; g < NQ; ++g)
#pragma unroll
                        for (int u = 0; u < NU; ++u) {
                            const int nrow = g * CP + rs * NU + u;
                            uint32_t hi[4], lo[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) split_tf32(av[g][e] * vv[u][e], hi[e], lo[e]);
                            const uint32_t off = (uint32_t)nrow * 128u + ((uint32_t)(jc ^ (nrow & 7)) << 4);
                            *reinterpret_cast<uint4*>(stage + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                            *reinterpret_cast<uint4*>(stage + BN * 128 + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                        }
                    // the tensor core reads the stage through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&sm.bfull[sb]);
                    if (PF) {
#pragma unroll
                        for (int g = 0; g < NQ; ++g)
#pragma unroll
                            for (int e = 0; e < 4; ++e) av[g][e] = an[g][e];
#pragma unroll
                        for (int u = 0; u < NU; ++u)
#pragma unroll
                            for (int e = 0; e < 4; ++e) vv[u][e] = vn[u][e];
                    }
                }
                if (!ok) break;
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else if (warp == 1) {
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk && ok; ++kt, ++it) ok = mma_step<BN>(sm, tmem, it, lane);
        }
        mma_drain(sm, ok, p.err);
    } else if (warp < 6) {
        // thread = row m of A (column j0 + m of the Z block); the stored tile is [64 points][128 columns]
        const int q = warp & 3, mrow = 32 * q + lane;
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                if (!mbar_wait(&sm.ufull[it % SU], (it / SU) & 1)) { ok = false; break; }
                if (it >= (uint32_t)NA && !wait_done<BN>(sm, it - NA)) { ok = false; break; }
                tc_fence_after();
                const float* R = reinterpret_cast<const float*>(sm.U + (it % SU) * SM::UBYTES) + mrow;
                float x[64];
#pragma unroll
                for (int k2 = 0; k2 < BK; ++k2) x[k2] = R[k2 * BM];
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.uempty[it % SU]);
                convert_publish<BN>(sm, tmem, it, q, lane, x);
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        for (uint32_t k = 0; ok; ++k) {
            const int64_t item = take_item<BN>(sm, k, true);
            if (item < 0) { ok = false; break; }
            if (item >= nitems) break;
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk && ok; ++kt, ++it) ok = promote_lean<BN>(sm, tmem, it, q, lane, acc);
            if (!ok) break;
            const int4 tl = p.tiles[item % p.ntiles];
            const int m = tl.x, ao = p.aoff[m], nq = p.acnt[m], zq = p.zcnt[m], g0 = tl.z / CP;
            const int64_t ch = item / p.ntiles;
            // this thread's row: a tail j (flag 0) or a pair q (flag 1); column group g: the pair
            // q0 + g or the tail j0 + g; U column of (q, j): wcol[aoff_m + q] + j
            const int row = tl.y + 32 * q + lane;
            if (row < (tl.w ? nq : zq)) {
#pragma unroll
                for (int g = 0; g < BN / CP; ++g) {
                    if (g0 + g >= (tl.w ? zq : nq)) continue;
                    const int64_t a = tl.w ? p.wcol[ao + row] + g0 + g : p.wcol[ao + g0 + g] + row;
#pragma unroll
                    for (int cc = 0; cc < CP; ++cc)
                        if (cc < p.c) p.part[(ch * p.c + cc) * p.r + a] = (double)acc[g * CP + cc];
                }
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    }
    cta_teardown<BN>(tmem, warp);
}

// m: the tail degree, plus kMfFlip when the phase takes the transposed roles (K = the pairs q of
// m, columns n = (j, c), A = the A0F block of m, the accumulator contracted with Z).
constexpr int kMfFlip = 1 << 16;
struct MfPhase {
    int m, n0, nk, y0;                  // tail degree (| kMfFlip), first column, K steps, row of its B tiles
};

struct MfUwTcArgs {
    int64_t n;                          // points
    int nphase;
    const MfPhase* phases;
    const int* zoff; const int* aoff; const int* acnt; const int* zcnt;
    const float* A0F; int ldA;
    const float* Z; int ldZ;
    int c;
    float* Y; int64_t ldy;
    int* err;
};

// Y for 128-point tiles (persistent over tiles), phases in order; CP = c padded to 16, 32 or
// 64 (a divisor of BN), so the column (q, cc) of accumulator entry j is q = (n0 + j) / CP,
// cc = j mod CP (for a transposed phase the column (j, cc) with the tail j = (n0 + j) / CP).
template <int BN, int CP>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_mf_uw(const __grid_constant__ CUtensorMap mZ, const __grid_constant__ CUtensorMap mA,
               const __grid_constant__ CUtensorMap mW, const __grid_constant__ CUtensorMap mWlo, MfUwTcArgs p) {
    using SM = Smem<BN>;
    static_assert(BN % CP == 0, "column groups must not straddle a tile");
    extern __shared__ unsigned char raw[];
    SM sm(raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tmem = cta_setup<BN>(sm, warp);
    const int64_t ntiles = (p.n + BM - 1) / BM;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int ph = 0; ph < p.nphase && ok; ++ph) {
                    const MfPhase P = p.phases[ph];
                    const bool fl = (P.m & kMfFlip) != 0;
                    const int m = P.m & (kMfFlip - 1);
                    const CUtensorMap* map = fl ? &mA : &mZ;
                    const int z0 = fl ? p.aoff[m] : p.zoff[m];
                    for (int kt = 0; kt < P.nk; ++kt, ++it) {
                        const uint32_t s = it % S_U;
                        if (!mbar_wait(&sm.uempty[s], ((it / S_U) & 1) ^ 1)) { ok = false; break; }
                        mbar_expect_tx(&sm.ufull[s], SM::UBYTES);
                        unsigned char* dst = sm.U + s * SM::UBYTES;
                        tma_load_2d(dst, map, z0 + kt * BK, (int)(tile * BM), &sm.ufull[s]);
                        tma_load_2d(dst + SM::UBYTES / 2, map, z0 + kt * BK + KH, (int)(tile * BM), &sm.ufull[s]);
                    }
                }
            }
            if (!producer_drain(sm.ufull, S_U, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 10) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
                for (int ph = 0; ph < p.nphase && ok; ++ph) {
                    const MfPhase P = p.phases[ph];
                    for (int kt = 0; kt < P.nk && ok; ++kt, ++it) ok = load_b<BN>(sm, it, &mW, &mWlo, kt * BK, P.y0);
                }
            if (!producer_drain(sm.bfull, SM::SB, it)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 1) {
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x)
            for (int ph = 0; ph < p.nphase && ok; ++ph) {
                const int nk = p.phases[ph].nk;
                for (int kt = 0; kt < nk && ok; ++kt, ++it) ok = mma_step<BN>(sm, tmem, it, lane);
            }
        mma_drain(sm, ok, p.err);
    } else if (warp < 6) {
        const int q = warp & 3, m = 32 * q + lane;
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int ph = 0; ph < p.nphase && ok; ++ph) {
                const int nk = p.phases[ph].nk;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    if (!convert_wait<BN>(sm, it)) { ok = false; break; }
                    const unsigned char* R = sm.U + (it % S_U) * SM::UBYTES + m * 128;
                    float x[64];
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 v = *reinterpret_cast<const float4*>(R + h * (SM::UBYTES / 2) + ((j ^ (m & 7)) << 4));
                            x[32 * h + 4 * j + 0] = v.x; x[32 * h + 4 * j + 1] = v.y;
                            x[32 * h + 4 * j + 2] = v.z; x[32 * h + 4 * j + 3] = v.w;
                        }
                    convert_release<BN>(sm, it, lane);
                    convert_publish<BN>(sm, tmem, it, q, lane, x);
                }
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            const int64_t row = tile * BM + 32 * q + lane;
            const bool rv = row < p.n;
            float y[CP];
#pragma unroll
            for (int j = 0; j < CP; ++j) y[j] = 0.f;
            for (int ph = 0; ph < p.nphase && ok; ++ph) {
                const MfPhase P = p.phases[ph];
                float acc[BN];
#pragma unroll
                for (int j = 0; j < BN; ++j) acc[j] = 0.f;
                for (int kt = 0; kt < P.nk && ok; ++kt, ++it) ok = promote_lean<BN>(sm, tmem, it, q, lane, acc);
                if (!ok) break;
                // contraction of the phase with its other factor: A0F (q = q0 + g) or, transposed, Z
                // (j = q0 + g)
                const bool fl = (P.m & kMfFlip) != 0;
                const int m = P.m & (kMfFlip - 1), q0 = P.n0 / CP;
                const float* fsrc = fl ? p.Z : p.A0F;
                const int64_t fld = fl ? (int64_t)p.ldZ : (int64_t)p.ldA;
                const int ao = fl ? p.zoff[m] : p.aoff[m], nq = fl ? p.zcnt[m] : p.acnt[m];
                // the BN / CP values of the point in one aligned load (blocks start on 16-byte
                // boundaries, q0 is a multiple of BN / CP), masked past the block
                constexpr int NG = BN / CP;
                float fv[NG];
                const float* fp = fsrc + row * fld + ao + q0;
                if constexpr (NG == 4) {
                    const float4 t = rv ? __ldg(reinterpret_cast<const float4*>(fp)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    fv[0] = t.x; fv[1] = t.y; fv[2] = t.z; fv[3] = t.w;
                } else if constexpr (NG == 2) {
                    const float2 t = rv ? __ldg(reinterpret_cast<const float2*>(fp)) : make_float2(0.f, 0.f);
                    fv[0] = t.x; fv[1] = t.y;
                } else {
                    fv[0] = rv ? __ldg(fp) : 0.f;
                }
#pragma unroll
                for (int g = 0; g < NG; ++g) {
                    const float f = q0 + g < nq ? fv[g] : 0.f;
#pragma unroll
                    for (int j = 0; j < CP; ++j) y[j] += f * acc[g * CP + j];
                }
            }
            if (!ok) break;
            if (rv) {
#pragma unroll
                for (int j = 0; j < CP; ++j)
                    if (j < p.c) p.Y[row + (int64_t)j * p.ldy] = y[j];
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    }
    cta_teardown<BN>(tmem, warp);
}

// B operand of k_tc_mf_uw: for phase p (rows y0 .. y0 + BN of hi / lo) and K index kk (a tail j),
// hi + lo = W[(wcol[aoff_m + q] + kk) c + cc] with (q, cc) = ((n0 + row) / CP, (n0 + row) mod CP),
// zero where q >= acnt_m, cc >= c or kk >= zcnt_m; for a transposed phase K runs over the pairs
// (kk = q) and the row is (j, cc): W[(wcol[aoff_m + kk] + j) c + cc].  Row-major [nphase BN][kpad].
__global__ void k_prep_mf_w(const float* __restrict__ W, int c, int cp, const MfPhase* __restrict__ phases, int nphase,
                            int bn, int64_t kpad, const int* __restrict__ zcnt, const int* __restrict__ aoff,
                            const int* __restrict__ acnt, const int64_t* __restrict__ wcol, float* __restrict__ hi,
                            float* __restrict__ lo) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nphase * bn * kpad) return;
    const int64_t rowg = idx / kpad, kk = idx % kpad;
    const MfPhase P = phases[rowg / bn];
    const int m = P.m & (kMfFlip - 1);
    const int nidx = P.n0 + (int)(rowg % bn), q = nidx / cp, cc = nidx % cp;
    float v = 0.f;
    if ((P.m & kMfFlip) != 0) {
        if (q < zcnt[m] && cc < c && kk < acnt[m]) v = W[(wcol[aoff[m] + kk] + q) * c + cc];
    } else {
        if (q < acnt[m] && cc < c && kk < zcnt[m]) v = W[(wcol[aoff[m] + q] + kk) * c + cc];
    }
    const float h = tf32_hi(v);
    hi[idx] = h;
    lo[idx] = v - h;
}

// Wt_hi[j * kpad + a] + Wt_lo[j * kpad + a] = W[a * c + j] (TF32 split, zero padding to kpad x bn).
__global__ void k_prep_wt(const float* __restrict__ W, int64_t r, int c, int bn, int64_t kpad, float* __restrict__ hi,
                          float* __restrict__ lo) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)bn * kpad) return;
    const int64_t j = idx / kpad, a = idx % kpad;
    const float v = (a < r && j < c) ? W[a * c + j] : 0.f;
    const float h = tf32_hi(v);
    hi[idx] = h;
    lo[idx] = v - h;
}

// Vhi[i + j * ldo] + Vlo[i + j * ldo] = V[i + j * ldv] (TF32 split; i < n, j < c).
__global__ void k_prep_v(const float* __restrict__ V, int64_t ldv, int64_t n, int c, int64_t ldo,
                         float* __restrict__ hi, float* __restrict__ lo) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)c * ldo) return;
    const int64_t j = idx / ldo, i = idx % ldo;
    const float v = (i < n) ? V[i + j * ldv] : 0.f;
    const float h = tf32_hi(v);
    hi[idx] = h;
    lo[idx] = v - h;
}

// Gram G = U^T U on the tensor cores, 64 columns at a time: the column block U[:, j0 : j0 + 64)
// is transposed through shared memory into the column-major TF32 hi / lo arrays that the U^T V
// kernel takes as its V operand.  hi[j ldo + i] + lo[j ldo + i] = U[i, j0 + j] (zero outside).
__global__ void __launch_bounds__(256) k_prep_ucols(const float* __restrict__ U, int64_t ldU, int64_t n,
                                                    int64_t r, int64_t j0, int64_t ldo, float* __restrict__ hi,
                                                    float* __restrict__ lo) {
    __shared__ float t[64][65];
    const int64_t i0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {        // rows i0 + e / 64, columns j0 + e % 64
        const int ii = e / 64, jj = e % 64;
        const int64_t i = i0 + ii, j = j0 + jj;
        t[ii][jj] = (i < n && j < r) ? U[i * ldU + j] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {        // columns e / 64, rows i0 + e % 64
        const int jj = e / 64, ii = e % 64;
        const int64_t i = i0 + ii;
        if (i >= ldo) continue;
        const float v = t[ii][jj];
        const float h = tf32_hi(v);
        hi[(int64_t)jj * ldo + i] = h;
        lo[(int64_t)jj * ldo + i] = v - h;
    }
}

// G[a * ldg + j0 + j] = sum over the row chunks of part[(chunk * 64 + j) * r + a], a < r, j0 + j < r.
__global__ void k_reduce_gram(const double* __restrict__ part, int nchunk, int64_t r, int64_t j0,
                              double* __restrict__ G, int64_t ldg) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= r * 64) return;
    const int64_t a = idx / 64;
    const int j = (int)(idx % 64);
    if (j0 + j >= r) return;
    double s = 0.0;
    for (int b = 0; b < nchunk; ++b) s += part[((int64_t)b * 64 + j) * r + a];
    G[a * ldg + j0 + j] = s;
}

// ------------------------------------------------------------------------- host side
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeFn encode_fn() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}

// 2-D FP32 tensor map: inner dimension `inner` (contiguous), outer `outer` with row stride
// `stride_bytes`; box {box_inner, box_outer}; zero fill out of bounds.
static bool make_map(CUtensorMap* m, const void* ptr, uint64_t inner, uint64_t outer, uint64_t stride_bytes,
                     uint32_t box_inner, uint32_t box_outer, bool swizzle128) {
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {stride_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int num_sms() {
    int dv = 0, nsm = 0;
    cudaGetDevice(&dv);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv);
    return std::max(nsm, 1);
}

template <int BN>
static hdf_status uw_bn(const float* U, int64_t ldU, int64_t n, int64_t r, const float* W, int c, float alpha,
                        const float* B, int64_t ldb, float beta, float* Y, int64_t ldy, float* work, int* err,
                        cudaStream_t st) {
    const int64_t kpad = ((r + BK - 1) / BK) * BK;
    float* hi = work;
    float* lo = work + (size_t)BN * kpad;
    HDF_COUNT_LAUNCH();
    k_prep_wt<<<(unsigned)(((int64_t)BN * kpad + 255) / 256), 256, 0, st>>>(W, r, c, BN, kpad, hi, lo);
    HDF_CUDA(cudaGetLastError());
    CUtensorMap mU, mW, mWl;
    if (!make_map(&mU, U, (uint64_t)ldU, (uint64_t)n, (uint64_t)ldU * 4, KH, BM, true) ||     // SW128 halves
        !make_map(&mW, hi, (uint64_t)kpad, BN, (uint64_t)kpad * 4, KH, BN, true) ||
        !make_map(&mWl, lo, (uint64_t)kpad, BN, (uint64_t)kpad * 4, KH, BN, true))
        return fail(HDF_ECUDA, "tensor-core matvec: cannot encode a tensor map");
    UwArgs a{n, (int)(kpad / BK), c, alpha, beta, B, ldb, Y, ldy, err};
    const size_t sm = Smem<BN>::bytes();
    HDF_CUDA(cudaFuncSetAttribute(k_tc_uw<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t ntiles = (n + BM - 1) / BM;
    const int grid = (int)std::min<int64_t>(ntiles, num_sms());
    HDF_COUNT_LAUNCH();
    k_tc_uw<BN><<<grid, NTHREADS, sm, st>>>(mU, mW, mWl, a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

template <int BN>
static hdf_status utv_bn(const float* U, int64_t ldU, int64_t n, int64_t r, const float* V, int64_t ldv, int c,
                         int64_t chunk, double* part, float* work, int* err, cudaStream_t st, bool part32 = false) {
    const int64_t ldo = ((n + 3) / 4) * 4;
    float* vhi = work;
    float* vlo = work + (size_t)c * ldo;
    if (V) {                     // V == nullptr: the caller has written the split into work
        HDF_COUNT_LAUNCH();
        k_prep_v<<<(unsigned)(((int64_t)c * ldo + 255) / 256), 256, 0, st>>>(V, ldv, n, c, ldo, vhi, vlo);
        HDF_CUDA(cudaGetLastError());
    }
    CUtensorMap mU, mV, mVl;
    if (!make_map(&mU, U, (uint64_t)ldU, (uint64_t)n, (uint64_t)ldU * 4, BM, BK, false) ||
        !make_map(&mV, vhi, (uint64_t)n, (uint64_t)c, (uint64_t)ldo * 4, KH, BN, true) ||
        !make_map(&mVl, vlo, (uint64_t)n, (uint64_t)c, (uint64_t)ldo * 4, KH, BN, true))
        return fail(HDF_ECUDA, "tensor-core matvec: cannot encode a tensor map");
    const int nch = (int)((n + chunk - 1) / chunk);
    int* next = reinterpret_cast<int*>(vlo + (size_t)c * ldo);      // one int past the split V
    HDF_CUDA(cudaMemsetAsync(next, 0, sizeof(int), st));
    UtvArgs a{r, n, chunk, nch, (int)((r + BM - 1) / BM), c, part, part32 ? reinterpret_cast<float*>(part) : nullptr,
              err, next};
    const size_t sm = Smem<BN>::bytes();
    HDF_CUDA(cudaFuncSetAttribute(k_tc_utv<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t nitems = (int64_t)a.mblocks * nch;
    const int grid = (int)std::min<int64_t>(nitems, num_sms());
    HDF_COUNT_LAUNCH();
    k_tc_utv<BN><<<grid, NTHREADS, sm, st>>>(mU, mV, mVl, a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

}  // namespace tc

bool encode_map_f32(CUtensorMap_st* map, const void* ptr, uint64_t inner, uint64_t outer, uint64_t stride_bytes,
                    uint32_t box_inner, uint32_t box_outer, bool swizzle128) {
    return tc::make_map(map, ptr, inner, outer, stride_bytes, box_inner, box_outer, swizzle128);
}

// Column count padded for the tensor-core path (16, 32 or 64); 0 if not eligible.
int tc_bn(int c) { return c <= 16 ? 16 : c <= 32 ? 32 : c <= 64 ? 64 : 0; }

size_t tc_work_floats(int64_t n, int64_t r, int c) {
    const int bn = tc_bn(c);
    const int64_t kpad = ((r + tc::BK - 1) / tc::BK) * tc::BK;
    const int64_t ldo = ((n + 3) / 4) * 4;
    return std::max<size_t>(2 * (size_t)bn * kpad, 2 * (size_t)c * ldo + 4);   // + the U^T V item counter
}

// Rows-per-chunk split for U^T V on the tensor cores: enough (column block, chunk) items.
void tc_utv_split(int64_t n, int64_t r, int64_t* chunk, int* nchunk) {
    // at least enough (column block, chunk) items to fill the GPU a few times, and chunks of at
    // most 8192 rows so that the FP32 register sums of the promoted steps stay short; chunks
    // are whole multiples of 64 rows (one K step), and *nchunk is the number of chunks that
    // really exist
    const int64_t mblocks = (r + tc::BM - 1) / tc::BM;
    const int64_t want = (4 * 152 + mblocks - 1) / mblocks;
    const int64_t by_len = (n + 8191) / 8192;
    const int64_t by_rows = std::max<int64_t>(1, n / (4 * tc::BK));
    const int64_t req = std::max<int64_t>(1, std::min<int64_t>(std::max(want, by_len), by_rows));
    const int64_t ch = (((n + req - 1) / req + tc::BK - 1) / tc::BK) * tc::BK;
    *chunk = ch;
    *nchunk = (int)((n + ch - 1) / ch);
}

hdf_status tc_utv(const float* U, int64_t ldU, int64_t n, int64_t r, const float* V, int64_t ldv, int c, int64_t chunk,
                  double* part, float* work, int* err, cudaStream_t st, bool part32) {
    switch (tc_bn(c)) {
        case 16: return tc::utv_bn<16>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st, part32);
        case 32: return tc::utv_bn<32>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st, part32);
        case 64: return tc::utv_bn<64>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st, part32);
    }
    return fail(HDF_EINVAL, "tc_utv: column count");
}

// G = U^T U (r x r, FP64, row-major) on the tensor cores (3xTF32 products, FP32 sums per row
// chunk, FP64 across chunks).  Work space from the stream-ordered pool.
hdf_status tc_gram(const float* U, int64_t ldU, int64_t n, int64_t r, double* G, int* err, cudaStream_t st) {
    int64_t chunk = 0;
    int nch = 0;
    tc_utv_split(n, r, &chunk, &nch);
    const int64_t ldo = ((n + 3) / 4) * 4;
    DevBuf work, part;
    HDF_CUDA(work.alloc_on(sizeof(float) * (2 * (size_t)64 * ldo + 4), st));
    HDF_CUDA(part.alloc_on(sizeof(double) * (size_t)nch * 64 * r, st));
    float* hi = work.as<float>();
    float* lo = hi + (size_t)64 * ldo;
    for (int64_t j0 = 0; j0 < r; j0 += 64) {
        HDF_COUNT_LAUNCH();
        tc::k_prep_ucols<<<(unsigned)((ldo + 63) / 64), 256, 0, st>>>(U, ldU, n, r, j0, ldo, hi, lo);
        HDF_CUDA(cudaGetLastError());
        hdf_status s = tc::utv_bn<64>(U, ldU, n, r, nullptr, 0, 64, chunk, part.as<double>(), work.as<float>(), err, st);
        if (s != HDF_OK) return s;
        HDF_COUNT_LAUNCH();
        tc::k_reduce_gram<<<(unsigned)((r * 64 + 255) / 256), 256, 0, st>>>(part.as<double>(), nch, r, j0, G, r);
        HDF_CUDA(cudaGetLastError());
    }
    return HDF_OK;
}

// Work-wait limit of the current device in clock cycles (<= 0: the default, about 2 s).
hdf_status set_wait_limit(long long cycles, long long* previous) {
    long long prev = 0;
    HDF_CUDA(cudaMemcpyFromSymbol(&prev, tc::d_wait_cycles, sizeof(prev)));
    const long long v = cycles > 0 ? cycles : tc::kDefaultWaitCycles;
    HDF_CUDA(cudaMemcpyToSymbol(tc::d_wait_cycles, &v, sizeof(v)));
    if (previous) *previous = prev;
    return HDF_OK;
}

namespace tc {
// Every FP32 bit pattern with a finite value: tf32_hi against the conversion instruction.
// bad[0] counts mismatches below 2^127 in magnitude, bad[1] those in the top binade (where
// rounding up overflows).
__global__ void k_tf32_check(unsigned long long* bad) {
    unsigned long long low = 0, top = 0;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < (1ull << 32); u += step) {
        const uint32_t b = (uint32_t)u;
        const uint32_t e = b & 0x7F800000u;
        if (e == 0x7F800000u) continue;
        const float x = __uint_as_float(b);
        uint32_t ref;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(ref) : "f"(x));
        if (__float_as_uint(tf32_hi(x)) != ref) {
            if (e == 0x7F000000u) ++top; else ++low;
        }
    }
    if (low) atomicAdd(&bad[0], low);
    if (top) atomicAdd(&bad[1], top);
}
}  // namespace tc

hdf_status tf32_check(unsigned long long* bad2) {
    DevBuf b;
    HDF_CUDA(b.alloc(2 * sizeof(unsigned long long)));
    HDF_CUDA(cudaMemset(b.p, 0, 2 * sizeof(unsigned long long)));
    HDF_COUNT_LAUNCH();
    tc::k_tf32_check<<<tc::num_sms() * 4, 256>>>(b.as<unsigned long long>());
    HDF_CUDA(cudaGetLastError());
    HDF_CUDA(cudaMemcpy(bad2, b.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    return HDF_OK;
}

// ---------------------------------------------------------- matrix-free products (host)
int tc_mf_cp(int c) { return c <= 16 ? 16 : c <= 32 ? 32 : 64; }

void tc_mf_lists(const std::vector<int>& zcnt, const std::vector<int>& acnt, int c, std::vector<int4>& tiles,
                 std::vector<int4>& phases, int* kpad) {
    tiles.clear();
    phases.clear();
    const int cp = tc_mf_cp(c);
    int kmax = tc::BK;
    for (size_t m = 0; m < zcnt.size(); ++m) {
        const int J = zcnt[m], Np = acnt[m] * cp, Nt = J * cp;
        if (J == 0 || acnt[m] == 0) continue;
        // U^T V tiles of degree m in the orientation with fewer tiles: rows = tails j, columns
        // (q, cc) (flag 0), or rows = the (k, s) pairs q of A0F, columns (j, cc) (flag 1; few
        // tails and many pairs, the small degrees)
        const int64_t n_rows_j = (int64_t)((J + tc::BM - 1) / tc::BM) * ((Np + 63) / 64);
        const int64_t n_rows_q = (int64_t)((acnt[m] + tc::BM - 1) / tc::BM) * ((Nt + 63) / 64);
        if (n_rows_q < n_rows_j) {
            for (int q0 = 0; q0 < acnt[m]; q0 += tc::BM)
                for (int n0 = 0; n0 < Nt; n0 += 64) tiles.push_back(make_int4((int)m, q0, n0, 1));
        } else {
            for (int j0 = 0; j0 < J; j0 += tc::BM)
                for (int n0 = 0; n0 < Np; n0 += 64) tiles.push_back(make_int4((int)m, j0, n0, 0));
        }
        // U W phases of degree m in the orientation with fewer K steps: K = the tails, columns
        // (q, cc), or (flagged) K = the pairs q, columns (j, cc)
        const int nk = (J + tc::BK - 1) / tc::BK, nkq = (acnt[m] + tc::BK - 1) / tc::BK;
        const int64_t steps_j = (int64_t)((Np + 63) / 64) * nk, steps_q = (int64_t)((Nt + 63) / 64) * nkq;
        if (steps_q < steps_j) {
            kmax = std::max(kmax, nkq * tc::BK);
            for (int n0 = 0; n0 < Nt; n0 += 64)
                phases.push_back(make_int4((int)m | tc::kMfFlip, n0, nkq, (int)phases.size() * 64));
        } else {
            kmax = std::max(kmax, nk * tc::BK);
            for (int n0 = 0; n0 < Np; n0 += 64)
                phases.push_back(make_int4((int)m, n0, nk, (int)phases.size() * 64));
        }
    }
    *kpad = kmax;
}

void tc_mf_chunks(int64_t n, int ntiles, int64_t* chunk, int* nchunk) {
    // chunks of at most 8192 points (short FP32 sums), enough items to fill the GPU a few times
    const int64_t want = (4 * 152 + std::max(ntiles, 1) - 1) / std::max(ntiles, 1);
    const int64_t by_len = (n + 8191) / 8192;
    const int64_t req = std::max<int64_t>(1, std::max(want, by_len));
    const int64_t ch = std::max<int64_t>(tc::BK, (((n + req - 1) / req + tc::BK - 1) / tc::BK) * tc::BK);
    *chunk = ch;
    *nchunk = (int)((n + ch - 1) / ch);
}

hdf_status tc_mf_utv(const MfTcView& v, const int4* tiles, int ntiles, const float* V, int64_t ldv, int c, double* part,
                     int* nchunk, int* err, cudaStream_t st) {
    int64_t chunk = 0;
    int nch = 0;
    tc_mf_chunks(v.n, ntiles, &chunk, &nch);
    *nchunk = nch;
    HDF_CUDA(cudaMemsetAsync(part, 0, sizeof(double) * (size_t)nch * c * v.r, st));
    if (ntiles == 0) return HDF_OK;
    CUtensorMap mZ, mA;
    if (!tc::make_map(&mZ, v.Z, (uint64_t)v.ldZ, (uint64_t)v.n, (uint64_t)v.ldZ * 4, tc::BM, tc::BK, false) ||
        !tc::make_map(&mA, v.A0F, (uint64_t)v.ldA, (uint64_t)v.n, (uint64_t)v.ldA * 4, tc::BM, tc::BK, false))
        return fail(HDF_ECUDA, "matrix-free product: cannot encode a tensor map");
    DevBuf next;
    HDF_CUDA(next.alloc_on(sizeof(int), st));
    HDF_CUDA(cudaMemsetAsync(next.p, 0, sizeof(int), st));
    tc::MfUtvTcArgs a{v.n, chunk, nch, ntiles, tiles, v.A0F, v.ldA, v.Z, v.ldZ, V, ldv, c,
                      v.zoff, v.zcnt, v.aoff, v.acnt, v.wcol, part, v.r, err, next.as<int>()};
    const size_t sm = tc::Smem<64>::bytes();
    const int64_t nitems = (int64_t)ntiles * nch;
    const int grid = (int)std::min<int64_t>(nitems, tc::num_sms());
    auto kern = c <= 16 ? tc::k_tc_mf_utv<64, 16> : c <= 32 ? tc::k_tc_mf_utv<64, 32> : tc::k_tc_mf_utv<64, 64>;
    HDF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HDF_COUNT_LAUNCH();
    kern<<<grid, tc::NTHREADS_MF, sm, st>>>(mZ, mA, a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

template <int CP>
static hdf_status mf_uw_cp(const MfTcView& v, const tc::MfPhase* phases, int nphase, int kpad, const float* hi,
                           const float* lo, int c, float* Y, int64_t ldy, int* err, cudaStream_t st) {
    CUtensorMap mZ, mA, mW, mWl;
    if (!tc::make_map(&mZ, v.Z, (uint64_t)v.ldZ, (uint64_t)v.n, (uint64_t)v.ldZ * 4, tc::KH, tc::BM, true) ||
        !tc::make_map(&mA, v.A0F, (uint64_t)v.ldA, (uint64_t)v.n, (uint64_t)v.ldA * 4, tc::KH, tc::BM, true) ||
        !tc::make_map(&mW, hi, (uint64_t)kpad, (uint64_t)nphase * 64, (uint64_t)kpad * 4, tc::KH, 64, true) ||
        !tc::make_map(&mWl, lo, (uint64_t)kpad, (uint64_t)nphase * 64, (uint64_t)kpad * 4, tc::KH, 64, true))
        return fail(HDF_ECUDA, "matrix-free product: cannot encode a tensor map");
    tc::MfUwTcArgs a{v.n, nphase, phases, v.zoff, v.aoff, v.acnt, v.zcnt, v.A0F, v.ldA, v.Z, v.ldZ, c, Y, ldy, err};
    const size_t sm = tc::Smem<64>::bytes();
    HDF_CUDA(cudaFuncSetAttribute(tc::k_tc_mf_uw<64, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t ntiles = (v.n + tc::BM - 1) / tc::BM;
    const int grid = (int)std::min<int64_t>(ntiles, tc::num_sms());
    HDF_COUNT_LAUNCH();
    tc::k_tc_mf_uw<64, CP><<<grid, tc::NTHREADS, sm, st>>>(mZ, mA, mW, mWl, a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

hdf_status tc_mf_uw(const MfTcView& v, const int4* phases, int nphase, int kpad, const float* W, int c, float* Y,
                    int64_t ldy, int* err, cudaStream_t st) {
    if (nphase == 0) {
        for (int j = 0; j < c; ++j) HDF_CUDA(cudaMemsetAsync(Y + j * ldy, 0, sizeof(float) * v.n, st));
        return HDF_OK;
    }
    const int cp = tc_mf_cp(c);
    DevBuf work;
    const size_t per = (size_t)nphase * 64 * kpad;
    HDF_CUDA(work.alloc_on(sizeof(float) * 2 * per, st));
    float* hi = work.as<float>();
    float* lo = hi + per;
    const tc::MfPhase* ph = reinterpret_cast<const tc::MfPhase*>(phases);
    HDF_COUNT_LAUNCH();
    tc::k_prep_mf_w<<<(unsigned)((per + 255) / 256), 256, 0, st>>>(W, c, cp, ph, nphase, 64, kpad, v.zcnt, v.aoff,
                                                                   v.acnt, v.wcol, hi, lo);
    HDF_CUDA(cudaGetLastError());
    switch (cp) {
        case 16: return mf_uw_cp<16>(v, ph, nphase, kpad, hi, lo, c, Y, ldy, err, st);
        case 32: return mf_uw_cp<32>(v, ph, nphase, kpad, hi, lo, c, Y, ldy, err, st);
        default: return mf_uw_cp<64>(v, ph, nphase, kpad, hi, lo, c, Y, ldy, err, st);
    }
}

hdf_status tc_uw(const float* U, int64_t ldU, int64_t n, int64_t r, const float* W, int c, float alpha, const float* B,
                 int64_t ldb, float beta, float* Y, int64_t ldy, float* work, int* err, cudaStream_t st) {
    switch (tc_bn(c)) {
        case 16: return tc::uw_bn<16>(U, ldU, n, r, W, c, alpha, B, ldb, beta, Y, ldy, work, err, st);
        case 32: return tc::uw_bn<32>(U, ldU, n, r, W, c, alpha, B, ldb, beta, Y, ldy, work, err, st);
        case 64: return tc::uw_bn<64>(U, ldU, n, r, W, c, alpha, B, ldb, beta, Y, ldy, work, err, st);
    }
    return fail(HDF_EINVAL, "tc_uw: column count");
}

}  // namespace hdf
