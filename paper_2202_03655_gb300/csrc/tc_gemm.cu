// Tensor-core GEMMs of the factored matvec K~V = U (S (U^T V)) for FP32 factors (sm_103a):
// tcgen05.mma (kind::tf32, accumulators in TMEM), operand tiles staged by TMA
// (cp.async.bulk.tensor) through an mbarrier pipeline, warp-specialised CTAs.
//
// Accuracy: one TF32 product keeps about 11 bits, far from what tol = 1e-6 needs, so every
// product is split three ways, A B ~= A_hi B_hi + A_hi B_lo + A_lo B_hi, with
// A_hi = A rounded to TF32 (cvt.rna.tf32.f32, exactly representable) and A_lo = A - A_hi.
// The high and low parts of the U tiles are formed in shared memory by converter warps, those
// of W and V by small preparation kernels.  The dropped A_lo B_lo term is ~2^-22 relative.
//
//   k_tc_uw  : Y = alpha U W + beta B.  M = 128 rows of U (points), N = BN >= c, K = rank.
//              A = U tile (K-major, SW128, TMA), B = W^T tile (K-major, SW128, TMA).
//   k_tc_utv : partial W = U^T V over a chunk of rows.  M = 128 columns of U, N = BN, K = rows.
//              U tiles are loaded as stored (row-major, M contiguous) and transposed by the
//              converter warps into K-major SW128 tiles (hi and lo), so only K-major operand
//              layouts reach the MMA.  B = V tiles (column-major V is K-major), SW128, TMA.
//
// The tensor core's FP32 accumulation is not rounded to nearest, and its error grows with
// the number of MMAs summed into one accumulator (about 1.7e-5 relative after 400 K steps).
// So each stage (32 K values, 12 MMAs) starts a fresh TMEM accumulator and the epilogue warps
// add it into FP32 registers (round to nearest); four TMEM buffers rotate so that the MMAs of
// the next stages run while earlier stages are promoted.
//
// CTA roles (10 warps): warp 0 TMA producer, warp 1 MMA issuer and TMEM owner, warps 2-5
// converters, warps 6-9 promotion and epilogue (TMEM -> registers -> global; warp w reads TMEM
// lanes 32 (w mod 4) .. +31).  Every wait on an mbarrier is bounded by a clock limit; on
// expiry the kernel records an error, drains its own copies and MMAs, frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "internal.h"

namespace hdf {
namespace tc {

constexpr int BM = 128;                 // MMA M
constexpr int BK = 32;                  // K elements per stage: one 128-byte swizzle row of FP32
constexpr int UW_STAGES = 4;
constexpr int UTV_STAGES = 3;
constexpr int NTHREADS = 320;
constexpr int NACC = 4;                 // TMEM accumulator buffers (one per stage in flight)
constexpr long long kWaitCycles = 4000000000ll;   // about 2 s at 2 GHz

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
// Waits for the completion of the phase with the given parity; false if the clock limit passes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
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

// Instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = BN.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_tf32() {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    return __uint_as_float(h);
}

template <int BN>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return (NACC * BN <= 32) ? 32 : (NACC * BN <= 64) ? 64 : (NACC * BN <= 128) ? 128 : (NACC * BN <= 256) ? 256 : 512;
}

struct UwArgs {
    int64_t n;          // rows of U
    int nkt;            // K steps (ceil(rank / 32))
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
    constexpr int S = UW_STAGES;
    constexpr uint32_t ABYTES = BM * BK * 4, BBYTES = BN * BK * 4;
    extern __shared__ unsigned char raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    float* A = reinterpret_cast<float*>(base);
    float* Alo = A + S * BM * BK;
    float* Bh = Alo + S * BM * BK;
    float* Bl = Bh + S * BN * BK;
    uint64_t* full = reinterpret_cast<uint64_t*>(Bl + S * BN * BK);
    uint64_t* lo = full + S;
    uint64_t* empty = lo + S;
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + NACC;
    uint64_t* drain = acce + NACC;
    uint32_t* slot = reinterpret_cast<uint32_t*>(drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&lo[s], 4); mbar_init(&empty[s], 1); }
        for (int b = 0; b < NACC; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], 4); }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(tmem_cols<BN>()));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const int64_t ntiles = (p.n + BM - 1) / BM;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int kt = 0; kt < p.nkt && ok; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&full[s], ABYTES + 2 * BBYTES);
                    tma_load_2d(A + s * BM * BK, &mU, kt * BK, (int)(tile * BM), &full[s]);
                    tma_load_2d(Bh + s * BN * BK, &mW, kt * BK, 0, &full[s]);
                    tma_load_2d(Bl + s * BN * BK, &mWlo, kt * BK, 0, &full[s]);
                }
            }
            // drain: every copy this thread issued has landed before the CTA leaves
            for (uint32_t q = (it > (uint32_t)S ? it - S : 0); q < it; ++q) {
                const int s = q % S;
                if (!mbar_wait(&full[s], (q / S) & 1)) ok = false;
            }
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32<BN>();
            uint32_t it = 0;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
                for (int kt = 0; kt < p.nkt; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1, buf = it % NACC, aph = (it / NACC) & 1;
                    if (!mbar_wait(&acce[buf], aph ^ 1)) { ok = false; break; }
                    if (!mbar_wait(&full[s], ph) || !mbar_wait(&lo[s], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + buf * BN;
                    const uint64_t da = sw128_desc(A + s * BM * BK), dal = sw128_desc(Alo + s * BM * BK);
                    const uint64_t db = sw128_desc(Bh + s * BN * BK), dbl = sw128_desc(Bl + s * BN * BK);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 32) >> 4;     // 8 TF32 = 32 bytes
                        mma_tf32(d, da + off, db + off, idesc, kk > 0 ? 1u : 0u);
                        mma_tf32(d, da + off, dbl + off, idesc, 1u);
                        mma_tf32(d, dal + off, db + off, idesc, 1u);
                    }
                    mma_commit(&empty[s]);
                    mma_commit(&accf[buf]);
                }
            }
            mma_commit(drain);                       // all MMAs of this thread complete
            if (!mbar_wait(drain, 0)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp < 6) {
        const int cw = warp - 2;                     // converter 0..3: a quarter of each A tile
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            for (int kt = 0; kt < p.nkt; ++kt, ++it) {
                const int s = it % S;
                const uint32_t ph = (it / S) & 1;
                if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                float4* hi4 = reinterpret_cast<float4*>(A + s * BM * BK) + cw * (BM * BK / 16);
                float4* lo4 = reinterpret_cast<float4*>(Alo + s * BM * BK) + cw * (BM * BK / 16);
#pragma unroll
                for (int q = 0; q < BM * BK / 16 / 32; ++q) {
                    const float4 v = hi4[q * 32 + lane];
                    float4 h, l;
                    h.x = tf32_hi(v.x); h.y = tf32_hi(v.y); h.z = tf32_hi(v.z); h.w = tf32_hi(v.w);
                    l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
                    hi4[q * 32 + lane] = h;
                    lo4[q * 32 + lane] = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&lo[s]);
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;                      // TMEM lane quadrant of this warp
        uint32_t it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            for (int kt = 0; kt < p.nkt; ++kt, ++it) {
                const uint32_t buf = it % NACC, aph = (it / NACC) & 1;
                if (!mbar_wait(&accf[buf], aph)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int j0 = 0; j0 < BN; j0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + buf * BN + j0, v);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) acc[j0 + jj] += v[jj];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[buf]);
            }
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
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols<BN>()));
    }
}

struct UtvArgs {
    int64_t r;          // columns of U (M extent)
    int64_t n;          // rows of U
    int64_t chunk;      // rows per K chunk
    int nchunk;
    int mblocks;        // ceil(r / 128)
    int c;
    double* part;       // part[(chunk * c + j) * r + a]
    int* err;
};

// Partial U^T V: items (column block of U, chunk of rows), persistent over items.
template <int BN>
__global__ void __launch_bounds__(NTHREADS, 1)
    k_tc_utv(const __grid_constant__ CUtensorMap mU, const __grid_constant__ CUtensorMap mV,
             const __grid_constant__ CUtensorMap mVlo, UtvArgs p) {
    constexpr int S = UTV_STAGES;
    constexpr uint32_t RAWBYTES = BM * BK * 4, BBYTES = BN * BK * 4;
    extern __shared__ unsigned char raw_[];
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(raw_) + 1023) & ~uintptr_t(1023));
    float* Raw = reinterpret_cast<float*>(base);          // S x [BK rows][BM cols] as stored
    float* Ah = Raw + S * BM * BK;                        // S x K-major SW128 hi
    float* Al = Ah + S * BM * BK;                         // S x K-major SW128 lo
    float* Bh = Al + S * BM * BK;
    float* Bl = Bh + S * BN * BK;
    uint64_t* full = reinterpret_cast<uint64_t*>(Bl + S * BN * BK);
    uint64_t* lo = full + S;
    uint64_t* empty = lo + S;
    uint64_t* accf = empty + S;
    uint64_t* acce = accf + NACC;
    uint64_t* drain = acce + NACC;
    uint32_t* slot = reinterpret_cast<uint32_t*>(drain + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&lo[s], 4); mbar_init(&empty[s], 1); }
        for (int b = 0; b < NACC; ++b) { mbar_init(&accf[b], 1); mbar_init(&acce[b], 4); }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(tmem_cols<BN>()));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const int64_t nitems = (int64_t)p.mblocks * p.nchunk;
    bool ok = true;
    auto ksteps = [&](int64_t item) -> int {
        const int64_t ch = item / p.mblocks;
        const int64_t i0 = ch * p.chunk, i1 = min(p.n, i0 + p.chunk);
        return (int)((i1 - i0 + BK - 1) / BK);
    };

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int64_t mb = item % p.mblocks, ch = item / p.mblocks;
                const int64_t i0 = ch * p.chunk;
                const int nk = ksteps(item);
                for (int kt = 0; kt < nk && ok; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1;
                    if (!mbar_wait(&empty[s], ph ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&full[s], RAWBYTES + 2 * BBYTES);
                    const int row = (int)(i0 + (int64_t)kt * BK);
                    tma_load_2d(Raw + s * BM * BK, &mU, (int)(mb * BM), row, &full[s]);
                    tma_load_2d(Bh + s * BN * BK, &mV, row, 0, &full[s]);
                    tma_load_2d(Bl + s * BN * BK, &mVlo, row, 0, &full[s]);
                }
            }
            for (uint32_t q = (it > (uint32_t)S ? it - S : 0); q < it; ++q) {
                const int s = q % S;
                if (!mbar_wait(&full[s], (q / S) & 1)) ok = false;
            }
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32<BN>();
            uint32_t it = 0;
            for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
                const int nk = ksteps(item);
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = it % S;
                    const uint32_t ph = (it / S) & 1, buf = it % NACC, aph = (it / NACC) & 1;
                    if (!mbar_wait(&acce[buf], aph ^ 1)) { ok = false; break; }
                    if (!mbar_wait(&full[s], ph) || !mbar_wait(&lo[s], ph)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + buf * BN;
                    const uint64_t da = sw128_desc(Ah + s * BM * BK), dal = sw128_desc(Al + s * BM * BK);
                    const uint64_t db = sw128_desc(Bh + s * BN * BK), dbl = sw128_desc(Bl + s * BN * BK);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 32) >> 4;
                        mma_tf32(d, da + off, db + off, idesc, kk > 0 ? 1u : 0u);
                        mma_tf32(d, da + off, dbl + off, idesc, 1u);
                        mma_tf32(d, dal + off, db + off, idesc, 1u);
                    }
                    mma_commit(&empty[s]);
                    mma_commit(&accf[buf]);
                }
            }
            mma_commit(drain);
            if (!mbar_wait(drain, 0)) ok = false;
            if (!ok) atomicExch(p.err, 1);
        }
    } else if (warp < 6) {
        // transpose the stored tile Raw[k][m] into K-major SW128 hi / lo tiles:
        // element (m, k) at byte (m/8)*1024 + (m%8)*128 + (((k/4) ^ (m%8)) * 16) + (k%4)*4
        const int cw = warp - 2;
        uint32_t it = 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const int s = it % S;
                const uint32_t ph = (it / S) & 1;
                if (!mbar_wait(&full[s], ph)) { ok = false; break; }
                const float* R = Raw + s * BM * BK;
                unsigned char* H = reinterpret_cast<unsigned char*>(Ah + s * BM * BK);
                unsigned char* Lo = reinterpret_cast<unsigned char*>(Al + s * BM * BK);
                // this warp: rows m in [32 cw, 32 cw + 32), all 8 k-chunks
                const int m = 32 * cw + lane;
#pragma unroll
                for (int kc = 0; kc < BK / 4; ++kc) {
                    float4 h, l;
                    const float x0 = R[(4 * kc + 0) * BM + m], x1 = R[(4 * kc + 1) * BM + m];
                    const float x2 = R[(4 * kc + 2) * BM + m], x3 = R[(4 * kc + 3) * BM + m];
                    h.x = tf32_hi(x0); h.y = tf32_hi(x1); h.z = tf32_hi(x2); h.w = tf32_hi(x3);
                    l.x = x0 - h.x; l.y = x1 - h.y; l.z = x2 - h.z; l.w = x3 - h.w;
                    const uint32_t off = (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((kc ^ (m & 7)) << 4));
                    *reinterpret_cast<float4*>(H + off) = h;
                    *reinterpret_cast<float4*>(Lo + off) = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&lo[s]);
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    } else {
        const int q = warp & 3;
        uint32_t it = 0;
        for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
            float acc[BN];
#pragma unroll
            for (int j = 0; j < BN; ++j) acc[j] = 0.f;
            const int nk = ksteps(item);
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const uint32_t buf = it % NACC, aph = (it / NACC) & 1;
                if (!mbar_wait(&accf[buf], aph)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int j0 = 0; j0 < BN; j0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + buf * BN + j0, v);
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) acc[j0 + jj] += v[jj];
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce[buf]);
            }
            if (!ok) break;
            const int64_t mb = item % p.mblocks, ch = item / p.mblocks;
            const int64_t a = mb * BM + 32 * q + lane;
            if (a < p.r) {
#pragma unroll
                for (int j = 0; j < BN; ++j)
                    if (j < p.c) p.part[((int64_t)ch * p.c + j) * p.r + a] = (double)acc[j];
            }
        }
        if (!ok && lane == 0) atomicExch(p.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols<BN>()));
    }
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

template <int BN>
static size_t uw_smem() {
    return 1024 + (size_t)UW_STAGES * (2 * BM * BK + 2 * BN * BK) * 4 + (3 * UW_STAGES + 2 * NACC + 1) * 8 + 16;
}
template <int BN>
static size_t utv_smem() {
    return 1024 + (size_t)UTV_STAGES * (3 * BM * BK + 2 * BN * BK) * 4 + (3 * UTV_STAGES + 2 * NACC + 1) * 8 + 16;
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
    if (!make_map(&mU, U, (uint64_t)ldU, (uint64_t)n, (uint64_t)ldU * 4, BK, BM, true) ||
        !make_map(&mW, hi, (uint64_t)kpad, BN, (uint64_t)kpad * 4, BK, BN, true) ||
        !make_map(&mWl, lo, (uint64_t)kpad, BN, (uint64_t)kpad * 4, BK, BN, true))
        return fail(HDF_ECUDA, "tensor-core matvec: cannot encode a tensor map");
    UwArgs a{n, (int)(kpad / BK), c, alpha, beta, B, ldb, Y, ldy, err};
    const size_t sm = uw_smem<BN>();
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
                         int64_t chunk, double* part, float* work, int* err, cudaStream_t st) {
    const int64_t ldo = ((n + 3) / 4) * 4;
    float* vhi = work;
    float* vlo = work + (size_t)c * ldo;
    HDF_COUNT_LAUNCH();
    k_prep_v<<<(unsigned)(((int64_t)c * ldo + 255) / 256), 256, 0, st>>>(V, ldv, n, c, ldo, vhi, vlo);
    HDF_CUDA(cudaGetLastError());
    CUtensorMap mU, mV, mVl;
    if (!make_map(&mU, U, (uint64_t)ldU, (uint64_t)n, (uint64_t)ldU * 4, BM, BK, false) ||
        !make_map(&mV, vhi, (uint64_t)n, (uint64_t)c, (uint64_t)ldo * 4, BK, BN, true) ||
        !make_map(&mVl, vlo, (uint64_t)n, (uint64_t)c, (uint64_t)ldo * 4, BK, BN, true))
        return fail(HDF_ECUDA, "tensor-core matvec: cannot encode a tensor map");
    const int nch = (int)((n + chunk - 1) / chunk);
    UtvArgs a{r, n, chunk, nch, (int)((r + BM - 1) / BM), c, part, err};
    const size_t sm = utv_smem<BN>();
    HDF_CUDA(cudaFuncSetAttribute(k_tc_utv<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t nitems = (int64_t)a.mblocks * nch;
    const int grid = (int)std::min<int64_t>(nitems, num_sms());
    HDF_COUNT_LAUNCH();
    k_tc_utv<BN><<<grid, NTHREADS, sm, st>>>(mU, mV, mVl, a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

}  // namespace tc

// Column count padded for the tensor-core path (16, 32 or 64); 0 if not eligible.
int tc_bn(int c) { return c <= 16 ? 16 : c <= 32 ? 32 : c <= 64 ? 64 : 0; }

size_t tc_work_floats(int64_t n, int64_t r, int c) {
    const int bn = tc_bn(c);
    const int64_t kpad = ((r + tc::BK - 1) / tc::BK) * tc::BK;
    const int64_t ldo = ((n + 3) / 4) * 4;
    return std::max<size_t>(2 * (size_t)bn * kpad, 2 * (size_t)c * ldo);
}

// Rows-per-chunk split for U^T V on the tensor cores: enough (column block, chunk) items.
void tc_utv_split(int64_t n, int64_t r, int64_t* chunk, int* nchunk) {
    // at least enough (column block, chunk) items to fill the GPU a few times, and chunks of at
    // most 8192 rows so that the FP32 register sums of the promoted stages stay short; chunks
    // are whole multiples of 32 rows, and *nchunk is the number of chunks that really exist
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
                  double* part, float* work, int* err, cudaStream_t st) {
    switch (tc_bn(c)) {
        case 16: return tc::utv_bn<16>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st);
        case 32: return tc::utv_bn<32>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st);
        case 64: return tc::utv_bn<64>(U, ldU, n, r, V, ldv, c, chunk, part, work, err, st);
    }
    return fail(HDF_EINVAL, "tc_utv: column count");
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
