// Batched factorization: many independent point sets (ragged sizes, one lengthscale each)
// built and applied together.
//
// Each set is factored exactly as hdf_build would factor it on its own (Algorithm 1,
// symmetric form); the batch changes only how the work is scheduled:
//  * A0 and A3 (centre, radius, mean-square kernel value, radial-basis Gram) run as segmented
//    reductions over all sets in one launch each, with per-item partials summed on the host in
//    item order (deterministic);
//  * A1-A2 and A4 (degree, cores, eigendecompositions, truncation, tables) run on host
//    threads, one set per task;
//  * A5 (radial factors and U) for all sets runs as persistent kernels that pull items from
//    device counters: one radial phase over (set, tiles) items, then one U-row phase per size
//    class of sets (sets grouped by the shared memory a warp needs, so each class runs with
//    its own warps per CTA); the launches are recorded as one CUDA graph and launched as a unit;
//  * K~V for all sets runs as persistent U^T V and U W kernels over (set, chunk, column block)
//    and (set, row block) items, recorded once in a CUDA graph and replayed.
// The shapes are chosen by an autotuner that times the candidates on first use and keeps the
// choice in a JSON cache ($HDF_AUTOTUNE_CACHE, default $HOME/.cache/hdf_gb300_autotune.json):
// tiles per item and CTAs per SM of the radial phase, warps per CTA (8, 16, 32) and CTAs per SM
// of each U class, and CTAs per SM of the products.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <sys/stat.h>
#include <vector>

#include "hdf_kernels.cuh"
#include "internal.h"
#include "planner.h"

using namespace hdf;

namespace {

constexpr int kMu2Sample = 512;

// Pinned host staging buffer for the batched build's table upload, kept between builds (grown
// on demand).  The caller holds the lock until the copy has completed; a build that finds it
// held uses pageable memory instead.
unsigned char* staging_acquire(size_t bytes, std::unique_lock<std::mutex>& lk) {
    static std::mutex mu;
    static unsigned char* buf = nullptr;
    static size_t cap = 0;
    std::unique_lock<std::mutex> l(mu, std::try_to_lock);
    if (!l.owns_lock()) return nullptr;
    if (cap < bytes) {
        if (buf) cudaFreeHost(buf);
        buf = nullptr;
        cap = 0;
        const size_t want = std::max(bytes, size_t(64) << 20);
        if (cudaMallocHost(reinterpret_cast<void**>(&buf), want) != cudaSuccess) {
            cudaGetLastError();
            buf = nullptr;
            return nullptr;
        }
        cap = want;
    }
    lk = std::move(l);
    return buf;
}
constexpr int kSegChunk = 8192;      // points per reduction item
constexpr int kGramChunk = 4096;     // points per Gram item

struct SegItem {
    int set;
    int pad;
    int64_t i0, i1;                  // global point range
};

struct SetGeom {                     // per set, for the segmented kernels
    int64_t off, n;
    double c[dev::kMaxD];
    double inv2R;
    int L, m;                        // degree, mu2 subsample size
    double ell;
};

// ------------------------------------------------------------ segmented reductions
__global__ void k_seg_sum(const double* __restrict__ x, int d, const SegItem* __restrict__ items,
                          double* __restrict__ part) {
    __shared__ double sh[256];
    const SegItem it = items[blockIdx.x];
    double acc[dev::kMaxD];
#pragma unroll
    for (int j = 0; j < dev::kMaxD; ++j) acc[j] = 0.0;
    for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x)
        for (int j = 0; j < d; ++j) acc[j] += x[i * d + j];
    for (int j = 0; j < d; ++j) {
        const double s = dev::block_sum_256(acc[j], sh);
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * d + j] = s;
    }
}

__global__ void k_seg_maxnorm(const double* __restrict__ x, int d, const SegItem* __restrict__ items,
                              const SetGeom* __restrict__ geo, double* __restrict__ part) {
    __shared__ double sh[256];
    const SegItem it = items[blockIdx.x];
    const SetGeom& g = geo[it.set];
    double m = 0.0;
    for (int64_t i = it.i0 + threadIdx.x; i < it.i1; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) { const double y = x[i * d + j] - g.c[j]; s += y * y; }
        m = fmax(m, s);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Sum over pairs i < j of K(x_i, x_j)^2 for sample rows i in [32 t, 32 t + 32) of set s
// (item (s, t)); the set's m strided sample points are staged in shared memory.  The host adds
// the diagonal m k(0)^2 and doubles nothing: part holds 2 x the half sum.  mu2 only sets the
// two error budgets, so the pairs run on the FP32 pipe (GB300's FP64 rate is a small fraction
// of it): coordinates relative to the set's centre (differences in FP64, then FP32), FP32
// kernel values (relative error ~1e-7), each thread's sum over one row in FP32 and the rest in
// FP64.
constexpr int kMu2Rows = 32;
__global__ void __launch_bounds__(256) k_seg_mu2_pairs(const double* __restrict__ x, int d,
                                                       const int2* __restrict__ items,
                                                       const SetGeom* __restrict__ geo, int kernel,
                                                       double* __restrict__ part) {
    __shared__ float xs[kMu2Sample * dev::kMaxD];
    __shared__ double sh[256];
    const int2 it = items[blockIdx.x];
    const SetGeom& g = geo[it.x];
    for (int u = threadIdx.x; u < g.m; u += blockDim.x) {
        const int64_t jj = g.off + ((int64_t)u * g.n) / g.m;
        for (int j = 0; j < d; ++j) xs[u * d + j] = (float)(x[jj * d + j] - g.c[j]);
    }
    __syncthreads();
    const float inv_ell = (float)(1.0 / g.ell);
    double acc = 0.0;
    const int r0 = it.y * kMu2Rows, r1 = min(g.m, r0 + kMu2Rows);
    for (int i = r0; i < r1; ++i) {
        float row = 0.f;
        for (int u = i + 1 + threadIdx.x; u < g.m; u += blockDim.x) {
            float s2 = 0.f;
            for (int j = 0; j < d; ++j) { const float y = xs[i * d + j] - xs[u * d + j]; s2 = fmaf(y, y, s2); }
            const float kv = dev::kernel_value_f(kernel, sqrtf(s2), inv_ell);
            row = fmaf(kv, kv, row);
        }
        acc += (double)row;
    }
    const double tot = dev::block_sum_256(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = 2.0 * tot;
}

// Chebyshev moments of one item (FP32 factors): part[poff + l], l < 2 L_s + 2.
__global__ void __launch_bounds__(256) k_seg_moments_df(const double* __restrict__ x, int d,
                                                        const SegItem* __restrict__ items,
                                                        const int64_t* __restrict__ poff,
                                                        const SetGeom* __restrict__ geo, double* __restrict__ part) {
    extern __shared__ float2 tsm_seg[];
    const SegItem it = items[blockIdx.x];
    const SetGeom& g = geo[it.set];
    const int nmom = 2 * g.L + 2;
    const double v = dev::moments_df_range(x, d, g.c, g.inv2R, nmom, it.i0, it.i1, tsm_seg);
    if (threadIdx.x < nmom) part[poff[blockIdx.x] + threadIdx.x] = v;
}

// Radial-basis Gram sums of one item: part[poff + q] (q < npairs) and part[poff + npairs + q].
__global__ void __launch_bounds__(256) k_seg_gram(const double* __restrict__ x, int d,
                                                  const SegItem* __restrict__ items,
                                                  const int64_t* __restrict__ poff,
                                                  const SetGeom* __restrict__ geo, double* __restrict__ part) {
    extern __shared__ double smem[];
    const SegItem it = items[blockIdx.x];
    const SetGeom& g = geo[it.set];
    const int L = g.L, LP1 = L + 1;
    const int npairs = LP1 * (LP1 + 1) / 2;
    double* Ts = smem;                              // [kGramTile][LP1]
    double* r2 = smem + dev::kGramTile * LP1;
    // this thread's pairs (l, l') in row order of the upper triangle
    int pl[dev::kGramMaxQ], pr[dev::kGramMaxQ];
#pragma unroll
    for (int q = 0; q < dev::kGramMaxQ; ++q) {
        int pi = threadIdx.x + 256 * q, l = 0;
        pl[q] = -1;
        pr[q] = 0;
        if (pi < npairs) {
            while (pi >= LP1 - l) { pi -= LP1 - l; ++l; }
            pl[q] = l;
            pr[q] = l + pi;
        }
    }
    double a0[dev::kGramMaxQ], a1[dev::kGramMaxQ];
#pragma unroll
    for (int q = 0; q < dev::kGramMaxQ; ++q) { a0[q] = 0.0; a1[q] = 0.0; }
    for (int64_t t0 = it.i0; t0 < it.i1; t0 += dev::kGramTile) {
        const int cnt = (int)min((int64_t)dev::kGramTile, it.i1 - t0);
        if (threadIdx.x < dev::kGramTile) {
            const int p = threadIdx.x;
            double* T = Ts + p * LP1;
            if (p < cnt) {
                const int64_t i = t0 + p;
                double s = 0.0;
                for (int j = 0; j < d; ++j) { const double y = (x[i * d + j] - g.c[j]) * g.inv2R; s += y * y; }
                const double u = 8.0 * s - 1.0;
                r2[p] = s;
                T[0] = 1.0;
                if (L >= 1) T[1] = u;
                for (int l = 2; l <= L; ++l) T[l] = 2.0 * u * T[l - 1] - T[l - 2];
            } else {
                r2[p] = 0.0;
                for (int l = 0; l <= L; ++l) T[l] = 0.0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < dev::kGramMaxQ; ++q) {
            if (pl[q] >= 0) {
                double s0 = 0.0, s1 = 0.0;
                for (int p = 0; p < cnt; ++p) {
                    const double v = Ts[p * LP1 + pl[q]] * Ts[p * LP1 + pr[q]];
                    s0 += v;
                    s1 += v * r2[p];
                }
                a0[q] += s0;
                a1[q] += s1;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < dev::kGramMaxQ; ++q) {
        const int pi = threadIdx.x + 256 * q;
        if (pi < npairs) {
            part[poff[blockIdx.x] + pi] = a0[q];
            part[poff[blockIdx.x] + npairs + pi] = a1[q];
        }
    }
}

// ------------------------------------------------------------- persistent build
struct BuildSet {
    dev::RFParams rf;
    dev::UWParams uw;
    int pre;
};

// Shared memory of the double-float radial phase of the batched build for `tiles` tiles per
// item: one buffer of basis pairs and rho per tile, then Q.
inline size_t batch_df_tile_smem(int L, int mt, int tiles) {
    return (size_t)tiles * dev::radialF_df_basis_bytes(L) + sizeof(float) * (size_t)mt * dev::kFTile;
}

// A5 for every set in two persistent phases, each with its own register and shared-memory budget:
// k_batch_radial computes the radial factors of (set, tiles) items; k_batch_urows writes the U rows
// of (set, point block) items and is launched once per size class of sets (sets grouped by the
// shared memory a warp needs), so that small sets run with many more warps per SM than the
// largest set of the batch would allow.
template <typename T>
__global__ void __launch_bounds__(256, 2) k_batch_radial(const BuildSet* __restrict__ sets,
                                                         const int2* __restrict__ items, int nitems, int* counter,
                                                         int tiles_per_item) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int2 w = items[it];
        const BuildSet& S = sets[w.x];
        const int64_t t0 = (int64_t)w.y * tiles_per_item * dev::kFTile;
        if constexpr (sizeof(T) == 4) {
            // FP32 sets always carry the double-float tables (QC).  First the basis values of all
            // the item's tiles at once (thread = point), then per tile Q (S.rf.kopt outputs per
            // thread) and F by all warps.
            const int LP1 = S.rf.L + 1;
            const size_t bb = dev::radialF_df_basis_bytes(S.rf.L);
            const int ntile = (int)min((int64_t)tiles_per_item, (S.rf.n - t0 + dev::kFTile - 1) / dev::kFTile);
            for (int pt = threadIdx.x; pt < ntile * dev::kFTile; pt += blockDim.x) {
                const int q = pt / dev::kFTile;
                float2* Tq = reinterpret_cast<float2*>(smem_raw + q * bb);
                dev::radialF_df_basis(S.rf, t0 + (int64_t)q * dev::kFTile, pt % dev::kFTile, Tq,
                                      reinterpret_cast<float*>(Tq + dev::kFTile * LP1));
            }
            __syncthreads();
            float* Qs = reinterpret_cast<float*>(smem_raw + tiles_per_item * bb);
            for (int q = 0; q < ntile; ++q) {
                const float2* Tq = reinterpret_cast<const float2*>(smem_raw + q * bb);
                const float* rq = reinterpret_cast<const float*>(Tq + dev::kFTile * LP1);
                if (S.rf.kopt == 2)
                    dev::radialF_df_q<2>(S.rf, Tq, rq, S.rf.QC, Qs, threadIdx.x, blockDim.x);
                else
                    dev::radialF_df_q<4>(S.rf, Tq, rq, S.rf.QC, Qs, threadIdx.x, blockDim.x);
                __syncthreads();
                dev::radialF_df_f(S.rf, t0 + (int64_t)q * dev::kFTile, Qs, reinterpret_cast<const float*>(S.rf.Wt),
                                  threadIdx.x, blockDim.x);
                __syncthreads();
            }
        } else {
            for (int q = 0; q < tiles_per_item; ++q) {
                const int64_t tq = t0 + (int64_t)q * dev::kFTile;
                if (tq >= S.rf.n) break;
                dev::radialF_tile<T>(S.rf, tq, smem_raw);
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_batch_urows(const BuildSet* __restrict__ sets, const int2* __restrict__ items,
                                                      int nitems, int* counter, int pts_per_item) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int2 w = items[it];
        const BuildSet& S = sets[w.x];
        const int levels = S.uw.d - 2;
        T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * S.uw.per_warp;
        T* cA = reinterpret_cast<T*>(smem_raw) + (size_t)nwarps * S.uw.per_warp;
        T* cB = cA + levels * S.uw.tri;
        for (int idx = threadIdx.x; idx < levels * S.uw.tri; idx += blockDim.x) {
            cA[idx] = reinterpret_cast<const T*>(S.uw.coefA)[idx];
            cB[idx] = reinterpret_cast<const T*>(S.uw.coefB)[idx];
        }
        __syncthreads();
        dev::uwriter_zero_slots<T>(S.uw, S.pre != 0, base, lane);
        const int64_t i0 = (int64_t)w.y * pts_per_item, i1 = min(i0 + pts_per_item, S.uw.n);
        const dev::UWTabs X{S.uw.qdesc, S.uw.chains, S.uw.gslot, S.uw.ychain};
        for (int64_t i = i0 + warp; i < i1; i += nwarps) dev::uwriter_point<T>(S.uw, X, S.pre != 0, i, cA, cB, base, lane);
        __syncthreads();
    }
}

// ------------------------------------------------------------ persistent matvec
struct MvSet {
    const void* U; int64_t ldU, n, r, off;
    const void* S;
    double* part;                    // nchunk x c x r
    void* W;                         // r x ldw (bulk type), row a = the c values of column a
    int ldw;                         // c, or the column tile width (zero-padded) for the streaming kernels
    int64_t chunk;
    int nchunk;
};

struct MvItem { int set, chunk; int64_t blk; };

template <typename T, int CT>
__global__ void __launch_bounds__(256) k_batch_utv(const MvSet* __restrict__ sets, const MvItem* __restrict__ items,
                                                   int nitems, int* counter, const T* __restrict__ V, int64_t ldv, int c) {
    __shared__ __align__(16) T Us[dev::kKT][dev::UtvShape<CT>::AB];
    __shared__ __align__(16) T Vs[dev::kKT][CT];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const MvItem w = items[it];
        const MvSet& S = sets[w.set];
        const int64_t i0 = (int64_t)w.chunk * S.chunk, i1 = min(S.n, i0 + S.chunk);
        dev::utv_tile_body<T, CT>(reinterpret_cast<const T*>(S.U), S.ldU, S.r, V + S.off, ldv, c, i0, i1,
                                  w.blk * dev::UtvShape<CT>::AB, S.part + (int64_t)w.chunk * c * S.r, Us, Vs);
        __syncthreads();
    }
}

template <typename T>
__global__ void k_batch_reduce(const MvSet* __restrict__ sets, const MvItem* __restrict__ items, int c) {
    const MvItem w = items[blockIdx.x];
    const MvSet& S = sets[w.set];
    const int64_t a = w.blk * 256 + threadIdx.x;
    if (a >= S.r) return;
    const T* Sv = reinterpret_cast<const T*>(S.S);
    T* W = reinterpret_cast<T*>(S.W);
    for (int j = 0; j < S.ldw; ++j) {
        double s = 0.0;
        if (j < c)
            for (int b = 0; b < S.nchunk; ++b) s += S.part[((int64_t)b * c + j) * S.r + a];
        W[a * S.ldw + j] = (T)(s * (double)Sv[a]);
    }
}

template <typename T, int CT>
__global__ void __launch_bounds__(256) k_batch_uw(const MvSet* __restrict__ sets, const MvItem* __restrict__ items,
                                                  int nitems, int* counter, T* __restrict__ Y, int64_t ldy, int c) {
    __shared__ __align__(16) T Us[dev::kKT][dev::UwShape<CT>::RB + dev::kUwPad];
    __shared__ __align__(16) T Ws[dev::kKT][CT];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const MvItem w = items[it];
        const MvSet& S = sets[w.set];
        dev::uw_tile_body<T, CT>(reinterpret_cast<const T*>(S.U), S.ldU, S.n, S.r, reinterpret_cast<const T*>(S.W), c,
                                 (T)1, nullptr, 0, (T)0, Y + S.off, ldy, w.blk * dev::UwShape<CT>::RB, Us, Ws);
        __syncthreads();
    }
}

// ------------------------------------------------ skinny FP32 matvec (c <= 16)
// Streaming kernels for few columns, where a register-tiled GEMM is bound by its shared-memory
// instructions rather than by HBM.  U^T V: lane = TA consecutive columns of U (one 8- or 16-byte
// load per row), the warps of a CTA stride over the rows of a chunk, V rows are staged in shared
// memory and read as broadcasts; the eight warps' partial sums are added in a fixed order.
// U W: k_batch_uw_b below (lane = row, U through bulk copies, W rows as broadcasts).
template <int CT> struct SkinnyShape {
    static constexpr int TA = CT <= 8 ? 4 : 2;      // U^T V: columns per lane
    static constexpr int AB = 32 * TA;              // U^T V: columns per item
    static constexpr int VR = CT <= 4 ? 512 : (CT == 8 ? 384 : 128);   // U^T V: V rows staged per pass
                                                                        // (static shared memory < 48 KB)
};

template <int N> struct FVec;
template <> struct FVec<2> {
    static __device__ __forceinline__ void ld(const float* p, float* o) {
        const float2 v = *reinterpret_cast<const float2*>(p); o[0] = v.x; o[1] = v.y;
    }
};
template <> struct FVec<4> {
    static __device__ __forceinline__ void ld(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p); o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};

template <int CT>
__device__ __forceinline__ void ld_row(const float* p, float* o) {
    if constexpr (CT % 4 == 0) {
#pragma unroll
        for (int j = 0; j < CT; j += 4) FVec<4>::ld(p + j, o + j);
    } else if constexpr (CT == 2) {
        FVec<2>::ld(p, o);
    } else {
        o[0] = p[0];
    }
}

template <int CT>
__global__ void __launch_bounds__(256) k_batch_utv_s(const MvSet* __restrict__ sets, const MvItem* __restrict__ items,
                                                     int nitems, int* counter, const float* __restrict__ V,
                                                     int64_t ldv, int c) {
    using SS = SkinnyShape<CT>;
    constexpr int TA = SS::TA, AB = SS::AB, VR = SS::VR, UNR = 4;
    __shared__ __align__(16) float Vs[VR][CT];
    __shared__ __align__(16) float red[8][AB][CT];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const MvItem w = items[it];
        const MvSet& S = sets[w.set];
        const float* U = reinterpret_cast<const float*>(S.U);
        const int64_t i0 = (int64_t)w.chunk * S.chunk, i1 = min(S.n, i0 + S.chunk);
        const int64_t a0 = w.blk * AB, a = a0 + (int64_t)lane * TA;
        const bool act = a < S.r;                    // S.r is a multiple of 4 (padded width)
        float acc[TA][CT];
#pragma unroll
        for (int q = 0; q < TA; ++q)
#pragma unroll
            for (int j = 0; j < CT; ++j) acc[q][j] = 0.f;
        for (int64_t k0 = i0; k0 < i1; k0 += VR) {
            const int nr = (int)min((int64_t)VR, i1 - k0);
            __syncthreads();
            for (int e = threadIdx.x; e < VR * CT; e += blockDim.x) {
                const int rr = e % VR, j = e / VR;
                Vs[rr][j] = (rr < nr && j < c) ? V[S.off + k0 + rr + (int64_t)j * ldv] : 0.f;
            }
            __syncthreads();
            if (!act) continue;
            for (int r0 = warp; r0 < nr; r0 += 8 * UNR) {
                float u[UNR][TA];
#pragma unroll
                for (int t = 0; t < UNR; ++t) {
                    const int rr = r0 + 8 * t;
                    if (rr < nr) {
                        FVec<TA>::ld(U + (k0 + rr) * S.ldU + a, u[t]);
                    } else {
#pragma unroll
                        for (int q = 0; q < TA; ++q) u[t][q] = 0.f;
                    }
                }
#pragma unroll
                for (int t = 0; t < UNR; ++t) {
                    const int rr = min(r0 + 8 * t, VR - 1);    // rows past nr carry u = 0
                    float v[CT];
                    ld_row<CT>(&Vs[rr][0], v);
#pragma unroll
                    for (int q = 0; q < TA; ++q)
#pragma unroll
                        for (int j = 0; j < CT; ++j) acc[q][j] += u[t][q] * v[j];
                }
            }
        }
        // partial sums of the eight warps, added in warp order
#pragma unroll
        for (int q = 0; q < TA; ++q)
#pragma unroll
            for (int j = 0; j < CT; ++j) red[warp][lane * TA + q][j] = acc[q][j];
        __syncthreads();
        for (int e = threadIdx.x; e < AB * CT; e += blockDim.x) {
            const int col = e / CT, j = e % CT;
            float sum = 0.f;
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) sum += red[ww][col][j];
            const int64_t aa = a0 + col;
            if (aa < S.r && j < c) S.part[((int64_t)w.chunk * c + j) * S.r + aa] = (double)sum;
        }
        __syncthreads();
    }
}

// ------------------------------------------------ pipelined U^T V (c <= 8)
// The loads of k_batch_utv_s land in registers, which caps the bytes a SM keeps in flight
// well below what HBM latency needs.  This variant streams U through a per-warp ring of
// shared-memory stages filled by cp.async (16 bytes per lane, zero fill outside the set),
// three tiles ahead of the arithmetic, so that registers hold only sums.  (The same ring for
// U W, with lane = 4 columns, measured slower than register loads: each lane reads its own W
// rows, and the ring's shared memory leaves L1 too small to keep the set's W resident.)
constexpr int kPipeStages = 4;      // tiles in flight per warp
constexpr int kPipeRows = 4;        // rows per tile
constexpr int kPipeCols = 128;      // columns per tile (4 per lane)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// floats of one U^T V stage: the U tile, then its kPipeRows x CT values of V
template <int CT> constexpr int utv_stage_floats() { return kPipeRows * kPipeCols + kPipeRows * CT; }
template <int CT> constexpr size_t utv_pipe_smem() {
    return sizeof(float) * (size_t)8 * kPipeStages * utv_stage_floats<CT>();
}

// Partial sums of U^T V as k_batch_utv_s (same items: set, 4096-row chunk, 128-column block).
// Warp w takes the row groups i0 + 4 (w + 8 t) .. + 3; each stage holds such a group's U tile and
// its V rows.  The eight warps' sums are added in warp order through shared memory that
// reuses the drained ring.
template <int CT>
__global__ void __launch_bounds__(256) k_batch_utv_p(const MvSet* __restrict__ sets, const MvItem* __restrict__ items,
                                                     int nitems, int* counter, const float* __restrict__ V,
                                                     int64_t ldv, int c) {
    static_assert(kPipeRows * CT <= 32, "one V value per lane and stage");
    constexpr int SF = utv_stage_floats<CT>();
    extern __shared__ __align__(16) float smp[];
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* ring = smp + (size_t)warp * kPipeStages * SF;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const MvItem w = items[it];
        const MvSet& S = sets[w.set];
        const float* U = reinterpret_cast<const float*>(S.U);
        const int64_t i0 = (int64_t)w.chunk * S.chunk, i1 = min(S.n, i0 + S.chunk);
        const int64_t a0 = w.blk * kPipeCols, a = a0 + 4 * lane;
        const bool act = a < S.r;                     // S.r is a multiple of 4 (padded width)
        const int ntiles = (int)((i1 - i0 + kPipeRows * 8 - 1) / (kPipeRows * 8));
        auto issue = [&](int t) {
            float* st = ring + (t % kPipeStages) * SF;
            const int64_t rb = i0 + (int64_t)kPipeRows * (warp + 8 * t);
#pragma unroll
            for (int q = 0; q < kPipeRows; ++q) {
                const int64_t i = rb + q;
                const bool ok = act && i < i1;
                cp_async16(st + q * kPipeCols + 4 * lane, ok ? (const void*)(U + i * S.ldU + a) : (const void*)U,
                           ok ? 16 : 0);
            }
            if (lane < kPipeRows * CT) {
                const int q = lane / CT, j = lane % CT;
                const int64_t i = rb + q;
                const bool ok = i < i1 && j < c;
                cp_async4(st + kPipeRows * kPipeCols + lane, ok ? (const void*)(V + S.off + i + (int64_t)j * ldv)
                                                                : (const void*)V, ok ? 4 : 0);
            }
        };
        float acc[4][CT];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int j = 0; j < CT; ++j) acc[q][j] = 0.f;
#pragma unroll
        for (int t = 0; t < kPipeStages - 1; ++t) {
            if (t < ntiles) issue(t);
            cp_commit();
        }
        for (int t = 0; t < ntiles; ++t) {
            if (t + kPipeStages - 1 < ntiles) issue(t + kPipeStages - 1);
            cp_commit();
            cp_wait<kPipeStages - 1>();
            __syncwarp();
            const float* st = ring + (t % kPipeStages) * SF;
#pragma unroll
            for (int q = 0; q < kPipeRows; ++q) {
                const float4 u = *reinterpret_cast<const float4*>(st + q * kPipeCols + 4 * lane);
                const float* vq = st + kPipeRows * kPipeCols + q * CT;
#pragma unroll
                for (int j = 0; j < CT; ++j) {
                    const float v = vq[j];
                    acc[0][j] = fmaf(u.x, v, acc[0][j]);
                    acc[1][j] = fmaf(u.y, v, acc[1][j]);
                    acc[2][j] = fmaf(u.z, v, acc[2][j]);
                    acc[3][j] = fmaf(u.w, v, acc[3][j]);
                }
            }
            __syncwarp();                              // the stage is refilled next iteration
        }
        cp_wait<0>();
        __syncthreads();                               // every warp's ring drained: reuse it
        float* red = smp;                              // [8][kPipeCols][CT]
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int j = 0; j < CT; ++j) red[((size_t)warp * kPipeCols + 4 * lane + q) * CT + j] = acc[q][j];
        __syncthreads();
        for (int e = threadIdx.x; e < kPipeCols * CT; e += blockDim.x) {
            const int col = e / CT, j = e % CT;
            float sum = 0.f;
#pragma unroll
            for (int ww = 0; ww < 8; ++ww) sum += red[((size_t)ww * kPipeCols + col) * CT + j];
            const int64_t aa = a0 + col;
            if (aa < S.r && j < c) S.part[((int64_t)w.chunk * c + j) * S.r + aa] = (double)sum;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ autotuner
std::mutex g_tune_mu;

std::string tune_path() {
    if (const char* p = std::getenv("HDF_AUTOTUNE_CACHE")) return p;
    const char* home = std::getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/hdf_gb300_autotune.json";
}

// Minimal JSON object of "key": integer pairs.
std::map<std::string, int> tune_load() {
    std::map<std::string, int> m;
    std::ifstream in(tune_path());
    if (!in) return m;
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string s = ss.str();
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        const size_t e = s.find('"', pos + 1);
        if (e == std::string::npos) break;
        const std::string key = s.substr(pos + 1, e - pos - 1);
        const size_t colon = s.find(':', e);
        if (colon == std::string::npos) break;
        m[key] = std::atoi(s.c_str() + colon + 1);
        pos = colon + 1;
    }
    return m;
}

void tune_store(const std::map<std::string, int>& m) {
    const std::string path = tune_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) mkdir(path.substr(0, slash).c_str(), 0755);   // one level, errors ignored
    std::ofstream out(path);
    if (!out) return;
    out << "{";
    bool first = true;
    for (const auto& kv : m) {
        out << (first ? "" : ", ") << "\"" << kv.first << "\": " << kv.second;
        first = false;
    }
    out << "}\n";
}

// ------------------------------------------------ U W with tensor copies (c <= 16)
// Lane = row of the item's 32-row tile (acc[CT] in registers), so that every lane reads the same
// W row (a shared-memory broadcast) instead of private ones.  The tile's U rows and the matching
// rows of W stream through a per-warp ring of shared-memory stages, kBwStages - 1 stages ahead of
// the arithmetic: per stage one TMA tensor copy brings the 32 x 32 block of U (the set's tensor
// map; rows past the set and columns past its width arrive as zeros; 128-byte swizzle, so that
// the 16-byte loads of eight consecutive rows hit distinct banks) and one bulk copy the 32 x CT
// block of W, both completing on the stage's mbarrier.  Items (set, 32-row tile) are taken per
// warp from a global counter, and the copies of the next items start while the current one is
// computed.  Every wait is bounded; a warp that gives up records the error, waits (bounded) for
// its copies in flight and leaves.
constexpr int kBwCols = 32;                     // columns of U per stage (one 128-byte swizzle row)
constexpr int kBwStages = 3;
constexpr int kBwWarps = 4;
constexpr long long kBwWait = 4000000000ll;     // about 2 s at 2 GHz
// bytes of one stage: the U block (32 rows of 128 bytes, 1024-byte aligned for the swizzle),
// then the W block, padded so that the next stage stays 1024-byte aligned
template <int CT> constexpr int bw_stage_bytes() { return 4096 + ((128 * CT + 1023) / 1024) * 1024; }
template <int CT> constexpr size_t bw_smem() { return 1024 + (size_t)kBwWarps * kBwStages * bw_stage_bytes<CT>(); }

__device__ __forceinline__ uint32_t b_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool b_mbar_try(uint32_t a, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool b_mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = b_smem_u32(bar);
    if (b_mbar_try(a, parity)) return true;
    const long long t0 = clock64();
    for (;;) {
        if (b_mbar_try(a, parity)) return true;
        if (clock64() - t0 > kBwWait) return false;
    }
}

// A set of k_batch_uw_b: its 32-row tiles are items tile0 .. tile0 + ceil(n / 32) - 1.
struct BwSet {
    const float* W;         // the set's W (r x CT)
    int64_t off;            // the set's first output row
    int64_t tile0;          // its first item
    int n;                  // rows
    int r;                  // padded width (a multiple of 4)
};

template <int CT>
__global__ void __launch_bounds__(32 * kBwWarps) k_batch_uw_b(const BwSet* __restrict__ bsets, int nsets, int nitems,
                                                              int* counter, const CUtensorMap* __restrict__ maps,
                                                              float* __restrict__ Y, int64_t ldy, int c, int* err) {
    extern __shared__ unsigned char smraw[];
    __shared__ __align__(8) uint64_t full[kBwWarps][kBwStages];
    constexpr int SB = bw_stage_bytes<CT>();
    constexpr int NQ = 8;                     // claimed items not yet finished: at most kBwStages + 1
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // 1024-byte alignment by an offset from the shared-memory pointer itself, so that the
    // compiler still sees shared-memory loads (a round trip through an integer would leave
    // generic ones)
    unsigned char* base = smraw + ((1024u - (b_smem_u32(smraw) & 1023u)) & 1023u);
    unsigned char* ring = base + (size_t)warp * kBwStages * SB;
    uint64_t* bar = full[warp];
    if (lane < kBwStages) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b_smem_u32(&bar[lane])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // The copies run ahead of the arithmetic across item boundaries: the issue cursor (stage ti
    // of ni of the current issue item) takes the item claimed one ahead (its record already
    // loaded) when its item is exhausted, and claims the next; lane (k mod NQ) keeps the width,
    // output offset and row count of the k-th item for the arithmetic, which follows in order.
    auto claim = [&]() -> int {
        int v = 0;
        if (lane == 0) v = atomicAdd(counter, 1);
        return __shfl_sync(0xffffffffu, v, 0);
    };
    uint32_t issued = 0, used = 0;            // stages issued and consumed by this warp (ring order)
    uint32_t q_head = 0, q_tail = 0;          // items: finished, handed to the issue cursor
    int q_r = 0, q_nrows = 0;
    int64_t q_yoff = 0;
    // an item's set (binary search over the sets' first items), first row and row count
    struct Item { const float* W; int64_t yoff; int row0, set, r, nrows; };
    auto item_of = [&](int v) {
        int lo = 0, hi = nsets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bsets[mid].tile0 <= v) lo = mid; else hi = mid - 1;
        }
        const BwSet& S = bsets[lo];
        Item t;
        t.row0 = (int)((v - S.tile0) * 32);
        t.W = S.W; t.yoff = S.off + t.row0; t.set = lo; t.r = S.r; t.nrows = min(32, S.n - t.row0);
        return t;
    };
    int ti = 0, ni = 0;
    Item cur{};                               // the issue cursor's item
    int nxt_idx = claim();                    // claimed one ahead, located ahead of use
    Item nxt{};
    if (nxt_idx < nitems) nxt = item_of(nxt_idx);
    bool ok = true;
    auto advance_issue = [&]() {
        if (ti >= ni) {                       // the issue item is exhausted (or there is none yet)
            if (nxt_idx >= nitems) return;
            cur = nxt;
            ti = 0;
            ni = (cur.r + kBwCols - 1) / kBwCols;
            if (lane == (int)(q_tail % NQ)) { q_r = cur.r; q_nrows = cur.nrows; q_yoff = cur.yoff; }
            ++q_tail;
            nxt_idx = claim();
            if (nxt_idx < nitems) nxt = item_of(nxt_idx);
        }
        const uint32_t slot = issued % kBwStages;
        const int a0 = ti * kBwCols;
        const uint32_t wbytes = (uint32_t)(min(kBwCols, cur.r - a0) * CT * 4);   // r: a multiple of 4
        unsigned char* st = ring + (size_t)slot * SB;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // earlier reads of the slot
        __syncwarp();
        if (lane == 0) {
            const uint32_t b = b_smem_u32(&bar[slot]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(4096u + wbytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];" ::"r"(b_smem_u32(st)),
                "l"((uint64_t)(maps + cur.set)), "r"(a0), "r"(cur.row0), "r"(b)
                : "memory");
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    b_smem_u32(st + 4096)),
                "l"(cur.W + (int64_t)a0 * CT), "r"(wbytes), "r"(b)
                : "memory");
        }
        ++issued;
        ++ti;
    };
    for (int k = 0; k < kBwStages - 1; ++k) advance_issue();
    while (ok && q_head < q_tail) {
        const int src = (int)(q_head % NQ);
        const int r = __shfl_sync(0xffffffffu, q_r, src);
        const int nrows = __shfl_sync(0xffffffffu, q_nrows, src);
        const int64_t yoff = __shfl_sync(0xffffffffu, q_yoff, src);
        const int nst = (r + kBwCols - 1) / kBwCols;
        float acc[CT];
#pragma unroll
        for (int j = 0; j < CT; ++j) acc[j] = 0.f;
        for (int t = 0; t < nst; ++t) {
            advance_issue();                  // keeps kBwStages - 1 stages ahead, across items
            const uint32_t slot = used % kBwStages;
            if (!__all_sync(0xffffffffu, b_mbar_wait(&bar[slot], (used / kBwStages) & 1))) { ok = false; break; }
            ++used;
            const unsigned char* su = ring + (size_t)slot * SB + lane * 128;     // this lane's row
            const float* sw = reinterpret_cast<const float*>(ring + (size_t)slot * SB + 4096);
            const int na = min(kBwCols, r - t * kBwCols);
            auto cols4 = [&](int jj) {                // columns 4 jj .. 4 jj + 3 (16-byte chunk jj)
                const float4 u = *reinterpret_cast<const float4*>(su + ((jj ^ (lane & 7)) << 4));
                const float uq[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float wv[CT];
                    ld_row<CT>(sw + (4 * jj + q) * CT, wv);
#pragma unroll
                    for (int j = 0; j < CT; ++j) acc[j] = fmaf(uq[q], wv[j], acc[j]);
                }
            };
            if (na == kBwCols) {
#pragma unroll 4
                for (int jj = 0; jj < kBwCols / 4; ++jj) cols4(jj);
            } else {
                for (int jj = 0; jj < na / 4; ++jj) cols4(jj);
            }
            __syncwarp();                     // every lane is done with the slot before it is refilled
        }
        if (!ok) break;
        if (lane < nrows) {
#pragma unroll
            for (int j = 0; j < CT; ++j)
                if (j < c) Y[yoff + lane + (int64_t)j * ldy] = acc[j];
        }
        ++q_head;
    }
    if (!ok) {
        // copies still in flight land before the warp leaves (bounded)
        for (; used < issued; ++used) b_mbar_wait(&bar[used % kBwStages], (used / kBwStages) & 1);
        if (lane == 0) atomicExch(err, 1);
    }
}

int ct_for(int c) { return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : c <= 32 ? 32 : 64; }

}  // namespace

// ------------------------------------------------------------------ batch object
struct hdf_batch {
    int nsets = 0, d = 0, prec = 0, kernel = 0;
    double tol = 0.0;
    size_t esz = 8;
    std::vector<int64_t> off;                       // nsets + 1
    std::vector<hdf_info> info;
    std::vector<std::vector<double>> S_host;
    std::vector<int64_t> uoff, soff;                // element offsets of U and S per set
    std::vector<std::vector<int64_t>> colmap;       // per set: padded column of each true column
    DevBuf U, S, arena, dsets;
    // matvec state
    DevBuf mvsets, mvitems_utv, mvitems_red, mvitems_uw, mvpart, mvW, counters;
    DevBuf derr;                                    // set by a matvec kernel that gave up a bounded wait
    DevBuf umaps;                                   // per set: TMA tensor map of U (32 x 32 boxes, FP32 batches)
    DevBuf bwsets;                                  // sets of the FP32 U W kernel (items: 32-row tiles)
    int mv_c = 0, n_utv = 0, n_red = 0, n_uw = 0, n_bw = 0;
    cudaGraphExec_t mv_exec = nullptr;
    const void* mv_V = nullptr;
    void* mv_Y = nullptr;
    int64_t mv_ldv = 0, mv_ldy = 0;
    cudaStream_t cap = nullptr;
    double t_ms[HDF_NPHASE] = {};
    int grid_build = 0;
    int nclass = 0;                                 // size classes of the U phase of the last build
    ~hdf_batch() {
        if (mv_exec) cudaGraphExecDestroy(mv_exec);
        if (cap) cudaStreamDestroy(cap);
    }
};

static double now_ms_b() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename T>
static hdf_status batch_build_t(hdf_batch* b, const double* x, const std::vector<double>& ells, double tol, double eta,
                                int p_max, cudaStream_t st, bool* all_reached) {
    const int ns = b->nsets, d = b->d;
    const double t_start = now_ms_b();
    std::vector<SetGeom> geo(ns);
    for (int s = 0; s < ns; ++s) {
        geo[s].off = b->off[s];
        geo[s].n = b->off[s + 1] - b->off[s];
        geo[s].ell = ells[s];
        geo[s].m = (int)std::min<int64_t>(geo[s].n, kMu2Sample);
    }
    // ---- A0: segmented centre, radius, mu2
    std::vector<SegItem> items;
    for (int s = 0; s < ns; ++s)
        for (int64_t i0 = 0; i0 < geo[s].n; i0 += kSegChunk)
            items.push_back({s, 0, geo[s].off + i0, geo[s].off + std::min<int64_t>(geo[s].n, i0 + kSegChunk)});
    const int nit = (int)items.size();
    std::vector<int2> mrows;                      // (set, tile of kMu2Rows sample rows)
    for (int s = 0; s < ns; ++s)
        for (int t = 0; t * kMu2Rows < geo[s].m; ++t) mrows.push_back(make_int2(s, t));
    DevBuf ditems, dgeo, dpart, drows;
    HDF_CUDA(ditems.alloc_on(sizeof(SegItem) * nit, st));
    HDF_CUDA(dgeo.alloc_on(sizeof(SetGeom) * ns, st));
    HDF_CUDA(drows.alloc_on(sizeof(int2) * mrows.size(), st));
    HDF_CUDA(dpart.alloc_on(sizeof(double) * std::max<size_t>((size_t)nit * d, mrows.size()), st));
    HDF_CUDA(cudaMemcpyAsync(ditems.p, items.data(), sizeof(SegItem) * nit, cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(drows.p, mrows.data(), sizeof(int2) * mrows.size(), cudaMemcpyHostToDevice, st));
    HDF_COUNT_LAUNCH();
    k_seg_sum<<<nit, 256, 0, st>>>(x, d, ditems.as<SegItem>(), dpart.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> hp((size_t)nit * d);
    HDF_CUDA(cudaMemcpyAsync(hp.data(), dpart.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    {
        std::vector<std::vector<double>> sums(ns, std::vector<double>(d, 0.0));
        for (int q = 0; q < nit; ++q)
            for (int j = 0; j < d; ++j) sums[items[q].set][j] += hp[(size_t)q * d + j];
        for (int s = 0; s < ns; ++s)
            for (int j = 0; j < d; ++j) {
                geo[s].c[j] = sums[s][j] / (double)geo[s].n;
                if (!std::isfinite(geo[s].c[j])) return fail(HDF_ENOTFINITE, "hdf_build_batched: non-finite points");
            }
    }
    HDF_CUDA(cudaMemcpyAsync(dgeo.p, geo.data(), sizeof(SetGeom) * ns, cudaMemcpyHostToDevice, st));
    HDF_COUNT_LAUNCH();
    k_seg_maxnorm<<<nit, 256, 0, st>>>(x, d, ditems.as<SegItem>(), dgeo.as<SetGeom>(), dpart.as<double>());
    HDF_CUDA(cudaGetLastError());
    HDF_CUDA(cudaMemcpyAsync(hp.data(), dpart.p, sizeof(double) * nit, cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<double> Rs(ns, 0.0);
    for (int q = 0; q < nit; ++q) Rs[items[q].set] = std::max(Rs[items[q].set], hp[q]);
    for (int s = 0; s < ns; ++s) {
        Rs[s] = std::sqrt(Rs[s]);
        if (!std::isfinite(Rs[s])) return fail(HDF_ENOTFINITE, "hdf_build_batched: non-finite points");
        if (Rs[s] == 0.0) Rs[s] = 1.0;
        geo[s].inv2R = 1.0 / (2.0 * Rs[s]);
    }
    HDF_CUDA(cudaMemcpyAsync(dgeo.p, geo.data(), sizeof(SetGeom) * ns, cudaMemcpyHostToDevice, st));
    HDF_COUNT_LAUNCH();
    k_seg_mu2_pairs<<<(unsigned)mrows.size(), 256, 0, st>>>(x, d, drows.as<int2>(), dgeo.as<SetGeom>(), b->kernel,
                                                           dpart.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> mp(mrows.size());
    HDF_CUDA(cudaMemcpyAsync(mp.data(), dpart.p, sizeof(double) * mp.size(), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<double> mu2(ns, 0.0);
    for (size_t q = 0; q < mrows.size(); ++q) mu2[mrows[q].x] += mp[q];
    for (int s = 0; s < ns; ++s) {
        const double k0 = kernel_value(b->kernel, 0.0, ells[s]);
        mu2[s] = (mu2[s] + geo[s].m * k0 * k0) / ((double)geo[s].m * (double)geo[s].m);
    }
    b->t_ms[0] = now_ms_b() - t_start;

    // ---- A1 per set on host threads (the radial cores, A2, follow while the device sums the
    //      radial moments below)
    double t0 = now_ms_b();
    std::vector<DegreePlan> dps(ns);
    parallel_for(ns, [&](int s) {
        plan_degree(b->kernel, ells[s], Rs[s], mu2[s], geo[s].n, tol, eta, p_max, d, false, dps[s], false);
    });
    // per-set host work in order of decreasing degree (the cost grows like p^5), so that the
    // largest sets do not start last on the worker pool
    std::vector<int> by_cost(ns);
    for (int s = 0; s < ns; ++s) by_cost[s] = s;
    std::stable_sort(by_cost.begin(), by_cost.end(), [&](int a, int b) { return dps[a].p > dps[b].p; });
    auto cores_all = [&]() {
        parallel_for(ns, [&](int t) {
            const int s = by_cost[t];
            radial_cores(dps[s].a.data(), dps[s].p, d, dps[s].cores, false);
        });
    };
    for (int s = 0; s < ns; ++s) geo[s].L = dps[s].L;
    b->t_ms[1] = now_ms_b() - t0;

    // ---- A3: segmented radial-basis Gram (FP32 factors: from Chebyshev moments, O(nL))
    t0 = now_ms_b();
    int Lmax = 0;
    for (int s = 0; s < ns; ++s) Lmax = std::max(Lmax, geo[s].L);
    std::vector<std::vector<double>> grams(ns);
    const size_t msm = sizeof(float2) * 256 * (size_t)(2 * Lmax + 3);
    if (sizeof(T) == 4 && msm <= 200 * 1024) {
        std::vector<SegItem> gitems;
        std::vector<int64_t> gpoff;
        int64_t gtot = 0;
        for (int s = 0; s < ns; ++s) {
            const int nmom = 2 * geo[s].L + 2;
            for (int64_t i0 = 0; i0 < geo[s].n; i0 += kGramChunk) {
                gitems.push_back({s, 0, geo[s].off + i0, geo[s].off + std::min<int64_t>(geo[s].n, i0 + kGramChunk)});
                gpoff.push_back(gtot);
                gtot += nmom;
            }
        }
        DevBuf dgi, dgpoff, dgpart;
        HDF_CUDA(dgi.alloc_on(sizeof(SegItem) * gitems.size(), st));
        HDF_CUDA(dgpoff.alloc_on(sizeof(int64_t) * gpoff.size(), st));
        HDF_CUDA(dgpart.alloc_on(sizeof(double) * gtot, st));
        HDF_CUDA(cudaMemcpyAsync(dgi.p, gitems.data(), sizeof(SegItem) * gitems.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaMemcpyAsync(dgpoff.p, gpoff.data(), sizeof(int64_t) * gpoff.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaMemcpyAsync(dgeo.p, geo.data(), sizeof(SetGeom) * ns, cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaFuncSetAttribute(k_seg_moments_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msm));
        HDF_COUNT_LAUNCH();
        k_seg_moments_df<<<(unsigned)gitems.size(), 256, msm, st>>>(x, d, dgi.as<SegItem>(), dgpoff.as<int64_t>(),
                                                                     dgeo.as<SetGeom>(), dgpart.as<double>());
        HDF_CUDA(cudaGetLastError());
        cores_all();            // A2 on the host while the device works (before the copy into
                                // pageable memory, which would wait for the kernel)
        std::vector<double> gp(gtot);
        HDF_CUDA(cudaMemcpyAsync(gp.data(), dgpart.p, sizeof(double) * gtot, cudaMemcpyDeviceToHost, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        std::vector<std::vector<double>> moms(ns);
        for (int s = 0; s < ns; ++s) moms[s].assign(2 * geo[s].L + 2, 0.0);
        for (size_t q = 0; q < gitems.size(); ++q) {
            std::vector<double>& m = moms[gitems[q].set];
            for (size_t e = 0; e < m.size(); ++e) m[e] += gp[gpoff[q] + e];
        }
        parallel_for(ns, [&](int s) { gram_from_moments(moms[s], geo[s].L, grams[s]); });
    } else {
    std::vector<SegItem> gitems;
    std::vector<int64_t> gpoff;
    int64_t gtot = 0;
    for (int s = 0; s < ns; ++s) {
        const int LP1 = geo[s].L + 1, npairs = LP1 * (LP1 + 1) / 2;
        for (int64_t i0 = 0; i0 < geo[s].n; i0 += kGramChunk) {
            gitems.push_back({s, 0, geo[s].off + i0, geo[s].off + std::min<int64_t>(geo[s].n, i0 + kGramChunk)});
            gpoff.push_back(gtot);
            gtot += 2 * npairs;
        }
    }
    DevBuf dgi, dgpoff, dgpart;
    HDF_CUDA(dgi.alloc_on(sizeof(SegItem) * gitems.size(), st));
    HDF_CUDA(dgpoff.alloc_on(sizeof(int64_t) * gpoff.size(), st));
    HDF_CUDA(dgpart.alloc_on(sizeof(double) * gtot, st));
    HDF_CUDA(cudaMemcpyAsync(dgi.p, gitems.data(), sizeof(SegItem) * gitems.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(dgpoff.p, gpoff.data(), sizeof(int64_t) * gpoff.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(dgeo.p, geo.data(), sizeof(SetGeom) * ns, cudaMemcpyHostToDevice, st));
    const size_t gsm = sizeof(double) * (dev::kGramTile * (Lmax + 1) + dev::kGramTile);
    HDF_CUDA(cudaFuncSetAttribute(k_seg_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    HDF_COUNT_LAUNCH();
    k_seg_gram<<<(unsigned)gitems.size(), 256, gsm, st>>>(x, d, dgi.as<SegItem>(), dgpoff.as<int64_t>(),
                                                           dgeo.as<SetGeom>(), dgpart.as<double>());
    HDF_CUDA(cudaGetLastError());
    cores_all();                // A2 on the host while the device works (before the copy)
    std::vector<double> gp(gtot);
    HDF_CUDA(cudaMemcpyAsync(gp.data(), dgpart.p, sizeof(double) * gtot, cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < ns; ++s) {
        const int LP1 = geo[s].L + 1;
        grams[s].assign(LP1 * (LP1 + 1), 0.0);
    }
    for (size_t q = 0; q < gitems.size(); ++q) {
        std::vector<double>& G = grams[gitems[q].set];
        for (size_t e = 0; e < G.size(); ++e) G[e] += gp[gpoff[q] + e];
    }
    }
    b->t_ms[2] = now_ms_b() - t0;

    // ---- A3-A4 per set on host threads, tables
    t0 = now_ms_b();
    const int vw = (sizeof(T) == 4) ? 4 : 2;
    std::vector<FactorChoice> fcs(ns);
    std::vector<DeviceTables> tbs(ns);
    std::vector<std::string> errs(ns);
    std::vector<char> ok(ns, 1);
    parallel_for(ns, [&](int t) {
        const int s = by_cost[t];
        plan_factor(grams[s], geo[s].L, d, dps[s].cores, dps[s].drop_budget, false, fcs[s]);
        ok[s] = make_tables(fcs[s], d, geo[s].L, vw, tbs[s], errs[s]) ? 1 : 0;
    });
    for (int s = 0; s < ns; ++s)
        if (!ok[s]) return fail(HDF_ETOOBIG, "hdf_build_batched: set " + std::to_string(s) + ": " + errs[s]);
    *all_reached = true;
    b->info.assign(ns, hdf_info{});
    b->colmap.assign(ns, std::vector<int64_t>());
    b->S_host.assign(ns, std::vector<double>());
    b->uoff.assign(ns + 1, 0);
    b->soff.assign(ns + 1, 0);
    std::vector<int64_t> foff(ns + 1, 0);
    for (int s = 0; s < ns; ++s) {
        hdf_info& I = b->info[s];
        const DegreePlan& dp = dps[s];
        const FactorChoice& fc = fcs[s];
        I.n = geo[s].n; I.d = d; I.precision = b->prec; I.p = dp.p; I.L = dp.L;
        I.reached = dp.reached ? 1 : 0;
        if (!dp.reached) *all_reached = false;
        I.rank = fc.rank; I.ldu = tbs[s].ldU; I.nharm = fc.nH;
        for (int j = 0; j < d; ++j) I.center[j] = geo[s].c[j];
        I.radius = Rs[s]; I.mu2 = mu2[s]; I.cheb_tail = dp.tail; I.tail_budget = dp.tail_budget;
        I.drop_budget = dp.drop_budget; I.dropped_cost = fc.dropped;
        I.err_bound = ((double)geo[s].n * dp.tail + fc.dropped) / ((double)geo[s].n * std::sqrt(mu2[s]));
        for (int k = 0; k <= std::min(dp.L, HDF_MAX_L); ++k) I.s_k[k] = fc.sk[k];
        b->S_host[s] = fc.S;
        b->uoff[s + 1] = b->uoff[s] + geo[s].n * tbs[s].ldU;
        b->soff[s + 1] = b->soff[s] + tbs[s].ldU;
        foff[s + 1] = foff[s] + geo[s].n * std::max(1, tbs[s].nF);
    }
    // arena of per-set tables, each piece 256-byte aligned: offsets first (serial), then the
    // pieces are copied on the worker pool into a pinned staging buffer and uploaded at once
    size_t arena_size = 0;
    struct Piece { const void* src; size_t bytes, off; };
    std::vector<std::vector<Piece>> pieces(ns);
    int cur_set = 0;
    auto put = [&](const void* src, size_t bytes) -> size_t {
        const size_t o = (arena_size + 255) & ~size_t(255);
        arena_size = o + std::max<size_t>(bytes, 16);
        pieces[cur_set].push_back({src, bytes, o});
        return o;
    };
    struct Offs { size_t q0, q1, qc, w, par, ch, qd, yc, gs, ca, cb; int mtp; };
    std::vector<Offs> offs(ns);
    std::vector<T> Sd(b->soff[ns], (T)0);
    // per-set conversions to the bulk type (and the FP32 Qmat pairs) on the worker pool
    struct Conv { std::vector<T> Wt, cA, cB; std::vector<float> qc; int mtp = 0; };
    std::vector<Conv> cv(ns);
    parallel_for(ns, [&](int s) {
        const DeviceTables& tb = tbs[s];
        const FactorChoice& fc = fcs[s];
        Conv& c = cv[s];
        c.Wt.resize(tb.Wt.size());
        c.cA.resize(tb.coefA.size());
        c.cB.resize(tb.coefB.size());
        for (size_t q = 0; q < c.Wt.size(); ++q) c.Wt[q] = (T)tb.Wt[q];
        for (size_t q = 0; q < c.cA.size(); ++q) { c.cA[q] = (T)tb.coefA[q]; c.cB[q] = (T)tb.coefB[q]; }
        if (sizeof(T) == 4) {
            // [Qmat0 | Qmat1] as (hi, lo) float pairs, (L+1) x mtp, odd columns zero in row L
            const int m0 = fc.m[0], m1 = fc.m[1], L = geo[s].L, mtp = ((m0 + m1 + 7) / 8) * 8;
            c.qc.assign((size_t)2 * (L + 1) * std::max(mtp, 8), 0.f);
            auto putq = [&](int l, int o, double v) {
                const float h = (float)v;
                c.qc[2 * ((size_t)l * mtp + o)] = h;
                c.qc[2 * ((size_t)l * mtp + o) + 1] = (float)(v - (double)h);
            };
            for (int l = 0; l < fc.nb[0]; ++l)
                for (int o = 0; o < m0; ++o) putq(l, o, fc.Qmat[0][(size_t)l * m0 + o]);
            for (int l = 0; l < fc.nb[1]; ++l)
                for (int o = 0; o < m1; ++o) putq(l, m0 + o, fc.Qmat[1][(size_t)l * m1 + o]);
            c.mtp = mtp;
        }
    });
    for (int s = 0; s < ns; ++s) {
        cur_set = s;
        const DeviceTables& tb = tbs[s];
        const FactorChoice& fc = fcs[s];
        const std::vector<T>& Wt = cv[s].Wt;
        const std::vector<T>& cA = cv[s].cA;
        const std::vector<T>& cB = cv[s].cB;
        offs[s].q0 = put(fc.Qmat[0].data(), sizeof(double) * fc.Qmat[0].size());
        offs[s].q1 = put(fc.Qmat[1].data(), sizeof(double) * fc.Qmat[1].size());
        offs[s].qc = 0;
        offs[s].mtp = 0;
        if (sizeof(T) == 4) {
            offs[s].qc = put(cv[s].qc.data(), sizeof(float) * cv[s].qc.size());
            offs[s].mtp = cv[s].mtp;
        }
        offs[s].w = put(Wt.data(), sizeof(T) * Wt.size());
        offs[s].par = put(tb.colpar.data(), tb.colpar.size());
        offs[s].ch = put(tb.chains.data(), sizeof(int16_t) * tb.chains.size());
        offs[s].qd = put(tb.qdesc.data(), sizeof(uint32_t) * tb.qdesc.size());
        offs[s].yc = put(tb.ychain.data(), sizeof(int32_t) * tb.ychain.size());
        offs[s].gs = put(tb.gslot.data(), sizeof(int32_t) * tb.gslot.size());
        offs[s].ca = put(cA.data(), sizeof(T) * cA.size());
        offs[s].cb = put(cB.data(), sizeof(T) * cB.size());
        for (int64_t a = 0; a < tb.ldU; ++a) Sd[b->soff[s] + a] = (T)tb.Spad[a];
        b->colmap[s] = tb.colmap;
    }
    std::unique_lock<std::mutex> staging_lock;
    unsigned char* stage = staging_acquire(arena_size, staging_lock);
    std::vector<unsigned char> arena_pageable;
    if (!stage) {                                    // another build holds the pinned buffer
        arena_pageable.resize(arena_size);
        stage = arena_pageable.data();
    }
    parallel_for(ns, [&](int s) {
        for (const Piece& pc : pieces[s])
            if (pc.bytes) std::memcpy(stage + pc.off, pc.src, pc.bytes);
    });
    HDF_CUDA(b->arena.alloc_on(arena_size, st));
    HDF_CUDA(cudaMemcpyAsync(b->arena.p, stage, arena_size, cudaMemcpyHostToDevice, st));
    HDF_CUDA(b->S.alloc_on(sizeof(T) * std::max<int64_t>(1, b->soff[ns]), st));
    HDF_CUDA(cudaMemcpyAsync(b->S.p, Sd.data(), sizeof(T) * Sd.size(), cudaMemcpyHostToDevice, st));
    const size_t ubytes = sizeof(T) * (size_t)std::max<int64_t>(1, b->uoff[ns]);
    if (b->U.alloc_on(ubytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(HDF_ENOMEM, "hdf_build_batched: cannot allocate U (" + std::to_string(ubytes) + " bytes)");
    }
    DevBuf dF;
    if (dF.alloc_on(sizeof(T) * (size_t)std::max<int64_t>(1, foff[ns]), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(HDF_ENOMEM, "hdf_build_batched: cannot allocate the radial factor buffer");
    }
    // set descriptors, shared-memory needs per phase and per set
    const size_t budget = 200 * 1024;
    std::vector<BuildSet> bs(ns);
    size_t smem_rf = 0;                               // radial phase: one tile per item
    int rf_L = 0, rf_mt = 0;                          // largest degree and basis count of the sets
    std::vector<size_t> pw_bytes(ns, 0), fixed_bytes(ns, 0);
    unsigned char* A = b->arena.as<unsigned char>();
    for (int s = 0; s < ns; ++s) {
        const DeviceTables& tb = tbs[s];
        const FactorChoice& fc = fcs[s];
        if (fc.rank == 0) continue;
        dev::RFParams& R = bs[s].rf;
        R.x = x + geo[s].off * d; R.n = geo[s].n; R.d = d;
        for (int j = 0; j < d; ++j) R.c.c[j] = geo[s].c[j];
        R.inv2R = geo[s].inv2R; R.L = geo[s].L;
        R.Qm0 = reinterpret_cast<const double*>(A + offs[s].q0); R.nb0 = fc.nb[0]; R.m0 = fc.m[0];
        R.Qm1 = reinterpret_cast<const double*>(A + offs[s].q1); R.nb1 = fc.nb[1]; R.m1 = fc.m[1];
        R.Wt = A + offs[s].w; R.colpar = A + offs[s].par; R.nF = tb.nF;
        if (sizeof(T) == 4 && offs[s].mtp > 0) {
            R.QC = reinterpret_cast<const float2*>(A + offs[s].qc);
            R.mtp = offs[s].mtp;
            R.kopt = std::min(4, dev::radialF_df_kopt(fc.m[0] + fc.m[1], 256 / 32));   // 2 or 4
        }
        R.F = dF.as<T>() + foff[s]; R.ldF = tb.nF;
        dev::UWParams& P = bs[s].uw;
        P.x = R.x; P.n = R.n; P.d = d; P.c = R.c; P.inv2R = R.inv2R;
        P.L = tb.L_used; P.tri = tb.tri;
        P.chains = reinterpret_cast<const int16_t*>(A + offs[s].ch); P.nH = tb.nH; P.cstride = chain_stride(d);
        P.ychain = reinterpret_cast<const int32_t*>(A + offs[s].yc); P.nYp = tb.nYp;
        P.gslot = reinterpret_cast<const int32_t*>(A + offs[s].gs);
        P.qdesc = reinterpret_cast<const uint32_t*>(A + offs[s].qd); P.nF = tb.nF;
        P.F = R.F; P.ldF = R.ldF;
        P.U = b->U.as<T>() + b->uoff[s]; P.ldU = tb.ldU;
        P.coefA = A + offs[s].ca; P.coefB = A + offs[s].cb;
        const int levels = d - 2;
        fixed_bytes[s] = dev::align16(sizeof(T) * 2 * levels * tb.tri);
        const int pw_pre = dev::uwriter_per_warp(levels, tb.tri, tb.L_used, tb.nYp, tb.nF, true);
        const int pw_fly = dev::uwriter_per_warp(levels, tb.tri, tb.L_used, tb.nYp, tb.nF, false);
        const bool pre = fixed_bytes[s] + sizeof(T) * 8 * (size_t)pw_pre <= budget / 2;
        bs[s].pre = pre ? 1 : 0;
        P.per_warp = pre ? pw_pre : pw_fly;
        pw_bytes[s] = sizeof(T) * (size_t)P.per_warp;
        const size_t need_rf = (sizeof(T) == 4) ? batch_df_tile_smem(geo[s].L, fc.m[0] + fc.m[1], 1)
                                                : dev::radialF_smem(geo[s].L, fc.m[0], fc.m[1], sizeof(T));
        smem_rf = std::max(smem_rf, need_rf);
        rf_L = std::max(rf_L, geo[s].L);
        rf_mt = std::max(rf_mt, fc.m[0] + fc.m[1]);
        if (fixed_bytes[s] + 8 * pw_bytes[s] > budget || need_rf > budget)
            return fail(HDF_ETOOBIG, "hdf_build_batched: per-set tables exceed shared memory");
    }
    // size classes of the U phase: sets by the shared memory a warp needs, classes at a quarter
    // and a half of the largest need
    size_t pw_max = 0;
    for (int s = 0; s < ns; ++s) pw_max = std::max(pw_max, pw_bytes[s]);
    struct UClass { std::vector<int> sets; size_t pw = 0, fixed = 0; int64_t points = 0; };
    std::vector<UClass> ucls(3);
    for (int s = 0; s < ns; ++s) {
        if (fcs[s].rank == 0) continue;
        const int c = (pw_bytes[s] * 4 <= pw_max) ? 0 : (pw_bytes[s] * 2 <= pw_max) ? 1 : 2;
        ucls[c].sets.push_back(s);
        ucls[c].pw = std::max(ucls[c].pw, pw_bytes[s]);
        ucls[c].fixed = std::max(ucls[c].fixed, fixed_bytes[s]);
        ucls[c].points += geo[s].n;
    }
    ucls.erase(std::remove_if(ucls.begin(), ucls.end(), [](const UClass& u) { return u.sets.empty(); }), ucls.end());
    HDF_CUDA(b->dsets.alloc_on(sizeof(BuildSet) * ns, st));
    HDF_CUDA(cudaMemcpyAsync(b->dsets.p, bs.data(), sizeof(BuildSet) * ns, cudaMemcpyHostToDevice, st));
    b->t_ms[3] = now_ms_b() - t0;

    // ---- A5: the radial phase and one U phase per class, shapes from the autotuner
    int nsm = 0, dv = 0;
    HDF_CUDA(cudaGetDevice(&dv));
    HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
    const int nclass = (int)ucls.size();
    DevBuf dcnt;
    HDF_CUDA(dcnt.alloc_on(sizeof(int) * (1 + nclass), st));
    int* cnt = dcnt.as<int>();
    // item lists depend on the shape (tiles per item, points per item): built per candidate
    auto radial_items = [&](int tpi) {
        std::vector<int2> it;
        const int64_t per = (int64_t)tpi * dev::kFTile;
        for (int s = 0; s < ns; ++s)
            if (fcs[s].rank > 0)
                for (int64_t t = 0; t * per < geo[s].n; ++t) it.push_back(make_int2(s, (int)t));
        return it;
    };
    auto urow_items = [&](const UClass& u, int ppi) {
        std::vector<int2> it;
        for (int s : u.sets)
            for (int64_t t = 0; t * ppi < geo[s].n; ++t) it.push_back(make_int2(s, (int)t));
        return it;
    };
    struct Shape { int a, per_sm; };                  // (tiles or warps, CTAs per SM)
    struct Plan { DevBuf items; int nitems = 0; int a = 0, per_sm = 1, pts = 0; size_t smem = 0; };
    std::vector<Plan> plans(1 + nclass);
    // FP32 radial phase: shared memory for `a` tiles per item (a basis buffer per tile)
    auto smem_rf_of = [&](int a) -> size_t {
        return (sizeof(T) == 4) ? std::max(smem_rf, batch_df_tile_smem(rf_L, rf_mt, a)) : smem_rf;
    };
    HDF_CUDA(cudaFuncSetAttribute(k_batch_radial<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)std::min(budget, smem_rf_of(8))));
    HDF_CUDA(cudaFuncSetAttribute(k_batch_urows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget));
    auto set_plan = [&](int ph, int a) -> hdf_status {
        Plan& P = plans[ph];
        std::vector<int2> it;
        if (ph == 0) {
            it = radial_items(a);
            P.smem = smem_rf_of(a);
            P.pts = a;
        } else {
            const UClass& u = ucls[ph - 1];
            P.pts = 8 * a;                             // points per item: 8 per warp
            it = urow_items(u, P.pts);
            P.smem = dev::align16(u.fixed + (size_t)a * u.pw);
        }
        P.a = a;
        P.nitems = (int)it.size();
        HDF_CUDA(P.items.alloc_on(sizeof(int2) * std::max<size_t>(1, it.size()), st));
        if (!it.empty()) HDF_CUDA(cudaMemcpyAsync(P.items.p, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaStreamSynchronize(st));      // the host item list is released on return
        return HDF_OK;
    };
    auto launch = [&](int ph, int per_sm) -> hdf_status {
        const Plan& P = plans[ph];
        if (P.nitems == 0) return HDF_OK;
        HDF_CUDA(cudaMemsetAsync(cnt + ph, 0, sizeof(int), st));
        HDF_COUNT_LAUNCH();
        if (ph == 0)
            k_batch_radial<T><<<nsm * per_sm, 256, P.smem, st>>>(b->dsets.as<BuildSet>(), P.items.as<int2>(), P.nitems,
                                                                cnt + ph, P.pts);
        else
            k_batch_urows<T><<<nsm * per_sm, 32 * P.a, P.smem, st>>>(b->dsets.as<BuildSet>(), P.items.as<int2>(),
                                                                     P.nitems, cnt + ph, P.pts);
        HDF_CUDA(cudaGetLastError());
        return HDF_OK;
    };
    auto occupancy = [&](int ph, int a, size_t smem) -> int {
        int occ = 0;
        if (ph == 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_radial<T>, 256, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_urows<T>, 32 * a, smem);
        cudaGetLastError();
        return occ;
    };
    cudaEvent_t e0, e1;
    HDF_CUDA(cudaEventCreate(&e0));
    HDF_CUDA(cudaEventCreate(&e1));
    struct EvG { cudaEvent_t a, b; ~EvG() { cudaEventDestroy(a); cudaEventDestroy(b); } } evg{e0, e1};
    for (int ph = 0; ph <= nclass; ++ph) {
        // candidates: radial tiles per item {1, 2, 4, 8}; U warps per CTA {8, 16, 32} within the
        // class's shared memory; CTAs per SM from 1 to the occupancy limit
        std::vector<int> as;
        int64_t work = 0;
        if (ph == 0) {
            for (int a : {1, 2, 4, 8})
                if (smem_rf_of(a) <= budget) as.push_back(a);
            for (int s = 0; s < ns; ++s) work += geo[s].n;
        } else {
            const UClass& u = ucls[ph - 1];
            for (int a : {8, 16, 32})
                if (u.fixed + (size_t)a * u.pw <= budget) as.push_back(a);
            work = u.points;
        }
        int bucket = 0;
        while ((int64_t(1) << (bucket + 1)) <= std::max<int64_t>(1, work / 1024)) ++bucket;
        char key[160];
        if (ph == 0)
            std::snprintf(key, sizeof(key), "batch_radial_v3:sm%d:d%d:%s:smem%zu:work2^%d", nsm, d,
                          sizeof(T) == 4 ? "fp32" : "fp64", smem_rf / 4096, bucket);
        else
            std::snprintf(key, sizeof(key), "batch_urows_v1:sm%d:d%d:%s:pw%zu:fixed%zu:work2^%d", nsm, d,
                          sizeof(T) == 4 ? "fp32" : "fp64", ucls[ph - 1].pw / 256, ucls[ph - 1].fixed / 1024, bucket);
        int code = 0;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto m = tune_load();
            auto itk = m.find(key);
            if (itk != m.end()) code = itk->second;
        }
        Shape best{0, 0};
        if (code > 0) {
            best = Shape{code / 100, code % 100};
            bool valid = std::find(as.begin(), as.end(), best.a) != as.end();
            if (valid) {
                if (hdf_status e = set_plan(ph, best.a); e != HDF_OK) return e;
                valid = best.per_sm >= 1 && best.per_sm <= std::max(1, occupancy(ph, best.a, plans[ph].smem));
            }
            if (!valid) best = Shape{0, 0};
        }
        if (best.a == 0) {
            float best_ms = 1e30f;
            for (int a : as) {
                if (hdf_status e = set_plan(ph, a); e != HDF_OK) return e;
                const int occ = std::max(1, occupancy(ph, a, plans[ph].smem));
                for (int per_sm = 1; per_sm <= occ; ++per_sm) {
                    float ms_min = 1e30f;
                    for (int rep = 0; rep < 2; ++rep) {           // the faster of two runs counts
                        HDF_CUDA(cudaEventRecord(e0, st));
                        if (hdf_status e = launch(ph, per_sm); e != HDF_OK) return e;
                        HDF_CUDA(cudaEventRecord(e1, st));
                        HDF_CUDA(cudaEventSynchronize(e1));
                        float ms = 0.f;
                        HDF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                        ms_min = std::min(ms_min, ms);
                    }
                    if (ms_min < best_ms) { best_ms = ms_min; best = Shape{a, per_sm}; }
                }
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto m = tune_load();
            m[key] = best.a * 100 + best.per_sm;
            tune_store(m);
        }
        if (plans[ph].a != best.a)
            if (hdf_status e = set_plan(ph, best.a); e != HDF_OK) return e;
        plans[ph].per_sm = best.per_sm;
    }
    b->grid_build = nsm * plans[0].per_sm;
    // the device work of A5 as one CUDA graph: counters, the radial phase, the U phases, with
    // events around the two halves; recorded on the batch's capture stream and launched on st
    if (!b->cap) HDF_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    cudaStream_t keep = st;
    st = b->cap;                                   // launch() enqueues on st
    HDF_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    hdf_status cs = HDF_OK;
    for (int ph = 0; ph <= nclass && cs == HDF_OK; ++ph) cs = launch(ph, plans[ph].per_sm);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    st = keep;
    if (cs != HDF_OK) { if (graph) cudaGraphDestroy(graph); return cs; }
    if (ce != cudaSuccess) return fail(HDF_ECUDA, std::string("hdf_build_batched: graph capture: ") + cudaGetErrorString(ce));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return fail(HDF_ECUDA, std::string("hdf_build_batched: graph: ") + cudaGetErrorString(ie));
    HDF_CUDA(cudaEventRecord(e0, st));
    const cudaError_t le = cudaGraphLaunch(exec, st);
    HDF_CUDA(cudaEventRecord(e1, st));
    const cudaError_t se = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (le != cudaSuccess || se != cudaSuccess)
        return fail(HDF_ECUDA, std::string("hdf_build_batched: graph launch: ") + cudaGetErrorString(le != cudaSuccess ? le : se));
    float ms = 0.f;
    HDF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    b->t_ms[4] = 0.0;                              // the radial phase is inside the graph of index 5
    b->t_ms[5] = ms;
    b->nclass = nclass;
    b->t_ms[HDF_NPHASE - 1] = now_ms_b() - t_start;
    return HDF_OK;
}

template <typename T>
static hdf_status batch_matvec_t(hdf_batch* b, const T* V, int64_t ldv, int c, T* Y, int64_t ldy, cudaStream_t st) {
    const int ns = b->nsets;
    if (c != b->mv_c) {
        // work space and items for this column count
        if (b->mv_exec) { cudaGraphExecDestroy(b->mv_exec); b->mv_exec = nullptr; }
        std::vector<MvSet> ms(ns);
        std::vector<MvItem> iu, ir, iw;
        const int ct = ct_for(c);
        const bool skinny = sizeof(T) == 4 && ct <= 16;
        int AB = (ct == 1) ? 256 : 128, RB = (ct == 1) ? 256 : 128;
        if (skinny) {                     // the streaming kernels' columns / rows per item
            AB = (ct <= 8) ? kPipeCols : SkinnyShape<16>::AB;
            RB = 32;                      // k_batch_uw_b: one 32-row tile per item (from the set table)
        }
        int64_t ptot = 0, wtot = 0;
        std::vector<int64_t> poff(ns), woff(ns);
        for (int s = 0; s < ns; ++s) {
            const int64_t n = b->info[s].n, r = (b->info[s].rank > 0) ? b->info[s].ldu : 0;   // padded width
            ms[s].n = n; ms[s].r = r; ms[s].ldU = b->info[s].ldu; ms[s].off = b->off[s];
            ms[s].chunk = 4096;
            ms[s].nchunk = (int)std::max<int64_t>(1, (n + ms[s].chunk - 1) / ms[s].chunk);
            poff[s] = ptot;
            ptot += (int64_t)ms[s].nchunk * c * std::max<int64_t>(1, r);
            woff[s] = wtot;
            ms[s].ldw = skinny ? ct : c;
            wtot += std::max<int64_t>(1, r) * ms[s].ldw;
            if (r == 0) continue;
            for (int q = 0; q < ms[s].nchunk; ++q)
                for (int64_t bl = 0; bl < (r + AB - 1) / AB; ++bl) iu.push_back({s, q, bl});
            for (int64_t bl = 0; bl < (r + 255) / 256; ++bl) ir.push_back({s, 0, bl});
            if (!skinny)                  // the FP32 U W kernel locates its tiles from the set table
                for (int64_t bl = 0; bl < (n + RB - 1) / RB; ++bl) iw.push_back({s, 0, bl});
        }
        HDF_CUDA(b->mvpart.alloc_on(sizeof(double) * std::max<int64_t>(1, ptot), st));
        HDF_CUDA(b->mvW.alloc_on(sizeof(T) * std::max<int64_t>(1, wtot), st));
        for (int s = 0; s < ns; ++s) {
            ms[s].U = b->U.as<T>() + b->uoff[s];
            ms[s].S = b->S.as<T>() + b->soff[s];
            ms[s].part = b->mvpart.as<double>() + poff[s];
            ms[s].W = b->mvW.as<T>() + woff[s];
        }
        if (skinny) {
            // the U W kernel's tensor maps: set s's U as ldU x n FP32, 32 x 32 boxes, 128-byte swizzle
            std::vector<CUtensorMap> maps(ns);
            for (int s = 0; s < ns; ++s) {
                const int64_t n = std::max<int64_t>(1, b->info[s].n), ld = std::max<int64_t>(4, b->info[s].ldu);
                if (!encode_map_f32(&maps[s], b->U.as<T>() + b->uoff[s], (uint64_t)ld, (uint64_t)n,
                                    (uint64_t)ld * sizeof(T), 32, 32, true))
                    return fail(HDF_ECUDA, "hdf_batch_matvec: cannot encode a tensor map");
            }
            HDF_CUDA(b->umaps.alloc(sizeof(CUtensorMap) * ns));
            HDF_CUDA(cudaMemcpyAsync(b->umaps.p, maps.data(), sizeof(CUtensorMap) * ns, cudaMemcpyHostToDevice, st));
            std::vector<BwSet> bw(ns);
            int64_t tiles = 0;
            for (int s = 0; s < ns; ++s) {
                bw[s].W = reinterpret_cast<const float*>(b->mvW.as<T>() + woff[s]);
                bw[s].off = b->off[s];
                bw[s].tile0 = tiles;
                bw[s].n = (int)ms[s].n;
                bw[s].r = (int)ms[s].r;
                if (ms[s].r > 0) tiles += (ms[s].n + 31) / 32;      // rank-0 sets: no items
            }
            b->n_bw = (int)tiles;
            HDF_CUDA(b->bwsets.alloc(sizeof(BwSet) * ns));
            HDF_CUDA(cudaMemcpyAsync(b->bwsets.p, bw.data(), sizeof(BwSet) * ns, cudaMemcpyHostToDevice, st));
            HDF_CUDA(cudaStreamSynchronize(st));      // the host table is released on return
        }
        HDF_CUDA(b->mvsets.alloc_on(sizeof(MvSet) * ns, st));
        HDF_CUDA(b->mvitems_utv.alloc_on(sizeof(MvItem) * std::max<size_t>(1, iu.size()), st));
        HDF_CUDA(b->mvitems_red.alloc_on(sizeof(MvItem) * std::max<size_t>(1, ir.size()), st));
        HDF_CUDA(b->mvitems_uw.alloc_on(sizeof(MvItem) * std::max<size_t>(1, iw.size()), st));
        HDF_CUDA(b->counters.alloc_on(sizeof(int) * 2, st));
        if (!b->derr.p) {
            HDF_CUDA(b->derr.alloc(sizeof(int)));
            HDF_CUDA(cudaMemsetAsync(b->derr.p, 0, sizeof(int), st));
        }
        HDF_CUDA(cudaMemcpyAsync(b->mvsets.p, ms.data(), sizeof(MvSet) * ns, cudaMemcpyHostToDevice, st));
        if (!iu.empty()) HDF_CUDA(cudaMemcpyAsync(b->mvitems_utv.p, iu.data(), sizeof(MvItem) * iu.size(), cudaMemcpyHostToDevice, st));
        if (!ir.empty()) HDF_CUDA(cudaMemcpyAsync(b->mvitems_red.p, ir.data(), sizeof(MvItem) * ir.size(), cudaMemcpyHostToDevice, st));
        if (!iw.empty()) HDF_CUDA(cudaMemcpyAsync(b->mvitems_uw.p, iw.data(), sizeof(MvItem) * iw.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        b->n_utv = (int)iu.size();
        b->n_red = (int)ir.size();
        b->n_uw = skinny ? b->n_bw : (int)iw.size();
        b->mv_c = c;
    }
    if (!b->mv_exec || b->mv_V != (const void*)V || b->mv_Y != (void*)Y || b->mv_ldv != ldv || b->mv_ldy != ldy) {
        if (b->mv_exec) { cudaGraphExecDestroy(b->mv_exec); b->mv_exec = nullptr; }
        if (!b->cap) HDF_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        int nsm = 0, dv = 0;
        HDF_CUDA(cudaGetDevice(&dv));
        HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
        const int ct = ct_for(c);
        const bool skinny = sizeof(T) == 4 && ct <= 16;
        int occ_u = 1, occ_w = 1;
        if (skinny) {
            switch (ct) {
#define HDF_B_OCC(CT)                                                                                             \
    case CT:                                                                                                      \
        HDF_CUDA(cudaFuncSetAttribute(k_batch_utv_p<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                      (int)utv_pipe_smem<CT>()));                                                 \
        HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, k_batch_utv_p<CT>, 256, utv_pipe_smem<CT>())); \
        HDF_CUDA(cudaFuncSetAttribute(k_batch_uw_b<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize,             \
                                      (int)bw_smem<CT>()));                                                       \
        HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_batch_uw_b<CT>, 32 * kBwWarps,          \
                                                               bw_smem<CT>()));                                   \
        break;
                HDF_B_OCC(1) HDF_B_OCC(2) HDF_B_OCC(4) HDF_B_OCC(8)
#undef HDF_B_OCC
                case 16:
                    HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, k_batch_utv_s<16>, 256, 0));
                    HDF_CUDA(cudaFuncSetAttribute(k_batch_uw_b<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)bw_smem<16>()));
                    HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, k_batch_uw_b<16>, 32 * kBwWarps,
                                                                           bw_smem<16>()));
                    break;
            }
        }
        HDF_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(b->counters.p, 0, sizeof(int) * 2, b->cap);
        const MvSet* S = b->mvsets.as<MvSet>();
        int* cnt = b->counters.as<int>();
        if (skinny) {
            switch (ct) {
#define HDF_B_SK(CT, UTV, UW, SU, SW)                                                                             \
    case CT:                                                                                                      \
        if (b->n_utv)                                                                                             \
            UTV<<<nsm * std::max(occ_u, 1), 256, SU, b->cap>>>(                                                   \
                S, b->mvitems_utv.as<MvItem>(), b->n_utv, cnt, reinterpret_cast<const float*>(V), ldv, c);        \
        if (b->n_red) k_batch_reduce<T><<<b->n_red, 256, 0, b->cap>>>(S, b->mvitems_red.as<MvItem>(), c);          \
        if (b->n_uw)                                                                                              \
            UW<<<nsm * std::max(occ_w, 1), 32 * kBwWarps, SW, b->cap>>>(                                          \
                b->bwsets.as<BwSet>(), ns, b->n_uw, cnt + 1, b->umaps.as<CUtensorMap>(),                          \
                reinterpret_cast<float*>(Y), ldy, c, b->derr.as<int>());                                          \
        break;
                HDF_B_SK(1, k_batch_utv_p<1>, k_batch_uw_b<1>, utv_pipe_smem<1>(), bw_smem<1>())
                HDF_B_SK(2, k_batch_utv_p<2>, k_batch_uw_b<2>, utv_pipe_smem<2>(), bw_smem<2>())
                HDF_B_SK(4, k_batch_utv_p<4>, k_batch_uw_b<4>, utv_pipe_smem<4>(), bw_smem<4>())
                HDF_B_SK(8, k_batch_utv_p<8>, k_batch_uw_b<8>, utv_pipe_smem<8>(), bw_smem<8>())
                HDF_B_SK(16, k_batch_utv_s<16>, k_batch_uw_b<16>, 0, bw_smem<16>())
#undef HDF_B_SK
            }
        } else
        switch (ct) {
#define HDF_B_MV(CT)                                                                                              \
    case CT:                                                                                                      \
        if (b->n_utv) k_batch_utv<T, CT><<<nsm * 3, 256, 0, b->cap>>>(S, b->mvitems_utv.as<MvItem>(), b->n_utv,   \
                                                                        cnt, V, ldv, c);                          \
        if (b->n_red) k_batch_reduce<T><<<b->n_red, 256, 0, b->cap>>>(S, b->mvitems_red.as<MvItem>(), c);          \
        if (b->n_uw) k_batch_uw<T, CT><<<nsm * 3, 256, 0, b->cap>>>(S, b->mvitems_uw.as<MvItem>(), b->n_uw,       \
                                                                      cnt + 1, Y, ldy, c);                        \
        break;
        HDF_B_MV(1) HDF_B_MV(2) HDF_B_MV(4) HDF_B_MV(8) HDF_B_MV(16) HDF_B_MV(32) HDF_B_MV(64) }
#undef HDF_B_MV
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
        if (ce != cudaSuccess) return fail(HDF_ECUDA, std::string("hdf_batch_matvec: capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&b->mv_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(HDF_ECUDA, std::string("hdf_batch_matvec: instantiate: ") + cudaGetErrorString(ce));
        b->mv_V = V; b->mv_Y = Y; b->mv_ldv = ldv; b->mv_ldy = ldy;
    }
    hdf::g_launches.fetch_add((b->n_utv ? 1 : 0) + (b->n_red ? 1 : 0) + (b->n_uw ? 1 : 0), std::memory_order_relaxed);
    HDF_CUDA(cudaGraphLaunch(b->mv_exec, st));
    return HDF_OK;
}

extern "C" {

hdf_status hdf_batch_device_errors(const hdf_batch* b, int* flag) {
    if (!b || !flag) return fail(HDF_EINVAL, "hdf_batch_device_errors: null argument");
    *flag = 0;
    if (!b->derr.p) return HDF_OK;
    HDF_CUDA(cudaDeviceSynchronize());
    int fl = 0;
    HDF_CUDA(cudaMemcpy(&fl, b->derr.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (fl) HDF_CUDA(cudaMemset(b->derr.p, 0, sizeof(int)));
    *flag = fl ? 1 : 0;
    return HDF_OK;
}

hdf_status hdf_build_batched(int nsets, const int64_t* offsets, const double* x_dev, int d, hdf_kernel kernel,
                             const double* lengthscales, double tol, hdf_precision prec, const hdf_options* opt,
                             hdf_stream stream, hdf_batch** out) {
    if (out) *out = nullptr;
    if (!out || !offsets || !x_dev || !lengthscales || nsets < 1 || d < 3 || d > HDF_MAX_D || kernel < 0 ||
        kernel > 3 || !(tol > 0 && tol < 1) || (prec != HDF_FP64 && prec != HDF_FP32))
        return fail(HDF_EINVAL, "hdf_build_batched: bad argument");
    if (offsets[0] != 0) return fail(HDF_EINVAL, "hdf_build_batched: offsets[0] must be 0");
    for (int s = 0; s < nsets; ++s) {
        if (offsets[s + 1] <= offsets[s]) return fail(HDF_EINVAL, "hdf_build_batched: every set needs >= 1 point");
        if (!(lengthscales[s] > 0)) return fail(HDF_EINVAL, "hdf_build_batched: lengthscales must be > 0");
    }
    int p_max = 64;
    double eta = 1.0;
    if (opt) {
        if (opt->p_max > 0) p_max = opt->p_max;
        if (opt->eta > 0) eta = opt->eta;
    }
    if (p_max > 2 * HDF_MAX_L) return fail(HDF_ETOOBIG, "hdf_build_batched: p_max > 128");
    p_max -= p_max % 2;
    hdf_batch* b = new hdf_batch();
    b->nsets = nsets;
    b->d = d;
    b->prec = prec;
    b->kernel = kernel;
    b->tol = tol;
    b->esz = (prec == HDF_FP64) ? 8 : 4;
    b->off.assign(offsets, offsets + nsets + 1);
    std::vector<double> ells(lengthscales, lengthscales + nsets);
    bool reached = true;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const hdf_status s = (prec == HDF_FP64) ? batch_build_t<double>(b, x_dev, ells, tol, eta, p_max, st, &reached)
                                             : batch_build_t<float>(b, x_dev, ells, tol, eta, p_max, st, &reached);
    if (s != HDF_OK) { delete b; return s; }
    *out = b;
    if (!reached) {
        fail(HDF_ETOL_UNREACHABLE, "hdf_build_batched: some sets were capped at p_max");
        return HDF_ETOL_UNREACHABLE;
    }
    return HDF_OK;
}

hdf_status hdf_batch_info(const hdf_batch* b, int set, hdf_info* info) {
    if (!b || !info || set < 0 || set >= b->nsets) return fail(HDF_EINVAL, "hdf_batch_info: bad argument");
    *info = b->info[set];
    return HDF_OK;
}

hdf_status hdf_batch_timings(const hdf_batch* b, double* t_ms) {
    if (!b || !t_ms) return fail(HDF_EINVAL, "hdf_batch_timings: bad argument");
    for (int q = 0; q < HDF_NPHASE; ++q) t_ms[q] = b->t_ms[q];
    return HDF_OK;
}

hdf_status hdf_batch_matvec(hdf_batch* b, const void* V_dev, int64_t ldv, int ncols, void* Y_dev, int64_t ldy,
                            hdf_stream stream) {
    const int64_t ntot = b ? b->off[b->nsets] : 0;
    if (!b || !V_dev || !Y_dev || ncols < 1 || ncols > 64 || ldv < ntot || ldy < ntot)
        return fail(HDF_EINVAL, "hdf_batch_matvec: bad argument (1 <= ncols <= 64)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (b->prec == HDF_FP64)
        return batch_matvec_t<double>(b, (const double*)V_dev, ldv, ncols, (double*)Y_dev, ldy, st);
    return batch_matvec_t<float>(b, (const float*)V_dev, ldv, ncols, (float*)Y_dev, ldy, st);
}

hdf_status hdf_batch_export(const hdf_batch* b, int set, void* U_host, double* S_host) {
    if (!b || set < 0 || set >= b->nsets) return fail(HDF_EINVAL, "hdf_batch_export: bad argument");
    const hdf_info& I = b->info[set];
    if (U_host && I.rank > 0) {
        std::vector<unsigned char> pad((size_t)I.n * I.ldu * b->esz);
        const unsigned char* src = b->U.as<unsigned char>() + b->uoff[set] * b->esz;
        HDF_CUDA(cudaMemcpy(pad.data(), src, pad.size(), cudaMemcpyDeviceToHost));
        unsigned char* out = static_cast<unsigned char*>(U_host);
        const std::vector<int64_t>& cm = b->colmap[set];
        for (int64_t i = 0; i < I.n; ++i)
            for (int64_t t = 0; t < I.rank; ++t)
                std::memcpy(out + ((size_t)i * I.rank + t) * b->esz, pad.data() + ((size_t)i * I.ldu + cm[t]) * b->esz,
                            b->esz);
    }
    if (S_host && I.rank > 0) std::memcpy(S_host, b->S_host[set].data(), sizeof(double) * I.rank);
    return HDF_OK;
}

void hdf_batch_free(hdf_batch* b) {
    if (!b) return;
    // the buffers come from the stream-ordered pool of the build / matvec streams: make sure no
    // kernel still reads them, then return them on the legacy stream
    cudaDeviceSynchronize();
    for (DevBuf* d : {&b->U, &b->S, &b->arena, &b->dsets, &b->mvsets, &b->mvitems_utv, &b->mvitems_red,
                      &b->mvitems_uw, &b->mvpart, &b->mvW, &b->counters})
        d->st = nullptr;
    delete b;
}

}  // extern "C"
