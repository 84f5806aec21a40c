// Internal declarations shared by the library's translation units (not part of the ABI):
// the factor object, error reporting, the launch counter and a device-buffer owner.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <string>
#include <vector>

#include "../../include/hdf.h"

struct DevBuf;

struct CUtensorMap_st;

namespace hdf {

// Sets the thread-local message returned by hdf_last_error and returns s.
hdf_status fail(hdf_status s, const std::string& msg);
// Counter of kernel launches reported by hdf_launch_count.
extern std::atomic<long long> g_launches;

// Tensor-core GEMMs of the FP32 matvec (tc_gemm.cu).  tc_bn: padded N (16, 32, 64) or 0.
int tc_bn(int c);
// 2-D FP32 tensor map for TMA: `inner` contiguous elements by `outer` rows of stride_bytes, box
// {box_inner, box_outer}, zero fill out of bounds, 128-byte swizzle if asked; false when the
// driver entry point is missing or refuses the arguments.
bool encode_map_f32(CUtensorMap_st* map, const void* ptr, uint64_t inner, uint64_t outer, uint64_t stride_bytes,
                    uint32_t box_inner, uint32_t box_outer, bool swizzle128);
size_t tc_work_floats(int64_t n, int64_t r, int c);
// Rows per chunk (a multiple of 32) and the number of chunks of the tensor-core U^T V split;
// tc_utv writes exactly that many partial slices.
void tc_utv_split(int64_t n, int64_t r, int64_t* chunk, int* nchunk);
// part32: the partial sums are written as FP32 into the same buffer (each is an FP32 register
// sum, so nothing is lost); else FP64.
hdf_status tc_utv(const float* U, int64_t ldU, int64_t n, int64_t r, const float* V, int64_t ldv, int c, int64_t chunk,
                  double* part, float* work, int* err, cudaStream_t st, bool part32 = false);
hdf_status tc_gram(const float* U, int64_t ldU, int64_t n, int64_t r, double* G, int* err, cudaStream_t st);
// Matrix-free products on the tensor cores (tc_gemm.cu) over the device views of a matrix-free
// factor: the U^T V tiles (m, j0, n0) and the U W phases (m, n0, K steps, B row) for c columns
// (tc_mf_lists), partial sums of U^T V into part (chunks x c x r, zeroed by the call), and Y = U W.
struct MfTcView {
    const float* Z; int ldZ;
    const float* A0F; int ldA;
    int64_t n, r;
    const int* zoff; const int* zcnt; const int* aoff; const int* acnt; const int64_t* wcol;
};
int tc_mf_cp(int c);
void tc_mf_lists(const std::vector<int>& zcnt, const std::vector<int>& acnt, int c, std::vector<int4>& tiles,
                 std::vector<int4>& phases, int* kpad);
// Points per chunk and chunks of the tensor-core U^T V partial sums (part holds nchunk x c x r).
void tc_mf_chunks(int64_t n, int ntiles, int64_t* chunk, int* nchunk);
hdf_status tc_mf_utv(const MfTcView& v, const int4* tiles, int ntiles, const float* V, int64_t ldv, int c, double* part,
                     int* nchunk, int* err, cudaStream_t st);
hdf_status tc_mf_uw(const MfTcView& v, const int4* phases, int nphase, int kpad, const float* W, int c, float* Y,
                    int64_t ldy, int* err, cudaStream_t st);
// Work-wait limit (clock cycles) of the tensor-core kernels on the current device.
hdf_status set_wait_limit(long long cycles, long long* previous);
// Mismatches of the tensor-core operand rounding (tf32_hi) against cvt.rna.tf32.f32 over all
// finite FP32 values: bad2[0] below 2^127 in magnitude, bad2[1] in the top binade.
hdf_status tf32_check(unsigned long long* bad2);
// HDF_ETIMEOUT (and the flag cleared) if a kernel on f gave up a bounded wait since the last
// check; synchronises the device.
hdf_status take_device_error(const hdf_factor* f);
// Matrix-free products (mfree.cu): partial sums of U^T V (c <= 64) into part (allocated by the
// call from the stream-ordered pool: *nchunk chunks of c x ldu, FP64) and Y = U W (W: ldu x c
// row-major, c <= 64).  FP32 factors run on the tensor cores unless HDF_FLAG_CUDA_CORES.
template <typename T>
hdf_status mf_utv(const hdf_factor* f, const T* V, int64_t ldv, int c, DevBuf& part, int* nchunk, cudaStream_t st);
template <typename T>
hdf_status mf_uw(const hdf_factor* f, const T* W, int c, T* Y, int64_t ldy, cudaStream_t st);
hdf_status tc_uw(const float* U, int64_t ldU, int64_t n, int64_t r, const float* W, int c, float alpha, const float* B,
                 int64_t ldb, float beta, float* Y, int64_t ldy, float* work, int* err, cudaStream_t st);

// W = S_scale .* (U^T V) for one group of c <= 64 columns: W (r x c row-major, bulk) and/or
// Wd (r x c, FP64).  S_scale may be null (no scaling).  Allocates its partial sums.
template <typename T>
hdf_status utv_reduce(const hdf_factor* f, const T* V, int64_t ldv, int c, const T* S_scale, T* W, double* Wd,
                      cudaStream_t st);

}  // namespace hdf

#define HDF_COUNT_LAUNCH() hdf::g_launches.fetch_add(1, std::memory_order_relaxed)

// A failed CUDA call returns HDF_ECUDA, or HDF_ENOMEM when it could not allocate memory.
#define HDF_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (e_ == cudaErrorMemoryAllocation) cudaGetLastError();                          \
            return hdf::fail(e_ == cudaErrorMemoryAllocation ? HDF_ENOMEM : HDF_ECUDA,        \
                             std::string(#call) + ": " + cudaGetErrorString(e_));             \
        }                                                                                     \
    } while (0)

namespace hdf {
// Host-side fault injection for tests (hdf_debug_fail_alloc): while g_alloc_fail_at >= 0 each
// device allocation through DevBuf counts it down, and the one that finds it at 0 reports
// cudaErrorMemoryAllocation without allocating (the countdown then stays off at -1).
extern std::atomic<long long> g_alloc_fail_at;
inline bool injected_alloc_failure() {
    long long v = g_alloc_fail_at.load(std::memory_order_relaxed);
    while (v >= 0)
        if (g_alloc_fail_at.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}
// Keeps freed stream-ordered allocations of the current device in its default memory pool
// (release threshold raised once per device), so that repeated builds and products reuse
// memory instead of mapping it again.
void pool_setup();
}  // namespace hdf

// Owns one device allocation.  alloc(): synchronous cudaMalloc; alloc_on(): stream-ordered
// from the device's memory pool, freed on the same stream (no device-wide synchronisation).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaStream_t st = nullptr;
    bool pooled = false;
    ~DevBuf() { release(); }
    void release() {
        if (!p) return;
        if (pooled) cudaFreeAsync(p, st); else cudaFree(p);
        p = nullptr;
    }
    cudaError_t alloc(size_t b) {
        release();
        bytes = b;
        pooled = false;
        if (b && hdf::injected_alloc_failure()) return cudaErrorMemoryAllocation;
        return b ? cudaMalloc(&p, b) : cudaSuccess;
    }
    cudaError_t alloc_on(size_t b, cudaStream_t s) {
        release();
        hdf::pool_setup();
        bytes = b;
        pooled = true;
        st = s;
        if (b && hdf::injected_alloc_failure()) return cudaErrorMemoryAllocation;
        return b ? cudaMallocAsync(&p, b, s) : cudaSuccess;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// What the build decided, kept for the adjoint (frozen structure) and for diagnostics.
struct FactorPlan {
    int d = 0, L = 0, L_used = 0, tri = 0, nF = 0, nH = 0, mmax = 0, p_max = 0;
    int nb[2] = {0, 0}, m[2] = {0, 0};
    double c[HDF_MAX_D] = {};
    double inv2R = 0.0;
    std::vector<double> Rf[2], Qmat[2];        // basis factor and its inverse map, per parity
    std::vector<std::vector<double>> Wk;       // kept eigenvectors per k (m x s_k, row-major)
    std::vector<int> sk, fbase, cbase, hbase;  // per k: kept count, F column, U column, harmonic bases
    // device copies: Qmat0, Qmat1 (FP64), Wt (m_max x nF, bulk), colk (F column -> k),
    // chains (nH x (d-1) int16), hk (harmonic -> k), ktab (per k: fbase, s_k, cbase, |H_k|, hbase,
    // padded |H_k|), qdesc (chunk descriptors), ychain (padded harmonic slots -> chain),
    // coefA/coefB (level recurrences, bulk)
    DevBuf dQ0, dQ1, dQC, dW, dcolk, dchains, dhk, dktab, dqdesc, dychain, dgslot, dA, dB;
    std::vector<int64_t> colmap;               // padded column of each true column of U
    std::vector<double> Spad;                  // S on the padded columns (0 on padding)
    // d S_k / d l (s_k x s_k), computed on first use by the adjoint
    std::vector<std::vector<double>> dSk;
    bool have_dS = false;
};

// Matrix-free form (mfree.cu): U is not stored; per point the Z row (tails of the harmonic
// chains) and the A0F row (first level factor times radial factor) replace the U row, and the
// products run over them.  Host and device copies of the layout of planner.h's FreeTables.
struct FreeFactor {
    static constexpr int64_t kChunk = 8192;          // points per partial sum of U^T V
    struct Items {                                  // U^T V tiles for one column count
        DevBuf buf;
        int count = 0;
    };
    bool on = false;
    int L_used = 0, nZ = 0, ldZ = 0, nA = 0, ldA = 0;
    DevBuf Z, A0F;                                  // n x ldZ, n x ldA (bulk type)
    DevBuf dzoff, dzcnt, daoff, dacnt, dwcol;
    std::vector<int> zoff, zcnt, aoff, acnt;
    std::unique_ptr<Items> items[128];              // FP32 c = 1..64, then FP64
    struct TcLists {                                // tensor-core tiles and phases for one column count
        DevBuf tiles, phases;
        int ntiles = 0, nphase = 0, kpad = 0;
    };
    std::unique_ptr<TcLists> tc[65];
    // true if a U of ubytes bytes may be stored on the current device (at most 80% of its memory)
    static bool fits(int64_t ubytes);
};

struct hdf_factor {
    FactorPlan plan;
    FreeFactor mf;
    hdf_info info{};
    int kernel = 0;
    double ell = 0, tol = 0;
    int prec = 0;
    size_t esz = 8;                 // bytes per bulk element
    DevBuf U, S;                    // U n x ldu, S rank (bulk type)
    std::vector<double> S_host;
    // solve core: U^T U (FP64, r x r, kept after the first solve), the LU factors of
    // lambda S^-1 + U^T U for core_lambda (row-major, in place) and their row permutation, S on
    // the padded columns (FP64), all on the device
    DevBuf core_G, core_lu, core_perm, core_S;
    double core_lambda = -1.0;
    // tensor-core matvec (FP32 factors): enabled unless HDF_FLAG_CUDA_CORES; dev_err is set by
    // a kernel whose bounded wait expired
    bool use_tc = true;
    DevBuf dev_err;
    // events around the kernels of the most recent matvec (first column group)
    cudaEvent_t mv_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool mv_recorded = false;
    // cross factor K(X, Y) ~= U S V^T: the Y side (its U is V, same columns and S); owned
    hdf_factor* ypart = nullptr;
    ~hdf_factor() {
        for (auto& e : mv_ev) if (e) cudaEventDestroy(e);
        delete ypart;
    }
};
