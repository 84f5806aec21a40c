// hdf_matvec_noalloc: K~ V with its work space in a fixed array that is part of the loaded
// library instead of memory obtained at call time.
//
// Some callers cannot allocate device memory at the moment they need a product: code whose
// device memory is owned by another allocator (a framework's caching pool holds the free
// memory, so a raw cudaMalloc can fail even though the framework has room), and latency-
// critical or real-time loops that reserve everything at start-up and must not enter the CUDA
// allocator.  For them the per-call partial sums live in g_noalloc_scratch below.
//
// The products always run on the CUDA-core tile kernels (k_utv_tile, k_uw_tile, as hdf_matvec
// does for FP64 factors).  For FP32 factors hdf_matvec uses the tensor cores where it can, so
// there the two entry points agree to FP32 rounding, not bit for bit, and this one is slower.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "hdf_kernels.cuh"
#include "internal.h"

namespace {

// 32 MiB of doubles.  Every device on which the library's module is loaded holds this
// array until the process exits.
constexpr size_t kScratchDoubles = size_t(1) << 22;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
constexpr int kGroup = 64;           // V columns per pass, as in hdf_matvec
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the symbol name
// is only a host-side stand-in, so the address is looked up once per device (with that
// device current) and cached.
hdf_status scratch_address(double** out) {
    int dev = 0;
    HDF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return hdf::fail(HDF_EINVAL, "hdf_matvec_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        HDF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = p;
    }
    *out = static_cast<double*>(g_addr[dev]);
    return HDF_OK;
}

int ct_for(int c) { return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : c <= 32 ? 32 : 64; }

template <typename T>
void utv(int ct, const T* U, int64_t ldU, int64_t n, int64_t r, const T* V, int64_t ldv, int c, int nchunk,
         int64_t chunk, double* part, cudaStream_t st) {
#define HDF_NA_UTV(CT)                                                                                 \
    case CT: {                                                                                         \
        dim3 g(nchunk, (unsigned)((r + hdf::dev::UtvShape<CT>::AB - 1) / hdf::dev::UtvShape<CT>::AB)); \
        HDF_COUNT_LAUNCH();                                                                            \
        hdf::dev::k_utv_tile<T, CT><<<g, 256, 0, st>>>(U, ldU, n, r, V, ldv, c, chunk, part);          \
        break;                                                                                         \
    }
    switch (ct) { HDF_NA_UTV(1) HDF_NA_UTV(2) HDF_NA_UTV(4) HDF_NA_UTV(8) HDF_NA_UTV(16) HDF_NA_UTV(32) HDF_NA_UTV(64) }
#undef HDF_NA_UTV
}

template <typename T>
void uw(int ct, const T* U, int64_t ldU, int64_t n, int64_t r, const T* W, int c, T* Y, int64_t ldy,
        cudaStream_t st) {
#define HDF_NA_UW(CT)                                                                                  \
    case CT: {                                                                                         \
        const unsigned g = (unsigned)((n + hdf::dev::UwShape<CT>::RB - 1) / hdf::dev::UwShape<CT>::RB);\
        HDF_COUNT_LAUNCH();                                                                            \
        hdf::dev::k_uw_tile<T, CT><<<g, 256, 0, st>>>(U, ldU, n, r, W, c, (T)1, nullptr, 0, (T)0, Y,  \
                                                       ldy);                                           \
        break;                                                                                         \
    }
    switch (ct) { HDF_NA_UW(1) HDF_NA_UW(2) HDF_NA_UW(4) HDF_NA_UW(8) HDF_NA_UW(16) HDF_NA_UW(32) HDF_NA_UW(64) }
#undef HDF_NA_UW
}

template <typename T>
hdf_status run(const hdf_factor* f, const T* V, int64_t ldv, int ncols, T* Y, int64_t ldy, cudaStream_t st) {
    const int64_t n = f->info.n, r = (f->info.rank > 0) ? f->info.ldu : 0;   // padded width of U
    if (r == 0) {
        for (int j = 0; j < ncols; ++j) HDF_CUDA(cudaMemsetAsync(Y + j * ldy, 0, n * sizeof(T), st));
        return HDF_OK;
    }
    const int cmax = std::min(ncols, kGroup);
    // Layout of the array: [W: r x cmax of T, rounded up to doubles][partials: nchunk x cmax x r]
    const int64_t w_doubles = (r * cmax * (int64_t)sizeof(T) + 7) / 8;
    const int64_t per_chunk = r * cmax;
    if (w_doubles + per_chunk > (int64_t)kScratchDoubles)
        return hdf::fail(HDF_ETOOBIG, "hdf_matvec_noalloc: ldu * min(ncols, 64) * (8 + element size) bytes "
                                      "exceeds the fixed 32 MiB work space");
    double* base = nullptr;
    hdf_status s = scratch_address(&base);
    if (s != HDF_OK) return s;
    T* W = reinterpret_cast<T*>(base);
    double* part = base + w_doubles;
    const int64_t by_rows = (n + 2047) / 2048;
    const int64_t by_space = ((int64_t)kScratchDoubles - w_doubles) / per_chunk;
    const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(by_rows, by_space), 1024));
    const int64_t chunk = (n + nchunk - 1) / nchunk;
    const T* U = f->U.as<T>();
    const T* S = f->S.as<T>();
    for (int j0 = 0; j0 < ncols; j0 += kGroup) {
        const int cg = std::min(kGroup, ncols - j0);
        const int ct = ct_for(cg);
        // every partial slot [0, nchunk * cg * r) is overwritten by k_utv_tile and every W entry
        // by k_reduce_scale, so nothing left from an earlier call is read
        utv<T>(ct, U, f->info.ldu, n, r, V + j0 * ldv, ldv, cg, nchunk, chunk, part, st);
        HDF_CUDA(cudaGetLastError());
        const int64_t work = r * cg;
        HDF_COUNT_LAUNCH();
        hdf::dev::k_reduce_scale<T><<<(unsigned)((work + 255) / 256), 256, 0, st>>>(part, nchunk, r, cg, S, W,
                                                                                    nullptr);
        HDF_CUDA(cudaGetLastError());
        uw<T>(ct, U, f->info.ldu, n, r, W, cg, Y + j0 * ldy, ldy, st);
        HDF_CUDA(cudaGetLastError());
    }
    return HDF_OK;
}

}  // namespace

extern "C" hdf_status hdf_matvec_noalloc(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols,
                                         void* Y_dev, int64_t ldy, hdf_stream stream) {
    if (!f || !V_dev || !Y_dev || ncols < 1 || ncols > 1024 || ldv < f->info.n || ldy < f->info.n)
        return hdf::fail(HDF_EINVAL, "hdf_matvec_noalloc: bad argument");
    if (f->ypart) return hdf::fail(HDF_EINVAL, "hdf_matvec_noalloc: symmetric factors only (use hdf_matvec)");
    if (f->mf.on) return hdf::fail(HDF_EINVAL, "hdf_matvec_noalloc: the factor stores no U (use hdf_matvec)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (f->prec == HDF_FP64)
        return run<double>(f, (const double*)V_dev, ldv, ncols, (double*)Y_dev, ldy, st);
    return run<float>(f, (const float*)V_dev, ldv, ncols, (float*)Y_dev, ldy, st);
}
