// Internal declarations shared by the library's translation units (not part of the ABI):
// the factor object, error reporting, the launch counter and a device-buffer owner.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hdf.h"

namespace hdf {

// Sets the thread-local message returned by hdf_last_error and returns s.
hdf_status fail(hdf_status s, const std::string& msg);
// Counter of kernel launches reported by hdf_launch_count.
extern std::atomic<long long> g_launches;

}  // namespace hdf

#define HDF_COUNT_LAUNCH() hdf::g_launches.fetch_add(1, std::memory_order_relaxed)

#define HDF_CUDA(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return hdf::fail(HDF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
        }                                                                                     \
    } while (0)

// Owns one device allocation.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t b) {
        if (p) { cudaFree(p); p = nullptr; }
        bytes = b;
        return b ? cudaMalloc(&p, b) : cudaSuccess;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct hdf_factor {
    hdf_info info{};
    int kernel = 0;
    double ell = 0, tol = 0;
    int prec = 0;
    size_t esz = 8;                 // bytes per bulk element
    DevBuf U, S;                    // U n x ldu, S rank (bulk type)
    std::vector<double> S_host;
    // solve core (lambda S^-1 + U^T U), LU factors on the host
    std::vector<double> G;
    double core_lambda = -1.0;
    std::vector<double> LU;
    std::vector<int> piv;
    // events around the kernels of the most recent matvec (first column group)
    cudaEvent_t mv_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool mv_recorded = false;
    ~hdf_factor() { for (auto& e : mv_ev) if (e) cudaEventDestroy(e); }
};
