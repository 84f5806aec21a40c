// The core of the Woodbury solve (Sec. 1, Sherman-Morrison-Woodbury, with the system of
// Eq. opt): C = lambda S^-1 + U^T U (r x r, FP64, row-major) is factored P C = L U by a blocked
// right-looking LU with partial pivoting.  S holds eigenvalues of both signs (the truncated
// expansion is not positive definite), so C is indefinite and needs pivoting.
//
// Work split.  Each panel of NB columns is factored with partial pivoting on the host (its
// rows split over the host threads, three barriers per column); the row interchanges of the
// panel are applied to the rest of the matrix on the device; U12 = L11^-1 A12 is one small GEMM
// with the host-inverted unit lower L11; the trailing update A22 -= L21 U12 -- nearly all of
// the 2/3 r^3 flops -- is an FP64 register-tiled GEMM on the device.  The factors stay on the
// device, and the solves L y = P z, U x = y run there as blocked substitutions (diagonal blocks
// in one CTA, the off-diagonal updates by the same GEMM).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

namespace hdf {
namespace lu {

constexpr int NB = 64;        // panel width (and block size of the substitutions)

// C = G + diag(lambda / S_a), with 1 on the diagonal of padding columns (S_a = 0: zero columns of U).
__global__ void k_core(const double* __restrict__ G, const double* __restrict__ Spad, double lambda, int64_t r,
                       double* __restrict__ C) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= r * r) return;
    const int64_t a = idx / r, b = idx % r;
    double v = G[idx];
    if (a == b) v += (Spad[a] != 0.0) ? lambda / Spad[a] : 1.0;
    C[idx] = v;
}

// Row interchanges j <-> piv[j], j = kb..ke-1 in order, on every column outside [kb, ke).
__global__ void k_swap_rows(double* __restrict__ A, int64_t r, int64_t kb, int64_t ke, const int* __restrict__ piv) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= r || (c >= kb && c < ke)) return;
    for (int64_t j = kb; j < ke; ++j) {
        const int64_t p = piv[j];
        if (p != j) {
            const double t = A[j * r + c];
            A[j * r + c] = A[p * r + c];
            A[p * r + c] = t;
        }
    }
}

// C (m x n) = beta C + alpha A (m x k) B (k x n), FP64, row-major with leading dimensions.
// 64 x 64 output tiles, 256 threads, 4 x 4 per thread, steps of 16 in k.  Every read of a tile's
// A rows and B columns precedes its writes, so B may be C's own rows when m <= 64 (one row tile).
constexpr int GT = 64, GK = 16;
__global__ void __launch_bounds__(256) k_dgemm(int64_t m, int64_t n, int64_t k, double alpha, const double* __restrict__ A,
                                               int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                                               int64_t ldc) {
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t r0 = (int64_t)blockIdx.y * GT, c0 = (int64_t)blockIdx.x * GT;
    double acc[4][4] = {};
    for (int64_t k0 = 0; k0 < k; k0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int kk = e % GK, rr = e / GK;
            const int64_t i = r0 + rr, kq = k0 + kk;
            As[kk][rr] = (i < m && kq < k) ? A[i * lda + kq] : 0.0;
            const int cc = e % GT, kb = e / GT;
            const int64_t j = c0 + cc, kp = k0 + kb;
            Bs[kb][cc] = (j < n && kp < k) ? B[kp * ldb + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t i = r0 + ty + 16 * u;
        if (i >= m) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t j = c0 + tx + 16 * v;
            if (j >= n) continue;
            const double old = (beta != 0.0) ? C[i * ldc + j] : 0.0;
            C[i * ldc + j] = beta * old + alpha * acc[u][v];
        }
    }
}

// z (rows of a w x nc block, row stride ldz) <- T^-1 z for the diagonal block T of the factors
// (rows and columns b0..b0+w of the r x r LU): lower with unit diagonal (lower = true) or upper.
// One CTA, thread j = column j of z.
__global__ void k_trsv_block(const double* __restrict__ LU, int64_t r, int64_t b0, int w, bool lower, double* z,
                             int64_t ldz, int nc) {
    __shared__ double T[NB][NB + 1];
    __shared__ double Z[NB][65];
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) T[e / w][e % w] = LU[(b0 + e / w) * r + b0 + e % w];
    for (int e = threadIdx.x; e < w * nc; e += blockDim.x) Z[e / nc][e % nc] = z[(e / nc) * ldz + e % nc];
    __syncthreads();
    const int j = threadIdx.x;
    if (j < nc) {
        if (lower) {
            for (int i = 0; i < w; ++i) {
                double s = Z[i][j];
                for (int l = 0; l < i; ++l) s -= T[i][l] * Z[l][j];
                Z[i][j] = s;
            }
        } else {
            for (int i = w - 1; i >= 0; --i) {
                double s = Z[i][j];
                for (int l = i + 1; l < w; ++l) s -= T[i][l] * Z[l][j];
                Z[i][j] = s / T[i][i];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < w * nc; e += blockDim.x) z[(e / nc) * ldz + e % nc] = Z[e / nc][e % nc];
}

// zo[a] = zi[perm[a]] (r x nc row-major): the row interchanges of the factorization, folded
// into one permutation on the host.
__global__ void k_gather_rows(const double* __restrict__ zi, double* __restrict__ zo, int64_t r, int nc,
                              const int* __restrict__ perm) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= r * nc) return;
    const int64_t a = idx / nc;
    zo[idx] = zi[(int64_t)perm[a] * nc + idx % nc];
}

// ------------------------------------------------------------------ host panel
// A sense-reversing spin barrier for the panel's threads.
struct SpinBarrier {
    std::atomic<int> count{0}, gen{0};
    int n = 1;
    void wait() {
        const int g = gen.load(std::memory_order_acquire);
        if (count.fetch_add(1, std::memory_order_acq_rel) + 1 == n) {
            count.store(0, std::memory_order_relaxed);
            gen.fetch_add(1, std::memory_order_acq_rel);
        } else {
            while (gen.load(std::memory_order_acquire) == g) std::this_thread::yield();
        }
    }
};

// LU with partial pivoting of the m x w row-major panel P (m >= w): piv[j] = row of P swapped
// with row j.  False if a pivot is zero or not finite.
bool panel_lu(int64_t m, int w, double* P, int* piv) {
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()),
                                                               16, m / 256 + 1}));
    SpinBarrier bar;
    bar.n = T;
    std::vector<double> bv(T);
    std::vector<int64_t> bi(T);
    std::atomic<bool> bad{false};
    double inv = 0.0;
    auto work = [&](int t) {
        const int64_t i0 = m * t / T, i1 = m * (t + 1) / T;
        for (int j = 0; j < w; ++j) {
            double best = -1.0;
            int64_t bidx = j;
            for (int64_t i = std::max<int64_t>(i0, j); i < i1; ++i) {
                const double a = std::fabs(P[i * w + j]);
                if (a > best) { best = a; bidx = i; }
            }
            bv[t] = best;
            bi[t] = bidx;
            bar.wait();
            if (t == 0) {
                double b = -1.0;
                int64_t p = j;
                for (int q = 0; q < T; ++q)
                    if (bv[q] > b) { b = bv[q]; p = bi[q]; }
                piv[j] = (int)p;
                if (!(b > 0.0) || !std::isfinite(b)) bad = true;
                if (p != j)
                    for (int c = 0; c < w; ++c) std::swap(P[j * w + c], P[p * w + c]);
                inv = bad ? 0.0 : 1.0 / P[j * w + j];
            }
            bar.wait();
            const double* Pj = P + (int64_t)j * w;
            for (int64_t i = std::max<int64_t>(i0, j + 1); i < i1; ++i) {
                double* Pi = P + i * w;
                const double l = Pi[j] * inv;
                Pi[j] = l;
                for (int c = j + 1; c < w; ++c) Pi[c] -= l * Pj[c];
            }
            bar.wait();
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < T; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& x : th) x.join();
    return !bad;
}

}  // namespace lu

// C = U^T U + diag(lambda / S) on the device (see k_core).
hdf_status core_init_device(const double* G, const double* Spad, double lambda, int64_t r, double* C, cudaStream_t st) {
    HDF_COUNT_LAUNCH();
    lu::k_core<<<(unsigned)((r * r + 255) / 256), 256, 0, st>>>(G, Spad, lambda, r, C);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

// P C = L U in place on the device (row-major r x r); dperm receives the row permutation
// (row a of P C is row perm[a] of C).  HDF_ESINGULAR if a pivot is zero.  Synchronises.
hdf_status lu_factor_device(int64_t r, double* C, DevBuf& dperm, cudaStream_t st) {
    using namespace lu;
    std::vector<int> piv_host(r, 0);
    DevBuf dpiv;
    HDF_CUDA(dpiv.alloc(sizeof(int) * std::max<int64_t>(1, r)));
    std::vector<double> panel, linv;
    DevBuf dlinv;
    HDF_CUDA(dlinv.alloc(sizeof(double) * NB * NB));
    for (int64_t kb = 0; kb < r; kb += NB) {
        const int64_t ke = std::min<int64_t>(r, kb + NB);
        const int w = (int)(ke - kb);
        const int64_t m = r - kb;
        panel.resize((size_t)m * w);
        HDF_CUDA(cudaMemcpy2DAsync(panel.data(), sizeof(double) * w, C + kb * r + kb, sizeof(double) * r,
                                   sizeof(double) * w, m, cudaMemcpyDeviceToHost, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        std::vector<int> pl(w);
        if (!panel_lu(m, w, panel.data(), pl.data())) return fail(HDF_ESINGULAR, "hdf_solve: singular core lambda S^-1 + U^T U");
        for (int j = 0; j < w; ++j) piv_host[kb + j] = (int)(kb + pl[j]);
        HDF_CUDA(cudaMemcpyAsync(dpiv.as<int>() + kb, piv_host.data() + kb, sizeof(int) * w, cudaMemcpyHostToDevice, st));
        // interchanges on the columns outside the panel, then the factored panel itself
        HDF_COUNT_LAUNCH();
        k_swap_rows<<<(unsigned)((r + 255) / 256), 256, 0, st>>>(C, r, kb, ke, dpiv.as<int>());
        HDF_CUDA(cudaGetLastError());
        HDF_CUDA(cudaMemcpy2DAsync(C + kb * r + kb, sizeof(double) * r, panel.data(), sizeof(double) * w,
                                   sizeof(double) * w, m, cudaMemcpyHostToDevice, st));
        if (ke == r) break;
        // U12 = L11^-1 A12 with the unit lower L11 inverted on the host (w x w)
        linv.assign((size_t)w * w, 0.0);
        for (int i = 0; i < w; ++i) {
            linv[(size_t)i * w + i] = 1.0;
            for (int j = 0; j < i; ++j) {
                double s = 0.0;
                for (int l = j; l < i; ++l) s -= panel[(size_t)i * w + l] * linv[(size_t)l * w + j];
                linv[(size_t)i * w + j] = s;
            }
        }
        HDF_CUDA(cudaMemcpyAsync(dlinv.p, linv.data(), sizeof(double) * w * w, cudaMemcpyHostToDevice, st));
        const int64_t nt = r - ke;
        HDF_COUNT_LAUNCH();
        k_dgemm<<<dim3((unsigned)((nt + GT - 1) / GT), 1), 256, 0, st>>>(w, nt, w, 1.0, dlinv.as<double>(), w,
                                                                       C + kb * r + ke, r, 0.0, C + kb * r + ke, r);
        // A22 -= L21 U12
        HDF_COUNT_LAUNCH();
        k_dgemm<<<dim3((unsigned)((nt + GT - 1) / GT), (unsigned)((nt + GT - 1) / GT)), 256, 0, st>>>(
            nt, nt, w, -1.0, C + ke * r + kb, r, C + kb * r + ke, r, 1.0, C + ke * r + ke, r);
        HDF_CUDA(cudaGetLastError());
        HDF_CUDA(cudaStreamSynchronize(st));     // panel and linv are reused
    }
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<int> perm(r);
    for (int64_t a = 0; a < r; ++a) perm[a] = (int)a;
    for (int64_t a = 0; a < r; ++a) std::swap(perm[a], perm[piv_host[a]]);
    HDF_CUDA(dperm.alloc(sizeof(int) * std::max<int64_t>(1, r)));
    HDF_CUDA(cudaMemcpy(dperm.p, perm.data(), sizeof(int) * r, cudaMemcpyHostToDevice));
    return HDF_OK;
}

// z (r x nc row-major, device, nc <= 64) = C^-1 zi with the factors of lu_factor_device; zi is
// left unchanged.
hdf_status lu_solve_device(int64_t r, const double* LU, const int* dperm, const double* zi, double* z, int nc,
                           cudaStream_t st) {
    using namespace lu;
    HDF_COUNT_LAUNCH();
    k_gather_rows<<<(unsigned)((r * nc + 255) / 256), 256, 0, st>>>(zi, z, r, nc, dperm);
    for (int64_t b0 = 0; b0 < r; b0 += NB) {                 // L y = P z
        const int w = (int)std::min<int64_t>(NB, r - b0);
        HDF_COUNT_LAUNCH();
        k_trsv_block<<<1, 64, 0, st>>>(LU, r, b0, w, true, z + b0 * nc, nc, nc);
        const int64_t rest = r - b0 - w;
        if (rest > 0) {
            HDF_COUNT_LAUNCH();
            k_dgemm<<<dim3((unsigned)((nc + GT - 1) / GT), (unsigned)((rest + GT - 1) / GT)), 256, 0, st>>>(
                rest, nc, w, -1.0, LU + (b0 + w) * r + b0, r, z + b0 * nc, nc, 1.0, z + (b0 + w) * nc, nc);
        }
    }
    const int64_t nblk = (r + NB - 1) / NB;
    for (int64_t b = nblk - 1; b >= 0; --b) {                // U x = y
        const int64_t b0 = b * NB;
        const int w = (int)std::min<int64_t>(NB, r - b0);
        HDF_COUNT_LAUNCH();
        k_trsv_block<<<1, 64, 0, st>>>(LU, r, b0, w, false, z + b0 * nc, nc, nc);
        if (b0 > 0) {
            HDF_COUNT_LAUNCH();
            k_dgemm<<<dim3((unsigned)((nc + GT - 1) / GT), (unsigned)((b0 + GT - 1) / GT)), 256, 0, st>>>(
                b0, nc, w, -1.0, LU + b0, r, z + b0 * nc, nc, 1.0, z, nc);
        }
    }
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

}  // namespace hdf
