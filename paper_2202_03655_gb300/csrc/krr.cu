// Kernel ridge regression of Sec. 4.2 on the device: k-means clustering (Lloyd's iteration),
// the operator K^ (HDF factors of the diagonal blocks through the batched factorization, exact
// off-diagonal blocks evaluated on the fly), the block-diagonal preconditioner (inverses of the
// exact lambda I + K_{C_i C_i}) and preconditioned conjugate gradients for Eq. (opt).
// Declarations and argument contracts are in include/hdf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "../../include/hdf.h"
#include "hdf_kernels.cuh"
#include "internal.h"
#include "planner.h"

using namespace hdf;

namespace {

double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int blocks_for(int64_t work, int per_block, int cap) {
    const int64_t g = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ------------------------------------------------------------------------- k-means
// Assignment step: label = nearest centre (squared distance summed over coordinates in order,
// the lowest index on ties); counts the points whose label changed.
__global__ void k_km_assign(const double* __restrict__ x, int64_t n, int d, int k, const double* __restrict__ C,
                            int* __restrict__ labels, int* __restrict__ changes) {
    extern __shared__ double Cs[];
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) Cs[e] = C[e];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[dev::kMaxD];
    for (int j = 0; j < d; ++j) xi[j] = x[i * d + j];
    double best = INFINITY;
    int bc = 0;
    for (int c = 0; c < k; ++c) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) { const double t = xi[j] - Cs[c * d + j]; s += t * t; }
        if (s < best) { best = s; bc = c; }
    }
    if (labels[i] != bc) { atomicAdd(changes, 1); labels[i] = bc; }
}

// Update step, first stage: block b sums the coordinates (and counts) of its chunk's points per
// cluster with fixed-order tree sums: part[(b k + c) (d + 1) + j], j = d the count.
__global__ void __launch_bounds__(256) k_km_partial(const double* __restrict__ x, int64_t n, int d, int k,
                                                    const int* __restrict__ labels, int64_t chunk,
                                                    double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int c = 0; c < k; ++c) {
        double acc[dev::kMaxD + 1];
        for (int j = 0; j <= d; ++j) acc[j] = 0.0;
        for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
            if (labels[i] == c) {
                for (int j = 0; j < d; ++j) acc[j] += x[i * d + j];
                acc[d] += 1.0;
            }
        for (int j = 0; j <= d; ++j) {
            const double t = dev::block_sum_256(acc[j], sh);
            if (threadIdx.x == 0) part[((int64_t)blockIdx.x * k + c) * (d + 1) + j] = t;
        }
    }
}

// Update step, second stage: centre c = mean of its points (partials added in block order); a
// centre without points stays where it is.
__global__ void k_km_finish(const double* __restrict__ part, int G, int k, int d, double* __restrict__ C) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    double s[dev::kMaxD + 1];
    for (int j = 0; j <= d; ++j) s[j] = 0.0;
    for (int b = 0; b < G; ++b)
        for (int j = 0; j <= d; ++j) s[j] += part[((int64_t)b * k + c) * (d + 1) + j];
    if (s[d] > 0.0)
        for (int j = 0; j < d; ++j) C[c * d + j] = s[j] / s[d];
}

__global__ void k_gather_rows(const double* __restrict__ x, int d, const int64_t* __restrict__ idx, int64_t m,
                              double* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= m * d) return;
    const int64_t r = e / d;
    out[e] = x[idx[r] * d + (e % d)];
}

// --------------------------------------------------------- direct kernel evaluation
constexpr int kDkRows = 128;     // rows (outputs) per block
constexpr int kDkTile = 128;     // columns staged per tile

// part[s m + i] = sum over columns j of split s of k(|a_i - b_j|) w_j, skipping j with
// cb[j] == ca[i] when ca is given (the off-diagonal blocks of K^).  Coordinates are FP32 copies
// shifted by a common point and the kernel values k_ij are FP32 (one fixed, exactly symmetric
// matrix); w_j = w_hi + w_lo as two FP32 numbers, each product k_ij w_hi formed exactly (fma)
// and the sums of one tile kept as FP32 pairs (TwoSum), so that the product is linear in w to
// about 1e-14 -- conjugate gradients need the same linear operator in every iteration.  Tiles
// are added in FP64 in column order.
template <int DD>
__global__ void __launch_bounds__(kDkRows) k_direct_kernel(const float* __restrict__ a, int64_t m,
                                                          const float* __restrict__ b, int64_t n, int kernel,
                                                          float inv_ell, const double* __restrict__ w,
                                                          const int* __restrict__ ca, const int* __restrict__ cb,
                                                          int64_t split, double* __restrict__ part) {
    constexpr int U = 4;                         // independent accumulators (pairs in flight)
    __shared__ float bs[kDkTile][DD];
    __shared__ float ws[kDkTile], wl[kDkTile];
    __shared__ int cs[kDkTile];
    const int64_t i = blockIdx.x * (int64_t)kDkRows + threadIdx.x;
    const bool act = i < m;
    float ai[DD];
#pragma unroll
    for (int j = 0; j < DD; ++j) ai[j] = act ? a[i * DD + j] : 0.f;
    const int myc = (ca && act) ? ca[i] : -1;
    const int64_t j0 = blockIdx.y * split, j1 = min(n, j0 + split);
    double acc = 0.0;
    for (int64_t t0 = j0; t0 < j1; t0 += kDkTile) {
        const int nt = (int)min((int64_t)kDkTile, j1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < kDkTile * DD; e += blockDim.x) {
            const int r = e / DD, q = e % DD;
            bs[r][q] = (r < nt) ? b[(t0 + r) * DD + q] : 0.f;
        }
        for (int r = threadIdx.x; r < kDkTile; r += blockDim.x) {
            const double wv = (r < nt) ? w[t0 + r] : 0.0;
            const float hi = (float)wv;
            ws[r] = hi;
            wl[r] = (float)(wv - (double)hi);
            cs[r] = (r < nt && cb) ? cb[t0 + r] : -2;        // rows past the tile carry w = 0
        }
        __syncthreads();
        float sh_[U], sl_[U];                    // tile sums as unevaluated FP32 pairs
#pragma unroll
        for (int u = 0; u < U; ++u) sh_[u] = sl_[u] = 0.f;
        const int ntu = (nt + U - 1) / U * U;    // the padded tail adds exact zeros (w = 0, k <= 1)
        for (int r0 = 0; r0 < ntu; r0 += U) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u;
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < DD; ++q) { const float t = ai[q] - bs[r][q]; s = fmaf(t, t, s); }
                float kv = dev::kernel_value_f(kernel, sqrtf(s), inv_ell);
                kv = (cs[r] == myc) ? 0.f : kv;
                const float p = kv * ws[r];
                const float e = fmaf(kv, wl[r], fmaf(kv, ws[r], -p));    // exact error of p, plus k w_lo
                float t1, t2;
                dev::two_sum(sh_[u], p, t1, t2);
                sh_[u] = t1;
                sl_[u] += t2 + e;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc += (double)sh_[u] + (double)sl_[u];
    }
    if (act) part[blockIdx.y * m + i] = acc;
}

// Launch of k_direct_kernel for the dimension d.
void launch_direct(int d, dim3 g, cudaStream_t st, const float* a, int64_t m, const float* b, int64_t n, int kernel,
                   float inv_ell, const double* w, const int* ca, const int* cb, int64_t split, double* part) {
#define HDF_DK(DD) case DD: k_direct_kernel<DD><<<g, kDkRows, 0, st>>>(a, m, b, n, kernel, inv_ell, w, ca, cb, split, part); break;
    switch (d) { HDF_DK(1) HDF_DK(2) HDF_DK(3) HDF_DK(4) HDF_DK(5) HDF_DK(6) HDF_DK(7) HDF_DK(8) }
#undef HDF_DK
}

// out[i] = alpha v[i] + (add ? add[i] : 0) + sum_s part[s m + i]
__global__ void k_direct_finish(const double* __restrict__ part, int S, int64_t m, double alpha,
                                const double* __restrict__ v, const double* __restrict__ add, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s = (v ? alpha * v[i] : 0.0) + (add ? add[i] : 0.0);
    for (int t = 0; t < S; ++t) s += part[t * m + i];
    out[i] = s;
}

// FP32 copy of row-major points shifted by the point o (FP64 differences first).
__global__ void k_shift_f32(const double* __restrict__ x, int64_t n, int d, const double* __restrict__ o,
                            float* __restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * d) return;
    out[e] = (float)(x[e] - o[e % d]);
}

// Column splits for the direct kernel: enough blocks to fill the GPU a few times.
int64_t direct_split(int64_t m, int64_t n, int* S) {
    const int64_t rb = (m + kDkRows - 1) / kDkRows;
    int64_t s = std::max<int64_t>(1, std::min<int64_t>((4 * 152 + rb - 1) / rb, (n + kDkTile - 1) / kDkTile));
    s = std::min<int64_t>(s, 64);
    int64_t split = (n + s - 1) / s;
    split = ((split + kDkTile - 1) / kDkTile) * kDkTile;
    *S = (int)std::max<int64_t>(1, (n + split - 1) / split);
    return split;
}

// ---------------------------------------------------------------- vector kernels
__global__ void k_gather_vec(const double* __restrict__ v, const int64_t* __restrict__ perm, int64_t n,
                             double* __restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) out[p] = v[perm[p]];
}

__global__ void k_scatter_vec(const double* __restrict__ v, const int64_t* __restrict__ perm, int64_t n,
                              double* __restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) out[perm[p]] = v[p];
}

__global__ void k_to_f32(const double* __restrict__ v, int64_t n, float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)v[i];
}

__global__ void k_to_f64(const float* __restrict__ v, int64_t n, double* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)v[i];
}

// part[b] = sum over the block's chunk of a_i b_i (fixed-order tree sums), two pairs at once.
__global__ void __launch_bounds__(256) k_dot2(const double* __restrict__ a, const double* __restrict__ b,
                                              const double* __restrict__ c, const double* __restrict__ e, int64_t n,
                                              int64_t chunk, double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double s1 = 0.0, s2 = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        s1 += a[i] * b[i];
        if (c) s2 += c[i] * e[i];
    }
    const double t1 = dev::block_sum_256(s1, sh);
    const double t2 = dev::block_sum_256(s2, sh);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = t1; part[2 * blockIdx.x + 1] = t2; }
}

// x += alpha p; r -= alpha q
__global__ void k_cg_step(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                          const double* __restrict__ q, double alpha, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

// p = z + beta p
__global__ void k_cg_dir(double* __restrict__ p, const double* __restrict__ z, double beta, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = z[i] + beta * p[i];
}

// ------------------------------------------------------------------- preconditioner
// Dense lambda I + K_{C_c C_c} of every cluster (exact kernel, FP64) into the packed array:
// block c at ioff[c], n_c x n_c row-major; one thread per entry.
__global__ void k_block_matrices(const double* __restrict__ xp, int d, const int64_t* __restrict__ offs,
                                 const int64_t* __restrict__ ioff, int nclus, int kernel, double ell, double lam,
                                 double* __restrict__ out) {
    const int c = blockIdx.y;
    const int64_t a0 = offs[c], nc = offs[c + 1] - a0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc * nc; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nc, j = e % nc;
        double s = 0.0;
        for (int q = 0; q < d; ++q) { const double t = xp[(a0 + i) * d + q] - xp[(a0 + j) * d + q]; s += t * t; }
        out[ioff[c] + e] = dev::kernel_value(kernel, sqrt(s), ell) + (i == j ? lam : 0.0);
    }
}

// z = M r: one warp per row of the block-diagonal inverse (packed as above).
__global__ void k_block_gemv(const double* __restrict__ inv, const int64_t* __restrict__ offs,
                             const int64_t* __restrict__ ioff, const int* __restrict__ cl, int64_t n,
                             const double* __restrict__ r, double* __restrict__ z) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const int c = cl[row];
    const int64_t a0 = offs[c], nc = offs[c + 1] - a0, i = row - a0;
    const double* M = inv + ioff[c] + i * nc;
    double s = 0.0;
    for (int64_t j = lane; j < nc; j += 32) s += M[j] * r[a0 + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) z[row] = s;
}

// --------------------------------------- block preconditioner: batched SPD inverse (FP64)
// A_c = lambda I + K_{C_c C_c} of every cluster c (packed row-major n_c x n_c at ioff[c]) is
// inverted on the device in 64 x 64 tiles, all clusters side by side (blockIdx.y = cluster):
//   Cholesky A = L L^T, right-looking, per panel j: the diagonal tile is factored in shared
//   memory and its inverse D_j = L_jj^-1 kept; L_ij = A_ij D_j^T for the tiles below; the
//   trailing lower tiles A_ik -= L_ij L_kj^T;
//   W = L^-1 by tile rows: W_ii = D_i, W_ij = -D_i sum_{j <= k < i} L_ik W_kj;
//   A^-1 = W^T W, both triangles written.
// A non-positive pivot sets *bad (the host reports HDF_ESINGULAR).
constexpr int kST = 64;                 // tile edge
constexpr int kSP = kST + 1;            // shared row stride (doubles)

struct SpdArgs {
    double* A;                          // packed blocks (overwritten by L in the lower tiles)
    double* W;                          // packed blocks: L^-1 (lower tiles), then A^-1 is written to A
    double* D;                          // per cluster: nb_c diagonal-tile inverses, 64 x 64 each
    const int64_t* offs;                // cluster c: rows offs[c] .. offs[c + 1]
    const int64_t* ioff;                // packed offsets of the blocks
    const int64_t* doff;                // offsets of the diagonal-tile inverses
    int* bad;
};

__device__ __forceinline__ int64_t spd_n(const SpdArgs& P, int c) { return P.offs[c + 1] - P.offs[c]; }

// tile (bi, bj) of the n x n row-major M -> s (kST x kSP), zeros outside the matrix
__device__ __forceinline__ void spd_load(const double* M, int64_t n, int bi, int bj, double* s) {
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) {
        const int r = e / kST, q = e % kST;
        const int64_t gr = (int64_t)bi * kST + r, gc = (int64_t)bj * kST + q;
        s[r * kSP + q] = (gr < n && gc < n) ? M[gr * n + gc] : 0.0;
    }
}
__device__ __forceinline__ void spd_store(double* M, int64_t n, int bi, int bj, const double* s, bool transpose) {
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) {
        const int r = e / kST, q = e % kST;
        const int64_t gr = (int64_t)bi * kST + r, gc = (int64_t)bj * kST + q;
        if (gr < n && gc < n) {
            if (transpose) M[gc * n + gr] = s[r * kSP + q];
            else M[gr * n + gc] = s[r * kSP + q];
        }
    }
}
// acc (4 x 4 per thread, 256 threads: rows 4 ty.., columns 4 tx..) += X Y^T or X Y (tiles in shared)
template <bool YT>
__device__ __forceinline__ void spd_mma(const double* X, const double* Y, double acc[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int m = 0; m < kST; ++m) {
        double xv[4], yv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[i] = X[(4 * ty + i) * kSP + m];
#pragma unroll
        for (int j = 0; j < 4; ++j) yv[j] = YT ? Y[(4 * tx + j) * kSP + m] : Y[m * kSP + 4 * tx + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
    }
}

// Panel j, step 1: factor the diagonal tile in shared memory, write L_jj to A, D_j = L_jj^-1.
__global__ void __launch_bounds__(256) k_spd_potrf(SpdArgs P, int j) {
    extern __shared__ double sh[];
    const int c = blockIdx.y;
    const int64_t n = spd_n(P, c);
    if ((int64_t)j * kST >= n) return;
    const int t = (int)min((int64_t)kST, n - (int64_t)j * kST);
    double* A = P.A + P.ioff[c];
    double* S = sh;                       // the tile
    double* X = sh + kST * kSP;           // its inverse
    spd_load(A, n, j, j, S);
    __syncthreads();
    for (int k = 0; k < t; ++k) {
        if (threadIdx.x == 0) {
            const double piv = S[k * kSP + k];
            if (!(piv > 0.0)) { atomicExch(P.bad, 1); S[k * kSP + k] = 1.0; }
            else S[k * kSP + k] = sqrt(piv);
        }
        __syncthreads();
        const double dk = S[k * kSP + k];
        for (int r = k + 1 + threadIdx.x; r < t; r += blockDim.x) S[r * kSP + k] /= dk;
        __syncthreads();
        // trailing lower triangle: S[r][q] -= S[r][k] S[q][k], k < q <= r < t
        const int m = t - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int r = k + 1 + e / m, q = k + 1 + e % m;
            if (q <= r) S[r * kSP + q] -= S[r * kSP + k] * S[q * kSP + k];
        }
        __syncthreads();
    }
    // zero the strict upper triangle and the padding, so that the tile is exactly L_jj
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) {
        const int r = e / kST, q = e % kST;
        if (q > r || r >= t) S[r * kSP + q] = (r == q && r >= t) ? 1.0 : 0.0;
    }
    __syncthreads();
    // X = L^-1, column q by thread q: X[r][q] = (delta_rq - sum_{q <= m < r} L[r][m] X[m][q]) / L[r][r]
    if (threadIdx.x < kST) {
        const int q = threadIdx.x;
        for (int r = 0; r < kST; ++r) {
            if (r < q) { X[r * kSP + q] = 0.0; continue; }
            double v = (r == q) ? 1.0 : 0.0;
            for (int m = q; m < r; ++m) v -= S[r * kSP + m] * X[m * kSP + q];
            X[r * kSP + q] = v / S[r * kSP + r];
        }
    }
    __syncthreads();
    spd_store(A, n, j, j, S, false);
    double* D = P.D + P.doff[c] + (int64_t)j * kST * kST;
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) D[e] = X[(e / kST) * kSP + e % kST];
}

// Panel j, step 2: L_ij = A_ij D_j^T for the tiles below the diagonal (blockIdx.x = i - j - 1).
__global__ void __launch_bounds__(256) k_spd_trsm(SpdArgs P, int j) {
    extern __shared__ double sh[];
    const int c = blockIdx.y;
    const int64_t n = spd_n(P, c);
    const int i = j + 1 + blockIdx.x;
    if ((int64_t)i * kST >= n) return;
    double* A = P.A + P.ioff[c];
    const double* D = P.D + P.doff[c] + (int64_t)j * kST * kST;
    double* Xs = sh;
    double* Ds = sh + kST * kSP;
    spd_load(A, n, i, j, Xs);
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) Ds[(e / kST) * kSP + e % kST] = D[e];
    __syncthreads();
    double acc[4][4] = {};
    spd_mma<true>(Xs, Ds, acc);
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) Xs[(4 * ty + a) * kSP + 4 * tx + b2] = acc[a][b2];
    __syncthreads();
    spd_store(A, n, i, j, Xs, false);
}

// Panel j, step 3: A_ik -= L_ij L_kj^T for j < k <= i (blockIdx.x enumerates the pairs).
__global__ void __launch_bounds__(256) k_spd_update(SpdArgs P, int j) {
    extern __shared__ double sh[];
    const int c = blockIdx.y;
    const int64_t n = spd_n(P, c);
    // pair index -> (i, k) with 0 <= kk <= ii, i = j + 1 + ii, k = j + 1 + kk
    const int e = blockIdx.x;
    int ii = (int)((sqrt(8.0 * e + 1.0) - 1.0) / 2.0);
    while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
    while (ii * (ii + 1) / 2 > e) --ii;
    const int kk = e - ii * (ii + 1) / 2;
    const int i = j + 1 + ii, k = j + 1 + kk;
    if ((int64_t)i * kST >= n) return;
    double* A = P.A + P.ioff[c];
    double* Li = sh;
    double* Lk = sh + kST * kSP;
    double* Cs = sh + 2 * kST * kSP;
    spd_load(A, n, i, j, Li);
    spd_load(A, n, k, j, Lk);
    spd_load(A, n, i, k, Cs);
    __syncthreads();
    double acc[4][4] = {};
    spd_mma<true>(Li, Lk, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) Cs[(4 * ty + a) * kSP + 4 * tx + b2] -= acc[a][b2];
    __syncthreads();
    spd_store(A, n, i, k, Cs, false);
}

// W = L^-1, tile row i (blockIdx.x = j <= i): W_ii = D_i, W_ij = -D_i sum_{j <= k < i} L_ik W_kj.
__global__ void __launch_bounds__(256) k_spd_winv(SpdArgs P, int i) {
    extern __shared__ double sh[];
    const int c = blockIdx.y;
    const int64_t n = spd_n(P, c);
    const int j = blockIdx.x;
    if ((int64_t)i * kST >= n || j > i) return;
    const double* A = P.A + P.ioff[c];
    double* W = P.W + P.ioff[c];
    const double* D = P.D + P.doff[c] + (int64_t)i * kST * kST;
    double* X = sh;
    double* Y = sh + kST * kSP;
    double* Z = sh + 2 * kST * kSP;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (j == i) {
        for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) Z[(e / kST) * kSP + e % kST] = D[e];
        __syncthreads();
        spd_store(W, n, i, i, Z, false);
        return;
    }
    double acc[4][4] = {};
    for (int k = j; k < i; ++k) {           // S = sum_k L_ik W_kj
        spd_load(A, n, i, k, X);
        spd_load(W, n, k, j, Y);
        __syncthreads();
        spd_mma<false>(X, Y, acc);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) Y[(4 * ty + a) * kSP + 4 * tx + b2] = acc[a][b2];
    for (int e = threadIdx.x; e < kST * kST; e += blockDim.x) X[(e / kST) * kSP + e % kST] = D[e];
    __syncthreads();
    double out[4][4] = {};
    spd_mma<false>(X, Y, out);              // D_i S
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) Z[(4 * ty + a) * kSP + 4 * tx + b2] = -out[a][b2];
    __syncthreads();
    spd_store(W, n, i, j, Z, false);
}

// A^-1 = W^T W: tile (i, j), j <= i (blockIdx.x enumerates the pairs) = sum_{k >= i} W_ki^T W_kj,
// written to (i, j) and, transposed, to (j, i).
__global__ void __launch_bounds__(256) k_spd_wtw(SpdArgs P) {
    extern __shared__ double sh[];
    const int c = blockIdx.y;
    const int64_t n = spd_n(P, c);
    const int nb = (int)((n + kST - 1) / kST);
    const int e = blockIdx.x;
    int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) / 2.0);
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    while (i * (i + 1) / 2 > e) --i;
    const int j = e - i * (i + 1) / 2;
    if (i >= nb) return;
    const double* W = P.W + P.ioff[c];
    double* A = P.A + P.ioff[c];
    double* X = sh;
    double* Y = sh + kST * kSP;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k = i; k < nb; ++k) {
        // X = W_ki^T (transposed on load), Y = W_kj
        for (int q = threadIdx.x; q < kST * kST; q += blockDim.x) {
            const int r = q / kST, s2 = q % kST;
            const int64_t gr = (int64_t)k * kST + r, gc = (int64_t)i * kST + s2;
            X[s2 * kSP + r] = (gr < n && gc < n) ? W[gr * n + gc] : 0.0;
        }
        spd_load(W, n, k, j, Y);
        __syncthreads();
        spd_mma<false>(X, Y, acc);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) X[(4 * ty + a) * kSP + 4 * tx + b2] = acc[a][b2];
    __syncthreads();
    spd_store(A, n, i, j, X, false);
    if (i != j) spd_store(A, n, i, j, X, true);
}

}  // namespace

struct hdf_krr {
    int64_t n = 0;
    int d = 0, nclus = 0, prec = 0, kernel = 0;
    double ell = 0.0, lam = 0.0;
    std::vector<int64_t> offs, ioff;
    DevBuf perm, xp, xp32, cl, doffs, dioff, inv;
    hdf_batch* batch = nullptr;
    DevBuf vb, yb, hd, part, dotp;       // work: bulk-typed vectors, HDF result, direct-kernel partials
    int S = 1;
    int64_t split = 0;
    double t_build = 0.0, t_precond = 0.0;
    ~hdf_krr() { if (batch) hdf_batch_free(batch); }
};

namespace {

// tp = lambda vp + K^ vp in cluster order (vp, tp length n, FP64, device)
hdf_status apply_perm(hdf_krr* K, const double* vp, double* tp, cudaStream_t st) {
    const int64_t n = K->n;
    const int gb = blocks_for(n, 256, 1 << 30);
    hdf_status s;
    if (K->prec == HDF_FP32) {
        HDF_COUNT_LAUNCH();
        k_to_f32<<<gb, 256, 0, st>>>(vp, n, K->vb.as<float>());
        s = hdf_batch_matvec(K->batch, K->vb.p, n, 1, K->yb.p, n, reinterpret_cast<hdf_stream>(st));
        if (s != HDF_OK) return s;
        HDF_COUNT_LAUNCH();
        k_to_f64<<<gb, 256, 0, st>>>(K->yb.as<float>(), n, K->hd.as<double>());
    } else {
        s = hdf_batch_matvec(K->batch, vp, n, 1, K->hd.p, n, reinterpret_cast<hdf_stream>(st));
        if (s != HDF_OK) return s;
    }
    dim3 g((unsigned)((n + kDkRows - 1) / kDkRows), (unsigned)K->S);
    HDF_COUNT_LAUNCH();
    launch_direct(K->d, g, st, K->xp32.as<float>(), n, K->xp32.as<float>(), n, K->kernel, (float)(1.0 / K->ell), vp,
                  K->cl.as<int>(), K->cl.as<int>(), K->split, K->part.as<double>());
    HDF_COUNT_LAUNCH();
    k_direct_finish<<<gb, 256, 0, st>>>(K->part.as<double>(), K->S, n, K->lam, vp, K->hd.as<double>(), tp);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

hdf_status precond_perm(hdf_krr* K, const double* rp, double* zp, cudaStream_t st) {
    HDF_COUNT_LAUNCH();
    k_block_gemv<<<blocks_for(K->n * 32, 256, 1 << 30), 256, 0, st>>>(K->inv.as<double>(), K->doffs.as<int64_t>(),
                                                                     K->dioff.as<int64_t>(), K->cl.as<int>(), K->n,
                                                                     rp, zp);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

// (a . b, c . e) with deterministic partial sums (c may be null)
hdf_status dot2(hdf_krr* K, const double* a, const double* b, const double* c, const double* e, double* r1,
                double* r2, cudaStream_t st) {
    const int64_t n = K->n;
    const int G = blocks_for(n, 4096, 256);
    const int64_t chunk = (n + G - 1) / G;
    HDF_COUNT_LAUNCH();
    k_dot2<<<G, 256, 0, st>>>(a, b, c, e, n, chunk, K->dotp.as<double>());
    HDF_CUDA(cudaGetLastError());
    double h[512];
    HDF_CUDA(cudaMemcpyAsync(h, K->dotp.p, sizeof(double) * 2 * G, cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    double s1 = 0.0, s2 = 0.0;
    for (int g = 0; g < G; ++g) { s1 += h[2 * g]; s2 += h[2 * g + 1]; }
    *r1 = s1;
    if (r2) *r2 = s2;
    return HDF_OK;
}

}  // namespace

extern "C" {

hdf_status hdf_kmeans(const double* x_dev, int64_t n, int d, int k, const int64_t* init_host, int max_iter,
                      int* labels_dev, double* centres_dev, int* iterations, hdf_stream stream) {
    if (!x_dev || !init_host || !labels_dev || n < 1 || d < 1 || d > HDF_MAX_D || k < 1 || k > n ||
        (int64_t)k * d > 6144 || max_iter < 1)
        return fail(HDF_EINVAL, "hdf_kmeans: bad argument (1 <= k <= n, k d <= 6144, 1 <= d <= 8)");
    for (int c = 0; c < k; ++c)
        if (init_host[c] < 0 || init_host[c] >= n) return fail(HDF_EINVAL, "hdf_kmeans: initial index out of range");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf C, idx, part, chg;
    HDF_CUDA(C.alloc_on(sizeof(double) * k * d, st));
    HDF_CUDA(idx.alloc_on(sizeof(int64_t) * k, st));
    HDF_CUDA(cudaMemcpyAsync(idx.p, init_host, sizeof(int64_t) * k, cudaMemcpyHostToDevice, st));
    HDF_COUNT_LAUNCH();
    k_gather_rows<<<blocks_for((int64_t)k * d, 256, 1 << 30), 256, 0, st>>>(x_dev, d, idx.as<int64_t>(), k,
                                                                           C.as<double>());
    HDF_CUDA(cudaMemsetAsync(labels_dev, 0xff, sizeof(int) * n, st));      // -1: every label changes first
    const int G = blocks_for(n, 2048, 512);
    const int64_t chunk = (n + G - 1) / G;
    HDF_CUDA(part.alloc_on(sizeof(double) * (size_t)G * k * (d + 1), st));
    HDF_CUDA(chg.alloc_on(sizeof(int), st));
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        HDF_CUDA(cudaMemsetAsync(chg.p, 0, sizeof(int), st));
        HDF_COUNT_LAUNCH();
        k_km_assign<<<blocks_for(n, 256, 1 << 30), 256, sizeof(double) * k * d, st>>>(x_dev, n, d, k, C.as<double>(),
                                                                                     labels_dev, chg.as<int>());
        HDF_CUDA(cudaGetLastError());
        int changes = 0;
        HDF_CUDA(cudaMemcpyAsync(&changes, chg.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        if (changes == 0 && it > 1) break;
        HDF_COUNT_LAUNCH();
        k_km_partial<<<G, 256, 0, st>>>(x_dev, n, d, k, labels_dev, chunk, part.as<double>());
        HDF_COUNT_LAUNCH();
        k_km_finish<<<blocks_for(k, 128, 1 << 20), 128, 0, st>>>(part.as<double>(), G, k, d, C.as<double>());
        HDF_CUDA(cudaGetLastError());
    }
    if (it > max_iter) it = max_iter;
    if (centres_dev) HDF_CUDA(cudaMemcpyAsync(centres_dev, C.p, sizeof(double) * k * d, cudaMemcpyDeviceToDevice, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    if (iterations) *iterations = it;
    return HDF_OK;
}

hdf_status hdf_kernel_matvec(const double* xq_dev, int64_t m, const double* x_dev, int64_t n, int d,
                             hdf_kernel kernel, double lengthscale, const double* w_dev, double* out_dev,
                             hdf_stream stream) {
    if (!xq_dev || !x_dev || !w_dev || !out_dev || m < 1 || n < 1 || d < 1 || d > HDF_MAX_D || kernel < 0 ||
        kernel > 3 || !(lengthscale > 0))
        return fail(HDF_EINVAL, "hdf_kernel_matvec: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf a, b, part;
    HDF_CUDA(a.alloc_on(sizeof(float) * m * d, st));
    HDF_CUDA(b.alloc_on(sizeof(float) * n * d, st));
    HDF_COUNT_LAUNCH();
    k_shift_f32<<<blocks_for(m * d, 256, 1 << 30), 256, 0, st>>>(xq_dev, m, d, x_dev, a.as<float>());
    HDF_COUNT_LAUNCH();
    k_shift_f32<<<blocks_for(n * d, 256, 1 << 30), 256, 0, st>>>(x_dev, n, d, x_dev, b.as<float>());
    int S = 1;
    const int64_t split = direct_split(m, n, &S);
    HDF_CUDA(part.alloc_on(sizeof(double) * (size_t)S * m, st));
    dim3 g((unsigned)((m + kDkRows - 1) / kDkRows), (unsigned)S);
    HDF_COUNT_LAUNCH();
    launch_direct(d, g, st, a.as<float>(), m, b.as<float>(), n, kernel, (float)(1.0 / lengthscale), w_dev, nullptr,
                  nullptr, split, part.as<double>());
    HDF_COUNT_LAUNCH();
    k_direct_finish<<<blocks_for(m, 256, 1 << 30), 256, 0, st>>>(part.as<double>(), S, m, 0.0, nullptr, nullptr,
                                                                 out_dev);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

hdf_status hdf_krr_build(const double* x_dev, int64_t n, int d, const int* labels_dev, hdf_kernel kernel,
                         double lengthscale, double lambda, double tol, hdf_precision prec, const hdf_options* opt,
                         hdf_stream stream, hdf_krr** out) {
    if (out) *out = nullptr;
    if (!x_dev || !labels_dev || !out || n < 1 || d < 3 || d > HDF_MAX_D || kernel < 0 || kernel > 3 ||
        !(lengthscale > 0) || !(lambda > 0) || !(tol > 0 && tol < 1) || (prec != HDF_FP64 && prec != HDF_FP32))
        return fail(HDF_EINVAL, "hdf_krr_build: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double t0 = wall_ms();
    // clusters in label order (empty labels dropped), points permuted cluster by cluster
    std::vector<int> lab(n);
    HDF_CUDA(cudaMemcpyAsync(lab.data(), labels_dev, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    int lmax = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (lab[i] < 0) return fail(HDF_EINVAL, "hdf_krr_build: negative label");
        lmax = std::max(lmax, lab[i]);
    }
    std::vector<int64_t> cnt((size_t)lmax + 1, 0);
    for (int64_t i = 0; i < n; ++i) cnt[lab[i]]++;
    std::vector<int> remap((size_t)lmax + 1, -1);
    hdf_krr* K = new hdf_krr();
    K->n = n; K->d = d; K->prec = prec; K->kernel = kernel; K->ell = lengthscale; K->lam = lambda;
    K->offs.push_back(0);
    for (int c = 0; c <= lmax; ++c)
        if (cnt[c] > 0) { remap[c] = (int)K->offs.size() - 1; K->offs.push_back(K->offs.back() + cnt[c]); }
    K->nclus = (int)K->offs.size() - 1;
    std::vector<int64_t> perm(n), pos(K->offs.begin(), K->offs.end() - 1);
    std::vector<int> clp(n);
    for (int64_t i = 0; i < n; ++i) {
        const int c = remap[lab[i]];
        perm[pos[c]] = i;
        clp[pos[c]++] = c;
    }
    auto bail = [&](hdf_status s) { delete K; return s; };
    hdf_status s = HDF_OK;
#define KRR_CUDA(call)                                                                            \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? HDF_ENOMEM : HDF_ECUDA,                \
                             std::string(#call) + ": " + cudaGetErrorString(e_)));                    \
    } while (0)
    KRR_CUDA(K->perm.alloc(sizeof(int64_t) * n));
    KRR_CUDA(K->xp.alloc(sizeof(double) * n * d));
    KRR_CUDA(K->xp32.alloc(sizeof(float) * n * d));
    KRR_CUDA(K->cl.alloc(sizeof(int) * n));
    KRR_CUDA(K->doffs.alloc(sizeof(int64_t) * K->offs.size()));
    KRR_CUDA(cudaMemcpyAsync(K->perm.p, perm.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    KRR_CUDA(cudaMemcpyAsync(K->cl.p, clp.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    KRR_CUDA(cudaMemcpyAsync(K->doffs.p, K->offs.data(), sizeof(int64_t) * K->offs.size(), cudaMemcpyHostToDevice, st));
    HDF_COUNT_LAUNCH();
    k_gather_rows<<<blocks_for(n * d, 256, 1 << 30), 256, 0, st>>>(x_dev, d, K->perm.as<int64_t>(), n, K->xp.as<double>());
    HDF_COUNT_LAUNCH();
    k_shift_f32<<<blocks_for(n * d, 256, 1 << 30), 256, 0, st>>>(K->xp.as<double>(), n, d, K->xp.as<double>(),
                                                                 K->xp32.as<float>());
    KRR_CUDA(cudaGetLastError());
    // HDF factors of the diagonal blocks: one batched build over the clusters
    std::vector<double> ells(K->nclus, lengthscale);
    s = hdf_build_batched(K->nclus, K->offs.data(), K->xp.as<double>(), d, kernel, ells.data(), tol, prec, opt, stream,
                          &K->batch);
    if (s != HDF_OK && s != HDF_ETOL_UNREACHABLE) return bail(s);
    const hdf_status build_status = s;
    K->t_build = wall_ms() - t0;
    // block preconditioner: exact blocks, inverted on the device (Cholesky, FP64)
    const double t1 = wall_ms();
    K->ioff.assign(K->nclus + 1, 0);
    for (int c = 0; c < K->nclus; ++c) {
        const int64_t nc = K->offs[c + 1] - K->offs[c];
        K->ioff[c + 1] = K->ioff[c] + nc * nc;
    }
    if (K->ioff.back() > ((int64_t)1 << 28))
        return bail(fail(HDF_ETOOBIG, "hdf_krr_build: sum of squared cluster sizes > 2^28 (block preconditioner)"));
    KRR_CUDA(K->dioff.alloc(sizeof(int64_t) * K->ioff.size()));
    KRR_CUDA(cudaMemcpyAsync(K->dioff.p, K->ioff.data(), sizeof(int64_t) * K->ioff.size(), cudaMemcpyHostToDevice, st));
    KRR_CUDA(K->inv.alloc(sizeof(double) * std::max<int64_t>(1, K->ioff.back())));
    {
        int64_t nmax = 0;
        for (int c = 0; c < K->nclus; ++c) nmax = std::max(nmax, K->offs[c + 1] - K->offs[c]);
        dim3 g((unsigned)blocks_for(nmax * nmax, 256, 4096), (unsigned)K->nclus);
        HDF_COUNT_LAUNCH();
        k_block_matrices<<<g, 256, 0, st>>>(K->xp.as<double>(), d, K->doffs.as<int64_t>(), K->dioff.as<int64_t>(),
                                            K->nclus, kernel, lengthscale, lambda, K->inv.as<double>());
        KRR_CUDA(cudaGetLastError());
    }
    {
        // invert every block on the device (batched tiles; see k_spd_potrf and its siblings)
        int nbmax = 0;
        std::vector<int64_t> doff(K->nclus + 1, 0);
        for (int c = 0; c < K->nclus; ++c) {
            const int nb = (int)((K->offs[c + 1] - K->offs[c] + kST - 1) / kST);
            nbmax = std::max(nbmax, nb);
            doff[c + 1] = doff[c] + (int64_t)nb * kST * kST;
        }
        DevBuf W, D, ddoff, bad;
        KRR_CUDA(W.alloc_on(sizeof(double) * std::max<int64_t>(1, K->ioff.back()), st));
        KRR_CUDA(D.alloc_on(sizeof(double) * std::max<int64_t>(1, doff.back()), st));
        KRR_CUDA(ddoff.alloc_on(sizeof(int64_t) * doff.size(), st));
        KRR_CUDA(bad.alloc_on(sizeof(int), st));
        KRR_CUDA(cudaMemcpyAsync(ddoff.p, doff.data(), sizeof(int64_t) * doff.size(), cudaMemcpyHostToDevice, st));
        KRR_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
        SpdArgs P{K->inv.as<double>(), W.as<double>(), D.as<double>(), K->doffs.as<int64_t>(),
                  K->dioff.as<int64_t>(), ddoff.as<int64_t>(), bad.as<int>()};
        const int tile = (int)(sizeof(double) * kST * kSP);
        KRR_CUDA(cudaFuncSetAttribute(k_spd_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * tile));
        KRR_CUDA(cudaFuncSetAttribute(k_spd_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * tile));
        KRR_CUDA(cudaFuncSetAttribute(k_spd_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * tile));
        KRR_CUDA(cudaFuncSetAttribute(k_spd_winv, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * tile));
        KRR_CUDA(cudaFuncSetAttribute(k_spd_wtw, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * tile));
        const unsigned ncl = (unsigned)K->nclus;
        for (int j = 0; j < nbmax; ++j) {
            HDF_COUNT_LAUNCH();
            k_spd_potrf<<<dim3(1, ncl), 256, 2 * tile, st>>>(P, j);
            const int nt = nbmax - j - 1;
            if (nt > 0) {
                HDF_COUNT_LAUNCH();
                k_spd_trsm<<<dim3((unsigned)nt, ncl), 256, 2 * tile, st>>>(P, j);
                HDF_COUNT_LAUNCH();
                k_spd_update<<<dim3((unsigned)(nt * (nt + 1) / 2), ncl), 256, 3 * tile, st>>>(P, j);
            }
        }
        for (int i = 0; i < nbmax; ++i) {
            HDF_COUNT_LAUNCH();
            k_spd_winv<<<dim3((unsigned)(i + 1), ncl), 256, 3 * tile, st>>>(P, i);
        }
        HDF_COUNT_LAUNCH();
        k_spd_wtw<<<dim3((unsigned)(nbmax * (nbmax + 1) / 2), ncl), 256, 2 * tile, st>>>(P);
        KRR_CUDA(cudaGetLastError());
        int hbad = 0;
        KRR_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        KRR_CUDA(cudaStreamSynchronize(st));
        if (hbad) return bail(fail(HDF_ESINGULAR, "hdf_krr_build: a block lambda I + K_cc is not positive definite"));
    }
    // work space
    K->split = direct_split(n, n, &K->S);
    KRR_CUDA(K->part.alloc(sizeof(double) * (size_t)K->S * n));
    KRR_CUDA(K->hd.alloc(sizeof(double) * n));
    KRR_CUDA(K->dotp.alloc(sizeof(double) * 512));
    if (prec == HDF_FP32) {
        KRR_CUDA(K->vb.alloc(sizeof(float) * n));
        KRR_CUDA(K->yb.alloc(sizeof(float) * n));
    }
    KRR_CUDA(cudaStreamSynchronize(st));
    K->t_precond = wall_ms() - t1;
#undef KRR_CUDA
    *out = K;
    return build_status;
}

hdf_status hdf_krr_apply(hdf_krr* K, const double* v_dev, double* out_dev, hdf_stream stream) {
    if (!K || !v_dev || !out_dev) return fail(HDF_EINVAL, "hdf_krr_apply: null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf vp, tp;
    HDF_CUDA(vp.alloc_on(sizeof(double) * K->n, st));
    HDF_CUDA(tp.alloc_on(sizeof(double) * K->n, st));
    const int gb = blocks_for(K->n, 256, 1 << 30);
    HDF_COUNT_LAUNCH();
    k_gather_vec<<<gb, 256, 0, st>>>(v_dev, K->perm.as<int64_t>(), K->n, vp.as<double>());
    if (hdf_status s = apply_perm(K, vp.as<double>(), tp.as<double>(), st); s != HDF_OK) return s;
    HDF_COUNT_LAUNCH();
    k_scatter_vec<<<gb, 256, 0, st>>>(tp.as<double>(), K->perm.as<int64_t>(), K->n, out_dev);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

hdf_status hdf_krr_precond(hdf_krr* K, const double* r_dev, double* z_dev, hdf_stream stream) {
    if (!K || !r_dev || !z_dev) return fail(HDF_EINVAL, "hdf_krr_precond: null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf rp, zp;
    HDF_CUDA(rp.alloc_on(sizeof(double) * K->n, st));
    HDF_CUDA(zp.alloc_on(sizeof(double) * K->n, st));
    const int gb = blocks_for(K->n, 256, 1 << 30);
    HDF_COUNT_LAUNCH();
    k_gather_vec<<<gb, 256, 0, st>>>(r_dev, K->perm.as<int64_t>(), K->n, rp.as<double>());
    if (hdf_status s = precond_perm(K, rp.as<double>(), zp.as<double>(), st); s != HDF_OK) return s;
    HDF_COUNT_LAUNCH();
    k_scatter_vec<<<gb, 256, 0, st>>>(zp.as<double>(), K->perm.as<int64_t>(), K->n, z_dev);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

hdf_status hdf_krr_solve(hdf_krr* K, const double* y_dev, double rtol, int max_iter, double* w_dev, int* iterations,
                         double* relres, hdf_stream stream) {
    if (!K || !y_dev || !w_dev || !(rtol > 0) || max_iter < 1) return fail(HDF_EINVAL, "hdf_krr_solve: bad argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = K->n;
    DevBuf buf;
    HDF_CUDA(buf.alloc_on(sizeof(double) * 5 * n, st));
    double *x = buf.as<double>(), *r = x + n, *z = r + n, *p = z + n, *q = p + n;
    const int gb = blocks_for(n, 256, 1 << 30);
    HDF_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    HDF_COUNT_LAUNCH();
    k_gather_vec<<<gb, 256, 0, st>>>(y_dev, K->perm.as<int64_t>(), n, r);
    if (hdf_status s = precond_perm(K, r, z, st); s != HDF_OK) return s;
    HDF_CUDA(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    double rz = 0.0, bb = 0.0;
    if (hdf_status s = dot2(K, r, z, r, r, &rz, &bb, st); s != HDF_OK) return s;
    const double nb = std::sqrt(bb);
    int it = 0;
    double res = (nb > 0.0) ? 1.0 : 0.0;
    if (nb > 0.0) {
        for (it = 1; it <= max_iter; ++it) {
            if (hdf_status s = apply_perm(K, p, q, st); s != HDF_OK) return s;
            double pq = 0.0;
            if (hdf_status s = dot2(K, p, q, nullptr, nullptr, &pq, nullptr, st); s != HDF_OK) return s;
            if (!(pq > 0.0)) return fail(HDF_ESINGULAR, "hdf_krr_solve: the operator is not positive definite");
            const double alpha = rz / pq;
            HDF_COUNT_LAUNCH();
            k_cg_step<<<gb, 256, 0, st>>>(x, r, p, q, alpha, n);
            HDF_CUDA(cudaGetLastError());
            if (hdf_status s = precond_perm(K, r, z, st); s != HDF_OK) return s;
            double rz_new = 0.0, rr = 0.0;
            if (hdf_status s = dot2(K, r, z, r, r, &rz_new, &rr, st); s != HDF_OK) return s;
            res = std::sqrt(rr) / nb;
            if (res <= rtol) break;
            HDF_COUNT_LAUNCH();
            k_cg_dir<<<gb, 256, 0, st>>>(p, z, rz_new / rz, n);
            HDF_CUDA(cudaGetLastError());
            rz = rz_new;
        }
        if (it > max_iter) it = max_iter;
    }
    HDF_COUNT_LAUNCH();
    k_scatter_vec<<<gb, 256, 0, st>>>(x, K->perm.as<int64_t>(), n, w_dev);
    HDF_CUDA(cudaGetLastError());
    HDF_CUDA(cudaStreamSynchronize(st));
    if (iterations) *iterations = it;
    if (relres) *relres = res;
    return (res <= rtol) ? HDF_OK : fail(HDF_ETOL_UNREACHABLE, "hdf_krr_solve: max_iter reached before rtol");
}

hdf_status hdf_krr_info(const hdf_krr* K, int* nclusters, int64_t* rank_total, double* t_ms) {
    if (!K) return fail(HDF_EINVAL, "hdf_krr_info: null argument");
    if (nclusters) *nclusters = K->nclus;
    if (rank_total) {
        int64_t tot = 0;
        for (int c = 0; c < K->nclus; ++c) {
            hdf_info I;
            if (hdf_status s = hdf_batch_info(K->batch, c, &I); s != HDF_OK) return s;
            tot += I.rank;
        }
        *rank_total = tot;
    }
    if (t_ms) { t_ms[0] = K->t_build; t_ms[1] = K->t_precond; }
    return HDF_OK;
}

void hdf_krr_free(hdf_krr* K) {
    if (!K) return;
    cudaDeviceSynchronize();
    delete K;
}

}  // extern "C"
