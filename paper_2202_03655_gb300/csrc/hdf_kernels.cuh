// Device kernels of the HDF factorization for sm_103a.
//
// Layout in HBM (all row-major unless stated):
//   x   n x d FP64 points (input, caller-owned)
//   F   n x ldF radial factors F[i, (k,s)] = f_{k,s}(|x'_i|)   (bulk type T)
//   U   n x ldU factor, column (k, s, h) = F[i, (k,s)] * Y_k^h(x_hat_i)   (bulk type T)
//   V,Y column-major n x c blocks (caller-owned)
// Every reduction over points is two-stage (per-block partials, then a fixed-order
// sum), so results do not depend on scheduling.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hdf {
namespace dev {

constexpr int kMaxD = 8;

struct Center {
    double c[kMaxD];
};

// ----------------------------------------------------------------- kernel values
__device__ __forceinline__ double kernel_value(int kernel, double r, double ell) {
    const double z = fabs(r) / ell;
    switch (kernel) {
        case 0: return exp(-0.5 * z * z);
        case 1: return 1.0 / (1.0 + z * z);
        case 2: { const double s = 1.7320508075688772 * z; return (1.0 + s) * exp(-s); }
        default: { const double s = 2.23606797749979 * z; return (1.0 + s + s * s / 3.0) * exp(-s); }
    }
}

// The same kernels in FP32 (r >= 0, inv_ell = 1 / l); values <= 1.
__device__ __forceinline__ float kernel_value_f(int kernel, float r, float inv_ell) {
    const float z = r * inv_ell;
    switch (kernel) {
        case 0: return expf(-0.5f * z * z);
        case 1: return 1.0f / (1.0f + z * z);
        case 2: { const float s = 1.7320508f * z; return (1.0f + s) * expf(-s); }
        default: { const float s = 2.2360680f * z; return (1.0f + s + s * s * (1.0f / 3.0f)) * expf(-s); }
    }
}

// Deterministic tree sum of one double per thread over the block (blockDim = 256).
__device__ __forceinline__ double block_sum_256(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double out = sh[0];
    __syncthreads();
    return out;
}

// ------------------------------------------------------------- A0: centre, radius
// part[b*d + j] = sum over the block's chunk of x[i, j].
static __global__ void k_sum_partial(const double* __restrict__ x, int64_t n, int d, int64_t chunk,
                              double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double acc[kMaxD];
#pragma unroll
    for (int j = 0; j < kMaxD; ++j) acc[j] = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x)
        for (int j = 0; j < d; ++j) acc[j] += x[i * d + j];
    for (int j = 0; j < d; ++j) {
        const double s = block_sum_256(acc[j], sh);
        if (threadIdx.x == 0) part[blockIdx.x * d + j] = s;
    }
}

// part[b] = max over the block's chunk of |x_i - c|^2.
static __global__ void k_maxnorm_partial(const double* __restrict__ x, int64_t n, int d, int64_t chunk,
                                  Center c, double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double m = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) { const double y = x[i * d + j] - c.c[j]; s += y * y; }
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

// Mean-square kernel value over the subsample idx(t) = floor(t n / m), t < m:
// part[t] = sum_u k(|x_idx(t) - x_idx(u)|)^2.
static __global__ void k_mu2_rows(const double* __restrict__ x, int64_t n, int d, int m, int kernel,
                           double ell, double* __restrict__ part) {
    __shared__ double sh[256];
    const int t = blockIdx.x;
    const int64_t i = ((int64_t)t * n) / m;
    double xi[kMaxD];
    for (int j = 0; j < d; ++j) xi[j] = x[i * d + j];
    double acc = 0.0;
    for (int u = threadIdx.x; u < m; u += blockDim.x) {
        const int64_t jj = ((int64_t)u * n) / m;
        double s = 0.0;
        for (int j = 0; j < d; ++j) { const double y = xi[j] - x[jj * d + j]; s += y * y; }
        const double kv = kernel_value(kernel, sqrt(s), ell);
        acc += kv * kv;
    }
    const double tot = block_sum_256(acc, sh);
    if (threadIdx.x == 0) part[t] = tot;
}

// Cross-pair version for K(X, Y): part[t] = sum_u k(|x_ix(t) - y_iy(u)|)^2 over the strided
// subsamples ix(t) = floor(t m / mx), t < mx, of X and iy(u) = floor(u n / my), u < my, of Y.
static __global__ void k_mu2_cross(const double* __restrict__ x, int64_t m, int mx, const double* __restrict__ y,
                                   int64_t n, int my, int d, int kernel, double ell, double* __restrict__ part) {
    __shared__ double sh[256];
    const int t = blockIdx.x;
    const int64_t i = ((int64_t)t * m) / mx;
    double xi[kMaxD];
    for (int j = 0; j < d; ++j) xi[j] = x[i * d + j];
    double acc = 0.0;
    for (int u = threadIdx.x; u < my; u += blockDim.x) {
        const int64_t jj = ((int64_t)u * n) / my;
        double s = 0.0;
        for (int j = 0; j < d; ++j) { const double z = xi[j] - y[jj * d + j]; s += z * z; }
        const double kv = kernel_value(kernel, sqrt(s), ell);
        acc += kv * kv;
    }
    const double tot = block_sum_256(acc, sh);
    if (threadIdx.x == 0) part[t] = tot;
}

// ----------------------------------------------------- A3: radial-basis Gram matrices
// B0[l] = T_l(u), l <= L and B1[l] = rho T_l(u), l < L, u = 8 rho^2 - 1, rho = |x - c|/(2R).
// part[b][q] (q < npairs) = sum_i B0[l] B0[l'] and part[b][npairs + q] = sum_i rho^2 T_l T_l'
// over the block's chunk, for the pairs (l, l') = pairs[q], l <= l'.
constexpr int kGramTile = 64;
constexpr int kGramMaxQ = 9;     // ceil(npairs / 256) for L <= 64

static __global__ void __launch_bounds__(256) k_radial_gram(const double* __restrict__ x, int64_t n, int d,
                                                     int64_t chunk, Center c, double inv2R, int L,
                                                     const uint16_t* __restrict__ pairs, int npairs,
                                                     double* __restrict__ part) {
    extern __shared__ double smem[];
    const int LP1 = L + 1;
    double* Ts = smem;                          // [kGramTile][LP1]
    double* r2 = smem + kGramTile * LP1;        // [kGramTile]
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double a0[kGramMaxQ], a1[kGramMaxQ];
#pragma unroll
    for (int q = 0; q < kGramMaxQ; ++q) { a0[q] = 0.0; a1[q] = 0.0; }
    for (int64_t t0 = i0; t0 < i1; t0 += kGramTile) {
        const int cnt = (int)min((int64_t)kGramTile, i1 - t0);
        if (threadIdx.x < kGramTile) {
            const int p = threadIdx.x;
            double* T = Ts + p * LP1;
            if (p < cnt) {
                const int64_t i = t0 + p;
                double s = 0.0;
                for (int j = 0; j < d; ++j) { const double y = (x[i * d + j] - c.c[j]) * inv2R; s += y * y; }
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
        for (int q = 0; q < kGramMaxQ; ++q) {
            const int pi = threadIdx.x + 256 * q;
            if (pi < npairs) {
                const int l = pairs[2 * pi], lp = pairs[2 * pi + 1];
                double s0 = 0.0, s1 = 0.0;
                for (int p = 0; p < cnt; ++p) {
                    const double v = Ts[p * LP1 + l] * Ts[p * LP1 + lp];
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
    for (int q = 0; q < kGramMaxQ; ++q) {
        const int pi = threadIdx.x + 256 * q;
        if (pi < npairs) {
            part[(int64_t)blockIdx.x * 2 * npairs + pi] = a0[q];
            part[(int64_t)blockIdx.x * 2 * npairs + npairs + pi] = a1[q];
        }
    }
}

// Chebyshev moments of the radial data: part[b][j] = sum over the block's chunk of T_j(u_i),
// u_i = 8 rho_i^2 - 1, j < nmom.  The radial-basis Gram matrices follow from them exactly
// (T_l T_l' = (T_{l+l'} + T_{|l-l'|}) / 2 and u T_j = (T_{j+1} + T_{|j-1|}) / 2), so the Gram
// costs O(n L) instead of O(n L^2).
constexpr int kMomTile = 64;

static __global__ void __launch_bounds__(256) k_radial_moments(const double* __restrict__ x, int64_t n, int d,
                                                               int64_t chunk, Center c, double inv2R, int nmom,
                                                               double* __restrict__ part) {
    extern __shared__ double smem[];
    double* Ts = smem;                          // [kMomTile][nmom]
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    double acc0 = 0.0, acc1 = 0.0;              // moments threadIdx.x and threadIdx.x + 256
    for (int64_t t0 = i0; t0 < i1; t0 += kMomTile) {
        const int cnt = (int)min((int64_t)kMomTile, i1 - t0);
        if (threadIdx.x < kMomTile) {
            const int p = threadIdx.x;
            double* T = Ts + p * nmom;
            if (p < cnt) {
                const int64_t i = t0 + p;
                double s = 0.0;
                for (int j = 0; j < d; ++j) { const double y = (x[i * d + j] - c.c[j]) * inv2R; s += y * y; }
                const double u = 8.0 * s - 1.0;
                T[0] = 1.0;
                if (nmom > 1) T[1] = u;
                for (int l = 2; l < nmom; ++l) T[l] = 2.0 * u * T[l - 1] - T[l - 2];
            } else {
                for (int l = 0; l < nmom; ++l) T[l] = 0.0;
            }
        }
        __syncthreads();
        if (threadIdx.x < nmom) {
            double s = 0.0;
            for (int p = 0; p < cnt; ++p) s += Ts[p * nmom + threadIdx.x];
            acc0 += s;
        }
        if (threadIdx.x + 256 < nmom) {
            double s = 0.0;
            for (int p = 0; p < cnt; ++p) s += Ts[p * nmom + threadIdx.x + 256];
            acc1 += s;
        }
        __syncthreads();
    }
    if (threadIdx.x < nmom) part[(int64_t)blockIdx.x * nmom + threadIdx.x] = acc0;
    if (threadIdx.x + 256 < nmom) part[(int64_t)blockIdx.x * nmom + threadIdx.x + 256] = acc1;
}

// out[j] = sum_b part[b * ncols + j] in block order.
static __global__ void k_reduce_cols(const double* __restrict__ part, int nblk, int64_t ncols,
                              double* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * ncols + j];
    out[j] = s;
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// ------------------------------------------------------------- A5a: radial factors
// Per point: B_par (FP64) -> Q_par = B_par Qmat_par (FP64, the orthonormalised radial basis
// of Eq. svd) -> F[i, col] = sum_l Q_par(col)[l] Wt[l, col] (type T).  Tiles of 32 points.
constexpr int kFTile = 32;

struct RFParams {
    const double* x; int64_t n; int d; Center c; double inv2R; int L;
    const double* Qm0; int nb0, m0;
    const double* Qm1; int nb1, m1;
    const float2* QC; int mtp;   // FP32 factors: [Qm0 | Qm1] as (hi, lo) float pairs, (L+1) x mtp
    int kopt;                    // FP32 factors in the batched build: outputs per thread of the Q part
    int stage_wt;                // FP32 factors: copy Wt into shared memory
    const void* Wt; const uint8_t* colpar; int nF;
    void* F; int64_t ldF;
};

// Dynamic shared memory of one radial tile, in bytes.
__host__ __device__ inline size_t radialF_smem(int L, int m0, int m1, size_t tsize) {
    return sizeof(double) * (kFTile * (L + 1) + kFTile) + tsize * (size_t)(m0 + m1) * kFTile;
}

// Compensated FP32 arithmetic for the radial basis of FP32 factors.  Q = B Qmat cancels (Qmat
// grows like the inverse square root of the smallest kept Gram eigenvalue), so a plain FP32
// sum is not enough; FP64 is, but runs at a small fraction of the FP32 rate on this GPU.  The
// basis values and Qmat are carried as unevaluated (hi, lo) float pairs (about 48 bits) and the
// dot product uses error-free transformations: TwoProd by fma (Dekker/Kahan) and TwoSum
// (Knuth), the "Dot2" scheme of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26, 2005), whose
// result is as accurate as a sum in twice the working precision.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// One Dot2 step: (sh, c) accumulates a * (bh + bl), a = (hi, lo).
__device__ __forceinline__ void dot2_step(float2 a, float bh, float bl, float& sh, float& c) {
    const float ph = a.x * bh;
    float pe = fmaf(a.x, bh, -ph);
    pe = fmaf(a.x, bl, fmaf(a.y, bh, pe));
    float s2, es;
    two_sum(sh, ph, s2, es);
    sh = s2;
    c += es + pe;
}

// FP32 factors (k_radial_F_df), one tile of kFTile points in three parts:
//   basis: u = 8 rho^2 - 1 and T_l(u) by the FP64 recurrence, split into (hi, lo) float pairs;
//   Q:     Q[o][p] = sum_l T_l(u_p) Qmat[l][o] by Dot2 against QC, the combined even | odd Qmat as
//          float pairs ((L+1) x mtp, odd columns zero in row L, mtp a multiple of 8), times rho
//          for the odd outputs;
//   F:     F[p][col] = sum_l Q[par(col) block + l][p] Wt[l][col] in FP32.
// The basis of the next tile is computed by one warp while the others form this tile's Q.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

// Chebyshev moments for FP32 factors: sum over the points [i0, i1) of T_l(u), l < nmom,
// u = 8 rho^2 - 1, by one 256-thread block.  Each thread runs one point's recurrence in
// double-float arithmetic (FP32 pairs; FP64 runs at a small fraction of the FP32 rate here),
// the values pass through shared memory (Tsm: 256 rows of nmom + 1 float2, an odd stride that
// keeps the 8-byte accesses conflict-free), thread l < nmom adds moment l over the tile with
// error-free sums, and the tile sums are added in FP64.  Thread l returns moment l.
__device__ __forceinline__ double moments_df_range(const double* __restrict__ x, int d, const double* cc,
                                                   double inv2R, int nmom, int64_t i0, int64_t i1, float2* Tsm) {
    const int S = nmom + 1;
    double acc = 0.0;
    for (int64_t t0 = i0; t0 < i1; t0 += 256) {
        const int cnt = (int)min((int64_t)256, i1 - t0);
        const int p = threadIdx.x;
        if (p < cnt) {
            float2* T = Tsm + p * S;
            const int64_t i = t0 + p;
            double s = 0.0;
            for (int j = 0; j < d; ++j) { const double y = (x[i * d + j] - cc[j]) * inv2R; s += y * y; }
            const double u = 8.0 * s - 1.0;
            const float uh = (float)u, ul = (float)(u - (double)uh);
            const float u2h = 2.f * uh, u2l = 2.f * ul;
            float ah = 1.f, al = 0.f, bh = uh, bl = ul;
            T[0] = make_float2(1.f, 0.f);
            if (nmom > 1) T[1] = make_float2(uh, ul);
            for (int l = 2; l < nmom; ++l) {
                const float ph = u2h * bh;
                float pl = fmaf(u2h, bh, -ph);
                pl = fmaf(u2h, bl, fmaf(u2l, bh, pl));
                float sh, se;
                two_sum(ph, -ah, sh, se);
                se += pl - al;
                float th, tl;
                fast_two_sum(sh, se, th, tl);
                T[l] = make_float2(th, tl);
                ah = bh; al = bl;
                bh = th; bl = tl;
            }
        }
        __syncthreads();
        if (threadIdx.x < nmom) {
            float mh = 0.f, ml = 0.f;
            for (int q = 0; q < cnt; ++q) {
                const float2 v = Tsm[q * S + threadIdx.x];
                float sh, se;
                two_sum(mh, v.x, sh, se);
                se += ml + v.y;
                fast_two_sum(sh, se, mh, ml);
            }
            acc += (double)mh + (double)ml;
        }
        __syncthreads();
    }
    return acc;
}

// Drop-in for k_radial_moments (same part layout) for FP32 factors.
static __global__ void __launch_bounds__(256) k_radial_moments_df(const double* __restrict__ x, int64_t n, int d,
                                                                  int64_t chunk, Center c, double inv2R, int nmom,
                                                                  double* __restrict__ part) {
    extern __shared__ float2 tsm_raw[];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    const double v = moments_df_range(x, d, c.c, inv2R, nmom, i0, i1, tsm_raw);
    if (threadIdx.x < nmom) part[(int64_t)blockIdx.x * nmom + threadIdx.x] = v;
}

// Basis values of one point in double-float arithmetic (FP32 pairs, about 48 bits): u and rho
// from FP64 coordinates (a few FP64 operations), then T_l(u) = 2 u T_{l-1} - T_{l-2} with
// error-free products and sums; the recurrence is stable on [-1, 1].
__device__ __forceinline__ void radialF_df_basis(const RFParams& P, int64_t t0, int p, float2* Ts, float* rh) {
    const int LP1 = P.L + 1;
    const int cnt = (int)min((int64_t)kFTile, P.n - t0);
    float2* Tp = Ts + p * LP1;
    double s = 0.0;
    if (p < cnt) {
        const int64_t i = t0 + p;
        for (int j = 0; j < P.d; ++j) { const double y = (P.x[i * P.d + j] - P.c.c[j]) * P.inv2R; s += y * y; }
    }
    const double u = 8.0 * s - 1.0;
    rh[p] = sqrtf((float)s);
    const float uh = (float)u, ul = (float)(u - (double)uh);
    const float u2h = 2.f * uh, u2l = 2.f * ul;                     // 2u, exact
    float ah = 1.f, al = 0.f, bh = uh, bl = ul;                       // T_{l-2}, T_{l-1}
    Tp[0] = make_float2(1.f, 0.f);
    if (P.L >= 1) Tp[1] = make_float2(uh, ul);
    for (int l = 2; l <= P.L; ++l) {
        // (ph, pl) = 2u * T_{l-1}
        const float ph = u2h * bh;
        float pl = fmaf(u2h, bh, -ph);
        pl = fmaf(u2h, bl, fmaf(u2l, bh, pl));
        // T_l = (ph, pl) - T_{l-2}
        float sh, se;
        two_sum(ph, -ah, sh, se);
        se += pl - al;
        float th, tl;
        fast_two_sum(sh, se, th, tl);
        Tp[l] = make_float2(th, tl);
        ah = bh; al = bl;
        bh = th; bl = tl;
    }
}

// Q part, by the nth compute threads (thread = point p and a group of kOpt outputs: each basis
// value read from shared memory serves kOpt outputs, one 16-byte load brings two outputs).
template <int kOpt = 8>
__device__ __forceinline__ void radialF_df_q(const RFParams& P, const float2* Ts, const float* rh, const float2* QC,
                                             float* Qs, int tid, int nth) {
    const int LP1 = P.L + 1;
    const int mt = P.m0 + P.m1;
    const int p = tid % kFTile;
    const float2* Tp = Ts + p * LP1;
    for (int o0 = (tid / kFTile) * kOpt; o0 < mt; o0 += (nth / kFTile) * kOpt) {
        float sh[kOpt], c[kOpt];
#pragma unroll
        for (int j = 0; j < kOpt; ++j) { sh[j] = 0.f; c[j] = 0.f; }
        for (int l = 0; l < LP1; ++l) {
            const float2 a = Tp[l];
            const float4* qr = reinterpret_cast<const float4*>(QC + (size_t)l * P.mtp + o0);
#pragma unroll
            for (int j2 = 0; j2 < kOpt / 2; ++j2) {
                const float4 b = qr[j2];
                dot2_step(a, b.x, b.y, sh[2 * j2], c[2 * j2]);
                dot2_step(a, b.z, b.w, sh[2 * j2 + 1], c[2 * j2 + 1]);
            }
        }
#pragma unroll
        for (int j = 0; j < kOpt; ++j) {
            const int o = o0 + j;
            if (o < mt) {
                float q = sh[j] + c[j];
                if (o >= P.m0) q *= rh[p];
                Qs[o * kFTile + p] = q;
            }
        }
    }
}

// F part: thread = column; Wt from shared memory (Ws, max(m0, m1) x nF) when staged.
__device__ __forceinline__ void radialF_df_f(const RFParams& P, int64_t t0, const float* Qs, const float* Ws,
                                             int tid, int nth) {
    const int cnt = (int)min((int64_t)kFTile, P.n - t0);
    float* F = reinterpret_cast<float*>(P.F);
    for (int col = tid; col < P.ldF; col += nth) {
        if (col >= P.nF) {                       // row padding: zeros, so that sectors are whole
#pragma unroll
            for (int p = 0; p < kFTile; ++p)
                if (p < cnt) F[(t0 + p) * P.ldF + col] = 0.f;
            continue;
        }
        const int par = P.colpar[col];
        const int ob = par ? P.m0 : 0, mp = par ? P.m1 : P.m0;
        float acc[kFTile];
#pragma unroll
        for (int p = 0; p < kFTile; ++p) acc[p] = 0.f;
#pragma unroll 4
        for (int l = 0; l < mp; ++l) {
            const float w = Ws[(size_t)l * P.nF + col];
            const float4* q = reinterpret_cast<const float4*>(Qs + (ob + l) * kFTile);
#pragma unroll
            for (int p4 = 0; p4 < kFTile / 4; ++p4) {
                const float4 v = q[p4];
                acc[4 * p4 + 0] += v.x * w;
                acc[4 * p4 + 1] += v.y * w;
                acc[4 * p4 + 2] += v.z * w;
                acc[4 * p4 + 3] += v.w * w;
            }
        }
#pragma unroll
        for (int p = 0; p < kFTile; ++p)
            if (p < cnt) F[(t0 + p) * P.ldF + col] = acc[p];
    }
}

// Radial factors of the points [t0, t0 + kFTile): block-wide, ends with a barrier.
template <typename T>
__device__ __forceinline__ void radialF_tile(const RFParams& P, int64_t t0, unsigned char* smem_raw) {
    const int LP1 = P.L + 1;
    double* Ts = reinterpret_cast<double*>(smem_raw);            // [kFTile][LP1]
    double* rh = Ts + kFTile * LP1;                              // [kFTile]
    T* Qs = reinterpret_cast<T*>(rh + kFTile);                   // [m0 + m1][kFTile]
    const T* Wt = reinterpret_cast<const T*>(P.Wt);
    T* F = reinterpret_cast<T*>(P.F);
    const int cnt = (int)min((int64_t)kFTile, P.n - t0);
    if (threadIdx.x < kFTile) {
        const int p = threadIdx.x;
        double* Tp = Ts + p * LP1;
        double s = 0.0;
        if (p < cnt) {
            const int64_t i = t0 + p;
            for (int j = 0; j < P.d; ++j) { const double y = (P.x[i * P.d + j] - P.c.c[j]) * P.inv2R; s += y * y; }
        }
        const double u = 8.0 * s - 1.0;
        rh[p] = sqrt(s);
        Tp[0] = 1.0;
        if (P.L >= 1) Tp[1] = u;
        for (int l = 2; l <= P.L; ++l) Tp[l] = 2.0 * u * Tp[l - 1] - Tp[l - 2];
    }
    __syncthreads();
    const int mt = P.m0 + P.m1;
    for (int idx = threadIdx.x; idx < mt * kFTile; idx += blockDim.x) {
        const int o = idx / kFTile, p = idx % kFTile;
        const double* Tp = Ts + p * LP1;
        double q = 0.0;
        if (o < P.m0) {
            for (int l = 0; l < P.nb0; ++l) q += Tp[l] * P.Qm0[l * P.m0 + o];
        } else {
            const int oo = o - P.m0;
            for (int l = 0; l < P.nb1; ++l) q += Tp[l] * P.Qm1[l * P.m1 + oo];
            q *= rh[p];
        }
        Qs[o * kFTile + p] = (T)q;
    }
    __syncthreads();
    for (int col = threadIdx.x; col < P.nF; col += blockDim.x) {
        const int par = P.colpar[col];
        const int ob = par ? P.m0 : 0, mp = par ? P.m1 : P.m0;
        T acc[kFTile];
#pragma unroll
        for (int p = 0; p < kFTile; ++p) acc[p] = (T)0;
        for (int l = 0; l < mp; ++l) {
            const T w = Wt[(int64_t)l * P.nF + col];
            const T* q = Qs + (ob + l) * kFTile;
#pragma unroll
            for (int p = 0; p < kFTile; ++p) acc[p] += q[p] * w;
        }
#pragma unroll
        for (int p = 0; p < kFTile; ++p)
            if (p < cnt) F[(t0 + p) * P.ldF + col] = acc[p];
    }
    __syncthreads();
}

// Per point: B_par (FP64) -> Q_par = B_par Qmat_par (FP64, the orthonormalised radial basis
// of Eq. svd) -> F[i, col] = sum_l Q_par(col)[l] Wt[l, col] (type T).  Tiles of 32 points.
template <typename T>
__global__ void __launch_bounds__(256) k_radial_F(RFParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t ntiles = (P.n + kFTile - 1) / kFTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) radialF_tile<T>(P, tile * kFTile, smem_raw);
}

// Shared memory of k_radial_F_df: QC, Wt (when staged), two buffers of basis values, Q.
__host__ __device__ inline size_t radialF_df_basis_bytes(int L) {
    return align16(sizeof(float2) * kFTile * (L + 1) + sizeof(float) * kFTile);
}
__host__ __device__ inline size_t radialF_df_smem(int L, int m0, int m1, int mtp, int nF, bool stage_wt) {
    const int mmax = m0 > m1 ? m0 : m1;
    return align16(sizeof(float2) * (size_t)(L + 1) * mtp) +
           (stage_wt ? align16(sizeof(float) * (size_t)mmax * nF) : 0) + 2 * radialF_df_basis_bytes(L) +
           sizeof(float) * (size_t)(m0 + m1) * kFTile;
}

// Outputs per thread of the Q part (2, 4 or 8) for mt outputs over qwarps warps: the fewest
// outputs per thread after rounding (each warp takes whole groups of kOpt outputs for its 32
// points), larger groups on ties (fewer shared loads per output).
__host__ __device__ inline int radialF_df_kopt(int mt, int qwarps) {
    int best = 8, cost = 1 << 30;
    for (int k = 8; k >= 2; k /= 2) {
        const int groups = (mt + k - 1) / k;
        const int c = ((groups + qwarps - 1) / qwarps) * k;
        if (c < cost) { cost = c; best = k; }
    }
    return best;
}

// FP32 factors, one CTA of kRfThreads per SM.  Per tile of kFTile points: warps 1.. form Q while
// warp 0 computes the basis values of the CTA's next tile into the other buffer, then all warps
// form F.  QC (and Wt when P.stage_wt) are staged per CTA.
constexpr int kRfThreads = 512;
template <int KOPT>
static __global__ void __launch_bounds__(kRfThreads, 1) k_radial_F_df(RFParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LP1 = P.L + 1;
    const int mmax = P.m0 > P.m1 ? P.m0 : P.m1;
    unsigned char* sp = smem_raw;
    float2* QC = reinterpret_cast<float2*>(sp);
    sp += align16(sizeof(float2) * (size_t)LP1 * P.mtp);
    const float* Ws = reinterpret_cast<const float*>(P.Wt);
    if (P.stage_wt) {
        float* w = reinterpret_cast<float*>(sp);
        for (int t = threadIdx.x; t < mmax * P.nF; t += blockDim.x) w[t] = reinterpret_cast<const float*>(P.Wt)[t];
        Ws = w;
        sp += align16(sizeof(float) * (size_t)mmax * P.nF);
    }
    float2* Tb[2];
    float* rb[2];
    for (int b = 0; b < 2; ++b) {
        Tb[b] = reinterpret_cast<float2*>(sp);
        rb[b] = reinterpret_cast<float*>(Tb[b] + kFTile * LP1);
        sp += radialF_df_basis_bytes(P.L);
    }
    float* Qs = reinterpret_cast<float*>(sp);
    for (int t = threadIdx.x; t < LP1 * P.mtp; t += blockDim.x) QC[t] = P.QC[t];
    const int64_t ntiles = (P.n + kFTile - 1) / kFTile;
    if (threadIdx.x < kFTile && blockIdx.x < ntiles) radialF_df_basis(P, blockIdx.x * kFTile, threadIdx.x, Tb[0], rb[0]);
    __syncthreads();
    int cur = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (threadIdx.x < 32) {
            const int64_t nxt = tile + gridDim.x;
            if (nxt < ntiles && threadIdx.x < kFTile) radialF_df_basis(P, nxt * kFTile, threadIdx.x, Tb[cur ^ 1], rb[cur ^ 1]);
        } else {
            radialF_df_q<KOPT>(P, Tb[cur], rb[cur], QC, Qs, threadIdx.x - 32, kRfThreads - 32);
        }
        __syncthreads();
        radialF_df_f(P, tile * kFTile, Qs, Ws, threadIdx.x, kRfThreads);
        __syncthreads();
        cur ^= 1;
    }
}

// ------------------------------------------------------- A5b: harmonics and U writer
// One warp per point.  Solid-harmonic form of the real hyperspherical harmonics:
//   Y = prod_j P_j(|mu_{j+1}|, mu_j - |mu_{j+1}|) * N_phi * {Re|Im} (x0 + i x1)^{|mu_{d-2}|},
//   P_j(m, n) = s_n r_j^n C_n^{m + alpha_j}(x_{D_j} / r_j),  D_j = d-1-j, r_j^2 = sum_{i<=D_j} x_i^2,
// a polynomial in (x_{D_j}, r_j^2) from the normalised three-term recurrence (coefA/coefB).
// Per-warp shared: level tables, trig powers, Y for all used harmonics, the point's F row.
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float4 type; static constexpr int w = 4; };
template <> struct Vec2<double> { typedef double2 type; static constexpr int w = 2; };

struct UWParams {
    const double* x; int64_t n; int d; Center c; double inv2R;
    int L;                     // highest harmonic degree with kept columns
    int tri;                   // (L+1)(L+2)/2
    const int16_t* chains;     // nH x cstride: level offsets, trig index, zero padding
    int nH, cstride;
    const int32_t* ychain;     // nYp padded harmonic slots -> chain (-1: padding)
    const int32_t* gslot;      // nH: padded slot of each harmonic
    int nYp;
    const uint32_t* qdesc;     // ldU / VW chunks, two words each (see make_tables)
    int nF;
    const void* F; int64_t ldF;
    void* U; int64_t ldU;
    const void* coefA; const void* coefB;   // (d-2) x tri, type T
    int per_warp;              // shared elements (type T) per warp
    int tab_bytes;             // bytes of index tables staged in shared memory (0: read from global)
};

// The index tables the U writer reads for every point (global, or staged in shared memory).
struct UWTabs {
    const uint32_t* qdesc;     // two words per chunk (see make_tables)
    const int16_t* chains;
    const int32_t* gslot;
    const int32_t* ychain;
};

// Bytes of the staged index tables: qdesc, chains, gslot, and ychain when harmonics are not
// precomputed; the kernel lays them out in this order, each 16-byte aligned.
__host__ __device__ inline size_t uwriter_tab_bytes(int64_t nq, int nH, int cstride, int nYp, bool pre) {
    return align16(sizeof(uint32_t) * 2 * nq) + align16(sizeof(int16_t) * (size_t)nH * cstride) +
           align16(sizeof(int32_t) * (size_t)nH) + (pre ? 0 : align16(sizeof(int32_t) * (size_t)nYp));
}

// Shared elements (type T) per warp of the U writer (a multiple of 16 bytes).
__host__ __device__ inline int uwriter_per_warp(int levels, int tri, int L, int nYp, int nF, bool pre) {
    return ((levels * tri + 2 * L + 1 + (pre ? nYp : 0) + nF + 1) + 3) & ~3;
}

// Direction x_hat of point i (differences in FP64, normalisation in the bulk precision T; the
// zero vector gets e_0), then the level tables of the normalised three-term recurrences
// (levels x tri, lanes over mu') and the trigonometric powers (x0 + i x1)^mu times the
// normalisers (2L+1, index L + mu), written by one warp into its shared tbl and trig.
template <typename T>
__device__ __forceinline__ void point_harmonic_tables(const double* __restrict__ x, int d, const Center& cen,
                                                      double inv2R, int L, int tri, const T* cA, const T* cB,
                                                      T* tbl, T* trig, int64_t i, int lane, bool have_x = false,
                                                      double x_lane = 0.0) {
    const int levels = d - 2;
    // FP32 factors: lane j forms coordinate j once and the warp shares it by shuffles (FP64
    // issues at a small fraction of the FP32 rate here).
    // xh is indexed with compile-time indices only (loops over kMaxD with the dimension as a
    // predicate), so that it stays in registers
    T xh[kMaxD];
    T s = (T)0;
    if constexpr (sizeof(T) == 4) {
        double cj = cen.c[0];                    // this lane's centre coordinate (register selects)
#pragma unroll
        for (int j = 1; j < kMaxD; ++j) cj = (lane == j) ? cen.c[j] : cj;
        // one FP64 sub, mul (x_lane: this lane's coordinate, loaded ahead by the caller)
        const double xd = (lane < d) ? ((have_x ? x_lane : x[i * d + lane]) - cj) * inv2R : 0.0;
        const float xf = (float)xd;
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            const float v = __shfl_sync(0xffffffffu, xf, j);      // zero for j >= d
            xh[j] = v;
            s += v * v;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) {
            xh[j] = (j < d) ? (T)((x[i * d + j] - cen.c[j]) * inv2R) : (T)0;
            s += xh[j] * xh[j];
        }
    }
    if (s > (T)0) {
        const T inv = (T)1 / sqrt(s);
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) xh[j] *= inv;
    } else {
#pragma unroll
        for (int j = 0; j < kMaxD; ++j) xh[j] = (j == 0) ? (T)1 : (T)0;
    }
    // level tables: lanes over mu'
    for (int j = 0; j < levels; ++j) {
        const int D = d - 1 - j;
        T q = (T)0, z = (T)0;
#pragma unroll
        for (int m = 0; m < kMaxD; ++m) {
            if (m <= D) q += xh[m] * xh[m];
            if (m == D) z = xh[m];
        }
        const T qq = q;
        const T* A = cA + j * tri;
        const T* B = cB + j * tri;
        T* tb = tbl + j * tri;
        for (int mu = lane; mu <= L; mu += 32) {
            const int o = mu * (L + 1) - mu * (mu - 1) / 2;
            const int nmax = L - mu;
            T pm2 = A[o];
            tb[o] = pm2;
            if (nmax >= 1) {
                T pm1 = A[o + 1] * z;
                tb[o + 1] = pm1;
                for (int nn = 2; nn <= nmax; ++nn) {
                    const T pn = A[o + nn] * z * pm1 - B[o + nn] * qq * pm2;
                    tb[o + nn] = pn;
                    pm2 = pm1;
                    pm1 = pn;
                }
            }
        }
    }
    // trig powers (x0 + i x1)^mu by binary powering in the bulk precision, lanes over mu
    for (int mu = lane; mu <= L; mu += 32) {
        T br = (T)xh[0], bi = (T)xh[1], rr = (T)1, ri = (T)0;
        int e = mu;
        while (e) {
            if (e & 1) { const T t = rr * br - ri * bi; ri = rr * bi + ri * br; rr = t; }
            const T t = br * br - bi * bi; bi = (T)2 * br * bi; br = t;
            e >>= 1;
        }
        if (mu == 0) {
            trig[L] = (T)0.3989422804014327;             // 1/sqrt(2 pi)
        } else {
            trig[L + mu] = rr * (T)0.5641895835477563;   // 1/sqrt(pi)
            trig[L - mu] = ri * (T)0.5641895835477563;
        }
    }
}

// One point's U row, executed by one warp.  cA/cB: level recurrences in shared memory;
// base: this warp's shared area (P.per_warp elements, 16-byte aligned), laid out as
// [harmonic slots (pre only)] [level tables] [trig powers] [radial factors].  pre: the
// harmonics of the point are computed once into the slots; otherwise each chunk's harmonics
// are multiplied out from the level tables as it is written.  A VW-wide chunk of the row meets
// one or two (k, s) blocks; its two descriptor words give each block's radial factor and first
// harmonic slot.
// The radial-factor slots of a warp's shared area (nF + 1, the last one zero).
template <typename T>
__device__ __forceinline__ T* uwriter_fs(const UWParams& P, bool pre, T* base) {
    return base + (pre ? P.nYp : 0) + (P.d - 2) * P.tri + 2 * P.L + 1;
}

// Radial factors and coordinate of one point loaded into registers one point ahead of use (FP32
// factors with nF <= 32 kPfF): lane l holds F[i, l + 32 k] and x[i, l] (l < d), so that their
// global-memory latency passes while the previous row is written.
constexpr int kPfF = 16;
template <typename T> struct PointPre { T f[kPfF]; double x; };
template <typename T>
__device__ __forceinline__ void point_prefetch(const UWParams& P, int64_t i, int lane, PointPre<T>& pp) {
    const T* Fg = reinterpret_cast<const T*>(P.F) + i * P.ldF;
#pragma unroll
    for (int k = 0; k < kPfF; ++k) {
        const int f = lane + 32 * k;
        pp.f[k] = (f < P.nF) ? Fg[f] : (T)0;
    }
    pp.x = (lane < P.d) ? P.x[i * P.d + lane] : 0.0;
}
template <typename T>
__device__ __forceinline__ void point_stage_f(const UWParams& P, const PointPre<T>& pp, T* Fs, int lane) {
#pragma unroll
    for (int k = 0; k < kPfF; ++k) {
        const int f = lane + 32 * k;
        if (f < P.nF) Fs[f] = pp.f[k];
    }
}

template <typename T>
__device__ __forceinline__ void uwriter_point(const UWParams& P, const UWTabs& X, bool pre, int64_t i, const T* cA,
                                              const T* cB, T* base, int lane, bool staged = false,
                                              double x_lane = 0.0) {
    const int levels = P.d - 2;
    T* Ys = base;                                // nYp (pre only)
    T* tbl = base + (pre ? P.nYp : 0);           // levels * tri
    T* trig = tbl + levels * P.tri;              // 2L+1, index L + mu
    T* Fs = trig + 2 * P.L + 1;                  // nF + 1
    const T* Fg = reinterpret_cast<const T*>(P.F);
    T* Ug = reinterpret_cast<T*>(P.U);
    typedef typename Vec2<T>::type VT;
    constexpr int VW = Vec2<T>::w;
    point_harmonic_tables<T>(P.x, P.d, P.c, P.inv2R, P.L, P.tri, cA, cB, tbl, trig, i, lane, staged, x_lane);
    // this point's radial factors (staged: already in Fs, written by the caller)
    if (!staged) {
        for (int f = lane; f < P.nF; f += 32) Fs[f] = Fg[i * P.ldF + f];
        if (lane == 0) Fs[P.nF] = (T)0;
    }
    __syncwarp();
    if (pre) {
        // padding slots were zeroed once per warp and are never written
        for (int g = lane; g < P.nH; g += 32) {
            const int16_t* c = X.chains + (int64_t)g * P.cstride;
            const int slot = X.gslot[g];
            T v = trig[P.L + c[levels]];
            for (int j = 0; j < levels; ++j) v *= tbl[j * P.tri + c[j]];
            Ys[slot] = v;
        }
    }
    __syncwarp();
    // row write: one VW-wide chunk per lane per step, four (FP64: two) steps in flight.  A chunk
    // is one radial factor times VW consecutive harmonic slots, or (where it meets the end of a
    // (k, s) block) the first e columns from one block and the rest from the next.
    T* row = Ug + i * P.ldU;
    const int64_t nq = P.ldU / VW;
    auto harm = [&](uint32_t y) -> T {          // the harmonic in slot y (0 for a padding slot)
        if (pre) return Ys[y];
        const int ch = X.ychain[y];
        T h = (T)0;
        if (ch >= 0) {
            const int16_t* c = X.chains + (int64_t)ch * P.cstride;
            h = trig[P.L + c[levels]];
            for (int j = 0; j < levels; ++j) h *= tbl[j * P.tri + c[j]];
        }
        return h;
    };
    auto chunk = [&](int64_t q) {
        const uint2 w = *reinterpret_cast<const uint2*>(X.qdesc + 2 * q);
        const uint32_t e = (w.x >> 18) & 3u;
        const T fa = Fs[w.x >> 20];
        const uint32_t ya = w.x & 0x3FFFFu;
        VT out;
        T v[VW];
        if (pre) {
            // one branch-free form for whole and split chunks (e = 0 reads as e = VW; the second
            // word of a whole chunk names valid slots and is never selected), so that the lanes of
            // a warp, whose chunks differ in kind and alignment, do not diverge
            const uint32_t ea = e ? e : (uint32_t)VW;
            const T fb = Fs[w.y >> 20];
            const uint32_t yb = (w.y & 0xFFFFFu) - ea;
            v[0] = fa * Ys[ya];
#pragma unroll
            for (int u = 1; u < VW; ++u) {
                const bool a = (uint32_t)u < ea;
                v[u] = (a ? fa : fb) * Ys[a ? ya + u : yb + u];
            }
        } else if (e == 0) {
#pragma unroll
            for (int u = 0; u < VW; ++u) v[u] = fa * harm(ya + u);
        } else {
            const T fb = Fs[w.y >> 20];
            const uint32_t yb = w.y & 0xFFFFFu;
#pragma unroll
            for (int u = 0; u < VW; ++u) v[u] = ((uint32_t)u < e) ? fa * harm(ya + u) : fb * harm(yb + u - e);
        }
        if constexpr (VW == 4) { out.x = v[0]; out.y = v[1]; out.z = v[2]; out.w = v[3]; }
        else { out.x = v[0]; out.y = v[1]; }
        return out;
    };
    constexpr int NF = (VW == 4) ? 4 : 2;        // chunks in flight per lane
    int64_t q = lane;
    for (; q + 32 * (NF - 1) < nq; q += 32 * NF) {
        VT o[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) o[f] = chunk(q + 32 * f);
#pragma unroll
        for (int f = 0; f < NF; ++f) *reinterpret_cast<VT*>(row + (q + 32 * f) * VW) = o[f];
    }
    for (; q < nq; q += 32) *reinterpret_cast<VT*>(row + q * VW) = chunk(q);
    __syncwarp();
}

// Zeroes a warp's harmonic slots once (the padding slots are never written afterwards).
template <typename T>
__device__ __forceinline__ void uwriter_zero_slots(const UWParams& P, bool pre, T* base, int lane) {
    if (pre)
        for (int g = lane; g < P.nYp; g += 32) base[g] = (T)0;
    __syncwarp();
}

// Shared memory of the U writer: [nwarps x per_warp][coefA][coefB] (elements of T).
// Shared memory: [nwarps x per_warp elements][cA][cB][staged index tables (tab_bytes)].
template <typename T, bool PRE, bool PF, bool STAGED>
__global__ void __launch_bounds__(1024) k_uwriter(UWParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int levels = P.d - 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * P.per_warp;
    T* cA = reinterpret_cast<T*>(smem_raw) + (size_t)nwarps * P.per_warp;
    T* cB = cA + levels * P.tri;
    for (int idx = threadIdx.x; idx < levels * P.tri; idx += blockDim.x) {
        cA[idx] = reinterpret_cast<const T*>(P.coefA)[idx];
        cB[idx] = reinterpret_cast<const T*>(P.coefB)[idx];
    }
    UWTabs X{P.qdesc, P.chains, P.gslot, P.ychain};
    if constexpr (STAGED) {
        // staged in shared memory (STAGED is a compile-time choice, so that the table reads
        // compile to shared-memory loads)
        unsigned char* tp = reinterpret_cast<unsigned char*>(smem_raw) +
                            align16(sizeof(T) * ((size_t)nwarps * P.per_warp + 2 * (size_t)levels * P.tri));
        const int64_t nq = P.ldU / Vec2<T>::w;
        uint32_t* q = reinterpret_cast<uint32_t*>(tp);
        for (int64_t k = threadIdx.x; k < 2 * nq; k += blockDim.x) q[k] = P.qdesc[k];
        X.qdesc = q;
        tp += align16(sizeof(uint32_t) * 2 * nq);
        int16_t* ch = reinterpret_cast<int16_t*>(tp);
        for (int64_t k = threadIdx.x; k < (int64_t)P.nH * P.cstride; k += blockDim.x) ch[k] = P.chains[k];
        tp += align16(sizeof(int16_t) * (size_t)P.nH * P.cstride);
        int32_t* gs = reinterpret_cast<int32_t*>(tp);
        for (int k = threadIdx.x; k < P.nH; k += blockDim.x) gs[k] = P.gslot[k];
        tp += align16(sizeof(int32_t) * (size_t)P.nH);
        X.chains = ch; X.gslot = gs;
        if (!PRE) {
            int32_t* yc = reinterpret_cast<int32_t*>(tp);
            for (int k = threadIdx.x; k < P.nYp; k += blockDim.x) yc[k] = P.ychain[k];
            X.ychain = yc;
        }
    }
    __syncthreads();
    uwriter_zero_slots<T>(P, PRE, base, lane);
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
    if constexpr (PF) {
        // PF: the next point's radial factors and coordinate travel in registers during this row
        T* Fs = uwriter_fs<T>(P, PRE, base);
        if (lane == 0) Fs[P.nF] = (T)0;
        PointPre<T> pp;
        if (gw < P.n) point_prefetch<T>(P, gw, lane, pp);
        for (int64_t i = gw; i < P.n; i += nw) {
            point_stage_f<T>(P, pp, Fs, lane);
            const double xl = pp.x;
            if (i + nw < P.n) point_prefetch<T>(P, i + nw, lane, pp);
            uwriter_point<T>(P, X, PRE, i, cA, cB, base, lane, true, xl);
        }
    } else {
        for (int64_t i = gw; i < P.n; i += nw) uwriter_point<T>(P, X, PRE, i, cA, cB, base, lane);
    }
}

// --------------------------------------------------------------------- A7: matvec
// Register-tiled GEMMs on the CUDA cores.  CT = padded column count of the V block (c <= CT).
// U^T V: a block owns 128 (256 when CT = 1) columns of U and a chunk of rows; each thread
// keeps a TA x TJ tile of the product.  Partials per chunk are summed in FP64 afterwards.
template <int CT> struct UtvShape {
    static constexpr int AB = (CT == 1) ? 256 : 128;                       // columns per block
    static constexpr int TA = (CT >= 8) ? 4 : (CT == 4 ? 2 : 1);            // columns per thread
    static constexpr int TJ = (CT * (AB / TA)) / 256;                       // V columns per thread
};
constexpr int kKT = 32;     // rows (k) per shared tile

template <typename T, int N> struct VecLd;
template <typename T> struct VecLd<T, 1> { static __device__ __forceinline__ void ld(const T* p, T* o) { o[0] = p[0]; } };
template <typename T> struct VecLd<T, 2> {
    static __device__ __forceinline__ void ld(const T* p, T* o) { o[0] = p[0]; o[1] = p[1]; }
};
template <> struct VecLd<float, 4> {
    static __device__ __forceinline__ void ld(const float* p, float* o) {
        const float4 v = *reinterpret_cast<const float4*>(p); o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct VecLd<double, 4> {
    static __device__ __forceinline__ void ld(const double* p, double* o) {
        const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
};
template <> struct VecLd<float, 8> {
    static __device__ __forceinline__ void ld(const float* p, float* o) { VecLd<float, 4>::ld(p, o); VecLd<float, 4>::ld(p + 4, o + 4); }
};
template <> struct VecLd<double, 8> {
    static __device__ __forceinline__ void ld(const double* p, double* o) { VecLd<double, 4>::ld(p, o); VecLd<double, 4>::ld(p + 4, o + 4); }
};

// part_chunk[j * r + a] = sum_{i0 <= i < i1} U[i, a] V[i + j ldv] for the columns [a0, a0 + AB).
template <typename T, int CT>
__device__ __forceinline__ void utv_tile_body(const T* __restrict__ U, int64_t ldU, int64_t r,
                                              const T* __restrict__ V, int64_t ldv, int c, int64_t i0, int64_t i1,
                                              int64_t a0, double* __restrict__ part_chunk,
                                              T (*Us)[UtvShape<CT>::AB], T (*Vs)[CT]) {
    using S = UtvShape<CT>;
    const int t = threadIdx.x;
    const int tx = t % (S::AB / S::TA), ty = t / (S::AB / S::TA);
    T acc[S::TA][S::TJ];
#pragma unroll
    for (int p = 0; p < S::TA; ++p)
#pragma unroll
        for (int q = 0; q < S::TJ; ++q) acc[p][q] = (T)0;
    for (int64_t k0 = i0; k0 < i1; k0 += kKT) {
        // U tile: kKT rows x AB columns, row segments are contiguous
        for (int e = t; e < kKT * S::AB; e += 256) {
            const int kk = e / S::AB, aa = e % S::AB;
            const int64_t i = k0 + kk, a = a0 + aa;
            Us[kk][aa] = (i < i1 && a < ldU) ? U[i * ldU + a] : (T)0;
        }
        // V tile: kKT rows x CT columns (column-major source: coalesced along rows)
        for (int e = t; e < kKT * CT; e += 256) {
            const int kk = e % kKT, j = e / kKT;
            const int64_t i = k0 + kk;
            Vs[kk][j] = (i < i1 && j < c) ? V[i + (int64_t)j * ldv] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKT; ++kk) {
            T ua[S::TA], vj[S::TJ];
            VecLd<T, S::TA>::ld(&Us[kk][tx * S::TA], ua);
            VecLd<T, S::TJ>::ld(&Vs[kk][ty * S::TJ], vj);
#pragma unroll
            for (int p = 0; p < S::TA; ++p)
#pragma unroll
                for (int q = 0; q < S::TJ; ++q) acc[p][q] += ua[p] * vj[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < S::TA; ++p) {
        const int64_t a = a0 + tx * S::TA + p;
#pragma unroll
        for (int q = 0; q < S::TJ; ++q) {
            const int j = ty * S::TJ + q;
            if (a < r && j < c) part_chunk[(int64_t)j * r + a] = (double)acc[p][q];
        }
    }
}

// part[(chunk * c + j) * r + a] = sum_{i in chunk} U[i, a] V[i + j ldv]
template <typename T, int CT>
__global__ void __launch_bounds__(256) k_utv_tile(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                                  const T* __restrict__ V, int64_t ldv, int c, int64_t chunk,
                                                  double* __restrict__ part) {
    __shared__ __align__(16) T Us[kKT][UtvShape<CT>::AB];
    __shared__ __align__(16) T Vs[kKT][CT];
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    utv_tile_body<T, CT>(U, ldU, r, V, ldv, c, i0, i1, blockIdx.y * (int64_t)UtvShape<CT>::AB,
                         part + (int64_t)blockIdx.x * c * r, Us, Vs);
}

// W[a * c + j] = scale_a * sum_chunk part[(chunk * c + j) * r + a]; scale = S[a] or 1.
template <typename T, typename P = double>
__global__ void k_reduce_scale(const P* __restrict__ part, int nchunk, int64_t r, int c,
                               const T* __restrict__ S, T* __restrict__ W, double* __restrict__ Wd) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= r * c) return;
    const int64_t a = idx / c;
    const int j = (int)(idx % c);
    double s = 0.0;
    for (int b = 0; b < nchunk; ++b) s += (double)part[((int64_t)b * c + j) * r + a];
    if (S) s *= (double)S[a];
    if (W) W[idx] = (T)s;
    if (Wd) Wd[idx] = s;
}

// Y[i + j ldy] = alpha * sum_a U[i, a] W[a * c + j] + beta * B[i + j ldb].
// A block owns RB rows and all CT columns; each thread keeps a TM x TN tile.
template <int CT> struct UwShape {
    static constexpr int RB = (CT == 1) ? 256 : 128;
    static constexpr int TM = (CT == 64) ? 8 : (CT >= 8 ? 4 : (CT == 4 ? 2 : 1));
    static constexpr int TN = (CT * (RB / TM)) / 256;
};

constexpr int kUwPad = 4;

// Rows [m0, m0 + RB) of Y = alpha U W + beta B.
template <typename T, int CT>
__device__ __forceinline__ void uw_tile_body(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                             const T* __restrict__ W, int c, T alpha, const T* __restrict__ B,
                                             int64_t ldb, T beta, T* __restrict__ Y, int64_t ldy, int64_t m0,
                                             T (*Us)[UwShape<CT>::RB + kUwPad], T (*Ws)[CT]) {
    using S = UwShape<CT>;
    const int t = threadIdx.x;
    const int tx = t % (S::RB / S::TM), ty = t / (S::RB / S::TM);
    T acc[S::TM][S::TN];
#pragma unroll
    for (int p = 0; p < S::TM; ++p)
#pragma unroll
        for (int q = 0; q < S::TN; ++q) acc[p][q] = (T)0;
    for (int64_t k0 = 0; k0 < r; k0 += kKT) {
        for (int e = t; e < kKT * S::RB; e += 256) {
            const int mm = e / kKT, kk = e % kKT;            // consecutive threads walk one row
            const int64_t i = m0 + mm, a = k0 + kk;
            Us[kk][mm] = (i < n && a < r) ? U[i * ldU + a] : (T)0;
        }
        for (int e = t; e < kKT * CT; e += 256) {
            const int kk = e / CT, j = e % CT;
            const int64_t a = k0 + kk;
            Ws[kk][j] = (a < r && j < c) ? W[a * c + j] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kKT; ++kk) {
            T um[S::TM], wn[S::TN];
            VecLd<T, S::TM>::ld(&Us[kk][tx * S::TM], um);
            VecLd<T, S::TN>::ld(&Ws[kk][ty * S::TN], wn);
#pragma unroll
            for (int p = 0; p < S::TM; ++p)
#pragma unroll
                for (int q = 0; q < S::TN; ++q) acc[p][q] += um[p] * wn[q];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < S::TN; ++q) {
        const int j = ty * S::TN + q;
        if (j >= c) continue;
#pragma unroll
        for (int p = 0; p < S::TM; ++p) {
            const int64_t i = m0 + tx * S::TM + p;
            if (i < n) {
                T out = alpha * acc[p][q];
                if (B) out += beta * B[i + (int64_t)j * ldb];
                Y[i + (int64_t)j * ldy] = out;
            }
        }
    }
}

template <typename T, int CT>
__global__ void __launch_bounds__(256) k_uw_tile(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                                 const T* __restrict__ W, int c, T alpha,
                                                 const T* __restrict__ B, int64_t ldb, T beta,
                                                 T* __restrict__ Y, int64_t ldy) {
    __shared__ __align__(16) T Us[kKT][UwShape<CT>::RB + kUwPad];
    __shared__ __align__(16) T Ws[kKT][CT];
    uw_tile_body<T, CT>(U, ldU, n, r, W, c, alpha, B, ldb, beta, Y, ldy, blockIdx.x * (int64_t)UwShape<CT>::RB,
                        Us, Ws);
}

// ----------------------------------------------------------------- A6: Gram U^T U
// G[a, b] for the 64 x 64 tile (blockIdx.x, blockIdx.y), b-tile >= a-tile; FP64 output.
template <typename T>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                              double* __restrict__ G) {
    if (blockIdx.y < blockIdx.x) return;
    __shared__ T As[16][64 + 1], Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int64_t a0 = blockIdx.x * 64, b0 = blockIdx.y * 64;
    double acc[4][4] = {};
    for (int64_t i0 = 0; i0 < n; i0 += 16) {
        for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
            const int rr = idx / 64, cc = idx % 64;
            const int64_t i = i0 + rr;
            As[rr][cc] = (i < n && a0 + cc < r) ? U[i * ldU + a0 + cc] : (T)0;
            Bs[rr][cc] = (i < n && b0 + cc < r) ? U[i * ldU + b0 + cc] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
            T av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { av[q] = As[rr][ty * 4 + q]; bv[q] = Bs[rr][tx * 4 + q]; }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[q][w] += (double)(av[q] * bv[w]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int64_t a = a0 + ty * 4 + q, b = b0 + tx * 4 + w;
            if (a < r && b < r) { G[a * r + b] = acc[q][w]; G[b * r + a] = acc[q][w]; }
        }
}

// Y = alpha * X + beta * Y on column-major blocks (used by the solve's refinement).
template <typename T>
__global__ void k_axpby(int64_t n, int c, T alpha, const T* __restrict__ X, int64_t ldx, T beta,
                        T* __restrict__ Y, int64_t ldy) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= n * c) return;
    const int64_t i = idx % n, j = idx / n;
    Y[i + j * ldy] = alpha * X[i + j * ldx] + beta * Y[i + j * ldy];
}

}  // namespace dev
}  // namespace hdf
