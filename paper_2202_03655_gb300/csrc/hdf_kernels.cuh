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
__global__ void k_sum_partial(const double* __restrict__ x, int64_t n, int d, int64_t chunk,
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
__global__ void k_maxnorm_partial(const double* __restrict__ x, int64_t n, int d, int64_t chunk,
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
__global__ void k_mu2_rows(const double* __restrict__ x, int64_t n, int d, int m, int kernel,
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

// ----------------------------------------------------- A3: radial-basis Gram matrices
// B0[l] = T_l(u), l <= L and B1[l] = rho T_l(u), l < L, u = 8 rho^2 - 1, rho = |x - c|/(2R).
// part[b][q] (q < npairs) = sum_i B0[l] B0[l'] and part[b][npairs + q] = sum_i rho^2 T_l T_l'
// over the block's chunk, for the pairs (l, l') = pairs[q], l <= l'.
constexpr int kGramTile = 64;
constexpr int kGramMaxQ = 9;     // ceil(npairs / 256) for L <= 64

__global__ void __launch_bounds__(256) k_radial_gram(const double* __restrict__ x, int64_t n, int d,
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

// out[j] = sum_b part[b * ncols + j] in block order.
__global__ void k_reduce_cols(const double* __restrict__ part, int nblk, int64_t ncols,
                              double* __restrict__ out) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * ncols + j];
    out[j] = s;
}

// ------------------------------------------------------------- A5a: radial factors
// Per point: B_par (FP64) -> Q_par = B_par Qmat_par (FP64, the orthonormalised radial basis
// of Eq. svd) -> F[i, col] = sum_l Q_par(col)[l] Wt[l, col] (type T).  Tiles of 32 points.
constexpr int kFTile = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_radial_F(
    const double* __restrict__ x, int64_t n, int d, Center c, double inv2R, int L,
    const double* __restrict__ Qm0, int nb0, int m0, const double* __restrict__ Qm1, int nb1, int m1,
    const T* __restrict__ Wt, const uint8_t* __restrict__ colpar, int nF,
    T* __restrict__ F, int64_t ldF) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int LP1 = L + 1;
    double* Ts = reinterpret_cast<double*>(smem_raw);            // [kFTile][LP1]
    double* rh = Ts + kFTile * LP1;                              // [kFTile]
    T* Qs = reinterpret_cast<T*>(rh + kFTile);                   // [m0 + m1][kFTile]
    const int64_t ntiles = (n + kFTile - 1) / kFTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = tile * kFTile;
        const int cnt = (int)min((int64_t)kFTile, n - t0);
        if (threadIdx.x < kFTile) {
            const int p = threadIdx.x;
            double* Tp = Ts + p * LP1;
            double s = 0.0;
            if (p < cnt) {
                const int64_t i = t0 + p;
                for (int j = 0; j < d; ++j) { const double y = (x[i * d + j] - c.c[j]) * inv2R; s += y * y; }
            }
            const double u = 8.0 * s - 1.0;
            rh[p] = sqrt(s);
            Tp[0] = 1.0;
            if (L >= 1) Tp[1] = u;
            for (int l = 2; l <= L; ++l) Tp[l] = 2.0 * u * Tp[l - 1] - Tp[l - 2];
        }
        __syncthreads();
        const int mt = m0 + m1;
        for (int idx = threadIdx.x; idx < mt * kFTile; idx += blockDim.x) {
            const int o = idx / kFTile, p = idx % kFTile;
            const double* Tp = Ts + p * LP1;
            double q = 0.0;
            if (o < m0) {
                for (int l = 0; l < nb0; ++l) q += Tp[l] * Qm0[l * m0 + o];
            } else {
                const int oo = o - m0;
                for (int l = 0; l < nb1; ++l) q += Tp[l] * Qm1[l * m1 + oo];
                q *= rh[p];
            }
            Qs[o * kFTile + p] = (T)q;
        }
        __syncthreads();
        for (int col = threadIdx.x; col < nF; col += blockDim.x) {
            const int par = colpar[col];
            const int ob = par ? m0 : 0, mp = par ? m1 : m0;
            T acc[kFTile];
#pragma unroll
            for (int p = 0; p < kFTile; ++p) acc[p] = (T)0;
            for (int l = 0; l < mp; ++l) {
                const T w = Wt[(int64_t)l * nF + col];
                const T* q = Qs + (ob + l) * kFTile;
#pragma unroll
                for (int p = 0; p < kFTile; ++p) acc[p] += q[p] * w;
            }
            for (int p = 0; p < cnt; ++p) F[(t0 + p) * ldF + col] = acc[p];
        }
        __syncthreads();
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
    const int16_t* chains;     // nH x (d-1)
    int nH;
    const uint32_t* desc;      // ldU entries: (fidx << 20) | hidx ; padding -> fidx = nF
    int nF;
    const void* F; int64_t ldF;
    void* U; int64_t ldU;
    const void* coefA; const void* coefB;   // (d-2) x tri, type T
    int per_warp;              // shared elements (type T) per warp
};

template <typename T>
__global__ void __launch_bounds__(256) k_uwriter(UWParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int levels = P.d - 2;
    T* cA = reinterpret_cast<T*>(smem_raw);
    T* cB = cA + levels * P.tri;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int idx = threadIdx.x; idx < levels * P.tri; idx += blockDim.x) {
        cA[idx] = reinterpret_cast<const T*>(P.coefA)[idx];
        cB[idx] = reinterpret_cast<const T*>(P.coefB)[idx];
    }
    __syncthreads();
    T* base = cB + levels * P.tri + (size_t)warp * P.per_warp;
    T* tbl = base;                               // levels * tri
    T* trig = tbl + levels * P.tri;              // 2L+1, index L + mu
    T* Ys = trig + 2 * P.L + 1;                  // nH
    T* Fs = Ys + P.nH;                           // nF + 1
    const T* Fg = reinterpret_cast<const T*>(P.F);
    T* Ug = reinterpret_cast<T*>(P.U);
    typedef typename Vec2<T>::type VT;
    constexpr int VW = Vec2<T>::w;
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
    for (int64_t i = gw; i < P.n; i += nw) {
        // direction x_hat (FP64), zero vector -> e_0
        double xh[kMaxD];
        double s = 0.0;
        for (int j = 0; j < P.d; ++j) { xh[j] = (P.x[i * P.d + j] - P.c.c[j]) * P.inv2R; s += xh[j] * xh[j]; }
        if (s > 0.0) {
            const double inv = 1.0 / sqrt(s);
            for (int j = 0; j < P.d; ++j) xh[j] *= inv;
        } else {
            for (int j = 0; j < P.d; ++j) xh[j] = (j == 0) ? 1.0 : 0.0;
        }
        // level tables: lanes over mu'
        for (int j = 0; j < levels; ++j) {
            const int D = P.d - 1 - j;
            double q = 0.0;
            for (int m = 0; m <= D; ++m) q += xh[m] * xh[m];
            const T z = (T)xh[D], qq = (T)q;
            const T* A = cA + j * P.tri;
            const T* B = cB + j * P.tri;
            T* tb = tbl + j * P.tri;
            for (int mu = lane; mu <= P.L; mu += 32) {
                const int o = mu * (P.L + 1) - mu * (mu - 1) / 2;
                const int nmax = P.L - mu;
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
        // trig powers (x0 + i x1)^mu by binary powering, lanes over mu
        for (int mu = lane; mu <= P.L; mu += 32) {
            double br = xh[0], bi = xh[1], rr = 1.0, ri = 0.0;
            int e = mu;
            while (e) {
                if (e & 1) { const double t = rr * br - ri * bi; ri = rr * bi + ri * br; rr = t; }
                const double t = br * br - bi * bi; bi = 2.0 * br * bi; br = t;
                e >>= 1;
            }
            if (mu == 0) {
                trig[P.L] = (T)0.3989422804014327;             // 1/sqrt(2 pi)
            } else {
                trig[P.L + mu] = (T)(rr * 0.5641895835477563);  // 1/sqrt(pi)
                trig[P.L - mu] = (T)(ri * 0.5641895835477563);
            }
        }
        // this point's radial factors
        for (int f = lane; f < P.nF; f += 32) Fs[f] = Fg[i * P.ldF + f];
        if (lane == 0) Fs[P.nF] = (T)0;
        __syncwarp();
        // harmonics
        for (int g = lane; g < P.nH; g += 32) {
            const int16_t* ch = P.chains + (int64_t)g * (levels + 1);
            T v = trig[P.L + ch[levels]];
            for (int j = 0; j < levels; ++j) v *= tbl[j * P.tri + ch[j]];
            Ys[g] = v;
        }
        __syncwarp();
        // row write, VW consecutive columns per lane per step
        T* row = Ug + i * P.ldU;
        for (int64_t c0 = (int64_t)lane * VW; c0 < P.ldU; c0 += 32 * VW) {
            T v[VW];
#pragma unroll
            for (int e = 0; e < VW; ++e) {
                const uint32_t dsc = __ldg(P.desc + c0 + e);
                v[e] = Fs[dsc >> 20] * Ys[dsc & 0xFFFFFu];
            }
            VT out;
            if constexpr (VW == 4) { out.x = v[0]; out.y = v[1]; out.z = v[2]; out.w = v[3]; }
            else { out.x = v[0]; out.y = v[1]; }
            *reinterpret_cast<VT*>(row + c0) = out;
        }
        __syncwarp();
    }
}

// --------------------------------------------------------------------- A7: matvec
// Partial W = U^T V over row chunks: part[(chunk * c + j) * r + a] (FP64), c <= kCB.
constexpr int kCB = 16;
constexpr int kUtvRows = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_utv(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                             const T* __restrict__ V, int64_t ldv, int c, int64_t chunk,
                                             double* __restrict__ part) {
    __shared__ T Vs[kUtvRows][kCB];
    const int64_t a = blockIdx.y * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    T acc[kCB];
#pragma unroll
    for (int j = 0; j < kCB; ++j) acc[j] = (T)0;
    for (int64_t t0 = i0; t0 < i1; t0 += kUtvRows) {
        const int cnt = (int)min((int64_t)kUtvRows, i1 - t0);
        for (int idx = threadIdx.x; idx < kUtvRows * kCB; idx += blockDim.x) {
            const int rr = idx % kUtvRows, j = idx / kUtvRows;
            Vs[rr][j] = (rr < cnt && j < c) ? V[(t0 + rr) + j * ldv] : (T)0;
        }
        __syncthreads();
        if (a < r) {
            for (int rr = 0; rr < cnt; ++rr) {
                const T u = U[(t0 + rr) * ldU + a];
#pragma unroll
                for (int j = 0; j < kCB; ++j) acc[j] += u * Vs[rr][j];
            }
        }
        __syncthreads();
    }
    if (a < r)
        for (int j = 0; j < c; ++j) part[((int64_t)blockIdx.x * c + j) * r + a] = (double)acc[j];
}

// W[a * c + j] = scale_a * sum_chunk part[(chunk * c + j) * r + a]; scale = S[a] or 1.
template <typename T>
__global__ void k_reduce_scale(const double* __restrict__ part, int nchunk, int64_t r, int c,
                               const T* __restrict__ S, T* __restrict__ W, double* __restrict__ Wd) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= r * c) return;
    const int64_t a = idx / c;
    const int j = (int)(idx % c);
    double s = 0.0;
    for (int b = 0; b < nchunk; ++b) s += part[((int64_t)b * c + j) * r + a];
    if (S) s *= (double)S[a];
    if (W) W[idx] = (T)s;
    if (Wd) Wd[idx] = s;
}

// Y[i + j ldy] = alpha * sum_a U[i, a] W[a * c + j] + beta * B[i + j ldb]; warp per row.
template <typename T>
__global__ void __launch_bounds__(256) k_uw(const T* __restrict__ U, int64_t ldU, int64_t n, int64_t r,
                                            const T* __restrict__ W, int c, T alpha,
                                            const T* __restrict__ B, int64_t ldb, T beta,
                                            T* __restrict__ Y, int64_t ldy) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = gw; i < n; i += nw) {
        T acc[kCB];
#pragma unroll
        for (int j = 0; j < kCB; ++j) acc[j] = (T)0;
        const T* row = U + i * ldU;
        for (int64_t a = lane; a < r; a += 32) {
            const T u = row[a];
            const T* w = W + a * c;
#pragma unroll
            for (int j = 0; j < kCB; ++j)
                if (j < c) acc[j] += u * w[j];
        }
#pragma unroll
        for (int j = 0; j < kCB; ++j) {
            T v = acc[j];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            acc[j] = v;
        }
        if (lane < c) {
            T v = (T)0;
#pragma unroll
            for (int j = 0; j < kCB; ++j)
                if (j == lane) v = acc[j];
            T out = alpha * v;
            if (B) out += beta * B[i + (int64_t)lane * ldb];
            Y[i + (int64_t)lane * ldy] = out;
        }
    }
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
