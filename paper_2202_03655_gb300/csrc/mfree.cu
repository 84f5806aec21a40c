// Matrix-free form of the factor: U (n x r) is never stored.  Per point the library keeps
//   Z[i, (m, j)]      = Z_m^j(x_hat_i), the tails of the harmonic chains: for a harmonic of degree
//                       k with chain (mu_1 = m, mu_2, ...), every level factor but the first and
//                       the trigonometric factor -- a harmonic of degree m in d-1 dimensions,
//   A0F[i, (m, k, s)] = P_0(m, k - m)(x_hat_i) F_i[k, s], the first level factor times the radial
//                       factor,
// so that U[i, (k, s, (m, j))] = A0F[i, (m, k, s)] Z[i, (m, j)] (the product form of the real
// hyperspherical harmonics, Eq. additiontheorem with the chain construction of the harmonics, and
// Algorithm 1's U = F * Y).  For d = 5 at degree 23 this is 4,900 + sum_k s_k (k+1) values per
// point instead of sum_k s_k |H_k|; the cost model of Sec. 3.6 and the limitation of Sec. 3.7
// (|H_k| grows like k^(d-2)) are why a factor with a large rank cannot be stored.
//
// The products, per tail degree m (q runs over the (k, s) pairs with k >= m, c over columns):
//   U^T V:  W[(k,s,m,j), c] = sum_i Z[i, (m,j)] (A0F[i, (m,q)] V[i, c])      (k_mf_utv)
//   U W:    Y[i, c] = sum_m sum_q A0F[i, (m,q)] sum_j Z[i, (m,j)] W[(k,s,m,j), c]   (k_mf_uw)
// Both are register-tiled FP32 (or FP64) GEMMs on the CUDA cores over the stored Z with the
// small second operand formed on the fly; W keeps the (k, s, h) padded row order of a stored
// factor, so scaling by S, the adjoint and every other consumer of U^T V are unchanged.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "hdf_kernels.cuh"
#include "internal.h"
#include "planner.h"

namespace hdf {
namespace dev {

// ------------------------------------------------------------------ Z and A0F rows
struct ZWParams {
    const double* x; int64_t n; int d; Center c; double inv2R;
    int L, tri;                      // highest kept degree, (L+1)(L+2)/2
    const int16_t* zchain; int cstride; int ldZ;
    const int32_t* zpair; const int32_t* gmap; int ng;   // product form (d = 4, 5), else zpair = null
    const int32_t* a0off; const int32_t* afcol; int nA; int ldA;   // a0off / afcol: ldA entries
    const void* F; int64_t ldF; int nF;
    void* Z; void* A0F;
    const void* coefA; const void* coefB;
    int per_warp;                    // shared elements per warp
    int stage;                       // 1: the index tables are copied to shared memory per CTA
};

// Bytes of the index tables k_zwriter stages in shared memory (each part 16-byte aligned): the
// product-form pairs and G recipe (d = 4, 5) or the chains, then a0off and afcol.
__host__ __device__ inline size_t zwriter_tab_bytes(bool pairs, int ldZ, int cstride, int ng, int ldA) {
    const size_t z = pairs ? align16(sizeof(int32_t) * (size_t)ldZ) + align16(sizeof(int32_t) * (size_t)(ng > 0 ? ng : 1))
                           : align16(sizeof(int16_t) * (size_t)ldZ * cstride);
    return z + 2 * align16(sizeof(int32_t) * (size_t)ldA);
}

// Per warp shared: level tables (levels x tri), trig (2L+1) and a zero slot, the point's F row
// (nF), and with d = 5 the point's G (ng + 1).
__host__ __device__ inline int zwriter_per_warp(int levels, int tri, int L, int nF, int gsz) {
    return (levels * tri + 2 * L + 2 + nF + gsz + 3) & ~3;
}

template <typename T> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void store(float* p, float a, float b, float c, float d) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void store(double* p, double a, double b, double c, double d) {
        *reinterpret_cast<double2*>(p) = make_double2(a, b);
        *reinterpret_cast<double2*>(p + 2) = make_double2(c, d);
    }
};

template <typename T>
__global__ void __launch_bounds__(1024) k_zwriter(ZWParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int levels = P.d - 2;
    const bool pairs = P.zpair != nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * P.per_warp;
    T* cA = reinterpret_cast<T*>(smem_raw) + (size_t)nwarps * P.per_warp;
    T* cB = cA + levels * P.tri;
    for (int idx = threadIdx.x; idx < levels * P.tri; idx += blockDim.x) {
        cA[idx] = reinterpret_cast<const T*>(P.coefA)[idx];
        cB[idx] = reinterpret_cast<const T*>(P.coefB)[idx];
    }
    const int16_t* zchain = P.zchain;
    const int32_t* zpair = P.zpair;
    const int32_t* gmap = P.gmap;
    const int32_t* a0off = P.a0off;
    const int32_t* afcol = P.afcol;
    if (P.stage) {
        unsigned char* tp = reinterpret_cast<unsigned char*>(cB + levels * P.tri);
        tp = reinterpret_cast<unsigned char*>(align16(reinterpret_cast<size_t>(tp)));
        if (pairs) {
            int32_t* zp = reinterpret_cast<int32_t*>(tp);
            for (int k = threadIdx.x; k < P.ldZ; k += blockDim.x) zp[k] = P.zpair[k];
            tp += align16(sizeof(int32_t) * (size_t)P.ldZ);
            int32_t* gm = reinterpret_cast<int32_t*>(tp);
            if (P.gmap)
                for (int k = threadIdx.x; k < P.ng; k += blockDim.x) gm[k] = P.gmap[k];
            tp += align16(sizeof(int32_t) * (size_t)(P.ng > 0 ? P.ng : 1));
            zpair = zp;
            if (P.gmap) gmap = gm;
        } else {
            int16_t* zc = reinterpret_cast<int16_t*>(tp);
            for (int64_t k = threadIdx.x; k < (int64_t)P.ldZ * P.cstride; k += blockDim.x) zc[k] = P.zchain[k];
            tp += align16(sizeof(int16_t) * (size_t)P.ldZ * P.cstride);
            zchain = zc;
        }
        int32_t* ao = reinterpret_cast<int32_t*>(tp);
        int32_t* af = ao + align16(sizeof(int32_t) * (size_t)P.ldA) / sizeof(int32_t);
        for (int k = threadIdx.x; k < P.ldA; k += blockDim.x) { ao[k] = P.a0off[k]; af[k] = P.afcol[k]; }
        a0off = ao;
        afcol = af;
    }
    __syncthreads();
    T* tbl = base;
    T* trig = tbl + levels * P.tri;
    T* Fs = trig + 2 * P.L + 2;
    // G of the product form: the trigonometric factors themselves (d = 4), else its own array;
    // its slot ng is zero (the padding columns)
    T* G = P.gmap ? Fs + P.nF : trig;
    if (pairs && lane == 0) G[P.ng] = (T)0;
    const T* Fg = reinterpret_cast<const T*>(P.F);
    const int tl = levels - 1;           // position of the trig index in a tail chain
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
    for (int64_t i = gw; i < P.n; i += nw) {
        point_harmonic_tables<T>(P.x, P.d, P.c, P.inv2R, P.L, P.tri, cA, cB, tbl, trig, i, lane);
        for (int f = lane; f < P.nF; f += 32) Fs[f] = Fg[i * P.ldF + f];
        T* zr = reinterpret_cast<T*>(P.Z) + i * (int64_t)P.ldZ;
        if (pairs) {
            // Z[i, t] = P_1[ia] G[ib] (P_1: the level-1 table), four consecutive columns per lane
            // (ldZ is a multiple of 8)
            if (P.gmap) {
                __syncwarp();
                for (int g = lane; g < P.ng; g += 32) {
                    const int32_t gm = gmap[g];
                    G[g] = tbl[2 * P.tri + (gm >> 16)] * trig[gm & 0xFFFF];   // level 2 x trig
                }
            }
            __syncwarp();
            const T* t1 = tbl + P.tri;
            for (int t4 = lane; 4 * t4 < P.ldZ; t4 += 32) {
                const int4 pr = *reinterpret_cast<const int4*>(zpair + 4 * t4);
                Vec4<T>::store(zr + 4 * t4, t1[pr.x >> 16] * G[pr.x & 0xFFFF], t1[pr.y >> 16] * G[pr.y & 0xFFFF],
                               t1[pr.z >> 16] * G[pr.z & 0xFFFF], t1[pr.w >> 16] * G[pr.w & 0xFFFF]);
            }
        } else {
            __syncwarp();
            for (int t = lane; t < P.ldZ; t += 32) {
                const int16_t* ch = zchain + (int64_t)t * P.cstride;
                const int tr = ch[tl];
                T v = (T)0;
                if (tr != 0x7fff) {                  // 0x7fff marks a padding column
                    v = trig[P.L + tr];
                    for (int l = 1; l < levels; ++l) v *= tbl[l * P.tri + ch[l - 1]];
                }
                zr[t] = v;
            }
        }
        // A0F[i, q] = P_0 entry times the radial factor, four columns per lane (ldA is a multiple
        // of 4); a0off = -1 marks a padding column
        T* ar = reinterpret_cast<T*>(P.A0F) + i * (int64_t)P.ldA;
        for (int q4 = lane; 4 * q4 < P.ldA; q4 += 32) {
            const int4 o = *reinterpret_cast<const int4*>(a0off + 4 * q4);
            const int4 fc = *reinterpret_cast<const int4*>(afcol + 4 * q4);
            Vec4<T>::store(ar + 4 * q4, o.x >= 0 ? tbl[o.x] * Fs[fc.x] : (T)0, o.y >= 0 ? tbl[o.y] * Fs[fc.y] : (T)0,
                           o.z >= 0 ? tbl[o.z] * Fs[fc.z] : (T)0, o.w >= 0 ? tbl[o.w] * Fs[fc.w] : (T)0);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------ GEMMs
// Thread tiles: 8 x 8 outputs in FP32, 4 x 8 in FP64 (register budget); 256 threads.
template <typename T> struct MfShape {
    static constexpr int TJ = (sizeof(T) == 4) ? 8 : 4;     // rows of the thread tile
    static constexpr int TN = 8;                            // columns of the thread tile
    static constexpr int KS = 16;                           // points per step of U^T V
    static constexpr int SMEM = KS * (16 * TJ + 1024);      // U^T V elements: A (KS x <= 16 TJ) + B (KS x <= 1024)
    // U W: Z^T tile (KJ x (BI + 4)) and W tile (KJ x BN), then the reduction buffer (16 x BI x 4)
    static constexpr int BI = 16 * TJ, BN = 16 * TN, KJ = 16, LDA = BI + 4;
    static constexpr int UW_SMEM = (KJ * LDA + KJ * BN > 16 * BI * 4) ? KJ * LDA + KJ * BN : 16 * BI * 4;
};

// Loads 4 consecutive elements of shared memory (16-byte aligned for FP32, two 16-byte loads
// for FP64).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* o) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else {
        const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
}

struct MfUtvArgs {
    const void* Z; int ldZ;
    const void* A0F; int ldA;
    const void* V; int64_t ldv; int c;
    int64_t n, chunk;
    const int4* items;               // (m, j0, n0, BJ) per tile
    const int* zoff; const int* zcnt; const int* aoff; const int* acnt;
    const int64_t* wcol;
    double* part; int64_t r;         // part[(chunk * c + cc) * r + a]
};

// One (tile, chunk) of U^T V per block (grid = tiles x chunks).  The tile covers rows
// j0..j0+BJ of the tails of degree m and columns n0..n0+BN of (q, c), BN = 256 TJ TN / BJ; the
// thread owns rows {g BJ / (TJ/4) + 4 tj + u} and columns {g BN / 2 + 4 tn + u}.
template <typename T>
__global__ void __launch_bounds__(256, 1) k_mf_utv(MfUtvArgs a) {
    using S = MfShape<T>;
    constexpr int TJ = S::TJ, TN = S::TN, KS = S::KS, GJ = TJ / 4, GN = TN / 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int4 it = a.items[blockIdx.x];
    const int m = it.x, j0 = it.y, n0 = it.z, BJ = it.w;
    const int nj = BJ / TJ, BN = (256 / nj) * TN;
    T* As = reinterpret_cast<T*>(smem_raw);          // KS x BJ
    T* Bs = As + KS * BJ;                            // KS x BN
    const int tid = threadIdx.x, tj = tid % nj, tn = tid / nj;
    const int J = a.zcnt[m], zo = a.zoff[m], ao = a.aoff[m], c = a.c, N = a.acnt[m] * c;
    const T* Z = reinterpret_cast<const T*>(a.Z);
    const T* A0F = reinterpret_cast<const T*>(a.A0F);
    const T* V = reinterpret_cast<const T*>(a.V);
    const int64_t ch = blockIdx.y, i0 = ch * a.chunk, i1 = min(a.n, i0 + a.chunk);
    T acc[TJ][TN];
#pragma unroll
    for (int u = 0; u < TJ; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] = (T)0;
    for (int64_t ib = i0; ib < i1; ib += KS) {
        for (int e = tid; e < KS * BJ; e += 256) {
            const int kk = e / BJ, jj = e % BJ;
            const int64_t i = ib + kk;
            As[e] = (i < i1 && j0 + jj < J) ? Z[i * a.ldZ + zo + j0 + jj] : (T)0;
        }
        for (int e = tid; e < KS * BN; e += 256) {
            const int kk = e / BN, nn = e % BN;
            const int64_t i = ib + kk;
            const int nidx = n0 + nn;
            T v = (T)0;
            if (i < i1 && nidx < N) {
                const int q = nidx / c, cc = nidx - q * c;
                v = A0F[i * a.ldA + ao + q] * V[i + cc * a.ldv];
            }
            Bs[e] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < KS; ++kk) {
            T x[TJ], y[TN];
#pragma unroll
            for (int g = 0; g < GJ; ++g) ld4<T>(As + kk * BJ + g * (BJ / GJ) + 4 * tj, x + 4 * g);
#pragma unroll
            for (int g = 0; g < GN; ++g) ld4<T>(Bs + kk * BN + g * (BN / GN) + 4 * tn, y + 4 * g);
#pragma unroll
            for (int u = 0; u < TJ; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) acc[u][v] += x[u] * y[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < TJ; ++u) {
        const int j = j0 + (u / 4) * (BJ / GJ) + 4 * tj + (u % 4);
        if (j >= J) continue;
#pragma unroll
        for (int v = 0; v < TN; ++v) {
            const int nidx = n0 + (v / 4) * (BN / GN) + 4 * tn + (v % 4);
            if (nidx >= N) continue;
            const int q = nidx / c, cc = nidx - q * c;
            a.part[(ch * c + cc) * a.r + a.wcol[ao + q] + j] = (double)acc[u][v];
        }
    }
}

struct MfUwArgs {
    const void* Z; int ldZ;
    const void* A0F; int ldA;
    const void* W; int c, cp;        // W: r x c row-major (padded U rows); cp: c padded to a power of 2 >= 4
    void* Y; int64_t ldy;
    int64_t n; int L;
    const int* zoff; const int* zcnt; const int* aoff; const int* acnt;
    const int64_t* wcol;
};

// Y for a tile of BI = 16 TI points (TI = TJ rows of the thread tile) over every tail degree m:
// Q = Z_m W_m in 128-column tiles of (q, c) (c padded to cp), then y += A0F[:, (m, q)] Q; the
// thread's columns {g 64 + 4 tn + u} share one c-set (4 tn mod cp) for every tile, so its y
// stays in registers; at the end the partial y of the threads with the same c-set are summed
// in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256, 1) k_mf_uw(MfUwArgs a) {
    using S = MfShape<T>;
    constexpr int TI = S::TJ, TN = S::TN, GI = TI / 4, GN = TN / 4;
    constexpr int BI = S::BI, BN = S::BN, KJ = S::KJ, LDA = S::LDA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*As)[LDA] = reinterpret_cast<T (*)[LDA]>(smem_raw);                   // Z^T tile: As[jj][point]
    T (*Bs)[BN] = reinterpret_cast<T (*)[BN]>(smem_raw + sizeof(T) * KJ * LDA);
    T (*red)[BI][4] = reinterpret_cast<T (*)[BI][4]>(smem_raw);             // after the products
    const int tid = threadIdx.x, ti = tid % 16, tn = tid / 16;
    const int64_t i0 = (int64_t)blockIdx.x * BI;
    const int c = a.c, cp = a.cp;
    const T* Z = reinterpret_cast<const T*>(a.Z);
    const T* A0F = reinterpret_cast<const T*>(a.A0F);
    const T* W = reinterpret_cast<const T*>(a.W);
    int pt[TI];                                      // this thread's points (tile offsets)
#pragma unroll
    for (int u = 0; u < TI; ++u) pt[u] = (u / 4) * (BI / GI) + 4 * ti + (u % 4);
    T y[TI][4];
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) y[u][v] = (T)0;
    for (int m = 0; m <= a.L; ++m) {
        const int J = a.zcnt[m], nq = a.acnt[m];
        if (J == 0 || nq == 0) continue;
        const int zo = a.zoff[m], ao = a.aoff[m], N = nq * cp;
        for (int n0 = 0; n0 < N; n0 += BN) {
            T acc[TI][TN];
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TN; ++v) acc[u][v] = (T)0;
            for (int j0 = 0; j0 < J; j0 += KJ) {
                for (int e = tid; e < KJ * BI; e += 256) {
                    const int p = e / KJ, jj = e % KJ;
                    const int64_t i = i0 + p;
                    As[jj][p] = (i < a.n && j0 + jj < J) ? Z[i * a.ldZ + zo + j0 + jj] : (T)0;
                }
                for (int e = tid; e < KJ * BN; e += 256) {
                    const int jj = e / BN, nn = e % BN;
                    const int nidx = n0 + nn, q = nidx / cp, cc = nidx % cp;
                    T v = (T)0;
                    if (q < nq && cc < c && j0 + jj < J) v = W[(a.wcol[ao + q] + j0 + jj) * c + cc];
                    Bs[jj][nn] = v;
                }
                __syncthreads();
#pragma unroll 4
                for (int jj = 0; jj < KJ; ++jj) {
                    T x[TI], w[TN];
#pragma unroll
                    for (int g = 0; g < GI; ++g) ld4<T>(&As[jj][g * (BI / GI) + 4 * ti], x + 4 * g);
#pragma unroll
                    for (int g = 0; g < GN; ++g) ld4<T>(&Bs[jj][g * (BN / GN) + 4 * tn], w + 4 * g);
#pragma unroll
                    for (int u = 0; u < TI; ++u)
#pragma unroll
                        for (int v = 0; v < TN; ++v) acc[u][v] += x[u] * w[v];
                }
                __syncthreads();
            }
            // y += A0F[i, (m, q_g)] Q[i, (q_g, c)] for the thread's two column groups
#pragma unroll
            for (int g = 0; g < GN; ++g) {
                const int q = (n0 + g * (BN / GN) + 4 * tn) / cp;
                if (q >= nq) continue;
#pragma unroll
                for (int u = 0; u < TI; ++u) {
                    const int64_t i = i0 + pt[u];
                    const T f = (i < a.n) ? A0F[i * a.ldA + ao + q] : (T)0;
#pragma unroll
                    for (int v = 0; v < 4; ++v) y[u][v] += f * acc[u][4 * g + v];
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) red[tn][pt[u]][v] = y[u][v];
    __syncthreads();
    T* Y = reinterpret_cast<T*>(a.Y);
    for (int e = tid; e < BI * c; e += 256) {
        const int p = e % BI, cc = e / BI;
        const int64_t i = i0 + p;
        if (i >= a.n) continue;
        const int set = (cc / 4) * 4, v = cc % 4;
        T sum = (T)0;
        for (int t = 0; t < 16; ++t)
            if ((4 * t) % cp == set) sum += red[t][p][v];
        Y[i + (int64_t)cc * a.ldy] = sum;
    }
}

}  // namespace dev

// ------------------------------------------------------------------------- host side
}  // namespace hdf

bool FreeFactor::fits(int64_t ubytes) {
    size_t fr = 0, total = 0;
    if (cudaMemGetInfo(&fr, &total) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return (double)ubytes <= 0.8 * (double)total;
}

namespace hdf {
namespace {

// Tiles of U^T V for c columns: per tail degree m the row block BJ (16, 32, 64 or 128 in FP32;
// half in FP64) that wastes the fewest padded products.
std::vector<int4> utv_items(const FreeFactor& mf, int c, bool fp32) {
    std::vector<int4> out;
    const int TJ = fp32 ? 8 : 4;
    for (int m = 0; m <= mf.L_used; ++m) {
        const int J = mf.zcnt[m], N = mf.acnt[m] * c;
        if (J == 0 || N == 0) continue;
        int best = 0;
        int64_t best_cost = -1;
        for (int nj = 2; nj <= 16; nj *= 2) {
            const int BJ = nj * TJ, BN = (256 / nj) * 8;
            const int64_t cost = (int64_t)((J + BJ - 1) / BJ) * BJ * ((N + BN - 1) / BN) * BN;
            if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = BJ; }
        }
        const int BN = (256 / (best / TJ)) * 8;
        for (int j0 = 0; j0 < J; j0 += best)
            for (int n0 = 0; n0 < N; n0 += BN) out.push_back(make_int4(m, j0, n0, best));
    }
    return out;
}

int pow2_at_least(int c, int lo) {
    int p = lo;
    while (p < c) p *= 2;
    return p;
}

}  // namespace

template <typename T>
hdf_status mf_write(hdf_factor* f, const double* x, int64_t n, int d, const dev::Center& cen, double inv2R,
                    const FactorChoice& fc, const DeviceTables& tb, const void* F, int64_t ldF, const void* coefA,
                    const void* coefB, cudaStream_t st) {
    FreeFactor& mf = f->mf;
    FreeTables ft;
    std::string err;
    if (!make_free_tables(fc, d, f->info.L, tb, ft, err)) return fail(HDF_EINVAL, "hdf_build: " + err);
    mf.on = true;
    mf.L_used = ft.L_used;
    mf.nZ = ft.nZ;
    mf.ldZ = ft.ldZ;
    mf.nA = ft.nA;
    mf.ldA = ft.ldA;
    mf.zoff = ft.zoff;
    mf.zcnt = ft.zcnt;
    mf.aoff = ft.aoff;
    mf.acnt = ft.acnt;
    const size_t zbytes = sizeof(T) * (size_t)n * ft.ldZ, abytes = sizeof(T) * (size_t)n * ft.ldA;
    if (mf.Z.alloc_on(zbytes, st) != cudaSuccess || mf.A0F.alloc_on(abytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(HDF_ENOMEM, "hdf_build: cannot allocate the matrix-free rows (" + std::to_string(zbytes + abytes) +
                                    " bytes)");
    }
    const int Lp = ft.L_used + 1;
    DevBuf dchain, da0, daf, dpair, dgmap;
    // the writer reads a0off / afcol four at a time over the whole row stride: padded to ldA
    std::vector<int32_t> a0p(ft.ldA, -1), afp(ft.ldA, 0);
    std::copy(ft.a0off.begin(), ft.a0off.end(), a0p.begin());
    std::copy(ft.afcol.begin(), ft.afcol.end(), afp.begin());
    const bool pairs = !ft.zpair.empty();
    HDF_CUDA(dchain.alloc_on(sizeof(int16_t) * ft.zchain.size(), st));
    HDF_CUDA(da0.alloc_on(sizeof(int32_t) * ft.ldA, st));
    HDF_CUDA(daf.alloc_on(sizeof(int32_t) * ft.ldA, st));
    if (pairs) {
        HDF_CUDA(dpair.alloc_on(sizeof(int32_t) * ft.zpair.size(), st));
        HDF_CUDA(cudaMemcpyAsync(dpair.p, ft.zpair.data(), sizeof(int32_t) * ft.zpair.size(), cudaMemcpyHostToDevice, st));
        if (!ft.gmap.empty()) {
            HDF_CUDA(dgmap.alloc_on(sizeof(int32_t) * ft.gmap.size(), st));
            HDF_CUDA(cudaMemcpyAsync(dgmap.p, ft.gmap.data(), sizeof(int32_t) * ft.gmap.size(), cudaMemcpyHostToDevice, st));
        }
    }
    HDF_CUDA(cudaMemcpyAsync(da0.p, a0p.data(), sizeof(int32_t) * ft.ldA, cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(daf.p, afp.data(), sizeof(int32_t) * ft.ldA, cudaMemcpyHostToDevice, st));
    HDF_CUDA(mf.dzoff.alloc(sizeof(int) * (Lp + 1)));
    HDF_CUDA(mf.dzcnt.alloc(sizeof(int) * Lp));
    HDF_CUDA(mf.daoff.alloc(sizeof(int) * (Lp + 1)));
    HDF_CUDA(mf.dacnt.alloc(sizeof(int) * Lp));
    HDF_CUDA(mf.dwcol.alloc(sizeof(int64_t) * std::max(1, ft.nA)));
    HDF_CUDA(cudaMemcpyAsync(dchain.p, ft.zchain.data(), sizeof(int16_t) * ft.zchain.size(), cudaMemcpyHostToDevice, st));
    if (ft.nA > 0)
        HDF_CUDA(cudaMemcpyAsync(mf.dwcol.p, ft.wcol.data(), sizeof(int64_t) * ft.nA, cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(mf.dzoff.p, ft.zoff.data(), sizeof(int) * (Lp + 1), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(mf.dzcnt.p, ft.zcnt.data(), sizeof(int) * Lp, cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(mf.daoff.p, ft.aoff.data(), sizeof(int) * (Lp + 1), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(mf.dacnt.p, ft.acnt.data(), sizeof(int) * Lp, cudaMemcpyHostToDevice, st));

    dev::ZWParams P{};
    P.x = x; P.n = n; P.d = d; P.c = cen; P.inv2R = inv2R;
    P.L = ft.L_used; P.tri = tb.tri;
    P.zchain = dchain.as<int16_t>(); P.cstride = chain_stride(d); P.ldZ = ft.ldZ;
    P.zpair = pairs ? dpair.as<int32_t>() : nullptr;
    P.gmap = ft.gmap.empty() ? nullptr : dgmap.as<int32_t>();
    P.ng = ft.ng;
    P.a0off = da0.as<int32_t>(); P.afcol = daf.as<int32_t>(); P.nA = ft.nA; P.ldA = ft.ldA;
    P.F = F; P.ldF = ldF; P.nF = tb.nF;
    P.Z = mf.Z.p; P.A0F = mf.A0F.p;
    P.coefA = coefA; P.coefB = coefB;
    const int levels = d - 2;
    P.per_warp = dev::zwriter_per_warp(levels, tb.tri, ft.L_used, tb.nF, ft.gmap.empty() ? 0 : ft.ng + 1);
    const size_t coef = sizeof(T) * 2 * (size_t)levels * tb.tri;
    const size_t budget = 200 * 1024;
    const size_t tabs = dev::zwriter_tab_bytes(pairs, ft.ldZ, chain_stride(d), ft.ng, ft.ldA) + 16;
    // stage the index tables only when 16 warps still fit beside them (fewer warps measured
    // slower); then as many warps as the budget holds, up to 32 (24 at d = 5, p = 64: 7% faster
    // than 16)
    P.stage = (coef + tabs + 16 * sizeof(T) * (size_t)P.per_warp <= budget) ? 1 : 0;
    const size_t fixed = coef + (P.stage ? tabs : 0);
    const int warps = (int)std::min<size_t>(32, (budget - std::min(budget, fixed)) / (sizeof(T) * P.per_warp));
    if (fixed + sizeof(T) * P.per_warp > budget || warps < 1)
        return fail(HDF_ETOOBIG, "hdf_build: matrix-free harmonic tables exceed shared memory");
    const size_t sm = fixed + sizeof(T) * (size_t)warps * P.per_warp;
    HDF_CUDA(cudaFuncSetAttribute(dev::k_zwriter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int occ = 0, nsm = 0, dv = 0;
    HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dev::k_zwriter<T>, warps * 32, sm));
    HDF_CUDA(cudaGetDevice(&dv));
    HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
    const int grid = std::max(1, std::min<int>(nsm * std::max(occ, 1), (int)((n + warps - 1) / warps)));
    HDF_COUNT_LAUNCH();
    dev::k_zwriter<T><<<grid, warps * 32, sm, st>>>(P);
    HDF_CUDA(cudaGetLastError());
    HDF_CUDA(cudaStreamSynchronize(st));            // the tables above are released on return
    return HDF_OK;
}
template hdf_status mf_write<float>(hdf_factor*, const double*, int64_t, int, const dev::Center&, double,
                                    const FactorChoice&, const DeviceTables&, const void*, int64_t, const void*,
                                    const void*, cudaStream_t);
template hdf_status mf_write<double>(hdf_factor*, const double*, int64_t, int, const dev::Center&, double,
                                     const FactorChoice&, const DeviceTables&, const void*, int64_t, const void*,
                                     const void*, cudaStream_t);

namespace {
// Device views and cached tensor-core lists of a matrix-free factor for c columns.
MfTcView tc_view(const hdf_factor* f) {
    const FreeFactor& mf = f->mf;
    return MfTcView{mf.Z.as<float>(), mf.ldZ, mf.A0F.as<float>(), mf.ldA, f->info.n, f->info.ldu,
                    mf.dzoff.as<int>(), mf.dzcnt.as<int>(), mf.daoff.as<int>(), mf.dacnt.as<int>(),
                    mf.dwcol.as<int64_t>()};
}

hdf_status tc_lists(const hdf_factor* f, int c, FreeFactor::TcLists** out) {
    FreeFactor& mf = const_cast<FreeFactor&>(f->mf);
    auto& slot = mf.tc[c];
    if (!slot) {
        std::vector<int4> tiles, phases;
        int kpad = 0;
        tc_mf_lists(mf.zcnt, mf.acnt, c, tiles, phases, &kpad);
        std::unique_ptr<FreeFactor::TcLists> L(new FreeFactor::TcLists());
        L->ntiles = (int)tiles.size();
        L->nphase = (int)phases.size();
        L->kpad = kpad;
        HDF_CUDA(L->tiles.alloc(sizeof(int4) * std::max<size_t>(1, tiles.size())));
        HDF_CUDA(L->phases.alloc(sizeof(int4) * std::max<size_t>(1, phases.size())));
        if (!tiles.empty()) HDF_CUDA(cudaMemcpy(L->tiles.p, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice));
        if (!phases.empty())
            HDF_CUDA(cudaMemcpy(L->phases.p, phases.data(), sizeof(int4) * phases.size(), cudaMemcpyHostToDevice));
        slot = std::move(L);
    }
    *out = slot.get();
    return HDF_OK;
}

bool use_tensor_cores(const hdf_factor* f) { return f->prec == HDF_FP32 && f->use_tc; }
}  // namespace

// Partial sums of U^T V (c <= 64 columns) into part[(chunk * c + cc) * r + a], r = ldu, part
// allocated here; *nchunk gets the number of chunks.
template <typename T>
hdf_status mf_utv(const hdf_factor* f, const T* V, int64_t ldv, int c, DevBuf& part, int* nchunk, cudaStream_t st) {
    FreeFactor& mf = const_cast<FreeFactor&>(f->mf);
    const int64_t n = f->info.n, r = f->info.ldu;
    if constexpr (sizeof(T) == 4) {
        if (use_tensor_cores(f)) {
            FreeFactor::TcLists* L = nullptr;
            if (hdf_status e = tc_lists(f, c, &L); e != HDF_OK) return e;
            int64_t chunk = 0;
            int nch = 0;
            tc_mf_chunks(n, L->ntiles, &chunk, &nch);
            HDF_CUDA(part.alloc_on(sizeof(double) * (size_t)nch * c * r, st));
            int got = 0;
            if (hdf_status e = tc_mf_utv(tc_view(f), L->tiles.as<int4>(), L->ntiles, reinterpret_cast<const float*>(V),
                                         ldv, c, part.as<double>(), &got, f->dev_err.as<int>(), st);
                e != HDF_OK)
                return e;
            *nchunk = got;
            return HDF_OK;
        }
    }
    auto& slot = mf.items[(sizeof(T) == 4 ? 0 : 64) + c - 1];
    if (!slot) {
        const std::vector<int4> it = utv_items(mf, c, sizeof(T) == 4);
        slot.reset(new FreeFactor::Items());
        slot->count = (int)it.size();
        HDF_CUDA(slot->buf.alloc(sizeof(int4) * std::max<size_t>(1, it.size())));
        if (!it.empty()) HDF_CUDA(cudaMemcpy(slot->buf.p, it.data(), sizeof(int4) * it.size(), cudaMemcpyHostToDevice));
    }
    const int64_t chunk = FreeFactor::kChunk;
    const int nch = (int)((n + chunk - 1) / chunk);
    *nchunk = nch;
    HDF_CUDA(part.alloc_on(sizeof(double) * (size_t)nch * c * r, st));
    HDF_CUDA(cudaMemsetAsync(part.p, 0, sizeof(double) * (size_t)nch * c * r, st));
    if (slot->count == 0) return HDF_OK;
    dev::MfUtvArgs a{};
    a.Z = mf.Z.p; a.ldZ = mf.ldZ; a.A0F = mf.A0F.p; a.ldA = mf.ldA;
    a.V = V; a.ldv = ldv; a.c = c;
    a.n = n; a.chunk = chunk;
    a.items = slot->buf.as<int4>();
    a.zoff = mf.dzoff.as<int>(); a.zcnt = mf.dzcnt.as<int>(); a.aoff = mf.daoff.as<int>(); a.acnt = mf.dacnt.as<int>();
    a.wcol = mf.dwcol.as<int64_t>();
    a.part = part.as<double>(); a.r = r;
    const size_t sm = sizeof(T) * (size_t)dev::MfShape<T>::SMEM;
    HDF_CUDA(cudaFuncSetAttribute(dev::k_mf_utv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HDF_COUNT_LAUNCH();
    dev::k_mf_utv<T><<<dim3((unsigned)slot->count, (unsigned)nch), 256, sm, st>>>(a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}
template hdf_status mf_utv<float>(const hdf_factor*, const float*, int64_t, int, DevBuf&, int*, cudaStream_t);
template hdf_status mf_utv<double>(const hdf_factor*, const double*, int64_t, int, DevBuf&, int*, cudaStream_t);

// Y = U W for W (ldu x c row-major, bulk type), c <= 64.
template <typename T>
hdf_status mf_uw(const hdf_factor* f, const T* W, int c, T* Y, int64_t ldy, cudaStream_t st) {
    const FreeFactor& mf = f->mf;
    const int64_t n = f->info.n;
    if constexpr (sizeof(T) == 4) {
        if (use_tensor_cores(f)) {
            FreeFactor::TcLists* L = nullptr;
            if (hdf_status e = tc_lists(f, c, &L); e != HDF_OK) return e;
            return tc_mf_uw(tc_view(f), L->phases.as<int4>(), L->nphase, L->kpad, reinterpret_cast<const float*>(W), c,
                            reinterpret_cast<float*>(Y), ldy, f->dev_err.as<int>(), st);
        }
    }
    dev::MfUwArgs a{};
    a.Z = mf.Z.p; a.ldZ = mf.ldZ; a.A0F = mf.A0F.p; a.ldA = mf.ldA;
    a.W = W; a.c = c; a.cp = pow2_at_least(c, 4);
    a.Y = Y; a.ldy = ldy;
    a.n = n; a.L = mf.L_used;
    a.zoff = mf.dzoff.as<int>(); a.zcnt = mf.dzcnt.as<int>(); a.aoff = mf.daoff.as<int>(); a.acnt = mf.dacnt.as<int>();
    a.wcol = mf.dwcol.as<int64_t>();
    constexpr int BI = dev::MfShape<T>::BI;
    const size_t sm = sizeof(T) * (size_t)dev::MfShape<T>::UW_SMEM;
    HDF_CUDA(cudaFuncSetAttribute(dev::k_mf_uw<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    HDF_COUNT_LAUNCH();
    dev::k_mf_uw<T><<<(unsigned)((n + BI - 1) / BI), 256, sm, st>>>(a);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}
template hdf_status mf_uw<float>(const hdf_factor*, const float*, int, float*, int64_t, cudaStream_t);
template hdf_status mf_uw<double>(const hdf_factor*, const double*, int, double*, int64_t, cudaStream_t);

}  // namespace hdf
