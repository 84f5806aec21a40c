// Adjoint of f = sum_j w_j^T K~ v_j with respect to the points and the lengthscale.
//
// The paper does not differentiate the factorization.  We use frozen-structure semantics:
// the scaling (c, R), the degree p, the radial-basis factor and the kept eigenvectors are
// those of the build, so that row i of U is an explicit smooth function of x_i,
//     U_i[(k,s,h)] = F_ks(|x'_i|) Y_k^h(x'_i / |x'_i|),  x' = (x - c)/(2R),
// and S depends on l only through the radial cores: S_k(l) = W_k^T R_f Gamma_k(l) R_f^T W_k.
// Then, with a = S U^T v and b = S U^T w,
//     grad_{x_i} f = (w_i a + v_i b) . dU_i/dx_i,     df/dl = (U^T w)^T (dS/dl) (U^T v).
// The kernel recomputes F, dF/drho, the harmonics and their gradients per point (nothing of
// U's Jacobian is stored): for a solid harmonic H of degree k (H(x_hat) = Y(x_hat)),
//     d/dx' [F(rho) Y(x'/rho)] = [F' - k F/rho] Y x_hat + (F/rho) grad H(x_hat).
// grad H comes from carrying d/dz and d/dq through the level recurrences
// P(n) = A z P(n-1) - B q P(n-2) (z = x_{D_j}, q = |x_{0..D_j}|^2) and from
// d(x0 + i x1)^mu = mu (x0 + i x1)^(mu-1) (dx0 + i dx1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "hdf_kernels.cuh"
#include "internal.h"

#include <type_traits>
#include "planner.h"

namespace {

using hdf::dev::kMaxD;

template <typename T>
struct AdjParams {
    const double* x; int64_t n; int d; double c[kMaxD]; double inv2R;
    int L;                         // degrees of the harmonic tables (L_used)
    int Lr;                        // radial degree: basis sizes Lr+1 (even), Lr (odd)
    int tri;
    const double* Qm0; int nb0, m0;
    const double* Qm1; int nb1, m1;
    const float2* QC; int mtp;                     // FP32 factors: [Qm0 | Qm1] as float pairs, (Lr+1) x mtp
    const T* Wt; const uint8_t* colk; int nF;
    const int16_t* chains; int nH, cstride; const uint8_t* hk; const int* ktab;
    const T* coefA; const T* coefB;
    const T* a; const T* b; int ab_stride;        // a[col * ab_stride], b[col * ab_stride]
    const T* v; const T* w;                        // this column of V and W (length n)
    T* grad; int accumulate;
    int per_warp_d;                                // doubles per warp
    int per_warp_t;                                // T elements per warp
};

// Double-float helpers for the FP32 form (FP32 pairs, error-free products and sums).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float2 df_norm(float s, float e) {
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {          // a * b
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    return df_norm(p, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {          // a + b
    float s, e;
    df_two_sum(a.x, b.x, s, e);
    e += a.y + b.y;
    return df_norm(s, e);
}
__device__ __forceinline__ void df_dot_step(float2 a, float2 b, float& sh, float& c) {   // Dot2 step
    const float ph = a.x * b.x;
    float pe = fmaf(a.x, b.x, -ph);
    pe = fmaf(a.x, b.y, fmaf(a.y, b.x, pe));
    float s2, es;
    df_two_sum(sh, ph, s2, es);
    sh = s2;
    c += es + pe;
}

// DD = the dimension d (a template parameter, so that the per-thread coordinate and gradient
// arrays stay in registers).
template <typename T, int DD>
__global__ void __launch_bounds__(128) k_adjoint(AdjParams<T> P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    constexpr int levels = DD - 2;
    double* dbase = reinterpret_cast<double*>(smem_raw) + (size_t)warp * P.per_warp_d;
    double* Tl = dbase;                        // Lr+1: T_l(u)
    double* dTl = Tl + (P.Lr + 1);             // Lr+1: T_l'(u)
    double* Q = dTl + (P.Lr + 1);              // m0+m1
    double* dQ = Q + (P.m0 + P.m1);            // m0+m1
    T* tbase = reinterpret_cast<T*>(reinterpret_cast<double*>(smem_raw) + (size_t)nwarps * P.per_warp_d) +
               (size_t)warp * P.per_warp_t;
    T* R1 = tbase;                             // nF
    T* R2 = R1 + P.nF;                         // nF
    T* tv = R2 + P.nF;                         // levels * tri: P
    T* tz = tv + levels * P.tri;               // dP/dz
    T* tq = tz + levels * P.tri;               // dP/dq
    T* trig = tq + levels * P.tri;             // 2L+1
    T* trx = trig + 2 * P.L + 1;               // d/dx0
    T* try_ = trx + 2 * P.L + 1;               // d/dx1
    const int64_t gw = (int64_t)blockIdx.x * nwarps + warp, nw = (int64_t)gridDim.x * nwarps;
    for (int64_t i = gw; i < P.n; i += nw) {
        T xh[kMaxD];
        double s2 = 0.0;
        if constexpr (sizeof(T) == 4) {
            // lane j forms coordinate j in FP64 once; |x'|^2 by an FP64 shuffle tree over the
            // first eight lanes; the warp shares the coordinates in FP32 (FP64 issues at a small
            // fraction of the FP32 rate on this GPU)
            double cj = P.c[0];                  // this lane's centre coordinate (register selects)
#pragma unroll
            for (int j = 1; j < DD; ++j) cj = (lane == j) ? P.c[j] : cj;
            const double xd = (lane < DD) ? (P.x[i * DD + lane] - cj) * P.inv2R : 0.0;   // one FP64 sub, mul
            double sq = xd * xd;
            sq += __shfl_xor_sync(0xffffffffu, sq, 4);
            sq += __shfl_xor_sync(0xffffffffu, sq, 2);
            sq += __shfl_xor_sync(0xffffffffu, sq, 1);
            s2 = __shfl_sync(0xffffffffu, sq, 0);
            const float xf = (float)xd;
#pragma unroll
            for (int j = 0; j < DD; ++j) xh[j] = __shfl_sync(0xffffffffu, xf, j);
        } else {
#pragma unroll
            for (int j = 0; j < DD; ++j) { xh[j] = (P.x[i * DD + j] - P.c[j]) * P.inv2R; s2 += xh[j] * xh[j]; }
        }
        double rho;
        if constexpr (sizeof(T) == 4) {
            // FP32 factors: the radial part in double-float / FP32 arithmetic (FP64 is slow here)
            const float s2f = (float)s2;
            const float rhof = sqrtf(s2f);
            rho = rhof;
            if (s2 > 0.0) { const float inv = 1.f / rhof; for (int j = 0; j < DD; ++j) xh[j] *= inv; }
            else { for (int j = 0; j < DD; ++j) xh[j] = (j == 0) ? 1.f : 0.f; }
            float2* Tl2 = reinterpret_cast<float2*>(Tl);
            float2* dTl2 = reinterpret_cast<float2*>(dTl);
            float* Qf = reinterpret_cast<float*>(Q);
            float* dQf = reinterpret_cast<float*>(dQ);
            if (lane == 0) {
                const double u = 8.0 * s2 - 1.0;
                const float uh = (float)u, ul = (float)(u - (double)uh);
                const float2 u2 = make_float2(2.f * uh, 2.f * ul);
                float2 t2 = make_float2(1.f, 0.f), t1 = make_float2(uh, ul);       // T_{l-2}, T_{l-1}
                float2 d2 = make_float2(0.f, 0.f), d1 = make_float2(1.f, 0.f);     // T'_{l-2}, T'_{l-1}
                Tl2[0] = t2; dTl2[0] = d2;
                if (P.Lr >= 1) { Tl2[1] = t1; dTl2[1] = d1; }
                for (int l = 2; l <= P.Lr; ++l) {
                    const float2 tn = df_add(df_mul(u2, t1), make_float2(-t2.x, -t2.y));
                    const float2 dn = df_add(df_add(make_float2(2.f * t1.x, 2.f * t1.y), df_mul(u2, d1)),
                                             make_float2(-d2.x, -d2.y));
                    Tl2[l] = tn; dTl2[l] = dn;
                    t2 = t1; t1 = tn;
                    d2 = d1; d1 = dn;
                }
            }
            __syncwarp();
            // S_T[o] = sum_l T_l Qmat[l][o], S_dT[o] = sum_l T'_l Qmat[l][o] (Dot2); then
            // even: Q = S_T, dQ = 16 rho S_dT;  odd: Q = rho S_T, dQ = S_T + 16 rho^2 S_dT
            for (int o = lane; o < P.m0 + P.m1; o += 32) {
                const bool odd = o >= P.m0;
                const int nb = odd ? P.nb1 : P.nb0;
                float th = 0.f, tc = 0.f, dh = 0.f, dc = 0.f;
                for (int l = 0; l < nb; ++l) {
                    const float2 qm = P.QC[(size_t)l * P.mtp + o];
                    df_dot_step(Tl2[l], qm, th, tc);
                    df_dot_step(dTl2[l], qm, dh, dc);
                }
                const float st = th + tc, sd = dh + dc;
                if (!odd) { Qf[o] = st; dQf[o] = 16.f * rhof * sd; }
                else { Qf[o] = rhof * st; dQf[o] = st + 16.f * s2f * sd; }
            }
            __syncwarp();
            for (int col = lane; col < P.nF; col += 32) {
                const int k = P.colk[col];
                const int par = k & 1, ob = par ? P.m0 : 0, mp = par ? P.m1 : P.m0;
                float F = 0.f, dF = 0.f;
                for (int l = 0; l < mp; ++l) {
                    const float wv = (float)P.Wt[(int64_t)l * P.nF + col];
                    F += Qf[ob + l] * wv;
                    dF += dQf[ob + l] * wv;
                }
                if (rhof > 1e-30f) {
                    R1[col] = (T)(dF - k * F / rhof);
                    R2[col] = (T)(F / rhof);
                } else {
                    R1[col] = (T)dF;
                    R2[col] = (T)0;
                }
            }
        } else {
        rho = sqrt(s2);
        if (s2 > 0.0) { for (int j = 0; j < DD; ++j) xh[j] = (T)(xh[j] / rho); }
        else { for (int j = 0; j < DD; ++j) xh[j] = (j == 0) ? (T)1 : (T)0; }
        const double u = 8.0 * s2 - 1.0;
        if (lane == 0) {
            Tl[0] = 1.0; dTl[0] = 0.0;
            if (P.Lr >= 1) { Tl[1] = u; dTl[1] = 1.0; }
            for (int l = 2; l <= P.Lr; ++l) {
                Tl[l] = 2.0 * u * Tl[l - 1] - Tl[l - 2];
                dTl[l] = 2.0 * Tl[l - 1] + 2.0 * u * dTl[l - 1] - dTl[l - 2];
            }
        }
        __syncwarp();
        // Q = B Qmat and dQ/drho; B0 = T_l, B0' = 16 rho T_l'; B1 = rho T_l, B1' = T_l + 16 rho^2 T_l'
        for (int o = lane; o < P.m0 + P.m1; o += 32) {
            double q = 0.0, dq = 0.0;
            if (o < P.m0) {
                for (int l = 0; l < P.nb0; ++l) {
                    const double qm = P.Qm0[l * P.m0 + o];
                    q += Tl[l] * qm;
                    dq += 16.0 * rho * dTl[l] * qm;
                }
            } else {
                const int oo = o - P.m0;
                for (int l = 0; l < P.nb1; ++l) {
                    const double qm = P.Qm1[l * P.m1 + oo];
                    q += rho * Tl[l] * qm;
                    dq += (Tl[l] + 16.0 * s2 * dTl[l]) * qm;
                }
            }
            Q[o] = q;
            dQ[o] = dq;
        }
        __syncwarp();
        // radial factors: R1 = F' - k F / rho, R2 = F / rho (tangential term dropped at rho = 0)
        for (int col = lane; col < P.nF; col += 32) {
            const int k = P.colk[col];
            const int par = k & 1, ob = par ? P.m0 : 0, mp = par ? P.m1 : P.m0;
            double F = 0.0, dF = 0.0;
            for (int l = 0; l < mp; ++l) {
                const double wv = (double)P.Wt[(int64_t)l * P.nF + col];
                F += Q[ob + l] * wv;
                dF += dQ[ob + l] * wv;
            }
            if (rho > 1e-30) {
                R1[col] = (T)(dF - k * F / rho);
                R2[col] = (T)(F / rho);
            } else {
                R1[col] = (T)dF;
                R2[col] = (T)0;
            }
        }
        }
        // level tables with d/dz and d/dq
        for (int j = 0; j < levels; ++j) {
            const int D = DD - 1 - j;
            T q = (T)0;
#pragma unroll
            for (int m = 0; m < DD; ++m)
                if (m <= D) q += xh[m] * xh[m];
            const T z = xh[D], qq = q;
            const T* A = P.coefA + j * P.tri;
            const T* B = P.coefB + j * P.tri;
            T* pv = tv + j * P.tri;
            T* pz = tz + j * P.tri;
            T* pq = tq + j * P.tri;
            for (int mu = lane; mu <= P.L; mu += 32) {
                const int o = mu * (P.L + 1) - mu * (mu - 1) / 2;
                const int nmax = P.L - mu;
                T v2 = A[o], z2 = (T)0, q2 = (T)0;
                pv[o] = v2; pz[o] = z2; pq[o] = q2;
                if (nmax >= 1) {
                    T v1 = A[o + 1] * z, z1 = A[o + 1], q1 = (T)0;
                    pv[o + 1] = v1; pz[o + 1] = z1; pq[o + 1] = q1;
                    for (int nn = 2; nn <= nmax; ++nn) {
                        const T an = A[o + nn], bn = B[o + nn];
                        const T v0 = an * z * v1 - bn * qq * v2;
                        const T z0 = an * (v1 + z * z1) - bn * qq * z2;
                        const T q0 = an * z * q1 - bn * (v2 + qq * q2);
                        pv[o + nn] = v0; pz[o + nn] = z0; pq[o + nn] = q0;
                        v2 = v1; z2 = z1; q2 = q1;
                        v1 = v0; z1 = z0; q1 = q0;
                    }
                }
            }
        }
        // (x0 + i x1)^mu and its derivatives, normalised as the harmonics
        typedef typename std::conditional<sizeof(T) == 4, float, double>::type TP;   // trig precision
        for (int mu = lane; mu <= P.L; mu += 32) {
            TP br = (TP)xh[0], bi = (TP)xh[1], rr = 1, ri = 0;     // z^mu
            TP pr = 1, pi = 0;                                      // z^(mu-1)
            int e = mu;
            while (e) {
                if (e & 1) { const TP t = rr * br - ri * bi; ri = rr * bi + ri * br; rr = t; }
                const TP t = br * br - bi * bi; bi = (TP)2 * br * bi; br = t;
                e >>= 1;
            }
            if (mu >= 1) {
                br = (TP)xh[0]; bi = (TP)xh[1]; e = mu - 1;
                while (e) {
                    if (e & 1) { const TP t = pr * br - pi * bi; pi = pr * bi + pi * br; pr = t; }
                    const TP t = br * br - bi * bi; bi = (TP)2 * br * bi; br = t;
                    e >>= 1;
                }
            }
            if (mu == 0) {
                trig[P.L] = (T)0.3989422804014327;
                trx[P.L] = (T)0;
                try_[P.L] = (T)0;
            } else {
                const TP nm = (TP)0.5641895835477563;
                trig[P.L + mu] = (T)(rr * nm);            // Re z^mu
                trig[P.L - mu] = (T)(ri * nm);            // Im z^mu
                trx[P.L + mu] = (T)(mu * pr * nm);        // d Re / dx0
                trx[P.L - mu] = (T)(mu * pi * nm);        // d Im / dx0
                try_[P.L + mu] = (T)(-mu * pi * nm);      // d Re / dx1
                try_[P.L - mu] = (T)(mu * pr * nm);       // d Im / dx1
            }
        }
        __syncwarp();
        const T wi = P.w[i], vi = P.v[i];
        T g[kMaxD];
#pragma unroll
        for (int m = 0; m < kMaxD; ++m) g[m] = (T)0;
        T xt[kMaxD];
#pragma unroll
        for (int m = 0; m < DD; ++m) xt[m] = (T)xh[m];
        for (int gi = lane; gi < P.nH; gi += 32) {
            const int k = P.hk[gi];
            const int* kt = P.ktab + hdf::kTabStride * k;
            const int fb = kt[0], sk = kt[1], cb = kt[2], hb = kt[4], dimp = kt[5];
            const int h = gi - hb;
            T al = (T)0, be = (T)0;
            for (int s = 0; s < sk; ++s) {
                const int64_t col = cb + (int64_t)s * dimp + h;
                const T cc = wi * P.a[col * P.ab_stride] + vi * P.b[col * P.ab_stride];
                al += cc * R1[fb + s];
                be += cc * R2[fb + s];
            }
            const int16_t* ch = P.chains + (int64_t)gi * P.cstride;
            const int tmu = ch[levels];
            T pvv[kMaxD], pzz[kMaxD], pqq[kMaxD];
#pragma unroll
            for (int j = 0; j < levels; ++j) {
                pvv[j] = tv[j * P.tri + ch[j]];
                pzz[j] = tz[j * P.tri + ch[j]];
                pqq[j] = tq[j * P.tri + ch[j]];
            }
            // suffix products suf[j] = prod_{j2 > j} P_j2, so that the product of all level
            // factors but one is (trig * prefix) * suffix: O(levels) per harmonic
            T suf[kMaxD];
            if (levels > 0) suf[levels - 1] = (T)1;
#pragma unroll
            for (int j = levels - 2; j >= 0; --j) suf[j] = suf[j + 1] * pvv[j + 1];
            const T pl = (levels > 0) ? pvv[0] * suf[0] : (T)1;      // all level factors
            const T tr = trig[P.L + tmu];
            const T prod = tr * pl;
            // Y x_hat term
#pragma unroll
            for (int m = 0; m < DD; ++m) g[m] += al * prod * xt[m];
            // grad H: level terms
            T pre = tr;                                  // trig * prod_{j2 < j} P_j2
#pragma unroll
            for (int j = 0; j < levels; ++j) {
                const T other = pre * suf[j];
                pre *= pvv[j];
                const int D = DD - 1 - j;
                const T cz = be * other * pzz[j], cq = be * other * pqq[j] * (T)2;
                g[D] += cz;
#pragma unroll
                for (int m = 0; m < DD; ++m)
                    if (m <= D) g[m] += cq * xt[m];
            }
            // grad H: trigonometric factor
            g[0] += be * pl * trx[P.L + tmu];
            g[1] += be * pl * try_[P.L + tmu];
        }
#pragma unroll
        for (int m = 0; m < DD; ++m) {
            T vsum = g[m];
            for (int o = 16; o > 0; o >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, o);
            g[m] = vsum;
        }
        if (lane < DD) {
            T vsum = (T)0;
#pragma unroll
    #pragma unroll
        for (int m = 0; m < DD; ++m) if (m == lane) vsum = g[m];
            const T out = vsum * (T)P.inv2R;
            T* dst = P.grad + i * DD + lane;
            *dst = P.accumulate ? *dst + out : out;
        }
        __syncwarp();
    }
}

// dS_k/dl = W_k^T R_f (dGamma_k/dl) R_f^T W_k with dGamma from the Chebyshev coefficients of
// d kappa/d l truncated at the build's degree (frozen p, c, R).
void compute_dS(hdf_factor* f) {
    FactorPlan& P = f->plan;
    const int M = hdf::cheb_nodes(P.p_max);          // the build's node count
    std::vector<double> a(std::max(M, 2 * P.L + 2));
    hdf::cheb_coeffs(f->kernel, f->ell, 1.0 / P.inv2R, M, true, a.data());
    for (size_t i = 2 * P.L + 1; i < a.size(); ++i) a[i] = 0.0;
    std::vector<std::vector<double>> dG;
    hdf::radial_cores(a.data(), 2 * P.L, P.d, dG);
    P.dSk.assign(P.L + 1, std::vector<double>());
    for (int k = 0; k <= P.L; ++k) {
        const int sk = P.sk[k];
        if (sk == 0) continue;
        const int par = k & 1, nb = P.nb[par], mk = P.m[par];
        const std::vector<double>& Rf = P.Rf[par];
        const std::vector<double>& W = P.Wk[k];
        // T1 = R_f dG R_f^T (mk x mk)
        std::vector<double> A((size_t)mk * nb, 0.0), T1((size_t)mk * mk, 0.0), T2((size_t)sk * mk, 0.0);
        for (int o = 0; o < mk; ++o)
            for (int l = 0; l < nb; ++l) {
                double s = 0.0;
                for (int t = 0; t < nb; ++t) s += Rf[(size_t)o * nb + t] * dG[k][(size_t)t * nb + l];
                A[(size_t)o * nb + l] = s;
            }
        for (int o = 0; o < mk; ++o)
            for (int o2 = 0; o2 < mk; ++o2) {
                double s = 0.0;
                for (int l = 0; l < nb; ++l) s += A[(size_t)o * nb + l] * Rf[(size_t)o2 * nb + l];
                T1[(size_t)o * mk + o2] = s;
            }
        for (int s_ = 0; s_ < sk; ++s_)
            for (int o2 = 0; o2 < mk; ++o2) {
                double s = 0.0;
                for (int o = 0; o < mk; ++o) s += W[(size_t)o * sk + s_] * T1[(size_t)o * mk + o2];
                T2[(size_t)s_ * mk + o2] = s;
            }
        std::vector<double> dS((size_t)sk * sk, 0.0);
        for (int s_ = 0; s_ < sk; ++s_)
            for (int t_ = 0; t_ < sk; ++t_) {
                double s = 0.0;
                for (int o2 = 0; o2 < mk; ++o2) s += T2[(size_t)s_ * mk + o2] * W[(size_t)o2 * sk + t_];
                dS[(size_t)s_ * sk + t_] = s;
            }
        P.dSk[k].swap(dS);
    }
    P.have_dS = true;
}

template <typename T>
hdf_status run(hdf_factor* f, const double* x, const T* V, int64_t ldv, const T* Wv, int64_t ldw, int ncols,
               T* grad, double* grad_l, double* value, cudaStream_t st) {
    FactorPlan& P = f->plan;
    const int64_t n = f->info.n, r = (f->info.rank > 0) ? f->info.ldu : 0;   // padded width of U
    const int d = P.d;
    if (r == 0) {
        HDF_CUDA(cudaMemsetAsync(grad, 0, sizeof(T) * n * d, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        if (grad_l) *grad_l = 0.0;
        if (value) *value = 0.0;
        return HDF_OK;
    }
    DevBuf ab, zd, vw;
    HDF_CUDA(ab.alloc(sizeof(T) * (size_t)r * ncols * 2));
    HDF_CUDA(zd.alloc_on(sizeof(double) * (size_t)r * ncols * 2, st));
    T* a = ab.as<T>();                         // S U^T V  (r x ncols)
    T* b = a + (size_t)r * ncols;              // S U^T W
    // U^T [V W] (FP64, r x 2 ncols row-major) in one pass over U when the 2 ncols columns fit
    // one group: [V W] is gathered into an n x 2 ncols column-major block first
    std::vector<double> hz((size_t)r * ncols * 2);
    const int c2 = 2 * ncols;
    if (c2 <= 64) {
        HDF_CUDA(vw.alloc_on(sizeof(T) * (size_t)n * c2, st));
        HDF_CUDA(cudaMemcpy2DAsync(vw.p, sizeof(T) * n, V, sizeof(T) * ldv, sizeof(T) * n, ncols,
                                   cudaMemcpyDeviceToDevice, st));
        HDF_CUDA(cudaMemcpy2DAsync(vw.as<T>() + (size_t)n * ncols, sizeof(T) * n, Wv, sizeof(T) * ldw, sizeof(T) * n,
                                   ncols, cudaMemcpyDeviceToDevice, st));
        hdf_status s = hdf::utv_reduce<T>(f, vw.as<T>(), n, c2, nullptr, nullptr, zd.as<double>(), st);
        if (s != HDF_OK) return s;
        HDF_CUDA(cudaMemcpyAsync(hz.data(), zd.p, sizeof(double) * hz.size(), cudaMemcpyDeviceToHost, st));
    } else {
        double* zv = zd.as<double>();
        double* zw = zv + (size_t)r * ncols;
        hdf_status s = hdf::utv_reduce<T>(f, V, ldv, ncols, nullptr, nullptr, zv, st);
        if (s != HDF_OK) return s;
        s = hdf::utv_reduce<T>(f, Wv, ldw, ncols, nullptr, nullptr, zw, st);
        if (s != HDF_OK) return s;
        std::vector<double> hv((size_t)r * ncols * 2);
        HDF_CUDA(cudaMemcpyAsync(hv.data(), zd.p, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        for (int64_t col = 0; col < r; ++col)          // into the [V W] row layout
            for (int j = 0; j < ncols; ++j) {
                hz[(size_t)col * c2 + j] = hv[(size_t)col * ncols + j];
                hz[(size_t)col * c2 + ncols + j] = hv[(size_t)r * ncols + (size_t)col * ncols + j];
            }
    }
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<T> ha((size_t)r * ncols), hb((size_t)r * ncols);
    double fval = 0.0;
    for (int64_t col = 0; col < r; ++col)
        for (int j = 0; j < ncols; ++j) {
            const size_t q = (size_t)col * ncols + j;
            const double sc = P.Spad[col];
            const double zv = hz[(size_t)col * c2 + j], zw = hz[(size_t)col * c2 + ncols + j];
            ha[q] = (T)(sc * zv);
            hb[q] = (T)(sc * zw);
            fval += zw * sc * zv;
        }
    HDF_CUDA(cudaMemcpyAsync(a, ha.data(), sizeof(T) * ha.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(b, hb.data(), sizeof(T) * hb.size(), cudaMemcpyHostToDevice, st));

    AdjParams<T> A{};
    A.x = x;
    A.n = n; A.d = d;
    for (int j = 0; j < d; ++j) A.c[j] = P.c[j];
    A.inv2R = P.inv2R;
    A.L = P.L_used; A.Lr = P.L; A.tri = P.tri;
    A.Qm0 = P.dQ0.as<double>(); A.nb0 = P.nb[0]; A.m0 = P.m[0];
    A.Qm1 = P.dQ1.as<double>(); A.nb1 = P.nb[1]; A.m1 = P.m[1];
    A.QC = P.dQC.as<float2>(); A.mtp = ((P.m[0] + P.m[1] + 7) / 8) * 8;
    if (sizeof(T) == 4 && A.QC == nullptr) return hdf::fail(HDF_EINVAL, "hdf_matvec_adjoint: factor lacks its FP32 radial tables");
    A.Wt = P.dW.as<T>(); A.colk = P.dcolk.as<uint8_t>(); A.nF = P.nF;
    A.chains = P.dchains.as<int16_t>(); A.nH = P.nH; A.cstride = hdf::chain_stride(d);
    A.hk = P.dhk.as<uint8_t>(); A.ktab = P.dktab.as<int>();
    A.coefA = P.dA.as<T>(); A.coefB = P.dB.as<T>();
    A.grad = grad;
    const int levels = d - 2;
    A.per_warp_d = 2 * (P.L + 1) + 2 * (P.m[0] + P.m[1]);
    A.per_warp_t = ((2 * P.nF + 3 * levels * P.tri + 3 * (2 * P.L_used + 1)) + 3) & ~3;
    const int warps = 4;
    const size_t sm = sizeof(double) * warps * A.per_warp_d + sizeof(T) * warps * A.per_warp_t;
    if (sm > 200 * 1024) return hdf::fail(HDF_ETOOBIG, "hdf_matvec_adjoint: per-point tables exceed shared memory");
    void (*kern)(AdjParams<T>) = d == 3 ? k_adjoint<T, 3> : d == 4 ? k_adjoint<T, 4> : d == 5 ? k_adjoint<T, 5>
                               : d == 6 ? k_adjoint<T, 6> : d == 7 ? k_adjoint<T, 7> : k_adjoint<T, 8>;
    HDF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int nsm = 0, dv = 0, occ = 0;
    HDF_CUDA(cudaGetDevice(&dv));
    HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
    HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm));
    const int grid = std::max(1, std::min<int>(nsm * std::max(occ, 1), (int)((n + warps - 1) / warps)));
    for (int j = 0; j < ncols; ++j) {
        A.a = a + j; A.b = b + j; A.ab_stride = ncols;
        A.v = V + j * ldv; A.w = Wv + j * ldw;
        A.accumulate = (j > 0);
        HDF_COUNT_LAUNCH();
        kern<<<grid, warps * 32, sm, st>>>(A);
        HDF_CUDA(cudaGetLastError());
    }
    // d f / d l on the host from U^T V, U^T W and the frozen dS_k/dl
    if (grad_l) {
        if (!P.have_dS) compute_dS(f);
        double gl = 0.0;
        std::vector<double> tmp;
        for (int k = 0; k <= P.L; ++k) {
            const int sk = P.sk[k];
            if (sk == 0) continue;
            const int dim = (int)hdf::harmonic_count(k, d);
            const int dimp = (k + 1 < (int)P.cbase.size() && sk > 0) ? (P.cbase[k + 1] - P.cbase[k]) / sk : dim;
            const std::vector<double>& dS = P.dSk[k];
            for (int j = 0; j < ncols; ++j)
                for (int h = 0; h < dim; ++h)
                    for (int s_ = 0; s_ < sk; ++s_) {
                        const int64_t cs = P.cbase[k] + (int64_t)s_ * dimp + h;
                        double acc = 0.0;
                        for (int t_ = 0; t_ < sk; ++t_) {
                            const int64_t ct = P.cbase[k] + (int64_t)t_ * dimp + h;
                            acc += dS[(size_t)s_ * sk + t_] * hz[(size_t)ct * c2 + j];
                        }
                        gl += hz[(size_t)cs * c2 + ncols + j] * acc;
                    }
        }
        *grad_l = gl;
    }
    if (value) *value = fval;
    HDF_CUDA(cudaStreamSynchronize(st));
    return hdf::take_device_error(f);
}

}  // namespace

extern "C" hdf_status hdf_matvec_adjoint(hdf_factor* f, const double* x_dev, const void* V_dev, int64_t ldv,
                                         const void* W_dev, int64_t ldw, int ncols, void* grad_x_dev,
                                         double* grad_l_host, double* value_host, hdf_stream stream) {
    if (!f || !x_dev || !V_dev || !W_dev || !grad_x_dev || ncols < 1 || ncols > 64 || ldv < f->info.n ||
        ldw < f->info.n)
        return hdf::fail(HDF_EINVAL, "hdf_matvec_adjoint: bad argument (1 <= ncols <= 64)");
    if (f->ypart) return hdf::fail(HDF_EINVAL, "hdf_matvec_adjoint: symmetric factors only");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (f->prec == HDF_FP64)
        return run<double>(f, x_dev, (const double*)V_dev, ldv, (const double*)W_dev, ldw, ncols, (double*)grad_x_dev,
                           grad_l_host, value_host, st);
    return run<float>(f, x_dev, (const float*)V_dev, ldv, (const float*)W_dev, ldw, ncols, (float*)grad_x_dev,
                      grad_l_host, value_host, st);
}
