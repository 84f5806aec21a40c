// Checks of the library's host numerics (planner.cpp) against their defining properties:
// the one-sided Jacobi SVD (A = U S V^T, orthonormal factors, sorted values, rank-deficient
// and wide inputs), the register-blocked rank-k update (against the plain triple loop), and
// the symmetric eigensolver (A V = V diag(w), V orthonormal).  Prints one line per check and
// exits non-zero on the first failure.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "planner.h"

using namespace hdf;

static int fails = 0;
static void report(const char* what, double err, double bound) {
    const bool ok = err <= bound;
    std::printf("%s %s err %.3e bound %.1e\n", ok ? "ok  " : "FAIL", what, err, bound);
    if (!ok) ++fails;
}

int main() {
    std::mt19937_64 g(7);
    std::normal_distribution<double> nd;
    // SVD
    const int shapes[][2] = {{1, 1}, {4, 1}, {1, 5}, {6, 3}, {3, 6}, {17, 17}, {40, 23}, {23, 40}, {65, 65}};
    for (auto& sh : shapes) {
        const int m = sh[0], n = sh[1], q = std::min(m, n);
        std::vector<double> A((size_t)m * n);
        for (auto& v : A) v = nd(g);
        if (m > 5 && n > 5)
            for (int j = 0; j < n; ++j) A[(size_t)3 * n + j] = 2.0 * A[(size_t)1 * n + j];   // rank drop
        std::vector<double> U((size_t)m * q), s(q), V((size_t)n * q);
        svd_jacobi(m, n, A.data(), U.data(), s.data(), V.data());
        double rec = 0.0, amax = 0.0, orth = 0.0, order = 0.0;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double t = 0.0;
                for (int o = 0; o < q; ++o) t += U[(size_t)i * q + o] * s[o] * V[(size_t)j * q + o];
                rec = std::max(rec, std::fabs(t - A[(size_t)i * n + j]));
                amax = std::max(amax, std::fabs(A[(size_t)i * n + j]));
            }
        for (int a = 0; a < q; ++a) {
            if (a > 0) order = std::max(order, s[a] - s[a - 1]);
            for (int b = 0; b < q; ++b) {
                double vv = 0.0, uu = 0.0;
                for (int j = 0; j < n; ++j) vv += V[(size_t)j * q + a] * V[(size_t)j * q + b];
                orth = std::max(orth, std::fabs(vv - (a == b)));
                if (s[a] > 1e-10 * s[0] && s[b] > 1e-10 * s[0]) {
                    for (int i = 0; i < m; ++i) uu += U[(size_t)i * q + a] * U[(size_t)i * q + b];
                    orth = std::max(orth, std::fabs(uu - (a == b)));
                }
            }
        }
        char buf[96];
        std::snprintf(buf, sizeof(buf), "svd %dx%d reconstruction", m, n);
        report(buf, rec / amax, 1e-13);
        std::snprintf(buf, sizeof(buf), "svd %dx%d orthonormality", m, n);
        report(buf, orth, 1e-12);
        std::snprintf(buf, sizeof(buf), "svd %dx%d decreasing values", m, n);
        report(buf, std::max(0.0, order), 0.0);
    }
    // rank-k update C -= A B
    const int dims[][3] = {{1, 1, 1}, {4, 8, 3}, {5, 9, 64}, {33, 70, 17}, {128, 131, 64}};
    for (auto& dm : dims) {
        const int m = dm[0], n = dm[1], k = dm[2];
        const int lda = k + 3, ldb = n + 5, ldc = n + 2;
        std::vector<double> A((size_t)m * lda), B((size_t)k * ldb), C((size_t)m * ldc), R;
        for (auto& v : A) v = nd(g);
        for (auto& v : B) v = nd(g);
        for (auto& v : C) v = nd(g);
        R = C;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double t = 0.0;
                for (int q = 0; q < k; ++q) t += A[(size_t)i * lda + q] * B[(size_t)q * ldb + j];
                R[(size_t)i * ldc + j] -= t;
            }
        gemm_minus(m, n, k, A.data(), lda, B.data(), ldb, C.data(), ldc);
        double err = 0.0;
        for (size_t e = 0; e < C.size(); ++e) err = std::max(err, std::fabs(C[e] - R[e]));
        char buf[96];
        std::snprintf(buf, sizeof(buf), "gemm_minus %dx%dx%d (padding columns untouched)", m, n, k);
        report(buf, err, 1e-12 * k);
    }
    // symmetric eigensolver
    for (int n : {1, 2, 9, 40}) {
        std::vector<double> A((size_t)n * n), Ac, w(n), V((size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j <= i; ++j) A[(size_t)i * n + j] = A[(size_t)j * n + i] = nd(g);
        Ac = A;
        sym_eig(n, Ac.data(), w.data(), V.data());
        double res = 0.0, orth = 0.0;
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < n; ++c) {
                double t = 0.0, o = 0.0;
                for (int j = 0; j < n; ++j) {
                    t += A[(size_t)i * n + j] * V[(size_t)j * n + c];
                    o += V[(size_t)j * n + i] * V[(size_t)j * n + c];
                }
                res = std::max(res, std::fabs(t - w[c] * V[(size_t)i * n + c]));
                orth = std::max(orth, std::fabs(o - (i == c)));
            }
        char buf[96];
        std::snprintf(buf, sizeof(buf), "sym_eig %d residual", n);
        report(buf, res, 1e-12 * n);
        std::snprintf(buf, sizeof(buf), "sym_eig %d orthonormality", n);
        report(buf, orth, 1e-12 * n);
    }
    // Matrix-free layout: for every kept U column (k, s, h) the chain of h splits into the level-0
    // offset of P_0(m, k - m) (a0off of the A0F column (m, k, s)) and the tail of degree m (the
    // zchain entry (m, j)), and wcol + j is the column's padded position; the tails are exactly
    // the chains of H_k with mu_1 = m, in the same order, for every k >= m.
    for (int d = 4; d <= 6; ++d) {
        const int L = 9;
        FactorChoice fc;
        fc.sk.assign(L + 1, 0);
        for (int k = 0; k <= L; ++k) fc.sk[k] = (k % 4 == 3) ? 0 : 1 + (L - k) % 3;   // gaps and varied ranks
        fc.m[0] = fc.m[1] = 3;
        fc.Wk.assign(L + 1, std::vector<double>());
        for (int k = 0; k <= L; ++k) fc.Wk[k].assign((size_t)3 * fc.sk[k], 0.5);
        int64_t rank = 0;
        for (int k = 0; k <= L; ++k) rank += harmonic_count(k, d) * fc.sk[k];
        fc.S.assign(rank, 1.0);
        DeviceTables tb;
        std::string err;
        FreeTables ft;
        if (!make_tables(fc, d, L, 4, tb, err) || !make_free_tables(fc, d, L, tb, ft, err)) {
            report("matrix-free tables built", 1.0, 0.0);
            continue;
        }
        const int levels = d - 2, stride = chain_stride(d);
        double bad = 0.0;
        int64_t cols = 0;
        for (int k = 0; k <= tb.L_used; ++k) {
            if (fc.sk[k] == 0) continue;
            const int hk = (int)harmonic_count(k, d);
            // chains of H_k in order; walk the groups of equal mu_1
            int h = 0;
            for (int m = 0; m <= k; ++m) {
                for (int j = 0; j < ft.zcnt[m]; ++j, ++h) {
                    const int16_t* full = &tb.chains[(size_t)(tb.hbase[k] + h) * stride];
                    const int16_t* tail = &ft.zchain[(size_t)(ft.zoff[m] + j) * stride];
                    for (int l = 1; l < levels; ++l) bad += (full[l] != tail[l - 1]);
                    bad += (full[levels] != tail[levels - 1]);
                    for (int s = 0; s < fc.sk[k]; ++s) {
                        int q = -1;
                        for (int t = ft.aoff[m]; t < ft.aoff[m] + ft.acnt[m]; ++t)
                            if (ft.afcol[t] == tb.fbase[k] + s) q = t;
                        if (q < 0) { bad += 1; continue; }
                        bad += (ft.a0off[q] != full[0]);
                        const int64_t col = tb.cbase[k] + (int64_t)s * tb.ktab[kTabStride * k + 5] + h;
                        bad += (ft.wcol[q] + j != col);
                        ++cols;
                    }
                }
            }
            bad += (h != hk);
        }
        // A0F blocks start on 16-byte boundaries; their padding columns are marked zero
        for (int m = 0; m <= tb.L_used; ++m) {
            bad += (ft.aoff[m] % 4 != 0);
            bad += (ft.aoff[m + 1] - ft.aoff[m] != (ft.acnt[m] + 3) / 4 * 4);
            for (int t = ft.aoff[m] + ft.acnt[m]; t < ft.aoff[m + 1]; ++t) bad += (ft.a0off[t] != -1);
        }
        bad += (ft.ldA % 4 != 0 || ft.ldA < ft.nA);
        // product form (d = 4, 5): each column's packed level-1 offset and G slot name the same
        // factors as its chain; padding columns name the zero slot
        if (d == 4 || d == 5) {
            bad += ((int)ft.zpair.size() != ft.ldZ);
            const int Lu = tb.L_used;
            for (int t = 0; t < ft.ldZ && (int)ft.zpair.size() == ft.ldZ; ++t) {
                const int ia = ft.zpair[t] >> 16, ib = ft.zpair[t] & 0xFFFF;
                const int16_t* ch = t < ft.nZ ? &ft.zchain[(size_t)t * stride] : nullptr;
                if (!ch || ch[levels - 1] == 0x7fff) { bad += (ib != ft.ng); continue; }
                bad += (ia != ch[0]);
                if (d == 4) bad += (ib != Lu + ch[1]);
                else bad += (ib >= ft.ng || ft.gmap[ib] != (((int32_t)ch[1] << 16) | (Lu + ch[2])));
            }
        } else {
            bad += !ft.zpair.empty();
        }
        char buf[96];
        std::snprintf(buf, sizeof(buf), "matrix-free layout d=%d (%lld columns)", d, (long long)cols);
        report(buf, bad + (cols != rank ? 1.0 : 0.0), 0.0);
    }
    // U chunk descriptors: for every stored column (k, s, h) the chunk's two words give the radial
    // factor of (k, s) and the slot of harmonic h, and every padding column decodes to the zero
    // factor (index nF) or to a padding slot; FP32 (4 columns per chunk) and FP64 (2)
    for (int d = 3; d <= 6; ++d)
        for (int vw : {4, 2}) {
            const int L = 11;
            FactorChoice fc;
            fc.sk.assign(L + 1, 0);
            for (int k = 0; k <= L; ++k) fc.sk[k] = (k % 5 == 4) ? 0 : 1 + (k * 7 + d) % 4;
            fc.m[0] = fc.m[1] = 2;
            fc.Wk.assign(L + 1, std::vector<double>());
            for (int k = 0; k <= L; ++k) fc.Wk[k].assign((size_t)2 * fc.sk[k], 0.25);
            int64_t rank = 0;
            for (int k = 0; k <= L; ++k) rank += harmonic_count(k, d) * fc.sk[k];
            fc.S.assign(rank, 1.0);
            DeviceTables tb;
            std::string err;
            if (!make_tables(fc, d, L, vw, tb, err)) { report("chunk tables built", 1.0, 0.0); continue; }
            auto decode = [&](int64_t c, uint32_t& F, uint32_t& slot) {
                const int64_t q = c / vw;
                const int u = (int)(c % vw);
                const uint32_t w0 = tb.qdesc[2 * q], w1 = tb.qdesc[2 * q + 1];
                const uint32_t e = (w0 >> 18) & 3u;
                if (e == 0 || (uint32_t)u < e) { F = w0 >> 20; slot = (w0 & 0x3FFFFu) + u; }
                else { F = w1 >> 20; slot = (w1 & 0xFFFFFu) + u - e; }
            };
            double bad = 0.0;
            std::vector<char> stored(tb.ldU, 0);
            for (int k = 0; k <= L; ++k)
                for (int s = 0; s < fc.sk[k]; ++s)
                    for (int h = 0; h < harmonic_count(k, d); ++h) {
                        const int64_t c = tb.cbase[k] + (int64_t)s * tb.ktab[kTabStride * k + 5] + h;
                        stored[c] = 1;
                        uint32_t F, slot;
                        decode(c, F, slot);
                        bad += (F != (uint32_t)(tb.fbase[k] + s)) + (slot != (uint32_t)tb.gslot[tb.hbase[k] + h]);
                    }
            for (int64_t c = 0; c < tb.ldU; ++c) {
                if (stored[c]) continue;
                uint32_t F, slot;
                decode(c, F, slot);
                bad += !(F == (uint32_t)tb.nF || (slot < tb.ychain.size() && tb.ychain[slot] < 0));
            }
            int64_t pad = 0;
            for (char x : stored) pad += !x;
            char buf[96];
            std::snprintf(buf, sizeof(buf), "U chunk descriptors d=%d vw=%d (%lld columns, %lld padding)", d, vw,
                          (long long)rank, (long long)pad);
            report(buf, bad + ((int64_t)tb.colmap.size() != rank ? 1.0 : 0.0), 0.0);
        }
    return fails ? 1 : 0;
}
