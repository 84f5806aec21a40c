// Host-side planning of the HDF factorization, FP64, no CUDA.
//
// Everything here costs O(p^4) or less (Sec. 3.6) and runs once per build on the host:
// kernel evaluation, Chebyshev coefficients and degree (Sec. 3.3, Remark 3), the radial
// cores r^(k) in a stable basis (Eq. rdef; App. A; Sec. 3.7), the symmetric eigen-solver
// used for the radial-basis factor and the per-degree eigendecompositions (Eq. svd,
// Remark 1), the truncation rule (Sec. 3.4-3.5), and the harmonic index tables (App. B).
#pragma once
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace hdf {

constexpr double kPi = 3.14159265358979323846;

// Kernels of Sec. 4.1 (Gaussian in the exp(-r^2/(2 l^2)) form).
double kernel_value(int kernel, double r, double ell);
double kernel_dz(int kernel, double z);                  // dk/dz, z = r/l
double kernel_dell(int kernel, double r, double ell);    // dk/dl

// Run fn(0..n-1) on up to hardware_concurrency host threads (each index independent).
void parallel_for(int n, const std::function<void(int)>& fn);

int cheb_nodes(int p_max);                               // 4 (p_max + 2)
// a[0..M-1] of f(|r|) on [-1,1], f(r) = k(two_r r; ell) (or dk/dl if dell), DCT-II.
void cheb_coeffs(int kernel, double ell, double two_r, int M, bool dell, double* a);
// tails[p] = sum_{p<i<M}|a_i| + sum_{i>=M/2}|a_i|.
void tail_sums(const double* a, int M, std::vector<double>& tails);
// smallest even p <= p_max with tails[p] <= budget; returns p, sets tail and reached.
int choose_degree(const double* a, int M, double budget, int p_max, double* tail, bool* reached);

// |S^{d-1}| and |H_k| (App. B).
double sphere_area(int d);
int64_t harmonic_count(int k, int d);

// Symmetric eigendecomposition by cyclic Jacobi rotations: A (n x n, row-major, destroyed),
// w (n eigenvalues), V (n x n row-major, column j = eigenvector j).
void sym_eig(int n, double* A, double* w, double* V);
// Gauss-Gegenbauer rule for the weight (1-t^2)^(lam-1/2) on [-1,1], N nodes (Golub-Welsch).
void gauss_gegenbauer(int N, double lam, double* t, double* w);
// The same, memoised per (N, lambda) for lambda a multiple of 1/1024 (half-integers here).
void gauss_gegenbauer_cached(int N, double lam, std::vector<double>& t, std::vector<double>& w);

// C (m x n, row stride ldc) -= A (m x kk, stride lda) B (kk x n, stride ldb), row-major, in
// 4 x 8 register blocks: the rank-kk update of the blocked host factorisations.
void gemm_minus(int64_t m, int64_t n, int64_t kk, const double* A, int64_t lda, const double* B, int64_t ldb,
                double* C, int64_t ldc);

// Radial cores Gamma_k (k = 0..p/2) of r^(k) in the basis rho^(k%2) T_l(8 rho^2 - 1):
// out[k] is a row-major nb_k x nb_k matrix, nb_k = L+1 (k even) or L (k odd).
// threads: spread the degrees over host threads.
void radial_cores(const double* a, int p, int d, std::vector<std::vector<double>>& out, bool threads = true);

// Per-level normalised Gegenbauer recurrences and the chain table of H_k (App. B) used
// by the harmonic kernel.  See hdf_kernels.cuh for the evaluation they feed.
struct HarmonicTables {
    int d = 0, L = 0, tri = 0;           // tri = (L+1)(L+2)/2 entries per level
    // coefA/coefB: (d-2) levels x tri, normalised recurrence
    //   P(0) = A[0], P(1) = A[1] z, P(n) = A[n] z P(n-1) - B[n] q P(n-2)
    std::vector<double> coefA, coefB;
    std::vector<int64_t> count;          // |H_k|, k = 0..L
};
void harmonic_tables(int d, int L, HarmonicTables& t);
// Offset of (mu', n) in a level table: rows mu' = 0..L of length L+1-mu'.
inline int tri_index(int L, int mu, int n) { return mu * (L + 1) - mu * (mu - 1) / 2 + n; }
// Append the chains of H_k (lexicographic in (mu_1..mu_{d-2})), chain_stride(d) int16 entries
// each: (d-2) level-table offsets, the signed mu_{d-2} (trigonometric index), zero padding so
// that one chain is one aligned 8- or 16-byte load.
inline int chain_stride(int d) { return (d - 1 <= 4) ? 4 : 8; }
void append_chains(int k, int d, int L, std::vector<int16_t>& out);

// ---------------------------------------------------------------- build planning
// A1-A2 for one problem: Chebyshev coefficients of kappa(r) = k(2R r; l), the degree from
// the tail budget tol sqrt(mu2)/2, the truncation budget eta tol n sqrt(mu2)/2, the cores.
struct DegreePlan {
    int p = 0, L = 0;
    bool reached = false;
    double tail = 0.0, tail_budget = 0.0, drop_budget = 0.0;
    std::vector<double> a;
    std::vector<std::vector<double>> cores;
};
// with_cores false leaves out.cores empty (the caller runs radial_cores itself, e.g. while the
// device computes the radial moments).
void plan_degree(int kernel, double ell, double R, double mu2, int64_t n, double tol, double eta, int p_max,
                 int d, bool threads, DegreePlan& out, bool with_cores = true);

// Radial-basis Gram sums (the layout plan_factor takes) from the Chebyshev moments
// m_j = sum_i T_j(u_i), j <= 2L+1, using T_l T_l' = (T_{l+l'} + T_{|l-l'|})/2 and
// rho^2 = (u + 1)/8, u T_j = (T_{j+1} + T_{|j-1|})/2.
void gram_from_moments(const std::vector<double>& m, int L, std::vector<double>& gram);

// A3-A4 for one problem from the radial-basis Gram sums (2 x npairs, pairs (l <= l') of the
// even basis in row order; the odd basis uses the leading L x L block of the second half):
// basis factor B = Q R_f (R_f = D^1/2 V^T, directions below 1e-13 nb lambda_max dropped),
// eigendecompositions of G_k = R_f Gamma_k R_f^T and the global truncation.
struct FactorChoice {
    int nb[2] = {0, 0}, m[2] = {0, 0};
    std::vector<double> Rf[2], Qmat[2];
    std::vector<std::vector<double>> Wk;     // per k: m x s_k, columns by decreasing |lambda|
    std::vector<int> sk;
    std::vector<double> S;                   // rank entries in (k, s, h) column order
    int64_t rank = 0, nH = 0;
    double dropped = 0.0;
};
void plan_factor(const std::vector<double>& gram, int L, int d, const std::vector<std::vector<double>>& cores,
                 double drop_budget, bool threads, FactorChoice& out);

// A = U diag(s) V^T of an m x n row-major matrix, q = min(m, n) triples by decreasing s:
// U (m x q), s (q), V (n x q), row-major (one-sided Jacobi).
void svd_jacobi(int m, int n, const double* A, double* U, double* s, double* V);

// A3-A4 for the cross block K(X, Y) (Algorithm 1, general form): basis factors of X and of Y
// from their Gram sums, SVDs of R_X Gamma_k R_Y^T = W_X Sigma W_Y^T and the global truncation
// with sigma in place of |lambda|.  fx gets W_X, fy gets W_Y; both get sigma as S, the same
// s_k, rank and column order.
void plan_factor_cross(const std::vector<double>& gram_x, const std::vector<double>& gram_y, int L, int d,
                       const std::vector<std::vector<double>>& cores, double drop_budget, bool threads,
                       FactorChoice& fx, FactorChoice& fy);

// Host images of the tables the device kernels read (FP64; cast to the bulk type on upload).
// U's columns come in blocks (k, s) of |H_k| harmonics, one after another; only a block of fewer
// than vw (16 bytes) harmonics is padded with zero columns to vw, so that a vw-wide chunk of a
// row meets at most two blocks (two radial factors, two runs of consecutive harmonic slots).
// Per point the harmonic slots are laid out per degree k (slot yoff_k + h, padded per k to vw).
// The padding columns of U carry S = 0 and leave K~ unchanged.
struct DeviceTables {
    int L_used = 0, tri = 0, nF = 0, nH = 0, mmax = 0, nYp = 0;
    int64_t ldU = 0;                         // padded width of U (a multiple of vw)
    std::vector<double> Wt;                  // mmax x nF
    std::vector<uint8_t> colpar, colk, hk;
    std::vector<int16_t> chains;             // nH x (d-1)
    std::vector<int32_t> ychain;             // nYp: chain of each padded Y slot, -1 for padding
    std::vector<int32_t> gslot;              // nH: padded Y slot of each harmonic
    std::vector<uint32_t> qdesc;             // 2 ldU / vw: per chunk (F << 20 | split << 18 | slot, F << 20 | slot)
    std::vector<int64_t> colmap;             // rank: padded column of each true column
    std::vector<double> Spad;                // ldU: S on the padded columns (0 on padding)
    std::vector<double> coefA, coefB;
    std::vector<int> ktab;                   // per k: fbase, s_k, cbase, |H_k|, hbase, columns per (k, s) block
    std::vector<int> fbase, cbase, hbase;
};
// vw: elements per 16 bytes of the bulk type.  False if a limit is exceeded.
bool make_tables(const FactorChoice& fc, int d, int L, int vw, DeviceTables& out, std::string& err);

// Matrix-free layout (d >= 4): U is never stored.  In the chain of a harmonic of degree k,
// (mu_1, ..., mu_{d-2}) with k >= mu_1 = m, the first level factor P_0(m, k - m) is the only
// one that depends on k; the rest -- the levels 1..d-3 and the trigonometric factor -- form
// Z_m^j, a harmonic of degree m in d-1 dimensions (j indexes the tails (mu_2..mu_{d-2}) in the
// order of H_k, the same for every k >= m).  So
//     U[i, (k, s, h = (m, j))] = F_i[k, s] P_0(m, k - m)(x_i) Z_m^j(x_i) = A0F[i, (m, k, s)] Z[i, (m, j)],
// and per point the library keeps the Z row (sum_m |H_m^(d-1)| values) and the A0F row
// (sum_k s_k (k + 1) values) instead of the U row (sum_k s_k |H_k|).
struct FreeTables {
    int L_used = 0;
    int nZ = 0, ldZ = 0;                     // Z columns (blocks padded to 8) and row stride
    int nA = 0, ldA = 0;                     // A0F columns and row stride (a multiple of 4)
    std::vector<int> zoff, zcnt;             // per m <= L_used: first Z column, |H_m^(d-1)|
    std::vector<int> aoff, acnt;             // per m: first A0F column (a multiple of 4), number of (k, s)
                                             // with k >= m (the block is padded to a multiple of 4)
    std::vector<int16_t> zchain;             // nZ x chain_stride(d): level-1..d-3 offsets, trig index
    std::vector<int32_t> a0off;              // nA: level-0 table offset of P_0(m, k - m); -1: padding (zero)
    std::vector<int32_t> afcol;              // nA: F column fbase[k] + s
    std::vector<int64_t> wcol;               // nA: padded U column of (k, s, h = first tail of m)
    // d = 4, 5: the product form of the tails, Z[i, t] = P_1[zpair_t >> 16] G[zpair_t & 0xFFFF] with
    // P_1 the level-1 table and G per point the product of the deeper factors: d = 4: G = the
    // trigonometric factors (slot L + mu_2); d = 5: G[mu_2^2 + mu_2 + mu_3] = P_2(mu_2 -> |mu_3|)
    // trig(mu_3), gmap = (level-2 offset << 16) | trig slot.  G[ng] = 0 serves the padding columns.
    // Empty for d >= 6.
    std::vector<int32_t> zpair, gmap;
    int ng = 0;
};
// From the tables of make_tables (its cbase, dimp, fbase); false (with err) if d < 4.
bool make_free_tables(const FactorChoice& fc, int d, int L, const DeviceTables& tb, FreeTables& out,
                      std::string& err);
constexpr int kTabStride = 6;               // ints per k in DeviceTables::ktab

}  // namespace hdf
