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

// Radial cores Gamma_k (k = 0..p/2) of r^(k) in the basis rho^(k%2) T_l(8 rho^2 - 1):
// out[k] is a row-major nb_k x nb_k matrix, nb_k = L+1 (k even) or L (k odd).
void radial_cores(const double* a, int p, int d, std::vector<std::vector<double>>& out);

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
// Append the chains of H_k (lexicographic in (mu_1..mu_{d-2})) as (d-1) int16 entries each:
// (d-2) level-table offsets, then the signed mu_{d-2} (trigonometric index).
void append_chains(int k, int d, int L, std::vector<int16_t>& out);

}  // namespace hdf
