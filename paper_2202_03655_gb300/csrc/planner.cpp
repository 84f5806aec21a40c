// Host-side planning of the HDF factorization (FP64).  See planner.h.
#include "planner.h"
#include <map>

#include <condition_variable>
#include <mutex>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <functional>
#include <thread>

namespace hdf {

// ------------------------------------------------------------------------- kernels
double kernel_value(int kernel, double r, double ell) {
    const double z = std::fabs(r) / ell;
    switch (kernel) {
        case 0: return std::exp(-0.5 * z * z);
        case 1: return 1.0 / (1.0 + z * z);
        case 2: { const double s = std::sqrt(3.0) * z; return (1.0 + s) * std::exp(-s); }
        case 3: { const double s = std::sqrt(5.0) * z; return (1.0 + s + s * s / 3.0) * std::exp(-s); }
    }
    return NAN;
}

double kernel_dz(int kernel, double z) {
    switch (kernel) {
        case 0: return -z * std::exp(-0.5 * z * z);
        case 1: { const double q = 1.0 + z * z; return -2.0 * z / (q * q); }
        case 2: return -3.0 * z * std::exp(-std::sqrt(3.0) * z);
        case 3: { const double s = std::sqrt(5.0) * z; return -(5.0 / 3.0) * z * (1.0 + s) * std::exp(-s); }
    }
    return NAN;
}

double kernel_dell(int kernel, double r, double ell) {
    const double z = std::fabs(r) / ell;
    return kernel_dz(kernel, z) * (-z / ell);
}

// Persistent worker pool: the workers are created once and sleep between jobs, so a planning
// step pays no thread start-up.  One job at a time; a concurrent or nested call runs serially.
namespace {
struct Pool {
    std::mutex m;
    std::condition_variable go, done;
    std::mutex busy;
    const std::function<void(int)>* job = nullptr;
    int n = 0, active = 0, workers = 0;
    uint64_t gen = 0;
    std::atomic<int> next{0};
    Pool() {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        workers = std::min(hw, 32) - 1;
        for (int t = 0; t < workers; ++t) std::thread([this]() { loop(); }).detach();
    }
    void loop() {
        uint64_t seen = 0;
        for (;;) {
            std::unique_lock<std::mutex> lk(m);
            go.wait(lk, [&]() { return gen != seen; });
            seen = gen;
            const std::function<void(int)>* f = job;
            const int N = n;
            lk.unlock();
            for (int i = next.fetch_add(1); i < N; i = next.fetch_add(1)) (*f)(i);
            lk.lock();
            if (--active == 0) done.notify_all();
        }
    }
};
Pool& pool() {
    static Pool* p = new Pool();     // never destroyed: detached workers outlive static destructors
    return *p;
}
}  // namespace

void parallel_for(int n, const std::function<void(int)>& fn) {
    Pool& P = pool();
    if (n <= 1 || P.workers == 0 || !P.busy.try_lock()) {
        for (int i = 0; i < n; ++i) fn(i);
        return;
    }
    {
        std::lock_guard<std::mutex> lk(P.m);
        P.job = &fn;
        P.n = n;
        P.next.store(0);
        P.active = P.workers;
        ++P.gen;
    }
    P.go.notify_all();
    for (int i = P.next.fetch_add(1); i < n; i = P.next.fetch_add(1)) fn(i);
    {
        std::unique_lock<std::mutex> lk(P.m);
        P.done.wait(lk, [&]() { return P.active == 0; });
    }
    P.busy.unlock();
}

// ----------------------------------------------------------------------- Chebyshev
int cheb_nodes(int p_max) { return 4 * (p_max + 2); }

// cos(pi q / (2M)) for q < 4M, built once per node count (the DCT below reads it with exact
// integer angle reduction instead of calling cos M^2/2 times per kernel).
static const std::vector<double>& dct_cos_table(int M) {
    static std::mutex mu;
    static std::map<int, std::vector<double>> tabs;
    std::lock_guard<std::mutex> lk(mu);
    std::vector<double>& t = tabs[M];
    if (t.empty()) {
        t.resize((size_t)4 * M);
        for (int q = 0; q < 4 * M; ++q) t[q] = std::cos(kPi * q / (2.0 * M));
    }
    return t;
}

void cheb_coeffs(int kernel, double ell, double two_r, int M, bool dell, double* a) {
    // a_i = (2/M) sum_j cos(i th_j) v_j, th_j = pi (j + 1/2) / M (first-kind nodes), halved at i = 0;
    // v_j depends on |cos th_j| only, so v_{M-1-j} = v_j, and for even i the two halves of the
    // sum are equal; odd a_i are zero exactly.
    const std::vector<double>& tab = dct_cos_table(M);
    const int M4 = 4 * M;
    std::vector<double> v(M);
    for (int j = 0; j < M; ++j) {
        const double r = std::fabs(tab[(2 * j + 1) % M4]);
        v[j] = dell ? kernel_dell(kernel, two_r * r, ell) : kernel_value(kernel, two_r * r, ell);
    }
    const int half = M / 2;
    for (int i = 0; i < M; ++i) {
        if (i & 1) { a[i] = 0.0; continue; }
        double s = 0.0;
        for (int j = 0; j < half; ++j) s += tab[((int64_t)i * (2 * j + 1)) % M4] * v[j];
        s *= 2.0;
        if (M & 1) s += tab[((int64_t)i * M) % M4] * v[half];
        a[i] = (2.0 / M) * s;
    }
    a[0] *= 0.5;
}

void tail_sums(const double* a, int M, std::vector<double>& tails) {
    tails.assign(M, 0.0);
    double guard = 0.0;
    for (int i = M / 2; i < M; ++i) guard += std::fabs(a[i]);
    double acc = 0.0;                       // sum_{i > p}
    for (int p = M - 1; p >= 0; --p) {
        tails[p] = acc + guard;
        acc += std::fabs(a[p]);
    }
}

int choose_degree(const double* a, int M, double budget, int p_max, double* tail, bool* reached) {
    std::vector<double> tails;
    tail_sums(a, M, tails);
    p_max -= p_max % 2;
    for (int p = 0; p <= p_max && p < M; p += 2) {
        if (tails[p] <= budget) { *tail = tails[p]; *reached = true; return p; }
    }
    *tail = tails[std::min(p_max, M - 1)];
    *reached = false;
    return p_max;
}

// ------------------------------------------------------------------ sphere, counts
double sphere_area(int d) { return 2.0 * std::pow(kPi, 0.5 * d) / std::tgamma(0.5 * d); }

static int64_t binom(int64_t n, int64_t k) {
    if (k < 0 || k > n) return 0;
    int64_t r = 1;
    for (int64_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

int64_t harmonic_count(int k, int d) { return binom(k + d - 1, k) - binom(k + d - 3, k - 2); }

// -------------------------------------------------------------- symmetric eigen
// Symmetric eigendecomposition A = V diag(w) V^T (row-major, V's columns the eigenvectors, in
// no particular order; A is overwritten).  Householder reduction to tridiagonal form, then the
// implicit symmetric QR iteration with Wilkinson shifts and deflation, rotations accumulated
// into V (Golub and Van Loan, Matrix Computations, Alg. 8.3.1 and 8.3.3).
void sym_eig(int n, double* A, double* w, double* V) {
    for (int i = 0; i < n * n; ++i) V[i] = 0.0;
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    if (n == 1) { w[0] = A[0]; return; }
    std::vector<double> v(n), pv(n), e(n, 0.0);
    // Householder: for column k, H = I - beta v v^T maps A[k+1:, k] to (alpha, 0, ..., 0)
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        double xn = 0.0;
        for (int i = 0; i < m; ++i) { v[i] = A[(k + 1 + i) * n + k]; xn += v[i] * v[i]; }
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        const double alpha = v[0] > 0.0 ? -xn : xn;
        v[0] -= alpha;
        double vn2 = 0.0;
        for (int i = 0; i < m; ++i) vn2 += v[i] * v[i];
        if (vn2 == 0.0) continue;
        const double beta = 2.0 / vn2;
        // p = beta A_sub v, K = (beta / 2) v^T p, q = p - K v, A_sub -= v q^T + q v^T
        double K = 0.0;
        for (int i = 0; i < m; ++i) {
            double t = 0.0;
            const double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
            for (int j = 0; j < m; ++j) t += row[j] * v[j];
            pv[i] = beta * t;
            K += v[i] * pv[i];
        }
        K *= 0.5 * beta;
        for (int i = 0; i < m; ++i) pv[i] -= K * v[i];
        for (int i = 0; i < m; ++i) {
            double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
            for (int j = 0; j < m; ++j) row[j] -= v[i] * pv[j] + pv[i] * v[j];
        }
        A[(k + 1) * n + k] = A[k * n + k + 1] = alpha;
        for (int i = 1; i < m; ++i) A[(k + 1 + i) * n + k] = A[k * n + k + 1 + i] = 0.0;
        // V <- V H on columns k+1 .. n-1
        for (int r = 0; r < n; ++r) {
            double* row = V + (size_t)r * n + (k + 1);
            double t = 0.0;
            for (int j = 0; j < m; ++j) t += row[j] * v[j];
            t *= beta;
            for (int j = 0; j < m; ++j) row[j] -= t * v[j];
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[i * n + i + 1];
    // implicit QR on the tridiagonal (w, e); rotation G in plane (k, k+1) with G_kk = G_k+1,k+1 = c,
    // G_k,k+1 = s, G_k+1,k = -s, T <- G^T T G, V <- V G.  The rotations are accumulated into
    // Vt = V^T, where columns k and k+1 of V are contiguous rows (the same arithmetic per entry).
    std::vector<double> Vt((size_t)n * n);
    for (int r2 = 0; r2 < n; ++r2)
        for (int c2 = 0; c2 < n; ++c2) Vt[(size_t)c2 * n + r2] = V[(size_t)r2 * n + c2];
    const double eps = 2.220446049250313e-16;
    int q = n - 1, iters = 0;
    while (q > 0 && iters < 64 * n) {
        for (int i = 0; i < q; ++i)
            if (std::fabs(e[i]) <= eps * (std::fabs(w[i]) + std::fabs(w[i + 1]))) e[i] = 0.0;
        while (q > 0 && e[q - 1] == 0.0) --q;
        if (q == 0) break;
        int p = q - 1;
        while (p > 0 && e[p - 1] != 0.0) --p;
        ++iters;
        // Wilkinson shift from the trailing 2 x 2 block
        const double dl = 0.5 * (w[q - 1] - w[q]), eq = e[q - 1];
        const double den = dl + (dl >= 0.0 ? 1.0 : -1.0) * std::hypot(dl, eq);
        const double mu = w[q] - eq * eq / den;
        double x = w[p] - mu, z = e[p];
        for (int k = p; k < q; ++k) {
            const double r = std::hypot(x, z);
            const double c = r == 0.0 ? 1.0 : x / r, s = r == 0.0 ? 0.0 : -z / r;
            if (k > p) e[k - 1] = r;
            const double a = w[k], f = e[k], g = w[k + 1];
            w[k] = c * c * a - 2.0 * c * s * f + s * s * g;
            w[k + 1] = s * s * a + 2.0 * c * s * f + c * c * g;
            e[k] = c * s * (a - g) + (c * c - s * s) * f;
            if (k + 1 < q) {
                const double h = e[k + 1];
                z = -s * h;                   // bulge T[k, k+2]
                e[k + 1] = c * h;
                x = e[k];
            }
            double* ck = Vt.data() + (size_t)k * n;
            double* ck1 = ck + n;
            for (int r2 = 0; r2 < n; ++r2) {
                const double vk = ck[r2], vk1 = ck1[r2];
                ck[r2] = c * vk - s * vk1;
                ck1[r2] = s * vk + c * vk1;
            }
        }
    }
    for (int r2 = 0; r2 < n; ++r2)
        for (int c2 = 0; c2 < n; ++c2) V[(size_t)r2 * n + c2] = Vt[(size_t)c2 * n + r2];
}

void gauss_gegenbauer(int N, double lam, double* t, double* w) {
    // Jacobi matrix of the monic Gegenbauer recurrence p_{j+1} = t p_j - b_j p_{j-1},
    // b_j = j (j + 2 lam - 1) / (4 (j + lam)(j + lam - 1)); nodes = eigenvalues,
    // weights = mu0 * (first eigenvector component)^2 (Golub-Welsch).
    std::vector<double> J(N * N, 0.0), V(N * N), ev(N);
    for (int j = 1; j < N; ++j) {
        const double b = j * (j + 2.0 * lam - 1.0) / (4.0 * (j + lam) * (j + lam - 1.0));
        J[(j - 1) * N + j] = J[j * N + j - 1] = std::sqrt(b);
    }
    sym_eig(N, J.data(), ev.data(), V.data());
    const double mu0 = std::exp(0.5 * std::log(kPi) + std::lgamma(lam + 0.5) - std::lgamma(lam + 1.0));
    std::vector<int> idx(N);
    for (int i = 0; i < N; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    for (int i = 0; i < N; ++i) {
        t[i] = ev[idx[i]];
        w[i] = mu0 * V[idx[i]] * V[idx[i]];     // row 0, column idx[i]
    }
}

// Gauss-Gegenbauer rules are shared by every problem of the same dimension: computed once per
// (N, lambda) and reused.
void gauss_gegenbauer_cached(int N, double lam, std::vector<double>& t, std::vector<double>& w) {
    static std::mutex mu;
    static std::map<std::pair<int, int64_t>, std::pair<std::vector<double>, std::vector<double>>> cache;
    const std::pair<int, int64_t> key(N, (int64_t)std::llround(lam * 1024.0));
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end() && it->first.second * (1.0 / 1024.0) == lam) {
            t = it->second.first;
            w = it->second.second;
            return;
        }
    }
    t.assign(N, 0.0);
    w.assign(N, 0.0);
    gauss_gegenbauer(N, lam, t.data(), w.data());
    if ((double)key.second * (1.0 / 1024.0) == lam) {
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = std::make_pair(t, w);
    }
}

// ------------------------------------------------------------------- radial cores
// F(s) = sum_q f_q T_q(2s - 1), f_q = a_{2q} (T_{2q}(r) = T_q(2 r^2 - 1)).  By Rodrigues'
// formula and k integrations by parts, the Gegenbauer coefficient of F(a^2+b^2-2abt) times
// the addition-theorem normaliser Z_k is
//   r^(k)(a,b) = (-1)^k |S^{d-1}| Gamma(alpha+1) / (sqrt(pi) Gamma(k+alpha+1/2))
//                (ab)^k int_{-1}^{1} F^(k)(a^2+b^2-2abt) (1-t^2)^(k+alpha-1/2) dt,
// the integrand being a polynomial of degree L-k in t: Gauss-Gegenbauer with parameter
// k+alpha and (L-k)/2+2 nodes is exact.  r^(k) is then interpolated at first-kind
// Chebyshev nodes in u = 8 rho^2 - 1 and converted to Chebyshev coefficients (DCT).
static void cheb_derivative(const std::vector<double>& c, std::vector<double>& dc, double scale) {
    const int N = (int)c.size() - 1;        // degree
    if (N <= 0) { dc.assign(1, 0.0); return; }
    std::vector<double> e(N + 2, 0.0);
    for (int q = N; q >= 1; --q) e[q - 1] = e[q + 1] + 2.0 * q * c[q];
    e[0] *= 0.5;
    dc.assign(N, 0.0);
    for (int q = 0; q < N; ++q) dc[q] = scale * e[q];
}

void radial_cores(const double* a, int p, int d, std::vector<std::vector<double>>& out, bool threads) {
    const int L = p / 2;
    const double alpha = 0.5 * d - 1.0;
    const double area = sphere_area(d);
    std::vector<std::vector<double>> deriv(L + 1);   // Chebyshev coefficients of F^(k)
    deriv[0].resize(L + 1);
    for (int q = 0; q <= L; ++q) deriv[0][q] = a[2 * q];
    for (int k = 1; k <= L; ++k) cheb_derivative(deriv[k - 1], deriv[k], 2.0);   // d/ds = 2 d/du
    out.assign(L + 1, std::vector<double>());
    std::vector<double> Dmat[2];                   // interpolation-to-coefficient maps, nb = L+1, L
    for (int par = 0; par < 2; ++par) {
        const int nb = par == 0 ? L + 1 : L;
        Dmat[par].resize((size_t)nb * nb);
        for (int l = 0; l < nb; ++l)
            for (int j = 0; j < nb; ++j)
                Dmat[par][(size_t)l * nb + j] = (l == 0 ? 1.0 : 2.0) / nb * std::cos(l * kPi * (j + 0.5) / nb);
    }
    auto one = [&](int k) {
        const std::vector<double>& Fk = deriv[k];
        const int nb = (k % 2 == 0) ? L + 1 : L;
        if (nb == 0) return;
        const int Nq = (L - k) / 2 + 2;
        std::vector<double> tq, wq;
        gauss_gegenbauer_cached(Nq, k + alpha, tq, wq);
        const double lpref = std::log(area) + std::lgamma(alpha + 1.0) - 0.5 * std::log(kPi)
                             - std::lgamma(k + alpha + 0.5);
        const double pref = ((k & 1) ? -1.0 : 1.0) * std::exp(lpref);
        std::vector<double> u(nb), rho(nb);
        for (int j = 0; j < nb; ++j) {
            u[j] = std::cos(kPi * (j + 0.5) / nb);
            rho[j] = std::sqrt((u[j] + 1.0) / 8.0);
        }
        std::vector<double> Vv(nb * nb), rpow(nb);
        for (int i = 0; i < nb; ++i) rpow[i] = std::pow(rho[i], (double)(k - (k & 1)));   // (ab)^k' = a^k' b^k'
        // Clenshaw at the Nq nodes of every pair (i, j <= i) of row i side by side: one long loop
        // of independent recurrences (element e = j Nq + q), then the per-pair quadrature sums
        std::vector<double> uqv((size_t)nb * Nq), b1v((size_t)nb * Nq), b2v((size_t)nb * Nq);
        double* uq = uqv.data();
        double* b1 = b1v.data();
        double* b2 = b2v.data();
        for (int i = 0; i < nb; ++i) {
            const int ne = (i + 1) * Nq;
            for (int j = 0; j <= i; ++j) {
                const double ab = rho[i] * rho[j];
                const double s0 = rho[i] * rho[i] + rho[j] * rho[j];
                for (int q = 0; q < Nq; ++q) uq[j * Nq + q] = 2.0 * (s0 - 2.0 * ab * tq[q]) - 1.0;
            }
            for (int e = 0; e < ne; ++e) { b1[e] = 0.0; b2[e] = 0.0; }
            for (int m = (int)Fk.size() - 1; m >= 1; --m) {
                const double cm = Fk[m];
                for (int e = 0; e < ne; ++e) {
                    const double b0 = 2.0 * uq[e] * b1[e] - b2[e] + cm;
                    b2[e] = b1[e];
                    b1[e] = b0;
                }
            }
            for (int j = 0; j <= i; ++j) {
                double integ = 0.0;
                for (int q = 0; q < Nq; ++q) {
                    const int e = j * Nq + q;
                    integ += wq[q] * (uq[e] * b1[e] - b2[e] + Fk[0]);
                }
                const double v = pref * rpow[i] * rpow[j] * integ;
                Vv[i * nb + j] = Vv[j * nb + i] = v;
            }
        }
        // Gamma = D V D^T with D[l][j] = (2 - delta_l0)/nb cos(l pi (j+1/2)/nb)
        const std::vector<double>& D = Dmat[k % 2];
        std::vector<double> T(nb * nb, 0.0), G(nb * nb, 0.0);
        for (int l = 0; l < nb; ++l)
            for (int j = 0; j < nb; ++j) {
                double s = 0.0;
                for (int m = 0; m < nb; ++m) s += D[l * nb + m] * Vv[m * nb + j];
                T[l * nb + j] = s;
            }
        for (int l = 0; l < nb; ++l)
            for (int m = 0; m < nb; ++m) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j) s += T[l * nb + j] * D[m * nb + j];
                G[l * nb + m] = s;
            }
        for (int l = 0; l < nb; ++l)
            for (int m = 0; m < l; ++m) G[l * nb + m] = G[m * nb + l] = 0.5 * (G[l * nb + m] + G[m * nb + l]);
        out[k].swap(G);
    };
    if (threads) {
        parallel_for(L + 1, one);
    } else {
        for (int k = 0; k <= L; ++k) one(k);
    }
}

// --------------------------------------------------------------- harmonic tables
void harmonic_tables(int d, int L, HarmonicTables& t) {
    t.d = d;
    t.L = L;
    t.tri = (L + 1) * (L + 2) / 2;
    const int levels = d - 2;
    t.coefA.assign((size_t)levels * t.tri, 0.0);
    t.coefB.assign((size_t)levels * t.tri, 0.0);
    for (int j = 0; j < levels; ++j) {
        const double alpha_j = 0.5 * (d - j - 2);
        for (int mu = 0; mu <= L; ++mu) {
            const double lam = mu + alpha_j;
            auto log_h = [&](int n) {       // log of the Gegenbauer norm h_n^lam
                return std::log(kPi) + (1.0 - 2.0 * lam) * std::log(2.0) + std::lgamma(n + 2.0 * lam)
                       - std::lgamma(n + 1.0) - std::log(n + lam) - 2.0 * std::lgamma(lam);
            };
            double* A = &t.coefA[(size_t)j * t.tri + tri_index(L, mu, 0)];
            double* B = &t.coefB[(size_t)j * t.tri + tri_index(L, mu, 0)];
            const int nmax = L - mu;
            A[0] = std::exp(-0.5 * log_h(0));
            if (nmax >= 1) A[1] = 2.0 * lam * std::exp(-0.5 * log_h(1));
            for (int n = 2; n <= nmax; ++n) {
                const double r1 = std::exp(0.5 * (log_h(n - 1) - log_h(n)));   // s_n / s_{n-1}
                const double r2 = std::exp(0.5 * (log_h(n - 2) - log_h(n)));   // s_n / s_{n-2}
                A[n] = 2.0 * (n + lam - 1.0) / n * r1;
                B[n] = (n + 2.0 * lam - 2.0) / n * r2;
            }
        }
    }
    t.count.resize(L + 1);
    for (int k = 0; k <= L; ++k) t.count[k] = harmonic_count(k, d);
}

void append_chains(int k, int d, int L, std::vector<int16_t>& out) {
    const int levels = d - 2;
    const int stride = chain_stride(d);
    std::vector<int> mu(d - 1);              // mu[0] = k, mu[1..d-2]
    mu[0] = k;
    std::function<void(int)> rec = [&](int pos) {
        if (pos == d - 2) {                   // last entry may be negative
            for (int m = -mu[pos - 1]; m <= mu[pos - 1]; ++m) {
                mu[pos] = m;
                for (int j = 0; j < levels; ++j) {
                    const int mnext = std::abs(mu[j + 1]);
                    out.push_back((int16_t)tri_index(L, mnext, mu[j] - mnext));
                }
                out.push_back((int16_t)m);
                for (int q = levels + 1; q < stride; ++q) out.push_back((int16_t)0);
            }
            return;
        }
        for (int m = 0; m <= mu[pos - 1]; ++m) {
            mu[pos] = m;
            rec(pos + 1);
        }
    };
    rec(1);
}

}  // namespace hdf

namespace hdf {

void plan_degree(int kernel, double ell, double R, double mu2, int64_t n, double tol, double eta, int p_max,
                 int d, bool threads, DegreePlan& out, bool with_cores) {
    const int M = cheb_nodes(p_max);
    out.a.assign(M, 0.0);
    cheb_coeffs(kernel, ell, 2.0 * R, M, false, out.a.data());
    out.tail_budget = 0.5 * tol * std::sqrt(mu2);
    out.drop_budget = 0.5 * eta * tol * (double)n * std::sqrt(mu2);
    out.p = choose_degree(out.a.data(), M, out.tail_budget, p_max, &out.tail, &out.reached);
    out.L = out.p / 2;
    if (with_cores) radial_cores(out.a.data(), out.p, d, out.cores, threads);
}

void gram_from_moments(const std::vector<double>& m, int L, std::vector<double>& gram) {
    const int nb0 = L + 1;
    const int npairs = nb0 * (nb0 + 1) / 2;
    gram.assign(2 * (size_t)npairs, 0.0);
    auto M = [&](int j) { return m[std::abs(j)]; };
    auto prodsum = [&](int l, int lp) { return 0.5 * (M(l + lp) + M(l - lp)); };          // sum T_l T_l'
    auto uprod = [&](int j) { return 0.5 * (M(j + 1) + M(j - 1)); };                       // sum u T_j
    int q = 0;
    for (int l = 0; l < nb0; ++l)
        for (int lp = l; lp < nb0; ++lp, ++q) {
            gram[q] = prodsum(l, lp);
            // sum rho^2 T_l T_l' = (1/8) sum (u + 1) T_l T_l'
            const double su = 0.5 * (uprod(l + lp) + uprod(l - lp));
            gram[(size_t)npairs + q] = 0.125 * (su + prodsum(l, lp));
        }
}

// C (m x n, row stride ldc) -= A (m x kk, stride lda) * B (kk x n, stride ldb), all row-major,
// in 4 x 8 register blocks (the sums over kk stay in registers; the fixed-size inner loops are
// left to the compiler's vectoriser).
void gemm_minus(int64_t m, int64_t n, int64_t kk, const double* A, int64_t lda, const double* B, int64_t ldb,
                       double* C, int64_t ldc) {
    int64_t i0 = 0;
    for (; i0 + 4 <= m; i0 += 4) {
        int64_t j0 = 0;
        for (; j0 + 8 <= n; j0 += 8) {
            double acc[4][8] = {};
            for (int64_t q = 0; q < kk; ++q) {
                const double* b = B + q * ldb + j0;
#pragma GCC unroll 4
                for (int r = 0; r < 4; ++r) {
                    const double a = A[(i0 + r) * lda + q];
#pragma GCC unroll 8
                    for (int c = 0; c < 8; ++c) acc[r][c] += a * b[c];
                }
            }
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 8; ++c) C[(i0 + r) * ldc + j0 + c] -= acc[r][c];
        }
        for (; j0 < n; ++j0)
            for (int r = 0; r < 4; ++r) {
                double s = 0.0;
                for (int64_t q = 0; q < kk; ++q) s += A[(i0 + r) * lda + q] * B[q * ldb + j0];
                C[(i0 + r) * ldc + j0] -= s;
            }
    }
    for (; i0 < m; ++i0)
        for (int64_t j0 = 0; j0 < n; ++j0) {
            double s = 0.0;
            for (int64_t q = 0; q < kk; ++q) s += A[i0 * lda + q] * B[q * ldb + j0];
            C[i0 * ldc + j0] -= s;
        }
}

// Radial-basis factor of one parity from its Gram sums: B = Q R_f with R_f = D^1/2 V^T and
// Q = B Qmat, Qmat = V D^-1/2, over the eigen-directions above 1e-13 nb lambda_max.
static void basis_factor(const std::vector<double>& gram, int L, int par, FactorChoice& out) {
    const int nb0 = L + 1, nb = out.nb[par];
    const int npairs = nb0 * (nb0 + 1) / 2;
    out.m[par] = 0;
    out.Rf[par].clear();
    out.Qmat[par].clear();
    if (nb == 0) return;
    std::vector<double> Gm((size_t)nb * nb), w(nb), V((size_t)nb * nb);
    int q = 0;
    for (int l = 0; l < nb0; ++l)
        for (int lp = l; lp < nb0; ++lp, ++q)
            if (l < nb && lp < nb) Gm[(size_t)l * nb + lp] = Gm[(size_t)lp * nb + l] = gram[(size_t)par * npairs + q];
    sym_eig(nb, Gm.data(), w.data(), V.data());
    double wmax = 0.0;
    for (int l = 0; l < nb; ++l) wmax = std::max(wmax, w[l]);
    const double floor_ = wmax * 1e-13 * nb;
    std::vector<int> keep;
    for (int l = 0; l < nb; ++l) if (w[l] > floor_) keep.push_back(l);
    const int mk = (int)keep.size();
    out.m[par] = mk;
    out.Rf[par].assign((size_t)mk * nb, 0.0);
    out.Qmat[par].assign((size_t)nb * mk, 0.0);
    for (int o = 0; o < mk; ++o) {
        const double sq = std::sqrt(w[keep[o]]);
        for (int l = 0; l < nb; ++l) {
            out.Rf[par][(size_t)o * nb + l] = sq * V[(size_t)l * nb + keep[o]];
            out.Qmat[par][(size_t)l * mk + o] = V[(size_t)l * nb + keep[o]] / sq;
        }
    }
}

// T = Ra Gamma_k Rb^T (ma x mb) for basis factors Ra (ma x nb) and Rb (mb x nb).
static void sandwich(const std::vector<double>& Ra, int ma, const std::vector<double>& Gk, int nb,
                     const std::vector<double>& Rb, int mb, std::vector<double>& T) {
    std::vector<double> T1((size_t)ma * nb, 0.0);
    for (int o = 0; o < ma; ++o)
        for (int l = 0; l < nb; ++l) {
            double s = 0.0;
            for (int t = 0; t < nb; ++t) s += Ra[(size_t)o * nb + t] * Gk[(size_t)t * nb + l];
            T1[(size_t)o * nb + l] = s;
        }
    T.assign((size_t)ma * mb, 0.0);
    for (int o = 0; o < ma; ++o)
        for (int o2 = 0; o2 < mb; ++o2) {
            double s = 0.0;
            for (int l = 0; l < nb; ++l) s += T1[(size_t)o * nb + l] * Rb[(size_t)o2 * nb + l];
            T[(size_t)o * mb + o2] = s;
        }
}

// Global truncation (Sec. 3.4-3.5): item j of block k costs |lam[k][j]| |H_k| / |S^{d-1}|;
// items are dropped in increasing (cost, k, j) order while the summed cost stays within the
// budget.  Returns per k the kept indices by decreasing |lam| (ties by index) and the cost.
static double select_kept(const std::vector<std::vector<double>>& lam, int d, double budget,
                          std::vector<std::vector<int>>& kept) {
    const int L = (int)lam.size() - 1;
    const double area = sphere_area(d);
    struct Item { double cost; int k, j; };
    std::vector<Item> items;
    for (int k = 0; k <= L; ++k) {
        const double hk = (double)harmonic_count(k, d);
        for (int j = 0; j < (int)lam[k].size(); ++j) items.push_back({std::fabs(lam[k][j]) * hk / area, k, j});
    }
    std::sort(items.begin(), items.end(), [](const Item& A, const Item& B) {
        if (A.cost != B.cost) return A.cost < B.cost;
        if (A.k != B.k) return A.k < B.k;
        return A.j < B.j;
    });
    std::vector<std::vector<char>> dropped(L + 1);
    for (int k = 0; k <= L; ++k) dropped[k].assign(lam[k].size(), 0);
    double acc = 0.0;
    for (const Item& it : items) {
        if (acc + it.cost > budget) break;
        acc += it.cost;
        dropped[it.k][it.j] = 1;
    }
    kept.assign(L + 1, std::vector<int>());
    for (int k = 0; k <= L; ++k) {
        std::vector<int>& idx = kept[k];
        for (int j = 0; j < (int)lam[k].size(); ++j) if (!dropped[k][j]) idx.push_back(j);
        std::sort(idx.begin(), idx.end(), [&](int A, int B) {
            const double fa = std::fabs(lam[k][A]), fb = std::fabs(lam[k][B]);
            if (fa != fb) return fa > fb;
            return A < B;
        });
    }
    return acc;
}

// Kept columns of the per-k vectors (vec[k]: m x q row-major) into out.Wk, out.sk, out.S (lam
// per column, repeated over the |H_k| harmonics), out.rank and out.nH.
static void fill_choice(const std::vector<std::vector<double>>& lam, const std::vector<std::vector<double>>& vec,
                        const std::vector<int>& qk, const std::vector<std::vector<int>>& kept, int d, int L,
                        FactorChoice& out) {
    out.sk.assign(L + 1, 0);
    out.Wk.assign(L + 1, std::vector<double>());
    out.S.clear();
    out.rank = 0;
    out.nH = 0;
    for (int k = 0; k <= L; ++k) {
        const int64_t hcount = harmonic_count(k, d);
        const std::vector<int>& idx = kept[k];
        out.sk[k] = (int)idx.size();
        if (out.sk[k] == 0) continue;
        const int mk = out.m[k % 2], q = qk[k];
        out.Wk[k].assign((size_t)mk * out.sk[k], 0.0);
        for (int s = 0; s < out.sk[k]; ++s)
            for (int o = 0; o < mk; ++o) out.Wk[k][(size_t)o * out.sk[k] + s] = vec[k][(size_t)o * q + idx[s]];
        out.rank += hcount * out.sk[k];
        out.nH += hcount;
        for (int s = 0; s < out.sk[k]; ++s)
            for (int64_t h = 0; h < hcount; ++h) out.S.push_back(lam[k][idx[s]]);
    }
}

void plan_factor(const std::vector<double>& gram, int L, int d, const std::vector<std::vector<double>>& cores,
                 double drop_budget, bool threads, FactorChoice& out) {
    out.nb[0] = L + 1;
    out.nb[1] = L;
    for (int par = 0; par < 2; ++par) basis_factor(gram, L, par, out);
    std::vector<std::vector<double>> lam(L + 1), vec(L + 1);
    std::vector<int> qk(L + 1, 0);
    auto one = [&](int k) {
        const int par = k % 2, nb = out.nb[par], mk = out.m[par];
        if (mk == 0 || nb == 0) return;
        std::vector<double> Gm;
        sandwich(out.Rf[par], mk, cores[k], nb, out.Rf[par], mk, Gm);
        for (int o = 0; o < mk; ++o)                       // exact symmetry: mirror the lower triangle
            for (int o2 = 0; o2 < o; ++o2) Gm[(size_t)o2 * mk + o] = Gm[(size_t)o * mk + o2];
        lam[k].resize(mk);
        vec[k].resize((size_t)mk * mk);
        qk[k] = mk;
        sym_eig(mk, Gm.data(), lam[k].data(), vec[k].data());
    };
    if (threads) {
        parallel_for(L + 1, one);
    } else {
        for (int k = 0; k <= L; ++k) one(k);
    }
    std::vector<std::vector<int>> kept;
    out.dropped = select_kept(lam, d, drop_budget, kept);
    fill_choice(lam, vec, qk, kept, d, L, out);
}

// ------------------------------------------------------------------ SVD (one-sided Jacobi)
// A = U diag(s) V^T for an m x n row-major A, q = min(m, n) triples by decreasing s: U (m x q),
// V (n x q), row-major.  Hestenes' one-sided Jacobi method: pairs of columns of W = A are
// rotated until all are mutually orthogonal to working precision; then s_j = |w_j|,
// U[:, j] = w_j / s_j, and V is the product of the rotations (Golub and Van Loan, Matrix
// Computations, Sec. 8.6.3).  A wide A is handled through its transpose.  Columns with
// s_j = 0 leave U[:, j] = 0.
void svd_jacobi(int m, int n, const double* A, double* U, double* s, double* V) {
    if (m < n) {                       // A^T = V S U^T
        std::vector<double> At((size_t)n * m);
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) At[(size_t)j * m + i] = A[(size_t)i * n + j];
        svd_jacobi(n, m, At.data(), V, s, U);
        return;
    }
    // column-major working copies: W (m x n), Vw (n x n)
    std::vector<double> W((size_t)m * n), Vw((size_t)n * n, 0.0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) W[(size_t)j * m + i] = A[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) Vw[(size_t)j * n + j] = 1.0;
    const double eps = 2.220446049250313e-16;
    for (int sweep = 0; sweep < 80; ++sweep) {
        double off = 0.0;
        for (int p = 0; p + 1 < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double* wp = &W[(size_t)p * m];
                double* wq = &W[(size_t)q * m];
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = 0; i < m; ++i) { al += wp[i] * wp[i]; be += wq[i] * wq[i]; ga += wp[i] * wq[i]; }
                if (al == 0.0 || be == 0.0) continue;
                const double rel = std::fabs(ga) / std::sqrt(al * be);
                if (!(rel > eps * m)) continue;
                off = std::max(off, rel);
                // rotation that zeroes the inner product of the two columns
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
                for (int i = 0; i < m; ++i) {
                    const double a = wp[i], b = wq[i];
                    wp[i] = c * a - sn * b;
                    wq[i] = sn * a + c * b;
                }
                double* vp = &Vw[(size_t)p * n];
                double* vq = &Vw[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    const double a = vp[i], b = vq[i];
                    vp[i] = c * a - sn * b;
                    vq[i] = sn * a + c * b;
                }
            }
        if (off == 0.0) break;
    }
    std::vector<double> nrm(n);
    std::vector<int> order(n);
    for (int j = 0; j < n; ++j) {
        double t = 0.0;
        for (int i = 0; i < m; ++i) t += W[(size_t)j * m + i] * W[(size_t)j * m + i];
        nrm[j] = std::sqrt(t);
        order[j] = j;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return nrm[a] > nrm[b]; });
    for (int o = 0; o < n; ++o) {
        const int j = order[o];
        s[o] = nrm[j];
        const double inv = nrm[j] > 0.0 ? 1.0 / nrm[j] : 0.0;
        for (int i = 0; i < m; ++i) U[(size_t)i * n + o] = W[(size_t)j * m + i] * inv;
        for (int i = 0; i < n; ++i) V[(size_t)i * n + o] = Vw[(size_t)j * n + i];
    }
}

void plan_factor_cross(const std::vector<double>& gram_x, const std::vector<double>& gram_y, int L, int d,
                       const std::vector<std::vector<double>>& cores, double drop_budget, bool threads,
                       FactorChoice& fx, FactorChoice& fy) {
    for (FactorChoice* f : {&fx, &fy}) { f->nb[0] = L + 1; f->nb[1] = L; }
    for (int par = 0; par < 2; ++par) { basis_factor(gram_x, L, par, fx); basis_factor(gram_y, L, par, fy); }
    std::vector<std::vector<double>> sig(L + 1), ux(L + 1), vy(L + 1);
    std::vector<int> qk(L + 1, 0);
    auto one = [&](int k) {
        const int par = k % 2, nb = fx.nb[par], mx = fx.m[par], my = fy.m[par];
        if (mx == 0 || my == 0 || nb == 0) return;
        std::vector<double> T;
        sandwich(fx.Rf[par], mx, cores[k], nb, fy.Rf[par], my, T);
        const int q = std::min(mx, my);
        sig[k].resize(q);
        ux[k].resize((size_t)mx * q);
        vy[k].resize((size_t)my * q);
        qk[k] = q;
        svd_jacobi(mx, my, T.data(), ux[k].data(), sig[k].data(), vy[k].data());
    };
    if (threads) {
        parallel_for(L + 1, one);
    } else {
        for (int k = 0; k <= L; ++k) one(k);
    }
    std::vector<std::vector<int>> kept;
    fx.dropped = fy.dropped = select_kept(sig, d, drop_budget, kept);
    fill_choice(sig, ux, qk, kept, d, L, fx);
    fill_choice(sig, vy, qk, kept, d, L, fy);
}

bool make_tables(const FactorChoice& fc, int d, int L, int vw, DeviceTables& t, std::string& err) {
    const std::vector<int>& sk = fc.sk;
    t.L_used = 0;
    for (int k = 0; k <= L; ++k) if (sk[k] > 0) t.L_used = k;
    // radial-factor columns: the blocks of even k first, then those of odd k, so that the
    // consecutive columns a warp forms share one parity (one radial basis, one loop length);
    // fbase[L + 1] holds the total nF
    t.fbase.assign(L + 2, 0);
    int fpos = 0;
    for (int par = 0; par < 2; ++par)
        for (int k = par; k <= L; k += 2) {
            t.fbase[k] = fpos;
            fpos += sk[k];
        }
    t.fbase[L + 1] = fpos;
    t.nF = fpos;
    t.mmax = std::max(fc.m[0], fc.m[1]);
    t.Wt.assign((size_t)std::max(1, t.mmax) * std::max(1, t.nF), 0.0);
    t.colpar.assign(std::max(1, t.nF), 0);
    t.colk.assign(std::max(1, t.nF), 0);
    for (int k = 0; k <= L; ++k)
        for (int s = 0; s < sk[k]; ++s) {
            const int col = t.fbase[k] + s, mk = fc.m[k % 2];
            t.colpar[col] = (uint8_t)(k % 2);
            t.colk[col] = (uint8_t)k;
            for (int o = 0; o < mk; ++o) t.Wt[(size_t)o * t.nF + col] = fc.Wk[k][(size_t)o * sk[k] + s];
        }
    HarmonicTables ht;
    harmonic_tables(d, t.L_used, ht);
    t.tri = ht.tri;
    t.coefA = ht.coefA;
    t.coefB = ht.coefB;
    t.chains.clear();
    t.hbase.assign(L + 2, 0);
    std::vector<int> yoff(L + 2, 0), dimp(L + 1, 0);
    for (int k = 0; k <= L; ++k) {
        t.hbase[k + 1] = t.hbase[k];
        yoff[k + 1] = yoff[k];
        if (sk[k] == 0) continue;
        append_chains(k, d, t.L_used, t.chains);
        const int dim = (int)ht.count[k];
        dimp[k] = ((dim + vw - 1) / vw) * vw;
        t.hbase[k + 1] += dim;
        yoff[k + 1] += dimp[k];
    }
    t.nH = t.hbase[L + 1];
    t.nYp = yoff[L + 1];
    if (t.nYp >= (1 << 20) || t.nF >= 4095) {
        err = "too many harmonics or radial columns for the column descriptors";
        return false;
    }
    t.hk.assign(std::max(1, t.nH), 0);
    t.ktab.assign(kTabStride * (L + 1), 0);
    t.cbase.assign(L + 2, 0);
    t.ychain.assign(std::max(1, t.nYp), -1);
    t.gslot.assign(std::max(1, t.nH), 0);
    // U's column blocks (k, s) follow each other without padding, except that a block of fewer
    // than vw harmonics (degree 0, and degree 1 in d = 3) is padded to vw zero-extended columns, so
    // that every vw-wide chunk of a row meets at most two blocks
    std::vector<int> ucols(L + 1, 0);
    for (int k = 0; k <= L; ++k) {
        for (int g = t.hbase[k]; g < t.hbase[k + 1]; ++g) {
            t.hk[g] = (uint8_t)k;
            t.ychain[yoff[k] + (g - t.hbase[k])] = g;
            t.gslot[g] = yoff[k] + (g - t.hbase[k]);
        }
        const int hkc = (sk[k] > 0) ? (int)ht.count[k] : 0;
        ucols[k] = (hkc > 0 && hkc < vw) ? vw : hkc;
        t.cbase[k + 1] = t.cbase[k] + ucols[k] * sk[k];
        int* kt = &t.ktab[kTabStride * k];
        kt[0] = t.fbase[k];
        kt[1] = sk[k];
        kt[2] = t.cbase[k];
        kt[3] = hkc;
        kt[4] = t.hbase[k];
        kt[5] = ucols[k];
    }
    // rows padded to an odd number of 8-element groups (32 bytes in FP32): every row of U starts
    // on a 32-byte sector (whole-sector stores and loads), and the odd stride spreads the rows of
    // a tile over the DRAM channels (a stride that is a multiple of 128 bytes measured slower)
    t.ldU = ((std::max<int64_t>(vw, t.cbase[L + 1]) + 7) / 8) * 8;
    if ((t.ldU / 8) % 2 == 0) t.ldU += 8;
    if (t.nYp >= (1 << 18)) {
        err = "too many harmonic slots for the column descriptors";
        return false;
    }
    t.colmap.clear();
    t.Spad.assign(t.ldU, 0.0);
    // per padded column: radial-factor index and harmonic slot (F index nF is a zero slot)
    std::vector<uint32_t> colF(t.ldU, (uint32_t)t.nF), colY(t.ldU, 0);
    std::vector<int64_t> blk_end(t.ldU, t.ldU);          // first column after the column's block
    int64_t tcol = 0;
    for (int k = 0; k <= L; ++k) {
        if (sk[k] == 0) continue;
        const int dim = (int)ht.count[k];
        for (int s = 0; s < sk[k]; ++s) {
            const int64_t c0 = t.cbase[k] + (int64_t)s * ucols[k];
            for (int h = 0; h < ucols[k]; ++h) {         // padding columns read zero slots
                colF[c0 + h] = (uint32_t)(t.fbase[k] + s);
                colY[c0 + h] = (uint32_t)(yoff[k] + h);
                blk_end[c0 + h] = c0 + ucols[k];
            }
            for (int h = 0; h < dim; ++h) {
                t.colmap.push_back(c0 + h);
                t.Spad[c0 + h] = fc.S[tcol++];
            }
        }
    }
    for (int64_t c = t.cbase[L + 1]; c < t.ldU; ++c) blk_end[c] = t.ldU;
    // chunk q (columns q vw .. q vw + vw - 1): two words.  w0 = (F << 20) | (e << 18) | slot of the
    // chunk's first column; e = 0 if the chunk lies in one block, else the number of its columns in
    // the first block; then w1 = (F << 20) | slot of the first column of the second block.
    const int64_t nq = t.ldU / vw;
    t.qdesc.assign(2 * nq, 0);
    for (int64_t q = 0; q < nq; ++q) {
        const int64_t c0 = q * vw;
        const int64_t e = std::min<int64_t>(vw, blk_end[c0] - c0);
        uint32_t w0 = (colF[c0] << 20) | colY[c0], w1 = 0;
        if (e < vw) {
            const int64_t cb = c0 + e;
            w0 |= (uint32_t)e << 18;
            w1 = (colF[cb] << 20) | colY[cb];
        }
        t.qdesc[2 * q] = w0;
        t.qdesc[2 * q + 1] = w1;
    }
    return true;
}

bool make_free_tables(const FactorChoice& fc, int d, int L, const DeviceTables& tb, FreeTables& ft,
                      std::string& err) {
    if (d < 4) {
        err = "the matrix-free layout needs d >= 4";
        return false;
    }
    const std::vector<int>& sk = fc.sk;
    const int Lu = tb.L_used, levels = d - 2, stride = chain_stride(d);
    ft.L_used = Lu;
    ft.zoff.assign(Lu + 2, 0);
    ft.zcnt.assign(Lu + 1, 0);
    ft.aoff.assign(Lu + 2, 0);
    ft.acnt.assign(Lu + 1, 0);
    ft.zchain.clear();
    // tails of degree m in the order of H_k: (mu_2, ..., mu_{d-2}) lexicographic, the last signed
    std::vector<int> mu(d - 1);
    for (int m = 0; m <= Lu; ++m) {
        const int cnt = (int)harmonic_count(m, d - 1);
        ft.zcnt[m] = cnt;
        mu[1] = m;
        std::function<void(int)> rec = [&](int pos) {
            if (pos == d - 2) {
                for (int v = -mu[pos - 1]; v <= mu[pos - 1]; ++v) {
                    mu[pos] = v;
                    for (int j = 1; j < levels; ++j) {
                        const int mnext = std::abs(mu[j + 1]);
                        ft.zchain.push_back((int16_t)tri_index(Lu, mnext, mu[j] - mnext));
                    }
                    ft.zchain.push_back((int16_t)v);
                    for (int q = levels; q < stride; ++q) ft.zchain.push_back((int16_t)0);
                }
                return;
            }
            for (int v = 0; v <= mu[pos - 1]; ++v) {
                mu[pos] = v;
                rec(pos + 1);
            }
        };
        rec(2);
        const int padded = (cnt + 7) / 8 * 8;               // each block starts on a 32-byte sector
        for (int q = cnt; q < padded; ++q)                   // padding tails: a zero trig slot
            for (int e = 0; e < stride; ++e) ft.zchain.push_back((int16_t)(e == levels - 1 ? 0x7fff : 0));
        ft.zoff[m + 1] = ft.zoff[m] + padded;
    }
    ft.nZ = ft.zoff[Lu + 1];
    ft.ldZ = ft.nZ;                                          // a multiple of 8
    if ((int64_t)ft.zchain.size() != (int64_t)ft.nZ * stride) {
        err = "matrix-free tail enumeration disagrees with the harmonic counts";
        return false;
    }
    ft.zpair.clear();
    ft.gmap.clear();
    ft.ng = 0;
    if (d == 4 || d == 5) {
        ft.ng = (d == 4) ? 2 * Lu + 1 : (Lu + 1) * (Lu + 1);
        ft.zpair.assign(ft.ldZ, ft.ng);                      // padding: level-1 entry 0 times the zero slot
        for (int t = 0; t < ft.nZ; ++t) {
            const int16_t* ch = &ft.zchain[(size_t)t * stride];
            const int tr = ch[levels - 1];
            if (tr == 0x7fff) continue;
            int g = Lu + tr;
            if (d == 5) {
                const int a = std::abs(tr), mu2 = a + (ch[1] - tri_index(Lu, a, 0));
                g = mu2 * mu2 + mu2 + tr;
            }
            ft.zpair[t] = ((int32_t)ch[0] << 16) | g;
        }
        if (d == 5) {
            ft.gmap.assign(ft.ng, 0);
            for (int mu2 = 0; mu2 <= Lu; ++mu2)
                for (int mu3 = -mu2; mu3 <= mu2; ++mu3) {
                    const int a = std::abs(mu3);
                    ft.gmap[mu2 * mu2 + mu2 + mu3] = (tri_index(Lu, a, mu2 - a) << 16) | (Lu + mu3);
                }
        }
    }
    // hoff[m]: offset of the tails of degree m inside H_k (the same for every k >= m)
    std::vector<int64_t> hoff(Lu + 2, 0);
    for (int m = 0; m <= Lu; ++m) hoff[m + 1] = hoff[m] + ft.zcnt[m];
    ft.a0off.clear();
    ft.afcol.clear();
    ft.wcol.clear();
    for (int m = 0; m <= Lu; ++m) {
        ft.aoff[m] = (int)ft.a0off.size();
        for (int k = m; k <= Lu; ++k) {
            if (k > L || sk[k] == 0) continue;
            const int dimp = tb.ktab[kTabStride * k + 5];
            for (int s2 = 0; s2 < sk[k]; ++s2) {
                ft.a0off.push_back(tri_index(Lu, m, k - m));
                ft.afcol.push_back(tb.fbase[k] + s2);
                ft.wcol.push_back((int64_t)tb.cbase[k] + (int64_t)s2 * dimp + hoff[m]);
            }
        }
        ft.acnt[m] = (int)ft.a0off.size() - ft.aoff[m];
        // every block starts on a 16-byte boundary of an A0F row, so the (up to four) columns
        // one product tile takes from a point are one aligned vector load; padding columns are
        // zero (a0off = -1) and belong to no (k, s)
        while (ft.a0off.size() % 4 != 0) {
            ft.a0off.push_back(-1);
            ft.afcol.push_back(0);
            ft.wcol.push_back(-1);
        }
    }
    ft.aoff[Lu + 1] = (int)ft.a0off.size();
    ft.nA = ft.aoff[Lu + 1];
    ft.ldA = (std::max(ft.nA, 1) + 3) / 4 * 4;
    return true;
}

}  // namespace hdf
