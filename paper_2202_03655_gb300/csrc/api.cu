// C ABI of the HDF library: orchestration of the device kernels and the host planner.
// Declarations and argument contracts are in include/hdf.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hdf.h"
#include "hdf_kernels.cuh"
#include "internal.h"
#include "planner.h"

using namespace hdf;

static thread_local std::string g_err;
constexpr int kMu2Sample = 512;     // mu2 from all pairs of at most this many strided points
namespace hdf {
std::atomic<long long> g_launches(0);     // kernels launched by this library
std::atomic<long long> g_alloc_fail_at(-1);

hdf_status take_device_error(const hdf_factor* f) {
    int flag = 0;
    HDF_CUDA(cudaDeviceSynchronize());
    for (const hdf_factor* g : {f, (const hdf_factor*)f->ypart}) {
        if (!g || !g->dev_err.p) continue;
        int fl = 0;
        HDF_CUDA(cudaMemcpy(&fl, g->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (fl) HDF_CUDA(cudaMemset(g->dev_err.p, 0, sizeof(int)));
        flag |= fl;
    }
    return flag ? fail(HDF_ETIMEOUT, "a device kernel gave up a bounded wait; its results are invalid") : HDF_OK;
}

hdf_status fail(hdf_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

void pool_setup() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}
}  // namespace hdf

// --------------------------------------------------------------------- helpers
static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int grid_for(int64_t work, int per_block, int cap) {
    int64_t g = (work + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

template <typename T>
static hdf_status build_device(hdf_factor* f, const double* x, int64_t n, int d, const dev::Center& cen,
                               double inv2R, const DegreePlan& dp, const FactorChoice& fc, cudaStream_t st);

extern "C" {

const char* hdf_status_string(hdf_status s) {
    switch (s) {
        case HDF_OK: return "ok";
        case HDF_EINVAL: return "invalid argument";
        case HDF_ENOMEM: return "out of memory";
        case HDF_ECUDA: return "CUDA error";
        case HDF_ETOL_UNREACHABLE: return "tolerance unreachable at the degree cap";
        case HDF_ENOTFINITE: return "non-finite input";
        case HDF_ESINGULAR: return "singular core";
        case HDF_ETIMEOUT: return "device wait timed out";
        case HDF_ETOOBIG: return "size exceeds a documented limit";
    }
    return "unknown status";
}

const char* hdf_last_error(void) { return g_err.c_str(); }

long long hdf_launch_count(void) { return hdf::g_launches.load(); }

int hdf_cheb_nodes(int p_max) { return cheb_nodes(p_max); }

hdf_status hdf_cheb_coeffs(hdf_kernel kernel, double lengthscale, double two_r, int M, double* a_host) {
    if (kernel < 0 || kernel > 3 || !(lengthscale > 0) || !(two_r >= 0) || M < 2 || !a_host)
        return fail(HDF_EINVAL, "hdf_cheb_coeffs: bad argument");
    cheb_coeffs(kernel, lengthscale, two_r, M, false, a_host);
    return HDF_OK;
}

hdf_status hdf_choose_degree(const double* a_host, int M, double budget, int p_max, int* p, double* tail,
                             int* reached) {
    if (!a_host || M < 2 || p_max < 0 || !p || !tail || !reached)
        return fail(HDF_EINVAL, "hdf_choose_degree: bad argument");
    bool ok = false;
    *p = choose_degree(a_host, M, budget, p_max, tail, &ok);
    *reached = ok ? 1 : 0;
    return HDF_OK;
}

hdf_status hdf_radial_cores(const double* a_host, int p, int d, double* cores_host, int64_t* count) {
    if (!a_host || p < 0 || (p & 1) || d < 3 || d > HDF_MAX_D || p > 2 * HDF_MAX_L || !count)
        return fail(HDF_EINVAL, "hdf_radial_cores: bad argument");
    const int L = p / 2;
    int64_t tot = 0;
    for (int k = 0; k <= L; ++k) { const int nb = (k % 2 == 0) ? L + 1 : L; tot += (int64_t)nb * nb; }
    *count = tot;
    if (!cores_host) return HDF_OK;
    std::vector<std::vector<double>> cores;
    radial_cores(a_host, p, d, cores);
    int64_t off = 0;
    for (int k = 0; k <= L; ++k) {
        std::memcpy(cores_host + off, cores[k].data(), cores[k].size() * sizeof(double));
        off += (int64_t)cores[k].size();
    }
    return HDF_OK;
}

hdf_status hdf_factor_info(const hdf_factor* f, hdf_info* info) {
    if (!f || !info) return fail(HDF_EINVAL, "hdf_factor_info: null argument");
    *info = f->info;
    return HDF_OK;
}

hdf_status hdf_factor_device(const hdf_factor* f, const void** U_dev, const void** S_dev) {
    if (!f) return fail(HDF_EINVAL, "hdf_factor_device: null factor");
    if (U_dev) *U_dev = f->U.p;
    if (S_dev) *S_dev = f->S.p;
    return HDF_OK;
}

}  // extern "C"

// Packed copy of a factor's U (true columns only) to the host.
static hdf_status export_u(const hdf_factor* f, void* U_host) {
    const int64_t n = f->info.n, r = f->info.rank, ld = f->info.ldu;
    if (!U_host || r == 0) return HDF_OK;
    // U is stored with zero padding columns; gather the true columns row by row
    std::vector<unsigned char> row((size_t)ld * f->esz * 1024);
    unsigned char* out = static_cast<unsigned char*>(U_host);
    for (int64_t i0 = 0; i0 < n; i0 += 1024) {
        const int64_t cnt = std::min<int64_t>(1024, n - i0);
        HDF_CUDA(cudaMemcpy(row.data(), f->U.as<unsigned char>() + (size_t)i0 * ld * f->esz,
                            (size_t)cnt * ld * f->esz, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < cnt; ++i)
            for (int64_t t = 0; t < r; ++t)
                std::memcpy(out + ((size_t)(i0 + i) * r + t) * f->esz,
                            row.data() + ((size_t)i * ld + f->plan.colmap[t]) * f->esz, f->esz);
    }
    return HDF_OK;
}

extern "C" {

hdf_status hdf_factor_export(const hdf_factor* f, void* U_host, double* S_host) {
    if (!f) return fail(HDF_EINVAL, "hdf_factor_export: null factor");
    if (f->mf.on && U_host) return fail(HDF_EINVAL, "hdf_factor_export: a matrix-free factor stores no U");
    if (hdf_status e = export_u(f, U_host); e != HDF_OK) return e;
    if (S_host && f->info.rank > 0) std::memcpy(S_host, f->S_host.data(), f->info.rank * sizeof(double));
    return HDF_OK;
}

hdf_status hdf_factor_export_y(const hdf_factor* f, void* V_host) {
    if (!f) return fail(HDF_EINVAL, "hdf_factor_export_y: null factor");
    if (!f->ypart) return fail(HDF_EINVAL, "hdf_factor_export_y: not a cross factor");
    return export_u(f->ypart, V_host);
}

void hdf_free(hdf_factor* f) {
    if (!f) return;
    // U and F come from the stream-ordered pool of the build's stream; make sure no kernel of
    // any stream still reads them, then return them to the pool on the legacy stream
    cudaDeviceSynchronize();
    f->U.st = nullptr;
    f->mf.Z.st = nullptr;
    f->mf.A0F.st = nullptr;
    if (f->ypart) f->ypart->U.st = nullptr;
    delete f;
}

hdf_status hdf_device_errors(const hdf_factor* f, int* flag) {
    if (!f || !flag) return fail(HDF_EINVAL, "hdf_device_errors: null argument");
    *flag = 0;
    const hdf_status s = take_device_error(f);
    if (s == HDF_ETIMEOUT) *flag = 1;
    return s == HDF_ETIMEOUT ? HDF_OK : s;
}

hdf_status hdf_set_wait_limit(long long cycles, long long* previous) {
    return hdf::set_wait_limit(cycles, previous);
}

hdf_status hdf_check_tf32_rounding(unsigned long long* mismatches) {
    if (!mismatches) return fail(HDF_EINVAL, "hdf_check_tf32_rounding: null argument");
    return hdf::tf32_check(mismatches);
}

void hdf_debug_fail_alloc(long long after) {
    hdf::g_alloc_fail_at.store(after >= 0 ? after : -1);
}

hdf_status hdf_matvec_timings(const hdf_factor* f, double* ms3) {
    if (!f || !ms3) return fail(HDF_EINVAL, "hdf_matvec_timings: null argument");
    if (!f->mv_recorded) return fail(HDF_EINVAL, "hdf_matvec_timings: no matvec recorded yet");
    for (int q = 0; q < 3; ++q) {
        float ms = 0.f;
        HDF_CUDA(cudaEventSynchronize(f->mv_ev[q + 1]));
        HDF_CUDA(cudaEventElapsedTime(&ms, f->mv_ev[q], f->mv_ev[q + 1]));
        ms3[q] = ms;
    }
    return HDF_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------- build
namespace {

struct BuildOpts {
    int p_max = 64;
    double eta = 1.0;
    bool use_tc = true;
    bool matrix_free = false;
};

hdf_status parse_opts(const hdf_options* opt, const char* who, BuildOpts& o) {
    if (opt) {
        if (opt->p_max > 0) o.p_max = opt->p_max;
        if (opt->eta > 0) o.eta = opt->eta;
        if (opt->flags & HDF_FLAG_CUDA_CORES) o.use_tc = false;
        if (opt->flags & HDF_FLAG_MATRIX_FREE) o.matrix_free = true;
    }
    if (o.p_max > 2 * HDF_MAX_L) return fail(HDF_ETOOBIG, std::string(who) + ": p_max > 128");
    o.p_max -= o.p_max % 2;
    return HDF_OK;
}

// Column sums of the row-major n x d points into sum[0..d) (two-stage reduction; synchronises).
hdf_status point_sums(const double* x, int64_t n, int d, DevBuf& part, double* sum, cudaStream_t st) {
    const int g = grid_for(n, 2048, 1024);
    const int64_t chunk = (n + g - 1) / g;
    HDF_COUNT_LAUNCH();
    dev::k_sum_partial<<<g, 256, 0, st>>>(x, n, d, chunk, part.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> hp((size_t)g * d);
    HDF_CUDA(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < d; ++j) {
        double t = 0.0;
        for (int b = 0; b < g; ++b) t += hp[(size_t)b * d + j];
        sum[j] = t;
    }
    return HDF_OK;
}

// max_i |x_i - c|^2 (two-stage reduction; synchronises).
hdf_status max_norm2(const double* x, int64_t n, int d, const dev::Center& cen, DevBuf& part, double* R2,
                     cudaStream_t st) {
    const int g = grid_for(n, 2048, 1024);
    const int64_t chunk = (n + g - 1) / g;
    HDF_COUNT_LAUNCH();
    dev::k_maxnorm_partial<<<g, 256, 0, st>>>(x, n, d, chunk, cen, part.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> hp(g);
    HDF_CUDA(cudaMemcpyAsync(hp.data(), part.p, g * sizeof(double), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    double r2 = 0.0;
    for (int b = 0; b < g; ++b) r2 = std::max(r2, hp[b]);
    *R2 = r2;
    return HDF_OK;
}

// Chebyshev moments sum_i T_j(8 rho_i^2 - 1), j <= 2L+1, of one point set, FP64 partial sums
// (double-float recurrences for FP32 factors), enqueued on the stream into job.msum;
// moments_to_host copies them into job.mom (a copy into pageable memory waits for the
// kernels, so host work meant to overlap them goes before it).
struct MomentJob {
    DevBuf mpart, msum;
    std::vector<double> mom;
};

hdf_status radial_moments(const double* x, int64_t n, int d, const dev::Center& cen, double inv2R, int L, int prec,
                          MomentJob& job, cudaStream_t st) {
    const int nmom = 2 * L + 2;
    const int gmom = grid_for(n, 8192, 2 * 152);
    const int64_t mchunk = (n + gmom - 1) / gmom;
    HDF_CUDA(job.mpart.alloc_on(sizeof(double) * (size_t)gmom * nmom, st));
    HDF_CUDA(job.msum.alloc_on(sizeof(double) * nmom, st));
    HDF_COUNT_LAUNCH();
    const size_t msm_df = sizeof(float2) * 256 * (size_t)(nmom + 1);
    if (prec == HDF_FP32 && msm_df <= 200 * 1024) {
        HDF_CUDA(cudaFuncSetAttribute(dev::k_radial_moments_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)msm_df));
        dev::k_radial_moments_df<<<gmom, 256, msm_df, st>>>(x, n, d, mchunk, cen, inv2R, nmom, job.mpart.as<double>());
    } else {
        const size_t msm = sizeof(double) * dev::kMomTile * nmom;
        dev::k_radial_moments<<<gmom, 256, msm, st>>>(x, n, d, mchunk, cen, inv2R, nmom, job.mpart.as<double>());
    }
    HDF_CUDA(cudaGetLastError());
    HDF_COUNT_LAUNCH();
    dev::k_reduce_cols<<<grid_for(nmom, 256, 1 << 20), 256, 0, st>>>(job.mpart.as<double>(), gmom, nmom,
                                                                    job.msum.as<double>());
    HDF_CUDA(cudaGetLastError());
    job.mom.assign(nmom, 0.0);
    return HDF_OK;
}

hdf_status moments_to_host(MomentJob& job, cudaStream_t st) {
    HDF_CUDA(cudaMemcpyAsync(job.mom.data(), job.msum.p, job.mom.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    return HDF_OK;
}

// A new factor object with the build's metadata; npts = rows of its U.
hdf_factor* new_factor(int64_t npts, int d, hdf_kernel kernel, double ell, double tol, hdf_precision prec,
                       const BuildOpts& o, const dev::Center& cen, double R, double inv2R, double mu2,
                       const DegreePlan& dp, const FactorChoice& fc) {
    hdf_factor* f = new hdf_factor();
    f->use_tc = o.use_tc;
    f->mf.on = o.matrix_free;           // requested; build_device may also choose it
    f->kernel = kernel;
    f->ell = ell;
    f->tol = tol;
    f->prec = prec;
    f->esz = (prec == HDF_FP64) ? 8 : 4;
    hdf_info& I = f->info;
    I.n = npts;
    I.d = d;
    I.precision = prec;
    I.p = dp.p;
    I.L = dp.L;
    I.reached = dp.reached ? 1 : 0;
    I.rank = fc.rank;
    I.nharm = fc.nH;
    for (int j = 0; j < d; ++j) I.center[j] = cen.c[j];
    I.radius = R;
    I.mu2 = mu2;
    I.cheb_tail = dp.tail;
    I.tail_budget = dp.tail_budget;
    I.drop_budget = dp.drop_budget;
    I.dropped_cost = fc.dropped;
    for (int k = 0; k <= std::min(dp.L, HDF_MAX_L); ++k) I.s_k[k] = fc.sk[k];
    f->S_host = fc.S;
    FactorPlan& P = f->plan;
    P.d = d;
    P.L = dp.L;
    P.p_max = o.p_max;
    for (int j = 0; j < d; ++j) P.c[j] = cen.c[j];
    P.inv2R = inv2R;
    for (int q = 0; q < 2; ++q) { P.nb[q] = fc.nb[q]; P.m[q] = fc.m[q]; P.Rf[q] = fc.Rf[q]; P.Qmat[q] = fc.Qmat[q]; }
    P.Wk = fc.Wk;
    P.sk = fc.sk;
    return f;
}

}  // namespace

extern "C" {

hdf_status hdf_build(const double* x_dev, int64_t n, int d, hdf_kernel kernel, double lengthscale,
                     double tol, hdf_precision prec, const hdf_options* opt, hdf_stream stream,
                     hdf_factor** out) {
    if (out) *out = nullptr;
    if (!x_dev || !out || n < 1 || d < 3 || d > HDF_MAX_D || kernel < 0 || kernel > 3 ||
        !(lengthscale > 0) || !(tol > 0 && tol < 1) || (prec != HDF_FP64 && prec != HDF_FP32))
        return fail(HDF_EINVAL, "hdf_build: bad argument (need n>=1, 3<=d<=8, l>0, 0<tol<1)");
    BuildOpts o;
    if (hdf_status e = parse_opts(opt, "hdf_build", o); e != HDF_OK) return e;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double tph[HDF_NPHASE] = {};
    const double t_start = now_ms();

    // ---- A0: centre (mean) and radius (max norm), two-stage reductions
    DevBuf part;
    HDF_CUDA(part.alloc(sizeof(double) * std::max<int64_t>(1024 * d, 2048)));
    dev::Center cen{};
    double sum[HDF_MAX_D];
    if (hdf_status e = point_sums(x_dev, n, d, part, sum, st); e != HDF_OK) return e;
    for (int j = 0; j < d; ++j) {
        cen.c[j] = sum[j] / (double)n;
        if (!std::isfinite(cen.c[j])) return fail(HDF_ENOTFINITE, "hdf_build: non-finite point coordinates");
    }
    double R2 = 0.0;
    if (hdf_status e = max_norm2(x_dev, n, d, cen, part, &R2, st); e != HDF_OK) return e;
    double R = std::sqrt(R2);
    if (!std::isfinite(R)) return fail(HDF_ENOTFINITE, "hdf_build: non-finite point coordinates");
    if (R == 0.0) R = 1.0;
    const double inv2R = 1.0 / (2.0 * R);

    // ---- mean-square kernel value on the strided subsample
    const int m = (int)std::min<int64_t>(n, kMu2Sample);
    HDF_COUNT_LAUNCH();
    dev::k_mu2_rows<<<m, 256, 0, st>>>(x_dev, n, d, m, kernel, lengthscale, part.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> mu_part(m);
    HDF_CUDA(cudaMemcpyAsync(mu_part.data(), part.p, m * sizeof(double), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    double mu2 = 0.0;
    for (int t = 0; t < m; ++t) mu2 += mu_part[t];
    mu2 /= (double)m * (double)m;

    tph[0] = now_ms() - t_start;
    double t0 = now_ms();
    // ---- A1: Chebyshev coefficients and degree (host)
    DegreePlan dp;
    plan_degree(kernel, lengthscale, R, mu2, n, tol, o.eta, o.p_max, d, true, dp, false);
    const int L = dp.L;

    // ---- A3: Chebyshev moments of the radial data (device) -> basis Gram matrices
    MomentJob mj;
    if (hdf_status e = radial_moments(x_dev, n, d, cen, inv2R, L, prec, mj, st); e != HDF_OK) return e;
    // ---- A2 (host, while the device sums the moments): radial cores of each degree
    radial_cores(dp.a.data(), dp.p, d, dp.cores, true);
    tph[1] = now_ms() - t0;
    t0 = now_ms();
    if (hdf_status e = moments_to_host(mj, st); e != HDF_OK) return e;
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<double> gram;
    gram_from_moments(mj.mom, L, gram);
    tph[2] = now_ms() - t0;
    t0 = now_ms();

    // ---- A3-A4 (host): basis factor, per-degree eigendecompositions, truncation
    FactorChoice fc;
    plan_factor(gram, L, d, dp.cores, dp.drop_budget, true, fc);

    hdf_factor* f = new_factor(n, d, kernel, lengthscale, tol, prec, o, cen, R, inv2R, mu2, dp, fc);
    hdf_info& I = f->info;
    I.err_bound = ((double)n * dp.tail + fc.dropped) / ((double)n * std::sqrt(mu2));
    tph[3] = now_ms() - t0;
    for (int q = 0; q < 4; ++q) I.t_ms[q] = tph[q];
    hdf_status st_dev = (prec == HDF_FP64)
        ? build_device<double>(f, x_dev, n, d, cen, inv2R, dp, fc, st)
        : build_device<float>(f, x_dev, n, d, cen, inv2R, dp, fc, st);
    if (st_dev != HDF_OK) { delete f; return st_dev; }
    I.t_ms[HDF_NPHASE - 1] = now_ms() - t_start;
    *out = f;
    if (!dp.reached) {
        g_err = "hdf_build: tolerance not reached at p_max; factor built at the cap";
        return HDF_ETOL_UNREACHABLE;
    }
    return HDF_OK;
}

hdf_status hdf_build_cross(const double* x_dev, int64_t m, const double* y_dev, int64_t n, int d,
                           hdf_kernel kernel, double lengthscale, double tol, hdf_precision prec,
                           const hdf_options* opt, hdf_stream stream, hdf_factor** out) {
    if (out) *out = nullptr;
    if (!x_dev || !y_dev || !out || m < 1 || n < 1 || d < 3 || d > HDF_MAX_D || kernel < 0 || kernel > 3 ||
        !(lengthscale > 0) || !(tol > 0 && tol < 1) || (prec != HDF_FP64 && prec != HDF_FP32))
        return fail(HDF_EINVAL, "hdf_build_cross: bad argument (need m,n>=1, 3<=d<=8, l>0, 0<tol<1)");
    BuildOpts o;
    if (hdf_status e = parse_opts(opt, "hdf_build_cross", o); e != HDF_OK) return e;
    if (o.matrix_free) return fail(HDF_EINVAL, "hdf_build_cross: the matrix-free form is for symmetric factors");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double tph[HDF_NPHASE] = {};
    const double t_start = now_ms();

    // ---- A0 for both sets with one map: centre = mean of the union, R = max distance from it
    DevBuf part;
    HDF_CUDA(part.alloc(sizeof(double) * std::max<int64_t>(1024 * d, 2048)));
    double sx[HDF_MAX_D], sy[HDF_MAX_D];
    if (hdf_status e = point_sums(x_dev, m, d, part, sx, st); e != HDF_OK) return e;
    if (hdf_status e = point_sums(y_dev, n, d, part, sy, st); e != HDF_OK) return e;
    dev::Center cen{};
    for (int j = 0; j < d; ++j) {
        cen.c[j] = (sx[j] + sy[j]) / ((double)m + (double)n);
        if (!std::isfinite(cen.c[j])) return fail(HDF_ENOTFINITE, "hdf_build_cross: non-finite point coordinates");
    }
    double R2x = 0.0, R2y = 0.0;
    if (hdf_status e = max_norm2(x_dev, m, d, cen, part, &R2x, st); e != HDF_OK) return e;
    if (hdf_status e = max_norm2(y_dev, n, d, cen, part, &R2y, st); e != HDF_OK) return e;
    double R = std::sqrt(std::max(R2x, R2y));
    if (!std::isfinite(R)) return fail(HDF_ENOTFINITE, "hdf_build_cross: non-finite point coordinates");
    if (R == 0.0) R = 1.0;
    const double inv2R = 1.0 / (2.0 * R);

    // ---- mean-square kernel value over cross pairs of the strided subsamples
    const int mx = (int)std::min<int64_t>(m, kMu2Sample), my = (int)std::min<int64_t>(n, kMu2Sample);
    HDF_COUNT_LAUNCH();
    dev::k_mu2_cross<<<mx, 256, 0, st>>>(x_dev, m, mx, y_dev, n, my, d, kernel, lengthscale, part.as<double>());
    HDF_CUDA(cudaGetLastError());
    std::vector<double> mu_part(mx);
    HDF_CUDA(cudaMemcpyAsync(mu_part.data(), part.p, mx * sizeof(double), cudaMemcpyDeviceToHost, st));
    HDF_CUDA(cudaStreamSynchronize(st));
    double mu2 = 0.0;
    for (int t = 0; t < mx; ++t) mu2 += mu_part[t];
    mu2 /= (double)mx * (double)my;

    tph[0] = now_ms() - t_start;
    double t0 = now_ms();
    // ---- A1: coefficients and degree; the truncation budget is eta tol |K_XY|_F / 2 with
    //      |K_XY|_F = sqrt(m n mu2)
    DegreePlan dp;
    plan_degree(kernel, lengthscale, R, mu2, m, tol, o.eta, o.p_max, d, true, dp, false);
    dp.drop_budget = 0.5 * o.eta * tol * std::sqrt((double)m * (double)n) * std::sqrt(mu2);
    const int L = dp.L;

    // ---- A3: radial moments of both sets (device) while the host computes the cores
    MomentJob jx, jy;
    if (hdf_status e = radial_moments(x_dev, m, d, cen, inv2R, L, prec, jx, st); e != HDF_OK) return e;
    if (hdf_status e = radial_moments(y_dev, n, d, cen, inv2R, L, prec, jy, st); e != HDF_OK) return e;
    radial_cores(dp.a.data(), dp.p, d, dp.cores, true);
    tph[1] = now_ms() - t0;
    t0 = now_ms();
    if (hdf_status e = moments_to_host(jx, st); e != HDF_OK) return e;
    if (hdf_status e = moments_to_host(jy, st); e != HDF_OK) return e;
    HDF_CUDA(cudaStreamSynchronize(st));
    std::vector<double> gx, gy;
    gram_from_moments(jx.mom, L, gx);
    gram_from_moments(jy.mom, L, gy);
    tph[2] = now_ms() - t0;
    t0 = now_ms();

    // ---- A3-A4 (host): both basis factors, per-degree SVDs, truncation
    FactorChoice fx, fy;
    plan_factor_cross(gx, gy, L, d, dp.cores, dp.drop_budget, true, fx, fy);

    hdf_factor* f = new_factor(m, d, kernel, lengthscale, tol, prec, o, cen, R, inv2R, mu2, dp, fx);
    f->ypart = new_factor(n, d, kernel, lengthscale, tol, prec, o, cen, R, inv2R, mu2, dp, fy);
    const double nrm = std::sqrt((double)m * (double)n);
    for (hdf_factor* g : {f, f->ypart}) {
        g->info.n_y = n;
        g->info.err_bound = (nrm * dp.tail + fx.dropped) / (nrm * std::sqrt(mu2));
    }
    f->ypart->info.n = n;
    tph[3] = now_ms() - t0;
    hdf_info& I = f->info;
    for (int q = 0; q < 4; ++q) I.t_ms[q] = tph[q];
    hdf_status st_dev = (prec == HDF_FP64)
        ? build_device<double>(f, x_dev, m, d, cen, inv2R, dp, fx, st)
        : build_device<float>(f, x_dev, m, d, cen, inv2R, dp, fx, st);
    if (st_dev == HDF_OK) {
        const float tx4 = (float)I.t_ms[4], tx5 = (float)I.t_ms[5];
        st_dev = (prec == HDF_FP64)
            ? build_device<double>(f->ypart, y_dev, n, d, cen, inv2R, dp, fy, st)
            : build_device<float>(f->ypart, y_dev, n, d, cen, inv2R, dp, fy, st);
        I.t_ms[4] = tx4 + f->ypart->info.t_ms[4];           // both sides' radial factors and U
        I.t_ms[5] = tx5 + f->ypart->info.t_ms[5];
    }
    if (st_dev != HDF_OK) { delete f; return st_dev; }
    if (f->info.ldu != f->ypart->info.ldu) {
        delete f;
        return fail(HDF_ECUDA, "hdf_build_cross: the two factors disagree on the padded width");
    }
    I.t_ms[HDF_NPHASE - 1] = now_ms() - t_start;
    *out = f;
    if (!dp.reached) {
        g_err = "hdf_build_cross: tolerance not reached at p_max; factor built at the cap";
        return HDF_ETOL_UNREACHABLE;
    }
    return HDF_OK;
}

}  // extern "C"

// -------------------------------------------------------------------------- matvec
static int ct_for(int c) { return c <= 1 ? 1 : c <= 2 ? 2 : c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : c <= 32 ? 32 : 64; }

template <typename T>
static void launch_utv(int ct, const T* U, int64_t ldU, int64_t n, int64_t r, const T* V, int64_t ldv, int c,
                       int nchunk, int64_t chunk, double* part, cudaStream_t st) {
#define HDF_UTV(CT)                                                                                    \
    case CT: {                                                                                         \
        dim3 g(nchunk, (unsigned)((r + dev::UtvShape<CT>::AB - 1) / dev::UtvShape<CT>::AB));           \
        HDF_COUNT_LAUNCH();                                                                            \
        dev::k_utv_tile<T, CT><<<g, 256, 0, st>>>(U, ldU, n, r, V, ldv, c, chunk, part);               \
        break;                                                                                         \
    }
    switch (ct) { HDF_UTV(1) HDF_UTV(2) HDF_UTV(4) HDF_UTV(8) HDF_UTV(16) HDF_UTV(32) HDF_UTV(64) }
#undef HDF_UTV
}

template <typename T>
static void launch_uw(int ct, const T* U, int64_t ldU, int64_t n, int64_t r, const T* W, int c, T alpha,
                      const T* B, int64_t ldb, T beta, T* Y, int64_t ldy, cudaStream_t st) {
#define HDF_UW(CT)                                                                                     \
    case CT: {                                                                                         \
        const unsigned g = (unsigned)((n + dev::UwShape<CT>::RB - 1) / dev::UwShape<CT>::RB);          \
        HDF_COUNT_LAUNCH();                                                                            \
        dev::k_uw_tile<T, CT><<<g, 256, 0, st>>>(U, ldU, n, r, W, c, alpha, B, ldb, beta, Y, ldy);     \
        break;                                                                                         \
    }
    switch (ct) { HDF_UW(1) HDF_UW(2) HDF_UW(4) HDF_UW(8) HDF_UW(16) HDF_UW(32) HDF_UW(64) }
#undef HDF_UW
}

// Row chunks for the split over n: enough blocks to fill the GPU, partials capped at 256 MB.
static int utv_chunks(int64_t n, int64_t r, int cg) {
    const int64_t by_rows = (n + 2047) / 2048;
    const int64_t by_mem = std::max<int64_t>(1, (int64_t)(256ll << 20) / (8 * std::max<int64_t>(1, r * cg)));
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min(by_rows, by_mem), 1024));
}

constexpr int kMaxGroup = 64;
constexpr int64_t kMaxSolveRank = 32768;      // the solve's r x r core and its factors on the device

// Per-column-group products U_in^T V and U W.  FP32 factors run both on the tensor cores
// (tcgen05, 3xTF32 with FP32 sums per row chunk) whenever the factor allows it (not disabled
// by HDF_FLAG_CUDA_CORES, 16-byte aligned rows, at least 256 rows and 64 columns); below that
// and for FP64 factors the CUDA-core tile kernels run.  One GroupWork serves every group of up
// to cmax columns of one call; its buffers come from the stream-ordered pool.
struct GroupWork {
    bool tc = false;         // tensor cores: the partial sums in `part` are FP32
    int nchunk = 0, tch = 0;
    int64_t chunk = 0, tchunk = 0;
    DevBuf part;             // partial sums: nchunk (or tch) x cmax x r, FP64
    DevBuf twork;            // tensor-core operand splits (V hi/lo, W hi/lo)
};

static bool tc_usable(const hdf_factor* f, int64_t n, int64_t r) {
    return f->prec == HDF_FP32 && f->use_tc && n >= 256 && r >= 64 &&
           reinterpret_cast<uintptr_t>(f->U.p) % 16 == 0 && f->info.ldu % 4 == 0;
}

static hdf_status group_setup(const hdf_factor* fin, const hdf_factor* fout, int64_t r, int cmax, GroupWork& g,
                              cudaStream_t st) {
    const int64_t nin = fin->info.n, nout = fout->info.n;
    g.tc = tc_usable(fin, nin, r) && tc_usable(fout, nout, r);
    if (g.tc) {
        tc_utv_split(nin, r, &g.tchunk, &g.tch);
        HDF_CUDA(g.part.alloc_on(sizeof(double) * (size_t)g.tch * cmax * r, st));
        HDF_CUDA(g.twork.alloc_on(sizeof(float) * tc_work_floats(std::max(nin, nout), r, cmax), st));
    } else {
        g.nchunk = utv_chunks(nin, r, cmax);
        g.chunk = (nin + g.nchunk - 1) / g.nchunk;
        HDF_CUDA(g.part.alloc_on(sizeof(double) * (size_t)g.nchunk * cmax * r, st));
    }
    return HDF_OK;
}

// Partial sums of U_in^T V for cg columns into g.part (*np slices of cg x r).
template <typename T>
static hdf_status group_utv(const hdf_factor* fin, int64_t r, const T* V, int64_t ldv, int cg, GroupWork& g,
                            int* np, cudaStream_t st) {
    const int64_t nin = fin->info.n;
    if constexpr (sizeof(T) == 4) {
        if (g.tc) {
            *np = g.tch;
            return tc_utv(reinterpret_cast<const float*>(fin->U.p), fin->info.ldu, nin, r,
                          reinterpret_cast<const float*>(V), ldv, cg, g.tchunk, g.part.as<double>(),
                          g.twork.as<float>(), fin->dev_err.as<int>(), st, true);
        }
    }
    *np = g.nchunk;
    launch_utv<T>(ct_for(cg), fin->U.as<T>(), fin->info.ldu, nin, r, V, ldv, cg, g.nchunk, g.chunk,
                  g.part.as<double>(), st);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

// W (or Wd) = S .* (sum of the np partial slices of g) for cg columns: FP32 partials from the
// tensor cores, FP64 from the CUDA-core kernels.
template <typename T>
static hdf_status group_reduce(const GroupWork& g, int np, int64_t r, int cg, const T* S, T* W, double* Wd,
                               cudaStream_t st) {
    HDF_COUNT_LAUNCH();
    if (g.tc)
        dev::k_reduce_scale<T, float><<<grid_for(r * cg, 256, 1 << 30), 256, 0, st>>>(
            reinterpret_cast<const float*>(g.part.p), np, r, cg, S, W, Wd);
    else
        dev::k_reduce_scale<T><<<grid_for(r * cg, 256, 1 << 30), 256, 0, st>>>(g.part.as<double>(), np, r, cg, S, W,
                                                                               Wd);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

// Y = alpha U_out W + beta B for cg columns (W: r x cg row-major, bulk type).
template <typename T>
static hdf_status group_uw(const hdf_factor* fout, int64_t r, const T* W, int cg, T alpha, const T* B, int64_t ldb,
                           T beta, T* Y, int64_t ldy, GroupWork& g, cudaStream_t st) {
    const int64_t nout = fout->info.n;
    if constexpr (sizeof(T) == 4) {
        if (g.tc)
            return tc_uw(reinterpret_cast<const float*>(fout->U.p), fout->info.ldu, nout, r,
                         reinterpret_cast<const float*>(W), cg, (float)alpha, reinterpret_cast<const float*>(B), ldb,
                         (float)beta, reinterpret_cast<float*>(Y), ldy, g.twork.as<float>(), fout->dev_err.as<int>(),
                         st);
    }
    launch_uw<T>(ct_for(cg), fout->U.as<T>(), fout->info.ldu, nout, r, W, cg, alpha, B, ldb, beta, Y, ldy, st);
    HDF_CUDA(cudaGetLastError());
    return HDF_OK;
}

// K~ V of a matrix-free factor (symmetric; alpha = 1, beta = 0), per group of <= 64 columns:
// partial sums of U^T V over chunks of points, their FP64 sum scaled by S, then U W.
template <typename T>
static hdf_status matvec_free(const hdf_factor* f, const T* V, int64_t ldv, int ncols, T* Y, int64_t ldy,
                              const T* S_scale, T alpha, const T* B, T beta, cudaStream_t st) {
    if (B || alpha != (T)1 || beta != (T)0) return fail(HDF_EINVAL, "matrix-free factor: plain products only");
    const int64_t n = f->info.n, r = f->info.ldu;
    const int cmax = std::min(ncols, kMaxGroup);
    (void)n;
    DevBuf part, W;
    HDF_CUDA(W.alloc_on(sizeof(T) * (size_t)r * cmax, st));
    hdf_factor* fm = const_cast<hdf_factor*>(f);
    const bool rec = fm->mv_ev[0] != nullptr;
    for (int j0 = 0; j0 < ncols; j0 += kMaxGroup) {
        const int cg = std::min(kMaxGroup, ncols - j0);
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[0], st));
        int np = 0;
        if (hdf_status e = mf_utv<T>(f, V + j0 * ldv, ldv, cg, part, &np, st); e != HDF_OK) return e;
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[1], st));
        HDF_COUNT_LAUNCH();
        dev::k_reduce_scale<T><<<grid_for(r * cg, 256, 1 << 30), 256, 0, st>>>(part.as<double>(), np, r, cg, S_scale,
                                                                               W.as<T>(), nullptr);
        HDF_CUDA(cudaGetLastError());
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[2], st));
        if (hdf_status e = mf_uw<T>(f, W.as<T>(), cg, Y + j0 * ldy, ldy, st); e != HDF_OK) return e;
        if (rec && j0 == 0) { HDF_CUDA(cudaEventRecord(fm->mv_ev[3], st)); fm->mv_recorded = true; }
    }
    return HDF_OK;
}

template <typename T>
// Y = alpha U_f (S_scale .* (U_in^T V)) + beta B, where U_in is the factor of fin (rows of V)
// and U_f that of f (rows of Y): fin = f for K~ V of a symmetric factor; for a cross factor
// K(X, Y) ~= U S V^T, (f, fin) = (X side, Y side) gives K~ V and the reverse gives K~^T V.
// Both factors have the same columns.
static hdf_status matvec_t(const hdf_factor* f, const hdf_factor* fin, const T* V, int64_t ldv, int ncols, T* Y,
                           int64_t ldy, const T* S_scale, T alpha, const T* B, int64_t ldb, T beta, cudaStream_t st) {
    // the GEMMs run over all ldu columns of U; padding columns are zero and carry S = 0
    const int64_t n = f->info.n, r = (f->info.rank > 0) ? f->info.ldu : 0;
    if (r == 0) {
        for (int j = 0; j < ncols; ++j) {
            if (B) {
                HDF_COUNT_LAUNCH();
                dev::k_axpby<T><<<grid_for(n, 256, 1 << 30), 256, 0, st>>>(n, 1, beta, B + j * ldb, ldb, (T)0,
                                                                          Y + j * ldy, ldy);
            } else {
                HDF_CUDA(cudaMemsetAsync(Y + j * ldy, 0, n * sizeof(T), st));
            }
        }
        HDF_CUDA(cudaGetLastError());
        return HDF_OK;
    }
    const int cmax = std::min(ncols, kMaxGroup);
    if (f->mf.on) return matvec_free<T>(f, V, ldv, ncols, Y, ldy, S_scale, alpha, B, beta, st);
    GroupWork g;
    if (hdf_status e = group_setup(fin, f, r, cmax, g, st); e != HDF_OK) return e;
    DevBuf W;
    HDF_CUDA(W.alloc_on(sizeof(T) * (size_t)r * cmax, st));
    hdf_factor* fm = const_cast<hdf_factor*>(f);
    const bool rec = fm->mv_ev[0] != nullptr;
    for (int j0 = 0; j0 < ncols; j0 += kMaxGroup) {
        const int cg = std::min(kMaxGroup, ncols - j0);
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[0], st));
        int np = 0;
        if (hdf_status e = group_utv<T>(fin, r, V + j0 * ldv, ldv, cg, g, &np, st); e != HDF_OK) return e;
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[1], st));
        if (hdf_status e = group_reduce<T>(g, np, r, cg, S_scale, W.as<T>(), nullptr, st); e != HDF_OK) return e;
        if (rec && j0 == 0) HDF_CUDA(cudaEventRecord(fm->mv_ev[2], st));
        if (hdf_status e = group_uw<T>(f, r, W.as<T>(), cg, alpha, B ? B + j0 * ldb : nullptr, ldb, beta,
                                       Y + j0 * ldy, ldy, g, st);
            e != HDF_OK)
            return e;
        if (rec && j0 == 0) { HDF_CUDA(cudaEventRecord(fm->mv_ev[3], st)); fm->mv_recorded = true; }
    }
    // the work buffers go back to the pool in stream order on return
    return HDF_OK;
}

namespace hdf {
template <typename T>
hdf_status utv_reduce(const hdf_factor* f, const T* V, int64_t ldv, int c, const T* S_scale, T* W, double* Wd,
                      cudaStream_t st) {
    const int64_t r = f->info.ldu;      // padded width (rows of W)
    if (c < 1 || c > kMaxGroup) return fail(HDF_EINVAL, "utv_reduce: 1 <= c <= 64");
    if (f->mf.on) {
        DevBuf part;
        int np = 0;
        if (hdf_status e = mf_utv<T>(f, V, ldv, c, part, &np, st); e != HDF_OK) return e;
        HDF_COUNT_LAUNCH();
        dev::k_reduce_scale<T><<<grid_for(r * c, 256, 1 << 30), 256, 0, st>>>(part.as<double>(), np, r, c, S_scale,
                                                                              W, Wd);
        HDF_CUDA(cudaGetLastError());
        return HDF_OK;
    }
    GroupWork g;
    if (hdf_status e = group_setup(f, f, r, c, g, st); e != HDF_OK) return e;
    int np = 0;
    if (hdf_status e = group_utv<T>(f, r, V, ldv, c, g, &np, st); e != HDF_OK) return e;
    if (hdf_status e = group_reduce<T>(g, np, r, c, S_scale, W, Wd, st); e != HDF_OK) return e;
    return HDF_OK;      // the partial sums return to the pool in stream order
}
template hdf_status utv_reduce<float>(const hdf_factor*, const float*, int64_t, int, const float*, float*, double*,
                                      cudaStream_t);
template hdf_status utv_reduce<double>(const hdf_factor*, const double*, int64_t, int, const double*, double*,
                                       double*, cudaStream_t);
}  // namespace hdf

// K~ V through the output side fout and the input side fin (see matvec_t).
static hdf_status matvec_sides(const hdf_factor* fout, const hdf_factor* fin, const void* V_dev, int64_t ldv,
                               int ncols, void* Y_dev, int64_t ldy, cudaStream_t st, const char* who) {
    if (!V_dev || !Y_dev || ncols < 1 || ncols > 1024 || ldv < fin->info.n || ldy < fout->info.n)
        return fail(HDF_EINVAL, std::string(who) + ": bad argument");
    if (fout->prec == HDF_FP64)
        return matvec_t<double>(fout, fin, (const double*)V_dev, ldv, ncols, (double*)Y_dev, ldy,
                                fout->S.as<double>(), 1.0, nullptr, 0, 0.0, st);
    return matvec_t<float>(fout, fin, (const float*)V_dev, ldv, ncols, (float*)Y_dev, ldy, fout->S.as<float>(),
                           1.0f, nullptr, 0, 0.0f, st);
}

extern "C" hdf_status hdf_matvec(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols, void* Y_dev, int64_t ldy,
                      hdf_stream stream) {
    if (!f) return fail(HDF_EINVAL, "hdf_matvec: null factor");
    return matvec_sides(f, f->ypart ? f->ypart : f, V_dev, ldv, ncols, Y_dev, ldy,
                        reinterpret_cast<cudaStream_t>(stream), "hdf_matvec");
}

extern "C" hdf_status hdf_matvec_transpose(const hdf_factor* f, const void* V_dev, int64_t ldv, int ncols,
                                           void* Y_dev, int64_t ldy, hdf_stream stream) {
    if (!f) return fail(HDF_EINVAL, "hdf_matvec_transpose: null factor");
    return matvec_sides(f->ypart ? f->ypart : f, f, V_dev, ldv, ncols, Y_dev, ldy,
                        reinterpret_cast<cudaStream_t>(stream), "hdf_matvec_transpose");
}

// --------------------------------------------------------------------------- solve

namespace hdf {
// The device LU of the Woodbury core (lu.cu).
hdf_status lu_factor_device(int64_t r, double* C, DevBuf& dperm, cudaStream_t st);
hdf_status lu_solve_device(int64_t r, const double* LU, const int* dperm, const double* zi, double* z, int nc,
                           cudaStream_t st);
hdf_status core_init_device(const double* G, const double* Spad, double lambda, int64_t r, double* C, cudaStream_t st);
}  // namespace hdf

namespace {
// y (bulk type) = z (FP64), n values.
template <typename T>
__global__ void k_cast_from_double(const double* __restrict__ z, T* __restrict__ y, int64_t n) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < n) y[idx] = (T)z[idx];
}
}  // namespace

// Xout = (lambda I + U S U^T)^{-1} Bin = (Bin - U C^{-1} U^T Bin) / lambda, C = lambda S^{-1} + U^T U,
// with C's LU factors on the device (f->core): per group of <= 64 columns, U^T Bin (FP64 sums),
// the two triangular solves on the device, then U times the result.
template <typename T>
static hdf_status woodbury_apply(hdf_factor* f, double lambda, const T* Bin, int64_t ldb, int ncols, T* Xout,
                                 int64_t ldx, cudaStream_t st) {
    const int64_t n = f->info.n, r = (f->info.rank > 0) ? f->info.ldu : 0;
    if (r == 0) {
        HDF_COUNT_LAUNCH();
        dev::k_axpby<T><<<grid_for(n * ncols, 256, 1 << 30), 256, 0, st>>>(n, ncols, (T)(1.0 / lambda), Bin, ldb,
                                                                           (T)0, Xout, ldx);
        HDF_CUDA(cudaGetLastError());
        return HDF_OK;
    }
    const int cmax = std::min(ncols, kMaxGroup);
    GroupWork g;
    if (hdf_status e = group_setup(f, f, r, cmax, g, st); e != HDF_OK) return e;
    DevBuf Wd, Zd, Wt;
    HDF_CUDA(Wd.alloc_on(sizeof(double) * (size_t)r * cmax, st));
    HDF_CUDA(Zd.alloc_on(sizeof(double) * (size_t)r * cmax, st));
    HDF_CUDA(Wt.alloc_on(sizeof(T) * (size_t)r * cmax, st));
    for (int j0 = 0; j0 < ncols; j0 += kMaxGroup) {
        const int cg = std::min(kMaxGroup, ncols - j0);
        int np = 0;
        if (hdf_status e = group_utv<T>(f, r, Bin + j0 * ldb, ldb, cg, g, &np, st); e != HDF_OK) return e;
        if (hdf_status e = group_reduce<T>(g, np, r, cg, (const T*)nullptr, (T*)nullptr, Wd.as<double>(), st);
            e != HDF_OK)
            return e;
        if (hdf_status e = lu_solve_device(r, f->core_lu.as<double>(), f->core_perm.as<int>(), Wd.as<double>(),
                                           Zd.as<double>(), cg, st);
            e != HDF_OK)
            return e;
        HDF_COUNT_LAUNCH();
        k_cast_from_double<T><<<grid_for(r * cg, 256, 1 << 30), 256, 0, st>>>(Zd.as<double>(), Wt.as<T>(), r * cg);
        HDF_CUDA(cudaGetLastError());
        if (hdf_status e = group_uw<T>(f, r, Wt.as<T>(), cg, (T)(-1.0 / lambda), Bin + j0 * ldb, ldb,
                                       (T)(1.0 / lambda), Xout + j0 * ldx, ldx, g, st);
            e != HDF_OK)
            return e;
    }
    return HDF_OK;
}

template <typename T>
static hdf_status solve_t(hdf_factor* f, double lambda, const T* B, int64_t ldb, int ncols, T* X, int64_t ldx,
                          int refine, cudaStream_t st) {
    const int64_t n = f->info.n, r = (f->info.rank > 0) ? f->info.ldu : 0;
    if (r > kMaxSolveRank) return fail(HDF_ETOOBIG, "hdf_solve: padded rank > 32768");
    if (r > 0 && !f->core_G.p) {
        DevBuf Gd;
        HDF_CUDA(Gd.alloc(sizeof(double) * (size_t)r * r));
        cudaEvent_t g0, g1;
        HDF_CUDA(cudaEventCreate(&g0));
        HDF_CUDA(cudaEventCreate(&g1));
        HDF_CUDA(cudaEventRecord(g0, st));
        const bool aligned = (reinterpret_cast<uintptr_t>(f->U.p) % 16 == 0) && (f->info.ldu % 4 == 0);
        if (sizeof(T) == 4 && f->use_tc && aligned && r >= 64 && n >= 32) {
            // U^T U on the tensor cores (FP32 factors)
            if (!f->dev_err.p) {
                HDF_CUDA(f->dev_err.alloc(sizeof(int)));
                HDF_CUDA(cudaMemsetAsync(f->dev_err.p, 0, sizeof(int), st));
            }
            hdf_status s = tc_gram(reinterpret_cast<const float*>(f->U.p), f->info.ldu, n, r, Gd.as<double>(),
                                   f->dev_err.as<int>(), st);
            if (s != HDF_OK) return s;
        } else {
            const unsigned nt = (unsigned)((r + 63) / 64);
            HDF_COUNT_LAUNCH();
            dev::k_gram<T><<<dim3(nt, nt), 256, 0, st>>>(f->U.as<T>(), f->info.ldu, n, r, Gd.as<double>());
            HDF_CUDA(cudaGetLastError());
        }
        HDF_CUDA(cudaEventRecord(g1, st));
        HDF_CUDA(cudaStreamSynchronize(st));
        float gms = 0.f;
        cudaEventElapsedTime(&gms, g0, g1);
        cudaEventDestroy(g0);
        cudaEventDestroy(g1);
        // a Gram matrix from a kernel that gave up a wait is not kept
        if (hdf_status e = take_device_error(f); e != HDF_OK) return e;
        std::swap(f->core_G.p, Gd.p);
        std::swap(f->core_G.bytes, Gd.bytes);
        f->info.t_ms[6] = gms;
        f->core_lambda = -1.0;
    }
    if (r > 0 && f->core_lambda != lambda) {
        // C = lambda S^-1 + U^T U (padding columns: zero columns of U with S = 0 get a unit
        // diagonal and solve to zero), factored on the device
        const double t0 = now_ms();
        if (!f->core_S.p) {
            HDF_CUDA(f->core_S.alloc(sizeof(double) * (size_t)r));
            HDF_CUDA(cudaMemcpy(f->core_S.p, f->plan.Spad.data(), sizeof(double) * r, cudaMemcpyHostToDevice));
        }
        if (!f->core_lu.p) HDF_CUDA(f->core_lu.alloc(sizeof(double) * (size_t)r * r));
        f->core_lambda = -1.0;
        if (hdf_status e = core_init_device(f->core_G.as<double>(), f->core_S.as<double>(), lambda, r,
                                            f->core_lu.as<double>(), st);
            e != HDF_OK)
            return e;
        if (hdf_status e = lu_factor_device(r, f->core_lu.as<double>(), f->core_perm, st); e != HDF_OK) return e;
        f->core_lambda = lambda;
        f->info.lu_ms = now_ms() - t0;
    }
    hdf_status s = woodbury_apply<T>(f, lambda, B, ldb, ncols, X, ldx, st);
    if (s != HDF_OK) return s;
    if (refine <= 0) {
        HDF_CUDA(cudaStreamSynchronize(st));
        return take_device_error(f);
    }
    DevBuf Rb, KX, dX;
    HDF_CUDA(Rb.alloc(sizeof(T) * (size_t)n * ncols));
    HDF_CUDA(KX.alloc(sizeof(T) * (size_t)n * ncols));
    HDF_CUDA(dX.alloc(sizeof(T) * (size_t)n * ncols));
    for (int it = 0; it < refine; ++it) {
        // Rb = B - lambda X - K~ X
        s = matvec_t<T>(f, f, X, ldx, ncols, KX.as<T>(), n, f->S.as<T>(), (T)1, nullptr, 0, (T)0, st);
        if (s != HDF_OK) return s;
        for (int j = 0; j < ncols; ++j)
            HDF_CUDA(cudaMemcpyAsync(Rb.as<T>() + j * n, B + j * ldb, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        HDF_COUNT_LAUNCH();
        dev::k_axpby<T><<<grid_for(n * ncols, 256, 1 << 30), 256, 0, st>>>(n, ncols, (T)(-lambda), X, ldx, (T)1,
                                                                           Rb.as<T>(), n);
        HDF_COUNT_LAUNCH();
        dev::k_axpby<T><<<grid_for(n * ncols, 256, 1 << 30), 256, 0, st>>>(n, ncols, (T)(-1), KX.as<T>(), n, (T)1,
                                                                           Rb.as<T>(), n);
        HDF_CUDA(cudaGetLastError());
        s = woodbury_apply<T>(f, lambda, Rb.as<T>(), n, ncols, dX.as<T>(), n, st);
        if (s != HDF_OK) return s;
        HDF_COUNT_LAUNCH();
        dev::k_axpby<T><<<grid_for(n * ncols, 256, 1 << 30), 256, 0, st>>>(n, ncols, (T)1, dX.as<T>(), n, (T)1, X,
                                                                           ldx);
        HDF_CUDA(cudaGetLastError());
    }
    HDF_CUDA(cudaStreamSynchronize(st));
    return take_device_error(f);
}

extern "C" hdf_status hdf_solve(hdf_factor* f, double lambda, const void* B_dev, int64_t ldb, int ncols,
                                void* X_dev, int64_t ldx, int refine_steps, hdf_stream stream) {
    if (!f || !B_dev || !X_dev || ncols < 1 || ncols > 1024 || !(lambda > 0) || ldb < f->info.n ||
        ldx < f->info.n || refine_steps < 0)
        return fail(HDF_EINVAL, "hdf_solve: bad argument");
    if (f->ypart) return fail(HDF_EINVAL, "hdf_solve: a cross factor K(X, Y) has no (lambda I + K~) system");
    if (f->mf.on) return fail(HDF_EINVAL, "hdf_solve: the Woodbury core needs the stored U (matrix-free factor)");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (f->prec == HDF_FP64)
        return solve_t<double>(f, lambda, (const double*)B_dev, ldb, ncols, (double*)X_dev, ldx, refine_steps, st);
    return solve_t<float>(f, lambda, (const float*)B_dev, ldb, ncols, (float*)X_dev, ldx, refine_steps, st);
}

// ---------------------------------------------------------- device part of build
namespace hdf {
// The matrix-free rows of a factor (mfree.cu): Z and P_0 F per point from the radial factors F.
template <typename T>
hdf_status mf_write(hdf_factor* f, const double* x, int64_t n, int d, const dev::Center& cen, double inv2R,
                    const FactorChoice& fc, const DeviceTables& tb, const void* F, int64_t ldF, const void* coefA,
                    const void* coefB, cudaStream_t st);
}  // namespace hdf

template <typename T>
static std::vector<T> cast_vec(const std::vector<double>& v) {
    std::vector<T> o(v.size());
    for (size_t q = 0; q < v.size(); ++q) o[q] = (T)v[q];
    return o;
}

template <typename T>
static hdf_status build_device(hdf_factor* f, const double* x, int64_t n, int d, const dev::Center& cen,
                               double inv2R, const DegreePlan& dp, const FactorChoice& fc, cudaStream_t st) {
    hdf_info& I = f->info;
    const int L = dp.L;
    const int64_t r = I.rank;
    const int vw = (sizeof(T) == 4) ? 4 : 2;
    HDF_CUDA(f->dev_err.alloc(sizeof(int)));
    HDF_CUDA(cudaMemsetAsync(f->dev_err.p, 0, sizeof(int), st));
    DeviceTables tb;
    std::string terr;
    if (!make_tables(fc, d, L, vw, tb, terr)) return fail(HDF_ETOOBIG, "hdf_build: " + terr);
    I.ldu = tb.ldU;
    f->plan.colmap = tb.colmap;
    f->plan.Spad = tb.Spad;
    // S on the device, on the padded columns
    {
        std::vector<T> Sd(I.ldu, (T)0);
        for (int64_t a = 0; a < I.ldu; ++a) Sd[a] = (T)tb.Spad[a];
        HDF_CUDA(f->S.alloc(sizeof(T) * I.ldu));
        HDF_CUDA(cudaMemcpyAsync(f->S.p, Sd.data(), sizeof(T) * I.ldu, cudaMemcpyHostToDevice, st));
    }
    const size_t ubytes = sizeof(T) * (size_t)n * (size_t)I.ldu;
    // the matrix-free form when asked for, or when U would not fit (d >= 4 only)
    bool mfree = f->mf.on && r > 0;
    if (mfree && d < 4) return fail(HDF_EINVAL, "hdf_build: the matrix-free form needs d >= 4");
    if (!mfree && d >= 4 && r > 0 && !FreeFactor::fits((int64_t)ubytes)) mfree = true;
    f->mf.on = false;                    // set by mf_write once the rows exist
    if (!mfree && f->U.alloc_on(ubytes, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(HDF_ENOMEM, "hdf_build: cannot allocate U (" + std::to_string(ubytes) + " bytes)");
    }
    if (r == 0) { HDF_CUDA(cudaStreamSynchronize(st)); return HDF_OK; }
    const int L_used = tb.L_used, nF = tb.nF, mmax = tb.mmax;
    const int64_t nH = tb.nH;
    const std::vector<double>* Qmat = fc.Qmat;
    const int nb0 = fc.nb[0], nb1 = fc.nb[1], m0 = fc.m[0], m1 = fc.m[1];
    std::vector<T> Wt = cast_vec<T>(tb.Wt), cA = cast_vec<T>(tb.coefA), cB = cast_vec<T>(tb.coefB);
    HarmonicTables ht;
    ht.tri = tb.tri;

    // upload (kept in the factor for the adjoint)
    FactorPlan& PL = f->plan;
    PL.L_used = L_used;
    PL.tri = tb.tri;
    PL.nF = nF;
    PL.nH = (int)nH;
    PL.mmax = mmax;
    PL.fbase = tb.fbase;
    PL.cbase = tb.cbase;
    PL.hbase = tb.hbase;
    DevBuf dpar, dF;
    DevBuf &dQ0 = PL.dQ0, &dQ1 = PL.dQ1, &dW = PL.dW, &dchains = PL.dchains, &dA = PL.dA, &dB = PL.dB;
    HDF_CUDA(PL.dcolk.alloc(tb.colk.size()));
    HDF_CUDA(PL.dhk.alloc(tb.hk.size() + 1));
    HDF_CUDA(PL.dktab.alloc(sizeof(int) * tb.ktab.size()));
    HDF_CUDA(cudaMemcpyAsync(PL.dcolk.p, tb.colk.data(), tb.colk.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(PL.dhk.p, tb.hk.data(), tb.hk.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(PL.dktab.p, tb.ktab.data(), sizeof(int) * tb.ktab.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(dQ0.alloc(sizeof(double) * std::max<size_t>(1, Qmat[0].size())));
    HDF_CUDA(dQ1.alloc(sizeof(double) * std::max<size_t>(1, Qmat[1].size())));
    HDF_CUDA(dW.alloc(sizeof(T) * Wt.size()));
    HDF_CUDA(dpar.alloc(tb.colpar.size()));
    HDF_CUDA(dchains.alloc(sizeof(int16_t) * std::max<size_t>(1, tb.chains.size())));
    HDF_CUDA(PL.dqdesc.alloc(sizeof(uint32_t) * tb.qdesc.size()));
    HDF_CUDA(PL.dychain.alloc(sizeof(int32_t) * tb.ychain.size()));
    HDF_CUDA(PL.dgslot.alloc(sizeof(int32_t) * tb.gslot.size()));
    HDF_CUDA(dA.alloc(sizeof(T) * cA.size() + 16));
    HDF_CUDA(dB.alloc(sizeof(T) * cB.size() + 16));
    const int64_t ldF = ((int64_t)nF + 31) / 32 * 32;       // 128-byte rows (FP32): whole-sector stores
    if (dF.alloc_on(sizeof(T) * (size_t)n * ldF, st) != cudaSuccess) {
        cudaGetLastError();
        return fail(HDF_ENOMEM, "hdf_build: cannot allocate the radial factor buffer");
    }
    if (!Qmat[0].empty()) HDF_CUDA(cudaMemcpyAsync(dQ0.p, Qmat[0].data(), sizeof(double) * Qmat[0].size(), cudaMemcpyHostToDevice, st));
    if (!Qmat[1].empty()) HDF_CUDA(cudaMemcpyAsync(dQ1.p, Qmat[1].data(), sizeof(double) * Qmat[1].size(), cudaMemcpyHostToDevice, st));
    // FP32 factors: [Qmat0 | Qmat1] as (hi, lo) float pairs for the compensated radial basis,
    // (L+1) x mtp with the odd columns zero in row L and mtp a multiple of 8
    const int mtp = ((m0 + m1 + 7) / 8) * 8;
    if (sizeof(T) == 4) {
        std::vector<float> qc((size_t)2 * (L + 1) * mtp, 0.f);
        auto put = [&](int l, int o, double v) {
            const float h = (float)v;
            qc[2 * ((size_t)l * mtp + o)] = h;
            qc[2 * ((size_t)l * mtp + o) + 1] = (float)(v - (double)h);
        };
        for (int l = 0; l < nb0; ++l)
            for (int o = 0; o < m0; ++o) put(l, o, Qmat[0][(size_t)l * m0 + o]);
        for (int l = 0; l < nb1; ++l)
            for (int o = 0; o < m1; ++o) put(l, m0 + o, Qmat[1][(size_t)l * m1 + o]);
        HDF_CUDA(PL.dQC.alloc(sizeof(float) * qc.size()));
        HDF_CUDA(cudaMemcpyAsync(PL.dQC.p, qc.data(), sizeof(float) * qc.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaStreamSynchronize(st));      // qc is a local buffer
    }
    HDF_CUDA(cudaMemcpyAsync(dW.p, Wt.data(), sizeof(T) * Wt.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(dpar.p, tb.colpar.data(), tb.colpar.size(), cudaMemcpyHostToDevice, st));
    if (!tb.chains.empty())
        HDF_CUDA(cudaMemcpyAsync(dchains.p, tb.chains.data(), sizeof(int16_t) * tb.chains.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(PL.dqdesc.p, tb.qdesc.data(), sizeof(uint32_t) * tb.qdesc.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(PL.dychain.p, tb.ychain.data(), sizeof(int32_t) * tb.ychain.size(), cudaMemcpyHostToDevice, st));
    HDF_CUDA(cudaMemcpyAsync(PL.dgslot.p, tb.gslot.data(), sizeof(int32_t) * tb.gslot.size(), cudaMemcpyHostToDevice, st));
    if (!cA.empty()) {
        HDF_CUDA(cudaMemcpyAsync(dA.p, cA.data(), sizeof(T) * cA.size(), cudaMemcpyHostToDevice, st));
        HDF_CUDA(cudaMemcpyAsync(dB.p, cB.data(), sizeof(T) * cB.size(), cudaMemcpyHostToDevice, st));
    }

    cudaEvent_t ev[3];
    for (int q = 0; q < 3; ++q) HDF_CUDA(cudaEventCreate(&ev[q]));
    struct EvGuard { cudaEvent_t* e; ~EvGuard() { for (int q = 0; q < 3; ++q) cudaEventDestroy(e[q]); } } evg{ev};
    HDF_CUDA(cudaEventRecord(ev[0], st));
    // A5a: radial factors F
    {
        dev::RFParams R{};
        R.x = x; R.n = n; R.d = d; R.c = cen; R.inv2R = inv2R; R.L = L;
        R.Qm0 = dQ0.as<double>(); R.nb0 = nb0; R.m0 = m0;
        R.Qm1 = dQ1.as<double>(); R.nb1 = nb1; R.m1 = m1;
        R.Wt = dW.p; R.colpar = dpar.as<uint8_t>(); R.nF = nF;
        R.F = dF.p; R.ldF = ldF;
        const int grid = grid_for((n + dev::kFTile - 1) / dev::kFTile, 1, 152 * 8);
        const size_t sm64 = dev::radialF_smem(L, m0, m1, sizeof(T));
        size_t sm32 = dev::radialF_df_smem(L, m0, m1, mtp, nF, true);
        R.stage_wt = 1;
        if (sm32 > 200 * 1024) { sm32 = dev::radialF_df_smem(L, m0, m1, mtp, nF, false); R.stage_wt = 0; }
        if (sizeof(T) == 4 && sm32 <= 200 * 1024) {
            R.QC = PL.dQC.as<float2>();
            R.mtp = mtp;
            const int kopt = dev::radialF_df_kopt(m0 + m1, dev::kRfThreads / 32 - 1);
            auto rk = kopt == 2 ? dev::k_radial_F_df<2> : kopt == 4 ? dev::k_radial_F_df<4> : dev::k_radial_F_df<8>;
            HDF_CUDA(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32));
            int occ = 0, nsm = 0, dv = 0;
            HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rk, dev::kRfThreads, sm32));
            HDF_CUDA(cudaGetDevice(&dv));
            HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
            const int g32 = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(occ, 1),
                                                                          (n + dev::kFTile - 1) / dev::kFTile));
            HDF_COUNT_LAUNCH();
            rk<<<g32, dev::kRfThreads, sm32, st>>>(R);
        } else {
            if (sm64 > 200 * 1024) return fail(HDF_ETOOBIG, "hdf_build: radial tile exceeds shared memory");
            HDF_CUDA(cudaFuncSetAttribute(dev::k_radial_F<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64));
            HDF_COUNT_LAUNCH();
            dev::k_radial_F<T><<<grid, 256, sm64, st>>>(R);
        }
        HDF_CUDA(cudaGetLastError());
    }
    HDF_CUDA(cudaEventRecord(ev[1], st));
    if (mfree) {
        // A5b, matrix-free: the Z and P_0 F rows instead of U
        if (hdf_status e = mf_write<T>(f, x, n, d, cen, inv2R, fc, tb, dF.p, ldF, dA.p, dB.p, st); e != HDF_OK)
            return e;
        I.matrix_free = 1;
        I.mf_row = (int64_t)f->mf.ldZ + f->mf.ldA;
    } else {
    // A5b: harmonics and U
        dev::UWParams P{};
        P.x = x; P.n = n; P.d = d; P.c = cen; P.inv2R = inv2R;
        P.L = L_used; P.tri = ht.tri;
        P.chains = dchains.as<int16_t>(); P.nH = (int)nH; P.cstride = chain_stride(d);
        P.ychain = PL.dychain.as<int32_t>(); P.nYp = tb.nYp; P.gslot = PL.dgslot.as<int32_t>();
        P.qdesc = PL.dqdesc.as<uint32_t>(); P.nF = nF;
        P.F = dF.p; P.ldF = ldF;
        P.U = f->U.p; P.ldU = I.ldu;
        P.coefA = dA.p; P.coefB = dB.p;
        const int levels = d - 2;
        // One CTA per SM with as many warps as shared memory holds (up to 32): the coefficient
        // tables and, when they fit, the per-point index tables are shared by all its warps.
        // Preference: harmonics precomputed per point (pre) with staged tables, then the
        // on-the-fly variant with staged tables, then either with tables read from global.
        const size_t coef = dev::align16(sizeof(T) * 2 * (size_t)levels * ht.tri);
        const size_t budget = 226 * 1024;
        const int64_t nq = I.ldu / (int64_t)(sizeof(T) == 4 ? 4 : 2);
        struct Cfg { bool pre, staged; int warps; size_t pw; size_t tabs; };
        Cfg pick{false, false, 0, 0, 0};
        for (int attempt = 0; attempt < 4 && pick.warps == 0; ++attempt) {
            const bool pre = (attempt % 2) == 0, staged = attempt < 2;
            const size_t pw = sizeof(T) * (size_t)dev::uwriter_per_warp(levels, ht.tri, L_used, tb.nYp, nF, pre);
            const size_t tabs = staged ? dev::uwriter_tab_bytes(nq, (int)nH, chain_stride(d), tb.nYp, pre) : 0;
            if (coef + tabs >= budget) continue;
            const int w = (int)std::min<size_t>(32, (budget - coef - tabs) / pw);
            if (w >= (attempt < 3 ? 8 : 1)) pick = Cfg{pre, staged, w, pw, tabs};
        }
        if (pick.warps == 0) return fail(HDF_ETOOBIG, "hdf_build: harmonic tables exceed shared memory");
        const bool pre = pick.pre;
        const int warps = pick.warps;
        P.per_warp = (int)(pick.pw / sizeof(T));
        P.tab_bytes = (int)pick.tabs;
        const size_t sm = dev::align16((size_t)warps * pick.pw + sizeof(T) * 2 * (size_t)levels * ht.tri) + pick.tabs;
        const bool stg = pick.staged;
        auto kern = pre ? (stg ? dev::k_uwriter<T, true, false, true> : dev::k_uwriter<T, true, false, false>)
                        : (stg ? dev::k_uwriter<T, false, false, true> : dev::k_uwriter<T, false, false, false>);
        // FP32 factors, harmonics precomputed, tables staged, nF <= 32 kPfF: the next point's
        // radial factors and coordinate are prefetched into registers
        if constexpr (sizeof(T) == 4)
            if (pre && stg && nF <= 32 * dev::kPfF) kern = dev::k_uwriter<T, true, true, true>;
        HDF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int occ = 0;
        HDF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, sm));
        int nsm = 0, dv = 0;
        HDF_CUDA(cudaGetDevice(&dv));
        HDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
        const int grid = std::max(1, std::min<int>(nsm * std::max(occ, 1), (int)((n + warps - 1) / warps)));
        HDF_COUNT_LAUNCH();
        kern<<<grid, warps * 32, sm, st>>>(P);   // P.tab_bytes: staged index tables
        HDF_CUDA(cudaGetLastError());
    }
    HDF_CUDA(cudaEventRecord(ev[2], st));
    HDF_CUDA(cudaStreamSynchronize(st));
    float ms1 = 0.f, ms2 = 0.f;
    HDF_CUDA(cudaEventElapsedTime(&ms1, ev[0], ev[1]));
    HDF_CUDA(cudaEventElapsedTime(&ms2, ev[1], ev[2]));
    I.t_ms[4] = ms1;
    I.t_ms[5] = ms2;
    for (auto& e : f->mv_ev) HDF_CUDA(cudaEventCreate(&e));
    return HDF_OK;
}
