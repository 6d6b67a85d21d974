// bx_api.cu -- host side of the C ABI (include/bx.h): argument validation, model
// creation (device copies of every toy, set-up kernel), workspace, and the evaluation
// driver that enqueues k_prep -> k_fwd_* -> k_mid -> [k_bwd_*] -> k_gather on the
// model's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bx_model.h"
#include "bx_internal.cuh"

using namespace bx;

static thread_local std::string g_err;

int bx_set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return bx_set_error(BX_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                __FILE__, __LINE__);                                              \
    } while (0)

extern "C" const char* bx_last_error(void) { return g_err.c_str(); }

extern "C" const char* bx_status_string(int s) {
    switch (s) {
        case BX_OK: return "ok";
        case BX_EINVAL: return "invalid argument";
        case BX_ENOMEM: return "out of memory";
        case BX_ECUDA: return "CUDA error";
        case BX_EDOMAIN: return "expected count <= 0 where data are present (or sigma^2 <= 0)";
        case BX_ETIMEOUT: return "device wait timed out";
        case BX_ENOTCONV: return "fit did not converge";
        default: return "unknown status";
    }
}

// ------------------------------------------------------------------ model

static int alloc_dev(bx_model* m, void** p, size_t bytes);

static bool finite_nonneg(const double* a, size_t n) {
    for (size_t j = 0; j < n; ++j)
        if (!std::isfinite(a[j]) || a[j] < 0.0) return false;
    return true;
}

// Groups of species by Birks multiplier (species-specific quenching): returns the number of
// groups (0 if there are more than MAX_SETS), their multipliers and each species' group.
static int quench_groups(const bx_model_desc& d, double* xi, int* set_of) {
    int n = 0;
    for (int k = 0; k < d.n_species; ++k) {
        const double q = d.quench ? d.quench[k] : 1.0;
        int c = 0;
        while (c < n && xi[c] != q) ++c;
        if (c == n) {
            if (n == MAX_SETS) return 0;
            xi[n++] = q;
        }
        set_of[k] = c;
    }
    return n;
}

static int validate_desc(const bx_model_desc& d, int t) {
#define REQ(cond, ...) \
    if (!(cond)) return bx_set_error(BX_EINVAL, __VA_ARGS__)
    REQ(d.n_grid >= 1 && d.n_grid <= MAX_CB * BCOLS, "toy %d: n_grid %d out of [1, %d]", t, d.n_grid, MAX_CB * BCOLS);
    REQ(std::isfinite(d.e_max) && d.e_max > 0.0, "toy %d: e_max must be > 0", t);
    REQ(d.n_species >= 1 && d.n_species <= KMAX, "toy %d: n_species %d out of [1, %d]", t, d.n_species, KMAX);
    REQ(d.shapes && finite_nonneg(d.shapes, (size_t)d.n_species * d.n_grid), "toy %d: shapes missing, negative or not finite", t);
    REQ(d.stop_pow, "toy %d: stop_pow missing", t);
    for (int i = 0; i < d.n_grid; ++i) REQ(std::isfinite(d.stop_pow[i]) && d.stop_pow[i] > 0.0, "toy %d: stop_pow[%d] must be > 0", t, i);
    if (d.tag_frac)
        for (int k = 0; k < d.n_species; ++k)
            REQ(d.tag_frac[k] >= 0.0 && d.tag_frac[k] <= 1.0, "toy %d: tag_frac[%d] out of [0, 1]", t, k);
    REQ(d.n_pileup >= 1 && d.n_pileup <= MAX_L, "toy %d: n_pileup %d out of [1, %d]", t, d.n_pileup, MAX_L);
    REQ(d.pileup && finite_nonneg(d.pileup, d.n_pileup), "toy %d: pileup missing, negative or not finite", t);
    REQ(std::isfinite(d.width) && d.width > 0.0, "toy %d: width must be > 0", t);
    REQ(d.m_lo >= 0 && d.m_hi > d.m_lo && d.m_hi <= MAX_TILES * TM, "toy %d: window [%d, %d) invalid (m_hi <= %d)", t, d.m_lo, d.m_hi, MAX_TILES * TM);
    const size_t nw = (size_t)(d.m_hi - d.m_lo);
    REQ(d.counts_sub && finite_nonneg(d.counts_sub, nw), "toy %d: counts_sub missing, negative or not finite", t);
    REQ(!d.tag_frac || (d.counts_tag && finite_nonneg(d.counts_tag, nw)), "toy %d: counts_tag required with tag_frac", t);
    REQ(d.n_rad >= 0 && d.n_rad <= MAX_RAD, "toy %d: n_rad out of [0, %d]", t, MAX_RAD);
    if (d.n_rad > 0) {
        REQ(d.rad_class && d.counts_rad && finite_nonneg(d.counts_rad, d.n_rad), "toy %d: radial term needs rad_class and counts_rad", t);
        for (int k = 0; k < d.n_species; ++k) REQ(d.rad_class[k] == 0 || d.rad_class[k] == 1, "toy %d: rad_class[%d] must be 0 or 1", t, k);
        REQ(d.r_fid > 0.0 && d.r_iv >= d.r_fid && d.att_len > 0.0, "toy %d: radial geometry invalid", t);
    }
    REQ(d.n_psd >= 0 && d.n_psd <= MAX_PSD, "toy %d: n_psd out of [0, %d]", t, MAX_PSD);
    if (d.quench) {
        for (int k = 0; k < d.n_species; ++k)
            REQ(std::isfinite(d.quench[k]) && d.quench[k] >= 0.0, "toy %d: quench[%d] must be finite and >= 0", t, k);
        double xi[MAX_SETS];
        int set_of[KMAX];
        const int ng = quench_groups(d, xi, set_of);
        REQ(ng >= 1, "toy %d: more than %d quenching groups", t, MAX_SETS);
        if (ng > 1) {
            REQ(d.n_rad2d + d.n_psd2d == 0, "toy %d: quenching groups with 2D histograms are not supported", t);
            const int ncs = (d.n_grid + BCOLS - 1) / BCOLS * BCOLS;
            REQ((ng - 1) * ncs + d.n_grid <= MAX_CB * BCOLS, "toy %d: %d quenching groups of %d columns exceed %d",
                t, ng, d.n_grid, MAX_CB * BCOLS);
        }
    }
    REQ(d.n_eslice >= 0 && d.n_eslice <= MAX_ES, "toy %d: n_eslice %d out of [0, %d]", t, d.n_eslice, MAX_ES);
    if (d.n_eslice > 0) {
        REQ(d.eslice_edges, "toy %d: n_eslice > 0 needs eslice_edges", t);
        REQ(d.eslice_edges[0] == 0 && d.eslice_edges[d.n_eslice] == (int)nw,
            "toy %d: energy slices must start at 0 and end at the window's %d bins", t, (int)nw);
        for (int q = 0; q < d.n_eslice; ++q)
            REQ(d.eslice_edges[q + 1] > d.eslice_edges[q], "toy %d: eslice_edges must rise strictly", t);
        REQ(d.n_eslice * d.n_rad <= MAX_RAD && d.n_eslice * d.n_psd <= MAX_PSD,
            "toy %d: energy slices x bins exceed %d", t, MAX_RAD);
        if (d.n_eslice > 1) REQ(d.n_rad2d + d.n_psd2d == 0, "toy %d: energy slices with 2D histograms are not supported", t);
    }
    REQ(d.n_rad2d >= 0 && d.n_psd2d >= 0 && d.n_rad2d <= NSL && d.n_psd2d <= NSL,
        "toy %d: n_rad2d, n_psd2d must lie in [0, %d]", t, NSL);
    REQ(d.joint2d == 0 || d.joint2d == 1, "toy %d: joint2d must be 0 or 1", t);
    REQ(std::isfinite(d.resp_skew) && std::isfinite(d.resp_kurt), "toy %d: resp_skew, resp_kurt must be finite", t);
    if (d.resp_skew != 0.0 || d.resp_kurt != 0.0)
        REQ(d.n_rad2d + d.n_psd2d == 0, "toy %d: the Gram-Charlier response is not supported with 2D histograms", t);
    if (d.joint2d) REQ(d.n_rad2d >= 1 && d.n_psd2d >= 1, "toy %d: the joint grid needs n_rad2d, n_psd2d >= 1", t);
    REQ(d.n_shell >= 0 && d.n_shell <= MAX_SETS, "toy %d: n_shell %d out of [0, %d]", t, d.n_shell, MAX_SETS);
    if (d.n_shell > 0) {   // the position-dependent response
        REQ(d.shell_ly && d.shell_frac, "toy %d: n_shell > 0 needs shell_ly and shell_frac", t);
        for (int r = 0; r < d.n_shell; ++r)
            REQ(std::isfinite(d.shell_ly[r]) && d.shell_ly[r] > 0.0, "toy %d: shell_ly[%d] must be > 0", t, r);
        REQ(finite_nonneg(d.shell_frac, (size_t)d.n_species * d.n_shell), "toy %d: shell_frac negative or not finite", t);
        REQ(d.n_rad2d + d.n_psd2d == 0, "toy %d: radial response shells with 2D histograms are not supported", t);
        double xi[MAX_SETS];
        int set_of[KMAX];
        REQ(quench_groups(d, xi, set_of) == 1, "toy %d: radial response shells need a single Birks multiplier", t);
        const int ncs = (d.n_grid + BCOLS - 1) / BCOLS * BCOLS;
        REQ((d.n_shell - 1) * ncs + d.n_grid <= MAX_CB * BCOLS, "toy %d: %d response shells of %d columns exceed %d",
            t, d.n_shell, d.n_grid, MAX_CB * BCOLS);
    }
    if (d.n_rad2d + d.n_psd2d > 0) {
        const int B2 = d.joint2d ? d.n_rad2d * d.n_psd2d : d.n_rad2d + d.n_psd2d;   // 2D slices
        const int n_sl = 1 + (d.tag_frac ? 1 : 0) + B2;
        REQ(n_sl <= NSL, "toy %d: %d slices (TFC spectra + 2D) exceed %d", t, n_sl, NSL);
        REQ(d.n_rad == 0 && d.n_psd == 0, "toy %d: 2D histograms replace the n_rad / n_psd terms", t);
        REQ(d.field2d && std::isfinite(d.field_amp) && d.field_amp >= 0.0 && d.field_amp < 1.0,
            "toy %d: 2D histograms need field2d and 0 <= field_amp < 1", t);
        for (size_t j = 0; j < (size_t)d.n_grid * B2; ++j)
            REQ(std::isfinite(d.field2d[j]) && std::fabs(d.field2d[j]) <= 1.0, "toy %d: field2d must lie in [-1, 1]", t);
        if (d.n_rad2d > 0) {
            const size_t nr = (size_t)(d.joint2d ? B2 : d.n_rad2d) * nw;   // the joint histogram in counts_rad2d
            REQ(d.rad_class && d.counts_rad2d && finite_nonneg(d.counts_rad2d, nr),
                "toy %d: energy x radius histogram needs rad_class and counts_rad2d", t);
            for (int k = 0; k < d.n_species; ++k) REQ(d.rad_class[k] == 0 || d.rad_class[k] == 1, "toy %d: rad_class[%d] must be 0 or 1", t, k);
            REQ(d.r_fid > 0.0 && d.r_iv >= d.r_fid && d.att_len > 0.0, "toy %d: radial geometry invalid", t);
        }
        if (d.n_psd2d > 0)
            REQ(d.psd2d_prob && finite_nonneg(d.psd2d_prob, (size_t)d.n_species * d.n_psd2d) &&
                    (d.joint2d || (d.counts_psd2d && finite_nonneg(d.counts_psd2d, (size_t)d.n_psd2d * nw))),
                "toy %d: energy x pulse-shape histogram needs psd2d_prob and counts_psd2d", t);
    }
    if (d.n_psd > 0)
        REQ(d.psd_prob && d.counts_psd && finite_nonneg(d.psd_prob, (size_t)d.n_species * d.n_psd) &&
                finite_nonneg(d.counts_psd, d.n_psd),
            "toy %d: pulse-shape term needs psd_prob and counts_psd", t);
#undef REQ
    return BX_OK;
}

static int alloc_dev(bx_model* m, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return bx_set_error(e == cudaErrorMemoryAllocation ? BX_ENOMEM : BX_ECUDA, "cudaMalloc(%zu): %s", bytes,
                            cudaGetErrorString(e));
    }
    m->allocs.push_back(*p);
    return BX_OK;
}

template <typename T>
static int upload(bx_model* m, const T* src, size_t n, const T** dst) {
    if (!src) {
        *dst = nullptr;
        return BX_OK;
    }
    void* p;
    int st = alloc_dev(m, &p, n * sizeof(T));
    if (st) return st;
    CU(cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, m->stream));
    *dst = static_cast<const T*>(p);
    return BX_OK;
}

static void free_model(bx_model* m) {
    if (!m) return;
    bx_fit_free(m);
    for (cudaEvent_t e : m->prof_ev) cudaEventDestroy(e);
    for (void* p : m->allocs) cudaFree(p);
    for (void* p : m->pinned) cudaFreeHost(p);
    delete m;
}

// n_est > 1: the toys are n_toys / n_est datasets of n_est energy estimators each (validated by
// bx_model_create_estimators); the workspace holds max_batch x n_est internal items.
static int model_create(const bx_model_desc* descs, int n_toys, const bx_options* opts, void* cuda_stream, int n_est,
                        bx_model** out) {
    if (!out) return bx_set_error(BX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs || n_toys < 1) return bx_set_error(BX_EINVAL, "need at least one model description");
    bx_options o{BX_FP32, 1, 8.0, 2.0};
    if (opts) o = *opts;
    if (o.precision != BX_FP64 && o.precision != BX_FP32 && o.precision != BX_TF32X3 && o.precision != BX_BF16X3)
        return bx_set_error(BX_EINVAL, "precision %d not supported (BX_FP64, BX_FP32, BX_BF16X3 or BX_TF32X3)",
                            o.precision);
    if (o.max_batch < 1) return bx_set_error(BX_EINVAL, "max_batch must be >= 1");
    if (o.band_sigmas == 0.0) o.band_sigmas = 8.0;
    if (o.watchdog_s == 0.0) o.watchdog_s = 2.0;
    if (!(o.band_sigmas >= 3.0 && o.band_sigmas <= 40.0)) return bx_set_error(BX_EINVAL, "band_sigmas out of [3, 40]");
    if (!(o.watchdog_s > 0.0 && o.watchdog_s <= 600.0)) return bx_set_error(BX_EINVAL, "watchdog_s out of (0, 600]");
    int n2d = 0;
    for (int t = 0; t < n_toys; ++t) {
        int st = validate_desc(descs[t], t);
        if (st) return st;
        n2d += descs[t].n_rad2d + descs[t].n_psd2d > 0 ? 1 : 0;
    }
    if (n2d != 0 && n2d != n_toys) return bx_set_error(BX_EINVAL, "toys of one model are either all 2D or none");
    for (int t = 0; t < n_toys; ++t) {
        double xi[MAX_SETS];
        int set_of[KMAX];
        if (quench_groups(descs[t], xi, set_of) > 1 && o.precision == BX_TF32X3)
            return bx_set_error(BX_EINVAL, "toy %d: quenching groups need BX_FP32 or BX_FP64", t);
        if (descs[t].n_eslice > 1 && o.precision == BX_TF32X3)
            return bx_set_error(BX_EINVAL, "toy %d: energy slices need BX_FP32 or BX_FP64", t);
        if (descs[t].n_shell > 0 && o.precision != BX_FP32 && o.precision != BX_FP64)
            return bx_set_error(BX_EINVAL, "toy %d: radial response shells need BX_FP32 or BX_FP64", t);
    }
    if (n2d && o.precision != BX_FP32 && o.precision != BX_BF16X3)
        return bx_set_error(BX_EINVAL, "2D histograms need BX_FP32 or BX_BF16X3");
    if (!n2d && o.precision == BX_BF16X3)
        return bx_set_error(BX_EINVAL, "BX_BF16X3 is the 2D models' response GEMM (the 1D models: BX_TF32X3)");
    for (int t = 0; t < n_toys; ++t) {   // the Gram-Charlier response: FP64 or FP32, density >= 0 within the band
        const double g1 = descs[t].resp_skew / 6.0, g2 = descs[t].resp_kurt / 24.0;
        if (g1 == 0.0 && g2 == 0.0) continue;
        if (o.precision != BX_FP64 && o.precision != BX_FP32)
            return bx_set_error(BX_EINVAL, "toy %d: the Gram-Charlier response needs BX_FP64 or BX_FP32", t);
        for (int j = 0; j <= 4000; ++j) {
            const double z = o.band_sigmas * (j / 2000.0 - 1.0), z2 = z * z;
            if (1.0 + g1 * z * (z2 - 3.0) + g2 * (z2 * (z2 - 6.0) + 3.0) < 0.0)
                return bx_set_error(BX_EINVAL, "toy %d: the Gram-Charlier density is negative at z = %.3f (within %g sigma)",
                                    t, z, o.band_sigmas);
        }
    }
    int dev = 0;
    CU(cudaGetDevice(&dev));
    int cc_major = 0, cc_minor = 0;
    CU(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    CU(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (cc_major != 10 || cc_minor != 3)
        return bx_set_error(BX_ECUDA, "device compute capability %d.%d: this library is built for sm_103a only",
                            cc_major, cc_minor);

    if (o.precision == BX_TF32X3) {
        // the tensor-core operand layout is verified once per process before first use
        static int tc_checked = 0;   // 0 unknown, 1 ok, -1 failed
        if (tc_checked == 0) {
            double err = 1.0;
            const int st = bx_selftest_tensor_core(&err);
            if (st) return st;
            tc_checked = err < 1e-5 ? 1 : -1;
        }
        if (tc_checked < 0)
            return bx_set_error(BX_ECUDA, "tensor-core self-test failed: TF32X3 path disabled, use BX_FP64");
    }
    bx_model* m = new bx_model();
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    m->n_toys = n_toys;
    m->precision = o.precision;
    m->cap = o.max_batch;
    m->n_est = n_est;
    m->n_data = n_toys / n_est;
    m->band = o.band_sigmas;
    m->watchdog_ns = (unsigned long long)(o.watchdog_s * 1e9);
    m->toys_h.resize(n_toys);
    int st = BX_OK;
    for (int t = 0; t < n_toys && !st; ++t) {
        const bx_model_desc& d = descs[t];
        Toy& T = m->toys_h[t];
        T = Toy{};
        T.K = d.n_species;
        T.N = d.n_grid;
        T.M = d.m_hi;
        T.m_lo = d.m_lo;
        T.nw = d.m_hi - d.m_lo;
        T.L = d.n_pileup;
        T.n_rad = d.n_rad;
        T.n_psd = d.n_psd;
        T.has_tag = d.tag_frac ? 1 : 0;
        T.n_r2 = d.n_rad2d;
        T.n_p2 = d.n_psd2d;
        T.b_r2 = 1 + T.has_tag;
        T.joint2 = d.joint2d;
        const int B2 = T.joint2 ? T.n_r2 * T.n_p2 : T.n_r2 + T.n_p2;   // 2D slices
        T.n_sl = (T.n_r2 + T.n_p2 > 0) ? T.b_r2 + B2 : 0;
        T.n_es = d.n_eslice > 1 ? d.n_eslice : 1;
        for (int q = 0; q < T.n_es; ++q) {
            T.es_lo[q] = T.m_lo + (d.n_eslice > 1 ? d.eslice_edges[q] : 0);
            T.es_hi[q] = T.m_lo + (d.n_eslice > 1 ? d.eslice_edges[q + 1] : T.nw);
        }
        T.nb = T.nw * (1 + T.has_tag) + T.n_es * (T.n_rad + T.n_psd) + B2 * T.nw;
        T.P = T.K + 7;
        T.n_tiles = (T.M + TM - 1) / TM;
        T.n_set = quench_groups(d, T.xi, T.set_of);
        T.n_shell = d.n_shell;
        if (T.n_shell > 0) {   // the sets are the radial shells, all with the one Birks multiplier
            T.n_set = T.n_shell;
            for (int c = 0; c < T.n_shell; ++c) {
                T.xi[c] = T.xi[0];
                T.lyf[c] = d.shell_ly[c];
                for (int k = 0; k < T.K; ++k) T.shw[c][k] = d.shell_frac[(size_t)k * d.n_shell + c];
            }
        }
        T.Ncs = T.n_set > 1 ? (T.N + BCOLS - 1) / BCOLS * BCOLS : T.N;
        T.Next = (T.n_set - 1) * T.Ncs + T.N;
        T.n_cb = (T.Next + BCOLS - 1) / BCOLS;
        T.n_kb = (T.N + KB - 1) / KB;
        T.dE = d.e_max / d.n_grid;
        T.w = d.width;
        T.gc1 = d.resp_skew / 6.0;
        T.gc2 = d.resp_kurt / 24.0;
        T.r_fid = d.r_fid;
        T.r_iv = d.r_iv;
        T.att_len = d.att_len;
        std::vector<double> cnt;
        cnt.insert(cnt.end(), d.counts_sub, d.counts_sub + T.nw);
        if (T.has_tag) cnt.insert(cnt.end(), d.counts_tag, d.counts_tag + T.nw);
        if (T.n_rad) cnt.insert(cnt.end(), d.counts_rad, d.counts_rad + (size_t)T.n_es * T.n_rad);
        if (T.n_psd) cnt.insert(cnt.end(), d.counts_psd, d.counts_psd + (size_t)T.n_es * T.n_psd);
        if (T.joint2) {
            cnt.insert(cnt.end(), d.counts_rad2d, d.counts_rad2d + (size_t)B2 * T.nw);
        } else {
            if (T.n_r2) cnt.insert(cnt.end(), d.counts_rad2d, d.counts_rad2d + (size_t)T.n_r2 * T.nw);
            if (T.n_p2) cnt.insert(cnt.end(), d.counts_psd2d, d.counts_psd2d + (size_t)T.n_p2 * T.nw);
        }
        if ((st = upload(m, d.shapes, (size_t)T.K * T.N, &T.shapes))) break;
        if ((st = upload(m, d.stop_pow, (size_t)T.N, &T.stop_pow))) break;
        {
            std::vector<float2> s32v(T.N);
            for (int i = 0; i < T.N; ++i) {
                const float h = (float)d.stop_pow[i];
                s32v[i] = make_float2(h, (float)(d.stop_pow[i] - (double)h));
            }
            if ((st = upload(m, s32v.data(), s32v.size(), &T.stop32))) break;
            CU(cudaStreamSynchronize(m->stream));
        }
        if ((st = upload(m, d.tag_frac, (size_t)T.K, &T.tag))) break;
        if ((st = upload(m, d.pileup, (size_t)T.L, &T.g))) break;
        if ((st = upload(m, cnt.data(), cnt.size(), &T.cnt))) break;
        {
            std::vector<float2> c32(cnt.size());
            for (size_t j = 0; j < cnt.size(); ++j) {
                const float h = (float)cnt[j];
                c32[j] = make_float2(h, (float)(cnt[j] - (double)h));
            }
            if ((st = upload(m, c32.data(), c32.size(), &T.cnt32))) break;
            CU(cudaStreamSynchronize(m->stream));   // c32 is released at the end of this scope
        }
        if ((st = upload(m, T.n_rad ? d.rad_class : nullptr, (size_t)T.K, &T.rad_class))) break;
        if ((st = upload(m, T.n_psd ? d.psd_prob : nullptr, (size_t)T.K * T.n_psd, &T.psd))) break;
        if (T.n_sl) {
            // template modulation per (column, slice) and its per-species column sums
            std::vector<float> ut((size_t)T.N * NSL, 0.f), utl((size_t)T.N * NSL, 0.f);
            std::vector<double> U2((size_t)T.K * NSL, 0.0);
            for (int i = 0; i < T.N; ++i)
                for (int b = 0; b < T.n_sl; ++b) {
                    const double u = b < T.b_r2 ? 1.0 : 1.0 + d.field_amp * d.field2d[(size_t)i * B2 + (b - T.b_r2)];
                    const float uh = (float)u;
                    ut[(size_t)i * NSL + b] = uh;
                    utl[(size_t)i * NSL + b] = (float)(u - (double)uh);
                    for (int k = 0; k < T.K; ++k) U2[(size_t)k * NSL + b] += d.shapes[(size_t)k * T.N + i] * u;
                }
            // template classes per slice set: species with the same slice probabilities (radial
            // class, pulse-shape row, or both on the joint grid) share one class
            for (int sset = 0; sset < 4; ++sset) {
                T.n_cls[sset] = 0;
                for (int k = 0; k < T.K; ++k) {
                    auto same = [&](int a, int b) {
                        const bool rad = (sset == 2) && T.n_r2 > 0;
                        const bool psd = (sset == 3 || (sset == 2 && T.joint2)) && T.n_p2 > 0;
                        if (rad && d.rad_class[a] != d.rad_class[b]) return false;
                        if (psd && memcmp(d.psd2d_prob + (size_t)a * T.n_p2, d.psd2d_prob + (size_t)b * T.n_p2,
                                          sizeof(double) * T.n_p2) != 0)
                            return false;
                        return true;
                    };
                    int c = 0;
                    while (c < T.n_cls[sset] && !same(k, T.cls_rep[sset][c])) ++c;
                    if (c == T.n_cls[sset]) T.cls_rep[sset][T.n_cls[sset]++] = k;
                    T.cls_of[sset][k] = c;
                }
            }
            std::vector<float> utmax(NSL, 0.f);
            for (int i = 0; i < T.N; ++i)
                for (int b = 0; b < T.n_sl; ++b) utmax[b] = std::max(utmax[b], std::fabs(ut[(size_t)i * NSL + b]));
            for (int b = 0; b < NSL; ++b) utmax[b] *= 1.0f + 1e-6f;   // above the double-float values too
            if ((st = upload(m, utmax.data(), utmax.size(), &T.utmax))) break;
            if ((st = upload(m, ut.data(), ut.size(), &T.ut))) break;
            if ((st = upload(m, utl.data(), utl.size(), &T.utl))) break;
            if ((st = upload(m, U2.data(), U2.size(), &T.U2))) break;
            if ((st = upload(m, T.n_p2 ? d.psd2d_prob : nullptr, (size_t)T.K * T.n_p2, &T.psd2))) break;
            if (T.n_r2 && !T.rad_class && (st = upload(m, d.rad_class, (size_t)T.K, &T.rad_class))) break;
            // the host copies are released when the model stream has consumed them
            CU(cudaStreamSynchronize(m->stream));
        }
        void *s32, *stiles, *g32, *gg;
        if ((st = alloc_dev(m, &s32, 2 * (size_t)T.K * T.N * sizeof(float)))) break;   // hi, then lo
        if ((st = alloc_dev(m, &stiles, (size_t)T.n_kb * 3 * US * KB * sizeof(float)))) break;
        if ((st = alloc_dev(m, &g32, (size_t)T.L * sizeof(float)))) break;
        if ((st = alloc_dev(m, &gg, (size_t)T.n_es * T.M * (sizeof(double) + sizeof(float))))) break;
        T.shapes32 = static_cast<float*>(s32);
        T.shapes32l = static_cast<float*>(s32) + (size_t)T.K * T.N;
        T.S_tiles = static_cast<float*>(stiles);
        T.g32 = static_cast<float*>(g32);
        T.Gg = static_cast<double*>(gg);
        T.Gg32 = reinterpret_cast<float*>(static_cast<double*>(gg) + (size_t)T.n_es * T.M);
        cudaError_t e = launch_setup_toy(T, static_cast<float*>(s32), const_cast<float*>(T.shapes32l),
                                         static_cast<float*>(stiles),
                                         static_cast<float*>(g32), static_cast<double*>(gg), m->stream);
        if (e != cudaSuccess) st = bx_set_error(BX_ECUDA, "set-up kernel: %s", cudaGetErrorString(e));
        m->Kmax = std::max(m->Kmax, T.K);
        m->Nmax = std::max(m->Nmax, T.Next);
        m->Mmax = std::max(m->Mmax, T.M);
        m->nwmax = std::max(m->nwmax, T.nw);
        m->nbmax = std::max(m->nbmax, T.nb);
        m->Lmax = std::max(m->Lmax, T.L);
        m->max_tiles = std::max(m->max_tiles, T.n_tiles);
        m->max_cb = std::max(m->max_cb, T.n_cb);
        m->any_tag |= T.has_tag;
        m->any_cols |= (T.n_rad > 0 || T.n_psd > 0) ? 1 : 0;
        m->is2d |= T.n_sl > 0 ? 1 : 0;
        if (T.n_sl > 0) m->ncs2d = std::max(m->ncs2d, T.n_cls[0] + T.n_cls[1] + T.n_cls[2] + T.n_cls[3]);
    }
    if (st) {
        cudaStreamSynchronize(m->stream);
        free_model(m);
        return st;
    }
    m->Pi = m->Kmax + 7;
    m->P = m->Pi + 4 * (m->n_est - 1);
    const int cap = m->cap * m->n_est;   // internal items
    Work& w = m->w;
    w = Work{};
    w.cap = cap;
    w.Npad = ((m->Nmax + 127) / 128) * 128;
    w.Mpad = ((m->Mmax + 127) / 128) * 128;
    w.nbmax = m->nbmax;
    w.pstride = m->Pi;
    w.precision = m->precision;
    w.lam_pairs = m->precision == BX_FP32;
    w.multi_set = 0;
    w.nes = 1;
    w.gc = 0;
    w.shells = 0;
    for (const Toy& T : m->toys_h) {
        w.shells |= T.n_shell > 0 ? 1 : 0;
        w.multi_set |= (T.n_set > 1 || T.n_shell > 0) ? 1 : 0;
        w.nes = std::max(w.nes, T.n_es);
        w.gc |= (T.gc1 != 0.0 || T.gc2 != 0.0) ? 1 : 0;
    }
    w.band = m->band;
    w.watchdog_ns = m->watchdog_ns;
    w.max_tiles = m->max_tiles;
    w.max_cb = m->max_cb;
    w.tr_kb = w.Npad / KB;
    w.row_kb = w.Mpad / KB;
    w.win_kb = (m->nwmax + KB - 1) / KB;
    w.win_tiles = (m->nwmax + TM - 1) / TM;
    w.Lmax = m->Lmax;
    w.ncs2d = m->ncs2d;
    if (!m->is2d) {   // the assembly stage holds one item's spectra and columns in shared memory
        size_t need = 0, avail = 0;
        const cudaError_t e = mid_smem_budget(w, m->Mmax, m->nwmax, m->Lmax, &need, &avail);
        const int bad = e != cudaSuccess ? 1 : need > avail ? 2 : 0;
        if (bad) {
            cudaStreamSynchronize(m->stream);
            const int nwm = m->nwmax, Mm = m->Mmax, Lm = m->Lmax, np = w.Npad;
            free_model(m);
            if (bad == 1) return bx_set_error(BX_ECUDA, "assembly kernel attributes: %s", cudaGetErrorString(e));
            return bx_set_error(BX_EINVAL,
                                "the assembly stage needs %zu B of shared memory per item (window %d, axis %d, "
                                "pile-up %d, %d columns); the device allows %zu B: use a smaller window, axis, "
                                "pile-up spectrum or grid",
                                need, nwm, Mm, Lm, np, avail);
        }
    }
    const size_t tv = m->precision == BX_FP64 ? sizeof(double) : sizeof(float);
    const bool species = m->precision == BX_TF32X3;
    struct A {
        void** p;
        size_t bytes;
    } plan[] = {
        {(void**)&w.toys, sizeof(Toy) * n_toys},
        {(void**)&w.toy_of, sizeof(int) * cap},
        {(void**)&w.col64, sizeof(Col64) * cap * w.Npad},
        {(void**)&w.colq, sizeof(double2) * cap * w.Npad},
        {(void**)&w.colf, sizeof(float4) * cap * w.Npad},
        {(void**)&w.colg, sizeof(ColG) * cap * w.Npad},
        {(void**)&w.colS, sizeof(double2) * cap * w.Npad},
        {(void**)&w.colS32, sizeof(float4) * cap * w.Npad},
        {(void**)&w.colAl, sizeof(float) * cap * w.Npad},
        {(void**)&w.aW, sizeof(double) * cap * w.nes * w.Npad},
        {(void**)&w.colr, sizeof(int2) * cap * w.Npad},
        {(void**)&w.lam, sizeof(double) * cap * 2 * w.Mpad},
        {(void**)&w.apart, m->any_cols && !species ? 2 * sizeof(float) * cap * m->max_tiles * w.nes * w.Npad : 16},
        {(void**)&w.tile_cols, sizeof(int2) * cap * MAX_SETS * MAX_TILES},
        {(void**)&w.cb_rows, sizeof(int2) * cap * MAX_CB},
        {(void**)&w.v, species ? 2 * tv * cap * w.Mpad * US : 16},   // hi, lo planes
        {(void**)&w.rowW, tv * cap * (2 + w.nes) * w.Mpad},
        {(void**)&w.coef, sizeof(double) * cap * (2 + w.nes) * KMAX},
        {(void**)&w.gmid, sizeof(double) * cap * PMAX},
        {(void**)&w.gpart, sizeof(double) * cap * MAX_CB * GPN},
        {(void**)&w.nll, sizeof(double) * cap},
        {(void**)&w.mu, sizeof(double) * cap * m->nbmax},
        {(void**)&w.status, sizeof(int) * cap},
        {(void**)&w.err, sizeof(unsigned)},
        {(void**)&w.units, sizeof(unsigned long long)},
        {(void**)&w.coef2d, m->is2d ? sizeof(float) * cap * 4 * KMAX * NSL : 16},
        {(void**)&w.tr2d, m->is2d ? sizeof(float) * cap * (w.Npad / KB) * 3 * NSL * KB : 16},
        {(void**)&w.trmax2d, m->is2d ? sizeof(unsigned) * cap * NSL : 16},
        {(void**)&w.alpha2d, m->is2d ? sizeof(float2) * cap * 4 * KMAX : 16},
        {(void**)&w.qcls2d, m->is2d ? sizeof(float2) * cap * NSL * KMAX : 16},
        {(void**)&w.wcls2d, m->is2d ? sizeof(float2) * cap * m->ncs2d * w.Npad : 16},
        {(void**)&w.y2d, m->is2d ? sizeof(float) * cap * (w.Mpad / KB) * 3 * NSL * KB : 16},
        {(void**)&w.w2d, m->is2d ? sizeof(float) * cap * ((m->nwmax + KB - 1) / KB) * 2 * NSL * KB : 16},
        {(void**)&w.wt2d, m->is2d ? sizeof(float) * cap * (w.Mpad / KB) * 2 * NSL * KB : 16},
        {(void**)&w.nll2d, m->is2d ? sizeof(double) * cap * MAX_TILES * 2 : 16},
        {(void**)&w.geps2d, m->is2d ? sizeof(double) * cap * MAX_TILES : 16},
        {(void**)&w.gpart2d, m->is2d ? sizeof(double) * cap * MAX_CB * (GPN + 1) : 16},
        {(void**)&m->theta_d, sizeof(double) * m->cap * m->P},
        {(void**)&m->nll_d, sizeof(double) * m->cap},
        {(void**)&m->grad_d, sizeof(double) * m->cap * m->P},
        {(void**)&m->est_theta, m->n_est > 1 ? sizeof(double) * cap * m->Pi : 16},
        {(void**)&m->est_nll, m->n_est > 1 ? sizeof(double) * cap : 16},
        {(void**)&m->est_grad, m->n_est > 1 ? sizeof(double) * cap * m->Pi : 16},
        {(void**)&m->est_skip, m->n_est > 1 ? (size_t)cap : 16},
    };
    for (auto& a : plan)
        if ((st = alloc_dev(m, a.p, a.bytes))) break;
    if (!st) {
        cudaError_t e = cudaMemcpyAsync((void*)w.toys, m->toys_h.data(), sizeof(Toy) * n_toys, cudaMemcpyHostToDevice,
                                        m->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.err, 0, sizeof(unsigned), m->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.units, 0, sizeof(unsigned long long), m->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync((void*)w.toy_of, 0, sizeof(int) * cap, m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) st = bx_set_error(BX_ECUDA, "model upload: %s", cudaGetErrorString(e));
    }
    if (st) {
        free_model(m);
        return st;
    }
    m->toy_cached.assign(cap, 0);
    *out = m;
    return BX_OK;
}

extern "C" void bx_model_destroy(bx_model* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    free_model(m);
}

extern "C" int bx_model_set_stream(bx_model* m, void* s) {
    if (!m) return bx_set_error(BX_EINVAL, "model is NULL");
    m->stream = static_cast<cudaStream_t>(s);
    return BX_OK;
}

extern "C" int bx_model_n_params(const bx_model* m) { return m ? m->P : 0; }

extern "C" int bx_model_create(const bx_model_desc* descs, int n_toys, const bx_options* opts, void* cuda_stream,
                               bx_model** out) {
    return model_create(descs, n_toys, opts, cuda_stream, 1, out);
}

// The estimators of one dataset see the same events: the same species shapes on the same grid,
// stopping power, tag fractions and quenching; only estimator 0 carries the radial and
// pulse-shape terms, and none carries 2D histograms or energy slices.
static int validate_estimators(const bx_model_desc* d, int n_data, int n_est) {
    if (n_data < 1 || n_est < 1 || n_est > MAX_EST)
        return bx_set_error(BX_EINVAL, "need n_data >= 1 and 1 <= n_est <= %d", MAX_EST);
    for (int t = 0; t < n_data; ++t) {
        const bx_model_desc& a = d[(size_t)t * n_est];
        for (int e = 0; e < n_est; ++e) {
            const bx_model_desc& b = d[(size_t)t * n_est + e];
            if (b.n_rad2d + b.n_psd2d > 0 || b.n_eslice > 1 || (n_est > 1 && b.n_shell > 0))
                return bx_set_error(BX_EINVAL, "dataset %d estimator %d: estimators take no 2D histograms, energy "
                                               "slices or radial response shells", t, e);
            if (e == 0) continue;
            if (b.n_rad > 0 || b.n_psd > 0)
                return bx_set_error(BX_EINVAL, "dataset %d estimator %d: the radial and pulse-shape terms belong to "
                                               "estimator 0", t, e);
            const size_t kn = (size_t)a.n_species * a.n_grid;
            const bool same = b.n_grid == a.n_grid && b.e_max == a.e_max && b.n_species == a.n_species &&
                              b.shapes && a.shapes && !memcmp(b.shapes, a.shapes, kn * sizeof(double)) && b.stop_pow &&
                              a.stop_pow && !memcmp(b.stop_pow, a.stop_pow, (size_t)a.n_grid * sizeof(double)) &&
                              (!a.tag_frac) == (!b.tag_frac) &&
                              (!a.tag_frac || !memcmp(a.tag_frac, b.tag_frac, (size_t)a.n_species * sizeof(double))) &&
                              (!a.quench) == (!b.quench) &&
                              (!a.quench || !memcmp(a.quench, b.quench, (size_t)a.n_species * sizeof(double)));
            if (!same)
                return bx_set_error(BX_EINVAL, "dataset %d estimator %d: grid, species shapes, stopping power, tag "
                                               "fractions and quenching must equal estimator 0's", t, e);
        }
    }
    return BX_OK;
}

extern "C" int bx_model_create_estimators(const bx_model_desc* descs, int n_data, int n_est, const bx_options* opts,
                                          void* cuda_stream, bx_model** out) {
    if (!out) return bx_set_error(BX_EINVAL, "out is NULL");
    *out = nullptr;
    if (!descs) return bx_set_error(BX_EINVAL, "need at least one model description");
    int st = validate_estimators(descs, n_data, n_est);
    if (st) return st;
    return model_create(descs, n_data * n_est, opts, cuda_stream, n_est, out);
}

int bx_fwd_tile_variants(const bx_model* m) { return m->precision == BX_FP32 && !m->is2d ? 2 : 1; }
void bx_set_fwd_tile(bx_model* m, int variant) { m->w.fwd_wpc = variant == 1 ? 1 : 2; }

int bx_public_P(const bx_model* m, int t) { return m->toys_h[(size_t)t * m->n_est].P + 4 * (m->n_est - 1); }

extern "C" int bx_model_n_bins(const bx_model* m, int toy) {
    if (!m || toy < 0 || toy >= m->n_data) return 0;
    int nb = 0;
    for (int e = 0; e < m->n_est; ++e) nb += m->toys_h[(size_t)toy * m->n_est + e].nb;
    return nb;
}

// Read and clear the sticky device error word (synchronises the stream).
int bx_take_device_error(bx_model* m) {
    unsigned err = 0;
    CU(cudaStreamSynchronize(m->stream));
    CU(cudaMemcpy(&err, m->w.err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) {
        CU(cudaMemset(m->w.err, 0, sizeof(unsigned)));
        return bx_set_error(BX_ETIMEOUT, "a device-side wait exceeded its time budget (error word 0x%x)", err);
    }
    return BX_OK;
}

extern "C" int bx_model_status(bx_model* m) {
    if (!m) return bx_set_error(BX_EINVAL, "model is NULL");
    return bx_take_device_error(m);
}

// ------------------------------------------------------------------ evaluation

// Public items j = 0..n-1 of datasets toy_idx[j]; with E estimators internal item j E + e is
// estimator e of dataset toy_idx[j] (toy toy_idx[j] E + e).  m->toy_tmp holds the public list.
int bx_set_items(bx_model* m, int n, const int* toy_idx) {
    if (n < 1 || n > m->cap) return bx_set_error(BX_EINVAL, "n = %d out of [1, max_batch = %d]", n, m->cap);
    std::vector<int>& tmp = m->toy_tmp;
    tmp.assign(n, 0);
    if (toy_idx)
        for (int j = 0; j < n; ++j) {
            if (toy_idx[j] < 0 || toy_idx[j] >= m->n_data)
                return bx_set_error(BX_EINVAL, "toy_idx[%d] = %d out of [0, %d)", j, toy_idx[j], m->n_data);
            tmp[j] = toy_idx[j];
        }
    const int E = m->n_est;
    std::vector<int> internal((size_t)n * E);
    for (int j = 0; j < n; ++j)
        for (int e = 0; e < E; ++e) internal[(size_t)j * E + e] = tmp[j] * E + e;
    if (!std::equal(internal.begin(), internal.end(), m->toy_cached.begin())) {
        // pageable source: the copy has consumed the list when the call returns
        CU(cudaMemcpyAsync((void*)m->w.toy_of, internal.data(), sizeof(int) * internal.size(), cudaMemcpyHostToDevice,
                           m->stream));
        std::copy(internal.begin(), internal.end(), m->toy_cached.begin());
    }
    return BX_OK;
}

static int prof_mark(bx_model* m, int stage) {
    if (!m->prof_on) return BX_OK;
    if (stage == 0 && m->prof_used + (BX_STAGES + 1) > m->prof_ev.size()) {
        for (int j = 0; j < BX_STAGES + 1; ++j) {
            cudaEvent_t e;
            CU(cudaEventCreate(&e));
            m->prof_ev.push_back(e);
        }
    }
    CU(cudaEventRecord(m->prof_ev[m->prof_used + stage], m->stream));
    if (stage == BX_STAGES) m->prof_used += BX_STAGES + 1;
    return BX_OK;
}

static int enqueue_items(bx_model* m, int n, const double* theta_dev, int tstride, int want_grad, int want_mu,
                         double* nll_dev, double* grad_dev) {
    Work w = m->w;
    w.theta = theta_dev;
    w.tstride = tstride;
    w.n_items = n;
    cudaStream_t s = m->stream;
    int st;
    BxRange eval_range("bx_eval");
    if ((st = prof_mark(m, 0))) return st;
    { BxRange r("bx_prep"); CU(launch_prep(w, n, s)); }
    if ((st = prof_mark(m, 1))) return st;
    if (m->is2d) {
        { BxRange r("bx_forward_2d"); CU(launch_eval2d(w, n, want_grad, want_mu, 1, s)); }
        if ((st = prof_mark(m, 2))) return st;
        { BxRange r("bx_pileup_nll_2d"); CU(launch_eval2d(w, n, want_grad, want_mu, 2, s)); }
        if ((st = prof_mark(m, 3))) return st;
        if (want_grad) { BxRange r("bx_adjoint_2d"); CU(launch_eval2d(w, n, want_grad, want_mu, 3, s)); }
        if ((st = prof_mark(m, 4))) return st;
        { BxRange r("bx_gather"); CU(launch_gather2d(w, n, nll_dev, grad_dev, want_grad, s)); }
        return prof_mark(m, 5);
    }
    {
        BxRange r("bx_forward");
        if (m->precision == BX_FP64) CU(launch_fwd_f64(w, n, m->max_tiles, m->any_tag, m->any_cols, s));
        else if (m->precision == BX_FP32) CU(launch_fwd_f32(w, n, m->max_tiles, m->any_tag, m->any_cols, s));
        else CU(launch_fwd_tc(w, n, m->max_tiles, s));
    }
    if ((st = prof_mark(m, 2))) return st;
    { BxRange r("bx_assembly"); CU(launch_mid(w, n, m->Mmax, m->nwmax, m->Lmax, want_grad, want_mu, s)); }
    if ((st = prof_mark(m, 3))) return st;
    if (want_grad) { BxRange r("bx_adjoint"); CU(launch_bwd(w, n, m->max_cb, s)); }
    if ((st = prof_mark(m, 4))) return st;
    { BxRange r("bx_gather"); CU(launch_gather(w, n, nll_dev, grad_dev, want_grad, s)); }
    if ((st = prof_mark(m, 5))) return st;
    return BX_OK;
}

// n public items: with several estimators, expanded to n E internal items (k_est_split), evaluated
// by the regular kernels, and joined (k_est_join: -lnL summed, gradients mapped back).
int bx_enqueue_eval(bx_model* m, int n, const double* theta_dev, int tstride, int want_grad, int want_mu,
                    double* nll_dev, double* grad_dev) {
    if (m->n_est == 1) return enqueue_items(m, n, theta_dev, tstride, want_grad, want_mu, nll_dev, grad_dev);
    const int E = m->n_est;
    const unsigned char* pub_skip = m->w.skip;
    CU(launch_est_split(theta_dev, tstride, n, E, m->w.toys, m->w.toy_of, pub_skip, m->est_theta, m->Pi,
                        pub_skip ? m->est_skip : nullptr, m->stream));
    m->w.skip = pub_skip ? m->est_skip : nullptr;
    const int st = enqueue_items(m, n * E, m->est_theta, m->Pi, want_grad, want_mu, m->est_nll, m->est_grad);
    m->w.skip = pub_skip;
    if (st) return st;
    CU(launch_est_join(m->est_nll, m->est_grad, m->Pi, n, E, m->w.toys, m->w.toy_of, nll_dev, grad_dev, m->P,
                       want_grad, m->stream));
    return BX_OK;
}

extern "C" int bx_model_profile(bx_model* m, int enable, double* stage_ms, int* n_evals, double* entries) {
    if (!m) return bx_set_error(BX_EINVAL, "model is NULL");
    CU(cudaStreamSynchronize(m->stream));
    if (stage_ms) {
        for (int j = 0; j < BX_STAGES; ++j) stage_ms[j] = 0.0;
        for (size_t b = 0; b + BX_STAGES < m->prof_used; b += BX_STAGES + 1)
            for (int j = 0; j < BX_STAGES; ++j) {
                float ms = 0.f;
                CU(cudaEventElapsedTime(&ms, m->prof_ev[b + j], m->prof_ev[b + j + 1]));
                stage_ms[j] += ms;
            }
    }
    if (n_evals) *n_evals = (int)(m->prof_used / (BX_STAGES + 1));
    unsigned long long u = 0;
    CU(cudaMemcpy(&u, m->w.units, sizeof u, cudaMemcpyDeviceToHost));
    CU(cudaMemset(m->w.units, 0, sizeof u));
    if (entries) *entries = (double)u;
    m->prof_on = enable ? 1 : 0;
    m->w.count_units = m->prof_on;
    m->prof_used = 0;
    return BX_OK;
}

static int eval_host(bx_model* m, int n, const int* toy_idx, const double* theta, int want_grad, int want_mu,
                     double* nll, double* grad) {
    int st = bx_set_items(m, n, toy_idx);
    if (st) return st;
    const int P = m->P;
    for (int j = 0; j < n; ++j) {
        const int t = m->toy_tmp[j];
        for (int q = 0; q < bx_public_P(m, t); ++q)
            if (!std::isfinite(theta[(size_t)j * P + q]))
                return bx_set_error(BX_EINVAL, "theta[%d][%d] is not finite", j, q);
    }
    CU(cudaMemcpyAsync(m->theta_d, theta, sizeof(double) * n * P, cudaMemcpyHostToDevice, m->stream));
    if ((st = bx_enqueue_eval(m, n, m->theta_d, P, want_grad, want_mu, m->nll_d, m->grad_d))) return st;
    if (nll) CU(cudaMemcpyAsync(nll, m->nll_d, sizeof(double) * n, cudaMemcpyDeviceToHost, m->stream));
    if (grad && want_grad)
        CU(cudaMemcpyAsync(grad, m->grad_d, sizeof(double) * n * P, cudaMemcpyDeviceToHost, m->stream));
    if ((st = bx_take_device_error(m))) return st;
    if (nll)
        for (int j = 0; j < n; ++j)
            if (std::isinf(nll[j]))
                return bx_set_error(BX_EDOMAIN, "item %d: expected count <= 0 in a bin with data, or invalid "
                                                "response parameters", j);
    return BX_OK;
}

extern "C" int bx_nll(bx_model* m, const double* theta, double* nll) {
    if (!m || !theta || !nll) return bx_set_error(BX_EINVAL, "NULL argument");
    return eval_host(m, 1, nullptr, theta, 0, 0, nll, nullptr);
}

extern "C" int bx_nll_grad(bx_model* m, const double* theta, double* nll, double* grad) {
    if (!m || !theta || !nll || !grad) return bx_set_error(BX_EINVAL, "NULL argument");
    return eval_host(m, 1, nullptr, theta, 1, 0, nll, grad);
}

extern "C" int bx_expected(bx_model* m, int toy, const double* theta, double* mu) {
    if (!m || !theta || !mu) return bx_set_error(BX_EINVAL, "NULL argument");
    if (toy < 0 || toy >= m->n_data) return bx_set_error(BX_EINVAL, "toy %d out of range", toy);
    double nll;
    int st = eval_host(m, 1, &toy, theta, 0, 1, &nll, nullptr);
    if (st && st != BX_EDOMAIN) return st;
    size_t off = 0;
    for (int e = 0; e < m->n_est; ++e) {   // internal item e: estimator e, its bins after the previous ones
        const int nb = m->toys_h[(size_t)toy * m->n_est + e].nb;
        CU(cudaMemcpyAsync(mu + off, m->w.mu + (size_t)e * m->nbmax, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                           m->stream));
        off += nb;
    }
    CU(cudaStreamSynchronize(m->stream));
    return BX_OK;
}

extern "C" int bx_nll_batch(bx_model* m, int n, const int* toy_idx, const double* theta, double* nll, double* grad,
                            int device_ptrs) {
    if (!m) return bx_set_error(BX_EINVAL, "NULL argument");
    if (n == 0) return BX_OK;   // an empty batch: nothing to evaluate
    if (!theta || !nll) return bx_set_error(BX_EINVAL, "NULL argument");
    if (!device_ptrs) return eval_host(m, n, toy_idx, theta, grad != nullptr, 0, nll, grad);
    int st = bx_set_items(m, n, toy_idx);
    if (st) return st;
    return bx_enqueue_eval(m, n, theta, m->P, grad != nullptr, 0, nll, grad ? grad : m->grad_d);
}

extern "C" int bx_selftest_watchdog(double budget_s) {
    if (!(budget_s > 0.0 && budget_s <= 10.0)) return bx_set_error(BX_EINVAL, "budget_s out of (0, 10]");
    unsigned* derr;
    unsigned herr = 0;
    CU(cudaMalloc(&derr, sizeof(unsigned)));
    cudaError_t e = cudaMemset(derr, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = launch_watchdog_selftest(derr, (unsigned long long)(budget_s * 1e9), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost);
    cudaFree(derr);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "watchdog self-test: %s", cudaGetErrorString(e));
    if (herr & ERR_TIMEOUT) return bx_set_error(BX_ETIMEOUT, "watchdog self-test: the unsatisfiable wait timed out");
    return BX_OK;
}

extern "C" int bx_selftest_tensor_core(double* max_rel_err) {
    if (!max_rel_err) return bx_set_error(BX_EINVAL, "NULL argument");
    // A[128][32], B[16][32]: values spanning several binades so the hi/lo split matters
    std::vector<float> A(TM * KB), B(US * KB), D(TM * US);
    unsigned s = 12345u;
    auto rnd = [&]() { s = s * 1664525u + 1013904223u; return (float)((s >> 8) & 0xFFFFFF) / 16777216.0f; };
    for (auto& x : A) x = rnd() * std::pow(2.0f, -(float)(int)(rnd() * 6));
    for (auto& x : B) x = rnd();
    float *dA, *dB, *dD;
    unsigned* derr;
    CU(cudaMalloc(&dA, A.size() * 4));
    CU(cudaMalloc(&dB, B.size() * 4));
    CU(cudaMalloc(&dD, D.size() * 4));
    CU(cudaMalloc(&derr, 4));
    CU(cudaMemcpy(dA, A.data(), A.size() * 4, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dB, B.data(), B.size() * 4, cudaMemcpyHostToDevice));
    CU(cudaMemset(dD, 0, D.size() * 4));
    CU(cudaMemset(derr, 0, 4));
    cudaError_t e = launch_umma_selftest(dA, dB, dD, derr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost);
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(derr);
    if (e != cudaSuccess) return bx_set_error(BX_ECUDA, "tensor-core self-test: %s", cudaGetErrorString(e));
    if (herr) return bx_set_error(BX_ETIMEOUT, "tensor-core self-test: MMA completion wait timed out");
    double worst = 0.0;
    for (int r = 0; r < TM; ++r)
        for (int n = 0; n < US; ++n) {
            double ref = 0.0;
            for (int c = 0; c < KB; ++c) ref += (double)A[r * KB + c] * (double)B[n * KB + c];
            worst = std::max(worst, std::fabs(D[r * US + n] - ref) / std::fabs(ref));
        }
    *max_rel_err = worst;
    return BX_OK;
}
