// vx_rates.cu -- host side of the C ABI declared in include/vx_rates.h.
//
// create(): validates the config and builds, in FP64 on the host, everything that does not depend
// on the zone state: Gauss-Legendre nodes in cos(omega) and electron energy, the energy weights,
// and per (unordered bin pair, omega node) the half-width |q|/2, the lower electron energy E-, and
// the three coefficients that turn the node moments into K_I and K_II. These are uploaded once.
// eval()/adjoint(): host-side argument checks, then one persistent launch (optionally replayed from
// a cached CUDA graph: work-counter reset + kernel).
#include "../../include/vx_rates.h"
#include "vx_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

namespace {

thread_local std::string g_err = "";

vx_status fail(vx_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define VX_CU(call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA,      \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Gauss-Legendre nodes (ascending, exactly antisymmetric) and weights on [-1, 1] into caller arrays
// of n entries: Newton's method on P_n from the asymptotic first guess cos(pi (k - 1/4) / (n + 1/2)).
// Used by vx_rates_create and, without heap storage, by vx_rates_eval_noalloc.
void gauss_legendre(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= n / 2 + (n & 1); ++k) {
        double r = std::cos(pi * (k - 0.25) / (n + 0.5));
        double dP = 1.0;
        for (int it = 0; it < 60; ++it) {
            double Pm = 1.0, P = r;  // P_0, P_1
            for (int m = 2; m <= n; ++m) {
                double Pn = ((2 * m - 1) * r * P - (m - 1) * Pm) / m;
                Pm = P;
                P = Pn;
            }
            if (n == 1) { P = r; Pm = 1.0; }
            dP = n * (Pm - r * P) / (1.0 - r * r);
            double step = P / dP;
            r -= step;
            if (std::fabs(step) <= 1e-17) {
                // one more evaluation of the derivative at the converged root
                Pm = 1.0; P = r;
                for (int m = 2; m <= n; ++m) {
                    double Pn = ((2 * m - 1) * r * P - (m - 1) * Pm) / m;
                    Pm = P;
                    P = Pn;
                }
                if (n == 1) { P = r; Pm = 1.0; }
                dP = n * (Pm - r * P) / (1.0 - r * r);
                break;
            }
        }
        double wk = 2.0 / ((1.0 - r * r) * dP * dP);
        x[n - k] = r;
        x[k - 1] = -r;
        w[n - k] = wk;
        w[k - 1] = wk;
    }
    if (n & 1) x[n / 2] = 0.0;
}

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    gauss_legendre(n, x.data(), w.data());
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }


}  // namespace

namespace vx {
// The last-error text for the library's other translation units (the block-tridiagonal solver).
vx_status set_error(vx_status s, const char *msg) { return fail(s, "%s", msg); }
}  // namespace vx

struct vx_rates {
    int device = 0;
    int nsm = 0;
    vx_config cfg{};
    std::vector<double> eps, w;
    std::vector<int> species;
    vx::Common common{};
    vx::Nodes32 n32{};
    vx::Nodes64 n64{};
    float4 *d_tab32 = nullptr;
    double *d_tab64 = nullptr;
    unsigned long long *d_counter = nullptr;
    int *d_flag = nullptr;
    // launch shapes: one thread per bin pair; mixed kernels in two register budgets
    int ms = 1, block = 32, block_mixed = 32;
    int grid_mixed[2][2] = {{0, 0}, {0, 0}};  // [forward, tangents][larger, smaller register budget]
    int minb[2] = {2, 3};                      // chosen budget per kind (autotuned with VX_AUTOTUNE)
    bool tuned[2] = {false, false};
    float tune_ms[2][2] = {{0, 0}, {0, 0}};
    int grid_64 = 0;
    size_t smem_fwd = 0, smem_adj = 0, smem_64 = 0;
    int cc_major = 0, cc_minor = 0;
    // one cached executable graph per kernel kind: mixed forward, mixed tangents, FP64
    cudaGraphExec_t gexec[3] = {nullptr, nullptr, nullptr};
    // host-buffer calls: two staging slots, each with its stream and work counter
    struct {
        size_t bytes = 0;                     // per slot
        double *buf[2] = {nullptr, nullptr};
        unsigned long long *cnt = nullptr;    // [2]
        cudaStream_t st[2] = {nullptr, nullptr};
    } hs;
};

namespace vx {
const void *kernel_mixed(bool adj, int minb, int n_e, bool split, bool prec) {
    if (prec) {
        if (adj) return minb == 3 ? kernel_mixed_adj_b3p(n_e, split) : kernel_mixed_adj_b2p(n_e, split);
        return minb == 3 ? kernel_mixed_fwd_b3p(n_e, split) : kernel_mixed_fwd_b2p(n_e, split);
    }
    if (adj) return minb == 3 ? kernel_mixed_adj_b3(n_e, split) : kernel_mixed_adj_b2(n_e, split);
    return minb == 3 ? kernel_mixed_fwd_b3(n_e, split) : kernel_mixed_fwd_b2(n_e, split);
}
cudaError_t launch_mixed(bool adj, int minb, const Launch &L, int grid, int block, size_t smem, cudaStream_t s) {
    if (L.c.precise) {
        if (adj) return minb == 3 ? launch_mixed_adj_b3p(L, grid, block, smem, s) : launch_mixed_adj_b2p(L, grid, block, smem, s);
        return minb == 3 ? launch_mixed_fwd_b3p(L, grid, block, smem, s) : launch_mixed_fwd_b2p(L, grid, block, smem, s);
    }
    if (adj) return minb == 3 ? launch_mixed_adj_b3(L, grid, block, smem, s) : launch_mixed_adj_b2(L, grid, block, smem, s);
    return minb == 3 ? launch_mixed_fwd_b3(L, grid, block, smem, s) : launch_mixed_fwd_b2(L, grid, block, smem, s);
}
}  // namespace vx

extern "C" {

const char *vx_status_string(vx_status s) {
    switch (s) {
        case VX_OK: return "VX_OK";
        case VX_ERR_INVALID_ARG: return "VX_ERR_INVALID_ARG";
        case VX_ERR_CUDA: return "VX_ERR_CUDA";
        case VX_ERR_OOM: return "VX_ERR_OOM";
        case VX_ERR_NUMERIC: return "VX_ERR_NUMERIC";
        case VX_ERR_UNSUPPORTED: return "VX_ERR_UNSUPPORTED";
        case VX_ERR_TIMEOUT: return "VX_ERR_TIMEOUT";
    }
    return "VX_ERR_UNKNOWN";
}

const char *vx_last_error(void) { return g_err.c_str(); }

static vx_status validate_config(const vx_config *c) {
    if (!c) return fail(VX_ERR_INVALID_ARG, "config is NULL");
    if (c->n_bins < 2 || c->n_bins > VX_MAX_BINS - 1)  // N (N+1)/2 bin pairs must fit one CTA
        return fail(VX_ERR_INVALID_ARG, "n_bins %d outside 2..%d", c->n_bins, VX_MAX_BINS - 1);
    if (!c->eps) return fail(VX_ERR_INVALID_ARG, "eps is NULL");
    for (int i = 0; i < c->n_bins; ++i) {
        if (!(c->eps[i] > 0.0) || !std::isfinite(c->eps[i]))
            return fail(VX_ERR_INVALID_ARG, "eps[%d] must be finite and > 0", i);
        if (i && !(c->eps[i] > c->eps[i - 1]))
            return fail(VX_ERR_INVALID_ARG, "eps must be strictly increasing (index %d)", i);
        if (c->weights && (!(c->weights[i] > 0.0) || !std::isfinite(c->weights[i])))
            return fail(VX_ERR_INVALID_ARG, "weights[%d] must be finite and > 0", i);
    }
    if (c->n_mu < 2 || c->n_mu > VX_MAX_MU) return fail(VX_ERR_INVALID_ARG, "n_mu %d outside 2..%d", c->n_mu, VX_MAX_MU);
    if (c->n_e < 2 || c->n_e > VX_MAX_NE) return fail(VX_ERR_INVALID_ARG, "n_e %d outside 2..%d", c->n_e, VX_MAX_NE);
    if (c->n_species < 1 || c->n_species > VX_MAX_SPECIES || !c->species)
        return fail(VX_ERR_INVALID_ARG, "n_species must be 1..3 with a species list");
    for (int s = 0; s < c->n_species; ++s) {
        int sp = c->species[s];
        if (sp < 0 || sp > 2) return fail(VX_ERR_INVALID_ARG, "species[%d] = %d is not a vx_species", s, sp);
        for (int t = 0; t < s; ++t)
            if (c->species[t] == sp) return fail(VX_ERR_INVALID_ARG, "species %d listed twice", sp);
    }
    for (int s = 0; s < c->n_species; ++s) {
        int want = c->species[s] == VX_NU_E ? VX_NU_EBAR : c->species[s] == VX_NU_EBAR ? VX_NU_E : VX_NU_X;
        bool ok = false;
        for (int t = 0; t < c->n_species; ++t) ok |= c->species[t] == want;
        if (!ok) return fail(VX_ERR_INVALID_ARG, "species %d needs its partner %d in the list", c->species[s], want);
    }
    if (!std::isfinite(c->sin2w) || !std::isfinite(c->g2) || !std::isfinite(c->norm))
        return fail(VX_ERR_INVALID_ARG, "sin2w, g2 and norm must be finite");
    if (!(c->eta_fp64 >= 0.0) || !std::isfinite(c->eta_fp64))
        return fail(VX_ERR_INVALID_ARG, "eta_fp64 must be finite and >= 0");
    if (c->eta_fp64 > 40.0)  // keeps two paired denominators below the FP32 range
        return fail(VX_ERR_INVALID_ARG, "eta_fp64 must be <= 40");
    if (c->prec != VX_PREC_FP64 && c->prec != VX_PREC_MIXED) return fail(VX_ERR_INVALID_ARG, "unknown precision");
    if (c->flags & ~(VX_USE_GRAPH | VX_AUTOTUNE | VX_QUAD_SPLIT | VX_PRECISE)) return fail(VX_ERR_INVALID_ARG, "unknown flag bits");
    if ((c->flags & VX_PRECISE) && c->prec != VX_PREC_MIXED)
        return fail(VX_ERR_UNSUPPORTED, "VX_PRECISE is a mode of the mixed form");
    if ((c->flags & VX_QUAD_SPLIT) && (c->n_e % 2 != 0))
        return fail(VX_ERR_INVALID_ARG, "VX_QUAD_SPLIT needs an even n_e (got %d)", c->n_e);
    if ((c->flags & VX_QUAD_SPLIT) && c->prec != VX_PREC_MIXED)
        return fail(VX_ERR_UNSUPPORTED, "VX_QUAD_SPLIT is provided for the mixed form");
    return VX_OK;
}

vx_status vx_rates_create(const vx_config *cfg, vx_rates **out) {
    if (!out) return fail(VX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    vx_status st = validate_config(cfg);
    if (st != VX_OK) return st;
    vx_rates *h = new vx_rates();
    h->cfg = *cfg;
    const int N = cfg->n_bins, S = cfg->n_species, nmu = cfg->n_mu, ne = cfg->n_e;
    h->eps.assign(cfg->eps, cfg->eps + N);
    h->species.assign(cfg->species, cfg->species + S);
    h->cfg.eps = h->eps.data();
    h->cfg.species = h->species.data();
    // energy weights eps^2 d(eps): edges at geometric midpoints, outer edges half a log step out
    h->w.resize(N);
    for (int i = 0; i < N; ++i) {
        if (cfg->weights) { h->w[i] = cfg->weights[i]; continue; }
        double lo = i ? std::sqrt(h->eps[i - 1] * h->eps[i]) : h->eps[0] * std::sqrt(h->eps[0] / h->eps[1]);
        double hi = i < N - 1 ? std::sqrt(h->eps[i] * h->eps[i + 1]) : h->eps[N - 1] * std::sqrt(h->eps[N - 1] / h->eps[N - 2]);
        h->w[i] = h->eps[i] * h->eps[i] * (hi - lo);
    }
    h->cfg.weights = h->w.data();
    if (h->cfg.eta_fp64 == 0.0) h->cfg.eta_fp64 = 20.0;

    vx::Common &C = h->common;
    C.N = N; C.n_mu = nmu; C.n_e = ne; C.S = S;
    C.npair = N * (N + 1) / 2;
    C.g2 = cfg->g2; C.norm = cfg->norm; C.eta_sw = h->cfg.eta_fp64;
    for (int i = 0; i < N; ++i) { C.eps[i] = h->eps[i]; C.w[i] = h->w[i]; }
    for (int s = 0; s < S; ++s) {
        int sp = h->species[s];
        int want = sp == VX_NU_E ? VX_NU_EBAR : sp == VX_NU_EBAR ? VX_NU_E : VX_NU_X;
        for (int t = 0; t < S; ++t) if (h->species[t] == want) C.partner[s] = t;
        C.species[s] = sp;
        // couplings: (C_V +- C_A)^2, C_V = +-1/2 + 2 sin^2(theta_W), C_A = +-1/2 (nu_e / nu_x);
        // anti-nu_e sees the transposed kernel, so its two terms swap
        double cv = (sp == VX_NU_X ? -0.5 : 0.5) + 2.0 * cfg->sin2w, ca = sp == VX_NU_X ? -0.5 : 0.5;
        double b1 = (cv + ca) * (cv + ca), b2 = (cv - ca) * (cv - ca);
        if (sp == VX_NU_EBAR) std::swap(b1, b2);
        C.bI64[s] = b1; C.bII64[s] = b2;
        C.bI[s] = (float)b1; C.bII[s] = (float)b2;
    }
    {
        int p = 0;
        for (int i = 0; i < N; ++i)
            for (int j = i; j < N; ++j) C.pij[p++] = (uint16_t)((i << 8) | j);
    }
    std::vector<double> tm, wm, tk, wk;
    gauss_legendre(nmu, tm, wm);
    gauss_legendre(ne, tk, wk);
    for (int m = 0; m < nmu; ++m) {
        C.t64[m] = tm[m];
        C.t_hi[m] = (float)tm[m];
        C.t_lo[m] = (float)(tm[m] - (double)C.t_hi[m]);
    }
    for (int k = 0; k < ne; ++k) {
        double u = 1.0 + tk[k], v = 1.0 - tk[k];
        h->n64.u[k] = u; h->n64.v[k] = v;
        h->n64.cp[k] = wk[k] * u * u; h->n64.cm[k] = wk[k] * v * v; h->n64.c0[k] = wk[k] * u * v;
        h->n32.u[k] = (float)u; h->n32.v[k] = (float)v;
        h->n32.cp[k] = (float)h->n64.cp[k]; h->n32.cm[k] = (float)h->n64.cm[k]; h->n32.c0[k] = (float)h->n64.c0[k];
        double uh = std::nearbyint(u * 2048.0) / 2048.0;
        h->n32.uh[k] = (float)uh;
        h->n32.ul[k] = (float)(u - uh);
    }
    C.split = (cfg->flags & VX_QUAD_SPLIT) ? 1 : 0;
    C.precise = (cfg->flags & VX_PRECISE) ? 1 : 0;
    if (C.split) {
        std::vector<double> th, wh;
        gauss_legendre(ne / 2, th, wh);
        for (int k = 0; k < ne / 2; ++k) {
            h->n32.hp[k] = (float)(1.0 + th[k]);
            h->n32.hm[k] = (float)(1.0 - th[k]);
            h->n32.hw[k] = (float)wh[k];
        }
    }
    // per (unordered pair p, omega node m) tables: FP32 records pair-major (a thread's consecutive
    // units are adjacent), FP64 records omega-major
    const int np = C.npair;
    std::vector<float4> t32((size_t)nmu * np * 2);
    std::vector<double> t64((size_t)nmu * np * 5);
    const double pi = 3.14159265358979323846;
    double hmax = 0.0, q0hmax = 0.0;
    for (int m = 0; m < nmu; ++m) {
        const double t = tm[m], y = 1.0 - t;
        for (int p = 0; p < np; ++p) {
            const int i = C.pij[p] >> 8, j = C.pij[p] & 0xff;
            const double e = h->eps[i], ep = h->eps[j];
            const double d = e - ep, g = e * ep * (1.0 + t);
            const double q2 = d * d + 2.0 * g, q = std::sqrt(q2), hh = 0.5 * q;
            const double q0 = e + ep, s = 2.0 * e * ep * y;
            const double Em = s / (2.0 * (q0 + q));
            // K = G2 pi eps eps' y^2 / (16 |q|^2) sum_k w_k O_k P(tau_k), with the omega weight folded in
            const double pref = wm[m] * pi * e * ep * y * y / (16.0 * q2);
            const double kp = pref * 0.25 * (q + d) * (q + d), km = pref * 0.25 * (q - d) * (q - d), k0 = pref * 2.0 * g;
            hmax = std::fmax(hmax, hh);
            q0hmax = std::fmax(q0hmax, 0.5 * q0);
            float4 *r = &t32[((size_t)p * nmu + m) * 2];
            const float fh = (float)hh, fEm = (float)Em;
            r[0] = make_float4(fh, (float)(hh - fh), fEm, (float)(Em - fEm));
            r[1] = make_float4((float)kp, (float)km, (float)k0, C.t_hi[m]);
            double *r64 = &t64[((size_t)m * np + p) * 5];
            r64[0] = hh; r64[1] = Em; r64[2] = kp; r64[3] = km; r64[4] = k0;
        }
    }
    C.h_max = hmax;
    C.q0h_max = q0hmax;

    // launch shape: one thread per unordered bin pair
    C.ms = 1;
    h->ms = 1;
    h->block = round_up(np, 32);                           // FP64 kernel (<= 496 pairs)
    h->block_mixed = std::min(round_up(np * nmu, 32), VX_BLOCK_MIXED);  // (pair, omega) units

    auto cleanup = [&](vx_status s) { vx_rates_destroy(h); return s; };
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) { vx_status s = fail(VX_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(ce)); delete h; return s; }
    cudaDeviceProp prop;
    if ((ce = cudaGetDeviceProperties(&prop, h->device)) != cudaSuccess) {
        vx_status s = fail(VX_ERR_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(ce));
        delete h;
        return s;
    }
    h->nsm = prop.multiProcessorCount;
#define VX_CUC(call)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            return cleanup(fail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "%s: %s", #call, \
                                cudaGetErrorString(e_)));                                              \
    } while (0)
    VX_CUC(cudaMalloc(&h->d_tab32, t32.size() * sizeof(float4)));
    VX_CUC(cudaMalloc(&h->d_tab64, t64.size() * sizeof(double)));
    VX_CUC(cudaMalloc(&h->d_counter, sizeof(unsigned long long)));
    VX_CUC(cudaMalloc(&h->d_flag, sizeof(int)));
    VX_CUC(cudaMemcpy(h->d_tab32, t32.data(), t32.size() * sizeof(float4), cudaMemcpyHostToDevice));
    VX_CUC(cudaMemcpy(h->d_tab64, t64.data(), t64.size() * sizeof(double), cudaMemcpyHostToDevice));
    VX_CUC(cudaMemset(h->d_flag, 0, sizeof(int)));

    h->smem_fwd = vx::smem_mixed_bytes(N, S, false, h->block_mixed, C.precise != 0);
    h->smem_adj = vx::smem_mixed_bytes(N, S, true, h->block_mixed, C.precise != 0);
    h->smem_64 = vx::smem_fp64(C);
    h->cc_major = prop.major;
    h->cc_minor = prop.minor;
    struct K { const void *fn; size_t smem; int *grid; int block; };
    const bool sp = C.split != 0, pr = C.precise != 0;
    K ks[5] = {{vx::kernel_mixed(false, 2, ne, sp, pr), h->smem_fwd, &h->grid_mixed[0][0], h->block_mixed},
               {vx::kernel_mixed(false, 3, ne, sp, pr), h->smem_fwd, &h->grid_mixed[0][1], h->block_mixed},
               {vx::kernel_mixed(true, 2, ne, sp, pr), h->smem_adj, &h->grid_mixed[1][0], h->block_mixed},
               {vx::kernel_mixed(true, 3, ne, sp, pr), h->smem_adj, &h->grid_mixed[1][1], h->block_mixed},
               {vx::kernel_fp64_fwd(ne), h->smem_64, &h->grid_64, h->block}};
    for (K &k : ks) {
        // opt in to the dynamic size always: the 48 KB default bounds static + dynamic together
        VX_CUC(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
        int occ = 0;
        VX_CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.block, k.smem));
        if (occ < 1) return cleanup(fail(VX_ERR_UNSUPPORTED, "kernel does not fit on an SM (block %d, smem %zu)", k.block, k.smem));
        *k.grid = occ * h->nsm;
    }
#undef VX_CUC
    *out = h;
    return VX_OK;
}

long long vx_rates_entries_per_zone(const vx_rates *h) {
    return h ? (long long)h->common.N * h->common.N : 0;
}

static vx_status check_device_ptr(const void *p, const char *name, size_t align = 8) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VX_ERR_INVALID_ARG, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(VX_ERR_INVALID_ARG, "%s must be device memory", name);
    if (((uintptr_t)p) % align) return fail(VX_ERR_INVALID_ARG, "%s must be %zu-byte aligned", name, align);
    return VX_OK;
}

static vx_status validate_batch(const vx_rates *h, const vx_batch *b) {
    if (!h) return fail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (!b) return fail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_zones < 0) return fail(VX_ERR_INVALID_ARG, "n_zones < 0");
    if (b->n_rays < 0) return fail(VX_ERR_INVALID_ARG, "n_rays < 0");
    if (b->ray_offsets) {  // device memory: the partition itself is checked by the launch
        if (b->n_rays == 0 && b->n_zones > 0) return fail(VX_ERR_INVALID_ARG, "n_zones > 0 with no rays");
        vx_status s0 = check_device_ptr(b->ray_offsets, "ray_offsets", 4);
        if (s0 != VX_OK) return s0;
    }
    if (b->n_zones == 0) return VX_OK;
    vx_status s;
    if ((s = check_device_ptr(b->state, "state")) != VX_OK) return s;
    if ((s = check_device_ptr(b->J, "J")) != VX_OK) return s;
    if ((s = check_device_ptr(b->H, "H")) != VX_OK) return s;
    return VX_OK;
}

static vx_status validate_out(const vx_out *o, bool allow_phi) {
    if (!o) return fail(VX_ERR_INVALID_ARG, "out is NULL");
    vx_status s;
    if ((s = check_device_ptr(o->j0, "out.j0")) != VX_OK) return s;
    if ((s = check_device_ptr(o->chi0, "out.chi0")) != VX_OK) return s;
    if ((s = check_device_ptr(o->j1, "out.j1")) != VX_OK) return s;
    if ((s = check_device_ptr(o->chi1, "out.chi1")) != VX_OK) return s;
    if (o->phi) {
        if (!allow_phi) return fail(VX_ERR_INVALID_ARG, "phi output is not produced by this call");
        if ((s = check_device_ptr(o->phi, "out.phi")) != VX_OK) return s;
    }
    return VX_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// Launch through a graph (memset node + kernel node), re-using the executable graph when the
// topology is unchanged and only the parameters differ.
static vx_status launch_graph(vx_rates *h, int slot, const void *fn, void *param, int grid, int block,
                              size_t smem, cudaStream_t s) {
    cudaGraphExec_t &gexec = h->gexec[slot];
    cudaGraph_t g = nullptr;
    cudaGraphNode_t nm = nullptr, nk = nullptr;
    VX_CU(cudaGraphCreate(&g, 0));
    cudaMemsetParams mp{};
    mp.dst = h->d_counter;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;
    mp.height = 1;
    mp.pitch = 0;
    cudaError_t e = cudaGraphAddMemsetNode(&nm, g, nullptr, 0, &mp);
    cudaKernelNodeParams kp{};
    kp.func = (void *)fn;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.sharedMemBytes = (unsigned)smem;
    void *args[1] = {param};
    kp.kernelParams = args;
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&nk, g, &nm, 1, &kp);
    if (e == cudaSuccess) {
        bool fresh = true;
        if (gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(gexec, g, &info) == cudaSuccess) fresh = false;
            else {
                cudaGetLastError();
                cudaGraphExecDestroy(gexec);
                gexec = nullptr;
            }
        }
        if (fresh) e = cudaGraphInstantiate(&gexec, g, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(gexec, s);
    }
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(VX_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return VX_OK;
}

static void fill_launch(const vx_rates *h, const vx_batch *b, vx::Launch &L) {
    L.c = h->common;
    L.n32 = h->n32;
    L.tab32 = h->d_tab32;
    L.tab64 = h->d_tab64;
    L.Z = b->n_zones;
    L.off = b->ray_offsets;
    L.n_rays = b->n_rays;
    L.state = b->state; L.J = b->J; L.H = b->H;
    L.j0 = L.chi0 = L.j1 = L.chi1 = L.phi = nullptr;
    L.jac = L.grad_state = nullptr;
    L.g_j0 = L.g_chi0 = L.g_j1 = L.g_chi1 = nullptr;
    L.blocks = L.grad_J = L.grad_H = nullptr;
    L.counter = h->d_counter;
    L.flag = h->d_flag;
}

// ---- autotuner ------------------------------------------------------------------------------
// Picks, per kernel kind, the register budget (minb 2 or 3: see k_pair_mixed) that runs a sample of the
// first batch fastest: the first zones of the batch, about 48 per CTA, each variant once to warm
// up and once timed with CUDA events (four launches in all). The choice is kept in the handle and, when the environment
// variable VX_AUTOTUNE_CACHE names a file, in that JSON file under a key of the quadrature, the
// kernel kind and the device (SM count, compute capability). Tuning synchronises the stream, so
// the first tuned call must not be inside a stream capture; its sample outputs are overwritten
// by the real launch that follows.
static std::string tune_key(const vx_rates *h, bool adj) {
    char k[160];
    snprintf(k, sizeof k, "N=%d,n_mu=%d,n_e=%d,S=%d,kind=%s%s%s,sm=%d,cc=%d.%d", h->common.N, h->common.n_mu,
             h->common.n_e, h->common.S, adj ? "tangents" : "forward", h->common.split ? "+split" : "",
             h->common.precise ? "+precise" : "", h->nsm, h->cc_major, h->cc_minor);
    return k;
}

static std::vector<std::pair<std::string, std::string>> cache_read(const char *path) {
    std::vector<std::pair<std::string, std::string>> m;
    FILE *f = fopen(path, "r");
    if (!f) return m;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        char *q0 = strchr(line, '"');
        if (!q0) continue;
        char *q1 = strchr(q0 + 1, '"');
        char *br = q1 ? strchr(q1, '{') : nullptr;
        char *be = br ? strchr(br, '}') : nullptr;
        if (!q1 || !br || !be) continue;
        m.emplace_back(std::string(q0 + 1, q1), std::string(br, be + 1));
    }
    fclose(f);
    return m;
}

static void cache_write(const char *path, const std::string &key, const std::string &val) {
    auto m = cache_read(path);
    bool found = false;
    for (auto &kv : m)
        if (kv.first == key) { kv.second = val; found = true; }
    if (!found) m.emplace_back(key, val);
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;  // the cache is an optimisation: an unwritable path is not an error
    fprintf(f, "{\n");
    for (size_t i = 0; i < m.size(); ++i)
        fprintf(f, "  \"%s\": %s%s\n", m[i].first.c_str(), m[i].second.c_str(), i + 1 < m.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

static vx_status autotune(vx_rates *h, bool adj, const vx::Launch &L, cudaStream_t s) {
    const int kind = adj ? 1 : 0;
    if (!(h->cfg.flags & VX_AUTOTUNE) || h->tuned[kind]) return VX_OK;
    const char *path = getenv("VX_AUTOTUNE_CACHE");
    const std::string key = tune_key(h, adj);
    if (path && *path) {
        for (auto &kv : cache_read(path)) {
            int mb = 0;
            if (kv.first == key && sscanf(kv.second.c_str(), "{\"minb\": %d", &mb) == 1 && (mb == 2 || mb == 3)) {
                h->minb[kind] = mb;
                h->tuned[kind] = true;
                return VX_OK;
            }
        }
    }
    // ~48 zones per CTA of the larger grid: long enough that start-up and tail effects of the
    // persistent grid do not decide the comparison
    const long long sample = std::min<long long>(L.Z, 48LL * h->grid_mixed[kind][1]);
    if (sample < 8LL * h->grid_mixed[kind][1]) return VX_OK;  // too small to tell apart: keep the default
    vx::Launch Ls = L;
    Ls.Z = sample;
    Ls.off = nullptr;  // the sample is a prefix of the zones, not a partition by rays
    const size_t smem = adj ? h->smem_adj : h->smem_fwd;
    cudaEvent_t e0, e1;
    VX_CU(cudaEventCreate(&e0));
    VX_CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestb = h->minb[kind];
    for (int mb = 2; mb <= 3; ++mb) {
        const int grid = (int)std::min<long long>(h->grid_mixed[kind][mb - 2], sample);
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            VX_CU(cudaMemsetAsync(Ls.counter, 0, sizeof(unsigned long long), s));
            if (rep) VX_CU(cudaEventRecord(e0, s));
            VX_CU(vx::launch_mixed(adj, mb, Ls, grid, h->block_mixed, smem, s));
            if (rep) VX_CU(cudaEventRecord(e1, s));
        }
        VX_CU(cudaEventSynchronize(e1));
        VX_CU(cudaEventElapsedTime(&ms, e0, e1));
        h->tune_ms[kind][mb - 2] = ms;
        if (ms < best) { best = ms; bestb = mb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->minb[kind] = bestb;
    h->tuned[kind] = true;
    if (path && *path) {
        char v[128];
        snprintf(v, sizeof v, "{\"minb\": %d, \"ms_b2\": %.4f, \"ms_b3\": %.4f, \"zones\": %lld}", bestb,
                 h->tune_ms[kind][0], h->tune_ms[kind][1], sample);
        cache_write(path, key, v);
    }
    return VX_OK;
}

vx_status vx_rates_eval(vx_rates *h, const vx_batch *b, const vx_out *out, vx_stream stream) {
    vx_status st = validate_batch(h, b);
    if (st != VX_OK) return st;
    if (b->n_zones == 0) return VX_OK;
    if ((st = validate_out(out, true)) != VX_OK) return st;
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool graph = (h->cfg.flags & VX_USE_GRAPH) != 0;
    if (h->cfg.prec == VX_PREC_MIXED) {
        vx::Launch L{};
        fill_launch(h, b, L);
        L.j0 = out->j0; L.chi0 = out->chi0; L.j1 = out->j1; L.chi1 = out->chi1; L.phi = out->phi;
        if ((st = autotune(h, false, L, s)) != VX_OK) return st;
        const int mb = h->minb[0];
        int grid = (int)std::min<long long>(h->grid_mixed[0][mb - 2], b->n_zones);
        if (graph) return launch_graph(h, 0, vx::kernel_mixed(false, mb, h->common.n_e, h->common.split != 0, h->common.precise != 0), &L, grid, h->block_mixed, h->smem_fwd, s);
        VX_CU(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), s));
        VX_CU(vx::launch_mixed(false, mb, L, grid, h->block_mixed, h->smem_fwd, s));
    } else {
        vx::Launch64 L;
        L.c = h->common;
        L.n64 = h->n64;
        L.tab64 = h->d_tab64;
        L.Z = b->n_zones;
        L.off = b->ray_offsets;
        L.n_rays = b->n_rays;
        L.state = b->state; L.J = b->J; L.H = b->H;
        L.j0 = out->j0; L.chi0 = out->chi0; L.j1 = out->j1; L.chi1 = out->chi1; L.phi = out->phi;
        L.counter = h->d_counter;
        L.flag = h->d_flag;
        int grid = (int)std::min<long long>(h->grid_64, b->n_zones);
        if (graph) return launch_graph(h, 2, vx::kernel_fp64_fwd(h->common.n_e), &L, grid, h->block, h->smem_64, s);
        VX_CU(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), s));
        VX_CU(vx::launch_fp64_fwd(L, grid, h->block, h->smem_64, s));
    }
    return VX_OK;
}

vx_status vx_rates_adjoint(vx_rates *h, const vx_batch *b, const vx_out *grad_out, double *jac,
                           double *grad_state, const vx_out *fwd, vx_stream stream) {
    vx_status st = validate_batch(h, b);
    if (st != VX_OK) return st;
    if (h->cfg.prec != VX_PREC_MIXED) return fail(VX_ERR_UNSUPPORTED, "the adjoint is provided for the mixed form");
    if (!jac && !grad_state && !fwd) return fail(VX_ERR_INVALID_ARG, "no output requested");
    if (grad_state && !grad_out) return fail(VX_ERR_INVALID_ARG, "grad_state needs grad_out");
    if (b->n_zones == 0) return VX_OK;
    if (jac && (st = check_device_ptr(jac, "jac")) != VX_OK) return st;
    if (grad_state && (st = check_device_ptr(grad_state, "grad_state")) != VX_OK) return st;
    if (fwd && (st = validate_out(fwd, false)) != VX_OK) return st;
    if (grad_state) {
        const double *g[4] = {grad_out->j0, grad_out->chi0, grad_out->j1, grad_out->chi1};
        const char *nm[4] = {"grad_out.j0", "grad_out.chi0", "grad_out.j1", "grad_out.chi1"};
        for (int k = 0; k < 4; ++k)
            if (g[k] && (st = check_device_ptr(g[k], nm[k])) != VX_OK) return st;
    }
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    vx::Launch L{};
    fill_launch(h, b, L);
    if (fwd) { L.j0 = fwd->j0; L.chi0 = fwd->chi0; L.j1 = fwd->j1; L.chi1 = fwd->chi1; }
    L.jac = jac;
    L.grad_state = grad_state;
    if (grad_state) { L.g_j0 = grad_out->j0; L.g_chi0 = grad_out->chi0; L.g_j1 = grad_out->j1; L.g_chi1 = grad_out->chi1; }
    if ((st = autotune(h, true, L, s)) != VX_OK) return st;
    const int mb = h->minb[1];
    int grid = (int)std::min<long long>(h->grid_mixed[1][mb - 2], b->n_zones);
    if (h->cfg.flags & VX_USE_GRAPH)
        return launch_graph(h, 1, vx::kernel_mixed(true, mb, h->common.n_e, h->common.split != 0, h->common.precise != 0), &L, grid, h->block_mixed, h->smem_adj, s);
    VX_CU(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), s));
    VX_CU(vx::launch_mixed(true, mb, L, grid, h->block_mixed, h->smem_adj, s));
    return VX_OK;
}

vx_status vx_rates_spectral(vx_rates *h, const vx_batch *b, const vx_out *grad_out, double *grad_J,
                            double *grad_H, double *blocks, const vx_out *fwd, vx_stream stream) {
    vx_status st = validate_batch(h, b);
    if (st != VX_OK) return st;
    if (h->cfg.prec != VX_PREC_MIXED) return fail(VX_ERR_UNSUPPORTED, "the spectral derivatives are provided for the mixed form");
    if (!blocks && !grad_J && !grad_H && !fwd) return fail(VX_ERR_INVALID_ARG, "no output requested");
    if (!grad_J != !grad_H) return fail(VX_ERR_INVALID_ARG, "grad_J and grad_H go together");
    if (grad_J && !grad_out) return fail(VX_ERR_INVALID_ARG, "grad_J and grad_H need grad_out");
    if (b->n_zones == 0) return VX_OK;
    if (blocks && (st = check_device_ptr(blocks, "blocks")) != VX_OK) return st;
    if (grad_J && (st = check_device_ptr(grad_J, "grad_J")) != VX_OK) return st;
    if (grad_H && (st = check_device_ptr(grad_H, "grad_H")) != VX_OK) return st;
    if (fwd && (st = validate_out(fwd, false)) != VX_OK) return st;
    if (grad_J) {
        const double *g[4] = {grad_out->j0, grad_out->chi0, grad_out->j1, grad_out->chi1};
        const char *nm[4] = {"grad_out.j0", "grad_out.chi0", "grad_out.j1", "grad_out.chi1"};
        for (int k = 0; k < 4; ++k)
            if (g[k] && (st = check_device_ptr(g[k], nm[k])) != VX_OK) return st;
    }
    DeviceGuard dg(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    vx::Launch L{};
    fill_launch(h, b, L);
    if (fwd) { L.j0 = fwd->j0; L.chi0 = fwd->chi0; L.j1 = fwd->j1; L.chi1 = fwd->chi1; }
    L.blocks = blocks;
    L.grad_J = grad_J;
    L.grad_H = grad_H;
    if (grad_J) { L.g_j0 = grad_out->j0; L.g_chi0 = grad_out->chi0; L.g_j1 = grad_out->j1; L.g_chi1 = grad_out->chi1; }
    if ((st = autotune(h, false, L, s)) != VX_OK) return st;
    const int mb = h->minb[0];
    int grid = (int)std::min<long long>(h->grid_mixed[0][mb - 2], b->n_zones);
    if (h->cfg.flags & VX_USE_GRAPH)
        return launch_graph(h, 0, vx::kernel_mixed(false, mb, h->common.n_e, h->common.split != 0, h->common.precise != 0), &L, grid, h->block_mixed, h->smem_fwd, s);
    VX_CU(cudaMemsetAsync(h->d_counter, 0, sizeof(unsigned long long), s));
    VX_CU(vx::launch_mixed(false, mb, L, grid, h->block_mixed, h->smem_fwd, s));
    return VX_OK;
}

// ---- host-buffer calls ----------------------------------------------------------------------
// The batch is processed in chunks of zones through two staging slots of device memory owned by
// the handle (VX_HOST_SLOT_BYTES each, or VX_HOST_SLOT_MB MiB from the environment, allocated on
// first use). Each call sizes its chunk to what
// one zone of its inputs and outputs occupies (~70k zones with the Jacobian, ~13k with spectral
// blocks at 21 bins and 3 species). Each slot has its own stream and work counter, so the copies
// of one chunk overlap the kernel of the next. Host arrays should be pinned for the copies to be
// asynchronous; the calls return when every output is in host memory.
#ifndef VX_HOST_SLOT_BYTES
#define VX_HOST_SLOT_BYTES (640ull << 20)
#endif

static vx_status host_prepare(vx_rates *h) {
    auto &hs = h->hs;
    if (hs.buf[0]) return VX_OK;
    hs.bytes = VX_HOST_SLOT_BYTES;
    if (const char *mb = getenv("VX_HOST_SLOT_MB")) {
        const long long v = atoll(mb);
        if (v >= 1 && v <= (1ll << 20)) hs.bytes = (size_t)v << 20;
    }
    for (int k = 0; k < 2; ++k) {
        cudaError_t e = cudaMalloc(&hs.buf[k], hs.bytes);
        if (e != cudaSuccess)
            return fail(e == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "staging slot: %s", cudaGetErrorString(e));
        if (!hs.st[k]) VX_CU(cudaStreamCreateWithFlags(&hs.st[k], cudaStreamNonBlocking));
    }
    if (!hs.cnt) VX_CU(cudaMalloc(&hs.cnt, 2 * sizeof(unsigned long long)));
    return VX_OK;
}

// What one host-buffer call reads and writes (host pointers; NULL = absent).
struct HostIO {
    int kind;                 // 0 forward, 1 forward + tangents, 2 spectral derivatives
    const vx_out *fwd;        // rates
    double *jac;              // [Z][S][N][4][3]
    const vx_out *seeds;      // VJP seeds (spectral)
    double *grad_J, *grad_H;  // [Z][S][N]
    double *blocks;           // [Z][S][4][N][N]
};

static vx_status host_validate_batch(const vx_rates *h, const vx_batch *b) {
    if (!h) return fail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (!b) return fail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (h->cfg.prec != VX_PREC_MIXED) return fail(VX_ERR_UNSUPPORTED, "the host-buffer calls are provided for the mixed form");
    if (b->n_zones < 0 || b->n_rays < 0) return fail(VX_ERR_INVALID_ARG, "negative size");
    if (b->ray_offsets) {
        if (b->ray_offsets[0] != 0) return fail(VX_ERR_INVALID_ARG, "ray_offsets[0] must be 0");
        for (int r = 0; r < b->n_rays; ++r)
            if (b->ray_offsets[r + 1] < b->ray_offsets[r])
                return fail(VX_ERR_INVALID_ARG, "ray_offsets must be non-decreasing (ray %d)", r);
        if ((long long)b->ray_offsets[b->n_rays] != b->n_zones)
            return fail(VX_ERR_INVALID_ARG, "ray_offsets[n_rays] = %d but n_zones = %lld", b->ray_offsets[b->n_rays], b->n_zones);
    }
    if (b->n_zones > 0 && (!b->state || !b->J || !b->H)) return fail(VX_ERR_INVALID_ARG, "state, J and H must be host arrays");
    return VX_OK;
}

static vx_status host_run(vx_rates *h, const vx_batch *b, const HostIO &io) {
    vx_status st = host_validate_batch(h, b);
    if (st != VX_OK) return st;
    if (io.fwd && (!io.fwd->j0 || !io.fwd->chi0 || !io.fwd->j1 || !io.fwd->chi1))
        return fail(VX_ERR_INVALID_ARG, "an output array is NULL");
    if (io.fwd && io.fwd->phi) return fail(VX_ERR_INVALID_ARG, "phi output is not produced by the host-buffer calls");
    if (b->n_zones == 0) return VX_OK;
    DeviceGuard dg(h->device);
    if ((st = host_prepare(h)) != VX_OK) return st;
    auto &hs = h->hs;
    const size_t S = h->common.S, N = h->common.N, SN = S * N;
    const double *seed[4] = {nullptr, nullptr, nullptr, nullptr};
    if (io.seeds) { seed[0] = io.seeds->j0; seed[1] = io.seeds->chi0; seed[2] = io.seeds->j1; seed[3] = io.seeds->chi1; }
    int nseed = 0;
    for (int k = 0; k < 4; ++k) nseed += seed[k] != nullptr;
    // doubles per zone in a slot
    const size_t per = 4 + 2 * SN + (io.fwd ? 4 * SN : 0) + (io.jac ? 12 * SN : 0) + nseed * SN +
                       (io.grad_J ? 2 * SN : 0) + (io.blocks ? 4 * N * N * S : 0);
    const long long chunk = (long long)(hs.bytes / (per * sizeof(double)));
    if (chunk < 1) return fail(VX_ERR_UNSUPPORTED, "one zone does not fit a staging slot");
    const long long Z = b->n_zones;
    const bool adj = io.kind == 1;
    const int kind = adj ? 1 : 0;
    const size_t smem = adj ? h->smem_adj : h->smem_fwd;
    for (long long c = 0, z0 = 0; z0 < Z; ++c, z0 += chunk) {
        const long long n = std::min(chunk, Z - z0);
        const int sl = (int)(c & 1);
        cudaStream_t s = hs.st[sl];
        double *p = hs.buf[sl];
        auto take = [&](size_t count) { double *q = p; p += count; return q; };
        double *d_state = take(4 * n), *d_J = take(SN * n), *d_H = take(SN * n);
        VX_CU(cudaMemcpyAsync(d_state, b->state + 4 * z0, 4 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        VX_CU(cudaMemcpyAsync(d_J, b->J + SN * z0, SN * n * sizeof(double), cudaMemcpyHostToDevice, s));
        VX_CU(cudaMemcpyAsync(d_H, b->H + SN * z0, SN * n * sizeof(double), cudaMemcpyHostToDevice, s));
        vx_batch db{0, n, nullptr, d_state, d_J, d_H};
        vx::Launch L{};
        fill_launch(h, &db, L);
        L.counter = hs.cnt + sl;
        double *d_out = nullptr, *d_jac = nullptr, *d_blk = nullptr, *d_gJ = nullptr, *d_gH = nullptr;
        if (io.fwd) {
            d_out = take(4 * SN * n);
            L.j0 = d_out; L.chi0 = d_out + SN * n; L.j1 = d_out + 2 * SN * n; L.chi1 = d_out + 3 * SN * n;
        }
        if (io.jac) L.jac = d_jac = take(12 * SN * n);
        if (nseed) {
            const double **gs[4] = {&L.g_j0, &L.g_chi0, &L.g_j1, &L.g_chi1};
            for (int k = 0; k < 4; ++k)
                if (seed[k]) {
                    double *q = take(SN * n);
                    VX_CU(cudaMemcpyAsync(q, seed[k] + SN * z0, SN * n * sizeof(double), cudaMemcpyHostToDevice, s));
                    *gs[k] = q;
                }
        }
        if (io.grad_J) { L.grad_J = d_gJ = take(SN * n); L.grad_H = d_gH = take(SN * n); }
        if (io.blocks) L.blocks = d_blk = take(4 * N * N * S * n);
        if ((st = autotune(h, adj, L, s)) != VX_OK) return st;
        const int mb = h->minb[kind];
        const int grid = (int)std::min<long long>(h->grid_mixed[kind][mb - 2], n);
        VX_CU(cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), s));
        VX_CU(vx::launch_mixed(adj, mb, L, grid, h->block_mixed, smem, s));
        if (io.fwd) {
            double *dst[4] = {io.fwd->j0, io.fwd->chi0, io.fwd->j1, io.fwd->chi1};
            for (int k = 0; k < 4; ++k)
                VX_CU(cudaMemcpyAsync(dst[k] + SN * z0, d_out + k * SN * n, SN * n * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
        }
        if (d_jac)
            VX_CU(cudaMemcpyAsync(io.jac + 12 * SN * z0, d_jac, 12 * SN * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (d_gJ) {
            VX_CU(cudaMemcpyAsync(io.grad_J + SN * z0, d_gJ, SN * n * sizeof(double), cudaMemcpyDeviceToHost, s));
            VX_CU(cudaMemcpyAsync(io.grad_H + SN * z0, d_gH, SN * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        if (d_blk)
            VX_CU(cudaMemcpyAsync(io.blocks + 4 * N * N * S * z0, d_blk, 4 * N * N * S * n * sizeof(double),
                                  cudaMemcpyDeviceToHost, s));
    }
    VX_CU(cudaStreamSynchronize(hs.st[0]));
    VX_CU(cudaStreamSynchronize(hs.st[1]));
    return VX_OK;
}

vx_status vx_rates_eval_host(vx_rates *h, const vx_batch *host_batch, const vx_out *host_out) {
    if (!host_out) return fail(VX_ERR_INVALID_ARG, "out is NULL");
    return host_run(h, host_batch, HostIO{0, host_out, nullptr, nullptr, nullptr, nullptr, nullptr});
}

vx_status vx_rates_adjoint_host(vx_rates *h, const vx_batch *host_batch, double *host_jac, const vx_out *host_fwd) {
    if (!host_jac && !host_fwd) return fail(VX_ERR_INVALID_ARG, "no output requested");
    return host_run(h, host_batch, HostIO{1, host_fwd, host_jac, nullptr, nullptr, nullptr, nullptr});
}

vx_status vx_rates_spectral_host(vx_rates *h, const vx_batch *host_batch, const vx_out *host_grad_out,
                                 double *host_grad_J, double *host_grad_H, double *host_blocks,
                                 const vx_out *host_fwd) {
    if (!host_blocks && !host_grad_J && !host_grad_H && !host_fwd) return fail(VX_ERR_INVALID_ARG, "no output requested");
    if (!host_grad_J != !host_grad_H) return fail(VX_ERR_INVALID_ARG, "grad_J and grad_H go together");
    if (host_grad_J && !host_grad_out) return fail(VX_ERR_INVALID_ARG, "grad_J and grad_H need grad_out");
    return host_run(h, host_batch,
                    HostIO{2, host_fwd, nullptr, host_grad_J ? host_grad_out : nullptr, host_grad_J, host_grad_H, host_blocks});
}

vx_status vx_rates_check(vx_rates *h, vx_stream stream) {
    if (!h) return fail(VX_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard dg(h->device);
    VX_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    VX_CU(cudaMemcpy(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        VX_CU(cudaMemset(h->d_flag, 0, sizeof(int)));
        return fail(VX_ERR_NUMERIC, "device numeric flag 0x%x (%s%s%s)", flag,
                    (flag & VX_FLAG_BAD_STATE) ? "invalid zone state; " : "",
                    (flag & VX_FLAG_NONFINITE) ? "non-finite result; " : "",
                    (flag & VX_FLAG_BAD_OFFSETS) ? "invalid ray offsets" : "");
    }
    return VX_OK;
}

void vx_rates_destroy(vx_rates *h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    cudaDeviceSynchronize();
    for (cudaGraphExec_t &g : h->gexec)
        if (g) cudaGraphExecDestroy(g);
    cudaFree(h->d_tab32);
    cudaFree(h->d_tab64);
    cudaFree(h->d_counter);
    cudaFree(h->d_flag);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->hs.buf[k]);
        if (h->hs.st[k]) cudaStreamDestroy(h->hs.st[k]);
    }
    cudaFree(h->hs.cnt);
    delete h;
}

}  // extern "C"

// =============================================================================================
// Allocation-free evaluation (vx_rates_eval_noalloc). Everything the forward mixed kernel needs
// besides the caller's inputs and outputs -- the work counter, the numeric flag and the
// (bin pair, omega node) table -- lives in one file-scope device array, so the call allocates
// nothing. Limits: at most VX_NOALLOC_MAX_BINS bins and VX_NOALLOC_MAX_MU cos(omega) nodes.
// =============================================================================================
#define VX_NOALLOC_MAX_BINS 24
#define VX_NOALLOC_MAX_MU 32
#define VX_NOALLOC_MAX_PAIRS (VX_NOALLOC_MAX_BINS * (VX_NOALLOC_MAX_BINS + 1) / 2)
#define VX_NOALLOC_TABLE_OFFSET 256
#define VX_NOALLOC_SCRATCH_BYTES \
    (VX_NOALLOC_TABLE_OFFSET + (size_t)VX_NOALLOC_MAX_PAIRS * VX_NOALLOC_MAX_MU * 2 * sizeof(float4))
#define VX_NOALLOC_MAX_DEVICES 64

// 307,456 bytes (256 + 300 pairs x 32 nodes x 2 float4) on every device that loads the library,
// held until the process exits. Layout: [0, 8) work counter, [8, 12) numeric flag, [256, ...) the
// pair table.
static_assert(VX_NOALLOC_SCRATCH_BYTES == 307456, "the header states the scratch size");
static __device__ __align__(256) unsigned char g_noalloc_scratch[VX_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device; the name itself is only a host-side stand-in.
static unsigned char *g_noalloc_ptr[VX_NOALLOC_MAX_DEVICES] = {nullptr};

namespace {

struct NoallocTab {
    double eps[VX_NOALLOC_MAX_BINS];
    double tm[VX_NOALLOC_MAX_MU], wm[VX_NOALLOC_MAX_MU];
    uint16_t pij[VX_NOALLOC_MAX_PAIRS];
    int N, n_mu, npair;
};

// Fills the (unordered pair, omega node) table in scratch with the records vx_rates_create builds
// on the host: half-width |q|/2 and lower electron energy E- (FP32 value plus remainder), the
// three moment coefficients and cos(omega).
__global__ void k_noalloc_table(const __grid_constant__ NoallocTab P, float4 *tab) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= P.n_mu * P.npair) return;
    const int m = e / P.npair, p = e % P.npair;
    const int i = P.pij[p] >> 8, j = P.pij[p] & 0xff;
    const double pi = 3.14159265358979323846;
    const double t = P.tm[m], y = 1.0 - t;
    const double ee = P.eps[i], ep = P.eps[j];
    const double d = ee - ep, g = ee * ep * (1.0 + t);
    const double q2 = d * d + 2.0 * g, q = sqrt(q2), hh = 0.5 * q;
    const double q0 = ee + ep, s = 2.0 * ee * ep * y;
    const double Em = s / (2.0 * (q0 + q));
    const double pref = P.wm[m] * pi * ee * ep * y * y / (16.0 * q2);
    const double kp = pref * 0.25 * (q + d) * (q + d), km = pref * 0.25 * (q - d) * (q - d), k0 = pref * 2.0 * g;
    float4 *r = tab + ((size_t)p * P.n_mu + m) * 2;
    const float fh = (float)hh, fEm = (float)Em;
    r[0] = make_float4(fh, (float)(hh - fh), fEm, (float)(Em - fEm));
    r[1] = make_float4((float)kp, (float)km, (float)k0, (float)t);
}

}  // namespace

// Kernel parameters of a config, built as vx_rates_create builds them, on the stack.
static void noalloc_params(const vx_config *cfg, vx::Launch &L, NoallocTab &T) {
    const int N = cfg->n_bins, S = cfg->n_species, nmu = cfg->n_mu, ne = cfg->n_e;
    vx::Common &C = L.c;
    memset(&L, 0, sizeof L);
    memset(&T, 0, sizeof T);
    C.N = N; C.n_mu = nmu; C.n_e = ne; C.S = S;
    C.npair = N * (N + 1) / 2;
    C.ms = 1;
    C.g2 = cfg->g2; C.norm = cfg->norm; C.eta_sw = cfg->eta_fp64 == 0.0 ? 20.0 : cfg->eta_fp64;
    const double *eps = cfg->eps;
    for (int i = 0; i < N; ++i) {
        double w;
        if (cfg->weights) w = cfg->weights[i];
        else {
            double lo = i ? std::sqrt(eps[i - 1] * eps[i]) : eps[0] * std::sqrt(eps[0] / eps[1]);
            double hi = i < N - 1 ? std::sqrt(eps[i] * eps[i + 1]) : eps[N - 1] * std::sqrt(eps[N - 1] / eps[N - 2]);
            w = eps[i] * eps[i] * (hi - lo);
        }
        C.eps[i] = eps[i];
        C.w[i] = w;
        T.eps[i] = eps[i];
    }
    for (int s = 0; s < S; ++s) {
        int sp = cfg->species[s];
        int want = sp == VX_NU_E ? VX_NU_EBAR : sp == VX_NU_EBAR ? VX_NU_E : VX_NU_X;
        for (int t = 0; t < S; ++t) if (cfg->species[t] == want) C.partner[s] = t;
        C.species[s] = sp;
        double cv = (sp == VX_NU_X ? -0.5 : 0.5) + 2.0 * cfg->sin2w, ca = sp == VX_NU_X ? -0.5 : 0.5;
        double b1 = (cv + ca) * (cv + ca), b2 = (cv - ca) * (cv - ca);
        if (sp == VX_NU_EBAR) std::swap(b1, b2);
        C.bI64[s] = b1; C.bII64[s] = b2;
        C.bI[s] = (float)b1; C.bII[s] = (float)b2;
    }
    int p = 0;
    for (int i = 0; i < N; ++i)
        for (int j = i; j < N; ++j) { C.pij[p] = (uint16_t)((i << 8) | j); T.pij[p] = C.pij[p]; ++p; }
    double tm[VX_MAX_MU], wm[VX_MAX_MU], tk[VX_MAX_NE], wk[VX_MAX_NE];
    gauss_legendre(nmu, tm, wm);
    gauss_legendre(ne, tk, wk);
    for (int m = 0; m < nmu; ++m) {
        C.t64[m] = tm[m];
        C.t_hi[m] = (float)tm[m];
        C.t_lo[m] = (float)(tm[m] - (double)C.t_hi[m]);
        T.tm[m] = tm[m];
        T.wm[m] = wm[m];
    }
    for (int k = 0; k < ne; ++k) {
        double u = 1.0 + tk[k], v = 1.0 - tk[k];
        L.n32.u[k] = (float)u; L.n32.v[k] = (float)v;
        L.n32.cp[k] = (float)(wk[k] * u * u); L.n32.cm[k] = (float)(wk[k] * v * v); L.n32.c0[k] = (float)(wk[k] * u * v);
        double uh = std::nearbyint(u * 2048.0) / 2048.0;
        L.n32.uh[k] = (float)uh;
        L.n32.ul[k] = (float)(u - uh);
    }
    double hmax = 0.0, q0hmax = 0.0;
    for (int m = 0; m < nmu; ++m)
        for (int q = 0; q < C.npair; ++q) {
            const int i = C.pij[q] >> 8, j = C.pij[q] & 0xff;
            const double d = eps[i] - eps[j], g = eps[i] * eps[j] * (1.0 + tm[m]);
            hmax = std::fmax(hmax, 0.5 * std::sqrt(d * d + 2.0 * g));
            q0hmax = std::fmax(q0hmax, 0.5 * (eps[i] + eps[j]));
        }
    C.h_max = hmax;
    C.q0h_max = q0hmax;
    T.N = N; T.n_mu = nmu; T.npair = C.npair;
}

extern "C" {

vx_status vx_rates_eval_noalloc(const vx_config *cfg, const vx_batch *b, const vx_out *out, vx_stream stream) {
    vx_status st = validate_config(cfg);
    if (st != VX_OK) return st;
    if (cfg->prec != VX_PREC_MIXED) return fail(VX_ERR_UNSUPPORTED, "vx_rates_eval_noalloc evaluates the mixed form only");
    if (cfg->n_bins > VX_NOALLOC_MAX_BINS || cfg->n_mu > VX_NOALLOC_MAX_MU)
        return fail(VX_ERR_UNSUPPORTED,
                    "vx_rates_eval_noalloc: %d bins x %d cos(omega) nodes exceed its fixed scratch of %zu bytes "
                    "(at most %d bins and %d nodes); use a handle from vx_rates_create",
                    cfg->n_bins, cfg->n_mu, (size_t)VX_NOALLOC_SCRATCH_BYTES, VX_NOALLOC_MAX_BINS, VX_NOALLOC_MAX_MU);
    if (!b) return fail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_zones < 0 || b->n_rays < 0) return fail(VX_ERR_INVALID_ARG, "negative batch size");
    if (b->n_zones == 0) return VX_OK;
    if (b->ray_offsets && (st = check_device_ptr(b->ray_offsets, "ray_offsets", 4)) != VX_OK) return st;
    if ((st = check_device_ptr(b->state, "state")) != VX_OK) return st;
    if ((st = check_device_ptr(b->J, "J")) != VX_OK) return st;
    if ((st = check_device_ptr(b->H, "H")) != VX_OK) return st;
    if ((st = validate_out(out, true)) != VX_OK) return st;

    int dev = 0;
    VX_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= VX_NOALLOC_MAX_DEVICES) return fail(VX_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    if (!g_noalloc_ptr[dev]) {  // once per device, with that device current
        void *ptr = nullptr;
        VX_CU(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_ptr[dev] = (unsigned char *)ptr;
    }
    unsigned char *scratch = g_noalloc_ptr[dev];

    vx::Launch L{};
    NoallocTab T;
    noalloc_params(cfg, L, T);
    L.tab32 = reinterpret_cast<const float4 *>(scratch + VX_NOALLOC_TABLE_OFFSET);
    L.tab64 = nullptr;
    L.Z = b->n_zones;
    L.state = b->state; L.J = b->J; L.H = b->H;
    L.j0 = out->j0; L.chi0 = out->chi0; L.j1 = out->j1; L.chi1 = out->chi1; L.phi = out->phi;
    L.counter = reinterpret_cast<unsigned long long *>(scratch);
    L.flag = reinterpret_cast<int *>(scratch + 8);

    const int ne = cfg->n_e, minb = 2;
    const int block = std::min(round_up(L.c.npair * cfg->n_mu, 32), VX_BLOCK_MIXED);
    const size_t smem = vx::smem_mixed_bytes(cfg->n_bins, cfg->n_species, false, block);
    const void *fn = vx::kernel_mixed(false, minb, ne, false, false);
    VX_CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nsm = 0, occ = 0;
    VX_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    VX_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem));
    if (occ < 1) return fail(VX_ERR_UNSUPPORTED, "kernel does not fit on an SM");
    const int grid = (int)std::min<long long>((long long)occ * nsm, b->n_zones);

    cudaStream_t s = (cudaStream_t)stream;
    VX_CU(cudaMemsetAsync(scratch, 0, 16, s));  // work counter and numeric flag start at zero
    const int nrec = T.n_mu * T.npair;
    k_noalloc_table<<<(nrec + 255) / 256, 256, 0, s>>>(T, reinterpret_cast<float4 *>(scratch + VX_NOALLOC_TABLE_OFFSET));
    VX_CU(cudaGetLastError());
    VX_CU(vx::launch_mixed(false, minb, L, grid, block, smem, s));
    return VX_OK;
}

}  // extern "C"
