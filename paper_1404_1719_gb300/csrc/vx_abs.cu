// vx_abs.cu -- charged-current absorption and emission on free nucleons (include/vx_abs.h).
//
// A streaming kernel: every (zone, species, bin) entry is independent and costs a few dozen
// arithmetic operations against 32 B (rates) or 128 B (rates and Jacobian) of output. A block
// takes a contiguous range of whole zones per iteration of a grid-stride loop, so a warp's stores
// are contiguous; the zone quantities its entries share (1/T, the nucleon densities, the state
// check) are formed once per zone into shared memory by the block's first threads. The lepton
// energy E and the prefactor (g2/pi)(1 + 3 gA^2) E^2 of every (species, bin) are formed on the
// host in FP64 and passed by value. (A block takes whole zones, and a thread the same entry of
// each: no 64-bit integer division per entry, which would run on the FP64 unit.)
// Forms: FP64 (library exp, true division, FP64 products) and mixed. GB300 issues FP64 about 75x
// slower than FP32, so the mixed form runs no FP64 arithmetic per entry. The exponent argument
// x = E/T -+ eta (up to ~1e3, more than FP32's 24 bits can resolve) is formed as an FP32 pair
// (double-float: exact products by FMA, two-sum) from pairs of E, 1/T and eta, and so is
// |x| log2(e) = n + fr with n an integer: the small occupation is (2^-fr r) 2^-n and the large one
// r = 1/(1 + 2^-fr 2^-n), 2^-fr from MUFU ex2 and r from the FP32 reciprocal. Every product is an
// FP32 mantissa, and the powers of two (2^-n, and that of the prefactor, so any global scale g2
// fits) are put into the FP64 result's exponent field with integer operations. Relative error
// about 2^-21 over the FP64 range.
#include "../../include/vx_abs.h"
#include "vx_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>

namespace vx {
vx_status set_error(vx_status s, const char *msg);
}

namespace {

constexpr double kQ = 1.29333236;            // m_n - m_p, MeV
constexpr double kGA = 1.2754;               // axial coupling
constexpr double kMu = 1.66053906660e-24;    // atomic mass unit, g
constexpr double kPi = 3.14159265358979323846;
constexpr int kAbsBlock = 256;
constexpr int kAbsWarps = kAbsBlock / 32;
constexpr int kZoneSlots = 32;  // zones a warp's 32 consecutive entries can span (S N >= 1)

vx_status afail(vx_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return vx::set_error(s, buf);
}

#define ABS_CU(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return afail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                             \
    } while (0)

vx_status device_ptr(const void *p, size_t align, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return afail(VX_ERR_INVALID_ARG, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return afail(VX_ERR_INVALID_ARG, "%s must be device memory", name);
    if ((uintptr_t)p % align) return afail(VX_ERR_INVALID_ARG, "%s must be %zu-byte aligned", name, align);
    return VX_OK;
}

// Per (species, bin): lepton energy and prefactor (0 where the reaction is closed); per species
// whether the lepton is a positron.
struct AbsConst {
    int N, S;
    int anti[3];
    double E[3][VX_MAX_BINS];
    double K[3][VX_MAX_BINS];
    float Ef[3][VX_MAX_BINS];  // mixed form: E as an FP32 pair, and K = Kf 2^kK with Kf in [1, 2)
    float El[3][VX_MAX_BINS];
    float Kf[3][VX_MAX_BINS];
    int kK[3][VX_MAX_BINS];
};

struct AbsLaunch {
    AbsConst c;
    long long Z;
    const int *off;
    int n_rays;
    const double *state;
    double *j0, *chi0, *j1, *chi1, *jac;
    int *flag;
};

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcpf(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// v 2^shift as an FP64 value, for v an FP32 value, with integer operations only (no FP64
// instruction, even predicated off): the FP64 exponent is set from v's bits; results below the
// FP64 normal range get the subnormal encoding of v's 24-bit significand (truncated), an FP32 zero
// or subnormal v gives a zero, a non-finite v the same non-finite FP64 value.
__device__ __forceinline__ double pow2scaled(float v, int shift) {
    const unsigned u = __float_as_uint(v);
    const int ev = (int)((u >> 23) & 0xffu);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63, m = u & 0x7fffffu;
    unsigned long long bits;
    const int e64 = ev - 127 + 1023 + shift;
    if (ev == 0) bits = sign;
    else if (ev == 255) bits = sign | 0x7ff0000000000000ull | (m << 29);
    else if (e64 >= 2047) bits = sign | 0x7ff0000000000000ull;
    else if (e64 >= 1) bits = sign | ((unsigned long long)e64 << 52) | (m << 29);
    else {  // subnormal: value = S 2^(e64 + 28) 2^-1074, S the 24-bit significand
        const unsigned long long S = m | 0x800000ull;
        const int sh = e64 + 28;
        bits = sign | (sh >= 0 ? (S << sh) : (sh > -25 ? (S >> -sh) : 0ull));
    }
    return __longlong_as_double((long long)bits);
}

// Occupation 1/(1 + e^x) and 1 - it, without cancellation.
template <bool F64>
__device__ __forceinline__ void occupation(double x, double &f, double &omf) {
    const double ax = fabs(x);
    double e, r;  // e = e^-|x|, r = 1/(1 + e)
    if (F64) {
        e = exp(-ax);
        r = 1.0 / (1.0 + e);
    } else {
        const double y = ax * 1.4426950408889634;  // |x| log2(e)
        const double n = floor(y);
        const double fr = (double)ex2f(-(float)(y - n));
        if (n <= 1022.0)
            e = fr * __longlong_as_double((long long)(1023 - (int)n) << 52);
        else if (n <= 1100.0)  // into the subnormal range: two exact powers of two
            e = fr * 0x1p-511 * __longlong_as_double((long long)(1023 - ((int)n - 511)) << 52);
        else
            e = 0.0;
        r = (double)rcpf((float)(1.0 + e));
    }
    if (x > 0.0) {
        f = e * r;
        omf = r;
    } else {
        f = r;
        omf = e * r;
    }
}

template <bool F64, bool ADJ>
__global__ void __launch_bounds__(kAbsBlock) k_abs(const __grid_constant__ AbsLaunch L) {
    // Each warp takes 32 consecutive zones at a time, with no CTA barrier: lane l forms zone l's
    // scalars in the warp's shared slots (the FP64 set-up with every lane busy), then the warp runs
    // through the group's entries (zone, species, bin) 32 at a time, staging their Jacobian rows in
    // its own slice of shared memory (row stride 13: banks) and storing them as one contiguous run.
    __shared__ double ziT[kAbsWarps][kZoneSlots], zeta[kAbsWarps][kZoneSlots], znb[kAbsWarps][kZoneSlots],
        zYe[kAbsWarps][kZoneSlots];
    __shared__ float znnf[kAbsWarps][kZoneSlots], znpf[kAbsWarps][kZoneSlots], znbf[kAbsWarps][kZoneSlots],
        ziT2f[kAbsWarps][kZoneSlots];
    __shared__ float ziTh[kAbsWarps][kZoneSlots], ziTl[kAbsWarps][kZoneSlots], zetah[kAbsWarps][kZoneSlots],
        zetal[kAbsWarps][kZoneSlots];
    __shared__ int zbad[kAbsWarps][kZoneSlots];
    __shared__ double sj[ADJ ? kAbsBlock * 13 : 1];
    const AbsConst &C = L.c;
    const int SN = C.S * C.N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double *sjw = sj + (ADJ ? warp * 32 * 13 : 0);
    vx::validate_offsets(L.off, L.n_rays, L.Z, L.flag);
    // entry q = lane of a group as (zone slot k0, species s0, bin i0), and the step of 32 entries
    const int k0 = lane / SN, s0 = (lane - k0 * SN) / C.N, i0 = lane - k0 * SN - s0 * C.N;
    const int dk = 32 / SN, dsi = 32 - dk * SN, ds = dsi / C.N, di = dsi - ds * C.N;
    for (long long zg = ((long long)blockIdx.x * kAbsWarps + warp) * kZoneSlots; zg < L.Z;
         zg += (long long)gridDim.x * kAbsWarps * kZoneSlots) {
        const int nz = (int)min((long long)kZoneSlots, L.Z - zg);
        if (lane < nz) {
            const int kk = lane;
            const double *st = L.state + 4 * (zg + kk);
            const double T = st[0], eta = st[1], Ye = st[2], rho = st[3];
            const bool bad = !(T > 0.0) || !isfinite(T) || !isfinite(eta) || !(Ye >= 0.0 && Ye <= 1.0) ||
                             !(rho >= 0.0) || !isfinite(rho);
            zbad[warp][kk] = bad;
            ziT[warp][kk] = bad ? 0.0 : 1.0 / T;
            zeta[warp][kk] = eta;
            zYe[warp][kk] = Ye;
            znb[warp][kk] = rho * (1e-39 / kMu);  // baryons per fm^3
            if (!F64) {
                const double nb = znb[warp][kk], iT = ziT[warp][kk];
                znbf[warp][kk] = (float)nb;
                znnf[warp][kk] = (float)(nb * (1.0 - Ye));
                znpf[warp][kk] = (float)(nb * Ye);
                ziT2f[warp][kk] = (float)fmin(iT * iT, 1e30);  // T >= 1e-15 MeV for the T-derivative
                ziTh[warp][kk] = (float)iT;
                ziTl[warp][kk] = (float)(iT - (double)ziTh[warp][kk]);
                zetah[warp][kk] = (float)eta;
                zetal[warp][kk] = (float)(eta - (double)zetah[warp][kk]);
            }
            if (bad) atomicOr(L.flag, VX_FLAG_BAD_STATE);
        }
        __syncwarp();
        const int nE = nz * SN;
        int k = k0, s = s0, i = i0;
        for (int c0 = 0; c0 < nE; c0 += 32) {
            const long long e = zg * SN + c0 + lane;
            const int last = min(31, nE - 1 - c0);
            if (c0 + lane < nE) {
                double j = 0.0, chi = 0.0, d[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
                const double K = C.K[s][i];
                if (zbad[warp][k]) {
                    j = chi = __longlong_as_double(0x7ff8000000000000ll);
                } else if (K > 0.0 && F64) {
                    const bool anti = C.anti[s] != 0;
                    const double E = C.E[s][i], iT = ziT[warp][k], nb = znb[warp][k], Ye = zYe[warp][k];
                    const double nn = nb * (1.0 - Ye), np = nb * Ye;
                    const double nin = anti ? np : nn, nout = anti ? nn : np;
                    const double x = fma(E, iT, anti ? zeta[warp][k] : -zeta[warp][k]);
                    double f, omf;
                    occupation<F64>(x, f, omf);
                    j = K * nout * f;
                    chi = K * nin * omf;
                    if (ADJ) {
                        // df/dx = -f (1 - f); dx/dT = -E/T^2; dx/deta = -1 (electron), +1 (positron)
                        const double g = f * omf, gT = g * E * iT * iT, ge = anti ? -g : g;
                        d[0][0] = K * nout * gT;   d[0][1] = K * nout * ge;   d[0][2] = K * (anti ? -nb : nb) * f;
                        d[1][0] = -K * nin * gT;   d[1][1] = -K * nin * ge;   d[1][2] = K * (anti ? nb : -nb) * omf;
                    }
                } else if (C.Kf[s][i] > 0.f) {
                    const bool anti = C.anti[s] != 0;
                    // x = E/T -+ eta as an FP32 pair: E (1/T) exactly by FMA, then a two-sum with -+eta
                    // (explicitly rounded operations: no contraction into FMAs may change the pair)
                    const float Eh = C.Ef[s][i], El = C.El[s][i], ih = ziTh[warp][k], il = ziTl[warp][k];
                    const float ph = __fmul_rn(Eh, ih);
                    const float pl = __fadd_rn(fmaf(Eh, ih, -ph), fmaf(Eh, il, __fmul_rn(El, ih)));
                    const float eh = anti ? zetah[warp][k] : -zetah[warp][k], el = anti ? zetal[warp][k] : -zetal[warp][k];
                    const float sh = __fadd_rn(ph, eh), sv = __fsub_rn(sh, ph);
                    const float xl0 = __fadd_rn(__fadd_rn(__fsub_rn(ph, __fsub_rn(sh, sv)), __fsub_rn(eh, sv)), __fadd_rn(pl, el));
                    const float xh = __fadd_rn(sh, xl0), xl = __fsub_rn(xl0, __fsub_rn(xh, sh));
                    // |x| log2(e) = yh + yl as an FP32 pair, then n = floor(yh) and fr = (yh - n) + yl
                    const float ah = fabsf(xh), al = xh < 0.f ? -xl : xl;
                    const float L2h = 1.44269502162933349609375f, L2l = 1.925963033500011079e-8f;
                    const float yh = __fmul_rn(ah, L2h);
                    const float yl = __fadd_rn(fmaf(ah, L2h, -yh), fmaf(ah, L2l, __fmul_rn(al, L2h)));
                    const bool huge = !(yh <= 2000.f);
                    const float nf = huge ? 2000.f : floorf(yh);
                    const int n = (int)nf;
                    const float ef = ex2f(huge ? 0.f : -__fadd_rn(__fsub_rn(yh, nf), yl));  // 2^-fr
                    const float e32 = n < 126 ? ef * __int_as_float((127 - n) << 23) : 0.f; // e^-|x|
                    const float r = rcpf(1.f + e32), sm = ef * r;  // large occupation; small one = sm 2^-n
                    const bool pos = xh > 0.f;
                    const float f = pos ? sm : r, omf = pos ? r : sm;
                    const int kf = C.kK[s][i] - (pos ? n : 0), ko = C.kK[s][i] - (pos ? 0 : n), kg = C.kK[s][i] - n;
                    const float Kf = C.Kf[s][i], nin = anti ? znpf[warp][k] : znnf[warp][k], nout = anti ? znnf[warp][k] : znpf[warp][k];
                    const float Kout = Kf * nout, Kin = Kf * nin;
                    j = pow2scaled(Kout * f, kf);
                    chi = pow2scaled(Kin * omf, ko);
                    if (ADJ) {
                        const float g = f * omf, gT = g * (C.Ef[s][i] * ziT2f[warp][k]), ge = anti ? -g : g;
                        const float Kb = Kf * znbf[warp][k];
                        d[0][0] = pow2scaled(Kout * gT, kg);  d[0][1] = pow2scaled(Kout * ge, kg);
                        d[0][2] = pow2scaled(anti ? -Kb * f : Kb * f, kf);
                        d[1][0] = pow2scaled(-Kin * gT, kg);  d[1][1] = pow2scaled(-Kin * ge, kg);
                        d[1][2] = pow2scaled(anti ? Kb * omf : -Kb * omf, ko);
                    }
                }
                if (L.j0) {
                    L.j0[e] = j;
                    L.chi0[e] = chi;
                    L.j1[e] = zbad[warp][k] ? j : 0.0;
                    L.chi1[e] = zbad[warp][k] ? j : 0.0;
                }
                if (ADJ && L.jac) {
                    double *J = sjw + lane * 13;
                    const double zero = zbad[warp][k] ? j : 0.0;
    #pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        J[c] = zbad[warp][k] ? j : d[0][c];
                        J[3 + c] = zbad[warp][k] ? j : d[1][c];
                        J[6 + c] = zero;
                        J[9 + c] = zero;
                    }
                }
                // (the FP64 class test on the FP64 pipe: in the mixed form on the results' exponent bits)
                const long long jb = __double_as_longlong(j), cb = __double_as_longlong(chi);
                const bool fin = F64 ? (isfinite(j) && isfinite(chi))
                                     : ((jb & 0x7ff0000000000000ll) != 0x7ff0000000000000ll &&
                                        (cb & 0x7ff0000000000000ll) != 0x7ff0000000000000ll);
                if (!zbad[warp][k] && !fin) atomicOr(L.flag, VX_FLAG_NONFINITE);
            }
            if (ADJ && L.jac) {  // the chunk's entries: 12 (last + 1) consecutive doubles
                __syncwarp();
                const int nv = 12 * (last + 1);
                double *dst = L.jac + (zg * SN + c0) * 12;
                for (int q = lane; q < nv; q += 32) {
                    const int ent = q / 12;
                    dst[q] = sjw[ent * 13 + (q - ent * 12)];
                }
                __syncwarp();
            }
            k += dk;  // the next 32 entries
            i += di;
            if (i >= C.N) {
                i -= C.N;
                ++s;
            }
            s += ds;
            if (s >= C.S) {
                s -= C.S;
                ++k;
            }
        }
        __syncwarp();  // the zone slots are read before the next group's set-up
    }
}

template <bool F64>
const void *abs_kernel(bool adj) {
    return adj ? (const void *)k_abs<F64, true> : (const void *)k_abs<F64, false>;
}

}  // namespace

struct vx_abs {
    int device = 0, grid = 0;
    int prec = VX_PREC_MIXED;
    AbsConst c{};
    int *d_flag = nullptr;
};

namespace {

vx_status abs_validate_batch(const vx_abs *h, const vx_batch *b) {
    if (!h) return afail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (!b) return afail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_zones < 0 || b->n_rays < 0) return afail(VX_ERR_INVALID_ARG, "negative batch size");
    if (b->n_zones == 0) return VX_OK;
    vx_status s;
    if (b->ray_offsets) {
        if (b->n_rays == 0) return afail(VX_ERR_INVALID_ARG, "n_zones > 0 with no rays");
        if ((s = device_ptr(b->ray_offsets, 4, "ray_offsets")) != VX_OK) return s;
    }
    if (b->n_zones > (1ll << 40)) return afail(VX_ERR_INVALID_ARG, "n_zones too large");
    return device_ptr(b->state, 8, "state");
}

vx_status abs_validate_out(const vx_out *o) {
    vx_status s;
    const double *a[4] = {o->j0, o->chi0, o->j1, o->chi1};
    const char *nm[4] = {"out.j0", "out.chi0", "out.j1", "out.chi1"};
    for (int k = 0; k < 4; ++k)
        if ((s = device_ptr(a[k], 8, nm[k])) != VX_OK) return s;
    if (o->phi) return afail(VX_ERR_INVALID_ARG, "out.phi must be NULL: these rates have no kernel to dump");
    return VX_OK;
}

vx_status abs_run(vx_abs *h, const vx_batch *b, const vx_out *out, double *jac, cudaStream_t s) {
    AbsLaunch L{};
    L.c = h->c;
    L.Z = b->n_zones;
    L.off = b->ray_offsets;
    L.n_rays = b->n_rays;
    L.state = b->state;
    if (out) { L.j0 = out->j0; L.chi0 = out->chi0; L.j1 = out->j1; L.chi1 = out->chi1; }
    L.jac = jac;
    L.flag = h->d_flag;
    const long long blocks = (b->n_zones + kAbsWarps * kZoneSlots - 1) / (kAbsWarps * kZoneSlots);  // 32 zones per warp
    const int grid = (int)std::min<long long>(h->grid, blocks);
    const bool f64 = h->prec == VX_PREC_FP64, adj = jac != nullptr;
    if (f64) adj ? k_abs<true, true><<<grid, kAbsBlock, 0, s>>>(L) : k_abs<true, false><<<grid, kAbsBlock, 0, s>>>(L);
    else adj ? k_abs<false, true><<<grid, kAbsBlock, 0, s>>>(L) : k_abs<false, false><<<grid, kAbsBlock, 0, s>>>(L);
    ABS_CU(cudaGetLastError());
    return VX_OK;
}

}  // namespace

extern "C" {

vx_status vx_abs_create(const vx_config *cfg, vx_abs **out) {
    if (!out) return afail(VX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return afail(VX_ERR_INVALID_ARG, "config is NULL");
    if (cfg->n_bins < 1 || cfg->n_bins > VX_MAX_BINS) return afail(VX_ERR_INVALID_ARG, "n_bins %d outside 1..%d", cfg->n_bins, VX_MAX_BINS);
    if (!cfg->eps) return afail(VX_ERR_INVALID_ARG, "eps is NULL");
    for (int i = 0; i < cfg->n_bins; ++i)
        if (!(cfg->eps[i] > 0.0) || !std::isfinite(cfg->eps[i])) return afail(VX_ERR_INVALID_ARG, "eps[%d] must be finite and > 0", i);
    if (cfg->n_species < 1 || cfg->n_species > 3 || !cfg->species) return afail(VX_ERR_INVALID_ARG, "n_species must be 1..3");
    for (int s = 0; s < cfg->n_species; ++s) {
        if (cfg->species[s] < 0 || cfg->species[s] > 2) return afail(VX_ERR_INVALID_ARG, "species[%d] is not a vx_species", s);
        for (int t = 0; t < s; ++t)
            if (cfg->species[t] == cfg->species[s]) return afail(VX_ERR_INVALID_ARG, "species listed twice");
    }
    if (!std::isfinite(cfg->g2)) return afail(VX_ERR_INVALID_ARG, "g2 must be finite");
    if (cfg->prec != VX_PREC_MIXED && cfg->prec != VX_PREC_FP64) return afail(VX_ERR_INVALID_ARG, "unknown precision");
    if (cfg->flags != 0) return afail(VX_ERR_UNSUPPORTED, "flags must be 0 for the absorption rates");

    vx_abs *h = new vx_abs();
    h->prec = cfg->prec;
    AbsConst &C = h->c;
    C.N = cfg->n_bins;
    C.S = cfg->n_species;
    const double pref = cfg->g2 / kPi * (1.0 + 3.0 * kGA * kGA);
    for (int s = 0; s < C.S; ++s) {
        const int sp = cfg->species[s];
        C.anti[s] = sp == VX_NU_EBAR;
        for (int i = 0; i < C.N; ++i) {
            const double E = sp == VX_NU_EBAR ? cfg->eps[i] - kQ : cfg->eps[i] + kQ;
            const bool open = sp != VX_NU_X && E > 0.0;
            C.E[s][i] = open ? E : 0.0;
            C.K[s][i] = open ? pref * E * E : 0.0;
            int ex = 0;
            const double m = open && C.K[s][i] > 0.0 ? std::frexp(C.K[s][i], &ex) : 0.0;  // K = m 2^ex, m in [1/2, 1)
            C.Ef[s][i] = (float)C.E[s][i];
            C.El[s][i] = (float)(C.E[s][i] - (double)C.Ef[s][i]);
            C.Kf[s][i] = (float)(2.0 * m);
            C.kK[s][i] = ex - 1;
        }
    }
    cudaDeviceProp prop;
    if (cudaGetDevice(&h->device) != cudaSuccess || cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
        delete h;
        return afail(VX_ERR_CUDA, "no CUDA device");
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, abs_kernel<false>(true), kAbsBlock, 0) != cudaSuccess || occ < 1)
        occ = 1;
    h->grid = occ * prop.multiProcessorCount;
    if (cudaMalloc(&h->d_flag, sizeof(int)) != cudaSuccess || cudaMemset(h->d_flag, 0, sizeof(int)) != cudaSuccess) {
        vx_abs_destroy(h);
        return afail(VX_ERR_OOM, "allocation failed");
    }
    *out = h;
    return VX_OK;
}

vx_status vx_abs_eval(vx_abs *h, const vx_batch *b, const vx_out *out, vx_stream stream) {
    vx_status st = abs_validate_batch(h, b);
    if (st != VX_OK) return st;
    if (!out) return afail(VX_ERR_INVALID_ARG, "out is NULL");
    if (b->n_zones == 0) return VX_OK;
    if ((st = abs_validate_out(out)) != VX_OK) return st;
    return abs_run(h, b, out, nullptr, (cudaStream_t)stream);
}

vx_status vx_abs_adjoint(vx_abs *h, const vx_batch *b, double *jac, const vx_out *fwd, vx_stream stream) {
    vx_status st = abs_validate_batch(h, b);
    if (st != VX_OK) return st;
    if (!jac && !fwd) return afail(VX_ERR_INVALID_ARG, "jac and fwd are both NULL");
    if (b->n_zones == 0) return VX_OK;
    if (jac && (st = device_ptr(jac, 8, "jac")) != VX_OK) return st;
    if (fwd && (st = abs_validate_out(fwd)) != VX_OK) return st;
    return abs_run(h, b, fwd, jac, (cudaStream_t)stream);
}

vx_status vx_abs_check(vx_abs *h, vx_stream stream) {
    if (!h) return afail(VX_ERR_INVALID_ARG, "handle is NULL");
    ABS_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int f = 0;
    ABS_CU(cudaMemcpy(&f, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        ABS_CU(cudaMemset(h->d_flag, 0, sizeof(int)));
        return afail(VX_ERR_NUMERIC, "absorption device flag 0x%x (%s%s%s)", f,
                     (f & VX_FLAG_BAD_STATE) ? "invalid zone state; " : "",
                     (f & VX_FLAG_NONFINITE) ? "non-finite result; " : "", (f & VX_FLAG_BAD_OFFSETS) ? "invalid ray offsets" : "");
    }
    return VX_OK;
}

void vx_abs_destroy(vx_abs *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_flag);
    delete h;
}

}  // extern "C"
