// vx_nes.cu -- inelastic neutrino-electron scattering (include/vx_nes.h) and the electron-gas
// closure (include/vx_eos.h).
//
// Work decomposition. One CTA owns one zone at a time (zones pulled from an atomic counter, as in
// the pair kernel). A bin pair (i >= j: the down-scattering order, eps_i >= eps_j) is one group of
// lpp lanes of a warp (lpp = n_mu rounded up to a power of two), one lane per cos(omega) node; each
// lane integrates its (pair, omega) unit over the electron energy, and the group sums the Legendre
// projections with a fixed shuffle tree (deterministic). The pair's kernel of the other order and
// the in-scattering kernel follow from time reversal and detailed balance in the contraction.
//
// Unit algebra. With t = E - E_min the azimuth-averaged matrix elements are quadratics with
// non-negative coefficients, <M_X> = a_X + b_X t + c t^2 (a, b, c built in FP64 on the host with
// the prefactor G2 w_omega 2 pi/(4 |q| eps eps') folded in), so each unit accumulates the three
// moments Sum W F t^k of the blocking factor F = f(E) (1 - f(E + q0)) (and, for the tangents, of its
// T and eta derivatives). The electron-energy rule has three panels: Gauss-Legendre below the lower
// Fermi edge (30 T deep), between the edges, and Gauss-Laguerre above the upper edge. The
// exponent arguments are anchored at the nearer edge (x2 at the lower, x1 at the upper one), so
// their rounding stays small where the factors change. On the Laguerre panel, e^x F is formed from
// the tabulated e^{-x_k} and two per-unit exponentials, with no exponential per node.
// A zone scale e^{min(eta, 0)} is taken out of the electron occupation, restored in FP64.
#include "../../include/vx_eos.h"
#include "../../include/vx_nes.h"
#include "vx_internal.h"

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace vx {
vx_status set_error(vx_status s, const char *msg);
}

namespace {

constexpr int kNesMaxP = 32;     // nodes per panel
constexpr int kNesMaxMu = 32;
constexpr int kNesBlock = 128;
constexpr double kTail = 30.0;   // depth of the lower panel below the lower Fermi edge, in T

vx_status nfail(vx_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return vx::set_error(s, buf);
}

#define NES_CU(call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return nfail(e_ == cudaErrorMemoryAllocation ? VX_ERR_OOM : VX_ERR_CUDA, "%s: %s", #call, \
                         cudaGetErrorString(e_));                                             \
    } while (0)

vx_status device_ptr(const void *p, size_t align, const char *name) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nfail(VX_ERR_INVALID_ARG, "%s: not a CUDA pointer", name);
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return nfail(VX_ERR_INVALID_ARG, "%s must be device memory", name);
    if ((uintptr_t)p % align) return nfail(VX_ERR_INVALID_ARG, "%s must be %zu-byte aligned", name, align);
    return VX_OK;
}

// Gauss-Legendre (Newton on P_n) and Gauss-Laguerre nodes and weights, FP64 on the host.
void gl_nodes(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= n / 2 + (n & 1); ++k) {
        double r = std::cos(pi * (k - 0.25) / (n + 0.5)), dP = 1.0;
        for (int it = 0; it < 100; ++it) {
            double Pm = 1.0, P = r;
            for (int m = 2; m <= n; ++m) {
                double Pn = ((2 * m - 1) * r * P - (m - 1) * Pm) / m;
                Pm = P;
                P = Pn;
            }
            if (n == 1) { P = r; Pm = 1.0; }
            dP = n * (Pm - r * P) / (1.0 - r * r);
            const double step = P / dP;
            r -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double Pm = 1.0, P = r;
        for (int m = 2; m <= n; ++m) {
            double Pn = ((2 * m - 1) * r * P - (m - 1) * Pm) / m;
            Pm = P;
            P = Pn;
        }
        if (n == 1) { P = r; Pm = 1.0; }
        dP = n * (Pm - r * P) / (1.0 - r * r);
        const double wk = 2.0 / ((1.0 - r * r) * dP * dP);
        x[n - k] = r; x[k - 1] = -r;
        w[n - k] = wk; w[k - 1] = wk;
    }
    if (n & 1) x[n / 2] = 0.0;
}

// L_n and L_{n-1} at x (three-term recurrence)
void lag_eval(int n, double x, double &ln, double &lm) {
    double p0 = 1.0, p1 = 1.0 - x;
    for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0 - x) * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    ln = n ? p1 : 1.0;
    lm = n ? p0 : 0.0;
}

// Roots of L_n as the eigenvalues of its Jacobi matrix (diagonal 2k + 1, off-diagonal k): the
// k-th eigenvalue by bisection on the Sturm count (the number of negative pivots of the LDL^T
// factorisation of the matrix minus x), inside the Gershgorin bound [0, 4n]; then two Newton steps
// on L_n. Weights x_k / ((n + 1) L_{n+1}(x_k))^2.
int sturm_below(int n, double x) {
    int neg = 0;
    double d = 1.0 - x;  // a_0 = 1
    if (d < 0.0) ++neg;
    for (int k = 1; k < n; ++k) {
        if (d == 0.0) d = 1e-300;
        d = (2.0 * k + 1.0 - x) - (double)k * (double)k / d;
        if (d < 0.0) ++neg;
    }
    return neg;
}

bool lag_nodes(int n, double *x, double *w) {
    for (int k = 0; k < n; ++k) {
        double lo = 0.0, hi = 4.0 * n + 2.0;
        for (int it = 0; it < 200 && hi - lo > 1e-15 * hi; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (sturm_below(n, mid) > k) hi = mid;
            else lo = mid;
        }
        double z = 0.5 * (lo + hi);
        for (int it = 0; it < 2; ++it) {
            double ln, lm;
            lag_eval(n, z, ln, lm);
            const double d = n * (ln - lm) / z;
            if (d != 0.0) z -= ln / d;
        }
        x[k] = z;
    }
    for (int k = 0; k < n; ++k) {
        if (!(x[k] > 0.0) || (k && !(x[k] > x[k - 1]))) return false;
        double l1, l0;
        lag_eval(n + 1, x[k], l1, l0);
        w[k] = x[k] / ((n + 1.0) * (n + 1.0) * l1 * l1);
    }
    return true;
}

}  // namespace

namespace vx {

struct NesCommon {
    int N, n_mu, n_p, npair, S, lpp, ppw;
    int species[3];
    double bI[3], bII[3];
    double eps[32], w[32];
    double g2, norm;
    // panel rules: Gauss-Legendre 1 + tau, 1 - tau, weight; Gauss-Laguerre x, weight, e^{-x}
    double gu[kNesMaxP], gv[kNesMaxP], gw[kNesMaxP], lx[kNesMaxP], lw[kNesMaxP], lg[kNesMaxP];
    unsigned char pi_[VX_MAX_PAIRS], pj_[VX_MAX_PAIRS];
};

// per (pair, omega) record: E_min, q0 (value + remainder), the five coefficients, cos(omega)
template <typename R>
struct NesRec {
    R em, em_lo, q0, q0_lo, aI, bI, aII, bII, c, t;
};

template <typename R>
struct NesLaunch {
    NesCommon c;
    const NesRec<R> *tab;  // [npair][n_mu]
    long long Z;
    const int *off;
    int n_rays;
    const double *state, *J, *H;
    double *j0, *chi0, *j1, *chi1, *phi, *jac;
    unsigned long long *counter;
    int *flag;
};

template <typename R> __device__ __forceinline__ R e2(R x);
template <> __device__ __forceinline__ float e2<float>(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double e2<double>(double x) { return exp2(x); }
template <typename R> __device__ __forceinline__ R rc(R x);
template <> __device__ __forceinline__ float rc<float>(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double rc<double>(double x) { return 1.0 / x; }

// Double-word value h + l (|l| <= ulp(h)/2) and the sums the per-unit set-up needs: Knuth's
// two-sum of the high parts, the low parts added to the error, renormalised.
template <typename R>
struct DW {
    R h, l;
};
template <typename R>
__device__ __forceinline__ DW<R> dw_add(DW<R> a, DW<R> b) {
    const R s = a.h + b.h;
    const R v = s - a.h;
    const R e = ((a.h - (s - v)) + (b.h - v)) + (a.l + b.l);
    DW<R> r;
    r.h = s + e;
    r.l = e - (r.h - s);
    return r;
}
template <typename R>
__device__ __forceinline__ DW<R> dw_neg(DW<R> a) {
    a.h = -a.h;
    a.l = -a.l;
    return a;
}

struct NesZone {
    double T, eta, scale, iT2;  // scale: e^{min(eta, 0)}, the zone scale restored at the end
    int bad;
};

// Moments of one (pair, omega) unit: F (q = 0), T^2 dF/dT (q = 1), dF/deta (q = 2), each against
// 1, t, t^2.
template <typename R, bool ADJ>
struct NesMom {
    R m[ADJ ? 3 : 1][3];
};

// Node constants in shared memory, one aligned record per node (a single shared-memory load):
// Gauss-Legendre 1 + tau, 1 - tau, weight; Gauss-Laguerre x, T w and e^{eta_s} e^{-x} (both set
// per zone) and e^{-x}.
template <typename R>
struct alignas(4 * sizeof(R)) NesGl {
    R u, v, w, pad;
};
template <typename R>
struct alignas(4 * sizeof(R)) NesLg {
    R x, wT, og, g;
};

template <typename R, bool ADJ, int NP>
__device__ __forceinline__ void nes_unit(const NesCommon &C, const NesGl<R> *gl, const NesLg<R> *lg,
                                         const NesRec<R> &rec, R mu_h, R mu_l, R T, R iTl, R one, R esl,
                                         NesMom<R, ADJ> &M) {
    const int np = NP > 0 ? NP : C.n_p;
    // offsets of the panels' ends relative to the Fermi edges, from double-word sums
    const DW<R> em = {rec.em, rec.em_lo}, mu = {mu_h, mu_l}, q0w = {rec.q0, rec.q0_lo};
    const DW<R> emr_w = dw_add(em, dw_neg(mu));        // E_min - mu (mu: the upper edge, q0 >= 0)
    const DW<R> emq_w = dw_add(emr_w, q0w);            // E_min - (mu - q0) (the lower edge)
    const R emr = emr_w.h + emr_w.l, emq = emq_w.h + emq_w.l;
    const R q0 = rec.q0, nq0 = -q0;
    const R crel = emr > (R)0 ? emr : (R)0;                 // c - mu, c = max(E_min, mu)
    const R brel = emr > -q0 ? emr : -q0;                    // b - mu, b = max(E_min, mu - q0)
    const R arel = emr > brel - (R)kTail * T ? emr : brel - (R)kTail * T;  // a - mu
    const R bq = emq > (R)0 ? emq : (R)0;                    // b - (mu - q0)
    const R aq = bq - (brel - arel);                         // a - (mu - q0)
    for (int q = 0; q < (ADJ ? 3 : 1); ++q) M.m[q][0] = M.m[q][1] = M.m[q][2] = (R)0;
    // wF: weighted blocking factor F; with the tangents dr = r2 - r1 (dF/deta = F dr) and
    // omr2 = 1 - r2, where r1 = one/(one + e1s) and r2 = 1/(1 + eb) are the two unblocked factors
    auto acc = [&](R wF, R t, R dr, R omr2, R E) {
        const R wt = wF * t;
        M.m[0][0] += wF; M.m[0][1] += wt; M.m[0][2] = fma(wt, t, M.m[0][2]);
        if (ADJ) {
            const R we = wF * dr;                                   // dF/deta
            const R wT = wF * fma(dr, E, omr2 * nq0);               // T^2 dF/dT
            const R wet = we * t, wTt = wT * t;
            M.m[2][0] += we; M.m[2][1] += wet; M.m[2][2] = fma(wet, t, M.m[2][2]);
            M.m[1][0] += wT; M.m[1][1] += wTt; M.m[1][2] = fma(wTt, t, M.m[1][2]);
        }
    };
    // one Gauss-Legendre node: F = 1/(a b), a = one + e1s, b = 1 + eb; r2 - r1 = F (e1s - one eb)
    // and 1 - r2 = eb/b = eb F a, free of cancellation
    auto gl_node = [&](R hw, R t, R e1s, R eb) {
        const R a = one + e1s;
        const R F = rc<R>(a * ((R)1 + eb));
        if (ADJ) acc(hw * F, t, F * fma(-one, eb, e1s), (F * a) * eb, rec.em + t);
        else acc(hw * F, t, (R)0, (R)0, (R)0);
    };
    // panels 1 and 2: Gauss-Legendre. x1 = (E - mu)/T, x2 = x1 + q0/T, in log2 units.
    {
        const R h1 = (R)0.5 * (brel - arel), h2 = (R)0.5 * (crel - brel);
        const R X2a = aq * iTl;                    // x2 at a, anchored at the lower edge
        const R X2b = bq * iTl;                    // x2 at b
        const R X1c = crel * iTl + esl;            // x1 at c, anchored at the upper edge, + eta_s
        const R c1 = esl - q0 * iTl;               // x1 + eta_s = x2 + c1
        const R t1 = arel - emr, t2 = brel - emr;  // t at a and at b
        const R h1l = h1 * iTl, h2l = h2 * iTl;
        // An empty panel (its ends clipped together at E_min) is skipped: there the exponent
        // arguments are unbounded, and its nodes carry zero weight anyway.
        if (h1 > (R)0) {
#pragma unroll 4
            for (int k = 0; k < np; ++k) {  // panel 1: [a, b], b the lower edge, X1 <= X2 <= 0
                const NesGl<R> g = gl[k];
                const R X2 = fma(h1l, g.u, X2a);
                gl_node(h1 * g.w, fma(h1, g.u, t1), e2<R>(X2 + c1), e2<R>(-X2));
            }
        }
        if (h2 > (R)0) {
#pragma unroll 4
            for (int k = 0; k < np; ++k) {  // panel 2: [b, c], c = mu, X1 <= 0 <= X2
                const NesGl<R> g = gl[k];
                const R X2 = fma(h2l, g.u, X2b);
                gl_node(h2 * g.w, fma(h2, g.u, t2), e2<R>(fma(-h2l, g.v, X1c)), e2<R>(-X2));
            }
        }
    }
    // panel 3: Gauss-Laguerre above c, E = c + T x: e^x F = 1 / ((one g + A)(1 + B g)), g = e^{-x}.
    // Where A overflows (the unit lies more than the format's range above the Fermi edge) every
    // node's F is below the format's range: the panel adds nothing.
    {
        const R A = e2<R>(crel * iTl + esl);   // e^{(c - mu)/T} e^{eta_s}
        const R B = e2<R>(-(crel + q0) * iTl);  // e^{-(c - mu + q0)/T}
        const R t3 = crel - emr;
        if (isfinite(A)) {
#pragma unroll 4
            for (int k = 0; k < np; ++k) {
                const NesLg<R> g = lg[k];
                const R Bg = B * g.g, s = g.og + A;
                const R Fx = rc<R>(s * ((R)1 + Bg));
                const R t = fma(T, g.x, t3);
                // r2 = 1/(1 + B g) = Fx s, r1 = og/(og + A): r2 - r1 = Fx (A - og B g), 1 - r2 = B g Fx s
                if (ADJ) acc(g.wT * Fx, t, Fx * fma(-g.og, Bg, A), (Bg * Fx) * s, rec.em + t);
                else acc(g.wT * Fx, t, (R)0, (R)0, (R)0);
            }
        }
    }
}

// Packed node loops (1) for the FP32 form's even unrolled panel sizes, or scalar (0); node pairs
// per unrolled chunk of the packed loops.
#ifndef VX_NES_X2
#define VX_NES_X2 1
#endif
#ifndef VX_NES_X2_UNROLL
#define VX_NES_X2_UNROLL 2
#endif
constexpr int kX2Unroll = VX_NES_X2_UNROLL;

// The FP32 form for even unrolled panel sizes, in packed FP32x2 arithmetic: lane x holds node k
// and lane y node k + NP/2 of the same panel, so an empty panel is still skipped whole. The same
// operations as nes_unit, half the FP32 instructions.
template <bool ADJ, int NP>
__device__ __forceinline__ void nes_unit_x2(const NesGl<float> *gl, const NesLg<float> *lg, const NesRec<float> &rec,
                                            float mu_h, float mu_l, float T, float iTl, float one, float esl,
                                            NesMom<float, ADJ> &M) {
    constexpr int H = NP / 2;
    const DW<float> em = {rec.em, rec.em_lo}, mu = {mu_h, mu_l}, q0w = {rec.q0, rec.q0_lo};
    const DW<float> emr_w = dw_add(em, dw_neg(mu));
    const DW<float> emq_w = dw_add(emr_w, q0w);
    const float emr = emr_w.h + emr_w.l, emq = emq_w.h + emq_w.l;
    const float q0 = rec.q0;
    const float crel = emr > 0.f ? emr : 0.f;
    const float brel = emr > -q0 ? emr : -q0;
    const float arel = emr > brel - (float)kTail * T ? emr : brel - (float)kTail * T;
    const float bq = emq > 0.f ? emq : 0.f;
    const float aq = bq - (brel - arel);
    auto f2 = [](float v) { return make_float2(v, v); };
    const float2 z2 = f2(0.f), one2 = f2(one), none2 = f2(-one), u2 = f2(1.f), nq02 = f2(-q0), Em2 = f2(rec.em);
    float2 m2[ADJ ? 3 : 1][3];
#pragma unroll
    for (int q = 0; q < (ADJ ? 3 : 1); ++q) m2[q][0] = m2[q][1] = m2[q][2] = z2;
    auto acc = [&](float2 wF, float2 t, float2 dr, float2 omr2, float2 E) {
        const float2 wt = __fmul2_rn(wF, t);
        m2[0][0] = __fadd2_rn(m2[0][0], wF); m2[0][1] = __fadd2_rn(m2[0][1], wt); m2[0][2] = __ffma2_rn(wt, t, m2[0][2]);
        if (ADJ) {
            const float2 we = __fmul2_rn(wF, dr);
            const float2 wT = __fmul2_rn(wF, __ffma2_rn(dr, E, __fmul2_rn(omr2, nq02)));
            const float2 wet = __fmul2_rn(we, t), wTt = __fmul2_rn(wT, t);
            m2[2][0] = __fadd2_rn(m2[2][0], we); m2[2][1] = __fadd2_rn(m2[2][1], wet); m2[2][2] = __ffma2_rn(wet, t, m2[2][2]);
            m2[1][0] = __fadd2_rn(m2[1][0], wT); m2[1][1] = __fadd2_rn(m2[1][1], wTt); m2[1][2] = __ffma2_rn(wTt, t, m2[1][2]);
        }
    };
    auto gl_node = [&](float2 hw, float2 t, float2 e1s, float2 eb) {
        const float2 a = __fadd2_rn(one2, e1s);
        const float2 ab = __fmul2_rn(a, __fadd2_rn(u2, eb));
        const float2 F = make_float2(rc<float>(ab.x), rc<float>(ab.y));
        if (ADJ) acc(__fmul2_rn(hw, F), t, __fmul2_rn(F, __ffma2_rn(none2, eb, e1s)), __fmul2_rn(__fmul2_rn(F, a), eb),
                     __fadd2_rn(Em2, t));
        else acc(__fmul2_rn(hw, F), t, z2, z2, z2);
    };
    {
        const float h1 = 0.5f * (brel - arel), h2 = 0.5f * (crel - brel);
        const float2 X2a = f2(aq * iTl), X2b = f2(bq * iTl), X1c = f2(crel * iTl + esl), c1 = f2(esl - q0 * iTl);
        const float2 t1 = f2(arel - emr), t2 = f2(brel - emr);
        const float2 h1v = f2(h1), h2v = f2(h2), h1l = f2(h1 * iTl), h2l = f2(h2 * iTl), nh2l = f2(-h2 * iTl);
        if (h1 > 0.f) {
#pragma unroll kX2Unroll
            for (int k = 0; k < H; ++k) {  // panel 1
                const NesGl<float> g0 = gl[k], g1 = gl[k + H];
                const float2 u = make_float2(g0.u, g1.u);
                const float2 X2 = __ffma2_rn(h1l, u, X2a);
                const float2 x1 = __fadd2_rn(X2, c1);
                gl_node(__fmul2_rn(h1v, make_float2(g0.w, g1.w)), __ffma2_rn(h1v, u, t1),
                        make_float2(e2<float>(x1.x), e2<float>(x1.y)), make_float2(e2<float>(-X2.x), e2<float>(-X2.y)));
            }
        }
        if (h2 > 0.f) {
#pragma unroll kX2Unroll
            for (int k = 0; k < H; ++k) {  // panel 2
                const NesGl<float> g0 = gl[k], g1 = gl[k + H];
                const float2 u = make_float2(g0.u, g1.u);
                const float2 X2 = __ffma2_rn(h2l, u, X2b);
                const float2 x1 = __ffma2_rn(nh2l, make_float2(g0.v, g1.v), X1c);
                gl_node(__fmul2_rn(h2v, make_float2(g0.w, g1.w)), __ffma2_rn(h2v, u, t2),
                        make_float2(e2<float>(x1.x), e2<float>(x1.y)), make_float2(e2<float>(-X2.x), e2<float>(-X2.y)));
            }
        }
    }
    {
        const float A = e2<float>(crel * iTl + esl), B = e2<float>(-(crel + q0) * iTl);
        if (isfinite(A)) {
            const float2 A2 = f2(A), B2 = f2(B), T2 = f2(T), t3 = f2(crel - emr);
#pragma unroll kX2Unroll
            for (int k = 0; k < H; ++k) {  // panel 3
                const NesLg<float> g0 = lg[k], g1 = lg[k + H];
                const float2 og = make_float2(g0.og, g1.og);
                const float2 Bg = __fmul2_rn(B2, make_float2(g0.g, g1.g)), s = __fadd2_rn(og, A2);
                const float2 den = __fmul2_rn(s, __fadd2_rn(u2, Bg));
                const float2 Fx = make_float2(rc<float>(den.x), rc<float>(den.y));
                const float2 t = __ffma2_rn(T2, make_float2(g0.x, g1.x), t3);
                const float2 wF = __fmul2_rn(make_float2(g0.wT, g1.wT), Fx);
                if (ADJ)
                    acc(wF, t, __fmul2_rn(Fx, __ffma2_rn(make_float2(-og.x, -og.y), Bg, A2)),
                        __fmul2_rn(__fmul2_rn(Bg, Fx), s), __fadd2_rn(Em2, t));
                else acc(wF, t, z2, z2, z2);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < (ADJ ? 3 : 1); ++q)
#pragma unroll
        for (int n = 0; n < 3; ++n) M.m[q][n] = m2[q][n].x + m2[q][n].y;
}


// Minimum CTAs per SM the register allocation is bounded for (1: no bound).
#ifndef VX_NES_MINB
#define VX_NES_MINB 1
#endif

template <typename R, bool ADJ, int NP>
__global__ void __launch_bounds__(kNesBlock, VX_NES_MINB) k_nes(const __grid_constant__ NesLaunch<R> L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ NesZone zs;
    __shared__ long long s_zone;
    __shared__ NesGl<R> sgl[kNesMaxP];
    __shared__ NesLg<R> slg[kNesMaxP];
    __shared__ R zr[6];  // mu (value, remainder), T, log2(e)/T, e^{eta_s}, eta_s log2(e)
    const NesCommon &C = L.c;
    const int N = C.N, N2 = N * N, S = C.S;
    constexpr int NQ = ADJ ? 3 : 1;
    // D[q][X][l][i][j] (i >= j filled): the down-scattering kernel and its tangents
    R *D = reinterpret_cast<R *>(smraw);
    R *Xf = D + (size_t)NQ * 4 * N2;  // [N][N] e^{-|eps_i - eps_j|/T} of the zone
    R *dE = Xf + N2;                  // [N][N] |eps_i - eps_j|
    R *vec = dE + N2;                 // [4][S][N] w_j (J_j, 1 - J_j, H_j, H_j) of the zone
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int k = tid; k < C.n_p; k += blockDim.x) {
        sgl[k].u = (R)C.gu[k];
        sgl[k].v = (R)C.gv[k];
        sgl[k].w = (R)C.gw[k];
        sgl[k].pad = (R)0;
        slg[k].x = (R)C.lx[k];
        slg[k].g = (R)C.lg[k];
    }
    for (int e = tid; e < N2; e += blockDim.x) dE[e] = (R)fabs(C.eps[e / N] - C.eps[e % N]);
    validate_offsets(L.off, L.n_rays, L.Z, L.flag);
    const int lpp = C.lpp, ppw = C.ppw, grp = lane / lpp, m = lane % lpp;
    const bool active = m < C.n_mu;
    const R L2E = (R)1.4426950408889634;
    for (;;) {
        if (tid == 0) {
            s_zone = (long long)atomicAdd(L.counter, 1ull);
            const long long z = s_zone;
            if (z < L.Z) {
                const double T = L.state[4 * z + 0], eta = L.state[4 * z + 1];
                zs.T = T;
                zs.eta = eta;
                zs.bad = !(T > 0.0) || !isfinite(T) || !isfinite(eta) || fabs(eta) > VX_ETA_MAX;
                if (!zs.bad) {  // the zone's scalars, once (FP64 here, R in the loops)
                    const double mu = eta * T, etas = eta < 0.0 ? eta : 0.0;
                    zr[0] = (R)mu;
                    zr[1] = (R)(mu - (double)zr[0]);
                    zr[2] = (R)T;
                    zr[3] = (R)(1.4426950408889634 / T);
                    zs.scale = exp(etas);
                    zr[4] = (R)zs.scale;
                    zr[5] = (R)(etas * 1.4426950408889634);
                    zs.iT2 = 1.0 / (T * T);
                    for (int k = 0; k < C.n_p; ++k) {  // the Laguerre panel's zone factors
                        slg[k].wT = (R)(T * C.lw[k]);
                        slg[k].og = (R)(zs.scale * C.lg[k]);
                    }
                }
            }
        }
        __syncthreads();
        const long long z = s_zone;
        if (z >= L.Z) break;
        if (zs.bad) {
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            for (int e = tid; e < S * N; e += blockDim.x) {
                const size_t o = (size_t)z * S * N + e;
                if (L.j0) { L.j0[o] = nan; L.chi0[o] = nan; L.j1[o] = nan; L.chi1[o] = nan; }
                if (ADJ && L.jac)
                    for (int q = 0; q < 12; ++q) L.jac[o * 12 + q] = nan;
            }
            if (L.phi)
                for (int e = tid; e < 8 * N2; e += blockDim.x) L.phi[(size_t)z * 8 * N2 + e] = nan;
            if (tid == 0) atomicOr(L.flag, VX_FLAG_BAD_STATE);
            __syncthreads();
            continue;
        }
        const R mu_h = zr[0], mu_l = zr[1], T = zr[2], iTl = zr[3], one = zr[4], esl = zr[5];
        // detailed-balance factors and contraction vectors of the zone
        for (int e = tid; e < N2; e += blockDim.x) Xf[e] = e2<R>(-dE[e] * iTl);
        for (int e = tid; e < 4 * S * N; e += blockDim.x) {
            const int o = e / (S * N), j = e % N;
            const double Jj = L.J[(size_t)z * S * N + e % (S * N)], Hj = L.H[(size_t)z * S * N + e % (S * N)];
            vec[e] = (R)(C.w[j] * (o == 0 ? Jj : o == 1 ? 1.0 - Jj : Hj));
        }
        // quadrature: groups of lpp lanes per bin pair, lanes over cos(omega)
        const int slots = (C.npair + nwarp * ppw - 1) / (nwarp * ppw);
        for (int sl = 0; sl < slots; ++sl) {
            const int p = (sl * nwarp + warp) * ppw + grp;
            R v[NQ][4];
#pragma unroll
            for (int q = 0; q < NQ; ++q) v[q][0] = v[q][1] = v[q][2] = v[q][3] = (R)0;
            if (active && p < C.npair) {
                const NesRec<R> rec = L.tab[(size_t)p * C.n_mu + m];
                NesMom<R, ADJ> M;
                if constexpr (std::is_same<R, float>::value && VX_NES_X2 && NP > 0 && NP % 2 == 0)
                    nes_unit_x2<ADJ, NP>(sgl, slg, rec, mu_h, mu_l, T, iTl, one, esl, M);
                else
                    nes_unit<R, ADJ, NP>(C, sgl, slg, rec, mu_h, mu_l, T, iTl, one, esl, M);
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const R kI = fma(rec.aI, M.m[q][0], fma(rec.bI, M.m[q][1], rec.c * M.m[q][2]));
                    const R kII = fma(rec.aII, M.m[q][0], fma(rec.bII, M.m[q][1], rec.c * M.m[q][2]));
                    v[q][0] = kI; v[q][1] = kII; v[q][2] = rec.t * kI; v[q][3] = rec.t * kII;
                }
            }
            // sum over the group's lanes (fixed butterfly: deterministic)
            for (int off = lpp >> 1; off > 0; off >>= 1)
#pragma unroll
                for (int q = 0; q < NQ; ++q)
#pragma unroll
                    for (int r = 0; r < 4; ++r) v[q][r] += __shfl_xor_sync(0xffffffffu, v[q][r], off);
            if (m == 0 && p < C.npair) {
                const int i = C.pi_[p], j = C.pj_[p];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    // [q][X][l]: v = {I l0, II l0, I l1, II l1}
                    D[((q * 2 + 0) * 2 + 0) * N2 + i * N + j] = v[q][0];
                    D[((q * 2 + 1) * 2 + 0) * N2 + i * N + j] = v[q][1];
                    D[((q * 2 + 0) * 2 + 1) * N2 + i * N + j] = v[q][2];
                    D[((q * 2 + 1) * 2 + 1) * N2 + i * N + j] = v[q][3];
                }
            }
        }
        __syncthreads();
        // kernel of a direction: out(i,j) = D(i,j) for i >= j, X D(j,i) above; in(i,j) = X D(i,j)
        // for i >= j, D(j,i) above. Tangents: dX/dT = X |de|/T^2 (q = 1 holds T^2 dD/dT).
        auto kern = [&](int q, int X, int l, int dir, int i, int j) -> R {
            const bool low = i >= j;
            const int a = low ? i : j, b = low ? j : i;
            const R d = D[((q * 2 + X) * 2 + l) * N2 + a * N + b];
            const bool scaled = (dir == 1) != low;  // out above the diagonal, in on and below it
            if (!scaled || i == j) return d;
            const R x = Xf[i * N + j];
            if (q == 1) {
                const R d0 = D[((0 * 2 + X) * 2 + l) * N2 + a * N + b];
                return x * fma(d0, dE[i * N + j], d);
            }
            return x * d;
        };
        const double scale = zs.scale, two_pi = 6.283185307179586;
        for (int e = tid; e < 4 * S * N; e += blockDim.x) {
            const int o = e / (S * N), s = (e / N) % S, i = e % N;
            const int l = o >> 1, dir = o & 1;  // j0: in l0, chi0: out l0, j1: in l1, chi1: out l1
            const R bI = (R)C.bI[s], bII = (R)C.bII[s];
            const size_t row = ((size_t)z * S + s) * N;
            const R *vo = vec + (size_t)(o * S + s) * N;
            double res[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                R acc = (R)0;
                for (int j = 0; j < N; ++j)
                    acc = fma(fma(bI, kern(q, 0, l, dir, i, j), bII * kern(q, 1, l, dir, i, j)), vo[j], acc);
                res[q] = (double)acc;
            }
            const double cl = (l ? -3.0 : 1.0) * two_pi * C.norm * scale;
            const size_t oi = row + i;
            const double fwd = cl * res[0];
            if (L.j0) {
                double *dst = o == 0 ? L.j0 : o == 1 ? L.chi0 : o == 2 ? L.j1 : L.chi1;
                dst[oi] = fwd;
                if (!isfinite(fwd)) atomicOr(L.flag, VX_FLAG_NONFINITE);
            }
            if (ADJ && L.jac) {
                const double dT = cl * res[1] * zs.iT2, dEta = cl * res[2];
                L.jac[oi * 12 + o * 3 + 0] = dT;
                L.jac[oi * 12 + o * 3 + 1] = dEta;
                L.jac[oi * 12 + o * 3 + 2] = 0.0;
                if (!isfinite(dT) || !isfinite(dEta)) atomicOr(L.flag, VX_FLAG_NONFINITE);
            }
        }
        if (L.phi) {  // [X][dir][l][i][j], G2 applied (in the table), zone scale restored
            for (int e = tid; e < 8 * N2; e += blockDim.x) {
                const int X = e / (4 * N2), dir = (e / (2 * N2)) & 1, l = (e / N2) & 1, ij = e % N2;
                L.phi[(size_t)z * 8 * N2 + e] = scale * (double)kern(0, X, l, dir, ij / N, ij % N);
            }
        }
        __syncthreads();
    }
}

template <typename R, bool ADJ>
const void *nes_kernel(int n_p) {
    switch (n_p) {
        case 8: return (const void *)k_nes<R, ADJ, 8>;
        case 16: return (const void *)k_nes<R, ADJ, 16>;
        default: return (const void *)k_nes<R, ADJ, 0>;
    }
}

template <typename R, bool ADJ>
cudaError_t nes_launch(const NesLaunch<R> &L, int grid, size_t smem, cudaStream_t s) {
    switch (L.c.n_p) {
        case 8: k_nes<R, ADJ, 8><<<grid, kNesBlock, smem, s>>>(L); break;
        case 16: k_nes<R, ADJ, 16><<<grid, kNesBlock, smem, s>>>(L); break;
        default: k_nes<R, ADJ, 0><<<grid, kNesBlock, smem, s>>>(L); break;
    }
    return cudaGetLastError();
}

// ---- electron-gas closure -------------------------------------------------------------------
// eta from the cubic eta^3 + pi^2 eta = q by Newton's method from a bracketing start (the
// function is increasing and convex for eta >= 0; from above the root Newton converges
// monotonically), then the derivatives by implicit differentiation.
__global__ void k_eos_eta(long long Z, double *state, double *deta) {
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= Z) return;
    const double hbarc = 1.973269804e-11, mu_g = 1.66053906660e-24, p = 9.869604401089358;  // pi^2
    const double T = state[4 * z + 0], ye = state[4 * z + 2], rho = state[4 * z + 3];
    double eta = __longlong_as_double(0x7ff8000000000000ll), d0 = eta, d1 = eta, d2 = eta;
    if (T > 0.0 && ye >= 0.0 && rho >= 0.0 && isfinite(T) && isfinite(ye) && isfinite(rho)) {
        const double r = hbarc / T;
        const double q = 3.0 * p * (rho * ye / mu_g) * r * r * r;
        // start above the root: eta^3 + p eta >= max(eta^3, p eta), so eta0 = max(cbrt(q), q/p) works
        double e = fmax(cbrt(q), q / p);
        for (int it = 0; it < 100; ++it) {
            const double f = fma(e * e, e, p * e) - q, df = fma(3.0 * e, e, p);
            const double step = f / df;
            e -= step;
            if (!(fabs(step) > 1e-16 * fmax(e, 1e-300))) break;
        }
        eta = e;
        const double dedq = 1.0 / fma(3.0 * e, e, p);
        d0 = dedq * (-3.0 * q / T);
        d1 = dedq * (ye > 0.0 ? q / ye : 3.0 * p * (rho / mu_g) * r * r * r);
        d2 = dedq * (rho > 0.0 ? q / rho : 3.0 * p * (ye / mu_g) * r * r * r);
    }
    state[4 * z + 1] = eta;
    if (deta) { deta[3 * z + 0] = d0; deta[3 * z + 1] = d1; deta[3 * z + 2] = d2; }
}

__global__ void k_eos_chain(long long Z, int rows, const double *deta, const double *jin, double *jout) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Z * rows) return;
    const long long z = e / rows;
    const double dT = jin[3 * e + 0], dE = jin[3 * e + 1], dY = jin[3 * e + 2];
    const double a = deta[3 * z + 0], b = deta[3 * z + 1], c = deta[3 * z + 2];
    jout[3 * e + 0] = fma(dE, a, dT);
    jout[3 * e + 1] = fma(dE, b, dY);
    jout[3 * e + 2] = dE * c;
}

}  // namespace vx

struct vx_nes {
    int device = 0, nsm = 0;
    vx::NesCommon c{};
    int prec = VX_PREC_MIXED;
    void *d_tab = nullptr;
    unsigned long long *d_counter = nullptr;
    int *d_flag = nullptr;
    size_t smem[2] = {0, 0};
    int grid[2] = {0, 0};
    // host-buffer calls: two staging slots of device memory, a stream and a work counter each
    double *hbuf[2] = {nullptr, nullptr};
    cudaStream_t hst[2] = {nullptr, nullptr};
    unsigned long long *hcnt = nullptr;
    size_t hbytes = 0;
};

namespace {

// Builds the (pair, omega) table in FP64: E_min = eps eps' y/(Q + q0), the coefficients of the
// azimuth-averaged matrix elements in t = E - E_min (all non-negative), with u = eps eps' y/Q,
// sigma = eps + eps', G = (eps eps')^2 y (2 - y), sigma - Q = 2 eps eps' (2 - y)/(sigma + Q):
//   a_I = u^2 Q^2 (sigma + Q)(sigma - Q)/(4 Q^2) + u^2 Q (sigma + Q)/2,  a_II = u^2 (sigma - Q)^2/4,
//   b_I = u^2 sigma^2/Q + u G/Q^2 + u^2 sigma,  b_II = u^2 sigma (sigma - Q)/Q + u G/Q^2,
//   c = u^2 sigma^2/Q^2 + u G/Q^3,
// each times G2 w_omega 2 pi/(4 Q eps eps').
template <typename R>
std::vector<vx::NesRec<R>> nes_table(const vx::NesCommon &C, const double *tmu, const double *wmu) {
    const double pi = 3.14159265358979323846;
    std::vector<vx::NesRec<R>> tab((size_t)C.npair * C.n_mu);
    for (int p = 0; p < C.npair; ++p) {
        const double e = C.eps[C.pi_[p]], ep = C.eps[C.pj_[p]];
        for (int m = 0; m < C.n_mu; ++m) {
            const double t = tmu[m], y = 1.0 - t, g = e * ep, q0 = e - ep;
            const double Q = std::sqrt(q0 * q0 + 2.0 * g * y), s = e + ep;
            const double Em = g * y / (Q + q0), u = g * y / Q, G = g * g * y * (2.0 - y);
            const double smQ = 2.0 * g * (2.0 - y) / (s + Q);
            const double pref = C.g2 * wmu[m] * 2.0 * pi / (4.0 * Q * g);
            const double aI = u * u * (Q * (s + Q)) * (Q * smQ) / (4.0 * Q * Q) + u * u * Q * (s + Q) / 2.0;
            const double aII = u * u * smQ * smQ / 4.0;
            const double bI = u * u * s * s / Q + u * G / (Q * Q) + u * u * s;
            const double bII = u * u * s * smQ / Q + u * G / (Q * Q);
            const double cc = u * u * s * s / (Q * Q) + u * G / (Q * Q * Q);
            vx::NesRec<R> &r = tab[(size_t)p * C.n_mu + m];
            r.em = (R)Em; r.em_lo = (R)(Em - (double)r.em);
            r.q0 = (R)q0; r.q0_lo = (R)(q0 - (double)r.q0);
            r.aI = (R)(pref * aI); r.bI = (R)(pref * bI); r.aII = (R)(pref * aII); r.bII = (R)(pref * bII);
            r.c = (R)(pref * cc); r.t = (R)t;
        }
    }
    return tab;
}

size_t nes_smem(const vx::NesCommon &C, bool adj, bool dbl) {
    const size_t r = dbl ? 8 : 4, N2 = (size_t)C.N * C.N;
    return ((adj ? 3 : 1) * 4 * N2 + 2 * N2 + 4 * (size_t)C.S * C.N) * r;
}

vx_status nes_validate_batch(const vx_nes *h, const vx_batch *b) {
    if (!h) return nfail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (!b) return nfail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_zones < 0 || b->n_rays < 0) return nfail(VX_ERR_INVALID_ARG, "negative batch size");
    if (b->n_zones == 0) return VX_OK;
    vx_status s;
    if (b->ray_offsets) {
        if (b->n_rays == 0) return nfail(VX_ERR_INVALID_ARG, "n_zones > 0 with no rays");
        if ((s = device_ptr(b->ray_offsets, 4, "ray_offsets")) != VX_OK) return s;
    }
    if ((s = device_ptr(b->state, 8, "state")) != VX_OK) return s;
    if ((s = device_ptr(b->J, 8, "J")) != VX_OK) return s;
    if ((s = device_ptr(b->H, 8, "H")) != VX_OK) return s;
    return VX_OK;
}

vx_status nes_validate_out(const vx_out *o, bool allow_phi) {
    vx_status s;
    const double *a[4] = {o->j0, o->chi0, o->j1, o->chi1};
    const char *nm[4] = {"out.j0", "out.chi0", "out.j1", "out.chi1"};
    for (int k = 0; k < 4; ++k)
        if ((s = device_ptr(a[k], 8, nm[k])) != VX_OK) return s;
    if (o->phi) {
        if (!allow_phi) return nfail(VX_ERR_INVALID_ARG, "phi output is not produced by this call");
        if ((s = device_ptr(o->phi, 8, "out.phi")) != VX_OK) return s;
    }
    return VX_OK;
}

template <typename R>
vx_status nes_run(vx_nes *h, const vx_batch *b, const vx_out *out, double *jac, cudaStream_t s,
                  unsigned long long *counter = nullptr) {
    vx::NesLaunch<R> L{};
    L.c = h->c;
    L.tab = reinterpret_cast<const vx::NesRec<R> *>(h->d_tab);
    L.Z = b->n_zones;
    L.off = b->ray_offsets;
    L.n_rays = b->n_rays;
    L.state = b->state; L.J = b->J; L.H = b->H;
    if (out) { L.j0 = out->j0; L.chi0 = out->chi0; L.j1 = out->j1; L.chi1 = out->chi1; L.phi = out->phi; }
    L.jac = jac;
    L.counter = counter ? counter : h->d_counter;
    L.flag = h->d_flag;
    const bool adj = jac != nullptr;
    const int grid = (int)std::min<long long>(h->grid[adj], b->n_zones);
    NES_CU(cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), s));
    const cudaError_t e = adj ? vx::nes_launch<R, true>(L, grid, h->smem[1], s) : vx::nes_launch<R, false>(L, grid, h->smem[0], s);
    NES_CU(e);
    return VX_OK;
}

// Host-buffer calls: the batch in chunks of zones through the handle's two staging slots
// (640 MiB each, or VX_HOST_SLOT_MB MiB from the environment, allocated on first use); each slot
// has its own stream and work counter, so the
// copies of one chunk overlap the kernel of the next. Host arrays should be pinned for the copies
// to be asynchronous; the call returns when every output is in host memory.
constexpr size_t kNesHostSlot = 640ull << 20;

vx_status nes_host_run(vx_nes *h, const vx_batch *b, const vx_out *fwd, double *jac) {
    if (!h) return nfail(VX_ERR_INVALID_ARG, "handle is NULL");
    if (!b) return nfail(VX_ERR_INVALID_ARG, "batch is NULL");
    if (b->n_zones < 0 || b->n_rays < 0) return nfail(VX_ERR_INVALID_ARG, "negative batch size");
    if (b->ray_offsets) {
        if (b->ray_offsets[0] != 0) return nfail(VX_ERR_INVALID_ARG, "ray_offsets[0] must be 0");
        for (int r = 0; r < b->n_rays; ++r)
            if (b->ray_offsets[r + 1] < b->ray_offsets[r])
                return nfail(VX_ERR_INVALID_ARG, "ray_offsets must be non-decreasing (ray %d)", r);
        if ((long long)b->ray_offsets[b->n_rays] != b->n_zones)
            return nfail(VX_ERR_INVALID_ARG, "ray_offsets[n_rays] does not equal n_zones");
    }
    if (fwd && (!fwd->j0 || !fwd->chi0 || !fwd->j1 || !fwd->chi1)) return nfail(VX_ERR_INVALID_ARG, "an output array is NULL");
    if (fwd && fwd->phi) return nfail(VX_ERR_INVALID_ARG, "phi output is not produced by the host-buffer calls");
    if (b->n_zones == 0) return VX_OK;
    if (!b->state || !b->J || !b->H) return nfail(VX_ERR_INVALID_ARG, "state, J and H must be host arrays");
    int cur = 0;
    NES_CU(cudaGetDevice(&cur));
    NES_CU(cudaSetDevice(h->device));
    struct Restore {
        int d;
        ~Restore() { cudaSetDevice(d); }
    } restore{cur};
    if (!h->hbuf[0]) {
        h->hbytes = kNesHostSlot;
        if (const char *mb = getenv("VX_HOST_SLOT_MB")) {  // slot size override, MiB
            const long long v = atoll(mb);
            if (v >= 1 && v <= (1ll << 20)) h->hbytes = (size_t)v << 20;
        }
        for (int k = 0; k < 2; ++k) {
            NES_CU(cudaMalloc(&h->hbuf[k], h->hbytes));
            NES_CU(cudaStreamCreateWithFlags(&h->hst[k], cudaStreamNonBlocking));
        }
        NES_CU(cudaMalloc(&h->hcnt, 2 * sizeof(unsigned long long)));
    }
    const size_t SN = (size_t)h->c.S * h->c.N;
    const size_t per = 4 + 2 * SN + (fwd ? 4 * SN : 0) + (jac ? 12 * SN : 0);  // doubles per zone
    const long long chunk = (long long)(h->hbytes / (per * sizeof(double)));
    if (chunk < 1) return nfail(VX_ERR_UNSUPPORTED, "one zone does not fit a staging slot");
    const long long Z = b->n_zones;
    for (long long c = 0, z0 = 0; z0 < Z; ++c, z0 += chunk) {
        const long long n = std::min(chunk, Z - z0);
        const int sl = (int)(c & 1);
        cudaStream_t s = h->hst[sl];
        double *p = h->hbuf[sl];
        auto take = [&](size_t count) { double *q = p; p += count; return q; };
        double *d_state = take(4 * n), *d_J = take(SN * n), *d_H = take(SN * n);
        NES_CU(cudaMemcpyAsync(d_state, b->state + 4 * z0, 4 * n * sizeof(double), cudaMemcpyHostToDevice, s));
        NES_CU(cudaMemcpyAsync(d_J, b->J + SN * z0, SN * n * sizeof(double), cudaMemcpyHostToDevice, s));
        NES_CU(cudaMemcpyAsync(d_H, b->H + SN * z0, SN * n * sizeof(double), cudaMemcpyHostToDevice, s));
        const vx_batch db{0, n, nullptr, d_state, d_J, d_H};
        vx_out dout{};
        double *d_out = nullptr, *d_jac = nullptr;
        if (fwd) {
            d_out = take(4 * SN * n);
            dout.j0 = d_out; dout.chi0 = d_out + SN * n; dout.j1 = d_out + 2 * SN * n; dout.chi1 = d_out + 3 * SN * n;
        }
        if (jac) d_jac = take(12 * SN * n);
        const vx_status st = h->prec == VX_PREC_FP64 ? nes_run<double>(h, &db, fwd ? &dout : nullptr, d_jac, s, h->hcnt + sl)
                                                     : nes_run<float>(h, &db, fwd ? &dout : nullptr, d_jac, s, h->hcnt + sl);
        if (st != VX_OK) return st;
        if (fwd) {
            double *dst[4] = {fwd->j0, fwd->chi0, fwd->j1, fwd->chi1};
            for (int k = 0; k < 4; ++k)
                NES_CU(cudaMemcpyAsync(dst[k] + SN * z0, d_out + k * SN * n, SN * n * sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
        }
        if (d_jac)
            NES_CU(cudaMemcpyAsync(jac + 12 * SN * z0, d_jac, 12 * SN * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    NES_CU(cudaStreamSynchronize(h->hst[0]));
    NES_CU(cudaStreamSynchronize(h->hst[1]));
    return VX_OK;
}

}  // namespace

extern "C" {

vx_status vx_nes_eval_host(vx_nes *h, const vx_batch *host_batch, const vx_out *host_out) {
    if (!host_out) return nfail(VX_ERR_INVALID_ARG, "out is NULL");
    return nes_host_run(h, host_batch, host_out, nullptr);
}

vx_status vx_nes_adjoint_host(vx_nes *h, const vx_batch *host_batch, double *host_jac, const vx_out *host_fwd) {
    if (!host_jac) return nfail(VX_ERR_INVALID_ARG, "jac is NULL");
    return nes_host_run(h, host_batch, host_fwd, host_jac);
}

vx_status vx_nes_create(const vx_config *cfg, vx_nes **out) {
    if (!out) return nfail(VX_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!cfg) return nfail(VX_ERR_INVALID_ARG, "config is NULL");
    if (cfg->n_bins < 2 || cfg->n_bins > VX_MAX_BINS - 1) return nfail(VX_ERR_INVALID_ARG, "n_bins %d outside 2..31", cfg->n_bins);
    if (!cfg->eps) return nfail(VX_ERR_INVALID_ARG, "eps is NULL");
    for (int i = 0; i < cfg->n_bins; ++i) {
        if (!(cfg->eps[i] > 0.0) || !std::isfinite(cfg->eps[i])) return nfail(VX_ERR_INVALID_ARG, "eps[%d] must be finite and > 0", i);
        if (i && !(cfg->eps[i] > cfg->eps[i - 1])) return nfail(VX_ERR_INVALID_ARG, "eps must be strictly increasing");
        if (cfg->weights && (!(cfg->weights[i] > 0.0) || !std::isfinite(cfg->weights[i])))
            return nfail(VX_ERR_INVALID_ARG, "weights[%d] must be finite and > 0", i);
    }
    if (cfg->n_mu < 2 || cfg->n_mu > kNesMaxMu) return nfail(VX_ERR_INVALID_ARG, "n_mu %d outside 2..%d", cfg->n_mu, kNesMaxMu);
    if (cfg->n_e < 6 || cfg->n_e > 3 * kNesMaxP || cfg->n_e % 3)
        return nfail(VX_ERR_INVALID_ARG, "n_e %d must be a multiple of 3 in 6..%d", cfg->n_e, 3 * kNesMaxP);
    if (cfg->n_species < 1 || cfg->n_species > 3 || !cfg->species) return nfail(VX_ERR_INVALID_ARG, "n_species must be 1..3");
    for (int s = 0; s < cfg->n_species; ++s) {
        if (cfg->species[s] < 0 || cfg->species[s] > 2) return nfail(VX_ERR_INVALID_ARG, "species[%d] is not a vx_species", s);
        for (int t = 0; t < s; ++t)
            if (cfg->species[t] == cfg->species[s]) return nfail(VX_ERR_INVALID_ARG, "species listed twice");
    }
    if (!std::isfinite(cfg->sin2w) || !std::isfinite(cfg->g2) || !std::isfinite(cfg->norm))
        return nfail(VX_ERR_INVALID_ARG, "sin2w, g2 and norm must be finite");
    if (cfg->prec != VX_PREC_MIXED && cfg->prec != VX_PREC_FP64) return nfail(VX_ERR_INVALID_ARG, "unknown precision");
    if (cfg->flags != 0 || cfg->eta_fp64 != 0.0) return nfail(VX_ERR_INVALID_ARG, "flags and eta_fp64 must be 0 for NES");

    vx_nes *h = new vx_nes();
    h->prec = cfg->prec;
    vx::NesCommon &C = h->c;
    const int N = cfg->n_bins;
    C.N = N; C.n_mu = cfg->n_mu; C.n_p = cfg->n_e / 3; C.S = cfg->n_species;
    C.npair = N * (N + 1) / 2;
    int lpp = 1;
    while (lpp < C.n_mu) lpp <<= 1;
    C.lpp = lpp;
    C.ppw = 32 / lpp;
    C.g2 = cfg->g2;
    C.norm = cfg->norm;
    for (int i = 0; i < N; ++i) {
        C.eps[i] = cfg->eps[i];
        if (cfg->weights) C.w[i] = cfg->weights[i];
        else {
            const double *e = cfg->eps;
            const double lo = i ? std::sqrt(e[i - 1] * e[i]) : e[0] * std::sqrt(e[0] / e[1]);
            const double hi = i < N - 1 ? std::sqrt(e[i] * e[i + 1]) : e[N - 1] * std::sqrt(e[N - 1] / e[N - 2]);
            C.w[i] = e[i] * e[i] * (hi - lo);
        }
    }
    for (int s = 0; s < C.S; ++s) {
        const int sp = cfg->species[s];
        C.species[s] = sp;
        const double cv = (sp == VX_NU_X ? -0.5 : 0.5) + 2.0 * cfg->sin2w, ca = sp == VX_NU_X ? -0.5 : 0.5;
        double b1 = (cv + ca) * (cv + ca), b2 = (cv - ca) * (cv - ca);
        if (sp == VX_NU_EBAR) std::swap(b1, b2);
        C.bI[s] = b1;
        C.bII[s] = b2;
    }
    {
        int p = 0;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j <= i; ++j) { C.pi_[p] = (unsigned char)i; C.pj_[p] = (unsigned char)j; ++p; }
    }
    double tmu[kNesMaxMu], wmu[kNesMaxMu], tg[kNesMaxP], wg[kNesMaxP], xl[kNesMaxP], wl[kNesMaxP];
    gl_nodes(C.n_mu, tmu, wmu);
    gl_nodes(C.n_p, tg, wg);
    if (!lag_nodes(C.n_p, xl, wl)) { delete h; return nfail(VX_ERR_INVALID_ARG, "Gauss-Laguerre nodes did not converge"); }
    for (int k = 0; k < C.n_p; ++k) {
        C.gu[k] = 1.0 + tg[k]; C.gv[k] = 1.0 - tg[k]; C.gw[k] = wg[k];
        C.lx[k] = xl[k]; C.lw[k] = wl[k]; C.lg[k] = std::exp(-xl[k]);
    }
    auto cleanup = [&](vx_status st) { vx_nes_destroy(h); return st; };
    cudaDeviceProp prop;
    if (cudaGetDevice(&h->device) != cudaSuccess || cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
        delete h;
        return nfail(VX_ERR_CUDA, "no CUDA device");
    }
    h->nsm = prop.multiProcessorCount;
    const bool dbl = h->prec == VX_PREC_FP64;
    size_t tb;
    if (dbl) {
        auto t = nes_table<double>(C, tmu, wmu);
        tb = t.size() * sizeof(t[0]);
        if (cudaMalloc(&h->d_tab, tb) != cudaSuccess || cudaMemcpy(h->d_tab, t.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(nfail(VX_ERR_OOM, "table upload failed"));
    } else {
        auto t = nes_table<float>(C, tmu, wmu);
        tb = t.size() * sizeof(t[0]);
        if (cudaMalloc(&h->d_tab, tb) != cudaSuccess || cudaMemcpy(h->d_tab, t.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(nfail(VX_ERR_OOM, "table upload failed"));
    }
    if (cudaMalloc(&h->d_counter, sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&h->d_flag, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->d_flag, 0, sizeof(int)) != cudaSuccess)
        return cleanup(nfail(VX_ERR_OOM, "allocation failed"));
    for (int adj = 0; adj < 2; ++adj) {
        h->smem[adj] = nes_smem(C, adj != 0, dbl);
        const void *fn = dbl ? (adj ? vx::nes_kernel<double, true>(C.n_p) : vx::nes_kernel<double, false>(C.n_p))
                             : (adj ? vx::nes_kernel<float, true>(C.n_p) : vx::nes_kernel<float, false>(C.n_p));
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem[adj]) != cudaSuccess)
            return cleanup(nfail(VX_ERR_CUDA, "shared memory attribute"));
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kNesBlock, h->smem[adj]) != cudaSuccess || occ < 1)
            return cleanup(nfail(VX_ERR_UNSUPPORTED, "NES kernel does not fit on an SM"));
        h->grid[adj] = occ * h->nsm;
    }
    *out = h;
    return VX_OK;
}

vx_status vx_nes_eval(vx_nes *h, const vx_batch *b, const vx_out *out, vx_stream stream) {
    vx_status st = nes_validate_batch(h, b);
    if (st != VX_OK) return st;
    if (!out) return nfail(VX_ERR_INVALID_ARG, "out is NULL");
    if (b->n_zones == 0) return VX_OK;
    if ((st = nes_validate_out(out, true)) != VX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return h->prec == VX_PREC_FP64 ? nes_run<double>(h, b, out, nullptr, s) : nes_run<float>(h, b, out, nullptr, s);
}

vx_status vx_nes_adjoint(vx_nes *h, const vx_batch *b, double *jac, const vx_out *fwd, vx_stream stream) {
    vx_status st = nes_validate_batch(h, b);
    if (st != VX_OK) return st;
    if (!jac) return nfail(VX_ERR_INVALID_ARG, "jac is NULL");
    if (b->n_zones == 0) return VX_OK;
    if ((st = device_ptr(jac, 8, "jac")) != VX_OK) return st;
    if (fwd && (st = nes_validate_out(fwd, false)) != VX_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    return h->prec == VX_PREC_FP64 ? nes_run<double>(h, b, fwd, jac, s) : nes_run<float>(h, b, fwd, jac, s);
}

vx_status vx_nes_check(vx_nes *h, vx_stream stream) {
    if (!h) return nfail(VX_ERR_INVALID_ARG, "handle is NULL");
    NES_CU(cudaStreamSynchronize((cudaStream_t)stream));
    int f = 0;
    NES_CU(cudaMemcpy(&f, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) {
        NES_CU(cudaMemset(h->d_flag, 0, sizeof(int)));
        return nfail(VX_ERR_NUMERIC, "NES device flag 0x%x (%s%s%s)", f, (f & VX_FLAG_BAD_STATE) ? "invalid zone state; " : "",
                     (f & VX_FLAG_NONFINITE) ? "non-finite result; " : "", (f & VX_FLAG_BAD_OFFSETS) ? "invalid ray offsets" : "");
    }
    return VX_OK;
}

void vx_nes_destroy(vx_nes *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    cudaFree(h->d_tab);
    cudaFree(h->d_counter);
    cudaFree(h->d_flag);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->hbuf[k]);
        if (h->hst[k]) cudaStreamDestroy(h->hst[k]);
    }
    cudaFree(h->hcnt);
    delete h;
}

vx_status vx_eos_eta(long long n_zones, double *state, double *deta, vx_stream stream) {
    if (n_zones < 0) return nfail(VX_ERR_INVALID_ARG, "n_zones < 0");
    if (n_zones == 0) return VX_OK;
    if (!state) return nfail(VX_ERR_INVALID_ARG, "state is NULL");
    vx_status st;
    if ((st = device_ptr(state, 8, "state")) != VX_OK) return st;
    if (deta && (st = device_ptr(deta, 8, "deta")) != VX_OK) return st;
    vx::k_eos_eta<<<(unsigned)((n_zones + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n_zones, state, deta);
    NES_CU(cudaGetLastError());
    return VX_OK;
}

vx_status vx_eos_chain(long long n_zones, int rows, const double *deta, const double *jac_in, double *jac_out,
                       vx_stream stream) {
    if (n_zones < 0 || rows < 0) return nfail(VX_ERR_INVALID_ARG, "negative size");
    if (n_zones == 0 || rows == 0) return VX_OK;
    if (!deta || !jac_in || !jac_out) return nfail(VX_ERR_INVALID_ARG, "NULL array");
    vx_status st;
    if ((st = device_ptr(deta, 8, "deta")) != VX_OK) return st;
    if ((st = device_ptr(jac_in, 8, "jac_in")) != VX_OK) return st;
    if ((st = device_ptr(jac_out, 8, "jac_out")) != VX_OK) return st;
    const long long n = n_zones * rows;
    vx::k_eos_chain<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(n_zones, rows, deta, jac_in, jac_out);
    NES_CU(cudaGetLastError());
    return VX_OK;
}

}  // extern "C"
