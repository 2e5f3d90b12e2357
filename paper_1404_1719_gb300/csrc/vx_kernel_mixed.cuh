// vx_kernel_mixed.cuh -- mixed-precision pair-process kernel: quadrature, Legendre projection,
// spectral contraction and (optionally) the T / eta tangents, fused in one persistent launch.
//
// Work decomposition. One CTA owns one zone at a time and pulls the next zone from a global
// atomic counter (zones of all rays are concatenated; every zone costs the same node count, so
// ragged rays need no special handling); several CTAs share an SM (4 or 6 of 128 threads), so
// one's per-zone set-up and contraction overlap the others' quadrature. The zone's
// npair * n_omega (pair, omega) units are split into equal contiguous ranges, one per thread;
// for each unit a thread loops over the n_e electron-energy nodes, whose constants are broadcast
// from shared memory.
//
// Kernel algebra (exact rewrites of the definition; see the oracle for the definition itself).
// With d = eps - eps', g = eps eps' (1 + cos w), |q|^2 = d^2 + 2 g, h = |q|/2, the electron energy
// on the Gauss-Legendre node tau is E = E- + h (1 + tau) and the positron's Ebar = E- + h (1 - tau).
// The azimuth-averaged squared matrix element of term I is, per node,
//     (s^2 / (16 |q|^2)) [ (|q| + d tau)^2 + g (1 - tau^2) ]
//   = (s^2 / (16 |q|^2)) [ (|q|+d)^2 (1+tau)^2 / 4 + (|q|-d)^2 (1-tau)^2 / 4 + 2 g (1 - tau^2) ],
// a sum of non-negative terms; term II is the same with d -> -d. So per (pair, omega) the node
// loop only accumulates three non-negative moments M+, M-, M0 of the blocking factor against
// w_k (1+tau)^2, w_k (1-tau)^2, w_k (1-tau^2), and K_I, K_II follow from three coefficients each
// (no cancellation anywhere). Terms I and II of (i,j) are terms II and I of (j,i), so only i <= j
// is integrated. Production follows from annihilation by detailed balance, e^{-(eps+eps')/T},
// applied in FP64 at the contraction.
//
// Blocking factor (1 - f_e)(1 - f_ebar) = 1 / ((1 + e1)(1 + e2)), e1 = exp(-x_e), e2 = exp(-x_p),
// x_e = (E - mu)/T, x_p = (Ebar + mu)/T, evaluated with MUFU ex2 / rcp. The zone is mapped to
// eta >= 0 (eta -> -eta exchanges e- and e+, i.e. tau -> -tau, i.e. M+ <-> M-).
//  * fast path (|eta| <= eta_sw): x arguments anchored at E- in FP32; nodes taken in mirror
//    pairs tau, -tau, which share one ex2 per node and (forward) one reciprocal per pair.
//  * degenerate path (|eta| > eta_sw): the electron argument B (1 + tau) + P is formed exactly:
//    B, P and 1 + tau are split into a high part on a power-of-two grid (chosen per zone so that
//    fma(B_hi, u_hi, P_hi) is exact in FP32) and a remainder, and exp2 of the exact high part and
//    of the small remainder are multiplied.
// The l = 1 omega projections and the spectral contraction are FP32 sums; their rounding is
// bounded by the same sums taken over absolute values, the scale that the parity metric uses
// for every l = 1 quantity (their omega sum cancels by up to ~760x at high degeneracy).
#pragma once
#include "vx_internal.h"

// Pair reciprocals (one rcp for two nodes) also in the tangent kernel's fast path.
#ifndef VX_ADJ_PAIR
#define VX_ADJ_PAIR 0
#endif
// Tangent kernel, packed loops: the blocking factor's own moments from the two energy tangents
// (1) instead of a separate accumulation (0). Per node GTa + GTp = O (E + Ebar) = O q0 with both
// terms non-negative, so M(O) = (M(GTa) + M(GTp)) / q0 loses nothing to cancellation.
#ifndef VX_MO_TANG
#define VX_MO_TANG 1
#endif
// Tangent kernel, packed fast loop (not the precise mode): the production tangent's moments as
// q0 M(O) - M(GTa) (1) instead of their own accumulation (0); GTp = O q0 - GTa on every node, and
// since f_ebar <= 1/2 in the eta >= 0 frame, GTp >= O Ebar / 2, so the difference cancels only by
// about q0 / Ebar on the moment's own weights. 2 of 24 FP32 lane operations per node fewer
// (GB300, workload 4: 625.0 against 658.3 ms on the same box). Loading each unit's record one
// unit ahead (626.8 ms), pair reciprocals (631.5 ms) and 32-node chunks (631.0 ms) on top of it
// measured slower.
#ifndef VX_TP_DIFF
#define VX_TP_DIFF 1
#endif
// Tangent kernel, fast zones with n_mu a multiple of 16: the nine moment sums per node on the
// tensor cores through warp-level MMA (1) or as FP32 FMAs (0); see mma_quadrature. Measured on
// GB300 (workload 4): 861.9 ms against 617.3 ms, although the FMAs it removes are worth ~190 ms (a
// copy without them ran in 424.1 ms): the TF32 splits cost more instructions than they save (+63 %
// warp instructions). With the remainder split packed and separate accumulators: 913.4 ms.
#ifndef VX_ADJ_MMA
#define VX_ADJ_MMA 0
#endif
// Packed loops: the positron energies of a mirror pair as the electron energies with the lanes
// exchanged (1; Ebar(tau) = E(-tau) bit for bit) or from their own fused multiply-add (0).
#ifndef VX_ESWAP
#define VX_ESWAP 1
#endif
// Fast path in packed FP32x2 arithmetic (one instruction for the same operation on a node and its
// mirror node) or in scalar FP32.
#ifndef VX_F32X2
#define VX_F32X2 1
#endif
// The second register budget ("minb 3"): 3 CTAs of 256 threads (80 registers) for the forward
// kernel; for the tangent kernel 640 threads per SM in CTAs of VX_BLOCK_MIXED (5 x 128: 96
// registers). GB300, tangent kernel at 96 vs 80 registers: workload 4 764 vs 772 ms, 16 x 48
// eta <= 63 workload 1377 vs 1388 ms; the forward kernel is faster at 80 (293 vs 296 ms).
#define VX_LB3_THREADS_ADJ VX_BLOCK_MIXED
#define VX_LB3_CTAS_ADJ (640 / VX_BLOCK_MIXED > 1 ? 640 / VX_BLOCK_MIXED : 1)
// Degenerate path: scalar (0), packed FP32x2 inline (1) or packed out of line (2), per kernel kind.
// Out of line, the packed loop gets its own register allocation and leaves the fast path's alone
// (GB300, tangent kernel: workload 4 773 / 781 / 772 ms, 16 x 48 eta <= 63 workload 1526 / 1410 /
// 1388 ms for 0 / 1 / 2).
#ifndef VX_DEG_PACK_ADJ
#define VX_DEG_PACK_ADJ 2
#endif
#ifndef VX_DEG_PACK_FWD
#define VX_DEG_PACK_FWD 1
#endif
// Unrolling of the node loops (unroll_depth): chunks of the cap where it divides n_e; else, where
// the loop may be unrolled whole, the whole rule if n_e is below the cap; else chunks of 16.
// GB300, tangent kernel: workload 4 674 / 668 / 646 ms at caps 16 / 32 / 64 (fast loop); 16 x 48
// eta <= 63 workload 1228 / 1211 ms with the degenerate loop in chunks of 16 / whole, but 1283 ms
// with the fast loop whole as well. Forward kernel: workload 4 290 / 278 ms at 16 / 64; 16 x 48
// workload 611 / 600 ms with the fast loop in chunks of 16 / whole, 617 / 600 ms with the
// degenerate loop in chunks of 16 / 48 (whole at n_e = 64 it spills in the smaller register budget).
#ifndef VX_UNROLL_FWD
#define VX_UNROLL_FWD 64
#endif
#ifndef VX_UNROLL_ADJ
#define VX_UNROLL_ADJ 64
#endif
#ifndef VX_UNROLL_DEG_FWD
#define VX_UNROLL_DEG_FWD 48
#endif
#ifndef VX_UNROLL_DEG_ADJ
#define VX_UNROLL_DEG_ADJ 64
#endif

namespace vx {

// Nodes per unrolled chunk of a node loop over NE nodes with unroll cap CAP (NE = 0: run-time n_e);
// WHOLE allows the whole loop below the cap.
template <int NE, int CAP, bool WHOLE>
__host__ __device__ constexpr int unroll_depth() {
    return NE > 0 && NE % CAP == 0 ? CAP : (WHOLE && NE > 0 && NE < CAP ? NE : 16);
}

__device__ __forceinline__ float ex2a(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ float rcpa(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2^-y (y > -1023) as an FP64 value: the integer part of y becomes an exact power of two, the
// fraction goes through MUFU ex2 (relative error ~2^-22, ample for factors that scale FP32 sums).
// Results below the FP64 range flush to 0, as the definition's own values do.
__device__ __forceinline__ double exp2neg(double y) {
    const double n = floor(y);
    if (n > 1022.0) return 0.0;
    const float f = (float)(y - n);  // in [0, 1)
    const double p2 = __longlong_as_double((long long)(1023 - (int)n) << 52);
    return (double)ex2a(-f) * p2;
}

// Projections of one quantity (blocking factor or one of its tangents) onto l = 0, 1 for
// coupling terms I and II.
// In the precise mode (PREC) every projection is carried as an unevaluated FP32 pair hi + lo
// (double-float): the l = 1 sums over cos(omega) cancel, and so do the eta-tangent sums.
struct Proj {
    float o0I, o0II, o1I, o1II;
    float l0I, l0II, l1I, l1II;  // low parts (precise mode only)
    __device__ __forceinline__ void zero() { o0I = o0II = o1I = o1II = 0.f; l0I = l0II = l1I = l1II = 0.f; }
};

// s + e = a + b exactly, s the rounded sum (Knuth's two-sum; no contraction, no reordering).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// hi + lo += t, with the rounding error of the high sum kept exactly.
__device__ __forceinline__ void acc2(float &hi, float &lo, float t) {
    float e;
    two_sum(hi, t, hi, e);
    lo = __fadd_rn(lo, e);
}

struct ZoneSh {
    double T, eta;
    float il_h, il_l;  // log2(e)/T
    float el_h, el_l;  // |eta| log2(e)
    float sB, sP;      // 2^kb and 2^(kb+11): grids of the exact split (degenerate path)
    float iB, iP;      // their inverses
    float sc;          // degenerate path: blocking factor carried as O 2^sc (keeps the deepest-
    float c1;          //   blocked nodes of the zone far from the FP32 underflow); c1 = 2^-sc
    float K;           // e^{-2|eta|}: e2 on a node from e1 on its mirror node (fast path)
    float mu_hi, mu_lo;  // |eta| T, the Fermi edge of the split rule, as an FP32 pair
    double unsc;       // 2^-sc, applied in FP64 to every result of the zone
    double iT2;        // 1/T^2
    int sv;            // production vectors carried as v 2^sv (degenerate zones); the two scales
                       //   share the FP32 exponent headroom so no product can overflow
    int deg, neg, bad;
    bool r2ok;         // degenerate path: r^2 stays in the FP32 range (tangents in the r^2 form)
};

// Moments of one quantity against the three non-negative basis weights.
struct Mom {
    float p, m, z;
    __device__ __forceinline__ void zero() { p = m = z = 0.f; }
};

// Electron-energy node constants, staged once per CTA in shared memory (uniform address within
// a warp, so every read is a broadcast): a = {1+tau, 1-tau, w(1+tau)^2, w(1-tau)^2},
// b = {w(1-tau^2), 1+tau on the 2^-11 grid, remainder, 0}.
struct NodeSm {
    float4 a, b;
};

// The first n_e/2 nodes again, laid out for packed FP32x2 arithmetic on a mirror pair (tau, -tau)
// (lane x: node k, lane y: node n_e-1-k): a = {1+tau, 1-tau, w(1+tau)^2, w(1-tau)^2} (1+tau of
// both nodes, then their first weights), b = {w(1-tau)^2, w(1+tau)^2, w(1-tau^2) twice} (their
// second and third weights), c = {uh of both nodes, ul of both nodes}, with uh and ul the split of
// 1 + tau used by the degenerate path. The fast path reads a and b, the degenerate path all three;
// 1 - tau of both nodes is a's first pair exchanged.
struct NodeMir {
    float4 a, b, c;
};

// Moments of the blocking factor from those of GTa and GTp: E + Ebar = 2 (h + E-) = q0 on every
// node, and both tangents are non-negative.
__device__ __forceinline__ void mo_from_tangents(Mom &mo, const Mom &ta, const Mom &tp, float h, float Em) {
    const float iq = 0.5f * rcpa(h + Em);
    mo.p = (ta.p + tp.p) * iq;
    mo.m = (ta.m + tp.m) * iq;
    mo.z = (ta.z + tp.z) * iq;
}

// Degenerate path, packed on mirror pairs: exact-split electron argument, direct positron argument,
// tangents from r^2 where the zone scale keeps r^2 in the FP32 range (R2), else first-order products
// with r (see node_loop), inline or as an out-of-line call (OUTLINE).
// (UD: unroll cap; the tangent kernel's loop may be unrolled whole. TPD: the production tangent's
// moments as q0 M(O) - M(GTa), as in the fast path; with the zone scale GTa + GTp = q0 r still holds
// node by node, and the moments of O are dominated by E above the Fermi edge, where f_e < 1/2.)
template <int NE, bool ADJ, bool OUTLINE, bool R2, int UD, bool TPD = false>
struct DegPacked {
    static __device__ __forceinline__ void body(const NodeMir *__restrict__ nm, float B, float Pp, float Bq, float Bl,
                                                float Pq, float Pl, float h, float Em, float c1, Mom &mo, Mom &ta,
                                                Mom &tp, Mom &et) {
        constexpr int U = unroll_depth<NE, UD, ADJ>();
        const float2 Bq2 = make_float2(Bq, Bq), Bl2 = make_float2(Bl, Bl), Pq2 = make_float2(Pq, Pq);
        const float2 Pl2 = make_float2(Pl, Pl), B2 = make_float2(B, B), Pp2 = make_float2(Pp, Pp);
        const float2 c12 = make_float2(c1, c1), h2 = make_float2(h, h), Em2 = make_float2(Em, Em);
        const float2 mone2 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
        float2 P2 = z2, M2 = z2, Z2 = z2;
        float2 TAp = z2, TAm = z2, TAz = z2, TPp = z2, TPm = z2, TPz = z2, ETp = z2, ETm = z2, ETz = z2;
#pragma unroll 1
        for (int k0 = 0; k0 < NE / 2; k0 += U / 2) {
#pragma unroll
            for (int kk = 0; kk < U / 2; ++kk) {
                const NodeMir q = nm[k0 + kk];
                const float2 u2 = make_float2(q.a.x, q.a.y), v2 = make_float2(q.a.y, q.a.x);
                const float2 cpm = make_float2(q.a.z, q.a.w), cmp = make_float2(q.b.x, q.b.y);
                const float2 c00 = make_float2(q.b.z, q.b.w);
                const float2 sx = __ffma2_rn(Bq2, make_float2(q.c.x, q.c.y), Pq2);  // exact by the grid choice
                const float2 lo = __ffma2_rn(Bq2, make_float2(q.c.z, q.c.w), __ffma2_rn(Bl2, u2, Pl2));
                const float2 e1 = __fmul2_rn(make_float2(ex2a(-sx.x), ex2a(-sx.y)), make_float2(ex2a(-lo.x), ex2a(-lo.y)));
                const float2 xp = __ffma2_rn(B2, v2, Pp2);
                const float2 e2 = make_float2(ex2a(-xp.x), ex2a(-xp.y));
                const float2 t = __fadd2_rn(c12, e1);
                const float2 d = __ffma2_rn(t, e2, t);
                const float2 r = make_float2(rcpa(d.x), rcpa(d.y));
                if (!(ADJ && VX_MO_TANG) || TPD) {
                    P2 = __ffma2_rn(cpm, r, P2);
                    M2 = __ffma2_rn(cmp, r, M2);
                    Z2 = __ffma2_rn(c00, r, Z2);
                }
                if (ADJ) {
                    const float2 E2 = __ffma2_rn(h2, u2, Em2);
                    const float2 Eb2 = VX_ESWAP ? make_float2(E2.y, E2.x) : __ffma2_rn(h2, v2, Em2);
                    float2 ga, gp = z2, ge;
                    if (R2) {
                        // r = 2^sc O with r^2 in the FP32 range (zone scale chosen for it):
                        // (1 - f_e) r = c1 (1 + e2) r^2, (1 - f_ebar) r = t r^2, f_e r = e1 (1 + e2) r^2,
                        // f_ebar r = e2 t r^2
                        const float2 r2 = __fmul2_rn(r, r);
                        const float2 s0 = __ffma2_rn(e2, r2, r2), p = __fmul2_rn(t, r2);
                        const float2 a1 = __fmul2_rn(e1, s0), a2 = __fmul2_rn(e2, p);
                        ga = __ffma2_rn(a1, E2, __fmul2_rn(a2, Eb2));
                        if (!TPD) gp = __ffma2_rn(__fmul2_rn(c12, s0), E2, __fmul2_rn(p, Eb2));
                        ge = __ffma2_rn(a1, mone2, a2);
                    } else {
                        const float2 qv = __ffma2_rn(e2, r, r);  // (1 + e2) r
                        const float2 se = __fmul2_rn(c12, qv);   // 1 - f_e
                        const float2 sp = __fmul2_rn(t, r);      // 1 - f_ebar
                        const float2 fe = __fmul2_rn(e1, qv), fp = __fmul2_rn(e2, sp);
                        ga = __fmul2_rn(__ffma2_rn(fe, E2, __fmul2_rn(fp, Eb2)), r);
                        if (!TPD) gp = __fmul2_rn(__ffma2_rn(se, E2, __fmul2_rn(sp, Eb2)), r);
                        ge = __fmul2_rn(__ffma2_rn(fe, mone2, fp), r);
                    }
                    TAp = __ffma2_rn(cpm, ga, TAp); TAm = __ffma2_rn(cmp, ga, TAm); TAz = __ffma2_rn(c00, ga, TAz);
                    if (!TPD) {
                        TPp = __ffma2_rn(cpm, gp, TPp); TPm = __ffma2_rn(cmp, gp, TPm); TPz = __ffma2_rn(c00, gp, TPz);
                    }
                    ETp = __ffma2_rn(cpm, ge, ETp); ETm = __ffma2_rn(cmp, ge, ETm); ETz = __ffma2_rn(c00, ge, ETz);
                }
            }
        }
        if (ADJ) {
            ta.p = TAp.x + TAp.y; ta.m = TAm.x + TAm.y; ta.z = TAz.x + TAz.y;
            et.p = ETp.x + ETp.y; et.m = ETm.x + ETm.y; et.z = ETz.x + ETz.y;
        }
        if (ADJ && TPD) {
            mo.p = P2.x + P2.y; mo.m = M2.x + M2.y; mo.z = Z2.x + Z2.y;
            const float q0 = 2.f * (h + Em);
            tp.p = fmaf(q0, mo.p, -ta.p); tp.m = fmaf(q0, mo.m, -ta.m); tp.z = fmaf(q0, mo.z, -ta.z);
        } else if (ADJ && VX_MO_TANG) {
            tp.p = TPp.x + TPp.y; tp.m = TPm.x + TPm.y; tp.z = TPz.x + TPz.y;
            mo_from_tangents(mo, ta, tp, h, Em);
        } else {
            if (ADJ) { tp.p = TPp.x + TPp.y; tp.m = TPm.x + TPm.y; tp.z = TPz.x + TPz.y; }
            mo.p = P2.x + P2.y; mo.m = M2.x + M2.y; mo.z = Z2.x + Z2.y;
        }
    }
    static __device__ __noinline__ void outline(const NodeMir *__restrict__ nm, float B, float Pp, float Bq,
                                                float Bl, float Pq, float Pl, float h, float Em, float c1, Mom *m4) {
        body(nm, B, Pp, Bq, Bl, Pq, Pl, h, Em, c1, m4[0], m4[1], m4[2], m4[3]);
    }
    static __device__ __forceinline__ void run(const NodeMir *__restrict__ nm, float B, float Pp, float Bq, float Bl,
                                               float Pq, float Pl, float h, float Em, float c1, Mom &mo, Mom &ta,
                                               Mom &tp, Mom &et) {
        if (OUTLINE) {
            Mom m4[4];
            outline(nm, B, Pp, Bq, Bl, Pq, Pl, h, Em, c1, m4);
            mo = m4[0]; ta = m4[1]; tp = m4[2]; et = m4[3];
        } else {
            body(nm, B, Pp, Bq, Bl, Pq, Pl, h, Em, c1, mo, ta, tp, et);
        }
    }
};

// Split rule, one (pair, omega) unit whose Fermi edge E_s lies inside (E-, E+): panels
// A = [E-, E_s] and B = [E_s, E+] share the n_e/2-node rule; lane x of every float2 is panel A's
// node, lane y panel B's. With rA = (E_s - E-)/(2h) and rB = 1 - rA, a node x of the rule sits at
// 1 + tau = rA (1 + x) (A) or 2 rA + rB (1 + x) (B) of the full interval, with weight r_P w, so the
// moment basis and the (pair, omega) coefficients are those of the standard rule. The electron
// argument X = (E - mu) log2(e)/T is formed relative to the edge: -rA B (1 - x) or rB B (1 + x)
// plus the rounding of the boundary and the zone scale (dls), accurate where the blocking factor
// changes; the positron argument is Qs - X with Qs = q0 log2(e)/T + sc. Tangents use the
// first-order products with r (r may be far below the FP32 normal range squared).
template <bool ADJ, bool OUTLINE>
struct SplitUnit {
    static __device__ __forceinline__ void body(const float4 *__restrict__ hs, int nh, float rA, float B, float dls,
                                                float Qs, float h, float Em, float c1, Mom &mo, Mom &ta, Mom &tp,
                                                Mom &et) {
        const float rB = 1.f - rA;
        const float2 rho = make_float2(rA, rB), au = make_float2(0.f, 2.f * rA), av = make_float2(2.f * rB, 0.f);
        const float2 nb = make_float2(-rA * B, rB * B), off = make_float2(dls, dls), mQ = make_float2(-Qs, -Qs);
        const float2 c12 = make_float2(c1, c1), h2 = make_float2(h, h), Em2 = make_float2(Em, Em);
        const float2 mone2 = make_float2(-1.f, -1.f), z2 = make_float2(0.f, 0.f);
        float2 P2 = z2, M2 = z2, Z2 = z2;
        float2 TAp = z2, TAm = z2, TAz = z2, TPp = z2, TPm = z2, TPz = z2, ETp = z2, ETm = z2, ETz = z2;
#pragma unroll 4
        for (int k = 0; k < nh; ++k) {
            const float4 q = hs[k];  // 1 + x, 1 - x, w
            const float2 u2 = __ffma2_rn(rho, make_float2(q.x, q.x), au);
            const float2 v2 = __ffma2_rn(rho, make_float2(q.y, q.y), av);
            const float2 W2 = __fmul2_rn(rho, make_float2(q.z, q.z));
            const float2 xs = __ffma2_rn(nb, make_float2(q.y, q.x), off);  // X + sc
            const float2 e1 = make_float2(ex2a(-xs.x), ex2a(-xs.y));        // e^{-x_e} 2^-sc
            const float2 xp = __fadd2_rn(xs, mQ);                           // -(x_p log2 e)
            const float2 e2 = make_float2(ex2a(xp.x), ex2a(xp.y));
            const float2 t = __fadd2_rn(c12, e1);
            const float2 d = __ffma2_rn(t, e2, t);
            const float2 r = make_float2(rcpa(d.x), rcpa(d.y));
            const float2 Wu = __fmul2_rn(W2, u2);
            const float2 cp = __fmul2_rn(Wu, u2), c0 = __fmul2_rn(Wu, v2), cm = __fmul2_rn(__fmul2_rn(W2, v2), v2);
            if (!(ADJ && VX_MO_TANG)) {
                P2 = __ffma2_rn(cp, r, P2);
                M2 = __ffma2_rn(cm, r, M2);
                Z2 = __ffma2_rn(c0, r, Z2);
            }
            if (ADJ) {
                const float2 qv = __ffma2_rn(e2, r, r);  // (1 + e2) r
                const float2 se = __fmul2_rn(c12, qv);   // 1 - f_e
                const float2 sp = __fmul2_rn(t, r);      // 1 - f_ebar
                const float2 fe = __fmul2_rn(e1, qv), fp = __fmul2_rn(e2, sp);
                const float2 E2 = __ffma2_rn(h2, u2, Em2), Eb2 = __ffma2_rn(h2, v2, Em2);
                const float2 ga = __fmul2_rn(__ffma2_rn(fe, E2, __fmul2_rn(fp, Eb2)), r);
                const float2 gp = __fmul2_rn(__ffma2_rn(se, E2, __fmul2_rn(sp, Eb2)), r);
                const float2 ge = __fmul2_rn(__ffma2_rn(fe, mone2, fp), r);
                TAp = __ffma2_rn(cp, ga, TAp); TAm = __ffma2_rn(cm, ga, TAm); TAz = __ffma2_rn(c0, ga, TAz);
                TPp = __ffma2_rn(cp, gp, TPp); TPm = __ffma2_rn(cm, gp, TPm); TPz = __ffma2_rn(c0, gp, TPz);
                ETp = __ffma2_rn(cp, ge, ETp); ETm = __ffma2_rn(cm, ge, ETm); ETz = __ffma2_rn(c0, ge, ETz);
            }
        }
        if (ADJ) {
            ta.p = TAp.x + TAp.y; ta.m = TAm.x + TAm.y; ta.z = TAz.x + TAz.y;
            tp.p = TPp.x + TPp.y; tp.m = TPm.x + TPm.y; tp.z = TPz.x + TPz.y;
            et.p = ETp.x + ETp.y; et.m = ETm.x + ETm.y; et.z = ETz.x + ETz.y;
        }
        if (ADJ && VX_MO_TANG) {
            mo_from_tangents(mo, ta, tp, h, Em);
        } else {
            mo.p = P2.x + P2.y; mo.m = M2.x + M2.y; mo.z = Z2.x + Z2.y;
        }
    }
    static __device__ __noinline__ void outline(const float4 *__restrict__ hs, int nh, float rA, float B, float dls,
                                                float Qs, float h, float Em, float c1, Mom *m4) {
        body(hs, nh, rA, B, dls, Qs, h, Em, c1, m4[0], m4[1], m4[2], m4[3]);
    }
    static __device__ __forceinline__ void run(const float4 *__restrict__ hs, int nh, float rA, float B, float dls,
                                               float Qs, float h, float Em, float c1, Mom &mo, Mom &ta, Mom &tp,
                                               Mom &et) {
        if (OUTLINE) {
            Mom m4[4];
            outline(hs, nh, rA, B, dls, Qs, h, Em, c1, m4);
            mo = m4[0]; ta = m4[1]; tp = m4[2]; et = m4[3];
        } else {
            body(hs, nh, rA, B, dls, Qs, h, Em, c1, mo, ta, tp, et);
        }
    }
};

// (ah + al) - (bh + bl) as a normalised FP32 pair (two-sum of the high parts; no contraction).
__device__ __forceinline__ void df_diff(float ah, float al, float bh, float bl, float &dh, float &dl) {
    const float s = __fsub_rn(ah, bh);
    const float v = __fsub_rn(s, ah);
    const float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, v)), __fsub_rn(-bh, v));
    const float t = __fadd_rn(e, __fsub_rn(al, bl));
    dh = __fadd_rn(s, t);
    dl = __fsub_rn(t, __fsub_rn(dh, s));
}

// One (pair, omega) node loop. Fills the moments of the blocking factor O and, with ADJ, of
// GTa = O (f_e E + f_ebar Ebar), GTp = O ((1-f_e) E + (1-f_ebar) Ebar), GEt = O (f_ebar - f_e).
// With the zone scale (degenerate path) e1 and the "1" of 1 + e1 carry the factor 2^-sc, so
// r = 2^sc O; c1 = 2^-sc recovers 1 - f_e, while f_e, f_ebar and 1 - f_ebar need no correction.
// The unroll depth of each loop is set by unroll_depth (the whole rule or chunks that divide n_e).
//
// Fast path, unrolled instantiations (even n_e): the Gauss-Legendre nodes come in exact mirror
// pairs tau, -tau (records k and n_e-1-k hold the same values with u <-> v and
// w(1+tau)^2 <-> w(1-tau)^2). On the mirror node the electron argument is the positron argument
// of tau less 2|eta|, so e2(tau) = e1(-tau) K and e2(-tau) = e1(tau) K with K = e^{-2|eta|}: one
// ex2 and half a record read per node, and (MPAIR) one reciprocal per node pair.
// SPLIT: the kernel carries the split rule too; its degenerate loop then stays in chunks of 16
// (unrolled whole beside the split loop it was slower: 16 x 48 eta <= 63 workload, 1758 vs
// 1805 ms).
// PREC (precise mode): the packed mirror loop forms the electron argument exactly as the
// degenerate path does (high part on the zone's grid, exact in FP32, remainder through a second
// ex2), so the blocking factor's relative error no longer grows like |x| 2^-24 with the argument.
template <int NE, bool ADJ, bool DEG, bool SPLIT, bool PREC, bool TPOK = true>
__device__ __forceinline__ void node_loop(const NodeSm *__restrict__ nd, const NodeMir *__restrict__ nm, int ne,
                                          float B, float Pe,
                                          float Pp, float Bq, float Bl, float Pq, float Pl, float h,
                                          float Em, float c1, float K, bool r2ok, Mom &mo, Mom &ta,
                                          Mom &tp, Mom &et) {
    constexpr bool MIRROR = !DEG && NE > 0;
    constexpr bool MPAIR = !ADJ || VX_ADJ_PAIR;
    constexpr int U = 16;
    // nodes per unrolled chunk of the mirror loop (a chunk must divide n_e)
    constexpr int UM0 = ADJ ? VX_UNROLL_ADJ : VX_UNROLL_FWD;
    constexpr int UM = unroll_depth<NE, UM0, !ADJ>();
    // tangent integrands of one node, accumulated with its basis weights (cp, cm, c0)
    auto tang = [&](float cp, float cm, float c0, float e1, float e2, float t, float r, float E, float Eb) {
        float ga, gp, ge;
        if (!DEG) {
            // r >= 1 / (2 (1 + e^40)) here, so r2 = r^2 stays normal: (1 - f_e) r = (1 + e2) r2,
            // (1 - f_ebar) r = t r2, f_e r = e1 (1 + e2) r2, f_ebar r = e2 t r2
            const float r2 = r * r;
            const float s0 = fmaf(e2, r2, r2), p = t * r2;
            const float a1 = e1 * s0, a2 = e2 * p;
            ga = fmaf(a1, E, a2 * Eb);
            gp = fmaf(s0, E, p * Eb);
            ge = a2 - a1;
        } else {
            // r = 2^sc O can lie near the FP32 floor: keep products with r to first order
            const float qv = fmaf(e2, r, r);  // (1 + e2) r
            const float se = c1 * qv;         // 1 - f_e
            const float sp = t * r;           // 1 - f_ebar
            const float fe = e1 * qv, fp = e2 * sp;
            ga = fmaf(fe, E, fp * Eb) * r;
            gp = fmaf(se, E, sp * Eb) * r;
            ge = (fp - fe) * r;
        }
        ta.p = fmaf(cp, ga, ta.p); ta.m = fmaf(cm, ga, ta.m); ta.z = fmaf(c0, ga, ta.z);
        tp.p = fmaf(cp, gp, tp.p); tp.m = fmaf(cm, gp, tp.m); tp.z = fmaf(c0, gp, tp.z);
        et.p = fmaf(cp, ge, et.p); et.m = fmaf(cm, ge, et.m); et.z = fmaf(c0, ge, et.z);
    };
    auto accum = [&](const NodeSm &q, float e1, float e2, float t, float r) {
        mo.p = fmaf(q.a.z, r, mo.p);
        mo.m = fmaf(q.a.w, r, mo.m);
        mo.z = fmaf(q.b.x, r, mo.z);
        if (ADJ) tang(q.a.z, q.a.w, q.b.x, e1, e2, t, r, fmaf(h, q.a.x, Em), fmaf(h, q.a.y, Em));
    };
    auto factors = [&](const NodeSm &q, float &e1, float &e2, float &t) {
        if (!DEG && !PREC) {
            e1 = ex2a(-fmaf(B, q.a.x, Pe));
            e2 = ex2a(-fmaf(B, q.a.y, Pp));
            t = 1.f + e1;
        } else {
            float s = fmaf(Bq, q.b.y, Pq);                      // exact by the grid choice
            float lo = fmaf(Bq, q.b.z, fmaf(Bl, q.a.x, Pl));    // small remainder
            e1 = ex2a(-s) * ex2a(-lo);
            e2 = ex2a(-fmaf(B, q.a.y, Pp));
            t = c1 + e1;
        }
    };
    if (MIRROR && VX_F32X2) {
        // packed form: lane x of every float2 is node tau, lane y its mirror -tau
        const float2 B2 = make_float2(B, B), Pe2 = make_float2(Pe, Pe), one2 = make_float2(1.f, 1.f);
        const float2 Bq2 = make_float2(Bq, Bq), Bl2 = make_float2(Bl, Bl);
        const float2 Pq2 = make_float2(Pq, Pq), Pl2 = make_float2(Pl, Pl);
        const float2 h2 = make_float2(h, h), Em2 = make_float2(Em, Em), mone2 = make_float2(-1.f, -1.f);
        const float2 z2 = make_float2(0.f, 0.f);
        float2 P2 = z2, M2 = z2, Z2 = z2;
        float2 TAp = z2, TAm = z2, TAz = z2, TPp = z2, TPm = z2, TPz = z2, ETp = z2, ETm = z2, ETz = z2;
        constexpr bool TPD = ADJ && VX_TP_DIFF && !PREC;
#pragma unroll 1
        for (int k0 = 0; k0 < NE / 2; k0 += UM / 2) {
#pragma unroll
            for (int kk = 0; kk < UM / 2; ++kk) {
                const NodeMir q = nm[k0 + kk];
                const float2 uv = make_float2(q.a.x, q.a.y), cpm = make_float2(q.a.z, q.a.w);
                const float2 cmp = make_float2(q.b.x, q.b.y), c00 = make_float2(q.b.z, q.b.w);
                float2 e;  // e1(tau), e1(-tau)
                if (PREC) {
                    const float2 sx = __ffma2_rn(Bq2, make_float2(q.c.x, q.c.y), Pq2);  // exact by the grid choice
                    const float2 lo = __ffma2_rn(Bq2, make_float2(q.c.z, q.c.w), __ffma2_rn(Bl2, uv, Pl2));
                    e = __fmul2_rn(make_float2(ex2a(-sx.x), ex2a(-sx.y)), make_float2(ex2a(-lo.x), ex2a(-lo.y)));
                } else {
                    const float2 x = __ffma2_rn(B2, uv, Pe2);
                    e = make_float2(ex2a(-x.x), ex2a(-x.y));
                }
                const float2 f = make_float2(e.y * K, e.x * K);  // e2(tau), e2(-tau)
                const float2 t = __fadd2_rn(e, one2);
                const float2 d = __ffma2_rn(t, f, t);
                float2 r;
                if (MPAIR) {
                    const float R = rcpa(d.x * d.y);  // finite: see the scalar form
                    r = make_float2(R * d.y, R * d.x);
                } else {
                    r = make_float2(rcpa(d.x), rcpa(d.y));
                }
                if (!(ADJ && VX_MO_TANG) || TPD) {
                    P2 = __ffma2_rn(cpm, r, P2);
                    M2 = __ffma2_rn(cmp, r, M2);
                    Z2 = __ffma2_rn(c00, r, Z2);
                }
                if (ADJ) {
                    const float2 vu = make_float2(q.a.y, q.a.x);
                    const float2 E2 = __ffma2_rn(h2, uv, Em2);
                    const float2 Eb2 = VX_ESWAP ? make_float2(E2.y, E2.x) : __ffma2_rn(h2, vu, Em2);
                    const float2 r2 = __fmul2_rn(r, r);
                    const float2 s0 = __ffma2_rn(f, r2, r2), p = __fmul2_rn(t, r2);
                    const float2 a1 = __fmul2_rn(e, s0), a2 = __fmul2_rn(f, p);
                    const float2 ga = __ffma2_rn(a1, E2, __fmul2_rn(a2, Eb2));
                    const float2 ge = __ffma2_rn(a1, mone2, a2);  // a2 - a1
                    TAp = __ffma2_rn(cpm, ga, TAp); TAm = __ffma2_rn(cmp, ga, TAm); TAz = __ffma2_rn(c00, ga, TAz);
                    if (!TPD) {
                        const float2 gp = __ffma2_rn(s0, E2, __fmul2_rn(p, Eb2));
                        TPp = __ffma2_rn(cpm, gp, TPp); TPm = __ffma2_rn(cmp, gp, TPm); TPz = __ffma2_rn(c00, gp, TPz);
                    }
                    ETp = __ffma2_rn(cpm, ge, ETp); ETm = __ffma2_rn(cmp, ge, ETm); ETz = __ffma2_rn(c00, ge, ETz);
                }
            }
        }
        if (ADJ) {
            ta.p = TAp.x + TAp.y; ta.m = TAm.x + TAm.y; ta.z = TAz.x + TAz.y;
            et.p = ETp.x + ETp.y; et.m = ETm.x + ETm.y; et.z = ETz.x + ETz.y;
        }
        if (TPD) {
            // GTp = O (E + Ebar) - GTa; GTa <= (E + Ebar) O max(f_e, f_ebar) and f_ebar <= 1/2 in
            // the eta >= 0 frame, so the difference keeps at least the positron's share
            mo.p = P2.x + P2.y; mo.m = M2.x + M2.y; mo.z = Z2.x + Z2.y;
            const float q0 = 2.f * (h + Em);
            tp.p = fmaf(q0, mo.p, -ta.p); tp.m = fmaf(q0, mo.m, -ta.m); tp.z = fmaf(q0, mo.z, -ta.z);
        } else if (ADJ && VX_MO_TANG) {
            tp.p = TPp.x + TPp.y; tp.m = TPm.x + TPm.y; tp.z = TPz.x + TPz.y;
            mo_from_tangents(mo, ta, tp, h, Em);
        } else {
            if (ADJ) { tp.p = TPp.x + TPp.y; tp.m = TPm.x + TPm.y; tp.z = TPz.x + TPz.y; }
            mo.p = P2.x + P2.y; mo.m = M2.x + M2.y; mo.z = Z2.x + Z2.y;
        }
    } else if (MIRROR) {
        static_assert(NE % U == 0 || NE == 0, "unrolled instantiations need a multiple of the unroll depth");
#pragma unroll 1
        for (int k0 = 0; k0 < NE / 2; k0 += UM / 2) {
#pragma unroll
            for (int kk = 0; kk < UM / 2; ++kk) {
                const NodeSm q = nd[k0 + kk];
                const float ea = ex2a(-fmaf(B, q.a.x, Pe));  // e1(tau)
                const float eb = ex2a(-fmaf(B, q.a.y, Pe));  // e1(-tau)
                const float fa = eb * K, fb = ea * K;        // e2(tau), e2(-tau)
                const float ta_ = 1.f + ea, tb_ = 1.f + eb;
                const float da = fmaf(ta_, fa, ta_), db = fmaf(tb_, fb, tb_);
                float ra, rb;
                if (MPAIR) {
                    // |eta| <= eta_sw <= 40: d <= 2 (1 + e^40), so the product stays finite
                    const float R = rcpa(da * db);
                    ra = R * db;
                    rb = R * da;
                } else {
                    ra = rcpa(da);
                    rb = rcpa(db);
                }
                mo.p = fmaf(q.a.z, ra, mo.p); mo.m = fmaf(q.a.w, ra, mo.m); mo.z = fmaf(q.b.x, ra, mo.z);
                mo.p = fmaf(q.a.w, rb, mo.p); mo.m = fmaf(q.a.z, rb, mo.m); mo.z = fmaf(q.b.x, rb, mo.z);
                if (ADJ) {
                    const float Ea = fmaf(h, q.a.x, Em), Eba = fmaf(h, q.a.y, Em);  // E(tau) = Ebar(-tau)
                    tang(q.a.z, q.a.w, q.b.x, ea, fa, ta_, ra, Ea, Eba);
                    tang(q.a.w, q.a.z, q.b.x, eb, fb, tb_, rb, Eba, Ea);
                }
            }
        }
    } else if (DEG && NE > 0 && VX_F32X2 && (ADJ ? VX_DEG_PACK_ADJ : VX_DEG_PACK_FWD)) {
        constexpr bool OL = (ADJ ? VX_DEG_PACK_ADJ : VX_DEG_PACK_FWD) == 2;
        constexpr int UDG = !ADJ ? VX_UNROLL_DEG_FWD : (SPLIT ? 16 : VX_UNROLL_DEG_ADJ);
        constexpr bool DTPD = ADJ && TPOK && VX_TP_DIFF;
        if (!ADJ || r2ok)
            DegPacked<NE, ADJ, OL, ADJ, UDG, DTPD>::run(nm, B, Pp, Bq, Bl, Pq, Pl, h, Em, c1, mo, ta, tp, et);
        else
            DegPacked<NE, ADJ, OL, false, UDG, DTPD>::run(nm, B, Pp, Bq, Bl, Pq, Pl, h, Em, c1, mo, ta, tp, et);
    } else if (NE > 0) {
#pragma unroll 1
        for (int k0 = 0; k0 < NE; k0 += U) {
#pragma unroll
            for (int kk = 0; kk < U; ++kk) {
                const NodeSm q = nd[k0 + kk];
                float e1, e2, t;
                factors(q, e1, e2, t);
                accum(q, e1, e2, t, rcpa(fmaf(t, e2, t)));
            }
        }
    } else {
#pragma unroll 2
        for (int k = 0; k < ne; ++k) {
            const NodeSm q = nd[k];
            float e1, e2, t;
            factors(q, e1, e2, t);
            accum(q, e1, e2, t, rcpa(fmaf(t, e2, t)));
        }
    }
}

// Coefficients that turn one (pair, omega) node's moments into its contributions: l = 0
// (kp, km, k0) and l = 1 (t kp, t km, t k0). (kp, km) are already exchanged for eta < 0.
struct Coef {
    float kp, km, k0;  // l = 0
    float lp, lm, l0;  // l = 1 (precise mode)
    float t;           // cos(omega): the l = 1 coefficients are t times the l = 0 ones
};

__device__ __forceinline__ Coef make_coef(float kp, float km, float k0, float t) {
    Coef c;
    c.kp = kp; c.km = km; c.k0 = k0;
    c.lp = t * kp; c.lm = t * km; c.l0 = t * k0;
    c.t = t;
    return c;
}

// Projection of one quantity's moments onto l = 0, 1 for terms I and II (term II of a pair uses
// the coefficients with kp and km exchanged).
// PREC: the l = 1 sums (and, for a quantity whose moments change sign -- SIGNED, the eta
// tangent -- the l = 0 sums too) go into double-float accumulators; sums of non-negative terms
// stay FP32, whose rounding is relative to the sum itself.
// Default mode: the l = 1 terms as cos(omega) times the l = 0 ones, fused into the accumulation.
template <bool PREC, bool SIGNED = false>
__device__ __forceinline__ void project(Proj &P, const Mom &M, const Coef &c) {
    const float a = fmaf(c.kp, M.p, fmaf(c.km, M.m, c.k0 * M.z));
    const float b = fmaf(c.km, M.p, fmaf(c.kp, M.m, c.k0 * M.z));
    if (PREC) {
        const float d = fmaf(c.lp, M.p, fmaf(c.lm, M.m, c.l0 * M.z));
        const float e = fmaf(c.lm, M.p, fmaf(c.lp, M.m, c.l0 * M.z));
        if (SIGNED) { acc2(P.o0I, P.l0I, a); acc2(P.o0II, P.l0II, b); }
        else { P.o0I += a; P.o0II += b; }
        acc2(P.o1I, P.l1I, d); acc2(P.o1II, P.l1II, e);
    } else {
        P.o0I += a; P.o0II += b;
        P.o1I = fmaf(c.t, a, P.o1I);
        P.o1II = fmaf(c.t, b, P.o1II);
    }
}

// Writes one pair's projections into the zone matrices [l][N][N]: term I of pair (i,j) is
// Phi_I(i,j), term II is Phi_I(j,i).
// (Precise mode: each double-float sum is rounded once, to nearest, on the way to FP32.)
template <bool PREC>
__device__ __forceinline__ void store_proj(float *q2, int N2, int N, int pi, int pj, const Proj &P) {
    float *M0 = q2, *M1 = q2 + N2;
    const int a = pi * N + pj, b = pj * N + pi;
    M0[a] = PREC ? __fadd_rn(P.o0I, P.l0I) : P.o0I;
    M1[a] = PREC ? __fadd_rn(P.o1I, P.l1I) : P.o1I;
    if (pi != pj) {
        M0[b] = PREC ? __fadd_rn(P.o0II, P.l0II) : P.o0II;
        M1[b] = PREC ? __fadd_rn(P.o1II, P.l1II) : P.o1II;
    }
}

// Partial projections of bin pairs split between threads: part[slot q][4 or 8][TB] floats (the
// precise mode adds the four low parts), thread index fastest, so a warp's stores and loads fall
// in distinct banks.
template <bool PREC>
__device__ __forceinline__ void part_put(float *part, int TB, int t, int sq, const Proj &P) {
    float *b = part + (size_t)sq * (PREC ? 8 : 4) * TB + t;
    b[0] = P.o0I; b[TB] = P.o0II; b[2 * TB] = P.o1I; b[3 * TB] = P.o1II;
    if (PREC) { b[4 * TB] = P.l0I; b[5 * TB] = P.l0II; b[6 * TB] = P.l1I; b[7 * TB] = P.l1II; }
}
template <bool PREC>
__device__ __forceinline__ Proj part_get(const float *part, int TB, int t, int sq) {
    const float *b = part + (size_t)sq * (PREC ? 8 : 4) * TB + t;
    Proj P;
    P.o0I = b[0]; P.o0II = b[TB]; P.o1I = b[2 * TB]; P.o1II = b[3 * TB];
    if (PREC) { P.l0I = b[4 * TB]; P.l0II = b[5 * TB]; P.l1I = b[6 * TB]; P.l1II = b[7 * TB]; }
    else { P.l0I = P.l0II = P.l1I = P.l1II = 0.f; }
    return P;
}

// One contraction term pair of the precise mode: (bI a + bII b) v added to hi + lo, with both
// products and the sum carried exactly to FP32-pair precision (two-product by FMA, two-sum).
__device__ __forceinline__ void contract2(float &hi, float &lo, float bI, float a, float bII, float b, float v) {
    const float p1 = __fmul_rn(bI, a), e1 = fmaf(bI, a, -p1);
    const float p2 = __fmul_rn(bII, b), e2 = fmaf(bII, b, -p2);
    float kh, kl;
    two_sum(p1, p2, kh, kl);
    kl = __fadd_rn(kl, __fadd_rn(e1, e2));
    const float th = __fmul_rn(kh, v), tl = fmaf(kh, v, -th);
    acc2(hi, lo, th);
    lo = fmaf(kl, v, __fadd_rn(lo, tl));
}

// bI a + bII b of the precise mode as an FP64 value (exact products, two-sum of the FP32 pair).
__device__ __forceinline__ double kern2(float bI, float a, float bII, float b) {
    const float p1 = __fmul_rn(bI, a), e1 = fmaf(bI, a, -p1);
    const float p2 = __fmul_rn(bII, b), e2 = fmaf(bII, b, -p2);
    float kh, kl;
    two_sum(p1, p2, kh, kl);
    return (double)kh + ((double)kl + ((double)e1 + (double)e2));
}

// ---- tangent kernel, fast zones: the moment sums on the tensor cores ----------------------------
// The moments of the three integrands O, GTa, GEt of a (pair, omega) unit are sums over the nodes
// of integrand x weight, with the weights w(1+tau)^2, w(1-tau)^2, w(1-tau^2) shared by every unit:
// a product [units x nodes] . [nodes x weights]. A warp takes 16 units at a time (units g and
// g + 8 in the 4-lane group g) and 8 nodes per MMA step (lane q of the group: mirror node pair
// k = 4 step + q, i.e. node k and node n_e - 1 - k, whose packed integrands are exactly the lane's
// A-fragment entries of m16n8k8). FP32 accuracy from TF32 operands: each integrand is split into
// a high part (its last 13 mantissa bits cleared) and the remainder, each weight into its nearest
// TF32 value and the remainder, held in B's columns (w_hi, w_lo) for the three weights; two MMAs
// per integrand (high and remainder rows) then carry every product but remainder x remainder
// (relative 2^-21). The projections onto l = 0, 1 are linear in the moments, so every lane
// accumulates its share (its weight column, its two units) over the pair's units and one
// butterfly reduces the warp per pair: a warp owns whole pairs, no partial pairs remain.
__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// v = hi + lo with hi the TF32 value of v's leading bits and lo the exact remainder, cut to TF32.
__device__ __forceinline__ void split_tf32(float v, unsigned &hi, unsigned &lo) {
    hi = __float_as_uint(v) & 0xffffe000u;
    lo = __float_as_uint(__fsub_rn(v, __uint_as_float(hi))) & 0xffffe000u;
}

// The packed integrands of one unit on a mirror node pair (lane x: node tau, lane y: node -tau),
// as in node_loop's packed fast path: O = r, GTa, GEt.
__device__ __forceinline__ void mma_integrands(float2 B2, float2 Pe2, float2 h2, float2 Em2, float2 uv, float K,
                                               float2 &r, float2 &ga, float2 &ge) {
    const float2 one2 = make_float2(1.f, 1.f), mone2 = make_float2(-1.f, -1.f);
    const float2 x = __ffma2_rn(B2, uv, Pe2);
    const float2 e = make_float2(ex2a(-x.x), ex2a(-x.y));
    const float2 f = make_float2(e.y * K, e.x * K);
    const float2 t = __fadd2_rn(e, one2);
    const float2 d = __ffma2_rn(t, f, t);
    r = make_float2(rcpa(d.x), rcpa(d.y));
    const float2 E2 = __ffma2_rn(h2, uv, Em2);
    const float2 Eb2 = make_float2(E2.y, E2.x);
    const float2 r2 = __fmul2_rn(r, r);
    const float2 s0 = __ffma2_rn(f, r2, r2), p = __fmul2_rn(t, r2);
    const float2 a1 = __fmul2_rn(e, s0), a2 = __fmul2_rn(f, p);
    ga = __ffma2_rn(a1, E2, __fmul2_rn(a2, Eb2));
    ge = __ffma2_rn(a1, mone2, a2);
}

template <int NE>
__device__ __forceinline__ void mma_quadrature(const NodeMir *__restrict__ nm, const float (*__restrict__ w8)[8],
                                               const float4 *__restrict__ tab, int npair, int nmu,
                                               const uint16_t *__restrict__ pij, float *mats, int N2, int N,
                                               float il_h, float el_h, float K, bool neg) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int pa = warp * npair / nwarp, pb = (warp + 1) * npair / nwarp;
#pragma unroll 1
    for (int p = pa; p < pb; ++p) {
        float acc[4][4];  // [O, GTa, GTp, GEt][l = 0 term I, term II, l = 1 term I, term II]
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[x][0] = acc[x][1] = acc[x][2] = acc[x][3] = 0.f;
#pragma unroll 1
        for (int m0 = 0; m0 < nmu; m0 += 16) {
            const int uA = p * nmu + m0 + g, uB = uA + 8;
            const float4 RA0 = __ldg(tab + 2 * uA), RA1 = __ldg(tab + 2 * uA + 1);
            const float4 RB0 = __ldg(tab + 2 * uB), RB1 = __ldg(tab + 2 * uB + 1);
            const float2 BA = make_float2(RA0.x * il_h, RA0.x * il_h), BB = make_float2(RB0.x * il_h, RB0.x * il_h);
            const float pA = fmaf(RA0.z, il_h, -el_h), pB = fmaf(RB0.z, il_h, -el_h);
            const float2 PA = make_float2(pA, pA), PB = make_float2(pB, pB);
            const float2 hA = make_float2(RA0.x, RA0.x), hB = make_float2(RB0.x, RB0.x);
            const float2 EA = make_float2(RA0.z, RA0.z), EB = make_float2(RB0.z, RB0.z);
            float D[3][4];
#pragma unroll
            for (int x = 0; x < 3; ++x) D[x][0] = D[x][1] = D[x][2] = D[x][3] = 0.f;
#pragma unroll 2
            for (int kb = 0; kb < NE / 8; ++kb) {
                const int k = 4 * kb + tq;
                const float2 uv = make_float2(nm[k].a.x, nm[k].a.y);
                const unsigned b0 = __float_as_uint(w8[k][g]), b1 = __float_as_uint(w8[NE - 1 - k][g]);
                float2 vA[3], vB[3];
                mma_integrands(BA, PA, hA, EA, uv, K, vA[0], vA[1], vA[2]);
                mma_integrands(BB, PB, hB, EB, uv, K, vB[0], vB[1], vB[2]);
#pragma unroll
                for (int x = 0; x < 3; ++x) {
                    unsigned h0, l0, h1, l1, h2, l2, h3, l3;
                    split_tf32(vA[x].x, h0, l0);
                    split_tf32(vB[x].x, h1, l1);
                    split_tf32(vA[x].y, h2, l2);
                    split_tf32(vB[x].y, h3, l3);
                    mma_tf32(D[x], h0, h1, h2, h3, b0, b1);
                    mma_tf32(D[x], l0, l1, l2, l3, b0, b1);
                }
            }
            // lane q < 3 holds weight q's moments: columns 2q, 2q + 1 = (w_hi, w_lo) of units A, B
            if (tq < 3) {
                // projection coefficients of this lane's weight: term I (kp, km, k0)[q], term II
                // (km, kp, k0)[q]; eta < 0 exchanges kp and km
                const bool sw = (tq == 0) != neg, sw2 = (tq == 1) != neg;
                const float caA = tq == 2 ? RA1.z : (sw ? RA1.x : RA1.y), cbA = tq == 2 ? RA1.z : (sw2 ? RA1.x : RA1.y);
                const float caB = tq == 2 ? RB1.z : (sw ? RB1.x : RB1.y), cbB = tq == 2 ? RB1.z : (sw2 ? RB1.x : RB1.y);
                const float q0A = 2.f * (RA0.x + RA0.z), q0B = 2.f * (RB0.x + RB0.z);
                float MA[4], MB[4];
                MA[0] = D[0][0] + D[0][1]; MA[1] = D[1][0] + D[1][1]; MA[3] = D[2][0] + D[2][1];
                MB[0] = D[0][2] + D[0][3]; MB[1] = D[1][2] + D[1][3]; MB[3] = D[2][2] + D[2][3];
                MA[2] = fmaf(q0A, MA[0], -MA[1]);  // GTp = O q0 - GTa
                MB[2] = fmaf(q0B, MB[0], -MB[1]);
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    const float aA = caA * MA[x], bA = cbA * MA[x], aB = caB * MB[x], bB = cbB * MB[x];
                    acc[x][0] += aA + aB;
                    acc[x][1] += bA + bB;
                    acc[x][2] += fmaf(RA1.w, aA, RB1.w * aB);
                    acc[x][3] += fmaf(RA1.w, bA, RB1.w * bB);
                }
            }
        }
        // the pair's sums over the warp (fixed butterfly), stored by lane 0
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[x][c] += __shfl_xor_sync(0xffffffffu, acc[x][c], off);
        if (lane == 0) {
            const int pi = pij[p] >> 8, pj = pij[p] & 0xff;
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                Proj P;
                P.zero();
                P.o0I = acc[x][0]; P.o0II = acc[x][1]; P.o1I = acc[x][2]; P.o1II = acc[x][3];
                store_proj<false>(mats + (size_t)x * 2 * N2, N2, N, pi, pj, P);
            }
        }
    }
}

// MINB selects one of two register budgets (2: up to 128 registers; 3: up to 80 for the forward
// kernel, 96 for the tangent kernel); both are compiled and the autotuner picks per kernel kind
// and quadrature. SPLIT compiles the split rule in (separate instantiations, so that the standard
// form's register allocation is not shaped by it).
template <int NE, bool ADJ, int MINB, bool SPLIT, bool PREC>
__global__ void __launch_bounds__(MINB == 3 ? (ADJ ? VX_LB3_THREADS_ADJ : VX_TPB_MIXED) : VX_TPB_MIXED,
                                  MINB == 3 ? (ADJ ? VX_LB3_CTAS_ADJ : 3) : MINB)
    k_pair_mixed(const __grid_constant__ Launch L) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ ZoneSh zs;
    __shared__ long long s_zone;
    __shared__ NodeSm s_nodes[VX_MAX_NE];
    __shared__ NodeMir s_mir[VX_MAX_NE / 2];
    __shared__ float4 s_half[VX_MAX_NE / 2];  // split rule: 1 + x, 1 - x, w of the n_e/2-node rule
    __shared__ uint16_t s_pij[VX_MAX_PAIRS];
    // tensor-core moments: per node the weights as (hi, lo) TF32 pairs, columns
    // (w(1+tau)^2, w(1-tau)^2, w(1-tau^2)) x (hi, lo) and two zero columns
    constexpr bool MMA = ADJ && !PREC && !SPLIT && NE > 0 && NE % 8 == 0 && VX_ADJ_MMA && VX_F32X2;
    __shared__ float s_w8[MMA ? VX_MAX_NE : 1][8];
    const Common &C = L.c;
    const int N = C.N, S = C.S, N2 = N * N, npair = C.npair;
    const int nq = ADJ ? 4 : 1;
    float *mats = reinterpret_cast<float *>(smraw);
    float *vec = mats + (size_t)nq * 2 * N2;
    size_t foff = ((size_t)nq * 2 * N2 + 4 * (size_t)S * N + 1) & ~(size_t)1;
    double *sc = reinterpret_cast<double *>(smraw + foff * 4);
    double *em = sc + N;
    double *shv = em + N;  // exp(-(eps_j - eps_0)/T) 2^sv
    double *red = shv + N;  // 64 doubles for block reductions
    float *part = reinterpret_cast<float *>(red + 64);  // [2 slots][nq][4 or 8][blockDim] partial projections
    const int tid = threadIdx.x;
    for (int k = tid; k < C.n_e; k += blockDim.x) {
        s_nodes[k].a = make_float4(L.n32.u[k], L.n32.v[k], L.n32.cp[k], L.n32.cm[k]);
        s_nodes[k].b = make_float4(L.n32.c0[k], L.n32.uh[k], L.n32.ul[k], 0.f);
        if (k < C.n_e / 2) {
            const int km = C.n_e - 1 - k;
            s_mir[k].a = make_float4(L.n32.u[k], L.n32.v[k], L.n32.cp[k], L.n32.cm[k]);
            s_mir[k].b = make_float4(L.n32.cm[k], L.n32.cp[k], L.n32.c0[k], L.n32.c0[k]);
            s_mir[k].c = make_float4(L.n32.uh[k], L.n32.uh[km], L.n32.ul[k], L.n32.ul[km]);
        }
    }
    for (int p = tid; p < npair; p += blockDim.x) s_pij[p] = C.pij[p];
    if (MMA)
        for (int k = tid; k < C.n_e; k += blockDim.x) {
            const float w3[3] = {L.n32.cp[k], L.n32.cm[k], L.n32.c0[k]};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float hi = __uint_as_float((__float_as_uint(w3[c]) + 0x1000u) & 0xffffe000u);  // nearest TF32
                s_w8[k][2 * c] = hi;
                s_w8[k][2 * c + 1] = __uint_as_float(__float_as_uint(w3[c] - hi) & 0xffffe000u);
            }
            s_w8[k][6] = s_w8[k][7] = 0.f;
        }
    if (SPLIT)
        for (int k = tid; k < C.n_e / 2; k += blockDim.x)
            s_half[k] = make_float4(L.n32.hp[k], L.n32.hm[k], L.n32.hw[k], 0.f);

    validate_offsets(L.off, L.n_rays, L.Z, L.flag);

    // Thread 0 reserves the next zone one iteration ahead and prefetches its inputs into L2 while
    // the current zone's quadrature runs, so a zone starts without an atomic or DRAM round trip.
    long long next_z = 0;
    if (tid == 0) next_z = (long long)atomicAdd(L.counter, 1ull);
    const int t_aux = blockDim.x > 32 ? 32 : 1;  // a thread of another warp for the set-up

    for (;;) {
        if (tid == 0) s_zone = next_z;
        __syncthreads();
        const long long z = s_zone;
        if (z >= L.Z) break;
        if (tid == 0) next_z = (long long)atomicAdd(L.counter, 1ull);

        // ---- zone set-up (FP64): the main scalars on thread 0, exponentials and 1/T^2 in parallel
        if (tid == t_aux) {
            const double T = L.state[4 * z + 0], ae = fabs(L.state[4 * z + 1]);
            zs.iT2 = 1.0 / (T * T);
            if (ae <= VX_ETA_MAX) {
                const double LOG2E = 1.4426950408889634;
                zs.K = (float)exp2neg(2.0 * ae * LOG2E);  // e^{-2|eta|}
            }
        }
        if (tid == 0) {
            double T = L.state[4 * z + 0], eta = L.state[4 * z + 1];
            int bad = !(T > 0.0) || !isfinite(T) || !isfinite(eta) || fabs(eta) > VX_ETA_MAX;
            zs.bad = bad;
            zs.T = T;
            zs.eta = eta;
            if (!bad) {
                const double LOG2E = 1.4426950408889634;
                double ae = fabs(eta);
                double il = LOG2E / T, el = ae * LOG2E;
                zs.il_h = (float)il;
                zs.il_l = (float)(il - (double)zs.il_h);
                zs.el_h = (float)el;
                zs.el_l = (float)(el - (double)zs.el_h);
                zs.neg = eta < 0.0;
                const double mu = ae * T;
                zs.mu_hi = (float)mu;
                zs.mu_lo = (float)(mu - (double)zs.mu_hi);
                zs.deg = ae > C.eta_sw;
                // zone scales: with O in [e^-|eta|, 1] and production vectors whose relevant
                // entries reach e^-|eta| times their row's largest, lift both off the FP32 floor.
                // sc also keeps r^2 = (2^sc O)^2 above 2^-126 (sc >= el - 62); sc + sv stays
                // floor(0.7 el), the headroom the contraction's products share
                int sc = zs.deg ? max((int)floor(0.3 * el), (int)ceil(el - 62.0)) : 0;
                zs.sv = zs.deg ? (int)floor(0.7 * el) - sc : 0;
                zs.sc = (float)sc;
                zs.c1 = ldexpf(1.f, -sc);
                zs.unsc = ldexp(1.0, -sc);
                // grid of the exact split: B_hi on 2^-kb with < 2^11 steps, P_hi and the sum on
                // 2^-(kb+11) with |sum| < 2^24 steps
                // (log2f is accurate to far better than the factor-2 margin left by the "- 1")
                float Bmax = (float)(C.h_max * il * 1.0001 + 1e-30);
                float Pmax = (float)(C.q0h_max * il + el + sc + 1.0);
                int kb = (int)floorf(fminf(11.f - log2f(Bmax), 13.f - log2f(Pmax + 2.f * Bmax))) - 1;
                kb = kb < -60 ? -60 : (kb > 60 ? 60 : kb);
                if (kb + 11 < 0) {  // grid coarser than 1: the integer shift would not be exact
                    zs.sc = 0.f;
                    zs.c1 = 1.f;
                    zs.unsc = 1.0;
                }
                zs.r2ok = zs.sc >= (float)(el - 62.0);  // the tangents' r^2 form is in range
                zs.sB = ldexpf(1.f, kb);
                zs.iB = ldexpf(1.f, -kb);
                zs.sP = ldexpf(1.f, kb + 11);
                zs.iP = ldexpf(1.f, -(kb + 11));
            }
        }
        __syncthreads();
        const double T = zs.T;
        if (zs.bad) {
            // invalid state: NaN outputs, raise the flag, skip the work
            const double nan = __longlong_as_double(0x7ff8000000000000ll);
            for (int e = tid; e < S * N; e += blockDim.x) {
                size_t o = (size_t)z * S * N + e;
                if (L.j0) { L.j0[o] = nan; L.chi0[o] = nan; L.j1[o] = nan; L.chi1[o] = nan; }
                if (ADJ && L.jac)
                    for (int q = 0; q < 12; ++q) L.jac[o * 12 + q] = nan;
            }
            if (L.phi)
                for (int e = tid; e < 4 * N2; e += blockDim.x) L.phi[(size_t)z * 4 * N2 + e] = nan;
            if (ADJ && L.grad_state && tid < 4) L.grad_state[4 * z + tid] = nan;
            if (!ADJ && L.blocks)
                for (int e = tid; e < S * 4 * N2; e += blockDim.x) L.blocks[(size_t)z * S * 4 * N2 + e] = nan;
            if (!ADJ && L.grad_J)
                for (int e = tid; e < S * N; e += blockDim.x) {
                    L.grad_J[(size_t)z * S * N + e] = nan;
                    L.grad_H[(size_t)z * S * N + e] = nan;
                }
            if (tid == 0) atomicOr(L.flag, VX_FLAG_BAD_STATE);
            __syncthreads();
            continue;
        }

        // ---- per-zone FP64 scales and contraction vectors -------------------------------------
        {
            const double il = 1.4426950408889634 / T;  // log2(e)/T
            for (int e = tid; e < 3 * N; e += blockDim.x) {
                const int i = e % N, which = e / N;
                if (which == 0) sc[i] = exp2neg((C.eps[i] + C.eps[0]) * il + (double)zs.sv);  // e^{-(eps_i+eps_0)/T} 2^-sv
                else if (which == 1) em[i] = exp2neg(C.eps[i] * il);                     // e^{-eps_i/T}
                else shv[i] = exp2neg((C.eps[i] - C.eps[0]) * il - (double)zs.sv);       // e^{-(eps_i-eps_0)/T} 2^sv
            }
        }
        __syncthreads();
        for (int e = tid; e < 4 * S * N; e += blockDim.x) {
            int o = e / (S * N), s = (e / N) % S, j = e % N;
            size_t a = ((size_t)z * S + C.partner[s]) * N + j;
            double v;
            if (o == 0) v = C.w[j] * (1.0 - L.J[a]) * shv[j];  // production: w (1 - J) e^{-(eps_j - eps_0)/T} 2^sv
            else if (o == 2) v = C.w[j] * L.H[a] * shv[j];
            else v = C.w[j] * (o == 1 ? L.J[a] : L.H[a]);
            vec[e] = (float)v;
        }

        if (tid == 0 && next_z < L.Z) {
            prefetch_l2(L.state + 4 * next_z);
            const size_t off = (size_t)next_z * S * N;
            for (int b = 0; b < S * N; b += 16) {
                prefetch_l2(L.J + off + b);
                prefetch_l2(L.H + off + b);
            }
        }

        // ---- quadrature: the npair * n_mu (pair, omega) units in equal contiguous ranges --------
        // A thread's range covers whole pairs and at most one partial pair at each end; partial
        // projections go to two slots per thread and are combined in thread order below.
        const int nmu = C.n_mu, U = npair * nmu, TB = blockDim.x;
        const int u0 = tid * U / TB, u1 = (tid + 1) * U / TB;
        const float il_h = zs.il_h, el_h = zs.el_h;
        const bool deg = zs.deg, neg = zs.neg;
        // One iteration per unit (28 or 29 per thread at N = 21, n_mu = 32): every lane runs the
        // node loop in step; only the flush at a pair boundary diverges.
        const bool use_mma = MMA && !deg && nmu % 16 == 0;
        if (use_mma)
            mma_quadrature<NE>(s_mir, s_w8, L.tab32, npair, nmu, s_pij, mats, N2, N, il_h, el_h, zs.K, neg);
        int p = u0 / nmu, m = u0 - (u0 / nmu) * nmu, mb = m;
        bool first = true;
        Proj PO, PTa, PTp, PEt;
        PO.zero();
        if (ADJ) { PTa.zero(); PTp.zero(); PEt.zero(); }
#pragma unroll 1
        for (int u = use_mma ? u1 : u0; u < u1; ++u) {
            {
                const float4 *rec = L.tab32 + ((size_t)p * nmu + m) * 2;  // a thread's units are consecutive records
                const float4 R0 = __ldg(rec), R1 = __ldg(rec + 1);
                const float h = R0.x, h_lo = R0.y, Em = R0.z, Em_lo = R0.w;
                float kp = R1.x, km = R1.y;
                const float k0 = R1.z;
                if (neg) {  // eta < 0: electron and positron exchange roles, M+ <-> M-
                    float t = kp; kp = km; km = t;
                }
                Mom mo, ta, tp, et;
                mo.zero();
                if (ADJ) { ta.zero(); tp.zero(); et.zero(); }
                const float B = h * il_h;
                const float Pp = fmaf(Em, il_h, el_h);
                // split rule (degenerate zones only): is the Fermi edge (|eta| T in the eta >= 0
                // frame) inside (E-, E+)? Decided on FP32 pairs (~2^-48 relative), like the
                // definition's FP64 comparison
                bool in_split = false;
                float rA = 0.f, dls = 0.f;
                if (SPLIT && deg) {
                    float dh, dl, gh, gl;
                    df_diff(zs.mu_hi, zs.mu_lo, Em, Em_lo, dh, dl);   // mu - E-
                    df_diff(2.f * h, 2.f * h_lo, dh, dl, gh, gl);     // E+ - mu
                    in_split = (dh > 0.f || (dh == 0.f && dl > 0.f)) && (gh > 0.f || (gh == 0.f && gl > 0.f));
                    if (in_split) {
                        rA = fminf(fmaxf(__fdividef(dh, 2.f * h), 0.f), 1.f);
                        // (E- + 2 h rA) - mu: the boundary's offset from the edge, then in log2 units
                        const float delta = fmaf(2.f * h, rA, -dh) + fmaf(2.f * h_lo, rA, -dl);
                        dls = fmaf(delta, il_h, zs.sc);
                    }
                }
                if (in_split) {
                    const float Qs = fmaf(2.f * (Em + h), il_h, zs.sc);
                    SplitUnit<ADJ, ADJ>::run(s_half, C.n_e / 2, rA, B, dls, Qs, h, Em, zs.c1, mo, ta, tp, et);
                    const Coef cf = make_coef(kp, km, k0, R1.w);
                    project<PREC>(PO, mo, cf);
                    if (ADJ) {
                        project<PREC>(PTa, ta, cf);
                        project<PREC>(PTp, tp, cf);
                        project<PREC, true>(PEt, et, cf);
                    }
                } else {
                    // exact split of the electron argument (degenerate path; every zone in the
                    // precise mode): B = h log2e/T and P = E- log2e/T - |eta| log2e as
                    // double-floats, their high parts on the zone's 2^-kb and 2^-(kb+11) grids
                    float Bq = 0.f, Bl = 0.f, Pq = 0.f, Pl = 0.f;
                    if (deg || PREC) {
                        const float il_l = zs.il_l, el_l = zs.el_l;
                        float bh = __fmul_rn(h, il_h);
                        float bl = __fadd_rn(fmaf(h, il_h, -bh), __fadd_rn(__fmul_rn(h, il_l), __fmul_rn(h_lo, il_h)));
                        Bq = __fmul_rn(rintf(__fmul_rn(bh, zs.sB)), zs.iB);
                        Bl = __fadd_rn(__fsub_rn(bh, Bq), bl);
                        float ph = __fmul_rn(Em, il_h);
                        float pl = __fadd_rn(fmaf(Em, il_h, -ph), __fadd_rn(__fmul_rn(Em, il_l), __fmul_rn(Em_lo, il_h)));
                        float s = __fsub_rn(ph, el_h);
                        float bb = __fsub_rn(s, ph);
                        float err = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, bb)), __fsub_rn(-el_h, bb));
                        float slo = __fsub_rn(__fadd_rn(err, pl), el_l);
                        Pq = __fmul_rn(rintf(__fmul_rn(s, zs.sP)), zs.iP);
                        Pl = __fadd_rn(__fsub_rn(s, Pq), slo);
                        Pq = __fadd_rn(Pq, zs.sc);  // exact: an integer on the same grid
                    }
                    if (!deg) {
                        const float Pe = fmaf(Em, il_h, -el_h);
                        node_loop<NE, ADJ, false, SPLIT, PREC>(s_nodes, s_mir, C.n_e, B, Pe, Pp, Bq, Bl, Pq, Pl, h, Em, 1.f, zs.K, false, mo, ta, tp, et);
                    } else {
                        node_loop<NE, ADJ, true, SPLIT, false, !PREC>(s_nodes, s_mir, C.n_e, B, 0.f, Pp, Bq, Bl, Pq, Pl, h, Em, zs.c1, 0.f, zs.r2ok, mo, ta, tp, et);
                    }
                    const Coef cf = make_coef(kp, km, k0, R1.w);
                    project<PREC>(PO, mo, cf);
                    if (ADJ) {
                        project<PREC>(PTa, ta, cf);
                        project<PREC>(PTp, tp, cf);
                        project<PREC, true>(PEt, et, cf);
                    }
                }
            }
            ++m;
            if (m == nmu || u + 1 == u1) {  // end of a pair or of this thread's range: flush
                if (mb == 0 && m == nmu) {  // the whole pair in this thread
                    const int pi = s_pij[p] >> 8, pj = s_pij[p] & 0xff;
                    store_proj<PREC>(mats + 0 * 2 * (size_t)N2, N2, N, pi, pj, PO);
                    if (ADJ) {
                        store_proj<PREC>(mats + 1 * 2 * (size_t)N2, N2, N, pi, pj, PTa);
                        store_proj<PREC>(mats + 2 * 2 * (size_t)N2, N2, N, pi, pj, PTp);
                        store_proj<PREC>(mats + 3 * 2 * (size_t)N2, N2, N, pi, pj, PEt);
                    }
                } else {
                    const int sq = (first ? 0 : 1) * nq;
                    part_put<PREC>(part, TB, tid, sq, PO);
                    if (ADJ) {
                        part_put<PREC>(part, TB, tid, sq + 1, PTa);
                        part_put<PREC>(part, TB, tid, sq + 2, PTp);
                        part_put<PREC>(part, TB, tid, sq + 3, PEt);
                    }
                }
                PO.zero();
                if (ADJ) { PTa.zero(); PTp.zero(); PEt.zero(); }
                first = false;
                ++p;
                m = 0;
                mb = 0;
            }
        }
        __syncthreads();
        // pairs split between threads: sum their partial projections over the owning threads in
        // order (owner of unit v: ceil((v+1) TB / U) - 1), then store
        for (int p = use_mma ? npair : tid; p < npair; p += TB) {
            const int ua = p * nmu, ub = ua + nmu - 1;
            const int ta = ((ua + 1) * TB + U - 1) / U - 1, tb = ((ub + 1) * TB + U - 1) / U - 1;
            if (ta == tb) continue;
            const int pi = s_pij[p] >> 8, pj = s_pij[p] & 0xff;
            for (int q = 0; q < nq; ++q) {
                Proj acc;
                acc.zero();
                for (int t = ta; t <= tb; ++t) {
                    const int sl = (t == ta && ua > t * U / TB) ? 1 : 0;
                    const Proj x = part_get<PREC>(part, TB, t, sl * nq + q);
                    if (PREC) {
                        acc2(acc.o0I, acc.l0I, x.o0I); acc.l0I = __fadd_rn(acc.l0I, x.l0I);
                        acc2(acc.o0II, acc.l0II, x.o0II); acc.l0II = __fadd_rn(acc.l0II, x.l0II);
                        acc2(acc.o1I, acc.l1I, x.o1I); acc.l1I = __fadd_rn(acc.l1I, x.l1I);
                        acc2(acc.o1II, acc.l1II, x.o1II); acc.l1II = __fadd_rn(acc.l1II, x.l1II);
                    } else {
                        acc.o0I += x.o0I;
                        acc.o0II += x.o0II;
                        acc.o1I += x.o1I;
                        acc.o1II += x.o1II;
                    }
                }
                store_proj<PREC>(mats + (size_t)q * 2 * N2, N2, N, pi, pj, acc);
            }
        }
        __syncthreads();

        // ---- contraction (and tangents) --------------------------------------------------------
        const double two_pi = 6.283185307179586;
        const double c0 = two_pi * C.norm * C.g2 * zs.unsc, c1 = 3.0 * c0;
        const double iT2 = zs.iT2;
        const double sgn = zs.neg ? -1.0 : 1.0;  // d/deta of the eta >= 0 mapping
        const int nout = 4 * S * N;
        double gT = 0.0, gE = 0.0;
        const bool want_fwd = L.j0 != nullptr;
        for (int e = tid; e < nout; e += blockDim.x) {
            const int o = e / (S * N), s = (e / N) % S, i = e % N;
            const int l = o >> 1;                 // j0, chi0: l = 0; j1, chi1: l = 1
            const bool prod = (o & 1) == 0;       // j0, j1 come from production
            const float bI = C.bI[s], bII = C.bII[s];
            const float *v = vec + (size_t)(o * S + s) * N;
            const double cl = l ? c1 : c0;
            const double scal = prod ? sc[i] : 1.0;
            double res[3];  // contraction of: the kernel, its T tangent, its eta tangent
            const int nres = ADJ ? 3 : 1;
#pragma unroll
            for (int r = 0; r < nres; ++r) {
                const int q = r == 0 ? 0 : r == 2 ? 3 : (prod ? 2 : 1);
                const float *M = mats + (size_t)(q * 2 + l) * N2;
                if (PREC && (l == 1 || q == 3)) {  // sums whose terms change sign
                    float ah = 0.f, al = 0.f;
                    for (int j = 0; j < N; ++j) contract2(ah, al, bI, M[i * N + j], bII, M[j * N + i], v[j]);
                    res[r] = (double)ah + (double)al;
                } else {
                    float acc = 0.f;
                    for (int j = 0; j < N; ++j) acc = fmaf(fmaf(bI, M[i * N + j], bII * M[j * N + i]), v[j], acc);
                    res[r] = (double)acc;
                }
            }
            const size_t oi = ((size_t)z * S + s) * N + i;
            const double fwd = cl * scal * res[0];
            if (want_fwd) {
                double *dst = o == 0 ? L.j0 : o == 1 ? L.chi0 : o == 2 ? L.j1 : L.chi1;
                dst[oi] = fwd;
                if (!isfinite(fwd)) atomicOr(L.flag, VX_FLAG_NONFINITE);
            }
            if (ADJ) {
                // production: d/dT = e^{-q0/T} GTp / T^2 ; annihilation: d/dT = -GTa / T^2
                const double dT = cl * scal * (prod ? 1.0 : -1.0) * res[1] * iT2;
                const double dE = cl * scal * sgn * res[2];
                if (L.jac) {
                    L.jac[oi * 12 + o * 3 + 0] = dT;
                    L.jac[oi * 12 + o * 3 + 1] = dE;
                    L.jac[oi * 12 + o * 3 + 2] = 0.0;
                    if (!isfinite(dT) || !isfinite(dE)) atomicOr(L.flag, VX_FLAG_NONFINITE);
                }
                const double *g = o == 0 ? L.g_j0 : o == 1 ? L.g_chi0 : o == 2 ? L.g_j1 : L.g_chi1;
                if (g) {
                    const double gv = g[oi];
                    gT += gv * dT;
                    gE += gv * dE;
                }
            }
        }
        if (ADJ && L.grad_state) {
            // deterministic block reduction: fixed shuffle tree, then warps in order
            for (int off = 16; off > 0; off >>= 1) {
                gT += __shfl_down_sync(0xffffffffu, gT, off);
                gE += __shfl_down_sync(0xffffffffu, gE, off);
            }
            const int nw = (blockDim.x + 31) >> 5;
            if ((tid & 31) == 0) { red[2 * (tid >> 5)] = gT; red[2 * (tid >> 5) + 1] = gE; }
            __syncthreads();
            if (tid == 0) {
                double a = 0.0, b = 0.0;
                for (int w = 0; w < nw; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
                L.grad_state[4 * z + 0] = a;
                L.grad_state[4 * z + 1] = b;
                L.grad_state[4 * z + 2] = 0.0;
                L.grad_state[4 * z + 3] = 0.0;
            }
        }
        if (!ADJ && L.blocks) {
            // d(rates)/d(partner spectrum): the coefficients of (1 - J), J, H, H in the contraction
            // above, scaled in FP64 (production carries e^{-(eps_i + eps_j)/T} = sc[i] shv[j])
            const int nb = 4 * N2;
            for (int e = tid; e < S * nb; e += blockDim.x) {
                const int s = e / nb, o = (e / N2) & 3, i = (e / N) % N, j = e % N;
                const float *M = mats + (size_t)(o >> 1) * N2;
                const double k = PREC ? kern2(C.bI[s], M[i * N + j], C.bII[s], M[j * N + i])
                                      : (double)fmaf(C.bI[s], M[i * N + j], C.bII[s] * M[j * N + i]);
                double f = ((o >> 1) ? c1 : c0) * C.w[j];
                if ((o & 1) == 0) f *= (o == 0 ? -sc[i] : sc[i]) * shv[j];
                L.blocks[(size_t)z * S * nb + e] = f * k;
            }
        }
        if (!ADJ && L.grad_J) {
            // vector-Jacobian product with those coefficients, per spectrum q and bin j; spectrum q
            // is read by species partner[q] (the pairing is an involution)
            for (int e = tid; e < 2 * S * N; e += blockDim.x) {
                const int hq = e / (S * N), q = (e / N) % S, j = e % N;
                const int s = C.partner[q];
                const float bI = C.bI[s], bII = C.bII[s];
                const float *M = mats + (size_t)hq * N2;
                const double *gp = hq ? L.g_j1 : L.g_j0, *ga = hq ? L.g_chi1 : L.g_chi0;
                const size_t row = ((size_t)z * S + s) * N;
                double sa = 0.0, sp = 0.0;  // annihilation and production sums over the species' bins i
                for (int i = 0; i < N; ++i) {
                    const double k = PREC ? kern2(bI, M[i * N + j], bII, M[j * N + i])
                                          : (double)fmaf(bI, M[i * N + j], bII * M[j * N + i]);
                    if (ga) sa = fma(k, ga[row + i], sa);
                    if (gp) sp = fma(k, gp[row + i] * sc[i], sp);
                }
                const double v = (hq ? c1 : c0) * C.w[j] * (hq ? sa + shv[j] * sp : sa - shv[j] * sp);
                (hq ? L.grad_H : L.grad_J)[((size_t)z * S + q) * N + j] = v;
            }
        }
        if (L.phi) {  // raw kernel of term I, G2 applied: [dir][l][i][j]
            for (int e = tid; e < 4 * N2; e += blockDim.x) {
                const int d = e / (2 * N2), l = (e / N2) & 1, ij = e % N2, i = ij / N, j = ij % N;
                double a = (double)mats[l * N2 + ij];
                double v = C.g2 * zs.unsc * (d == 0 ? em[i] * em[j] * a : a);
                L.phi[(size_t)z * 4 * N2 + e] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace vx
