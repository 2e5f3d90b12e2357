/*
 * vx_nes.h -- C ABI of the inelastic neutrino-electron scattering (NES) rate kernel.
 *
 * Where it sits in the method. Marek et al. (arXiv:1404.1719, sec. 2.1) list the neutrinos'
 * emission, absorption and scattering rates among the components of the transport system that
 * each ray's implicit Newton solve needs; like the pair process of vx_rates.h, the scattering
 * kernels are not written down in the paper. The kernel evaluated here is the standard one for
 * nu + e- -> nu + e- with massless electrons and Fermi-Dirac blocking:
 *
 *   R^out_X(eps, eps', w) = (G2/(eps eps')) Int d3p/(2E) d3p'/(2E') d4(k + p - k' - p')
 *                           f(E) (1 - f(E')) M_X,   M_I = (k.p)(k'.p'),  M_II = (k.p')(k'.p),
 *   R^in = e^{-(eps - eps')/T} R^out (detailed balance), Phi^dir_l = Int d(cos w) P_l(cos w) R^dir,
 *
 * with couplings (C_V +- C_A)^2 per species as for the pair kernel (nu_e; anti-nu_e with the two
 * terms swapped; nu_x), each species scattering within its own spectrum. Scattering on positrons
 * is not included. Readings:
 *   - Gauss-Legendre in cos(omega) (n_mu nodes, 2..32);
 *   - the electron energy E in [E_min, inf), E_min = (|q| - q0)/2, on three panels of n_e/3 nodes
 *     each: Gauss-Legendre from 30 T below the lower Fermi edge (mu_e - max(q0, 0)) up to it,
 *     Gauss-Legendre between the two edges, Gauss-Laguerre (scale T) above the upper edge
 *     (mu_e + max(-q0, 0)), every panel clipped at E_min;
 *   - each bin pair is integrated in the down-scattering order (eps_i >= eps_j) and the other
 *     order follows from time reversal, so the discrete kernel obeys detailed balance and time
 *     reversal exactly.
 *   Outputs per zone z, species s and bin i, with J, H the species' own moments, w_j = eps_j^2 d(eps_j)
 *   and C = `norm`:
 *     j0   =  2 pi C sum_j w_j Phi^in_0(i,j) J_j,     chi0 =  2 pi C sum_j w_j Phi^out_0(i,j) (1 - J_j),
 *     j1   = -6 pi C sum_j w_j Phi^in_1(i,j) H_j,     chi1 = -6 pi C sum_j w_j Phi^out_1(i,j) H_j,
 *   so that the source of the occupation f(eps, mu) has the same form as for the pair process,
 *   (1 - f)(j0 - mu j1) - f (chi0 + mu chi1).
 *
 * Conventions are those of vx_rates.h: device arrays of the current device owned by the caller,
 * asynchronous calls on `stream`, host-side argument checks before any launch (VX_ERR_INVALID_ARG,
 * nothing written), device numeric problems (T <= 0 or non-finite, |eta_e| > 80, a non-finite
 * result) give NaN outputs for the zone and a flag read by vx_nes_check. A handle is not
 * thread-safe.
 */
#ifndef VX_NES_H
#define VX_NES_H

#include "vx_rates.h" /* vx_status, vx_stream, vx_config, vx_batch, vx_out */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vx_nes vx_nes; /* opaque handle */

/* Builds the handle for one energy grid and quadrature from a vx_config:
 *   n_bins 2..31, eps and weights as in vx_rates.h; n_mu 2..32; n_e a multiple of 3, 6..96
 *   (n_e/3 nodes per panel); n_species 1..3 distinct vx_species in any combination; sin2w, g2,
 *   norm as in vx_rates.h; prec VX_PREC_MIXED (FP32 quadrature, FP64 scaling) or VX_PREC_FP64;
 *   eta_fp64 and flags must be 0.
 * Builds the (bin pair, omega) table in FP64 on the host and uploads it. Errors:
 * VX_ERR_INVALID_ARG, VX_ERR_OOM, VX_ERR_CUDA; *out is NULL then. */
vx_status vx_nes_create(const vx_config *cfg, vx_nes **out);

/* Forward NES rates of every zone into *out (j0, chi0, j1, chi1 device [Z][S][N]); out->phi, if not
 * NULL, receives the kernel, device [Z][2 X][2 dir][2 l][N][N] FP64 (X = I, II; dir 0 = in, 1 = out;
 * G2 applied, couplings not). batch: as in vx_rates.h (ray_offsets device memory or NULL, validated
 * on the device; state T, eta_e used). */
vx_status vx_nes_eval(vx_nes *h, const vx_batch *batch, const vx_out *out, vx_stream stream);

/* Derivatives with respect to the zone state from one pass: jac device [Z][S][N][4][3],
 * d(j0, chi0, j1, chi1)/d(T, eta_e, Y_e) at fixed nodes (the rule applied to the integrand's
 * derivative; the panels' nodes are those placed for the zone); the Y_e column is 0 (compose with
 * vx_eos_chain of vx_eos.h for derivatives at fixed rho and Y_e). fwd, if not NULL, receives the
 * forward rates of the same pass (its phi member must be NULL). Both precisions. */
vx_status vx_nes_adjoint(vx_nes *h, const vx_batch *batch, double *jac, const vx_out *fwd, vx_stream stream);

/* The same computations on HOST arrays (vx_nes_eval, vx_nes_adjoint with host pointers; host
 * ray_offsets, validated on the host): the batch goes through the handle's two staging slots of
 * device memory (640 MiB each, allocated on first use) in chunks of zones, one stream per slot,
 * so the copies of one chunk overlap the kernel of the next. Host arrays should be pinned for the
 * copies to be asynchronous. Synchronous: returns when every output is in host memory; the
 * numeric flag is reported by vx_nes_check as for the device calls. out->phi must be NULL.
 * Errors: VX_ERR_INVALID_ARG (NULL arrays, invalid offsets), VX_ERR_OOM, VX_ERR_CUDA. */
vx_status vx_nes_eval_host(vx_nes *h, const vx_batch *host_batch, const vx_out *host_out);
vx_status vx_nes_adjoint_host(vx_nes *h, const vx_batch *host_batch, double *host_jac, const vx_out *host_fwd);

/* Synchronises `stream`, reads and clears the device numeric flag: VX_OK or VX_ERR_NUMERIC. */
vx_status vx_nes_check(vx_nes *h, vx_stream stream);

/* Releases the handle (NULL is a no-op). Synchronises the device. */
void vx_nes_destroy(vx_nes *h);

#ifdef __cplusplus
}
#endif
#endif /* VX_NES_H */
