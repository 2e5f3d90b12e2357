/*
 * vx_abs.h -- charged-current neutrino absorption and emission on free nucleons, per zone,
 * species and energy bin, with their Jacobian.
 *
 * Where it sits in the method. The implicit transport step of Marek et al., arXiv:1404.1719,
 * sec. 2.1, couples the neutrino moments to the matter through the emission, absorption and
 * scattering rates; the Newton iteration needs each rate and its derivatives with respect to the
 * matter state. This entry family supplies the absorption and emission of electron neutrinos
 * and antineutrinos on nucleons, beside the pair kernel (vx_rates.h) and neutrino-electron
 * scattering (vx_nes.h). The paper does not write the rates down; the definition used is:
 *   - reactions nu_e + n <-> e- + p and anti-nu_e + p <-> e+ + n (heavy-lepton neutrinos: none);
 *   - zero recoil: lepton energy E = eps + Q (nu_e), eps - Q (anti-nu_e, nothing at or below
 *     eps = Q), Q = m_n - m_p = 1.29333236 MeV; massless leptons;
 *   - chi(eps) = (g2/pi)(1 + 3 gA^2) n_in E^2 (1 - f_l(E)), j(eps) = (g2/pi)(1 + 3 gA^2) n_out E^2
 *     f_l(E), gA = 1.2754, f_l the electron (positron) occupation at eta_e (-eta_e);
 *   - non-degenerate free nucleons without nuclei: n_p = rho Y_e / m_u, n_n = rho (1 - Y_e) / m_u
 *     in fm^-3 (m_u = 1.66053906660e-24 g); n_in = n_n, n_out = n_p for nu_e and the reverse for
 *     anti-nu_e (the nucleons' final-state blocking integral equals the target density then);
 *   - the rates are isotropic: j1 = chi1 = 0.
 * The rates obey detailed balance j/chi = exp(-(eps - mu_nu)/T), mu_nu = eta_e T - Q -
 * T ln((1 - Y_e)/Y_e) for nu_e.
 *
 * Conventions as in vx_rates.h: a handle per energy grid and species list, caller-owned device
 * arrays, asynchronous on `stream`, argument checks on the host before any launch; a bad zone
 * state gives NaN for that zone and raises the numeric flag (vx_abs_check).
 */
#ifndef VX_ABS_H
#define VX_ABS_H

#include "vx_rates.h" /* vx_config, vx_batch, vx_out, vx_status, vx_stream */

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vx_abs vx_abs;

/* Creates a handle. Reads from cfg: n_bins (1..32), eps (host, positive), n_species (1..3),
 * species (host, distinct vx_species values), g2 (the rates' global scale, finite, non-zero
 * magnitudes of any size) and prec (VX_PREC_MIXED: the exponent argument in FP64, the occupation
 * factors and products in FP32 with their powers of two carried exactly into the FP64 results,
 * relative error ~1e-6; the T-derivative needs T >= 1e-15 MeV there. VX_PREC_FP64: FP64 throughout).
 * weights, n_mu, n_e, sin2w, norm and eta_fp64 are not used; flags must be 0.
 * Errors: VX_ERR_INVALID_ARG, VX_ERR_UNSUPPORTED (flags), VX_ERR_OOM, VX_ERR_CUDA. */
vx_status vx_abs_create(const vx_config *cfg, vx_abs **out);

/* Rates of every zone: out->j0, chi0, j1, chi1 (device [Z][S][N], FP64; j1 = chi1 = 0), from
 * batch->state (device [Z][4]: T in MeV, eta_e, Y_e, rho in g/cm^3). batch->J and batch->H are
 * not read (may be NULL); batch->ray_offsets as in vx_rates.h (device int32 [R+1] or NULL,
 * validated, only reported). out->phi must be NULL (these rates have no kernel to dump).
 * A zone with T <= 0, a non-finite input, Y_e outside [0, 1] or rho < 0 gets NaN and raises the
 * numeric flag. Errors: VX_ERR_INVALID_ARG (NULL handle, batch or out; non-device or misaligned
 * pointers; n_zones < 0). */
vx_status vx_abs_eval(vx_abs *h, const vx_batch *batch, const vx_out *out, vx_stream stream);

/* Jacobian (device [Z][S][N][4][3], FP64, NULL to skip) of (j0, chi0, j1, chi1) with respect to
 * (T at fixed eta_e, Y_e, rho; eta_e; Y_e at fixed T, eta_e, rho), and, if fwd is not NULL, the
 * rates of the same pass. Every rate is proportional to rho at fixed (T, eta_e, Y_e), so its
 * derivative in rho is rate / rho (not stored). vx_eos_chain turns the columns into derivatives
 * at fixed density and electron fraction. Errors as vx_abs_eval. */
vx_status vx_abs_adjoint(vx_abs *h, const vx_batch *batch, double *jac, const vx_out *fwd, vx_stream stream);

/* VX_OK, or VX_ERR_NUMERIC if a call since the last check met a bad zone state, a non-finite
 * result or invalid ray offsets (then clears the flag). Synchronises `stream`. */
vx_status vx_abs_check(vx_abs *h, vx_stream stream);

/* Frees the handle (NULL is allowed). */
void vx_abs_destroy(vx_abs *h);

#ifdef __cplusplus
}
#endif
#endif /* VX_ABS_H */
