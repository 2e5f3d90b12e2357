/*
 * vx_eos.h -- the electron-gas closure eta_e(rho, Y_e, T) and the chain rule that turns the rate
 * kernels' derivatives at fixed eta_e into derivatives at fixed density and electron fraction.
 *
 * Where it sits in the method. The paper (Marek et al., arXiv:1404.1719, sec. 2.1) closes the
 * hydrodynamic and transport system with an equation of state; the rate kernels of vx_rates.h
 * and vx_nes.h take the electron degeneracy eta_e = mu_e/T as an input. This closure supplies
 * eta_e from the hydrodynamic variables, so that the implicit Newton step (sec. 2.1) can take
 * the rates' derivatives with respect to T, Y_e and rho. READING: electrons and positrons are a
 * massless ideal Fermi gas in equilibrium (the same massless leptons as the kernels), so the net
 * electron density is (T/hbar c)^3 (eta^3 + pi^2 eta)/(3 pi^2) = rho Y_e / m_u, a cubic in eta
 * with one real root; hbar c = 197.3269804 MeV fm, m_u = 1.66053906660e-24 g. Nuclei, the
 * electron mass and the rest of a stellar equation of state are out of scope.
 *
 * Conventions as in vx_rates.h (device arrays owned by the caller, asynchronous on `stream`,
 * argument checks on the host before any launch).
 */
#ifndef VX_EOS_H
#define VX_EOS_H

#include "vx_rates.h" /* vx_status, vx_stream */

#ifdef __cplusplus
extern "C" {
#endif

/* For every zone of state (device [Z][4]: T in MeV, eta_e, Y_e, rho in g/cm^3) writes eta_e into
 * state[z][1] from T, Y_e and rho, and, if deta is not NULL, deta (device [Z][3]) =
 * d eta_e / d(T, Y_e, rho). A zone with T <= 0, Y_e < 0, rho < 0 or a non-finite input gets NaN.
 * Errors: VX_ERR_INVALID_ARG (n_zones < 0, NULL or non-device state with n_zones > 0). */
vx_status vx_eos_eta(long long n_zones, double *state, double *deta, vx_stream stream);

/* Chain rule for jacobians laid out [Z][rows][3] with columns d/dT (at fixed eta_e), d/deta_e and
 * d/dY_e at fixed (T, eta_e, rho) (the rate kernels' [Z][S][N][4][3] has rows = 4 S N; that
 * column is zero for the pair and scattering kernels, whose rates depend on Y_e only through
 * eta_e): writes jac_out [Z][rows][3] = (d/dT, d/dY_e, d/drho) at fixed (rho, Y_e), (T, rho) and
 * (T, Y_e):
 *   d/dT|_{rho,Ye} = d/dT|_eta + d/deta * deta/dT,  d/dY_e = d/dY_e|_eta + d/deta * deta/dY_e,
 *   d/drho = d/deta * deta/drho,  with deta from vx_eos_eta. A rate with its own dependence on rho
 *   at fixed eta_e (the absorption rates of vx_abs.h: rate / rho) needs that term added by the
 *   caller. jac_out may equal jac_in.
 * Errors: VX_ERR_INVALID_ARG (negative sizes, NULL or non-device arrays with work to do). */
vx_status vx_eos_chain(long long n_zones, int rows, const double *deta, const double *jac_in, double *jac_out,
                       vx_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* VX_EOS_H */
