/*
 * vx_abs_oracle.c -- TEST INFRASTRUCTURE ONLY. Plain FP64 reference of the charged-current
 * neutrino absorption and emission rates on free nucleons (the "absorption, emission" rates the
 * paper lists among the components of the implicit transport system, Marek et al.,
 * arXiv:1404.1719, sec. 2.1). Only tests/, the smoke check and the bench's CPU baseline call it;
 * the library never links or loads it.
 *
 * The paper does not write these rates down. The definition used here, with every choice stated
 * as a reading:
 *   A1 reactions: nu_e + n <-> e- + p (species 0) and anti-nu_e + p <-> e+ + n (species 1); the
 *      heavy-lepton neutrinos (species 2) have no charged-current reaction: all their rates are 0.
 *   A2 zero recoil: the nucleons are infinitely heavy, so the charged lepton takes the neutrino
 *      energy plus the mass difference: E = eps + Q (nu_e), E = eps - Q (anti-nu_e, zero at and
 *      below the threshold eps <= Q), Q = m_n - m_p = 1.29333236 MeV. Leptons are massless, as in
 *      the pair and scattering kernels. The rates are then isotropic: j1 = chi1 = 0.
 *   A3 rates (per unit length, in the units the global scale g2 gives them):
 *        chi(eps) = (g2 / pi) (1 + 3 gA^2) n_in  E^2 (1 - f_l(E))     absorption
 *        j(eps)   = (g2 / pi) (1 + 3 gA^2) n_out E^2 f_l(E)           emission
 *      with gA = 1.2754; for nu_e n_in = n_n, n_out = n_p, f_l the electron occupation
 *      1/(1 + exp(E/T - eta_e)); for anti-nu_e n_in = n_p, n_out = n_n, f_l the positron
 *      occupation 1/(1 + exp(E/T + eta_e)).
 *   A4 nucleons: a free, non-degenerate (Maxwell-Boltzmann) gas of neutrons and protons without
 *      nuclei, n_p = rho Y_e / m_u, n_n = rho (1 - Y_e) / m_u (charge neutrality), in fm^-3 with
 *      rho in g/cm^3, m_u = 1.66053906660e-24 g, 1 fm^3 = 1e-39 cm^3. The final-state blocking
 *      integral of the nucleons, (n_n - n_p) / (1 - exp((mu_p - mu_n)/T)) with kinetic chemical
 *      potentials, then equals n_n exactly (and n_p for the reverse reaction).
 *   A5 outputs as for the other kernels: j0 = j, chi0 = chi, j1 = chi1 = 0 per zone, species and
 *      bin, and the Jacobian [Z][S][N][4][3] with columns d/dT (at fixed eta_e, Y_e, rho),
 *      d/deta_e and d/dY_e (at fixed T, eta_e, rho). Every rate is proportional to rho at fixed
 *      (T, eta_e, Y_e), so d/drho = rate / rho.
 *   A zone with T <= 0, a non-finite input, Y_e outside [0, 1] or rho < 0 gets NaN.
 *
 * Detailed balance follows from A3-A4: j/chi = exp(-(eps - mu_nu)/T) with
 * mu_nu = mu_e + mu_p - mu_n = eta_e T - Q - T ln(n_n/n_p) for nu_e (and -mu_nu for anti-nu_e).
 * The tests check that, the threshold, Pauli blocking, the scalings in rho and Y_e, and the
 * Jacobian against central differences.
 */
#include <math.h>
#include <stddef.h>

static const double kQ = 1.29333236;          /* m_n - m_p, MeV */
static const double kGA = 1.2754;             /* axial coupling */
static const double kMu = 1.66053906660e-24;  /* atomic mass unit, g */
static const double kPi = 3.14159265358979323846;

/* Occupation of a massless fermion 1/(1 + e^x) and 1 - of it, without cancellation. */
static void occupation(double x, double *f, double *omf)
{
    if (x > 0.0) {
        const double e = exp(-x);
        *f = e / (1.0 + e);
        *omf = 1.0 / (1.0 + e);
    } else {
        const double e = exp(x);
        *f = 1.0 / (1.0 + e);
        *omf = e / (1.0 + e);
    }
}

/* Rates of one zone (A1-A5): j0, chi0, j1, chi1 at [s][i], jac (may be NULL) at [s][i][4][3]. */
void vxo_abs_zone(int N, const double *eps, int S, const int *species, double g2, const double *st,
                  double *j0, double *chi0, double *j1, double *chi1, double *jac)
{
    const double T = st[0], eta = st[1], Ye = st[2], rho = st[3];
    const int bad = !(T > 0.0) || !isfinite(T) || !isfinite(eta) || !(Ye >= 0.0 && Ye <= 1.0) || !(rho >= 0.0) ||
                    !isfinite(rho);
    const double nb = rho / kMu * 1e-39;  /* baryons per fm^3 */
    const double nn = nb * (1.0 - Ye), np = nb * Ye;
    for (int s = 0; s < S; ++s) {
        for (int i = 0; i < N; ++i) {
            const size_t o = (size_t)s * N + i;
            double j = 0.0, chi = 0.0, d[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
            if (bad) {
                j = chi = NAN;
                for (int a = 0; a < 2; ++a)
                    for (int c = 0; c < 3; ++c) d[a][c] = NAN;
            } else if (species[s] == 0 || species[s] == 1) {
                const int anti = species[s] == 1;
                const double E = anti ? eps[i] - kQ : eps[i] + kQ;
                if (E > 0.0) {
                    const double K = g2 / kPi * (1.0 + 3.0 * kGA * kGA) * E * E;
                    const double nin = anti ? np : nn, nout = anti ? nn : np;
                    const double dnin = anti ? nb : -nb, dnout = anti ? -nb : nb; /* d/dY_e */
                    const double x = anti ? E / T + eta : E / T - eta;
                    double f, omf;
                    occupation(x, &f, &omf);
                    j = K * nout * f;
                    chi = K * nin * omf;
                    /* df/dx = -f (1 - f); dx/dT = -E/T^2, dx/deta = -1 (electron), +1 (positron) */
                    const double dfdx = -f * omf;
                    const double dxdT = -E / (T * T), dxde = anti ? 1.0 : -1.0;
                    d[0][0] = K * nout * dfdx * dxdT;
                    d[0][1] = K * nout * dfdx * dxde;
                    d[0][2] = K * dnout * f;
                    d[1][0] = -K * nin * dfdx * dxdT;
                    d[1][1] = -K * nin * dfdx * dxde;
                    d[1][2] = K * dnin * omf;
                }
            }
            j0[o] = j;
            chi0[o] = chi;
            j1[o] = bad ? NAN : 0.0;
            chi1[o] = bad ? NAN : 0.0;
            if (jac) {
                double *J = jac + o * 12;
                for (int q = 0; q < 12; ++q) J[q] = bad ? NAN : 0.0;
                for (int c = 0; c < 3; ++c) {
                    J[0 * 3 + c] = d[0][c];
                    J[1 * 3 + c] = d[1][c];
                }
            }
        }
    }
}

/* All zones: state [Z][4], outputs [Z][S][N], jac [Z][S][N][4][3] or NULL. */
void vxo_abs_eval(int N, const double *eps, int S, const int *species, double g2, long long Z, const double *state,
                  double *j0, double *chi0, double *j1, double *chi1, double *jac)
{
    const size_t zs = (size_t)S * N;
    for (long long z = 0; z < Z; ++z)
        vxo_abs_zone(N, eps, S, species, g2, state + 4 * z, j0 + z * zs, chi0 + z * zs, j1 + z * zs, chi1 + z * zs,
                     jac ? jac + z * zs * 12 : NULL);
}
