/*
 * vx_nes_oracle.c -- plain, slow FP64 CPU oracle for inelastic neutrino-electron scattering (NES)
 * and for the electron-gas closure eta_e(rho, Y_e, T).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or loads this file; only
 * the tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no code, header,
 * table or constant with the GPU path. It is compiled into the same test library as vx_oracle.c
 * and uses that file's Gauss-Legendre routine.
 *
 * What it computes. The paper (Marek et al., sec. 2.1) lists the neutrinos' emission, absorption
 * and SCATTERING rates among the components of the transport system and the equation of state as
 * a closure; it defines neither. The definitions below are the standard ones with massless
 * electrons; each choice the paper leaves open is marked READING.
 *
 * (1) NES kernel. nu(k) + e-(p) -> nu(k') + e-(p'), k = (eps, k), k' = (eps', k'), angle omega,
 *   y = 1 - cos(omega), q = k - k', q0 = eps - eps', Q = |q| = sqrt(eps^2 + eps'^2 - 2 eps eps' cos w).
 *   f(E) = 1/(exp(E/T - eta) + 1) is the electron occupation.
 *
 *   R^dir_X(eps, eps', y) = (G2/(eps eps')) Int d3p/(2E) Int d3p'/(2E') d4(k + p - k' - p') F_dir M_X
 *     M_I  = (k.p)(k'.p')      M_II = (k.p')(k'.p)                 (Minkowski products, +---)
 *     F_out = f(E) (1 - f(E'))  (neutrino scatters out of eps into eps')
 *     F_in  = (1 - f(E)) f(E')  (the inverse process: into eps from eps')
 *   Phi^dir_{l,X}(eps, eps') = Int_{-1}^{1} d(cos w) P_l(cos w) R^dir_X,   l = 0, 1.
 *
 *   Reduction: p' = p + q fixes cos(p, q) through E; what remains is an integral over
 *   E in [E_min, inf), E_min = (Q - q0)/2, with the azimuth of p about q averaged analytically:
 *     R^dir_X = (G2/(eps eps')) (2 pi/(4Q)) Int_{E_min}^inf dE F_dir(E, E + q0) <M_X>
 *     E c* = (E q0 - eps eps' y)/Q,  <a.p> = E a0 - (E c*)(a.q)/Q for a lightlike a,
 *     <(a.p)(b.p)> = <a.p><b.p> + (E^2 - (E c*)^2)/2 (a_perp . b_perp),
 *     k.q = eps (eps - eps' cos w), k'.q = eps' (eps cos w - eps'),
 *     k_perp = k'_perp (k' = k - q), |k_perp|^2 = eps^2 eps'^2 y (2 - y)/Q^2,
 *     k'.p' = k'.p + eps eps' y,  k.p' = k.p - eps eps' y   (k.k' = eps eps' y), so
 *     <M_I>  = <(k.p)(k'.p)> + eps eps' y <k.p>,   <M_II> = <(k.p)(k'.p)> - eps eps' y <k'.p>.
 *
 * Discrete rule in electron energy (READING: the workload text's "Gauss-Laguerre in electron
 *   energy", made accurate where the electrons are degenerate). With mu = eta T, the blocking
 *   factor F_out switches at the two Fermi edges e_lo = mu - max(q0, 0) and e_hi = mu + max(-q0, 0).
 *   Three panels of n_p = n_e/3 nodes each:
 *     P1: Gauss-Legendre on [a, b], b = max(E_min, e_lo), a = max(E_min, b - 30 T)
 *         (below a the factor is under e^-30 of its value at the edge: the tail is dropped);
 *     P2: Gauss-Legendre on [b, c], c = max(E_min, e_hi)  (between the edges);
 *     P3: Gauss-Laguerre on [c, inf) in x = (E - c)/T, weights w_k e^{x_k} T.
 *   Empty panels (a = b or b = c) contribute nothing. The same nodes serve F_in.
 *   READING (which ordered pairs are integrated): the kernel of a bin pair is integrated in the
 *   down-scattering order only, eps_i >= eps_j (from the point (eps_i, eps_j), both F_out and F_in);
 *   for eps_i < eps_j time reversal gives Phi^out(i,j) = Phi^in at the point (eps_j, eps_i) and
 *   Phi^in(i,j) = Phi^out at (eps_j, eps_i). The rule's nodes move with q0, so integrating both
 *   orders would break the exchange symmetry at the rule's accuracy (~1e-5 at n_p = 16); this way
 *   the discrete kernel obeys detailed balance and time reversal exactly.
 *   Against an adaptive quadrature of the integral the rule is within 1e-5 at n_p = 16 (T 0.5-30
 *   MeV, eta -5..60, eps 1-380 MeV), 1e-10 at n_p = 32 (pins in tests/test_nes_pins.py).
 *
 * Species (READING, as for the pair kernel): couplings beta_I = (CV + CA)^2, beta_II = (CV - CA)^2,
 *   nu_e: CV = 1/2 + 2 sin^2(theta_W), CA = 1/2; anti-nu_e: the two swap; nu_x: CV = -1/2 +
 *   2 sin^2(theta_W), CA = -1/2. Phi_s = beta_I Phi_I + beta_II Phi_II. Each species scatters
 *   within its own spectrum. READING: scattering on positrons is not included (it is the same
 *   kernel at -eta with the two terms swapped; it matters only where eta_e is near 0 or below).
 *
 * Contraction (READING: the same conventions as the pair kernel: R = sum_l (2l+1)/2 Phi_l P_l,
 *   f(mu') = J + 3 mu' H, and signs chosen so that the source of f(eps, mu) has the same form,
 *   df/dt = (1 - f)(j0 - mu j1) - f (chi0 + mu chi1)):
 *     j0(i)   =  2 pi C sum_j w_j Phi^in_0(i,j) J_j      chi0(i) =  2 pi C sum_j w_j Phi^out_0(i,j) (1 - J_j)
 *     j1(i)   = -6 pi C sum_j w_j Phi^in_1(i,j) H_j      chi1(i) = -6 pi C sum_j w_j Phi^out_1(i,j) H_j
 *   with J, H the species' own moments, w_j = eps_j^2 d(eps_j).
 *
 * Gradients: analytic derivatives with respect to T and eta at fixed nodes (the panels' nodes as
 *   placed for the zone) and spectra (READING: the rule's edges move with mu and T; the derivative
 *   returned is the rule applied to the integrand's derivative).
 *
 * (2) Electron-gas closure (READING: massless electrons and positrons in equilibrium, the only EOS
 *   content the kernels need). The net electron density of a massless Fermi gas is
 *     n_e- - n_e+ = (T/hbar c)^3 (F_2(eta) - F_2(-eta))/pi^2 = (T/hbar c)^3 (eta^3 + pi^2 eta)/(3 pi^2),
 *   and charge neutrality sets it to rho Y_e / m_u. eta follows from the depressed cubic
 *   eta^3 + pi^2 eta = 3 pi^2 rho Y_e (hbar c/T)^3 / m_u (one real root, Cardano's formula);
 *   its derivatives from implicit differentiation. hbar c = 197.3269804 MeV fm,
 *   m_u = 1.66053906660e-24 g.
 *
 * Arithmetic: FP64, loops in the order written, plain "+=", built with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NESO_PI 3.14159265358979323846
#define NESO_TAIL 30.0
#define NESO_MAXP 128

int vxo_gauss_legendre(int n, double *x, double *w);

/* ---------------------------------------------------------------------------------------- */
/* Laguerre polynomial L_n(x) and L_{n-1}(x) by the recurrence                              */
/* (k+1) L_{k+1} = (2k+1-x) L_k - k L_{k-1}.                                                  */
static void laguerre(int n, double x, double *ln, double *lnm1)
{
    double p0 = 1.0, p1 = 1.0 - x;
    if (n == 0) { *ln = 1.0; *lnm1 = 0.0; return; }
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0 - x) * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *ln = p1;
    *lnm1 = p0;
}

/* Gauss-Laguerre nodes (ascending) and weights for Int_0^inf e^{-x} g(x) dx: the roots of L_n are
 * bracketed on a grid that is dense near 0 (all lie in (0, 4n + 2)), bisected, then polished by
 * Newton; w_k = x_k / ((n + 1) L_{n+1}(x_k))^2. */
int vxo_gauss_laguerre(int n, double *x, double *w)
{
    if (n < 1 || n > 200 || !x || !w) return -1;
    const int M = 200000;
    const double top = 4.0 * n + 10.0;
    int found = 0;
    double xa = 0.0, la, tmp;
    laguerre(n, xa, &la, &tmp);
    for (int i = 1; i <= M && found < n; i++) {
        double r = (double)i / M;
        double xb = top * r * r;
        double lb;
        laguerre(n, xb, &lb, &tmp);
        if ((la < 0.0) != (lb < 0.0)) {
            double lo = xa, hi = xb, flo = la;
            for (int it = 0; it < 200; it++) {
                double mid = 0.5 * (lo + hi), fm;
                laguerre(n, mid, &fm, &tmp);
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; }
                else hi = mid;
                if (hi - lo <= 1e-15 * hi) break;
            }
            double z = 0.5 * (lo + hi);
            for (int it = 0; it < 3; it++) {  /* L_n' = n (L_n - L_{n-1}) / x */
                double ln, lm;
                laguerre(n, z, &ln, &lm);
                double d = n * (ln - lm) / z;
                if (d != 0.0) z -= ln / d;
            }
            x[found++] = z;
        }
        xa = xb;
        la = lb;
    }
    if (found != n) return -2;
    for (int k = 0; k < n; k++) {
        double l1, l0;
        laguerre(n + 1, x[k], &l1, &l0);
        w[k] = x[k] / ((n + 1.0) * (n + 1.0) * l1 * l1);
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
static double occ(double E, double T, double eta) { return 1.0 / (exp(E / T - eta) + 1.0); }
static double occ_c(double E, double T, double eta) { return 1.0 / (1.0 + exp(eta - E / T)); } /* 1 - f */

/* Azimuth-averaged <M_I>, <M_II> at electron energy E (definition above). */
static void nes_matrix(double eps, double epsp, double y, double E, double *mI, double *mII)
{
    double c = 1.0 - y, q0 = eps - epsp;
    double Q2 = eps * eps + epsp * epsp - 2.0 * eps * epsp * c, Q = sqrt(Q2);
    double kk = eps * epsp * y;
    double Ec = (E * q0 - kk) / Q;
    double kq = eps * (eps - epsp * c), kpq = epsp * (eps * c - epsp);
    double kp = E * eps - Ec * kq / Q;
    double kpp = E * epsp - Ec * kpq / Q;
    double kperp2 = eps * eps * epsp * epsp * y * (2.0 - y) / Q2;
    double prod = kp * kpp + 0.5 * (E * E - Ec * Ec) * kperp2;
    *mI = prod + kk * kp;
    *mII = prod - kk * kpp;
}

/* Nodes E_k and weights W_k (the dE measure included) of the three-panel rule for one
 * (eps, eps', y) and zone (T, eta): 3 n_p entries (empty panels get zero weights). */
void vxo_nes_nodes(double eps, double epsp, double y, double T, double eta, int n_p, const double *tg,
                   const double *wg, const double *xl, const double *wl, double *E, double *W)
{
    double c = 1.0 - y, q0 = eps - epsp;
    double Q = sqrt(eps * eps + epsp * epsp - 2.0 * eps * epsp * c);
    double Emin = 0.5 * (Q - q0);
    double mu = eta * T;
    double elo = mu - (q0 > 0.0 ? q0 : 0.0), ehi = mu + (q0 < 0.0 ? -q0 : 0.0);
    double cc = ehi > Emin ? ehi : Emin;
    double b = elo > Emin ? elo : Emin;
    double a = b - NESO_TAIL * T > Emin ? b - NESO_TAIL * T : Emin;
    for (int k = 0; k < n_p; k++) {
        E[k] = 0.5 * (a + b) + 0.5 * (b - a) * tg[k];
        W[k] = 0.5 * (b - a) * wg[k];
        E[n_p + k] = 0.5 * (b + cc) + 0.5 * (cc - b) * tg[k];
        W[n_p + k] = 0.5 * (cc - b) * wg[k];
        E[2 * n_p + k] = cc + T * xl[k];
        W[2 * n_p + k] = T * wl[k] * exp(xl[k]);
    }
}

/* Kernel at one point: K[dir][X] (dir 0 = in, 1 = out; X 0 = I, 1 = II) with G2 = 1; optional
 * dK[dir][X][v] (v: d/dT, d/deta) and Kabs[dir][X] (sum of |terms|). boltzmann != 0 replaces the
 * occupations by f = e^{eta - E/T}, 1 - f = 1 (no blocking: the non-degenerate limit). */
void vxo_nes_point(double eps, double epsp, double y, double T, double eta, int boltzmann, int n_p,
                   const double *tg, const double *wg, const double *xl, const double *wl, double *K,
                   double *dK, double *Kabs)
{
    double E[3 * NESO_MAXP], W[3 * NESO_MAXP];
    vxo_nes_nodes(eps, epsp, y, T, eta, n_p, tg, wg, xl, wl, E, W);
    double c = 1.0 - y, q0 = eps - epsp;
    double Q = sqrt(eps * eps + epsp * epsp - 2.0 * eps * epsp * c);
    double pref = (1.0 / (eps * epsp)) * 2.0 * NESO_PI / (4.0 * Q);
    double s[2][2] = {{0, 0}, {0, 0}}, ds[2][2][2], sa[2][2] = {{0, 0}, {0, 0}};
    memset(ds, 0, sizeof ds);
    for (int k = 0; k < 3 * n_p; k++) {
        if (W[k] == 0.0) continue;
        double Ek = E[k], Ep = Ek + q0;
        double mI, mII;
        nes_matrix(eps, epsp, y, Ek, &mI, &mII);
        double Fin, Fout, gin[2], gout[2];
        if (boltzmann) {
            Fout = exp(eta - Ek / T);
            Fin = exp(eta - Ep / T);
            gout[0] = Ek / (T * T); gout[1] = 1.0;
            gin[0] = Ep / (T * T); gin[1] = 1.0;
        } else {
            double fE = occ(Ek, T, eta), cE = occ_c(Ek, T, eta);
            double fP = occ(Ep, T, eta), cP = occ_c(Ep, T, eta);
            Fout = fE * cP;
            Fin = cE * fP;
            /* d ln F / dT at fixed eta, d ln F / d eta at fixed T */
            gout[0] = (cE * Ek - fP * Ep) / (T * T);
            gout[1] = cE - fP;
            gin[0] = (-fE * Ek + cP * Ep) / (T * T);
            gin[1] = -fE + cP;
        }
        double F[2] = {Fin, Fout}, m[2] = {mI, mII};
        for (int d = 0; d < 2; d++)
            for (int x = 0; x < 2; x++) {
                double t = W[k] * F[d] * m[x];
                s[d][x] += t;
                sa[d][x] += fabs(t);
                if (dK) {
                    double *g = d ? gout : gin;
                    ds[d][x][0] += t * g[0];
                    ds[d][x][1] += t * g[1];
                }
            }
    }
    for (int d = 0; d < 2; d++)
        for (int x = 0; x < 2; x++) {
            K[2 * d + x] = pref * s[d][x];
            if (Kabs) Kabs[2 * d + x] = pref * sa[d][x];
            if (dK) {
                dK[4 * d + 2 * x + 0] = pref * ds[d][x][0];
                dK[4 * d + 2 * x + 1] = pref * ds[d][x][1];
            }
        }
}

static void nes_betas(int species, double sin2w, double *bI, double *bII)
{
    double cv, ca;
    if (species == 2) { cv = -0.5 + 2.0 * sin2w; ca = -0.5; }
    else { cv = 0.5 + 2.0 * sin2w; ca = 0.5; }
    double b1 = (cv + ca) * (cv + ca), b2 = (cv - ca) * (cv - ca);
    if (species == 1) { double t = b1; b1 = b2; b2 = t; }
    *bI = b1;
    *bII = b2;
}

static void nes_weights(int n, const double *eps, double *w)
{
    for (int i = 0; i < n; i++) {
        double lo = i ? sqrt(eps[i - 1] * eps[i]) : eps[0] / sqrt(eps[1] / eps[0]);
        double hi = i < n - 1 ? sqrt(eps[i] * eps[i + 1]) : eps[n - 1] * sqrt(eps[n - 1] / eps[n - 2]);
        w[i] = eps[i] * eps[i] * (hi - lo);
    }
}

/* Phi^dir_{l,X}(i,j) of one zone (G2 applied): phi[X][dir][l][i][j]; optional dphi[..][v] and
 * |P_l|-weighted magnitudes pabs (same layout as phi). */
void vxo_nes_phi_zone(int n, const double *eps, int n_mu, const double *tmu, const double *wmu, int n_p,
                      const double *tg, const double *wg, const double *xl, const double *wl, double g2, double T,
                      double eta, double *phi, double *dphi, double *pabs, double *dabs)
{
    int N2 = n * n;
    memset(phi, 0, sizeof(double) * 8 * N2);
    if (dphi) memset(dphi, 0, sizeof(double) * 16 * N2);
    if (pabs) memset(pabs, 0, sizeof(double) * 8 * N2);
    if (dabs) memset(dabs, 0, sizeof(double) * 16 * N2);
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            /* down-scattering order: the point (eps_hi, eps_lo); for i < j the directions swap */
            const int rev = i < j;
            const double ea = rev ? eps[j] : eps[i], eb = rev ? eps[i] : eps[j];
            for (int m = 0; m < n_mu; m++) {
                double t = tmu[m], y = 1.0 - t;
                double K[4], dK[8], Ka[4];
                vxo_nes_point(ea, eb, y, T, eta, 0, n_p, tg, wg, xl, wl, K, (dphi || dabs) ? dK : NULL, Ka);
                for (int x = 0; x < 2; x++)
                    for (int d = 0; d < 2; d++)
                        for (int l = 0; l < 2; l++) {
                            const int dp = rev ? 1 - d : d;  /* direction of the point's kernel used */
                            double P = l ? t : 1.0;
                            int o = (((x * 2 + d) * 2 + l) * n + i) * n + j;
                            phi[o] += g2 * wmu[m] * P * K[2 * dp + x];
                            if (pabs) pabs[o] += g2 * wmu[m] * fabs(P) * Ka[2 * dp + x];
                            for (int v = 0; v < 2; v++) {
                                double dv = g2 * wmu[m] * P * dK[4 * dp + 2 * x + v];
                                if (dphi) dphi[2 * o + v] += dv;
                                if (dabs) dabs[2 * o + v] += fabs(dv);
                            }
                        }
            }
        }
}

/* Rates of Z zones (definition above): out arrays [Z][S][N] (j0, chi0, j1, chi1); optional phi dump
 * [Z][2 X][2 dir][2 l][N][N] (G2 applied), Jacobian jac [Z][S][N][4][3] (d/dT, d/deta, d/dY_e = 0),
 * magnitudes (sums of |terms|) j1_abs, chi1_abs, phi_abs, jac_abs. Returns the thread count. */
int vxo_nes_eval(int n, const double *eps, const double *weights, int n_mu, int n_e, int S, const int *species,
                 double sin2w, double g2, double norm, long Z, const double *state, const double *J, const double *H,
                 double *j0, double *chi0, double *j1, double *chi1, double *phi_out, double *jac,
                 double *j1_abs, double *chi1_abs, double *phi_abs, double *jac_abs, int threads)
{
    if (n < 2 || n > 64 || n_mu < 1 || n_e < 3 || n_e % 3 || n_e / 3 > NESO_MAXP || S < 1 || S > 3) return -1;
    int n_p = n_e / 3;
    double *tmu = malloc(sizeof(double) * n_mu), *wmu = malloc(sizeof(double) * n_mu);
    double tg[NESO_MAXP], wg[NESO_MAXP], xl[NESO_MAXP], wl[NESO_MAXP];
    double w[64];
    vxo_gauss_legendre(n_mu, tmu, wmu);
    vxo_gauss_legendre(n_p, tg, wg);
    if (vxo_gauss_laguerre(n_p, xl, wl) != 0) { free(tmu); free(wmu); return -2; }
    if (weights) memcpy(w, weights, sizeof(double) * n);
    else nes_weights(n, eps, w);
    int N2 = n * n, used = 1;
    const int need_d = jac != NULL || jac_abs != NULL;
    const int need_a = j1_abs || chi1_abs || phi_abs || jac_abs;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long z = 0; z < Z; z++) {
        double T = state[4 * z + 0], eta = state[4 * z + 1];
        double *phi = malloc(sizeof(double) * 8 * N2), *pa = malloc(sizeof(double) * 8 * N2);
        double *dphi = need_d ? malloc(sizeof(double) * 16 * N2) : NULL;
        double *da = need_d ? malloc(sizeof(double) * 16 * N2) : NULL;
        vxo_nes_phi_zone(n, eps, n_mu, tmu, wmu, n_p, tg, wg, xl, wl, g2, T, eta, phi, dphi, need_a ? pa : NULL,
                         need_d ? da : NULL);
        if (phi_out) memcpy(phi_out + (size_t)z * 8 * N2, phi, sizeof(double) * 8 * N2);
        if (phi_abs) memcpy(phi_abs + (size_t)z * 8 * N2, pa, sizeof(double) * 8 * N2);
        for (int s = 0; s < S; s++) {
            double bI, bII;
            nes_betas(species[s], sin2w, &bI, &bII);
            for (int i = 0; i < n; i++) {
                double r[4] = {0, 0, 0, 0}, ra[4] = {0, 0, 0, 0}, dr[4][2], dra[4][2];
                memset(dr, 0, sizeof dr);
                memset(dra, 0, sizeof dra);
                for (int j = 0; j < n; j++) {
                    size_t sp = ((size_t)z * S + s) * n + j;
                    /* output o: 0 j0 (in, l 0, J), 1 chi0 (out, l 0, 1 - J), 2 j1 (in, l 1, H), 3 chi1 (out, l 1, H) */
                    for (int o = 0; o < 4; o++) {
                        int d = (o == 0 || o == 2) ? 0 : 1, l = o >> 1;
                        double v = o == 0 ? J[sp] : o == 1 ? 1.0 - J[sp] : H[sp];
                        double c = (l ? -6.0 : 2.0) * NESO_PI * norm * w[j] * v;
                        int oI = ((0 * 2 + d) * 2 + l) * N2 + i * n + j, oII = ((1 * 2 + d) * 2 + l) * N2 + i * n + j;
                        double k = bI * phi[oI] + bII * phi[oII];
                        r[o] += c * k;
                        if (need_a) ra[o] += fabs(c) * (bI * pa[oI] + bII * pa[oII]);
                        if (need_d)
                            for (int v2 = 0; v2 < 2; v2++) {
                                dr[o][v2] += c * (bI * dphi[2 * oI + v2] + bII * dphi[2 * oII + v2]);
                                dra[o][v2] += fabs(c) * (bI * da[2 * oI + v2] + bII * da[2 * oII + v2]);
                            }
                    }
                }
                size_t oi = ((size_t)z * S + s) * n + i;
                j0[oi] = r[0]; chi0[oi] = r[1]; j1[oi] = r[2]; chi1[oi] = r[3];
                if (j1_abs) j1_abs[oi] = ra[2];
                if (chi1_abs) chi1_abs[oi] = ra[3];
                for (int o = 0; o < 4; o++) {
                    if (jac) {
                        jac[oi * 12 + o * 3 + 0] = dr[o][0];
                        jac[oi * 12 + o * 3 + 1] = dr[o][1];
                        jac[oi * 12 + o * 3 + 2] = 0.0;
                    }
                    if (jac_abs) {
                        jac_abs[oi * 12 + o * 3 + 0] = dra[o][0];
                        jac_abs[oi * 12 + o * 3 + 1] = dra[o][1];
                        jac_abs[oi * 12 + o * 3 + 2] = 0.0;
                    }
                }
            }
        }
        free(phi); free(pa); free(dphi); free(da);
    }
    free(tmu);
    free(wmu);
    return used;
}

/* ---------------------------------------------------------------------------------------- */
/* Electron-gas closure: eta_e of every zone from (T, Y_e, rho) in state [Z][4] (T, -, Y_e, rho);
 * eta[z] and, if deta != NULL, deta[z][3] = d eta / d(T, Y_e, rho). Cardano's formula for the
 * one real root of eta^3 + p eta - q = 0, p = pi^2, q = 3 pi^2 n (hbar c / T)^3, n = rho Y_e/m_u. */
#define NESO_HBARC_MEV_CM 1.973269804e-11
#define NESO_MU_G 1.66053906660e-24
void vxo_eos_eta(long Z, const double *state, double *eta, double *deta)
{
    for (long z = 0; z < Z; z++) {
        double T = state[4 * z + 0], ye = state[4 * z + 2], rho = state[4 * z + 3];
        double n = rho * ye / NESO_MU_G;
        double r = NESO_HBARC_MEV_CM / T;
        double p = NESO_PI * NESO_PI, q = 3.0 * p * n * r * r * r;
        double disc = sqrt(q * q / 4.0 + p * p * p / 27.0);
        /* Cardano: e = cbrt(q/2 + disc) + cbrt(q/2 - disc); the two cube roots multiply to -p/3,
         * so the second is written -p/(3 A), which does not cancel when q is large */
        double A = cbrt(q / 2.0 + disc);
        double e = A - p / (3.0 * A);
        eta[z] = e;
        if (deta) {
            double dedq = 1.0 / (3.0 * e * e + p);
            deta[3 * z + 0] = dedq * (-3.0 * q / T);
            deta[3 * z + 1] = dedq * (q / ye);
            deta[3 * z + 2] = dedq * (q / rho);
        }
    }
}
