/*
 * vx_oracle.c -- plain, slow FP64 CPU oracle for the e+e- pair-process rate kernel.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library calls, links or loads this file;
 * only the tests, the smoke check and the benchmark's CPU-baseline leg do. It shares no code,
 * header, table or constant with the GPU path.
 *
 * What it computes. The paper (Marek et al., "Towards Petaflops Capability of the VERTEX
 * Supernova Code", sec. 2.1) counts the neutrinos' emission, absorption and scattering rates
 * among the components of the PDE system and uses the neutrino occupation f, the intensity
 * I = c/(2 pi hbar c)^3 eps^3 f, and the angular moments J, H of I (the one numbered equation of
 * sec. 2.1). It does not define the rate kernels. The definition below is the standard
 * electroweak e- e+ <-> nu nubar kernel with massless leptons and Fermi-Dirac blocking; each
 * choice the paper leaves open is marked READING.
 *
 *   nu momentum k = (eps, k), nubar momentum k' = (eps', k'), angle omega between them,
 *   y = 1 - cos(omega), Q = k + k', q0 = eps + eps', s = Q.Q = 2 eps eps' y, |q|^2 = q0^2 - s.
 *   Electron (E, p), positron (Ebar, pbar), f_e(E) = 1/(exp(E/T - eta) + 1),
 *   f_ebar(Ebar) = 1/(exp(Ebar/T + eta) + 1), eta = electron degeneracy mu_e/T.
 *
 *   K^X_dir(eps, eps', y) = (G2/(eps eps')) Int d3p/(2E) Int d3pbar/(2Ebar) d4(p + pbar - Q) O_dir M_X
 *     M_I  = (p.k')(pbar.k)     M_II = (p.k)(pbar.k')           (Minkowski products, +---)
 *     O_p  = f_e f_ebar (production)   O_a = (1 - f_e)(1 - f_ebar) (annihilation)
 *   Phi^dir_{l,X}(eps, eps') = Int_{-1}^{1} d(cos w) P_l(cos w) K^X_dir,   l = 0, 1.
 *
 *   The delta function fixes pbar = Q - p and cos(p, q) through E, leaving an integral over
 *   E in [E-, E+], E+- = (q0 +- |q|)/2, with the azimuth of p about q averaged analytically:
 *     K^X = (G2/(eps eps')) Int dE O_dir(E, q0 - E) (2 pi / (4|q|)) [<p.a>(Q.b) - <(p.a)(p.b)>]
 *     (a, b) = (k', k) for I and (k, k') for II;  Q.k = Q.k' = s/2;
 *     E c* = (2 q0 E - s)/(2|q|);  <p.a> = E a0 - (E c*)(a.q)/|q|;
 *     <(p.a)(p.b)> = <p.a><p.b> + (E^2 - (E c*)^2)/2 (a_perp . b_perp);
 *     k.q = eps (q0 - eps' y), k'.q = eps' (q0 - eps y),
 *     |k_perp|^2 = |k'_perp|^2 = -k_perp.k'_perp = eps^2 eps'^2 y (2 - y)/|q|^2.
 *
 * Discrete rule (what both GPU forms must reproduce):
 *   Gauss-Legendre in cos(omega) (n_mu nodes t_m, y_m = 1 - t_m) and Gauss-Legendre on the
 *   finite electron-energy interval [E-, E+] (n_e nodes). READING: the workload text says
 *   "Gauss-Laguerre in electron energy", but for fixed (eps, eps', omega) the electron energy
 *   lives on a finite interval where a Laguerre rule does not apply.
 *   O_p and O_a are evaluated independently, each from its own formula.
 *   Split rule (the E-panel variant, an alternative discrete rule): in zones with |eta| above a
 *   threshold eta_split, where the Fermi edge of the degenerate lepton lies inside (E-, E+), two
 *   Gauss-Legendre panels of n_e/2 nodes meet at it (vxo_kernel_point_split); elsewhere the
 *   standard rule. READING: the edge is the electron's, E = mu_e, for eta >= 0 and the
 *   positron's, Ebar = -mu_e, for eta < 0 (the two cases are mirror images). The threshold
 *   (default 20, the GPU's precision switch) keeps the standard rule in cold, mildly degenerate
 *   zones, where half the nodes on a panel that spans ~100 T of Boltzmann tail do worse.
 *
 * Species (READING): nu_e uses couplings beta_I = (CV + CA)^2, beta_II = (CV - CA)^2 with
 * CV = 1/2 + 2 sin^2(theta_W), CA = 1/2 and partner spectrum anti-nu_e; anti-nu_e uses the
 * transposed kernel Phi(eps', eps) (beta_I and beta_II swap) with partner nu_e; nu_x uses
 * CV = -1/2 + 2 sin^2(theta_W), CA = -1/2 with its own spectrum as partner (no flavour factor).
 *
 * Contraction (READING of the moment equation of sec. 2.1 with f(mu') = J + 3 mu' H and the
 * Legendre convention R = sum_l (2l+1)/2 Phi_l P_l):
 *   j0(i)  = 2 pi C sum_j w_j Phi^p_0(i,j) (1 - Jbar_j)     chi0(i) = 2 pi C sum_j w_j Phi^a_0 Jbar_j
 *   j1(i)  = 6 pi C sum_j w_j Phi^p_1(i,j) Hbar_j           chi1(i) = 6 pi C sum_j w_j Phi^a_1 Hbar_j
 *   so that df/dt = (1 - f)(j0 - mu j1) - f (chi0 + mu chi1); w_j = eps_j^2 d(eps_j) and C is the
 *   phase-space constant c/(2 pi hbar c)^3 of sec. 2.1 (a parameter, default 1).
 *
 * Gradients: analytic derivatives of the above with respect to T and eta at fixed nodes and
 * spectra; the Y_e and rho derivatives are identically zero for this process.
 *
 * Arithmetic: FP64, loops in the order written, plain "+=", built with -ffp-contract=off.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define VXO_PI 3.14159265358979323846

#define VXO_MAX_HALF 512 /* largest panel rule of the split form */

/* ---------------------------------------------------------------------------------------- */
/* Gauss-Legendre nodes (ascending) and weights on [-1, 1]: Newton iteration on P_n, using the */
/* three-term recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1} and                          */
/* P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1); weight 2 / ((1 - x^2) P_n'(x)^2).               */
int vxo_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || !x || !w) return -1;
    for (int i = 0; i < (n + 1) / 2; i++) {
        double z = cos(VXO_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; k++) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute the derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; k++) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = wi;
        w[n - 1 - i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
    return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Energy-bin weights w_i = eps_i^2 d(eps_i). READING: bin edges at the geometric midpoints   */
/* of neighbouring centres, the two outer edges half a logarithmic step beyond the end centres. */
int vxo_energy_weights(int n, const double *eps, double *w)
{
    if (n < 2 || !eps || !w) return -1;
    for (int i = 0; i < n; i++) {
        double lo, hi;
        if (i == 0) lo = eps[0] / sqrt(eps[1] / eps[0]);
        else lo = sqrt(eps[i - 1] * eps[i]);
        if (i == n - 1) hi = eps[n - 1] * sqrt(eps[n - 1] / eps[n - 2]);
        else hi = sqrt(eps[i] * eps[i + 1]);
        w[i] = eps[i] * eps[i] * (hi - lo);
    }
    return 0;
}

/* Couplings beta_I, beta_II of one species (READING above). */
static void species_betas(int species, double sin2w, double *bI, double *bII)
{
    double cv, ca;
    if (species == 2) { cv = -0.5 + 2.0 * sin2w; ca = -0.5; }
    else { cv = 0.5 + 2.0 * sin2w; ca = 0.5; }
    double b1 = (cv + ca) * (cv + ca), b2 = (cv - ca) * (cv - ca);
    if (species == 1) { *bI = b2; *bII = b1; } /* anti-nu_e: transposed kernel */
    else { *bI = b1; *bII = b2; }
}

/* ---------------------------------------------------------------------------------------- */
/* The kernel at one point (eps, eps', y): K^X_dir and, if dK != NULL, its T and eta           */
/* derivatives. Output layout K[dir][X] with dir 0 = production, 1 = annihilation and          */
/* X 0 = I, 1 = II; dK[dir][X][0] = d/dT, dK[dir][X][1] = d/deta.  G2 = 1 here.               */
/* occ selects the statistics: 0 = Fermi-Dirac (the kernel); 1 = Boltzmann limit (O_p =        */
/* exp(-q0/T), O_a = 1), used only to check the kinematics against the closed form.           */
/* Kinematics of one point (eps, eps', y) and the electron-energy sums of one kernel point. */
typedef struct {
    double eps, epsp, q0, s, q, Ep, Em, kq, kpq, perp, Qk;
} kin_t;

typedef struct {
    double sum[2][2], dsum[2][2][2], dabs[2][2][2];
} acc_t;

static void kin_init(double eps, double epsp, double y, kin_t *k)
{
    k->eps = eps;
    k->epsp = epsp;
    k->q0 = eps + epsp;
    k->s = 2.0 * eps * epsp * y;
    k->q = sqrt(k->q0 * k->q0 - k->s);
    k->Ep = 0.5 * (k->q0 + k->q);
    k->Em = k->s / (2.0 * (k->q0 + k->q));
    k->kq = eps * (k->q0 - epsp * y);    /* k . q  */
    k->kpq = epsp * (k->q0 - eps * y);   /* k' . q */
    k->perp = eps * eps * epsp * epsp * y * (2.0 - y) / (k->q * k->q); /* |k_perp|^2 */
    k->Qk = 0.5 * k->s;                  /* Q.k = Q.k' */
}

/* Adds one electron-energy node E with quadrature weight W (dE measure) to the sums. */
static void node_add(const kin_t *k, double E, double W, double T, double eta, int occ, int want_d,
                     int want_abs, acc_t *a)
{
    double Eb = k->q0 - E;
    double xe = E / T - eta;
    double xp = Eb / T + eta;
    double Op = 1.0 / ((exp(xe) + 1.0) * (exp(xp) + 1.0));
    double Oa = 1.0 / ((1.0 + exp(-xe)) * (1.0 + exp(-xp)));
    if (occ == 1) { Op = exp(-k->q0 / T); Oa = 1.0; }
    double Ec = (2.0 * k->q0 * E - k->s) / (2.0 * k->q);
    double pk = E * k->eps - Ec * k->kq / k->q;     /* <p.k>  */
    double pkp = E * k->epsp - Ec * k->kpq / k->q;  /* <p.k'> */
    double half_sin2 = 0.5 * (E * E - Ec * Ec);
    /* (a,b) = (k',k): <p.k'>(Q.k) - [<p.k'><p.k> + (E^2 - Ec^2)/2 (k'_perp.k_perp)] */
    double MI = pkp * k->Qk - (pkp * pk - half_sin2 * k->perp);
    /* (a,b) = (k,k'): <p.k>(Q.k') - [<p.k><p.k'> + (E^2 - Ec^2)/2 (k_perp.k'_perp)] */
    double MII = pk * k->Qk - (pk * pkp - half_sin2 * k->perp);
    a->sum[0][0] += W * Op * MI;
    a->sum[0][1] += W * Op * MII;
    a->sum[1][0] += W * Oa * MI;
    a->sum[1][1] += W * Oa * MII;
    if (want_d) {
        double fe = 1.0 / (exp(xe) + 1.0);   /* electron occupation   */
        double fp = 1.0 / (exp(xp) + 1.0);   /* positron occupation   */
        /* dO_p/dT = O_p [(1-f_e) E + (1-f_ebar) Ebar]/T^2,  dO_p/deta = O_p (f_ebar - f_e) */
        double dOpT = Op * ((1.0 - fe) * E + (1.0 - fp) * Eb) / (T * T);
        double dOpe = Op * (fp - fe);
        /* dO_a/dT = -O_a [f_e E + f_ebar Ebar]/T^2,      dO_a/deta = O_a (f_ebar - f_e) */
        double dOaT = -Oa * (fe * E + fp * Eb) / (T * T);
        double dOae = Oa * (fp - fe);
        a->dsum[0][0][0] += W * dOpT * MI;  a->dsum[0][0][1] += W * dOpe * MI;
        a->dsum[0][1][0] += W * dOpT * MII; a->dsum[0][1][1] += W * dOpe * MII;
        a->dsum[1][0][0] += W * dOaT * MI;  a->dsum[1][0][1] += W * dOae * MI;
        a->dsum[1][1][0] += W * dOaT * MII; a->dsum[1][1][1] += W * dOae * MII;
        if (want_abs) { /* the same sums of absolute values: the rounding bound of each derivative */
            a->dabs[0][0][0] += W * fabs(dOpT * MI);  a->dabs[0][0][1] += W * fabs(dOpe * MI);
            a->dabs[0][1][0] += W * fabs(dOpT * MII); a->dabs[0][1][1] += W * fabs(dOpe * MII);
            a->dabs[1][0][0] += W * fabs(dOaT * MI);  a->dabs[1][0][1] += W * fabs(dOae * MI);
            a->dabs[1][1][0] += W * fabs(dOaT * MII); a->dabs[1][1][1] += W * fabs(dOae * MII);
        }
    }
}

static void kernel_finish(const kin_t *k, const acc_t *a, double *K, double *dK, double *dKabs)
{
    double pref = 2.0 * VXO_PI / (4.0 * k->q * k->eps * k->epsp);
    for (int d = 0; d < 2; d++)
        for (int X = 0; X < 2; X++) {
            K[2 * d + X] = pref * a->sum[d][X];
            if (dK) {
                dK[(2 * d + X) * 2 + 0] = pref * a->dsum[d][X][0];
                dK[(2 * d + X) * 2 + 1] = pref * a->dsum[d][X][1];
            }
            if (dKabs) {
                dKabs[(2 * d + X) * 2 + 0] = pref * a->dabs[d][X][0];
                dKabs[(2 * d + X) * 2 + 1] = pref * a->dabs[d][X][1];
            }
        }
}

void vxo_kernel_point(double eps, double epsp, double y, double T, double eta, int occ,
                      int n_e, const double *tE, const double *wE, double *K, double *dK,
                      double *dKabs)
{
    kin_t k;
    acc_t a;
    memset(&a, 0, sizeof a);
    kin_init(eps, epsp, y, &k);
    for (int i = 0; i < n_e; i++) {
        double E = 0.5 * (k.Ep + k.Em) + 0.5 * (k.Ep - k.Em) * tE[i];
        double W = 0.5 * (k.Ep - k.Em) * wE[i];
        node_add(&k, E, W, T, eta, occ, dK != NULL, dKabs != NULL, &a);
    }
    kernel_finish(&k, &a, K, dK, dKabs);
}

/* The split rule (E-panel variant): if the Fermi edge of the degenerate lepton, E_s = mu_e for  */
/* eta >= 0 (electron) and E_s = q0 + mu_e for eta < 0 (the positron's edge Ebar = -mu_e), lies */
/* strictly inside (E-, E+), the interval is split there into two Gauss-Legendre panels, each    */
/* with the n_h-node rule (tH, wH); otherwise the standard n_e-node rule (tE, wE) is used.       */
void vxo_kernel_point_split(double eps, double epsp, double y, double T, double eta, int occ,
                            int n_e, const double *tE, const double *wE, int n_h, const double *tH,
                            const double *wH, double *K, double *dK, double *dKabs)
{
    kin_t k;
    kin_init(eps, epsp, y, &k);
    double Es = eta >= 0.0 ? eta * T : k.q0 + eta * T;
    if (!(k.Em < Es && Es < k.Ep)) {
        vxo_kernel_point(eps, epsp, y, T, eta, occ, n_e, tE, wE, K, dK, dKabs);
        return;
    }
    acc_t a;
    memset(&a, 0, sizeof a);
    double hA = 0.5 * (Es - k.Em), hB = 0.5 * (k.Ep - Es);
    for (int i = 0; i < n_h; i++) {
        node_add(&k, Es - hA * (1.0 - tH[i]), hA * wH[i], T, eta, occ, dK != NULL, dKabs != NULL, &a);
        node_add(&k, Es + hB * (1.0 + tH[i]), hB * wH[i], T, eta, occ, dK != NULL, dKabs != NULL, &a);
    }
    kernel_finish(&k, &a, K, dK, dKabs);
}

/* ---------------------------------------------------------------------------------------- */
/* Phi^dir_{l,X}(i,j) of one zone for all ordered bin pairs (i = nu bin, j = nubar bin).       */
/* phi layout [dir][X][l][i][j]; dphi (optional) [dir][X][l][i][j][2] with d/dT, d/deta.        */
/* phiabs (optional): the same sums with |P_l|, i.e. the magnitude that bounds the rounding of   */
/* the l = 1 projection (whose terms change sign with cos(omega)); equal to phi for l = 0.       */
void vxo_phi_zone(int n, const double *eps, int n_mu, const double *tmu, const double *wmu,
                  int n_e, const double *tE, const double *wE, double g2, double T, double eta,
                  int occ, int split, double eta_split, double *phi, double *dphi, double *phiabs,
                  double *dphiabs)
{
    size_t NN = (size_t)n * n;
    int n_h = n_e / 2;
    double tH[VXO_MAX_HALF], wH[VXO_MAX_HALF];
    split = split && fabs(eta) > eta_split;
    if (split) vxo_gauss_legendre(n_h, tH, wH);
    memset(phi, 0, 8 * NN * sizeof(double));
    if (phiabs) memset(phiabs, 0, 8 * NN * sizeof(double));
    if (dphiabs) memset(dphiabs, 0, 16 * NN * sizeof(double));
    if (dphi) memset(dphi, 0, 16 * NN * sizeof(double));
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int m = 0; m < n_mu; m++) {
                double y = 1.0 - tmu[m];
                double K[4], dK[8], dKa[8];
                if (split)
                    vxo_kernel_point_split(eps[i], eps[j], y, T, eta, occ, n_e, tE, wE, n_h, tH, wH, K,
                                           dphi ? dK : NULL, dphiabs ? dKa : NULL);
                else
                    vxo_kernel_point(eps[i], eps[j], y, T, eta, occ, n_e, tE, wE, K, dphi ? dK : NULL,
                                     dphiabs ? dKa : NULL);
                for (int d = 0; d < 2; d++)
                    for (int X = 0; X < 2; X++)
                        for (int l = 0; l < 2; l++) {
                            double Pl = (l == 0) ? 1.0 : tmu[m];
                            size_t o = (((size_t)(d * 2 + X) * 2 + l) * n + i) * n + j;
                            phi[o] += wmu[m] * Pl * g2 * K[2 * d + X];
                            if (phiabs) phiabs[o] += wmu[m] * fabs(Pl) * g2 * K[2 * d + X];
                            if (dphi) {
                                dphi[2 * o + 0] += wmu[m] * Pl * g2 * dK[(2 * d + X) * 2 + 0];
                                dphi[2 * o + 1] += wmu[m] * Pl * g2 * dK[(2 * d + X) * 2 + 1];
                            }
                            if (dphiabs) {
                                dphiabs[2 * o + 0] += wmu[m] * fabs(Pl) * g2 * dKa[(2 * d + X) * 2 + 0];
                                dphiabs[2 * o + 1] += wmu[m] * fabs(Pl) * g2 * dKa[(2 * d + X) * 2 + 1];
                            }
                        }
            }
}

/* phi[dir][X][l][i][j] and dphi[dir][X][l][i][j][v] of one zone, ij = i*N + j */
#define PHI(a, d, X, l, ij) (a)[(((size_t)(d) * 2 + (X)) * 2 + (l)) * NN + (ij)]
#define DPHI(a, d, X, l, ij, v) (a)[2 * ((((size_t)(d) * 2 + (X)) * 2 + (l)) * NN + (ij)) + (v)]

/* Index (within the species list) of the spectrum a species' kernel is contracted with:
 * nu_e <-> anti-nu_e, nu_x with itself; -1 if it is not in the list. */
static int partner_index(int S, const int *species, int si)
{
    int sp = species[si];
    int want = (sp == 0) ? 1 : (sp == 1) ? 0 : 2;
    for (int k = 0; k < S; k++)
        if (species[k] == want) return k;
    return -1;
}

/* ---------------------------------------------------------------------------------------- */
/* Full evaluation over Z zones (OpenMP over zones: the paper's ray-to-thread mapping,        */
/* sec. 2.2). Arrays: state [Z][4] = (T, eta, Y_e, rho); J, H, j0, chi0, j1, chi1 [Z][S][N].   */
/* weights: NULL -> vxo_energy_weights. phi_out: NULL or [Z][2 dir][2 l][N][N] for K^I.       */
/* jac: NULL or [Z][S][N][4 outputs j0,chi0,j1,chi1][3 inputs T,eta,Y_e].                      */
/* j1abs, chi1abs [Z][S][N], phiabs_out [Z][2][2][N][N] (optional): the same results with every   */
/* term replaced by its absolute value (|P_l|, |H|), which bound the rounding of a sum whose      */
/* terms cancel; for the l = 0 outputs the terms never change sign. jacabs, like jac: the same    */
/* for the derivatives, whose node terms can change sign as well.                                 */
/* dsrc: NULL or [Z][S][4][N][N], the derivatives of the rates with respect to the partner       */
/* spectrum they are contracted with (the rates are affine in J and linear in H):                */
/*   [z][s][0][i][j] = d j0[z][s][i] / d J[z][p(s)][j],   [1] = d chi0 / d J,                    */
/*   [2] = d j1 / d H[z][p(s)][j],   [3] = d chi1 / d H,   p(s) = the partner species' index.    */
/* dsrcabs (like dsrc): the same with |P_l| in the omega sum (equal to |dsrc| for l = 0).        */
/* split: 0 = the standard discrete rule, 1 = the split rule (vxo_kernel_point_split; n_e even) */
/* in zones with |eta| > eta_split.                                                              */
/* Returns the number of threads used (>= 1), or -1 on a bad argument.                         */
int vxo_eval(int n, const double *eps, const double *weights, int n_mu, int n_e,
             int n_species, const int *species, double sin2w, double g2, double norm,
             long Z, const double *state, const double *J, const double *H,
             double *j0, double *chi0, double *j1, double *chi1, double *phi_out, double *jac,
             double *j1abs, double *chi1abs, double *phiabs_out, double *jacabs, double *dsrc,
             double *dsrcabs, int split, double eta_split, int n_threads)
{
    if (n < 2 || n_mu < 1 || n_e < 1 || n_species < 1 || Z < 0 || !eps || !species) return -1;
    if (split && (n_e % 2 != 0 || n_e / 2 > VXO_MAX_HALF)) return -1;
    for (int k = 0; k < n_species; k++)
        if (species[k] < 0 || species[k] > 2 || partner_index(n_species, species, k) < 0) return -1;
    double *w = (double *)malloc(n * sizeof(double));
    double *tmu = (double *)malloc(n_mu * sizeof(double)), *wmu = (double *)malloc(n_mu * sizeof(double));
    double *tE = (double *)malloc(n_e * sizeof(double)), *wE = (double *)malloc(n_e * sizeof(double));
    if (weights) memcpy(w, weights, n * sizeof(double));
    else vxo_energy_weights(n, eps, w);
    vxo_gauss_legendre(n_mu, tmu, wmu);
    vxo_gauss_legendre(n_e, tE, wE);
    int S = n_species, N = n;
    size_t NN = (size_t)N * N;
    int used = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel
    {
#ifdef _OPENMP
#pragma omp single
        used = omp_get_num_threads();
#endif
        double *phi = (double *)malloc(8 * NN * sizeof(double));
        double *dphi = jac ? (double *)malloc(16 * NN * sizeof(double)) : NULL;
        int want_abs = j1abs || chi1abs || phiabs_out || dsrcabs;
        double *pabs = want_abs ? (double *)malloc(8 * NN * sizeof(double)) : NULL;
        double *dpabs = (jac && jacabs) ? (double *)malloc(16 * NN * sizeof(double)) : NULL;
#pragma omp for schedule(dynamic, 1)
        for (long z = 0; z < Z; z++) {
            double T = state[4 * z + 0], eta = state[4 * z + 1];
            vxo_phi_zone(N, eps, n_mu, tmu, wmu, n_e, tE, wE, g2, T, eta, 0, split, eta_split, phi, dphi, pabs,
                         dpabs);
            if (phiabs_out)
                for (int d = 0; d < 2; d++)
                    for (int l = 0; l < 2; l++)
                        memcpy(phiabs_out + (((size_t)z * 2 + d) * 2 + l) * NN, &PHI(pabs, d, 0, l, 0),
                               NN * sizeof(double));
            if (phi_out) /* K^I only: [dir][l][i][j] */
                for (int d = 0; d < 2; d++)
                    for (int l = 0; l < 2; l++)
                        memcpy(phi_out + (((size_t)z * 2 + d) * 2 + l) * NN, &PHI(phi, d, 0, l, 0),
                               NN * sizeof(double));
            for (int si = 0; si < S; si++) {
                int sp = species[si];
                int pk = partner_index(S, species, si);
                double bI, bII;
                species_betas(sp, sin2w, &bI, &bII);
                const double *Jp = J + ((size_t)z * S + pk) * N;
                const double *Hp = H + ((size_t)z * S + pk) * N;
                const double c0 = 2.0 * VXO_PI * norm, c1 = 6.0 * VXO_PI * norm;
                double *D = dsrc ? dsrc + ((size_t)z * S + si) * 4 * NN : NULL;
                double *Da = dsrcabs ? dsrcabs + ((size_t)z * S + si) * 4 * NN : NULL;
                for (int i = 0; i < N; i++) {
                    double a_j0 = 0, a_c0 = 0, a_j1 = 0, a_c1 = 0, m_j1 = 0, m_c1 = 0;
                    double g[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
                    double ga[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
                    for (int j = 0; j < N; j++) {
                        size_t ij = (size_t)i * N + j;
                        /* species kernel = beta_I Phi_I + beta_II Phi_II, per direction and l */
                        double pp0 = bI * PHI(phi, 0, 0, 0, ij) + bII * PHI(phi, 0, 1, 0, ij);
                        double pp1 = bI * PHI(phi, 0, 0, 1, ij) + bII * PHI(phi, 0, 1, 1, ij);
                        double pa0 = bI * PHI(phi, 1, 0, 0, ij) + bII * PHI(phi, 1, 1, 0, ij);
                        double pa1 = bI * PHI(phi, 1, 0, 1, ij) + bII * PHI(phi, 1, 1, 1, ij);
                        a_j0 += w[j] * pp0 * (1.0 - Jp[j]);
                        a_c0 += w[j] * pa0 * Jp[j];
                        a_j1 += w[j] * pp1 * Hp[j];
                        a_c1 += w[j] * pa1 * Hp[j];
                        if (D) { /* coefficients of (1 - J), J, H, H in the four sums above */
                            D[0 * NN + ij] = -c0 * w[j] * pp0;
                            D[1 * NN + ij] = c0 * w[j] * pa0;
                            D[2 * NN + ij] = c1 * w[j] * pp1;
                            D[3 * NN + ij] = c1 * w[j] * pa1;
                        }
                        if (Da) {
                            Da[0 * NN + ij] = c0 * w[j] * fabs(pp0);
                            Da[1 * NN + ij] = c0 * w[j] * fabs(pa0);
                            Da[2 * NN + ij] = c1 * w[j] * (bI * PHI(pabs, 0, 0, 1, ij) + bII * PHI(pabs, 0, 1, 1, ij));
                            Da[3 * NN + ij] = c1 * w[j] * (bI * PHI(pabs, 1, 0, 1, ij) + bII * PHI(pabs, 1, 1, 1, ij));
                        }
                        if (pabs) {
                            m_j1 += w[j] * (bI * PHI(pabs, 0, 0, 1, ij) + bII * PHI(pabs, 0, 1, 1, ij)) * fabs(Hp[j]);
                            m_c1 += w[j] * (bI * PHI(pabs, 1, 0, 1, ij) + bII * PHI(pabs, 1, 1, 1, ij)) * fabs(Hp[j]);
                        }
                        if (jac)
                            for (int v = 0; v < 2; v++) {
                                double dpp0 = bI * DPHI(dphi, 0, 0, 0, ij, v) + bII * DPHI(dphi, 0, 1, 0, ij, v);
                                double dpp1 = bI * DPHI(dphi, 0, 0, 1, ij, v) + bII * DPHI(dphi, 0, 1, 1, ij, v);
                                double dpa0 = bI * DPHI(dphi, 1, 0, 0, ij, v) + bII * DPHI(dphi, 1, 1, 0, ij, v);
                                double dpa1 = bI * DPHI(dphi, 1, 0, 1, ij, v) + bII * DPHI(dphi, 1, 1, 1, ij, v);
                                g[0][v] += w[j] * dpp0 * (1.0 - Jp[j]);
                                g[1][v] += w[j] * dpa0 * Jp[j];
                                g[2][v] += w[j] * dpp1 * Hp[j];
                                g[3][v] += w[j] * dpa1 * Hp[j];
                                if (dpabs) {
                                    ga[0][v] += w[j] * (bI * DPHI(dpabs, 0, 0, 0, ij, v) + bII * DPHI(dpabs, 0, 1, 0, ij, v)) * fabs(1.0 - Jp[j]);
                                    ga[1][v] += w[j] * (bI * DPHI(dpabs, 1, 0, 0, ij, v) + bII * DPHI(dpabs, 1, 1, 0, ij, v)) * fabs(Jp[j]);
                                    ga[2][v] += w[j] * (bI * DPHI(dpabs, 0, 0, 1, ij, v) + bII * DPHI(dpabs, 0, 1, 1, ij, v)) * fabs(Hp[j]);
                                    ga[3][v] += w[j] * (bI * DPHI(dpabs, 1, 0, 1, ij, v) + bII * DPHI(dpabs, 1, 1, 1, ij, v)) * fabs(Hp[j]);
                                }
                            }
                    }
                    size_t o = ((size_t)z * S + si) * N + i;
                    j0[o] = c0 * a_j0;
                    chi0[o] = c0 * a_c0;
                    j1[o] = c1 * a_j1;
                    chi1[o] = c1 * a_c1;
                    if (j1abs) j1abs[o] = c1 * m_j1;
                    if (chi1abs) chi1abs[o] = c1 * m_c1;
                    if (jac) {
                        double c[4] = {c0, c0, c1, c1};
                        for (int out = 0; out < 4; out++) {
                            jac[o * 12 + out * 3 + 0] = c[out] * g[out][0];
                            jac[o * 12 + out * 3 + 1] = c[out] * g[out][1];
                            jac[o * 12 + out * 3 + 2] = 0.0; /* Y_e: no dependence */
                            if (dpabs) {
                                jacabs[o * 12 + out * 3 + 0] = c[out] * ga[out][0];
                                jacabs[o * 12 + out * 3 + 1] = c[out] * ga[out][1];
                                jacabs[o * 12 + out * 3 + 2] = 0.0;
                            }
                        }
                    }
                }
            }
        }
        free(phi);
        free(dphi);
        free(pabs);
        free(dpabs);
    }
    free(w); free(tmu); free(wmu); free(tE); free(wE);
    return used;
}
