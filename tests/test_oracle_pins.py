"""Pins of the FP64 oracle against facts fixed by mathematics, independent of its own code.

Each test below would fail for a plausible mistake in the oracle (a dropped term, a wrong sign,
a swapped operand, a wrong normalisation). None of them re-types the oracle's formulas:
  * Gauss-Legendre exactness on polynomials (and numpy's leggauss);
  * the Boltzmann-limit closed form of the pair kernel, from the Lorentz-covariant phase-space
    integral  Int d3p/(2E) d3pbar/(2Ebar) d4(p+pbar-Q) p^mu pbar^nu = (pi/24)(Q^2 g^munu + 2 Q^mu Q^nu);
  * detailed balance, the eps<->eps' exchange, and the eta = 0 electron/positron symmetry;
  * a continuum identity linking the kernel to complete Fermi-Dirac integrals F_3, F_4, and the
    closed forms that pin the F_k routine used there (F_2(0) = 3 zeta(3)/2, ...);
  * brute-force azimuth averaging with explicit four-vectors;
  * a brute-force angular integral that fixes the Legendre convention of the contraction;
  * central finite differences for the analytic gradients.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
import vx_inputs

SIN2W = 0.23


def fermi(k, eta):
    """Complete Fermi-Dirac integral F_k(eta) = Int_0^inf x^k / (exp(x - eta) + 1) dx (scipy quad)."""
    f = lambda x: x ** k * special.expit(eta - x)
    hi = max(eta, 0.0) + 80.0
    pts = [max(eta, 0.0)] if eta > 0 else None
    v, _ = integrate.quad(f, 0.0, hi, points=pts, epsabs=0, epsrel=1e-13, limit=400)
    return v


# ---------------------------------------------------------------------------------- quadrature
@pytest.mark.parametrize("n", [1, 2, 5, 16, 32, 48, 64])
def test_gauss_legendre_exact_on_polynomials(n):
    x, w = oracle.gauss_legendre(n)
    assert np.all(np.diff(x) > 0)
    for k in range(2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * x ** k) - exact) < 1e-14 * max(1.0, n / 8)
    xn, wn = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xn)) < 1e-14 and np.max(np.abs(w - wn)) < 1e-14


def test_energy_weights_log_grid():
    eps = vx_inputs.energy_centres(17, 1.0, 300.0)
    w = oracle.energy_weights(eps)
    r = eps[1] / eps[0]
    # on a logarithmic grid every bin spans eps*(r^1/2 - r^-1/2)
    np.testing.assert_allclose(w, eps ** 3 * (np.sqrt(r) - 1 / np.sqrt(r)), rtol=1e-13)
    # the widths telescope to the full span between the outer edges
    assert abs(np.sum(w / eps ** 2) - (eps[-1] * np.sqrt(r) - eps[0] / np.sqrt(r))) < 1e-10


# ---------------------------------------------------------------------- Boltzmann closed forms
@pytest.mark.parametrize("n_e", [2, 5, 32])
def test_boltzmann_closed_form_point(n_e):
    """(pi/24) s^2 (G2/(eps eps')) with s = 2 eps eps' y: K = (pi/6) eps eps' y^2 e^{-q0/T}."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        e, ep = np.exp(rng.uniform(0, np.log(380), 2))
        y = rng.uniform(1e-3, 2.0 - 1e-3)
        T = rng.uniform(1, 30)
        K = oracle.kernel_point(e, ep, y, T, rng.uniform(0, 20), n_e, boltzmann=True)
        cf = np.pi / 6 * e * ep * y * y
        np.testing.assert_allclose(K[1], [cf, cf], rtol=1e-12)
        np.testing.assert_allclose(K[0], [cf * np.exp(-(e + ep) / T)] * 2, rtol=1e-12)


@pytest.mark.parametrize("n_mu", [2, 16])
def test_boltzmann_phi_moments(n_mu):
    """Phi_0 = Int_0^2 dy (pi/6) eps eps' y^2 = (4 pi/9) eps eps';  Phi_1/Phi_0 = -1/2."""
    eps = vx_inputs.energy_centres(9, 1.0, 300.0)
    T, g2 = 7.0, 2.5
    ph = oracle.phi_zone(eps, n_mu, 3, T, 4.0, g2=g2, boltzmann=True)
    ee = np.outer(eps, eps)
    q0 = eps[:, None] + eps[None, :]
    for X in (0, 1):
        np.testing.assert_allclose(ph[1, X, 0], g2 * 4 * np.pi / 9 * ee, rtol=1e-12)
        np.testing.assert_allclose(ph[0, X, 0], g2 * 4 * np.pi / 9 * ee * np.exp(-q0 / T), rtol=1e-12)
        np.testing.assert_allclose(ph[:, X, 1] / ph[:, X, 0], -0.5, rtol=1e-12)


# ---------------------------------------------------------------------------------- symmetries
@pytest.mark.parametrize("T,eta", [(1.0, 0.0), (3.0, 5.0), (10.0, 20.0), (30.0, 60.0), (2.0, -4.0)])
def test_detailed_balance(T, eta):
    """O_a/O_p = exp((E + Ebar)/T) = exp(q0/T) at every node, so Phi^a = e^{q0/T} Phi^p."""
    eps = vx_inputs.energy_centres(11, 1.0, 300.0)
    ph = oracle.phi_zone(eps, 8, 16, T, eta)
    q0 = eps[:, None] + eps[None, :]
    ok = q0 / T < 600  # production flushes towards the FP64 underflow range beyond this
    for X in (0, 1):
        for l in (0, 1):
            ratio = ph[1, X, l][ok] / (ph[0, X, l][ok] * np.exp(q0[ok] / T))
            np.testing.assert_allclose(ratio, 1.0, rtol=2e-13)


@pytest.mark.parametrize("T,eta", [(1.0, 7.0), (5.0, 3.0), (30.0, 40.0)])
def test_exchange_symmetry(T, eta):
    """Exchanging nu and nubar (eps <-> eps') maps M_I onto M_II: Phi_II(i,j) = Phi_I(j,i)."""
    eps = vx_inputs.energy_centres(9, 1.0, 380.0)
    ph = oracle.phi_zone(eps, 8, 16, T, eta)
    np.testing.assert_allclose(ph[:, 1], np.swapaxes(ph[:, 0], -1, -2), rtol=1e-13, atol=0)


def test_eta_zero_particle_symmetry():
    """At eta = 0 electrons and positrons are interchangeable: Phi_I = Phi_II, so Phi_I is symmetric."""
    eps = vx_inputs.energy_centres(9, 1.0, 380.0)
    ph = oracle.phi_zone(eps, 8, 16, 4.0, 0.0)
    np.testing.assert_allclose(ph[:, 0], ph[:, 1], rtol=1e-12)
    np.testing.assert_allclose(ph[:, 0], np.swapaxes(ph[:, 0], -1, -2), rtol=1e-12)


def test_eta_sign_swaps_terms():
    """eta -> -eta exchanges the roles of e- and e+ (p <-> pbar), which maps M_I onto M_II."""
    eps = vx_inputs.energy_centres(7, 1.0, 300.0)
    a = oracle.phi_zone(eps, 8, 16, 6.0, 3.5)
    b = oracle.phi_zone(eps, 8, 16, 6.0, -3.5)
    np.testing.assert_allclose(a[:, 0], b[:, 1], rtol=1e-12)


# ------------------------------------------------------------------------ Fermi integrals + continuum
def test_fermi_integral_closed_forms():
    zeta3 = 1.2020569031595942
    assert abs(fermi(2, 0.0) - 1.5 * zeta3) < 1e-12
    assert abs(fermi(3, 0.0) - 7 * np.pi ** 4 / 120) < 1e-11
    for eta in (0.5, 2.0, 6.0, 15.0):
        assert abs((fermi(2, eta) - fermi(2, -eta)) - (eta ** 3 + np.pi ** 2 * eta) / 3) < 1e-10 * eta ** 3
        s3 = eta ** 4 / 4 + np.pi ** 2 * eta ** 2 / 2 + 7 * np.pi ** 4 / 60
        assert abs((fermi(3, eta) + fermi(3, -eta)) - s3) < 1e-10 * s3


@pytest.mark.parametrize("T,eta", [(2.0, 4.0), (5.0, 0.0), (1.5, -2.0)])
def test_continuum_fermi_identity(T, eta):
    """Int Int eps^2 eps'^2 Phi^p_{0,X} deps deps' = G2 (4 pi/9) T^8 F3(eta) F3(-eta), and with the
    weight (eps + eps'): T^9 (4 pi/9) [F4(eta) F3(-eta) + F3(eta) F4(-eta)].

    Total pair emission integrates the Lorentz-covariant neutrino phase space first, which leaves
    the electron-positron integral of (p.pbar)^2 f_e f_ebar. The eps, eps' integrals use Gauss-Laguerre.
    """
    xg, wg = np.polynomial.laguerre.laggauss(60)
    eps = T * xg
    ph = oracle.phi_zone(eps, 48, 48, T, eta)[0, :, 0]  # production, l = 0, [X][i][j]
    wl = T * wg * np.exp(xg) * eps ** 2
    ref0 = 4 * np.pi / 9 * T ** 8 * fermi(3, eta) * fermi(3, -eta)
    ref1 = 4 * np.pi / 9 * T ** 9 * (fermi(4, eta) * fermi(3, -eta) + fermi(3, eta) * fermi(4, -eta))
    for X in (0, 1):
        tot0 = wl @ ph[X] @ wl
        tot1 = wl @ (ph[X] * (eps[:, None] + eps[None, :])) @ wl
        assert abs(tot0 / ref0 - 1) < 1e-9
        assert abs(tot1 / ref1 - 1) < 1e-9


# ------------------------------------------------------------------------ brute-force kinematics
def _mink(a, b):
    return a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)


def _kernel_bruteforce(e, ep, y, T, eta, n_e, n_phi=12):
    """K^X_dir from explicit four-vectors: for each electron energy on the E-grid fix the polar
    angle of p about q by energy conservation, average M over the azimuth numerically."""
    cw = 1.0 - y
    k = np.array([e, 0.0, 0.0, e])
    kp = np.array([ep, ep * np.sqrt(1 - cw * cw), 0.0, ep * cw])
    Q = k + kp
    qv = Q[1:]
    q = np.linalg.norm(qv)
    qh = qv / q
    e1 = np.cross(qh, [0.0, 1.0, 0.0]); e1 /= np.linalg.norm(e1)
    e2 = np.cross(qh, e1)
    q0 = Q[0]
    s = _mink(Q, Q)
    Ep, Em = (q0 + q) / 2, (q0 - q) / 2
    t, w = np.polynomial.legendre.leggauss(n_e)
    phis = 2 * np.pi * np.arange(n_phi) / n_phi
    out = np.zeros((2, 2))
    for tk, wk in zip(t, w):
        E = (Ep + Em) / 2 + (Ep - Em) / 2 * tk
        W = (Ep - Em) / 2 * wk
        c = (2 * q0 * E - s) / (2 * q * E)
        sn = np.sqrt(max(0.0, 1 - c * c))
        pv = E * (c * qh[None, :] + sn * (np.cos(phis)[:, None] * e1 + np.sin(phis)[:, None] * e2))
        p = np.concatenate([np.full((n_phi, 1), E), pv], axis=1)
        pb = Q[None, :] - p
        assert np.allclose(_mink(pb, pb), 0.0, atol=1e-9 * q0 * q0)  # positron on its mass shell
        MI = np.mean(_mink(p, kp[None]) * _mink(pb, k[None]))
        MII = np.mean(_mink(p, k[None]) * _mink(pb, kp[None]))
        Eb = q0 - E
        fe = 1 / (np.exp(E / T - eta) + 1)
        fp = 1 / (np.exp(Eb / T + eta) + 1)
        for d, O in enumerate((fe * fp, (1 - fe) * (1 - fp))):
            out[d, 0] += W * O * MI
            out[d, 1] += W * O * MII
    return out * 2 * np.pi / (4 * q) / (e * ep)


@pytest.mark.parametrize("e,ep,y,T,eta", [(7.0, 19.0, 0.3, 5.0, 3.0), (150.0, 2.0, 1.9, 8.0, 12.0),
                                          (40.0, 41.0, 1.0, 2.0, -1.0), (300.0, 300.0, 0.02, 30.0, 20.0)])
def test_azimuth_average_bruteforce(e, ep, y, T, eta):
    ref = _kernel_bruteforce(e, ep, y, T, eta, 16)
    got = oracle.kernel_point(e, ep, y, T, eta, 16)
    np.testing.assert_allclose(got, ref, rtol=1e-11)


def test_precision_floor_against_mpmath():
    """The oracle's own FP64 rounding at a cancellation-prone point (eps >> eps', y near 2,
    degenerate electrons) compared with the same discrete rule evaluated in 40-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    e, ep, T, eta, n_e = 380.0, 1.0, 30.0, 20.0, 32
    t_mu, _ = np.polynomial.legendre.leggauss(32)
    y = 1.0 - t_mu[0]  # the node nearest to back-to-back emission
    tk, wk = np.polynomial.legendre.leggauss(n_e)
    E1, E2, Y, TT, ET = mp.mpf(e), mp.mpf(ep), mp.mpf(y), mp.mpf(T), mp.mpf(eta)
    q0 = E1 + E2
    s = 2 * E1 * E2 * Y
    q = mp.sqrt(q0 * q0 - s)
    Ep, Em = (q0 + q) / 2, s / (2 * (q0 + q))
    kq, kpq = E1 * (q0 - E2 * Y), E2 * (q0 - E1 * Y)
    perp = E1 ** 2 * E2 ** 2 * Y * (2 - Y) / q ** 2
    acc = [mp.mpf(0)] * 4
    for t, w in zip(tk, wk):
        E = (Ep + Em) / 2 + (Ep - Em) / 2 * mp.mpf(t)
        W = (Ep - Em) / 2 * mp.mpf(w)
        Ec = (2 * q0 * E - s) / (2 * q)
        pk, pkp = E * E1 - Ec * kq / q, E * E2 - Ec * kpq / q
        hs = (E * E - Ec * Ec) / 2
        MI = pkp * s / 2 - (pkp * pk - hs * perp)
        MII = pk * s / 2 - (pk * pkp - hs * perp)
        xe, xp = E / TT - ET, (q0 - E) / TT + ET
        Op = 1 / ((mp.exp(xe) + 1) * (mp.exp(xp) + 1))
        Oa = 1 / ((1 + mp.exp(-xe)) * (1 + mp.exp(-xp)))
        acc = [acc[0] + W * Op * MI, acc[1] + W * Op * MII, acc[2] + W * Oa * MI, acc[3] + W * Oa * MII]
    pref = 2 * mp.pi / (4 * q * E1 * E2)
    ref = np.array([float(pref * a) for a in acc]).reshape(2, 2)
    got = oracle.kernel_point(e, ep, y, T, eta, n_e)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


# ------------------------------------------------------------------------ contraction convention
def _betas(species):
    cv, ca = (-0.5 + 2 * SIN2W, -0.5) if species == 2 else (0.5 + 2 * SIN2W, 0.5)
    b1, b2 = (cv + ca) ** 2, (cv - ca) ** 2
    return (b2, b1) if species == 1 else (b1, b2)


def test_contraction_angular_bruteforce():
    """With R(cos w) = sum_l (2l+1)/2 Phi_l P_l(cos w) and f(mu') = J + 3 mu' H, integrating the
    production and absorption terms over the partner's direction gives j0 - mu j1 and chi0 + mu chi1."""
    eps = vx_inputs.energy_centres(6, 2.0, 120.0)
    N = len(eps)
    state = np.array([[6.0, 2.5, 0.3, 1e12]])
    rng = np.random.default_rng(5)
    J = rng.uniform(0.05, 0.9, (1, 3, N))
    H = rng.uniform(0.0, 0.3, (1, 3, N)) * J
    out = oracle.evaluate(eps, 8, 12, [0, 1, 2], state, J, H, sin2w=SIN2W)
    ph = oracle.phi_zone(eps, 8, 12, 6.0, 2.5)  # [dir][X][l][i][j]
    w = oracle.energy_weights(eps)
    mup, wmup = np.polynomial.legendre.leggauss(6)
    phis = 2 * np.pi * np.arange(8) / 8
    for si, sp in enumerate((0, 1, 2)):
        pk = {0: 1, 1: 0, 2: 2}[sp]
        bI, bII = _betas(sp)
        kern = bI * ph[:, 0] + bII * ph[:, 1]  # [dir][l][i][j]
        for mu in (-0.7, 0.2, 0.9):
            cw = mu * mup[:, None] + np.sqrt(1 - mu * mu) * np.sqrt(1 - mup[:, None] ** 2) * np.cos(phis)[None, :]
            for i in range(N):
                prod = absn = 0.0
                for j in range(N):
                    fbar = J[0, pk, j] + 3 * mup[:, None] * H[0, pk, j]
                    Rp = 0.5 * kern[0, 0, i, j] + 1.5 * kern[0, 1, i, j] * cw
                    Ra = 0.5 * kern[1, 0, i, j] + 1.5 * kern[1, 1, i, j] * cw
                    dphi = 2 * np.pi / len(phis)
                    prod += w[j] * np.sum(wmup[:, None] * dphi * Rp * (1 - fbar))
                    absn += w[j] * np.sum(wmup[:, None] * dphi * Ra * fbar)
                np.testing.assert_allclose(out["j0"][0, si, i] - mu * out["j1"][0, si, i], prod, rtol=1e-12)
                np.testing.assert_allclose(out["chi0"][0, si, i] + mu * out["chi1"][0, si, i], absn, rtol=1e-12)


def test_phi_dump_matches_zone_kernel():
    b = vx_inputs.make_batch(1, rays=[0])
    st = b["state"][:3]
    out = oracle.evaluate(b["eps"], 4, 6, b["species"], st, b["J"][:3], b["H"][:3], phi=True)
    for z in range(3):
        ph = oracle.phi_zone(b["eps"], 4, 6, st[z, 0], st[z, 1])
        np.testing.assert_array_equal(out["phi"][z], ph[:, 0])


def test_norm_and_g2_scale_linearly():
    eps = vx_inputs.energy_centres(5, 1.0, 100.0)
    st, J, H = vx_inputs.random_zones(2, 3, n_bins=5)
    a = oracle.evaluate(eps, 4, 6, [0, 1, 2], st, J, H)
    b = oracle.evaluate(eps, 4, 6, [0, 1, 2], st, J, H, g2=3.0, norm=0.5)
    for k in ("j0", "chi0", "j1", "chi1"):
        np.testing.assert_allclose(b[k], 1.5 * a[k], rtol=1e-14)


# -------------------------------------------------------------------------------- gradients
def test_gradient_central_differences():
    """Analytic d/dT and d/deta against central differences (h_T = 1e-4 T, h_eta = 1e-4 max(|eta|,1))."""
    eps = vx_inputs.energy_centres(7, 1.0, 300.0)
    st, J, H = vx_inputs.random_zones(4, 11, n_bins=7, eta_range=(0.0, 25.0))
    st[0, 1] = 0.0
    args = (eps, 6, 12, [0, 1, 2])
    base = oracle.evaluate(*args, st, J, H, jac=True)
    jac = base["jac"]
    keys = ("j0", "chi0", "j1", "chi1")
    for v, rel in ((0, lambda s: 1e-4 * s[:, 0]), (1, lambda s: 1e-4 * np.maximum(np.abs(s[:, 1]), 1.0))):
        h = rel(st)
        sp, sm = st.copy(), st.copy()
        sp[:, v] += h
        sm[:, v] -= h
        fp = oracle.evaluate(*args, sp, J, H)
        fm = oracle.evaluate(*args, sm, J, H)
        for o, k in enumerate(keys):
            fd = (fp[k] - fm[k]) / (2 * h[:, None, None])
            an = jac[..., o, v]
            for z in range(st.shape[0]):
                for s in range(3):
                    nrm = np.max(np.abs(an[z, s]))
                    if nrm < 1e-300:
                        continue
                    assert np.max(np.abs(fd[z, s] - an[z, s])) / nrm < 1e-6, (k, v, z, s)
    assert np.all(jac[..., 2] == 0.0)


def test_rejects_missing_partner_and_accepts_empty_batch():
    eps = vx_inputs.energy_centres(4, 1.0, 50.0)
    st, J, H = vx_inputs.random_zones(1, 0, n_bins=4, n_species=1)
    with pytest.raises(ValueError):
        oracle.evaluate(eps, 2, 2, [0], st, J, H)  # nu_e without its anti-nu_e partner
    out = oracle.evaluate(eps, 2, 2, [2], st[:0], J[:0], H[:0])
    assert out["j0"].shape == (0, 1, 4)


# ------------------------------------------------------------------ magnitude companions (l = 1)
def test_magnitude_companions_bound_and_limit():
    """The |P_l| sums bound |Phi_l| entrywise, equal Phi_0 for l = 0, and in the Boltzmann limit
    (K ~ (1 - cos w)^2) tend to Int |t| (1-t)^2 dt / Int (1-t)^2 dt = (3/2)/(8/3) = 9/16 of Phi_0."""
    eps = vx_inputs.energy_centres(7, 1.0, 300.0)
    ph = oracle.phi_zone(eps, 16, 12, 9.0, 30.0)
    pa = oracle.phi_zone(eps, 16, 12, 9.0, 30.0, mag=True)
    assert np.all(pa[:, :, 1] >= np.abs(ph[:, :, 1]) * (1 - 1e-15))
    np.testing.assert_array_equal(pa[:, :, 0], ph[:, :, 0])
    for n_mu, tol in ((32, 2e-3), (64, 5e-4)):
        mb = oracle.phi_zone(eps, n_mu, 4, 5.0, 0.0, boltzmann=True)
        mba = oracle.phi_zone(eps, n_mu, 4, 5.0, 0.0, boltzmann=True, mag=True)
        np.testing.assert_allclose(mba[1, 0, 1] / mb[1, 0, 0], 9 / 16, rtol=tol)
    st, J, H = vx_inputs.random_zones(3, 2, n_bins=7)
    out = oracle.evaluate(eps, 8, 8, [0, 1, 2], st, J, H, mag=True, jac=True)
    assert np.all(out["j1_abs"] >= np.abs(out["j1"])) and np.all(out["chi1_abs"] >= np.abs(out["chi1"]))
    assert np.all(out["jac_abs"] >= np.abs(out["jac"]) * (1 - 1e-14))


# -------------------------------------------------------------- derivatives w.r.t. the spectra
def _spectral_case(species=(0, 1, 2), zones=3, seed=5):
    b = vx_inputs.make_batch(1, seed=seed)
    st, J, H = b["state"][:zones], b["J"][:zones], b["H"][:zones]
    sp = np.array(species, np.int32)
    if len(sp) != J.shape[1]:
        J, H = J[:, : len(sp)].copy(), H[:, : len(sp)].copy()
    return b, st, J, H, sp


def _ev(b, sp, st, J, H, **kw):
    return oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], sp, st, J, H, **kw)


@pytest.mark.parametrize("species", [(0, 1, 2), (1, 0), (2,)])
def test_spectral_blocks_are_the_affine_coefficients(species):
    """The rates are affine in J (j0 through 1 - J, chi0 through J) and linear in H, so a
    perturbation of the partner spectra changes them by exactly the blocks times the perturbation,
    and j1 = D2 H, chi1 = D3 H, chi0 = D1 J, j0(J = 0) = -sum_j D0. These identities tie the blocks
    to the forward rates (pinned above) and catch a wrong sign, factor, partner or transposition."""
    b, st, J, H, sp = _spectral_case(species)
    ref = _ev(b, sp, st, J, H, spectral=True)
    D = ref["dsrc"]
    pk = oracle.partner_indices(sp)
    rng = np.random.default_rng(11)
    dJ = rng.uniform(-0.2, 0.2, J.shape)
    dH = rng.uniform(-0.2, 0.2, H.shape)
    moved = _ev(b, sp, st, J + dJ, H + dH)
    scale = lambda k: np.abs(ref[k]).max() + np.abs(moved[k]).max()
    for s in range(len(sp)):
        p = pk[s]
        for k, o, dX in (("j0", 0, dJ), ("chi0", 1, dJ), ("j1", 2, dH), ("chi1", 3, dH)):
            pred = np.einsum("zij,zj->zi", D[:, s, o], dX[:, p])
            assert np.abs(moved[k][:, s] - ref[k][:, s] - pred).max() <= 1e-12 * scale(k), (k, s)
        assert np.allclose(ref["chi0"][:, s], np.einsum("zij,zj->zi", D[:, s, 1], J[:, p]), rtol=1e-12, atol=0)
        assert np.allclose(ref["j1"][:, s], np.einsum("zij,zj->zi", D[:, s, 2], H[:, p]), rtol=1e-11,
                           atol=1e-13 * np.abs(ref["j1"]).max())
        assert np.allclose(ref["chi1"][:, s], np.einsum("zij,zj->zi", D[:, s, 3], H[:, p]), rtol=1e-11,
                           atol=1e-13 * np.abs(ref["chi1"]).max())
    zero = _ev(b, sp, st, np.zeros_like(J), H)
    assert np.allclose(zero["j0"], -D[:, :, 0].sum(axis=-1), rtol=1e-12, atol=0)
    assert np.all(D[:, :, 0] <= 0) and np.all(D[:, :, 1] >= 0)


def test_spectral_vjp_is_the_adjoint_of_the_perturbation():
    """<g, f(J + dJ, H + dH) - f(J, H)> = <grad_J, dJ> + <grad_H, dH> for random seeds g: pins the
    partner bookkeeping of the vector-Jacobian product against the forward oracle."""
    b, st, J, H, sp = _spectral_case((1, 2, 0), zones=2, seed=9)
    ref = _ev(b, sp, st, J, H, spectral=True)
    rng = np.random.default_rng(3)
    g = {k: rng.normal(size=J.shape) for k in ("j0", "chi0", "j1", "chi1")}
    gJ, gH = oracle.spectral_vjp(ref["dsrc"], sp, g["j0"], g["chi0"], g["j1"], g["chi1"])
    dJ = rng.uniform(-0.1, 0.1, J.shape)
    dH = rng.uniform(-0.1, 0.1, H.shape)
    moved = _ev(b, sp, st, J + dJ, H + dH)
    lhs = sum(np.sum(g[k] * (moved[k] - ref[k])) for k in g)
    rhs = np.sum(gJ * dJ) + np.sum(gH * dH)
    mag = sum(np.sum(np.abs(g[k]) * (np.abs(moved[k]) + np.abs(ref[k]))) for k in g)
    assert abs(lhs - rhs) <= 1e-12 * mag


def test_spectral_blocks_exchange_symmetry_between_nu_e_and_anti_nu_e():
    """The anti-neutrino's couplings are the neutrino's with (C_V + C_A)^2 and (C_V - C_A)^2
    exchanged, and term II(i, j) is term I(j, i). So both species' chi0 blocks follow from the raw
    term-I dump (pinned above through the zone kernel): nu_e uses beta_I Phi_I + beta_II Phi_I^T,
    anti-nu_e beta_II Phi_I + beta_I Phi_I^T, each times 2 pi w_j."""
    b, st, J, H, sp = _spectral_case((0, 1), zones=2, seed=4)
    ref = _ev(b, sp, st, J, H, spectral=True, phi=True)
    D, phi, w = ref["dsrc"], ref["phi"], oracle.energy_weights(b["eps"])
    cv, ca = 0.5 + 2 * SIN2W, 0.5
    bI, bII = (cv + ca) ** 2, (cv - ca) ** 2
    c0 = 2.0 * math.pi
    for z in range(st.shape[0]):
        KI = phi[z, 1, 0]  # annihilation, l = 0, term I
        k_nu = bI * KI + bII * KI.T
        k_nubar = bII * KI + bI * KI.T
        assert np.allclose(D[z, 0, 1], c0 * k_nu * w[None, :], rtol=1e-12, atol=0)
        assert np.allclose(D[z, 1, 1], c0 * k_nubar * w[None, :], rtol=1e-12, atol=0)


# --------------------------------------------------------------------- the split discrete rule
SPLIT_STATES = [(2.0, 15.0), (5.0, 30.0), (1.0, 60.0), (3.0, -20.0), (10.0, 5.0)]


def test_split_rule_without_an_edge_is_the_standard_rule():
    """With eta = 0 the Fermi edge sits at E = 0 <= E-, outside every interval: the split rule is
    the standard rule, bit for bit."""
    eps = vx_inputs.energy_centres(9, 1.0, 300.0)
    a = oracle.phi_zone(eps, 6, 16, 4.0, 0.0, grad=True)
    b = oracle.phi_zone(eps, 6, 16, 4.0, 0.0, grad=True, split=True, eta_split=0.0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # below the degeneracy threshold the split form keeps the standard rule
    a = oracle.phi_zone(eps, 6, 16, 2.0, 15.0)
    b = oracle.phi_zone(eps, 6, 16, 2.0, 15.0, split=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("T,eta", SPLIT_STATES)
def test_split_and_standard_rules_share_their_limit(T, eta):
    """Both rules discretise the same integral, so at 1024 nodes they agree to rounding; a wrong
    panel map, weight or edge would leave a finite gap."""
    eps = vx_inputs.energy_centres(9, 1.0, 300.0)
    a = oracle.phi_zone(eps, 6, 1024, T, eta)
    b = oracle.phi_zone(eps, 6, 1024, T, eta, split=True, eta_split=0.0)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


@pytest.mark.parametrize("T,eta", SPLIT_STATES[:4])
def test_split_rule_converges_faster_at_high_degeneracy(T, eta):
    """Where the Fermi edge cuts the electron-energy interval, panels meeting at the edge converge
    much faster: at 64 nodes the split rule is at least 100x closer to the converged value."""
    eps = vx_inputs.energy_centres(13, 1.0, 300.0)
    ref = oracle.phi_zone(eps, 8, 1024, T, eta, split=True, eta_split=0.0)
    scale = np.abs(ref).max(axis=-1, keepdims=True) + 1e-300
    err_std = np.max(np.abs(oracle.phi_zone(eps, 8, 64, T, eta) - ref) / scale)
    err_split = np.max(np.abs(oracle.phi_zone(eps, 8, 64, T, eta, split=True, eta_split=0.0) - ref) / scale)
    assert err_split * 100 <= err_std, (err_split, err_std)


@pytest.mark.parametrize("T,eta", SPLIT_STATES)
def test_split_rule_boltzmann_limit_matches_the_standard_rule(T, eta):
    """With Boltzmann statistics the integrand is a polynomial of degree 2 in E, integrated exactly
    by either rule, whatever the panels: the two agree to rounding (the Boltzmann closed form pins
    the standard rule above)."""
    for (e, ep, y) in ((10.0, 40.0, 0.3), (150.0, 20.0, 1.7), (80.0, 80.0, 1.0)):
        a = oracle.kernel_point(e, ep, y, T, eta, 16, boltzmann=True)
        b = oracle.kernel_point(e, ep, y, T, eta, 16, boltzmann=True, split=True)
        assert np.allclose(a, b, rtol=1e-13, atol=0)


def test_split_rule_gradient_central_differences():
    """Analytic d/dT and d/deta under the split rule against central differences. The panel
    boundary moves with mu_e = eta T; the integral does not depend on it, so at a converged node
    count (256 here) the difference is the finite-difference error alone. At 64 nodes the
    boundary's motion adds the derivative of the discretisation error (3e-4 in a T = 1.3 MeV zone
    with |q|/T ~ 100): the returned Jacobian is the split-rule quadrature of the derivatives."""
    eps = vx_inputs.energy_centres(7, 1.0, 300.0)
    st, J, H = vx_inputs.random_zones(3, 12, n_bins=7, eta_range=(8.0, 40.0))
    args = (eps, 6, 256, [0, 1, 2])
    base = oracle.evaluate(*args, st, J, H, jac=True, split=True, eta_split=0.0)
    keys = ("j0", "chi0", "j1", "chi1")
    for v, rel in ((0, lambda s: 1e-4 * s[:, 0]), (1, lambda s: 1e-4 * np.maximum(np.abs(s[:, 1]), 1.0))):
        h = rel(st)
        sp, sm = st.copy(), st.copy()
        sp[:, v] += h
        sm[:, v] -= h
        fp = oracle.evaluate(*args, sp, J, H, split=True, eta_split=0.0)
        fm = oracle.evaluate(*args, sm, J, H, split=True, eta_split=0.0)
        for o, k in enumerate(keys):
            fd = (fp[k] - fm[k]) / (2 * h[:, None, None])
            an = base["jac"][..., o, v]
            for z in range(st.shape[0]):
                for s in range(3):
                    nrm = np.max(np.abs(an[z, s]))
                    if nrm < 1e-300:
                        continue
                    assert np.max(np.abs(fd[z, s] - an[z, s])) / nrm < 1e-5, (k, v, z, s)


def test_split_rule_rejects_an_odd_node_count():
    eps = vx_inputs.energy_centres(5, 1.0, 100.0)
    st, J, H = vx_inputs.random_zones(2, 1, n_bins=5)
    with pytest.raises(ValueError):
        oracle.evaluate(eps, 4, 15, [0, 1, 2], st, J, H, split=True)
