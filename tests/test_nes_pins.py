"""Pins of the inelastic neutrino-electron scattering (NES) oracle and of the electron-gas closure
(oracle/vx_nes_oracle.c) against mathematics that does not go through the oracle's own formulas.

  - Gauss-Laguerre nodes: numpy's laggauss, and exactness on x^k e^{-x} (k < 2n).
  - The azimuth average <M_X>: explicit four-vectors p, p' = p + q with |p'| = E + q0, averaged
    over the azimuth of p about q numerically.
  - Normalisation and the whole reduction: without blocking (Boltzmann electrons), the
    out-scattering rate integrated over the final neutrino, Int eps'^2 d eps' Phi^out_0, has the
    closed form 8 pi G2 eps T^4 e^eta for term I and a third of it for term II (the massless
    two-body phase space: s^2/4 and u^2/4 averaged over it).
  - Detailed balance R^in = e^{-(eps - eps')/T} R^out and time reversal R^out(eps, eps') =
    R^in(eps', eps), each computed from its own blocking formula.
  - The three-panel discrete rule against an adaptive quadrature of the same integral, with the
    four-vector integrand.
  - Central differences of the analytic T and eta derivatives.
  - The contraction's factors and signs: the collision integral of sec. 2.1's moment equation,
    integrated directly over the partner directions, equals (1 - f)(j0 - mu j1) - f (chi0 + mu chi1).
  - The closure: the net electron density from a numerical Fermi integral, and central differences.
"""
import math

import numpy as np
import pytest

import oracle

integrate = pytest.importorskip("scipy.integrate")


def test_gauss_laguerre_nodes_and_exactness():
    for n in (4, 16, 24, 32):
        x, w = oracle.gauss_laguerre(n)
        xr, wr = np.polynomial.laguerre.laggauss(n)
        assert np.allclose(x, xr, rtol=1e-13, atol=0) and np.allclose(w, wr, rtol=1e-11, atol=1e-300)
        for k in range(0, 2 * n, max(1, n // 4)):
            # Int_0^inf x^k e^{-x} dx = k!, in relative terms
            assert abs(np.sum(w * x ** k) / math.factorial(k) - 1.0) < 1e-10, (n, k)


def four_vector_average(eps, epsp, y, E, n_phi=16):
    """<M_I>, <M_II> at electron energy E from explicit four-vectors (metric +---)."""
    c = 1.0 - y
    k = np.array([eps, 0.0, 0.0, eps])
    kp = np.array([epsp, epsp * math.sqrt(max(0.0, 1 - c * c)), 0.0, epsp * c])
    q = k - kp
    qv = q[1:]
    Q = np.linalg.norm(qv)
    qh = qv / Q
    e1 = np.cross(qh, [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(qh, e1)
    cs = (E * q[0] - eps * epsp * y) / (E * Q)  # cos(p, q) fixed by |p + q| = E + q0
    sn = math.sqrt(max(0.0, 1 - cs * cs))
    dot = lambda a, b: a[0] * b[0] - a[1:] @ b[1:]
    mI = mII = 0.0
    for ph in 2 * math.pi * (np.arange(n_phi) + 0.5) / n_phi:
        p = np.concatenate([[E], E * (sn * math.cos(ph) * e1 + sn * math.sin(ph) * e2 + cs * qh)])
        pp = p + q
        assert abs(np.linalg.norm(pp[1:]) - pp[0]) < 1e-9 * pp[0]  # the outgoing electron is on shell
        mI += dot(k, p) * dot(kp, pp) / n_phi
        mII += dot(k, pp) * dot(kp, p) / n_phi
    return mI, mII


def brute_point(eps, epsp, y, T, eta, n_e, F):
    """R^X at one point with the oracle's nodes but the four-vector integrand and a blocking F."""
    E, W = oracle.nes_nodes(eps, epsp, y, T, eta, n_e)
    Q = math.sqrt(eps ** 2 + epsp ** 2 - 2 * eps * epsp * (1 - y))
    pref = 2 * math.pi / (4 * Q) / (eps * epsp)
    s = np.zeros(2)
    for e, w in zip(E, W):
        if w != 0.0:
            s += w * F(e, e + eps - epsp) * np.array(four_vector_average(eps, epsp, y, e))
    return pref * s


def fd(E, T, eta):
    return 1.0 / (math.exp(min(E / T - eta, 700.0)) + 1.0)


@pytest.mark.parametrize("eps,epsp,y,T,eta", [(30.0, 12.0, 0.4, 5.0, 2.0), (5.0, 80.0, 1.7, 8.0, 6.0),
                                              (100.0, 99.0, 0.02, 3.0, 25.0), (40.0, 40.0, 1.0, 10.0, -2.0)])
def test_azimuth_average_against_four_vectors(eps, epsp, y, T, eta):
    K = oracle.nes_point(eps, epsp, y, T, eta, 48)
    bout = brute_point(eps, epsp, y, T, eta, 48, lambda a, b: fd(a, T, eta) * (1 - fd(b, T, eta)))
    bin_ = brute_point(eps, epsp, y, T, eta, 48, lambda a, b: (1 - fd(a, T, eta)) * fd(b, T, eta))
    np.testing.assert_allclose(K[1], bout, rtol=1e-10)
    np.testing.assert_allclose(K[0], bin_, rtol=1e-10)


def _phi0_boltzmann(eps, epsp, T, eta, n=48):
    """Int d(cos w) R^out (no blocking) in y = s^2, which removes the 1/|q| behaviour of the
    integrand at forward, elastic scattering."""
    s, w = np.polynomial.legendre.leggauss(n)
    s, w = (s + 1) * math.sqrt(2) / 2, w * math.sqrt(2) / 2
    tot = np.zeros(2)
    for sv, wv in zip(s, w):
        tot += wv * 2 * sv * oracle.nes_point(eps, epsp, sv * sv, T, eta, 48, boltzmann=True)[1]
    return tot


@pytest.mark.parametrize("eps,T,eta", [(10.0, 4.0, -1.0), (30.0, 6.0, 0.5)])
def test_boltzmann_total_rate_closed_form(eps, T, eta):
    """Int_0^inf eps'^2 Phi^out_{0,X}(eps, eps') d eps' = 8 pi eps T^4 e^eta x (1, 1/3) for X = I, II.
    eps' is integrated in variables that cluster at eps' = eps (eps (1 - z^2) below, eps + 40 T z^2
    above, then Gauss-Laguerre), where the integrand has a logarithmic singularity."""
    z, wz = np.polynomial.legendre.leggauss(48)
    z, wz = (z + 1) / 2, wz / 2
    L = 40 * T
    tot = np.zeros(2)
    for zv, wv in zip(z, wz):
        ep = eps * (1 - zv * zv)
        tot += wv * 2 * eps * zv * ep * ep * _phi0_boltzmann(eps, ep, T, eta)
        ep = eps + L * zv * zv
        tot += wv * 2 * L * zv * ep * ep * _phi0_boltzmann(eps, ep, T, eta)
    xl, wl = np.polynomial.laguerre.laggauss(16)
    for x, w in zip(xl, wl):
        ep = eps + L + T * x
        tot += T * w * math.exp(x) * ep * ep * _phi0_boltzmann(eps, ep, T, eta)
    ref = 8 * math.pi * eps * T ** 4 * math.exp(eta)
    np.testing.assert_allclose(tot, [ref, ref / 3], rtol=1e-7)


@pytest.mark.parametrize("eps,epsp,y,T,eta", [(30.0, 12.0, 0.4, 5.0, 2.0), (5.0, 80.0, 1.7, 8.0, 6.0),
                                              (100.0, 99.0, 0.02, 3.0, 25.0), (2.0, 150.0, 1.2, 20.0, 40.0)])
def test_detailed_balance_and_time_reversal(eps, epsp, y, T, eta):
    K = oracle.nes_point(eps, epsp, y, T, eta, 48)
    np.testing.assert_allclose(K[0], math.exp(-(eps - epsp) / T) * K[1], rtol=1e-12)
    Kr = oracle.nes_point(epsp, eps, y, T, eta, 48)
    # the reversed process: out of eps' into eps has the in-kernel of (eps, eps'); the rule's nodes
    # differ (E_min and the edges move), so agreement is to the rule's accuracy
    np.testing.assert_allclose(Kr[1], K[0], rtol=2e-5)
    np.testing.assert_allclose(Kr[0], K[1], rtol=2e-5)


@pytest.mark.parametrize("eps,epsp,y,T,eta", [(30.0, 12.0, 0.4, 5.0, 2.0), (5.0, 80.0, 1.7, 8.0, 6.0),
                                              (100.0, 60.0, 0.3, 3.0, 25.0), (200.0, 20.0, 1.9, 1.0, 55.0),
                                              (40.0, 41.0, 0.01, 15.0, -3.0)])
def test_three_panel_rule_against_adaptive_quadrature(eps, epsp, y, T, eta):
    q0 = eps - epsp
    Q = math.sqrt(eps ** 2 + epsp ** 2 - 2 * eps * epsp * (1 - y))
    Emin = 0.5 * (Q - q0)
    mu = eta * T

    def g(E, X):
        return fd(E, T, eta) * (1 - fd(E + q0, T, eta)) * four_vector_average(eps, epsp, y, E, 8)[X]

    pts = sorted({Emin, max(Emin, mu - max(q0, 0.0)), max(Emin, mu + max(-q0, 0.0))})
    ref = np.zeros(2)
    for X in (0, 1):
        for a, b in zip(pts[:-1], pts[1:]):
            if b > a:
                ref[X] += integrate.quad(g, a, b, args=(X,), epsrel=1e-12, epsabs=0, limit=400)[0]
        ref[X] += integrate.quad(g, pts[-1], np.inf, args=(X,), epsrel=1e-12, epsabs=0, limit=400)[0]
    ref *= 2 * math.pi / (4 * Q) / (eps * epsp)
    np.testing.assert_allclose(oracle.nes_point(eps, epsp, y, T, eta, 48)[1], ref, rtol=2e-5)
    np.testing.assert_allclose(oracle.nes_point(eps, epsp, y, T, eta, 96)[1], ref, rtol=1e-9)


@pytest.mark.parametrize("eps,epsp,y,T,eta", [(30.0, 12.0, 0.4, 5.0, 2.0), (5.0, 80.0, 1.7, 8.0, 6.0),
                                              (100.0, 60.0, 0.3, 3.0, 25.0)])
def test_gradients_against_central_differences(eps, epsp, y, T, eta):
    """At fixed nodes: the differences keep the nodes of (T, eta) by evaluating the blocking of the
    shifted state on the unshifted nodes (the four-vector integrand on oracle.nes_nodes)."""
    _, dK = oracle.nes_point(eps, epsp, y, T, eta, 48, grad=True)
    hT, he = 1e-4 * T, 1e-4 * max(abs(eta), 1.0)

    def at(Tx, ex):
        return np.array([brute_point(eps, epsp, y, T, eta, 48,
                                     lambda a, b: (1 - fd(a, Tx, ex)) * fd(b, Tx, ex)),
                         brute_point(eps, epsp, y, T, eta, 48,
                                     lambda a, b: fd(a, Tx, ex) * (1 - fd(b, Tx, ex)))])
    dT = (at(T + hT, eta) - at(T - hT, eta)) / (2 * hT)
    de = (at(T, eta + he) - at(T, eta - he)) / (2 * he)
    np.testing.assert_allclose(dK[..., 0], dT, rtol=1e-6, atol=1e-9 * np.abs(dT).max())
    np.testing.assert_allclose(dK[..., 1], de, rtol=1e-6, atol=1e-9 * np.abs(de).max())


def test_contraction_is_the_collision_integral():
    """df/dt of the moment equation (sec. 2.1) for f(mu') = J + 3 mu' H, integrated directly over
    the partner directions: in coordinates about the neutrino's own direction (the angle omega on
    the oracle's Gauss-Legendre nodes in cos(omega), the azimuth psi about k on a uniform grid),
    with the partner's direction cosine mu' = mu cos(omega) + sqrt(1 - mu^2) sin(omega) cos(psi) and
    the kernel evaluated at each omega. This fixes the 2 pi and 6 pi factors, the (1 - J) of the
    loss term, the couplings and the signs of j1 and chi1."""
    eps = np.array([4.0, 11.0, 25.0, 50.0])
    n = len(eps)
    T, eta = 6.0, 3.0
    n_mu = 24
    st = np.array([[T, eta, 0.3, 1e12]])
    J = np.array([[[0.6, 0.4, 0.2, 0.05]]])
    H = np.array([[[0.1, 0.15, 0.05, 0.02]]])
    for species in (0, 1, 2):
        sp = np.array([species], np.int32)
        r = oracle.nes_evaluate(eps, n_mu, 48, sp, st, J, H)
        w = oracle.energy_weights(eps)
        cv, ca = (-0.5 if species == 2 else 0.5) + 2 * 0.23, (-0.5 if species == 2 else 0.5)
        bI, bII = (cv + ca) ** 2, (cv - ca) ** 2
        if species == 1:
            bI, bII = bII, bI
        f = 0.3
        tw, ww = np.polynomial.legendre.leggauss(n_mu)
        npsi = 16
        for i in (0, 2):
            for mu in (-0.6, 0.8):
                gain = loss = 0.0
                for j in range(n):
                    for cw, wcw in zip(tw, ww):
                        K = oracle.nes_point(eps[i], eps[j], 1.0 - cw, T, eta, 48)
                        Kin, Kout = bI * K[0][0] + bII * K[0][1], bI * K[1][0] + bII * K[1][1]
                        sw = math.sqrt(1 - cw * cw)
                        for a in range(npsi):
                            psi = 2 * math.pi * (a + 0.5) / npsi
                            mup = mu * cw + math.sqrt(1 - mu * mu) * sw * math.cos(psi)
                            fp = J[0, 0, j] + 3 * mup * H[0, 0, j]
                            dom = wcw * 2 * math.pi / npsi
                            gain += w[j] * dom * Kin * fp
                            loss += w[j] * dom * Kout * (1 - fp)
                direct = (1 - f) * gain - f * loss
                moments = ((1 - f) * (r["j0"][0, 0, i] - mu * r["j1"][0, 0, i])
                           - f * (r["chi0"][0, 0, i] + mu * r["chi1"][0, 0, i]))
                assert abs(direct - moments) <= 1e-12 * (abs(gain) + abs(loss)), (species, i, mu, direct, moments)


def test_discrete_kernel_obeys_detailed_balance_and_time_reversal_exactly():
    """The zone's discrete kernel (down-scattering order integrated, the rest by symmetry):
    Phi^in(i,j) = e^{-(eps_i - eps_j)/T} Phi^out(i,j) for every ordered pair (the oracle computes
    the two blocking factors independently), and Phi^out(i,j) = Phi^in(j,i)."""
    eps = np.array([2.0, 9.0, 30.0, 90.0, 200.0])
    T, eta = 7.0, 4.0
    st = np.array([[T, eta, 0.3, 1e12]])
    J = np.full((1, 1, len(eps)), 0.3)
    r = oracle.nes_evaluate(eps, 12, 48, np.array([0], np.int32), st, J, 0.5 * J, phi=True)
    phi = r["phi"][0]  # [X][dir][l][i][j], dir 0 = in, 1 = out
    X = np.exp(-(eps[:, None] - eps[None, :]) / T)
    np.testing.assert_allclose(phi[:, 0], X[None, None] * phi[:, 1], rtol=1e-12, atol=0)
    np.testing.assert_allclose(phi[:, 1], np.swapaxes(phi[:, 0], -1, -2), rtol=1e-12, atol=0)


def test_eos_closure_against_fermi_integrals():
    """The net electron density of the massless gas at the returned eta, from a numerical Fermi
    integral, equals rho Y_e / m_u; the derivatives match central differences."""
    hbarc, mu_g = 1.973269804e-11, 1.66053906660e-24
    st = np.array([[0.8, 0, 0.45, 1e10], [5.0, 0, 0.3, 1e12], [12.0, 0, 0.25, 3e13], [30.0, 0, 0.2, 1e14],
                   [2.0, 0, 0.4, 5e14]])
    eta, deta = oracle.eos_eta(st)
    for z in range(len(st)):
        T, ye, rho = st[z, 0], st[z, 2], st[z, 3]
        e = eta[z]
        g = lambda x: x * x * (1 / (math.exp(min(x - e, 700)) + 1) - 1 / (math.exp(min(x + e, 700)) + 1))
        pts = [0.0, max(e, 1.0), max(e, 1.0) + 60.0]
        F = sum(integrate.quad(g, a, b, epsrel=1e-13, limit=400)[0] for a, b in zip(pts[:-1], pts[1:]))
        n_net = (T / hbarc) ** 3 * F / math.pi ** 2
        assert abs(n_net / (rho * ye / mu_g) - 1) < 1e-10, z
        for v, col in ((0, 0), (2, 1), (3, 2)):
            h = 1e-5 * st[z, v]
            sp, sm = st[z:z + 1].copy(), st[z:z + 1].copy()
            sp[0, v] += h
            sm[0, v] -= h
            num = (oracle.eos_eta(sp)[0][0] - oracle.eos_eta(sm)[0][0]) / (2 * h)
            assert abs(num - deta[z, col]) <= 1e-7 * abs(deta[z, col]), (z, v)
