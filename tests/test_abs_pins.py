"""Pins of the charged-current absorption and emission oracle (oracle/vx_abs_oracle.c) against what
physics and mathematics fix, not against a restatement of its formulas:

- detailed balance: j/chi = exp(-(eps - mu_nu)/T) with the beta-equilibrium chemical potential
  mu_nu = mu_e + mu_p - mu_n of non-degenerate nucleons, mu_n - mu_p = (m_n - m_p) + T ln(n_n/n_p),
  the mass difference taken from the nucleon masses (pins the lepton energy eps + Q or eps - Q,
  the lepton's occupation, the assignment of n_n and n_p);
- the equilibrium spectrum at mu_nu makes the source (1 - f) j - f chi vanish;
- the anti-nu_e threshold at eps = m_n - m_p, and the (eps - Q)^2 rise above it;
- Pauli blocking: absorption into occupied electron states vanishes in degenerate electrons;
- the scalings: every rate proportional to rho; nu_e absorption to the neutron fraction 1 - Y_e,
  its emission to the proton fraction Y_e, the reverse for anti-nu_e; nothing for nu_x;
- the Jacobian against fourth-order central differences in T, eta_e and Y_e.
"""
import numpy as np
import pytest
from scipy.special import expit

import oracle

Q_MASSES = 939.56542052 - 938.27208816  # m_n - m_p (MeV) from the nucleon masses
SP = np.array([0, 1, 2], np.int32)


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def zones(n, seed=0):
    rng = np.random.default_rng(seed)
    st = np.empty((n, 4))
    st[:, 0] = np.exp(rng.uniform(np.log(0.5), np.log(30.0), n))
    st[:, 1] = rng.uniform(-10.0, 40.0, n)
    st[:, 2] = rng.uniform(0.05, 0.6, n)
    st[:, 3] = np.exp(rng.uniform(np.log(1e8), np.log(1e14), n))
    return st


def grid(n=21):
    return np.geomspace(1.0, 300.0, n)


def mu_nu(st):
    T, eta, Ye = st[:, 0], st[:, 1], st[:, 2]
    return eta * T - Q_MASSES - T * np.log((1.0 - Ye) / Ye)


def test_detailed_balance_with_the_beta_equilibrium_chemical_potential():
    eps, st = grid(), zones(60, 1)
    r = oracle.abs_evaluate(eps, SP, st)
    T, mnu = st[:, 0][:, None], mu_nu(st)[:, None]
    for s, sign in ((0, 1.0), (1, -1.0)):  # anti-nu_e: mu = -mu_nu
        j, chi = r["j0"][:, s], r["chi0"][:, s]
        ok = (j > 1e-280) & (chi > 1e-280)
        assert ok.sum() > 500
        expect = -(eps[None, :] - sign * mnu) / T
        with np.errstate(divide="ignore", invalid="ignore"):
            got = np.log(j) - np.log(chi)
        assert np.max(np.abs(got - expect)[ok] / np.maximum(1.0, np.abs(expect[ok]))) < 1e-12


def test_equilibrium_spectrum_is_stationary():
    eps, st = grid(), zones(40, 2)
    r = oracle.abs_evaluate(eps, SP, st)
    T, mnu = st[:, 0][:, None], mu_nu(st)[:, None]
    for s, sign in ((0, 1.0), (1, -1.0)):
        a = (eps[None, :] - sign * mnu) / T
        f, omf = expit(-a), expit(a)  # Fermi-Dirac occupation at mu_nu and 1 - it
        j, chi = r["j0"][:, s], r["chi0"][:, s]
        src = omf * j - f * chi
        scale = omf * j + f * chi
        assert np.all(np.abs(src) <= 1e-13 * scale + 1e-300)


def test_antineutrino_threshold_and_rise_above_it():
    st = np.array([[2.0, 3.0, 0.3, 1e12]])
    below = np.array([0.2, 0.9, Q_MASSES * (1 - 1e-9)])
    r = oracle.abs_evaluate(below, SP, st)
    assert np.all(r["chi0"][0, 1] == 0.0) and np.all(r["j0"][0, 1] == 0.0)
    assert np.all(r["chi0"][0, 0] > 0.0)  # nu_e absorbs at any energy (E = eps + Q > 0)
    for d in (1e-3, 1e-5):
        r = oracle.abs_evaluate(np.array([Q_MASSES + d, Q_MASSES + 2 * d]), SP, st)
        c = r["chi0"][0, 1]
        assert abs(c[1] / c[0] - 4.0) < 10 * d  # (eps - Q)^2 at the threshold


def test_pauli_blocking_in_degenerate_electrons():
    T = 0.5
    eps = np.linspace(1.0, 80.0, 80)
    deg = np.array([[T, 80.0, 0.3, 1e13]])   # mu_e = 40 MeV
    hot = np.array([[T, -50.0, 0.3, 1e13]])  # no electrons: no blocking
    rd, rh = oracle.abs_evaluate(eps, SP, deg), oracle.abs_evaluate(eps, SP, hot)
    ratio = rd["chi0"][0, 0] / rh["chi0"][0, 0]
    E = eps + Q_MASSES
    assert np.all(ratio[E < 40.0 - 10 * T] < np.exp(-10.0))
    assert np.all(ratio[E > 40.0 + 10 * T] > 1.0 - np.exp(-10.0))
    # and emission needs occupied electron states: none without electrons
    assert np.all(rh["j0"][0, 0] < 1e-20 * rd["j0"][0, 0])


def test_scalings_in_density_and_electron_fraction():
    eps, st = grid(), zones(20, 3)
    base = oracle.abs_evaluate(eps, SP, st)
    s2 = st.copy()
    s2[:, 3] *= 2.0
    r2 = oracle.abs_evaluate(eps, SP, s2)
    for k in ("j0", "chi0"):
        np.testing.assert_allclose(r2[k], 2.0 * base[k], rtol=1e-15, atol=0)
    s3 = st.copy()
    s3[:, 2] = 0.5 * st[:, 2]
    r3 = oracle.abs_evaluate(eps, SP, s3)
    fp = (s3[:, 2] / st[:, 2])[:, None]               # proton fraction ratio
    fn = ((1 - s3[:, 2]) / (1 - st[:, 2]))[:, None]   # neutron fraction ratio
    np.testing.assert_allclose(r3["chi0"][:, 0], fn * base["chi0"][:, 0], rtol=1e-14)
    np.testing.assert_allclose(r3["j0"][:, 0], fp * base["j0"][:, 0], rtol=1e-14)
    np.testing.assert_allclose(r3["chi0"][:, 1], fp * base["chi0"][:, 1], rtol=1e-14)
    np.testing.assert_allclose(r3["j0"][:, 1], fn * base["j0"][:, 1], rtol=1e-14)
    for k in ("j0", "chi0", "j1", "chi1"):
        assert np.all(base[k][:, 2] == 0.0)
    assert np.all(base["j1"] == 0.0) and np.all(base["chi1"] == 0.0)


def test_jacobian_against_central_differences():
    eps, st = grid(9), zones(12, 4)
    r = oracle.abs_evaluate(eps, SP, st, jac=True)
    steps = (1e-5, 1e-4, 1e-4)  # relative in T, absolute in eta and Y_e
    for c, col in enumerate((0, 1, 2)):
        vals = []
        for k in (-2, -1, 1, 2):
            s = st.copy()
            h = steps[c] * (st[:, 0] if c == 0 else 1.0)
            s[:, col] = st[:, col] + k * h
            vals.append(oracle.abs_evaluate(eps, SP, s))
        h = (steps[c] * (st[:, 0] if c == 0 else np.ones(len(st))))[:, None, None]
        for o, key in ((0, "j0"), (1, "chi0")):
            fd = (vals[0][key] - 8 * vals[1][key] + 8 * vals[2][key] - vals[3][key]) / (12 * h)
            an = r["jac"][..., o, c]
            # per row: 1e-7 of the largest derivative, plus the stencil's rounding floor (a rate
            # that is nearly constant in the input has a derivative below what differences resolve)
            floor = 1e-13 * np.max(np.abs(r[key]), axis=-1, keepdims=True) / h
            tol = 1e-7 * np.max(np.abs(an), axis=-1, keepdims=True) + floor
            assert np.all(np.abs(fd - an) <= tol), (key, c)
            assert np.sum(np.abs(an) > 1e3 * floor) > 20  # and most rows do resolve the derivative
        assert np.all(r["jac"][..., 2:, :] == 0.0)


def test_invalid_zones_give_nan():
    st = zones(5, 5)
    st[1, 0] = -1.0
    st[2, 2] = 1.5
    st[3, 3] = np.nan
    r = oracle.abs_evaluate(grid(5), SP, st, jac=True)
    for k in ("j0", "chi0", "j1", "chi1"):
        assert np.all(np.isnan(r[k][[1, 2, 3]])) and np.all(np.isfinite(r[k][[0, 4]]))
    assert np.all(np.isnan(r["jac"][[1, 2, 3]]))
