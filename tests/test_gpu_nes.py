"""GPU parity of the inelastic neutrino-electron scattering (NES) kernel and of the electron-gas
closure, through the C ABI (include/vx_nes.h, include/vx_eos.h), against the FP64 oracle
(oracle/vx_nes_oracle.c) on the same seeded inputs.

Tolerances as for the pair kernel: 1e-12 for the FP64 form and 1e-5 for the mixed form, per
output row (zone, species) over the bins; sums whose terms change sign (the l = 1 projections,
the derivatives) are measured against the oracle's sum of absolute values (tests/_metrics.py).
"""
import numpy as np
import pytest

import oracle
import vx_inputs
from _metrics import worst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("j0", "chi0", "j1", "chi1")
TOL = {"fp64": 1e-12, "mixed": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()
    oracle.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def edge_batch(n_e=24):
    eps = vx_inputs.energy_centres(13, 1.0, 300.0)
    rows = [(T, eta) for T in (0.3, 1.0, 7.0, 40.0) for eta in (-45.0, -12.0, -3.0, 0.0, 2.5, 9.999, 25.0, 60.0, 79.5)]
    st, J, H = vx_inputs.random_zones(len(rows), 31, n_bins=13)
    st[:, 0] = [r[0] for r in rows]
    st[:, 1] = [r[1] for r in rows]
    return dict(eps=eps, n_mu=8, n_e=n_e, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)


def nes_case(name):
    """NES quadrature: n_mu cos(omega) nodes, n_e = 48 (16 nodes per electron-energy panel)."""
    if name == "workload1":
        b = vx_inputs.make_batch(1)
        return dict(b, n_mu=8, n_e=48)
    if name == "workload2":  # every fourth zone of the 400-zone ray (profiles T 30 -> 1 MeV, eta 20 -> 0)
        b = vx_inputs.make_batch(2)
        z = np.arange(0, 400, 4)
        return dict(b, state=b["state"][z], J=b["J"][z], H=b["H"][z], n_mu=16, n_e=48)
    if name == "degenerate":  # eta up to ~63
        b = vx_inputs.make_batch(5, rays=[7])
        z = np.arange(0, 400, 8)
        return dict(b, state=b["state"][z], J=b["J"][z], H=b["H"][z], n_mu=16, n_e=48)
    if name == "edge":
        return edge_batch(24)
    if name == "edge-generic":  # 10 nodes per panel: the instantiation without an unrolled count
        return edge_batch(30)
    raise KeyError(name)


CASES = ("workload1", "workload2", "degenerate", "edge", "edge-generic")


def rates(b, precision):
    from paper_1404_1719_gb300 import NesRates
    return NesRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], precision=precision)


def reference(b, jac=False):
    return oracle.nes_evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"], b["J"], b["H"], phi=True,
                               jac=jac, mag=True)


def mags(ref, k):
    return ref.get(k + "_abs")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES)
def test_nes_rates_and_kernel_against_oracle(case, precision):
    b = nes_case(case)
    r = rates(b, precision)
    out = r.evaluate(dev(b["state"]), dev(b["J"]), dev(b["H"]), phi=True)
    assert r.check()
    r.close()
    ref = reference(b)
    tol = TOL[precision]
    for k in KEYS:
        e = worst(out[k].cpu().numpy(), ref[k], mag=mags(ref, k))
        assert e <= tol, f"{k}: {e:.3e}"
    # kernel dump, rows (zone, X, dir, l, i) over j, against |P_l|-weighted magnitudes. The mixed
    # form carries the kernel in FP32: a row whose every entry lies more than the FP32 exponent
    # range (1e-30) below the zone's largest entry (in cold zones, in-scattering into the top bins
    # from far below) is out of its range and is not compared; the FP64 form is compared everywhere.
    g, o, m = out["phi"].cpu().numpy(), ref["phi"], ref["phi_abs"]
    if precision == "mixed":
        zmax = np.max(np.abs(o).reshape(o.shape[0], -1), axis=1)[:, None, None, None, None, None]
        keep = np.max(m, axis=-1, keepdims=True) >= 1e-30 * zmax
        g, o, m = np.where(keep, g, 0.0), np.where(keep, o, 0.0), np.where(keep, m, 0.0)
    e = worst(g, o, mag=m)
    assert e <= tol, f"phi: {e:.3e}"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ("workload1", "degenerate", "edge"))
def test_nes_jacobian_against_oracle(case, precision):
    b = nes_case(case)
    r = rates(b, precision)
    res = r.adjoint(dev(b["state"]), dev(b["J"]), dev(b["H"]), forward=True)
    assert r.check()
    r.close()
    ref = reference(b, jac=True)
    gj, oj, ma = res["jac"].cpu().numpy(), ref["jac"], ref["jac_abs"]
    assert np.all(gj[..., 2] == 0.0)
    tol = TOL[precision]
    for v in (0, 1):
        e = worst(np.swapaxes(gj[..., v], 2, 3), np.swapaxes(oj[..., v], 2, 3), mag=np.swapaxes(ma[..., v], 2, 3))
        assert e <= tol, f"input {v}: {e:.3e}"
    for k in KEYS:  # the forward rates of the same pass
        assert worst(res[k].cpu().numpy(), ref[k], mag=mags(ref, k)) <= tol, k


def test_nes_discrete_kernel_detailed_balance_on_device():
    """Phi^in(i,j) = e^{-(eps_i - eps_j)/T} Phi^out(i,j) in the dump (FP64 form: to rounding)."""
    b = nes_case("workload1")
    r = rates(b, "fp64")
    phi = r.evaluate(dev(b["state"]), dev(b["J"]), dev(b["H"]), phi=True)["phi"].cpu().numpy()
    r.close()
    T = b["state"][:, 0]
    X = np.exp(-(b["eps"][:, None] - b["eps"][None, :])[None] / T[:, None, None])
    lhs, rhs = phi[:, :, 0], X[:, None, None] * phi[:, :, 1]
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def test_nes_invalid_state_and_argument_checks():
    from paper_1404_1719_gb300 import capi
    b = nes_case("workload1")
    st = b["state"][:5].copy()
    st[1, 0] = -2.0   # T <= 0
    st[3, 1] = 90.0   # |eta| beyond the supported range
    r = rates(b, "mixed")
    out = r.evaluate(dev(st), dev(b["J"][:5]), dev(b["H"][:5]))
    assert capi.vx_nes_check(r.handle, torch.cuda.current_stream().cuda_stream) == capi.VX_ERR_NUMERIC
    j0 = out["j0"].cpu().numpy()
    assert np.all(np.isnan(j0[[1, 3]])) and np.all(np.isfinite(j0[[0, 2, 4]]))
    with pytest.raises(ValueError):  # host offsets that are not a partition
        r.evaluate(dev(st), dev(b["J"][:5]), dev(b["H"][:5]), ray_offsets=[0, 3])
    r.close()
    eps = np.asarray(b["eps"], np.float64)
    sp = np.array([0, 1, 2], np.int32)
    for n_e, n_mu in ((32, 8), (48, 40)):  # n_e not a multiple of 3; n_mu above 32
        cfg = capi.vx_config(n_bins=len(eps), eps=eps.ctypes.data_as(capi._dp), weights=None, n_mu=n_mu, n_e=n_e,
                             n_species=3, species=sp.ctypes.data_as(capi._ip), sin2w=0.23, g2=1.0, norm=1.0,
                             eta_fp64=0.0, prec=capi.VX_PREC_MIXED, flags=0)
        with pytest.raises(capi.VxError) as e:
            capi.vx_nes_create(cfg)
        assert e.value.status == capi.VX_ERR_INVALID_ARG


def test_eos_closure_and_chain_rule_against_oracle():
    """eta_e(rho, Y_e, T) and its derivatives against the oracle's Cardano solution; the chain rule
    applied to the NES and pair Jacobians gives d/d(T, Y_e, rho) at fixed (rho, Y_e) etc., and the
    Y_e column is no longer zero."""
    from paper_1404_1719_gb300 import NesRates, PairRates, eos_chain, eos_eta
    b = vx_inputs.make_batch(2)
    z = np.arange(0, 400, 10)
    st = b["state"][z].copy()
    st[:, 1] = -99.0  # overwritten by the closure
    dst = dev(st)
    deta = eos_eta(dst)
    eta_o, deta_o = oracle.eos_eta(st)
    np.testing.assert_allclose(dst[:, 1].cpu().numpy(), eta_o, rtol=1e-13, atol=0)
    np.testing.assert_allclose(deta.cpu().numpy(), deta_o, rtol=1e-11, atol=0)
    st_o = st.copy()
    st_o[:, 1] = eta_o
    J, H = b["J"][z], b["H"][z]
    for kind in ("nes", "pair"):
        if kind == "nes":
            r = NesRates(b["eps"], 8, 24, species=b["species"], precision="fp64")
            ref = oracle.nes_evaluate(b["eps"], 8, 24, b["species"], st_o, J, H, jac=True)["jac"]
            jac = r.adjoint(dst, dev(J), dev(H))["jac"]
        else:
            r = PairRates(b["eps"], 8, 16, species=b["species"])
            ref = oracle.evaluate(b["eps"], 8, 16, b["species"], st_o, J, H, jac=True)["jac"]
            jac = r.adjoint(dst, dev(J), dev(H), jacobian=True)["jac"]
        assert r.check()
        r.close()
        tot = eos_chain(jac, deta).cpu().numpy()
        g = jac.cpu().numpy()
        # the chain rule itself, from the kernel's own columns and the closure's derivatives
        dT, dE, dY = g[..., 0], g[..., 1], g[..., 2]
        assert np.all(dY == 0.0)  # these rates depend on Y_e only through eta_e
        d = deta.cpu().numpy()[:, None, None, None, :]
        exp = np.stack([dT + dE * d[..., 0], dY + dE * d[..., 1], dE * d[..., 2]], axis=-1)
        size = np.stack([np.abs(dT) + np.abs(dE * d[..., 0]), np.abs(dE * d[..., 1]), np.abs(dE * d[..., 2])], axis=-1)
        assert np.all(np.abs(tot - exp) <= 1e-14 * size)  # the T column is a sum that can cancel
        assert np.any(tot[..., 1] != 0.0)  # the Y_e column
        # and the Y_e column against the oracle's eta-derivative and the oracle's closure
        oy = ref[..., 1] * deta_o[:, None, None, None, 1]
        tol = 1e-10 if kind == "nes" else 1e-5
        scale = np.max(np.abs(oy), axis=2, keepdims=True)
        assert np.max(np.abs(tot[..., 1] - oy) / np.where(scale > 0, scale, 1)) <= tol
