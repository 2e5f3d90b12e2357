"""GPU parity of the charged-current absorption and emission rates (include/vx_abs.h) against the
FP64 oracle (oracle/vx_abs_oracle.c), through the C ABI, on the same seeded inputs.

Tolerances as for the other kernels, per output row (zone, species) over the bins: 1e-12 for the
FP64 form, 1e-5 for the mixed form (normwise and elementwise on entries >= 1e-3 of the row's
largest, tests/_metrics.py). Every term of these rates has one sign, so |o| is the magnitude.
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
SP = np.array([0, 1, 2], np.int32)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()
    oracle.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def edge_state():
    """T from 0.05 to 80 MeV, eta_e from -80 to 80, Y_e at 0 and 1 and between, rho from 0 to 1e15:
    occupations at both ends of the FP64 range, empty nucleon species, the anti-nu_e threshold."""
    rows = [(T, eta, ye, rho) for T in (0.05, 1.0, 80.0) for eta in (-80.0, -5.0, 0.0, 30.0, 80.0)
            for ye, rho in ((0.0, 1e12), (0.45, 1e15), (1.0, 1e9), (0.3, 0.0))]
    return np.array(rows, dtype=np.float64)


def case(name):
    if name == "workload1":
        b = vx_inputs.make_batch(1)
        return b["eps"], b["state"]
    if name == "workload2":
        b = vx_inputs.make_batch(2)
        return b["eps"], b["state"]
    if name == "degenerate":  # eta up to ~63
        b = vx_inputs.make_batch(5, rays=[7])
        return b["eps"], b["state"]
    if name == "edge":
        return np.concatenate([[0.5, 1.2, 1.29333236, 1.3], np.geomspace(2.0, 300.0, 17)]), edge_state()
    if name == "max-bins":  # 32 bins, the threshold inside the grid
        return np.geomspace(0.4, 400.0, 32), vx_inputs.make_batch(1)["state"][:20]
    raise KeyError(name)


CASES = ("workload1", "workload2", "degenerate", "edge", "max-bins")


def rates(eps, precision):
    from paper_1404_1719_gb300 import AbsRates
    return AbsRates(eps, species=SP, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", CASES)
def test_rates_and_jacobian_against_oracle(name, precision):
    eps, st = case(name)
    r = rates(eps, precision)
    res = r.adjoint(dev(st), forward=True)
    fw = r.evaluate(dev(st))
    assert r.check()
    r.close()
    ref = oracle.abs_evaluate(eps, SP, st, jac=True)
    tol = TOL[precision]
    for k in KEYS:
        g, o = res[k].cpu().numpy(), ref[k]
        assert worst(g, o) <= tol, f"{k}: {worst(g, o):.3e}"
        assert np.array_equal(fw[k].cpu().numpy(), g), k  # the forward call computes the same values
    gj, oj = res["jac"].cpu().numpy(), ref["jac"]
    for c in range(3):
        e = worst(np.swapaxes(gj[..., c], 2, 3), np.swapaxes(oj[..., c], 2, 3))
        assert e <= tol, f"column {c}: {e:.3e}"
    assert np.all(gj[..., 2:, :] == 0.0) and np.all(res["j1"].cpu().numpy() == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("species,nbins,nzones", [((0,), 1, 45), ((0,), 5, 101), ((1, 2), 13, 77)])
def test_few_entries_per_zone(species, nbins, nzones, precision):
    """Fewer than 32 entries (species x bins) per zone, so that a warp's 32 consecutive entries span
    several zones and the entry counter carries across zones; zone counts not multiples of 32."""
    from paper_1404_1719_gb300 import AbsRates
    sp = np.array(species, np.int32)
    eps = np.geomspace(0.8, 120.0, nbins) if nbins > 1 else np.array([7.5])
    st = vx_inputs.make_batch(2)["state"][:nzones]
    r = AbsRates(eps, species=sp, precision=precision)
    res = r.adjoint(dev(st), forward=True)
    assert r.check()
    r.close()
    ref = oracle.abs_evaluate(eps, sp, st, jac=True)
    tol = TOL[precision]
    for k in ("j0", "chi0"):
        assert worst(res[k].cpu().numpy(), ref[k]) <= tol, k
    gj, oj = res["jac"].cpu().numpy(), ref["jac"]
    for c in range(3):
        assert worst(np.swapaxes(gj[..., c], 2, 3), np.swapaxes(oj[..., c], 2, 3)) <= tol, c


def test_full_size_workload_sampled():
    """The bench's configuration (workload 4, 1.64 M zones, mixed form, forward + Jacobian) against
    the oracle on a sample of zones spread over the whole batch."""
    b = vx_inputs.make_batch(4)
    r = rates(b["eps"], "mixed")
    offs = torch.from_numpy(np.asarray(b["ray_offsets"], dtype=np.int32)).cuda()
    res = r.adjoint(dev(b["state"]), forward=True, ray_offsets=offs)
    assert r.check()
    r.close()
    zs = np.random.default_rng(0).choice(len(b["state"]), 2000, replace=False)
    ref = oracle.abs_evaluate(b["eps"], SP, b["state"][zs], jac=True)
    for k in ("j0", "chi0"):
        assert worst(res[k].cpu().numpy()[zs], ref[k]) <= 1e-5, k
    gj = res["jac"].cpu().numpy()[zs]
    for c in range(3):
        assert worst(np.swapaxes(gj[..., c], 2, 3), np.swapaxes(ref["jac"][..., c], 2, 3)) <= 1e-5, c


def test_detailed_balance_on_device():
    """j/chi = exp(-(eps - mu_nu)/T), mu_nu = eta T - Q - T ln((1 - Y_e)/Y_e), from the FP64 form."""
    eps, st = case("workload2")
    r = rates(eps, "fp64")
    out = r.evaluate(dev(st))
    r.close()
    T, eta, Ye = st[:, 0:1], st[:, 1:2], st[:, 2:3]
    mu = eta * T - (939.56542052 - 938.27208816) - T * np.log((1 - Ye) / Ye)
    j, chi = out["j0"].cpu().numpy()[:, 0], out["chi0"].cpu().numpy()[:, 0]
    ok = (j > 1e-280) & (chi > 1e-280)
    got = np.log(j[ok]) - np.log(chi[ok])
    expect = (-(eps[None, :] - mu) / T)[ok]
    assert np.max(np.abs(got - expect) / np.maximum(1.0, np.abs(expect))) < 1e-12


def test_chain_rule_gives_the_total_electron_fraction_derivative():
    """With eta_e from the electron-gas closure, eos_chain of this Jacobian is the derivative at
    fixed (T, rho): compared with central differences of the oracle through the oracle's closure."""
    from paper_1404_1719_gb300 import eos_chain, eos_eta
    b = vx_inputs.make_batch(2)
    st = b["state"][::20].copy()
    dst = dev(st)
    deta = eos_eta(dst)
    r = rates(b["eps"], "fp64")
    jac = r.adjoint(dst)["jac"]
    r.close()
    tot = eos_chain(jac, deta).cpu().numpy()

    def rates_at(ye):
        s = st.copy()
        s[:, 2] = ye
        s[:, 1] = oracle.eos_eta(s)[0]
        return oracle.abs_evaluate(b["eps"], SP, s)

    h = 1e-5
    ye = st[:, 2]
    v = [rates_at(ye + k * h) for k in (-2, -1, 1, 2)]
    for o, key in ((0, "j0"), (1, "chi0")):
        fd = (v[0][key] - 8 * v[1][key] + 8 * v[2][key] - v[3][key]) / (12 * h)
        an = tot[..., o, 1]
        scale = np.max(np.abs(an), axis=-1, keepdims=True) + 1e-300
        assert np.max(np.abs(fd - an) / scale) < 1e-6, key


def test_invalid_states_offsets_and_arguments():
    from paper_1404_1719_gb300 import capi
    eps, st = case("workload1")
    st = st[:6].copy()
    st[1, 0] = 0.0      # T <= 0
    st[3, 2] = 1.2      # Y_e > 1
    st[4, 3] = -1.0     # rho < 0
    r = rates(eps, "mixed")
    out = r.evaluate(dev(st))
    assert capi.vx_abs_check(r.handle, torch.cuda.current_stream().cuda_stream) == capi.VX_ERR_NUMERIC
    j0 = out["j0"].cpu().numpy()
    assert np.all(np.isnan(j0[[1, 3, 4]])) and np.all(np.isfinite(j0[[0, 2, 5]]))
    ok = vx_inputs.make_batch(1)["state"][:6]
    r.evaluate(dev(ok), ray_offsets=torch.tensor([0, 4, 3, 6], dtype=torch.int32, device="cuda"))
    assert capi.vx_abs_check(r.handle, torch.cuda.current_stream().cuda_stream) == capi.VX_ERR_NUMERIC
    with pytest.raises(ValueError):  # host offsets that are not a partition
        r.evaluate(dev(ok), ray_offsets=[0, 2])
    with pytest.raises(ValueError):  # state on the host
        r.evaluate(torch.from_numpy(ok))
    # a host pointer reaches the C ABI: rejected before any launch
    b = capi.vx_batch(n_rays=1, n_zones=6, ray_offsets=None, state=ok.ctypes.data, J=None, H=None)
    o = {k: torch.empty((6, 3, len(eps)), dtype=torch.float64, device="cuda") for k in KEYS}
    with pytest.raises(capi.VxError) as e:
        capi.vx_abs_eval(r.handle, b, capi.vx_out(*(o[k].data_ptr() for k in KEYS), None))
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    b.state = dev(ok).data_ptr()
    phi = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.VxError) as e:  # no kernel to dump
        capi.vx_abs_eval(r.handle, b, capi.vx_out(*(o[k].data_ptr() for k in KEYS), phi.data_ptr()))
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    r.close()
    sp = np.array([0, 0], np.int32)
    cfg = capi.vx_config(n_bins=len(eps), eps=np.ascontiguousarray(eps).ctypes.data_as(capi._dp), weights=None,
                         n_mu=0, n_e=0, n_species=2, species=sp.ctypes.data_as(capi._ip), sin2w=0.0, g2=1.0,
                         norm=1.0, eta_fp64=0.0, prec=capi.VX_PREC_MIXED, flags=0)
    with pytest.raises(capi.VxError) as e:  # a species twice
        capi.vx_abs_create(cfg)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
