"""GPU tangents: the adjoint kernel against the oracle's analytic T / eta derivatives (1e-5, per
(zone, species, output, input) row over the energy bins), the vector-Jacobian product against the
Jacobian, the torch.autograd path, and the forward rates produced by the same pass."""
import numpy as np
import pytest

import oracle
import vx_inputs
from _metrics import magnitudes, worst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("j0", "chi0", "j1", "chi1")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()
    oracle.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def rates_for(b, **kw):
    from paper_1404_1719_gb300 import PairRates
    return PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], **kw)


def check_jac(gj, ref, tol=1e-5):
    """Rows (zone, species, output) over the bins, per input; derivative sums whose terms change
    sign are measured against the oracle's sum of absolute values. The Y_e column must be 0."""
    oj, ma = ref["jac"], ref.get("jac_abs")
    assert np.all(gj[..., 2] == 0.0)
    for v in (0, 1):
        # [Z][S][N][4] -> rows (zone, species, output) over the bins
        m = None if ma is None else np.swapaxes(ma[..., v], 2, 3)
        e = worst(np.swapaxes(gj[..., v], 2, 3), np.swapaxes(oj[..., v], 2, 3), mag=m)
        assert e <= tol, f"input {v}: {e:.3e}"


@pytest.mark.parametrize("workload,rays", [(1, None), (2, None), (5, [3])])
def test_jacobian_against_oracle(workload, rays):
    b = vx_inputs.make_batch(workload, rays=rays)
    r = rates_for(b)
    res = r.adjoint(dev(b["state"]), dev(b["J"]), dev(b["H"]), jacobian=True, forward=True)
    assert r.check()
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"], b["J"], b["H"], jac=True,
                          mag=True)
    check_jac(res["jac"].cpu().numpy(), ref)
    fw = r.evaluate(dev(b["state"]), dev(b["J"]), dev(b["H"]))
    mg = magnitudes(ref)
    for k in KEYS:
        assert worst(res[k].cpu().numpy(), ref[k], mag=mg[k]) <= 1e-5
        # two FP32 instantiations: l = 1 sums that cancel differ at rounding times their absolute sum
        assert worst(res[k].cpu().numpy(), fw[k].cpu().numpy(), mag=mg[k]) <= 2e-6
    r.close()


def test_jacobian_edge_states():
    eps = vx_inputs.energy_centres(11, 1.0, 300.0)
    rows = [(T, eta) for T in (0.5, 4.0, 35.0) for eta in (-30.0, -5.0, 0.0, 6.0, 19.9, 20.1, 40.0, 75.0)]
    st, J, H = vx_inputs.random_zones(len(rows), 8, n_bins=11)
    st[:, 0] = [a for a, _ in rows]
    st[:, 1] = [c for _, c in rows]
    b = dict(eps=eps, n_mu=8, n_e=24, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)
    r = rates_for(b)
    res = r.adjoint(dev(st), dev(J), dev(H), jacobian=True)
    assert r.check()
    ref = oracle.evaluate(eps, 8, 24, b["species"], st, J, H, jac=True, mag=True)
    check_jac(res["jac"].cpu().numpy(), ref)
    r.close()


def test_vjp_matches_jacobian_and_autograd():
    from paper_1404_1719_gb300 import VxRatesFn
    b = vx_inputs.make_batch(1)
    r = rates_for(b)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    g = {k: torch.randn(J.shape, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(i))
         for i, k in enumerate(KEYS)}
    res = r.adjoint(st, J, H, grad_out=g, jacobian=True)
    jac = res["jac"]
    manual = torch.zeros(st.shape[0], 2, dtype=torch.float64, device="cuda")
    scale = torch.zeros_like(manual)
    for o, k in enumerate(KEYS):
        manual += torch.einsum("zsi,zsiv->zv", g[k], jac[..., o, :2])
        scale += torch.einsum("zsi,zsiv->zv", g[k].abs(), jac[..., o, :2].abs())
    gs = res["grad_state"]
    assert torch.all((gs[:, :2] - manual).abs() <= 1e-12 * scale)
    assert torch.all(gs[:, 2:] == 0)
    # autograd through the Function
    s2 = st.clone().requires_grad_(True)
    outs = VxRatesFn.apply(r, s2, J, H)
    torch.autograd.backward(outs, [g[k] for k in KEYS])
    np.testing.assert_allclose(s2.grad.cpu().numpy(), gs.cpu().numpy(), rtol=1e-12, atol=0)
    r.close()


def test_full_size_forward_adjoint_sampled():
    """4096 rays x 400 zones: Jacobian and forward from one pass; sampled zones vs the oracle."""
    b = vx_inputs.make_batch(4)
    Z = b["state"].shape[0]
    r = rates_for(b)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    res = r.adjoint(st, J, H, jacobian=True, forward=True, ray_offsets=b["ray_offsets"])
    assert r.check()
    rng = np.random.default_rng(4)
    pick = np.unique(np.concatenate([rng.integers(0, Z, 16), [0, 399, 400, Z - 1]]))
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"][pick], b["J"][pick],
                          b["H"][pick], jac=True, mag=True)
    check_jac(res["jac"][torch.as_tensor(pick, device="cuda")].cpu().numpy(), ref)
    mg = magnitudes(ref)
    for k in KEYS:
        assert worst(res[k][torch.as_tensor(pick, device="cuda")].cpu().numpy(), ref[k], mag=mg[k]) <= 1e-5
    r.close()


def test_maximum_sizes_forward_and_tangents():
    """31 bins (496 bin pairs) with 64 x 64 quadrature: the largest grid and node counts."""
    eps = vx_inputs.energy_centres(31, 0.5, 400.0)
    st, J, H = vx_inputs.random_zones(9, 31, n_bins=31, T_range=(0.8, 35.0), eta_range=(-5.0, 45.0))
    b = dict(eps=eps, n_mu=64, n_e=64, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)
    r = rates_for(b)
    res = r.adjoint(dev(st), dev(J), dev(H), jacobian=True, forward=True)
    assert r.check()
    ref = oracle.evaluate(eps, 64, 64, b["species"], st, J, H, jac=True, mag=True)
    check_jac(res["jac"].cpu().numpy(), ref)
    mg = magnitudes(ref)
    for k in KEYS:
        assert worst(res[k].cpu().numpy(), ref[k], mag=mg[k]) <= 1e-5, k
    r.close()


def test_3d_scale_workload_full_size_sampled():
    """16200 rays x 400 zones (6.48 M zones), 16 x 48 quadrature, eta_e up to ~63: forward and
    Jacobian of every zone in one pass; sampled zones against the oracle."""
    b = vx_inputs.make_batch(5)
    Z = b["state"].shape[0]
    r = rates_for(b, graph=True)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    res = r.adjoint(st, J, H, jacobian=True, forward=True, ray_offsets=b["ray_offsets"])
    assert r.check()
    rng = np.random.default_rng(5)
    pick = np.unique(np.concatenate([rng.integers(0, Z, 14), [0, 1, 399, Z - 1]]))
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"][pick], b["J"][pick],
                          b["H"][pick], jac=True, mag=True)
    ix = torch.as_tensor(pick, device="cuda")
    check_jac(res["jac"][ix].cpu().numpy(), ref)
    mg = magnitudes(ref)
    for k in KEYS:
        assert worst(res[k][ix].cpu().numpy(), ref[k], mag=mg[k]) <= 1e-5, k
    assert torch.isfinite(res["jac"]).all() and torch.isfinite(res["j0"]).all()
    r.close()
