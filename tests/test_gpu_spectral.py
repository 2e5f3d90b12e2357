"""GPU derivatives of the rates with respect to the partner spectra (vx_rates_spectral): the
blocks d(j0, chi0)/dJ, d(j1, chi1)/dH and the vector-Jacobian product against the oracle (1e-5,
rows (zone, species, output, bin i) over the partner bins j; l = 1 blocks against their |P_1|
companions), the autograd path for J and H, and the argument checks."""
import numpy as np
import pytest

import oracle
import vx_inputs
from _metrics import worst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("j0", "chi0", "j1", "chi1")
TOL = 1e-5


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


def _edge_batch():
    eps = vx_inputs.energy_centres(13, 1.0, 300.0)
    rows = [(T, eta) for T in (0.3, 2.0, 40.0) for eta in (-30.0, -3.0, 0.0, 9.0, 19.99, 20.01, 45.0, 79.0)]
    st, J, H = vx_inputs.random_zones(len(rows), 31, n_bins=13)
    st[:, 0] = [a for a, _ in rows]
    st[:, 1] = [c for _, c in rows]
    return dict(eps=eps, n_mu=8, n_e=20, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)


def _cases():
    return {
        "w1": vx_inputs.make_batch(1),
        "w2": vx_inputs.make_batch(2),
        "w5ray": vx_inputs.make_batch(5, rays=[7]),
        "edge": _edge_batch(),
    }


def _seeds(shape, seed=0):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(size=shape) for k in KEYS}


@pytest.mark.parametrize("case", ["w1", "w2", "w5ray", "edge"])
def test_blocks_and_vjp_against_oracle(case):
    b = _cases()[case]
    st, J, H = b["state"], b["J"], b["H"]
    r = rates_for(b)
    g = _seeds(J.shape, seed=len(case))
    res = r.spectral(dev(st), dev(J), dev(H), grad_out={k: dev(v) for k, v in g.items()}, blocks=True, forward=True)
    assert r.check()
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], st, J, H, spectral=True, mag=True)
    blk = res["blocks"].cpu().numpy()
    e = worst(blk, ref["dsrc"], mag=ref["dsrc_abs"])  # rows (z, s, o, i) over j
    assert e <= TOL, f"blocks: {e:.3e}"
    # VJP: against the oracle's blocks contracted in FP64, measured against |blocks| . |g|
    gJ, gH = oracle.spectral_vjp(ref["dsrc"], b["species"], g["j0"], g["chi0"], g["j1"], g["chi1"])
    aJ, aH = oracle.spectral_vjp(ref["dsrc_abs"], b["species"], *(np.abs(g[k]) for k in KEYS))
    assert worst(res["grad_J"].cpu().numpy(), gJ, mag=aJ) <= TOL
    assert worst(res["grad_H"].cpu().numpy(), gH, mag=aH) <= TOL
    # the forward rates of the same pass
    mags = {"j0": None, "chi0": None, "j1": ref["j1_abs"], "chi1": ref["chi1_abs"]}
    for k in KEYS:
        assert worst(res[k].cpu().numpy(), ref[k], mag=mags[k]) <= TOL, k
    r.close()


def test_vjp_is_the_blocks_contracted():
    """The in-kernel vector-Jacobian product equals the kernel's own blocks contracted with the
    seeds (FP64 arithmetic on both sides, so agreement to ~1e-12)."""
    b = vx_inputs.make_batch(2)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    r = rates_for(b)
    g = _seeds(b["J"].shape, seed=7)
    res = r.spectral(st, J, H, grad_out={k: dev(v) for k, v in g.items()}, blocks=True)
    assert r.check()
    blk = res["blocks"].cpu().numpy()
    gJ, gH = oracle.spectral_vjp(blk, b["species"], g["j0"], g["chi0"], g["j1"], g["chi1"])
    aJ, aH = oracle.spectral_vjp(np.abs(blk), b["species"], *(np.abs(g[k]) for k in KEYS))
    assert worst(res["grad_J"].cpu().numpy(), gJ, mag=aJ) <= 1e-11
    assert worst(res["grad_H"].cpu().numpy(), gH, mag=aH) <= 1e-11
    r.close()


def test_autograd_gradients_for_spectra():
    """torch.autograd through VxRatesFn: the J and H gradients are the spectral VJP, and, the rates
    being affine in J and linear in H, they predict a finite change of the spectra exactly up to
    the FP32 rounding of the two forward evaluations."""
    from paper_1404_1719_gb300 import VxRatesFn
    b = vx_inputs.make_batch(1)
    r = rates_for(b)
    st = dev(b["state"])
    J = dev(b["J"]).requires_grad_(True)
    H = dev(b["H"]).requires_grad_(True)
    g = _seeds(b["J"].shape, seed=3)
    outs = VxRatesFn.apply(r, st, J, H)
    loss = sum((o * dev(g[k])).sum() for o, k in zip(outs, KEYS))
    gJ, gH = torch.autograd.grad(loss, (J, H))
    ref = r.spectral(st, J.detach(), H.detach(), grad_out={k: dev(v) for k, v in g.items()}, blocks=False)
    assert torch.equal(gJ, ref["grad_J"]) and torch.equal(gH, ref["grad_H"])
    rng = np.random.default_rng(5)
    dJ, dH = dev(rng.uniform(-0.05, 0.05, b["J"].shape)), dev(rng.uniform(-0.05, 0.05, b["H"].shape))
    with torch.no_grad():
        moved = VxRatesFn.apply(r, st, J + dJ, H + dH)
        lhs = sum(((m - o) * dev(g[k])).sum() for m, o, k in zip(moved, outs, KEYS)).item()
        rhs = ((gJ * dJ).sum() + (gH * dH).sum()).item()
        mag = sum((dev(np.abs(g[k])) * (m.abs() + o.abs())).sum() for m, o, k in zip(moved, outs, KEYS)).item()
    assert abs(lhs - rhs) <= 1e-5 * mag
    # state gradients still flow when only the state requires them
    st2 = st.clone().requires_grad_(True)
    outs2 = VxRatesFn.apply(r, st2, J.detach(), H.detach())
    gs, = torch.autograd.grad(sum((o * dev(g[k])).sum() for o, k in zip(outs2, KEYS)), (st2,))
    assert torch.isfinite(gs).all() and gs.abs().sum() > 0
    r.close()


def test_invalid_zone_gives_nan_blocks_and_flag():
    b = vx_inputs.make_batch(1)
    st = b["state"].copy()
    st[5, 0] = -1.0  # T <= 0
    r = rates_for(b)
    g = _seeds(b["J"].shape)
    res = r.spectral(dev(st), dev(b["J"]), dev(b["H"]), grad_out={k: dev(v) for k, v in g.items()})
    assert not r.check()
    blk = res["blocks"].cpu().numpy()
    assert np.all(np.isnan(blk[5])) and np.all(np.isfinite(np.delete(blk, 5, axis=0)))
    assert np.all(np.isnan(res["grad_J"].cpu().numpy()[5])) and np.all(np.isnan(res["grad_H"].cpu().numpy()[5]))
    r.close()


def test_spectral_argument_checks():
    from paper_1404_1719_gb300 import capi
    b = vx_inputs.make_batch(1)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    r = rates_for(b)
    bt = r._batch(st, J, H, None)
    gJ = torch.empty_like(J)
    with pytest.raises(capi.VxError) as e:  # nothing requested
        capi.vx_rates_spectral(r.handle, bt, None, None, None, None, None)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    with pytest.raises(capi.VxError) as e:  # grad_J without grad_H
        capi.vx_rates_spectral(r.handle, bt, capi.vx_out(None, None, None, None, None), gJ.data_ptr(), None, None, None)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    with pytest.raises(capi.VxError) as e:  # VJP without seeds
        capi.vx_rates_spectral(r.handle, bt, None, gJ.data_ptr(), gJ.data_ptr(), None, None)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    r.close()
    r64 = rates_for(b, precision="fp64")
    with pytest.raises(capi.VxError) as e:
        r64.spectral(st, J, H)
    assert e.value.status == capi.VX_ERR_UNSUPPORTED
    r64.close()
