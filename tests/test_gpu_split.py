"""GPU split discrete rule (VX_QUAD_SPLIT): rates, Phi, Jacobian and spectral blocks against the
oracle's split rule (1e-5, the parity metric), the identity with the standard form where no Fermi
edge cuts an interval, and the accuracy gain against a converged reference."""
import numpy as np
import pytest

import oracle
import vx_inputs
from _metrics import magnitudes, worst

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
    rows = [(T, eta) for T in (0.3, 1.0, 7.0, 40.0)
            for eta in (-45.0, -12.0, -3.0, 0.0, 2.5, 9.999, 19.999, 20.001, 25.0, 60.0, 79.5)]
    st, J, H = vx_inputs.random_zones(len(rows), 23, n_bins=13)
    st[:, 0] = [r[0] for r in rows]
    st[:, 1] = [r[1] for r in rows]
    return dict(eps=eps, n_mu=8, n_e=20, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)


def _cases():
    return {"w1": vx_inputs.make_batch(1), "w2": vx_inputs.make_batch(2),
            "w5ray": vx_inputs.make_batch(5, rays=[7]), "edge": _edge_batch()}


@pytest.mark.parametrize("case", ["w1", "w2", "w5ray", "edge"])
def test_split_form_against_oracle(case):
    b = _cases()[case]
    st, J, H = b["state"], b["J"], b["H"]
    r = rates_for(b, split=True)
    out = r.evaluate(dev(st), dev(J), dev(H), phi=True)
    adj = r.adjoint(dev(st), dev(J), dev(H), jacobian=True, forward=True)
    blk = r.spectral(dev(st), dev(J), dev(H))["blocks"]
    assert r.check()
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], st, J, H, phi=True, jac=True,
                          spectral=True, mag=True, split=True, eta_split=20.0)
    mg = magnitudes(ref)
    for k in KEYS:
        assert worst(out[k].cpu().numpy(), ref[k], mag=mg[k]) <= TOL, k
        assert worst(adj[k].cpu().numpy(), ref[k], mag=mg[k]) <= TOL, k
    assert worst(out["phi"].cpu().numpy(), ref["phi"], mag=mg["phi"]) <= TOL
    gj, oj, ma = adj["jac"].cpu().numpy(), ref["jac"], ref["jac_abs"]
    for v in (0, 1):
        e = worst(np.swapaxes(gj[..., v], 2, 3), np.swapaxes(oj[..., v], 2, 3), mag=np.swapaxes(ma[..., v], 2, 3))
        assert e <= TOL, f"jacobian input {v}: {e:.3e}"
    assert worst(blk.cpu().numpy(), ref["dsrc"], mag=ref["dsrc_abs"]) <= TOL
    r.close()


def test_split_form_equals_standard_form_below_the_threshold():
    """Zones with |eta| <= 20 (the precision switch) keep the standard rule: the split handle
    returns the standard form's bits."""
    b = vx_inputs.make_batch(1)
    st = b["state"].copy()
    st[:, 1] = np.clip(st[:, 1], -20.0, 20.0)
    args = (dev(st), dev(b["J"]), dev(b["H"]))
    r0, r1 = rates_for(b), rates_for(b, split=True)
    a0 = r0.adjoint(*args, jacobian=True, forward=True)
    a1 = r1.adjoint(*args, jacobian=True, forward=True)
    assert r0.check() and r1.check()
    for k in KEYS + ("jac",):
        assert torch.equal(a0[k], a1[k]), k
    r0.close(), r1.close()


def test_split_form_is_more_accurate_at_high_degeneracy():
    """Cold, strongly degenerate zones on the 3-D-scale grid (21 bins, 16 x 48 quadrature), where
    the Fermi edge is sharp on the electron-energy interval: against a converged reference (the
    oracle's split rule with 512 energy nodes) the split form is at least 20x closer than the
    standard form (FP64 oracle at 48 nodes: 1.0e-4 against 1.0e-2)."""
    b = vx_inputs.make_batch(5, rays=[7])
    rows = [(T, eta) for T in (0.5, 1.0, 2.0) for eta in (30.0, 45.0, 60.0)]
    st, J, H = vx_inputs.random_zones(len(rows), 41, n_bins=len(b["eps"]))
    st[:, 0] = [a for a, _ in rows]
    st[:, 1] = [c for _, c in rows]
    ref = oracle.evaluate(b["eps"], b["n_mu"], 512, b["species"], st, J, H, split=True, eta_split=0.0)
    errs = {}
    for split in (False, True):
        r = rates_for(b, split=split)
        out = r.evaluate(dev(st), dev(J), dev(H))
        assert r.check()
        errs[split] = max(worst(out[k].cpu().numpy(), ref[k]) for k in ("j0", "chi0"))
        r.close()
    assert errs[True] <= 1e-3 and errs[True] * 20 <= errs[False], errs


def test_split_needs_an_even_node_count_and_the_mixed_form():
    from paper_1404_1719_gb300 import capi
    b = vx_inputs.make_batch(1)
    with pytest.raises(capi.VxError) as e:
        from paper_1404_1719_gb300 import PairRates
        PairRates(b["eps"], b["n_mu"], 15, species=b["species"], split=True)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    with pytest.raises(capi.VxError) as e:
        rates_for(b, split=True, precision="fp64")
    assert e.value.status == capi.VX_ERR_UNSUPPORTED
