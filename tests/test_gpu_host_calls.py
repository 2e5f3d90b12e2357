"""Host-buffer calls (vx_rates_eval_host, vx_rates_adjoint_host, and the NES kernel's
vx_nes_eval_host, vx_nes_adjoint_host): the same bits as the device calls on a batch of three
staging chunks (both slots, a partial last chunk), from pinned and from pageable host memory, and
their argument checks."""
import numpy as np
import pytest

import vx_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("j0", "chi0", "j1", "chi1")
Z = 140_000  # > 2 chunks of 65,536 zones


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()


@pytest.fixture(scope="module")
def case():
    from paper_1404_1719_gb300 import PairRates
    eps = vx_inputs.energy_centres(11, 1.0, 300.0)
    st, J, H = vx_inputs.random_zones(Z, 77, n_bins=11)
    r = PairRates(eps, 8, 16, species=(0, 1, 2))
    yield r, st, J, H
    r.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_eval_host_matches_device_call(case):
    r, st, J, H = case
    ref = r.evaluate(_dev(st), _dev(J), _dev(H))
    pinned = [torch.from_numpy(x).pin_memory() for x in (st, J, H)]
    got = r.evaluate_host(*pinned)
    assert r.check()
    for k in KEYS:
        assert torch.equal(got[k], ref[k].cpu()), k
    got2 = r.evaluate_host(st, J, H)  # pageable numpy input
    for k in KEYS:
        assert torch.equal(got2[k], ref[k].cpu()), k


def test_adjoint_host_matches_device_call(case):
    r, st, J, H = case
    ref = r.adjoint(_dev(st), _dev(J), _dev(H), jacobian=True, forward=True)
    got = r.adjoint_host(st, J, H, forward=True)
    assert r.check()
    assert torch.equal(got["jac"], ref["jac"].cpu())
    for k in KEYS:
        assert torch.equal(got[k], ref[k].cpu()), k
    only = r.adjoint_host(st[:1000], J[:1000], H[:1000], forward=False)
    assert set(only) == {"jac"} and torch.equal(only["jac"], ref["jac"][:1000].cpu())


def test_host_call_argument_checks(case):
    from paper_1404_1719_gb300 import PairRates, capi
    r, st, J, H = case
    b, _ = r._host_batch(st[:10], J[:10], H[:10], None)
    with pytest.raises(capi.VxError) as e:
        capi.vx_rates_adjoint_host(r.handle, b, None, None)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    with pytest.raises(capi.VxError) as e:
        capi.vx_rates_eval_host(r.handle, b, capi.vx_out(None, None, None, None, None))
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    r64 = PairRates(vx_inputs.energy_centres(11, 1.0, 300.0), 8, 16, precision="fp64")
    with pytest.raises(capi.VxError) as e:
        r64.evaluate_host(st[:10], J[:10], H[:10])
    assert e.value.status == capi.VX_ERR_UNSUPPORTED
    r64.close()


def test_spectral_host_matches_device_call(monkeypatch):
    """Blocks, J/H gradients and rates through vx_rates_spectral_host equal the device call's bits,
    with 8 MiB staging slots so that a 3000-zone batch spans six chunks."""
    from paper_1404_1719_gb300 import PairRates
    monkeypatch.setenv("VX_HOST_SLOT_MB", "8")
    eps = vx_inputs.energy_centres(11, 1.0, 300.0)
    st, J, H = vx_inputs.random_zones(3000, 5, n_bins=11)
    rng = np.random.default_rng(2)
    g = {k: rng.normal(size=J.shape) for k in KEYS}
    r = PairRates(eps, 8, 16, species=(0, 1, 2))
    ref = r.spectral(_dev(st), _dev(J), _dev(H), grad_out={k: _dev(v) for k, v in g.items()}, blocks=True,
                     forward=True)
    got = r.spectral_host(st, J, H, grad_out=g, blocks=True, forward=True)
    assert r.check()
    for k in ("blocks", "grad_J", "grad_H") + KEYS:
        assert torch.equal(got[k], ref[k].cpu()), k
    r.close()


def test_nes_host_calls_match_device_calls(monkeypatch):
    """NES through 8 MiB staging slots: 1,753 zones per chunk at 11 bins, 3 species, so 5,000
    zones take three chunks."""
    from paper_1404_1719_gb300 import NesRates, capi
    monkeypatch.setenv("VX_HOST_SLOT_MB", "8")
    eps = vx_inputs.energy_centres(11, 1.0, 300.0)
    st, J, H = vx_inputs.random_zones(5000, 91, n_bins=11)
    r = NesRates(eps, 8, 24, species=(0, 1, 2))
    ref = r.adjoint(_dev(st), _dev(J), _dev(H), forward=True)
    pinned = [torch.from_numpy(x).pin_memory() for x in (st, J, H)]
    got = r.adjoint_host(*pinned, forward=True, ray_offsets=[0, 1200, 5000])
    for k in KEYS + ("jac",):
        assert torch.equal(got[k], ref[k].cpu()), k
    ref2 = r.evaluate(_dev(st), _dev(J), _dev(H))  # the forward kernel (its own instantiation)
    got2 = r.evaluate_host(st, J, H)  # pageable numpy arrays
    for k in KEYS:
        assert torch.equal(got2[k], ref2[k].cpu()), k
    assert r.check()
    with pytest.raises(capi.VxError):  # offsets that are not a partition, rejected on the host
        r.adjoint_host(*pinned, ray_offsets=[0, 6000, 5000])
    r.close()
