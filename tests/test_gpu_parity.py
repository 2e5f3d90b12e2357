"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: 1e-12 for the plain FP64 form, 1e-5 for the mixed form, measured per output row
(zone, species) over the energy bins, normwise and elementwise on entries >= 1e-3 of the row max.
"""
import numpy as np
import pytest

import oracle
import vx_inputs
from _metrics import magnitudes, row_errors, worst

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


def make(b, precision, **kw):
    from paper_1404_1719_gb300 import PairRates
    return PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"], precision=precision, **kw)


def run_pair(b, precision, zones=None, **kw):
    st, J, H = b["state"], b["J"], b["H"]
    if zones is not None:
        st, J, H = st[zones], J[zones], H[zones]
    rates = make(b, precision, **kw)
    out = rates.evaluate(dev(st), dev(J), dev(H), phi=True)
    ok = rates.check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    rates.close()
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], st, J, H, phi=True, mag=True)
    return got, ref, ok


def err(got, ref, k):
    """Worst error of output k; sums whose terms change sign (l = 1) are measured against the
    same sum of absolute values (their rounding bound), the others against their own values."""
    return worst(got[k], ref[k], mag=magnitudes(ref).get(k))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("workload", [1, 2])
def test_parity_small_workloads(workload, precision):
    b = vx_inputs.make_batch(workload)
    got, ref, ok = run_pair(b, precision)
    assert ok
    tol = TOL[precision]
    for k in KEYS:
        e = err(got, ref, k)
        assert e <= tol, f"{k}: {e:.3e} > {tol}"
    # raw kernel dump: rows (zone, dir, l, i) over j
    assert err(got, ref, "phi") <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_degenerate_ray(precision):
    """One ray of the 3-D-scale workload: eta_e up to ~63, 16 x 48 quadrature."""
    b = vx_inputs.make_batch(5, rays=[7])
    got, ref, ok = run_pair(b, precision)
    assert ok
    for k in KEYS:
        assert err(got, ref, k) <= TOL[precision], k
    assert err(got, ref, "phi") <= TOL[precision]


def _edge_batch():
    eps = vx_inputs.energy_centres(13, 1.0, 300.0)
    rows = []
    for T in (0.3, 1.0, 7.0, 40.0):
        for eta in (-45.0, -12.0, -3.0, 0.0, 2.5, 9.999, 19.999, 20.001, 25.0, 60.0, 79.5):
            rows.append((T, eta))
    st, J, H = vx_inputs.random_zones(len(rows), 21, n_bins=13)
    st[:, 0] = [r[0] for r in rows]
    st[:, 1] = [r[1] for r in rows]
    return dict(eps=eps, n_mu=8, n_e=20, species=np.array([0, 1, 2], np.int32), state=st, J=J, H=H)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_parity_edge_states(precision):
    """Negative and large degeneracy, both sides of the precision switch, cold and hot zones,
    an electron-energy node count without an unrolled instantiation."""
    b = _edge_batch()
    got, ref, ok = run_pair(b, precision)
    assert ok
    for k in KEYS:
        assert err(got, ref, k) <= TOL[precision], k
    assert err(got, ref, "phi") <= TOL[precision]


@pytest.mark.parametrize("species", [[2], [1, 0], [0, 2, 1]])
def test_species_subsets_and_order(species):
    b = vx_inputs.make_batch(1, rays=[0])
    sp = np.array(species, np.int32)
    st, J, H = vx_inputs.random_zones(24, 3, n_bins=17, n_species=len(sp))
    bb = dict(eps=b["eps"], n_mu=8, n_e=16, species=sp, state=st, J=J, H=H)
    got, ref, ok = run_pair(bb, "mixed")
    assert ok
    for k in KEYS:
        assert err(got, ref, k) <= 1e-5


def test_invalid_state_raises_flag_and_spares_other_zones():
    from paper_1404_1719_gb300 import capi
    b = vx_inputs.make_batch(1, rays=[0])
    st = b["state"][:6].copy()
    st[2, 0] = -1.0        # T <= 0
    st[4, 1] = 95.0        # |eta| beyond the supported range
    rates = make(b, "mixed")
    out = rates.evaluate(dev(st), dev(b["J"][:6]), dev(b["H"][:6]))
    assert capi.vx_rates_check(rates.handle, torch.cuda.current_stream().cuda_stream) == capi.VX_ERR_NUMERIC
    assert rates.check()  # the flag is cleared by the read
    j0 = out["j0"].cpu().numpy()
    assert np.all(np.isnan(j0[[2, 4]])) and np.all(np.isfinite(j0[[0, 1, 3, 5]]))
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], st[[0, 1, 3, 5]], b["J"][[0, 1, 3, 5]],
                          b["H"][[0, 1, 3, 5]], mag=True)
    assert worst(j0[[0, 1, 3, 5]], ref["j0"]) <= 1e-5  # l = 0: no cancellation
    rates.close()


def test_host_argument_checks():
    from paper_1404_1719_gb300 import capi
    b = vx_inputs.make_batch(1, rays=[0])
    rates = make(b, "mixed")
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    Z = st.shape[0]
    with pytest.raises(ValueError):  # host offsets that do not cover the zones: caught before the C call
        rates.evaluate(st, J, H, ray_offsets=[0, 10, 20])
    import ctypes
    host_offs = np.array([0, Z], np.int32)
    bt = capi.vx_batch(n_rays=1, n_zones=Z, ray_offsets=host_offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                       state=st.data_ptr(), J=J.data_ptr(), H=H.data_ptr())
    good = rates._alloc(Z)
    o = capi.vx_out(*(good[k].data_ptr() for k in KEYS), None)
    with pytest.raises(capi.VxError) as e:  # offsets in host memory: the device calls take device offsets
        capi.vx_rates_eval(rates.handle, bt, o, 0)
    assert e.value.status == capi.VX_ERR_INVALID_ARG and "ray_offsets" in str(e.value)
    with pytest.raises(ValueError):  # a caller-supplied output of the wrong shape
        rates.evaluate(st, J, H, out={k: torch.empty(3, dtype=torch.float64, device="cuda") for k in KEYS})
    bt = capi.vx_batch(n_rays=1, n_zones=st.shape[0], ray_offsets=None, state=st.data_ptr(), J=J.data_ptr(),
                       H=H.data_ptr())
    host = np.zeros(st.shape[0] * 3 * 17)
    o = capi.vx_out(host.ctypes.data, host.ctypes.data, host.ctypes.data, host.ctypes.data, None)
    with pytest.raises(capi.VxError) as e:  # host memory as an output
        capi.vx_rates_eval(rates.handle, bt, o, 0)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    empty = torch.empty((0, 4), dtype=torch.float64, device="cuda")
    rates.evaluate(empty, torch.empty((0, 3, 17), dtype=torch.float64, device="cuda"),
                   torch.empty((0, 3, 17), dtype=torch.float64, device="cuda"))
    assert rates.check()
    rates.close()


def test_device_ray_offsets_validated_on_the_device():
    """ray_offsets are device memory: a valid partition passes, an invalid one raises the device
    flag (VX_ERR_NUMERIC) while every zone is still evaluated (the rates do not depend on rays)."""
    from paper_1404_1719_gb300 import capi
    b = vx_inputs.make_batch(1, rays=[0])
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    Z = st.shape[0]
    for graph in (False, True):
        rates = make(b, "mixed", graph=graph)
        ref = rates.evaluate(st, J, H)
        ref = {k: v.clone() for k, v in ref.items()}
        good = torch.tensor([0, 20, 20, Z], dtype=torch.int32, device="cuda")
        out = rates.evaluate(st, J, H, ray_offsets=good)
        assert rates.check()
        for k in KEYS:
            assert torch.equal(out[k], ref[k])
        for bad in ([0, 30, 20, Z], [1, 20, 30, Z], [0, 20, 30, Z - 1]):
            out = rates.evaluate(st, J, H, ray_offsets=torch.tensor(bad, dtype=torch.int32, device="cuda"))
            status = capi.vx_rates_check(rates.handle, torch.cuda.current_stream().cuda_stream)
            assert status == capi.VX_ERR_NUMERIC and "invalid ray offsets" in capi.vx_last_error()
            for k in KEYS:
                assert torch.equal(out[k], ref[k])
        assert rates.check()
        rates.close()


def test_graph_replay_is_bitwise_deterministic():
    b = vx_inputs.make_batch(2)
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    ra = make(b, "mixed", graph=True)
    rb = make(b, "mixed", graph=False)
    a1 = ra.evaluate(st, J, H)
    a1 = {k: v.clone() for k, v in a1.items()}
    a2 = ra.evaluate(st, J, H)
    c = rb.evaluate(st, J, H)
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(a1[k], a2[k]) and torch.equal(a1[k], c[k]), k
    ra.close()
    rb.close()


def test_ragged_rays_full_size_sampled():
    """2048 rays of 300..550 zones in one launch, graph-captured; sampled zones against the oracle."""
    b = vx_inputs.make_batch(3)
    Z = b["state"].shape[0]
    rates = make(b, "mixed", graph=True)
    out = rates.evaluate(dev(b["state"]), dev(b["J"]), dev(b["H"]), ray_offsets=b["ray_offsets"])
    assert rates.check()
    rng = np.random.default_rng(3)
    offs = b["ray_offsets"]
    pick = np.unique(np.concatenate([rng.integers(0, Z, 24), offs[1:-1][:4], offs[1:][-3:] - 1, [0, Z - 1]]))
    ref = oracle.evaluate(b["eps"], b["n_mu"], b["n_e"], b["species"], b["state"][pick], b["J"][pick], b["H"][pick],
                          mag=True)
    got = {k: out[k][torch.as_tensor(pick, device="cuda")].cpu().numpy() for k in KEYS}
    for k in KEYS:
        assert err(got, ref, k) <= 1e-5, k
    rates.close()


def test_autotune_picks_a_variant_and_caches_it(tmp_path, monkeypatch):
    """VX_AUTOTUNE times both register budgets on the first batch, writes the choice to the JSON
    file named by VX_AUTOTUNE_CACHE, and a second handle reads it back; results stay within the
    mixed tolerance of an untuned handle."""
    import json
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("VX_AUTOTUNE_CACHE", str(cache))
    b = vx_inputs.make_batch(3, rays=range(96))  # ~41k zones: more than the tuning sample
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    r1 = make(b, "mixed", autotune=True)
    # with the batch's ray offsets: the tuning sample (a prefix of the zones) must not trip the
    # device-side check of the offsets
    o1 = r1.adjoint(st, J, H, jacobian=True, forward=True, ray_offsets=b["ray_offsets"])
    assert r1.check()
    data = json.loads(cache.read_text())
    (key, val), = data.items()
    assert "kind=tangents" in key and val["minb"] in (2, 3) and val["ms_b2"] > 0 and val["ms_b3"] > 0
    r2 = make(b, "mixed", autotune=True)
    o2 = r2.adjoint(st, J, H, jacobian=True, forward=True)
    r0 = make(b, "mixed")
    o0 = r0.adjoint(st, J, H, jacobian=True, forward=True)
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(o1[k], o2[k])
        assert worst(o1[k].cpu().numpy(), o0[k].cpu().numpy()) <= 2e-6
    for r in (r0, r1, r2):
        r.close()
