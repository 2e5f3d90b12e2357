"""The allocation-free entry point vx_rates_eval_noalloc, called through the C ABI.

It serves callers that must not have the library allocate device memory (their memory belongs
to their own pool, or their time step cannot afford the synchronisation of cudaMalloc/cudaFree).
Its rates must match those of vx_rates_eval on a mixed-precision handle within the mixed
tolerance, call after call, although every call reuses the same fixed device scratch.
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

import vx_inputs
from _metrics import worst

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
KEYS = ("j0", "chi0", "j1", "chi1")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def config(capi, b, keep):
    eps = np.ascontiguousarray(b["eps"], dtype=np.float64)
    sp = np.ascontiguousarray(b["species"], dtype=np.int32)
    keep += [eps, sp]
    return capi.vx_config(n_bins=len(eps), eps=eps.ctypes.data_as(capi._dp), weights=None, n_mu=b["n_mu"],
                          n_e=b["n_e"], n_species=len(sp), species=sp.ctypes.data_as(capi._ip), sin2w=0.23,
                          g2=1.0, norm=1.0, eta_fp64=0.0, prec=capi.VX_PREC_MIXED, flags=0)


def noalloc(capi, b, keep, free_bytes=None):
    """One call; with free_bytes (a list) it also records the device's free memory just before and
    just after the call (inputs and outputs are allocated beforehand)."""
    st, J, H = dev(b["state"]), dev(b["J"]), dev(b["H"])
    keep += [st, J, H]
    Z, S, N = J.shape
    out = {k: torch.full((Z, S, N), float("nan"), dtype=torch.float64, device="cuda") for k in KEYS}
    batch = capi.vx_batch(n_rays=1, n_zones=Z, ray_offsets=None, state=st.data_ptr(), J=J.data_ptr(), H=H.data_ptr())
    o = capi.vx_out(*(out[k].data_ptr() for k in KEYS), None)
    cfg = config(capi, b, keep)
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    capi.vx_rates_eval_noalloc(cfg, batch, o, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if free_bytes is not None:
        free_bytes.append((before, torch.cuda.mem_get_info()[0]))
    return out


def with_handle(b):
    from paper_1404_1719_gb300 import PairRates
    r = PairRates(b["eps"], b["n_mu"], b["n_e"], species=b["species"])
    res = r.evaluate(dev(b["state"]), dev(b["J"]), dev(b["H"]))
    assert r.check()
    out = {k: v.cpu().numpy() for k, v in res.items()}
    r.close()
    return out


def test_noalloc_matches_handle_on_consecutive_calls():
    from paper_1404_1719_gb300 import capi
    keep = []
    # calls in a row with different grids and quadratures: each rebuilds the shared table. After
    # the first (which also loads the kernels), a call leaves the device's free memory unchanged.
    free = []
    for n, b in enumerate((vx_inputs.make_batch(2), vx_inputs.make_batch(1), vx_inputs.make_batch(5, rays=[7]))):
        got = noalloc(capi, b, keep, free if n else None)
        ref = with_handle(b)
        for k in KEYS:
            g = got[k].cpu().numpy()
            assert np.all(np.isfinite(g)), k
            assert worst(g, ref[k]) <= 1e-5, k
    assert free and all(a == b for a, b in free), free


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1404_1719_gb300 import capi
    keep = []
    b = vx_inputs.make_batch(1, rays=[0])
    b = dict(b, eps=vx_inputs.energy_centres(25, 1.0, 300.0), J=np.zeros((64, 3, 25)), H=np.zeros((64, 3, 25)))
    with pytest.raises(capi.VxError) as e:
        noalloc(capi, b, keep)
    assert e.value.status == capi.VX_ERR_UNSUPPORTED and "at most 24 bins" in str(e.value)
