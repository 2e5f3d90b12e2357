"""C ABI checks that need no GPU: the library builds for sm_103a, loads, exports every entry point
include/*.h declares, and rejects invalid configurations on the host before any CUDA call.
Also checks that the product package is independent of the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1404_1719_gb300 import _build, capi as c
    _build.build()
    return c


def header_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(vx_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(capi):
    names = header_functions()
    assert len(names) >= 8
    lib = capi.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(capi.SYMBOLS) == set(names)


def test_status_strings(capi):
    assert capi.vx_status_string(capi.VX_OK) == "VX_OK"
    assert capi.vx_status_string(capi.VX_ERR_NUMERIC) == "VX_ERR_NUMERIC"


def _cfg(capi, keep, **over):
    eps = np.geomspace(1, 300, 17)
    sp = np.array([0, 1, 2], np.int32)
    d = dict(n_bins=17, eps=eps, weights=None, n_mu=16, n_e=32, species=sp, n_species=3, sin2w=0.23, g2=1.0,
             norm=1.0, eta_fp64=0.0, prec=capi.VX_PREC_MIXED, flags=0)
    d.update(over)
    keep.extend([d["eps"], d["species"], d["weights"]])
    return capi.vx_config(
        n_bins=d["n_bins"], eps=d["eps"].ctypes.data_as(capi._dp) if d["eps"] is not None else None,
        weights=d["weights"].ctypes.data_as(capi._dp) if d["weights"] is not None else None,
        n_mu=d["n_mu"], n_e=d["n_e"], n_species=d["n_species"],
        species=d["species"].ctypes.data_as(capi._ip) if d["species"] is not None else None,
        sin2w=d["sin2w"], g2=d["g2"], norm=d["norm"], eta_fp64=d["eta_fp64"], prec=d["prec"], flags=d["flags"])


@pytest.mark.parametrize("over", [
    dict(n_bins=1), dict(n_bins=32), dict(eps=np.geomspace(300, 1, 17)), dict(eps=np.r_[0.0, np.geomspace(1, 300, 16)]),
    dict(n_mu=1), dict(n_mu=65), dict(n_e=1), dict(n_e=65), dict(n_species=0), dict(species=np.array([0, 2, 2], np.int32)),
    dict(species=np.array([0, 2, 2], np.int32)), dict(n_species=1, species=np.array([0], np.int32)),
    dict(species=np.array([0, 1, 7], np.int32)), dict(sin2w=float("nan")), dict(eta_fp64=-1.0),
    dict(eta_fp64=50.0), dict(prec=9), dict(flags=64), dict(weights=-np.ones(17)),
])
def test_create_rejects_invalid_config(capi, over):
    keep = []
    cfg = _cfg(capi, keep, **over)
    h = ctypes.c_void_p()
    st = capi.lib().vx_rates_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == capi.VX_ERR_INVALID_ARG, capi.vx_last_error()
    assert not h.value
    assert capi.vx_last_error()


def test_null_arguments_are_rejected(capi):
    lib = capi.lib()
    h = ctypes.c_void_p()
    assert lib.vx_rates_create(None, ctypes.byref(h)) == capi.VX_ERR_INVALID_ARG
    assert lib.vx_rates_eval(None, None, None, None) == capi.VX_ERR_INVALID_ARG
    assert lib.vx_rates_check(None, None) == capi.VX_ERR_INVALID_ARG
    lib.vx_rates_destroy(None)
    assert lib.vx_rates_entries_per_zone(None) == 0


def test_btd_create_rejects_invalid_arguments(capi):
    """Checked on the host before any CUDA call."""
    lib = capi.lib()
    h = ctypes.c_void_p()
    for m, z, n in ((0, 4, 2), (129, 4, 2), (-3, 4, 2), (4, -1, 2), (4, 4, -1), (4, 4, 9)):
        assert lib.vx_btd_create(m, z, n, ctypes.byref(h)) == capi.VX_ERR_INVALID_ARG
        assert not h.value
    assert lib.vx_btd_create(4, 4, 2, None) == capi.VX_ERR_INVALID_ARG
    assert lib.vx_btd_solve(None, 1, 1, *([None] * 7)) == capi.VX_ERR_INVALID_ARG
    assert lib.vx_btd_check(None, None) == capi.VX_ERR_INVALID_ARG
    lib.vx_btd_destroy(None)


def test_product_package_does_not_use_the_oracle():
    pkg = os.path.join(ROOT, "paper_1404_1719_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert not re.search(r"\bimport\s+oracle\b|\bfrom\s+oracle\b|vx_oracle|libvx_oracle", txt), f


def test_library_is_built_for_sm_103a():
    from paper_1404_1719_gb300 import _build
    assert ["-gencode", "arch=compute_103a,code=sm_103a"] == _build.ARCH
