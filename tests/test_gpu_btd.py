"""GPU block-tridiagonal Newton solve (vx_btd_*) against the banded-LU oracle: random and
transport-shaped systems over ragged rays (empty and one-zone rays included) for m from 1 to the
maximum 128, full-length rays at the benchmark's block size, the FP32-only result without
refinement, singular blocks, invalid offsets, argument checks, reproducibility and the host-buffer
path."""
import numpy as np
import pytest

from oracle import btd as obtd
from vx_inputs import btd as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-12  # normwise over a ray, after two FP64 refinement sweeps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build
    _build.build()


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def run(s, n_refine=2, solver=None):
    from paper_1404_1719_gb300 import BlockTridiagSolver
    Z = s["d"].shape[0]
    sv = solver or BlockTridiagSolver(s["m"], max(Z, 1), n_refine)
    x = sv.solve(dev(s["offsets"], torch.int32), dev(s["A"]), dev(s["B"]), dev(s["C"]), dev(s["d"]))
    ok = sv.check()
    out = x.cpu().numpy()
    if solver is None:
        sv.close()
    return out, ok


def ray_errors(x, ref, offsets):
    errs = []
    for r in range(len(offsets) - 1):
        a, b = offsets[r], offsets[r + 1]
        if b > a:
            errs.append(np.abs(x[a:b] - ref[a:b]).max() / np.abs(ref[a:b]).max())
    return max(errs)


@pytest.mark.parametrize("m", [1, 2, 7, 32, 33, 42, 63, 64, 65, 84, 96, 97, 128])  # every register-tile size and its edges
def test_random_systems_against_oracle(m):
    s = gen.random_system([5, 0, 1, 9, 17, 2], m, seed=m)
    x, ok = run(s)
    assert ok
    ref = obtd.solve(s["A"], s["B"], s["C"], s["d"], s["offsets"])
    e = ray_errors(x, ref, s["offsets"])
    assert e <= TOL, f"m={m}: {e:.3e}"


@pytest.mark.parametrize("m", [2, 7, 33, 84, 97, 128])
def test_row_exchanges(m):
    """The equations of every zone shuffled (one row permutation applied to A_k, B_k, C_k and d_k):
    the solution is unchanged, but the dominant entries leave the diagonal, so partial pivoting
    exchanges rows in every block. Checked against the oracle and against the unshuffled solve."""
    s = gen.random_system([5, 0, 1, 9, 17, 2], m, seed=200 + m)
    ref = obtd.solve(s["A"], s["B"], s["C"], s["d"], s["offsets"])
    rng = np.random.default_rng(m)
    t = {k: s[k].copy() for k in ("A", "B", "C", "d")}
    for z in range(s["d"].shape[0]):
        p = rng.permutation(m)
        if m > 1 and np.all(p == np.arange(m)):
            p = np.roll(p, 1)
        for k in ("A", "B", "C", "d"):
            t[k][z] = t[k][z][p]
    t.update(offsets=s["offsets"], m=m)
    x, ok = run(t)
    assert ok
    e = ray_errors(x, ref, s["offsets"])
    assert e <= TOL, f"m={m}: {e:.3e}"
    assert e <= TOL and ray_errors(x, obtd.solve(t["A"], t["B"], t["C"], t["d"], t["offsets"]), s["offsets"]) <= TOL


@pytest.mark.parametrize("pair", [True, False])
def test_newton_systems_against_oracle(pair):
    s = gen.newton_system([40, 25, 0, 3, 1], n_bins=21, pair=pair, seed=1)
    assert s["m"] == (84 if pair else 42)
    x, ok = run(s)
    assert ok
    ref = obtd.solve(s["A"], s["B"], s["C"], s["d"], s["offsets"])
    assert ray_errors(x, ref, s["offsets"]) <= TOL


def test_full_length_rays_sampled():
    """Rays of 400 zones at m = 84, the benchmark's ray shape and launch configuration: two rays
    against the oracle, every ray through its FP64 residual."""
    s = gen.newton_system([400] * 6, n_bins=21, seed=0)
    x, ok = run(s)
    assert ok
    o = s["offsets"]
    ref = obtd.solve(s["A"], s["B"], s["C"], s["d"], o, rays=[0, 5])
    for r in (0, 5):
        a, b = o[r], o[r + 1]
        assert np.abs(x[a:b] - ref[a:b]).max() <= TOL * np.abs(ref[a:b]).max()
    res = s["d"] - obtd.apply(s["A"], s["B"], s["C"], x, o)
    assert np.abs(res).max() <= 1e-13 * np.abs(s["d"]).max()


@pytest.mark.parametrize("shuffle", [False, True])
def test_without_refinement_is_fp32_accurate(shuffle):
    """FP32 accuracy of the factors alone; shuffled: the equations of every zone permuted, so that
    only a sound pivot choice keeps the FP32 factorisation at this accuracy."""
    s = gen.newton_system([60, 30], n_bins=8, seed=2)
    ref = obtd.solve(s["A"], s["B"], s["C"], s["d"], s["offsets"])
    if shuffle:
        rng = np.random.default_rng(5)
        for z in range(s["d"].shape[0]):
            p = rng.permutation(s["m"])
            for k in ("A", "B", "C", "d"):
                s[k][z] = s[k][z][p]
    x0, ok0 = run(s, n_refine=0)
    x1, ok1 = run(s, n_refine=1)
    x2, ok2 = run(s, n_refine=2)
    assert ok0 and ok1 and ok2
    e0, e1, e2 = (ray_errors(x, ref, s["offsets"]) for x in (x0, x1, x2))
    assert 1e-9 < e0 < 1e-4, e0  # FP32 factorisation, no refinement
    assert e1 < e0 * 1e-3 and e2 <= TOL, (e0, e1, e2)


def test_singular_block_gives_nan_ray_and_flag():
    s = gen.random_system([4, 5, 3], 6, seed=3)
    o = s["offsets"]
    A, B, C = s["A"].copy(), s["B"].copy(), s["C"].copy()
    k = o[1] + 2  # ray 1, third zone: an all-zero block row with no coupling
    A[k] = 0.0
    B[k] = 0.0
    C[k] = 0.0
    A[k + 1] = 0.0
    C[k - 1] = 0.0
    x, ok = run(dict(s, A=A, B=B, C=C))
    assert not ok
    assert np.isnan(x[o[1]:o[2]]).all()
    ref = obtd.solve(A, B, C, s["d"], o, rays=[0, 2])
    for r in (0, 2):
        assert np.abs(x[o[r]:o[r + 1]] - ref[o[r]:o[r + 1]]).max() <= TOL * np.abs(ref[o[r]:o[r + 1]]).max()


def test_invalid_offsets_solve_nothing_and_flag():
    from paper_1404_1719_gb300 import BlockTridiagSolver
    s = gen.random_system([4, 6], 5, seed=4)
    sv = BlockTridiagSolver(5, 10, 2)
    for bad in ([0, 6, 4], [1, 4, 10], [0, 4, 9]):  # decreasing, not starting at 0, not ending at Z
        x = torch.full((10, 5), 7.0, dtype=torch.float64, device="cuda")
        sv.solve(dev(np.array(bad, np.int32), torch.int32), dev(s["A"]), dev(s["B"]), dev(s["C"]), dev(s["d"]), out=x)
        assert not sv.check()
        assert bool((x == 7.0).all())  # nothing written
    x = sv.solve(dev(s["offsets"], torch.int32), dev(s["A"]), dev(s["B"]), dev(s["C"]), dev(s["d"]))
    assert sv.check()  # the flag was cleared and a valid call passes
    sv.close()


def test_argument_checks():
    from paper_1404_1719_gb300 import BlockTridiagSolver, capi
    for m, z, n in ((0, 4, 2), (129, 4, 2), (4, -1, 2), (4, 4, -1), (4, 4, 9)):
        with pytest.raises(capi.VxError) as e:
            BlockTridiagSolver(m, z, n)
        assert e.value.status == capi.VX_ERR_INVALID_ARG
    s = gen.random_system([3, 2], 4, seed=5)
    sv = BlockTridiagSolver(4, 4, 1)
    off, A, B, C, d = dev(s["offsets"], torch.int32), dev(s["A"]), dev(s["B"]), dev(s["C"]), dev(s["d"])
    with pytest.raises(capi.VxError) as e:  # more zones than the handle was made for
        sv.solve(off, A, B, C, d)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    sv.close()
    sv = BlockTridiagSolver(4, 5, 1)
    with pytest.raises(capi.VxError) as e:  # x aliasing d
        sv.solve(off, A, B, C, d, out=d)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    with pytest.raises(capi.VxError) as e:
        capi.vx_btd_solve(sv.handle, 2, 5, off.data_ptr(), A.data_ptr(), None, C.data_ptr(), d.data_ptr(),
                          torch.empty_like(d).data_ptr())
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    # offsets in host memory (the rate calls' host-buffer convention): rejected before any launch
    host_off = s["offsets"].astype(np.int32)
    with pytest.raises(capi.VxError) as e:
        capi.vx_btd_solve(sv.handle, 2, 5, host_off.ctypes.data, A.data_ptr(), B.data_ptr(), C.data_ptr(),
                          d.data_ptr(), torch.empty_like(d).data_ptr())
    assert e.value.status == capi.VX_ERR_INVALID_ARG and "ray_offsets must be device memory" in str(e.value)
    host_x = np.zeros(d.shape)
    with pytest.raises(capi.VxError) as e:  # a host output
        capi.vx_btd_solve(sv.handle, 2, 5, off.data_ptr(), A.data_ptr(), B.data_ptr(), C.data_ptr(),
                          d.data_ptr(), host_x.ctypes.data)
    assert e.value.status == capi.VX_ERR_INVALID_ARG
    # a caller-supplied solution tensor of the wrong shape, type or place: caught in Python
    for bad in (torch.empty(4, 4, dtype=torch.float64, device="cuda"), torch.empty_like(d, dtype=torch.float32),
                torch.empty(d.shape, dtype=torch.float64)):
        with pytest.raises(ValueError):
            sv.solve(off, A, B, C, d, out=bad)
    torch.cuda.synchronize()
    assert sv.check()
    sv.close()


def test_reproducible_and_host_path():
    from paper_1404_1719_gb300 import BlockTridiagSolver
    s = gen.newton_system([30, 12], n_bins=6, seed=6)
    Z = s["d"].shape[0]
    sv = BlockTridiagSolver(s["m"], Z, 2)
    args = (dev(s["offsets"], torch.int32), dev(s["A"]), dev(s["B"]), dev(s["C"]), dev(s["d"]))
    x1 = sv.solve(*args).cpu()
    x2 = sv.solve(*args).cpu()
    assert torch.equal(x1, x2)
    host = [torch.from_numpy(np.ascontiguousarray(s[k])).pin_memory() for k in ("A", "B", "C", "d")]
    xh = sv.solve_host(torch.from_numpy(s["offsets"]).pin_memory(), *host)
    assert torch.equal(xh, x1)
    assert sv.check()
    sv.close()
