"""Pins of the block-tridiagonal oracle (oracle/btd.py) to what the mathematics fixes: closed-form
solutions, Cramer's rule, a manufactured solution whose right-hand side comes from index loops,
the block-diagonal special case, and ragged/empty rays. No GPU."""
import numpy as np
import pytest

from oracle import btd
from vx_inputs import btd as gen


def test_poisson_closed_form():
    """m = 1, blocks (-1, 2, -1), d = 1: the discrete Poisson problem, x_k = k (n + 1 - k) / 2 for
    k = 1..n."""
    n = 37
    A = -np.ones((n, 1, 1))
    B = 2 * np.ones((n, 1, 1))
    C = -np.ones((n, 1, 1))
    d = np.ones((n, 1))
    k = np.arange(1, n + 1)
    exact = k * (n + 1 - k) / 2.0
    for x in (btd.solve_ray(A, B, C, d), btd.solve_dense(A, B, C, d)):
        assert np.allclose(x[:, 0], exact, rtol=1e-13, atol=0)


def test_two_zone_cramer():
    """m = 1, two zones, A and C different: [[b0, c0], [a1, b1]] x = d by Cramer's rule. A swap of
    the sub- and super-diagonal blocks changes the answer."""
    a1, b0, b1, c0, d0, d1 = 0.3, 2.0, -1.5, 0.7, 1.25, -0.5
    A = np.array([[[99.0]], [[a1]]])  # A_0 multiplies nothing
    B = np.array([[[b0]], [[b1]]])
    C = np.array([[[c0]], [[99.0]]])  # nor does C_{n-1}
    d = np.array([[d0], [d1]])
    det = b0 * b1 - c0 * a1
    exact = np.array([(d0 * b1 - c0 * d1) / det, (b0 * d1 - a1 * d0) / det])
    assert np.allclose(btd.solve_ray(A, B, C, d)[:, 0], exact, rtol=1e-14)
    assert np.allclose(btd.solve_dense(A, B, C, d)[:, 0], exact, rtol=1e-14)


def _loop_product(A, B, C, x, offsets):
    """A_k x_{k-1} + B_k x_k + C_k x_{k+1}, written as plain index loops (brute force)."""
    Z, m = x.shape
    y = np.zeros((Z, m))
    for r in range(len(offsets) - 1):
        a, b = offsets[r], offsets[r + 1]
        for k in range(a, b):
            for i in range(m):
                s = 0.0
                for j in range(m):
                    s += B[k, i, j] * x[k, j]
                    if k > a:
                        s += A[k, i, j] * x[k - 1, j]
                    if k + 1 < b:
                        s += C[k, i, j] * x[k + 1, j]
                y[k, i] = s
    return y


def test_apply_matches_index_loops():
    s = gen.random_system([3, 0, 1, 4], 3, seed=2)
    x = np.random.default_rng(1).standard_normal(s["d"].shape)
    ref = _loop_product(s["A"], s["B"], s["C"], x, s["offsets"])
    assert np.allclose(btd.apply(s["A"], s["B"], s["C"], x, s["offsets"]), ref, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("m,lengths", [(1, [5, 1, 0, 9]), (3, [4, 2, 7]), (6, [1, 12, 0, 3])])
def test_manufactured_solution(m, lengths):
    """Choose x*, form d = M x* by index loops, solve: x* comes back (non-symmetric blocks, so a
    transposed block or a swapped neighbour would not)."""
    s = gen.random_system(lengths, m, seed=m)
    xs = np.random.default_rng(7).standard_normal(s["d"].shape)
    d = _loop_product(s["A"], s["B"], s["C"], xs, s["offsets"])
    x = btd.solve(s["A"], s["B"], s["C"], d, s["offsets"])
    assert np.allclose(x, xs, rtol=0, atol=1e-12 * np.abs(xs).max())


def test_manufactured_newton_system():
    s = gen.newton_system([6, 3], n_bins=4, seed=3)
    assert s["m"] == 16
    xs = np.random.default_rng(8).standard_normal(s["d"].shape)
    d = btd.apply(s["A"], s["B"], s["C"], xs, s["offsets"])
    x = btd.solve(s["A"], s["B"], s["C"], d, s["offsets"])
    assert np.abs(x - xs).max() <= 1e-11 * np.abs(xs).max()


def test_block_diagonal_reduces_to_independent_solves():
    s = gen.random_system([4, 3], 5, seed=4)
    A, C = np.zeros_like(s["A"]), np.zeros_like(s["C"])
    x = btd.solve(A, s["B"], C, s["d"], s["offsets"])
    ref = np.stack([np.linalg.solve(s["B"][k], s["d"][k]) for k in range(len(s["d"]))])
    assert np.allclose(x, ref, rtol=1e-13, atol=1e-15)


def test_banded_equals_dense_and_rays_are_independent():
    s = gen.random_system([5, 1, 6], 4, seed=5)
    o = s["offsets"]
    x = btd.solve(s["A"], s["B"], s["C"], s["d"], o)
    for r in range(3):
        a, b = o[r], o[r + 1]
        xd = btd.solve_dense(s["A"][a:b], s["B"][a:b], s["C"][a:b], s["d"][a:b])
        assert np.allclose(x[a:b], xd, rtol=1e-12, atol=1e-14)
    only = btd.solve(s["A"], s["B"], s["C"], s["d"], o, rays=[1])
    assert np.array_equal(only[o[1]:o[2]], x[o[1]:o[2]]) and np.isnan(only[:o[1]]).all()


def test_newton_generator_is_reproducible_by_ray():
    full = gen.newton_system([3, 5, 2], n_bins=3, seed=9)
    one = gen.newton_system([3, 5, 2], n_bins=3, seed=9, rays=[1])
    o = full["offsets"]
    for k in ("A", "B", "C", "d"):
        assert np.array_equal(one[k], full[k][o[1]:o[2]])
    # the ends of a ray couple to nothing
    assert not full["A"][o[0]].any() and not full["C"][o[1] - 1].any()
