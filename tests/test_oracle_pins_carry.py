"""Pins of the oracle's solve with L-BFGS pairs carried across time steps.

Carrying the pairs is an addition to the paper's Algorithm 1 (which starts each step's
quasi-Newton iteration with an empty history).  The pins check the oracle's two-loop
recursion with carried pairs against the recursive BFGS update of the inverse Hessian
written out densely (Nocedal & Wright Eq. 6.17, applied pair by pair from H0 = H~^-1),
which fixes the pairs' order and scaling; that the pair a solve appends is the step it
took; that an empty carry is the plain solve; and that a trajectory converges to the
same positions with or without the carried pairs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

DT = 0.1


@pytest.fixture(scope="module")
def m162():
    rest, tris = W.discocyte(162)
    return O.Model(rest, tris, W.material_vector(), DT)


def _state(m, seed, noise=0.5):
    rng = np.random.default_rng(seed)
    x = m.rest + rng.normal(0, 0.02, m.rest.shape)
    v = rng.normal(0, 1e-3, x.shape)
    f = rng.normal(0, noise, x.shape)
    return x, v, f


def _pairs(m, seed, k):
    """k history pairs of a real solve (max_iter k from y, empty history)."""
    x, v, f = _state(m, seed)
    y = m.first_guess(x, v, f)
    _, st, (S, Y) = m.solve_carry(y, y, None, O.make_opts(max_iter=k, tol=0.0))
    assert len(S) == k and st.iterations == k
    return S, Y


def _bfgs_inverse(m, S, Y):
    """H~^-1 updated by every pair, oldest first:
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / (s^T y)."""
    n = m.n
    H = np.kron(np.linalg.inv(m.hessian()), np.eye(3))  # AoS: index 3 i + c
    I = np.eye(3 * n)
    for s, y in zip(S, Y):
        s, y = s.reshape(-1), y.reshape(-1)
        rho = 1.0 / (s @ y)
        V = I - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


def test_empty_carry_is_the_plain_solve(m162):
    x, v, f = _state(m162, 1)
    y = m162.first_guess(x, v, f)
    o = O.make_opts(tol=1e-9, max_iter=100)
    xa, sa = m162.solve(y, y, o)
    xb, sb, (S, Y) = m162.solve_carry(y, y, None, o)
    assert np.array_equal(xa, xb)
    assert (sa.iterations, sa.evaluations, sa.status) == (sb.iterations, sb.evaluations, sb.status)
    assert 0 < len(S) <= 5 and S.shape == Y.shape == (len(S), m162.n, 3)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_first_direction_is_the_recursive_bfgs_update(m162, k):
    S, Y = _pairs(m162, 2, k)
    # another problem: new state and force, the carried pairs as history
    x, v, f = _state(m162, 3)
    y = m162.first_guess(x, v, f)
    x0 = y + np.random.default_rng(4).normal(0, 1e-3, y.shape)
    x1, st, _ = m162.solve_carry(x0, y, (S, Y), O.make_opts(max_iter=1, tol=0.0, fixed_alpha=1))
    assert st.iterations == 1
    _, g0, _ = m162.objective(x0, y)
    d = -_bfgs_inverse(m162, S, Y) @ g0.reshape(-1)
    step = (x1 - x0).reshape(-1)
    assert np.abs(step - d).max() <= 1e-9 * np.abs(d).max()
    # the pairs in the other order give another direction (the pin sees the order)
    if k > 1:
        d_rev = -_bfgs_inverse(m162, S[::-1], Y[::-1]) @ g0.reshape(-1)
        assert np.abs(d_rev - d).max() > 1e-4 * np.abs(d).max()


def test_appended_pair_is_the_step_taken(m162):
    S, Y = _pairs(m162, 5, 5)
    x, v, f = _state(m162, 6)
    y = m162.first_guess(x, v, f)
    x1, st, (S1, Y1) = m162.solve_carry(y, y, (S, Y), O.make_opts(max_iter=1, tol=0.0))
    assert st.iterations == 1 and len(S1) == 5
    _, g0, _ = m162.objective(y, y)
    _, g1, _ = m162.objective(x1, y)
    assert np.allclose(S1[-1], x1 - y, rtol=0, atol=1e-15 * np.abs(x1).max())
    assert np.allclose(Y1[-1], g1 - g0, rtol=0, atol=1e-12 * np.abs(g1 - g0).max())
    # the window keeps the newest lbfgs_m pairs: the oldest carried one dropped
    assert np.array_equal(S1[:-1], S[1:]) and np.array_equal(Y1[:-1], Y[1:])


def test_pairs_unchanged_when_accepted_at_the_first_iterate(m162):
    x, v, f = _state(m162, 7)
    y = m162.first_guess(x, v, f)
    o = O.make_opts(tol=1e-8, max_iter=100)
    xs, st, pairs = m162.solve_carry(y, y, None, o)
    assert st.iterations > 0
    x2, st2, (S2, Y2) = m162.solve_carry(xs, y, pairs, o)
    assert st2.iterations == 0 and np.array_equal(x2, xs)
    assert np.array_equal(S2, pairs[0]) and np.array_equal(Y2, pairs[1])


def test_failed_line_search_drops_the_pairs(m162):
    S, Y = _pairs(m162, 8, 3)
    x, v, f = _state(m162, 9)
    y = m162.first_guess(x, v, f)
    _, st, (S1, _) = m162.solve_carry(y + 0.5, y, (S, Y), O.make_opts(max_iter=5, tol=0.0, max_halvings=0, c1=0.99,
                                                                       c2=0.999))
    if st.status == 2:
        assert len(S1) == 0
    else:  # the full step passed every test: nothing to check here
        pytest.skip("line search did not fail")


def test_trajectory_with_carried_pairs_reaches_the_same_steps(m162):
    x = m162.rest.copy()
    v = np.zeros_like(x)
    f = W.shear_forces(x[None], m162.tris, np.array([500.0]))[0] + np.random.default_rng(11).normal(0, 0.5, x.shape)
    o = O.make_opts(tol=1e-10, max_iter=200)
    xa, va, sa = m162.trajectory(x, v, f, 12, o, carry_pairs=False)
    xb, vb, sb = m162.trajectory(x, v, f, 12, o, carry_pairs=True)
    assert all(s.status == 0 for s in sa + sb)
    assert np.abs(xa - xb).max() <= 1e-8 * m162.lbar
    assert np.abs(va - vb).max() <= 1e-7 * m162.lbar / DT
    # the carried curvature pays once the trajectory has settled (fixed force)
    ia = np.mean([s.iterations for s in sa[4:]])
    ib = np.mean([s.iterations for s in sb[4:]])
    assert ib < ia, (ia, ib)


def test_carry_rule_that_never_fires_is_the_plain_trajectory(m162):
    # carry_max_iters below every step's iteration count: no solve starts from carried
    # pairs, so the trajectory is the one without them, bit for bit
    x = m162.rest.copy()
    v = np.zeros_like(x)
    f = W.shear_forces(x[None], m162.tris, np.array([500.0]))[0]
    o = O.make_opts(tol=1e-9, max_iter=200)
    xa, va, sa = m162.trajectory(x, v, f, 6, o, carry_pairs=False)
    xb, vb, sb = m162.trajectory(x, v, f, 6, o, carry_pairs=True, carry_max_iters=-1)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert [s.iterations for s in sa] == [s.iterations for s in sb]
