"""Pins of the collision oracle (Sec. 3.3): the collision energy's closed form and
finite-difference gradient, its cancellation outside the neighbouring body, the
detection against a point-in-body test of two overlapping cells, a plain double
loop on a small case, and the effect on a time step."""
import numpy as np
import pytest

from oracle import collision as Co
from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

DT = 0.1
WCOL = 2000.0


def _model(n=66):
    rest, tris = W.discocyte(n)
    return O.Model(rest, tris, W.material_vector(), DT), rest, tris


def test_collision_energy_closed_form_and_cancellation():
    m, rest, _ = _model()
    col = np.zeros((m.n, 4))
    nrm = np.array([0.6, 0.0, 0.8])
    col[5, :3] = nrm
    col[5, 3] = np.dot(nrm, rest[5]) + 0.01  # vertex 5 lies 0.01 um behind the plane
    col[7, :3] = nrm
    col[7, 3] = np.dot(nrm, rest[7]) - 0.02  # vertex 7 is outside: no term
    E, g = m.energy_collision(rest, col, WCOL)
    assert E == pytest.approx(0.5 * WCOL * 0.01 ** 2, rel=1e-12)
    assert np.allclose(g[5], -WCOL * 0.01 * nrm, rtol=1e-12)
    assert np.abs(np.delete(g, 5, axis=0)).max() == 0.0
    # continuous at the plane: the term vanishes as the vertex reaches it
    x = rest.copy()
    x[5] += 0.01 * nrm
    assert m.energy_collision(x, col, WCOL)[0] == pytest.approx(0.0, abs=1e-18)


def test_collision_gradient_matches_finite_differences():
    m, rest, _ = _model()
    rng = np.random.default_rng(1)
    x = rest + 0.02 * m.lbar * rng.standard_normal(rest.shape)
    y = x + 0.01 * m.lbar * rng.standard_normal(rest.shape)
    col = np.zeros((m.n, 4))
    for i in range(0, m.n, 3):
        nv = rng.standard_normal(3)
        nv /= np.linalg.norm(nv)
        col[i, :3] = nv
        col[i, 3] = np.dot(nv, x[i]) + rng.uniform(-0.05, 0.05)  # some in, some out
    mk = W.material_vector(k_vol=0.0)  # exact gradients elsewhere (no linearised volume projection)
    m2 = O.Model(rest, W.discocyte(66)[1], mk, DT)
    E, G = m2.objective_col(x, y, col, WCOL)
    h = 1e-6 * m.lbar
    fd = np.zeros_like(x)
    for i in range(m.n):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            fd[i, c] = (m2.objective_col(xp, y, col, WCOL)[0] - m2.objective_col(xm, y, col, WCOL)[0]) / (2 * h)
    assert np.abs(fd - G).max() <= 1e-6 * np.abs(G).max()


def _inside(x_pts, xb, tris):
    """Point-in-closed-surface by the winding number (solid angle / 4 pi)."""
    a, b, c = (xb[tris[:, k]][None] - x_pts[:, None] for k in range(3))
    la, lb, lc = (np.linalg.norm(v, axis=-1) for v in (a, b, c))
    num = np.einsum("pti,pti->pt", a, np.cross(b, c))
    den = la * lb * lc + (a * b).sum(-1) * lc + (a * c).sum(-1) * lb + (b * c).sum(-1) * la
    return (2 * np.arctan2(num, den)).sum(1) / (4 * np.pi) > 0.5


def test_detection_agrees_with_point_in_body():
    rest, tris = W.discocyte(258)
    xa = rest.copy()
    xb = rest + np.array([6.5, 0.3, 0.1])  # the rims overlap by ~1.3 um
    planes = Co.detect([(np.stack([xa, xb]), tris)], cutoff=1.0)[0]
    pa = planes[0]
    has = np.abs(pa[:, :3]).sum(1) > 0
    assert has.sum() > 10
    pen = pa[:, 3] - (pa[:, :3] * xa).sum(1) > 0
    inside = _inside(xa, xb, tris)
    # every vertex of A inside B within the cutoff of B's surface is detected as penetrating,
    # and the tangent-plane test agrees with the exact inside test on nearly all of them
    near = has
    agree = (pen[near] == inside[near]).mean()
    assert agree >= 0.95, agree
    assert not has[xa[:, 0] < 0].any()  # the far side of A sees nothing
    assert np.allclose(np.linalg.norm(pa[has, :3], axis=1), 1.0)


def test_detection_matches_double_loop():
    rest, tris = W.discocyte(66)
    rng = np.random.default_rng(3)
    xs = np.stack([rest, rest + [5.5, 0.5, 0.2], rest + [2.0, 5.0, -0.3]]) + 0.01 * rng.standard_normal((3, 66, 3))
    planes = Co.detect([(xs, tris)], cutoff=1.2)[0].reshape(-1, 4)
    from oracle.ibm import vertex_area_normal
    nrm = np.concatenate([vertex_area_normal(xs[c], tris)[1] for c in range(3)])
    X = xs.reshape(-1, 3)
    for i in range(len(X)):
        best, bd = -1, np.inf
        for j in range(len(X)):
            if j // 66 == i // 66:
                continue
            d = np.sum((X[i] - X[j]) ** 2)
            if d <= 1.2 ** 2 and d < bd:
                best, bd = j, d
        if best < 0:
            assert (planes[i] == 0).all()
        else:
            assert np.allclose(planes[i, :3], nrm[best]) and planes[i, 3] == pytest.approx(nrm[best] @ X[best])


def test_collision_step_pushes_cells_apart_and_far_cells_are_unaffected():
    m, rest, tris = _model(258)
    xs = np.stack([rest, rest + [6.8, 0.0, 0.0]])
    v = np.zeros_like(xs)
    f = np.zeros_like(xs)
    planes = Co.detect([(xs, tris)], cutoff=1.0)[0]
    opts = O.make_opts(tol=1e-9, max_iter=200)
    x1, _, st = m.step_batch(xs, v, f, opts, col=planes, wcol=WCOL)
    x0, _, _ = m.step_batch(xs, v, f, opts)
    depth = lambda x: np.clip(planes[..., 3] - (planes[..., :3] * x).sum(-1), 0, None).sum()
    # one 0.1 us step moves a vertex by about (h^2 / m) w_col d / (1 + h^2 w_col / m), ~5 % of
    # its depth; without the term the cells do not separate at all
    assert depth(xs) > 0 and depth(x1) < 0.97 * depth(xs) and depth(x1) < depth(x0) - 0.02 * depth(xs)
    assert all(s.status == 0 for s in st)
    # cells out of reach: the planes are empty and the step is the plain step, bit for bit
    far = np.stack([rest, rest + [30.0, 0.0, 0.0]])
    pf = Co.detect([(far, tris)], cutoff=1.0)[0]
    assert (pf == 0).all()
    a, _, _ = m.step_batch(far, v, f, opts, col=pf, wcol=WCOL)
    b, _, _ = m.step_batch(far, v, f, opts)
    assert np.array_equal(a, b)
