"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a closed form, an
invariant, a printed value (tests/golden), a finite difference, a textbook
routine (scipy) or a brute-force search.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DT = 0.1  # us


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out[k] = [float(t) for t in v] if len(v) > 1 else float(v[0])
    return out


@pytest.fixture(scope="module")
def m642():
    rest, tris = W.discocyte(642)
    return O.Model(rest, tris, W.material_vector(), DT)


@pytest.fixture(scope="module")
def m66():
    rest, tris = W.discocyte(66)
    return O.Model(rest, tris, W.material_vector(), DT)


def deformed(model, amp=0.03, seed=0, affine=True):
    rng = np.random.default_rng(seed)
    X = model.rest
    A = np.eye(3) + (0.05 * rng.standard_normal((3, 3)) if affine else 0)
    return X @ A.T + amp * model.lbar * rng.standard_normal(X.shape)


def rot(seed):
    return W.random_rotations(np.random.default_rng(seed), 1)[0]


# ---------------------------------------------------------------------------------------
# rest geometry against the printed RBC dimensions (Sec. 1) and 1-D quadrature
# ---------------------------------------------------------------------------------------
def _profile_quadrature():
    D = W.DISCOCYTE_D
    r = np.linspace(0.0, D / 2, 400001)
    q = np.clip(1 - 4 * r ** 2 / D ** 2, 0, None)
    z = D * np.sqrt(q) * (W.ES_A0 + W.ES_A1 * r ** 2 / D ** 2 + W.ES_A2 * r ** 4 / D ** 4)
    V = np.trapezoid(2 * math.pi * r * 2 * z, r)
    dz = np.gradient(z, r)
    A = 2 * np.trapezoid(2 * math.pi * r * np.sqrt(1 + dz ** 2), r)
    return V, A, 2 * z[0], 2 * z.max()


def test_rest_shape_matches_printed_rbc():
    g = read_golden("rbc_rest_geometry.txt")
    V, A, t0, tmax = _profile_quadrature()
    assert abs(V - g["volume_um3"]) / g["volume_um3"] < 0.01
    assert abs(A - g["area_um2"]) / g["area_um2"] < 0.01
    assert abs(t0 - g["thickness_dimple_um"]) < 0.005
    assert abs(tmax - g["thickness_rim_um"]) < 0.01


@pytest.mark.parametrize("n", [258, 642, 2562])
def test_mesh_volume_area_converge_to_profile(n):
    V, A, _, _ = _profile_quadrature()
    rest, tris = W.discocyte(n)
    m = O.Model(rest, tris, W.material_vector(), DT)
    # an inscribed polyhedron under-estimates both, and the gap shrinks with refinement
    tol = {258: 0.035, 642: 0.015, 2562: 0.004}[n]
    assert V * (1 - tol) < m.V0 < V
    assert A * (1 - tol) < m.A0 < A * 1.001


def test_rest_volume_area_independent_formulae(m642):
    X, T = m642.rest, m642.tris
    tri = X[T]
    V = np.einsum("ti,ti->t", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0
    A = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    assert abs(m642.V0 - V) < 1e-12 * V
    assert abs(m642.A0 - A) < 1e-12 * A
    assert abs(m642.mtotal - 1000.0 * V) < 1e-9 * m642.mtotal
    assert abs(m642.masses().sum() - m642.mtotal) < 1e-9 * m642.mtotal


def test_volume_exact_on_polyhedra():
    # octahedron with unit circumradius: volume 4/3; cube of side 2: volume 8
    s, t = W.sphere_mesh(6)
    m = O.Model(s, t, W.material_vector(), DT)
    assert abs(m.volume(s) - 4.0 / 3.0) < 1e-14
    cube = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], float)
    faces = np.array([[0, 1, 3], [0, 3, 2], [4, 6, 7], [4, 7, 5], [0, 4, 5], [0, 5, 1],
                      [2, 3, 7], [2, 7, 6], [0, 2, 6], [0, 6, 4], [1, 5, 7], [1, 7, 3]], np.int32)
    mc = O.Model(cube, faces, W.material_vector(), DT)
    assert abs(mc.volume(cube) - 8.0) < 1e-13
    assert abs(mc.area(cube) - 24.0) < 1e-13


# ---------------------------------------------------------------------------------------
# zero energy / gradient at rest, rigid-motion invariance, conservation
# ---------------------------------------------------------------------------------------
def test_zero_energy_and_gradient_at_rest(m642):
    X = m642.rest
    scale = 5000.0 * m642.A0  # pN um, stiffness x area
    for name in ("energy_area", "energy_skalak", "energy_bend", "energy_vol"):
        e, g = getattr(m642, name)(X)
        assert abs(e) < 1e-14 * scale, name
        assert np.abs(g).max() < 1e-11 * 5000.0 * m642.lbar, name


@pytest.mark.parametrize("seed", [1, 2])
def test_rigid_motion_invariance(m642, seed):
    x = deformed(m642, seed=seed)
    Q, t = rot(seed + 10), np.array([31.0, -7.0, 55.0])
    y = x @ Q.T + t
    for name in ("energy_area", "energy_skalak", "energy_bend", "energy_vol"):
        e0, g0 = getattr(m642, name)(x)
        e1, g1 = getattr(m642, name)(y)
        assert abs(e1 - e0) <= 1e-9 * abs(e0) + 1e-12, name
        assert np.abs(g1 - g0 @ Q.T).max() <= 1e-8 * np.abs(g0).max(), name


def test_internal_forces_sum_and_torque_vanish(m642):
    x = deformed(m642, seed=3)
    _, g = m642.internal_energy(x)
    F = -g
    ref = np.abs(F).max() * len(F)
    assert np.abs(F.sum(0)).max() < 1e-11 * ref
    assert np.abs(np.cross(x - x.mean(0), F).sum(0)).max() < 1e-11 * ref * 10


# ---------------------------------------------------------------------------------------
# finite differences
# ---------------------------------------------------------------------------------------
def fd_grad(fun, x, h, idx):
    g = np.zeros(len(idx))
    for q, (i, c) in enumerate(idx):
        xp = x.copy(); xp[i, c] += h
        xm = x.copy(); xm[i, c] -= h
        g[q] = (fun(xp) - fun(xm)) / (2 * h)
    return g


@pytest.mark.parametrize("name", ["energy_area", "energy_skalak", "energy_bend"])
def test_gradients_match_finite_differences_all_coords(m66, name):
    x = deformed(m66, seed=4, amp=0.05)
    e, g = getattr(m66, name)(x)
    idx = [(i, c) for i in range(m66.n) for c in range(3)]
    fd = fd_grad(lambda z: getattr(m66, name)(z)[0], x, 1e-6 * m66.lbar, idx)
    ga = np.array([g[i, c] for i, c in idx])
    assert np.linalg.norm(fd - ga) <= 1e-7 * np.linalg.norm(ga)


@pytest.mark.parametrize("name", ["energy_area", "energy_skalak", "energy_bend"])
def test_gradients_match_finite_differences_642(m642, name):
    x = deformed(m642, seed=5)
    e, g = getattr(m642, name)(x)
    rng = np.random.default_rng(7)
    idx = [(int(i), int(c)) for i, c in zip(rng.integers(0, m642.n, 40), rng.integers(0, 3, 40))]
    fd = fd_grad(lambda z: getattr(m642, name)(z)[0], x, 1e-6 * m642.lbar, idx)
    ga = np.array([g[i, c] for i, c in idx])
    assert np.linalg.norm(fd - ga) <= 1e-7 * np.linalg.norm(ga)


def test_volume_gradient_is_exact_dV_dx(m66):
    x = deformed(m66, seed=6)
    gc = m66.volume_gradient(x)
    idx = [(i, c) for i in range(m66.n) for c in range(3)]
    fd = fd_grad(m66.volume, x, 1e-6 * m66.lbar, idx)
    ga = np.array([gc[i, c] for i, c in idx])
    assert np.linalg.norm(fd - ga) <= 1e-8 * np.linalg.norm(ga)


def test_volume_pd_gradient_vs_exact_shrinks_with_dV(m66):
    # The PD gradient w (x - p) of the volume term differs from dE/dx by a term of
    # relative size O(C): halving the volume error halves the mismatch.
    X = m66.rest
    rng = np.random.default_rng(8)
    dirn = rng.standard_normal(X.shape)
    rel = []
    for amp in (0.02, 0.01, 0.005):
        x = X * (1 + amp) + 1e-3 * dirn * m66.lbar
        e, g = m66.energy_vol(x)
        idx = [(i, c) for i in range(m66.n) for c in range(3)]
        fd = fd_grad(lambda z: m66.energy_vol(z)[0], x, 1e-7 * m66.lbar, idx)
        ga = np.array([g[i, c] for i, c in idx])
        rel.append(np.linalg.norm(fd - ga) / np.linalg.norm(ga))
    assert rel[0] < 0.1
    assert 1.6 < rel[0] / rel[1] < 2.4 and 1.6 < rel[1] / rel[2] < 2.4


# ---------------------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------------------
def _sl2_closed_isotropic(s):
    return 1.0 if s <= 2.0 else (s + math.sqrt(s * s - 4.0)) / 2.0


def test_sl2_projection_special_cases():
    for s in (0.3, 0.9, 1.0, 1.5, 2.0, 2.5, 4.0):
        assert abs(O.sl2_project(s, s) - _sl2_closed_isotropic(s)) < 1e-13 * max(1, s)
    # a point already on the manifold projects to itself
    for a in (1.0, 1.2, 3.0):
        assert abs(O.sl2_project(a, 1.0 / a) - a) < 1e-13 * a


def test_sl2_projection_matches_grid_search():
    rng = np.random.default_rng(11)
    grid = np.exp(np.linspace(np.log(1e-3), np.log(1e3), 2_000_001))
    for _ in range(60):
        s1 = rng.uniform(0.05, 5.0)
        s2 = rng.uniform(0.0, s1)
        a = O.sl2_project(s1, s2)
        phi = (grid - s1) ** 2 + (1 / grid - s2) ** 2
        ag = grid[np.argmin(phi)]
        phia = (a - s1) ** 2 + (1 / a - s2) ** 2
        assert phia <= phi.min() + 1e-12
        assert abs(a - ag) < 1e-4 * a
        assert abs(a ** 4 - s1 * a ** 3 + s2 * a - 1) < 1e-12 * (1 + s1 * a ** 3)  # stationarity


def test_skalak_valanis_landel_equals_invariant_form():
    # Sec. 2.1.3: with D = 0 and g dropped, f(l1) + f(l2) (shifted) equals the
    # printed (B/4)(I1^2/2 + I1 - I2) part of Skalak's density.
    rng = np.random.default_rng(12)
    B = 5.0
    for _ in range(50):
        l1, l2 = rng.uniform(0.3, 2.5, 2)
        I1 = l1 ** 2 + l2 ** 2 - 2
        I2 = l1 ** 2 * l2 ** 2 - 1
        lhs = O.skalak_f(l1, B, 0.0) + O.skalak_f(l2, B, 0.0)
        assert abs(lhs - B / 4 * (0.5 * I1 ** 2 + I1 - I2)) < 1e-12 * (1 + abs(lhs))
    # the correction term of the modified energy is D (l - 1)^4 / 4
    assert abs(O.skalak_f(1.5, B, 35.0) - O.skalak_f(1.5, B, 0.0) - 35.0 * 0.5 ** 4 / 4) < 1e-13


def test_drucker_stability_of_modified_skalak():
    # Sec. 2.1.3: f'' > 0; with B = 5, D = 35 the minimum is about 4.5 near l = 0.933.
    lam = np.linspace(0.05, 3.0, 5901)
    h = 1e-5
    f2 = np.array([(O.skalak_fp(l + h, 5, 35) - O.skalak_fp(l - h, 5, 35)) / (2 * h) for l in lam])
    assert f2.min() > 0
    i = np.argmin(f2)
    assert abs(f2[i] - 4.5) < 0.05 and abs(lam[i] - 0.933) < 0.01
    f2o = np.array([(O.skalak_fp(l + h, 5, 0) - O.skalak_fp(l - h, 5, 0)) / (2 * h) for l in lam])
    assert f2o[lam < 1 / math.sqrt(3) - 0.01].max() < 0  # original Skalak loses stability
    assert abs(O.skalak_f(1.0, 5, 35)) < 1e-15 and abs(O.skalak_fp(1.0, 5, 35)) < 1e-15


@pytest.mark.parametrize("s", [0.97, 1.03, 1.6, 2.6])
def test_isotropic_scaling_closed_forms(m642, s):
    # x = s Q X + t stretches every element by l1 = l2 = s.
    Q = rot(21)
    x = s * m642.rest @ Q.T + 3.0
    A0 = m642.A0
    e_sk, _ = m642.energy_skalak(x)
    assert abs(e_sk - A0 * 2 * O.skalak_f(s, 5.0, 35.0)) < 1e-10 * abs(e_sk)
    a = _sl2_closed_isotropic(s)
    e_ar, _ = m642.energy_area(x)
    assert abs(e_ar - 0.5 * 5000.0 * A0 * ((s - a) ** 2 + (s - 1 / a) ** 2)) < 1e-10 * abs(e_ar)
    e_v, gv = m642.energy_vol(x)
    gc0 = m642.volume_gradient(m642.rest)
    Cv = (s ** 3 - 1) * m642.V0
    assert abs(e_v - 0.5 * 250.0 * Cv ** 2 / (s ** 4 * (gc0 ** 2).sum())) < 1e-10 * e_v
    # bending: delta_f = s R delta_g, so E scales like (s - 1)^2 times the E at s = 2
    e_b, _ = m642.energy_bend(x)
    e_b2, _ = m642.energy_bend(2.0 * m642.rest)
    assert abs(e_b - e_b2 * (s - 1) ** 2) < 1e-9 * abs(e_b)


# ---------------------------------------------------------------------------------------
# operators: L, H~, masses, first guess
# ---------------------------------------------------------------------------------------
def test_laplacian_structure(m642):
    L = m642.laplacian()
    assert np.abs(L - L.T).max() < 1e-9 * np.abs(L).max()
    # PD descriptors annihilate translations, so L 1 = k_vol 1 (volume term has G = I)
    assert np.abs(L.sum(1) - 250.0).max() < 1e-8 * np.abs(L).max()
    assert np.linalg.eigvalsh(L).min() > 0


def test_hessian_solve(m642):
    H = m642.hessian()
    rng = np.random.default_rng(13)
    b = rng.standard_normal((m642.n, 3))
    z = m642.apply_hinv(b)
    assert np.abs(H @ z - b).max() < 1e-10 * np.abs(b).max()
    import scipy.linalg as sl
    assert np.abs(z - sl.cho_solve(sl.cho_factor(H), b)).max() < 1e-12 * np.abs(z).max()
    M = m642.masses()
    assert np.allclose(np.diag(H) - M / DT ** 2, np.diag(m642.laplacian()), rtol=1e-12)


def test_first_guess_lumped(m642):
    rng = np.random.default_rng(14)
    x, v, f = (rng.standard_normal((m642.n, 3)) for _ in range(3))
    y = m642.first_guess(x, v, f)
    M = m642.masses()[:, None]
    assert np.abs(y - (x + DT * v + DT ** 2 * f / M)).max() < 1e-14


def flat_vertex_configuration(model, i):
    """Rest shape with vertex i moved to the cotangent-weighted centre of its one-ring,
    where delta_f = sum_j c_ij (x_j - x_i) vanishes (the 1/(2 A_i) factor of c_ij is
    common to the ring and drops out); also the current area-weighted normal there."""
    x = model.rest.copy()
    T = model.tris
    wsum, acc = 0.0, np.zeros(3)
    for t in T:
        for a in range(3):
            # the edge opposite corner a gets cot(angle at a) for both its ends
            p, q, r = t[a], t[(a + 1) % 3], t[(a + 2) % 3]
            u, v = x[q] - x[p], x[r] - x[p]
            cot = np.dot(u, v) / np.linalg.norm(np.cross(u, v))
            if q == i:
                wsum += cot; acc += cot * x[r]
            elif r == i:
                wsum += cot; acc += cot * x[q]
    x[i] = acc / wsum
    nrm = np.zeros(3)
    for t in T:
        if i in t:
            nrm += 0.5 * np.cross(x[t[1]] - x[t[0]], x[t[2]] - x[t[0]])
    return x, nrm / np.linalg.norm(nrm)


def test_bending_flat_vertex_branch():
    # Bending (Sec. 2.1.2): at delta_f = 0 the closest point on the sphere {R delta_g} is
    # not unique; the reading takes it along the current vertex normal, oriented as
    # delta_g is to the rest normal (inward on the convex rim).  Moving the vertex
    # outward by eps keeps that projection (delta_f = eps csum n points inward), so
    # g along the ray is smooth for eps >= 0: the branch's energy must be the ray's
    # limit at 0 and its gradient the one-sided derivative (a sign error flips it).
    rest, tris = W.discocyte(258)
    m = O.Model(rest, tris, W.material_vector(), DT)
    i = int(np.argmax(np.hypot(rest[:, 0], rest[:, 1])))  # a rim vertex (convex)
    x0, nhat = flat_vertex_configuration(m, i)
    E = lambda e: m.energy_bend(np.where(np.arange(m.n)[:, None] == i, x0 + e * nhat, x0))[0]
    E0, G0 = m.energy_bend(x0)
    h = 1e-4 * m.lbar
    E1, E2, E3 = E(h), E(2 * h), E(3 * h)
    assert abs(E0 - (3 * E1 - 3 * E2 + E3)) <= 1e-9 * E0
    d1 = (-3 * E0 + 4 * E1 - E2) / (2 * h)
    assert abs(np.dot(G0[i], nhat) - d1) <= 1e-5 * np.abs(G0).max()
    # the other side of the vertex is a different branch: the derivative differs
    Em = lambda e: E(-e)
    dm = (-3 * E0 + 4 * Em(h) - Em(2 * h)) / (2 * h)
    assert abs(-np.dot(G0[i], nhat) - dm) > 1e-2 * np.abs(G0).max()


def test_first_guess_rayleigh_beta():
    # beta_D > 0 (Sec. 2.1.4, C = alpha_D M + beta_D L with the PD matrix L standing in
    # for the stiffness): M~ = M + h C is not diagonal, and the first guess of
    # Eq. preOptimizationNewton is the solution of M~ (y - x) = h M v + h^2 F_ext.
    # M~ is formed here from the oracle's masses and L, the residual is dense.
    rest, tris = W.discocyte(258)
    beta, alpha = 0.01, 0.002
    m = O.Model(rest, tris, W.material_vector(beta_D=beta, alpha_D=alpha), DT)
    rng = np.random.default_rng(31)
    x, v, f = rest.copy(), 0.01 * rng.standard_normal(rest.shape), 2.0 * rng.standard_normal(rest.shape)
    y = m.first_guess(x, v, f)
    Mv = m.masses()[:, None]
    Mt = np.diag(m.masses() * (1 + DT * alpha)) + DT * beta * m.laplacian()
    rhs = DT * Mv * v + DT ** 2 * f
    assert np.abs(Mt @ (y - x) - rhs).max() <= 1e-12 * np.abs(rhs).max()
    # the coupling is not negligible: y differs from the lumped first guess
    y_lumped = x + rhs / (Mv * (1 + DT * alpha))
    assert np.abs(y - y_lumped).max() > 1e-3 * np.abs(y_lumped - x).max()
    # H~ = M~ / h^2 + L (Sec. 2.1.1)
    assert np.abs(m.hessian() - (Mt / DT ** 2 + m.laplacian())).max() <= 1e-12 * np.abs(m.hessian()).max()


def test_objective_gradient_rayleigh_beta_finite_differences():
    # With beta_D > 0 the inertia term (1/2h^2)(x - y)^T M~ (x - y) couples vertices; its
    # gradient M~ (x - y) / h^2 plus the exact energy gradients (no volume term, whose PD
    # gradient is the linearised projection) must match central differences of g.
    rest, tris = W.discocyte(66)
    m = O.Model(rest, tris, W.material_vector(beta_D=0.02, k_vol=0.0), DT)
    rng = np.random.default_rng(32)
    x = rest + 0.02 * m.lbar * rng.standard_normal(rest.shape)
    y = x + 0.01 * m.lbar * rng.standard_normal(rest.shape)
    E, G, parts = m.objective(x, y)
    Mt = np.diag(m.masses()) + DT * 0.02 * m.laplacian()
    assert abs(parts[0] - 0.5 / DT ** 2 * np.sum((x - y) * (Mt @ (x - y)))) <= 1e-12 * parts[0]
    h = 1e-6 * m.lbar
    fd = np.zeros_like(x)
    for i in range(m.n):
        for c in range(3):
            xp = x.copy(); xp[i, c] += h
            xm = x.copy(); xm[i, c] -= h
            fd[i, c] = (m.objective(xp, y)[0] - m.objective(xm, y)[0]) / (2 * h)
    assert np.abs(fd - G).max() <= 1e-6 * np.abs(G).max()


def test_rayleigh_modal_damping_ratio_small():
    # Reading of beta_D = 0.01 in microseconds: zeta = beta omega / 2 <= 0.1 for all
    # modes of L x = omega^2 M x (Sec. 2.1.4).
    import scipy.linalg as sl
    rest, tris = W.discocyte(258)
    m = O.Model(rest, tris, W.material_vector(beta_D=0.01), DT)
    w2 = sl.eigh(m.laplacian(), np.diag(m.masses()), eigvals_only=True)
    assert 0.5 * 0.01 * math.sqrt(w2.max()) <= 0.1


# ---------------------------------------------------------------------------------------
# solver behaviour
# ---------------------------------------------------------------------------------------
def test_objective_decreases_every_iteration(m642):
    p = W.population(642, 1, 3, forces="noise", noise_pN=200.0)
    x0, v0, f0 = p["x"][0], p["v"][0], p["f"][0]
    y = m642.first_guess(x0, v0, f0)
    prev = None
    for k in range(0, 9):
        x, st = m642.solve(y, y, O.make_opts(max_iter=k, tol=0.0))
        assert st.iterations == k
        if prev is not None:
            assert st.objective <= prev
        prev = st.objective


def test_zero_stiffness_returns_first_guess():
    rest, tris = W.discocyte(258)
    m = O.Model(rest, tris, W.material_vector(B=0, C=0, D=0, k_bend=0, k_vol=0, k_mat_hess=0), DT)
    p = W.population(258, 1, 4, forces="noise", noise_pN=1.0)
    x1, v1, st = m.step(p["x"][0], p["v"][0], p["f"][0], O.make_opts(tol=1e-12))
    M = m.masses()[:, None]
    y = p["x"][0] + DT ** 2 * p["f"][0] / M
    assert st.iterations == 0
    assert np.abs(x1 - y).max() < 1e-13


def test_local_global_solver_monotone():
    # Appendix A: pure PD energies, no history, alpha = 1 is the alternating solver,
    # whose objective never increases.
    rest, tris = W.discocyte(258)
    m = O.Model(rest, tris, W.material_vector(B=0, D=0, k_mat_hess=0, k_vol=0), DT)
    p = W.population(258, 1, 5, forces="noise", noise_pN=300.0)
    y = m.first_guess(p["x"][0], p["v"][0], p["f"][0])
    objs = []
    for k in range(0, 12):
        _, st = m.solve(y, y, O.make_opts(lbfgs_m=0, max_iter=k, tol=0.0, fixed_alpha=1))
        objs.append(st.objective)
    assert all(b <= a * (1 + 1e-14) for a, b in zip(objs, objs[1:]))
    assert objs[-1] < objs[0]


@pytest.mark.parametrize("nv", [6, 12])
def test_brute_force_newton_matches_lbfgs(nv):
    # Without the volume term every gradient is the exact gradient of g (exact
    # projections), so L-BFGS with the Armijo search must reach Newton's root.  The
    # volume term's PD gradient uses the paper's linearised projection and is pinned
    # separately by finite differences.
    rest, tris = W.discocyte(nv)
    m = O.Model(rest, tris, W.material_vector(k_vol=0.0), DT)
    rng = np.random.default_rng(nv)
    x0 = rest + 0.02 * m.lbar * rng.standard_normal(rest.shape)
    v0 = 0.001 * rng.standard_normal(rest.shape)
    f0 = 500.0 * rng.standard_normal(rest.shape)
    y = m.first_guess(x0, v0, f0)
    x_lb, st = m.solve(y, y, O.make_opts(tol=1e-11, max_iter=200))
    # FP64 rounding of g (x - y is ~1e-3 of x) stalls the Armijo test near r ~ 1e-11
    assert st.residual < 1e-10
    # Newton on grad g = 0 with a central-difference Jacobian
    x = y.copy()
    for _ in range(30):
        _, g, _ = m.objective(x, y)
        if np.linalg.norm(g) < 1e-13 * 5000:
            break
        h = 1e-6 * m.lbar
        J = np.zeros((3 * nv, 3 * nv))
        for q in range(3 * nv):
            xp = x.copy().ravel(); xp[q] += h
            xm = x.copy().ravel(); xm[q] -= h
            J[:, q] = (m.objective(xp.reshape(-1, 3), y)[1].ravel() - m.objective(xm.reshape(-1, 3), y)[1].ravel()) / (2 * h)
        x = x - np.linalg.solve(0.5 * (J + J.T), g.ravel()).reshape(-1, 3)
    assert np.abs(x - x_lb).max() < 1e-10 * m.lbar


def test_step_conserves_momentum_without_external_force(m642):
    # With F_ext = 0 and no Rayleigh damping, sum m (v_{n+1} - v_n) = -h sum grad g
    # (the internal forces sum to zero), so momentum drifts only by the residual:
    # |dP| <= h * n * r * lbar * max(m) / h^2.  The post step conserves P exactly.
    rng = np.random.default_rng(15)
    x0 = m642.rest @ rot(16).T + 0.002 * m642.lbar * rng.standard_normal(m642.rest.shape) + 40.0
    v0 = 1e-3 * rng.standard_normal(x0.shape)
    M = m642.masses()[:, None]
    x1, v1, st = m642.step(x0, v0, np.zeros_like(x0), O.make_opts(tol=1e-8, max_iter=200))
    assert O.STATUS[st.status] == "OK"
    dP = np.abs((M * v1).sum(0) - (M * v0).sum(0)).max()
    bound = m642.n * st.residual * m642.lbar * M.max() / DT
    assert dP <= bound
    assert dP < 1e-6 * np.abs(M * v0).sum()


def test_post_step_conserves_linear_and_angular_momentum(m642):
    rng = np.random.default_rng(17)
    x = deformed(m642, seed=18) + 20.0
    v = rng.standard_normal(x.shape)
    M = m642.masses()[:, None]
    v2 = m642.post_step(x, v, 0.6)
    assert np.abs((M * v2).sum(0) - (M * v).sum(0)).max() < 1e-9 * np.abs(M * v).sum() / len(v)
    xc = (M * x).sum(0) / M.sum()
    L0 = np.cross(x - xc, M * v).sum(0)
    L1 = np.cross(x - xc, M * v2).sum(0)
    assert np.abs(L1 - L0).max() < 1e-9 * np.abs(np.cross(x - xc, M * v)).sum() / len(v)
    # kappa = 1 leaves exactly the rigid-body velocity field; kappa = 0 changes nothing
    v1 = m642.post_step(x, v, 1.0)
    rigid = v1 - v1.mean(0)  # = omega x r + (vcm - mean) ; check it is a rotation field
    Wm = np.linalg.lstsq(np.stack([np.cross(np.eye(3)[k], x - xc) for k in range(3)], -1).reshape(-1, 3),
                         (v1 - (M * v).sum(0) / M.sum()).reshape(-1), rcond=None)
    assert Wm[1].size == 0 or Wm[1][0] < 1e-16 * (v ** 2).sum()
    assert np.abs(m642.post_step(x, v, 0.0) - v).max() == 0.0


def test_printed_parameter_table_defaults():
    g = read_golden("material_parameters.txt")
    d = W.DEFAULT_MATERIAL
    for k in ("B", "C", "D"):
        assert d[k] == g[k]
    assert d["k_vol"] == g["k_volume"] and d["alpha_D"] == g["alpha_D"] and d["kappa"] == g["kappa_damping"]
    # readings: bending at the physiological 2e-19 J; beta_D off (its unit is not printed)
    assert d["k_bend"] == 0.2 and d["beta_D"] == 0.0
    assert 258 in g["mesh_resolutions"] and 66 in g["mesh_resolutions"] and 1026 in g["mesh_resolutions"]
