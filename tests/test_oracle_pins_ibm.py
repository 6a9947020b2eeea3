"""Pins of the immersed-boundary oracle (oracle/ibm.py, Sec. 2.3) against what the
mathematics fixes: the moment conditions of the four-point kernel, exact
interpolation of linear fields, Eq. Fext under a uniform or linear stress in closed
form, conservation and adjointness of spreading, the closed-form slip contraction
of one multi-direct forcing cycle for an isolated point, and brute-force sums over
the lattice for the stencil gather."""
import numpy as np
import pytest

from oracle import ibm as I
from paper_1903_06479_gb300 import workloads as W


def test_kernel_values_and_continuity():
    # w(0) = 1/2, w(+-1) = 1/4 from both branches, w(+-2) = 0, zero beyond
    assert I.w1(0.0) == pytest.approx(0.5, abs=1e-15)
    assert I.w1(1.0) == pytest.approx(0.25, abs=1e-15)
    assert I.w1(1.0 + 1e-12) == pytest.approx(0.25, abs=1e-9)
    assert I.w1(2.0) == pytest.approx(0.0, abs=1e-15)
    assert I.w1(2.5) == 0.0 and I.w1(-3.0) == 0.0
    r = np.linspace(-2.5, 2.5, 2001)
    assert np.allclose(I.w1(r), I.w1(-r), atol=0)


@pytest.mark.parametrize("seed", [0, 1])
def test_kernel_moment_conditions(seed):
    # the stencil's defining sums (Peskin): sum_j w(r - j) = 1, sum_j (r - j) w(r - j)
    # = 0 and sum_j w(r - j)^2 = 3/8 for every r
    r = np.random.default_rng(seed).uniform(-5, 5, 1000)
    j = np.floor(r)[:, None] + np.arange(-2, 4)[None, :]
    w = I.w1(r[:, None] - j)
    assert np.abs(w.sum(1) - 1).max() < 1e-14
    assert np.abs(((r[:, None] - j) * w).sum(1)).max() < 1e-14
    assert np.abs((w ** 2).sum(1) - 3 / 8).max() < 1e-14


def _lattice():
    return I.Lattice(origin=(-6.0, -6.0, -5.0), dx=0.5, shape_xyz=(25, 25, 21))


def test_stencil_gather_matches_brute_force_sum():
    lat = _lattice()
    rng = np.random.default_rng(3)
    field = rng.standard_normal((lat.nz, lat.ny, lat.nx, 2))
    X = rng.uniform(-4, 4, (20, 3))
    got = I.interpolate(field, X, lat)
    kk, jj, ii = np.meshgrid(np.arange(lat.nz), np.arange(lat.ny), np.arange(lat.nx), indexing="ij")
    nodes = lat.node(ii, jj, kk)
    for p in range(len(X)):
        Wt = np.prod(I.w1((nodes - X[p]) / lat.dx), axis=-1)  # every lattice node
        ref = np.einsum("kji,kjic->c", Wt, field)
        assert np.abs(got[p] - ref).max() < 1e-13


def test_linear_fields_are_interpolated_exactly():
    lat = _lattice()
    rng = np.random.default_rng(4)
    a, B = rng.standard_normal(3), rng.standard_normal((3, 3))
    kk, jj, ii = np.meshgrid(np.arange(lat.nz), np.arange(lat.ny), np.arange(lat.nx), indexing="ij")
    field = a + lat.node(ii, jj, kk) @ B.T
    X = rng.uniform(-4, 4, (50, 3))
    assert np.abs(I.interpolate(field, X, lat) - (a + X @ B.T)).max() < 1e-12


def _cell():
    rest, tris = W.discocyte(642)
    return rest, tris


def test_vertex_areas_and_normals():
    rest, tris = _cell()
    A, n = I.vertex_area_normal(rest, tris)
    e1 = rest[tris[:, 1]] - rest[tris[:, 0]]
    e2 = rest[tris[:, 2]] - rest[tris[:, 0]]
    assert abs(A.sum() - 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum()) < 1e-12 * A.sum()
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    # outward on the rim: the normal of the outermost vertex points away from the axis
    k = int(np.argmax(np.hypot(rest[:, 0], rest[:, 1])))
    assert np.dot(n[k, :2], rest[k, :2]) > 0.9 * np.linalg.norm(rest[k, :2])


def test_fext_uniform_and_linear_stress_closed_forms():
    rest, tris = _cell()
    lat = _lattice()
    A, n = I.vertex_area_normal(rest, tris)
    eta, g = 1.2e3, 500e-6  # plasma viscosity, shear rate 500/s in 1/us
    s6 = np.zeros((lat.nz, lat.ny, lat.nx, 6))
    s6[..., 3] = eta * g  # sigma_xy: a linear shear flow
    F = I.ext_forces(rest, tris, s6, lat, rho=1.0)
    exp = np.zeros_like(F)
    exp[:, 0] = eta * g * A * n[:, 1]
    exp[:, 1] = eta * g * A * n[:, 0]
    assert np.abs(F - exp).max() < 1e-12 * np.abs(exp).max()
    # a stress linear in position (a Poiseuille-type profile) is sampled exactly
    kk, jj, ii = np.meshgrid(np.arange(lat.nz), np.arange(lat.ny), np.arange(lat.nx), indexing="ij")
    P = lat.node(ii, jj, kk)
    s6 = np.zeros((lat.nz, lat.ny, lat.nx, 6))
    s6[..., 4] = -2.0 * P[..., 0]  # sigma_xz = -2 x
    s6[..., 5] = -2.0 * P[..., 1]  # sigma_yz = -2 y
    F = I.ext_forces(rest, tris, s6, lat, rho=2.0)
    sxz, syz = -2.0 * rest[:, 0], -2.0 * rest[:, 1]
    exp = 2.0 * A[:, None] * np.stack([sxz * n[:, 2], syz * n[:, 2], sxz * n[:, 0] + syz * n[:, 1]], axis=1)
    assert np.abs(F - exp).max() < 1e-11 * np.abs(exp).max()
    # the exterior variants sample the same uniform stress
    s6 = np.zeros((lat.nz, lat.ny, lat.nx, 6)); s6[..., 3] = 1.0
    F0 = I.ext_forces(rest, tris, s6, lat, mode=0)
    for mode in (1, 2):
        assert np.abs(I.ext_forces(rest, tris, s6, lat, mode=mode) - F0).max() < 1e-12 * np.abs(F0).max()


def test_exterior_modes_see_only_the_outside():
    # a stress that jumps across the membrane: inside the cell 0, outside 1 (sigma_xz);
    # the exterior variants ignore the inside, the full stencil does not
    rest, tris = _cell()
    lat = _lattice()
    kk, jj, ii = np.meshgrid(np.arange(lat.nz), np.arange(lat.ny), np.arange(lat.nx), indexing="ij")
    P = lat.node(ii, jj, kk)
    r = np.hypot(P[..., 0], P[..., 1])
    inside = (r < 3.0) & (np.abs(P[..., 2]) < 0.3)  # nodes inside the membrane, between the dimples
    s6 = np.zeros((lat.nz, lat.ny, lat.nx, 6)); s6[..., 4] = np.where(inside, 0.0, 1.0)
    A, n = I.vertex_area_normal(rest, tris)
    k = int(np.argmax(rest[:, 2] - 10 * (np.hypot(rest[:, 0], rest[:, 1]) > 0.5)))  # the top of the dimple
    assert n[k, 2] > 0.99
    for mode in (1, 2):
        F = I.ext_forces(rest, tris, s6, lat, mode=mode)
        assert F[k, 0] == pytest.approx(A[k] * n[k, 2], rel=1e-12)
    F = I.ext_forces(rest, tris, s6, lat, mode=0)
    assert F[k, 0] < 0.99 * A[k] * n[k, 2]  # the full stencil also sees the inside


def test_spreading_conserves_total_force_and_is_adjoint_to_interpolation():
    lat = _lattice()
    rng = np.random.default_rng(5)
    X = rng.uniform(-4, 4, (30, 3))
    fk = rng.standard_normal((30, 3))
    A = rng.uniform(0.1, 0.3, 30)
    f = I.spread(fk, X, A, lat)
    assert np.abs(f.sum((0, 1, 2)) * lat.dx ** 3 - (fk * (A * lat.dx)[:, None]).sum(0)).max() < 1e-12
    g = rng.standard_normal((lat.nz, lat.ny, lat.nx, 3))
    lhs = (g * f).sum() * lat.dx ** 3
    rhs = ((A * lat.dx)[:, None] * fk * I.interpolate(g, X, lat)).sum()
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_multi_direct_forcing_isolated_point_closed_form():
    # one Lagrangian point: one cycle shrinks the slip U - u by the factor
    # 1 - (A / dx^2) (3/8)^3 (the stencil's sum of squared weights), and L cycles by
    # its L-th power
    lat = _lattice()
    X = np.array([[0.123, -0.456, 0.789]])
    U = np.array([[0.3, -0.2, 0.1]])
    A = np.array([0.2])
    u0 = np.zeros((lat.nz, lat.ny, lat.nx, 3)); u0[..., 0] = 0.05
    c = A[0] / lat.dx ** 2 * (3 / 8) ** 3
    slip0 = U - I.interpolate(u0, X, lat)
    for L in range(4):
        f, fimm = I.multi_direct_forcing(u0, X, U, A, lat, dt=0.1, cycles=L)
        ul = I.interpolate(u0 + fimm * 0.1, X, lat)
        assert np.abs((U - ul) - slip0 * (1 - c) ** (L + 1)).max() < 1e-13
