"""Pins of the seeded input generators that the oracle and the GPU path share
(paper_1903_06479_gb300/workloads.py): rigid placements, the shear-traction stand-in
for the immersed-boundary force (Eq. Fext) and its noise."""
import numpy as np
import pytest

from paper_1903_06479_gb300 import workloads as W


def _volume(x, tris):
    a, b, c = x[..., tris[:, 0], :], x[..., tris[:, 1], :], x[..., tris[:, 2], :]
    return np.einsum("...i,...i->...", a, np.cross(b, c)).sum(-1) / 6.0


def test_population_is_deterministic_and_placements_rigid():
    p = W.population(258, 6, seed=3, forces="shear", noise_pN=0.5)
    q = W.population(258, 6, seed=3, forces="shear", noise_pN=0.5)
    for k in ("x", "v", "f", "f_shear"):
        assert np.array_equal(p[k], q[k])
    rest, tris = p["rest"], p["tris"]
    # proper rotations plus translations: edge lengths and the signed volume are kept
    e_rest = np.linalg.norm(rest[tris[:, 1]] - rest[tris[:, 0]], axis=-1)
    e = np.linalg.norm(p["x"][:, tris[:, 1]] - p["x"][:, tris[:, 0]], axis=-1)
    assert np.allclose(e, e_rest[None], rtol=0, atol=1e-12)
    assert np.allclose(_volume(p["x"], tris), _volume(rest, tris), rtol=1e-12)
    centres = p["x"].mean(axis=1) - rest.mean(axis=0)
    assert (centres >= 0).all() and (centres <= 100.0).all()
    assert not np.any(p["v"])


def test_vertex_area_normals_integrate_to_three_volumes_and_close():
    """Sum_k x_k . (A n)_k = 3V (each face's area vector dotted with any of its
    corners gives 3 V_f) and Sum_k (A n)_k = 0 on a closed surface."""
    p = W.population(642, 3, seed=5, forces="shear", noise_pN=0.0)
    an = W._vertex_area_normals(p["x"], p["tris"])
    v3 = np.einsum("cni,cni->c", p["x"], an)
    assert np.allclose(v3, 3.0 * _volume(p["x"], p["tris"]), rtol=1e-12)
    assert np.abs(an.sum(axis=1)).max() < 1e-12 * np.abs(an).sum(axis=1).max()


def test_shear_traction_closed_surface_and_components():
    """F_k = sigma (A n)_k with sigma = eta gamma (e_x e_y^T + e_y e_x^T): no z component,
    the x and y components swap the normal's y and x, and the net force vanishes."""
    p = W.population(642, 4, seed=2, forces="shear", noise_pN=0.0)
    g = np.array([10.0, 100.0, 500.0, 1000.0])
    f = W.shear_forces(p["x"], p["tris"], g)
    an = W._vertex_area_normals(p["x"], p["tris"])
    sig = W.PLASMA_ETA * g * 1e-6
    assert np.allclose(f[..., 0], sig[:, None] * an[..., 1], rtol=1e-14, atol=0)
    assert np.allclose(f[..., 1], sig[:, None] * an[..., 0], rtol=1e-14, atol=0)
    assert not np.any(f[..., 2])
    assert np.abs(f.sum(axis=1)).max() < 1e-12 * np.abs(f).sum(axis=(1, 2)).max()
    # noise-free population forces are this traction at the placement
    assert np.array_equal(p["f"], p["f_shear"])


def test_force_noise_and_redrawn_draws():
    p = W.population(642, 16, seed=1, forces="shear", noise_pN=0.5)
    noise = p["f"] - p["f_shear"]
    assert abs(noise.mean()) < 0.01 and abs(noise.std() - 0.5) < 0.005
    draws = W.noise_redrawn_forces(p, 16, seed=7)
    assert len(draws) == 4
    nz = [d - p["f_shear"] for d in draws]
    for a in nz:
        assert abs(a.std() - 0.5) < 0.005
    for a, b in zip(nz, nz[1:] + nz[:1]):
        assert abs(np.corrcoef(a.ravel(), b.ravel())[0, 1]) < 0.01  # independent draws
    assert np.array_equal(W.noise_redrawn_forces(p, 16, seed=7)[2], draws[2])


def test_soa_round_trip():
    a = np.random.Generator(np.random.PCG64(0)).normal(size=(5, 7, 3))
    s = W.to_soa(a)
    assert s.shape == (5, 3, 7) and s.flags["C_CONTIGUOUS"]
    assert np.array_equal(W.from_soa(s), a)


def test_stretch_forces_balance_and_bead_patches():
    rest, tris = W.discocyte(258)
    for F in (0.0, 50.0, 200.0):
        f = W.stretch_forces(rest, F, 2.0)
        assert np.abs(f.sum(0)).max() < 1e-12  # equal and opposite
        left, right = W.bead_vertices(rest, 2.0)
        assert f[right, 0].sum() == pytest.approx(F) and f[left, 0].sum() == pytest.approx(-F)
        assert (rest[right, 0] > 0).all() and (rest[left, 0] < 0).all()
    # torque-free: the patches are mirror images on the x axis
    assert np.abs(np.cross(rest, W.stretch_forces(rest, 100.0)).sum(0)).max() < 1e-9


def test_elongation_index_and_recovery_fit():
    from paper_1903_06479_gb300 import validation as V
    lam0, linf = 2.4, 1.0
    assert V.elongation_index(lam0, lam0, linf) == pytest.approx(1.0)
    assert V.elongation_index(linf, lam0, linf) == pytest.approx(0.0)
    t = np.linspace(0, 5000, 40)
    tc, delta, r2 = V.fit_recovery_time(t, np.exp(-t / 1234.0))
    assert tc == pytest.approx(1234.0, rel=1e-9) and delta == pytest.approx(1.0) and r2 == pytest.approx(1.0)
    tc, delta, r2 = V.fit_recovery_time(t, np.exp(-(t / 2500.0) ** 0.7))
    assert tc == pytest.approx(2500.0, rel=1e-9) and delta == pytest.approx(0.7) and r2 == pytest.approx(1.0)
    x = np.random.default_rng(0).standard_normal((50, 3))
    DA, DT = V.diameters(x)
    assert DA == pytest.approx(np.ptp(x[:, 0])) and DT == pytest.approx(np.ptp(x[:, 1]))
