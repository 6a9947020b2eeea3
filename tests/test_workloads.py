"""Pins of the seeded input generators that the oracle and the GPU path share
(paper_1903_06479_gb300/workloads.py): rigid placements, the shear-traction stand-in
for the immersed-boundary force (Eq. Fext) and its noise."""
import numpy as np

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
