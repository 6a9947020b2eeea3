"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests, the benchmark and the oracle wrapper; it
holds none of the solver's arithmetic (no energies, projections, operators or
solver steps).  It builds:

* closed triangle meshes of the red-blood-cell membrane: subdivided octahedra
  (66, 258, 1026 vertices, the paper's own resolutions in its parameter table)
  and subdivided icosahedra (162, 642, 2562 vertices), projected on the unit
  sphere and mapped to the Evans-Skalak biconcave discocyte of the paper's
  introduction (diameter 7.82 um, dimple 0.81 um, rim 2.57 um);
* random rigid placements (uniform SO(3) from normalised Gaussian quaternions,
  translations uniform in a 100 um cube);
* external forces: i.i.d. Gaussian noise, and a stand-in for the immersed-boundary
  force of the paper's Eq. (Fext), F_k = A_k sigma n_k, with sigma a linear shear
  stress eta * gamma_dot * (e_x e_y^T + e_y e_x^T) of plasma viscosity 1.2 cP.

Units are um, us and pN throughout.  Random numbers come from numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

DISCOCYTE_D = 7.82  # um, Sec. 1
# Evans-Skalak coefficients of the discocyte profile
ES_A0, ES_A1, ES_A2 = 0.0518, 2.0026, -4.491
PLASMA_ETA = 1.2e3  # 1.2 cP in pN us / um^2

# Default material (parameter table of the results section; bending modulus at
# the physiological 2e-19 J = 0.2 pN um; density 1000 kg/m^3 = 1000 mass units
# per um^3 with mass unit pN us^2 / um)
DEFAULT_MATERIAL = dict(B=5.0, C=5000.0, D=35.0, k_bend=0.2, k_vol=250.0, k_mat_hess=5.0,
                        density=1000.0, alpha_D=0.0, beta_D=0.0, kappa=0.6)
MATERIAL_ORDER = ("B", "C", "D", "k_bend", "k_vol", "k_mat_hess", "density", "alpha_D", "beta_D", "kappa")


def _subdivide(verts: list, tris: np.ndarray) -> tuple[list, np.ndarray]:
    cache: dict = {}
    out = []

    def mid(a, b):
        key = (a, b) if a < b else (b, a)
        if key not in cache:
            p = verts[a] + verts[b]
            verts.append(p / np.linalg.norm(p))
            cache[key] = len(verts) - 1
        return cache[key]

    for a, b, c in tris:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    return verts, np.asarray(out, dtype=np.int32)


def _base_octahedron():
    v = [np.array(p, dtype=np.float64) for p in
         [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]]
    t = np.array([(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4),
                  (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)], dtype=np.int32)
    return v, t


def _base_icosahedron():
    p = (1.0 + 5 ** 0.5) / 2.0
    raw = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0), (0, -1, p), (0, 1, p),
           (0, -1, -p), (0, 1, -p), (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    v = [np.array(q, dtype=np.float64) / np.linalg.norm(q) for q in raw]
    t = np.array([(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
                  (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
                  (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)], dtype=np.int32)
    return v, t


def sphere_mesh(n_verts: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit-sphere triangulation with outward (counter-clockwise) faces.

    n_verts in {6, 18, 66, 258, 1026} (octahedron family) or {12, 42, 162, 642, 2562}
    (icosahedron family)."""
    octa = {6: 0, 18: 1, 66: 2, 258: 3, 1026: 4, 4098: 5}
    ico = {12: 0, 42: 1, 162: 2, 642: 3, 2562: 4}
    if n_verts in octa:
        v, t = _base_octahedron()
        levels = octa[n_verts]
    elif n_verts in ico:
        v, t = _base_icosahedron()
        levels = ico[n_verts]
    else:
        raise ValueError(f"no sphere mesh with {n_verts} vertices")
    for _ in range(levels):
        v, t = _subdivide(v, t)
    verts = np.asarray(v)
    # orient every face outward
    c = verts[t].mean(axis=1)
    nrm = np.cross(verts[t[:, 1]] - verts[t[:, 0]], verts[t[:, 2]] - verts[t[:, 0]])
    flip = (nrm * c).sum(1) < 0
    t[flip] = t[flip][:, [0, 2, 1]]
    return verts, t


def discocyte(n_verts: int, diameter: float = DISCOCYTE_D) -> tuple[np.ndarray, np.ndarray]:
    """Biconcave rest shape: (x, y) <- (D/2)(x_s, y_s) and
    z <- sign(z_s) D sqrt(1 - 4 r^2/D^2) (a0 + a1 r^2/D^2 + a2 r^4/D^4)."""
    s, t = sphere_mesh(n_verts)
    D = diameter
    xy = 0.5 * D * s[:, :2]
    r2 = (xy ** 2).sum(1)
    q = np.clip(1.0 - 4.0 * r2 / D ** 2, 0.0, None)
    prof = D * np.sqrt(q) * (ES_A0 + ES_A1 * r2 / D ** 2 + ES_A2 * r2 ** 2 / D ** 4)
    z = np.sign(s[:, 2]) * np.abs(prof)
    return np.column_stack([xy, z]), t


def random_rotations(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform rotations from normalised Gaussian quaternions, shape [count, 3, 3]."""
    q = rng.standard_normal((count, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((count, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def place_cells(rest: np.ndarray, rng: np.random.Generator, count: int, box: float = 100.0,
                rotate: bool = True) -> np.ndarray:
    """Copies of the rest shape, randomly rotated and translated: [count, n, 3]."""
    R = random_rotations(rng, count) if rotate else np.broadcast_to(np.eye(3), (count, 3, 3))
    t = rng.uniform(0.0, box, size=(count, 1, 3))
    return np.einsum("cij,nj->cni", R, rest) + t


def _vertex_area_normals(x: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Per-vertex share A_k n_k of the area-weighted normals (one third of each
    incident face), for the force stand-in only.  x: [cells, n, 3]."""
    import scipy.sparse as sp
    cells, n = x.shape[0], x.shape[1]
    e1 = x[:, tris[:, 1]] - x[:, tris[:, 0]]
    e2 = x[:, tris[:, 2]] - x[:, tris[:, 0]]
    an = np.cross(e1, e2) / 6.0  # [cells, nt, 3]
    nt = tris.shape[0]
    inc = sp.csr_matrix((np.ones(3 * nt), (tris.T.ravel(), np.tile(np.arange(nt), 3))), shape=(n, nt))
    out = inc @ np.transpose(an, (1, 0, 2)).reshape(nt, cells * 3)
    return np.transpose(np.asarray(out).reshape(n, cells, 3), (1, 0, 2))


def shear_forces(x: np.ndarray, tris: np.ndarray, gamma_dot_per_s: np.ndarray) -> np.ndarray:
    """Traction F_k = A_k sigma n_k of a linear shear flow (stand-in for Eq. Fext).

    x: [cells, n, 3] positions; gamma_dot_per_s: [cells] shear rates in 1/s."""
    an = _vertex_area_normals(x, tris)
    sig = PLASMA_ETA * np.asarray(gamma_dot_per_s, dtype=np.float64) * 1e-6  # 1/s -> 1/us
    f = np.zeros_like(x)
    f[..., 0] = sig[:, None] * an[..., 1]
    f[..., 1] = sig[:, None] * an[..., 0]
    return f


def population(n_verts: int, cells: int, seed: int, forces: str = "shear", noise_pN: float = 0.5,
               gamma_range=(10.0, 1000.0), gamma_fixed: float | None = None, box: float = 100.0,
               rotate: bool = True):
    """A seeded population: returns dict(rest, tris, x [cells, n, 3], v, f), all float64,
    and for "shear" also f_shear, the traction without the noise.

    forces: "noise" (i.i.d. N(0, noise_pN)) or "shear" (traction of a linear shear flow at
    rate U(gamma_range) per cell, or gamma_fixed, plus N(0, noise_pN) noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rest, tris = discocyte(n_verts)
    x = place_cells(rest, rng, cells, box=box, rotate=rotate)
    v = np.zeros_like(x)
    out = dict(rest=rest, tris=tris, x=x, v=v)
    if forces == "noise":
        out["f"] = rng.normal(0.0, noise_pN, size=x.shape)
    elif forces == "shear":
        g = np.full(cells, gamma_fixed) if gamma_fixed is not None else rng.uniform(*gamma_range, size=cells)
        out["f_shear"] = shear_forces(x, tris, g)
        out["f"] = out["f_shear"] + rng.normal(0.0, noise_pN, size=x.shape)
    else:
        raise ValueError(forces)
    return out


def noise_redrawn_forces(pop: dict, cells: int, seed: int, draws: int = 4, noise_pN: float = 0.5) -> list:
    """Force fields for a run whose noise is redrawn every step: the shear traction of
    the population's first `cells` cells plus `draws` independent N(0, noise_pN) draws,
    used in turn (step k takes draw k mod draws)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = pop["f_shear"][:cells]
    return [base + rng.normal(0.0, noise_pN, size=base.shape) for _ in range(draws)]


def material_vector(**overrides) -> np.ndarray:
    m = dict(DEFAULT_MATERIAL)
    m.update(overrides)
    return np.array([m[k] for k in MATERIAL_ORDER], dtype=np.float64)


def to_soa(a: np.ndarray) -> np.ndarray:
    """[cells, n, 3] -> [cells, 3, n] (the library's component-major layout)."""
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def from_soa(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.swapaxes(a, -1, -2))


def bead_vertices(rest: np.ndarray, patch_um: float = 2.0) -> tuple[np.ndarray, np.ndarray]:
    """Vertices held by the two optical-tweezers beads of the stretching experiment
    (Sec. 3.1): those within patch_um of the rest shape's extreme points along x
    (left, right)."""
    left = np.where(np.linalg.norm(rest - rest[np.argmin(rest[:, 0])], axis=1) <= patch_um)[0]
    right = np.where(np.linalg.norm(rest - rest[np.argmax(rest[:, 0])], axis=1) <= patch_um)[0]
    return left, right


def stretch_forces(rest: np.ndarray, force_pN: float, patch_um: float = 2.0) -> np.ndarray:
    """Equal and opposite total forces +-force_pN along x, spread evenly over each
    bead's vertices: [n, 3]."""
    left, right = bead_vertices(rest, patch_um)
    f = np.zeros_like(rest)
    f[right, 0] = force_pN / len(right)
    f[left, 0] = -force_pN / len(left)
    return f
