"""FP64 CPU oracle of the immersed-boundary force step (Sec. 2.3 of arXiv:1903.06479).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package.

Plain numpy, FP64, written from the paper's definitions:

* the 1-D four-point kernel w(r) and the Dirac stencil W(x, y, z) = w(x/dx) w(y/dx)
  w(z/dx) / dx^3 (Sec. 2.3, the two equations after the interpolation formula);
* interpolation of a lattice field to a Lagrangian point,
  u(X_k) = sum_x u(x) W(x - X_k) dx^3;
* the external force of Eq. Fext, F_k = rho A_k (sum_x sigma(x) W(x - X_k) dx^3) n_k,
  with A_k the surface area of vertex k and n_k its unit normal;
* the multi-direct forcing iteration (Steps 0-5 of Sec. 2.3).

Readings where the paper leaves a choice (each is also stated in the design notes):

1. Eq. Fext is printed in lattice units (dx = 1); in physical units the sum carries
   the dx^3 of the interpolation formula, i.e. the weights are the products of w.
2. A_k is one third of the areas of the triangles around vertex k (barycentric
   share); n_k is the normalised area-weighted vertex normal.
3. Spreading (Step 1) is printed in lattice units, f(x) = sum_k f_k W(x - X_k) A_k;
   in physical units the Lagrangian volume element is A_k dx (a membrane one lattice
   spacing thick), which keeps spreading the adjoint of interpolation.
4. With L cycles of Steps 1-4, the Eulerian force f_imm is the spread of the final
   Lagrangian force f_L (L = 0 is plain direct forcing of f_0).
5. Stencil nodes outside the lattice contribute nothing.
6. The exterior variants: mode 1 sums only the stencil nodes on the outside of the
   membrane ((x - X_k) . n_k > 0) with their weights renormalised to sum to one;
   mode 2 takes sigma of the exterior stencil node farthest from X_k (the first in
   z, y, x order among equals).

Lattice: node (i, j, k) sits at origin + dx (i, j, k), 0 <= i < nx, ...; lattice
fields are arrays [nz, ny, nx, c].  Vertex arrays are [n, 3] (one cell) or
[cells, n, 3].
"""
from __future__ import annotations

import numpy as np


def w1(r):
    """The paper's four-point kernel of one coordinate (lattice units)."""
    a = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(a)
    m1 = a <= 1.0
    m2 = (a > 1.0) & (a <= 2.0)
    out[m1] = (3.0 - 2.0 * a[m1] + np.sqrt(1.0 + 4.0 * a[m1] - 4.0 * a[m1] ** 2)) / 8.0
    out[m2] = (5.0 - 2.0 * a[m2] - np.sqrt(np.maximum(-7.0 + 12.0 * a[m2] - 4.0 * a[m2] ** 2, 0.0))) / 8.0
    return out


class Lattice:
    def __init__(self, origin, dx, shape_xyz):
        self.origin = np.asarray(origin, dtype=np.float64)
        self.dx = float(dx)
        self.nx, self.ny, self.nz = (int(s) for s in shape_xyz)

    def node(self, i, j, k):
        return self.origin + self.dx * np.stack([i, j, k], axis=-1)


def stencil(X, lat: Lattice):
    """The 64 stencil nodes of each point X [P, 3]: integer node indices [P, 64, 3]
    (x, y, z), their weights prod_d w(r_d - j_d) [P, 64] (zero outside the lattice)
    and node positions [P, 64, 3]."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    r = (X - lat.origin) / lat.dx
    base = np.floor(r).astype(np.int64) - 1
    offs = np.array([(a, b, c) for c in range(4) for b in range(4) for a in range(4)])  # z, y, x order
    idx = base[:, None, :] + offs[None, :, :]
    wts = np.prod(w1(r[:, None, :] - idx), axis=-1)
    inside = ((idx >= 0) & (idx < np.array([lat.nx, lat.ny, lat.nz]))).all(-1)
    wts = np.where(inside, wts, 0.0)
    pos = lat.origin + lat.dx * idx
    return idx, wts, pos, inside


def gather(field, idx, inside):
    """field[nz, ny, nx, c] at the stencil nodes (zero outside): [P, 64, c]."""
    nz, ny, nx = field.shape[:3]
    i = np.clip(idx[..., 0], 0, nx - 1)
    j = np.clip(idx[..., 1], 0, ny - 1)
    k = np.clip(idx[..., 2], 0, nz - 1)
    v = field[k, j, i]
    return np.where(inside[..., None], v, 0.0)


def interpolate(field, X, lat: Lattice):
    """u(X_k) = sum_x u(x) W(x - X_k) dx^3 for each point: [P, c]."""
    idx, wts, _, inside = stencil(X, lat)
    return np.einsum("pq,pqc->pc", wts, gather(field, idx, inside))


def vertex_area_normal(x, tris):
    """A_k (one third of the incident triangle areas) and the unit area-weighted normal
    n_k of every vertex of one cell x [n, 3]."""
    x = np.asarray(x, dtype=np.float64)
    e1 = x[tris[:, 1]] - x[tris[:, 0]]
    e2 = x[tris[:, 2]] - x[tris[:, 0]]
    c = np.cross(e1, e2)  # 2 A_t n_t
    area = 0.5 * np.linalg.norm(c, axis=1)
    A = np.zeros(x.shape[0])
    N = np.zeros_like(x)
    for a in range(3):
        np.add.at(A, tris[:, a], area / 3.0)
        np.add.at(N, tris[:, a], 0.5 * c)
    n = N / np.linalg.norm(N, axis=1, keepdims=True)
    return A, n


def sym_from6(s6):
    """[..., 6] (xx, yy, zz, xy, xz, yz) -> [..., 3, 3]."""
    s = np.empty(s6.shape[:-1] + (3, 3))
    s[..., 0, 0], s[..., 1, 1], s[..., 2, 2] = s6[..., 0], s6[..., 1], s6[..., 2]
    s[..., 0, 1] = s[..., 1, 0] = s6[..., 3]
    s[..., 0, 2] = s[..., 2, 0] = s6[..., 4]
    s[..., 1, 2] = s[..., 2, 1] = s6[..., 5]
    return s


def ext_forces(x, tris, sigma6, lat: Lattice, rho=1.0, mode=0):
    """Eq. Fext for one cell: F_k = rho A_k sigma_k n_k with sigma_k the stencil
    average of the lattice stress sigma6 [nz, ny, nx, 6] (mode 0), of its exterior
    nodes (mode 1) or the stress of the farthest exterior node (mode 2)."""
    A, n = vertex_area_normal(x, tris)
    idx, wts, pos, inside = stencil(x, lat)
    s6 = gather(sigma6, idx, inside)  # [n, 64, 6]
    if mode == 0:
        sk = np.einsum("pq,pqc->pc", wts, s6)
    else:
        ext = (np.einsum("pqc,pc->pq", pos - x[:, None, :], n) > 0.0) & inside
        if mode == 1:
            we = np.where(ext, wts, 0.0)
            tot = we.sum(1, keepdims=True)
            sk = np.einsum("pq,pqc->pc", np.where(tot > 0, we / np.where(tot > 0, tot, 1.0), 0.0), s6)
        else:
            d2 = np.where(ext, ((pos - x[:, None, :]) ** 2).sum(-1), -1.0)
            q = np.argmax(d2, axis=1)  # first index among equals
            sk = np.where((d2.max(1) >= 0)[:, None], s6[np.arange(len(q)), q], 0.0)
    S = sym_from6(sk)
    return rho * A[:, None] * np.einsum("pij,pj->pi", S, n)


def spread(fk, X, A, lat: Lattice):
    """Step 1: f(x) = sum_k f_k W(x - X_k) A_k dx (reading 3) on the lattice
    [nz, ny, nx, 3]."""
    out = np.zeros((lat.nz, lat.ny, lat.nx, 3))
    idx, wts, _, inside = stencil(X, lat)
    scale = np.asarray(A, dtype=np.float64) * lat.dx / lat.dx ** 3
    contrib = wts[..., None] * (scale[:, None, None] * np.asarray(fk, dtype=np.float64)[:, None, :])
    sel = inside
    np.add.at(out, (idx[..., 2][sel], idx[..., 1][sel], idx[..., 0][sel]), contrib[sel])
    return out


def multi_direct_forcing(u_star, X, U, A, lat: Lattice, dt, cycles):
    """Steps 0-5 of the multi-direct forcing: returns the Lagrangian force f_L [P, 3]
    and the Eulerian body force f_imm (the spread of f_L, reading 4)."""
    X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
    U = np.asarray(U, dtype=np.float64).reshape(-1, 3)
    f = (U - interpolate(u_star, X, lat)) / dt  # Step 0
    for _ in range(cycles):
        fl = spread(f, X, A, lat)  # Step 1
        ul = u_star + fl * dt  # Step 2
        f = f + (U - interpolate(ul, X, lat)) / dt  # Steps 3-4
    return f, spread(f, X, A, lat)
