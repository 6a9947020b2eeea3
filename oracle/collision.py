"""FP64 CPU oracle of the collision detection of Sec. 3.3 (Proof of capability).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product package.

Plain numpy, brute force over every pair of vertices of different cells.  The paper
gives each colliding vertex x_i a desired position p_i "defined from the colliding
neighbors and their normals" and checks at every iteration whether x_i still
penetrates; the energy itself is in the C oracle (or_energy_collision).  Readings:

1. The colliding neighbour of vertex i is the nearest vertex j of another cell with
   |x_j - x_i| <= cutoff, at the positions the step starts from; ties go to the
   lowest global vertex index (cells of all groups numbered in order).
2. p_i is x_i moved onto the tangent plane of the neighbouring body at j: unit
   normal n_j (the normalised area-weighted vertex normal, outward) and offset
   c_i = n_j . x_j.  Vertex i penetrates while c_i - n_j . x_i > 0.
3. Vertices without a neighbour within the cutoff get the plane (0, 0, 0, 0).
"""
from __future__ import annotations

import numpy as np

from .ibm import vertex_area_normal


def detect(groups, cutoff: float):
    """groups: list of (x [cells, n, 3], tris).  Returns, per group, planes
    [cells, n, 4] = (n_j, c_i) in absolute coordinates."""
    X, cell_id, normals = [], [], []
    cid = 0
    for x, tris in groups:
        for c in range(x.shape[0]):
            X.append(np.asarray(x[c], dtype=np.float64))
            cell_id.append(np.full(x.shape[1], cid))
            normals.append(vertex_area_normal(x[c], tris)[1])
            cid += 1
    X = np.concatenate(X)
    cell_id = np.concatenate(cell_id)
    normals = np.concatenate(normals)
    V = X.shape[0]
    planes = np.zeros((V, 4))
    cut2 = cutoff * cutoff
    for a in range(0, V, 512):
        b = min(V, a + 512)
        d2 = ((X[a:b, None, :] - X[None, :, :]) ** 2).sum(-1)
        d2[cell_id[a:b, None] == cell_id[None, :]] = np.inf
        d2[d2 > cut2] = np.inf
        j = np.argmin(d2, axis=1)  # the first index among equal distances
        ok = np.isfinite(d2[np.arange(b - a), j])
        nj = normals[j]
        planes[a:b, :3] = np.where(ok[:, None], nj, 0.0)
        planes[a:b, 3] = np.where(ok, (nj * X[j]).sum(1), 0.0)
    out, off = [], 0
    for x, _ in groups:
        c, n = x.shape[:2]
        out.append(planes[off:off + c * n].reshape(c, n, 4))
        off += c * n
    return out
