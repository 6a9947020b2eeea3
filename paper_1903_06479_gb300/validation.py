"""Solid-only validation runs of the paper's Sec. 3.1-3.2 on the GPU path.

Stretching (Sec. 3.1): equal and opposite forces on the vertices under two beads at
the ends of the cell's long axis, raised in increments up to 200 pN; at every
increment the cell is stepped until it stops moving (the paper applies the next
increment only at equilibrium), and the axial and transverse diameters are read.
The paper's mesh independence is checked by running several resolutions in one
batched npfem_step call (one group per mesh).

Recovery (Sec. 3.2): a cell stretched to equilibrium is released and its shape
ratio lambda = D_A / D_T is followed in time through the elongation index
e(t) = (lambda - l_inf)(l_0 + l_inf) / ((lambda + l_inf)(l_0 - l_inf))
(Eq. ElongationIndex), fitted by exp(-(t / t_c)^delta).

Everything here is host-side orchestration and measurement; every time step is an
npfem_step call (no CPU path).
"""
from __future__ import annotations

import numpy as np

from . import npfem as N
from . import workloads as W

PAPER_MATERIAL = dict(k_bend=1.0)  # the results section's parameter table (bending 1 pN um)


def diameters(x: np.ndarray) -> tuple[float, float]:
    """Axial (along x, the stretching axis) and transverse (along y, in the plane of
    the disc) diameters of one cell [n, 3]."""
    return float(x[:, 0].max() - x[:, 0].min()), float(x[:, 1].max() - x[:, 1].min())


def elongation_index(lam, lam0: float, lam_inf: float):
    """Eq. ElongationIndex of Hochmuth et al. as printed in Sec. 3.2."""
    lam = np.asarray(lam, dtype=np.float64)
    return (lam - lam_inf) * (lam0 + lam_inf) / ((lam + lam_inf) * (lam0 - lam_inf))


def fit_recovery_time(t, e, e_lo: float = 0.02, e_hi: float = 0.98) -> tuple[float, float, float]:
    """Fit of Eq. ElongationIndex, e = exp(-(t / t_c)^delta): least squares of
    log(-log e) = delta log t - delta log t_c over the samples with e_lo < e < e_hi and
    t > 0.  Returns (t_c, delta, coefficient of determination of that linear fit)."""
    t = np.asarray(t, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    m = (e > e_lo) & (e < e_hi) & (t > 0)
    xs, ys = np.log(t[m]), np.log(-np.log(e[m]))
    A = np.stack([xs, np.ones_like(xs)], axis=1)
    (delta, c0), *_ = np.linalg.lstsq(A, ys, rcond=None)
    res = ys - (delta * xs + c0)
    r2 = 1.0 - np.dot(res, res) / max(np.dot(ys - ys.mean(), ys - ys.mean()), 1e-300)
    return float(np.exp(-c0 / delta)), float(delta), float(r2)


def _device(a, dtype):
    import torch
    return torch.tensor(a, dtype=dtype, device="cuda")


def stretching(sizes=(66, 258, 1026), forces_pN=(25, 50, 75, 100, 125, 150, 175, 200), dt: float = 2.0,
               tol: float | None = None, max_iter: int = 300, precision: str = "fp64", patch_um: float = 2.0,
               move_tol: float = 1e-5, max_steps: int = 2000, material: dict | None = None):
    """Quasi-static stretching of one cell per mesh resolution, all resolutions in one
    batched npfem_step per time step.  The time step only sets how fast the cell
    settles: at 2 us each step's solve converges on every mesh (at 10 us the 1026-vertex
    mesh stalls short of the tolerance).  The residual r = RMS(h^2 |grad g| / m) / lbar
    grows with h^2, so the default tolerance is 1e-6 in FP64 and 1e-4 in FP32 (a force
    balance of ~1e-3 pN per vertex, which FP32 resolves in forces of 100 pN).  Returns {n: {"force", "DA", "DT", "steps",
    "move", "x"}} with one entry per force level (the last step's largest vertex move,
    um) and the final positions x [n, 3]."""
    import torch
    mat = dict(PAPER_MATERIAL)
    mat.update(material or {})
    td = torch.float64 if precision == "fp64" else torch.float32
    if tol is None:
        tol = 1e-6 if precision == "fp64" else 1e-4
    hs, rests, bead = [], [], []
    for n in sizes:
        rest, tris = W.discocyte(n)
        hs.append(N.Handle(rest, tris, N.material(**mat),
                           N.default_opts(precision=precision, tol=tol, max_iter=max_iter, warm_history=0), dt=dt))
        rests.append(rest)
    cells = [1] * len(sizes)
    x = _device(np.concatenate([W.to_soa(r[None]).ravel() for r in rests]), td)
    v = torch.zeros_like(x)
    f = torch.zeros_like(x)
    out = {n: {"force": [], "DA": [], "DT": [], "steps": [], "move": []} for n in sizes}
    split = lambda a: np.split(a, np.cumsum([3 * n for n in sizes])[:-1])
    for F in forces_pN:
        f.copy_(_device(np.concatenate([W.to_soa(W.stretch_forces(r, F, patch_um)[None]).ravel() for r in rests]), td))
        moves = np.full(len(sizes), np.inf)
        k = 0
        while k < max_steps and moves.max() > move_tol:
            x0 = x.clone()
            N.step(hs, cells, x, v, f, dt)
            d = (x - x0).abs().cpu().numpy()
            moves = np.array([p.max() for p in split(d)])
            k += 1
        xs = [W.from_soa(p.reshape(1, 3, n))[0] for p, n in zip(split(x.double().cpu().numpy()), sizes)]
        for n, xc, mv in zip(sizes, xs, moves):
            DA, DT = diameters(xc)
            out[n]["force"].append(float(F))
            out[n]["DA"].append(DA)
            out[n]["DT"].append(DT)
            out[n]["steps"].append(k)
            out[n]["move"].append(float(mv))
    for n, xc in zip(sizes, xs):
        out[n]["x"] = xc
    for h in hs:
        h.close()
    return out


def recovery(n: int = 258, force_pN: float = 100.0, dt_stretch: float = 2.0, dt: float = 0.1, steps: int = 4000,
             every: int = 20, precision: str = "fp64", beta_D: float = 0.01, patch_um: float = 2.0,
             material: dict | None = None, tol: float | None = None):
    """Stretch one cell to equilibrium at force_pN (two increments, as in `stretching`),
    then release it (F = 0, at rest) and step it with time step dt (us) under Rayleigh
    damping beta_D and the post-convergence dissipation.  The released cell moves ~1e-4 um
    per step, so the residual tolerance sets how far each step stops short of its
    minimiser relative to that motion: the default is 1e-9 in FP64 and 1e-6 in FP32.  Returns t (us), lambda(t), e(t), lambda_0, lambda_inf,
    the fitted t_c (us) and the fit's R^2."""
    import torch
    mat = dict(PAPER_MATERIAL)
    mat.update(material or {})
    st = stretching((n,), (force_pN / 2, force_pN), dt=dt_stretch, precision=precision, patch_um=patch_um,
                    material=mat)
    rest, tris = W.discocyte(n)
    td = torch.float64 if precision == "fp64" else torch.float32
    x = _device(W.to_soa(st[n]["x"][None]).ravel(), td)
    v = torch.zeros_like(x)
    x0 = W.from_soa(x.double().cpu().numpy().reshape(1, 3, n))[0]
    DA0, DT0 = diameters(x0)
    lam0 = DA0 / DT0
    lam_inf = 1.0  # the rest discocyte: D_A = D_T
    mat_r = dict(mat)
    mat_r["beta_D"] = beta_D
    if tol is None:
        tol = 1e-9 if precision == "fp64" else 1e-6
    h = N.Handle(rest, tris, N.material(**mat_r), N.default_opts(precision=precision, tol=tol, max_iter=200), dt=dt)
    v.zero_()
    f = torch.zeros_like(x)
    ts, lams = [0.0], [lam0]
    for k in range(1, steps + 1):
        N.step([h], [1], x, v, f, dt)
        if k % every == 0:
            xc = W.from_soa(x.double().cpu().numpy().reshape(1, 3, n))[0]
            DA, DT = diameters(xc)
            ts.append(k * dt)
            lams.append(DA / DT)
    h.close()
    ts, lams = np.array(ts), np.array(lams)
    e = elongation_index(lams, lam0, lam_inf)
    tc, delta, r2 = fit_recovery_time(ts, e)
    return {"t_us": ts, "lambda": lams, "e": e, "lambda0": lam0, "lambda_inf": lam_inf, "t_c_us": tc,
            "delta": delta, "r2": r2, "stretch": st}
