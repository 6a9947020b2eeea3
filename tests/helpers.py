"""Shared helpers for the GPU parity tests: seeded inputs, oracle runs, tolerances."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

DT = 0.1  # us


_MODELS = {}


def oracle_model(n_verts, **mat):
    """Oracle model of the discocyte mesh (cached: the FP64 set-up of large meshes
    factors a dense matrix)."""
    key = (n_verts, tuple(sorted(mat.items())))
    if key not in _MODELS:
        rest, tris = W.discocyte(n_verts)
        _MODELS[key] = (O.Model(rest, tris, W.material_vector(**mat), DT), rest, tris)
    return _MODELS[key]


def population32(n_verts, cells, seed, **kw):
    """Seeded population rounded to FP32 (the exact inputs both sides see)."""
    p = W.population(n_verts, cells, seed, **kw)
    for k in ("x", "v", "f"):
        p[k] = p[k].astype(np.float32).astype(np.float64)
    return p


def oracle_steps(model, x, v, f, steps=1, threads=8, **opts):
    """Run the oracle on [cells, n, 3] float64 arrays; returns x, v, stats list."""
    return model.step_batch(x, v, f, O.make_opts(**opts), steps=steps, threads=threads)


def gpu_step_device(handle, x, v, f, steps=1, dtype="float32", stats=True, static=False):
    """Run npfem_step (npfem_step_static with static) on torch device tensors built
    from [cells, n, 3] arrays."""
    import torch
    from paper_1903_06479_gb300 import npfem
    td = torch.float64 if dtype == "float64" else torch.float32
    xs = torch.tensor(W.to_soa(x), dtype=td, device="cuda")
    vs = torch.tensor(W.to_soa(v), dtype=td, device="cuda")
    fs = torch.tensor(W.to_soa(f), dtype=td, device="cuda")
    cells = x.shape[0]
    st = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda") if stats else None
    fn = npfem.step_static if static else npfem.step
    for _ in range(steps):
        fn([handle], [cells], xs, vs, fs, handle.dt, stats=st)
    torch.cuda.synchronize()
    out_st = None
    if stats:
        out_st = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(cells)
    return (W.from_soa(xs.double().cpu().numpy()), W.from_soa(vs.double().cpu().numpy()), out_st)


def max_rel_disp(xa, xb, lbar):
    return float(np.linalg.norm(xa - xb, axis=-1).max() / lbar)


def fp32_store_allowance(x, lbar):
    """Half an ulp of the largest |coordinate| per component, as a fraction of lbar:
    the rounding of storing x_{n+1} in FP32, which no solver accuracy can remove."""
    return float(np.sqrt(3.0) * np.spacing(np.abs(x).max().astype(np.float32)) / lbar)
