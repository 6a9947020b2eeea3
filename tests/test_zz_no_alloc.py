"""The allocation-free entry point npfem_step_static.

Callers that cannot allocate device memory while stepping (a framework's caching
allocator owns the GPU, or cudaMalloc's device-wide synchronisation would stall
the time loop) use npfem_step_static, whose scratch is a fixed array compiled into
the library.  This test steps the same cells with npfem_step and with
npfem_step_static, twice in a row, and requires the same result within the FP32
parity tolerance of the other tests (max |dx| / lbar <= 1e-5).  It uses
2562-vertex cells, whose solver vectors overflow shared memory into the scratch.
The file is named to be collected last.
"""
import numpy as np
import pytest

from helpers import DT, max_rel_disp, population32
from paper_1903_06479_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_static_step_matches_step_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    rest, tris = W.discocyte(2562)
    h = N.Handle(rest, tris, N.material(), N.default_opts(precision="fp32", tol=1e-6), dt=DT)
    _, info = h.rest_info()
    cells = 3
    p = population32(2562, cells, seed=31, forces="shear", noise_pN=0.5, box=10.0)
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    xa, va, fa = mk(p["x"]), mk(p["v"]), mk(p["f"])
    xb, vb = xa.clone(), va.clone()
    sa = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
    sb = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
    for call in range(2):
        N.step([h], [cells], xa, va, fa, DT, stats=sa)
        N.step_static([h], [cells], xb, vb, fa, DT, stats=sb)
        torch.cuda.synchronize()
        ga = sa.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(cells)
        gb = sb.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(cells)
        assert (gb["status"] == 0).all() and (gb["residual"] <= 1e-6).all(), gb
        X = lambda t: W.from_soa(t.double().cpu().numpy())
        assert max_rel_disp(X(xb), X(xa), info["lbar"]) <= 1e-5, call
        assert max_rel_disp(DT * X(vb), DT * X(va), info["lbar"]) <= 1e-5, call


def _step_both(N, handles, cells, p_list, dtype, calls=2):
    """Steps the same concatenated groups with npfem_step and npfem_step_static;
    yields both states and both stats arrays after each call."""
    import torch
    mk = lambda a: torch.tensor(np.concatenate([W.to_soa(p[a]).ravel() for p in p_list]), dtype=dtype, device="cuda")
    xa, va, fa = mk("x"), mk("v"), mk("f")
    xb, vb = xa.clone(), va.clone()
    total = sum(cells)
    sa = torch.zeros((total, 32), dtype=torch.uint8, device="cuda")
    sb = torch.zeros((total, 32), dtype=torch.uint8, device="cuda")
    for _ in range(calls):
        N.step(handles, cells, xa, va, fa, DT, stats=sa)
        N.step_static(handles, cells, xb, vb, fa, DT, stats=sb)
        torch.cuda.synchronize()
        ga = sa.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(total)
        gb = sb.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(total)
        yield xa.double().cpu().numpy(), xb.double().cpu().numpy(), ga, gb


def test_static_step_two_groups_every_cell_stats():
    """Two meshes of different resolution in one call: positions and every cell's
    statistics (the per-group offsets into the stats array) agree with npfem_step."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    sizes, cells = (258, 642), [5, 3]
    handles, pops, lbar = [], [], []
    for nv, c, seed in zip(sizes, cells, (41, 42)):
        rest, tris = W.discocyte(nv)
        # the static path has no temporal warm start: compare against npfem_step without it
        h = N.Handle(rest, tris, N.material(), N.default_opts(precision="fp32", tol=1e-6, warm_history=0), dt=DT)
        handles.append(h)
        lbar.append(h.rest_info()[1]["lbar"])
        pops.append(population32(nv, c, seed=seed, forces="shear", noise_pN=0.5, box=10.0))
    for xa, xb, ga, gb in _step_both(N, handles, cells, pops, torch.float32):
        assert (gb["status"] == 0).all() and (gb["residual"] <= 1e-6).all(), gb
        for k in ("iterations", "evaluations", "status"):
            assert (ga[k] == gb[k]).all(), (k, ga[k], gb[k])
        np.testing.assert_allclose(gb["residual"], ga["residual"], rtol=1e-3, atol=1e-9)
        np.testing.assert_allclose(gb["volume"], ga["volume"], rtol=1e-9)
        off = 0
        for nv, c, lb in zip(sizes, cells, lbar):
            n = 3 * nv * c
            A = W.from_soa(xa[off:off + n].reshape(c, 3, nv))
            B = W.from_soa(xb[off:off + n].reshape(c, 3, nv))
            assert max_rel_disp(B, A, lb) <= 1e-5
            off += n


def test_static_step_fp64():
    """The FP64 branch of the allocation-free step agrees with npfem_step to the FP64
    parity tolerance."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    rest, tris = W.discocyte(642)
    h = N.Handle(rest, tris, N.material(), N.default_opts(precision="fp64", tol=1e-8, warm_history=0), dt=DT)
    lb = h.rest_info()[1]["lbar"]
    p = population32(642, 3, seed=43, forces="shear", noise_pN=0.5, box=10.0)
    for xa, xb, ga, gb in _step_both(N, [h], [3], [p], torch.float64):
        assert (gb["status"] == 0).all(), gb
        assert (ga["iterations"] == gb["iterations"]).all()
        A = W.from_soa(xa.reshape(3, 3, 642))
        B = W.from_soa(xb.reshape(3, 3, 642))
        assert max_rel_disp(B, A, lb) <= 1e-10
