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
