"""Collisions between cells (Sec. 3.3) on the GPU against the FP64 oracle
(oracle/collision.py and the collision energy of the C oracle).

* Detection: the nearest vertex of another cell within the cutoff and its tangent
  plane.  The GPU measures distances in FP32, so a vertex whose two candidates (or
  whose distance and the cutoff) are within rounding may resolve differently; all but
  0.5 % of the vertices must agree, and agreeing planes to 1e-5.
* A step with collision planes: FP64 with the same planes on both sides, fixed
  iteration count, max |dx| / lbar <= 1e-10; FP32 and BF16 at tolerance 1e-6 with the
  GPU's own detection, max |dx| / lbar <= 1e-5 plus the FP32 storage rounding.
"""
import numpy as np
import pytest

from helpers import DT, fp32_store_allowance, max_rel_disp, oracle_model
from oracle import collision as Co
from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

pytestmark = pytest.mark.gpu
WCOL = 2000.0
CUT = 0.6


@pytest.fixture(scope="module")
def npfem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    N.lib()
    return N


def _cells(n=258, seed=300):
    """Four cells: three lying flat and overlapping at their rims, one far away; each
    turned about its axis by a random angle; FP32-rounded."""
    rest, tris = W.discocyte(n)
    th = np.random.default_rng(seed).uniform(0.0, 2 * np.pi, 4)
    R = np.zeros((4, 3, 3))
    R[:, 0, 0], R[:, 0, 1], R[:, 1, 0], R[:, 1, 1], R[:, 2, 2] = np.cos(th), -np.sin(th), np.sin(th), np.cos(th), 1.0
    shifts = np.array([[0.0, 0.0, 0.0], [6.9, 0.4, 0.2], [3.2, 6.6, -0.3], [40.0, 40.0, 40.0]])
    x = np.einsum("cij,nj->cni", R, rest) + shifts[:, None, :] + 20.0
    return rest, tris, x.astype(np.float32).astype(np.float64)


def _detect_gpu(N, hs, counts, x_soa, cutoff):
    import torch
    total = x_soa.numel() // 3
    planes = torch.zeros(4 * total, dtype=torch.float32, device="cuda")
    stats = torch.zeros(2, dtype=torch.int32, device="cuda")
    N.collision_detect(hs, counts, x_soa, cutoff, planes, stats)
    torch.cuda.synchronize()
    return planes, stats.cpu().numpy()


def _to_absolute(pl_local, x):
    """[cells, n, 4] planes with offsets relative to each cell's vertex 0 -> absolute."""
    out = pl_local.astype(np.float64).copy()
    out[..., 3] += (out[..., :3] * x[:, :1, :]).sum(-1)
    return out


def test_detection_matches_oracle(npfem):
    import torch
    rest, tris, x = _cells()
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT)
    xs = torch.tensor(W.to_soa(x).ravel(), dtype=torch.float32, device="cuda")
    planes, stats = _detect_gpu(npfem, [h], [4], xs, CUT)
    pg = _to_absolute(planes.cpu().numpy().reshape(4, -1, 4), x)
    po = Co.detect([(x, tris)], CUT)[0]
    hg = np.abs(pg[..., :3]).sum(-1) > 0
    ho = np.abs(po[..., :3]).sum(-1) > 0
    assert ho.sum() > 50 and not ho[3].any()
    assert stats[0] == hg.sum() and stats[1] == 0
    both = hg & ho
    assert (hg != ho).sum() <= 0.005 * hg.size
    same = both & (np.abs(pg[..., :3] - po[..., :3]).max(-1) <= 1e-5) & (np.abs(pg[..., 3] - po[..., 3]) <= 1e-4)
    assert (both & ~same).sum() <= 0.005 * hg.size


def test_two_groups_detection_crosses_meshes(npfem):
    # a 642-vertex cell overlapping a 258-vertex cell: each sees the other
    import torch
    r1, t1 = W.discocyte(642)
    r2, t2 = W.discocyte(258)
    x1 = (r1 + 30.0)[None].astype(np.float32).astype(np.float64)
    x2 = (r2 + [37.0, 30.0, 30.0])[None].astype(np.float32).astype(np.float64)
    hs = [npfem.Handle(r, t, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT) for r, t in ((r1, t1), (r2, t2))]
    xs = torch.tensor(np.concatenate([W.to_soa(x1).ravel(), W.to_soa(x2).ravel()]), dtype=torch.float32, device="cuda")
    planes, stats = _detect_gpu(npfem, hs, [1, 1], xs, CUT)
    p = planes.cpu().numpy().reshape(-1, 4)
    g1 = _to_absolute(p[:642][None], x1)[0]
    g2 = _to_absolute(p[642:][None], x2)[0]
    o1, o2 = Co.detect([(x1, t1), (x2, t2)], CUT)
    for g, o in ((g1, o1[0]), (g2, o2[0])):
        hg, ho = np.abs(g[:, :3]).sum(1) > 0, np.abs(o[:, :3]).sum(1) > 0
        assert ho.sum() > 5 and (hg != ho).sum() <= 2
        both = hg & ho
        assert np.abs(g[both, :3] - o[both, :3]).max() <= 1e-5


def test_step_with_collisions_fp64_fixed_iterations(npfem):
    import torch
    rest, tris, x = _cells()
    m = O.Model(rest, tris, W.material_vector(), DT)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp64", tol=0.0, max_iter=8,
                                                                      armijo_noise=0.0), dt=DT)
    # the oracle's planes, rounded to FP32 in the library's local form, on both sides
    po = Co.detect([(x, tris)], CUT)[0]
    loc = po.copy()
    loc[..., 3] -= (po[..., :3] * x[:, :1, :]).sum(-1)
    loc = loc.astype(np.float32)
    po_same = _to_absolute(loc, x)
    rng = np.random.default_rng(301)
    v = (0.01 * rng.standard_normal(x.shape)).astype(np.float32).astype(np.float64)
    f = np.zeros_like(x)
    xo, vo, st = m.step_batch(x, v, f, O.make_opts(tol=0.0, max_iter=8), col=po_same, wcol=WCOL, threads=4)
    dev = lambda a: torch.tensor(W.to_soa(a).ravel(), dtype=torch.float64, device="cuda")
    xs, vs, fs = dev(x), dev(v), dev(f)
    pl = torch.tensor(loc.ravel(), dtype=torch.float32, device="cuda")
    h.set_collisions(pl, WCOL)
    npfem.step([h], [4], xs, vs, fs, DT)
    torch.cuda.synchronize()
    xg = W.from_soa(xs.cpu().numpy().reshape(4, 3, -1))
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    # and the planes changed the step: without them the overlapping cells end elsewhere
    xn, _, _ = m.step_batch(x, v, f, O.make_opts(tol=0.0, max_iter=8), threads=4)
    assert max_rel_disp(xn[:3], xo[:3], m.lbar) > 1e-4
    assert max_rel_disp(xn[3:], xo[3:], m.lbar) == 0.0  # the far cell has no planes


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_step_with_collisions_at_tolerance(npfem, prec):
    import torch
    rest, tris, x = _cells(seed=302)
    m = O.Model(rest, tris, W.material_vector(), DT)
    # without the temporal warm start, so that the last step below starts from the first guess
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision=prec, tol=1e-6, warm_history=0), dt=DT)
    dev = lambda a: torch.tensor(W.to_soa(a).ravel(), dtype=torch.float32, device="cuda")
    f = np.zeros_like(x)
    xs, vs, fs = dev(x), dev(np.zeros_like(x)), dev(f)
    planes, _ = _detect_gpu(npfem, [h], [4], xs, CUT)
    pg = _to_absolute(planes.cpu().numpy().reshape(4, -1, 4), x)
    xo, _, st = m.step_batch(x, np.zeros_like(x), f, O.make_opts(tol=1e-10, max_iter=300), col=pg, wcol=WCOL, threads=4)
    h.set_collisions(planes, WCOL)
    stt = torch.zeros((4, 32), dtype=torch.uint8, device="cuda")
    npfem.step([h], [4], xs, vs, fs, DT, stats=stt)
    torch.cuda.synchronize()
    sg = stt.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(4)
    assert (sg["status"] == 0).all(), sg
    xg = W.from_soa(xs.double().cpu().numpy().reshape(4, 3, -1))
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(x, m.lbar)
    # removing the planes gives the plain step again
    h.set_collisions(None, 0.0)
    xs2, vs2 = dev(x), dev(np.zeros_like(x))
    h2 = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision=prec, tol=1e-6, warm_history=0),
                      dt=DT)
    xs3, vs3 = dev(x), dev(np.zeros_like(x))
    npfem.step([h], [4], xs2, vs2, fs, DT)
    npfem.step([h2], [4], xs3, vs3, fs, DT)
    torch.cuda.synchronize()
    assert torch.equal(xs2, xs3)
