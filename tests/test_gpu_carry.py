"""L-BFGS pairs carried across time steps (opts.warm_history = 2) on the GPU path.

An addition to the paper's Algorithm 1, which starts each step's quasi-Newton
iteration with an empty history: along a trajectory each solve also starts from the
cell's pairs of its previous solve, while that solve took at most 3 iterations (the
oracle's trajectory applies the same rule, carry_max_iters=3).  Tolerances:
  * FP64, fixed iteration count, exact Armijo test: max_i |dx_i| / lbar <= 1e-10
    against the oracle's trajectory with the same carried pairs (oracle
    Model.trajectory), and visibly apart from the oracle without them;
  * FP32 / BF16 at tolerance 1e-6: the linear accumulation of the one-step bound
    (steps x 1e-5 lbar, plus the FP32 storage rounding) against the oracle's plain
    steps at tolerance 1e-10, the same bound as the temporal warm start's.
"""
import numpy as np
import pytest

from helpers import DT, fp32_store_allowance, gpu_step_device, max_rel_disp, oracle_model, oracle_steps, population32
from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

pytestmark = pytest.mark.gpu

_ORACLE = {}


@pytest.fixture(scope="module")
def npfem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    N.lib()
    return N


def make_handle(N, n_verts, precision, **kw):
    rest, tris = W.discocyte(n_verts)
    return N.Handle(rest, tris, N.material(), N.default_opts(precision=precision, **kw), dt=DT)


def _stats_steps(N, h, p, steps, dtype="float32"):
    """steps calls of npfem_step on one trajectory; positions and per-step stats."""
    import torch
    td = torch.float64 if dtype == "float64" else torch.float32
    xs, vs, fs = (torch.tensor(W.to_soa(p[k]), dtype=td, device="cuda") for k in ("x", "v", "f"))
    cells = p["x"].shape[0]
    st = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
    out = []
    for _ in range(steps):
        N.step([h], [cells], xs, vs, fs, DT, stats=st)
        out.append(st.cpu().numpy().view(N.CELL_STATS_DTYPE).reshape(cells).copy())
    return W.from_soa(xs.double().cpu().numpy()), W.from_soa(vs.double().cpu().numpy()), out


def test_carried_pairs_fp64_fixed_iterations_match_oracle(npfem):
    # tol 0: three iterations every step, so every step after the first starts from the
    # previous step's pairs (up to the window of 5) and the two sides take the same path
    steps, cells, nv = 4, 3, 258
    m, _, _ = oracle_model(nv)
    p = population32(nv, cells, seed=71, forces="shear", noise_pN=0.5, box=6.0)
    h = make_handle(npfem, nv, "fp64", tol=0.0, max_iter=3, armijo_noise=0.0, warm_history=2)
    xg, vg, sts = _stats_steps(npfem, h, p, steps, dtype="float64")
    assert all((s["iterations"] == 3).all() and (s["status"] == 1).all() for s in sts)
    o = O.make_opts(tol=0.0, max_iter=3)
    for c in range(cells):
        xc, vc, so = m.trajectory(p["x"][c], p["v"][c], p["f"][c], steps, o, carry_pairs=True, carry_max_iters=3)
        assert [s.iterations for s in so] == [3] * steps
        assert max_rel_disp(xg[c], xc, m.lbar) <= 1e-10
        assert np.abs(vg[c] - vc).max() <= 1e-10 * m.lbar / DT
        # the carried pairs change the path: the oracle without them ends elsewhere
        xp, _, _ = m.trajectory(p["x"][c], p["v"][c], p["f"][c], steps, o, carry_pairs=False)
        assert max_rel_disp(xp, xc, m.lbar) > 1e-6


def test_carried_pairs_fp64_converged_trajectory(npfem):
    # converged steps (tol 1e-7): positions on the oracle's trajectory under the same
    # rule, and the carried pairs take fewer iterations than the temporal warm start
    # alone (oracle: 1.25 against 2.28 per step in steps 5-16)
    steps, cells, nv = 16, 3, 258
    m, _, _ = oracle_model(nv)
    p = population32(nv, cells, seed=72, forces="shear", noise_pN=0.5, box=6.0)
    its = {}
    for wh in (1, 2):
        h = make_handle(npfem, nv, "fp64", tol=1e-7, max_iter=200, armijo_noise=0.0, warm_history=wh)
        xg, _, sts = _stats_steps(npfem, h, p, steps, dtype="float64")
        assert all((s["status"] == 0).all() for s in sts)
        its[wh] = np.mean([s["iterations"].mean() for s in sts[4:]])
        o = O.make_opts(tol=1e-7, max_iter=200)
        for c in range(cells):
            xc, _, so = m.trajectory(p["x"][c], p["v"][c], p["f"][c], steps, o, carry_pairs=wh == 2,
                                     carry_max_iters=3)
            assert max_rel_disp(xg[c], xc, m.lbar) <= 1e-6
    assert its[2] < its[1] - 0.5, its


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_carried_pairs_converge_and_cut_iterations(npfem, prec):
    steps, cells = 20, 8
    m, _, _ = oracle_model(642)
    p = population32(642, cells, seed=90, forces="shear", noise_pN=0.5)
    if "plain20" not in _ORACLE:
        _ORACLE["plain20"] = oracle_steps(m, p["x"], p["v"], p["f"], steps=steps, tol=1e-10, max_iter=200)[0]
    xo = _ORACLE["plain20"]
    its = {}
    for wh in (1, 2):
        h = make_handle(npfem, 642, prec, tol=1e-6, warm_history=wh)
        xg, _, sts = _stats_steps(npfem, h, p, steps)
        assert all((s["status"] == 0).all() and (s["residual"] <= 1e-6).all() for s in sts)
        assert max_rel_disp(xg, xo, m.lbar) <= steps * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
        its[wh] = np.mean([s["iterations"].mean() for s in sts[5:]])
    assert its[2] < its[1], its


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_carried_pairs_mixed_resolutions(npfem, prec):
    """258/642/2562-vertex groups in one call: each group's records at its own offset
    (2562 vertices keep their vectors in the global per-block slots)."""
    import torch
    steps = 4
    sizes = [(2562, 2), (642, 3), (258, 3)]
    hs, ms, pops = [], [], []
    for k, (nv, c) in enumerate(sizes):
        hs.append(make_handle(npfem, nv, prec, tol=1e-6, warm_history=2))
        ms.append(oracle_model(nv)[0])
        pops.append(population32(nv, c, seed=120 + k, forces="shear", noise_pN=0.5, box=6.0))
    flat = lambda key: np.concatenate([W.to_soa(p[key]).ravel() for p in pops])
    xs, vs, fs = (torch.tensor(flat(k), dtype=torch.float32, device="cuda") for k in ("x", "v", "f"))
    total = sum(c for _, c in sizes)
    st = torch.zeros((total, 32), dtype=torch.uint8, device="cuda")
    iters = []
    for _ in range(steps):
        npfem.step(hs, [c for _, c in sizes], xs, vs, fs, DT, stats=st)
        sg = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(total)
        assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
        iters.append(sg["iterations"].copy())
    xg = xs.double().cpu().numpy()
    off = 0
    for k, ((nv, c), m, p) in enumerate(zip(sizes, ms, pops)):
        key = ("mixed", nv, c, 120 + k)
        if key not in _ORACLE:
            _ORACLE[key] = oracle_steps(m, p["x"], p["v"], p["f"], steps=steps, tol=1e-10, max_iter=200)[0]
        part = W.from_soa(xg[off:off + 3 * nv * c].reshape(c, 3, nv))
        off += 3 * nv * c
        assert max_rel_disp(part, _ORACLE[key], m.lbar) <= steps * 1e-5 + fp32_store_allowance(p["x"], m.lbar)


def test_carried_pairs_reset_with_a_new_layout(npfem):
    # a call with other cell counts starts a new trajectory: no correction, no pairs
    # (the step from y equals the plain one)
    m, _, _ = oracle_model(642)
    p = population32(642, 6, seed=91, forces="shear", noise_pN=0.5)
    h = make_handle(npfem, 642, "fp32", tol=1e-6, warm_history=2)
    _stats_steps(npfem, h, p, 3)
    q = {k: p[k][:4] for k in ("x", "v", "f")}
    xa, va, sa = gpu_step_device(h, q["x"], q["v"], q["f"])
    h0 = make_handle(npfem, 642, "fp32", tol=1e-6, warm_history=0)
    xb, vb, sb = gpu_step_device(h0, q["x"], q["v"], q["f"])
    assert np.array_equal(xa, xb) and np.array_equal(sa["iterations"], sb["iterations"])


def test_carried_pairs_left_out_while_solves_take_more_than_three_iterations(npfem):
    # noise redrawn every step: every solve takes 4 or more iterations, so the rule never
    # loads the carried pairs and the trajectory is the one without them, bit for bit
    # (compared while every cell's last solve took more than 3 iterations)
    import torch
    cells = 8
    p = population32(642, cells, seed=93, forces="shear", noise_pN=0.5)
    rng = np.random.default_rng(5)
    draws = [W.to_soa(p["f_shear"] + rng.normal(0, 0.5, p["x"].shape)) for _ in range(10)]
    out = {}
    for wh in (1, 2):
        h = make_handle(npfem, 642, "fp32", tol=1e-6, warm_history=wh)
        xs, vs = (torch.tensor(W.to_soa(p[k]), dtype=torch.float32, device="cuda") for k in ("x", "v"))
        st = torch.zeros((cells, 32), dtype=torch.uint8, device="cuda")
        xk, its = [], []
        for f in draws:
            fs = torch.tensor(f, dtype=torch.float32, device="cuda")
            npfem.step([h], [cells], xs, vs, fs, DT, stats=st)
            s = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(cells)
            assert (s["status"] == 0).all()
            xk.append(xs.cpu().numpy().copy())
            its.append(s["iterations"].copy())
        out[wh] = (xk, its)
    k = 0
    while k < len(draws) and (k == 0 or (out[1][1][k - 1] > 3).all()):
        assert np.array_equal(out[1][0][k], out[2][0][k]), k
        assert np.array_equal(out[1][1][k], out[2][1][k]), k
        k += 1
    assert k >= 5, (k, [i.min() for i in out[1][1]])
