"""Parity of the CUDA path (called through the C-ABI) with the FP64 CPU oracle.

Tolerances (stated per test):
  * FP64 GPU path, fixed iteration count, exact Armijo test: max_i |dx_i| / lbar <= 1e-10.
  * FP32 GPU path at tolerance 1e-6: max_i |dx_i| / lbar <= 1e-5, plus the FP32
    storage rounding of x_{n+1} (half an ulp of the largest coordinate) where cells
    sit far from the origin.
"""
import numpy as np
import pytest

from helpers import DT, fp32_store_allowance, gpu_step_device, max_rel_disp, oracle_model, oracle_steps, population32
from paper_1903_06479_gb300 import workloads as W

_ORACLE = {}  # oracle results shared by parametrisations with identical inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npfem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    N.lib()
    return N


def make_handle(N, n_verts, precision="fp32", **kw):
    rest, tris = W.discocyte(n_verts)
    mat = {k: kw.pop(k) for k in list(kw) if k in W.DEFAULT_MATERIAL}
    opts = N.default_opts(precision=precision, **kw)
    return N.Handle(rest, tris, N.material(**mat), opts, dt=DT)


# ---------------------------------------------------------------------------------
# setup: rest tables and the FP64 inverse
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("n_verts", [258, 642])
def test_setup_matches_oracle(npfem, n_verts):
    h = make_handle(npfem, n_verts, "fp64")
    m, rest, tris = oracle_model(n_verts)
    masses, sc = h.rest_info()
    assert np.allclose(masses, m.masses(), rtol=1e-12)
    assert abs(sc["V0"] - m.V0) < 1e-12 * m.V0 and abs(sc["A0"] - m.A0) < 1e-12 * m.A0
    assert abs(sc["lbar"] - m.lbar) < 1e-12 * m.lbar
    Ainv = h.inverse()
    H = m.hessian()
    assert np.abs(Ainv @ H - np.eye(n_verts)).max() < 1e-11
    assert np.abs(Ainv - Ainv.T).max() == 0.0


# ---------------------------------------------------------------------------------
# objective and gradient, energy by energy
# ---------------------------------------------------------------------------------
def _eval_case(n_verts, cells, seed):
    m, rest, tris = oracle_model(n_verts)
    rng = np.random.default_rng(seed)
    x = W.place_cells(rest, rng, cells, box=30.0)
    x = x + 0.03 * m.lbar * rng.standard_normal(x.shape)
    x[0] = x[0] * 1.02  # one cell with a volume error
    y = x + 0.002 * m.lbar * rng.standard_normal(x.shape)
    return m, x, y


@pytest.mark.parametrize("prec,tol_e,tol_g", [("fp64", 1e-11, 1e-10), ("fp32", 3e-5, 2e-4)])
@pytest.mark.parametrize("n_verts", [258, 642])
def test_eval_parity(npfem, prec, tol_e, tol_g, n_verts):
    import torch
    h = make_handle(npfem, n_verts, prec)
    cells = 6
    m, x, y = _eval_case(n_verts, cells, 3 + n_verts)
    td = torch.float64 if prec == "fp64" else torch.float32
    if prec == "fp32":
        x = x.astype(np.float32).astype(np.float64)
        y = y.astype(np.float32).astype(np.float64)
    xs = torch.tensor(W.to_soa(x), dtype=td, device="cuda")
    ys = torch.tensor(W.to_soa(y), dtype=td, device="cuda")
    g = torch.zeros_like(xs)
    parts = torch.zeros((cells, 8), dtype=torch.float64, device="cuda")
    h.eval(cells, xs, ys, g, parts)
    torch.cuda.synchronize()
    g = W.from_soa(g.double().cpu().numpy())
    parts = parts.cpu().numpy()
    for c in range(cells):
        E, G, P = m.objective(x[c], y[c])
        # parts: inertia, area, skalak, bend, volume energy, V, g, r
        for q, name in [(0, "inertia"), (1, "area"), (2, "skalak"), (3, "bend")]:
            assert abs(parts[c, q] - P[q]) <= tol_e * max(abs(P[q]), 1e-3 * abs(E)), (c, name, parts[c, q], P[q])
        assert abs(parts[c, 5] - P[5]) <= tol_e * P[5] * 10
        assert abs(parts[c, 6] - E) <= tol_e * abs(E)
        assert np.abs(g[c] - G).max() <= tol_g * np.abs(G).max(), (c, np.abs(g[c] - G).max(), np.abs(G).max())
        assert abs(parts[c, 7] - m.residual(G)) <= tol_g * m.residual(G)


# ---------------------------------------------------------------------------------
# one time step
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("n_verts,cells", [(258, 4), (642, 5)])
def test_step_parity_fp64_fixed_iterations(npfem, n_verts, cells):
    # tol = 0 and a fixed cap of 8 iterations: both sides take the same steps
    h = make_handle(npfem, n_verts, "fp64", tol=0.0, max_iter=8, armijo_noise=0.0)
    m, _, _ = oracle_model(n_verts)
    p = population32(n_verts, cells, seed=n_verts, forces="shear", noise_pN=1.0)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=0.0, max_iter=8)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-10
    for c in range(cells):
        assert sg["iterations"][c] == st[c].iterations


@pytest.mark.parametrize("n_verts,cells,seed", [(258, 6, 1), (642, 8, 2)])
def test_step_parity_fp32_at_tolerance(npfem, n_verts, cells, seed):
    h = make_handle(npfem, n_verts, "fp32", tol=1e-6)
    m, _, _ = oracle_model(n_verts)
    p = population32(n_verts, cells, seed=seed, forces="shear", noise_pN=0.5)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert all(s == 0 for s in sg["status"]), sg
    assert (sg["residual"] <= 1e-6).all()
    allow = fp32_store_allowance(p["x"], m.lbar)
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + allow
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-5


def test_step_parity_fp32_near_origin_strict(npfem):
    # cells within 10 um of the origin: the storage rounding is < 1e-6 lbar
    h = make_handle(npfem, 642, "fp32", tol=1e-6)
    m, _, _ = oracle_model(642)
    p = population32(642, 4, seed=9, forces="noise", noise_pN=2.0, box=2.0)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5


def test_several_steps_fp32(npfem):
    h = make_handle(npfem, 642, "fp32", tol=1e-6)
    m, _, _ = oracle_model(642)
    p = population32(642, 3, seed=4, forces="shear", gamma_fixed=1000.0, noise_pN=2.0, box=4.0)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], steps=5, tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=5)
    assert max_rel_disp(xg, xo, m.lbar) <= 5e-5


@pytest.mark.parametrize("prec,tune", [("fp32", False), ("bf16", False), ("bf16", True), ("tf32", False)])
def test_mixed_resolutions_one_step(npfem, prec, tune):
    """One step over 2562-, 642- and 258-vertex groups: a single persistent SIMT launch
    (FP32), cluster launches for the groups that fit the tensor-core kernel plus a SIMT
    launch for the rest (BF16), and the same after the autotuner picked each group's
    launch shape (which leaves x, v untouched)."""
    import torch
    sizes = [(2562, 2), (642, 3), (258, 3)]
    hs, ms, pops = [], [], []
    for k, (nv, c) in enumerate(sizes):
        hs.append(make_handle(npfem, nv, prec, tol=1e-6))
        ms.append(oracle_model(nv)[0])
        pops.append(population32(nv, c, seed=20 + k, forces="shear", noise_pN=0.5, box=6.0))
    flat = lambda key: np.concatenate([W.to_soa(p[key]).ravel() for p in pops])
    xs = torch.tensor(flat("x"), dtype=torch.float32, device="cuda")
    vs = torch.tensor(flat("v"), dtype=torch.float32, device="cuda")
    fs = torch.tensor(flat("f"), dtype=torch.float32, device="cuda")
    total = sum(c for _, c in sizes)
    st = torch.zeros((total, 32), dtype=torch.uint8, device="cuda")
    if tune:
        x0 = xs.clone()
        shapes = npfem.autotune(hs, [c for _, c in sizes], xs, vs, fs, DT, trial_steps=1)
        assert torch.equal(xs, x0)
        assert not shapes[0]["tensor_core"]  # 2562 vertices do not fit the cluster kernel
        assert all(sh["simt_threads"] in (512, 640) for sh in shapes)
    npfem.step(hs, [c for _, c in sizes], xs, vs, fs, DT, stats=st)
    torch.cuda.synchronize()
    sg = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(total)
    assert (sg["status"] == 0).all()
    xg = xs.double().cpu().numpy()
    off = 0
    for k, ((nv, c), m, p) in enumerate(zip(sizes, ms, pops)):
        key = ("mixed", nv, c, 20 + k)
        if key not in _ORACLE:  # the same inputs for every parametrisation
            _ORACLE[key] = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)[0]
        xo = _ORACLE[key]
        part = W.from_soa(xg[off:off + 3 * nv * c].reshape(c, 3, nv))
        off += 3 * nv * c
        assert max_rel_disp(part, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


def test_step_host_matches_device(npfem):
    # the same step twice from the same state: without the temporal warm start, which
    # would start the second from the first one's answer
    h = make_handle(npfem, 642, "fp32", tol=1e-6, warm_history=0)
    p = population32(642, 4, seed=5)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    xh = W.to_soa(p["x"]).astype(np.float32)
    vh = W.to_soa(p["v"]).astype(np.float32)
    fh = W.to_soa(p["f"]).astype(np.float32)
    st = np.zeros(4, dtype=npfem.CELL_STATS_DTYPE)
    h.step_host(xh, vh, fh, st)
    assert np.array_equal(W.from_soa(xh.astype(np.float64)), xg)
    assert np.array_equal(st["iterations"], sg["iterations"])


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_step_host_pinned_in_place_matches_device(npfem, prec):
    # pinned host buffers are stepped in place (the kernels read and write them over the
    # host link): three steps of a trajectory, bit for bit those of device buffers (the
    # idle-SM blocks off on both sides, as npfem_step_host runs)
    import torch
    cells = 6
    p = population32(642, cells, seed=7, forces="shear", noise_pN=0.5)
    hd = make_handle(npfem, 642, prec, tol=1e-6, fill_idle_sms=0)
    hh = make_handle(npfem, 642, prec, tol=1e-6, fill_idle_sms=0)
    xg, vg, sg = gpu_step_device(hd, p["x"], p["v"], p["f"], steps=3)
    xs, vs, fs = (torch.tensor(W.to_soa(p[k]), dtype=torch.float32).pin_memory() for k in ("x", "v", "f"))
    st = torch.zeros((cells, 32), dtype=torch.uint8).pin_memory()
    sv = st.numpy().view(npfem.CELL_STATS_DTYPE).reshape(cells)
    for _ in range(3):
        hh.step_host(xs.numpy(), vs.numpy(), fs.numpy(), sv)
    assert np.array_equal(W.from_soa(xs.double().numpy()), xg)
    assert np.array_equal(W.from_soa(vs.double().numpy()), vg)
    assert np.array_equal(sv["iterations"], sg["iterations"]) and (sv["status"] == 0).all()


# ---------------------------------------------------------------------------------
# edge cases and failure reporting (host-made failures only)
# ---------------------------------------------------------------------------------
def test_zero_cells_and_invalid_args(npfem):
    import torch
    h = make_handle(npfem, 258, "fp32")
    x = torch.zeros(3 * 258, device="cuda")
    npfem.step([h], [0], x, x, x, DT)  # no work, no error
    with pytest.raises(npfem.NpfemError) as e:
        npfem.step([h], [1], x, x, x, DT * 2)
    assert e.value.code == -1
    rest, tris = W.discocyte(258)
    with pytest.raises(npfem.NpfemError) as e:
        npfem.Handle(rest, tris[:-1], opts=npfem.default_opts())  # open mesh
    assert e.value.code == -2
    bad = tris.copy()
    bad[:, [1, 2]] = bad[:, [2, 1]]  # clockwise: negative rest volume
    with pytest.raises(npfem.NpfemError) as e:
        npfem.Handle(rest, bad, opts=npfem.default_opts())
    assert e.value.code == -2


def test_nonfinite_force_flags_only_that_cell(npfem):
    h = make_handle(npfem, 642, "fp32", tol=1e-6)
    p = population32(642, 3, seed=6)
    p["f"][1, 7, 0] = np.nan
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert list(sg["status"]) == [0, 3, 0]
    assert np.array_equal(xg[1], p["x"][1]) and (vg[1] == 0).all()
    assert np.isfinite(xg).all()


def test_iteration_cap_reports_maxiter(npfem):
    h = make_handle(npfem, 642, "fp32", tol=1e-12, max_iter=1)
    p = population32(642, 2, seed=7, forces="noise", noise_pN=50.0)
    _, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert (sg["status"] == 1).all() and (sg["iterations"] == 1).all()


# ---------------------------------------------------------------------------------
# full size: 16384 cells of 642 vertices in the benchmark's launch configuration,
# checked on sampled cells against the oracle and by invariants on all cells
# ---------------------------------------------------------------------------------
def test_full_size_sampled(npfem):
    h = make_handle(npfem, 642, "fp32", tol=1e-6)
    m, _, _ = oracle_model(642)
    p = population32(642, 16384, seed=3, forces="shear", gamma_fixed=1000.0, noise_pN=2.0)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    assert np.isfinite(xg).all() and np.isfinite(vg).all()
    Mv = m.masses()
    # sum m (v_{n+1} - v_n) = h sum F_ext - h sum grad g (internal forces sum to zero,
    # the post step conserves momentum), and |h sum grad g| <= n r lbar max(m) / h
    P_gpu = (Mv[None, :, None] * vg).sum(1)
    P_exp = (Mv[None, :, None] * p["v"]).sum(1) + DT * p["f"].sum(1)
    bound = 642 * sg["residual"].astype(np.float64) * m.lbar * Mv.max() / DT
    assert (np.abs(P_gpu - P_exp).max(1) <= bound + 1e-4 * np.abs(P_exp).max(1)).all()
    sample = np.random.default_rng(0).choice(16384, 8, replace=False)
    xo, vo, _ = oracle_steps(m, p["x"][sample], p["v"][sample], p["f"][sample], tol=1e-10, max_iter=200)
    assert max_rel_disp(xg[sample], xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


# ---------------------------------------------------------------------------------
# BF16 tensor-core contraction (A^-1 resident in tensor memory across a cluster):
# the direction changes only through H0, so the converged step must still meet the
# FP32 parity tolerance at the same residual tolerance.
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("n_verts,cells,refine", [(642, 13, 1), (642, 8, 0), (258, 7, 1)])
def test_step_bf16_tensor_core(npfem, n_verts, cells, refine):
    h = make_handle(npfem, n_verts, "bf16", tol=1e-6, refine=refine)
    m, _, _ = oracle_model(n_verts)
    p = population32(n_verts, cells, seed=40 + n_verts, forces="shear", noise_pN=0.5)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    h.check_device()
    assert (sg["status"] == 0).all(), sg
    assert (sg["residual"] <= 1e-6).all()
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-5


def test_bf16_iterations_close_to_fp32(npfem):
    p = population32(642, 64, seed=50, forces="shear", noise_pN=0.5)
    out = {}
    for prec in ("fp32", "bf16"):
        h = make_handle(npfem, 642, prec, tol=1e-6)
        _, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
        out[prec] = sg["iterations"].mean()
    assert out["bf16"] <= out["fp32"] + 1.0, out


def test_bf16_full_size_sampled(npfem):
    h = make_handle(npfem, 642, "bf16", tol=1e-6)
    m, _, _ = oracle_model(642)
    p = population32(642, 16384, seed=3, forces="shear", gamma_fixed=1000.0, noise_pN=2.0)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    h.check_device()
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    sample = np.random.default_rng(1).choice(16384, 8, replace=False)
    xo, vo, _ = oracle_steps(m, p["x"][sample], p["v"][sample], p["f"][sample], tol=1e-10, max_iter=200)
    assert max_rel_disp(xg[sample], xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


@pytest.mark.parametrize("n_verts,cells,refine", [(642, 13, 1), (642, 8, 0), (258, 7, 1), (2562, 2, 0)])
def test_step_tf32_tensor_core(npfem, n_verts, cells, refine):
    # TF32 A^-1 streamed through the tensor cores by every SIMT block (2562 vertices: 21
    # row tiles, 336 accumulator columns)
    h = make_handle(npfem, n_verts, "tf32", tol=1e-6, refine=refine)
    m, _, _ = oracle_model(n_verts)
    p = population32(n_verts, cells, seed=40 + n_verts, forces="shear", noise_pN=0.5)
    key = ("tc", n_verts, cells)
    if key not in _ORACLE:
        _ORACLE[key] = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xo, vo, st = _ORACLE[key]
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    h.check_device()
    assert (sg["status"] == 0).all(), sg
    assert (sg["residual"] <= 1e-6).all()
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-5


def test_tf32_iterations_close_to_fp32(npfem):
    # the TF32 contraction changes the direction by ~2^-11 relative: iteration counts stay
    # those of the FP32 contraction
    p = population32(642, 64, seed=50, forces="shear", noise_pN=0.5)
    out = {}
    for prec in ("fp32", "tf32"):
        h = make_handle(npfem, 642, prec, tol=1e-6, warm_history=0)
        _, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
        out[prec] = sg["iterations"].mean()
    assert out["tf32"] <= out["fp32"] + 0.5, out


def test_tf32_full_size_sampled(npfem):
    h = make_handle(npfem, 642, "tf32", tol=1e-6)
    m, _, _ = oracle_model(642)
    p = population32(642, 16384, seed=3, forces="shear", gamma_fixed=1000.0, noise_pN=2.0)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    h.check_device()
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    sample = np.random.default_rng(1).choice(16384, 8, replace=False)
    xo, vo, _ = oracle_steps(m, p["x"][sample], p["v"][sample], p["f"][sample], tol=1e-10, max_iter=200)
    assert max_rel_disp(xg[sample], xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


def _volumes(x, tris):
    a, b, c = x[:, tris[:, 0]], x[:, tris[:, 1]], x[:, tris[:, 2]]
    return np.einsum("cti,cti->ct", a, np.cross(b, c)).sum(1) / 6.0


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_multistep_drift_against_fp64_oracle(npfem, prec):
    """20 steps of 8 cells under N(0, 2 pN) noise plus 1000/s shear: positions and
    volumes against the FP64 oracle (run to 1e-10).  Each step converges to 1e-6 and
    carries at most the one-step bound 1e-5 l̄ (FP32 and BF16 alike); errors of
    successive steps add at most linearly, so 20 steps stay within 2e-4 l̄, and the
    relative volume error within 3 * 2e-4 l̄ / R (R the cell's mean radius)."""
    steps = 20
    h = make_handle(npfem, 642, prec, tol=1e-6)
    m, rest, tris = oracle_model(642)
    p = population32(642, 8, seed=60, forces="shear", gamma_fixed=1000.0, noise_pN=2.0)
    if "drift" not in _ORACLE:
        _ORACLE["drift"] = oracle_steps(m, p["x"], p["v"], p["f"], steps=steps, tol=1e-10, max_iter=200)[0]
    xo = _ORACLE["drift"]
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=steps)
    assert (sg["status"] == 0).all()
    drift = max_rel_disp(xg, xo, m.lbar)
    assert drift <= steps * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
    R = np.linalg.norm(rest - rest.mean(0), axis=1).mean()
    verr = np.abs(_volumes(xg, tris) / _volumes(xo, tris) - 1.0).max()
    assert verr <= 3 * steps * 1e-5 * m.lbar / R


def test_bf16_idle_sm_fill_matches_clusters_only(npfem):
    """With more cells than cluster blocks, SMs the clusters leave idle solve cells with
    the SIMT kernel from the same work counter; every cell converges either way and the
    two splits agree to the solver tolerance (and both to the oracle on a sample)."""
    cells = 400
    m, _, _ = oracle_model(642)
    p = population32(642, cells, seed=70, forces="shear", noise_pN=0.5)
    out = {}
    for fill in (0, 1):
        h = make_handle(npfem, 642, "bf16", tol=1e-6, fill_idle_sms=fill)
        n0 = npfem.launch_count()
        xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=2)
        out[fill] = (xg, npfem.launch_count() - n0)
        h.check_device()
        assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    assert max_rel_disp(out[0][0], out[1][0], m.lbar) <= 2e-5
    # clusters only: one launch on the first step; on the second (temporal warm start)
    # the first-iterate pass and the clusters
    assert out[0][1] == 3 and out[1][1] >= 3
    sample = [0, 137, 399]
    xo, _, _ = oracle_steps(m, p["x"][sample], p["v"][sample], p["f"][sample], steps=2, tol=1e-10, max_iter=200)
    assert max_rel_disp(out[1][0][sample], xo, m.lbar) <= 2e-5 + fp32_store_allowance(p["x"], m.lbar)


def test_single_cell_fp64_ten_steps(npfem):
    """One 258-vertex discocyte, FP64 on the GPU, i.i.d. N(0, 1 pN) forces from seed 0,
    10 steps at tolerance 1e-8 with the iteration cap 50: the same iterates as the
    FP64 oracle (the FP64 path differs from it only by rounding order)."""
    h = make_handle(npfem, 258, "fp64", tol=1e-8, max_iter=50, armijo_noise=0.0, warm_history=0)
    m, _, _ = oracle_model(258)
    p = W.population(258, 1, 0, forces="noise", noise_pN=1.0)
    xo, vo, so = oracle_steps(m, p["x"], p["v"], p["f"], steps=10, tol=1e-8, max_iter=50)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=10, dtype="float64")
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-8).all()
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_graph_replay_matches_eager_steps(npfem, prec):
    """Three steps captured as one CUDA graph and replayed equal three eager steps:
    bitwise for the FP32 path (each cell's arithmetic does not depend on the block that
    takes it), to the solver tolerance for BF16 (the idle-SM split between tensor-core
    and SIMT blocks is dynamic)."""
    import torch
    m, rest, tris = oracle_model(642)
    # eager and captured steps start from the same state: no temporal warm start
    h = make_handle(npfem, 642, prec, tol=1e-6, warm_history=0)
    p = population32(642, 300, seed=80, forces="shear", noise_pN=0.5)
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    xa, va, f = mk(p["x"]), mk(p["v"]), mk(p["f"])
    xb, vb = xa.clone(), va.clone()
    for _ in range(3):
        npfem.step([h], [300], xa, va, f, DT)
    g = npfem.StepGraph([h], [300], xb, vb, f, DT, steps=3)
    assert torch.equal(xb, mk(p["x"]))  # creation does not touch the state
    n0 = npfem.launch_count()
    g.launch()
    torch.cuda.synchronize()
    assert npfem.launch_count() > n0
    g.close()
    if prec == "fp32":
        assert torch.equal(xa, xb) and torch.equal(va, vb)
    else:
        assert max_rel_disp(W.from_soa(xa.double().cpu().numpy()), W.from_soa(xb.double().cpu().numpy()),
                            m.lbar) <= 3e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_temporal_warm_start(npfem, prec):
    """With warm_history each step starts from y + (x_n - y_{n-1}) of the same cell: the
    steps still converge to the tolerance (positions against the FP64 oracle after 10
    steps within the linear accumulation of the one-step bound) and take fewer
    iterations than from y."""
    steps = 10
    m, _, _ = oracle_model(642)
    p = population32(642, 8, seed=90, forces="shear", noise_pN=0.5)
    if "temporal" not in _ORACLE:
        _ORACLE["temporal"] = oracle_steps(m, p["x"], p["v"], p["f"], steps=steps, tol=1e-10, max_iter=200)[0]
    xo = _ORACLE["temporal"]
    its = {}
    for hist in (0, 1):
        h = make_handle(npfem, 642, prec, tol=1e-6, warm_history=hist)
        xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=steps)
        assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
        assert max_rel_disp(xg, xo, m.lbar) <= steps * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
        its[hist] = sg["iterations"].mean()  # iterations of the last step
    assert its[1] < its[0] - 1.0, its


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_compensated_positions(npfem, prec):
    """With the temporal warm start the FP32 positions carry their rounding residue from
    step to step.  Rounding x to FP32 in absolute coordinates perturbs the shape by up
    to half an ulp of ~60 um each step, which keeps settled trajectories near two
    iterations per step (test_oracle_rounding.py shows it on the FP64 oracle).
    Compensated, the GPU trajectory takes <= 1 iteration per step on average once it
    has settled, and stays on the FP64 oracle's positions."""
    steps = 100
    m, _, _ = oracle_model(642)
    p = population32(642, 8, seed=90, forces="shear", noise_pN=0.5)
    h = make_handle(npfem, 642, prec, tol=1e-6, warm_history=1)
    import torch
    xs, vs, fs = (torch.tensor(W.to_soa(p[k]), dtype=torch.float32, device="cuda") for k in ("x", "v", "f"))
    st = torch.zeros((8, 32), dtype=torch.uint8, device="cuda")
    its = []
    need = 0
    for k in range(steps):
        npfem.step([h], [8], xs, vs, fs, h.dt, stats=st)
        s = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE).reshape(8)
        assert (s["status"] == 0).all() and (s["residual"] <= 1e-6).all()
        its.append(s["iterations"].mean())
        it, ev = s["iterations"], s["evaluations"]
        if prec == "bf16" and k >= 1 and (k == 1 or 2 * need <= 8):
            # the first-iterate pass evaluated (at most half of the cells needed
            # iterations in the step before): it accepts with one evaluation, and a cell
            # it leaves to the clusters is evaluated there again at the same point
            assert (ev[it == 0] == 1).all() and (ev[it > 0] >= it[it > 0] + 2).all(), (k, it, ev)
        else:
            assert (ev >= it + 1).all(), (k, it, ev)
        need = int((it > 0).sum())
    assert np.mean(its[-40:]) <= 1.0, its[-40:]
    if "compensated" not in _ORACLE:
        # 1e-8: two orders below the GPU's tolerance, which sets the bound below
        _ORACLE["compensated"] = oracle_steps(m, p["x"], p["v"], p["f"], steps=steps, tol=1e-8, max_iter=200)[0]
    xg = W.from_soa(xs.double().cpu().numpy())
    assert max_rel_disp(xg, _ORACLE["compensated"], m.lbar) <= steps * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
