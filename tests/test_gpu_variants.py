"""Solver variants the paper describes, on the GPU against the FP64 oracle.

* Local/global alternating solver (Appendix A, Eq. x_star): projective energies only,
  no L-BFGS history (lbfgs_m = 0) and step length fixed at 1; its objective never
  increases from one iteration to the next.
* Original Skalak law (Sec. 2.1.3 with D = 0) next to the modified law (D = 35).
* Stiffness-proportional Rayleigh damping (Sec. 2.1.4, beta_D > 0): M~ = M + h beta_D L
  is not diagonal, so the first guess of Eq. preOptimizationNewton applies M~^-1 and
  the inertia term couples vertices.

Tolerances are those of the other parity tests: FP64 with a fixed iteration count
and the exact Armijo test, max |dx| / lbar <= 1e-10; FP32 and BF16 at residual 1e-6,
max |dx| / lbar <= 1e-5 plus the FP32 storage rounding of x_{n+1}.
"""
import numpy as np
import pytest

from helpers import DT, fp32_store_allowance, gpu_step_device, max_rel_disp, oracle_model, oracle_steps, population32
from paper_1903_06479_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PURE_PD = dict(B=0.0, D=0.0, k_mat_hess=0.0)  # area preservation, bending, volume: projective terms only
BETA = dict(beta_D=0.01)  # the paper's parameter table, read in microseconds


@pytest.fixture(scope="module")
def npfem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    N.lib()
    return N


def make_handle(N, n_verts, precision, mat, **opts):
    rest, tris = W.discocyte(n_verts)
    return N.Handle(rest, tris, N.material(**mat), N.default_opts(precision=precision, **opts), dt=DT)


# ---------------------------------------------------------------------------------
# local/global solver (Appendix A)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("n_verts,cells", [(258, 3), (642, 3)])
def test_local_global_fp64_fixed_iterations(npfem, n_verts, cells):
    lg = dict(lbfgs_m=0, fixed_alpha=1, tol=0.0, max_iter=8)
    h = make_handle(npfem, n_verts, "fp64", PURE_PD, armijo_noise=0.0, **lg)
    m, _, _ = oracle_model(n_verts, **PURE_PD)
    p = population32(n_verts, cells, seed=70 + n_verts, forces="noise", noise_pN=200.0, box=10.0)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], **lg)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-10
    assert (sg["iterations"] == 8).all() and (sg["status"] == 1).all()  # MAXITER with tol = 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_local_global_objective_never_increases(npfem, prec):
    # the same cells stepped with caps of 0..10 iterations: the final objective
    # (per-cell stats) must not increase with the cap (Appendix A)
    import torch
    m, _, _ = oracle_model(258, **PURE_PD)
    p = population32(258, 4, seed=77, forces="noise", noise_pN=300.0, box=10.0)
    objs = []
    for k in range(0, 11):
        h = make_handle(npfem, 258, prec, PURE_PD, lbfgs_m=0, fixed_alpha=1, tol=0.0, max_iter=k, armijo_noise=0.0,
                        warm_history=0)
        _, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64" if prec == "fp64" else "float32")
        objs.append(sg["objective"].copy())
        h.close()
    objs = np.array(objs)
    slack = 1e-13 if prec == "fp64" else 1e-6  # the objective's own rounding in FP32
    assert (objs[1:] <= objs[:-1] + slack * np.abs(objs[:-1])).all(), objs
    assert (objs[-1] < objs[0]).all()


def test_local_global_fp32_fixed_iterations(npfem):
    lg = dict(lbfgs_m=0, fixed_alpha=1, tol=0.0, max_iter=8)
    h = make_handle(npfem, 642, "fp32", PURE_PD, **lg)
    m, _, _ = oracle_model(642, **PURE_PD)
    p = population32(642, 3, seed=72, forces="noise", noise_pN=200.0, box=10.0)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], **lg)
    xg, vg, _ = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


# ---------------------------------------------------------------------------------
# original (D = 0) and modified (D = 35) Skalak law
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("D", [0.0, 35.0])
def test_skalak_law_fp64_fixed_iterations(npfem, D):
    h = make_handle(npfem, 258, "fp64", dict(D=D), tol=0.0, max_iter=8, armijo_noise=0.0)
    m, _, _ = oracle_model(258, D=D)
    p = population32(258, 3, seed=80, forces="noise", noise_pN=100.0, box=10.0)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=0.0, max_iter=8)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    assert [int(s) for s in sg["iterations"]] == [s.iterations for s in st]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_original_skalak_at_tolerance(npfem, prec):
    h = make_handle(npfem, 642, prec, dict(D=0.0), tol=1e-6)
    m, _, _ = oracle_model(642, D=0.0)
    p = population32(642, 5, seed=81, forces="shear", noise_pN=0.5)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"])
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all(), sg
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


def test_original_and_modified_skalak_differ_at_large_strain(npfem):
    # the D term stiffens large strains: under the same large force the modified law
    # deforms less (a check that D reaches the kernel at all)
    p = population32(258, 2, seed=82, forces="noise", noise_pN=3000.0, box=10.0)
    out = {}
    for D in (0.0, 35.0):
        h = make_handle(npfem, 258, "fp64", dict(D=D), tol=1e-8, max_iter=200)
        xg, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
        assert (sg["status"] == 0).all()
        out[D] = xg
    m, _, _ = oracle_model(258)
    assert max_rel_disp(out[0.0], out[35.0], m.lbar) > 1e-6


# ---------------------------------------------------------------------------------
# Rayleigh damping with beta_D > 0
# ---------------------------------------------------------------------------------
def test_rayleigh_beta_first_guess(npfem):
    # max_iter = 0: x_{n+1} is the first guess y = x_n + M~^-1 (h M v_n + h^2 F_ext);
    # v_{n+1} = (y - x_n)/h before the post-step; compare y against the oracle's
    m, _, _ = oracle_model(258, **BETA)
    h = make_handle(npfem, 258, "fp64", BETA, tol=0.0, max_iter=0, armijo_noise=0.0)
    p = population32(258, 3, seed=90, forces="noise", noise_pN=5.0, box=10.0)
    rng = np.random.default_rng(91)
    p["v"] = (0.02 * rng.standard_normal(p["v"].shape)).astype(np.float32).astype(np.float64)
    xg, _, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
    for c in range(3):
        y = m.first_guess(p["x"][c], p["v"][c], p["f"][c])
        assert np.abs(xg[c] - y).max() <= 1e-10 * m.lbar
        # and it is not the lumped first guess
        Mv = m.masses()[:, None]
        yl = p["x"][c] + DT * p["v"][c] + DT ** 2 * p["f"][c] / Mv
        assert np.abs(y - yl).max() > 1e-4 * np.abs(yl - p["x"][c]).max()


def test_rayleigh_beta_eval_parity(npfem):
    import torch
    m, rest, tris = oracle_model(258, **BETA)
    h = make_handle(npfem, 258, "fp64", BETA)
    rng = np.random.default_rng(92)
    x = W.place_cells(rest, rng, 3, box=20.0) + 0.03 * m.lbar * rng.standard_normal((3, 258, 3))
    y = x + 0.01 * m.lbar * rng.standard_normal(x.shape)
    xs = torch.tensor(W.to_soa(x), dtype=torch.float64, device="cuda")
    ys = torch.tensor(W.to_soa(y), dtype=torch.float64, device="cuda")
    g = torch.zeros_like(xs)
    parts = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    h.eval(3, xs, ys, g, parts)
    torch.cuda.synchronize()
    g = W.from_soa(g.cpu().numpy())
    parts = parts.cpu().numpy()
    for c in range(3):
        E, G, P = m.objective(x[c], y[c])
        assert abs(parts[c, 0] - P[0]) <= 1e-11 * abs(P[0])  # inertia with h beta_D L
        assert abs(parts[c, 6] - E) <= 1e-11 * abs(E)
        assert np.abs(g[c] - G).max() <= 1e-10 * np.abs(G).max()


@pytest.mark.parametrize("n_verts", [258, 642])
def test_rayleigh_beta_fp64_fixed_iterations(npfem, n_verts):
    h = make_handle(npfem, n_verts, "fp64", BETA, tol=0.0, max_iter=8, armijo_noise=0.0)
    m, _, _ = oracle_model(n_verts, **BETA)
    p = population32(n_verts, 3, seed=93, forces="shear", noise_pN=1.0)
    xo, vo, st = oracle_steps(m, p["x"], p["v"], p["f"], tol=0.0, max_iter=8)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], dtype="float64")
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-10
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 1e-10
    assert [int(s) for s in sg["iterations"]] == [s.iterations for s in st]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_rayleigh_beta_at_tolerance(npfem, prec):
    h = make_handle(npfem, 642, prec, BETA, tol=1e-6)
    m, _, _ = oracle_model(642, **BETA)
    p = population32(642, 6, seed=94, forces="shear", noise_pN=0.5)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200, steps=3)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=3)
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all(), sg
    assert max_rel_disp(xg, xo, m.lbar) <= 3 * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
    assert max_rel_disp(DT * vg, DT * vo, m.lbar) <= 3 * 1e-5


def test_rayleigh_beta_rejects_learned_warm_start(npfem):
    h = make_handle(npfem, 258, "fp32", BETA)
    P = np.zeros(npfem.mlp_nparam(), dtype=np.float32)
    P[-12:-3] = 1.0  # sigma
    with pytest.raises(npfem.NpfemError):
        h.set_warmstart(P, 1)


# ---------------------------------------------------------------------------------
# set-up: the one-time FP64 inversion (Sec. 2.1.1) in a handful of launches
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("prec,mat", [("fp32", {}), ("bf16", {}), ("fp64", BETA), ("bf16", BETA)])
def test_setup_launch_count_and_inverse(npfem, prec, mat):
    c0 = npfem.launch_count()
    h = make_handle(npfem, 642, prec, mat)
    launches = npfem.launch_count() - c0
    assert launches < 50, launches
    m, _, _ = oracle_model(642, **mat)
    Ainv = h.inverse()
    assert np.abs(Ainv @ m.hessian() - np.eye(642)).max() < 1e-11
