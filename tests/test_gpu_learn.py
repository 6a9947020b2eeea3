"""GPU parity and benefit of the learned warm start (an addition to the paper's
method): the library's training kernels against the oracle's FP64 network, its
feature kernels against the oracle's features, and the iteration count of a
trained network against the plain first guess at the same residual tolerance."""
import numpy as np
import pytest

from helpers import DT, fp32_store_allowance, gpu_step_device, max_rel_disp, oracle_model, oracle_steps, population32
from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W
from test_oracle_pins_learn import rand_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def npfem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_06479_gb300 import npfem as N
    N.lib()
    return N


def dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")


def test_mlp_loss_and_gradient_match_oracle(npfem):
    import torch
    rng = np.random.default_rng(10)
    P = rand_params(11).astype(np.float32)
    feat = rng.normal(0, 1, (300, 9)).astype(np.float32)  # 4 full tiles and a partial one
    tgt = rng.normal(0, 1, (300, 3)).astype(np.float32)
    idx = rng.permutation(300)[:257].astype(np.int32)
    grad = torch.zeros(npfem.mlp_nparam(), device="cuda")
    loss = torch.zeros(1, device="cuda")
    npfem.mlp_loss_grad(dev(P), dev(feat), dev(tgt), dev(idx, torch.int32), 257, grad, loss)
    lo, go = O.mlp_loss_grad(P.astype(np.float64), feat[idx].astype(np.float64), tgt[idx].astype(np.float64), True)
    g = grad.cpu().numpy()
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def test_adam_step(npfem):
    rng = np.random.default_rng(12)
    n = npfem.mlp_nparam()
    P, m, v, g = (rng.normal(0, 1, n).astype(np.float32) for _ in range(4))
    v = np.abs(v)
    tp, tm, tv = dev(P), dev(m), dev(v)
    npfem.mlp_adam(tp, tm, tv, dev(g), 3, lr=1e-3)
    k = n - 21
    m2 = 0.9 * m[:k] + 0.1 * g[:k]
    v2 = 0.999 * v[:k] + 0.001 * g[:k] ** 2
    P2 = P[:k] - 1e-3 * (m2 / (1 - 0.9 ** 3)) / (np.sqrt(v2 / (1 - 0.999 ** 3)) + 1e-8)
    assert np.allclose(tp.cpu().numpy()[:k], P2, rtol=1e-5, atol=1e-7)
    assert np.array_equal(tp.cpu().numpy()[k:], P[k:])


def test_features_and_targets_match_oracle(npfem):
    import torch
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT)
    p = population32(642, 3, seed=13, forces="shear", noise_pN=1.0, box=20.0)
    p["x"] = (p["x"] + 0.01 * m.lbar * np.random.default_rng(14).standard_normal(p["x"].shape)).astype(np.float32).astype(np.float64)
    xn = p["x"] + 1e-4 * np.random.default_rng(15).standard_normal(p["x"].shape)
    xn = xn.astype(np.float32).astype(np.float64)
    feat = torch.zeros((3 * 642, 9), device="cuda")
    tgt = torch.zeros((3 * 642, 3), device="cuda")
    h.ws_features(3, dev(W.to_soa(p["x"])), dev(W.to_soa(p["v"])), dev(W.to_soa(p["f"])), feat,
                  x_next=dev(W.to_soa(xn)), target=tgt)
    fg = feat.cpu().numpy().reshape(3, 642, 9)
    tg = tgt.cpu().numpy().reshape(3, 642, 3)
    for c in range(3):
        y = m.first_guess(p["x"][c], p["v"][c], p["f"][c])
        fo, R = m.ws_features(y, p["f"][c])
        scale = np.abs(fo).max(0)
        assert np.all(np.abs(fg[c] - fo).max(0) <= 2e-4 * scale + 1e-9), (np.abs(fg[c] - fo).max(0), scale)
        to = (xn[c] - y) @ R
        assert np.abs(tg[c] - to).max() <= 2e-4 * np.abs(to).max()


def test_warm_start_guess_matches_oracle(npfem):
    import torch
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT)
    P = rand_params(16)
    P[-3:] = 1e-4  # small output scale: a plausible correction
    h.set_warmstart(P.astype(np.float32), 1)
    p = population32(642, 2, seed=17, forces="shear", noise_pN=1.0, box=20.0)
    x1 = torch.zeros((2, 3, 642), device="cuda")
    h.ws_guess(2, dev(W.to_soa(p["x"])), dev(W.to_soa(p["v"])), dev(W.to_soa(p["f"])), x1)
    xg = W.from_soa(x1.double().cpu().numpy())
    for c in range(2):
        xo = m.ws_guess(P.astype(np.float32).astype(np.float64), p["x"][c], p["v"][c], p["f"][c], True)
        y = m.first_guess(p["x"][c], p["v"][c], p["f"][c])
        corr = np.abs(xo - y).max()
        assert corr > 1e-6
        assert np.abs(xg[c] - xo).max() <= 1e-3 * corr + 2 * np.spacing(np.float32(25.0))


@pytest.mark.parametrize("prec,static,mode", [("bf16", False, 1), ("fp32", False, 1), ("fp32", True, 1),
                                              ("bf16", False, 2)])
def test_warm_started_step_matches_oracle(npfem, prec, static, mode):
    """Same converged step from a learned first iterate: through the separate
    warm-start launch (npfem_step, SIMT and tensor-core kernels) and through the
    solver's in-kernel warm start (npfem_step_static)."""
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision=prec, refine=0, tol=1e-6), dt=DT)
    P = rand_params(18)
    P[-3:] = 1e-4
    h.set_warmstart(P.astype(np.float32), mode)
    p = population32(642, 6, seed=19, forces="shear", noise_pN=0.5)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], static=static)
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    assert max_rel_disp(xg, xo, m.lbar) <= 1e-5 + fp32_store_allowance(p["x"], m.lbar)


def test_trained_network_cuts_iterations(npfem):
    import torch
    from paper_1903_06479_gb300 import learn
    rest, tris = W.discocyte(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32", tol=1e-6, warm_history=0),
                     dt=DT)
    P, info = learn.train_warmstart(h, n_cells=256, steps=60, seed=200, train_steps=1500)
    assert info["loss_final"] < 0.5 * info["loss_init"]
    # held-out cells, advanced 40 plain steps from rest, then one step each way
    p = W.population(642, 128, 999, forces="shear", noise_pN=0.5)
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    x, v, f = mk(p["x"]), mk(p["v"]), mk(p["f"])
    for _ in range(40):
        npfem.step([h], [128], x, v, f, DT)
    iters = {}
    for mode in (0, 1):
        h.set_warmstart(P if mode else None, mode)
        xa, va = x.clone(), v.clone()
        st = torch.zeros((128, 32), dtype=torch.uint8, device="cuda")
        npfem.step([h], [128], xa, va, f, DT, stats=st)
        s = st.cpu().numpy().view(npfem.CELL_STATS_DTYPE)
        assert (s["status"] == 0).all() and (s["residual"] <= 1e-6).all()
        iters[mode] = float(s["iterations"].mean())
    assert iters[1] < iters[0] - 0.5, iters


# ---------------------------------------------------------------------------------
# temporal network along a trajectory
# ---------------------------------------------------------------------------------
def _temporal_inputs(seed, m, cells=3):
    p = population32(642, cells, seed=seed, forces="shear", noise_pN=1.0, box=20.0)
    rng = np.random.default_rng(seed + 1)
    r32 = lambda a: a.astype(np.float32).astype(np.float64)
    p["x"] = r32(p["x"] + 0.01 * m.lbar * rng.standard_normal(p["x"].shape))
    f_prev = r32(p["f"] + rng.normal(0, 0.5, p["f"].shape))
    c1 = r32(1e-3 * rng.standard_normal(p["x"].shape))
    c2 = r32(c1 + 2e-4 * rng.standard_normal(p["x"].shape))
    return p, f_prev, c1, c2


def test_temporal_features_targets_and_corrections_match_oracle(npfem):
    import torch
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT)
    p, f_prev, c1, c2 = _temporal_inputs(60, m)
    xn = (p["x"] + 1e-4 * np.random.default_rng(61).standard_normal(p["x"].shape)).astype(np.float32).astype(np.float64)
    S = lambda a: dev(W.to_soa(a))
    feat = torch.zeros((3 * 642, 9), device="cuda")
    tgt = torch.zeros((3 * 642, 3), device="cuda")
    cn = torch.zeros((3, 3, 642), device="cuda")
    h.ws_features_temporal(3, S(p["x"]), S(p["v"]), S(p["f"]), S(f_prev), S(c1), S(c2), feat, x_next=S(xn),
                           target=tgt, c_out=cn)
    fg = feat.cpu().numpy().reshape(3, 642, 9)
    tg = tgt.cpu().numpy().reshape(3, 642, 3)
    cg = W.from_soa(cn.double().cpu().numpy())
    for c in range(3):
        y = m.first_guess(p["x"][c], p["v"][c], p["f"][c])
        fo, R = m.ws_features_temporal(y, p["f"][c], f_prev[c], c1[c], c2[c])
        scale = np.abs(fo).max(0)
        assert np.all(np.abs(fg[c] - fo).max(0) <= 2e-4 * scale + 1e-12), (np.abs(fg[c] - fo).max(0), scale)
        co = xn[c] - y
        assert np.abs(cg[c] - co).max() <= 2e-4 * np.abs(co).max() + 4e-6
        to = (co - c1[c]) @ R
        assert np.abs(tg[c] - to).max() <= 2e-4 * np.abs(co).max() + 4e-6


def test_temporal_guess_matches_oracle(npfem):
    import torch
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision="fp32"), dt=DT)
    P = rand_params(62)
    P[-3:] = 1e-4
    h.set_warmstart_temporal(P.astype(np.float32))
    p, f_prev, c1, c2 = _temporal_inputs(63, m, cells=2)
    S = lambda a: dev(W.to_soa(a))
    u = torch.zeros((2, 3, 642), device="cuda")
    h.ws_guess_temporal(2, S(p["x"]), S(p["v"]), S(p["f"]), S(f_prev), S(c1), S(c2), u)
    ug = W.from_soa(u.double().cpu().numpy())
    for c in range(2):
        xo = m.ws_guess_temporal(P.astype(np.float32).astype(np.float64), p["x"][c], p["v"][c], p["f"][c], f_prev[c],
                                 c1[c], c2[c], True)
        y = m.first_guess(p["x"][c], p["v"][c], p["f"][c])
        corr = np.abs(xo - y - c1[c]).max()
        assert corr > 1e-6
        assert np.abs((p["x"][c] + ug[c]) - xo).max() <= 1e-3 * corr + 2 * np.spacing(np.float32(25.0))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_temporal_network_trajectory_matches_oracle(npfem, prec):
    # any first iterate converges to the same step: 6 steps with the network installed
    # against the oracle's 6 steps from y
    m, rest, tris = oracle_model(642)
    h = npfem.Handle(rest, tris, npfem.material(), npfem.default_opts(precision=prec, tol=1e-6), dt=DT)
    P = rand_params(64)
    P[-3:] = 1e-5
    h.set_warmstart_temporal(P.astype(np.float32))
    p = population32(642, 5, seed=65, forces="shear", noise_pN=0.5, box=10.0)
    xo, vo, _ = oracle_steps(m, p["x"], p["v"], p["f"], steps=6, tol=1e-10, max_iter=200)
    xg, vg, sg = gpu_step_device(h, p["x"], p["v"], p["f"], steps=6)
    assert (sg["status"] == 0).all() and (sg["residual"] <= 1e-6).all()
    assert max_rel_disp(xg, xo, m.lbar) <= 6 * 1e-5 + fp32_store_allowance(p["x"], m.lbar)
