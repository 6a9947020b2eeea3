"""Training driver of the learned warm start (an addition to the paper's method).

The plain solver (npfem_step with the first guess y) generates trajectories; for
every step the library computes the per-vertex features at y and the rest-frame
target R^T (x_{n+1} - y) (npfem_ws_features).  The network is trained by the
library's own kernels (npfem_mlp_loss_grad, npfem_mlp_adam); this module only
allocates device buffers, draws minibatch indices and loops.
"""
from __future__ import annotations

import numpy as np

from . import npfem as N
from . import workloads as W

DT = 0.1


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases, identity normalisation."""
    rng = np.random.default_rng(seed)
    P = np.zeros(N.mlp_nparam(), dtype=np.float32)
    sizes = [(64, 9), (64, 64), (3, 64)]
    off = 0
    for fo, fi in sizes:
        lim = np.sqrt(6.0 / (fi + fo))
        P[off:off + fo * fi] = rng.uniform(-lim, lim, fo * fi)
        off += fo * fi + fo
    P[off:off + 9] = 0.0          # mu
    P[off + 9:off + 18] = 1.0     # sigma
    P[off + 18:off + 21] = 1.0    # s_out
    return P


def generate(handle: N.Handle, n_cells: int, steps: int, seed: int, vertices_per_step: int = 32,
             tol: float = 1e-7, gamma_range=(10.0, 1000.0), noise_pN: float = 0.5):
    """Trajectories of the plain solver from rest; returns device tensors (feat [S, 9],
    target [S, 3]) with `vertices_per_step` random vertices per cell and step."""
    import torch
    pop = W.population(handle.n, n_cells, seed, forces="shear", noise_pN=noise_pN, gamma_range=gamma_range)
    assert pop["rest"].shape[0] == handle.n
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    x, v, f = mk(pop["x"]), mk(pop["v"]), mk(pop["f"])
    n = handle.n
    plain = N.Handle(pop["rest"], pop["tris"], handle.material, N.default_opts(precision="fp32", tol=tol, max_iter=200),
                     dt=handle.dt)
    feat_all = torch.empty((n_cells * n, 9), dtype=torch.float32, device="cuda")
    tgt_all = torch.empty((n_cells * n, 3), dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    feats, tgts = [], []
    for _ in range(steps):
        x0, v0 = x.clone(), v.clone()
        N.step([plain], [n_cells], x, v, f, plain.dt)
        plain.ws_features(n_cells, x0, v0, f, feat_all, x_next=x, target=tgt_all)
        pick = torch.randint(0, n, (n_cells, vertices_per_step), device="cuda", generator=g)
        rows = (torch.arange(n_cells, device="cuda")[:, None] * n + pick).reshape(-1)
        feats.append(feat_all[rows].clone())
        tgts.append(tgt_all[rows].clone())
    torch.cuda.synchronize()
    return torch.cat(feats), torch.cat(tgts)


def set_normalisation(P: np.ndarray, feat, target) -> np.ndarray:
    """Input mean/std and per-component output scale from the training set."""
    P = P.copy()
    mu = feat.mean(0).double().cpu().numpy()
    sd = feat.std(0).double().cpu().numpy()
    so = target.std(0).double().cpu().numpy()
    base = N.mlp_nparam() - 21
    P[base:base + 9] = mu
    P[base + 9:base + 18] = np.maximum(sd, 1e-12)
    P[base + 18:base + 21] = np.maximum(so, 1e-12)
    return P


def train(P: np.ndarray, feat, target, steps: int = 4000, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          lr_final: float = 1e-4, log_every: int = 0):
    """Adam on minibatches drawn uniformly; returns (params, list of (step, loss))."""
    import torch
    dev = "cuda"
    p = torch.tensor(P, dtype=torch.float32, device=dev)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    grad = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    S = feat.shape[0]
    hist = []
    for k in range(1, steps + 1):
        idx = torch.randint(0, S, (batch,), device=dev, generator=g, dtype=torch.int32)
        N.mlp_loss_grad(p, feat, target, idx, batch, grad, loss)
        lr_k = lr * (lr_final / lr) ** ((k - 1) / max(1, steps - 1))
        N.mlp_adam(p, m, v, grad, k, lr=lr_k)
        if log_every and (k % log_every == 0 or k == steps):
            hist.append((k, float(loss.item())))
    torch.cuda.synchronize()
    return p.cpu().numpy(), hist


def validation_loss(P: np.ndarray, feat, target) -> float:
    import torch
    p = torch.tensor(P, dtype=torch.float32, device="cuda")
    grad = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    N.mlp_loss_grad(p, feat, target, None, feat.shape[0], grad, loss)
    return float(loss.item())


def train_warmstart(handle: N.Handle, n_cells: int = 1000, steps: int = 200, seed: int = 100, train_steps: int = 4000,
                    vertices_per_step: int = 32, log_every: int = 0):
    """Full pipeline: generate n_cells x steps step pairs with the plain solver, fit the
    normalisation, train.  Returns (params, info)."""
    feat, target = generate(handle, n_cells, steps, seed, vertices_per_step=vertices_per_step)
    P = set_normalisation(init_params(seed), feat, target)
    base = validation_loss(P * 0 + P, feat, target)
    P, hist = train(P, feat, target, steps=train_steps, seed=seed, log_every=log_every)
    return P, {"samples": int(feat.shape[0]), "step_pairs": n_cells * steps, "loss_init": base,
               "loss_final": validation_loss(P, feat, target), "history": hist}


def generate_temporal(handle: N.Handle, n_cells: int, steps: int, seed: int, vertices_per_step: int = 32,
                      tol: float = 1e-7, noise_pN: float = 0.5, regen_fraction: float = 0.5,
                      gamma_range=(10.0, 1000.0)):
    """Training data of the temporal network: trajectories of the plain solver from rest,
    the first cells under a force held fixed, the last `regen_fraction` of them with the
    N(0, noise_pN) noise redrawn every step; (features, targets) of steps >= 2 at
    `vertices_per_step` random vertices per cell and step (device tensors)."""
    import torch
    pop = W.population(handle.n, n_cells, seed, forces="shear", noise_pN=noise_pN, gamma_range=gamma_range)
    mk = lambda a: torch.tensor(W.to_soa(a), dtype=torch.float32, device="cuda")
    x, v, f, fsh = mk(pop["x"]), mk(pop["v"]), mk(pop["f"]), mk(pop["f_shear"])
    n = handle.n
    plain = N.Handle(pop["rest"], pop["tris"], handle.material,
                     N.default_opts(precision="fp32", tol=tol, max_iter=200, warm_history=0), dt=handle.dt)
    regen = int(round(regen_fraction * n_cells))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    c1, c2 = torch.zeros_like(x), torch.zeros_like(x)
    cn = torch.zeros_like(x)
    f_prev = f.clone()
    feat_all = torch.empty((n_cells * n, 9), dtype=torch.float32, device="cuda")
    tgt_all = torch.empty((n_cells * n, 3), dtype=torch.float32, device="cuda")
    feats, tgts = [], []
    for k in range(steps):
        if regen:
            f[n_cells - regen:] = fsh[n_cells - regen:] + noise_pN * torch.randn(
                fsh[n_cells - regen:].shape, device="cuda", generator=g)
        x0, v0 = x.clone(), v.clone()
        N.step([plain], [n_cells], x, v, f, plain.dt)
        plain.ws_features_temporal(n_cells, x0, v0, f, f_prev, c1, c2, feat_all, x_next=x, target=tgt_all, c_out=cn)
        if k >= 2:
            pick = torch.randint(0, n, (n_cells, vertices_per_step), device="cuda", generator=g)
            rows = (torch.arange(n_cells, device="cuda")[:, None] * n + pick).reshape(-1)
            feats.append(feat_all[rows].clone())
            tgts.append(tgt_all[rows].clone())
        c2, c1 = c1, cn.clone()
        f_prev = f.clone()
    torch.cuda.synchronize()
    plain.close()
    return torch.cat(feats), torch.cat(tgts)


def train_temporal_warmstart(handle: N.Handle, n_cells: int = 500, steps: int = 60, seed: int = 300,
                             train_steps: int = 20000, vertices_per_step: int = 32, regen_fraction: float = 0.5):
    """Full pipeline of the temporal network: generate, normalise, train.  Returns
    (params, info)."""
    feat, target = generate_temporal(handle, n_cells, steps, seed, vertices_per_step=vertices_per_step,
                                     regen_fraction=regen_fraction)
    P = set_normalisation(init_params(seed), feat, target)
    base = validation_loss(P, feat, target)
    P, hist = train(P, feat, target, steps=train_steps, seed=seed)
    return P, {"samples": int(feat.shape[0]), "step_pairs": n_cells * (steps - 2), "loss_init": base,
               "loss_final": validation_loss(P, feat, target), "history": hist}
