"""Pins of the oracle's learned-warm-start reference (features, network, gradient).

The warm start is an addition to the paper's method; these pins check the FP64
reference against finite differences, a brute-force BF16 rounding and the
invariances the features are built to have."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1903_06479_gb300 import workloads as W

DT = 0.1


def rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    P = rng.normal(0.0, scale, O.mlp_nparam())
    base = O.mlp_nparam() - 21
    P[base:base + 9] = rng.normal(0, 0.1, 9)
    P[base + 9:base + 18] = rng.uniform(0.5, 2.0, 9)
    P[base + 18:base + 21] = rng.uniform(0.5, 2.0, 3)
    return P.astype(np.float32).astype(np.float64)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = rand_params(1)
    feat = rng.normal(0, 1, (37, 9))
    tgt = rng.normal(0, 1, (37, 3))
    loss, g = O.mlp_loss_grad(P, feat, tgt, bf16_operands=False)
    h = 1e-6
    for q in list(rng.choice(O.mlp_nparam() - 21, 60, replace=False)) + [0, 575, 576, 4735, 4991, 4994]:
        Pp = P.copy(); Pp[q] += h
        Pm = P.copy(); Pm[q] -= h
        fd = (O.mlp_loss_grad(Pp, feat, tgt, False)[0] - O.mlp_loss_grad(Pm, feat, tgt, False)[0]) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 * max(1.0, abs(g).max()), q
    assert np.all(g[O.mlp_nparam() - 21:] == 0.0)


def test_bf16_rounding_is_nearest_ties_to_even():
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.normal(0, 1, 2000), rng.normal(0, 1e-3, 500), [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]])
    for x in xs.astype(np.float32):
        b = O.bf16(x)
        u = np.frombuffer(np.float32(b).tobytes(), dtype=np.uint32)[0]
        assert u & 0xFFFF == 0  # 8 significant bits
        # neighbours on the BF16 grid around x
        ux = np.frombuffer(np.float32(x).tobytes(), dtype=np.uint32)[0] & 0xFFFF0000
        cands = [np.frombuffer(np.uint32(c).tobytes(), dtype=np.float32)[0] for c in (ux, ux + 0x10000)]
        d = [abs(float(c) - float(x)) for c in cands]
        best = min(d)
        assert abs(abs(b - float(x)) - best) == 0.0
        if d[0] == d[1]:  # tie: even significand
            assert (u >> 16) & 1 == 0
    assert O.bf16(1.0 + 2 ** -8) == 1.0 and O.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


@pytest.fixture(scope="module")
def m642():
    rest, tris = W.discocyte(642)
    return O.Model(rest, tris, W.material_vector(), DT)


def test_features_vanish_on_a_rigid_placement(m642):
    Q = W.random_rotations(np.random.default_rng(3), 1)[0]
    y = m642.rest @ Q.T + np.array([40.0, 2.0, -7.0])
    feat, R = m642.ws_features(y, np.zeros_like(y))
    assert np.abs(R - Q).max() < 1e-12
    assert np.abs(feat).max() < 1e-11


def test_features_are_rotation_invariant(m642):
    rng = np.random.default_rng(4)
    y = m642.rest + 0.02 * m642.lbar * rng.standard_normal(m642.rest.shape)
    f = rng.normal(0, 2.0, y.shape)
    Q = W.random_rotations(rng, 1)[0]
    fa, Ra = m642.ws_features(y, f)
    fb, Rb = m642.ws_features(y @ Q.T + 5.0, f @ Q.T)
    assert np.abs(fa - fb).max() < 1e-10 * np.abs(fa).max()
    assert np.abs(Rb - Q @ Ra).max() < 1e-12


def test_warm_start_with_zero_output_is_the_first_guess(m642):
    P = rand_params(5)
    P[4800:4995] = 0.0  # W3 and b3
    p = W.population(642, 1, 6, forces="noise", noise_pN=1.0)
    x1 = m642.ws_guess(P, p["x"][0], p["v"][0], p["f"][0])
    y = m642.first_guess(p["x"][0], p["v"][0], p["f"][0])
    assert np.abs(x1 - y).max() == 0.0


def test_bf16_operand_network_within_rounding_bound():
    """The BF16-operand network (weights, normalised inputs and first hidden layer
    rounded to BF16, unit roundoff 2^-9) differs from the FP64 network by no more than
    the first-order propagation of those roundings through |W3| |W2| |W1|, and it does
    differ (the rounding is applied)."""
    rng = np.random.default_rng(21)
    P = rand_params(22)
    feat = rng.normal(0, 1, (64, 9))
    o64 = O.mlp_predict(P, feat, bf16_operands=False)
    o16 = O.mlp_predict(P, feat, bf16_operands=True)
    base = O.mlp_nparam() - 21
    mu, sig, sout = P[base:base + 9], P[base + 9:base + 18], P[base + 18:]
    W1, W2, W3 = P[:576].reshape(64, 9), P[640:4736].reshape(64, 64), P[4800:4992].reshape(3, 64)
    u = 2.0 ** -9
    xn = (feat - mu) / sig
    # |delta pre-activation 1| <= u |W1| |xn| (weights) + u |W1| |xn| (inputs), tanh is 1-Lipschitz
    d1 = 2 * u * np.abs(xn) @ np.abs(W1).T
    h1 = np.tanh(xn @ W1.T + P[576:640])
    # layer 2: weight and operand rounding plus the propagated layer-1 error
    d2 = (2 * u * np.abs(h1) + d1) @ np.abs(W2).T
    h2 = np.tanh(h1 @ W2.T + P[4736:4800])
    d3 = (u * np.abs(h2) + d2) @ np.abs(W3).T
    bound = 1.05 * d3 * sout + 1e-12
    err = np.abs(o16 - o64)
    assert np.all(err <= bound), (err / bound).max()
    assert err.max() > 1e-3 * bound.max()


# ---------------------------------------------------------------------------------------
# temporal network: features of the force change and of the corrections' trend
# ---------------------------------------------------------------------------------------
def test_temporal_features_vanish_on_a_steady_trajectory(m642):
    # F_n = F_{n-1} and c_{n-1} = c_{n-2}: nothing changes between steps, every feature is 0
    rng = np.random.default_rng(40)
    y = m642.rest + 0.02 * m642.lbar * rng.standard_normal(m642.rest.shape)
    f = rng.normal(0, 1.0, y.shape)
    c = 1e-3 * rng.standard_normal(y.shape)
    feat, _ = m642.ws_features_temporal(y, f, f, c, c)
    assert np.abs(feat).max() == 0.0


def test_temporal_features_closed_forms_and_rotation_invariance(m642):
    rng = np.random.default_rng(41)
    y = m642.rest + 0.02 * m642.lbar * rng.standard_normal(m642.rest.shape)
    M = m642.masses()[:, None]
    # a force change that is a uniform displacement h^2 dF / m = a: u = R^T a everywhere and
    # its Laplacian vanishes (the cotangent weights' rows sum to c_ii)
    a = np.array([0.003, -0.001, 0.002])
    df = a[None, :] * M / DT ** 2
    c1, c2 = rng.standard_normal(y.shape) * 1e-3, rng.standard_normal(y.shape) * 1e-3
    f0 = rng.normal(0, 1.0, y.shape)
    feat, R = m642.ws_features_temporal(y, f0 + df, f0, c1, c2)
    assert np.abs(feat[:, 3:6] - (a @ R)[None, :]).max() < 1e-14
    assert np.abs(feat[:, 6:9]).max() < 1e-10 * np.abs(a).max() / m642.lbar ** 2
    assert np.abs(feat[:, 0:3] - (c1 - c2) @ R).max() < 1e-15
    # rigid motion of the whole state rotates nothing in the features
    Q = W.random_rotations(rng, 1)[0]
    f1 = rng.normal(0, 1.0, y.shape)
    fa, Ra = m642.ws_features_temporal(y, f1, f0, c1, c2)
    fb, Rb = m642.ws_features_temporal(y @ Q.T + 7.0, f1 @ Q.T, f0 @ Q.T, c1 @ Q.T, c2 @ Q.T)
    assert np.abs(fa - fb).max() < 1e-10 * np.abs(fa).max()


def test_temporal_guess_with_zero_output_is_the_temporal_warm_start(m642):
    P = rand_params(42)
    P[4800:4995] = 0.0  # W3 and b3
    p = W.population(642, 1, 43, forces="noise", noise_pN=1.0)
    rng = np.random.default_rng(44)
    c1, c2 = 1e-3 * rng.standard_normal(p["x"][0].shape), 1e-3 * rng.standard_normal(p["x"][0].shape)
    f_prev = p["f"][0] + rng.normal(0, 0.5, p["f"][0].shape)
    x1 = m642.ws_guess_temporal(P, p["x"][0], p["v"][0], p["f"][0], f_prev, c1, c2)
    y = m642.first_guess(p["x"][0], p["v"][0], p["f"][0])
    assert np.abs(x1 - (y + c1)).max() < 1e-15 * np.abs(y).max() + 1e-18
