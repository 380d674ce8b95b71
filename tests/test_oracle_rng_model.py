"""Pins of the oracle's initialisation, MLP predictor, backward pass and optimiser."""
import os

import numpy as np
import pytest

from oracle.mixer import loss_grads, mix, softmax
from oracle.model import (ADAM_EPS, Shape, adam_step, backward, forward, init_params, views)
from oracle.rng import splitmix64_draws, uniform_pm1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_values():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    assert [int(x) for x in splitmix64_draws(0, 0, 3)] == want
    # counter-based: draw i is independent of where the range starts
    assert int(splitmix64_draws(0, 2, 1)[0]) == want[2]


def test_init_values_exact_and_bounded():
    sh = Shape(A=64, E=16, t=16, H=32)
    p = init_params(sh, 42)
    assert p.dtype == np.float32 and p.size == sh.count == 11360
    emb, w1, b1, w2, b2 = views(p, sh)
    assert np.all(b1 == 0) and np.all(b2 == 0) and not np.signbit(b1).any()
    assert np.abs(emb).max() <= 1 and np.abs(w1).max() <= 1 / 16 and np.abs(w2).max() <= 1 / np.sqrt(32) + 1e-7
    # fan_in 256 -> bound exactly 1/16, so W1 lies on the 2^-27 grid
    assert np.all(w1.astype(np.float64) * 2 ** 27 == np.round(w1.astype(np.float64) * 2 ** 27))
    u = uniform_pm1(42, 0, 4).astype(np.float64)
    assert np.all(u * 2 ** 23 == np.round(u * 2 ** 23)) and np.all((u >= -1) & (u < 1))


def _loops_forward(p, sh, ctx):
    """Brute-force forward with explicit index loops (tiny shapes only)."""
    emb, w1, b1, w2, b2 = (np.asarray(v, dtype=np.float64) for v in views(p, sh))
    x = [emb[c][e] for c in ctx for e in range(sh.E)]
    h = []
    for j in range(sh.H):
        acc = b1[j]
        for i in range(len(x)):
            acc += x[i] * w1[i][j]
        h.append(max(acc, 0.0))
    out = []
    for a in range(sh.A):
        acc = b2[a]
        for j in range(sh.H):
            acc += h[j] * w2[j][a]
        out.append(acc)
    return np.array(out)


def _setup(seed=3):
    sh = Shape(A=16, E=3, t=4, H=5)
    p = init_params(sh, seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    p += rng.normal(0, 0.3, p.size)  # nonzero biases, generic point
    ctx = rng.integers(0, sh.A, (6, sh.t))
    ctx[1, :2] = ctx[1, 2]  # repeated tokens inside one context
    tgt = rng.integers(0, sh.A, 6)
    Lu = rng.normal(0, 1, (6, sh.A))
    return sh, p, ctx, tgt, Lu


def test_forward_matches_index_loops():
    sh, p, ctx, _, _ = _setup()
    L = forward(p, sh, ctx)[3]
    for r in range(ctx.shape[0]):
        assert np.allclose(L[r], _loops_forward(p, sh, ctx[r]), rtol=0, atol=1e-12)


def _loss(p, sh, ctx, tgt, Lu, alpha):
    Lm = forward(p, sh, ctx)[3]
    P = softmax(mix(Lu, Lm, alpha))
    return -np.log(P[np.arange(len(tgt)), tgt]).mean()


def test_gradient_matches_central_differences():
    sh, p, ctx, tgt, Lu = _setup()
    alpha = 0.37
    X, a, h, Lm = forward(p, sh, ctx)
    P = softmax(mix(Lu, Lm, alpha))
    dLm, dalpha = loss_grads(P, tgt, Lu, Lm, alpha)
    g = backward(p, sh, ctx, X, a, h, dLm)
    eps = 1e-6
    near_kink = np.abs(a).min() < 1e-4
    assert not near_kink
    for i in range(p.size):
        q = p.copy(); q[i] += eps
        r = p.copy(); r[i] -= eps
        fd = (_loss(q, sh, ctx, tgt, Lu, alpha) - _loss(r, sh, ctx, tgt, Lu, alpha)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
    fda = (_loss(p, sh, ctx, tgt, Lu, alpha + eps) - _loss(p, sh, ctx, tgt, Lu, alpha - eps)) / (2 * eps)
    assert abs(fda - dalpha) <= 1e-8 + 1e-6 * abs(fda)


def test_gradient_without_static_model():
    sh, p, ctx, tgt, _ = _setup(7)
    alpha = 0.5
    X, a, h, Lm = forward(p, sh, ctx)
    P = softmax(mix(None, Lm, alpha, S=(0, 0, 1)))
    dLm, dalpha = loss_grads(P, tgt, None, Lm, alpha, S=(0, 0, 1))
    f = lambda al: -np.log(softmax((1 - al) * Lm)[np.arange(6), tgt]).mean()
    fda = (f(alpha + 1e-6) - f(alpha - 1e-6)) / 2e-6
    assert abs(fda - dalpha) < 1e-7
    g = backward(p, sh, ctx, X, a, h, dLm)
    i = sh.offsets()["w2"][0] + 3
    q = p.copy(); q[i] += 1e-6
    r = p.copy(); r[i] -= 1e-6
    fw = lambda pp: -np.log(softmax((1 - alpha) * forward(pp, sh, ctx)[3])[np.arange(6), tgt]).mean()
    assert abs((fw(q) - fw(r)) / 2e-6 - g[i]) < 1e-8


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.zeros(4); m = np.zeros(4); v = np.zeros(4)
    adam_step(th, m, v, g, 1, 1e-3)
    # bias-corrected first step: -lr * g / (|g| + eps)
    assert np.allclose(th, -1e-3 * g / (np.abs(g) + ADAM_EPS), rtol=1e-9, atol=0)
    adam_step(th, m, v, g, 2, 1e-3)  # constant gradient keeps the step at -lr*sign
    assert np.allclose(th, -2e-3 * g / (np.abs(g) + ADAM_EPS), rtol=1e-9, atol=0)


def test_forward_backward_and_mixer_gradients_match_torch_autograd():
    """An independent implementation: torch.nn.functional in float64 (embedding lookup, linear
    layers, ReLU) with autograd through Eq. (1), the softmax and the mean cross entropy of Eq. (2).
    The oracle's logits, its parameter gradient (the embedding's scattered adds included) and
    d alpha agree to rounding."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    sh = Shape(A=16, E=3, t=4, H=5)
    rng = np.random.default_rng(8)
    p = init_params(sh, 4).astype(np.float64) + rng.normal(0, 0.3, sh.count)
    ctx = rng.integers(0, sh.A, (7, sh.t))
    ctx[3, :] = ctx[3, 0]  # one token repeated inside a context: several adds into one embedding row
    tgt = rng.integers(0, sh.A, 7)
    Lu = rng.normal(0, 1, (7, sh.A))
    alpha = 0.37
    X, a, h, Lm = forward(p, sh, ctx)
    P = softmax(mix(Lu, Lm, alpha, (1, 0, 1)))
    dLm, dal = loss_grads(P, tgt, Lu, Lm, alpha, (1, 0, 1))
    g = backward(p, sh, ctx, X, a, h, dLm)

    off = sh.offsets()
    tp = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    ta = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    emb = tp[off["emb"][0]:off["emb"][1]].view(sh.A, sh.E)
    w1t = tp[off["w1"][0]:off["w1"][1]].view(sh.H, sh.t * sh.E)
    b1 = tp[off["b1"][0]:off["b1"][1]]
    w2 = tp[off["w2"][0]:off["w2"][1]].view(sh.H, sh.A)
    b2 = tp[off["b2"][0]:off["b2"][1]]
    xt = F.embedding(torch.from_numpy(ctx), emb).reshape(7, sh.t * sh.E)
    lm = F.linear(F.relu(F.linear(xt, w1t, b1)), w2.T, b2)
    z = ta * torch.from_numpy(Lu) + (1 - ta) * lm
    loss = F.cross_entropy(z, torch.from_numpy(tgt))
    loss.backward()
    np.testing.assert_allclose(Lm, lm.detach().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(P, torch.softmax(z, 1).detach().numpy(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(g, tp.grad.numpy(), rtol=0, atol=1e-12)
    assert abs(dal - float(ta.grad)) < 1e-12


def test_adam_matches_torch_optim_adam():
    """torch.optim.Adam (float64; betas 0.9 / 0.999, eps 1e-8, bias correction by the step count,
    eps added after the square root) over 25 steps of varying gradients, zeros included: the
    parameters and both moments agree to rounding."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    th = rng.normal(0, 1, 40)
    m, v = np.zeros(40), np.zeros(40)
    tp = torch.tensor(th.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=ADAM_EPS)
    for tau in range(1, 26):
        g = rng.normal(0, 10.0 ** rng.uniform(-4, 1), 40)
        g[rng.integers(0, 40, 5)] = 0.0
        adam_step(th, m, v, g, tau, 1e-3)
        tp.grad = torch.from_numpy(g.copy())
        opt.step()
    st = opt.state[tp]
    np.testing.assert_allclose(th, tp.detach().numpy(), rtol=0, atol=1e-14)
    np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-13, atol=0)
    np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-13, atol=0)
