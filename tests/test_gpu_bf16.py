"""BF16 batched form: tensor-core predictor GEMMs with the optimiser fused into the
weight-gradient epilogues.  Bars: probabilities within 2e-2 of the FP64 oracle for a
single step from identical state; exact round trips; bits/base within 0.5 % of the
FP32 plain form on the same input."""
import numpy as np
import pytest

import synth
from oracle.mixer import mix, softmax
from oracle.model import Shape, forward, init_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2507_12805_gb300 as P
    return P


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# shapes on both engines: tcgen05/TMA (every GEMM dimension a multiple of 64: several 128-row
# tiles, two column tiles for H > 256, 4^6 tokens gathered from global memory) and mma.sync
@pytest.mark.parametrize("k,E,t,H,rows", [(4, 32, 32, 128, 130), (6, 32, 8, 256, 65), (4, 16, 20, 320, 140),
                                          (3, 16, 8, 64, 300), (3, 16, 16, 32, 70), (3, 8, 5, 48, 300),
                                          (2, 3, 5, 20, 9)])
def test_predict_bf16_within_tolerance(P, torch, k, E, t, H, rows):
    rng = np.random.default_rng(k * 101 + rows)
    sh = Shape(4 ** k, E, t, H)
    params = (init_params(sh, 3).astype(np.float64) + rng.normal(0, 0.05, sh.count)).astype(np.float32)
    ctx = rng.integers(0, sh.A, (rows, t))
    want = forward(params, sh, ctx)[3]
    d_out = torch.zeros((rows, sh.A), dtype=torch.float32, device="cuda")
    P.pmklc_predict(dev(torch, params), k, E, t, H, dev(torch, ctx.astype(np.uint16).view(np.int16)), d_out,
                    precision=P.PMKLC_BF16_BATCHED)
    got = d_out.cpu().numpy()
    # the probabilities are what the coder uses: compare softmax(logits) at the 2e-2 bar
    assert np.abs(softmax(got) - softmax(want)).max() < 2e-2
    assert np.abs(got - want).max() < 2e-2 * max(1.0, np.abs(want).max())


def _bf16(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _bf16_operand_grads(flat, sh, ctx, dLm):
    """The oracle's backward (oracle.model) with its GEMM operands rounded to BF16 where the BF16
    form stores them (weights, h, dz, dh), accumulated in FP64: what a correct BF16 kernel computes
    up to FP32 accumulation order and the rounding of its own FP32 forward."""
    from oracle.model import views
    emb, w1, b1, w2, b2 = views(np.asarray(flat, np.float64), sh)
    w1b, w2b, embb = _bf16(w1), _bf16(w2), _bf16(emb)
    R = ctx.shape[0]
    X = embb[ctx].reshape(R, -1)
    h = _bf16(np.maximum(X @ w1b + b1, 0.0))
    dz = _bf16(dLm)
    dh = _bf16((dz @ w2b.T) * (h > 0))
    g = np.zeros(sh.count)
    gemb, gw1, gb1, gw2, gb2 = views(g, sh)
    gw2[...] = h.T @ dz
    gb2[...] = dz.sum(axis=0)
    gw1[...] = X.T @ dh
    gb1[...] = dh.sum(axis=0)
    np.add.at(gemb, ctx.reshape(-1), (dh @ w1b.T).reshape(R * sh.t, sh.E))
    return g


# Gradient of every parameter block.  BF16 operands alone move the embedding and W1 gradients by
# up to ~7 % (relative L2) from the exact FP64 gradient on these inputs (cancellation in the sums
# over rows), so each block is held to 2e-2 of the BF16-operand restatement of the oracle's
# backward, and to 0.15 of the exact oracle gradient; a transposed or misplaced operand gives
# errors of order 1 in both.  Shapes: the first three take the tcgen05/TMA engine (every GEMM
# dimension a multiple of 64) with two 128-row tiles, ragged last K stages of the lane reductions
# (150 and 200 predicted lanes), H > 256 and, for 4^6 tokens, embedding gathers from global
# memory; the last three take the mma.sync engine.
GRAD_CASES = [
    # k, E, t, H, G, M, static (E, t, H) or None
    (4, 32, 8, 64, 3, 37, (32, 4, 64)),
    (4, 16, 12, 192, 2, 150, None),
    (4, 8, 16, 320, 2, 200, (16, 8, 64)),
    (6, 8, 8, 64, 2, 90, None),
    (4, 32, 8, 64, 3, 37, (16, 12, 48)),
    (4, 16, 12, 144, 2, 150, None),
    # 4^6 x 32 embedding table: too large to sum in shared memory, so the dX GEMM stores its rows and
    # a second kernel sums them into the table (tcgen05 engine)
    (6, 32, 8, 64, 2, 150, (32, 8, 64)),
]


@pytest.mark.parametrize("k,E,t,H,G,M,stat", GRAD_CASES)
def test_train_step_bf16_gradient_blocks(P, torch, k, E, t, H, G, M, stat):
    from oracle.codec import Config
    from oracle.mixer import loss_grads, mix, softmax
    from oracle.model import forward
    from tests.test_gpu_steps import _model, _oracle_step
    rng = np.random.default_rng(k * 1000 + E * 7 + H + M)
    use_static = stat is not None
    es, ts, hs = stat if use_static else (16, 12, 48)
    cfg_o = Config(s=2, k=k, use_static=use_static, emb_s=es, ctx_s=ts, hid_s=hs, emb_d=E, ctx_d=t, hid_d=H,
                   lr=1e-3)
    dsh, ssh = cfg_o.dm_shape, cfg_o.static_shape
    params = np.stack([_model(rng, dsh, 5 + g, 0.05) for g in range(G)])
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    alpha = np.full(G, 0.5, np.float32)
    az = np.zeros(G, np.float32)
    static = _model(rng, ssh, 77, 0.05) if use_static else None
    ctx = rng.integers(0, dsh.A, (G * M, cfg_o.t_eff))
    tgt = rng.integers(0, dsh.A, G * M)
    want = _oracle_step(cfg_o, params, m, v, alpha, az, az, static, ctx, tgt, 1, G, M)
    cfg = P.ModelConfig(s=2, k=k, use_static=use_static, emb_s=es, ctx_s=ts, hid_s=hs, emb_d=E, ctx_d=t,
                        hid_d=H, lr=1e-3, static_weights=static, precision=P.PMKLC_BF16_BATCHED)
    d = {k_: dev(torch, x) for k_, x in dict(params=params, m=m, v=v, alpha=alpha, am=az, av=az).items()}
    d_grad = torch.zeros(params.shape, dtype=torch.float32, device="cuda")
    P.pmklc_train_step(cfg, G, M, d["params"], d["m"], d["v"], d["alpha"], d["am"], d["av"],
                       dev(torch, static) if use_static else None,
                       dev(torch, ctx.astype(np.uint16).view(np.int16)), dev(torch, tgt.astype(np.uint16).view(np.int16)),
                       1, None, d_grad, None)
    gg = d_grad.cpu().numpy()
    S = (1 if use_static else 0, 0, 1)
    for g in range(G):
        rows = slice(g * M, (g + 1) * M)
        cd = ctx[rows, ctx.shape[1] - t:]
        Lm = forward(params[g].astype(np.float64), dsh, cd)[3]
        Lu = forward(static.astype(np.float64), ssh, ctx[rows, ctx.shape[1] - ts:])[3] if use_static else None
        dLm = loss_grads(softmax(mix(Lu, Lm, 0.5, S)), tgt[rows], Lu, Lm, 0.5, S)[0]
        emu = _bf16_operand_grads(params[g], dsh, cd, dLm)
        exact = want[g][1]
        for name, (lo, hi) in dsh.offsets().items():
            got = gg[g, lo:hi].astype(np.float64)
            for ref, bar in ((emu[lo:hi], 2e-2), (exact[lo:hi], 0.15)):
                rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
                assert rel < bar, (g, name, bar, rel)


@pytest.mark.parametrize("use_static", [0, 1])
def test_train_step_bf16_within_tolerance(P, torch, use_static):
    from oracle.codec import Config
    from tests.test_gpu_steps import _model, _oracle_step
    rng = np.random.default_rng(21 + use_static)
    cfg_o = Config(s=2, k=4, use_static=bool(use_static), emb_s=16, ctx_s=12, hid_s=48, emb_d=32, ctx_d=8,
                   hid_d=64, lr=1e-3)
    G, M = 3, 37
    dsh = cfg_o.dm_shape
    params = np.stack([_model(rng, dsh, 5 + g, 0.05) for g in range(G)])
    m = (rng.normal(0, 1e-3, params.shape)).astype(np.float32)
    v = (1e-6 + rng.random(params.shape) * 1e-5).astype(np.float32)
    alpha = np.array([0.5, 0.25, 0.8], np.float32)
    am = np.array([1e-3, 0, -1e-3], np.float32)
    av = np.array([1e-6, 1e-7, 2e-6], np.float32)
    static = _model(rng, cfg_o.static_shape, 77, 0.05) if use_static else None
    ctx = rng.integers(0, dsh.A, (G * M, cfg_o.t_eff))
    tgt = rng.integers(0, dsh.A, G * M)
    tau = 5
    want = _oracle_step(cfg_o, params, m, v, alpha, am, av, static, ctx, tgt, tau, G, M)
    cfg = P.ModelConfig(s=2, k=4, use_static=bool(use_static), emb_s=16, ctx_s=12, hid_s=48, emb_d=32, ctx_d=8,
                        hid_d=64, lr=1e-3, static_weights=static, precision=P.PMKLC_BF16_BATCHED)
    d = {k: dev(torch, x) for k, x in dict(params=params, m=m, v=v, alpha=alpha, am=am, av=av).items()}
    d_P = torch.zeros((G * M, dsh.A), dtype=torch.float32, device="cuda")
    d_da = torch.zeros(G, dtype=torch.float32, device="cuda")
    P.pmklc_train_step(cfg, G, M, d["params"], d["m"], d["v"], d["alpha"], d["am"], d["av"],
                       dev(torch, static) if use_static else None,
                       dev(torch, ctx.astype(np.uint16).view(np.int16)), dev(torch, tgt.astype(np.uint16).view(np.int16)),
                       tau, d_P, None, d_da)
    gP, gth, gal = d_P.cpu().numpy(), d["params"].cpu().numpy(), d["alpha"].cpu().numpy()
    for g in range(G):
        Pr, gr, dal, th, mm, vv, al = want[g]
        assert np.abs(gP[g * M:(g + 1) * M] - Pr).max() < 2e-2
        step_err = np.abs((gth[g] - params[g]) - (th - params[g].astype(np.float64)))
        assert np.quantile(step_err, 0.999) <= 0.1 * cfg.lr and step_err.max() <= 2 * cfg.lr
        assert abs(gal[g] - al) <= 0.1 * cfg.lr


def _cfg(P, **kw):
    base = dict(s=2, k=3, use_static=True, emb_s=8, ctx_s=3, hid_s=16, emb_d=8, ctx_d=4, hid_d=16,
                lanes_per_block=3, count_order=3, smp_mode=P.PMKLC_SMP_TREE, smp_fraction=0.2,
                precision=P.PMKLC_BF16_BATCHED)
    base.update(kw)
    return base


@pytest.mark.parametrize("kw", [dict(), dict(use_static=False, smp_mode=1), dict(optimizer=1, lr=0.05, fallback=0),
                                dict(s=3, k=6, emb_d=8, ctx_d=6, hid_d=24, lanes_per_block=7, fallback=0),
                                dict(emb_d=5, emb_s=3, fallback=0)])
def test_bf16_round_trip_and_determinism(P, kw):
    kw = _cfg(P, **kw)
    sw = init_params(Shape(4 ** kw["k"], kw["emb_s"], kw["ctx_s"], kw["hid_s"]), 5) if kw["use_static"] else None
    seq = synth.markov(3000, 2, 0.4, 31).tobytes()
    lens = [1400, 1000, 2, 0, 598]
    cfg = P.ModelConfig(**kw, static_weights=sw)
    out = P.pmklc_compress(seq, lens, cfg)
    assert out == P.pmklc_compress(seq, lens, cfg)
    back, bl = P.pmklc_decompress(out, sw)
    assert back == seq and list(bl) == lens


@pytest.mark.parametrize("s,k,E", [(2, 4, 16), (3, 6, 32)])
def test_masked_train_step_bf16_matches_oracle(P, torch, s, k, E):
    """Overlap-masked coding: the logits layer and dh are formed over each row's coded slice only
    (4^s columns selected by the previous token).  One BF16 step against the FP64 oracle's masked
    step (softmax over the slice, zero elsewhere): probabilities within 2e-2, every gradient block
    within 2e-2 of the BF16-operand restatement and 0.15 of the exact gradient (the bars of the
    unmasked test above).  Slices of 16 and 64 columns, 150 rows per group (two 16-row chunks of
    one slice and many one-row slices)."""
    from oracle.codec import Config
    from oracle.mixer import loss_grads
    from oracle.model import backward
    rng = np.random.default_rng(500 + 10 * s + k)
    G, M, t, H = 2, 150, 8, 64
    cfg_o = Config(s=s, k=k, use_static=True, emb_s=E, ctx_s=8, hid_s=64, emb_d=E, ctx_d=t, hid_d=H, lr=1e-3)
    dsh, ssh = cfg_o.dm_shape, cfg_o.static_shape
    W, mod = 4 ** s, 4 ** (k - s)
    params = np.stack([_model_params(rng, dsh, g) for g in range(G)])
    static = _model_params(rng, ssh, 77)
    ctx = rng.integers(0, dsh.A, (G * M, cfg_o.t_eff))
    ctx[:40, -1] = 5  # forty rows of group 0 share one slice
    base = (ctx[:, -1] % mod) * W
    tgt = base + rng.integers(0, W, G * M)
    z0 = np.zeros(G, np.float32)
    cfg = P.ModelConfig(s=s, k=k, use_static=True, emb_s=E, ctx_s=8, hid_s=64, emb_d=E, ctx_d=t, hid_d=H, lr=1e-3,
                        static_weights=static, precision=P.PMKLC_BF16_BATCHED, overlap_mask=1)
    d = {k_: dev(torch, x) for k_, x in dict(params=params, m=np.zeros_like(params), v=np.zeros_like(params),
                                             alpha=np.full(G, 0.5, np.float32), am=z0, av=z0).items()}
    d_P = torch.zeros((G * M, dsh.A), dtype=torch.float32, device="cuda")
    d_grad = torch.zeros(params.shape, dtype=torch.float32, device="cuda")
    P.pmklc_train_step(cfg, G, M, d["params"], d["m"], d["v"], d["alpha"], d["am"], d["av"], dev(torch, static),
                       dev(torch, ctx.astype(np.uint16).view(np.int16)), dev(torch, tgt.astype(np.uint16).view(np.int16)),
                       1, d_P, d_grad, None)
    gP, gg = d_P.cpu().numpy(), d_grad.cpu().numpy()
    for g in range(G):
        rows = slice(g * M, (g + 1) * M)
        cd = ctx[rows, ctx.shape[1] - t:]
        X, a, h, Lm = forward(params[g].astype(np.float64), dsh, cd)
        Lu = forward(static.astype(np.float64), ssh, ctx[rows, ctx.shape[1] - 8:])[3]
        zz = mix(Lu, Lm, 0.5, (1, 0, 1))
        Pr = np.zeros_like(zz)
        for i, b in enumerate(base[rows]):
            Pr[i, b:b + W] = softmax(zz[i, b:b + W])
        assert np.abs(gP[rows] - Pr).max() < 2e-2
        dLm = loss_grads(Pr, tgt[rows], Lu, Lm, 0.5, (1, 0, 1))[0]
        emu = _bf16_operand_grads(params[g], dsh, cd, dLm)
        exact = backward(params[g].astype(np.float64), dsh, cd, X, a, h, dLm)
        for name, (lo, hi) in dsh.offsets().items():
            got = gg[g, lo:hi].astype(np.float64)
            for ref, bar in ((emu[lo:hi], 2e-2), (exact[lo:hi], 0.15)):
                rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
                assert rel < bar, (g, name, bar, rel)


def _model_params(rng, sh, seed):
    from tests.test_gpu_steps import _model
    return _model(rng, sh, seed, 0.05)


def test_bf16_bits_per_base_close_to_fp32(P):
    w = synth.workload("plain", scale=1 / 16)
    kw = dict(s=2, k=4, use_static=True, emb_s=32, ctx_s=32, hid_s=128, emb_d=32, ctx_d=32, hid_d=128,
              lanes_per_block=16, smp_mode=2, fallback=0)
    sw = P.pmklc_init_model(4, 32, 32, 128, 2001)
    a = P.pmklc_compress(w.seq, w.block_lens, P.ModelConfig(**kw, static_weights=sw))
    b = P.pmklc_compress(w.seq, w.block_lens, P.ModelConfig(**kw, static_weights=sw, precision=1))
    assert P.pmklc_decompress(b, sw)[0] == w.seq.tobytes()
    assert abs(len(b) - len(a)) <= 0.005 * len(a), (len(a), len(b))


@pytest.mark.parametrize("optimizer,M", [(0, 150), (1, 150), (0, 200), (0, 500), (1, 1000)])
def test_update_in_gradient_epilogues_equals_the_streaming_optimiser(P, torch, optimizer, M):
    """On the tcgen05 engine W1 and W2 are updated in the epilogues of their gradient GEMMs; when the
    gradient is exported they are stored and the streaming optimiser applies the same rule.  Both
    paths give the same parameters, moments and mixing weight bit for bit (the update arithmetic is
    explicitly rounded, the gradients are the same FP32 values).  Lane counts whose last K block is
    partial and whose stage buffers are reused (more K blocks than buffers) cover the tail stage's
    synchronisation."""
    from oracle.codec import Config
    from tests.test_gpu_steps import _model
    rng = np.random.default_rng(88 + optimizer + M)
    cfg_o = Config(s=2, k=4, use_static=True, emb_s=16, ctx_s=8, hid_s=64, emb_d=16, ctx_d=8, hid_d=128)
    G = 3
    dsh = cfg_o.dm_shape
    params = np.stack([_model(rng, dsh, 5 + g, 0.05) for g in range(G)])
    m = (rng.normal(0, 1e-3, params.shape)).astype(np.float32)
    v = (1e-6 + rng.random(params.shape) * 1e-5).astype(np.float32)
    alpha = np.array([0.5, 0.25, 0.8], np.float32)
    am = np.array([1e-3, 0, -1e-3], np.float32)
    av = np.array([1e-6, 1e-7, 2e-6], np.float32)
    static = _model(rng, cfg_o.static_shape, 77, 0.05)
    ctx = rng.integers(0, dsh.A, (G * M, cfg_o.t_eff)).astype(np.uint16).view(np.int16)
    tgt = rng.integers(0, dsh.A, G * M).astype(np.uint16).view(np.int16)
    cfg = P.ModelConfig(s=2, k=4, use_static=True, emb_s=16, ctx_s=8, hid_s=64, emb_d=16, ctx_d=8, hid_d=128,
                        lr=1e-3, optimizer=optimizer, static_weights=static, precision=P.PMKLC_BF16_BATCHED,
                        update_path=P.PMKLC_UPDATE_FUSED)
    out = []
    for export in (False, True):
        d = {k_: dev(torch, x) for k_, x in dict(params=params, m=m, v=v, alpha=alpha, am=am, av=av).items()}
        d_grad = torch.zeros(params.shape, dtype=torch.float32, device="cuda") if export else None
        P.pmklc_train_step(cfg, G, M, d["params"], d["m"], d["v"], d["alpha"], d["am"], d["av"], dev(torch, static),
                           dev(torch, ctx), dev(torch, tgt), 3, None, d_grad, None)
        out.append({k_: x.cpu().numpy() for k_, x in d.items()})
    assert not np.array_equal(out[0]["params"], params)  # the step updated the parameters
    for name in ("params", "m", "v", "alpha", "am", "av"):
        assert np.array_equal(out[0][name].view(np.uint32), out[1][name].view(np.uint32)), name


def test_update_paths_give_identical_containers(P):
    """A whole BF16 run on tcgen05 shapes with W1 and W2 updated in the gradient GEMMs' epilogues,
    by the streaming optimiser, and by the size rule: the same container byte for byte but for the
    variant field that records the path, and it decodes."""
    import synth
    from oracle.model import Shape, init_params
    seq = synth.markov(24000, 5, 0.40, 77).tobytes()
    lens = [8000, 8000, 8000]
    kw = dict(s=2, k=4, use_static=True, emb_s=16, ctx_s=8, hid_s=64, emb_d=16, ctx_d=8, hid_d=128,
              lanes_per_block=24, smp_mode=P.PMKLC_SMP_TREE, fallback=0, overlap_mask=1,
              precision=P.PMKLC_BF16_BATCHED)
    sw = init_params(Shape(256, 16, 8, 64), 3)
    outs = [P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, update_path=u))
            for u in (P.PMKLC_UPDATE_STREAM, P.PMKLC_UPDATE_FUSED, P.PMKLC_UPDATE_AUTO)]
    # identical except the variant field (bytes 72-76), which records the path taken
    for out in outs[1:]:
        assert out[:72] == outs[0][:72] and out[76:] == outs[0][76:]
    assert P.pmklc_decompress(outs[1], sw)[0] == seq


@pytest.mark.parametrize("s,k,E", [(2, 4, 16), (3, 6, 32)])
def test_kernel_variants_give_identical_containers(P, torch, s, k, E):
    """Every kernel variant the autotuner offers (row-GEMM tile caps 0 / 128 / 64 x update path
    streaming / fused) codes the same bytes: the containers differ only in the variant field that
    records the choice, every one decodes, and the autotuner picks one of them.  (3,6) with E 32
    sums the embedding gradient from stored dX rows, (2,4) in the dX tiles."""
    import synth
    from oracle.model import Shape, init_params
    seq = synth.markov(24000, 5, 0.40, 78)
    lens = [8000, 8000, 8000]
    kw = dict(s=s, k=k, use_static=True, emb_s=E, ctx_s=8, hid_s=64, emb_d=E, ctx_d=8, hid_d=128,
              lanes_per_block=24, smp_mode=P.PMKLC_SMP_TREE, fallback=0, overlap_mask=1,
              precision=P.PMKLC_BF16_BATCHED)
    sw = init_params(Shape(4 ** k, E, 8, 64), 4)
    codes = [t | (u << 2) for t in (0, 1, 2) for u in (P.PMKLC_UPDATE_STREAM, P.PMKLC_UPDATE_FUSED)]
    outs = []
    for code in codes:
        out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, gemm_tiles=code & 3,
                                                        update_path=code >> 2))
        variant = int.from_bytes(out[72:76], "little")
        assert (variant >> 8) & 3 == code & 3 and (variant >> 10) & 3 == code >> 2 and variant & 1 == 1
        outs.append(out)
        assert P.pmklc_decompress(out, sw)[0] == seq.tobytes()
    for out in outs[1:]:
        assert out[:72] == outs[0][:72] and out[76:] == outs[0][76:]
    cfg = P.ModelConfig(**kw, static_weights=sw)
    chosen, ms = P.pmklc_autotune_variant(torch.from_numpy(seq).cuda(), lens, cfg, codes, head_bases=4000)
    assert chosen in codes and len(ms) == len(codes) and np.all(ms > 0)


@pytest.mark.parametrize("lanes", [200, 1000])
def test_many_lanes_per_block_round_trip_on_both_update_paths(P, lanes):
    """Uneven blocks with a lane-length target and up to `lanes` lanes per block (K blocks beyond
    the stage buffers in the lane-reducing GEMMs, partial last K blocks), network only: both update
    paths decode exactly and code the same bytes."""
    import synth
    from oracle.model import Shape, init_params
    tabs = synth.species_tables()
    lens = [400_000, 100_000, 30_000]
    seq = np.concatenate([synth.sample(L, tabs[i], 950 + i) for i, L in enumerate(lens)])
    kw = dict(s=3, k=4, use_static=True, emb_s=16, ctx_s=8, hid_s=64, emb_d=16, ctx_d=8, hid_d=128,
              lanes_per_block=lanes, lane_tokens=128, smp_mode=P.PMKLC_SMP_TREE, fallback=0, overlap_mask=1,
              precision=P.PMKLC_BF16_BATCHED)
    sw = init_params(Shape(256, 16, 8, 64), 6)
    outs = []
    for upd in (P.PMKLC_UPDATE_STREAM, P.PMKLC_UPDATE_FUSED):
        out = P.pmklc_compress(seq, lens, P.ModelConfig(**kw, static_weights=sw, update_path=upd))
        assert P.pmklc_decompress(out, sw)[0] == seq.tobytes()
        outs.append(out)
    assert outs[0][:72] == outs[1][:72] and outs[0][76:] == outs[1][76:]
