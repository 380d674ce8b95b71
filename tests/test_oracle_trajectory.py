"""The oracle's whole online-learning run on one block, against an independent restatement in
torch (float64 autograd and torch.optim.Adam): the lanes of the block, the uniform prefix, the
mixer of Eq. (1) with a trainable alpha, the mean cross entropy of Eq. (2) over the lanes that
predict at a step, one Adam update per step, and, with overlap masking, the slice each token is
coded over.  Every probability the oracle codes, at every step of the run, agrees to rounding:
this pins the run's bookkeeping (which rows predict and train, when the update count advances,
what alpha sees), which the per-step pins alone do not."""
import numpy as np
import pytest

import synth
from oracle import codec as ocodec
from oracle.model import Shape, init_params


def _torch_run(torch, seq, cfg: ocodec.Config, static_w, init=None, snapshot_at=None):
    """Independent restatement, one block, network only: returns ({j: P rows of the predicting
    lanes in lane order}, the state (weights, alpha, optimiser) as it stood before local step
    snapshot_at).  init: a state to start from (a copy of a parent's), else the seeded init."""
    import copy
    F = torch.nn.functional
    s, k, A = cfg.s, cfg.k, 4 ** cfg.k
    codes = np.frombuffer(seq, np.uint8)
    digit = np.zeros(256, np.int64)
    digit[[ord("A"), ord("C"), ord("G"), ord("T")]] = [0, 1, 2, 3]
    d = digit[codes]
    l = (len(d) - k) // s + 1
    tok = np.array([int("".join(str(x) for x in d[i * s:i * s + k]), 4) for i in range(l)])
    M = min(cfg.lanes_per_block, l)
    base, extra = divmod(l, M)
    lens = [base + (r < extra) for r in range(M)]
    starts = [r * base + min(r, extra) for r in range(M)]
    t_eff = max(cfg.ctx_d, cfg.ctx_s if cfg.use_static else 0)

    def views(p, sh):
        o = sh.offsets()
        g = lambda n: p[o[n][0]:o[n][1]]
        return (g("emb").view(sh.A, sh.E), g("w1").view(sh.H, sh.t * sh.E), g("b1"), g("w2").view(sh.H, sh.A),
                g("b2"))

    def logits(p, sh, ctx):
        emb, w1t, b1, w2, b2 = views(p, sh)
        x = F.embedding(ctx, emb).reshape(ctx.shape[0], sh.t * sh.E)
        return F.linear(F.relu(F.linear(x, w1t, b1)), w2.T, b2)

    dsh, ssh = cfg.dm_shape, cfg.static_shape
    theta = torch.tensor(init_params(dsh, cfg.seed).astype(np.float64), requires_grad=True)
    alpha = torch.tensor(float(np.float32(cfg.alpha_init)), dtype=torch.float64, requires_grad=True)
    sw = torch.tensor(np.asarray(static_w, np.float32).astype(np.float64)) if cfg.use_static else None
    if cfg.optimizer == ocodec.ADAM:
        opt = torch.optim.Adam([theta, alpha], lr=float(np.float32(cfg.lr)), betas=(0.9, 0.999), eps=1e-8)
    else:
        opt = torch.optim.SGD([theta, alpha], lr=float(np.float32(cfg.lr)))
    if init is not None:
        with torch.no_grad():
            theta.copy_(init[0])
            alpha.copy_(init[1])
        opt.load_state_dict(copy.deepcopy(init[2]))
    out, snap = {}, None
    for j in range(max(lens)):
        if j == snapshot_at:
            snap = (theta.detach().clone(), alpha.detach().clone(), copy.deepcopy(opt.state_dict()))
        rows = [r for r in range(M) if t_eff <= j < lens[r]]
        if not rows:
            continue
        pos = [starts[r] + j for r in rows]
        cd = torch.tensor(np.stack([tok[q - cfg.ctx_d:q] for q in pos]))
        z = (1 - alpha) * logits(theta, dsh, cd)
        if cfg.use_static:
            cs = torch.tensor(np.stack([tok[q - cfg.ctx_s:q] for q in pos]))
            z = z + alpha * logits(sw, ssh, cs)
        loss, Ps = 0.0, []
        for i, q in enumerate(pos):
            if cfg.overlap_mask and j > 0:
                W = 4 ** s
                b0 = (int(tok[q - 1]) % 4 ** (k - s)) * W
            else:
                b0, W = 0, A
            zs = z[i, b0:b0 + W]
            P = torch.zeros(A, dtype=torch.float64)
            P[b0:b0 + W] = torch.softmax(zs.detach(), 0)
            Ps.append(P.numpy())
            loss = loss - torch.log_softmax(zs, 0)[int(tok[q]) - b0]
        out[j] = np.stack(Ps)
        opt.zero_grad()
        (loss / len(pos)).backward()
        opt.step()
    if snap is None and snapshot_at is not None:  # the parent ended first: its final state
        snap = (theta.detach().clone(), alpha.detach().clone(), copy.deepcopy(opt.state_dict()))
    return out, snap


@pytest.mark.parametrize("s,k,mask", [(1, 2, 0), (1, 3, 1), (2, 2, 0)])
def test_oracle_run_matches_an_independent_torch_restatement(s, k, mask):
    torch = pytest.importorskip("torch")
    seq = synth.markov(700, 3, 0.45, 3 + k).tobytes()
    cfg = ocodec.Config(s=s, k=k, use_static=True, emb_s=3, ctx_s=2, hid_s=5, emb_d=4, ctx_d=3, hid_d=6,
                        lanes_per_block=4, fallback=0, smp_mode=ocodec.SMP_NONE, overlap_mask=mask,
                        alpha_init=0.5, lr=3e-3)
    sw = init_params(Shape(4 ** k, 3, 2, 5), 2001)
    got = {}
    ocodec.compress(seq, [len(seq)], cfg, sw, on_probs=lambda g, j, P: got.__setitem__(j, np.array(P)))
    want, _ = _torch_run(torch, seq, cfg, sw)
    assert sorted(got) == sorted(want) and len(want) > 80
    worst = max(np.abs(got[j] - want[j]).max() for j in want)
    print(f"(s,k) = ({s},{k}) mask {mask}: {len(want)} steps, worst |P - P_torch| = {worst:.2e}")
    assert worst < 1e-10, worst


def test_chain_hand_over_inside_the_trajectory():
    """Two blocks under CHAIN step-wise model passing (f = 0.25): block 1 starts at global step
    ceil(f L_0) from a full copy of block 0's state as it stands then (weights, Adam moments and
    step count, alpha).  Both blocks' probabilities at every step agree with the restatement, which
    runs block 0 alone, copies its state before its local step ceil(f L_0) and runs block 1 from it."""
    import math
    torch = pytest.importorskip("torch")
    s, k = 1, 2
    seq = synth.markov(1200, 3, 0.45, 9).tobytes()
    lens = [700, 500]
    cfg = ocodec.Config(s=s, k=k, use_static=True, emb_s=3, ctx_s=2, hid_s=5, emb_d=4, ctx_d=3, hid_d=6,
                        lanes_per_block=4, fallback=0, smp_mode=ocodec.SMP_CHAIN, smp_fraction=0.25,
                        alpha_init=0.5, lr=3e-3)
    sw = init_params(Shape(4 ** k, 3, 2, 5), 2001)
    got = {0: {}, 1: {}}
    ocodec.compress(seq, lens, cfg, sw, on_probs=lambda g, j, P: got[g].__setitem__(j, np.array(P)))
    L0 = -(-((lens[0] - k) // s + 1) // 4)  # block 0's steps: its longest lane
    hand = math.ceil(float(np.float32(0.25)) * L0)
    w0, snap = _torch_run(torch, seq[:lens[0]], cfg, sw, snapshot_at=hand)
    w1, _ = _torch_run(torch, seq[lens[0]:], cfg, sw, init=snap)
    for g, want in ((0, w0), (1, w1)):
        assert sorted(got[g]) == sorted(want)
        worst = max(np.abs(got[g][j] - want[j]).max() for j in want)
        assert worst < 1e-10, (g, worst)
    # the hand-over matters: block 1 from the seeded init codes other probabilities
    cold, _ = _torch_run(torch, seq[lens[0]:], cfg, sw)
    assert max(np.abs(got[1][j] - cold[j]).max() for j in cold) > 1e-3


@pytest.mark.parametrize("use_static,optimizer", [(False, 0), (True, 1)])
def test_trajectory_without_static_model_and_with_sgd(use_static, optimizer):
    """The same restatement for Eq. (1) without a static model (S0 = 0: z = (1 - alpha) L^m, alpha
    still trained) and for the plain SGD update of the weights and alpha."""
    torch = pytest.importorskip("torch")
    seq = synth.markov(600, 3, 0.45, 21).tobytes()
    static = dict(use_static=True, emb_s=3, ctx_s=2, hid_s=5) if use_static else {}
    cfg = ocodec.Config(s=1, k=2, emb_d=4, ctx_d=3, hid_d=6, lanes_per_block=3, fallback=0,
                        smp_mode=ocodec.SMP_NONE, alpha_init=0.5, lr=0.05 if optimizer else 3e-3,
                        optimizer=optimizer, **static)
    sw = init_params(Shape(16, 3, 2, 5), 2001) if use_static else None
    got = {}
    ocodec.compress(seq, [len(seq)], cfg, sw, on_probs=lambda g, j, P: got.__setitem__(j, np.array(P)))
    want, _ = _torch_run(torch, seq, cfg, sw)
    assert sorted(got) == sorted(want) and len(want) > 150
    assert max(np.abs(got[j] - want[j]).max() for j in want) < 1e-10
