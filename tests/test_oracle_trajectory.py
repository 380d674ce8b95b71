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


def _torch_run(torch, seq, cfg: ocodec.Config, static_w):
    """Independent restatement, one block, network only: returns {(j): P rows of the predicting
    lanes in lane order}."""
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
    t_eff = max(cfg.ctx_d, cfg.ctx_s)

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
    sw = torch.tensor(np.asarray(static_w, np.float32).astype(np.float64))
    opt = torch.optim.Adam([theta, alpha], lr=float(np.float32(cfg.lr)), betas=(0.9, 0.999), eps=1e-8)
    out = {}
    for j in range(max(lens)):
        rows = [r for r in range(M) if t_eff <= j < lens[r]]
        if not rows:
            continue
        pos = [starts[r] + j for r in rows]
        cd = torch.tensor(np.stack([tok[q - cfg.ctx_d:q] for q in pos]))
        cs = torch.tensor(np.stack([tok[q - cfg.ctx_s:q] for q in pos]))
        z = alpha * logits(sw, ssh, cs) + (1 - alpha) * logits(theta, dsh, cd)
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
    return out


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
    want = _torch_run(torch, seq, cfg, sw)
    assert sorted(got) == sorted(want) and len(want) > 80
    worst = max(np.abs(got[j] - want[j]).max() for j in want)
    print(f"(s,k) = ({s},{k}) mask {mask}: {len(want)} steps, worst |P - P_torch| = {worst:.2e}")
    assert worst < 1e-10, worst
