"""GPU parity of the learned proposal's kernels against the FP64 oracle (oracle/mlp.py and the
oracle's mixture move): network forward (the FP32-accurate training products on either engine,
and the BF16 tcgen05 network kernel), loss gradient and Adam on either engine, features, warm
start and the mixture move."""
import numpy as np
import pytest

import oracle
import oracle.mlp as omlp
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _params(qam, seed=5, noise=0.05):
    rng = np.random.default_rng(seed + 100)
    p = omlp.init_params(qam, seed) + noise * rng.standard_normal(omlp.param_count(qam))
    return p.astype(np.float32).astype(np.float64)     # the values the GPU holds


def _features(rows, seed=0):
    """Feature rows of the scale the detector produces (level units, log Gt_ii, log sigma^2)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 6))
    X[:, :4] = rng.normal(0.0, 4.0, (rows, 4))
    X[:, 4] = rng.normal(-2.0, 0.5, rows)
    X[:, 5] = rng.uniform(-7.0, -2.0, rows)
    return X.astype(np.float32).astype(np.float64)


def _mlp(qam, params, max_rows=4096, train_tc=None):
    from paper_2407_06042_gb300 import Mlp
    m = Mlp(qam, max_rows=max_rows)
    m.set_params(params.astype(np.float32))
    if train_tc is not None:
        m.set_train_engine(train_tc)
    return m


# Products of the forward and training passes on tcgen05 with each FP32 operand split into three
# BF16 terms (to 2^-26 of itself) and the six leading term products accumulated in FP32: each
# product is as accurate as an FP32 one, but the tensor core adds several products per step
# into its FP32 accumulator with a rounding of its own rather than one FMA at a time, and it
# accumulates 18 term products per 16 values of k; the tensor-core path gets twice the room
# (the QPSK weight gradient over 1000 rows, the tightest case, measured 1.2e-4 of max |g|).
TC_SLACK = {False: 1.0, True: 2.0}


@pytest.mark.parametrize("train_tc", [False, True])
@pytest.mark.parametrize("qam", [4, 16, 64])
def test_forward_fp32_matches_oracle(qam, train_tc):
    import torch
    p = _params(qam)
    X = _features(1000 + qam)
    m = _mlp(qam, p, max_rows=384, train_tc=train_tc)   # several chunks and a ragged one
    out = m.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = omlp.forward(p, X, qam)[0]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(out, ref, atol=2e-5 * TC_SLACK[train_tc] * scale, rtol=0)
    m.destroy()


@pytest.mark.parametrize("qam,rows", [(4, 128 * 40 + 77), (16, 128 * 40 + 77), (64, 128 * 40 + 77),
                                      (16, 128 * 152 * 3 + 77), (64, 128 * 152 * 3 + 77),
                                      (16, 1), (4, 129)])
def test_forward_tensor_cores_match_quantised_oracle(qam, rows):
    """BF16 tcgen05 forward against the oracle's quantised network (hidden activations and
    layer-2/3 weights rounded to BF16). The two differ by FP32 vs FP64 accumulation, except
    where an activation sits within FP32 error of a BF16 rounding boundary and rounds the other
    way (~1e-5 of activations): such a row moves by about one BF16 ulp of one activation times
    its weights. The larger row counts give every CTA of the persistent kernel several tiles,
    so its pipeline (layer 1 of one tile beside the MMAs and epilogues of the previous one)
    runs through every buffer's phases several times."""
    import torch
    p = _params(qam)
    X = _features(rows, seed=1)
    m = _mlp(qam, p)
    out = m.forward(torch.tensor(X, dtype=torch.float32, device="cuda"),
                    tensor_cores=True).cpu().numpy()
    ref = omlp.forward(p, X, qam, quant=True)[0]
    scale = np.abs(ref).max()
    err = np.abs(out - ref).max(axis=1)
    assert np.mean(err <= 5e-5 * scale) >= 0.9, np.quantile(err / scale, [0.5, 0.9, 0.99])
    assert err.max() <= 2e-2 * scale, err.max() / scale
    exact = omlp.forward(p, X, qam)[0]
    assert np.abs(out - exact).max() <= 0.1 * scale      # BF16 network stays close to FP64
    m.destroy()


def _decided_rows(p, X, qam, idx, margin=1e-5):
    """The rows of idx whose ReLU decisions FP32 arithmetic takes as FP64 does: every hidden
    pre-activation at least `margin` of its layer's largest from zero. A pre-activation closer to
    zero than an FP32 sum's rounding (about 1e-7 of the terms for K = 256) may land on either
    side in any FP32 evaluation order; the mask it sets then moves a weight gradient by a whole
    row's term (up to 2e-3 of max |g| in the QPSK case), which says nothing about the kernel."""
    _, (_, a1, _, a2, _) = omlp.forward(p, X[idx], qam)
    ok = ((np.abs(a1) >= margin * np.abs(a1).max()).all(axis=1)
          & (np.abs(a2) >= margin * np.abs(a2).max()).all(axis=1))
    return idx[ok]


@pytest.mark.parametrize("train_tc", [False, True])
@pytest.mark.parametrize("qam,rows", [(16, 300), (4, 1000), (64, 257), (16, 4096)])
def test_loss_and_gradient_match_oracle(qam, rows, train_tc):
    import torch
    p = _params(qam, seed=7)
    X = _features(rows + 50, seed=2)
    rng = np.random.default_rng(3)
    labels = rng.integers(0, qam, rows + 50).astype(np.int32)
    idx = _decided_rows(p, X, qam, rng.permutation(rows + 50)[:rows]).astype(np.int32)
    m = _mlp(qam, p, train_tc=train_tc)
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dl = torch.tensor(labels, device="cuda")
    di = torch.tensor(idx, device="cuda")
    loss, grad = m.loss_grad(dX, dl, di)
    ref_loss, ref_grad = omlp.loss_and_grad(p, X[idx], labels[idx], qam)
    k = TC_SLACK[train_tc]
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * k * abs(ref_loss)
    g = grad.cpu().numpy()
    o = 0
    for name, shp in omlp.shapes(qam):
        n = int(np.prod(shp))
        gs, rs = g[o:o + n], ref_grad[o:o + n]
        assert np.abs(gs - rs).max() <= 1e-4 * k * np.abs(rs).max() + 1e-7, (name, np.abs(gs - rs).max() / np.abs(rs).max())
        o += n
    # without an index list: rows 0 .. rows-1
    loss2, grad2 = m.loss_grad(dX, dl, None, rows=rows)
    ref_loss2, _ = omlp.loss_and_grad(p, X[:rows], labels[:rows], qam)
    assert abs(float(loss2.item()) - ref_loss2) <= 1e-5 * k * abs(ref_loss2)
    # determinism: a second evaluation is bit-identical
    _, grad3 = m.loss_grad(dX, dl, di)
    assert torch.equal(grad, grad3)
    m.destroy()


def test_adam_steps_match_oracle():
    import torch
    qam, rows = 16, 256
    p = _params(qam, seed=9)
    X = _features(3 * rows, seed=4)
    labels = np.random.default_rng(5).integers(0, qam, 3 * rows).astype(np.int32)
    m = _mlp(qam, p)
    dX = torch.tensor(X, dtype=torch.float32, device="cuda")
    dl = torch.tensor(labels, device="cuda")
    ref = p.copy()
    mm, vv = np.zeros_like(p), np.zeros_like(p)
    lr = 1e-3
    for s in range(3):
        idx = np.arange(s * rows, (s + 1) * rows, dtype=np.int32)
        loss = torch.zeros(1, device="cuda")
        m.train_step(dX, dl, torch.tensor(idx, device="cuda"), lr, loss)
        _, g = omlp.loss_and_grad(ref, X[idx], labels[idx], qam)
        ref, mm, vv = omlp.adam(ref, mm, vv, g, s + 1, lr)
    got = m.get_params().astype(np.float64)
    # Adam's first steps move each weight by ~lr; FP32 gradients agree to ~1e-4 relative, so
    # the update of a weight with a tiny gradient may differ by up to lr in sign-sensitive cases
    diff = np.abs(got - ref)
    assert np.quantile(diff, 0.999) <= 0.05 * lr, np.quantile(diff, [0.5, 0.999])
    assert diff.max() <= 3 * lr
    m.destroy()


def _learned_detector(batch, chains, precision="fp32", seed=3):
    return H.make_detector(batch, chains=chains, precision=precision, seed=seed)


def test_features_match_oracle():
    b = workload.generate([(4, 6, 16, 14.0), (3, 3, 64, 20.0), (8, 8, 4, 9.0)], 21)
    det = _learned_detector(b, 8)
    det.run_chains(3)
    X = det.features().cpu().numpy()
    X0 = det.features(at_zero=True).cpu().numpy()
    flat, _ = det.get_chains()
    st = H.split_states(det, b, flat)
    r0 = r = 0
    for ch in range(b.n_channels):
        Hc, y, s2 = b.channel(ch)
        nt, q = int(b.nt[ch]), int(b.qam[ch])
        ref0 = omlp.features(Hc, y, s2, q)
        np.testing.assert_allclose(X0[r0:r0 + nt], ref0, rtol=2e-4, atol=2e-4 * np.abs(ref0).max())
        r0 += nt
        for c in range(8):
            ref = omlp.features(Hc, y, s2, q, st[ch][c])
            np.testing.assert_allclose(X[r:r + nt], ref, rtol=2e-4, atol=2e-4 * np.abs(ref).max())
            r += nt
    det.destroy()


def test_warm_start_matches_oracle():
    b = workload.generate([(4, 4, 16, 12.0), (6, 6, 16, 16.0), (3, 3, 4, 8.0)], 22)
    p = _params(16, seed=11, noise=0.2)
    m = _mlp(16, p)
    det = _learned_detector(b, 16)
    det.set_model(m, 0.5)
    det.init_learned()
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    bad = 0
    for ch in range(b.n_channels):
        if int(b.qam[ch]) != 16:
            continue
        lp = tg[ch].nn_logp(p)
        for c in range(16):
            exp = tg[ch].init_state_learned(3, ch, c, lp)
            if not np.array_equal(exp, st[ch][c]):
                bad += 1
            fx = oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(st[ch][c]))
            assert abs(f[ch * 16 + c] - fx) <= 1e-9 * abs(fx)
    assert bad <= 1, bad          # a CDF boundary within FP32 error of the uniform is ~1e-5 rare
    det.destroy()
    m.destroy()


def _mix_parity(det, b, tg, p, lam, steps, w_cat, w_acc, quant=False, seed=3):
    flat, _ = det.get_chains()
    cur = H.split_states(det, b, flat)
    res = dict(steps=0, mism=0, excused=0, bad=0, detail=[], acc=0)
    for s in range(steps):
        t = 5 + s
        det.mix_step(t)
        flat, _ = det.get_chains()
        nxt = H.split_states(det, b, flat)
        for ch in tg:
            for c in range(det.cfg.chains):
                exp, info = tg[ch].mix_step(seed, ch, c, t, cur[ch][c], lam, p, quant=quant)
                res["steps"] += 1
                res["acc"] += int(info.accepted)
                if np.array_equal(exp, nxt[ch][c]):
                    continue
                res["mism"] += 1
                if info.cat_margin < w_cat or abs(info.log_a - info.log_u) < w_acc:
                    res["excused"] += 1
                else:
                    res["bad"] += 1
                    if len(res["detail"]) < 5:
                        res["detail"].append((t, ch, c, info.cat_margin, info.log_a - info.log_u))
        cur = nxt
    return res


@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0])
def test_mixture_move_parity_fp32(lam):
    """FP32 handle, CUDA-core network: the FP32 windows of the plain sampler apply (2e-4 on the
    CDF margin, 2e-3 on |log A - log u|)."""
    b = workload.generate([(4, 4, 16, 12.0), (6, 8, 16, 18.0), (2, 2, 4, 6.0)], 23)
    p = _params(16, seed=12, noise=0.2)
    m = _mlp(16, p)
    det = _learned_detector(b, 16)
    det.run_chains(4)
    det.set_model(m, lam)
    tg = {ch: t for ch, t in H.targets(b).items() if int(b.qam[ch]) == 16}
    r = _mix_parity(det, b, tg, p, lam, 4, 2e-4, 2e-3)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(2, r["steps"] // 200), r
    # the untouched QPSK channel's chains did not move
    det.destroy()
    m.destroy()


def test_mixture_move_parity_tensor_cores():
    """MIXED handle, tcgen05 network against the oracle's quantised network: logits agree to
    ~1e-5 of their scale except on rows with a BF16 rounding flip (~1e-3), which widens the
    windows to 5e-3 (CDF margin) and 5e-2 (|log A - log u|, a sum over antennas)."""
    b = workload.generate([(8, 8, 16, 14.0), (4, 6, 16, 10.0)], 24)
    p = _params(16, seed=13, noise=0.2)
    m = _mlp(16, p)
    det = _learned_detector(b, 32, precision="mixed")
    det.run_chains(4)
    det.set_model(m, 0.5, tensor_cores=True)
    tg = H.targets(b)
    r = _mix_parity(det, b, tg, p, 0.5, 3, 5e-3, 5e-2, quant=True)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(3, r["steps"] // 50), r
    det.destroy()
    m.destroy()


def test_mixture_moves_keep_tracked_energies():
    b = workload.generate([(6, 6, 16, 16.0)] * 3, 25)
    p = _params(16, seed=14, noise=0.2)
    m = _mlp(16, p)
    det = _learned_detector(b, 32, precision="mixed")
    det.set_model(m, 0.5, tensor_cores=True)
    det.init_learned()
    det.run_mixed(12, 3)
    out = det.estimate(stats=True)
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    for ch in range(b.n_channels):
        for c in range(32):
            fx = oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(st[ch][c]))
            assert abs(f[ch * 32 + c] - fx) <= 1e-4 * abs(fx) + 1e-3
    assert out["stats"]["transitions"] == 12 * 3 * 32
    assert out["stats"]["accepts"] > 0
    det.destroy()
    m.destroy()
