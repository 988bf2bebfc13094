"""GPU parity of the tensor-core (MIXED precision) chain kernel against the FP64 oracle.

The Gram products run on tcgen05 from BF16 split terms of Gt and P~Gt with FP32 accumulation;
everything else is FP32. With three split terms the products carry ~24 significant bits, as in
FP32, and the FP32 windows apply (2e-3 on |log A - log u|, 2e-4 on the CDF margin). With two
terms (~16 bits) the same protocol runs with windows 32x wider: the split error 2^-17 relative
per product replaces FP32's 2^-24 in the error of Gt x' and of the drift slope.
"""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

TC = 2            # MCMC_ENGINE_TC: these tests pin the tensor-core kernel itself
TRACE = 16        # MCMC_ENGINE_TRACE: log A and log u of every chain's latest test
GRAPH = 4         # MCMC_ENGINE_GRAPH
NO_CLUSTER = 8    # MCMC_ENGINE_NO_CLUSTER: N > 128 on the single-CTA kernel (operand streamed)


def _small(n=16, snr=12.0, seed=1001):
    return workload.rayleigh_batch(4, 4, 16, [snr], n, seed)


@pytest.mark.parametrize("terms,w_cat,w_acc", [(3, 2e-4, 2e-3), (2, 6.4e-3, 6.4e-2)])
def test_mixed_step_parity(terms, w_cat, w_acc):
    b = _small(16)
    det = H.make_detector(b, chains=32, precision="mixed", split_terms=terms, seed=0,
                          engine=TC | TRACE)
    r = H.step_parity(det, b, H.targets(b), seed=0, steps=25, w_cat=w_cat, w_acc=w_acc,
                      energies=True, label=f"mixed_s{terms}_4x4")
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 1000), r
    assert r["max_dloga"] <= w_acc, r
    # the energies the chains hold after each launch (exact evaluations at the end of a run),
    # against the oracle's f of their states
    assert r["energy_rel_max"] <= 1e-10, r
    det.destroy()


@pytest.mark.parametrize("big", [False, True])
def test_mixed_one_launch_equals_single_step_launches(big):
    # big: N = 200 on four-CTA clusters, whose decisions come from exchanged partial sums
    b = workload.generate([(100, 100, 16, 20.0)] * 2, 97) if big else _small(6)
    steps = 8 if big else 20
    d1 = H.make_detector(b, chains=32, precision="mixed", engine=TC)
    d1.run_chains(steps)
    s1, f1 = d1.get_chains()
    d2 = H.make_detector(b, chains=32, precision="mixed", engine=TC)
    for t in range(steps):
        d2.run_chains(1, t)
    s2, f2 = d2.get_chains()
    np.testing.assert_array_equal(s1, s2)
    d1.destroy()
    d2.destroy()


@pytest.mark.parametrize("shapes", [
    [(36, 40, 16, 18.0), (33, 33, 64, 26.0)],          # N = 72, 66: ragged K and dimensions
    [(64, 64, 16, 20.0), (64, 128, 4, 8.0)],           # N = 128: two A-operand tiles
    [(1, 2, 4, 6.0), (3, 3, 64, 20.0), (8, 16, 16, 14.0)],
    [(80, 96, 16, 18.0), (100, 100, 4, 12.0)],         # N = 160, 200: 3- / 4-CTA clusters
    [(128, 128, 64, 28.0)],                            # N = 256: the largest channel
])
@pytest.mark.parametrize("flags", [0, NO_CLUSTER])
def test_mixed_step_parity_shapes(shapes, flags):
    # flags: N > 128 on thread-block clusters (resident operand tiles), or on the single-CTA
    # kernel that streams the operand from L2
    b = workload.generate(shapes, 91)
    det = H.make_detector(b, chains=36, precision="mixed", split_terms=3, seed=2, engine=TC | flags)
    r = H.step_parity(det, b, H.targets(b), seed=2, steps=6, w_cat=2e-4, w_acc=2e-3)
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 500), r
    det.destroy()


@pytest.mark.parametrize("tile,terms,shapes", [
    (64, 2, [(128, 128, 64, 28.0), (120, 128, 16, 24.0)]),   # N = 256, 240: 64 chains per CTA
    (16, 2, [(70, 80, 4, 14.0)]),                             # N = 140: three-CTA clusters
    (32, 3, [(100, 100, 64, 26.0)]),                          # N = 200: fourth tile a quarter full
])
def test_mixed_cluster_tiles(tile, terms, shapes):
    """N > 128 on thread-block clusters (one resident operand tile per CTA; x' slices and the
    chains' partial sums exchanged through distributed shared memory) at every chain tile: step
    parity against the oracle with full and partial work items (100 chains per channel)."""
    b = workload.generate(shapes, 95)
    det = H.make_detector(b, chains=100, precision="mixed", split_terms=terms, seed=6, engine=TC,
                          tile=tile)
    w = 1.0 if terms == 3 else 32.0
    r = H.step_parity(det, b, H.targets(b), seed=6, steps=4, w_cat=2e-4 * w, w_acc=2e-3 * w)
    assert r["steps"] == 4 * 100 * b.n_channels
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 500), r
    det.destroy()


def test_mixed_ber_within_binomial_interval_of_oracle():
    """4x4 16-QAM at 12 dB, 1000 channels, 32 chains x 100 iterations: the GPU's uncoded BER of
    sign(LLR) lies inside the 95% Clopper-Pearson interval of the oracle's."""
    from scipy.stats import beta
    b = workload.workload("rayleigh_4x4_16qam")
    det = H.make_detector(b, chains=32, precision="mixed", seed=0, engine=TC)
    det.run_chains(100)
    out = det.estimate()
    det.destroy()
    ref = oracle.detect_batch(b, chains=32, iterations=100, seed=0)
    bits = b.tx_bits.astype(int)
    e_gpu = int(((out["llr"] < 0).astype(int) != bits).sum())
    e_ref = int(((np.concatenate([r["llr"] for r in ref]) < 0).astype(int) != bits).sum())
    n = bits.size
    lo = beta.ppf(0.025, e_ref, n - e_ref + 1) if e_ref else 0.0
    hi = beta.ppf(0.975, e_ref + 1, n - e_ref)
    assert lo <= e_gpu / n <= hi, (e_gpu, e_ref, n)


def test_mixed_energies_refresh():
    """Exact refresh every R transitions and at the end of every run: the energies the chains
    hold (exported as they are) equal the oracle's f of the states after a run that ends on a
    refresh point and after one that ends between refresh points; the largest correction a
    refresh made stays small."""
    b = _small(4, snr=20.0)
    det = H.make_detector(b, chains=32, precision="mixed", refresh_period=10, engine=TC)
    tg = H.targets(b)

    def check(tol):
        st = H.states_now(det, b)
        f, _ = det.get_tracked()
        for ch in range(b.n_channels):
            for c in range(32):
                fx = H.fp64_energy(tg[ch], st[ch][c])
                assert abs(f[ch * 32 + c] - fx) <= tol * abs(fx), (ch, c, f[ch * 32 + c], fx)

    det.run_chains(30)
    check(1e-10)             # transition 30 is a refresh point
    det.run_chains(5, 30)
    check(1e-10)             # five FP32 increments past it, then the end-of-run refresh
    out = det.estimate(stats=True)
    assert out["stats"]["refresh_drift"] < 1e-2
    assert out["stats"]["refresh_drift_rel"] < 1e-3
    det.destroy()


def test_uneven_batch_autotuned_and_graph_replay():
    """Uneven batch (Nt in {2..16}, Nr in {Nt, 2Nt}, QPSK..64-QAM): the autotuned engines keep
    oracle parity, and replaying the launches from a captured CUDA graph gives bit-identical
    chains."""
    b = workload.uneven_batch(40, 1003, nts=(2, 4, 8, 16), snr_range=(8.0, 20.0))
    det = H.make_detector(b, chains=32, precision="mixed", split_terms=3, seed=4)
    r = H.step_parity(det, b, H.targets(b), seed=4, steps=5, w_cat=2e-4, w_acc=2e-3)
    assert r["bad"] == 0, r
    det.destroy()
    d1 = H.make_detector(b, chains=32, precision="mixed", seed=4)
    d1.run_chains(15)
    d1.run_chains(10, 15)
    o1 = d1.estimate()
    d2 = H.make_detector(b, chains=32, precision="mixed", seed=4, engine=GRAPH)
    d2.run_chains(15)
    d2.run_chains(10, 15)
    o2 = d2.estimate()
    np.testing.assert_array_equal(d1.get_chains()[0], d2.get_chains()[0])
    np.testing.assert_array_equal(o1["llr"], o2["llr"])
    d1.destroy()
    d2.destroy()


def test_cluster_graph_replay():
    """N = 200 and 256 on thread-block clusters, launched directly and replayed from a captured
    CUDA graph (with the FP64 refresh): bit-identical chains and LLRs."""
    b = workload.generate([(100, 100, 16, 20.0), (128, 128, 64, 26.0)], 99)
    outs = []
    for flags in (TC, TC | GRAPH):
        det = H.make_detector(b, chains=64, precision="mixed", seed=8, refresh_period=5, engine=flags)
        det.run_chains(7)
        det.run_chains(6, 7)
        outs.append((det.get_chains()[0], det.estimate()["llr"]))
        det.destroy()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("flags", [0, NO_CLUSTER])
def test_mixed_kronecker_256_refresh(flags):
    """128x128 64-QAM Kronecker channels (N = 256: four-CTA clusters, or the single-CTA kernel
    with the operand streamed) with the FP64 refresh every 10 transitions: step parity, then
    tracked energies equal to FP64 evaluations right after a refresh point. The clusters'
    refresh rounds G to 53 bits below its largest diagonal entry: at most about 2e-14 of the
    quadratic term, which the cancellation in f = -|y - Hx|^2 / sigma^2 (30 dB) raises to about
    2e-11 of f, below the 1e-10 asked here."""
    b = workload.kronecker_batch(128, 128, 64, [30.0], 2, 0.5, 77)
    det = H.make_detector(b, chains=32, precision="mixed", split_terms=3, refresh_period=10,
                          seed=5, engine=TC | flags)
    r = H.step_parity(det, b, H.targets(b), seed=5, steps=3, w_cat=2e-4, w_acc=2e-3)
    assert r["bad"] == 0, r
    det.run_chains(17, 3)
    out = det.estimate(stats=True)
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    ftr, _ = det.get_tracked()
    for ch in range(b.n_channels):
        for c in range(32):
            fx = oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(st[ch][c]))
            assert abs(f[ch * 32 + c] - fx) <= 1e-10 * abs(fx)
            assert abs(ftr[ch * 32 + c] - fx) <= 1e-10 * abs(fx)
    # the largest correction a refresh made to the FP32-tracked energies (ten transitions apart)
    assert out["stats"]["refresh_drift_rel"] < 1e-3, out["stats"]
    det.destroy()


@pytest.mark.parametrize("tile,shapes", [
    (16, [(16, 16, 16, 16.0)] * 3),                  # N = 32: every work item full, 2 x 16 chains
    (32, [(16, 16, 16, 16.0), (16, 20, 4, 10.0)]),   # 2 x 32 chains per CTA (64 per work item)
    (16, [(15, 15, 16, 14.0), (9, 12, 64, 22.0)]),   # N = 30, 18: ragged dimensions in each group
])
def test_mixed_two_chain_groups(tile, shapes):
    """Channels of N <= 32 run two chain groups per CTA (the operand rows held twice); step
    parity against the oracle with full and partial work items and both tiles."""
    b = workload.generate(shapes, 93)
    det = H.make_detector(b, chains=96, precision="mixed", split_terms=2, seed=5, engine=TC, tile=tile)
    r = H.step_parity(det, b, H.targets(b), seed=5, steps=4, w_cat=2e-4, w_acc=2e-3)
    assert r["steps"] == 4 * 96 * b.n_channels
    assert r["bad"] == 0, r
    assert r["mism"] <= max(4, r["steps"] // 500), r
    det.destroy()


def test_deferred_initial_energies_and_kernel_timing():
    """The exact initial energies are evaluated by the first run after preprocess (read-outs
    before it hand out FP64 evaluations of the initial states, for f and the running best), so
    a run that follows equals the oracle's energies at the 1e-10 bar whether or not something
    was read out in between; the run's chain-kernel time excludes the evaluations around it and
    is no longer than the whole run."""
    import torch
    b = _small(4, snr=20.0)
    tg = H.targets(b)
    det = H.make_detector(b, chains=32, precision="mixed", engine=TC, seed=3)
    st0 = H.states_now(det, b)
    f0, best0 = det.get_tracked()
    for ch in range(b.n_channels):
        for c in range(32):
            fx = H.fp64_energy(tg[ch], st0[ch][c])
            assert abs(f0[ch * 32 + c] - fx) <= 1e-10 * abs(fx)
            assert best0[ch * 32 + c] == f0[ch * 32 + c]
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    det.run_chains(20)
    ev1.record(stream)
    torch.cuda.synchronize()
    (kms,) = det.run_kernel_ms(1)
    assert 0.0 < kms <= ev0.elapsed_time(ev1)
    st = H.states_now(det, b)
    f, _ = det.get_tracked()
    for ch in range(b.n_channels):
        for c in range(32):
            fx = H.fp64_energy(tg[ch], st[ch][c])
            assert abs(f[ch * 32 + c] - fx) <= 1e-10 * abs(fx)
    # the same seed without the read-out before the run: identical chains and energies
    det2 = H.make_detector(b, chains=32, precision="mixed", engine=TC, seed=3)
    det2.run_chains(20)
    f2, best2 = det2.get_tracked()
    _, best = det.get_tracked()
    np.testing.assert_array_equal(f2, f)
    np.testing.assert_array_equal(best2, best)
    assert len(det2.run_kernel_ms(1)) == 1
    det.destroy()
    det2.destroy()


KERNEL_REFRESH = 128   # MCMC_ENGINE_KERNEL_REFRESH: in-run refreshes inside the chain kernels


@pytest.mark.parametrize("case", ["cluster", "streamed", "one_tile", "simt_fp32"])
def test_in_run_refresh_between_launches(case):
    """A run with in-run refreshes is cut into launches at the refresh points, with the exact
    refresh kernel between them; the in-kernel refreshes (MCMC_ENGINE_KERNEL_REFRESH) give the
    same chains: equal states, acceptances, near-tie counts, best samples and LLRs, and energies
    equal to within the two exact evaluations' rounding. The second run starts between refresh
    points."""
    if case in ("cluster", "streamed"):
        b = workload.kronecker_batch(128, 128, 64, [30.0], 2, 0.5, 78)
        kw = dict(chains=64, precision="mixed", split_terms=2,
                  engine=TC | (NO_CLUSTER if case == "streamed" else 0))
    elif case == "one_tile":
        b = workload.rayleigh_batch(32, 32, 64, [26.0], 8, 79)
        kw = dict(chains=32, precision="mixed", split_terms=2, engine=TC)
    else:
        b = workload.rayleigh_batch(32, 32, 64, [26.0], 8, 79)
        kw = dict(chains=32, precision="fp32", engine=1)   # MCMC_ENGINE_SIMT
    outs = []
    for extra in (0, KERNEL_REFRESH):
        kx = dict(kw)
        kx["engine"] = kw["engine"] | extra
        det = H.make_detector(b, seed=11, refresh_period=7, **kx)
        det.run_chains(17)
        det.run_chains(9, 17)
        flat, _ = det.get_chains()
        ftr, fbest = det.get_tracked()
        est = det.estimate(stats=True)
        outs.append((flat.copy(), ftr.copy(), fbest.copy(), est))
        det.destroy()
    (s0, f0, b0, e0), (s1, f1, b1, e1) = outs
    np.testing.assert_array_equal(s0, s1)
    assert e0["stats"]["accepts"] == e1["stats"]["accepts"]
    assert e0["stats"]["near_ties"] == e1["stats"]["near_ties"]
    assert e0["stats"]["accepts"] > 0
    np.testing.assert_allclose(f0, f1, rtol=1e-10, atol=0)
    np.testing.assert_allclose(b0, b1, rtol=1e-10, atol=0)
    np.testing.assert_array_equal(e0["best_idx"], e1["best_idx"])
    np.testing.assert_allclose(e0["llr"], e1["llr"], rtol=1e-5, atol=1e-5)
