"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances (derivation in the design notes):
 * FP64 mode: chain states bit-exact; a mismatch is excused only at a near-tie of the oracle's
   own decision, |log A - log u| < 1e-6 or a categorical CDF margin < 1e-6 (of S_total);
   LLRs within 1e-9 (abs) + 1e-9 (rel); energies within 1e-10 relative.
 * FP32 mode: the same protocol with FP32 windows, 2e-3 for |log A - log u| and 2e-4 for the
   CDF margin (FP32 rounding of Gt x' amplified by 1/(tau sigma^2) and the proposal slope);
   unexcused mismatches must be zero, excused ones rare.
"""
import numpy as np
import pytest

import oracle
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _small(n=16, snr=12.0, seed=1001):
    return workload.rayleigh_batch(4, 4, 16, [snr], n, seed)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_initial_states_and_energies(precision):
    b = _small(8)
    det = H.make_detector(b, chains=32, precision=precision, seed=5)
    tg = H.targets(b)
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    for ch in range(b.n_channels):
        for c in range(32):
            np.testing.assert_array_equal(st[ch][c], tg[ch].init_state(5, ch, c))
            fx = oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(st[ch][c]))
            assert abs(f[ch * 32 + c] - fx) <= 1e-10 * max(1.0, abs(fx))
    det.destroy()


TRACE = 16   # MCMC_ENGINE_TRACE: the kernels record log A and log u of every chain's latest test


def test_fp64_step_parity():
    b = _small(16)
    det = H.make_detector(b, chains=32, precision="fp64", seed=0, engine=TRACE)
    r = H.step_parity(det, b, H.targets(b), seed=0, steps=25, energies=True, label="fp64_4x4")
    assert r["bad"] == 0, r
    assert r["mism"] <= 2, r
    # FP64 chains track energies and log A (Eq. (18)) to rounding
    assert r["energy_rel_max"] <= 1e-10, r
    assert r["max_dloga"] <= 1e-9, r
    det.destroy()


@pytest.mark.parametrize("precond", [True, False])
def test_fp64_full_run_matches_oracle(precond):
    b = _small(24)
    T = 100
    det = H.make_detector(b, chains=32, precision="fp64", seed=0, preconditioned=precond)
    det.run_chains(T)
    out = det.estimate(stats=True)
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    ref = oracle.detect_batch(b, chains=32, iterations=T, seed=0, preconditioned=precond)
    diverged = 0
    for ch in range(b.n_channels):
        diverged += int(np.any(ref[ch]["final_states"] != st[ch], axis=1).sum())
    assert diverged <= 1, diverged
    nb = 4 * 4
    for ch in range(b.n_channels):
        if np.any(ref[ch]["final_states"] != st[ch]):
            continue
        np.testing.assert_allclose(out["llr"][ch * nb:(ch + 1) * nb], ref[ch]["llr"],
                                   rtol=1e-6, atol=1e-4)
        np.testing.assert_allclose(f[ch * 32:(ch + 1) * 32], ref[ch]["final_f"], rtol=1e-10)
        assert abs(out["best_f"][ch] - ref[ch]["best_f"]) <= 1e-10 * abs(ref[ch]["best_f"])
    assert out["stats"]["transitions"] == T * 32 * b.n_channels
    det.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_one_launch_equals_single_step_launches(precision):
    b = _small(6)
    d1 = H.make_detector(b, chains=32, precision=precision)
    d1.run_chains(20)
    s1, _ = d1.get_chains()
    d2 = H.make_detector(b, chains=32, precision=precision)
    for t in range(20):
        d2.run_chains(1, t)
    s2, _ = d2.get_chains()
    np.testing.assert_array_equal(s1, s2)
    d1.destroy()
    d2.destroy()


def test_fp32_step_parity():
    b = _small(16)
    det = H.make_detector(b, chains=32, precision="fp32", seed=0, engine=TRACE)
    r = H.step_parity(det, b, H.targets(b), seed=0, steps=25, w_cat=2e-4, w_acc=2e-3,
                      energies=True, label="fp32_4x4")
    assert r["bad"] == 0, r
    assert r["mism"] <= max(3, r["steps"] // 2000), r
    # the energies the chains hold after each launch: FP32 increments from exact initial values,
    # replaced by exact evaluations when the launch ends (refresh_period 0)
    assert r["energy_rel_max"] <= 1e-10, r
    # the kernel's log A against the oracle's: well inside the accept window
    assert r["max_dloga"] <= 2e-3, r
    det.destroy()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_estimate_matches_oracle_on_gpu_states(precision):
    b = _small(12, snr=10.0)
    det = H.make_detector(b, chains=32, precision=precision)
    det.run_chains(40)
    out = det.estimate()
    flat, f = det.get_chains()
    st = H.split_states(det, b, flat)
    tg = H.targets(b)
    nb = 16
    tol = 1e-6 if precision == "fp64" else 2e-3
    for ch in range(b.n_channels):
        ref = tg[ch].llr_is(st[ch])
        np.testing.assert_allclose(out["llr"][ch * nb:(ch + 1) * nb], ref, rtol=tol, atol=tol)
        lev = H.levels_from_labels(out["best_idx"][ch * 4:(ch + 1) * 4], 4, 4)
        fb = oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(lev))
        assert abs(out["best_f"][ch] - fb) <= 1e-10 * abs(fb)
        fin = max(oracle.f_value(tg[ch].Hr, tg[ch].yr, tg[ch].sigma2, tg[ch].values(s))
                  for s in st[ch])
        # FP32 modes track energies with FP32 differences: the running best may miss a final
        # state by the tracking error only
        btol = 1e-9 if precision == "fp64" else 1e-4
        assert out["best_f"][ch] >= fin - btol * abs(fin)
    det.destroy()


def test_ragged_shapes_and_mixed_modulations_fp64():
    """Odd Nt (N = 2, 6, 10), Nr below / above Nt, QPSK / 16 / 64-QAM in one batch, a chain count
    that is not a multiple of the kernel's chain tile."""
    shapes = [(1, 1, 4, 10.0), (3, 2, 16, 14.0), (5, 7, 64, 22.0), (3, 6, 4, 6.0), (2, 2, 64, 25.0)]
    b = workload.generate(shapes, 77)
    for precond in (True, False):
        det = H.make_detector(b, chains=36, precision="fp64", seed=3, preconditioned=precond)
        r = H.step_parity(det, b, H.targets(b, preconditioned=precond), seed=3, steps=12)
        assert r["bad"] == 0, r
        det.destroy()


def test_host_io_equals_device_io():
    b = _small(5)
    d1 = H.make_detector(b, chains=32, precision="fp32")
    d1.run_chains(30)
    o1 = d1.estimate()
    d2 = H.make_detector(b, chains=32, precision="fp32", host_io=True)
    d2.run_chains(30)
    o2 = d2.estimate()
    for k in ("best_idx", "llr", "best_f"):
        np.testing.assert_array_equal(o1[k], o2[k])
    d1.destroy()
    d2.destroy()


def test_resume_is_exact():
    b = _small(4)
    d1 = H.make_detector(b, chains=32, precision="fp32")
    d1.run_chains(60)
    d2 = H.make_detector(b, chains=32, precision="fp32")
    d2.run_chains(25)
    s, _ = d2.get_chains()
    d3 = H.make_detector(b, chains=32, precision="fp32")
    d3.set_chains(s)
    d3.run_chains(35, 25)
    np.testing.assert_array_equal(d1.get_chains()[0], d3.get_chains()[0])
    for d in (d1, d2, d3):
        d.destroy()


def test_error_paths():
    from paper_2407_06042_gb300 import Detector, McmcError
    b = _small(2)
    with pytest.raises(McmcError) as e:
        Detector(max_channels=1, max_nt=4, max_nr=4, chains=30)      # chains % 4 != 0
    assert e.value.status == 1
    det = Detector(max_channels=2, max_nt=4, max_nr=4, chains=32)
    with pytest.raises(McmcError) as e:
        det.run_chains(5)
    assert e.value.status == 6                                        # before preprocess
    Hd, yd, s2 = H.upload(b)
    with pytest.raises(McmcError) as e:
        det.preprocess(b.nt, b.nr, np.array([16, 8]), Hd, b.H_off, yd, b.y_off, s2)
    assert e.value.status == 1                                        # bad QAM order
    det.preprocess(b.nt, b.nr, b.qam, Hd, b.H_off, yd, b.y_off, s2)
    bad = np.full(2 * 32 * 8, 9, np.int8)
    with pytest.raises(McmcError) as e:
        det.set_chains(bad)
    assert e.value.status == 1                                        # level out of range
    det.destroy()
