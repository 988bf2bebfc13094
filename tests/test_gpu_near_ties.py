"""Near-tie accounting of the parity protocol, per precision, at the 4x4 16-QAM and the 32x32
64-QAM shapes: many single-transition steps compared with the FP64 oracle (step mode, the
oracle re-synchronised to the GPU state after every step).

For every transition the oracle's own margins are recorded (|log A - log u| of Eq. (18) and the
categorical CDF margin of Eqs. (16)-(17)/(21)); every GPU/oracle mismatch is put in a band of
that margin (< 1e-6, < 1e-4, < the precision's window). The kernels' own log A (recorded with
MCMC_ENGINE_TRACE) is compared with the oracle's on every transition whose proposal is
unambiguous, and the energies the chains track are compared with the oracle's f of their states
after every step. The kernels also count their own near-ties (mcmc_stats.near_ties). Each case
appends its figures to $MCMC_PARITY_REPORT when that variable names a file.

Windows: FP64 1e-6 (the bar stated for FP64 accept decisions); FP32 and MIXED with three split terms 2e-4 (CDF) and 2e-3
(accept), the FP32 rounding of Gt x' amplified by 1/(tau sigma^2); MIXED with two terms 32x
those (the split error 2^-17 per product instead of 2^-24)."""
import numpy as np
import pytest

import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

TRACE = 16
WINDOWS = {"fp64": (1e-6, 1e-6), "fp32": (2e-4, 2e-3), "mixed3": (2e-4, 2e-3),
           "mixed2": (6.4e-3, 6.4e-2)}
SHAPES = {"4x4_16qam": dict(nt=4, qam=16, snr=[12.0], n=128, chains=32, steps=24),
          "32x32_64qam": dict(nt=32, qam=64, snr=[20.0, 26.0, 32.0], n=16, chains=64, steps=10)}


@pytest.mark.parametrize("shape", sorted(SHAPES))
@pytest.mark.parametrize("form", ["fp64", "fp32", "mixed3", "mixed2"])
def test_near_tie_bands(form, shape):
    sp = SHAPES[shape]
    b = workload.rayleigh_batch(sp["nt"], sp["nt"], sp["qam"], sp["snr"], sp["n"], 2024)
    prec = "mixed" if form.startswith("mixed") else form
    kw = dict(split_terms=int(form[-1])) if prec == "mixed" else {}
    det = H.make_detector(b, chains=sp["chains"], precision=prec, seed=11, engine=TRACE, **kw)
    w_cat, w_acc = WINDOWS[form]
    r = H.step_parity(det, b, H.targets(b), seed=11, steps=sp["steps"], w_cat=w_cat, w_acc=w_acc,
                      energies=True, label=f"near_ties_{form}_{shape}")
    out = det.estimate(stats=True)
    det.destroy()
    n = r["steps"]
    assert n == sp["n"] * len(sp["snr"]) * sp["chains"] * sp["steps"]
    assert r["bad"] == 0, r
    # excused mismatches are rare: at most 1 % of the transitions, and none in FP64 beyond the
    # oracle's own near-ties
    assert r["mism"] <= max(4, n // 100), r
    # the kernel's log A against the oracle's, on unambiguous proposals: inside the window
    assert r["max_dloga"] is not None and r["max_dloga"] <= w_acc, r
    # the kernel's own near-tie counts cover every transition it took (the probe launches of
    # the autotuner are not counted)
    ties = out["stats"]["near_ties"]
    assert ties[0] <= ties[1] <= ties[2] <= out["stats"]["transitions"], ties
    if form in ("fp64", "fp32", "mixed3"):
        assert r["energy_rel_max"] <= 1e-5, r
