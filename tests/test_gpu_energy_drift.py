"""The energies the chains track between exact evaluations, at the 32x32 64-QAM headline shape
(SNR 20..32 dB, 64 chains, 200 transitions).

FP32 and MIXED chains add FP32 energy differences (Algorithm 1's MH ratio, Eq. (18)) to an
exact starting value. By default every run ends with an exact evaluation (refresh_period 0), so
the read-outs see exact energies; with refresh_period -1 there is none, and the tracked values
show the drift the increments accumulate. That drift is absolute: each increment
(1/sigma^2) sum_n (xt'_n - xt_n)(2 zt_n - (Gt xt)_n - (Gt xt')_n) is formed from terms of size
|zt_n| and rounded to FP32 (MIXED also multiplies by Gt's BF16 split, 2^-17 relative per entry
with two terms), while |f| near the transmitted vector is only about 2 Nr. At 32 dB that makes
the relative drift after 200 transitions larger than 1e-5 in every FP32 form; the measured
figures are written to $MCMC_PARITY_REPORT, and the bounds below are a few times them.
"""
import json
import os

import numpy as np
import pytest

import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

BOUND = {"fp32": 1e-4, "mixed3": 3e-4, "mixed2": 1e-3}
SAMPLE = [0, 1, 200, 300, 511, 600, 700, 895]


@pytest.fixture(scope="module")
def batch():
    w = workload.WORKLOADS["rayleigh_32x32_64qam"]
    return workload.rayleigh_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], 128, w["seed"])


@pytest.mark.parametrize("form", ["fp32", "mixed3", "mixed2"])
def test_tracked_energy_drift(batch, form):
    b = batch
    prec = "mixed" if form.startswith("mixed") else form
    kw = dict(split_terms=int(form[-1])) if prec == "mixed" else {}
    out = {}
    for R in (-1, 0):
        det = H.make_detector(b, chains=64, precision=prec, seed=0, refresh_period=R, **kw)
        det.run_chains(200)
        ftr, _ = det.get_tracked()
        _, fx = det.get_chains()            # exact evaluations (the handle keeps its values)
        st = det.estimate(stats=True)["stats"]
        states = H.states_now(det, b)
        det.destroy()
        rel = np.abs(ftr - fx) / np.abs(fx)
        out[R] = dict(max=float(rel.max()), p99=float(np.quantile(rel, 0.99)),
                      median=float(np.median(rel)), drift_rel=st["refresh_drift_rel"])
        # the exact evaluations against the oracle's f on a sample
        tg = H.targets(b, channels=SAMPLE)
        for ch in SAMPLE:
            for c in range(0, 64, 9):
                fo = H.fp64_energy(tg[ch], states[ch][c])
                assert abs(fx[ch * 64 + c] - fo) <= 1e-10 * abs(fo)
    path = os.environ.get("MCMC_PARITY_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(dict(label=f"energy_drift_{form}_32x32_64qam_T200",
                                     no_refresh=out[-1], default=out[0])) + "\n")
    # without any refresh: the drift stays within the stated bound
    assert out[-1]["max"] <= BOUND[form], out
    # default: the run ends with exact energies, and the correction it made is the drift
    assert out[0]["max"] <= 1e-10, out
    assert out[0]["drift_rel"] <= BOUND[form], out
