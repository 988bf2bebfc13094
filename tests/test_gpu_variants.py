"""The detector on the paper's other channel conditions (Sec. IV-C/D/F): step parity against the
oracle on an imperfect-CSI batch (both see the estimate H^ = H + E), the BER's growth with the
estimate's NMSE, and the correlated 16x16 16-QAM channel of Fig. 9 in MIXED precision."""
import numpy as np
import pytest

import bench
import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,w", [("fp64", (1e-6, 1e-6)), ("fp32", (2e-4, 2e-3))])
def test_csi_step_parity(precision, w):
    b = workload.csi_batch(4, 4, 16, 12.0, [-20.0, -10.0], 3, 41)
    det = H.make_detector(b, chains=16, precision=precision, seed=9)
    r = H.step_parity(det, b, H.targets(b), seed=9, steps=4, w_cat=w[0], w_acc=w[1])
    assert r["steps"] == 4 * 16 * b.n_channels
    assert r["bad"] == 0, r
    det.destroy()


def _ber(b, chains, T, precision="mixed"):
    det = H.make_detector(b, chains=chains, precision=precision, seed=0)
    det.run_chains(T)
    out = det.estimate()
    det.destroy()
    return bench.ber_of(b, out["llr"], out["best_idx"])


def test_csi_ber_grows_with_the_estimation_error():
    b = workload.csi_batch(16, 16, 16, 16.5, [-30.0, -10.0], 128, 42)
    ber = _ber(b, 64, 50)
    assert ber["nmse-10"]["ber_llr"] > 2 * ber["nmse-30"]["ber_llr"], ber


def test_correlated_16x16_16qam_mixed_matches_fp32():
    """Fig. 9's channel: the MIXED form and the plain FP32 sampler run the same chains up to
    rounding, so their BERs agree closely."""
    b = workload.kronecker_batch(16, 16, 16, [18.0], 256, 0.5, 43)
    m = _ber(b, 64, 60, "mixed")["18"]["ber_llr"]
    f = _ber(b, 64, 60, "fp32")["18"]["ber_llr"]
    assert abs(m - f) <= max(0.1 * f, 2e-4), (m, f)
