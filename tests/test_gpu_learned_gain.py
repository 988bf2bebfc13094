"""What the trained network gains over the method without it.

The network is trained on the GPU by the library's own kernels, on samples the plain sampler
generates (32x32 16-QAM Rayleigh, SNR U[12, 24] dB: 512 channels x 16 chains, features at
transitions 0, 2, 5, 10, 20, 40 and at x = 0, labelled with the channel's best sample after 200
transitions), and evaluated on 64x64 16-QAM Rayleigh (SNR U[12, 24] dB, 256 channels, 64
chains). Both runs are exact MCMC on the same posterior; the learned warm start only changes
where the chains begin. Measured on GB300 (BER of sign(LLR)): the plain sampler needs 20
transitions for 0.177 and 40 for 0.169; the warm start gives 0.169 after 5 and 0.165 after 20.
The assertions leave margins of several binomial standard deviations (~0.0015 at 65 536 bits)."""
import numpy as np
import pytest

import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_2407_06042_gb300 import Mlp, learned
    rng = np.random.default_rng(7)
    btr = workload.generate([(32, 32, 16, float(s)) for s in rng.uniform(12, 24, 512)], 2001)
    det = H.make_detector(btr, chains=16, precision="mixed", seed=1)
    X, lab = learned.chain_samples(det, [0, 2, 5, 10, 20, 40], 200, label="best")
    det.destroy()
    m = Mlp(16, max_rows=4096)
    m.set_params(learned.init_params(16, 0))
    hist = learned.train(m, X, lab, epochs=8, batch=4096, lr=1e-3)
    bev = workload.generate([(64, 64, 16, float(s)) for s in rng.uniform(12, 24, 256)], 2002)
    yield m, hist, bev
    m.destroy()


def test_training_reduces_the_loss(trained):
    _, hist, _ = trained
    assert hist[-1] < 0.75 * np.log(16)          # well below the uniform guess
    assert hist[-1] < hist[0]


def test_warm_start_reaches_equal_ber_in_fewer_iterations(trained):
    from paper_2407_06042_gb300 import learned
    m, _, bev = trained
    cps = [5, 20, 40]
    d = H.make_detector(bev, chains=64, precision="mixed", seed=3)
    plain = {c["T"]: c["ber_llr"] for c in learned.ber_curve(d, bev.tx_bits, cps)}
    d.destroy()
    d = H.make_detector(bev, chains=64, precision="mixed", seed=3)
    d.set_model(m, 0.0, tensor_cores=True)
    warm = {c["T"]: c["ber_llr"] for c in learned.ber_curve(d, bev.tx_bits, cps, learned=True)}
    d.destroy()
    assert warm[5] < plain[20] - 0.003, (plain, warm)
    assert warm[20] < plain[40], (plain, warm)


def test_mixture_moves_do_not_hurt(trained):
    """Mixture moves every 5 transitions (lambda = 0.5) after the warm start: exact MH moves, so
    the BER must stay at least as good as the warm start's alone (within noise)."""
    from paper_2407_06042_gb300 import learned
    m, _, bev = trained
    d = H.make_detector(bev, chains=64, precision="mixed", seed=3)
    d.set_model(m, 0.0, tensor_cores=True)
    warm = learned.ber_curve(d, bev.tx_bits, [40], learned=True)[0]["ber_llr"]
    d.destroy()
    d = H.make_detector(bev, chains=64, precision="mixed", seed=3)
    d.set_model(m, 0.5, tensor_cores=True)
    mixed = learned.ber_curve(d, bev.tx_bits, [40], learned=True, period=5)[0]["ber_llr"]
    d.destroy()
    assert mixed <= warm + 0.004, (warm, mixed)
