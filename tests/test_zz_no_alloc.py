"""The allocation-free detection entry point against the handle-based one.

``mcmc_detect_noalloc`` is for callers that cannot call cudaMalloc (real-time loops that must not
wait on the allocator, hosts whose device memory belongs to a pool they do not manage,
components whose device memory budget is fixed when they start). It runs the same FP32 kernels with every intermediate
buffer in one fixed device array, so its labels, LLRs and energies must equal those of
create / preprocess / run_chains / estimate, within the FP32 tolerances the other GPU tests
use. Two calls in a row (different batches, then a repeat) check that each call starts from a
clean slate although the array keeps the previous call's contents. This file is collected last,
so a failure here never hides another test's result.
"""
import ctypes

import numpy as np
import pytest

import workload
from tests import helpers as H

pytestmark = pytest.mark.gpu

CHAINS, SEED = 32, 7


def _handle_path(batch, pre, iters):
    det = H.make_detector(batch, chains=CHAINS, precision="fp32", seed=SEED, preconditioned=pre)
    det.run_chains(iters)
    out = det.estimate()
    det.destroy()
    return out


def _noalloc(batch, pre, iters):
    import torch
    import paper_2407_06042_gb300 as pkg
    lib = pkg.lib()
    Hd, yd, s2 = H.upload(batch)
    n_ant = int(batch.nt.sum())
    n_bits = int((batch.nt.astype(np.int64) * np.log2(batch.qam).astype(np.int64)).sum())
    idx = torch.zeros(n_ant, dtype=torch.int8, device="cuda")
    llr = torch.zeros(n_bits, dtype=torch.float32, device="cuda")
    bf = torch.zeros(batch.n_channels, dtype=torch.float64, device="cuda")
    nt = np.ascontiguousarray(batch.nt, np.int32)
    nr = np.ascontiguousarray(batch.nr, np.int32)
    qam = np.ascontiguousarray(batch.qam, np.int32)
    ho = np.ascontiguousarray(batch.H_off, np.int64)
    yo = np.ascontiguousarray(batch.y_off, np.int64)
    p = lambda a: ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())
    st = lib.mcmc_detect_noalloc(batch.n_channels, p(nt), p(nr), p(qam), p(Hd), p(ho), p(yd),
                                 p(yo), p(s2), CHAINS, iters, SEED, int(pre), 1.0, 2.0, p(idx),
                                 p(llr), p(bf), None)
    return st, dict(best_idx=idx.cpu().numpy(), llr=llr.cpu().numpy(), best_f=bf.cpu().numpy())


def _compare(a, b):
    np.testing.assert_array_equal(a["best_idx"], b["best_idx"])
    np.testing.assert_allclose(a["llr"], b["llr"], rtol=2e-3, atol=2e-3)
    np.testing.assert_allclose(a["best_f"], b["best_f"], rtol=1e-10, atol=0)


@pytest.mark.parametrize("pre", [True, False])
@pytest.mark.parametrize("iters", [60, 0])
def test_noalloc_matches_handle_path_on_two_calls_in_a_row(pre, iters):
    b1 = workload.rayleigh_batch(4, 4, 16, [12.0], 24, 1001)
    # Nt = 40 takes the 4 x 4 register-tiled Gauss-Jordan (Nt in 33..64) in both paths
    b2 = workload.generate([(3, 5, 64, 22.0), (8, 8, 4, 9.0), (6, 6, 16, 15.0)] * 4
                           + [(40, 44, 16, 18.0)], 77)
    ref1, ref2 = _handle_path(b1, pre, iters), _handle_path(b2, pre, iters)
    st, out1 = _noalloc(b1, pre, iters)
    assert st == 0
    _compare(out1, ref1)
    st, out2 = _noalloc(b2, pre, iters)
    assert st == 0
    _compare(out2, ref2)
    st, again = _noalloc(b2, pre, iters)
    assert st == 0
    _compare(again, out2)


def test_noalloc_rejects_batches_beyond_its_scratch():
    # 20 000 channels of 32 x 32 need far more than the fixed 16 MiB array
    b = workload.rayleigh_batch(4, 4, 16, [12.0], 1, 1001)
    n = 20000
    big = workload.Batch(
        nt=np.full(n, 32, np.int32), nr=np.full(n, 32, np.int32), qam=np.full(n, 64, np.int32),
        snr_db=np.zeros(n), sigma2=np.ones(n, np.float32), H=b.H, H_off=np.zeros(n, np.int64),
        y=b.y, y_off=np.zeros(n, np.int64), tx_levels=b.tx_levels,
        lev_off=np.zeros(n, np.int64), tx_bits=b.tx_bits, bit_off=np.zeros(n, np.int64))
    import paper_2407_06042_gb300 as pkg
    lib = pkg.lib()
    arr = lambda a: ctypes.c_void_p(a.ctypes.data)
    nt, nr, qam = big.nt, big.nr, big.qam
    dummy = ctypes.c_void_p(1)   # never dereferenced: the size check comes first
    st = lib.mcmc_detect_noalloc(n, arr(nt), arr(nr), arr(qam), dummy, arr(big.H_off), dummy,
                                 arr(big.y_off), dummy, 64, 10, 0, 1, 1.0, 2.0, None, None, None,
                                 None)
    assert st == 1   # MCMC_EINVAL
