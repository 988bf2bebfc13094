"""CPU checks of the synthetic workloads of the paper's other experiments: the imperfect-CSI batch
(Sec. IV-F) keeps the true system and adds an estimation error of the requested NMSE; the
large-MIMO and correlated workloads (Figs. 7-9) materialise with their shapes; the bench groups
BER by NMSE point."""
import numpy as np
import pytest

import bench
import workload


def test_csi_batch_error_has_the_requested_nmse():
    pts = [-25.0, -15.0]
    b = workload.csi_batch(16, 16, 16, 16.5, pts, 256, 77)
    ref = workload.generate([(16, 16, 16, 16.5)] * 512, 77)
    # the true system: same symbols, noise and received vectors as the perfect-CSI draw
    np.testing.assert_array_equal(b.y, ref.y)
    np.testing.assert_array_equal(b.tx_bits, ref.tx_bits)
    np.testing.assert_array_equal(b.sigma2, ref.sigma2)
    E = (b.H.astype(np.complex128) - ref.H.astype(np.complex128)).reshape(512, 256)
    Ht = ref.H.astype(np.complex128).reshape(512, 256)
    for i, p in enumerate(pts):
        sl = slice(256 * i, 256 * (i + 1))
        nmse = np.sum(np.abs(E[sl]) ** 2) / np.sum(np.abs(Ht[sl]) ** 2)
        assert abs(10 * np.log10(nmse) - p) < 0.1, (p, 10 * np.log10(nmse))
        # circular, zero mean, uncorrelated with the channel
        e = E[sl].reshape(-1)
        assert abs(np.mean(e)) < 4 * np.sqrt(np.mean(np.abs(e) ** 2) / e.size)
        assert abs(np.mean(e.real ** 2) / np.mean(e.imag ** 2) - 1) < 0.05
        c = np.vdot(Ht[sl].reshape(-1), e) / np.sqrt(np.vdot(e, e).real * np.vdot(Ht[sl], Ht[sl]).real)
        assert abs(c) < 0.02
    np.testing.assert_array_equal(b.nmse_db, np.repeat(pts, 256))
    s = b.subset([3, 300])
    np.testing.assert_array_equal(s.nmse_db, [-25.0, -15.0])


@pytest.mark.parametrize("name,shape", [("rayleigh_16x16_16qam", (16, 16, 16)),
                                        ("rayleigh_24x24_16qam", (24, 24, 16)),
                                        ("kronecker_16x16_16qam", (16, 16, 16)),
                                        ("csi_16x16_16qam", (16, 16, 16))])
def test_paper_workloads_materialise(name, shape):
    b, w = bench.load_batch(0.01, 0, name)
    assert b.n_channels >= 4
    assert set(b.nt.tolist()) == {shape[0]} and set(b.nr.tolist()) == {shape[1]}
    assert set(b.qam.tolist()) == {shape[2]}
    assert w["chains"] == 128 and w["iterations"] == 100


def test_ber_grouped_by_nmse():
    b = workload.csi_batch(2, 2, 4, 10.0, [-20.0, -10.0], 3, 5)
    nbits = int(b.tx_bits.size)
    llr = np.where(b.tx_bits == 0, 1.0, -1.0).astype(np.float32)
    llr[0] = -llr[0]                                   # one error in the first NMSE group
    idx = np.zeros(int(b.nt.sum()), np.int8)
    ber = bench.ber_of(b, llr, idx)
    assert list(ber) == ["nmse-20", "nmse-10"]
    assert ber["nmse-20"]["ber_llr"] == 1 / (nbits // 2) and ber["nmse-10"]["ber_llr"] == 0.0
