"""Where the posterior is enumerable, the sampler detects like the exact MAP detector: on 4x4
16-QAM Rayleigh at 20 dB (150 channels, the paper's 32 chains x 100 transitions, IS-LLR), the
oracle's DMALA makes the same number of bit errors as sign(exact LLR) (Eq. (4)) to within two
bits, and both are far below a linear MMSE detector. This pins the whole oracle chain (proposal,
MH, tempering, IS-LLR) against the exact answer, not against itself."""
import numpy as np

import oracle
import workload


def _mmse_bits(b, ch):
    Hc, y, s2 = b.channel(ch)
    nt, qam = Hc.shape[1], int(b.qam[ch])
    L, d = int(np.sqrt(qam)), np.sqrt(3.0 / (2.0 * (qam - 1)))
    xh = np.linalg.solve(Hc.conj().T @ Hc + s2 * np.eye(nt), Hc.conj().T @ y)
    nb = int(np.log2(L))

    def bits(v):
        k = np.clip(np.round((v / d + (L - 1)) / 2), 0, L - 1).astype(int)
        return ((k ^ (k >> 1))[:, None] >> np.arange(nb - 1, -1, -1)) & 1

    return np.concatenate([bits(xh.real), bits(xh.imag)], axis=1).reshape(-1)


def test_dmala_detects_like_exact_map_on_4x4_16qam():
    b = workload.rayleigh_batch(4, 4, 16, [20.0], 150, 1001)
    res = oracle.detect_batch(b, chains=32, iterations=100, seed=0)
    llr = np.concatenate([r["llr"] for r in res])
    e_dmala = int(((llr < 0).astype(np.uint8) != b.tx_bits).sum())
    e_map = e_mmse = 0
    for ch in range(b.n_channels):
        Hc, y, s2 = b.channel(ch)
        t = oracle.Target.from_channel(Hc, y, s2, 16, preconditioned=True, tau=2.0)
        tb = b.tx_bits[b.bit_off[ch]:b.bit_off[ch] + 16]
        e_map += int(((t.exact_llr() < 0).astype(np.uint8) != tb).sum())
        e_mmse += int((_mmse_bits(b, ch) != tb).sum())
    assert abs(e_dmala - e_map) <= 2, (e_dmala, e_map)
    assert e_mmse > 4 * max(e_map, 1), (e_mmse, e_map)
