"""Seeded synthetic MIMO workloads: the transmitter and the channel, never the detector.

This module is shared by the CPU oracle (``oracle/``), the CUDA path's tests and ``bench.py``.
It holds only the system model's random draws (paper Sec. II-A, Eq. (1); Sec. IV-A and IV-D for
the channel models), none of the detector's arithmetic:

* transmitted symbols: each complex antenna carries a square Qc-QAM point whose in-phase and
  quadrature parts are independent PAM levels ``k in {0..L-1}`` (``L = sqrt(Qc)``), drawn
  uniformly, i.e. uniform bits under a per-dimension binary-reflected Gray label
  ``k ^ (k >> 1)``; the transmitted bits per antenna are the in-phase label (MSB first) followed
  by the quadrature label; unit average symbol energy;
* channel: iid Rayleigh with entries CN(0, 1/Nr), or Kronecker ``R_r^{1/2} G R_t^{1/2}`` with the
  exponential correlation ``[R]_ij = rho^|i-j|`` (Sec. IV-D, Eq. (37)), square roots by eigendecomposition;
* noise: CN(0, sigma^2) per receive antenna with ``sigma^2 = Nt / (Nr * 10^(SNR/10))``, which is
  the paper's SNR definition ``E||Hx||^2 / E||n||^2`` (footnote of Sec. III-B) for these channels;
* imperfect CSI (Sec. IV-F): the receiver's estimate ``H^ = H + E`` with E entries
  CN(0, sigma_e^2); for CN(0, 1/Nr) channels the NMSE ``E||E||_F^2 / E||H||_F^2`` equals
  ``Nr sigma_e^2``. y is generated with the true H; the batch carries H^, the detector's view.

H, y and sigma^2 are rounded to single precision once, here, so that every consumer (the FP64
oracle and the FP32 device path) detects exactly the same problem.
"""
from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Batch", "generate", "rayleigh_batch", "kronecker_batch", "uneven_batch", "csi_batch",
    "WORKLOADS", "workload",
]


@dataclasses.dataclass
class Batch:
    """A packed batch of channel realisations.

    Complex arrays are packed back to back; ``H_off[b]`` / ``y_off[b]`` are offsets in complex
    elements. ``H`` of channel b is stored column-major (Nr x Nt): element (r, c) sits at
    ``H_off[b] + c * Nr + r``.
    """

    nt: np.ndarray          # int32 [B]
    nr: np.ndarray          # int32 [B]
    qam: np.ndarray         # int32 [B] 4 | 16 | 64
    snr_db: np.ndarray      # float64 [B]
    sigma2: np.ndarray      # float32 [B] complex noise variance
    H: np.ndarray           # complex64 packed
    H_off: np.ndarray       # int64 [B]
    y: np.ndarray           # complex64 packed
    y_off: np.ndarray       # int64 [B]
    tx_levels: np.ndarray   # int8 packed, per channel 2*Nt levels: [Re dims; Im dims]
    lev_off: np.ndarray     # int64 [B]
    tx_bits: np.ndarray     # uint8 packed, per channel Nt*log2(Qc) bits
    bit_off: np.ndarray     # int64 [B]
    nmse_db: Optional[np.ndarray] = None   # float64 [B] NMSE of the channel estimate (imperfect CSI)

    @property
    def n_channels(self) -> int:
        return int(self.nt.shape[0])

    def channel(self, b: int):
        """(H [Nr,Nt] complex128, y [Nr] complex128, sigma2 float) of channel b."""
        nt, nr = int(self.nt[b]), int(self.nr[b])
        h = self.H[self.H_off[b]: self.H_off[b] + nt * nr].astype(np.complex128)
        H = h.reshape(nt, nr).T.copy()
        y = self.y[self.y_off[b]: self.y_off[b] + nr].astype(np.complex128)
        return H, y, float(self.sigma2[b])

    def levels(self, b: int) -> np.ndarray:
        return self.tx_levels[self.lev_off[b]: self.lev_off[b] + 2 * int(self.nt[b])]

    def bits(self, b: int) -> np.ndarray:
        nb = int(self.nt[b]) * int(np.log2(self.qam[b]))
        return self.tx_bits[self.bit_off[b]: self.bit_off[b] + nb]

    def subset(self, idx: Sequence[int]) -> "Batch":
        """A new packed batch holding the channels ``idx`` in that order."""
        parts = [(self.channel(int(b)), int(b)) for b in idx]
        out = _pack(
            [self.nt[b] for _, b in parts], [self.nr[b] for _, b in parts],
            [self.qam[b] for _, b in parts], [self.snr_db[b] for _, b in parts],
            [self.sigma2[b] for _, b in parts], [p[0] for p, _ in parts],
            [p[1] for p, _ in parts], [self.levels(b) for _, b in parts],
        )
        if self.nmse_db is not None:
            out.nmse_db = np.asarray([self.nmse_db[b] for _, b in parts], np.float64)
        return out


def _gray_bits(levels: np.ndarray, nbits: int) -> np.ndarray:
    g = levels ^ (levels >> 1)
    return ((g[..., None] >> np.arange(nbits - 1, -1, -1)) & 1).astype(np.uint8)


def _sqrtm_psd(R: np.ndarray) -> np.ndarray:
    w, V = np.linalg.eigh(R)
    return (V * np.sqrt(np.clip(w, 0.0, None))) @ V.T


def _exp_corr(n: int, rho: float) -> np.ndarray:
    i = np.arange(n)
    return rho ** np.abs(i[:, None] - i[None, :])


def _draw_group(rng: np.random.Generator, count: int, nt: int, nr: int, qam: int,
                snr_db: np.ndarray, rho: Optional[float]):
    L = int(round(np.sqrt(qam)))
    if L * L != qam or L not in (2, 4, 8):
        raise ValueError(f"unsupported QAM order {qam}")
    dmin = np.sqrt(3.0 / (2.0 * (qam - 1)))
    lev = rng.integers(0, L, size=(count, 2 * nt))                 # [Re; Im] per antenna
    amp = (2 * lev - (L - 1)) * dmin
    x = amp[:, :nt] + 1j * amp[:, nt:]
    G = (rng.standard_normal((count, nr, nt)) + 1j * rng.standard_normal((count, nr, nt)))
    G *= np.sqrt(0.5 / nr)
    if rho is not None and rho != 0.0:
        Rr = _sqrtm_psd(_exp_corr(nr, rho))
        Rt = _sqrtm_psd(_exp_corr(nt, rho))
        G = Rr[None] @ G @ Rt[None]
    H = G.astype(np.complex64)
    sigma2 = (nt / (nr * 10.0 ** (snr_db / 10.0))).astype(np.float32)
    n = (rng.standard_normal((count, nr)) + 1j * rng.standard_normal((count, nr)))
    n *= np.sqrt(sigma2.astype(np.float64) / 2.0)[:, None]
    y = (np.einsum("brt,bt->br", H.astype(np.complex128), x) + n).astype(np.complex64)
    return H, y, sigma2, lev.astype(np.int8)


def _pack(nt, nr, qam, snr_db, sigma2, Hs, ys, levs) -> Batch:
    nt = np.asarray(nt, np.int32)
    nr = np.asarray(nr, np.int32)
    qam = np.asarray(qam, np.int32)
    B = nt.shape[0]
    H_off = np.zeros(B, np.int64)
    y_off = np.zeros(B, np.int64)
    lev_off = np.zeros(B, np.int64)
    bit_off = np.zeros(B, np.int64)
    if B:
        H_off[1:] = np.cumsum((nt * nr).astype(np.int64))[:-1]
        y_off[1:] = np.cumsum(nr.astype(np.int64))[:-1]
        lev_off[1:] = np.cumsum(2 * nt.astype(np.int64))[:-1]
        nbits = nt.astype(np.int64) * np.log2(qam).astype(np.int64)
        bit_off[1:] = np.cumsum(nbits)[:-1]
    Hp = np.concatenate([np.asarray(h, np.complex64).T.reshape(-1) for h in Hs]) if B else \
        np.zeros(0, np.complex64)
    yp = np.concatenate([np.asarray(v, np.complex64) for v in ys]) if B else np.zeros(0, np.complex64)
    lp = np.concatenate([np.asarray(v, np.int8) for v in levs]) if B else np.zeros(0, np.int8)
    bits = []
    for b in range(B):
        L = int(round(np.sqrt(qam[b])))
        nb = int(np.log2(L))
        lv = np.asarray(levs[b], np.int64)
        t = int(nt[b])
        gi = _gray_bits(lv[:t], nb)
        gq = _gray_bits(lv[t:], nb)
        bits.append(np.concatenate([gi, gq], axis=1).reshape(-1))
    bp = np.concatenate(bits).astype(np.uint8) if B else np.zeros(0, np.uint8)
    return Batch(nt, nr, qam, np.asarray(snr_db, np.float64), np.asarray(sigma2, np.float32),
                 Hp, H_off, yp, y_off, lp, lev_off, bp, bit_off)


def generate(shapes: Sequence[tuple], seed: int, rho: Optional[float] = None) -> Batch:
    """Draw one channel per entry of ``shapes`` = [(nt, nr, qam, snr_db), ...].

    Channels with equal (nt, nr, qam) are drawn together (vectorised); the draw order is fixed
    by the sorted set of shapes, so the output depends only on ``shapes`` and ``seed``.
    """
    rng = np.random.default_rng(seed)
    shapes = [(int(a), int(b), int(c), float(d)) for a, b, c, d in shapes]
    B = len(shapes)
    out_H = [None] * B
    out_y = [None] * B
    out_s = np.zeros(B, np.float32)
    out_l = [None] * B
    groups = {}
    for i, (nt, nr, qam, _) in enumerate(shapes):
        groups.setdefault((nt, nr, qam), []).append(i)
    for key in sorted(groups):
        idx = groups[key]
        snr = np.array([shapes[i][3] for i in idx])
        H, y, s2, lev = _draw_group(rng, len(idx), key[0], key[1], key[2], snr, rho)
        for j, i in enumerate(idx):
            out_H[i], out_y[i], out_s[i], out_l[i] = H[j], y[j], s2[j], lev[j]
    return _pack([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes],
                 [s[3] for s in shapes], out_s, out_H, out_y, out_l)


def rayleigh_batch(nt: int, nr: int, qam: int, snr_db: Sequence[float], per_snr: int,
                   seed: int) -> Batch:
    """``per_snr`` iid Rayleigh channels at each SNR point, SNR-major order."""
    shapes = [(nt, nr, qam, s) for s in snr_db for _ in range(per_snr)]
    return generate(shapes, seed)


def kronecker_batch(nt: int, nr: int, qam: int, snr_db: Sequence[float], total: int,
                    rho: float, seed: int) -> Batch:
    """``total`` Kronecker-correlated channels with the SNR points assigned in equal blocks."""
    pts = list(snr_db)
    shapes = [(nt, nr, qam, pts[(i * len(pts)) // total]) for i in range(total)]
    return generate(shapes, seed, rho=rho)


def csi_batch(nt: int, nr: int, qam: int, snr_db: float, nmse_db: Sequence[float],
              per_point: int, seed: int) -> Batch:
    """``per_point`` Rayleigh channels at each NMSE point (point-major order) seen through an
    imperfect estimate H^ = H + E, E entries CN(0, 10^(NMSE/10) / Nr). The true channels, symbols
    and noise are those of ``generate`` with the same seed; E comes from its own stream."""
    pts = [float(v) for v in nmse_db]
    b = generate([(nt, nr, qam, snr_db)] * (per_point * len(pts)), seed)
    nm = np.repeat(np.asarray(pts, np.float64), per_point)
    rng = np.random.default_rng(seed + 104729)
    n = nt * nr
    E = rng.standard_normal((b.n_channels, n, 2))
    se = np.sqrt(10.0 ** (nm / 10.0) / nr / 2.0)
    E = (E[..., 0] + 1j * E[..., 1]) * se[:, None]
    Hh = b.H.astype(np.complex128).reshape(b.n_channels, n) + E
    return dataclasses.replace(b, H=Hh.astype(np.complex64).reshape(-1), nmse_db=nm)


def uneven_batch(count: int, seed: int, nts=(8, 16, 32, 64), qams=(4, 16, 64),
                 snr_range=(10.0, 30.0)) -> Batch:
    """Mixed-shape batch: Nt ~ U(nts), Nr ~ U{Nt, 2Nt}, Qc ~ U(qams), SNR ~ U[snr_range]."""
    rng = np.random.default_rng(seed + 7919)
    nt = rng.choice(np.asarray(nts), size=count)
    nr = nt * rng.integers(1, 3, size=count)
    qam = rng.choice(np.asarray(qams), size=count)
    snr = rng.uniform(snr_range[0], snr_range[1], size=count)
    return generate(list(zip(nt, nr, qam, snr)), seed)


# Named workloads (sizes of the paper's and the benchmark's experiments). Each entry gives the
# batch recipe plus the sampler settings used with it.
WORKLOADS = {
    # 4x4 16-QAM Rayleigh at 12 dB, 1000 channels, 32 chains x 100 iterations (65 536 states:
    # exact posterior and MAP enumerable).
    "rayleigh_4x4_16qam": dict(kind="rayleigh", nt=4, nr=4, qam=16, snr_db=[12.0], per_snr=1000,
                               chains=32, iterations=100, seed=1001),
    # 32x32 64-QAM Rayleigh, SNR 20..32 dB step 2, 4096 channels per point, 64 x 200.
    "rayleigh_32x32_64qam": dict(kind="rayleigh", nt=32, nr=32, qam=64,
                                 snr_db=[20.0, 22.0, 24.0, 26.0, 28.0, 30.0, 32.0],
                                 per_snr=4096, chains=64, iterations=200, seed=1002),
    # 16384 channels of mixed Nt/Nr/QAM, SNR U[10,30] dB, 128 x 150.
    "uneven_16384": dict(kind="uneven", count=16384, chains=128, iterations=150, seed=1003),
    # 128x128 64-QAM Kronecker rho=0.5, SNR 26..34 dB, 1024 channels, 256 x 300.
    "kronecker_128x128_64qam": dict(kind="kronecker", nt=128, nr=128, qam=64,
                                    snr_db=[26.0, 28.0, 30.0, 32.0, 34.0], total=1024, rho=0.5,
                                    chains=256, iterations=300, seed=1004),
    # Learned proposal: evaluation on 64x64 16-QAM Rayleigh, SNR U[12,24] dB, 8192 channels,
    # 64 chains, the plain sampler's reference at 40 iterations; the network is trained on plain-
    # sampler samples of 32x32 16-QAM Rayleigh at SNR U[12,24] dB (512 channels x 16 chains,
    # features at 7 points of each chain: ~1.8M rows).
    # Convergence diagnostics of Figs. 2-3 (Sec. III-B): 2x2 QPSK Rayleigh (16 states), 100
    # channel realisations at each of 4, 6, 8, 10 dB; exact transition kernels of both proposals,
    # their spectra and total-variation curves over 50 transitions.
    "convergence_2x2_qpsk": dict(kind="convergence", nt=2, nr=2, qam=4,
                                 snr_db=[4.0, 6.0, 8.0, 10.0], per_snr=100, chains=1,
                                 iterations=50, seed=1006),
    # Large MIMO of Figs. 7-8 (Sec. IV-C): 16x16 and 24x24 16-QAM Rayleigh, 128 chains, T = 100
    # (the paper's default, Sec. IV-A).
    "rayleigh_16x16_16qam": dict(kind="rayleigh", nt=16, nr=16, qam=16,
                                 snr_db=[10.0, 12.0, 14.0, 16.0, 18.0], per_snr=2048, chains=128,
                                 iterations=100, seed=1007),
    "rayleigh_24x24_16qam": dict(kind="rayleigh", nt=24, nr=24, qam=16,
                                 snr_db=[12.0, 14.0, 16.0, 18.0, 20.0], per_snr=1024, chains=128,
                                 iterations=100, seed=1008),
    # Correlated channels of Fig. 9 (Sec. IV-D): 16x16 16-QAM Kronecker, rho = 0.5.
    "kronecker_16x16_16qam": dict(kind="kronecker", nt=16, nr=16, qam=16,
                                  snr_db=[14.0, 16.0, 18.0, 20.0, 22.0], total=5120, rho=0.5,
                                  chains=128, iterations=100, seed=1009),
    # Imperfect CSI of Fig. 11 (Sec. IV-F): 16x16 16-QAM Rayleigh at 16.5 dB, channel-estimate
    # NMSE -30..-15 dB.
    "csi_16x16_16qam": dict(kind="csi", nt=16, nr=16, qam=16, snr_db=[16.5],
                            nmse_db=[-30.0, -25.0, -20.0, -15.0], per_point=1024, chains=128,
                            iterations=100, seed=1010),
    "learned_64x64_16qam": dict(kind="learned", nt=64, nr=64, qam=16, snr_range=(12.0, 24.0),
                                count=8192, chains=64, iterations=40, seed=1005,
                                checkpoints=[1, 2, 5, 10, 20, 40],
                                train=dict(nt=32, nr=32, channels=512, chains=16,
                                           feature_times=[0, 2, 5, 10, 20, 40], label_time=200,
                                           label="best", epochs=8, batch=4096, lr=1e-3)),
}


def workload(name: str, scale: float = 1.0) -> Batch:
    """Materialise a named workload; ``scale`` < 1 keeps that fraction of the channels."""
    w = WORKLOADS[name]
    if w["kind"] in ("rayleigh", "convergence"):
        n = max(1, int(round(w["per_snr"] * scale)))
        return rayleigh_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], n, w["seed"])
    if w["kind"] == "kronecker":
        n = max(1, int(round(w["total"] * scale)))
        return kronecker_batch(w["nt"], w["nr"], w["qam"], w["snr_db"], n, w["rho"], w["seed"])
    if w["kind"] == "uneven":
        n = max(1, int(round(w["count"] * scale)))
        return uneven_batch(n, w["seed"])
    if w["kind"] == "csi":
        n = max(1, int(round(w["per_point"] * scale)))
        return csi_batch(w["nt"], w["nr"], w["qam"], w["snr_db"][0], w["nmse_db"], n, w["seed"])
    if w["kind"] == "learned":
        n = max(1, int(round(w["count"] * scale)))
        return learned_eval_batch(w, n)
    raise KeyError(name)


def learned_eval_batch(w: dict, n: int, seed_offset: int = 0) -> Batch:
    """Evaluation channels of a learned-proposal workload (SNR uniform in its range)."""
    rng = np.random.default_rng(w["seed"] + seed_offset)
    snr = rng.uniform(w["snr_range"][0], w["snr_range"][1], n)
    return generate([(w["nt"], w["nr"], w["qam"], float(s)) for s in snr], w["seed"] + seed_offset)


def learned_train_batch(w: dict, seed_offset: int = 0) -> Batch:
    """Training channels of a learned-proposal workload."""
    t = w["train"]
    rng = np.random.default_rng(w["seed"] + 500 + seed_offset)
    snr = rng.uniform(w["snr_range"][0], w["snr_range"][1], t["channels"])
    return generate([(t["nt"], t["nr"], w["qam"], float(s)) for s in snr],
                    w["seed"] + 500 + seed_offset)
