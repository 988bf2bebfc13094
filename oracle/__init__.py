"""FP64 CPU oracle for the DMALA MIMO detector -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It wraps ``dmala_oracle.c`` (plain C, FP64, the paper's definitions written out)
through ctypes and shares no code with the CUDA library: the two meet only through the seeded
inputs of ``workload``.

Parity status of each oracle function (what pins it is listed in ``tests/test_oracle_pins.py``):
every function is pinned except ``transition_matrix``'s use for the convergence rate of the
paper's one printed 2x2 example (r = 0.657, Sec. III-B): that channel is not printed, so that
single number is "parity unpinned"; the matrix itself is pinned by row sums, detailed balance
and stationarity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmala_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, portable flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Problem(ctypes.Structure):
    """Mirror of ``oracle_problem``: one real-valued DMALA target and proposal."""
    _fields_ = [
        ("M", ctypes.c_int), ("N", ctypes.c_int), ("L", ctypes.c_int),
        ("H", _dp), ("y", _dp), ("P", _dp),
        ("sigma2", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
        ("tau", ctypes.c_double), ("dmin", ctypes.c_double),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [("log_a", ctypes.c_double), ("log_u", ctypes.c_double),
                ("cat_margin", ctypes.c_double), ("f_new", ctypes.c_double),
                ("accepted", ctypes.c_int)]


class DetectCfg(ctypes.Structure):
    _fields_ = [("preconditioned", ctypes.c_int), ("alpha_scale", ctypes.c_double),
                ("tau", ctypes.c_double), ("chains", ctypes.c_int),
                ("iterations", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("channel", ctypes.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            l.oracle_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            l.oracle_uniform.restype = ctypes.c_double
            l.oracle_uniform.argtypes = [ctypes.c_uint32]
            l.oracle_real_model.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            l.oracle_dmin.restype = ctypes.c_double
            l.oracle_dmin.argtypes = [ctypes.c_int]
            l.oracle_f.restype = ctypes.c_double
            l.oracle_f.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
            l.oracle_grad_f.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        _dp, _dp]
            l.oracle_preconditioner.restype = ctypes.c_int
            l.oracle_preconditioner.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
            pp = ctypes.POINTER(Problem)
            l.oracle_log_q.restype = ctypes.c_double
            l.oracle_log_q.argtypes = [pp, _ip, _ip]
            l.oracle_log_accept.restype = ctypes.c_double
            l.oracle_log_accept.argtypes = [pp, _ip, _ip]
            l.oracle_init_state.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, _ip]
            l.oracle_step.restype = ctypes.c_int
            l.oracle_step.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, _ip, ctypes.POINTER(StepInfo)]
            l.oracle_step_chains.restype = None
            l.oracle_step_chains.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_int, ctypes.c_uint32, _ip,
                                             ctypes.POINTER(StepInfo)]
            l.oracle_mix_log_q.restype = ctypes.c_double
            l.oracle_mix_log_q.argtypes = [pp, ctypes.c_double, _ip, _dp, _ip]
            l.oracle_mix_propose.restype = ctypes.c_double
            l.oracle_mix_propose.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_double, _ip, _dp, _ip]
            l.oracle_mix_accept.restype = ctypes.c_int
            l.oracle_mix_accept.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_double, _ip, _ip, _dp, _dp,
                                            ctypes.c_double, ctypes.POINTER(StepInfo)]
            l.oracle_init_state_learned.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32,
                                                    ctypes.c_uint32, _dp, _ip]
            l.oracle_run_chain.restype = ctypes.c_int
            l.oracle_run_chain.argtypes = [pp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint32, ctypes.c_int, _ip, _dp, _ip, _dp]
            l.oracle_llr_is.argtypes = [pp, ctypes.c_int, _ip, _dp]
            l.oracle_all_f.argtypes = [pp, _dp]
            l.oracle_exact_llr.argtypes = [pp, _dp]
            l.oracle_transition_matrix.argtypes = [pp, _dp]
            l.oracle_llr_list.argtypes = [pp, ctypes.c_int, _ip, ctypes.c_double, _dp]
            l.oracle_detect.restype = ctypes.c_int
            l.oracle_detect.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                        ctypes.c_double, ctypes.POINTER(DetectCfg), _ip, _dp, _ip,
                                        _dp, _dp, ctypes.POINTER(ctypes.c_long)]
            l.oracle_problem_size.restype = ctypes.c_int
            if l.oracle_problem_size() != ctypes.sizeof(Problem):
                raise RuntimeError("oracle_problem layout mismatch")
            _lib = l
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    return a.ctypes.data_as(_ip)


# --------------------------------------------------------------------------------------------
# Thin wrappers
# --------------------------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(word: int) -> float:
    return lib().oracle_uniform(int(word) & 0xFFFFFFFF)


def dmin(qc: int) -> float:
    return lib().oracle_dmin(int(qc))


def real_model(H: np.ndarray, y: np.ndarray):
    """Stacked real-valued model of a complex (Nr x Nt) channel: (H_r [2Nr,2Nt], y_r [2Nr])."""
    nr, nt = H.shape
    Hc = np.ascontiguousarray(np.asarray(H, np.complex128).T).view(np.float64).reshape(-1).copy()
    yc = np.ascontiguousarray(np.asarray(y, np.complex128)).view(np.float64).copy()
    Hr = np.zeros((2 * nr, 2 * nt))
    yr = np.zeros(2 * nr)
    lib().oracle_real_model(nr, nt, _d(Hc), _d(yc), _d(Hr), _d(yr))
    return Hr, yr


def f_value(Hr: np.ndarray, yr: np.ndarray, sigma2: float, x: np.ndarray) -> float:
    Hr = np.ascontiguousarray(Hr, np.float64)
    yr = np.ascontiguousarray(yr, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    return lib().oracle_f(_d(Hr), _d(yr), Hr.shape[0], Hr.shape[1], float(sigma2), _d(x))


def grad_f(Hr: np.ndarray, yr: np.ndarray, sigma2: float, x: np.ndarray) -> np.ndarray:
    Hr = np.ascontiguousarray(Hr, np.float64)
    yr = np.ascontiguousarray(yr, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    g = np.zeros(Hr.shape[1])
    lib().oracle_grad_f(_d(Hr), _d(yr), Hr.shape[0], Hr.shape[1], float(sigma2), _d(x), _d(g))
    return g


def preconditioner(Hr: np.ndarray, gamma: float) -> np.ndarray:
    Hr = np.ascontiguousarray(Hr, np.float64)
    N = Hr.shape[1]
    P = np.zeros((N, N))
    if lib().oracle_preconditioner(_d(Hr), Hr.shape[0], N, float(gamma), _d(P)) != 0:
        raise np.linalg.LinAlgError("singular")
    return P


class Target:
    """A DMALA problem (real-valued H, y; proposal parameters) held alive for the C side."""

    def __init__(self, Hr, yr, sigma2, L, dmin_, *, alpha, beta=1.0, tau=1.0, P=None):
        self.Hr = np.ascontiguousarray(Hr, np.float64)
        self.yr = np.ascontiguousarray(yr, np.float64)
        self.P = None if P is None else np.ascontiguousarray(P, np.float64)
        self.M, self.N = self.Hr.shape
        self.L = int(L)
        self.dmin = float(dmin_)
        self.sigma2 = float(sigma2)
        self.s = Problem(self.M, self.N, self.L, _d(self.Hr), _d(self.yr),
                         _d(self.P) if self.P is not None else _dp(),
                         self.sigma2, float(alpha), float(beta), float(tau), self.dmin)

    @classmethod
    def from_channel(cls, H, y, sigma2, qam, *, preconditioned=True, alpha_scale=1.0, tau=2.0):
        """Paper defaults (Sec. IV-A): alpha = sigma^2, beta = dmin^2/sigma^2,
        gamma = sigma^2/(2 dmin^2) for the preconditioned proposal; beta = 1, no P otherwise."""
        Hr, yr = real_model(H, y)
        L = int(round(np.sqrt(qam)))
        d = dmin(qam)
        P, beta = None, 1.0
        if preconditioned:
            P = preconditioner(Hr, sigma2 / (2.0 * d * d))
            beta = d * d / sigma2
        t = cls(Hr, yr, sigma2, L, d, alpha=alpha_scale * sigma2, beta=beta, tau=tau, P=P)
        t.Hc, t.yc = np.asarray(H), np.asarray(y)
        return t

    @property
    def ptr(self):
        return ctypes.byref(self.s)

    def values(self, k) -> np.ndarray:
        return (2 * np.asarray(k, np.float64) - self.L + 1) * self.dmin

    def log_q(self, k_from, k_to) -> float:
        a = np.ascontiguousarray(k_from, np.int32)
        b = np.ascontiguousarray(k_to, np.int32)
        return lib().oracle_log_q(self.ptr, _i(a), _i(b))

    def log_accept(self, k, kp) -> float:
        a = np.ascontiguousarray(k, np.int32)
        b = np.ascontiguousarray(kp, np.int32)
        return lib().oracle_log_accept(self.ptr, _i(a), _i(b))

    def init_state(self, seed, channel, chain) -> np.ndarray:
        k = np.zeros(self.N, np.int32)
        lib().oracle_init_state(self.ptr, int(seed), int(channel), int(chain), _i(k))
        return k

    def step(self, seed, channel, chain, t, k):
        """One transition numbered t from state k: (new state, StepInfo)."""
        kk = np.ascontiguousarray(k, np.int32).copy()
        info = StepInfo()
        lib().oracle_step(self.ptr, int(seed), int(channel), int(chain), int(t), _i(kk),
                          ctypes.byref(info))
        return kk, info

    def step_chains(self, seed, channel, t, states, chain0=0):
        """Transition t of chains chain0.. from states [chains, N]: (new states, infos dict)."""
        st = np.ascontiguousarray(states, np.int32).copy()
        n = st.shape[0]
        infos = (StepInfo * n)()
        lib().oracle_step_chains(self.ptr, int(seed), int(channel), int(chain0), n, int(t),
                                 _i(st), infos)
        info = dict(log_a=np.array([x.log_a for x in infos]), log_u=np.array([x.log_u for x in infos]),
                    cat_margin=np.array([x.cat_margin for x in infos]),
                    accepted=np.array([x.accepted for x in infos], bool))
        return st, info

    def nn_logp(self, params, k=None, quant=False) -> np.ndarray:
        """Network log-probabilities [Nt, Qc] at level indices k (None: x = 0) for a channel
        built by from_channel."""
        from oracle import mlp
        F = mlp.features(self.Hc, self.yc, self.sigma2, self.L * self.L, k)
        return mlp.log_softmax(mlp.forward(params, F, self.L * self.L, quant)[0])

    def mix_log_q(self, lam, k_from, nnlogp_from, k_to) -> float:
        return lib().oracle_mix_log_q(self.ptr, float(lam), _i(np.ascontiguousarray(k_from, np.int32)),
                                      _d(np.ascontiguousarray(nnlogp_from, np.float64)),
                                      _i(np.ascontiguousarray(k_to, np.int32)))

    def mix_step(self, seed, channel, chain, t, k, lam, params=None, nn=None, quant=False):
        """Learned mixture move numbered t from level indices k (see oracle_mix_propose). The
        network is params (evaluated by oracle.mlp) or a callable nn(k) -> [Nt, Qc] log-probs."""
        nnf = nn if nn is not None else (lambda kk: self.nn_logp(params, kk, quant))
        kk = np.ascontiguousarray(k, np.int32).copy()
        lx = np.ascontiguousarray(nnf(kk), np.float64)
        kp = np.zeros(self.N, np.int32)
        margin = lib().oracle_mix_propose(self.ptr, int(seed), int(channel), int(chain), int(t),
                                          float(lam), _i(kk), _d(lx), _i(kp))
        lxp = np.ascontiguousarray(nnf(kp), np.float64)
        info = StepInfo()
        lib().oracle_mix_accept(self.ptr, int(seed), int(channel), int(chain), int(t), float(lam),
                                _i(kk), _i(kp), _d(lx), _d(lxp), margin, ctypes.byref(info))
        return kk, info

    def init_state_learned(self, seed, channel, chain, nnlogp0) -> np.ndarray:
        k = np.zeros(self.N, np.int32)
        lp = np.ascontiguousarray(nnlogp0, np.float64)
        lib().oracle_init_state_learned(self.ptr, int(seed), int(channel), int(chain), _d(lp), _i(k))
        return k

    def run_chain(self, seed, channel, chain, t_offset, iters, k):
        kk = np.ascontiguousarray(k, np.int32).copy()
        bf = ctypes.c_double(-np.inf)
        bk = np.zeros(self.N, np.int32)
        gap = ctypes.c_double(0.0)
        acc = lib().oracle_run_chain(self.ptr, int(seed), int(channel), int(chain),
                                     int(t_offset), int(iters), _i(kk), ctypes.byref(bf), _i(bk),
                                     ctypes.byref(gap))
        return kk, dict(accepts=acc, best_f=bf.value, best_k=bk, min_gap=gap.value)

    def llr_is(self, samples) -> np.ndarray:
        s = np.ascontiguousarray(samples, np.int32)
        B = int(np.log2(self.L))
        out = np.zeros(self.N * B)
        lib().oracle_llr_is(self.ptr, s.shape[0], _i(s), _d(out))
        return out

    def llr_list(self, samples, clip: float) -> np.ndarray:
        """List-based LLR of Eq. (31) over the distinct samples, clipped to [-clip, clip]."""
        s = np.ascontiguousarray(samples, np.int32)
        B = int(np.log2(self.L))
        out = np.zeros(self.N * B)
        lib().oracle_llr_list(self.ptr, s.shape[0], _i(s), float(clip), _d(out))
        return out

    def n_states(self) -> int:
        return self.L ** self.N

    def all_f(self) -> np.ndarray:
        out = np.zeros(self.n_states())
        lib().oracle_all_f(self.ptr, _d(out))
        return out

    def exact_llr(self) -> np.ndarray:
        B = int(np.log2(self.L))
        out = np.zeros(self.N * B)
        lib().oracle_exact_llr(self.ptr, _d(out))
        return out

    def transition_matrix(self) -> np.ndarray:
        S = self.n_states()
        if S > 4096:
            raise ValueError("state space too large for a dense transition matrix")
        out = np.zeros((S, S))
        lib().oracle_transition_matrix(self.ptr, _d(out))
        return out

    def state_levels(self, idx: int) -> np.ndarray:
        k = np.zeros(self.N, np.int32)
        for n in range(self.N - 1, -1, -1):
            k[n] = idx % self.L
            idx //= self.L
        return k

    def state_index(self, k) -> int:
        idx = 0
        for v in np.asarray(k):
            idx = idx * self.L + int(v)
        return idx


# --------------------------------------------------------------------------------------------
# Whole detections
# --------------------------------------------------------------------------------------------
def detect(H, y, sigma2, qam, *, chains, iterations, seed=0, channel=0, preconditioned=True,
           alpha_scale=1.0, tau=2.0) -> dict:
    """Algorithm 2 around Algorithm 1 for one channel, FP64. Returns final states [chains, 2Nt]
    levels, final_f [chains], best_state [2Nt], best_f, llr [Nt log2 Qc], accepts."""
    nr, nt = H.shape
    N = 2 * nt
    Hc = np.ascontiguousarray(np.asarray(H, np.complex128).T).view(np.float64).reshape(-1).copy()
    yc = np.ascontiguousarray(np.asarray(y, np.complex128)).view(np.float64).copy()
    cfg = DetectCfg(int(preconditioned), float(alpha_scale), float(tau), int(chains),
                    int(iterations), int(seed), int(channel))
    fs = np.zeros((chains, N), np.int32)
    ff = np.zeros(chains)
    bs = np.zeros(N, np.int32)
    bf = ctypes.c_double(0.0)
    nb = N * int(np.log2(int(round(np.sqrt(qam)))))
    llr = np.zeros(nb)
    acc = ctypes.c_long(0)
    rc = lib().oracle_detect(nr, nt, int(qam), _d(Hc), _d(yc), float(sigma2), ctypes.byref(cfg),
                             _i(fs), _d(ff), _i(bs), ctypes.byref(bf), _d(llr), ctypes.byref(acc))
    if rc != 0:
        raise ValueError("oracle_detect rejected its input")
    return dict(final_states=fs, final_f=ff, best_state=bs, best_f=bf.value, llr=llr,
                accepts=acc.value)


def detect_batch(batch, *, chains, iterations, seed=0, preconditioned=True, alpha_scale=1.0,
                 tau=2.0, channels=None, threads: Optional[int] = None):
    """``detect`` over channels of a ``workload.Batch`` on a thread pool (the C call releases
    the GIL). The channel id in the Philox counter is the channel's index in the batch."""
    idx = list(range(batch.n_channels)) if channels is None else list(channels)
    threads = threads or os.cpu_count() or 1

    def one(b):
        H, y, s2 = batch.channel(b)
        return detect(H, y, s2, int(batch.qam[b]), chains=chains, iterations=iterations,
                      seed=seed, channel=b, preconditioned=preconditioned,
                      alpha_scale=alpha_scale, tau=tau)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, idx))


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
