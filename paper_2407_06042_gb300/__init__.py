"""GB300 (sm_103a) DMALA MIMO detector: Python binding of the C-ABI library ``libmcmcdet.so``.

The binding only marshals arguments: every step of the detection (Gram / matched filter,
preconditioner, chains, read-out) runs in the library's CUDA kernels. The functions below carry
the C names of ``include/mcmcdet.h``; :class:`Detector` is a convenience wrapper over them that
accepts torch tensors (device memory, ``host_io = 0``) or numpy / CPU tensors (host memory,
``host_io = 1``). Importing this package fails loudly when the library cannot be built or
loaded: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "Detector", "Config", "Stats", "lib", "load", "MCMC_PREC_FP64", "MCMC_PREC_FP32",
    "MCMC_PREC_MIXED", "MCMC_ENGINE_AUTO", "MCMC_ENGINE_SIMT", "MCMC_ENGINE_TC",
    "MCMC_ENGINE_GRAPH", "MCMC_ENGINE_NO_CLUSTER", "MCMC_ENGINE_TRACE", "MCMC_ENGINE_NO_PACK",
    "MCMC_ENGINE_NO_GRAPH", "MCMC_ENGINE_KERNEL_REFRESH", "McmcError", "Mlp",
    "ABI_FUNCTIONS", "ABI_FUNCTIONS_LEARNED", "ABI_FUNCTIONS_DIAG", "transition_diagnostics",
]

MCMC_PREC_FP64, MCMC_PREC_FP32, MCMC_PREC_MIXED = 0, 1, 2
MCMC_ENGINE_AUTO, MCMC_ENGINE_SIMT, MCMC_ENGINE_TC, MCMC_ENGINE_GRAPH = 0, 1, 2, 4
MCMC_ENGINE_NO_CLUSTER = 8
MCMC_ENGINE_TRACE = 16
MCMC_ENGINE_NO_PACK = 32
MCMC_ENGINE_NO_GRAPH = 64
MCMC_ENGINE_KERNEL_REFRESH = 128
_PREC = {"fp64": MCMC_PREC_FP64, "fp32": MCMC_PREC_FP32, "mixed": MCMC_PREC_MIXED}
STATUS = {0: "MCMC_OK", 1: "MCMC_EINVAL", 2: "MCMC_ENOMEM", 3: "MCMC_ECUDA", 4: "MCMC_ETIMEOUT",
          5: "MCMC_ENUMERIC", 6: "MCMC_ESTATE", 7: "MCMC_EUNSUPPORTED"}

# Every entry point of include/mcmcdet.h.
ABI_FUNCTIONS = [
    "mcmc_config_default", "mcmc_detect_create", "mcmc_detect_preprocess",
    "mcmc_detect_run_chains", "mcmc_detect_estimate", "mcmc_detect_get_chains",
    "mcmc_detect_set_chains", "mcmc_detect_synchronize", "mcmc_detect_destroy",
    "mcmc_status_string", "mcmc_detect_last_error", "mcmc_detect_kernel_launches",
    "mcmc_detect_noalloc", "mcmc_detect_llr_list", "mcmc_detect_get_tracked",
    "mcmc_detect_get_trace", "mcmc_detect_launch_groups", "mcmc_detect_run_kernel_ms",
]

# Every entry point of include/mcmcdet_learned.h.
ABI_FUNCTIONS_LEARNED = [
    "mcmc_mlp_param_count", "mcmc_mlp_create", "mcmc_mlp_destroy", "mcmc_mlp_last_error",
    "mcmc_mlp_set_params", "mcmc_mlp_get_params", "mcmc_mlp_forward", "mcmc_mlp_loss_grad",
    "mcmc_mlp_set_train_engine",
    "mcmc_mlp_train_step", "mcmc_detect_features", "mcmc_detect_set_model",
    "mcmc_detect_init_learned", "mcmc_detect_mix_step",
]


# Every entry point of include/mcmcdet_diag.h.
ABI_FUNCTIONS_DIAG = ["mcmc_diag_transition"]


class McmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    """Mirror of ``mcmc_config``."""
    _fields_ = [
        ("max_channels", ctypes.c_int32), ("max_nt", ctypes.c_int32), ("max_nr", ctypes.c_int32),
        ("chains", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("preconditioned", ctypes.c_int32), ("refresh_period", ctypes.c_int32),
        ("split_terms", ctypes.c_int32), ("engine", ctypes.c_int32), ("tile", ctypes.c_int32),
        ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
    ]


class Stats(ctypes.Structure):
    """Mirror of ``mcmc_stats``."""
    _fields_ = [("transitions", ctypes.c_int64), ("accepts", ctypes.c_int64),
                ("numeric_faults", ctypes.c_int32), ("near_tie_windows", ctypes.c_int32),
                ("refresh_drift", ctypes.c_double), ("near_ties", ctypes.c_int64 * 3),
                ("refresh_drift_rel", ctypes.c_double)]


_lib = None


def load(path: Optional[str] = None):
    """Load (building first if stale) the C-ABI library and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.build()
    l = ctypes.CDLL(p)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    l.mcmc_config_default.argtypes = [ctypes.POINTER(Config)]
    l.mcmc_config_default.restype = None
    l.mcmc_detect_create.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    l.mcmc_detect_create.restype = ctypes.c_int
    l.mcmc_detect_preprocess.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_float,
                                         ctypes.c_float, i32]
    l.mcmc_detect_preprocess.restype = ctypes.c_int
    l.mcmc_detect_run_chains.argtypes = [vp, i32, i64]
    l.mcmc_detect_run_chains.restype = ctypes.c_int
    l.mcmc_detect_estimate.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Stats), i32]
    l.mcmc_detect_estimate.restype = ctypes.c_int
    l.mcmc_detect_get_chains.argtypes = [vp, vp, vp, i32]
    l.mcmc_detect_llr_list.argtypes = [vp, vp, ctypes.c_float, i32]
    l.mcmc_detect_llr_list.restype = ctypes.c_int
    l.mcmc_detect_get_chains.restype = ctypes.c_int
    l.mcmc_detect_get_tracked.argtypes = [vp, vp, vp, i32]
    l.mcmc_detect_get_tracked.restype = ctypes.c_int
    l.mcmc_detect_launch_groups.argtypes = [vp, vp, i32]
    l.mcmc_detect_launch_groups.restype = ctypes.c_int32
    l.mcmc_detect_run_kernel_ms.argtypes = [vp, i32, vp]
    l.mcmc_detect_run_kernel_ms.restype = ctypes.c_int
    l.mcmc_detect_get_trace.argtypes = [vp, vp, i32]
    l.mcmc_detect_get_trace.restype = ctypes.c_int
    l.mcmc_detect_set_chains.argtypes = [vp, vp, i32]
    l.mcmc_detect_set_chains.restype = ctypes.c_int
    l.mcmc_detect_synchronize.argtypes = [vp]
    l.mcmc_detect_synchronize.restype = ctypes.c_int
    l.mcmc_detect_destroy.argtypes = [vp]
    l.mcmc_detect_destroy.restype = ctypes.c_int
    l.mcmc_status_string.argtypes = [ctypes.c_int]
    l.mcmc_status_string.restype = ctypes.c_char_p
    l.mcmc_detect_last_error.argtypes = [vp]
    l.mcmc_detect_last_error.restype = ctypes.c_char_p
    l.mcmc_detect_kernel_launches.argtypes = [vp]
    l.mcmc_detect_kernel_launches.restype = ctypes.c_int64
    l.mcmc_detect_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32,
                                      ctypes.c_uint64, i32, ctypes.c_float, ctypes.c_float, vp,
                                      vp, vp, vp]
    l.mcmc_detect_noalloc.restype = ctypes.c_int
    l.mcmc_mlp_param_count.argtypes = [i32]
    l.mcmc_mlp_param_count.restype = i64
    l.mcmc_mlp_create.argtypes = [i32, i32, vp, ctypes.POINTER(vp)]
    l.mcmc_mlp_destroy.argtypes = [vp]
    l.mcmc_mlp_last_error.argtypes = [vp]
    l.mcmc_mlp_last_error.restype = ctypes.c_char_p
    l.mcmc_mlp_set_params.argtypes = [vp, vp, i32]
    l.mcmc_mlp_set_train_engine.argtypes = [vp, i32]
    l.mcmc_mlp_get_params.argtypes = [vp, vp, i32]
    l.mcmc_mlp_forward.argtypes = [vp, i64, vp, vp, i32]
    l.mcmc_mlp_loss_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    l.mcmc_mlp_train_step.argtypes = [vp, i32, vp, vp, vp, ctypes.c_float, vp]
    l.mcmc_detect_features.argtypes = [vp, i32, vp]
    l.mcmc_detect_set_model.argtypes = [vp, vp, ctypes.c_float, i32]
    l.mcmc_detect_init_learned.argtypes = [vp]
    l.mcmc_detect_mix_step.argtypes = [vp, i64]
    for n in ABI_FUNCTIONS_LEARNED:
        if n not in ("mcmc_mlp_param_count", "mcmc_mlp_last_error"):
            getattr(l, n).restype = ctypes.c_int
    l.mcmc_diag_transition.argtypes = [i32, i32, i32, i32, vp, vp, vp, i32, ctypes.c_float,
                                       ctypes.c_float, vp, vp, vp, i32, vp, vp]
    l.mcmc_diag_transition.restype = ctypes.c_int
    if path is None:
        _lib = l
    return l


def lib():
    return load()


def _ptr(x) -> int:
    """Address of a torch tensor / numpy array / None."""
    if x is None:
        return 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return int(x.ctypes.data)
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return int(x.data_ptr())
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _is_host(x) -> bool:
    if isinstance(x, np.ndarray):
        return True
    return hasattr(x, "device") and x.device.type == "cpu"


class Detector:
    """One ``mcmc_detector`` handle (see include/mcmcdet.h for every argument's meaning)."""

    def __init__(self, *, max_channels: int, max_nt: int, max_nr: int, chains: int,
                 precision: str = "fp32", preconditioned: bool = True, refresh_period: int = 0,
                 split_terms: int = 2, engine: int = MCMC_ENGINE_AUTO, seed: int = 0,
                 stream=None, tile: int = 0):
        self._l = lib()
        cfg = Config()
        self._l.mcmc_config_default(ctypes.byref(cfg))
        cfg.max_channels, cfg.max_nt, cfg.max_nr = int(max_channels), int(max_nt), int(max_nr)
        cfg.chains = int(chains)
        cfg.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        cfg.preconditioned = int(bool(preconditioned))
        cfg.refresh_period = int(refresh_period)
        cfg.split_terms = int(split_terms)
        cfg.engine = int(engine)
        cfg.tile = int(tile)
        cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
        cfg.stream = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else (stream or None)
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = self._l.mcmc_detect_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise McmcError(st, self._l.mcmc_status_string(st).decode())
        self._h = h
        self.batch_meta = None

    # -- helpers --------------------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            msg = self._l.mcmc_detect_last_error(self._h).decode()
            raise McmcError(st, msg or self._l.mcmc_status_string(st).decode())

    @property
    def handle(self):
        return self._h

    def kernel_launches(self) -> int:
        return int(self._l.mcmc_detect_kernel_launches(self._h))

    # -- C ABI ----------------------------------------------------------------------------
    def preprocess(self, nt, nr, qam, H, H_off, y, y_off, noise_var, *, alpha_scale=1.0,
                   tau=2.0):
        nt = np.ascontiguousarray(nt, np.int32)
        nr = np.ascontiguousarray(nr, np.int32)
        qam = np.ascontiguousarray(qam, np.int32)
        H_off = np.ascontiguousarray(H_off, np.int64)
        y_off = np.ascontiguousarray(y_off, np.int64)
        host = _is_host(H)
        if host != _is_host(y) or host != _is_host(noise_var):
            raise ValueError("H, y and noise_var must all be host or all be device buffers")
        self._keep = (nt, nr, qam, H_off, y_off, H, y, noise_var)
        st = self._l.mcmc_detect_preprocess(
            self._h, int(nt.shape[0]), _ptr(nt), _ptr(nr), _ptr(qam), _ptr(H), _ptr(H_off),
            _ptr(y), _ptr(y_off), _ptr(noise_var), float(alpha_scale), float(tau), int(host))
        self._check(st)
        L = np.round(np.sqrt(qam)).astype(np.int64)
        nb = np.log2(L).astype(np.int64)
        self.batch_meta = dict(nt=nt, nr=nr, qam=qam, N=2 * nt.astype(np.int64), L=L, log2L=nb,
                               n_channels=int(nt.shape[0]))

    def run_chains(self, iterations: int, t_offset: int = 0):
        self._check(self._l.mcmc_detect_run_chains(self._h, int(iterations), int(t_offset)))

    def sizes(self):
        m = self.batch_meta
        n_ant = int(m["nt"].sum())
        n_bits = int((m["nt"].astype(np.int64) * 2 * m["log2L"]).sum())
        n_states = int(self.cfg.chains * m["N"].sum())
        return n_ant, n_bits, n_states

    def estimate(self, best_idx=None, llr=None, best_f=None, *, host_io: Optional[bool] = None,
                 stats: bool = False):
        """Fills the given buffers; with no buffers, returns new host numpy arrays."""
        ret_new = best_idx is None and llr is None and best_f is None
        if ret_new:
            n_ant, n_bits, _ = self.sizes()
            best_idx = np.zeros(n_ant, np.int8)
            llr = np.zeros(n_bits, np.float32)
            best_f = np.zeros(self.batch_meta["n_channels"], np.float64)
        bufs = [b for b in (best_idx, llr, best_f) if b is not None]
        if host_io is None:
            host_io = _is_host(bufs[0]) if bufs else True
        s = Stats()
        st = self._l.mcmc_detect_estimate(self._h, _ptr(best_idx), _ptr(llr), _ptr(best_f),
                                          ctypes.byref(s) if stats else None, int(host_io))
        self._check(st)
        out = dict(best_idx=best_idx, llr=llr, best_f=best_f)
        if stats:
            out["stats"] = dict(transitions=s.transitions, accepts=s.accepts,
                                refresh_drift=s.refresh_drift,
                                refresh_drift_rel=s.refresh_drift_rel,
                                numeric_faults=s.numeric_faults,
                                near_ties=[int(v) for v in s.near_ties],
                                near_tie_windows=[1e-6, 1e-4, 1e-2])
        return out

    def llr_list(self, clip: float, llr=None, *, host_io: Optional[bool] = None):
        """List-based LLRs (Eq. (31)) of the current states, clipped to [-clip, clip]; with no
        buffer, returns a new host numpy array."""
        if llr is None:
            _, n_bits, _ = self.sizes()
            llr = np.zeros(n_bits, np.float32)
        if host_io is None:
            host_io = _is_host(llr)
        self._check(self._l.mcmc_detect_llr_list(self._h, _ptr(llr), float(clip), int(host_io)))
        return llr

    def get_chains(self, states=None, f=None, *, host_io: Optional[bool] = None):
        if states is None and f is None:
            _, _, n_states = self.sizes()
            states = np.zeros(n_states, np.int8)
            f = np.zeros(self.batch_meta["n_channels"] * self.cfg.chains, np.float64)
        if host_io is None:
            host_io = _is_host(states if states is not None else f)
        self._check(self._l.mcmc_detect_get_chains(self._h, _ptr(states), _ptr(f), int(host_io)))
        return states, f

    def get_tracked(self, f=None, best_f=None, *, host_io: Optional[bool] = None):
        """Tracked energies of the current states and of each chain's best visited state, as
        the chains hold them (no FP64 re-evaluation); new host arrays when none are given."""
        if f is None and best_f is None:
            n = self.batch_meta["n_channels"] * self.cfg.chains
            f = np.zeros(n, np.float64)
            best_f = np.zeros(n, np.float64)
        if host_io is None:
            host_io = _is_host(f if f is not None else best_f)
        self._check(self._l.mcmc_detect_get_tracked(self._h, _ptr(f), _ptr(best_f), int(host_io)))
        return f, best_f

    def get_trace(self, trace=None, *, host_io: Optional[bool] = None):
        """Per chain [log acceptance ratio, log u] of its latest transition (handles created with
        MCMC_ENGINE_TRACE); a new host array [n_channels * chains, 2] when none is given."""
        if trace is None:
            trace = np.zeros((self.batch_meta["n_channels"] * self.cfg.chains, 2), np.float64)
        if host_io is None:
            host_io = _is_host(trace)
        self._check(self._l.mcmc_detect_get_trace(self._h, _ptr(trace), int(host_io)))
        return trace

    def launch_groups(self):
        """The batch's launch groups: dicts of engine, tile, packed, max_n, items, ctas_per_sm."""
        n = int(self._l.mcmc_detect_launch_groups(self._h, None, 0))
        buf = (ctypes.c_int32 * (6 * max(n, 1)))()
        self._l.mcmc_detect_launch_groups(self._h, buf, n)
        keys = ("engine", "tile", "packed", "max_n", "items", "ctas_per_sm")
        return [dict(zip(keys, buf[6 * i:6 * i + 6])) for i in range(n)]

    def run_kernel_ms(self, n: int = 1):
        """Device time (ms) of the chain kernels of the latest n runs, oldest first, without the
        exact energy evaluations around them (waits for those runs)."""
        buf = (ctypes.c_float * max(int(n), 1))()
        self._check(self._l.mcmc_detect_run_kernel_ms(self._h, int(n), buf))
        return [float(v) for v in buf[:int(n)]]

    def set_chains(self, states, *, host_io: Optional[bool] = None):
        if host_io is None:
            host_io = _is_host(states)
        if host_io:
            states = np.ascontiguousarray(states, np.int8)
        self._check(self._l.mcmc_detect_set_chains(self._h, _ptr(states), int(host_io)))

    def synchronize(self):
        self._check(self._l.mcmc_detect_synchronize(self._h))

    # -- learned proposal (include/mcmcdet_learned.h) --------------------------------------
    def features(self, X=None, *, at_zero: bool = False):
        """Network features of the current states (or of x = 0) into a device tensor."""
        import torch
        m = self.batch_meta
        rows = int(m["nt"].sum()) * (1 if at_zero else self.cfg.chains)
        if X is None:
            X = torch.empty((rows, 6), dtype=torch.float32, device="cuda")
        self._check(self._l.mcmc_detect_features(self._h, int(at_zero), _ptr(X)))
        return X

    def set_model(self, mlp, lam: float, *, tensor_cores: bool = False):
        self._model = mlp
        self._check(self._l.mcmc_detect_set_model(self._h, mlp.handle if mlp else None,
                                                  float(lam), int(tensor_cores)))

    def init_learned(self):
        self._check(self._l.mcmc_detect_init_learned(self._h))

    def mix_step(self, t: int):
        self._check(self._l.mcmc_detect_mix_step(self._h, int(t)))

    def run_mixed(self, iterations: int, period: int, t_offset: int = 0):
        """Transitions t_offset+1 .. t_offset+iterations; transition t is a mixture move when
        t % period == 0 and an Algorithm 1 transition otherwise."""
        t = t_offset
        end = t_offset + iterations
        while t < end:
            nxt = min(end, (t // period + 1) * period)
            plain = nxt - t - (1 if nxt % period == 0 else 0)
            if plain:
                self.run_chains(plain, t)
            t += plain
            if t < end and (t + 1) % period == 0:
                self.mix_step(t + 1)
                t += 1

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._l.mcmc_detect_destroy(self._h)
            self._h = ctypes.c_void_p()

    close = destroy

    def __del__(self):  # pragma: no cover
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


class Mlp:
    """One ``mcmc_mlp`` handle: the learned proposal's network (include/mcmcdet_learned.h)."""

    def __init__(self, qam: int, *, max_rows: int = 65536, stream=None):
        self._l = load()
        self.qam = int(qam)
        h = ctypes.c_void_p()
        sp = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else stream
        st = self._l.mcmc_mlp_create(self.qam, int(max_rows), ctypes.c_void_p(sp) if sp else None,
                                     ctypes.byref(h))
        if st != 0:
            raise McmcError(st, self._l.mcmc_status_string(st).decode())
        self._h = h
        self.max_rows = int(max_rows)
        self.param_count = int(self._l.mcmc_mlp_param_count(self.qam))

    @property
    def handle(self):
        return self._h

    def _check(self, st: int):
        if st != 0:
            msg = self._l.mcmc_mlp_last_error(self._h).decode()
            raise McmcError(st, msg or self._l.mcmc_status_string(st).decode())

    def set_train_engine(self, tensor_cores: bool):
        """Training products on tcgen05 (split-BF16, the default on sm_103) or CUDA cores."""
        self._check(self._l.mcmc_mlp_set_train_engine(self._h, int(bool(tensor_cores))))

    def set_params(self, params):
        if _is_host(params):
            params = np.ascontiguousarray(params, np.float32)
        self._check(self._l.mcmc_mlp_set_params(self._h, _ptr(params), int(_is_host(params))))

    def get_params(self, out=None):
        if out is None:
            out = np.zeros(self.param_count, np.float32)
        self._check(self._l.mcmc_mlp_get_params(self._h, _ptr(out), int(_is_host(out))))
        return out

    def forward(self, X, logits=None, *, tensor_cores: bool = False):
        import torch
        rows = int(X.shape[0])
        if logits is None:
            logits = torch.empty((rows, self.qam), dtype=torch.float32, device=X.device)
        self._check(self._l.mcmc_mlp_forward(self._h, rows, _ptr(X), _ptr(logits),
                                             int(tensor_cores)))
        return logits

    def loss_grad(self, X, labels, idx=None, rows=None):
        """(loss, gradient) as device tensors; rows defaults to len(idx) or len(X)."""
        import torch
        if rows is None:
            rows = int(idx.shape[0]) if idx is not None else int(X.shape[0])
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        grad = torch.zeros(self.param_count, dtype=torch.float32, device=X.device)
        self._check(self._l.mcmc_mlp_loss_grad(self._h, int(rows), _ptr(X), _ptr(labels),
                                               _ptr(idx), _ptr(loss), _ptr(grad)))
        return loss, grad

    def train_step(self, X, labels, idx, lr: float, loss=None, rows=None):
        if rows is None:
            rows = int(idx.shape[0]) if idx is not None else int(X.shape[0])
        self._check(self._l.mcmc_mlp_train_step(self._h, int(rows), _ptr(X), _ptr(labels),
                                                _ptr(idx), float(lr), _ptr(loss)))
        return loss

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._l.mcmc_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    close = destroy

    def __del__(self):  # pragma: no cover
        try:
            self.destroy()
        except Exception:
            pass


def transition_diagnostics(H, y, noise_var, nt: int, nr: int, qam: int, *, preconditioned=True,
                           alpha_scale: float = 1.0, tau: float = 2.0, tv_steps: int = 0,
                           eigenvalues: bool = False, stream=None):
    """Exact transition kernels of a batch of small channels of one shape, on the GPU (see
    include/mcmcdet_diag.h). H, y: device float32 tensors with the complex entries interleaved
    (channel b at H[b * nr * nt * 2:], column-major nr x nt; y[b * nr * 2:]); noise_var: device
    float32 [n_channels]. Returns device float64 tensors: P [B, S, S], pi [B, S], and, when
    asked for, eig [B, S] (descending) and tv [B, tv_steps + 1]."""
    import torch
    n = int(noise_var.numel())
    L = {4: 2, 16: 4, 64: 8}.get(int(qam), 0)
    S = L ** (2 * int(nt)) if L else 0
    if not S or S > 256 or n < 1:
        raise McmcError(1, "shape outside the diagnostics' range")
    dev = noise_var.device
    P = torch.empty((n, S, S), dtype=torch.float64, device=dev)
    pi = torch.empty((n, S), dtype=torch.float64, device=dev)
    eig = torch.empty((n, S), dtype=torch.float64, device=dev) if eigenvalues else None
    tv = torch.empty((n, tv_steps + 1), dtype=torch.float64, device=dev) if tv_steps > 0 else None
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = load().mcmc_diag_transition(n, int(nt), int(nr), int(qam), _ptr(H), _ptr(y),
                                     _ptr(noise_var), int(bool(preconditioned)),
                                     float(alpha_scale), float(tau), _ptr(P), _ptr(pi), _ptr(eig),
                                     int(tv_steps), _ptr(tv), ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise McmcError(rc, "mcmc_diag_transition")
    out = {"P": P, "pi": pi}
    if eig is not None:
        out["eig"] = eig
    if tv is not None:
        out["tv"] = tv
    return out
