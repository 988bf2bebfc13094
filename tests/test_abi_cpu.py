"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every entry point
that include/mcmcdet.h, include/mcmcdet_learned.h and include/mcmcdet_diag.h declare. Only
host-only entry points and host-side argument checks are called (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions(name="mcmcdet.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcmc_[a-z_]+)\s*\(", src)))


@pytest.mark.parametrize("header,attr", [("mcmcdet.h", "ABI_FUNCTIONS"),
                                         ("mcmcdet_learned.h", "ABI_FUNCTIONS_LEARNED"),
                                         ("mcmcdet_diag.h", "ABI_FUNCTIONS_DIAG")])
def test_library_builds_and_exports_every_declared_symbol(header, attr):
    import paper_2407_06042_gb300 as pkg
    lib = pkg.load()
    declared = _header_functions(header)
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), f"{name} not exported"
    assert sorted(getattr(pkg, attr)) == declared


def test_learned_host_only_entry_points():
    """Parameter counts agree with the oracle network's layout; argument checks run on the
    host before any device call."""
    import paper_2407_06042_gb300 as pkg
    import oracle.mlp as omlp
    lib = pkg.load()
    for q in (4, 16, 64):
        assert lib.mcmc_mlp_param_count(q) == omlp.param_count(q)
    assert lib.mcmc_mlp_param_count(8) == 0
    h = ctypes.c_void_p()
    assert lib.mcmc_mlp_create(8, 16, None, ctypes.byref(h)) == 1
    assert lib.mcmc_mlp_create(16, 0, None, ctypes.byref(h)) == 1
    assert lib.mcmc_mlp_create(16, 16, None, None) == 1
    assert lib.mcmc_mlp_destroy(None) == 1
    assert lib.mcmc_mlp_last_error(None) == b"null handle"
    assert lib.mcmc_mlp_set_train_engine(None, 1) == 1
    assert lib.mcmc_detect_mix_step(None, 1) == 1
    assert lib.mcmc_detect_set_model(None, None, 0.5, 0) == 1


def test_host_only_entry_points():
    import paper_2407_06042_gb300 as pkg
    lib = pkg.load()
    cfg = pkg.Config()
    lib.mcmc_config_default(ctypes.byref(cfg))
    assert cfg.chains == 32 and cfg.precision == pkg.MCMC_PREC_FP32 and cfg.preconditioned == 1
    assert lib.mcmc_status_string(0) == b"ok"
    assert lib.mcmc_status_string(1) == b"invalid argument"
    assert lib.mcmc_detect_destroy(None) == 0
    assert lib.mcmc_detect_kernel_launches(None) == 0
    assert lib.mcmc_detect_last_error(None) == b"null handle"
    assert lib.mcmc_detect_llr_list(None, None, 1.0, 0) == 1
    assert lib.mcmc_detect_run_chains(None, 1, 0) == 1
    assert lib.mcmc_detect_create(None, None) == 1
    assert lib.mcmc_detect_get_tracked(None, None, None, 0) == 1
    assert lib.mcmc_detect_get_trace(None, None, 0) == 1
    assert lib.mcmc_detect_launch_groups(None, None, 0) == 0
    assert lib.mcmc_detect_run_kernel_ms(None, 1, None) == 1


def test_config_struct_matches_header():
    import paper_2407_06042_gb300 as pkg
    # int32 x 10 + uint64 + pointer
    assert ctypes.sizeof(pkg.Config) == 10 * 4 + 8 + 8
    # int64 x 2 + int32 x 2 + double + int64 x 3 (near-tie counts) + double
    assert ctypes.sizeof(pkg.Stats) == 8 + 8 + 4 + 4 + 8 + 3 * 8 + 8


def test_diag_argument_checks_on_the_host():
    """Arguments outside the diagnostics' range are rejected before any device call."""
    import paper_2407_06042_gb300 as pkg
    lib = pkg.load()
    d = ctypes.c_void_p(16)          # never dereferenced: every call below fails its checks
    call = lib.mcmc_diag_transition
    bad = [
        (0, 2, 2, 4, d, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),    # no channels
        (1, 3, 3, 16, d, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),   # S = 4^6 > 256
        (1, 5, 5, 4, d, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),    # N = 10 > 8
        (1, 2, 2, 16, d, d, d, 1, 1.0, 2.0, d, None, d, 0, None, None),      # spectrum of S = 256
        (1, 1, 33, 4, d, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),   # nr > 32
        (1, 1, 1, 8, d, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),    # qam
        (1, 1, 1, 4, d, d, d, 2, 1.0, 2.0, d, None, None, 0, None, None),    # flag
        (1, 1, 1, 4, d, d, d, 1, 0.0, 2.0, d, None, None, 0, None, None),    # alpha_scale
        (1, 1, 1, 4, d, d, d, 1, 1.0, 0.5, d, None, None, 0, None, None),    # tau < 1
        (1, 1, 1, 4, d, d, d, 1, 1.0, 2.0, None, None, None, 0, None, None),  # no P
        (1, 1, 1, 4, None, d, d, 1, 1.0, 2.0, d, None, None, 0, None, None),  # no H
        (1, 1, 1, 4, d, d, d, 1, 1.0, 2.0, d, None, None, -1, d, None),      # tv_steps
    ]
    for args in bad:
        assert call(*args) == 1, args


def test_config_validation_on_the_host():
    """mcmc_detect_create rejects an invalid configuration before any device call (EINVAL). A
    valid one passes validation and, on a machine without a GPU, stops at the device query
    (EUNSUPPORTED); with a GPU it creates a handle, which is destroyed again."""
    import paper_2407_06042_gb300 as pkg
    lib = pkg.load()
    TC, AUTO, GRAPH, NOCL = pkg.MCMC_ENGINE_TC, pkg.MCMC_ENGINE_AUTO, pkg.MCMC_ENGINE_GRAPH, pkg.MCMC_ENGINE_NO_CLUSTER
    MIXED, FP32 = pkg.MCMC_PREC_MIXED, pkg.MCMC_PREC_FP32

    def create(**kw):
        cfg = pkg.Config()
        lib.mcmc_config_default(ctypes.byref(cfg))
        for k, v in kw.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        st = lib.mcmc_detect_create(ctypes.byref(cfg), ctypes.byref(h))
        if st == 0:
            lib.mcmc_detect_destroy(h)
        return st

    for kw in [dict(precision=MIXED, engine=TC, tile=64, max_nt=128, max_nr=128),
               dict(precision=MIXED, engine=TC | NOCL, tile=32),
               dict(precision=MIXED, engine=TC | GRAPH | NOCL),
               dict(precision=MIXED, engine=AUTO | NOCL),
               dict(precision=FP32, engine=pkg.MCMC_ENGINE_SIMT, tile=64),
               dict(precision=MIXED, engine=AUTO | pkg.MCMC_ENGINE_KERNEL_REFRESH, refresh_period=10)]:
        assert create(**kw) in (0, 7), kw
    for kw in [dict(engine=256), dict(engine=3), dict(precision=MIXED, engine=TC, tile=48),
               dict(precision=MIXED, engine=AUTO, tile=64), dict(precision=FP32, engine=TC),
               dict(max_nt=129), dict(chains=6), dict(split_terms=4),
               dict(refresh_period=-2)]:
        assert create(**kw) == 1, kw
