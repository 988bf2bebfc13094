"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every entry point
that include/mcmcdet.h declares. Only host-only entry points are called (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "mcmcdet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mcmc_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    import paper_2407_06042_gb300 as pkg
    lib = pkg.load()
    declared = _header_functions()
    assert declared, "no declarations parsed"
    for name in declared:
        assert hasattr(lib, name), f"{name} not exported"
    assert sorted(pkg.ABI_FUNCTIONS) == declared


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
    assert lib.mcmc_detect_run_chains(None, 1, 0) == 1
    assert lib.mcmc_detect_create(None, None) == 1


def test_config_struct_matches_header():
    import paper_2407_06042_gb300 as pkg
    # int32 x 10 + uint64 + pointer
    assert ctypes.sizeof(pkg.Config) == 10 * 4 + 8 + 8
    assert ctypes.sizeof(pkg.Stats) == 8 + 8 + 4 + 4 + 8
