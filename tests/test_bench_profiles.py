"""bench.py's use of the committed ncu summaries (host logic, no GPU): the DRAM traffic and the
instruction count per chain x dimension x transition are quoted only while the summary's source
hash equals the hash of the kernel sources it was captured from, and only for the workload it
was captured on."""
import os

import bench


def _summary(tmp_path, h, workload="rayleigh_32x32_64qam"):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel source\n")
    prof = tmp_path / "summary.md"
    prof.write_text(f"# summary\n\nsource_hash: {h}\ndram_bytes_per_full_launch: 1.5e+09\n"
                    f"profile_workload: {workload}\nwarp_instructions_per_chain_dim_transition: 4.25\n")
    return src, prof


def _patch(monkeypatch, tmp_path, src, prof):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "CHAIN_SOURCES", {"mixed": [os.path.basename(src)]})
    monkeypatch.setattr(bench, "PROFILE_FILES", {"mixed": os.path.basename(prof)})
    monkeypatch.setattr(bench, "ISSUE_PROFILES",
                        {("mixed", "rayleigh_32x32_64qam"): os.path.basename(prof),
                         ("mixed", "kronecker_128x128_64qam"): os.path.basename(prof)})


def test_current_summary_is_quoted(monkeypatch, tmp_path):
    src, prof = _summary(tmp_path, "0" * 16)
    _patch(monkeypatch, tmp_path, src, prof)
    h = bench._kernel_hash(bench.CHAIN_SOURCES["mixed"])
    prof.write_text(prof.read_text().replace("0" * 16, h))
    assert bench.profiled_traffic("mixed", "rayleigh_32x32_64qam") == 1.5e9
    assert bench.profiled_traffic("mixed", "kronecker_128x128_64qam") is None
    assert bench.profiled_issue("mixed", "rayleigh_32x32_64qam") == 4.25
    # another workload's instruction count is not this one's
    assert bench.profiled_issue("mixed", "kronecker_128x128_64qam") is None


def test_stale_summary_is_not_quoted(monkeypatch, tmp_path):
    src, prof = _summary(tmp_path, "0" * 16)
    _patch(monkeypatch, tmp_path, src, prof)
    h = bench._kernel_hash(bench.CHAIN_SOURCES["mixed"])
    prof.write_text(prof.read_text().replace("0" * 16, h))
    src.write_text("// kernel source, changed since the capture\n")
    assert bench.profiled_traffic("mixed", "rayleigh_32x32_64qam") is None
    assert bench.profiled_issue("mixed", "rayleigh_32x32_64qam") is None


def test_committed_summaries_name_their_workload():
    for (precision, workload), f in bench.ISSUE_PROFILES.items():
        text = open(os.path.join(bench.ROOT, f)).read()
        assert f"profile_workload: {workload}" in text, f
        assert "warp_instructions_per_chain_dim_transition:" in text, f
        assert "source_hash:" in text, f


def test_missing_summary(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profiled_traffic("mixed", "rayleigh_32x32_64qam") is None
    assert bench.profiled_issue("mixed", "rayleigh_32x32_64qam") is None
    assert bench.profiled_issue("fp64", "rayleigh_32x32_64qam") is None
