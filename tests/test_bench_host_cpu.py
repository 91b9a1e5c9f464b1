"""Host logic of bench.py's roofline (no GPU): the committed ncu summaries name kernels that exist
in the sources and carry figures that parse; the DRAM traffic is scaled to a launch by its moves
and dropped once the kernel's sources (code only, without comments) no longer hash to the profiled
ones."""
import os
import re

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_1411_4212_gb300", "csrc")


def _kernel_names():
    names = set()
    for f in os.listdir(CSRC):
        if f.endswith(".cu"):
            names |= set(re.findall(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s+)?(\w+)",
                                    open(os.path.join(CSRC, f)).read()))
    return names


def _profiles():
    out = []
    for name in sorted(os.listdir(bench.PROFILES)):
        if name.endswith(".md"):
            fields = bench.profile_fields(os.path.join(bench.PROFILES, name))
            if "kernel" in fields:
                out.append((name, fields))
    return out


def test_profiles_name_existing_kernels_and_parse():
    kernels = _kernel_names()
    profs = _profiles()
    assert profs
    for name, f in profs:
        assert f["kernel"].split("<")[0] in kernels, name
        assert re.fullmatch(r"[0-9a-f]{64}", f["source_sha256"]), name
        assert int(f["moves_per_launch"]) > 0 and float(f["dram_bytes_per_launch"]) > 0, name


def test_profiled_traffic_scales_and_expires(tmp_path, monkeypatch):
    k = "walker_pipe_kernel<false,2>"
    good = tmp_path / "p.md"
    good.write_text(f"- kernel: `{k}`\n- source_sha256: `{bench.kernel_source_hash()}`\n"
                    "- moves_per_launch: 1000\n- dram_bytes_per_launch: 5000\n")
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.profiled_traffic(k, 3000) == pytest.approx(15000.0)
    assert bench.profiled_traffic("walker_pipe_kernel<false,4>", 3000) is None
    good.write_text(f"- kernel: `{k}`\n- source_sha256: `{'0' * 64}`\n"
                    "- moves_per_launch: 1000\n- dram_bytes_per_launch: 5000\n")
    assert bench.profiled_traffic(k, 3000) is None


def test_hbm_peak_reads_the_measured_file_or_falls_back(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 1234.5}')
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.hbm_peak()
    assert peak == pytest.approx(1234.5e9) and "measured" in src
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    peak, src = bench.hbm_peak()
    assert peak == pytest.approx(6.8e12) and "fallback" in src


def test_source_hash_covers_code_not_comments():
    code = 'int f(int x) {\n  return x + 1;  // one more\n}\n/* block\n comment */ const char* s = "a // b";\n'
    same = 'int f(int x) { return x + 1; }\n  const char* s = "a // b";  // another comment\n'
    other = 'int f(int x) {\n  return x + 2;\n}\nconst char* s = "a // b";\n'
    assert bench._code_only(code) == bench._code_only(same)
    assert bench._code_only(code) != bench._code_only(other)
    assert '"a // b"' in bench._code_only(code)               # string literals are code
    assert "'//'" in bench._code_only("char c = '//';")       # and so are character literals
