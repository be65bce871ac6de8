"""bench.py's use of the committed ncu summaries: a kernel's recorded DRAM
bytes are reported only for the source hash the summary was taken on, and the
recorded figures are in the units bench.py reports them in."""
import os
import re

import bench

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")


def _field(name, key):
    text = open(os.path.join(PROFILES, name)).read()
    m = re.search(rf"^{key}:\s*(\S+)", text, re.M)
    assert m, (name, key)
    return m.group(1)


def test_fit_traffic_only_for_its_sources():
    h = _field("fit_kernel_fit_workload.txt", "source_hash")
    t = bench.recorded_traffic(h)
    assert t == float(_field("fit_kernel_fit_workload.txt", "dram_bytes_per_launch"))
    assert bench.recorded_traffic("0" * 16) is None
    # bytes per launch of the 2M-track, 10-layer workload: within a factor of
    # two of its algorithmic bytes (inputs read once, outputs written once)
    algo = float(_field("fit_kernel_fit_workload.txt", "algorithmic_bytes_per_launch"))
    assert 0.5 * algo < t < 2.0 * algo


def test_build_traffic_only_for_its_sources():
    h = _field("build_kernel_build_workload.txt", "source_hash")
    t = bench.recorded_build_traffic(h)
    parts = [float(_field("build_kernel_build_workload.txt", k)) for k in
             ("dram_bytes_read_per_launch", "dram_bytes_write_per_launch", "binning_dram_bytes_per_launch")]
    assert t == sum(parts)
    assert bench.recorded_build_traffic("0" * 16) is None


def test_source_hash_covers_included_headers(tmp_path, monkeypatch):
    """The hash follows #include "..." into the package's csrc/ headers: a
    change to a header the translation unit includes changes the hash; the
    public header (declarations and their documentation) does not."""
    csrc = tmp_path / "paper_1705_02876_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "include").mkdir()
    (tmp_path / "paper_1705_02876_gb300" / "build.py").write_text("# build\n")
    (csrc / "unit.cu").write_text('#include "a.cuh"\n#include "kf.h"\n')
    (csrc / "a.cuh").write_text("// a\n")
    (tmp_path / "include" / "kf.h").write_text("/* h */\n")
    (csrc / "other.cuh").write_text("// not included\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash("unit.cu")
    (csrc / "other.cuh").write_text("// changed, still not included\n")
    assert bench.kernel_source_hash("unit.cu") == h0
    (tmp_path / "include" / "kf.h").write_text("/* h, changed */\n")
    assert bench.kernel_source_hash("unit.cu") == h0
    (csrc / "a.cuh").write_text("// a, changed\n")
    assert bench.kernel_source_hash("unit.cu") != h0
