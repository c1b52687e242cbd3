"""The ncu figures bench.py folds into its roofline lines (DRAM bytes per
corner ray, warp instructions per update or per ray, issue-active share) are
read from profiles/<kernel>_c2_reduced.md only while the profiled kernel's
sources hash to the value that summary records; otherwise the line reports
no traffic.  Checked on a throw-away tree, independent of the real sources."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _tree(tmp_path, kernel):
    csrc = tmp_path / "paper_2211_00354_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for i, fn in enumerate(bench.PROFILE_SOURCES[kernel]):
        (csrc / fn).write_text("// source %d of %s\n" % (i, kernel))
    (tmp_path / "profiles").mkdir()
    return csrc


@pytest.mark.parametrize("kernel", sorted(bench.PROFILE_SOURCES))
def test_figures_are_read_only_for_matching_sources(tmp_path, monkeypatch, kernel):
    csrc = _tree(tmp_path, kernel)
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    sha = bench.sources_sha(kernel)
    (tmp_path / "profiles" / (kernel + "_c2_reduced.md")).write_text(
        "summary\n\n    source-sha256: %s\n    dram-bytes-per-corner-ray: 16.5\n"
        "    warp-instructions-per-update: 5.697\n    issue-active-pct: 82.0\n" % sha)
    assert bench.profile_figures(kernel) == {"dram-bytes-per-corner-ray": 16.5,
                                             "warp-instructions-per-update": 5.697,
                                             "issue-active-pct": 82.0}
    # any change to one of the kernel's sources voids the figures
    first = bench.PROFILE_SOURCES[kernel][0]
    (csrc / first).write_text((csrc / first).read_text() + "// changed\n")
    assert bench.sources_sha(kernel) != sha
    assert bench.profile_figures(kernel) == {}


def test_missing_summary_gives_no_figures(tmp_path, monkeypatch):
    _tree(tmp_path, "k_eval32")
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    assert bench.profile_figures("k_eval32") == {}
