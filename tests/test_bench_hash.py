"""bench.py's key for stored DRAM counters (no GPU): a kernel's translation unit and the
local headers it includes, with comments and blank space ignored."""
from __future__ import annotations

import os
import shutil

import bench


def _tree(tmp_path):
    root = tmp_path / "tree"
    shutil.copytree(os.path.join(bench.ROOT, "paper_1303_0383_gb300", "csrc"),
                    root / "paper_1303_0383_gb300" / "csrc",
                    ignore=shutil.ignore_patterns("*.o", "_build"))
    shutil.copytree(os.path.join(bench.ROOT, "include"), root / "include")
    return root


def _edit(path, old, new):
    s = path.read_text()
    assert old in s
    path.write_text(s.replace(old, new, 1))


def test_unit_hash_follows_the_units_own_sources(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    csrc = root / "paper_1303_0383_gb300" / "csrc"
    unit0 = bench.kernel_source_hash("select_mixed.cu")
    all0 = bench.kernel_source_hash()
    assert unit0 != bench.kernel_source_hash("select.cu")
    # code of another kernel: the library's hash moves, the unit's does not
    (csrc / "mle.cu").write_text((csrc / "mle.cu").read_text() + "\nint lagp_hash_probe;\n")
    assert bench.kernel_source_hash() != all0
    assert bench.kernel_source_hash("select_mixed.cu") == unit0
    # a comment and blank lines in the unit itself: no change
    _edit(csrc / "select_mixed.cu", "#include", "// a comment\n\n#include")
    assert bench.kernel_source_hash("select_mixed.cu") == unit0
    # code in a header the unit includes (through predict_loc.cuh): the unit's hash moves
    _edit(csrc / "fp64_chol.cuh", "#pragma once", "#pragma once\nstatic int lagp_hash_probe2;")
    assert bench.kernel_source_hash("select_mixed.cu") != unit0
    # the FP64 selection unit does not include that header
    assert "fp64_chol.cuh" not in (csrc / "select.cu").read_text()
