"""Host logic of bench.py that decides whether the committed ncu counters still describe the exact
kernel: the code-only fingerprint of its sources, and the reading of the committed launch list."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
bench = pytest.importorskip("bench")


def test_code_only_drops_comments_and_blank_lines():
    src = "int a; // one\n\n/* two\n   lines */ int b;  \n   // three\nint c; /* four */ int d;\n"
    assert bench.code_only(src) == "int a;\n int b;\nint c;  int d;"


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources and the launch list, with bench.py pointed at it."""
    csrc = tmp_path / "paper_1201_2501_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(ROOT, "paper_1201_2501_gb300", "csrc", f), csrc / f)
    prof = tmp_path / "launches.md"
    shutil.copy(bench.TRAFFIC_PROFILE, prof)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    return csrc, prof


def test_a_comment_edit_keeps_the_fingerprint_and_a_code_edit_changes_it(tree):
    csrc, _ = tree
    fp0 = bench.kernel_fingerprint()
    f = csrc / "sfft_internal.h"
    text = f.read_text(encoding="utf-8")
    f.write_text(text + "\n// a note\n/* and a block\n   comment */\n\n", encoding="utf-8")
    assert bench.kernel_fingerprint() == fp0
    f.write_text(text + "\nconstexpr int kProbeOnly = 1;\n", encoding="utf-8")
    assert bench.kernel_fingerprint() != fp0


def _with_fingerprint(prof, fp, tag=None):
    import re

    text = prof.read_text(encoding="utf-8")
    text = re.sub(r"sources_sha256_16 = [0-9a-f]{16}", f"sources_sha256_16 = {fp}", text)
    if tag is not None:
        text = re.sub(r"workload_tag = [A-Za-z0-9_.]+", f"workload_tag = {tag}", text)
    prof.write_text(text, encoding="utf-8")


def test_traffic_is_read_only_when_sources_and_workload_match(tree):
    csrc, prof = tree
    import re

    traffic = int(re.search(r"traffic_per_step_bytes = (\d+)", prof.read_text(encoding="utf-8")).group(1))
    _with_fingerprint(prof, bench.kernel_fingerprint())
    assert bench.profiled_traffic() == traffic
    _with_fingerprint(prof, bench.kernel_fingerprint(), tag="n22_k64_b256_other")
    assert bench.profiled_traffic() is None
    _with_fingerprint(prof, "0" * 16, tag=bench.WORKLOAD_TAG)
    assert bench.profiled_traffic() is None
