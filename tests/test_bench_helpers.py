"""Host-side helpers of bench.py that decide what the benchmark line reports.

A DRAM figure measured by ncu on a kernel is reported (roofline.traffic) only
while that kernel's sources are unchanged: the key is a hash of the kernel's
files with comments and blank lines left out, so a change of wording keeps the
figure and any change of code drops it.  No GPU needed."""
import json
import os

import pytest

import bench


@pytest.fixture()
def fake_tree(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2511_18071_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("// the kernel\n__global__ void k(float *a) {\n    a[0] = 1.f;  /* one */\n}\n")
    (csrc / "h.cuh").write_text("#pragma once\nconstexpr int N = 4;\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setitem(bench.KERNEL_SOURCES, "fake_kernel", ["k.cu", "h.cuh"])
    return tmp_path, csrc


def _record(root, sha):
    json.dump({"fake_kernel": {"source_sha": sha, "dram_bytes_per_launch": 1234}},
              open(os.path.join(root, "profiles", "traffic.json"), "w"))


def test_traffic_reported_while_sources_unchanged(fake_tree):
    root, csrc = fake_tree
    _record(root, bench.source_hash("fake_kernel"))
    assert bench.profile_traffic("fake_kernel") == 1234


def test_comment_edits_keep_the_figure(fake_tree):
    root, csrc = fake_tree
    _record(root, bench.source_hash("fake_kernel"))
    (csrc / "k.cu").write_text("// the kernel, reworded\n\n__global__ void k(float *a) {\n"
                               "    a[0] = 1.f;  /* the first entry */\n}\n")
    assert bench.profile_traffic("fake_kernel") == 1234


@pytest.mark.parametrize("edit", [("k.cu", "a[0] = 1.f;", "a[0] = 2.f;"), ("h.cuh", "N = 4", "N = 8")])
def test_code_edits_drop_the_figure(fake_tree, edit):
    root, csrc = fake_tree
    _record(root, bench.source_hash("fake_kernel"))
    f, old, new = edit
    p = csrc / f
    p.write_text(p.read_text().replace(old, new))
    assert bench.profile_traffic("fake_kernel") is None


def test_unknown_kernel_has_no_figure(fake_tree):
    root, _ = fake_tree
    _record(root, "0" * 16)
    assert bench.profile_traffic("other_kernel") is None
