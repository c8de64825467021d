"""Host logic of the benchmark (CPU): the recorded DRAM traffic of a kernel is reported only while
the kernel's sources are the ones it was measured on, and the replica timing takes the slowest
rank."""
import json
import os
import shutil

import pytest

import bench


def _copy_tree(tmp_path):
    root = tmp_path / "repo"
    (root / "paper_2606_31842_b300").mkdir(parents=True)
    shutil.copytree(os.path.join(bench.ROOT, "paper_2606_31842_b300", "csrc"),
                    root / "paper_2606_31842_b300" / "csrc")
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), root / "profiles")
    return root


def test_kernel_text_is_one_definition():
    src = open(os.path.join(bench.ROOT, "paper_2606_31842_b300", "csrc", "stencil.cu")).read()
    t3 = bench._kernel_text(src, "k_step3d")
    t32 = bench._kernel_text(src, "k_step3d2")
    assert t3.startswith("__global__") and t3.rstrip().endswith("}")
    assert "k_step3d2" not in t3 and t32 != t3
    assert t3.count("{") == t3.count("}")
    with pytest.raises(KeyError):
        bench._kernel_text(src, "no_such_kernel")


def test_traffic_records_match_current_sources():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for key, r in rec.items():
        kernel, prec = key.split(":")
        assert bench.traffic_for(kernel, prec) == r["dram_bytes_per_launch"], key


def test_traffic_is_null_once_the_kernel_changes(tmp_path, monkeypatch):
    root = _copy_tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_for("k_step3d", "fp32") is not None
    # editing another part of the same file keeps the record ...
    p = root / "paper_2606_31842_b300" / "csrc" / "stencil.cu"
    src = p.read_text()
    i = src.index("k_step_df(")
    j = src.index("{", i)
    p.write_text(src[:j + 1] + "  // edited\n" + src[j + 1:])
    assert bench.traffic_for("k_step3d", "fp32") is not None
    # ... and so does a comment inside the kernel ...
    src = p.read_text()
    j = src.index("T acc_c = acc[idx];")
    p.write_text(src[:j] + "/* note */ " + src[j:])
    assert bench.traffic_for("k_step3d", "fp32") is not None
    # ... editing the kernel's code drops it
    src = p.read_text()
    j = src.index("T acc_c = acc[idx];")
    p.write_text(src[:j] + "T acc_c = acc[idx] * T(1);" + src[j + len("T acc_c = acc[idx];"):])
    assert bench.traffic_for("k_step3d", "fp32") is None
    assert bench.traffic_for("k_step3d2", "fp32") is not None
    # a shared header drops every kernel built from it
    h = root / "paper_2606_31842_b300" / "csrc" / "whv_device.cuh"
    h.write_text(h.read_text() + "\nconstexpr int kEdited = 1;\n")
    assert bench.traffic_for("k_step3d2", "fp32") is None
    assert bench.traffic_for("unknown_kernel", "fp32") is None


def test_aggregate_single_process_is_identity():
    assert bench.aggregate_max(3.5, 1) == 3.5
