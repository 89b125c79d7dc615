"""Host-side pieces of bench.py that decide reported numbers (CPU only): the algorithmic flop model
of a primitive quartet (the roofline's numerator) and the gate that reads the committed ncu traffic
only while the J-engine sources are the ones it was taken on."""
import os
import shutil

import numpy as np

import bench


def test_flop_model_values():
    """40 + 3 sum_{k <= L} N(k) + 2 N(L_P) N(L_Q), N(L) = (L+1)(L+2)(L+3)/6: 45 flops for (ss|ss)
    (L_P = L_Q = 0), 450 for (pp|pp) (L_P = L_Q = 2); the class table sums class counts times these."""
    assert [bench.nh(L) for L in range(5)] == [1, 4, 10, 20, 35]
    assert bench.flops_per_prim_quartet(0, 0) == 45
    assert bench.flops_per_prim_quartet(2, 2) == 450
    assert bench.flops_per_prim_quartet(1, 0) == 40 + 3 * 5 + 2 * 4
    cq = np.zeros((5, 5))
    cq[0, 0], cq[2, 2] = 10, 3
    assert bench.algorithmic_flops(cq) == 10 * 45 + 3 * 450


def test_traffic_read_only_for_matching_sources(tmp_path, monkeypatch):
    """A profile summary carries the SHA-1 prefixes of jengine.cu and common.cuh; its DRAM bytes per
    build are reported only while both match, and a changed source turns the figure into None."""
    import hashlib
    root = tmp_path / "repo"
    csrc = root / "paper_1708_03377_gb300" / "csrc"
    (root / "profiles").mkdir(parents=True)
    csrc.mkdir(parents=True)
    for f in ("jengine.cu", "common.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1708_03377_gb300", "csrc", f), csrc)
    sha = {f: hashlib.sha1(open(csrc / f, "rb").read()).hexdigest()[:12] for f in ("jengine.cu", "common.cuh")}
    (root / "profiles" / "jengine_water64_fp64.txt").write_text(
        "summary\n"
        f"jengine_source_sha1: {sha['jengine.cu']}\n"
        f"common_source_sha1: {sha['common.cuh']}\n"
        "dram_bytes_per_build: 1234567\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profile_traffic() == 1234567.0
    with open(csrc / "common.cuh", "a") as fh:
        fh.write("\n// changed\n")
    assert bench.profile_traffic() is None

