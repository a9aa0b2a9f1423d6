"""Measurement plumbing on the CPU: the kernel source hash that ties a
committed ncu summary to the code it was taken on, the traffic lookup that
bench.py reports from it, and the autotuner's result cache."""
import json
import os
import shutil

import pytest

import bench
from paper_1805_12258_gb300 import autotune

CSRC = os.path.join("paper_1805_12258_gb300", "csrc")


def _copy_sources(root):
    os.makedirs(os.path.join(root, CSRC))
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(bench.ROOT, CSRC, f), os.path.join(root, CSRC, f))


def test_hash_ignores_comments_and_spacing(tmp_path, monkeypatch):
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    path = os.path.join(tmp_path, CSRC, bench.KERNEL_SOURCES[0])
    src = open(path).read()
    open(path, "w").write("// a new comment\n/* and a block\n comment */\n" +
                          src.replace("\n", "\n\n", 3))
    assert bench.kernel_source_hash() == h0
    open(path, "w").write(src + "\nint x;\n")
    assert bench.kernel_source_hash() != h0


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    # a table entry counts only for its kernel name and the source hash it
    # was taken on; any later change of the kernel's code voids it
    _copy_sources(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_hash()
    key = "staged 85x2097152 H=16 f32 tb=128 order=semitone"
    os.makedirs(os.path.join(tmp_path, "profiles"))
    with open(os.path.join(tmp_path, "profiles", "traffic.txt"), "w") as fh:
        fh.write("# kernel | dram_bytes_per_launch | kernel_sha | summary\n")
        fh.write(f"{key} | 765780224 | {sha} | x.md\n")
        fh.write(f"{key.replace('f32', 'bf16')} | 368234496 | 0123456789abcdef | y.md\n")
    assert bench.profiled_traffic(key) == 765780224
    assert bench.profiled_traffic(key.replace("semitone", "octave")) is None
    assert bench.profiled_traffic(key.replace("f32", "bf16")) is None  # other source
    path = os.path.join(tmp_path, CSRC, "hs_device.cuh")
    open(path, "a").write("\nstatic int changed;\n")
    assert bench.profiled_traffic(key) is None


def test_committed_traffic_table_is_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.txt")) as fh:
        rows = [ln.split("|") for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        name, traffic, sha, summary = (x.strip() for x in r)
        assert name.startswith(("staged ", "generic ")) and int(traffic) > 0
        assert len(sha) == 16 and int(sha, 16) >= 0
        assert os.path.exists(os.path.join(bench.ROOT, "profiles", summary))


def test_instructions_only_for_the_profiled_source(tmp_path, monkeypatch):
    # an instruction count counts only for its run's name and the hash of
    # the files its entry names; a code change in any of them voids it
    files = ["hs_hfrac.cu", "hs_device.cuh"]
    os.makedirs(os.path.join(tmp_path, CSRC))
    for f in files:
        shutil.copy(os.path.join(bench.ROOT, CSRC, f), os.path.join(tmp_path, CSRC, f))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    key = "staged hfrac 85x2097152 H=16 f32 tb=64"
    os.makedirs(os.path.join(tmp_path, "profiles"))
    with open(os.path.join(tmp_path, "profiles", "instructions.txt"), "w") as fh:
        fh.write("# kernel | warp_instructions_per_run | source_sha | files | summary\n")
        fh.write(f"{key} | 3600000000 | {bench.source_hash(files)} | {', '.join(files)} | x.md\n")
        fh.write(f"{key.replace('64', '128')} | 1 | {bench.source_hash(files)} | missing.cu | y.md\n")
    assert bench.profiled_instructions(key) == 3600000000
    assert bench.profiled_instructions(key.replace("64", "128")) is None  # no such file
    assert bench.profiled_instructions("staged 85x2097152 H=16 f32") is None
    open(os.path.join(tmp_path, CSRC, "hs_hfrac.cu"), "a").write("\nstatic int changed;\n")
    assert bench.profiled_instructions(key) is None


def test_issue_roofline_arithmetic():
    # 152 SMs x 4 schedulers x 2070 MHz = 1.25856e12 warp-instructions/s
    r = bench.issue_roofline(1.25856e9, 1000.0, {"sm_mhz": 2070.0}, 152)
    assert r["bound"] == "issue" and r["peak"] == 152 * 4 * 2070e6
    assert abs(r["achieved"] - 1.25856e12) < 1.0 and abs(r["frac"] - 1.0) < 1e-12
    assert bench.issue_roofline(None, 1000.0, {"sm_mhz": 2070.0}, 152) is None
    assert bench.issue_roofline(1e9, 1000.0, {}, 152) is None


def test_committed_instruction_table_is_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "instructions.txt")) as fh:
        rows = [ln.split("|") for ln in fh if ln.strip() and not ln.startswith("#")]
    assert rows
    for r in rows:
        name, inst, sha, files, summary = (x.strip() for x in r)
        assert name.startswith("staged ") and int(inst) > 0
        assert len(sha) == 16 and int(sha, 16) >= 0
        for f in files.split(","):
            assert os.path.exists(os.path.join(bench.ROOT, CSRC, f.strip()))
        assert os.path.exists(os.path.join(bench.ROOT, "profiles", summary))


def test_order_names():
    assert bench.ORDER_NAMES[0] == bench.ORDER_NAMES[4] == "53-step"
    assert bench.ORDER_NAMES[3] == "semitone"
    assert bench.ORDER_NAMES[1] == "linear" and bench.ORDER_NAMES[2] == "octave"


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("HS_TUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}
    k = autotune.key_of("plane", 85, 16, "f32", 2 ** 21)
    assert k == "plane:85x16:f32:2^21"
    # bin counts are classed by the nearest power of two
    assert autotune.key_of("plane", 85, 16, "f32", 3_000_000) == "plane:85x16:f32:2^22"
    autotune._store(k, {"best": {"tile_bins": 128}, "table": []})
    autotune._store("other", {"best": {}, "table": []})
    d = json.loads(path.read_text())
    assert d[k]["best"] == {"tile_bins": 128} and "other" in d
    path.write_text("{ not json")
    assert autotune._load() == {}


def test_window_parity_compares_records_inside_the_window():
    import numpy as np

    import oracle
    from paper_1805_12258_gb300 import hs
    o = np.zeros(3, oracle.CAND_DTYPE)
    o["f"], o["z"], o["k"], o["power"] = [100, 150, 199], [0, -3, 5], [1, 4, 16], [20.0, 30.0, 50.0]
    near = np.zeros(1, oracle.CAND_DTYPE)
    near["f"], near["z"], near["k"], near["power"] = 160, 1, 2, 17.0
    g = np.zeros(5, hs.CAND_DTYPE)
    # three in-window records equal to the oracle's, one near-threshold
    # record, one outside the window (bin 50)
    g["bin"], g["z"], g["k"] = [100, 150, 199, 160, 50], [0, -3, 5, 1, 0], [1, 4, 16, 2, 1]
    g["power"] = [20.0, 30.0, 50.0, 17.0, 99.0]
    cpu = {"_window": (100, 200), "_records": o, "_near": near}
    r = bench.window_parity(g, cpu)
    assert r["equal"] and r["gpu_records"] == 4 and r["oracle_records"] == 3
    g2 = g.copy()
    g2["power"][1] = 30.0 * (1 + 3e-6)  # a power off by more than 1e-6
    assert not bench.window_parity(g2, cpu)["equal"]
    g3 = g[[0, 2, 3, 4]]  # a record missing
    r3 = bench.window_parity(g3, cpu)
    assert not r3["equal"] and r3["only_oracle"] == 1
    g4 = np.concatenate([g, g[:1]])  # a duplicate record
    assert not bench.window_parity(g4, cpu)["equal"]
