"""Host-side pieces of bench.py (CPU only): the code hash that gates the committed ncu traffic,
the peak denominators and the reference arm's line."""

import json
import os
import subprocess
import sys

import bench


def test_strip_comments_keeps_code_and_literals():
    src = ('int a = 1; // trailing\n'
           '/* block\n   comment */ const char* s = "x // not a comment \\" /* nor this */";\n'
           "char q = '\"';  // quote in a char literal\n"
           '\n   \n'
           'asm volatile("mov.u32 %0, %1;" : "=r"(a) : "r"(b));  /* tail */\n')
    out = bench.strip_comments(src)
    assert out == ('int a = 1;\n'
                   ' const char* s = "x // not a comment \\" /* nor this */";\n'
                   "char q = '\"';\n"
                   'asm volatile("mov.u32 %0, %1;" : "=r"(a) : "r"(b));')


def test_code_hash_ignores_comment_edits(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1911_03813_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "fg_tc.cu").write_text("// header\n__global__ void k() { int x = 1; }\n")
    (csrc / "tc_common.cuh").write_text("#pragma once\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    (csrc / "fg_tc.cu").write_text("// another header\n\n__global__ void k() { int x = 1; }  "
                                   "/* note */\n")
    assert bench.kernel_source_hash() == h0
    (csrc / "fg_tc.cu").write_text("__global__ void k() { int x = 2; }\n")
    assert bench.kernel_source_hash() != h0


def test_traffic_is_reported_only_for_the_captured_code(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_1911_03813_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "fg_tc.cu").write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    entry = {"source_hash": bench.kernel_source_hash(), "dram_bytes_per_launch_full": 123.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"fg_pass_bf16": entry}))
    assert bench.ncu_traffic("fg_pass_bf16") == 123.0
    (csrc / "fg_tc.cu").write_text("__global__ void k() { return; }\n")
    assert bench.ncu_traffic("fg_pass_bf16") is None


def test_committed_traffic_entry_is_consistent():
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["fg_pass_bf16"]
    scale = bench.P_FULL / t["p_captured"]
    per_launch = (t["dram_bytes_read_captured"] + t["dram_bytes_write_captured"]) * scale
    assert abs(per_launch - t["dram_bytes_per_launch_full"]) <= 1.0
    assert t["algorithmic_bytes_per_launch_full"] == bench.P_FULL * bench.N_FEAT * 2
    # traffic at or just above the algorithmic bytes: V is read once per launch
    assert 1.0 <= per_launch / t["algorithmic_bytes_per_launch_full"] < 1.05


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    pk = bench.measured_peaks()
    assert pk["src"] == "fallback" and pk["hbm_gbs"] == 6800.0 and pk["sm_max_mhz"] == 2070.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 7000.0}))
    pk = bench.measured_peaks()
    assert pk["src"] == "measured" and pk["hbm_gbs"] == 7000.0


def test_serving_sweep_argument():
    class A:
        serving_sweep = "0.5, 1.0,,1.2"
    assert bench.sweep_of(A) == (0.5, 1.0, 1.2)
    A.serving_sweep = ""
    assert bench.sweep_of(A) == ()


def test_reference_arm_line_without_a_gpu():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and prints one JSON
    line with the contract's keys (a short run: one step, no warm-up)."""
    out = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl",
                          "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=bench.ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["config"]["workload"] == bench.WORKLOAD
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
