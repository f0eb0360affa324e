"""Host-side logic of bench.py (no GPU): the traffic record and its source check,
the clock sampler's summary, and the per-stage work the roofline divides."""
import os

import bench


def test_traffic_record_is_read_while_the_source_is_unchanged(tmp_path, monkeypatch):
    import hashlib
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic_stage_x.md").write_text(
        "# a summary\n\nCommand: something: with colons\n\n"
        f"source: kernel.cu\nsource_sha256_16: {digest}\ndram_bytes_per_launch: 1234567\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_from_profile("stage_x") == 1234567.0
    assert bench.traffic_from_profile("stage_y") is None  # no record
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.traffic_from_profile("stage_x") is None  # counters taken on another source


def test_committed_traffic_record_parses():
    path = os.path.join(bench.ROOT, "profiles", "traffic_inc_patch.md")
    text = open(path).read()
    assert "source: paper_2212_11296_gb300/csrc/k_incremental.cu" in text
    assert "dram_bytes_per_launch:" in text


def test_clock_summary_reports_throttle_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    rows = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    path.write_text("\n".join(rows) + "\n")
    c = bench.ClockSampler(0)
    c.path = str(path)
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    path.write_text("0, 1500, 2070, 800.0, 0x8, Active, Not Active, Not Active, Not Active\n")  # summary() removed it
    c2 = bench.ClockSampler(0)
    c2.path = str(path)
    assert c2.summary()["reasons"] == ["hw_slowdown"]


def test_stage_work_of_the_incremental_bf16_path():
    w = {"d_model": 256, "K": 256, "layers": 8, "L": 16}
    st = {"unique_rows": [10, 20, 30, 40, 50, 60, 70, 80, 90], "inc_searched_rows": 1000, "active_rows": 5000,
          "samples": 15, "attn_pairs": 0, "inc_base_rows": 3840, "inc_patched_rows": 4000,
          "inc_patch_pairs": 9000, "inc_full_pairs": 7000, "inc_whole_pairs": 11000}
    d, K = 256, 256
    assert bench.stage_flops("vq_argmin", st, w, True, True) == (1000 * 2.0 * K * d, "tensor")
    assert bench.stage_flops("inc_certificate", st, w, True, True) == (3840 * 2.0 * K * d, "tensor")
    assert bench.stage_flops("inc_certificate", st, w, False, True) == (3840 * 2.0 * K * d, "alu")
    # patch: 8 d per (row, changed key) pair; recompute: 4 d per pair; tensor cores on the BF16 path
    assert bench.stage_flops("inc_patch", st, w, True, True) == (9000 * 8.0 * d, "tensor")
    assert bench.stage_flops("inc_patch", st, w, False, True) == (9000 * 8.0 * d, "alu")
    assert bench.stage_flops("inc_recompute", st, w, True, True) == (7000 * 4.0 * d, "tensor")
    assert bench.stage_flops("inc_recompute", st, w, False, True) == (7000 * 4.0 * d, "alu")
    assert bench.stage_flops("inc_recompute_whole", st, w, True, True) == (11000 * 4.0 * d, "tensor")
    assert bench.stage_flops("qkv_gemm", st, w, True, True) == (sum(st["unique_rows"][:8]) * 6.0 * d * d, "tensor")
    assert bench.stage_flops("mlp_up", st, w, False, False) == (sum(st["unique_rows"][1:9]) * 8.0 * d * d, "alu")
    assert bench.stage_flops("dedupe", st, w, True, True) == (0.0, "hbm")
