"""The bench's work counts and roofline arithmetic (CPU only, no GPU).

The ALU kernels' roofline has two pipes that issue side by side: t_roof =
max(flops / FP32 peak, special ops / SFU peak), `frac` = t_roof / measured
time.  The tensor kernels count the J rows and Gram blocks the method needs
once the channel-independent jump columns are stored once.
"""
import pytest

import bench


PIPES = {"fp32_tflops": 80.0, "sfu_gops": 5000.0}


def test_tensor_counts_take_the_jump_columns_once():
    # 128 curves: n_c = 2,048 (1,024 position + 1,024 jump columns per channel)
    n, P, Nb, nc = 1000, 8192, 1024, 2048
    jr, b1 = bench.step_work("tc_jrows", n, P, Nb, nc)
    sy, b2 = bench.step_work("tc_syrk", n, P, Nb, nc)
    assert b1 == b2 == "tensor"
    assert jr == 2.0 * 4096 * Nb * n                  # 3 x 1,024 position rows + 1,024 jump rows
    assert sy == (3 * 2048 * 2049 - 2 * 1024 * 1025) * n


def test_alu_roofline_takes_the_binding_pipe():
    n, P, Nb, nc = 1 << 20, 2048, 1024, 512
    (F, T), bound = bench.step_work("k_field", n, P, Nb, nc)
    assert bound == "alu_per_launch"
    assert F == n * (P * bench.FWD_HANDLE[0] + Nb * bench.FWD_BOUND[0])
    assert T == n * (P * bench.FWD_HANDLE[1] + Nb * bench.FWD_BOUND[1])
    t_fp, t_sf = F / 80e12, T / 5e12
    ms = 2.0 * max(t_fp, t_sf) * 1e3                 # a launch at half its roofline speed
    roofs = bench.rooflines({"k_field": (ms, 1)}, 1, n, P, Nb, nc, PIPES, cfg=2)
    (r,) = roofs
    assert r["frac"] == pytest.approx(0.5, rel=1e-12)
    assert r["bound"] == ("sfu" if t_sf > t_fp else "fp32")
    assert r["fp32_pipe_frac"] == pytest.approx(t_fp / (ms / 1e3), rel=1e-12)
    assert r["sfu_pipe_frac"] == pytest.approx(t_sf / (ms / 1e3), rel=1e-12)
    # the FP32-only recount: every special op as one flop
    assert r["fp32_only"]["frac"] == pytest.approx((F + T) / (ms / 1e3) / 80e12, rel=1e-12)


def test_per_step_work_is_split_over_launches():
    n, P, Nb, nc = 262144 * 4, 8192, 1024, 2048
    (F, T), bound = bench.step_work("k_frows", n, P, Nb, nc)
    assert bound == "alu"
    steps, launches = 3, 3 * 5
    ms = launches * 10.0
    (r,) = bench.rooflines({"k_frows": (ms, launches)}, steps, n, P, Nb, nc, PIPES, cfg=4)
    per = F * steps / launches
    assert r["flops_per_launch"] == pytest.approx(per, rel=1e-12)
    assert r["bound"] == "fp32"
    assert r["achieved"] == pytest.approx(per / 10e-3 / 1e12, rel=1e-12)


def test_compensated_schemes_count_three_products():
    n, P, Nb, nc = 262144, 8192, 1024, 2048
    jr, _ = bench.step_work("tc_jrows", n, P, Nb, nc)
    ms = 5.0
    prof = {"tc_jrows": (ms, 1)}
    (b,) = bench.rooflines(prof, 1, n, P, Nb, nc, PIPES, cfg=4, jtj="bf16")
    (x,) = bench.rooflines(prof, 1, n, P, Nb, nc, PIPES, cfg=4, jtj="bf16x3")
    (t,) = bench.rooflines(prof, 1, n, P, Nb, nc, PIPES, cfg=4, jtj="3xtf32")
    assert b["flops_per_launch"] == jr and x["flops_per_launch"] == 3 * jr
    assert x["frac"] == pytest.approx(3 * b["frac"], rel=1e-12)
    assert t["peak"] == pytest.approx(b["peak"] * 1.1 / 2.25, rel=1e-12)
    assert x["traffic"] is None and t["traffic"] is None


def test_traffic_record_is_dropped_when_its_kernel_source_changes(tmp_path, monkeypatch):
    """`traffic` comes from the committed ncu record only while the kernel's
    sources hash to the recorded SHA-256 and the workload is the recorded one."""
    import hashlib
    import json
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"k": {"bytes_per_launch": 123, "sources": ["k.cu"], "config": 4,
                 "sha256": hashlib.sha256(src.read_bytes()).hexdigest()}}
    (tmp_path / "profiles" / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("k", 4) == 123
    assert bench.kernel_traffic("k", 2) is None          # another workload
    assert bench.kernel_traffic("other", 4) is None      # no record
    src.write_text("__global__ void k() { }\n")         # the kernel changed
    assert bench.kernel_traffic("k", 4) is None


def test_committed_traffic_records_match_their_sources():
    """Every committed DRAM-traffic record is keyed to the sources as they
    stand, so the bench reports it (a source change re-captures or re-keys)."""
    import hashlib
    import json
    import os
    with open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as f:
        recs = json.load(f)
    for name, rec in recs.items():
        h = hashlib.sha256()
        for s in rec["sources"]:
            with open(os.path.join(bench.ROOT, s), "rb") as f:
                h.update(f.read())
        assert h.hexdigest() == rec["sha256"], name
        assert bench.kernel_traffic(name, rec["config"]) == rec["bytes_per_launch"]
