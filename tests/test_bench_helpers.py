"""The bench's roofline arithmetic and profile lookups, on the host.

achieved = algorithmic work per launch / the launch's measured time; frac =
achieved / peak, the peak from the measured file (3xTF32: the TF32 rate, the
measured BF16 rate times the nominal TF32/BF16 ratio, over three products);
a profiled DRAM traffic counts only while the kernel's source is unchanged.
The reference arm (the FP64 oracle on the host cores) prints its own line on
rank 0 only."""
import os
import types

import pytest

import bench


def _scene(m=100, n_newton=5):
    return types.SimpleNamespace(m=m, n_newton=n_newton)


def _prof(**ms_per_launch):
    return {k: {"launches_per_step": n, "ms_per_launch": t, "ms_per_step": n * t} for k, (n, t) in ms_per_launch.items()}


def test_tensor_roofline_is_flops_per_launch_over_time():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2000.0}
    info = {"flops_front_tc": 6e11, "flops_front_simt": 0.0, "flops_contract_tc": 2e11, "flops_contract_simt": 0.0}
    prof = _prof(k_front_gemm_tc=(6, 0.5), k_contract_tc=(1, 1.0))
    out = bench.rooflines(_scene(), "tissue_c3", prof, info, {"build_WH": 2.0}, [], peaks, 150)
    tf32x3 = 1800.0 * bench.TF32_PER_BF16 / 3.0
    fg = out["k_front_gemm_tc"]
    assert fg["per_launch"] == pytest.approx(1e11)                  # 6e11 flops over 6 launches
    assert fg["achieved"] == pytest.approx(1e11 / 0.5e-3 / 1e12)     # TFLOP/s
    assert fg["peak"] == pytest.approx(tf32x3) and fg["frac"] == pytest.approx(fg["achieved"] / tf32x3)
    ct = out["k_contract_tc"]
    assert ct["achieved"] == pytest.approx(2e11 / 1e-3 / 1e12)
    # the whole build against the same 3xTF32 rate, from the build phase's time
    assert out["w_h_build"]["achieved"] == pytest.approx(8e11 / 2e-3 / 1e12)
    # shares of the step add up over the profiled kernels
    assert fg["share_of_step"] + ct["share_of_step"] == pytest.approx(1.0)


def test_memory_rooflines_use_the_dense_definitions():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0}
    m, nn = 100, 5
    m3 = 3 * m
    info = {"flops_front_tc": 0.0, "flops_front_simt": 0.0, "flops_contract_tc": 0.0, "flops_contract_simt": 0.0}
    prof = _prof(k_update_W=(nn, 0.01), k_pgs=(nn, 0.2))
    stats = [{"sweeps": s, "sweeps_s_only": 0, "deferred_folds": 0, "rechecks": 0, "joins": 0, "n_stick": 0,
              "n_slip": 3} for s in (50, 1, 1, 1, 1)]
    out = bench.rooflines(_scene(m, nn), "tissue_c3", prof, info, {"build_WH": 1.0}, stats, peaks, 150)
    uw = out["k_update_W"]
    # W_H read and W written once per Newton iteration, plus the directions
    assert uw["per_launch"] == pytest.approx(2.0 * m3 * m3 * 4 + 9 * m * 4)
    assert uw["achieved"] == pytest.approx(uw["per_launch"] / 1e-5 / 1e9) and uw["peak"] == 6000.0
    pg = out["k_pgs"]
    # one read of W per sweep run (54 sweeps in the step) and the gaps, per launch
    assert pg["per_launch"] == pytest.approx((54 * m3 * m3 * 4.0 + nn * m3 * 4 * 3) / nn)
    assert pg["latency"]["sweeps_per_launch"] == [50, 1, 1, 1, 1]
    assert pg["latency"]["ns_per_contact_visit"] == pytest.approx(0.2e-3 * 1e9 / (54 * m / nn))


def test_fallback_peaks_are_named():
    out = bench.rooflines(_scene(), "tissue_c3", _prof(k_update_W=(5, 0.01)),
                          {"flops_front_tc": 0.0, "flops_front_simt": 0.0, "flops_contract_tc": 0.0,
                           "flops_contract_simt": 0.0}, {"build_WH": 1.0}, [], {}, 150)
    assert out["k_update_W"]["peak"] == 6800.0 and "fallback" in out["k_update_W"]["peak_note"]


def test_profiled_traffic_follows_the_source_hash():
    # the committed profile of the current source is found; any other hash is not
    got = bench.profiled_traffic("k_contract_tc", "tissue_c3")
    sha = bench.source_sha("k_contract_tc")
    table = open(os.path.join(bench.ROOT, "profiles", "traffic_tissue_c3.md")).read()
    if f"| {sha} |" in table:
        assert isinstance(got, int) and got > 0
    else:
        assert got is None
    assert bench.profiled_traffic("k_contract_tc", "no_such_workload") is None
    assert bench.profiled_traffic("k_unknown", "tissue_c3") is None


def test_reference_arm_prints_its_line(monkeypatch, capsys):
    # the oracle arm on the 9k-DOF liver scene: one JSON line with the arm's
    # keys, copies declared as none, and the host cores the solves kept busy
    import json
    monkeypatch.setattr(bench, "WORKLOAD", "liver_c1")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.run_reference(types.SimpleNamespace(steps=3, warmup=1, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 3 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] == pytest.approx(1e3 / line["value"])
    assert line["config"]["contacts"] == 300 and line["config"]["workload"].startswith("liver_c1")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and 1 <= cb["cores"] <= (os.cpu_count() or 1)
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["gpu_launches"] == 0


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(types.SimpleNamespace(steps=3, warmup=1, gpus=2))
    assert capsys.readouterr().out == ""
