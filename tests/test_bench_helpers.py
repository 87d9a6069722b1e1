"""Host helpers of bench.py: the FP8-e4m3 and BF16 roundings of the FP8 scan
study against PyTorch's own conversions, the roofline arithmetic and the
clock record of the timed region."""
import os
import sys

import numpy as np
import pytest
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _values(rng, n=20000):
    v = np.concatenate([
        rng.standard_normal(n) * 10.0,
        rng.uniform(-448, 448, n),
        rng.uniform(-2 ** -6, 2 ** -6, n),           # subnormal range of e4m3
        np.ldexp(rng.integers(1, 16, 1000), -9) * rng.choice([-1, 1], 1000),
    ])
    return v.astype(np.float32).astype(np.float64)


def test_round_bf16_matches_torch():
    v = _values(np.random.default_rng(1))
    want = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bench.round_bf16(v), want)


def test_round_e4m3_matches_torch():
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this torch")
    v = _values(np.random.default_rng(2))
    v = v[np.abs(v) <= 448.0]  # the study saturates beyond; torch maps to NaN
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(bench.round_e4m3(v), want)


def test_round_e4m3_grid_and_saturation():
    # every e4m3 value is a fixed point; halfway points go to the even neighbour
    grid = [0.0]
    for e in range(-6, 9):
        for mnt in range(8):
            grid.append((1 + mnt / 8) * 2.0 ** e)
    grid += [k * 2.0 ** -9 for k in range(1, 8)]
    grid = np.array(sorted(set(g for g in grid if g <= 448)))
    assert np.array_equal(bench.round_e4m3(grid), grid)
    assert bench.round_e4m3(np.array([1.0625]))[0] == 1.0     # tie to even mantissa 000
    assert bench.round_e4m3(np.array([1.1875]))[0] == 1.25    # tie to even mantissa 010
    assert bench.round_e4m3(np.array([1e6]))[0] == 448.0      # saturates
    assert bench.round_e4m3(np.array([-1e6]))[0] == -448.0


def test_stage_work_and_alu_peak():
    # the estimator's bytes are m rows of d FP32 values (+ query, ids, output)
    b, f = bench.stage_work("estimate", 10, 1000, 128, 8, 16, 100, 5.0)
    assert b == 10 * (100 * 128 * 4 + 128 * 4 + 16 * 4 + 4) and f == 0.0
    # the scan reads the lists once and writes every candidate's value
    b, f = bench.stage_work("scan", 10, 1000, 128, 8, 16, 100, 50.0)
    assert f == 2.0 * 10 * 50.0 * 128 and b == 1000 * 128 * 2 + 10 * 50.0 * 4
    b, _ = bench.stage_work("scan", 10, 1000, 130, 8, 16, 100, 50.0, "fp32")
    assert b == 1000 * 132 * 4 + 10 * 50.0 * 4
    b, _ = bench.stage_work("scan", 10, 1000, 130, 8, 16, 100, 50.0, "bf16x3")
    assert b == 3 * 1000 * 192 * 2 + 10 * 50.0 * 4
    # the selection reads them back and, unless the scan was the split one,
    # the k neighbours' FP32 rows
    b, _ = bench.stage_work("select", 10, 1000, 128, 8, 16, 100, 50.0, "fp32")
    assert b == 10 * (50.0 * 4 + 16 * 128 * 4 + 16 * 4)
    b, _ = bench.stage_work("select", 10, 1000, 128, 8, 16, 100, 50.0, "bf16x3")
    assert b == 10 * (50.0 * 4 + 16 * 4)
    # the method-only count leaves out the candidates' write and read-back
    b, f = bench.stage_work("scan", 10, 1000, 128, 8, 16, 100, 50.0, method_only=True)
    assert b == 1000 * 128 * 2 and f == 2.0 * 10 * 50.0 * 128
    b, _ = bench.stage_work("select", 10, 1000, 128, 8, 16, 100, 50.0, "bf16x3",
                            method_only=True)
    assert b == 10 * 16 * 4
    assert bench.fp32_alu_tflops(2070.0) == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_ncu_traffic_requires_same_schedule_and_source(tmp_path, monkeypatch):
    """A committed DRAM-traffic figure is used only for the schedule it was
    captured at and while the kernel's source is unchanged."""
    import json
    src = tmp_path / "paper_2107_02736_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "sample.cu").write_text("kernel v1")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sched = {"k": 1536, "m": 4000, "nprobe": 8, "precision": "bf16"}
    entry = {"kernel": "k_estimate<32>", "source": "sample.cu",
             "src_sha": bench.src_digest("sample.cu"), "schedule": sched,
             "bytes_per_launch_full": 123}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"estimate": entry}))
    assert bench.ncu_traffic("estimate", dict(sched)) == 123
    assert bench.ncu_traffic("estimate", dict(sched, m=8000)) is None
    assert bench.ncu_traffic("estimate", dict(sched, precision="fp32")) is None
    # several entries per stage: the one captured at the run's schedule
    other = dict(entry, schedule=dict(sched, precision="bf16x3"), bytes_per_launch_full=456)
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"estimate": [entry, other]}))
    assert bench.ncu_traffic("estimate", dict(sched, precision="bf16x3")) == 456
    assert bench.ncu_traffic("estimate", dict(sched)) == 123
    assert bench.ncu_traffic("select", sched) is None
    (src / "sample.cu").write_text("kernel v2")
    assert bench.ncu_traffic("estimate", sched) is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_of_the_timed_region(tmp_path):
    """Only samples stamped inside [mark_begin, mark_end] are summarised; the
    reasons are those seen there; with none inside, every sample is used."""
    import datetime
    base = datetime.datetime(2026, 12, 4, 2, 46, 43)
    def line(dt_ms, sm, reasons=("Not Active",) * 4):
        t = base + datetime.timedelta(milliseconds=dt_ms)
        stamp = t.strftime("%Y/%m/%d %H:%M:%S.") + f"{t.microsecond // 1000:03d}"
        return ", ".join([stamp, str(sm), "2070", "900.5", "0x0"] + list(reasons))
    rows = [line(0, 1200, ("Active", "Not Active", "Not Active", "Not Active")),
            line(20, 2070), line(40, 2055),
            line(60, 2070, ("Not Active", "Not Active", "Not Active", "Active")),
            line(80, 900)]
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clk.csv")
    open(c.path, "w").write("\n".join(rows) + "\n")
    c.proc = _Done()
    c.t_begin = (base + datetime.timedelta(milliseconds=15)).timestamp()
    c.t_end = (base + datetime.timedelta(milliseconds=65)).timestamp()
    got = c.stop()
    assert got["samples_in_region"] == 3 and got["samples_total"] == 5
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0
    assert got["reasons"] == ["sw_power_cap"]
    # a region between two samples: every sample is summarised
    c.path = str(tmp_path / "clk2.csv")
    open(c.path, "w").write("\n".join(rows) + "\n")
    c.t_begin = (base + datetime.timedelta(milliseconds=5)).timestamp()
    c.t_end = (base + datetime.timedelta(milliseconds=10)).timestamp()
    got = c.stop()
    assert got["samples_in_region"] == 0 and got["samples"] == 5
    assert got["reasons"] == ["hw_slowdown", "sw_power_cap"]


def _representative_headline():
    """A headline line with every section bench.py fills, at realistic sizes."""
    r = bench.row(1536, 4000, 8, 1.9e6, 9.0e-3)
    return bench.sig({
        "metric": "kde_queries_per_s_at_1e-2_mean_rel_err", "value": 1.94e6,
        "unit": "queries/s", "n_gpus": 1, "steps": 20, "warmup": 5, "ms_per_step": 5.15,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": bench.WORKLOAD, "kernel": "gaussian", "h": 12.806247, "k": 1536,
                   "m": 4000, "nprobe": 8, "scan_precision": "bf16",
                   "parallelism": "replicas x1", "l2": "inputs > L2 (X 512 MB)"},
        "mean_rel_err": 0.0090123, "max_step_rel_err": 0.0091234, "meets_target": True,
        "val_rel_err": 0.0087654,
        "e2e": {"value": 1.91e6, "unit": "queries/s", "h2d_bytes_per_step": 5120000,
                "d2h_bytes_per_step": 40000},
        "gpu_launches": 480,
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 7},
        "roofline": {"bound": "hbm", "achieved": 7412.3456, "peak": 6781.4, "unit": "GB/s",
                     "frac": 1.0930123, "traffic": 17212345678, "stage": "estimate",
                     "ms_per_call": 2.7712345, "t_min_ms": 3.0212345,
                     "peak_source": "measured hbm_gbs"},
        "stage_ms_per_step": {s: 1.2345678 for s in ("stage", "coarse", "plan", "scan",
                                                     "select", "estimate")},
        "path_roofline": {"frac": 0.8912345, "t_min_ms": 4.5712345, "frac_method": 0.8512345},
        "cpu_baseline": {"value": 1321.12345, "unit": "queries/s", "cores": 16, "kind": "oracle",
                         "sample": "10000 test queries, IVF search + DEANN, FP64, 12.3 s",
                         "single_thread_qps": 72.512345},
        "baselines": {"exact": {"qps": 551234.5, "tflops_algorithmic": 141.23456,
                                "frac_algorithmic": 0.0741234, "split_products": 6,
                                "peak": 1901.8},
                      "rs_qps": 12612.345, "rs_m": 1310720, "rs_rel_err": 0.0089123,
                      "scans": {"fp32": r, "bf16": r, "bf16x3": r}, "deannp": r},
        "forms": {"fixed_params_exp": {"deannp_qps": 2.5e6, "deannp_err": 0.036,
                                       "deann_qps": 2.1e6, "deann_err": 0.04, "recall": 0.83},
                  "recall": 0.9912345, "adjoint": {"qps": 2.02e6, "frac": 0.84123},
                  "mean_shift_qsteps": 6.8e6, "exponential": {"row": r, "exact_qps": 91234.5},
                  "d784": {"exact_qps": 121234.0, "fp32_fixed": r, "fp32": r, "bf16_fixed": r,
                           "bf16": r, "bf16x3_fixed": r, "bf16x3": r, "same_nbrs": True},
                  "n4M_batched": {"fixed": r, "tuned": r,
                                  "one_call_qps": [1.45123e6, 1.41234e6],
                                  "with_backward_qps": [1.09123e6, 1.31234e6]}},
        "margin_failures": 0, "build_s": 3.2123456,
    }, 4)


def test_headline_line_fits_the_driver_tail():
    """The full headline fits in the bytes kept for it and the forms summary
    printed before it in its own; together they fit the driver's 3 KB tail.
    When the headline would not fit, optional sections move to a side line and
    the required keys stay."""
    import json
    line = _representative_headline()
    forms = dict(line.pop("forms"), row_fields=bench.ROW_FIELDS)
    text, moved = bench.fit_headline(line)
    assert moved == {} and len(text) <= bench.HEADLINE_LIMIT, len(text)
    ftext = json.dumps({"side": "forms", **bench.sig(forms, 4)})
    assert len(ftext) <= bench.FORMS_LIMIT, len(ftext)
    assert len(text) + len(ftext) + 40 <= 3000
    text, moved = bench.fit_headline(line, limit=1500)
    assert len(text) <= 1500 and "baselines" in moved
    got = json.loads(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "dtype", "config", "e2e", "clocks", "roofline",
                "cpu_baseline", "gpu_launches"):
        assert key in got
