"""Host logic of bench.py that needs no GPU: the clock and throttle-reason
summary taken from nvidia-smi samples during the timed region."""
import bench

IDLE = "2070, 2070, 950.12, 0x0000000000000000, Not Active, Not Active, " \
       "Not Active, Not Active"


def line(sm, reasons=()):
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
             "sw_power_cap")
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return ", ".join([str(sm), "2070", "1200.5", "0x4"] + flags)


def test_median_clock_and_no_reasons():
    out = bench.parse_clock_lines([line(2070), line(2055), line(1980)])
    assert out == {"sm_mhz": 2055, "sm_max_mhz": 2070.0, "reasons": [],
                   "samples": 3}
    assert bench.parse_clock_lines([IDLE])["reasons"] == []


def test_every_active_reason_is_reported_once():
    out = bench.parse_clock_lines([
        line(1900, ("sw_power_cap",)), line(1850, ("hw_slowdown",)),
        line(1870, ("sw_power_cap", "sw_thermal_slowdown"))])
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap",
                              "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1870


def test_malformed_and_unavailable_samples_are_skipped():
    out = bench.parse_clock_lines([
        "", "clocks.current.sm [MHz], clocks.max.sm [MHz]",
        "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        line(2070)])
    assert out["samples"] == 1 and out["sm_mhz"] == 2070
    assert bench.parse_clock_lines([])["sm_mhz"] is None


def run_bench(*args, nproc=1):
    import json
    import socket
    import subprocess
    import sys
    cmd = [sys.executable, bench.__file__]
    if nproc > 1:
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
               f"--nproc-per-node={nproc}", "--master-addr", "127.0.0.1",
               "--master-port", str(port), bench.__file__]
    p = subprocess.run(cmd + list(args), capture_output=True, text=True,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_contract_line():
    """The reference arm (the FP64 oracle on the host cores, a bounded
    sample of the workload per step) needs no GPU."""
    (line,) = run_bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert line["impl"] == "reference"
    for key in ("metric", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data",
                "config"):
        assert key in line, key
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["metric"] == bench.METRIC and line["higher_is_better"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    lines = run_bench("--impl", "reference", "--gpus", "2", "--steps", "1",
                      "--warmup", "0", nproc=2)
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_study_jobs_and_aggregation(monkeypatch, capsys):
    """bench.py --study: the paper's configurations become the right runs,
    and the per-configuration summaries (worst error over the models, the
    dynamic-vs-fixed counts and geometric mean) are formed correctly; the
    GPU runs are replaced by a fake that returns known errors."""
    import argparse
    import json
    import math

    seen = []

    def fake(job, span):
        seen.append(job)
        k = len(job["seeds"])
        base = [1e-3 * (1 + s % 10) for s in job["seeds"]]
        if job["era"] == "dynamic":
            # half the fixed era's error for three models, twice for seven
            worst = [b * (0.5 if s % 10 < 3 else 2.0)
                     for b, s in zip(base, job["seeds"])]
        else:
            worst = base
        return dict(job, worst=worst, at_end=[0.0] * k, block_steps=10 * k,
                    seconds=0.0)
    monkeypatch.setattr(bench, "study_job", fake)
    args = argparse.Namespace(study_span=3, study_precision="fp64",
                              study_workers=2, study_only="", study_eras="")
    assert bench.study(args) == 0
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    res = out["results"]["fp64"]
    # Sec. 3: 5 eras x 2 pass counts (100 bodies), 7 eras (500 bodies)
    assert len(res["sec3_n100"]) == 10 and len(res["sec3_n500"]) == 7
    assert sum(j["n"] == 100 and j["study"] == "sec3_n100" for j in seen) == 10
    # Sec. 4: one fixed-era ensemble of ten models + ten dynamic runs, twice
    dyn = [j for j in seen if j["era"] == "dynamic"]
    assert len(dyn) == 20 and all(len(j["seeds"]) == 1 for j in dyn)
    s4 = res["sec4_n100"]
    assert s4["models"] == 10 and s4["dynamic_at_most_fixed"] == 3
    assert math.isclose(s4["geomean_ratio_dynamic_over_fixed"], 2.0 ** 0.4)
    assert math.isclose(s4["worst_fixed"], 1e-2)
    assert math.isclose(s4["worst_dynamic"], 2e-2)
    assert out["runs"] == len(seen) == 39


def test_study_selection(monkeypatch, capsys):
    import argparse
    import json
    seen = []

    def fake(job, span):
        seen.append(job)
        k = len(job["seeds"])
        return dict(job, worst=[1e-3] * k, at_end=[0.0] * k, block_steps=1,
                    seconds=0.0)
    monkeypatch.setattr(bench, "study_job", fake)
    args = argparse.Namespace(study_span=2, study_precision="both",
                              study_workers=2, study_only="sec3_n100",
                              study_eras="0.25")
    assert bench.study(args) == 0
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    # three and five passes at era 1/4, in both precisions
    assert len(seen) == 4
    assert {(j["n_iter"], j["era"], j["precision"]) for j in seen} == {
        (3, 0.25, "fp64"), (5, 0.25, "fp64"), (3, 0.25, "mixed"),
        (5, 0.25, "mixed")}
    assert set(out["results"]["mixed"]) == {"sec3_n100"}
