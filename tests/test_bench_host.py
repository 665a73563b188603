"""The benchmark's host-side contract on CPU: the reference arm (the FP64 oracle timed on
the host) prints one JSON line with the contract's keys, only rank 0 prints under a
multi-rank launch, and the roofline byte counts follow the per-pass formulas."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline", "impl"}


def _run(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_the_contract_line():
    p = _run({}, "--impl", "reference", "--workload", "vol32_iso9_n3_k3", "--steps", "2", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert KEYS <= set(rec)
    assert rec["impl"] == "reference" and rec["steps"] == 2 and rec["warmup"] == 1
    assert rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert rec["config"]["workload"] == "vol32_iso9_n3_k3"


def test_reference_arm_other_ranks_print_nothing():
    p = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference",
             "--workload", "vol32_iso9_n3_k3", "--steps", "1", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_algorithmic_bytes_formulas():
    sys.path.insert(0, ROOT)
    import bench

    class Vol:
        n = (64, 64, 64)

    class PlanInfo:
        K = 15
        precision = "fp32"
        info = {"E": (78, 78, 94), "P_conv": (80, 80, 96), "P_cert": (128, 128, 128), "real_table": True}

    V, VE, H2, H2c = 64 ** 3, 78 * 78 * 94, 49, 65
    ab = lambda tag: bench.algorithmic_bytes(tag, PlanInfo, Vol)   # noqa: E731
    # certificate axis 0: input spectrum + real FP32 table + K output spectra
    assert ab("cert_axis0") == 64 * 128 * H2c * 8 + 15 * 128 * 128 * H2c * 4 + 15 * 64 * 128 * H2c * 8
    assert ab("cert_tail") == 15 * 64 * 128 * H2c * 8
    assert ab("blur_head") == VE * 4 + 78 * 80 * H2 * 8
    assert ab("blur_tail") == 64 * 80 * H2 * 8 + V * 8
    assert ab("bp_head") == V * 4 + 64 * 80 * H2 * 8
    assert ab("bp_tail") == 78 * 80 * H2 * 8 + VE * 4
    assert ab("not_a_pass") == 0.0


@pytest.mark.parametrize("tag", ["cert_axis0_tc", "cert_c2r_tc", "cert_axis0"])
def test_traffic_record_matches_sources_or_is_ignored(tag):
    """The committed DRAM bytes are used only for their workload, while the kernel sources
    still match the digest they were captured on, and only for the tags they cover."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "dram_traffic.json")))
    got = bench.ncu_traffic(tag, rec["workload"])
    if rec["source_digest"] == bench.source_digest() and tag in rec["bytes_per_launch"]:
        assert got == rec["bytes_per_launch"][tag]
    else:
        assert got is None
    assert bench.ncu_traffic(tag, "another_workload") is None


def test_clock_summary_parses_samples_and_reasons(tmp_path):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0, str(tmp_path))
    assert c.path == str(tmp_path / "clocks_rank0.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2040, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    open(c.path, "w").write("\n".join(rows) + "\n")
    c.proc = object()          # as if nvidia-smi had run
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.proc = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_bounds_many_steps():
    """With more steps than whole oracle steps fit in the time budget, each step is a sample
    of grid candidates evaluated by the oracle's direct sums, and the run stays bounded."""
    import time
    t0 = time.perf_counter()
    p = _run({"SFW_REF_BUDGET_S": "2"}, "--impl", "reference", "--workload", "vol32_iso9_n3_k3",
             "--steps", "400", "--warmup", "3")
    assert p.returncode == 0, p.stderr[-2000:]
    assert time.perf_counter() - t0 < 60
    rec = json.loads([l for l in p.stdout.splitlines() if l.startswith("{")][0])
    assert rec["steps"] == 400 and rec["value"] > 0
    assert rec["config"]["candidates_per_step"] >= 1
    assert "direct sums" in rec["cpu_baseline"]["sample"]
