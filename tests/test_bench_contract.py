"""The benchmark's output contract, checked on the CPU: the reference arm's JSON line (the FP64
oracle timed on the host cores) and the algorithmic work counted per particle-step."""
import json
import os
import subprocess
import sys

import pytest

import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line_with_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--ref-samples", "4"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["unit"] == "particle-steps/s" and d["value"] > 0
    assert d["config"]["workload"] == "racing_K4096_M64_T40"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_work_per_particle_step():
    """Counted from the method's formulas: the bicycle's 5 substeps, 6 Gaussians (1.5 Philox calls,
    3 Box-Muller pairs), the disturbance and the moment sums."""
    import bench
    assert bench.algorithmic_flops_per_particle_step(workload.config1()) == 967.0
    assert bench.algorithmic_flops_per_particle_step(workload.double_integrator_problem(1, 2, 1)) == 213.0
    p = workload.config1()
    p.n_sub = 10  # the model term scales with the substeps, nothing else does
    assert bench.algorithmic_flops_per_particle_step(p) - 967.0 == 5 * 131  # 131 per Euler substep


@pytest.mark.parametrize("world,ms,expect", [(1, 0.5, 2 * 4096 * 64 * 40 * 1e3 / 2 / 0.5),
                                             (4, 1.0, 4 * 4096 * 64 * 40 * 1e3 / 1.0)])
def test_whole_job_throughput(world, ms, expect):
    import bench
    assert bench.whole_job_throughput(4096 * 64 * 40, ms, world) == pytest.approx(expect)


def test_gpus_flag_must_match_the_launchers_rank_count():
    """--gpus N under a launcher that started another number of ranks fails loudly (it never prints
    a line for the wrong number of GPUs)."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "4", "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--ref-samples", "4"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, env=env)
    assert out.returncode != 0 and "WORLD_SIZE" in out.stderr
    assert not out.stdout.strip()


def test_gpus_flag_without_a_launcher_starts_that_many_ranks():
    """--gpus 2 without torchrun re-launches the script as two ranks (here the reference arm, which
    only rank 0 runs and prints); the line reports both ranks."""
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl", "reference",
                          "--steps", "1", "--warmup", "3", "--ref-samples", "4"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(l) for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def test_cpu_baseline_reports_all_cores_and_one_thread():
    import bench
    import oracle
    p = workload.config0()
    r = bench.run_cpu_baseline(p, budget_s=0.5)
    assert r["kind"] == "oracle" and r["cores"] == oracle.host_threads() and r["value"] > 0
    assert r["one_thread"]["cores"] == 1 and r["one_thread"]["value"] > 0
    assert r["cpu"]
