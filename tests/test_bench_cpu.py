"""bench.py's reference arm on the host (no GPU): one JSON line with the contract's keys, and
under a multi-rank launch only rank 0 prints it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_the_contract_line():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    res = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in res, key
    assert res["impl"] == "reference" and res["steps"] == 2 and res["warmup"] == 1
    assert res["value"] > 0 and res["higher_is_better"] is True
    cb = res["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == res["value"] and cb["cores"] >= 1 and cb["sample"]
    assert 0 < cb["cores_busy"] <= cb["cores"] + 0.5
    e2e = res["e2e"]
    assert e2e["value"] == res["value"] and e2e["unit"] == res["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "workload" in res["config"]


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_cpu_baseline_leg_measures_busy_cores():
    """The oracle leg of the GPU arm (run here on a small cell): the oracle's Davidson on at
    least one k-point, whose eigenvalues are the dense ones to the metric's 1e-8 Ry."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle import hamiltonian as ham
    from paper_2412_01695_gb300 import synth
    prob = synth.make_config(1)
    res, eigs = bench.cpu_baseline(prob, budget_s=0.5)
    assert res["kind"] == "oracle" and res["value"] > 0 and len(eigs) >= 1
    assert 0 < res["cores_busy"] <= res["cores"] + 0.5
    for ik, e in eigs.items():
        w = np.linalg.eigvalsh(ham.problem_h(prob, ik))[:prob.nb]
        assert np.max(np.abs(e - w)) <= bench.EIG_TOL


def test_traffic_figures_name_their_profile_and_sources():
    """Every DRAM-traffic figure bench.py reports comes from a profile summary under
    profiles/ and names the kernel sources whose digest gates it (a figure whose sources
    changed since the capture is reported as null)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    assert b.TRAFFIC
    for name, t in b.TRAFFIC.items():
        assert t["bytes"] > 0, name
        assert os.path.isfile(os.path.join(ROOT, t["profile"])), (name, t["profile"])
        for src in t["sources"]:
            assert os.path.isfile(os.path.join(ROOT, "paper_2412_01695_gb300", "csrc", src)), (name, src)
        assert len(t["digest"]) == 12
        got = b.traffic_for(name)
        assert got == (None, None) or got == (t["bytes"], t["profile"])
