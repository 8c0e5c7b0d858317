"""The bench's CPU legs (CPU only): the block-parallel oracle baseline (one
spawned process per core, the field shared through shared memory) and the
reference arm's JSON line (rank 0 prints it, other ranks print nothing)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_parallel_oracle_baseline():
    sys.path.insert(0, ROOT)
    import bench
    x = np.random.default_rng(0).standard_normal(1 << 18).astype(np.float32)
    msgs = [(np.random.default_rng(i).standard_normal(5000).astype(np.float32), 1e-3)
            for i in range(3)]
    r = bench.cpu_parallel(x, msgs, x.size)
    assert r["unit"] == "GB/s" and r["value"] > 0
    assert r["cores"] == (os.cpu_count() or 1)
    assert "%d segments" % r["cores"] in r["sample"]


def _reference(env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--side", "32", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    sys.path.insert(0, ROOT)
    import bench
    (line,) = _reference({"WORLD_SIZE": "1", "RANK": "0"})
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "GB/s" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["config"]["workload"].startswith("grf512_rel1e-3_L32")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "sample" in cb
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_print_nothing():
    assert _reference({"WORLD_SIZE": "2", "RANK": "1"}) == []
