"""The CPU arm of bench.py (the oracle as the reference implementation) keeps the JSON
contract: one line with the metric, unit, value, timing and baseline fields; ranks other
than 0 of a torchrun launch exit 0 without printing.  Runs on the host only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")


def _run(extra_env=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.update(extra_env or {})
    cmd = [sys.executable, BENCH, "--impl", "reference", "--workload", "born", "--steps", "3",
           "--warmup", "3", "--ref-rows", "16"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "Mnode/s" and d["higher_is_better"] is True
    assert d["steps"] == 3 and d["warmup"] == 3 and d["value"] > 0
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert "workload" in d["config"] and "2562 nodes" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_oracle_near_setup_timing_covers_the_oracle_near_set():
    """The bench's separately timed oracle near-field setup samples whole near sets: with
    every row of a small mesh sampled it times exactly the oracle's near CSR entries."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import synthetic
    mol = synthetic.born_ion()
    rate, rows, entries, dt = bench.oracle_near_rate(mol, seconds=60.0)
    assert rows == mol.n_nodes and rate > 0 and dt > 0
    rp, _, _ = oracle.Oracle.for_molecule(mol).near_csr()
    assert entries == rp[-1]
