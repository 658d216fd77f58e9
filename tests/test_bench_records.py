"""The measurement records bench.py reads are consistent with the sources (CPU):
the committed DRAM-traffic record was captured on the current sweep source (so a
change to the sweeps without a new ncu capture reports traffic as unknown, not
stale), and the oracle's operation counts of the benchmark workload match its
recorded trace."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_record_matches_the_sweep_source():
    bench = load_bench()
    rec = bench.traffic_record()
    assert rec is not None, "sweep.cuh changed since the ncu traffic capture: recapture it"
    algorithmic = 4 * 4096 * 4096  # FP32 cost bytes of one sweep at n = m = 4096
    for k in ("cg_row_sweep", "cg_col_sweep"):
        t = rec["dram_bytes_per_launch"][k]
        assert algorithmic <= t <= 1.05 * algorithmic, (k, t)


def test_reference_arm_uses_the_recorded_oracle_trace():
    bench = load_bench()
    trace = json.load(open(os.path.join(ROOT, "tests", "golden", "grid4096_oracle_trace.json")))
    t = trace["sqeuclid"]
    ops = bench.oracle_ops_of_workload()
    # priced as CG steps: the recorded CG iterations plus Alg. 2's two outer
    # products per Newton step; everything else as LSE updates
    assert ops["cg_like"] == t["cg_iters"] + 2 * t["newton_steps"]
    assert ops["lse_like"] == 2 * t["stages"] + 2 * t["newton_steps"] + t["ls_trials"] + 2 * t["sinkhorn_iters"]
    assert t["cg_iters"] > 0 and t["stages"] > 0
    # the estimate prices those counts at the sampled per-operation times
    est = bench.oracle_estimate({"t_lse": 2.0, "t_cg": 0.5}, ops)
    assert est == 2.0 * ops["lse_like"] + 0.5 * ops["cg_like"]
