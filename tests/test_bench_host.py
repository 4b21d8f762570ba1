"""Host-side helpers of bench.py that need no GPU: the bounded CPU-oracle
samples behind the cpu_baseline objects of the workload lines."""
import bench
from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W


def test_oracle_prefix_runs_at_least_min_ops_and_stops_on_budget():
    c = W.random_noisy_circuit(4, 30, 11)
    done, dt = bench.oracle_prefix_time(c.n, c.ops, 0.0, min_ops=3)
    assert done == 3 and dt >= 0.0                  # budget already spent: the minimum only
    done, _ = bench.oracle_prefix_time(c.n, c.ops, 1e9)
    assert done == len(c.ops)                       # generous budget: the whole circuit


def test_sweep_estimate_scales_per_size_op_times_by_each_circuits_ops():
    cs = [W.random_noisy_circuit(n, d, 20 + i) for i, (n, d) in enumerate([(3, 20), (4, 10), (3, 40)])]
    total, sample = bench.cpu_baseline_circuits(cs, budget_per_n=1e9)
    # with an unbounded budget each size's first circuit runs whole, so the
    # estimate is (that circuit's time / its ops) x the ops of all circuits of that size
    assert total > 0.0
    assert "n=3" in sample and "n=4" in sample
    assert f"{len(cs[0].ops)} ops at n=3" in sample   # the first 3-qubit circuit is the sample
    rho = O.run_circuit(3, cs[2].ops)                   # the sampled circuits still run on the oracle
    assert abs(O.trace(rho).real - 1.0) < 1e-12
