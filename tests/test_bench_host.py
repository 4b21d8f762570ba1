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
    total, sample, full = bench.cpu_baseline_circuits(cs, budget_per_n=1e9, full_count=0)
    # with an unbounded budget each size's first circuit runs whole, so the
    # estimate is (that circuit's time / its ops) x the ops of all circuits of that size
    assert total > 0.0 and full == {}
    assert "n=3" in sample and "n=4" in sample
    assert f"{len(cs[0].ops)} ops at n=3" in sample   # the first 3-qubit circuit is the sample
    rho = O.run_circuit(3, cs[2].ops)                   # the sampled circuits still run on the oracle
    assert abs(O.trace(rho).real - 1.0) < 1e-12


def test_sweep_whole_circuit_sample_keeps_the_oracle_readouts():
    cs = [W.random_noisy_circuit(n, d, 30 + i) for i, (n, d) in enumerate([(3, 20), (7, 5), (4, 10), (2, 8)])]
    total, sample, full = bench.cpu_baseline_circuits(cs, budget_per_n=1e9, masks=(1, 3), full_max_n=4, full_count=2)
    # the first two circuits of at most 4 qubits run whole: indices 0 and 2
    assert sorted(full) == [0, 2] and "2 whole circuits" in sample
    rho = O.run_circuit(4, cs[2].ops)
    assert abs(full[2][0] - O.trace(rho).real) < 1e-15
    assert abs(full[2][2] - O.expect_z(rho, 1)) < 1e-15 and abs(full[2][3] - O.expect_z(rho, 3)) < 1e-15
    assert "n=7" in sample and "n=2" in sample         # the other sizes still get a prefix timing
    assert total > 0.0


def test_gate_slices_attach_channels_to_their_gate():
    ops = [("h", [0], ()), ("depol", [0], (1e-3,)), ("ad", [0], (1e-4,)), ("cx", [0, 1], ()),
           ("depol", [0, 1], (1e-2,)), ("rz", [1], (0.3,))]
    g = bench.gate_slices(ops)
    assert [len(x) for x in g] == [3, 2, 1] and g[1][0][0] == "cx"


def test_served_speedup_counts_only_completed_requests():
    serve = {"_completed": [(5, 100), (6, 200)], "wall_s": 2.0}
    plain = {5: (1.0, 50), 6: (2.0, 50)}              # ms per gate
    r = bench.served_vs_plain(serve, plain)
    assert abs(r["plain_fp64_s_for_completed"] - 0.5) < 1e-12   # 100 x 1 ms + 200 x 2 ms
    assert abs(r["speedup_vs_plain_fp64"] - 0.25) < 1e-12
    assert abs(r["plain_fp64_circuits_per_s"] - 4.0) < 1e-12


def test_oracle_tfim_zz_reads_each_step_of_the_ring_circuit():
    # one <Z0 Z1> per Trotter step, equal to the oracle run step by step
    zz = bench.oracle_tfim_zz(4, 3)
    c = W.tfim_ring(4, 3)
    rho = O.zero_state(4)
    want = []
    for a, b in c.steps:
        for op in c.ops[a:b]:
            rho = O.apply_op(rho, op)
        want.append(float(O.expect_z(rho, bench.ZZ_MASK)))
    assert zz == want and len(zz) == 3
    assert all(abs(z) <= 1.0 for z in zz) and zz[0] > 0.9   # |0000> starts at <Z0 Z1> = 1; small dt
