"""Serving loop (tq_server): continuous batching of circuit requests. Each
request's result must match the single-state path (FP64: bitwise for
requests resident in shared memory, whose arithmetic per group is identical; within
1e-12 for the others), admission must respect the HBM budget,
and results must match the oracle."""
import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
SPLIT_Z = 1e-5              # stated split-precision bound on <Z> (trace-renormalised)
SPLIT_TRACE_DRIFT = 1e-5    # stated bound on |Tr rho - 1| before renormalisation


def _requests(count, seed, n_lo=2, n_hi=9):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        c = W.served_request(rng, n_min=n_lo, n_max=n_hi, d_min=10, d_max=80)
        out.append((c.n, c.ops, [1, (1 << c.n) - 1]))
    return out


def _single(tq, precision, n, ops, masks):
    # FP64: the same canonical-group DFMA arithmetic as the batch kernel
    with tq.State(n, precision, hermitian=precision == "fp64", engine="dfma") as st:
        st.run(ops, width=2)
        tr = st.trace()
        return np.concatenate([[tr.real, tr.imag], st.expect_z(masks)])


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_served_results_same_alone_and_in_mix(tq, precision):
    reqs = _requests(16, 5)
    srv = tq.Server(precision, rho_budget=64 << 20, max_live=6)
    ids = []
    # arrivals spread over ticks: four requests join before every tick
    pending = list(range(len(reqs)))
    done = {}
    ticks = 0
    while (pending or len(done) < len(reqs)) and ticks < 10000:
        for _ in range(4):
            if pending:
                k = pending.pop(0)
                n, ops, masks = reqs[k]
                ids.append((k, srv.submit(n, ops, width=2, masks=masks)))
        live, queued, fin = srv.step()
        assert live <= 6
        ticks += 1
        for k, rid in ids:
            if k not in done:
                st, res = srv.poll(rid)
                if st == 2:
                    done[k] = res
    assert len(done) == len(reqs)
    assert srv.info()["rho_live_bytes"] == 0
    for k, (n, ops, masks) in enumerate(reqs):
        alone = _single(tq, precision, n, ops, masks)
        got = done[k].copy()
        want = O.run_circuit(n, ops)
        if precision == "split":
            # <Z> of both split paths is already divided by the trace
            assert np.max(np.abs(got - alone)) < 1e-6
            assert abs(got[0] - O.trace(want).real) < SPLIT_TRACE_DRIFT
            for i, m in enumerate(masks):
                assert abs(got[2 + i] - O.expect_z(want, m)) < SPLIT_Z, (k, i)
        else:
            if 16 * 4 ** n <= 64 * 1024:
                assert np.array_equal(got, alone), k    # resident: the same DFMA arithmetic, same order
            else:
                assert np.max(np.abs(got - alone)) < TOL64, k   # tile jobs: width-2 blocks may run in the Pauli basis
            assert abs(got[0] - O.trace(want).real) < TOL64
            for i, m in enumerate(masks):
                assert abs(got[2 + i] - O.expect_z(want, m)) < TOL64
    srv.free()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_pipelined_ticks_give_the_same_results(tq, precision):
    # tq_server_step_async collects the previous tick and launches the next
    # without waiting; every request's result equals the synchronous run's
    reqs = _requests(12, 7)
    runs = []
    for mode in ("sync", "async"):
        srv = tq.Server(precision, rho_budget=64 << 20, max_live=5)
        ids = [srv.submit(n, ops, width=2, masks=masks) for n, ops, masks in reqs[:6]]
        pending = list(reqs[6:])
        done, ticks = {}, 0
        while len(done) < len(reqs) and ticks < 10000:
            if pending:
                n, ops, masks = pending.pop(0)
                ids.append(srv.submit(n, ops, width=2, masks=masks))
            live, queued, fin = srv.step() if mode == "sync" else srv.step_async()
            assert live <= 5
            ticks += 1
            for k, rid in enumerate(ids):
                if k not in done:
                    st, res = srv.poll(rid)
                    if st == 2:
                        done[k] = res
        assert len(done) == len(reqs)
        assert srv.info()["rho_live_bytes"] == 0 and srv.gpu_ms() > 0
        runs.append(done)
        srv.free()
    for k in range(len(reqs)):
        if precision == "fp64":
            assert np.array_equal(runs[0][k], runs[1][k]), k
        else:
            assert np.max(np.abs(runs[0][k] - runs[1][k])) < 1e-6, k


def test_admission_respects_the_hbm_budget(tq):
    # room for exactly two 8-qubit FP64 density matrices (1 MiB each): at most
    # two requests can be admitted (and so finish) per tick
    srv = tq.Server("fp64", rho_budget=2 << 20, max_live=8)
    c = W.random_noisy_circuit(8, 30, 9)
    ids = [srv.submit(8, c.ops, width=2, masks=[3]) for _ in range(5)]
    finished_per_tick = []
    guard = 0
    while any(srv.poll(i)[0] != 2 for i in ids) and guard < 1000:
        live, queued, fin = srv.step()
        finished_per_tick.append(fin)
        assert live + fin <= 2
        assert srv.info()["rho_live_bytes"] <= 2 << 20
        guard += 1
    assert max(finished_per_tick) == 2 and len(finished_per_tick) == 3
    want = O.run_circuit(8, c.ops)
    for i in ids:
        st, res = srv.poll(i)
        assert st == 2 and abs(res[2] - O.expect_z(want, 3)) < TOL64
    with pytest.raises(tq.TqError) as e:
        srv.submit(10, c.ops, width=2)                 # 16 MiB can never fit a 2 MiB budget
    assert e.value.status == 3                          # TQ_ERR_OOM
    srv.free()


def test_long_requests_stay_live_across_ticks(tq):
    # 12-qubit requests advance 8 blocks per tick: they stay resident over
    # several ticks while short ones arriving later finish first
    srv = tq.Server("fp64", rho_budget=1 << 30, max_live=8)
    long_c = W.random_noisy_circuit(12, 200, 21, gate_set=("h", "rz", "cx"))
    short_c = W.random_noisy_circuit(5, 20, 22)
    a = srv.submit(12, long_c.ops, width=2, masks=[1])
    srv.step()
    assert srv.poll(a)[0] == 1
    b = srv.submit(5, short_c.ops, width=2, masks=[1])
    srv.step()
    assert srv.poll(b)[0] == 2 and srv.poll(a)[0] == 1
    guard = 0
    while srv.poll(a)[0] != 2 and guard < 1000:
        srv.step()
        guard += 1
    res = srv.poll(a)[1]
    with tq.State(12, "fp64") as st:
        st.run(long_c.ops, width=2)
        assert abs(res[2] - st.expect_z([1])[0]) < TOL64   # readouts reduce in a different order
    srv.free()


def test_submit_rejects_tables_beyond_the_table_budget(tq):
    # a request whose superoperator tables can never fit the table arena is
    # refused at submit (it would otherwise block the FIFO head for good);
    # smaller requests queued behind the refused one still run
    srv = tq.Server("fp64", rho_budget=64 << 20, table_budget=256 << 10, max_live=4)
    big = W.random_noisy_circuit(6, 400, 31)       # > 100 fused 4 KiB superoperators alone
    with pytest.raises(tq.TqError) as e:
        srv.submit(6, big.ops, width=2, masks=[1])
    assert e.value.status == 3                          # TQ_ERR_OOM
    small = W.random_noisy_circuit(4, 5, 32)     # tables of a few superoperators: well below 256 KiB
    rid = srv.submit(4, small.ops, width=2, masks=[1])
    guard = 0
    while srv.poll(rid)[0] != 2 and guard < 100:
        srv.step()
        guard += 1
    st, res = srv.poll(rid)
    want = O.run_circuit(4, small.ops)
    assert st == 2 and abs(res[2] - O.expect_z(want, 1)) < TOL64
    srv.free()


def test_submit_rejects_blocks_wider_than_two_qubits(tq):
    # the serving loop applies blocks of at most 2 qubits: a fusion width
    # above 2, or an op on 3 qubits, is refused at submit and queues nothing;
    # a valid request submitted afterwards still runs
    srv = tq.Server("fp64", rho_budget=64 << 20, table_budget=16 << 20, max_live=4)
    c = W.random_noisy_circuit(4, 10, 33)
    with pytest.raises(tq.TqError) as e:
        srv.submit(4, c.ops, width=3, masks=[1])
    assert e.value.status == 7                          # TQ_ERR_UNSUPPORTED
    U = np.eye(8, dtype=complex)
    with pytest.raises(tq.TqError) as e:
        srv.submit(4, [("unitary", [0, 1, 2], [U])], width=2, masks=[1])
    assert e.value.status == 7
    rid = srv.submit(4, c.ops, width=2, masks=[1])
    guard = 0
    while srv.poll(rid)[0] != 2 and guard < 100:
        srv.step()
        guard += 1
    st, res = srv.poll(rid)
    want = O.run_circuit(4, c.ops)
    assert st == 2 and abs(res[2] - O.expect_z(want, 1)) < TOL64
    srv.free()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_large_requests_run_through_single_state_kernels(tq, precision):
    # requests of >= 12 qubits advance by single-state launches (tensor cores:
    # split width 2, and FP64 with the tensor engine) after the tick's batch
    # kernel, while small ones stay in it; every result must equal the
    # request's single-state run (FP64: the DFMA engine, held to the oracle
    # by the parity tests) within the precision's tolerance
    rng = np.random.default_rng(41)
    reqs = []
    for n, depth in ((12, 12), (5, 40), (13, 6), (7, 30), (12, 10)):
        c = W.served_request(rng, n_min=n, n_max=n, d_min=depth, d_max=depth)
        reqs.append((n, c.ops, [1, 3, (1 << n) - 1]))
    srv = tq.Server(precision, rho_budget=8 << 30, max_live=3, engine="tensor")
    ids = [srv.submit(n, ops, width=-1, masks=m) for n, ops, m in reqs]
    guard = 0
    while any(srv.poll(i)[0] != 2 for i in ids) and guard < 5000:
        srv.step_async()
        guard += 1
    srv.step()
    tol = TOL64 if precision == "fp64" else 1e-6
    for (n, ops, masks), rid in zip(reqs, ids):
        st_, got = srv.poll(rid)
        assert st_ == 2
        with tq.State(n, precision, engine="dfma") as st:
            st.run(ops, width=-1)
            tr = st.trace()
            want = np.concatenate([[tr.real, tr.imag], st.expect_z(masks)])
        assert np.max(np.abs(got - want)) < tol, (n, np.max(np.abs(got - want)))
    srv.free()
