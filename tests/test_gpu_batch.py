"""Batched execution (tq_batch): many independent circuits in one persistent
launch captured in a CUDA graph. Each job must match the oracle (FP64
1e-12) and the single-state path, alone and in the mix."""
import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _jobs(count, n_lo, n_hi, seed, depth=(10, 40)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(*depth))
        p = float(10 ** rng.uniform(-4, -2))
        c = W.random_noisy_circuit(n, d, int(rng.integers(1 << 30)), gate_set=("h", "rz", "rx", "cx", "su2"),
                                   p1=p, p2=p, gamma=1e-3)
        masks = [1, (1 << n) - 1] + ([0b11] if n > 1 else [])
        out.append((n, c.ops, masks))
    return out


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_batch_matches_oracle_and_replays(tq, precision):
    jobs = _jobs(24, 2, 8, 1)        # resident (n <= 6) and tiled (7, 8) jobs
    b = tq.Batch(precision)
    for n, ops, masks in jobs:
        b.add(n, ops, width=-1, masks=masks)
    tol = TOL64 if precision == "fp64" else 2e-6
    for rep in range(2):                 # first run captures the graph, the second replays it
        b.run()
        b.wait()
        info = b.info()
        assert info["jobs"] == len(jobs) and info["items"] > 0
        for j, (n, ops, masks) in enumerate(jobs):
            want = O.run_circuit(n, ops)
            got = b.rho(j)
            assert np.max(np.abs(got - want)) < tol, (rep, j, n)
            res = b.result(j)
            assert abs(res[0] - O.trace(want).real) < (TOL64 if precision == "fp64" else 1e-5)
            for i, m in enumerate(masks):
                wz = O.expect_z(want, m) / (1.0 if precision == "fp64" else O.trace(want).real)
                assert abs(res[2 + i] - wz) < (TOL64 if precision == "fp64" else 1e-5)
    b.free()


def _block_superops(tq, n, ops, width, precision):
    """(width, superoperator) of every fused block, composed with numpy from
    the library's gate matrices in the planner's blocks (local order: the
    qubits as they first appear; local index r + 2^w c, bit j = qubit j)."""
    block_of, widths = tq.plan_fusion(n, ops, width, precision)
    out = []
    for b, w in enumerate(widths):
        members = [ops[i] for i in range(len(ops)) if block_of[i] == b]
        qs = []
        for _, q, _ in members:
            for v in q:
                if v not in qs:
                    qs.append(v)
        D = 4 ** w
        S = np.eye(D, dtype=complex)
        for name, q, params in members:
            U = tq.gate_matrix(name, params)
            k = len(q)
            So = np.kron(U.conj(), U)                     # local index r + 2^k c of the op
            pos = [qs.index(v) for v in q]
            E = np.zeros((D, D), dtype=complex)
            for i in range(D):
                for j in range(D):
                    if any(((i >> t) & 1) != ((j >> t) & 1) or ((i >> (w + t)) & 1) != ((j >> (w + t)) & 1)
                           for t in range(w) if t not in pos):
                        continue
                    li = sum((((i >> pos[t]) & 1) << t) | (((i >> (pos[t] + w)) & 1) << (k + t)) for t in range(k))
                    lj = sum((((j >> pos[t]) & 1) << t) | (((j >> (pos[t] + w)) & 1) << (k + t)) for t in range(k))
                    E[i, j] = So[li, lj]
            S = E @ S
        out.append((w, S))
    return out


def _pauli_nonzeros(S):
    """Nonzeros of R' = T S T^dagger / 16 (the Pauli-basis matrix the batch
    kernel builds for width-2 blocks), entries at most 2^-47 of the largest
    dropped as the kernel does."""
    t1 = {0: {(0, 0): 1, (1, 1): 1}, 1: {(0, 1): 1, (1, 0): 1}, 2: {(0, 1): 1j, (1, 0): -1j},
          3: {(0, 0): 1, (1, 1): -1}}
    T = np.zeros((16, 16), dtype=complex)
    for P0 in range(4):
        for P1 in range(4):
            slot = [0, 1, 4, 5][P0] + [0, 2, 8, 10][P1]
            for l in range(16):
                r0, r1, c0, c1 = l & 1, (l >> 1) & 1, (l >> 2) & 1, (l >> 3) & 1
                T[slot, l] = t1[P0].get((r0, c0), 0) * t1[P1].get((r1, c1), 0)
    R = (T @ S @ T.conj().T).real / 16
    return int(np.sum(np.abs(R) > np.max(np.abs(R)) * 2.0 ** -47))


def _expected_work(tq, precision, n, ops, width, diagonal_fp64):
    """Flops and HBM bytes tq_batch_work must report for one job, from the
    plan's blocks: every job runs its canonical groups (Hermitian mode);
    FP64 counts nonzeros (a diagonal block has D of them), split counts all;
    width-2 blocks of tile jobs that the kernel runs in the Pauli basis count
    4 per real-times-complex product plus 128: FP64 per nonzero of R' (when
    that is cheaper than 4 per nonzero of S), split always, dense (256).
    FP64 tile jobs on the batched tensor-core pass (the default FP64 engine)
    count the dense product."""
    esz = 16 if precision == "fp64" else 8
    resident = esz * 4 ** n <= 64 * 1024
    herm = True
    flops = bytes_ = 0
    for w, S in _block_superops(tq, n, ops, width, precision):
        M = 2 ** (n - w)
        groups = M * (M + 1) // 2 if herm else 4 ** (n - w)
        nnz = 4 ** w if (precision == "fp64" and diagonal_fp64) else 16 ** w
        per = 8 * nnz
        if precision == "fp64" and not resident and n >= 6:
            per = 8 * 16 ** w          # batched tensor-core pass: the dense algorithmic count
        elif not resident and w == 2:
            if precision == "split":
                per = 4 * 256 + 128
            else:
                nr = _pauli_nonzeros(S)
                if 2 * nr + 128 < 4 * nnz:
                    per = 4 * nr + 128
        flops += per * groups
        if not resident:
            bytes_ += ((4 ** n + 2 ** n) if herm else 2 * 4 ** n) * esz
    if resident and widths_nonempty(tq, n, ops, width, precision):
        bytes_ += 2 * 4 ** n * esz
    return flops, bytes_


def widths_nonempty(tq, n, ops, width, precision):
    return len(tq.plan_fusion(n, ops, width, precision)[1]) > 0


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("width", [1, 2])
def test_batch_work_counts(tq, precision, width):
    # diagonal circuits (RZ, CZ, RZZ): every fused FP64 block has exactly D
    # nonzeros, so the device count is known in closed form; split counts
    # dense products. Resident (n <= 6) and tile (7, 8) jobs.
    rng = np.random.default_rng(7)
    jobs = []
    for n in (3, 6, 7, 8):
        ops = []
        for _ in range(30):
            if rng.random() < 0.5:
                ops.append(("rz", [int(rng.integers(n))], (float(rng.uniform(-3, 3)),)))
            else:
                a, c = (int(v) for v in rng.choice(n, 2, replace=False))
                ops.append(("cz", [a, c], ()) if rng.random() < 0.5 else ("rzz", [a, c], (float(rng.uniform(-3, 3)),)))
        jobs.append((n, ops))
    b = tq.Batch(precision)
    with pytest.raises(tq.TqError):
        b.work()                      # nothing has run yet
    for n, ops in jobs:
        b.add(n, ops, width=width)
    b.run()
    b.wait()
    want_f = want_b = 0
    for n, ops in jobs:
        f, by = _expected_work(tq, precision, n, ops, width, diagonal_fp64=True)
        want_f += f
        want_b += by
    got = b.work()
    assert got["flops"] == want_f and got["bytes"] == want_b
    for j, (n, ops) in enumerate(jobs):
        tol = TOL64 if precision == "fp64" else 2e-6
        assert np.max(np.abs(b.rho(j) - O.run_circuit(n, ops))) < tol
    b.free()


def test_batch_job_alone_equals_in_mix_and_single_state(tq):
    jobs = _jobs(40, 4, 9, 2, depth=(20, 60))
    mix = tq.Batch("fp64")
    for n, ops, masks in jobs:
        mix.add(n, ops, width=2, masks=masks)
    mix.run()
    mix.wait()
    for j in (0, 7, 19, 33):
        n, ops, masks = jobs[j]
        alone = tq.Batch("fp64")
        alone.add(n, ops, width=2, masks=masks)
        alone.run()
        alone.wait()
        assert np.array_equal(alone.rho(0), mix.rho(j))          # bitwise: same kernels, same order
        assert np.array_equal(alone.result(0), mix.result(j))
        with tq.State(n, "fp64", engine="dfma") as st:
            st.run(ops, width=2)
            if 16 * 4 ** n <= 64 * 1024:
                # resident jobs: both compute the canonical groups with the
                # same DFMA arithmetic in the same order
                assert np.array_equal(st.rho(), mix.rho(j))
            else:
                # tile jobs may run width-2 blocks in the Pauli basis (other
                # rounding): both FP64, each within 1e-12 of the other
                assert np.max(np.abs(st.rho() - mix.rho(j))) < TOL64
        alone.free()
    mix.free()


@pytest.mark.parametrize("tile_log2", [4, 8, 12, 18])
def test_batch_tile_sizes_agree(tq, tile_log2):
    jobs = _jobs(6, 7, 9, 3)
    ref = tq.Batch("fp64")
    tb = tq.Batch("fp64")
    for n, ops, masks in jobs:
        ref.add(n, ops, width=2, masks=masks)
        tb.add(n, ops, width=2, masks=masks)
    for n in (7, 8, 9):
        tb.set_tile(n, tile_log2)
    ref.run()
    tb.run()
    for j in range(len(jobs)):
        assert np.array_equal(ref.rho(j), tb.rho(j))
    ref.free()
    tb.free()


def test_batch_rejects_wide_blocks(tq):
    b = tq.Batch("fp64")
    ops = [("h", [0], ()), ("cx", [0, 1], ())]
    with pytest.raises(tq.TqError) as e:
        b.add(3, ops, width=3)
    assert e.value.status == 7          # TQ_ERR_UNSUPPORTED
    U = np.eye(8, dtype=complex)
    with pytest.raises(tq.TqError) as e:
        b.add(4, [("unitary", [0, 1, 2], [U])], width=2)
    assert e.value.status == 7
    b.free()


def test_batch_wait_timeout_is_reported_and_recoverable(tq):
    # a job whose device-side waits can never be satisfied: the bounded wait
    # runs out, the kernel sets its error flag and returns normally
    jobs = _jobs(4, 8, 8, 4)
    b = tq.Batch("fp64")
    for n, ops, masks in jobs:
        b.add(n, ops, width=2, masks=masks)
    b.test_wait_limit(20000, never_ready_job=1)
    b.run()
    with pytest.raises(tq.TqError) as e:
        b.wait()
    assert e.value.status == 5          # TQ_ERR_TIMEOUT
    # the context is still usable: normal waits give correct results
    b.test_wait_limit(20000000, never_ready_job=-1)
    b.run()
    b.wait()
    for j, (n, ops, masks) in enumerate(jobs):
        assert np.max(np.abs(b.rho(j) - O.run_circuit(n, ops))) < TOL64
    b.free()
    with tq.State(3, "fp64") as st:      # and other work still runs
        st.run(W.ghz(3), width=2)
        assert abs(st.trace() - 1) < TOL64


def test_autotune_picks_a_valid_candidate_and_caches(tq, tmp_path):
    cache = str(tmp_path / "tune.txt")
    t, w, ms = tq.autotune("fp64", 8, cache)
    assert w in (1, 2) and 4 <= t <= 16 and ms > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].split()[1:3] == ["fp64", "8"]
    assert tq.autotune("fp64", 8, cache) == (t, w, ms)          # answered from the cache
    assert len(open(cache).read().splitlines()) == 1
    # the DFMA engine is tuned on its own and cached under its own key
    td, wd, msd = tq.autotune("fp64", 8, cache, engine="dfma")
    assert wd in (1, 2) and 4 <= td <= 16 and msd > 0
    lines = open(cache).read().splitlines()
    assert len(lines) == 2 and lines[1].split()[1:3] == ["fp64-dfma", "8"]
    # the tuned settings give the same results as the defaults
    jobs = _jobs(5, 8, 8, 11)
    a, b = tq.Batch("fp64"), tq.Batch("fp64")
    for n, ops, masks in jobs:
        a.add(n, ops, width=w, masks=masks)
        b.add(n, ops, width=w, masks=masks)
    b.set_tile(8, t)
    a.run()
    b.run()
    for j in range(len(jobs)):
        assert np.array_equal(a.rho(j), b.rho(j))


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("engine", ["auto", "dfma", "tensor"])
def test_tile_jobs_on_either_engine_match_the_oracle(tq, precision, engine):
    # tile jobs (7-9 qubits) run on the batched tensor-core pass (FP64: auto
    # or tensor; split: tensor), otherwise on the persistent kernel; resident
    # jobs on the persistent kernel always; one job alone equals itself in
    # the mix
    jobs = _jobs(12, 4, 9, 13, depth=(20, 60))
    esz = 16 if precision == "fp64" else 8
    tol = TOL64 if precision == "fp64" else 2e-6
    ztol = TOL64 if precision == "fp64" else 1e-5
    b = tq.Batch(precision, engine=engine)
    for n, ops, masks in jobs:
        b.add(n, ops, width=-1, masks=masks)
    b.run()
    b.wait()
    tiles = sum(1 for n, _, _ in jobs if esz * 4 ** n > 64 * 1024)
    on_tensor = engine == "tensor" or (engine == "auto" and precision == "fp64")
    assert b.tensor_jobs() == (tiles if on_tensor else 0)
    for j, (n, ops, masks) in enumerate(jobs):
        want = O.run_circuit(n, ops)
        assert np.max(np.abs(b.rho(j) - want)) < tol, (j, n)
        res = b.result(j)
        for i, m in enumerate(masks):
            wz = O.expect_z(want, m) / (1.0 if precision == "fp64" else O.trace(want).real)
            assert abs(res[2 + i] - wz) < ztol
    k = next(j for j, (n, _, _) in enumerate(jobs) if esz * 4 ** n > 64 * 1024)
    alone = tq.Batch(precision, engine=engine)
    alone.add(jobs[k][0], jobs[k][1], width=-1, masks=jobs[k][2])
    alone.run()
    alone.wait()
    assert np.array_equal(alone.rho(0), b.rho(k))
    alone.free()
    b.free()

