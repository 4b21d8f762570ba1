"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 states must match within 1e-12 max-abs (entries, trace, <Z> values).
Split states (complex64 storage, FP32 products) are checked against the
bound stated for them: 2e-6 max-abs per entry after one op on a unit-trace
state, and the per-result bounds of the circuit tests below."""
import itertools
import math

import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def random_general_matrix(n, seed):
    """A unit-trace Hermitian state plus a non-Hermitian part, so that a
    missing conjugate or a transposed operand shows up."""
    rho = W.random_density_matrix(n, seed)
    rng = np.random.default_rng(seed + 1)
    N = 1 << n
    return rho + 0.2 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / N


def maxabs(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))))


QUBIT_CASES = {
    1: [(0,)],
    2: [(0,), (1,), (0, 1), (1, 0)],
    3: [(0,), (2,), (2, 0), (1, 2), (0, 1, 2), (2, 0, 1)],
    5: [(0,), (4,), (1, 3), (4, 0), (0, 2, 4), (3, 1, 0), (0, 1, 2, 3), (4, 2, 0, 1)],
    7: [(0,), (3,), (6,), (0, 1), (6, 5), (2, 6), (0, 1, 2), (6, 3, 0), (0, 1, 2, 3), (6, 0, 4, 2)],
}


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("n", sorted(QUBIT_CASES))
def test_single_kraus_op_every_position(tq, n, precision):
    rho = random_general_matrix(n, 100 + n)
    for ci, qubits in enumerate(QUBIT_CASES[n]):
        k = len(qubits)
        Ks = W.random_kraus(k, 2, 1000 * n + ci)
        want = O.apply_kraus(rho, Ks, list(qubits))
        with tq.State(n, precision) as st:
            st.set_rho(rho)
            st.apply_kraus(list(qubits), Ks)
            got = st.rho()
        tol = TOL64 if precision == "fp64" else 2e-6
        assert maxabs(got, want) < tol, (qubits, maxabs(got, want))


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_unitary_ops(tq, precision):
    n = 6
    rho = random_general_matrix(n, 7)
    rng = np.random.default_rng(3)
    for k in (1, 2, 3, 4):
        a = rng.standard_normal((1 << k, 1 << k)) + 1j * rng.standard_normal((1 << k, 1 << k))
        U, _ = np.linalg.qr(a)
        qubits = [int(v) for v in rng.choice(n, size=k, replace=False)]
        want = O.apply_kraus(rho, [U], qubits)
        with tq.State(n, precision) as st:
            st.set_rho(rho)
            st.apply_gate(qubits, U)
            got = st.rho()
        assert maxabs(got, want) < (TOL64 if precision == "fp64" else 2e-6), (k, qubits)


def test_plain_6q_unfused_matches_oracle(tq):
    c = W.plain_6q()
    want = O.run_circuit(c.n, c.ops)
    with tq.State(c.n, "fp64") as st:
        nb = st.run(c.ops, width=0)
        assert nb == len(c.ops)
        got = st.rho()
        tr = st.trace()
        zs = st.expect_z([1 << q for q in range(c.n)])
    assert maxabs(got, want) < TOL64
    assert abs(tr - O.trace(want)) < TOL64
    for q in range(c.n):
        assert abs(zs[q] - O.expect_z(want, 1 << q)) < TOL64


@pytest.mark.parametrize("engine", ["auto", "dfma"])
@pytest.mark.parametrize("width", [0, 1, 2, 3, 4, -1])
@pytest.mark.parametrize("n", [4, 5, 8])
def test_fused_circuits_match_oracle_fp64(tq, n, width, engine):
    c = W.random_noisy_circuit(n, 60, 40 + n, gate_set=("h", "s", "rz", "cx", "su2", "rzz"))
    c.ops += [("thermal", [0, n - 1], (300e-9, 100e-6, 80e-6)), ("pd", [n // 2], (0.05,))]
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "fp64", engine=engine) as st:
        st.run(c.ops, width=width)
        got = st.rho()
    assert maxabs(got, want) < TOL64


@pytest.mark.parametrize("width", [0, 2, 3, 4])
def test_fused_circuits_split_bound(tq, width):
    n = 7
    c = W.random_noisy_circuit(n, 120, 77, gate_set=("h", "rx", "rz", "cx", "su2"))
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "split") as st:
        st.run(c.ops, width=width)
        got = st.rho()
        zs = st.expect_z([1 << q for q in range(n)] + [3, 0b1010101])
    assert maxabs(got, want) < 2e-6
    wz = [O.expect_z(want, m) for m in [1 << q for q in range(n)] + [3, 0b1010101]]
    assert maxabs(zs, wz) < 1e-5


@pytest.mark.parametrize("width", [0, 1, 2, 3, 4])
def test_layered_thermal_widths_match_oracle(tq, width):
    # the 12-qubit layered thermal workload's structure at 8 qubits and 200 gates
    c = W.layered_thermal(n=8, n_gates=200)
    want = O.run_circuit(c.n, c.ops)
    with tq.State(c.n, "fp64") as st:
        st.run(c.ops, width=width)
        got = st.rho()
    assert maxabs(got, want) < TOL64


@pytest.mark.parametrize("precision,tol", [("fp64", TOL64), ("split", 2e-5)])
def test_tfim_8q_zz_per_step(tq, precision, tol):
    c = W.tfim_ring(n=8, steps=30)
    rho = O.zero_state(c.n)
    with tq.State(c.n, precision) as st:
        worst = 0.0
        for (s0, s1) in c.steps:
            step_ops = c.ops[s0:s1]
            rho = O.run_circuit(c.n, step_ops, rho)
            st.run(step_ops, width=-1)
            zz = st.expect_z([0b11])[0]
            worst = max(worst, abs(zz - O.expect_z(rho, 0b11)))
        assert worst < tol, worst
        assert abs(st.trace() - 1) < (TOL64 if precision == "fp64" else 1e-5)


def test_readouts(tq):
    n = 7
    rho = random_general_matrix(n, 9)
    masks = list(range(1, 21)) + [(1 << n) - 1]       # > 16 masks: several reduction launches
    with tq.State(n, "fp64") as st:
        st.set_rho(rho)
        tr = st.trace()
        zs = st.expect_z(masks)
        p = st.probs()
    assert abs(tr - O.trace(rho)) < TOL64
    assert maxabs(zs, [O.expect_z(rho, m) for m in masks]) < TOL64
    assert maxabs(p, O.probabilities(rho)) < TOL64


def test_split_readouts_are_renormalised(tq):
    n = 5
    rho = W.random_density_matrix(n, 2) * 1.5     # trace 1.5: readouts divide by it
    with tq.State(n, "split") as st:
        st.set_rho(rho)
        assert abs(st.trace() - 1.5) < 1e-6
        zs = st.expect_z([1, 6, 31])
        p = st.probs()
    want = [O.expect_z(rho, m) / 1.5 for m in (1, 6, 31)]
    assert maxabs(zs, want) < 1e-6
    assert abs(np.sum(p) - 1) < 1e-6


def test_edge_cases(tq):
    # one qubit; a block as wide as the register (a single group); empty circuit
    for n, k in [(1, 1), (2, 2), (3, 3), (4, 4)]:
        rho = random_general_matrix(n, 30 + n)
        Ks = W.random_kraus(k, 3, 50 + n)
        want = O.apply_kraus(rho, Ks, list(range(k))[::-1])
        for precision, tol in [("fp64", TOL64), ("split", 2e-6)]:
            with tq.State(n, precision) as st:
                st.set_rho(rho)
                st.apply_kraus(list(range(k))[::-1], Ks)
                assert maxabs(st.rho(), want) < tol
    with tq.State(3, "fp64") as st:
        assert st.run([], width=2) == 0
        assert abs(st.rho()[0, 0] - 1) == 0
        st.run(W.ghz(3), width=2)
        before = st.rho()
        for bad in ([("h", [3], ())], [("cx", [1, 1], ())], [("depol", [0], (2.0,))],
                    [("thermal", [0], (1e-6, 1e-6, 5e-6))]):
            with pytest.raises(tq.TqError):
                st.run(bad, width=2)
        with pytest.raises(tq.TqError) as e:
            st.apply_gate([5], np.eye(2))
        assert e.value.status == 2                     # TQ_ERR_QUBIT
        assert maxabs(st.rho(), before) == 0           # errors leave the state unchanged
        st.reset()
        assert st.rho()[0, 0] == 1 and abs(st.trace() - 1) == 0


def test_ghz_depolarizing_closed_form_at_12q(tq):
    n, p = 12, 0.03
    ops = W.ghz(n) + [("depol", [q], (p,)) for q in range(n)]
    with tq.State(n, "fp64") as st:
        st.run(ops, width=-1)
        zz = st.expect_z([0b11, (1 << 11) | 1, 1 << 5])
    assert abs(zz[0] - (1 - p) ** 2) < TOL64
    assert abs(zz[1] - (1 - p) ** 2) < TOL64
    assert abs(zz[2]) < TOL64


def _factorised_check(tq, n, subset, width, precision, n_gates, seed, n_samples=4096, tol=TOL64, engine=None):
    """Full-size check: a product state (random SU(2) + amplitude damping on
    every qubit), then a noisy circuit on `subset` only. rho factorises into
    the oracle's small results, so sampled entries of the 4^n vector can be
    computed one by one."""
    import torch

    prefix = W.product_prefix(n, seed)
    sub = W.random_noisy_circuit(len(subset), n_gates, seed + 1, gate_set=("h", "rz", "cx", "su2", "rzz"))
    body = [(name, [subset[q] for q in qs], params) for name, qs, params in sub.ops]
    # oracle pieces
    factors = {}
    for q in range(n):
        if q not in subset:
            ops_q = [(nm, [0], pr) for nm, qs, pr in prefix if qs == [q]]
            factors[q] = O.run_circuit(1, ops_q)
    local = {q: j for j, q in enumerate(subset)}
    ops_s = [(nm, [local[qs[0]]], pr) for nm, qs, pr in prefix if qs[0] in local] + sub.ops
    rho_s = O.run_circuit(len(subset), ops_s)

    with tq.State(n, precision, engine=engine) as st:
        st.run(prefix + body, width=width)
        tr = st.trace()
        st.device_ptr()                                  # every entry current (Hermitian mode)
        vec = st._buf.view(torch.complex128 if precision == "fp64" else torch.complex64)
        N = 1 << n
        rng = np.random.default_rng(seed)
        r = rng.integers(0, N, n_samples)
        c = rng.integers(0, N, n_samples)
        r[:3] = [0, N - 1, 0]
        c[:3] = [0, N - 1, N - 1]
        idx = torch.as_tensor(r + c * N, device="cuda")
        got = vec[idx].cpu().numpy().astype(np.complex128)
    want = np.empty(n_samples, dtype=np.complex128)
    for s in range(n_samples):
        rs = sum(((int(r[s]) >> q) & 1) << j for j, q in enumerate(subset))
        cs = sum(((int(c[s]) >> q) & 1) << j for j, q in enumerate(subset))
        v = rho_s[rs, cs]
        for q, f in factors.items():
            v *= f[(int(r[s]) >> q) & 1, (int(c[s]) >> q) & 1]
        want[s] = v
    assert abs(tr - 1) < (1e-11 if precision == "fp64" else 1e-5)
    err = float(np.max(np.abs(got - want)))
    assert err < tol, err


@pytest.mark.parametrize("engine", ["auto", "dfma"])
@pytest.mark.parametrize("width", [0, 1, 2, 3, 4])
def test_full_size_12q_factorised(tq, width, engine):
    _factorised_check(tq, 12, [0, 5, 10, 11], width, "fp64", 40, 12, engine=engine)


def test_full_size_15q_factorised_fp64(tq):
    # the 15-qubit register in the launch configuration of the benchmark, on
    # the DFMA engine (the tensor-core engine has its own checks)
    _factorised_check(tq, 15, [0, 6, 13, 14], -1, "fp64", 12, 15, engine="dfma")


def test_full_size_15q_factorised_split(tq):
    _factorised_check(tq, 15, [1, 7, 12, 14], -1, "split", 30, 16, tol=2e-6)


def test_max_size_16q_factorised_fp64(tq):
    # the largest register (vec(rho) = 64 GiB in FP64; vec indices up to 2^32 - 1), DFMA engine
    _factorised_check(tq, 16, [0, 7, 14, 15], -1, "fp64", 10, 17, engine="dfma")


def test_max_size_16q_factorised_split(tq):
    _factorised_check(tq, 16, [2, 8, 13, 15], -1, "split", 20, 18, tol=2e-6)


@pytest.mark.parametrize("precision", ["fp64", "split"])
@pytest.mark.parametrize("n,width", [(3, 1), (6, 2), (8, 2), (6, 0)])
def test_small_register_program_runs_on_a_cluster(tq, precision, n, width):
    # n <= 8 and widths <= 2: tq_program_run applies every block in ONE
    # kernel on a thread-block cluster (cluster barriers between blocks);
    # the second run replays the captured graph
    c = W.random_noisy_circuit(n, 60, 300 + n, gate_set=("h", "rx", "rz", "cx", "su2", "rzz"))
    prog = tq.DeviceProgram(n, c.ops, width=width, precision=precision)
    assert prog.n_blocks >= 2 and prog.max_width <= 2
    want = O.run_circuit(n, c.ops)
    tol = TOL64 if precision == "fp64" else 2e-6
    with tq.State(n, precision) as st:
        for _ in range(2):
            st.reset()
            l0 = st.launch_count()
            st.run_program(prog)
            assert st.launch_count() - l0 == 3            # superoperator build, fusion, the cluster kernel
            assert maxabs(st.rho(), want) < tol
            assert abs(st.trace().real - O.trace(want).real) < (TOL64 if precision == "fp64" else 1e-5)
    prog.free()


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_device_program_equals_host_call(tq, precision):
    import torch
    n = 9
    c = W.tfim_ring(n, steps=1)
    prog = tq.DeviceProgram(n, c.ops, width=-1, precision=precision)
    assert prog.n_ops == len(c.ops) and prog.n_blocks >= 1 and prog.table_bytes > 0
    masks = torch.tensor([0b11, 1 << 8], dtype=torch.int64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with tq.State(n, precision) as a, tq.State(n, precision) as b:
        for _ in range(3):
            a.run_program(prog)
            b.run(c.ops, width=-1)
        a.expect_z_device(masks.data_ptr(), 2, out.data_ptr())
        va, vb = a.vec(), b.vec()
        zb = b.expect_z([0b11, 1 << 8])
    assert np.array_equal(va, vb)                  # same kernels, same order: bitwise equal
    assert np.array_equal(out.cpu().numpy(), zb)
    prog.free()
    with pytest.raises(tq.TqError):
        with tq.State(n - 1, precision) as st:
            st.run_program(tq.DeviceProgram(n, c.ops, precision=precision))


def test_profile_counts_launches(tq):
    n = 8
    c = W.tfim_ring(n, steps=2)
    with tq.State(n, "fp64") as st:
        st.profile(True)
        l0 = st.launch_count()
        nb = st.run(c.ops, width=2)
        st.expect_z([3])
        stats = st.profile_stats()
        packs = stats.get("sparse_pack", {"launches": 0})["launches"]
        assert st.launch_count() - l0 == 1 + 1 + packs + nb + 2
    applies = {k: v for k, v in stats.items() if k.startswith("apply")}
    assert sum(v["launches"] for v in applies.values()) == nb
    assert stats["superop_build"]["launches"] == 1 and stats["fuse"]["launches"] == 1
    assert stats["reduce"]["launches"] == 2
    # Hermitian mode computes the canonical groups only: M (M + 1) / 2 of M^2
    M = 2 ** (n - 2)
    groups = M * (M + 1) // 2
    for k, v in applies.items():
        assert v["bytes"] == 2 * 16 * groups * 16
        assert 0 < v["flops"] <= 8.0 * groups * 16 * 16


def test_profile_counts_the_row_list_nonzeros_applied(tq):
    # unfused single ops whose superoperators have closed-form nonzero counts
    # (local index l = r + 2 c, S = conj(K) (x) K summed over the Kraus set):
    #   1-qubit depolarising: S00,00 S00,11 S11,00 S11,11 and the two
    #   coherences S01,01 S10,10 -> 6 of 16;
    #   amplitude damping: S00,00 S00,11 S11,11 S01,01 S10,10 -> 5;
    #   CX (a permutation of the 16 local entries): 16 of 256.
    # The row-list kernels' flops per launch are 8 x (canonical groups) x
    # those counts, read back from the device's row lists.
    n = 7
    cases = [([("depol", [2], (0.01,))], "apply_f64_sparse_w1", 1, 6),
             ([("ad", [5], (0.2,))], "apply_f64_sparse_w1", 1, 5),
             ([("cx", [1, 4], ())], "apply_f64_sparse_w2", 2, 16)]
    for ops, kind, w, nnz in cases:
        with tq.State(n, "fp64", engine="dfma") as st:
            st.profile(True)
            st.run(ops, width=0)
            stats = st.profile_stats()
        M = 2 ** (n - w)
        assert stats[kind]["launches"] == 1
        assert stats[kind]["flops"] == 8.0 * (M * (M + 1) // 2) * nnz, (ops, stats[kind]["flops"])
    assert all(v["total_ms"] > 0 for v in stats.values())


def test_layered_thermal_12q_fusion_widths_agree(tq):
    # the 12-qubit layered thermal workload at full register size (first 400
    # gates): every fusion width gives the unfused result within 1e-12
    import torch
    c = W.layered_thermal(n=12, n_gates=400)
    masks = [1 << q for q in range(12)] + [0b11, (1 << 12) - 1]
    idx = torch.as_tensor(np.random.default_rng(1).integers(0, 1 << 24, 8192), device="cuda")
    ref = None
    for width in (0, 1, 2, 3, 4):
        with tq.State(12, "fp64") as st:
            nb = st.run(c.ops, width=width)
            z = st.expect_z(masks)
            tr = st.trace()
            st.device_ptr()
            v = st._buf.view(torch.complex128)[idx].cpu().numpy()
        assert abs(tr - 1) < 1e-11
        if ref is None:
            ref = (z, v, nb)
            continue
        assert nb < ref[2]
        assert maxabs(z, ref[0]) < TOL64, width
        assert maxabs(v, ref[1]) < TOL64, width


@pytest.mark.parametrize("width", [0, 1, 2, 3, 4])
def test_hermitian_mode_matches_full_update_and_oracle(tq, width):
    n = 7
    c = W.random_noisy_circuit(n, 80, 61 + width, gate_set=("h", "s", "rx", "cx", "su2", "rzz"))
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "fp64") as a, tq.State(n, "fp64", hermitian=False) as b:
        assert a.hermitian_mode() and not b.hermitian_mode()
        a.run(c.ops, width=width)
        b.run(c.ops, width=width)
        ra, rb = a.rho(), b.rho()
        za, zb = a.expect_z([1, 6, 127]), b.expect_z([1, 6, 127])
    assert maxabs(ra, want) < TOL64 and maxabs(rb, want) < TOL64
    off = ~np.eye(1 << n, dtype=bool)                   # the lower triangle mirrors the upper exactly;
    assert np.array_equal(ra[off], ra.conj().T[off])    # the diagonal keeps rounding-level Im parts
    assert np.max(np.abs(np.diag(ra).imag)) < 1e-15
    assert maxabs(za, zb) < TOL64


def test_hermitian_mode_follows_set_rho(tq):
    n = 5
    with tq.State(n, "fp64") as st:
        st.set_rho(random_general_matrix(n, 3))         # not Hermitian: full updates
        assert not st.hermitian_mode()
        herm = W.random_density_matrix(n, 4)
        herm = 0.5 * (herm + herm.conj().T)
        st.set_rho(herm)
        assert st.hermitian_mode()
        st.run([("cx", [0, 3], ()), ("depol", [0, 3], (0.1,))], width=2)
        assert maxabs(st.rho(), O.run_circuit(n, [("cx", [0, 3], ()), ("depol", [0, 3], (0.1,))], herm)) < TOL64
        st.set_hermitian(False)                          # fills the lower half, then full updates
        assert not st.hermitian_mode()
        st.reset()
        st.set_hermitian(True)
        assert st.hermitian_mode()


@pytest.mark.parametrize("width", [0, 1, 2, 3, -1])
@pytest.mark.parametrize("n", [5, 6, 9, 11])
def test_split_hermitian_mode_matches_oracle(tq, n, width):
    # split Hermitian mode runs widths 1-2 through coalesced 16 x 16 group
    # tiles (direct or transposed per local index); width-3 blocks in the mix
    # fill the lower triangle first and update every group
    c = W.random_noisy_circuit(n, 70, 90 + n + width, gate_set=("h", "s", "rx", "cx", "su2", "rzz"))
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "split") as a, tq.State(n, "split", hermitian=False) as b:
        assert a.hermitian_mode()
        a.run(c.ops, width=width)
        b.run(c.ops, width=width)
        ra, rb = a.rho(), b.rho()
        masks = [1, 3, (1 << n) - 1]
        za = a.expect_z(masks)
    assert maxabs(ra, want) < 2e-6
    assert maxabs(ra, rb) < 2e-6
    assert maxabs(za, [O.expect_z(want, m) for m in masks]) < 1e-5


def test_split_precision_bounds_tfim_8q(tq):
    # the split path's stated bounds on the 8-qubit ring TFIM (30 Trotter
    # steps, 900 noisy gates) against the oracle: <Z0 Z1> after every step,
    # every entry of rho, the trace drift before renormalisation, and the
    # most negative eigenvalue (the oracle's state is positive to 1e-12)
    n = 8
    c = W.tfim_ring(n, 30)
    rho = O.zero_state(n)
    with tq.State(n, "split") as st:
        for a, b in c.steps:
            for op in c.ops[a:b]:
                rho = O.apply_op(rho, op)
            st.run(c.ops[a:b], width=-1)
            assert abs(st.expect_z([3])[0] - O.expect_z(rho, 3) / O.trace(rho).real) < 1e-5
        got = st.rho()
        tr = st.trace().real
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12
    assert maxabs(got, rho) < 2e-6
    assert abs(tr - 1.0) < 1e-5
    assert np.min(np.linalg.eigvalsh((got + got.conj().T) / 2)) > -1e-6


def test_split_tensor_core_wait_timeout_is_reported(tq):
    # failure path of the split tensor-core pass: with its MMAs (and their
    # commit) skipped, the bounded MMA wait runs out with nothing in flight;
    # the kernel frees its tensor memory and returns, the next readout of the
    # state reports TQ_ERR_TIMEOUT and poisons it, and the context stays usable
    n = 9
    c = W.tfim_ring(n, 1)
    try:
        tq.test_tc_wait_limit(2000, skip_mma=True)
        with tq.State(n, "split") as st:
            assert st.hermitian_mode()
            st.run(c.ops, width=2)
            with pytest.raises(tq.TqError) as e:
                st.expect_z([3])
            assert e.value.status == 5          # TQ_ERR_TIMEOUT
            with pytest.raises(tq.TqError) as e:
                st.trace()
            assert e.value.status == 6          # TQ_ERR_STATE: poisoned
    finally:
        tq.test_tc_wait_limit(0, skip_mma=False)
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "split") as st:
        st.run(c.ops, width=2)
        assert maxabs(st.rho(), want) < 2e-6
        assert abs(st.trace().real - 1.0) < 1e-5
