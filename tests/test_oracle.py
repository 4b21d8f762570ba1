"""Pins of the CPU oracle to things other than itself: closed forms, library
routines (numpy.kron, scipy.linalg.expm), a separate state-vector simulator,
brute-force Kronecker expansion and invariants. CPU only."""
import itertools
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
I2 = np.eye(2, dtype=complex)


def ket(n, x):
    r = np.zeros((1 << n, 1 << n), dtype=complex)
    r[x, x] = 1
    return r


# ---------------------------------------------------------------- gates

@pytest.mark.parametrize("theta", [0.0, 0.3, 1.7, -2.9, 6.1])
def test_rotations_match_matrix_exponential(theta):
    assert np.allclose(O.gate_matrix("rx", (theta,)), scipy.linalg.expm(-0.5j * theta * X), atol=1e-14)
    assert np.allclose(O.gate_matrix("ry", (theta,)), scipy.linalg.expm(-0.5j * theta * Y), atol=1e-14)
    assert np.allclose(O.gate_matrix("rz", (theta,)), scipy.linalg.expm(-0.5j * theta * Z), atol=1e-14)
    # RZZ on local order (b0 = Q[0], b1 = Q[1]); Z(x)Z is symmetric so the order is immaterial
    assert np.allclose(O.gate_matrix("rzz", (theta,)), scipy.linalg.expm(-0.5j * theta * np.kron(Z, Z)), atol=1e-14)


def test_fixed_gates_textbook_relations():
    g = O.gate_matrix
    assert np.allclose(g("x"), X) and np.allclose(g("y"), Y) and np.allclose(g("z"), Z)
    assert np.allclose(g("h") @ g("z") @ g("h"), X)
    assert np.allclose(g("s") @ g("s"), Z)
    assert np.allclose(g("t") @ g("t"), g("s"))
    assert np.allclose(g("sx") @ g("sx"), X)
    assert np.allclose(g("sdg") @ g("s"), I2)
    assert np.allclose(g("tdg") @ g("t"), I2)
    for name in O.ONE_QUBIT_GATES + O.TWO_QUBIT_GATES:
        params = (0.37, -1.2, 0.5, 2.0) if name == "su2" else (0.81,)
        U = g(name, params)
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14), name
    # CX with control b0 and target b1, in numpy.kron order (left factor = high bit b1)
    P0, P1 = np.diag([1, 0]).astype(complex), np.diag([0, 1]).astype(complex)
    assert np.allclose(g("cx"), np.kron(I2, P0) + np.kron(X, P1))
    assert np.allclose(g("cz"), np.kron(I2, P0) + np.kron(Z, P1))


def test_su2_from_quaternion():
    U = O.gate_matrix("su2", (3.0, 0.0, 0.0, 0.0))
    assert np.allclose(U, I2)
    U = O.gate_matrix("su2", (0.0, 2.0, 0.0, 0.0))
    assert np.allclose(U, 1j * Z)
    rng = np.random.default_rng(5)
    for _ in range(20):
        U = O.gate_matrix("su2", tuple(rng.standard_normal(4)))
        assert abs(np.linalg.det(U) - 1) < 1e-13
        assert np.allclose(U.conj().T @ U, I2, atol=1e-14)


def test_cx_convention_on_basis_states():
    # qubit 0 is the control (bit 0), qubit 1 the target (bit 1)
    out = O.apply_op(ket(2, 0b01), ("cx", [0, 1], ()))
    assert np.allclose(out, ket(2, 0b11))
    out = O.apply_op(ket(2, 0b10), ("cx", [0, 1], ()))
    assert np.allclose(out, ket(2, 0b10))
    # reversed qubit list: control is qubit 1
    out = O.apply_op(ket(2, 0b10), ("cx", [1, 0], ()))
    assert np.allclose(out, ket(2, 0b11))
    # in a larger register with a non-adjacent pair
    out = O.apply_op(ket(4, 0b0100), ("cx", [2, 0], ()))
    assert np.allclose(out, ket(4, 0b0101))


# ------------------------------------------------------ brute-force expansions

def test_kron_expansion_matches_numpy_kron_for_adjacent_qubits():
    rng = np.random.default_rng(1)
    n = 5
    rho = W.random_density_matrix(n, 11)
    for k in (1, 2, 3):
        for q in range(n - k + 1):
            Ks = W.random_kraus(k, 2, int(rng.integers(1 << 30)))
            qubits = list(range(q, q + k))
            # numpy.kron: left factor holds the high bits
            fulls = [np.kron(np.eye(1 << (n - q - k)), np.kron(K, np.eye(1 << q))) for K in Ks]
            want = sum(F @ rho @ F.conj().T for F in fulls)
            assert np.allclose(O.apply_kraus_kron(rho, Ks, qubits), want, atol=1e-14)


def test_local_action_matches_kron_expansion_for_all_qubit_orders():
    rng = np.random.default_rng(2)
    n = 4
    rho = W.random_density_matrix(n, 12) + 0.1j * W.random_density_matrix(n, 13)  # non-Hermitian too
    for k in (1, 2, 3):
        for qubits in itertools.permutations(range(n), k):
            Ks = W.random_kraus(k, 3, int(rng.integers(1 << 30)))
            a = O.apply_kraus(rho, Ks, list(qubits))
            b = O.apply_kraus_kron(rho, Ks, list(qubits))
            assert np.max(np.abs(a - b)) < 1e-14, qubits


def test_statevector_matches_kron_statevector():
    # independent pin of sv_run: full-register unitaries from numpy.kron on adjacent qubits
    rng = np.random.default_rng(3)
    n = 5
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    ops = []
    for _ in range(30):
        if rng.uniform() < 0.4:
            q = int(rng.integers(n - 1))
            ops.append(("unitary", [q, q + 1], [W.random_kraus(2, 1, int(rng.integers(1 << 30)))[0]]))
        else:
            q = int(rng.integers(n))
            ops.append(("su2", [q], tuple(rng.standard_normal(4))))
    for name, qubits, params in ops:
        U = params[0] if name == "unitary" else O.gate_matrix(name, params)
        k = len(qubits)
        F = np.kron(np.eye(1 << (n - qubits[0] - k)), np.kron(U, np.eye(1 << qubits[0])))
        psi = F @ psi
    assert np.allclose(O.sv_run(n, ops), psi, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_noise_free_density_matrix_equals_pure_state(seed):
    n = 5
    rng = np.random.default_rng(seed)
    names = list(O.ONE_QUBIT_GATES) + list(O.TWO_QUBIT_GATES)
    ops = []
    for _ in range(60):
        g = names[int(rng.integers(len(names)))]
        if g in O.TWO_QUBIT_GATES:
            q = [int(v) for v in rng.choice(n, 2, replace=False)]
        else:
            q = [int(rng.integers(n))]
        params = tuple(rng.standard_normal(4)) if g == "su2" else (float(rng.uniform(0, 6.3)),)
        ops.append((g, q, params))
    psi = O.sv_run(n, ops)
    rho = O.run_circuit(n, ops)
    assert np.max(np.abs(rho - np.outer(psi, psi.conj()))) < 1e-13


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("p", [0.0, 1e-3, 0.2, 1.0])
def test_depolarizing_closed_forms(p):
    out = O.apply_op(ket(1, 0), ("depol", [0], (p,)))
    assert np.allclose(out, np.diag([1 - p / 2, p / 2]), atol=1e-15)
    out = O.apply_op(ket(2, 0), ("depol", [0, 1], (p,)))
    assert np.allclose(out, (1 - p) * ket(2, 0) + p * np.eye(4) / 4, atol=1e-15)
    # on two qubits of a three-qubit |000>: the third qubit is untouched
    out = O.apply_op(ket(3, 0), ("depol", [2, 0], (p,)))
    want = (1 - p) * ket(3, 0)
    for x in (0b000, 0b001, 0b100, 0b101):
        want[x, x] += p / 4
    assert np.allclose(out, want, atol=1e-15)


@pytest.mark.parametrize("p", [0.01, 0.3])
def test_depolarizing_equals_pauli_twirl(p):
    # the same channel as a mixture of the 4^k Pauli conjugations
    rho = W.random_density_matrix(3, 4) + 0.2j * W.random_density_matrix(3, 5)
    paulis = [I2, X, Y, Z]
    for qubits in ([1], [2, 0]):
        k = len(qubits)
        Ks = []
        for idx in itertools.product(range(4), repeat=k):
            P = np.array([[1.0 + 0j]])
            for j in reversed(range(k)):      # kron left factor = high local bit
                P = np.kron(P, paulis[idx[j]])
            w = (1 - p + p / 4 ** k) if all(i == 0 for i in idx) else p / 4 ** k
            Ks.append(math.sqrt(w) * P)
        a = O.apply_op(rho, ("depol", qubits, (p,)))
        b = O.apply_kraus(rho, Ks, qubits)
        assert np.max(np.abs(a - b)) < 1e-14


@pytest.mark.parametrize("g", [0.0, 5e-4, 0.3, 1.0])
def test_amplitude_damping_closed_forms(g):
    assert np.allclose(O.apply_op(ket(1, 0), ("ad", [0], (g,))), ket(1, 0))
    assert np.allclose(O.apply_op(ket(1, 1), ("ad", [0], (g,))), np.diag([g, 1 - g]))
    plus = np.full((2, 2), 0.5, dtype=complex)
    s = math.sqrt(1 - g) / 2
    assert np.allclose(O.apply_op(plus, ("ad", [0], (g,))), [[(1 + g) / 2, s], [s, (1 - g) / 2]])


def test_thermal_relaxation_closed_forms():
    t, t1, t2 = 300e-9, 100e-6, 80e-6
    plus = np.full((2, 2), 0.5, dtype=complex)
    out = O.apply_op(plus, ("thermal", [0], (t, t1, t2)))
    assert abs(out[0, 0] - (1 - math.exp(-t / t1) / 2)) < 1e-15
    assert abs(out[0, 1] - math.exp(-t / t2) / 2) < 1e-15
    assert abs(out[1, 0] - math.exp(-t / t2) / 2) < 1e-15
    # T2 = 2 T1 is pure amplitude damping with gamma = 1 - exp(-t/T1)
    rho = W.random_density_matrix(2, 7)
    a = O.apply_op(rho, ("thermal", [1], (t, t1, 2 * t1)))
    b = O.apply_op(rho, ("ad", [1], (1 - math.exp(-t / t1),)))
    assert np.max(np.abs(a - b)) < 1e-15
    # general T2: amplitude damping then phase damping with 1-lambda = exp(-2t/T2)/exp(-t/T1)
    lam = 1 - math.exp(-2 * t / t2) / math.exp(-t / t1)
    c = O.apply_op(O.apply_op(rho, ("ad", [0], (1 - math.exp(-t / t1),))), ("pd", [0], (lam,)))
    d = O.apply_op(rho, ("thermal", [0], (t, t1, t2)))
    assert np.max(np.abs(c - d)) < 1e-15
    # semigroup: relaxing for t then s equals relaxing for t + s
    e = O.apply_op(O.apply_op(rho, ("thermal", [0], (t, t1, t2))), ("thermal", [0], (2 * t, t1, t2)))
    f = O.apply_op(rho, ("thermal", [0], (3 * t, t1, t2)))
    assert np.max(np.abs(e - f)) < 1e-15
    # long time: everything decays to |0><0| on that qubit
    g = O.apply_op(rho, ("thermal", [0, 1], (1.0, t1, t2)))
    assert np.allclose(g, ket(2, 0), atol=1e-12)
    with pytest.raises(ValueError):
        O.apply_op(rho, ("thermal", [0], (t, 1e-6, 3e-6)))


@pytest.mark.parametrize("n", [2, 3, 5])
def test_ghz_density_matrix(n):
    rho = O.run_circuit(n, W.ghz(n))
    want = np.zeros_like(rho)
    N = 1 << n
    for r in (0, N - 1):
        for c in (0, N - 1):
            want[r, c] = 0.5
    assert np.max(np.abs(rho - want)) < 1e-15


@pytest.mark.parametrize("p", [1e-3, 0.1])
def test_ghz_with_depolarizing_correlations(p):
    n = 4
    ops = W.ghz(n) + [("depol", [q], (p,)) for q in range(n)]
    rho = O.run_circuit(n, ops)
    for i, j in itertools.combinations(range(n), 2):
        assert abs(O.expect_z(rho, (1 << i) | (1 << j)) - (1 - p) ** 2) < 1e-14
    for i in range(n):
        assert abs(O.expect_z(rho, 1 << i)) < 1e-15


def _teleport_ops(out_noise_p=0.0):
    # deferred-measurement teleportation of qubit 0 to qubit 2
    ops = [("h", [1], ()), ("cx", [1, 2], ()), ("cx", [0, 1], ()), ("h", [0], ()),
           ("cx", [1, 2], ()), ("cz", [0, 2], ())]
    if out_noise_p:
        ops.append(("depol", [2], (out_noise_p,)))
    return ops


def _teleport_channel(rho_in, ops):
    zero = np.diag([1, 0]).astype(complex)
    full = np.kron(zero, np.kron(zero, rho_in))     # qubit 0 = low bit
    out = O.run_circuit(3, ops, full).reshape(2, 4, 2, 4)   # (q2, q1q0) x (q2, q1q0)
    return np.einsum("aibi->ab", out)


def _chi_matrix(channel):
    # linear inversion: E(rho) = sum_mn chi_mn P_m rho P_n
    P = [I2, X, Y, Z]
    rows, rhs = [], []
    for i in range(2):
        for j in range(2):
            E = np.zeros((2, 2), dtype=complex)
            E[i, j] = 1
            out = channel(E)
            basis = [P[m] @ E @ P[nn] for m in range(4) for nn in range(4)]
            rows.append(np.array([b.reshape(-1) for b in basis]).T)
            rhs.append(out.reshape(-1))
    A = np.vstack(rows)
    b = np.concatenate(rhs)
    chi = np.linalg.solve(A, b)
    return chi.reshape(4, 4)


def test_teleportation_chi_identity(golden):
    chi = _chi_matrix(lambda E: _teleport_channel(E, _teleport_ops()))
    assert np.max(np.abs(chi - golden("teleport_chi_ideal.txt"))) < 1e-13


@pytest.mark.parametrize("p", [0.02, 0.1])
def test_teleportation_with_output_depolarizing(p):
    chi = _chi_matrix(lambda E: _teleport_channel(E, _teleport_ops(p)))
    want = np.diag([1 - 3 * p / 4, p / 4, p / 4, p / 4])
    assert np.max(np.abs(chi - want)) < 1e-13
    rng = np.random.default_rng(9)
    for _ in range(5):
        v = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        v /= np.linalg.norm(v)
        out = _teleport_channel(np.outer(v, v.conj()), _teleport_ops(p))
        assert abs(np.real(v.conj() @ out @ v) - (1 - p / 2)) < 1e-13


# ---------------------------------------------------------------- readouts

def test_readouts_match_kron_observables():
    n = 4
    rho = W.random_density_matrix(n, 21)
    for mask in range(1 << n):
        Zm = np.array([[1.0 + 0j]])
        for q in reversed(range(n)):
            Zm = np.kron(Zm, Z if (mask >> q) & 1 else I2)
        assert abs(O.expect_z(rho, mask) - np.real(np.trace(rho @ Zm))) < 1e-14
    p = O.probabilities(rho)
    for x in range(1 << n):
        proj = np.zeros((1 << n, 1 << n))
        proj[x, x] = 1
        assert abs(p[x] - np.real(np.trace(rho @ proj))) < 1e-15
    assert abs(O.trace(rho) - 1) < 1e-14


# -------------------------------------------------------------- invariants

def test_invariants_on_noisy_circuits():
    circ = W.random_noisy_circuit(6, 120, 77, gate_set=("h", "x", "s", "rz", "cx", "su2", "rzz"))
    circ.ops += [("thermal", [0, 3], (300e-9, 100e-6, 80e-6)), ("pd", [5], (0.1,))]
    rho = O.run_circuit(circ.n, circ.ops)
    assert abs(O.trace(rho) - 1) < 1e-12
    assert np.max(np.abs(rho - rho.conj().T)) < 1e-12
    assert np.min(np.linalg.eigvalsh(rho)) > -1e-12
    assert abs(np.sum(O.probabilities(rho)) - O.trace(rho).real) < 1e-13
    for q in range(circ.n):
        assert -1 <= O.expect_z(rho, 1 << q) <= 1


def test_workload_shapes():
    c1 = W.plain_6q()
    assert c1.n == 6 and c1.n_gates == 200
    c2 = W.layered_thermal()
    assert c2.n == 12 and sum(1 for o in c2.ops if o[0] != "thermal") == 2000
    c3 = W.tfim_ring()
    assert c3.n == 15 and c3.n_gates == 900 and len(c3.steps) == 30
    assert sum(1 for o in c3.ops if o[0] in ("rzz", "rx")) == 900
    assert W.plain_6q().ops == c1.ops          # seeded: identical on regeneration


# ------------------------------------------------ measurement, reset, readout

def test_reset_closed_forms():
    assert np.allclose(O.apply_op(ket(1, 1), ("reset", [0], ())), ket(1, 0))
    rho = W.random_density_matrix(3, 8)
    out = O.apply_op(rho, ("reset", [1], ()))
    # qubit 1 ends in |0>, the reduced state of qubits 0 and 2 is unchanged
    t_in = rho.reshape(2, 2, 2, 2, 2, 2)      # (q2, q1, q0) x (q2, q1, q0)
    t_out = out.reshape(2, 2, 2, 2, 2, 2)
    assert np.allclose(np.einsum("aibcid->abcd", t_in), np.einsum("aibcid->abcd", t_out), atol=1e-15)
    assert np.allclose(t_out[:, 1], 0) and np.allclose(t_out[:, :, :, :, 1], 0)
    assert abs(O.trace(out) - 1) < 1e-14


def test_measurement_closed_forms():
    n = 3
    ghz = O.run_circuit(n, W.ghz(n))
    m, p, post = O.measure(ghz, 1, 0.25)
    assert m == 0 and abs(p - 0.5) < 1e-15 and np.allclose(post, ket(n, 0))
    m, p, post = O.measure(ghz, 2, 0.75)
    assert m == 1 and abs(p - 0.5) < 1e-15 and np.allclose(post, ket(n, 7))
    # |+> on qubit 0: measuring gives each outcome with probability 1/2; a mixed state keeps its rest
    rho = O.run_circuit(2, [("h", [0], ()), ("ad", [1], (0.3,)), ("h", [1], ())])
    m, p, post = O.measure(rho, 0, 0.9)
    assert m == 1 and abs(p - 0.5) < 1e-15
    assert abs(O.trace(post) - 1) < 1e-15 and abs(O.expect_z(post, 1) + 1) < 1e-15


def test_readout_and_sampling():
    # one qubit: the confusion matrix itself
    out = O.readout_probabilities([0.8, 0.2], [0.1], [0.3])
    assert np.allclose(out, [0.8 * 0.9 + 0.2 * 0.3, 0.8 * 0.1 + 0.2 * 0.7])
    # independent qubits: a product distribution stays a product of confused factors
    pa, pb = np.array([0.6, 0.4]), np.array([0.25, 0.75])
    p = np.kron(pb, pa)                               # qubit 0 = low bit
    e10, e01 = [0.02, 0.05], [0.1, 0.07]
    want = np.kron(O.readout_probabilities(pb, [e10[1]], [e01[1]]), O.readout_probabilities(pa, [e10[0]], [e01[0]]))
    assert np.allclose(O.readout_probabilities(p, e10, e01), want, atol=1e-15)
    assert abs(np.sum(O.readout_probabilities(np.full(8, 1 / 8), [0.1] * 3, [0.2] * 3)) - 1) < 1e-15
    assert list(O.sample([0.5, 0.0, 0.25, 0.25], [0.1, 0.49, 0.5, 0.74, 0.76, 0.999])) == [0, 0, 2, 2, 3, 3]
    assert list(O.sample(np.eye(4)[2], [0.0, 0.5, 0.9999])) == [2, 2, 2]


# ------------------------------------------------- case studies (Sec. 5)

def _dejmps(A, B, C, D):
    # Deutsch et al. (1996): Bell-diagonal weights (Phi+, Psi-, Psi+, Phi-)
    # after one successful round, and the success probability
    N = (A + B) ** 2 + (C + D) ** 2
    return ((A * A + B * B) / N, 2 * C * D / N, (C * C + D * D) / N, 2 * A * B / N), N


@pytest.mark.parametrize("rounds", [1, 2])
@pytest.mark.parametrize("F", [0.55, 0.7, 0.9])
def test_purification_matches_dejmps_recurrence(rounds, F):
    from paper_2404_13184_gb300 import case_studies as C
    n, ops = C.purification_ops(F, 0.0, rounds)
    rho = O.run_circuit(n, ops)
    tr = O.trace(rho).real
    # after the Bell-basis change |Phi+> -> |00> on qubits 0, 1
    p00 = sum(rho[x, x].real for x in range(1 << n) if x & 3 == 0)
    w, succ = _dejmps(F, (1 - F) / 3, (1 - F) / 3, (1 - F) / 3)
    if rounds == 2:
        # two independent first-round successes, then the second round
        w, N2 = _dejmps(*w)
        succ = succ * succ * N2
    assert abs(p00 / tr - w[0]) < 1e-13
    assert abs(tr - succ) < 1e-13


@pytest.mark.parametrize("e10,e01", [(0.02, 0.02), (0.02, 0.06), (0.1, 0.0)])
def test_teleportation_readout_error_is_a_pauli_channel(e10, e01):
    # every Bell-measurement outcome has probability 1/4 whatever the input,
    # so each recorded bit is flipped with probability e = (e10 + e01)/2,
    # independently: a wrong m1 leaves an X error, a wrong m0 a Z error
    from paper_2404_13184_gb300 import case_studies as C
    noise = C.DeviceNoise(e10=e10, e01=e01)
    chan = lambda E: _teleport_channel(E, C.teleport_ops(noise, [], []))
    chi = _chi_matrix(chan)
    e = (e10 + e01) / 2
    want = np.diag([(1 - e) ** 2, e * (1 - e), e * e, e * (1 - e)])
    assert np.max(np.abs(chi - want)) < 1e-13
