"""CPU pins of the change of basis that the batch kernel's width-2 tile items
use (csrc/tq_batch_kernels.cuh: k_pauli_lists, pauli_fwd, pauli_inv). A
two-qubit block's superoperator S is taken to the basis of Pauli products,
R' = T S T^dagger / 16, where T = T1 (x) T1 and T1 maps a qubit's 2 x 2
block (a00, a10, a01, a11) to (I, X, Y, Z) = (a00 + a11, a01 + a10,
i(a01 - a10), a00 - a11). A group's update is then y = T^dagger R' (T x).

These tests pin the facts the kernel relies on against the Pauli transfer
matrix Tr(P_a E(P_b)), which is computed from the oracle's own action of
each op on 4 x 4 matrices (operators on 2 qubits):
- R' is real for every Kraus map;
- S = T^dagger R' T;
- R' is a signed permutation (16 nonzeros) for a Clifford gate, diagonal
  for a Pauli channel, and 24-nonzero for a rotation about one axis.
The GPU tests hold the kernel itself to the oracle."""
import itertools

import numpy as np
import pytest

from oracle import dm_oracle as O

PAULI = [np.eye(2, dtype=np.complex128),
         np.array([[0, 1], [1, 0]], dtype=np.complex128),
         np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
         np.array([[1, 0], [0, -1]], dtype=np.complex128)]
# a qubit's 2 x 2 block, taken in the order (a00, a10, a01, a11), to (I, X, Y, Z)
T1 = np.array([[1, 0, 0, 1],
               [0, 1, 1, 0],
               [0, -1j, 1j, 0],
               [1, 0, 0, -1]], dtype=np.complex128)
T = np.kron(T1, T1)  # pair index of qubit 1 high: m = p0 + 4 p1


def pair_order():
    """perm[m] = column-stacked vec index r + 4c of the entry whose per-qubit
    pairs are p0 = r0 + 2 c0, p1 = r1 + 2 c1 (m = p0 + 4 p1)."""
    perm = np.zeros(16, dtype=np.int64)
    for r0, r1, c0, c1 in itertools.product(range(2), repeat=4):
        m = (r0 + 2 * c0) + 4 * (r1 + 2 * c1)
        perm[m] = (r0 + 2 * r1) + 4 * (c0 + 2 * c1)
    return perm


def channel(ops):
    """E(A): the ops, one after another, on a 2-qubit register (linear in A)."""
    def E(A):
        for op in ops:
            A = O.apply_op(A, op)
        return A
    return E


def superop(E):
    """S with S vec(A) = vec(E(A)) (column-stacked vec), column by column:
    column j is vec of E applied to the j-th unit matrix."""
    S = np.zeros((16, 16), dtype=np.complex128)
    for j in range(16):
        U = np.zeros(16, dtype=np.complex128)
        U[j] = 1.0
        S[:, j] = E(U.reshape(4, 4, order="F")).reshape(16, order="F")
    return S


def pauli_of(S):
    """R' = T S T^dagger / 16, with S in the per-qubit pair order."""
    perm = pair_order()
    Sp = S[np.ix_(perm, perm)]
    return T @ Sp @ T.conj().T / 16.0


def transfer(E):
    """Tr(P_a E(P_b)) / 16 for the products P_a = P_a1 (x) P_a0, a = a0 + 4 a1
    (register index r = r0 + 2 r1, so qubit 1 is the left factor)."""
    P = [np.kron(PAULI[a1], PAULI[a0]) for a1 in range(4) for a0 in range(4)]
    return np.array([[np.trace(Pa @ E(Pb)) for Pb in P] for Pa in P]) / 16.0


RNG = np.random.default_rng(11)
MAPS = {
    "h_q0": [("h", [0], ())],
    "cx": [("cx", [0, 1], ())],
    "rx_rzz": [("rx", [1], (0.37,)), ("rzz", [0, 1], (1.1,))],
    "su2_pair": [("su2", [0], tuple(RNG.standard_normal(4))), ("su2", [1], tuple(RNG.standard_normal(4))),
                 ("cz", [0, 1], ())],
    "depol2": [("depol", [0, 1], (0.03,))],
    "depol1_ad": [("depol", [1], (0.05,)), ("ad", [0], (0.2,))],
    "thermal_pd": [("thermal", [0, 1], (1.0, 50.0, 70.0)), ("pd", [1], (0.1,))],
    "fused_noisy": [("h", [0], ()), ("cx", [0, 1], ()), ("depol", [0, 1], (0.01,)),
                    ("rz", [1], (0.8,)), ("ad", [1], (0.05,))],
}


@pytest.mark.parametrize("name", sorted(MAPS))
def test_pauli_matrix_is_the_real_transfer_matrix(name):
    E = channel(MAPS[name])
    R = pauli_of(superop(E))
    assert np.max(np.abs(R.imag)) < 1e-15
    assert np.allclose(R, transfer(E), rtol=0, atol=1e-15)
    # trace preservation: the identity row is (1/4) e_0
    want = np.zeros(16)
    want[0] = 0.25
    assert np.allclose(R[0], want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("name", sorted(MAPS))
def test_update_through_the_pauli_basis_equals_the_product(name):
    S = superop(channel(MAPS[name]))
    R = pauli_of(S).real
    perm = pair_order()
    Sp = S[np.ix_(perm, perm)]
    x = RNG.standard_normal(16) + 1j * RNG.standard_normal(16)
    y = T.conj().T @ (R @ (T @ x))
    assert np.allclose(y, Sp @ x, rtol=0, atol=1e-13)
    # T / 2 is unitary, which is what lets the transform be undone by T^dagger
    assert np.allclose(T @ T.conj().T, 4 * np.eye(16), rtol=0, atol=0)


def test_sparsity_of_clifford_gates_pauli_channels_and_rotations():
    for ops in (MAPS["h_q0"], MAPS["cx"], [("s", [1], ())], [("swap", [0, 1], ())]):
        R = pauli_of(superop(channel(ops))).real
        nz = np.abs(R) > 1e-15
        assert nz.sum() == 16                                      # a signed permutation ...
        assert np.all(nz.sum(axis=0) == 1) and np.all(nz.sum(axis=1) == 1)
        assert np.allclose(np.abs(R[nz]), 0.25, rtol=0, atol=1e-15)  # ... of 1/4s
    R = pauli_of(superop(channel(MAPS["depol2"]))).real
    assert np.allclose(R, np.diag(np.diag(R)), rtol=0, atol=1e-15)  # a Pauli channel is diagonal
    # its diagonal: 1/4 on the identity, (1 - p) / 4 on the other 15 products
    assert np.allclose(np.diag(R), [0.25] + [0.25 * (1 - 0.03)] * 15, rtol=0, atol=1e-15)
    R = pauli_of(superop(channel([("rz", [0], (0.7,))]))).real
    # RZ mixes X and Y of qubit 0 (a 2 x 2 rotation block), times 4 products on qubit 1
    assert (np.abs(R) > 1e-15).sum() == 4 * (2 + 4)
    # against the complex S: RZ is diagonal there (16 nonzeros); the
    # depolarising channel has 28 in S (populations mix) against 16 in R';
    # a fused noisy block (H, CX, depolarising, RZ, damping) 84 against 28
    assert (np.abs(superop(channel([("rz", [0], (0.7,))]))) > 1e-15).sum() == 16
    S = superop(channel(MAPS["depol2"]))
    assert (np.abs(S) > 1e-15).sum() == 28 and (np.abs(pauli_of(S)) > 1e-15).sum() == 16
    S = superop(channel(MAPS["fused_noisy"]))
    assert (np.abs(S) > 1e-15).sum() == 84 and (np.abs(pauli_of(S).real) > 1e-15).sum() == 28
