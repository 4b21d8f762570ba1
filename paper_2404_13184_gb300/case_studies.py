"""Case-study workloads run on the batch engine (TANQ-Sim Sec. 5: teleportation
channel tomography, Case Study-1; nested entanglement purification, Case
Study-2). Circuits are lists of ops in the binding's format; every density
matrix is evolved and every readout (trace, <Z...Z>) is reduced on the GPU.
The host only turns the readouts into a 2x2 output state, a chi matrix or a
fidelity, which are a few dozen flops.

Noise is synthetic (the paper's ibm_toronto calibration is not available):
1- and 2-qubit depolarising after each gate, zero-temperature thermal
relaxation (T1, T2, gate time) on each gate qubit, and a readout confusion
(e10 = P(read 1 | 0), e01 = P(read 0 | 1)) on measured qubits.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# --- teleportation ------------------------------------------------------------


@dataclass(frozen=True)
class DeviceNoise:
    """Per-gate noise of a synthetic device. Zero fields switch a term off."""
    p1: float = 0.0          # 1-qubit depolarising after each 1-qubit gate
    p2: float = 0.0          # 2-qubit depolarising after each 2-qubit gate
    t1: float = 0.0          # T1 (s); 0: no thermal relaxation
    t2: float = 0.0          # T2 (s), <= 2 T1
    t_1q: float = 35e-9      # 1-qubit gate time (s)
    t_2q: float = 300e-9     # 2-qubit gate time (s)
    e10: float = 0.0         # readout: P(read 1 | state 0)
    e01: float = 0.0         # readout: P(read 0 | state 1)


NOISELESS = DeviceNoise()
# a device-like setting (transmon-scale error rates and coherence times)
DEVICE = DeviceNoise(p1=3e-4, p2=1e-2, t1=100e-6, t2=80e-6, e10=0.02, e01=0.04)
# the same device with 1- and 2-qubit gate errors raised to 0.1 (Sec. 5, Fig. (c))
DEVICE_WORSE = DeviceNoise(p1=0.1, p2=0.1, t1=100e-6, t2=80e-6, e10=0.02, e01=0.04)


def _channels(noise: DeviceNoise, qubits, two_qubit: bool):
    """Depolarising and thermal-relaxation channels after a gate on `qubits`
    (1- or 2-qubit rates and gate time by `two_qubit`)."""
    ops = []
    p = noise.p2 if two_qubit else noise.p1
    if p > 0:
        ops.append(("depol", list(qubits), (p,)))
    if noise.t1 > 0:
        t = noise.t_2q if two_qubit else noise.t_1q
        ops += [("thermal", [q], (t, noise.t1, noise.t2)) for q in qubits]
    return ops


def _noisy(noise: DeviceNoise, name: str, qubits, params=()):
    """A gate followed by its channels."""
    return [(name, list(qubits), params)] + _channels(noise, qubits, len(qubits) == 2)


def readout_confusion(e10: float, e01: float):
    """Kraus set of a Z measurement whose recorded bit flips with P(1|0) = e10
    and P(0|1) = e01, in deferred-measurement form: the qubit then acts only
    as a control, so the dephasing the set implies changes nothing else."""
    K0 = np.diag([np.sqrt(1 - e10), np.sqrt(1 - e01)]).astype(complex)
    K1 = np.array([[0, 0], [np.sqrt(e10), 0]], dtype=complex)
    K2 = np.array([[0, np.sqrt(e01)], [0, 0]], dtype=complex)
    return [K for K in (K0, K1, K2) if np.any(K)]


# tomography inputs on qubit 0: |0>, |1>, |+>, |+i>
TOMO_INPUTS = {
    "0": [],
    "1": [("x", [0], ())],
    "+": [("h", [0], ())],
    "+i": [("h", [0], ()), ("s", [0], ())],
}
# basis changes that map X, Y, Z of qubit 2 onto Z
_HSDG = np.array([[1, -1j], [1, 1j]]) / np.sqrt(2)   # U Y U^dagger = Z
BASIS = {"z": [], "x": [("h", [2], ())], "y": [("unitary", [2], [_HSDG])]}


def teleport_ops(noise: DeviceNoise, prep, basis):
    """Teleport qubit 0 to qubit 2 in deferred-measurement form: Bell pair
    (1, 2); Bell-basis change on (0, 1); readout confusion on the measured
    qubits 0, 1; corrections X^{m1} Z^{m0} on qubit 2 as CX(1, 2), CZ(0, 2).
    The corrections are physically 1-qubit gates on qubit 2, so they carry
    1-qubit noise. State preparation and the tomography basis change are
    ideal (they belong to the tomography, not the channel)."""
    ops = list(prep)
    ops += _noisy(noise, "h", [1]) + _noisy(noise, "cx", [1, 2])
    ops += _noisy(noise, "cx", [0, 1]) + _noisy(noise, "h", [0])
    if noise.e10 > 0 or noise.e01 > 0:
        K = readout_confusion(noise.e10, noise.e01)
        ops += [("kraus", [0], K), ("kraus", [1], K)]
    ops += [("cx", [1, 2], ())] + _channels(noise, [2], False)
    ops += [("cz", [0, 2], ())] + _channels(noise, [2], False)
    return ops + list(basis)


_PAULI = [np.eye(2, dtype=complex), np.array([[0, 1], [1, 0]], dtype=complex),
          np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], dtype=complex)]


def bloch_state(x: float, y: float, z: float, tr: float = 1.0):
    """2x2 density matrix tr (I + x X + y Y + z Z) / 2."""
    return tr * (_PAULI[0] + x * _PAULI[1] + y * _PAULI[2] + z * _PAULI[3]) / 2


def chi_from_outputs(out: dict):
    """Process matrix of a 1-qubit channel in the Pauli basis (I, X, Y, Z),
    E(rho) = sum_ij chi_ij P_i rho P_j, from its outputs on |0>, |1>, |+>,
    |+i> (keys "0", "1", "+", "+i"). The outputs on |0><1| and |1><0| follow
    by linearity: with a = 2E(|+><+|) - E(0) - E(1) and b = 2E(|+i><+i|) -
    E(0) - E(1), E(|0><1|) = (a + i b)/2 and E(|1><0|) = (a - i b)/2; chi
    then solves the 16 linear equations E(E_kl) = sum_ij chi_ij P_i E_kl P_j."""
    e0, e1 = out["0"], out["1"]
    a = 2 * out["+"] - e0 - e1
    b = 2 * out["+i"] - e0 - e1
    images = {(0, 0): e0, (1, 1): e1, (0, 1): (a + 1j * b) / 2, (1, 0): (a - 1j * b) / 2}
    M = np.zeros((16, 16), dtype=complex)
    rhs = np.zeros(16, dtype=complex)
    row = 0
    for (k, l), img in images.items():
        E = np.zeros((2, 2), dtype=complex)
        E[k, l] = 1
        for r in range(2):
            for c in range(2):
                for i in range(4):
                    for j in range(4):
                        M[row, 4 * i + j] = (_PAULI[i] @ E @ _PAULI[j])[r, c]
                rhs[row] = img[r, c]
                row += 1
    return np.linalg.solve(M, rhs).reshape(4, 4)


def teleport_chi(tq, noises, precision: str = "fp64"):
    """chi matrix of the teleportation channel for each noise setting: 4
    tomography inputs x 3 readout bases per setting, all in one batch run.
    Returns (list of chi, list of {input: 2x2 output state}, batch wall time
    in ms)."""
    import time
    b = tq.Batch(precision)
    index = []
    for s, noise in enumerate(noises):
        for inp, prep in TOMO_INPUTS.items():
            for ax, rot in BASIS.items():
                j = b.add(3, teleport_ops(noise, prep, rot), width=2, masks=[4])
                index.append((s, inp, ax, j))
    t0 = time.perf_counter()
    b.run()
    b.wait()
    ms = (time.perf_counter() - t0) * 1e3
    bloch = {}
    for s, inp, ax, j in index:
        r = b.result(j)
        # FP64 readouts are Re Tr(rho Z); split ones are already divided by the trace
        bloch[(s, inp, ax)] = (r[0], r[2] / r[0] if precision == "fp64" else r[2])
    b.free()
    chis, outs = [], []
    for s in range(len(noises)):
        out = {}
        for inp in TOMO_INPUTS:
            tr = bloch[(s, inp, "z")][0]
            x, y, z = (bloch[(s, inp, ax)][1] for ax in ("x", "y", "z"))
            out[inp] = bloch_state(x, y, z, tr)
        outs.append(out)
        chis.append(chi_from_outputs(out))
    return chis, outs, ms


def process_fidelity(chi) -> float:
    """Overlap with the identity channel: chi_00."""
    return float(np.real(chi[0, 0]))


# --- nested purification --------------------------------------------------------

# Bell pairs (A_i, B_i) on qubits (2i, 2i+1); four pairs purified in two rounds
PAIRS = [(0, 1), (2, 3), (4, 5), (6, 7)]


def werner_prep(pair, fidelity: float):
    """Ideal Bell pair |Phi+> on (A, B) followed by the 2-qubit depolarising
    channel of parameter 4(1 - F)/3, which gives the Werner state of
    fidelity F (F >= 1/4)."""
    a, bq = pair
    lam = 4.0 * (1.0 - fidelity) / 3.0
    ops = [("h", [a], ()), ("cx", [a, bq], ())]
    if lam > 0:
        ops.append(("depol", [a, bq], (lam,)))
    return ops


_KEEP_EVEN = np.diag([1.0, 0.0, 0.0, 1.0]).astype(complex)   # outcomes 00 and 11 on (A, B)


def dejmps_round(keep, sacrifice, p_cx: float):
    """One purification step of Deutsch et al. (1996) on pairs `keep` and
    `sacrifice`: RX(pi/2) on Alice's qubits, RX(-pi/2) on Bob's, bilateral CX
    keep -> sacrifice (each followed by a 2-qubit depolarising error p_cx),
    Z measurement of the sacrificed pair with success when both outcomes
    agree, kept as the projector |00><00| + |11><11| (the trace of the result
    is the success probability)."""
    (a1, b1), (a2, b2) = keep, sacrifice
    ops = [("rx", [a1], (np.pi / 2,)), ("rx", [a2], (np.pi / 2,)),
           ("rx", [b1], (-np.pi / 2,)), ("rx", [b2], (-np.pi / 2,))]
    for c, t in ((a1, a2), (b1, b2)):
        ops.append(("cx", [c, t], ()))
        if p_cx > 0:
            ops.append(("depol", [c, t], (p_cx,)))
    ops.append(("kraus", [a2, b2], [_KEEP_EVEN]))
    return ops


def purification_ops(fidelity: float, p_cx: float, rounds: int = 2):
    """`rounds` nested purification rounds over 2^rounds Werner pairs of
    fidelity F, ending with the Bell-basis change CX(A, B), H(A) on the kept
    pair (0, 1), which maps |Phi+> to |00>. rounds 1: 4 qubits, 2: 8."""
    if rounds not in (1, 2):
        raise ValueError("rounds must be 1 or 2")
    pairs = PAIRS[: 1 << rounds]
    ops = []
    for p in pairs:
        ops += werner_prep(p, fidelity)
    live = list(pairs)
    for _ in range(rounds):
        nxt = []
        for i in range(0, len(live), 2):
            ops += dejmps_round(live[i], live[i + 1], p_cx)
            nxt.append(live[i])
        live = nxt
    ops += [("cx", [0, 1], ()), ("h", [0], ())]
    return 2 << rounds, ops


def fidelity_from_readouts(tr: float, z0: float, z1: float, z01: float, normalized: bool = False):
    """Fidelity with |Phi+> after the Bell-basis change: P(00 on qubits 0, 1)
    / Tr = (Tr + <Z0> + <Z1> + <Z0 Z1>) / (4 Tr); `normalized`: the <Z>
    readouts are already divided by the trace."""
    if normalized:
        return (1.0 + z0 + z1 + z01) / 4.0
    return (tr + z0 + z1 + z01) / (4.0 * tr)


def purification_curves(tq, fidelities, p_values, rounds: int = 2, precision: str = "fp64"):
    """Output fidelity and success probability for every (p_cx, F_in), all
    circuits in one batch run. Returns ({p: [(F_in, F_out, P_success)]}, ms)."""
    import time
    b = tq.Batch(precision)
    jobs = []
    for p in p_values:
        for f in fidelities:
            n, ops = purification_ops(f, p, rounds)
            jobs.append((p, f, b.add(n, ops, width=2, masks=[1, 2, 3])))
    t0 = time.perf_counter()
    b.run()
    b.wait()
    ms = (time.perf_counter() - t0) * 1e3
    curves = {p: [] for p in p_values}
    for p, f, j in jobs:
        r = b.result(j)
        curves[p].append((f, fidelity_from_readouts(r[0], r[2], r[3], r[4], precision != "fp64"), r[0]))
    b.free()
    return curves, ms
