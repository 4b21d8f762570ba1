"""Case studies of Sec. 5 on the batch engine: teleportation channel
tomography (Case Study-1) and nested purification (Case Study-2). CPU tests
cover the host-side analysis; GPU tests compare the engine's readouts with
the oracle (FP64 1e-12) and with closed forms."""
import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import case_studies as C

TOL64 = 1e-12
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]])
PZ = np.diag([1.0, -1.0]).astype(complex)
INPUT_STATES = {"0": np.array([1, 0], complex), "1": np.array([0, 1], complex),
                "+": np.array([1, 1], complex) / np.sqrt(2), "+i": np.array([1, 1j]) / np.sqrt(2)}


def _outputs(channel):
    return {k: channel(np.outer(v, v.conj())) for k, v in INPUT_STATES.items()}


# ------------------------------------------------------------- host logic

def test_chi_of_a_pauli_channel_is_its_probabilities():
    p = np.array([0.7, 0.1, 0.15, 0.05])
    chan = lambda r: p[0] * r + p[1] * PX @ r @ PX + p[2] * PY @ r @ PY + p[3] * PZ @ r @ PZ
    chi = C.chi_from_outputs(_outputs(chan))
    assert np.max(np.abs(chi - np.diag(p))) < 1e-14


def test_chi_of_a_unitary_is_rank_one():
    th = 0.8
    U = np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)])      # RZ(th) = cos I - i sin Z
    c = np.array([np.cos(th / 2), 0, 0, -1j * np.sin(th / 2)])
    chi = C.chi_from_outputs(_outputs(lambda r: U @ r @ U.conj().T))
    assert np.max(np.abs(chi - np.outer(c, c.conj()))) < 1e-14


def test_bloch_state_and_readout_fidelity():
    r = C.bloch_state(0.1, -0.2, 0.3, 0.9)
    assert abs(np.trace(r) - 0.9) < 1e-15
    assert abs(np.trace(r @ PY).real / 0.9 + 0.2) < 1e-15
    # |Phi+> after CX(0, 1), H(0) is |00>: readouts Tr = 1, <Z0> = <Z1> = <Z0Z1> = 1
    assert C.fidelity_from_readouts(1.0, 1.0, 1.0, 1.0) == 1.0
    assert C.fidelity_from_readouts(0.5, 0.5, 0.5, 0.5) == 1.0
    assert C.fidelity_from_readouts(0.5, 1.0, 1.0, 1.0, normalized=True) == 1.0


def test_circuit_shapes():
    n, ops = C.purification_ops(0.8, 0.02, 2)
    assert n == 8 and sum(1 for o in ops if o[0] == "kraus") == 3
    n, ops = C.purification_ops(0.8, 0.0, 1)
    assert n == 4 and all(max(o[1]) < 4 for o in ops)
    with pytest.raises(ValueError):
        C.purification_ops(0.8, 0.0, 3)
    ops = C.teleport_ops(C.DEVICE, C.TOMO_INPUTS["+i"], C.BASIS["y"])
    assert all(max(o[1]) < 3 for o in ops)
    assert sum(1 for o in ops if o[0] == "kraus") == 2          # readout on qubits 0 and 1


# ------------------------------------------------------------------- GPU

def _oracle_output(noise, inp):
    """2x2 state of qubit 2 after the teleportation circuit (oracle)."""
    rho = O.run_circuit(3, C.teleport_ops(noise, C.TOMO_INPUTS[inp], []))
    return np.einsum("aibi->ab", rho.reshape(2, 4, 2, 4))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_teleportation_chi_on_the_engine(tq, golden, precision):
    noises = [C.NOISELESS, C.DEVICE, C.DEVICE_WORSE, C.DeviceNoise(e10=0.02, e01=0.06)]
    chis, outs, _ = C.teleport_chi(tq, noises, precision)
    tol = TOL64 if precision == "fp64" else 2e-6
    assert np.max(np.abs(chis[0] - golden("teleport_chi_ideal.txt"))) < tol
    e = 0.04
    assert np.max(np.abs(chis[3] - np.diag([(1 - e) ** 2, e * (1 - e), e * e, e * (1 - e)]))) < tol
    for noise, chi, out in zip(noises, chis, outs):
        for k in INPUT_STATES:      # the channel's output states against the oracle
            assert np.max(np.abs(out[k] - _oracle_output(noise, k))) < tol, k
        # a channel: chi Hermitian, trace 1, positive semidefinite
        assert np.max(np.abs(chi - chi.conj().T)) < tol
        assert abs(np.trace(chi) - 1) < tol
        assert np.min(np.linalg.eigvalsh((chi + chi.conj().T) / 2)) > -10 * tol
    # noise lowers the process fidelity, more noise lowers it more
    f = [C.process_fidelity(c) for c in chis[:3]]
    assert f[0] > f[1] > f[2]


@pytest.mark.gpu
def test_purification_curves_on_the_engine(tq):
    Fs = [0.55, 0.7, 0.85, 0.95]
    ps = [0.0, 0.03, 0.1]
    curves, _ = C.purification_curves(tq, Fs, ps, rounds=2)
    for p in ps:
        for F, f_out, succ in curves[p]:
            n, ops = C.purification_ops(F, p, 2)
            rho = O.run_circuit(n, ops)
            tr = O.trace(rho).real
            p00 = sum(rho[x, x].real for x in range(1 << n) if x & 3 == 0)
            assert abs(succ - tr) < TOL64
            assert abs(f_out - p00 / tr) < TOL64
    # noise-free purification improves every input above 1/2; a 10% CX error
    # makes it worse than doing nothing for high-fidelity inputs
    assert all(f_out > F for F, f_out, _ in curves[0.0])
    assert curves[0.1][-1][1] < 0.95
