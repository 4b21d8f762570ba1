"""GPU parity of the FP64-accurate tensor-core engine (TQ_ENGINE_TENSOR):
FP64 states whose width-1 and width-2 blocks run on the tcgen05 tensor cores
through fixed-point digit slicing (csrc/tq_apply_oz.cu). The bar is the FP64
one: 1e-12 max-abs against the oracle on every entry, trace and <Z>."""
import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W
from test_gpu_parity import TOL64, _factorised_check, maxabs, random_general_matrix

pytestmark = pytest.mark.gpu

# registers of at least 6 qubits (the tile walk needs 16 row-rest values);
# every ordered target pattern: low and high bits, reversed order, adjacent
# and far apart
CASES = {
    6: [(0,), (5,), (0, 1), (1, 0), (5, 4), (0, 5), (3, 1)],
    7: [(0,), (3,), (6,), (0, 1), (6, 5), (2, 6), (6, 0)],
    9: [(4,), (8,), (0, 8), (7, 2), (4, 5)],
}


@pytest.mark.parametrize("n", sorted(CASES))
def test_single_kraus_op_every_position(tq, n):
    rho = W.random_density_matrix(n, 200 + n)
    for ci, qubits in enumerate(CASES[n]):
        k = len(qubits)
        Ks = W.random_kraus(k, 3, 2000 * n + ci)          # generic, not trace preserving
        want = O.apply_kraus(rho, Ks, list(qubits))
        with tq.State(n, "fp64", engine="tensor") as st:
            assert st.fp64_on_tensor() and st.hermitian_mode()
            st.set_rho(rho)
            assert st.hermitian_mode()
            st.apply_kraus(list(qubits), Ks)
            got = st.rho()
        assert maxabs(got, want) < TOL64, (qubits, maxabs(got, want))


def test_scaled_operands_keep_relative_accuracy(tq):
    # entries far from 1 and a superoperator with large entries: the digit
    # alignment follows the exponents of each group and each row
    n = 6
    rho = W.random_density_matrix(n, 7) * 3.0e-7
    Ks = [k * 40.0 for k in W.random_kraus(2, 2, 8)]
    want = O.apply_kraus(rho, Ks, [1, 4])
    with tq.State(n, "fp64", engine="tensor") as st:
        st.set_rho(rho)
        st.apply_kraus([1, 4], Ks)
        got = st.rho()
    assert maxabs(got, want) < 1e-14 * np.max(np.abs(want)) * 64, maxabs(got, want) / np.max(np.abs(want))


@pytest.mark.parametrize("width", [0, 1, 2, -1])
@pytest.mark.parametrize("n", [6, 8, 10])
def test_noisy_circuits_match_oracle(tq, n, width):
    c = W.random_noisy_circuit(n, 80, 500 + n, gate_set=("h", "rx", "rz", "cx", "su2", "rzz"))
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "fp64", engine="tensor") as st:
        st.run(c.ops, width=width)
        got = st.rho()
        tr = st.trace()
        z = st.expect_z([1, 3, (1 << n) - 1])
    assert maxabs(got, want) < TOL64
    assert abs(tr - O.trace(want)) < TOL64
    for v, m in zip(z, [1, 3, (1 << n) - 1]):
        assert abs(v - O.expect_z(want, m)) < TOL64


def test_tfim_8q_zz_per_step(tq):
    c = W.tfim_ring(n=8, steps=30)
    rho = O.zero_state(c.n)
    worst = 0.0
    with tq.State(c.n, "fp64", engine="tensor") as st:
        for (s0, s1) in c.steps:
            rho = O.run_circuit(c.n, c.ops[s0:s1], rho)
            st.run(c.ops[s0:s1], width=-1)
            worst = max(worst, abs(st.expect_z([0b11])[0] - O.expect_z(rho, 0b11)))
        assert abs(st.trace() - 1) < TOL64
        got = st.rho()
    assert worst < TOL64, worst
    assert maxabs(got, rho) < TOL64


def test_layered_thermal_matches_oracle(tq):
    c = W.layered_thermal(n=8, n_gates=200)
    want = O.run_circuit(c.n, c.ops)
    with tq.State(c.n, "fp64", engine="tensor") as st:
        st.run(c.ops, width=2)
        assert maxabs(st.rho(), want) < TOL64


def test_engines_agree_and_device_program_matches(tq):
    # the same circuit on DFMA and tensor engines (to FP64 accuracy), and a
    # device program (captured graph, replayed twice) equal to the host call
    n = 9
    c = W.random_noisy_circuit(n, 60, 77, gate_set=("h", "rx", "rz", "cx", "su2", "rzz"))
    with tq.State(n, "fp64", engine="dfma") as st:
        st.run(c.ops, width=2)
        ref = st.rho()
    with tq.State(n, "fp64", engine="tensor") as st:
        st.run(c.ops, width=2)
        host = st.rho()
    assert maxabs(host, ref) < TOL64
    prog = tq.DeviceProgram(n, c.ops, width=2, precision="fp64")
    with tq.State(n, "fp64", engine="tensor") as st:
        for _ in range(2):
            st.reset()
            st.run_program(prog)
            assert np.array_equal(st.rho(), host)
    prog.free()


def test_full_size_15q_factorised(tq):
    # the 15-qubit register of the benchmark, sampled entries against the
    # oracle's factors
    _factorised_check(tq, 15, [0, 6, 13, 14], -1, "fp64", 12, 15, engine="tensor")


def test_max_size_16q_factorised(tq):
    _factorised_check(tq, 16, [0, 7, 14, 15], 2, "fp64", 10, 17, engine="tensor")


def test_tensor_wait_timeout_is_reported(tq):
    # failure path: MMAs and commit skipped, the bounded wait runs out, the
    # next readout reports TQ_ERR_TIMEOUT and poisons the state, the context
    # stays usable
    n = 8
    c = W.tfim_ring(n, 1)
    try:
        tq.test_tc_wait_limit(2000, skip_mma=True)
        with tq.State(n, "fp64", engine="tensor") as st:
            st.run(c.ops, width=2)
            with pytest.raises(tq.TqError) as e:
                st.expect_z([3])
            assert e.value.status == 5          # TQ_ERR_TIMEOUT
            with pytest.raises(tq.TqError) as e:
                st.trace()
            assert e.value.status == 6          # TQ_ERR_STATE
    finally:
        tq.test_tc_wait_limit(0, skip_mma=False)
    want = O.run_circuit(n, c.ops)
    with tq.State(n, "fp64", engine="tensor") as st:
        st.run(c.ops, width=2)
        assert maxabs(st.rho(), want) < TOL64
