"""Measurement, reset, readout error and sampling on the GPU against the
oracle (FP64 1e-12; split within its bound)."""
import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _circuit(n, seed):
    c = W.random_noisy_circuit(n, 40, seed, gate_set=("h", "rx", "rz", "cx", "su2"))
    return c.ops + [("reset", [n - 1], ()), ("h", [n - 1], ()), ("depol", [n - 1], (0.05,))]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 2e-6)])
def test_reset_in_circuits(tq, precision, tol):
    n = 6
    ops = _circuit(n, 3)
    want = O.run_circuit(n, ops)
    with tq.State(n, precision) as st:
        st.run(ops, width=-1)
        assert np.max(np.abs(st.rho() - want)) < tol


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_selective_measurement_sequence(tq, precision):
    n = 6
    ops = _circuit(n, 4)
    rho = O.run_circuit(n, ops)
    rng = np.random.default_rng(7)
    with tq.State(n, precision) as st:
        st.run(ops, width=-1)
        for q in (0, 3, 5, 1):
            u = float(rng.uniform())
            m_want, p_want, rho = O.measure(rho, q, u)
            m, p = st.measure(q, u)
            if precision == "split" and abs(u - (p_want if m_want == 0 else 1 - p_want)) < 1e-5:
                pytest.skip("draw too close to the outcome boundary for FP32 storage")
            assert m == m_want
            assert abs(p - p_want) < (1e-12 if precision == "fp64" else 1e-6)
            assert np.max(np.abs(st.rho() - rho)) < (1e-12 if precision == "fp64" else 5e-6)
        # measured qubits now have definite values
        for q in (0, 3, 5, 1):
            z = st.expect_z([1 << q])[0]
            assert abs(abs(z) - 1) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("split", 1e-6)])
def test_readout_probabilities(tq, precision, tol):
    n = 7
    ops = _circuit(n, 5)
    rho = O.run_circuit(n, ops)
    rng = np.random.default_rng(8)
    e10 = rng.uniform(0, 0.05, n)
    e01 = rng.uniform(0, 0.1, n)
    want = O.readout_probabilities(O.probabilities(rho), e10, e01)
    with tq.State(n, precision) as st:
        st.run(ops, width=-1)
        got = st.probs_readout(e10, e01)
        plain = st.probs()
    assert np.max(np.abs(got - want)) < tol
    assert abs(np.sum(got) - 1) < tol * 10
    assert np.max(np.abs(plain - O.probabilities(rho))) < tol


def test_sampling_matches_inverse_cdf(tq):
    n = 8
    ops = _circuit(n, 6)
    rho = O.run_circuit(n, ops)
    rng = np.random.default_rng(9)
    u = rng.uniform(size=20000)
    e10, e01 = np.full(n, 0.02), np.full(n, 0.04)
    with tq.State(n, "fp64") as st:
        st.run(ops, width=-1)
        got = st.sample(u)
        got_ro = st.sample(u, e10, e01)
    for probs, g in ((O.probabilities(rho), got), (O.readout_probabilities(O.probabilities(rho), e10, e01), got_ro)):
        want = O.sample(probs, u)
        cdf = np.cumsum(probs) / np.sum(probs)
        diff = np.nonzero(g != want)[0]
        # outcomes may differ only where u sits on a CDF boundary (summation order)
        for i in diff:
            assert np.min(np.abs(cdf - u[i])) < 1e-12
        assert len(diff) <= 2
        # and the histogram matches the probabilities
        hist = np.bincount(g.astype(np.int64), minlength=1 << n) / len(u)
        assert np.max(np.abs(hist - probs)) < 0.02


def test_measurement_argument_errors(tq):
    with tq.State(3, "fp64") as st:
        with pytest.raises(tq.TqError):
            st.measure(3, 0.5)
        with pytest.raises(tq.TqError):
            st.measure(0, 1.0)
        with pytest.raises(tq.TqError):
            st.probs_readout([0.1, 0.2, 1.5], [0, 0, 0])
        with pytest.raises(tq.TqError):
            st.sample([0.2, -0.1])
        assert list(st.sample([0.0, 0.5, 0.999])) == [0, 0, 0]      # |000>
