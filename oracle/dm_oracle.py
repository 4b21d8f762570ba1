"""Plain FP64 CPU oracle for noisy density-matrix circuit simulation.

TEST INFRASTRUCTURE ONLY. This module is the independent checker of the GPU
library. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it. The product path never calls it, and it
shares no code, table or helper with the CUDA library.

What it computes (TANQ-Sim, arXiv 2404.13184):

* Sec. 2.1, Eq. 1 (``eq:onegate``) and Eq. 2 (``eq:dmsim``): a circuit maps
  rho_in to rho_out = G_{m-1}( ... G_0(rho_in) ... ), where each step is a
  gate G rho G^dagger or, with noise, a channel.
* Sec. 3.1 (the Kraus sum under "When considering noise"): a noisy channel is
  a set of Kraus matrices K_i and acts as rho -> sum_i K_i rho K_i^dagger.
* Sec. 2.1 (text after Eq. 2): a k-qubit matrix acts on the n-qubit register
  as its Kronecker product with the identity on the other qubits.

The oracle applies these definitions directly to a dense (2^n, 2^n) complex128
matrix ``rho[r, c]``. It deliberately does not use the paper's vectorised
superoperator form (Sec. 3.1, Eq. ``eq:sp``): that is the method under test.

Conventions (the paper leaves them open; these readings are shared with the
library only through its documented API, never through code):

* qubit q is bit q of the row index r and of the column index c;
* a k-qubit matrix acts on an ordered qubit list Q; bit j of its local index
  is qubit Q[j] (Q[0] is the least significant local bit);
* CX on (Q[0], Q[1]) flips Q[1] when Q[0] is 1;
* RZ(t) = diag(e^{-it/2}, e^{it/2}), RX(t) = exp(-i t X/2),
  RZZ(t) = exp(-i t Z(x)Z/2);
* depolarising on k qubits with parameter p is
  E(rho) = (1-p) rho + p * (I_Q / 2^k) (x) Tr_Q(rho);
* amplitude damping with gamma has K0 = [[1,0],[0,sqrt(1-gamma)]],
  K1 = [[0,sqrt(gamma)],[0,0]];
* thermal relaxation (zero temperature) for time t with T1, T2 <= 2 T1 maps
  rho00 -> rho00 + (1-e^{-t/T1}) rho11, rho11 -> e^{-t/T1} rho11 and
  rho01 -> e^{-t/T2} rho01 (rho10 likewise);
* phase damping with lambda keeps populations and scales coherences by
  sqrt(1-lambda);
* reset of a qubit to |0> has Kraus operators |0><0| and |0><1|;
* measuring qubit q with outcome m projects with P_m = |m><m| on q and
  renormalises: rho -> P_m rho P_m / Tr(P_m rho); the outcome is 0 when a
  uniform draw u is below Tr(P_0 rho) / Tr(rho);
* readout error (Sec. 3.5): qubit q reads 1 when prepared in 0 with
  probability e10[q] and 0 when prepared in 1 with e01[q], independently per
  qubit, applied to the outcome probabilities of measuring every qubit;
* sampling a shot from outcome probabilities p takes the smallest x with
  u < sum_{y <= x} p[y] / sum p (inverse cumulative distribution).

The measurement and reset section announced in the paper is missing from
its text; these are the textbook definitions.

An op is a tuple ``(name, qubits, params)`` as produced by the workload
generators; ``("kraus", qubits, [K0, K1, ...])`` and ``("unitary", qubits,
[U])`` carry explicit matrices.

Every function here is pinned by ``tests/test_oracle.py`` to closed forms,
library routines (``numpy.kron``, ``scipy.linalg.expm``), a separate
state-vector simulator and brute-force Kronecker expansion.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "gate_matrix", "kraus_matrices", "apply_kraus", "apply_kraus_kron",
    "apply_depolarizing", "apply_thermal", "apply_op", "zero_state",
    "run_circuit", "trace", "expect_z", "probabilities", "sv_run",
    "measure", "readout_probabilities", "sample",
    "ONE_QUBIT_GATES", "TWO_QUBIT_GATES",
]

ONE_QUBIT_GATES = ("id", "h", "x", "y", "z", "s", "sdg", "t", "tdg", "sx",
                   "rx", "ry", "rz", "su2")
TWO_QUBIT_GATES = ("cx", "cz", "swap", "rzz")


# --------------------------------------------------------------------------
# Gates (textbook definitions)
# --------------------------------------------------------------------------

def gate_matrix(name: str, params=()) -> np.ndarray:
    """Unitary matrix of a named gate, in the local index order above."""
    c = complex
    if name == "id":
        return np.eye(2, dtype=np.complex128)
    if name == "h":
        return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    if name == "x":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if name == "y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if name == "z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if name == "s":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if name == "sdg":
        return np.array([[1, 0], [0, -1j]], dtype=np.complex128)
    if name == "t":
        return np.array([[1, 0], [0, np.exp(1j * math.pi / 4)]], dtype=np.complex128)
    if name == "tdg":
        return np.array([[1, 0], [0, np.exp(-1j * math.pi / 4)]], dtype=np.complex128)
    if name == "sx":
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
    if name == "rx":
        t = float(params[0])
        return np.array([[math.cos(t / 2), -1j * math.sin(t / 2)],
                         [-1j * math.sin(t / 2), math.cos(t / 2)]], dtype=np.complex128)
    if name == "ry":
        t = float(params[0])
        return np.array([[math.cos(t / 2), -math.sin(t / 2)],
                         [math.sin(t / 2), math.cos(t / 2)]], dtype=np.complex128)
    if name == "rz":
        t = float(params[0])
        return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)
    if name == "su2":
        # Haar-random SU(2) from four i.i.d. normal draws: normalising them
        # gives a uniform unit quaternion (a, b, c, d) (Shoemake 1992).
        a, b, cc, d = (float(v) for v in params)
        nrm = math.sqrt(a * a + b * b + cc * cc + d * d)
        a, b, cc, d = a / nrm, b / nrm, cc / nrm, d / nrm
        return np.array([[c(a, b), c(cc, d)], [c(-cc, d), c(a, -b)]], dtype=np.complex128)
    if name == "cx":
        # local index = b0 + 2*b1, b0 = control, b1 = target
        m = np.zeros((4, 4), dtype=np.complex128)
        for b0 in range(2):
            for b1 in range(2):
                out_b1 = b1 ^ b0
                m[b0 + 2 * out_b1, b0 + 2 * b1] = 1.0
        return m
    if name == "cz":
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if name == "swap":
        m = np.zeros((4, 4), dtype=np.complex128)
        for b0 in range(2):
            for b1 in range(2):
                m[b1 + 2 * b0, b0 + 2 * b1] = 1.0
        return m
    if name == "rzz":
        t = float(params[0])
        # Z(x)Z eigenvalue is +1 when the two bits agree, -1 otherwise
        ph = [np.exp(-0.5j * t * (1 if ((i & 1) == (i >> 1)) else -1)) for i in range(4)]
        return np.diag(ph).astype(np.complex128)
    raise ValueError(f"unknown gate {name!r}")


# --------------------------------------------------------------------------
# Kraus sets for channels that are defined by their Kraus operators
# --------------------------------------------------------------------------

def kraus_matrices(name: str, params=()) -> list[np.ndarray]:
    """Kraus operators of the channels the oracle applies through Kraus sums."""
    if name == "ad":
        g = float(params[0])
        k0 = np.array([[1, 0], [0, math.sqrt(1 - g)]], dtype=np.complex128)
        k1 = np.array([[0, math.sqrt(g)], [0, 0]], dtype=np.complex128)
        return [k0, k1]
    if name == "pd":
        lam = float(params[0])
        k0 = np.array([[1, 0], [0, math.sqrt(1 - lam)]], dtype=np.complex128)
        k1 = np.array([[0, 0], [0, math.sqrt(lam)]], dtype=np.complex128)
        return [k0, k1]
    if name == "reset":
        k0 = np.array([[1, 0], [0, 0]], dtype=np.complex128)
        k1 = np.array([[0, 1], [0, 0]], dtype=np.complex128)
        return [k0, k1]
    raise ValueError(f"no Kraus set for {name!r}")


# --------------------------------------------------------------------------
# Index helpers: which rows of the register a local matrix touches
# --------------------------------------------------------------------------

def _local_split(n: int, qubits) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """For every register index x in [0, 2^n): its local index (bits of x at
    ``qubits``), its base (x with those bits cleared), and for every local
    index b the register offset that sets those bits to b."""
    x = np.arange(1 << n, dtype=np.int64)
    loc = np.zeros_like(x)
    base = x.copy()
    for j, q in enumerate(qubits):
        bit = (x >> q) & 1
        loc |= bit << j
        base &= ~(np.int64(1) << q)
    k = len(qubits)
    dep = np.zeros(1 << k, dtype=np.int64)
    for b in range(1 << k):
        for j, q in enumerate(qubits):
            if (b >> j) & 1:
                dep[b] |= np.int64(1) << q
    return loc, base, dep


def _check_qubits(n: int, qubits) -> None:
    if len(set(qubits)) != len(qubits) or any(q < 0 or q >= n for q in qubits):
        raise ValueError(f"bad qubit list {qubits} for n={n}")


# --------------------------------------------------------------------------
# Channel application
# --------------------------------------------------------------------------

def apply_kraus(rho: np.ndarray, kraus, qubits) -> np.ndarray:
    """sum_i K_i rho K_i^dagger with each K_i acting on ``qubits``.

    (K rho)[r, :] = sum_b K[loc(r), b] * rho[base(r) | dep(b), :]   (row action)
    (A K^dag)[:, c] = sum_b A[:, base(c) | dep(b)] * conj(K[loc(c), b])
    """
    n = int(round(math.log2(rho.shape[0])))
    _check_qubits(n, qubits)
    loc, base, dep = _local_split(n, qubits)
    out = np.zeros_like(rho)
    for K in kraus:
        K = np.asarray(K, dtype=np.complex128)
        left = np.zeros_like(rho)
        for b in range(K.shape[1]):
            left += K[loc, b][:, None] * rho[base | dep[b], :]
        for b in range(K.shape[1]):
            out += left[:, base | dep[b]] * np.conj(K[loc, b])[None, :]
    return out


def apply_kraus_kron(rho: np.ndarray, kraus, qubits) -> np.ndarray:
    """Same channel through the full 2^n x 2^n operator (Kronecker product of
    K with the identity on the other qubits, Sec. 2.1) and dense matmuls.
    O(8^n): for small registers only, as a check of ``apply_kraus``."""
    n = int(round(math.log2(rho.shape[0])))
    _check_qubits(n, qubits)
    loc, base, _ = _local_split(n, qubits)
    same_rest = base[:, None] == base[None, :]
    out = np.zeros_like(rho)
    for K in kraus:
        full = np.where(same_rest, np.asarray(K, dtype=np.complex128)[loc[:, None], loc[None, :]], 0)
        out += full @ rho @ full.conj().T
    return out


def apply_depolarizing(rho: np.ndarray, p: float, qubits) -> np.ndarray:
    """(1-p) rho + p (I_Q / 2^k) (x) Tr_Q(rho) on the qubits Q."""
    n = int(round(math.log2(rho.shape[0])))
    _check_qubits(n, qubits)
    loc, base, dep = _local_split(n, qubits)
    k = len(qubits)
    # partial trace over Q, broadcast back to every (r, c): depends only on base(r), base(c)
    part = np.zeros_like(rho)
    for b in range(1 << k):
        idx = base | dep[b]
        part += rho[np.ix_(idx, idx)]
    same_loc = loc[:, None] == loc[None, :]
    return (1.0 - p) * rho + (p / (1 << k)) * np.where(same_loc, part, 0)


def apply_thermal(rho: np.ndarray, t: float, t1: float, t2: float, qubit: int) -> np.ndarray:
    """Zero-temperature thermal relaxation on one qubit, by its action on the
    2x2 blocks of rho (population transfer and coherence decay)."""
    if t2 > 2.0 * t1:
        raise ValueError("thermal relaxation needs T2 <= 2 T1")
    n = int(round(math.log2(rho.shape[0])))
    _check_qubits(n, [qubit])
    e1 = math.exp(-t / t1)
    e2 = math.exp(-t / t2)
    x = np.arange(1 << n, dtype=np.int64)
    a = ((x >> qubit) & 1)[:, None]
    b = ((x >> qubit) & 1)[None, :]
    flip = x | (np.int64(1) << qubit)
    out = np.where(a != b, e2 * rho, rho)
    out = np.where((a == 1) & (b == 1), e1 * rho, out)
    gain = (1.0 - e1) * rho[np.ix_(flip, flip)]
    out = np.where((a == 0) & (b == 0), rho + gain, out)
    return out


def apply_op(rho: np.ndarray, op) -> np.ndarray:
    """Apply one op ``(name, qubits, params)`` to rho."""
    name, qubits, params = op
    qubits = list(qubits)
    if name in ONE_QUBIT_GATES or name in TWO_QUBIT_GATES:
        return apply_kraus(rho, [gate_matrix(name, params)], qubits)
    if name == "unitary":
        return apply_kraus(rho, [np.asarray(params[0])], qubits)
    if name == "kraus":
        return apply_kraus(rho, [np.asarray(K) for K in params], qubits)
    if name == "depol":
        return apply_depolarizing(rho, float(params[0]), qubits)
    if name in ("ad", "pd", "reset"):
        return apply_kraus(rho, kraus_matrices(name, params), qubits)
    if name == "thermal":
        t, t1, t2 = (float(v) for v in params)
        for q in qubits:  # independently on each qubit of the gate
            rho = apply_thermal(rho, t, t1, t2, q)
        return rho
    raise ValueError(f"unknown op {name!r}")


def zero_state(n: int) -> np.ndarray:
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def run_circuit(n: int, ops, rho: np.ndarray | None = None) -> np.ndarray:
    """Eq. 2: apply the ops in order, starting from |0..0><0..0| by default."""
    rho = zero_state(n) if rho is None else np.array(rho, dtype=np.complex128)
    for op in ops:
        rho = apply_op(rho, op)
    return rho


# --------------------------------------------------------------------------
# Readouts
# --------------------------------------------------------------------------

def trace(rho: np.ndarray) -> complex:
    return complex(np.trace(rho))


def expect_z(rho: np.ndarray, mask: int) -> float:
    """Re Tr(rho Z_mask), Z_mask = tensor product of Z on the qubits in mask."""
    x = np.arange(rho.shape[0], dtype=np.int64)
    par = np.zeros_like(x)
    m = x & int(mask)
    while np.any(m):
        par ^= m & 1
        m >>= 1
    sign = 1.0 - 2.0 * par
    return float(np.sum(sign * np.real(np.diag(rho))))


def probabilities(rho: np.ndarray) -> np.ndarray:
    """Outcome probabilities of measuring every qubit: the real diagonal."""
    return np.real(np.diag(rho)).copy()


# --------------------------------------------------------------------------
# Separate state-vector simulator (noise-free circuits), for cross-checks
# --------------------------------------------------------------------------

def sv_run(n: int, ops) -> np.ndarray:
    """Apply unitary ops to |0..0> with tensor contractions over qubit axes.
    The state is reshaped to n axes of size 2, axis n-1-q holding qubit q."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    psi = psi.reshape((2,) * n)
    for name, qubits, params in ops:
        if name == "unitary":
            U = np.asarray(params[0], dtype=np.complex128)
        elif name in ONE_QUBIT_GATES or name in TWO_QUBIT_GATES:
            U = gate_matrix(name, params)
        else:
            raise ValueError(f"sv_run handles unitary ops only, got {name!r}")
        k = len(qubits)
        # U as a tensor: out axes (bit k-1 .. bit 0), then in axes likewise
        Ut = U.reshape((2,) * (2 * k))
        in_axes = [k + (k - 1 - j) for j in range(k)]          # U input axis of local bit j
        st_axes = [n - 1 - qubits[j] for j in range(k)]        # state axis of qubit Q[j]
        res = np.tensordot(Ut, psi, axes=(in_axes, st_axes))   # out axes of U first
        # result axes: U out (bit k-1..0), then the untouched state axes in order
        rest = [a for a in range(n) if a not in st_axes]
        order = [None] * n
        for j in range(k):
            order[n - 1 - qubits[j]] = (k - 1 - j)
        for pos, a in enumerate(rest):
            order[a] = k + pos
        psi = np.transpose(res, order)
    return psi.reshape(-1)


# --------------------------------------------------------------------------
# Measurement, readout error and sampling
# --------------------------------------------------------------------------

def measure(rho: np.ndarray, qubit: int, u: float):
    """Selective measurement of one qubit: (outcome, probability, new rho)."""
    n = int(round(math.log2(rho.shape[0])))
    _check_qubits(n, [qubit])
    d = np.real(np.diag(rho))
    x = np.arange(rho.shape[0])
    p0 = float(np.sum(d[((x >> qubit) & 1) == 0]))
    tr = float(np.sum(d))
    m = 0 if u < p0 / tr else 1
    pm = p0 if m == 0 else tr - p0
    P = np.zeros((2, 2), dtype=np.complex128)
    P[m, m] = 1.0
    out = apply_kraus(rho, [P], [qubit]) / pm
    return m, pm / tr, out


def readout_probabilities(p: np.ndarray, e10, e01) -> np.ndarray:
    """Outcome probabilities after independent per-qubit readout errors:
    the 2x2 confusion matrix [[1-e10, e01], [e10, 1-e01]] on every qubit."""
    p = np.array(p, dtype=np.float64)
    n = int(round(math.log2(p.shape[0])))
    t = p.reshape((2,) * n)
    for q in range(n):
        A = np.array([[1 - e10[q], e01[q]], [e10[q], 1 - e01[q]]])
        ax = n - 1 - q
        t = np.moveaxis(np.tensordot(A, t, axes=([1], [ax])), 0, ax)
    return t.reshape(-1)


def sample(p: np.ndarray, uniforms) -> np.ndarray:
    """Inverse-CDF samples: for each u the smallest x with u < cdf[x] / cdf[-1]."""
    cdf = np.cumsum(np.asarray(p, dtype=np.float64))
    return np.searchsorted(cdf / cdf[-1], np.asarray(uniforms), side="right")
