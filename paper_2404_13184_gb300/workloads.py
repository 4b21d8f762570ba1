"""Seeded synthetic circuits shaped like the paper's workloads.

This module only draws random numbers and lists ops; it holds none of the
simulation arithmetic. Both the GPU library (through its Python binding) and
the CPU oracle consume its output, so it must stay free of either.

An op is ``(name, qubits, params)``:

* gates: ``h x y z s sdg t tdg sx rx ry rz su2`` (1 qubit) and
  ``cx cz swap rzz`` (2 qubits); ``rx/ry/rz/rzz`` take one angle,
  ``su2`` takes four i.i.d. standard-normal draws (the library and the
  oracle each normalise them into a unit quaternion);
* channels: ``depol`` (p; on the op's 1 or 2 qubits), ``ad`` (gamma; 1
  qubit), ``pd`` (lambda; 1 qubit), ``thermal`` (t, T1, T2; independently on
  every listed qubit).

A "noisy gate" (the unit of the throughput metric) is one circuit gate
together with the channels attached after it (TANQ-Sim Sec. 3.1 builds one
superoperator per noisy gate).

The paper's own benchmark circuits (QASMBench, Table 3 and Table 4) are not
used; these generators stand in for them with the same scale: 4-15 qubits,
hundreds to thousands of basis-level gates, 1- and 2-qubit gates with
depolarising, amplitude-damping and thermal-relaxation noise (Sec. 3.5).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2404_13184


@dataclasses.dataclass
class Circuit:
    n: int
    ops: list
    n_gates: int                      # noisy gates (circuit gates)
    steps: list | None = None         # op index ranges per Trotter step (TFIM)
    label: str = ""


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_noisy_circuit(n: int, n_gates: int, seed: int, gate_set=("h", "x", "s", "rz", "cx"),
                         p1: float = 1e-3, p2: float = 1e-2, gamma: float = 5e-4) -> Circuit:
    """Gates drawn uniformly from ``gate_set``; each 1-qubit gate is followed
    by 1-qubit depolarising p1, each 2-qubit gate by 2-qubit depolarising p2
    and amplitude damping gamma on both of its qubits (p/gamma of 0 omit the
    channel). Targets are uniform over distinct qubits."""
    rng = _rng(seed)
    ops = []
    for _ in range(n_gates):
        g = gate_set[int(rng.integers(len(gate_set)))]
        if g in ("cx", "cz", "swap", "rzz"):
            q = [int(v) for v in rng.choice(n, size=2, replace=False)]
            params = (float(rng.uniform(0, 2 * math.pi)),) if g == "rzz" else ()
            ops.append((g, q, params))
            if p2 > 0:
                ops.append(("depol", q, (p2,)))
            if gamma > 0:
                ops.append(("ad", [q[0]], (gamma,)))
                ops.append(("ad", [q[1]], (gamma,)))
        else:
            q = [int(rng.integers(n))]
            if g in ("rx", "ry", "rz"):
                params = (float(rng.uniform(0, 2 * math.pi)),)
            elif g == "su2":
                params = tuple(float(v) for v in rng.standard_normal(4))
            else:
                params = ()
            ops.append((g, q, params))
            if p1 > 0:
                ops.append(("depol", q, (p1,)))
    return Circuit(n=n, ops=ops, n_gates=n_gates, label=f"random{n}q{n_gates}g")


def plain_6q(seed: int = SEED_BASE + 1) -> Circuit:
    """6 qubits, 200 random gates from {H, X, S, RZ, CX}; depolarising 1e-3
    after 1-qubit gates, 2-qubit depolarising 1e-2 plus amplitude damping
    5e-4 on both qubits after CX. Run unfused in FP64."""
    c = random_noisy_circuit(6, 200, seed)
    c.label = "plain-6q-200g"
    return c


def layered_thermal(n: int = 12, n_gates: int = 2000, seed: int = SEED_BASE + 2,
                    t1: float = 100e-6, t2: float = 80e-6, t_1q: float = 50e-9,
                    t_2q: float = 300e-9) -> Circuit:
    """Alternating layers: n Haar SU(2) gates, then CX on a brick pattern of a
    line (even pairs (0,1),(2,3),..., next time odd pairs (1,2),(3,4),...),
    repeated until exactly ``n_gates`` gates (the last layer truncated).
    Every gate is followed by thermal relaxation (T1, T2) for its gate time,
    independently on each of its qubits."""
    rng = _rng(seed)
    ops = []
    count = 0
    layer = 0
    while count < n_gates:
        if layer % 2 == 0:
            for q in range(n):
                if count >= n_gates:
                    break
                ops.append(("su2", [q], tuple(float(v) for v in rng.standard_normal(4))))
                ops.append(("thermal", [q], (t_1q, t1, t2)))
                count += 1
        else:
            start = 0 if (layer // 2) % 2 == 0 else 1
            for a in range(start, n - 1, 2):
                if count >= n_gates:
                    break
                ops.append(("cx", [a, a + 1], ()))
                ops.append(("thermal", [a, a + 1], (t_2q, t1, t2)))
                count += 1
        layer += 1
    return Circuit(n=n, ops=ops, n_gates=n_gates, label=f"layered-thermal-{n}q-{n_gates}g")


def tfim_ring(n: int = 15, steps: int = 30, J: float = 1.0, h: float = 0.5, dt: float = 0.1,
              p: float = 5e-4) -> Circuit:
    """Transverse-field Ising Trotter circuit on a ring: per step RZZ(2 J dt)
    on every neighbour pair (i, i+1 mod n), then RX(2 h dt) on every qubit;
    2-qubit depolarising p after every RZZ and 1-qubit depolarising p after
    every RX. ``steps`` lists the op range of each Trotter step; the
    observable is <Z_0 Z_1> after each step. Deterministic (no draws)."""
    ops = []
    ranges = []
    for _ in range(steps):
        s0 = len(ops)
        for i in range(n):
            pair = [i, (i + 1) % n]
            ops.append(("rzz", pair, (2 * J * dt,)))
            ops.append(("depol", pair, (p,)))
        for i in range(n):
            ops.append(("rx", [i], (2 * h * dt,)))
            ops.append(("depol", [i], (p,)))
        ranges.append((s0, len(ops)))
    return Circuit(n=n, ops=ops, n_gates=2 * n * steps, steps=ranges, label=f"tfim-ring-{n}q-{steps}steps")


def sweep(count: int = 1024, seed: int = SEED_BASE + 4, n_min: int = 4, n_max: int = 11,
          d_min: int = 50, d_max: int = 500) -> list[Circuit]:
    """Batched noise-parameter sweep: ``count`` circuits, n ~ U{n_min..n_max},
    depth ~ U{d_min..d_max}, gates uniform over {H, RZ, RX, CX}, depolarising
    p log-uniform in [1e-4, 1e-2] per circuit (1-qubit after 1-qubit gates,
    2-qubit after CX)."""
    rng = _rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_min, n_max + 1))
        depth = int(rng.integers(d_min, d_max + 1))
        p = float(10 ** rng.uniform(-4, -2))
        sub_seed = int(rng.integers(1 << 62))
        c = random_noisy_circuit(n, depth, sub_seed, gate_set=("h", "rz", "rx", "cx"), p1=p, p2=p, gamma=0.0)
        c.label = f"sweep{i}-{n}q-{depth}g-p{p:.2e}"
        out.append(c)
    return out


def served_request(rng: np.random.Generator, n_min: int = 5, n_max: int = 15, d_min: int = 50,
                   d_max: int = 2000, frac_2q: float = 0.3) -> Circuit:
    """One served request: n ~ U{n_min..n_max}, depth ~ U{d_min..d_max}, a
    fraction ``frac_2q`` of CX gates, other gates uniform over {H, RX, RZ};
    per request depolarising p log-uniform in [1e-4, 1e-2] after every gate and
    amplitude damping gamma log-uniform in [1e-5, 1e-3] on every gate qubit."""
    n = int(rng.integers(n_min, n_max + 1))
    depth = int(rng.integers(d_min, d_max + 1))
    p = float(10 ** rng.uniform(-4, -2))
    gamma = float(10 ** rng.uniform(-5, -3))
    # per-gate draws in bulk: gate kind, qubits (a CX pair uniform over
    # ordered pairs of distinct qubits), 1-qubit gate and angle
    two = (rng.uniform(size=depth) < frac_2q).tolist()
    qa = rng.integers(n, size=depth).tolist()
    qb = rng.integers(max(1, n - 1), size=depth).tolist()
    g1 = rng.integers(3, size=depth).tolist()
    ang = rng.uniform(0, 2 * math.pi, size=depth).tolist()
    ops = []
    for t in range(depth):
        a = qa[t]
        if two[t]:
            b = qb[t] + (qb[t] >= a)
            q = [a, b]
            ops.append(("cx", q, ()))
            ops.append(("depol", q, (p,)))
            ops.append(("ad", [a], (gamma,)))
            ops.append(("ad", [b], (gamma,)))
        else:
            g = ("h", "rx", "rz")[g1[t]]
            q = [a]
            ops.append((g, q, () if g == "h" else (ang[t],)))
            ops.append(("depol", q, (p,)))
            ops.append(("ad", q, (gamma,)))
    return Circuit(n=n, ops=ops, n_gates=depth, label=f"req-{n}q-{depth}g")


def poisson_arrivals(rate: float = 200.0, duration: float = 60.0, seed: int = SEED_BASE + 5) -> list[float]:
    """Arrival times of a Poisson process with ``rate`` per second on [0, duration)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            return out
        out.append(t)


def ghz(n: int) -> list:
    """Noise-free GHZ preparation: H on qubit 0, then CX (0, i) for i = 1..n-1."""
    ops = [("h", [0], ())]
    for i in range(1, n):
        ops.append(("cx", [0, i], ()))
    return ops


def product_prefix(n: int, seed: int) -> list:
    """A random single-qubit SU(2) followed by amplitude damping on every
    qubit: leaves a product state whose factors are each a generic 2x2
    density matrix (used for full-size checks that factor over qubits)."""
    rng = _rng(seed)
    ops = []
    for q in range(n):
        ops.append(("su2", [q], tuple(float(v) for v in rng.standard_normal(4))))
        ops.append(("ad", [q], (float(rng.uniform(0.05, 0.3)),)))
    return ops


def random_kraus(k: int, m: int, seed: int) -> list[np.ndarray]:
    """m random complex 2^k x 2^k matrices (i.i.d. normal entries), unnormalised:
    generic non-CPTP Kraus sets are allowed (the paper's G need not be unitary)."""
    rng = _rng(seed)
    d = 1 << k
    return [(rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / d for _ in range(m)]


def random_density_matrix(n: int, seed: int) -> np.ndarray:
    """A random full-rank density matrix (Wishart, normalised to trace 1)."""
    rng = _rng(seed)
    d = 1 << n
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    r = a @ a.conj().T
    return r / np.trace(r).real
