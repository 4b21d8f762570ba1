"""CPU tests of the C-ABI library: it loads, exports every function the
header declares, and its host-side logic (gate and channel library, fusion
planner, group-base index) is right. No GPU work is started."""
import itertools
import math
import os
import re
import subprocess

import numpy as np
import pytest

from oracle import dm_oracle as O
from paper_2404_13184_gb300 import binding as B
from paper_2404_13184_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tanq.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2404_13184_gb300 import build
        build.build()
    return B.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tq_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tq_[a-z0-9_]+)\b", out))
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(lib, f)
    bound = {name for name, _, _ in B._SIGNATURES}
    assert set(declared) == bound, set(declared) ^ bound


def _enum_values(body: str) -> dict:
    vals, nxt = {}, 0
    for item in body.split(","):
        item = item.strip()
        if not item:
            continue
        if "=" in item:
            name, v = item.split("=")
            nxt = int(v.strip())
            name = name.strip()
        else:
            name = item
        vals[name] = nxt
        nxt += 1
    return vals


def test_binding_enums_match_header():
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    enums = {}
    for body, name in re.findall(r"typedef enum \{(.*?)\}\s*(\w+);", src, flags=re.S):
        enums[name] = _enum_values(body)
    g = enums["tq_gate"]
    for k, v in B.GATES.items():
        assert g["TQ_GATE_" + k.upper()] == v, k
    c = enums["tq_channel"]
    names = {"depol": "TQ_CH_DEPOLARIZING", "ad": "TQ_CH_AMPLITUDE_DAMPING", "pd": "TQ_CH_PHASE_DAMPING",
             "thermal": "TQ_CH_THERMAL", "reset": "TQ_CH_RESET"}
    for k, v in B.CHANNELS.items():
        assert c[names[k]] == v
    assert enums["tq_precision"] == {"TQ_FP64": 0, "TQ_SPLIT": 1}
    assert enums["tq_op_kind"]["TQ_OP_KRAUS"] == B.OP_KRAUS
    assert enums["tq_op_kind"]["TQ_OP_CHANNEL"] == B.OP_CHANNEL
    st = enums["tq_status"]
    for v, name in B.STATUS.items():
        assert st[name] == v


def test_op_struct_layout():
    # C layout: 8 int32 (32 B), 4 doubles (32 B), one pointer -> 72 bytes
    assert B.ctypes.sizeof(B.TqOp) == 72
    assert B.TqOp.params.offset == 32 and B.TqOp.mats.offset == 64


@pytest.mark.parametrize("name", sorted(B.GATES))
def test_gate_library_matches_oracle(lib, name):
    params = (0.3, -1.1, 0.7, 2.2) if name == "su2" else (1.234,)
    assert np.max(np.abs(B.gate_matrix(name, params) - O.gate_matrix(name, params))) < 1e-15


@pytest.mark.parametrize("name,k,params", [
    ("depol", 1, (0.013,)), ("depol", 2, (0.2,)), ("depol", 1, (1.0,)),
    ("ad", 1, (5e-4,)), ("ad", 1, (0.4,)), ("pd", 1, (0.3,)),
    ("thermal", 1, (50e-9, 100e-6, 80e-6)), ("thermal", 2, (300e-9, 100e-6, 80e-6)),
    ("thermal", 1, (2e-5, 10e-6, 20e-6)), ("reset", 1, ()),
])
def test_channel_kraus_sets_act_like_the_oracle_channels(lib, name, k, params):
    Ks = B.channel_kraus(name, k, params)
    d = 1 << k
    # trace preserving
    tp = sum(K.conj().T @ K for K in Ks)
    assert np.max(np.abs(tp - np.eye(d))) < 1e-14
    # same action as the oracle's definition of the channel, on random states
    n = 3
    rho = W.random_density_matrix(n, 3) + 0.3j * W.random_density_matrix(n, 4)
    for qubits in itertools.permutations(range(n), k):
        want = O.apply_op(rho, (name, list(qubits), params))
        got = O.apply_kraus(rho, Ks, list(qubits))
        assert np.max(np.abs(got - want)) < 1e-14


def test_host_argument_errors(lib):
    with pytest.raises(B.TqError):
        B.channel_kraus("thermal", 1, (1e-6, 1e-5, 3e-5))   # T2 > 2 T1
    with pytest.raises(B.TqError):
        B.channel_kraus("depol", 3, (0.1,))
    with pytest.raises(B.TqError):
        B.channel_kraus("ad", 1, (1.5,))
    with pytest.raises(B.TqError):
        B.gate_matrix("su2", (0, 0, 0, 0))
    with pytest.raises(B.TqError):
        B.plan_fusion(3, [("h", [3], ())], 2)                # qubit out of range
    with pytest.raises(B.TqError):
        B.plan_fusion(3, [("cx", [1, 1], ())], 2)            # repeated qubit


def test_group_base_is_the_papers_s_i_for_one_qubit(lib):
    # Sec. 3.1: s_i = floor(floor(i/2^q)/2^(n-1)) 2^(q+n+1) + (floor(i/2^q) % 2^(n-1)) 2^(q+1) + (i % 2^q)
    for n in range(1, 6):
        for q in range(n):
            for i in range(4 ** (n - 1)):
                t = i // 2 ** q
                s_i = (t // 2 ** (n - 1)) * 2 ** (q + n + 1) + (t % 2 ** (n - 1)) * 2 ** (q + 1) + i % 2 ** q
                assert B.group_base(i, [q, q + n]) == s_i


def test_group_base_enumerates_each_index_once(lib):
    # the bases of all groups plus all target-bit offsets tile [0, 4^n) exactly once
    n = 4
    for qubits in [(0,), (3,), (1, 2), (2, 0), (0, 1, 3), (3, 1, 0, 2)]:
        k = len(qubits)
        pos = list(qubits) + [q + n for q in qubits]
        seen = np.zeros(4 ** n, dtype=int)
        for g in range(4 ** (n - k)):
            base = B.group_base(g, pos)
            for l in range(4 ** k):
                off = sum(((l >> j) & 1) << qubits[j] for j in range(k))
                off += sum(((l >> (k + j)) & 1) << (qubits[j] + n) for j in range(k))
                seen[base + off] += 1
        assert np.all(seen == 1)


def _check_plan_valid(n, ops, boo, widths, cap):
    nb = len(widths)
    assert all(0 <= b < nb for b in boo)
    # every block's width = number of distinct qubits of its ops, within the cap
    for b in range(nb):
        qs = set()
        for i, o in enumerate(ops):
            if boo[i] == b:
                qs |= set(o[1])
        assert len(qs) == widths[b] and widths[b] <= cap
    # ops sharing a qubit keep their order (block index non-decreasing), so the
    # fused product equals the circuit
    for i, j in itertools.combinations(range(len(ops)), 2):
        if set(ops[i][1]) & set(ops[j][1]):
            assert boo[i] <= boo[j], (i, j)


@pytest.mark.parametrize("width", [0, 1, 2, 3, 4, -1])
@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_fusion_plans_are_valid(lib, width, precision):
    circ = W.random_noisy_circuit(7, 150, 5, gate_set=("h", "rz", "cx", "su2", "rzz"))
    boo, widths = B.plan_fusion(circ.n, circ.ops, width, precision)
    cap = 4 if width == -1 else width
    if width == 0:
        assert boo == list(range(len(circ.ops)))
        assert widths == [len(o[1]) for o in circ.ops]
    else:
        _check_plan_valid(circ.n, circ.ops, boo, widths, max(cap, 2))
        if width >= 2:
            assert len(widths) < len(circ.ops)


def test_fusion_merges_noisy_gate_and_its_channels(lib):
    # a CX with its 2q depolarising and the two amplitude-damping channels: one block at width 2
    ops = [("cx", [0, 2], ()), ("depol", [0, 2], (0.01,)), ("ad", [0], (1e-3,)), ("ad", [2], (1e-3,))]
    boo, widths = B.plan_fusion(3, ops, 2)
    assert boo == [0, 0, 0, 0] and widths == [2]
    # TFIM step at width 2: RZZ blocks absorb the RX that follow on their qubits
    c = W.tfim_ring(6, 1)
    boo, widths = B.plan_fusion(6, c.ops, 2)
    assert len(widths) == 6 and all(w == 2 for w in widths)
    # width 1 cannot hold a 2-qubit op: it gets its own block
    boo, widths = B.plan_fusion(3, ops, 1)
    assert widths[boo[0]] == 2


def test_fusion_respects_commutation_barriers(lib):
    # H(0); CX(0,1); H(0): the second H must not join the first H's block
    ops = [("h", [0], ()), ("cx", [0, 1], ()), ("h", [0], ())]
    boo, widths = B.plan_fusion(2, ops, 1)
    assert boo[0] != boo[2] and boo[0] < boo[1] < boo[2]
    boo, widths = B.plan_fusion(2, ops, 2)
    assert boo == [0, 0, 0]


def _superop(Ks):
    # S = sum conj(K) (x) K with local index r + d c: numpy.kron(conj(K), K)
    return sum(np.kron(np.conj(K), K) for K in Ks)


@pytest.mark.parametrize("op", [
    ("rzz", [0, 1], (0.3,)), ("cx", [0, 1], ()), ("cz", [1, 0], ()), ("rz", [0], (1.1,)), ("h", [0], ()),
    ("rx", [0], (0.4,)), ("su2", [0], (0.1, 0.2, 0.3, 0.4)),
    ("depol", [0], (0.01,)), ("depol", [0, 1], (0.05,)), ("ad", [0], (0.2,)), ("pd", [0], (0.3,)),
    ("thermal", [0], (5e-8, 1e-4, 8e-5)),
])
def test_op_patterns_cover_the_superoperator(lib, op):
    name, q, params = op
    pat = B.op_pattern(op)
    if name in O.ONE_QUBIT_GATES or name in O.TWO_QUBIT_GATES:
        Ks = [O.gate_matrix(name, params)]
    elif name == "depol":
        Ks = B.channel_kraus("depol", len(q), params)
    elif name == "thermal":
        Ks = B.channel_kraus("thermal", 1, params)
    else:
        Ks = O.kraus_matrices(name, params)
    S = _superop(Ks)
    nz = np.abs(S) > 1e-15
    assert pat.shape == S.shape
    assert np.all(pat[nz])                       # every nonzero is in the pattern
    if name in ("rzz", "cx", "cz", "rz", "depol", "ad"):
        assert np.array_equal(pat, nz)           # and the pattern is exact here


def test_sparsity_aware_planning():
    # FP64 is DFMA-bound, so the automatic planner prices a block by its
    # nonzeros: the TFIM step stays in blocks of at most 2 qubits
    c = W.tfim_ring(6, 1)
    _, w64 = B.plan_fusion(6, c.ops, -1, "fp64")
    _, w32 = B.plan_fusion(6, c.ops, -1, "split")
    assert max(w64) <= 2 and w32 == [2] * 6
    assert B.op_pattern(("rzz", [0, 1], (0.2,))).sum() == 16        # diagonal
    assert B.op_pattern(("depol", [0, 1], (0.1,))).sum() == 28      # 12 coherences + 4 x 4 populations
    assert B.op_pattern(("depol", [0], (0.1,))).sum() == 6
    assert B.op_pattern(("cx", [0, 1], ())).sum() == 16             # a permutation


def test_register_size_limits_are_checked_before_any_gpu_work(lib):
    # n in [1, 16]: outside it tq_create / tq_batch_add fail with TQ_ERR_ARG
    # and touch no device (this runs on machines without a GPU)
    h = B.ctypes.c_void_p()
    for n in (0, 17, -1):
        assert lib.tq_create(n, 0, None, B.ctypes.byref(h)) == 1
        assert not h.value
    assert lib.tq_create(3, 7, None, B.ctypes.byref(h)) == 1          # unknown precision


def test_tensor_core_wait_hook_arguments(lib):
    # the failure-path hook of the split tensor-core pass only sets host-side
    # launch values: negative limits are rejected, 0 restores the default
    assert lib.tq_test_tc_wait_limit(-1, 0) == 1          # TQ_ERR_ARG
    assert lib.tq_test_tc_wait_limit(1000, 1) == 0
    assert lib.tq_test_tc_wait_limit(0, 0) == 0
