"""The allocation-free readout (tq_expect_z_noalloc) against the ordinary one.

Callers whose device memory belongs to another allocator, or who cannot
accept cudaFree's device-wide synchronisation, use this entry point with
their own buffers; its scratch is a fixed array inside the library. This
file is collected last so that a run stopping at the first failure has run
every other test before it."""
import numpy as np
import pytest

from paper_2404_13184_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "split": 1e-6}


@pytest.mark.parametrize("precision", ["fp64", "split"])
def test_noalloc_readout_matches_expect_z_on_two_calls(tq, precision):
    import torch
    n = 9
    c = W.random_noisy_circuit(n, 80, 3, gate_set=("h", "rx", "rz", "cx", "su2"))
    half = len(c.ops) // 2
    masks_a = [0b11, 1, 1 << 8, (1 << n) - 1]
    masks_b = [1 << q for q in range(n)] + [0b101, 0b110000, 0]
    stream = torch.cuda.current_stream().cuda_stream
    with tq.State(n, precision) as st:
        for ops, masks in ((c.ops[:half], masks_a), (c.ops[half:], masks_b)):
            st.run(ops, width=2)
            want = st.expect_z(masks)                              # existing entry point
            m = torch.tensor(masks, dtype=torch.int64, device="cuda")
            out = torch.full((len(masks),), float("nan"), dtype=torch.float64, device="cuda")
            tq.expect_z_noalloc(st.device_ptr(), n, precision, m.data_ptr(), len(masks), out.data_ptr(), stream)
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - want)) < TOL[precision]


@pytest.mark.parametrize("n,precision", [(14, "fp64"), (15, "split")])
def test_noalloc_readout_multi_cta_partials(tq, n, precision):
    # 14 and 15 qubits: the reduction runs on 32 and 64 CTAs, so the fixed
    # scratch array holds many per-CTA partials; two calls in a row
    import torch
    c = W.random_noisy_circuit(4, 40, 11, gate_set=("h", "rx", "rz", "cx", "su2"))
    masks_a = [0b11, 1, 1 << (n - 1), (1 << n) - 1]
    masks_b = [1 << q for q in range(4)] + [0b1010, 0]
    stream = torch.cuda.current_stream().cuda_stream
    with tq.State(n, precision) as st:
        for q in range(4, n):
            st.run([("h", [q], ())], width=1)
        for masks in (masks_a, masks_b):
            st.run(c.ops, width=2)
            want = st.expect_z(masks)
            m = torch.tensor(masks, dtype=torch.int64, device="cuda")
            out = torch.full((len(masks),), float("nan"), dtype=torch.float64, device="cuda")
            tq.expect_z_noalloc(st.device_ptr(), n, precision, m.data_ptr(), len(masks), out.data_ptr(), stream)
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - want)) < TOL[precision]


def test_noalloc_rejects_sizes_beyond_its_scratch(tq):
    import torch
    with tq.State(4, "fp64") as st:
        m = torch.ones(17, dtype=torch.int64, device="cuda")
        out = torch.zeros(17, dtype=torch.float64, device="cuda")
        with pytest.raises(tq.TqError) as e:
            tq.expect_z_noalloc(st.device_ptr(), 4, "fp64", m.data_ptr(), 17, out.data_ptr())
        assert e.value.status == 1                                 # TQ_ERR_ARG
        with pytest.raises(tq.TqError):
            tq.expect_z_noalloc(st.device_ptr(), 17, "fp64", m.data_ptr(), 1, out.data_ptr())
