"""The residual entry point that allocates no device memory.

It exists for callers that cannot allocate device memory when they need the
residual (another runtime owns the device pool, a fixed footprint after
start-up, or work between launches that an allocation would synchronise).
Its scratch is a fixed array built into the library, so these checks compare
it with the residual ibdvm_step reports, on two calls in a row (the second
call finds the previous call's partial sums still in the shared array), and
check that a size beyond the array's capacity is refused with a clear message,
that a small call after a large one ignores the larger call's partial sums,
and that the largest size the array serves works in 2D and 3D.
This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2512_20252_gb300 import ibdvm
from paper_2512_20252_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("case", ["cylinder_48", "sphere"])
def test_residual_without_allocation_matches_step(torch, case):
    c = wl.cylinder_48() if case == "cylinder_48" else wl._case(3, 14, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6))
    solver = ibdvm.Solver(c)
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        W0, _, t = solver.moments()
        r_step = solver.step(1)
        W1, _, _ = solver.moments()
        d0 = torch.tensor(W0, device="cuda")
        d1 = torch.tensor(W1, device="cuda")
        dt = torch.tensor(t, device="cuda")
        ibdvm.residual_noalloc(d0.data_ptr(), d1.data_ptr(), dt.data_ptr(), W0.shape[0], solver.dim,
                               out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(r_step, rel=1e-11, abs=0.0)
        assert r_step > 0.0
    solver.close()


def _host_residual(W0, W1, types):
    """max_i sqrt(sum_j dW_ij^2) / sum_j |W_ij| over the fluid cells, components
    with sum |W| = 0 skipped (the convergence criterion of Sec. 4)."""
    fl = types == 0
    d, w = (W1 - W0)[fl], np.abs(W1[fl])
    num, den = np.sqrt(np.sum(d * d, axis=0)), np.sum(w, axis=0)
    return float(max(n / m for n, m in zip(num, den) if m != 0.0))


def test_small_call_after_a_large_one_and_the_capacity_edge(torch):
    """A call over few blocks after a call over many must ignore the partial
    sums the larger call left in the shared array; and the largest size the
    array serves (2,097,152 cells) works in 2D and 3D.  Synthetic fields, each
    result against the host reduction."""
    rng = np.random.default_rng(11)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for dim, n in ((2, 2_097_152), (3, 2_097_152), (3, 1_000), (2, 300)):
        nw = dim + 2
        W0 = 1.0 + rng.random((n, nw))
        W1 = W0 + 1e-3 * rng.standard_normal((n, nw))
        W1[:, 1] = W0[:, 1]  # one component without change
        types = (rng.random(n) < 0.97).astype(np.uint8) ^ 1  # about 3 % not fluid
        d0, d1 = torch.tensor(W0, device="cuda"), torch.tensor(W1, device="cuda")
        dt = torch.tensor(types, device="cuda")
        ibdvm.residual_noalloc(d0.data_ptr(), d1.data_ptr(), dt.data_ptr(), n, dim, out.data_ptr(),
                               stream.cuda_stream)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(_host_residual(W0, W1, types), rel=1e-12), (dim, n)


def test_residual_without_allocation_rejects_oversize(torch):
    w = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ibdvm.IbdvmError) as e:
        ibdvm.residual_noalloc(w.data_ptr(), w.data_ptr(), None, 2_097_153, 2, out.data_ptr())
    assert e.value.status == 1
    assert "2097152" in str(e.value)
