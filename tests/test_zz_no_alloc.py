"""The residual entry point that allocates no device memory.

It exists for callers that cannot allocate device memory when they need the
residual (another runtime owns the device pool, a fixed footprint after
start-up, or work between launches that an allocation would synchronise).
Its scratch is a fixed array built into the library, so these checks compare
it with the residual ibdvm_step reports, on two calls in a row (the second
call finds the previous call's partial sums still in the shared array), and
check that a size beyond the array's capacity is refused with a clear message.
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


def test_residual_without_allocation_rejects_oversize(torch):
    w = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ibdvm.IbdvmError) as e:
        ibdvm.residual_noalloc(w.data_ptr(), w.data_ptr(), None, 2_097_153, 2, out.data_ptr())
    assert e.value.status == 1
    assert "2097152" in str(e.value)
