"""Failure detection without a GPU fault: the bounded device waits of the TMA
sweeps give up and report IBDVM_E_TIMEOUT instead of hanging, and the device
stays usable afterwards (a solve right after the timeout is still exact)."""
import numpy as np
import pytest

import oracle
from paper_2512_20252_gb300 import ibdvm
from paper_2512_20252_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def test_bounded_wait_completes_when_the_bytes_arrive():
    st, sec = ibdvm.selftest_bounded_wait(True, 1000)
    assert st == ibdvm.OK


def test_bounded_wait_times_out_when_nothing_arrives():
    st, sec = ibdvm.selftest_bounded_wait(False, 2000)  # a barrier nothing completes
    assert st == 7  # IBDVM_E_TIMEOUT
    assert sec < 30.0
    # the context is intact: a solve right after matches the oracle
    case = wl.small_2d("circle", n=12, nv=6, precision="fp64")
    g = ibdvm.Solver(case)
    o = oracle.OracleCase(case)
    g.step(3)
    o.step(3)
    fl = o.cell_types() == oracle.FLUID
    err = np.abs(g.get_f()[fl] - o.get_f()[fl]).max() / np.abs(o.get_f()[fl]).max()
    assert err < 1e-11


def test_bounded_wait_rejects_bad_limits():
    assert ibdvm.selftest_bounded_wait(False, -1)[0] == 1
    assert ibdvm.selftest_bounded_wait(False, (1 << 18) + 1)[0] == 1
