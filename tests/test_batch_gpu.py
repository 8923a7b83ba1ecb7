"""The batched form (grouped launches over many 2D FP32 cases) through the C-ABI.

A member of a batch takes exactly the steps that ibdvm_step takes on its own
(the same kernel bodies), so with the same velocity chunking its state,
residual and step forces are bit-identical to a twin stepped alone; with a
different chunking (64- instead of 128-velocity chunks) only the grouping of
the FP32 moment partial sums changes.  Membership may change between steps
(continuous batching) without changing any member's result.
"""
import numpy as np
import pytest

import oracle
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


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def mixed_cases():
    """Uneven members: 64, 144 and 256 velocities (quadrants padded to
    64-velocity chunks), three body kinds, grids that are not multiples of the
    8-column strip."""
    a = wl.small_2d("circle", n=40, nv=16, Ma=0.4, precision="mixed")            # 256 velocities
    b = wl.small_2d("ellipse", n=24, nv=8, Ma=0.6, precision="mixed")           # 64 velocities
    b["n"] = [27, 21]
    b["lo"], b["hi"] = [-2.2, -1.7], [2.0, 1.9]
    c = wl.small_2d("naca", n=36, nv=12, Ma=0.5, precision="mixed", Kn=0.05)     # 144 velocities
    d = wl.small_2d("circle", n=19, nv=16, Ma=0.2, precision="mixed", Kn=0.5)
    d["n"] = [19, 45]
    d["lo"], d["hi"] = [-1.5, -3.5], [1.5, 3.5]
    return [a, b, c, d]


def twins(torch, cases, stream):
    solo = [ibdvm.Solver(c, stream=stream.cuda_stream) for c in cases]
    mem = [ibdvm.Solver(c, stream=stream.cuda_stream) for c in cases]
    return solo, mem


def assert_same(s, m):
    np.testing.assert_array_equal(s.get_f(), m.get_f())
    Ws, qs, _ = s.moments()
    Wm, qm, _ = m.moments()
    np.testing.assert_array_equal(Ws, Wm)
    np.testing.assert_array_equal(qs, qm)


def test_batch_bit_identical_to_members_stepped_alone(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    solo, mem = twins(torch, cases, stream)
    b = ibdvm.Batch(stream=stream.cuda_stream)
    for m in mem:
        b.add(m)
    assert len(b) == 4
    for nsteps in (5, 2, 1):  # graph pairs and single steps, both parities
        rs = [s.step(nsteps) for s in solo]
        rb, st = b.step(nsteps)
        assert list(st) == [0] * 4
        assert list(rb) == rs
        for s, m in zip(solo, mem):
            assert_same(s, m)
    F, Q, CD, CL = b.forces()
    for i, s in enumerate(solo):
        Fs, Qs, CDs, CLs = s.step_forces()
        assert CD[i] == CDs and CL[i] == CLs and Q[i] == Qs
        np.testing.assert_array_equal(F[i], Fs)
    t = b.tiling()
    assert t["nitems"] > 0 and t["grid"] > 0 and t["graphs"] == 1
    kt = b.kernel_times()
    assert kt["sweep"][1] == 8  # one persistent sweep launch per step
    b.close()


def test_continuous_batching_members_join_and_leave(torch):
    """A result is the same alone and in the mix: members join and leave
    between steps, and each still matches its twin stepped alone."""
    stream = torch.cuda.Stream()
    cases = mixed_cases()[:3]
    solo, mem = twins(torch, cases, stream)
    A, B, C = mem
    b = ibdvm.Batch(stream=stream.cuda_stream)
    b.add(A)
    b.step(3)
    b.add(B)
    b.step(4)
    b.remove(A)
    b.add(C)
    b.step(3)
    b.step(2)
    solo[0].step(7)
    solo[1].step(9)
    solo[2].step(5)
    for s, m in zip(solo, mem):
        assert_same(s, m)
    assert [m is x for m, x in zip(b.members, (B, C))] == [True, True]
    # a member that leaves keeps stepping on its own
    b.remove(B)
    B.step(2)
    solo[1].step(2)
    assert_same(solo[1], B)
    b.close()
    # destroying a member takes it out of its batch
    b2 = ibdvm.Batch(stream=stream.cuda_stream)
    b2.add(C)
    C.close()
    assert b2.lib.ibdvm_batch_size(b2.h) == 0
    b2.members = []
    b2.close()


@pytest.mark.parametrize("rows,kpt", [(16, 4), (8, 0), (16, 2), (0, 2)])
def test_tilings(torch, rows, kpt):
    stream = torch.cuda.Stream()
    cases = mixed_cases()
    solo, mem = twins(torch, cases, stream)
    b = ibdvm.Batch(stream=stream.cuda_stream)
    for m in mem:
        b.add(m)
    b.set_tiling(rows, kpt)
    b.step(4)
    for s in solo:
        s.step(4)
    # the row tiling does not change any cell's arithmetic (kpt has no effect)
    for s, m in zip(solo, mem):
        assert_same(s, m)
    assert b.tiling()["kpt"] in (2, 4, 6)
    b.close()


def test_autotuner_keeps_a_candidate_and_steps_stay_correct(torch):
    stream = torch.cuda.Stream()
    cases = mixed_cases()[:2]
    solo, mem = twins(torch, cases, stream)
    b = ibdvm.Batch(stream=stream.cuda_stream)
    for m in mem:
        b.add(m)
    best = b.tune(2)
    assert best > 0
    t = b.tiling()
    assert t["rows"] in (16, 32, 64, 128, 0) and t["kpt"] in (2, 4, 6)
    nsteps = 5 * (2 + 2)  # five trials of a warm-up pair and two timed steps
    for s in solo:
        s.step(nsteps)
    for s, m in zip(solo, mem):
        Ws, _, typ = s.moments()
        Wm, _, _ = m.moments()
        fl = typ == 0
        for i in range(4):
            if np.abs(Ws[fl, i]).max() > 1e-9:
                assert rel_err(Wm[fl, i], Ws[fl, i]) < 1e-5
    b.close()


def test_batch_against_the_oracle(torch):
    """Two members against the FP64 CPU oracle (mixed-precision tolerance)."""
    stream = torch.cuda.Stream()
    cases = mixed_cases()[1:3]
    mem = [ibdvm.Solver(c, stream=stream.cuda_stream) for c in cases]
    orc = [oracle.OracleCase(c) for c in cases]
    b = ibdvm.Batch(stream=stream.cuda_stream)
    for m in mem:
        b.add(m)
    rb, _ = b.step(6)
    F, Q, CD, CL = b.forces()
    for i, (m, o) in enumerate(zip(mem, orc)):
        ro = o.step(6)
        t = o.cell_types()
        fl = t == oracle.FLUID
        Wm, _, _ = m.moments()
        Wo, _ = o.moments()
        for k in range(4):
            if np.abs(Wo[fl, k]).max() > 1e-9:
                assert rel_err(Wm[fl, k], Wo[fl, k]) < 1e-5, (i, k)
        assert rb[i] == pytest.approx(ro, rel=1e-3)
    b.close()


def test_batch_rejects_bad_members(torch):
    stream = torch.cuda.Stream()
    other = torch.cuda.Stream()
    b = ibdvm.Batch(stream=stream.cuda_stream)
    fp64 = ibdvm.Solver(wl.small_2d("circle", n=12, nv=8), stream=stream.cuda_stream)
    with pytest.raises(ibdvm.IbdvmError) as e:
        b.add(fp64)
    assert e.value.status == 1
    ok = ibdvm.Solver(wl.small_2d("circle", n=12, nv=8, precision="mixed"), stream=other.cuda_stream)
    with pytest.raises(ibdvm.IbdvmError):
        b.add(ok)  # bound to another stream
    ok.set_stream(stream.cuda_stream)
    b.add(ok)
    s3 = ibdvm.Solver(wl._case(3, 8, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6), precision="mixed"),
                      stream=stream.cuda_stream)
    with pytest.raises(ibdvm.IbdvmError):
        b.add(s3)  # the members of a batch have one dimension
    b2 = ibdvm.Batch(stream=stream.cuda_stream)
    with pytest.raises(ibdvm.IbdvmError) as e:
        b2.add(ok)
    assert e.value.status == 8
    with pytest.raises(ibdvm.IbdvmError):
        ok.set_stream(other.cuda_stream)  # a member stays on the batch's stream
    with pytest.raises(ibdvm.IbdvmError):
        b.set_tiling(-1, 0)
    with pytest.raises(ibdvm.IbdvmError):
        b.tune(3)
    r, st = b.step(0)
    assert list(st) == [0]
    b2.close()
    b.close()


def test_stretched_velocity_grid_member(torch):
    """A member on a stretched velocity grid (partly specular wall: the
    specular part bisects the node grid) steps in the batch exactly as alone."""
    stream = torch.cuda.Stream()
    a = wl.stretched(wl._case(2, 32, 2.0, 16, 4.5, 0.1, 0.4, wl.circle(0.7, accom=0.7), precision="mixed"), 0.3)
    cases = [a, mixed_cases()[1]]
    solo, mem = twins(torch, cases, stream)
    b = ibdvm.Batch(stream=stream.cuda_stream)
    for m in mem:
        b.add(m)
    rb, st = b.step(4)
    rs = [s.step(4) for s in solo]
    assert list(st) == [0, 0] and list(rb) == rs
    for s, m in zip(solo, mem):
        assert_same(s, m)
    b.close()
