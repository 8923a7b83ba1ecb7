"""The tree-refined 2D grid (reading C28) and a body on it (C29) through the
C-ABI against the oracle's tree: the neighbour tables, the FP64 path within
1e-11 on f and W after several steps from a perturbed state, the mixed path
within 1e-5, the surface force, one-level trees against the uniform grid's
GPU path, and the refusals."""
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


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _perturbed(o, seed, amp=0.2):
    rng = np.random.default_rng(seed)
    return o.get_f() * (1.0 + amp * rng.uniform(-1.0, 1.0, size=o.shape()))


@pytest.mark.parametrize("metric,levels", [("point", 2), ("point", 3), ("x", 2)])
def test_tree_fp64_against_the_oracle(metric, levels):
    case = wl.tree_case(16, levels, nv=10, Ma=0.5, metric=metric,
                        radii=[0.9, 0.5, 0.3][:levels] if metric == "x" else None)
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    assert g.ncell == o.nleaf and g.dt == pytest.approx(o.dt, rel=1e-14)
    np.testing.assert_array_equal(g.tree_neighbours(), o.neighbours())
    f0 = _perturbed(o, 7)
    o.set_f(f0)
    g.set_f(f0)
    ro = o.step(6)
    rg = g.step(6)
    assert rel_err(g.get_f(), o.get_f()) < 1e-11
    Wg, qg, t = g.moments()
    Wo, qo = o.moments()
    assert np.all(t == ibdvm.FLUID)
    for i in range(4):
        if np.abs(Wo[:, i]).max() > 1e-9:
            assert rel_err(Wg[:, i], Wo[:, i]) < 1e-11, i
    assert float(np.abs(qg - qo).max() / max(np.abs(qo).max(), 1e-3)) < 1e-8
    assert rg == pytest.approx(ro, rel=1e-9)
    g.close()


@pytest.mark.parametrize("metric,levels,nv", [("point", 2, 12), ("point", 3, 16), ("y", 2, 15)])
def test_tree_mixed_against_the_oracle(metric, levels, nv):
    """FP32 storage: f within 1e-5 of the oracle's FP64 after eight steps from
    a perturbed state, W within 1e-5; leaves of one level on every side and
    leaves at coarse-fine interfaces and domain edges, velocity counts whose
    quadrants end inside a warp."""
    case = wl.tree_case(16, levels, nv=nv, Ma=0.5, precision="mixed", metric=metric,
                        radii=[0.9, 0.5, 0.3][:levels] if metric == "y" else None)
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    f0 = _perturbed(o, 11)
    o.set_f(f0)
    g.set_f(f0)
    o.step(8)
    g.step(8)
    assert rel_err(g.get_f(), o.get_f()) < 1e-5
    Wg, _, _ = g.moments()
    Wo, _ = o.moments()
    for i in range(4):
        if np.abs(Wo[:, i]).max() > 1e-9:
            assert rel_err(Wg[:, i], Wo[:, i]) < 1e-5, i
    g.close()


def test_one_level_tree_matches_the_uniform_gpu_path():
    n = 24
    case = wl._case(2, n, 2.0, 10, 4.5, 0.1, 0.4, {"kind": "none"})
    u = ibdvm.Solver(case)
    tree = {"maxlevel": 1, "level": [1] * (n * n), "ix": [i for _ in range(n) for i in range(n)],
            "iy": [j for j in range(n) for _ in range(n)]}
    t = ibdvm.Solver(dict(case, n=[n // 2, n // 2], tree=tree))
    rng = np.random.default_rng(2)
    f0 = u.get_f() * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=u.get_f().shape))
    u.set_f(f0)
    t.set_f(f0)
    u.step(5)
    t.step(5)
    assert rel_err(t.get_f(), u.get_f()) < 1e-12
    u.close()
    t.close()


def test_tree_refusals():
    case = wl.tree_case(8, 2, nv=6)
    g = ibdvm.Solver(case)
    with pytest.raises(ibdvm.IbdvmError):
        g.set_domain(wl.box_walls(2, 1.0))
    F, Q, CD, CL = g.forces()
    assert np.all(F == 0.0) and Q == 0.0
    g.close()
    bad = dict(case["tree"])
    bad["level"] = list(bad["level"])[1:]
    bad["ix"] = list(bad["ix"])[1:]
    bad["iy"] = list(bad["iy"])[1:]
    with pytest.raises(ibdvm.IbdvmError, match="hole"):
        ibdvm.Solver(dict(case, tree=bad))
    # a body whose ghost band reaches a coarser leaf (C29)
    with pytest.raises(ibdvm.IbdvmError, match="finest level"):
        ibdvm.Solver(dict(case, body=wl.circle(0.55)))
    with pytest.raises(ValueError, match="finest level"):
        oracle.OracleTree(dict(case, body=wl.circle(0.55)))


def _body_tree(precision, nv=10):
    return wl.tree_case(16, 2, nv=nv, Ma=0.5, radii=[1.4, 1.0], body=wl.circle(0.3), precision=precision)


def test_tree_with_a_body_fp64_against_the_oracle():
    """C29: a cylinder in the finest level of a three-level tree; FP64 within
    1e-11 of the oracle on f, W, the surface force and the residual after six
    steps from a perturbed state."""
    case = _body_tree("fp64")
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    assert g.info.nfluid == o.nfluid
    f0 = _perturbed(o, 5, amp=0.1)
    o.set_f(f0)
    g.set_f(f0)
    ro = o.step(6)
    rg = g.step(6)
    assert rel_err(g.get_f(), o.get_f()) < 1e-11
    Wg, _, t = g.moments()
    Wo, _ = o.moments()
    np.testing.assert_array_equal(t, o.cell_types())
    fl = t == ibdvm.FLUID
    for i in range(4):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-11, i
    Fg, Qg, CDg, _ = g.forces()
    Fo, Qo, CDo, _ = o.forces()
    assert np.abs(Fg - Fo).max() < 1e-10 * np.abs(Fo).max()
    assert CDg == pytest.approx(CDo, rel=1e-10)
    assert Qg == pytest.approx(Qo, rel=1e-8, abs=1e-12)
    assert rg == pytest.approx(ro, rel=1e-9)
    g.close()


def test_tree_with_a_body_mixed_against_the_oracle():
    case = _body_tree("mixed", nv=12)
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    f0 = _perturbed(o, 9, amp=0.1)
    o.set_f(f0)
    g.set_f(f0)
    o.step(8)
    g.step(8)
    assert rel_err(g.get_f(), o.get_f()) < 1e-5
    Wg, _, t = g.moments()
    Wo, _ = o.moments()
    fl = t == ibdvm.FLUID
    for i in range(4):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    _, _, CDg, _ = g.forces()
    _, _, CDo, _ = o.forces()
    assert CDg == pytest.approx(CDo, rel=1e-4)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_level_tree_with_a_body_matches_the_uniform_gpu_path(precision):
    n = 32
    case = wl._case(2, n, 2.0, 10, 4.5, 0.1, 0.4, wl.circle(0.5), precision=precision)
    u = ibdvm.Solver(case)
    tree = {"maxlevel": 1, "level": [1] * (n * n), "ix": [i for _ in range(n) for i in range(n)],
            "iy": [j for j in range(n) for _ in range(n)]}
    t = ibdvm.Solver(dict(case, n=[n // 2, n // 2], tree=tree))
    rng = np.random.default_rng(4)
    f0 = u.get_f() * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=u.get_f().shape))
    u.set_f(f0)
    t.set_f(f0)
    u.step(5)
    t.step(5)
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert rel_err(t.get_f(), u.get_f()) < tol
    _, _, CDu, _ = u.forces()
    _, _, CDt, _ = t.forces()
    assert CDt == pytest.approx(CDu, rel=1e-10 if precision == "fp64" else 1e-5)
    u.close()
    t.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tree_wall_quantities_against_the_oracle(precision):
    """Wall-point quantities of a body on a tree (C29) through the C-ABI
    against the oracle's finest grid under the tree, after a few steps."""
    case = _body_tree(precision)
    g = ibdvm.Solver(case)
    o = oracle.OracleTree(case)
    g.step(4)
    o.step(4)
    wg = g.wall()
    wo = o.finest_case().wall_quantities()
    assert wg.shape == wo.shape and wo.shape[0] > 8
    tol = 1e-10 if precision == "fp64" else 1e-4
    for i, c in enumerate(oracle.OracleCase.WALL_COLUMNS):
        err = np.abs(wg[:, i] - wo[:, i]).max() / max(np.abs(wo[:, i]).max(), 1e-3)
        assert err < tol, (c, err)
    g.close()


@pytest.mark.parametrize("workload,steps", [("tree_2d", 5), ("cylinder_hypersonic_tree", 5)])
def test_tree_full_size_mixed_against_fp64(workload, steps):
    """The tree workloads at their full size and launch shape: the mixed path
    (gather-first leaves, FP32 ghost values) against the FP64 path (which
    matches the oracle to 1e-11 on the smaller trees) after a few steps from
    the bench's start: W within 1e-5 of its largest magnitude per component
    (at least 1% of the largest density: a momentum component near zero by
    symmetry carries FP32 rounding of order 1e-8), C_D within 1e-4."""
    out = {}
    for prec in ("fp64", "mixed"):
        case = getattr(wl, workload)(precision=prec)
        g = ibdvm.Solver(case)
        if case["body"]["kind"] == "none":
            xc = wl.tree_centres(case)
            f = g.get_f()
            f *= (1.0 + 0.2 * np.exp(-(xc[:, 0] ** 2 + xc[:, 1] ** 2) / 2.0))[:, None, None]
            g.set_f(f)
            del f
        g.step(steps)
        W, q, t = g.moments()
        _, _, CD, _ = g.forces()
        out[prec] = (W, t, CD)
        g.close()
    (Wd, t, CDd), (Wm, _, CDm) = out["fp64"], out["mixed"]
    fl = t == ibdvm.FLUID
    for i in range(Wd.shape[1]):
        scale = max(np.abs(Wd[fl, i]).max(), 1e-2 * np.abs(Wd[fl, 0]).max())
        assert np.abs(Wm[fl, i] - Wd[fl, i]).max() < 1e-5 * scale, i
    assert abs(CDm - CDd) <= 1e-4 * abs(CDd)


# ---------------------------------------------------------------------------
# octrees (3D)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("body", [False, True])
def test_octree_fp64_against_the_oracle(body):
    """An octree with four finer leaves across some faces, with and without a
    sphere in its finest level (C29): FP64 within 1e-11 of the oracle on f,
    W, the surface force and the residual after four steps from a perturbed
    state; the neighbour tables equal."""
    case = wl.tree_case_3d(8, 2, nv=6, Ma=0.5, radii=[1.6, 1.2] if body else None,
                           body=wl.sphere(0.4) if body else None)
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    assert g.ncell == o.nleaf and g.info.nfluid == o.nfluid
    np.testing.assert_array_equal(g.tree_neighbours(), o.neighbours())
    f0 = _perturbed(o, 13, amp=0.1)
    o.set_f(f0)
    g.set_f(f0)
    ro = o.step(4)
    rg = g.step(4)
    assert rel_err(g.get_f(), o.get_f()) < 1e-11
    Wg, _, t = g.moments()
    Wo, _ = o.moments()
    np.testing.assert_array_equal(t, o.cell_types())
    fl = t == ibdvm.FLUID
    for i in range(5):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-11, i
    assert rg == pytest.approx(ro, rel=1e-9)
    if body:
        Fg, Qg, CDg, _ = g.forces()
        Fo, Qo, CDo, _ = o.forces()
        assert np.abs(Fg - Fo).max() < 1e-10 * np.abs(Fo).max()
        assert CDg == pytest.approx(CDo, rel=1e-10)
    g.close()


def test_octree_mixed_against_the_oracle():
    case = wl.tree_case_3d(8, 2, nv=8, Ma=0.5, radii=[1.6, 1.2], body=wl.sphere(0.4), precision="mixed")
    o = oracle.OracleTree(case)
    g = ibdvm.Solver(case)
    f0 = _perturbed(o, 17, amp=0.1)
    o.set_f(f0)
    g.set_f(f0)
    o.step(6)
    g.step(6)
    assert rel_err(g.get_f(), o.get_f()) < 1e-5
    Wg, _, t = g.moments()
    Wo, _ = o.moments()
    fl = t == ibdvm.FLUID
    for i in range(5):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    _, _, CDg, _ = g.forces()
    _, _, CDo, _ = o.forces()
    assert CDg == pytest.approx(CDo, rel=1e-4)
    g.close()


def test_one_level_octree_matches_the_uniform_gpu_path():
    n = 12
    case = wl._case(3, n, 2.0, 6, 4.5, 0.1, 0.4, wl.sphere(0.7))
    u = ibdvm.Solver(case)
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    tree = {"maxlevel": 1, "level": [1] * n ** 3, "ix": ix.T.ravel().tolist(), "iy": iy.T.ravel().tolist(),
            "iz": iz.T.ravel().tolist()}
    t = ibdvm.Solver(dict(case, n=[n // 2] * 3, tree=tree))
    rng = np.random.default_rng(8)
    f0 = u.get_f() * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=u.get_f().shape))
    u.set_f(f0)
    t.set_f(f0)
    u.step(4)
    t.step(4)
    assert rel_err(t.get_f(), u.get_f()) < 1e-12
    _, _, CDu, _ = u.forces()
    _, _, CDt, _ = t.forces()
    assert CDt == pytest.approx(CDu, rel=1e-10)
    u.close()
    t.close()
