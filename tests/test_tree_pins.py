"""Pins of the oracle's tree-refined grids (reading C28) against what the
mathematics fixes: on a tree of one level the step is the uniform grid's;
a uniform state stays uniform; data linear along an axis are transported
exactly on a tree refined in stripes across that axis; the fluxes through
coarse-fine interfaces conserve every velocity's total; mirror symmetry; and
trees that do not tile the domain or break the 2:1 rule are refused."""
import numpy as np
import pytest

import oracle
from paper_2512_20252_gb300 import workloads as wl


def _uniform_tree(n, level):
    """All leaves at one level over a root of n / 2^level cells per axis."""
    root = n >> level
    ix, iy, lev = [], [], []
    for j in range(n):
        for i in range(n):
            ix.append(i)
            iy.append(j)
            lev.append(level)
    return root, {"maxlevel": level, "level": lev, "ix": ix, "iy": iy}


@pytest.mark.parametrize("level", [0, 1])
def test_one_level_tree_is_the_uniform_step(level):
    n = 16
    case = wl._case(2, n, 2.0, 8, 4.5, 0.1, 0.4, {"kind": "none"})
    u = oracle.OracleCase(case)
    root, tree = _uniform_tree(n, level)
    tcase = dict(case, n=[root, root], tree=tree)
    t = oracle.OracleTree(tcase)
    assert t.nleaf == u.ncell and t.dt == pytest.approx(u.dt, rel=1e-15)
    rng = np.random.default_rng(3)
    f0 = u.get_f() * (1.0 + 0.3 * rng.uniform(-1.0, 1.0, size=u.shape()))
    u.set_f(f0)
    t.set_f(f0)
    ru = u.step(4)
    rt = t.step(4)
    fu, ft = u.get_f(), t.get_f()
    assert np.abs(ft - fu).max() < 1e-13 * np.abs(fu).max()
    assert rt == pytest.approx(ru, rel=1e-10)


def test_uniform_state_stays_uniform():
    """A uniform state across the coarse-fine interfaces stays uniform: after
    two steps every leaf beyond the reach of the domain edges (two cells of
    any level per step: four root cells) holds the same values."""
    case = wl.tree_case(16, 2, nv=8)
    t = oracle.OracleTree(case)
    t.step(2)
    f = t.get_f()
    xc = t.centres()
    inner = np.where(np.abs(xc).max(axis=1) < 2.0 - 4 * 0.25)[0]
    lev = np.asarray(case["tree"]["level"])
    assert set(lev[inner]) == {0, 1, 2}
    fi = f[inner]
    assert np.abs(fi - fi[:1]).max() < 1e-14 * np.abs(fi).max()


@pytest.mark.parametrize("axis", [0, 1])
def test_linear_data_are_transported_exactly_on_stripes(axis):
    """f_k = finf_k (1 + eps (x_a - x0)) on a tree refined in stripes across
    axis a (every cell's neighbours along the other axis share its level):
    the limited slopes equal the gradient, the face values the linear data,
    so one step moves every cell by -dt xi_a finf_k eps (relaxation made
    negligible by a huge Knudsen number), away from the domain edges."""
    L = 2.0
    case = wl.tree_case(16, 2, L=L, nv=8, Kn=1e12, metric="xy"[axis], radii=[0.8, 0.4])
    t = oracle.OracleTree(case)
    lev = np.asarray(case["tree"]["level"])
    assert set(lev) == {0, 1, 2}
    xc = t.centres()
    f0 = t.get_f()
    finf = f0[0].copy()
    eps = 0.05
    f0 = finf[None] * (1.0 + eps * (xc[:, axis] - 0.1))[:, None, None]
    t.set_f(f0)
    t.step(1)
    f1 = t.get_f()
    xi = np.asarray(oracle.OracleCase(dict(case, tree=None)).velocities()[0])[:, axis]
    expect = f0 - t.dt * xi[None, :, None] * finf[None] * eps
    # two root cells from every domain edge: the freestream halo is not linear
    inner = np.abs(xc).max(axis=1) < L - 2 * (2 * L / 16)
    scale = np.abs(t.dt * xi[None, :, None] * finf[None] * eps).max()
    assert np.abs(f1[inner] - expect[inner]).max() < 1e-9 * scale


def test_coarse_fine_fluxes_conserve_every_velocity():
    """A perturbation inside a refined tree: the area-weighted total of every
    velocity's distribution changes only by the boundary fluxes, which cancel
    for a freestream boundary; relaxation made negligible."""
    case = wl.tree_case(16, 2, nv=8, Kn=1e12)
    t = oracle.OracleTree(case)
    xc, hs = t.centres(), t.sizes()
    area = hs[:, 0] * hs[:, 1]
    f0 = t.get_f()
    bump = 0.2 * np.exp(-((xc[:, 0] - 0.2) ** 2 + (xc[:, 1] + 0.1) ** 2) / 0.1)
    f0 = f0 * (1.0 + bump)[:, None, None]
    t.set_f(f0)
    t.step(1)
    f1 = t.get_f()
    d = np.einsum("c,ckm->km", area, f1 - f0)
    ref = np.einsum("c,ckm->km", area, np.abs(f0 - f0[:1]))
    assert np.abs(d).max() < 1e-10 * np.abs(ref).max()


def test_mirror_symmetry_on_a_refined_tree():
    """A state symmetric about y = 0 (a bump across the refined region, the
    freestream along x) stays symmetric: a side's two finer neighbours enter
    its slopes and fluxes alike."""
    case = wl.tree_case(16, 2, nv=8, Ma=0.5)
    t = oracle.OracleTree(case)
    xc = t.centres()
    f0 = t.get_f() * (1.0 + 0.2 * np.exp(-((xc[:, 0] - 0.2) ** 2 + xc[:, 1] ** 2) / 0.1))[:, None, None]
    t.set_f(f0)
    t.step(6)
    W, _ = t.moments()
    tr = case["tree"]
    key = {(l, i, j): c for c, (l, i, j) in enumerate(zip(tr["level"], tr["ix"], tr["iy"]))}
    mir = np.array([key[(l, i, (16 << l) - 1 - j)] for l, i, j in zip(tr["level"], tr["ix"], tr["iy"])])
    assert np.abs(W[mir, 0] - W[:, 0]).max() < 1e-13
    assert np.abs(W[mir, 2] + W[:, 2]).max() < 1e-13


def test_invalid_trees_are_refused():
    case = wl.tree_case(4, 2, nv=4)
    tr = case["tree"]
    # a hole: drop a leaf
    bad = {k: (v[1:] if isinstance(v, list) else v) for k, v in tr.items()}
    with pytest.raises(ValueError):
        oracle.OracleTree(dict(case, tree=bad))
    # two levels apart: a level-2 block next to a level-0 cell
    lev, ix, iy = [], [], []
    for j in range(4):
        for i in range(4):
            if (i, j) == (1, 1):
                for jj in range(4):
                    for ii in range(4):
                        lev.append(2)
                        ix.append(4 + ii)
                        iy.append(4 + jj)
            else:
                lev.append(0)
                ix.append(i)
                iy.append(j)
    with pytest.raises(ValueError):
        oracle.OracleTree(dict(case, tree={"maxlevel": 2, "level": lev, "ix": ix, "iy": iy}))
    # the balanced generator's trees are accepted and tile the domain
    t = oracle.OracleTree(case)
    hs = t.sizes()
    assert np.sum(hs[:, 0] * hs[:, 1]) == pytest.approx((case["hi"][0] - case["lo"][0]) ** 2)


def _bump(x):
    return 1.0 + 0.2 * np.exp(-((x[:, 0] - 0.1) ** 2 + (x[:, 1] + 0.05) ** 2) / 0.3)


def _uniform_centres(case):
    n = case["n"]
    h = [(case["hi"][a] - case["lo"][a]) / n[a] for a in range(2)]
    i, j = np.meshgrid(np.arange(n[0]), np.arange(n[1]), indexing="xy")
    return np.stack([case["lo"][0] + (i.ravel() + 0.5) * h[0], case["lo"][1] + (j.ravel() + 0.5) * h[1]], axis=1)


def test_one_level_tree_with_a_body_is_the_uniform_case():
    """C29 on a tree of one level: the ghost band, the fluid cells next to the
    ghosts, the solid cells, the residual and the surface force are the
    uniform grid's with the same body."""
    n = 32
    case = wl._case(2, n, 2.0, 8, 4.5, 0.1, 0.4, wl.circle(0.5))
    u = oracle.OracleCase(case)
    root, tree = _uniform_tree(n, 1)
    t = oracle.OracleTree(dict(case, n=[root, root], tree=tree))
    np.testing.assert_array_equal(t.cell_types(), u.cell_types())
    assert t.nfluid == u.nfluid
    f0 = u.get_f() * _bump(_uniform_centres(case))[:, None, None]
    u.set_f(f0)
    t.set_f(f0)
    ru = u.step(3)
    rt = t.step(3)
    fu, ft = u.get_f(), t.get_f()
    assert np.abs(ft - fu).max() < 1e-13 * np.abs(fu).max()
    assert rt == pytest.approx(ru, rel=1e-10)
    Fu, Qu, CDu, _ = u.forces()
    Ft, Qt, CDt, _ = t.forces()
    assert np.abs(Ft - Fu).max() < 1e-12 * np.abs(Fu).max()
    assert Qt == pytest.approx(Qu, rel=1e-10, abs=1e-14)
    assert CDt == pytest.approx(CDu, rel=1e-12)


def test_body_on_a_refined_tree_is_the_finest_grid_near_it():
    """A body in the finest level of a three-level tree: one step from the
    same smooth state gives, at every finest leaf whose neighbourhood of
    three finest cells holds no coarser leaf (the body's ghost band and its
    donors among them), the values of the uniform finest grid with the same
    body, and the same surface force."""
    case = wl.tree_case(16, 2, nv=8, radii=[1.4, 1.0], body=wl.circle(0.3))
    t = oracle.OracleTree(case)
    ucase = dict(case, n=[64, 64])
    ucase.pop("tree")
    u = oracle.OracleCase(ucase)
    tr = case["tree"]
    lev = np.asarray(tr["level"])
    # the level of every finest-grid cell, and the finest leaves' cells
    levmap = np.zeros((64, 64), dtype=int)
    for l, i, j in zip(tr["level"], tr["ix"], tr["iy"]):
        s = 1 << (2 - l)
        levmap[i * s:(i + 1) * s, j * s:(j + 1) * s] = l
    fine = np.where(lev == 2)[0]
    vcell = np.asarray(tr["ix"])[fine] + 64 * np.asarray(tr["iy"])[fine]
    ok = np.array([levmap[max(i - 3, 0):i + 4, max(j - 3, 0):j + 4].min() == 2
                   for i, j in zip(np.asarray(tr["ix"])[fine], np.asarray(tr["iy"])[fine])])
    np.testing.assert_array_equal(t.cell_types()[fine], u.cell_types()[vcell])
    assert ok.sum() > 300 and np.any(t.cell_types()[fine][ok] == 1)
    t.set_f(t.get_f() * _bump(t.centres())[:, None, None])
    u.set_f(u.get_f() * _bump(_uniform_centres(ucase))[:, None, None])
    t.step(1)
    u.step(1)
    ft, fu = t.get_f()[fine][ok], u.get_f()[vcell][ok]
    assert np.abs(ft - fu).max() < 1e-14 * np.abs(fu).max()
    Ft, Qt, CDt, _ = t.forces()
    Fu, Qu, CDu, _ = u.forces()
    assert np.abs(Ft - Fu).max() < 1e-13 * np.abs(Fu).max()
    assert CDt == pytest.approx(CDu, rel=1e-13)


def test_a_body_outside_the_finest_level_is_refused():
    with pytest.raises(ValueError, match="finest level"):
        oracle.OracleTree(wl.tree_case(16, 2, nv=6, body=wl.circle(0.55)))
    with pytest.raises(ValueError, match="finest level"):
        oracle.OracleTree(wl.tree_case(16, 2, nv=6, body=wl.circle(0.2, center=(1.0, 0.0))))
    oracle.OracleTree(wl.tree_case(16, 2, nv=6, body=wl.circle(0.3)))


# ---------------------------------------------------------------------------
# octrees (3D): the same pins, with four finer leaves across a face
# ---------------------------------------------------------------------------

def _uniform_tree_3d(n, level):
    root = n >> level
    ix, iy, iz = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return root, {"maxlevel": level, "level": [level] * n ** 3, "ix": ix.T.ravel().tolist(),
                  "iy": iy.T.ravel().tolist(), "iz": iz.T.ravel().tolist()}


@pytest.mark.parametrize("body", [False, True])
def test_one_level_octree_is_the_uniform_step(body):
    n = 12
    case = wl._case(3, n, 2.0, 6, 4.5, 0.1, 0.4, wl.sphere(0.7) if body else {"kind": "none"})
    u = oracle.OracleCase(case)
    root, tree = _uniform_tree_3d(n, 1)
    t = oracle.OracleTree(dict(case, n=[root] * 3, tree=tree))
    np.testing.assert_array_equal(t.cell_types(), u.cell_types())
    assert t.dt == pytest.approx(u.dt, rel=1e-15)
    rng = np.random.default_rng(6)
    f0 = u.get_f() * (1.0 + 0.2 * rng.uniform(-1.0, 1.0, size=u.shape()))
    u.set_f(f0)
    t.set_f(f0)
    ru = u.step(3)
    rt = t.step(3)
    fu, ft = u.get_f(), t.get_f()
    assert np.abs(ft - fu).max() < 1e-13 * np.abs(fu).max()
    assert rt == pytest.approx(ru, rel=1e-10)
    if body:
        Fu, _, CDu, _ = u.forces()
        Ft, _, CDt, _ = t.forces()
        assert np.abs(Ft - Fu).max() < 1e-12 * np.abs(Fu).max()


def test_octree_uniform_state_and_conservation():
    """On a three-level octree: a uniform state stays uniform away from the
    domain edges, and with relaxation made negligible the volume-weighted
    total of every velocity changes only by the (cancelling) freestream
    boundary fluxes, across faces with four finer neighbours."""
    case = wl.tree_case_3d(16, 2, nv=6)
    t = oracle.OracleTree(case)
    nb = t.neighbours()
    assert (nb[:, :, 3] >= 0).any()  # faces with four finer neighbours
    t.step(2)
    f = t.get_f()
    xc = t.centres()
    inner = np.where(np.abs(xc).max(axis=1) < 2.0 - 4 * 0.25)[0]
    lev = np.asarray(case["tree"]["level"])
    assert set(lev[inner]) == {0, 1, 2}
    assert np.abs(f[inner] - f[inner][:1]).max() < 1e-14 * np.abs(f[inner]).max()
    case = wl.tree_case_3d(8, 2, nv=6, Kn=1e12)
    t = oracle.OracleTree(case)
    xc, hs = t.centres(), t.sizes()
    vol = hs.prod(axis=1)
    f0 = t.get_f() * (1.0 + 0.2 * np.exp(-((xc - [0.2, -0.1, 0.05]) ** 2).sum(axis=1) / 0.1))[:, None, None]
    t.set_f(f0)
    t.step(1)
    d = np.einsum("c,ckm->km", vol, t.get_f() - f0)
    ref = np.einsum("c,ckm->km", vol, np.abs(f0 - f0[:1]))
    assert np.abs(d).max() < 1e-10 * np.abs(ref).max()


def test_invalid_octrees_are_refused():
    case = wl.tree_case_3d(4, 2, nv=4)
    tr = case["tree"]
    bad = {k: (v[1:] if isinstance(v, list) else v) for k, v in tr.items()}
    with pytest.raises(ValueError):
        oracle.OracleTree(dict(case, tree=bad))
    # a level-2 block next to level-0 cells
    lev, ix, iy, iz = [], [], [], []
    for k in range(4):
        for j in range(4):
            for i in range(4):
                if (i, j, k) == (1, 1, 1):
                    for kk in range(4):
                        for jj in range(4):
                            for ii in range(4):
                                lev.append(2)
                                ix.append(4 + ii)
                                iy.append(4 + jj)
                                iz.append(4 + kk)
                else:
                    lev.append(0)
                    ix.append(i)
                    iy.append(j)
                    iz.append(k)
    with pytest.raises(ValueError):
        oracle.OracleTree(dict(case, tree={"maxlevel": 2, "level": lev, "ix": ix, "iy": iy, "iz": iz}))
    t = oracle.OracleTree(case)
    assert np.sum(t.sizes().prod(axis=1)) == pytest.approx(4.0 ** 3)


def test_body_on_a_refined_octree_is_the_finest_grid_near_it():
    case = wl.tree_case_3d(8, 2, nv=6, radii=[1.6, 1.2], body=wl.sphere(0.4))
    t = oracle.OracleTree(case)
    ucase = dict(case, n=[32, 32, 32])
    ucase.pop("tree")
    u = oracle.OracleCase(ucase)
    tr = case["tree"]
    lev = np.asarray(tr["level"])
    levmap = np.zeros((32, 32, 32), dtype=int)
    for l, i, j, k in zip(tr["level"], tr["ix"], tr["iy"], tr["iz"]):
        s = 1 << (2 - l)
        levmap[i * s:(i + 1) * s, j * s:(j + 1) * s, k * s:(k + 1) * s] = l
    fine = np.where(lev == 2)[0]
    I, J, K = (np.asarray(tr[q])[fine] for q in ("ix", "iy", "iz"))
    vcell = I + 32 * (J + 32 * K)
    ok = np.array([levmap[max(i - 3, 0):i + 4, max(j - 3, 0):j + 4, max(k - 3, 0):k + 4].min() == 2
                   for i, j, k in zip(I, J, K)])
    np.testing.assert_array_equal(t.cell_types()[fine], u.cell_types()[vcell])
    assert ok.sum() > 100 and np.any(t.cell_types()[fine][ok] == 1)
    bump = lambda x: 1.0 + 0.2 * np.exp(-((x - [0.1, -0.05, 0.02]) ** 2).sum(axis=1) / 0.3)
    uc = np.stack(np.meshgrid(*[ucase["lo"][a] + (np.arange(32) + 0.5) * 4.0 / 32 for a in range(3)],
                              indexing="ij"), axis=-1).transpose(2, 1, 0, 3).reshape(-1, 3)
    t.set_f(t.get_f() * bump(t.centres())[:, None, None])
    u.set_f(u.get_f() * bump(uc)[:, None, None])
    t.step(1)
    u.step(1)
    ft, fu = t.get_f()[fine][ok], u.get_f()[vcell][ok]
    assert np.abs(ft - fu).max() < 1e-14 * np.abs(fu).max()
    Ft, _, CDt, _ = t.forces()
    Fu, _, CDu, _ = u.forces()
    assert np.abs(Ft - Fu).max() < 1e-13 * np.abs(Fu).max()
