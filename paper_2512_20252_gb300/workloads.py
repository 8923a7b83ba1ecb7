"""Workload presets and seeded synthetic case generators.

This module holds case descriptions only (grid sizes, velocity grids, gas and
body parameters, seeded draws of batched and served cases).  It contains none
of the method's arithmetic, so both the CUDA path and the CPU oracle can be
driven from the same dicts.

Case dict keys: dim, n, lo, hi (physical grid); nv, vlo, vhi, rule (velocity
grid, rule "trapezoid", "midpoint" or "nodes" with vnodes = the nodes of each
axis); Kn, Ma, Pr, gamma, omega_vhs, alpha_vhs, rho_inf, T_inf, dir, cfl, dt
(gas, non-dimensional as in Sec. 4 of the paper); body = {kind, center,
radii, angle, verts, accom, Tw, Uw, Lref}; domain_walls (six faces: None or
{Tw, Uw}); cutcell, upwind, ghost_nonneg (method switches); precision
("fp64" or "mixed"); steps.

The workloads stand in for the paper's cases (Sec. 4: the cavity with a
cylinder, the hypersonic cylinder, the supersonic airfoil and sphere, on
uniform grids) and for the sizes of the benchmark configurations; the paper
measures on no public dataset.
"""
from __future__ import annotations

import math

import numpy as np

ARGON = dict(Pr=2.0 / 3.0, gamma=5.0 / 3.0, omega_vhs=0.81, alpha_vhs=1.0, rho_inf=1.0, T_inf=1.0)


def _case(dim, n, L, nv, V, Kn, Ma, body, precision="fp64", steps=200, rule="trapezoid", **kw):
    lo = [-L] * dim if np.isscalar(L) else list(L[0])
    hi = [L] * dim if np.isscalar(L) else list(L[1])
    d = dict(
        dim=dim,
        n=[n] * dim if np.isscalar(n) else list(n),
        lo=lo,
        hi=hi,
        nv=[nv] * dim if np.isscalar(nv) else list(nv),
        vlo=[-V] * dim if np.isscalar(V) else list(V[0]),
        vhi=[V] * dim if np.isscalar(V) else list(V[1]),
        rule=rule,
        Kn=Kn,
        Ma=Ma,
        dir=[1.0, 0.0, 0.0],
        cfl=0.5,
        dt=0.0,
        body=body,
        cutcell=1,
        upwind=1,
        precision=precision,
        steps=steps,
        **ARGON,
    )
    d.update(kw)
    return d


def circle(r=0.5, center=(0.0, 0.0), **wall):
    b = dict(kind="circle", center=list(center) + [0.0], radii=[r, r, 0.0], accom=1.0, Tw=1.0,
             Uw=[0.0, 0.0, 0.0])
    b.update(wall)
    return b


def sphere(r=0.5, center=(0.0, 0.0, 0.0), **wall):
    b = dict(kind="sphere", center=list(center), radii=[r, r, r], accom=1.0, Tw=1.0,
             Uw=[0.0, 0.0, 0.0])
    b.update(wall)
    return b


def ellipse(a=0.5, aspect=2.0, angle=0.0, center=(0.0, 0.0), **wall):
    b = dict(kind="ellipse", center=list(center) + [0.0], radii=[a, a / aspect, 0.0], angle=angle,
             accom=1.0, Tw=1.0, Uw=[0.0, 0.0, 0.0], Lref=2.0 * a)
    b.update(wall)
    return b


def naca0012(chord=1.0, aoa_deg=0.0, npts=80, center=(0.0, 0.0), **wall):
    """NACA 0012 polygon from the public 4-digit thickness law with a closed
    trailing edge, counter-clockwise, rotated by the angle of attack about the
    quarter chord and placed with the quarter chord at ``center``."""
    t = 0.12
    beta = np.linspace(0.0, math.pi, npts + 1)
    x = 0.5 * (1.0 - np.cos(beta))  # cosine spacing, 0 .. 1
    yt = 5 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2 + 0.2843 * x**3 - 0.1036 * x**4)
    # counter-clockwise: trailing edge -> lower surface -> leading edge -> upper surface
    lower = np.stack([x[::-1], -yt[::-1]], axis=1)  # TE .. LE
    upper = np.stack([x[1:-1], yt[1:-1]], axis=1)  # LE .. TE (exclusive)
    pts = np.concatenate([lower, upper], axis=0) * chord
    pts[:, 0] -= 0.25 * chord
    a = -math.radians(aoa_deg)  # positive angle of attack: nose up
    R = np.array([[math.cos(a), -math.sin(a)], [math.sin(a), math.cos(a)]])
    pts = pts @ R.T + np.asarray(center)[None, :]
    b = dict(kind="polygon", verts=pts.reshape(-1).tolist(), center=list(center) + [0.0],
             radii=[0.0, 0.0, 0.0], accom=1.0, Tw=1.0, Uw=[0.0, 0.0, 0.0], Lref=chord)
    b.update(wall)
    return b


# -------------------------------------------------------------------------
# workloads: the benchmark configurations and the paper's cases
# -------------------------------------------------------------------------

def cylinder_48():
    """2D flow past a circular cylinder, FP64: [-4,4]^2 on 48^2 cells, r = 0.5,
    24^2 trapezoid velocities on [-5,5]^2, Kn 0.1, Ma 0.3, 200 steps, CFL 0.5."""
    return _case(2, 48, 4.0, 24, 5.0, 0.1, 0.3, circle(0.5), precision="fp64", steps=200)


def cylinder_512(Kn=0.1, precision="mixed", steps=200):
    """2D cylinder, 512^2 cells on [-8,8]^2, r = 0.5, 48^2 velocities on [-6,6]^2,
    Ma 0.5 (604M f values per component pair)."""
    return _case(2, 512, 8.0, 48, 6.0, Kn, 0.5, circle(0.5), precision=precision, steps=steps)


def stretched_axis(n, V, h_min):
    """n velocity nodes on [-V, V], symmetric about 0, spaced h_min at the
    centre and growing geometrically toward the ends (a stretched grid,
    refined where the distributions of a gas near rest vary fastest)."""
    if n % 2:
        raise ValueError("an even node count keeps 0 between two nodes")
    m = n // 2
    # half-spacings h_min q^i, i < m, sum to V - h_min / 2 past the first node
    lo, hi = 1.0, 10.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = h_min * (q ** (m - 1) - 1.0) / (q - 1.0) if q != 1.0 else h_min * (m - 1)
        lo, hi = (q, hi) if h_min / 2 + s < V else (lo, q)
    q = 0.5 * (lo + hi)
    half = [h_min / 2]
    for i in range(1, m):
        half.append(half[-1] + h_min * q ** (i - 1))
    half = np.array(half) * (V / half[-1])
    return list(-half[::-1]) + list(half)


def stretched(case, h_min):
    """The case on stretched velocity grids (the same node count and interval
    per axis, spacing h_min at the centre)."""
    c = dict(case)
    c["rule"] = "nodes"
    c["vnodes"] = [stretched_axis(int(c["nv"][a]), float(c["vhi"][a]), h_min) for a in range(c["dim"])]
    return c


def box_walls(dim=2, Tw=1.0, lid=None, lid_T=None):
    """Diffuse walls on every domain face (x-, x+, y-, y+, z-, z+) at Tw; lid:
    the velocity of the top face (y+ in 2D, z+ in 3D), its temperature lid_T."""
    walls = [{"Tw": Tw, "Uw": [0.0, 0.0, 0.0]} for _ in range(2 * dim)] + [None] * (6 - 2 * dim)
    top = 2 * (dim - 1) + 1
    if lid is not None:
        walls[top] = {"Tw": Tw if lid_T is None else lid_T, "Uw": list(lid) + [0.0] * (3 - len(lid))}
    return walls


def cavity(n=64, nv=40, Kn=0.075, lid=0.15, precision="fp64", steps=200, cutcell=1, body=True):
    """Lid-driven cavity with a stationary cylinder at its centre (Sec. 4.1):
    [0,1]^2 on n^2 cells, diffuse walls at T_w = 1, the top wall moving at
    U_w = lid along x, a cylinder of diameter 0.25 at (0.5, 0.5) with T_w = 1,
    nv^2 velocities on [-5,5]^2, Kn 0.075, the gas initially at rest."""
    b = circle(0.125, center=(0.5, 0.5)) if body else {"kind": "none"}
    return _case(2, n, ([0.0, 0.0], [1.0, 1.0]), nv, 5.0, Kn, 0.0, b, precision=precision, steps=steps,
                 cutcell=cutcell, domain_walls=box_walls(2, 1.0, lid=(lid, 0.0)))


def sphere_96(precision="mixed", steps=200):
    """3D flow past a sphere: 96^3 cells on [-4,4]^3, r = 0.5, 20^3 velocities on
    [-5,5]^3, Kn 0.1, Ma 0.5."""
    return _case(3, 96, 4.0, 20, 5.0, 0.1, 0.5, sphere(0.5), precision=precision, steps=steps)


def sphere_96_tree(precision="mixed", steps=200, root=32, maxlevel=2, radii=(2.4, 1.5)):
    """The flow of sphere_96 (r = 0.5, Ma 0.5, Kn 0.1, 20^3 velocities on
    [-5,5]^3, [-4,4]^3) on an octree: a root of root^3 cells refined about the
    centre to level l within radii[l] (the finest edge 1/16 at the wall, the
    96^3 grid's is 1/12), 2:1 balanced, leaves in Z order."""
    d = _case(3, root, 4.0, 20, 5.0, 0.1, 0.5, sphere(0.5), precision=precision, steps=steps)
    d["tree"] = tree_leaves_3d((root,) * 3, maxlevel, d["lo"], d["hi"], (0.0, 0.0, 0.0), list(radii))
    d["tree_spec"] = {"center": [0.0, 0.0, 0.0], "radii": list(radii),
                      "sample": {"root": [8, 8, 8], "maxlevel": 2, "radii": list(radii)}}
    return d


def sphere_supersonic(n=64, nv=24, precision="mixed", steps=200):
    """The supersonic sphere of Sec. 4.4 on a uniform grid: Ma 3.834, Kn 0.03,
    T_w = 1 + (gamma - 1) Ma^2 / 2, n^3 cells on [-4,4]^3, r = 0.5, nv^3
    velocities on a stretched grid over [-3 sqrt(T_w), 3 sqrt(T_w)]^3 with
    central spacing 0.2275 (the paper's smallest), nonnegative ghost values
    (an impulsive start on this grid loses positivity without them)."""
    Ma, gamma = 3.834, 5.0 / 3.0
    Tw = 1.0 + 0.5 * (gamma - 1.0) * Ma * Ma
    c = _case(3, n, 4.0, nv, 3.0 * np.sqrt(Tw), 0.03, Ma, sphere(0.5, Tw=Tw), precision=precision,
              steps=steps, ghost_nonneg=1)
    return stretched(c, 0.2275)


def cylinder_hypersonic(n=1536, nv=60, precision="mixed", steps=200):
    """The hypersonic cylinder of Sec. 4.2: Ma 5, Kn 0.1, radius 1 (the
    reference length), T_w = 1, the domain [-16,16]^2 on a uniform n^2 grid
    (the paper refines to 0.01 at the wall), nv^2 velocities on
    [-10,10]^2, nonnegative ghost values (an impulsive start loses
    positivity in the wake without them)."""
    return _case(2, n, 16.0, nv, 10.0, 0.1, 5.0, circle(1.0), precision=precision, steps=steps,
                 ghost_nonneg=1)


def cylinder_hypersonic_tree(nv=60, precision="mixed", steps=200, root=128, maxlevel=4,
                             radii=(8.0, 4.0, 2.2, 1.5)):
    """The hypersonic cylinder of Sec. 4.2 on a tree-refined grid (C28, C29):
    Ma 5, Kn 0.1, radius 1, T_w = 1, the domain [-16,16]^2 on a root grid of
    root^2 cells refined about the cylinder's centre to level l within
    radii[l] (the finest edge 32 / (root 2^maxlevel) = 1/64 at the wall, the
    paper's wall spacing is 0.01), 2:1 balanced, nv^2 velocities on
    [-10,10]^2, nonnegative ghost values."""
    d = _case(2, root, 16.0, nv, 10.0, 0.1, 5.0, circle(1.0), precision=precision, steps=steps, ghost_nonneg=1)
    d["tree"] = tree_leaves((root, root), maxlevel, d["lo"], d["hi"], (0.0, 0.0), list(radii))
    d["tree_spec"] = {"center": [0.0, 0.0], "radii": list(radii),
                      "sample": {"root": [16, 16], "maxlevel": 3, "radii": [8.0, 4.0, 2.2]}}
    return d


def naca_supersonic_tree(nv=60, precision="mixed", steps=200, root=(80, 112), maxlevel=4,
                         radii=(1.5, 0.6, 0.25, 0.1)):
    """The NACA0012 airfoil of Sec. 4.3 (Ma 2, Kn 0.026, T_w = 1, angle of
    attack 0, chord 1 from the origin) on a tree-refined grid (C28, C29):
    the domain [-3,7] x [-7,7] on a root grid of 80 x 112 cells (edge 1/8)
    refined about the chord to level l within radii[l] of it (the finest
    edge 1/128 within 0.1 of the chord), 2:1 balanced, nv^2 velocities on
    [-4,8] x [-6,6].  Like the uniform grid, it loses positivity after about
    550 steps from the impulsive start; throughput runs are short."""
    body = naca0012(1.0, 0.0, 400, center=(0.25, 0.0))
    root = (root, root * 7 // 5) if np.isscalar(root) else root
    d = _case(2, list(root), ([-3.0, -7.0], [7.0, 7.0]), nv, ([-4.0, -6.0], [8.0, 6.0]), 0.026, 2.0, body,
              precision=precision, steps=steps)
    d["tree"] = tree_leaves(tuple(root), maxlevel, d["lo"], d["hi"], (0.5, 0.0), list(radii), metric="segment",
                            segment=((0.0, 0.0), (1.0, 0.0)))
    d["tree_spec"] = {"center": [0.5, 0.0], "radii": list(radii), "metric": "segment",
                      "segment": [[0.0, 0.0], [1.0, 0.0]],
                      "sample": {"root": [20, 28], "maxlevel": 3, "radii": [1.5, 0.6, 0.25]}}
    return d


def naca_supersonic(cells_per_unit=100, nv=60, precision="mixed", steps=200):
    """The NACA0012 airfoil of Sec. 4.3: Ma 2, Kn 0.026, T_w = 1, angle of
    attack 0, chord 1 with the leading edge at the origin, the domain
    [-3,7] x [-7,7] on a uniform grid of cells_per_unit cells per unit length
    (1000 x 1400 by default), nv^2 velocities on [-4,8] x [-6,6].  From the
    impulsive start the state loses positivity after about 550 steps (the
    same on a tree refined about the chord); throughput runs are short."""
    n = [10 * cells_per_unit, 14 * cells_per_unit]
    body = naca0012(1.0, 0.0, 400, center=(0.25, 0.0))
    return _case(2, n, ([-3.0, -7.0], [7.0, 7.0]), nv, ([-4.0, -6.0], [8.0, 6.0]), 0.026, 2.0, body,
                 precision=precision, steps=steps)


def sphere_96_stretched(precision="mixed", steps=200):
    """The 96^3 sphere (Ma 0.5, Kn 0.1) on a stretched velocity grid: 20^3
    nodes on [-5,5]^3, spacing 0.25 at the centre (0.53 on the uniform grid)
    growing toward the ends."""
    return stretched(sphere_96(precision=precision, steps=steps), 0.25)


def sphere_24(precision="fp64", steps=50):
    """The 3D sphere downscaled to 24^3 cells and 12^3 velocities (50 steps)."""
    return _case(3, 24, 4.0, 12, 5.0, 0.1, 0.5, sphere(0.5), precision=precision, steps=steps)


def batched_2d(seed=0, ncases=64, precision="mixed"):
    """64 seeded 2D cases of uneven size: n ~ U{64..384} cells per axis on
    [-4,4]^2, m ~ U{16..40} velocities per axis on [-6,6]^2, body in {circle,
    ellipse with aspect U[1,3], NACA0012 at AoA U[0,10] deg}, Kn log-uniform in
    [0.01, 1], Ma uniform in [0.1, 0.8]."""
    rng = np.random.default_rng(seed)
    cases = []
    for i in range(ncases):
        n = int(rng.integers(64, 385))
        m = int(rng.integers(16, 41))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            body = circle(0.5)
        elif kind == 1:
            body = ellipse(0.5, float(rng.uniform(1.0, 3.0)), 0.0)
        else:
            body = naca0012(1.0, float(rng.uniform(0.0, 10.0)))
        Kn = float(10.0 ** rng.uniform(-2.0, 0.0))
        Ma = float(rng.uniform(0.1, 0.8))
        c = _case(2, n, 4.0, m, 6.0, Kn, Ma, body, precision=precision, steps=200)
        c["name"] = f"batch{seed}_{i}"
        cases.append(c)
    return cases


def served_stream(seed=0, nreq=200, rate=20.0):
    """Poisson arrivals (rate per second) of mixed requests: 80% 2D cases shaped
    like batched_2d, 20% 3D spheres with n ~ U{32..64} cells per axis on
    [-4,4]^3 and m ~ U{12..20} velocities per axis on [-5,5]^3.  Returns a list
    of (arrival_time_s, case)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    pool2d = batched_2d(seed + 1000, ncases=nreq)
    for i in range(nreq):
        t += float(rng.exponential(1.0 / rate))
        if rng.uniform() < 0.8:
            c = dict(pool2d[i])
        else:
            n = int(rng.integers(32, 65))
            m = int(rng.integers(12, 21))
            c = _case(3, n, 4.0, m, 5.0, 0.1, 0.5, sphere(0.5), precision="mixed", steps=0)
        c["name"] = f"req{i}"
        out.append((t, c))
    return out


def small_2d(body="circle", n=16, nv=8, precision="fp64", **kw):
    """A small 2D case that the oracle finishes in well under a second per step."""
    b = {"circle": circle(0.7), "ellipse": ellipse(0.8, 1.7, 0.4), "naca": naca0012(2.5, 7.0, 60),
         "none": {"kind": "none"}}[body]
    return _case(2, n, 2.0, nv, 4.5, kw.pop("Kn", 0.1), kw.pop("Ma", 0.3), b, precision=precision,
                 steps=kw.pop("steps", 5), **kw)


# ---------------------------------------------------------------------------
# quadtree meshes (the tree-refined physical grids of Sec. 4.2-4.4)
# ---------------------------------------------------------------------------

def tree_leaves(root, maxlevel, lo, hi, center, radii, metric="point", segment=None):
    """Leaves (level, ix, iy) of a 2:1-balanced quadtree over a root grid of
    root[0] x root[1] cells on [lo, hi]: a cell of level l < maxlevel is split
    while its centre lies within radii[l] of `center` (radii decreasing with
    the level; metric "point": the distance to the point, "x" or "y": the
    distance along that axis only, which refines stripes, "segment": the
    distance to the segment ((x0, y0), (x1, y1)) given as `segment`, which
    refines about a thin body), then any leaf with a face neighbour two or
    more levels finer is split until the tree is balanced.  Integer
    coordinates are those of the leaf's level (0 <= ix < root[0] 2^level).
    Geometry only."""
    nx0, ny0 = root
    hx0, hy0 = (hi[0] - lo[0]) / nx0, (hi[1] - lo[1]) / ny0
    L = maxlevel
    # leaf level of every finest cell: the tree as a level map
    nf = (nx0 << L, ny0 << L)
    lev = np.zeros(nf, dtype=np.int64)

    def blocks(l):
        """level map in blocks of level-l cells: (nx_l, s, ny_l, s)"""
        s = 1 << (L - l)
        return lev.reshape(nx0 << l, s, ny0 << l, s)

    def uniform_at(l):
        """level-l cells that are one leaf of level l"""
        bl = blocks(l)
        return (bl.min(axis=(1, 3)) == l) & (bl.max(axis=(1, 3)) == l)

    def split(l, mask):
        s = 1 << (L - l)
        up = np.repeat(np.repeat(mask, s, axis=0), s, axis=1)
        lev[up] = l + 1

    for l in range(L):
        h = 2.0 ** -l
        xc = lo[0] + (np.arange(nx0 << l) + 0.5) * hx0 * h
        yc = lo[1] + (np.arange(ny0 << l) + 0.5) * hy0 * h
        X, Y = np.meshgrid(xc, yc, indexing="ij")
        if metric == "segment":
            (x0, y0), (x1, y1) = segment
            ex, ey = x1 - x0, y1 - y0
            t = np.clip(((X - x0) * ex + (Y - y0) * ey) / (ex * ex + ey * ey), 0.0, 1.0)
            near = np.hypot(X - x0 - t * ex, Y - y0 - t * ey) <= radii[l]
        elif metric == "x":
            near = np.abs(X - center[0]) <= radii[l]
        elif metric == "y":
            near = np.abs(Y - center[1]) <= radii[l]
        else:
            near = np.hypot(X - center[0], Y - center[1]) <= radii[l]
        split(l, uniform_at(l) & near)
    # 2:1 balance across faces: raise a leaf whose face neighbour is two or more
    # levels finer (one level at a time, until nothing changes)
    changed = True
    while changed:
        changed = False
        for l in range(L):
            s = 1 << (L - l)
            nxl, nyl = nx0 << l, ny0 << l
            leaf = uniform_at(l)
            # the largest level in the strip of finest cells beyond each face
            big = np.zeros((nxl, nyl), dtype=bool)
            first = lev[0::s, :].reshape(nxl, nyl, s).max(axis=2)   # x-first finest column of each block
            last = lev[s - 1::s, :].reshape(nxl, nyl, s).max(axis=2)
            big[1:, :] |= last[:-1, :] >= l + 2
            big[:-1, :] |= first[1:, :] >= l + 2
            firsty = lev[:, 0::s].reshape(nxl, s, nyl).max(axis=1)
            lasty = lev[:, s - 1::s].reshape(nxl, s, nyl).max(axis=1)
            big[:, 1:] |= lasty[:, :-1] >= l + 2
            big[:, :-1] |= firsty[:, 1:] >= l + 2
            m = leaf & big
            if m.any():
                split(l, m)
                changed = True
    # the leaves in the tree's depth-first (Z) order: root cells row by row,
    # the four children of a cell as (0,0), (1,0), (0,1), (1,1), so that
    # consecutive leaves are close in space
    level, ix, iy = [], [], []

    def visit(l, i, j):
        s = 1 << (L - l)
        if lev[i * s, j * s] == l:
            level.append(l)
            ix.append(i)
            iy.append(j)
            return
        for dj in (0, 1):
            for di in (0, 1):
                visit(l + 1, 2 * i + di, 2 * j + dj)

    for j in range(ny0):
        for i in range(nx0):
            visit(0, i, j)
    return {"maxlevel": L, "level": level, "ix": ix, "iy": iy}


def tree_leaves_3d(root, maxlevel, lo, hi, center, radii):
    """Leaves (level, ix, iy, iz) of a 2:1-balanced octree over a root grid of
    root[0] x root[1] x root[2] cells on [lo, hi]: a cell of level l <
    maxlevel is split while its centre lies within radii[l] of `center`, then
    any leaf with a face neighbour two or more levels finer is split until
    the tree is balanced; listed depth first (Z order: root cells with x
    fastest, the eight children with x, then y, then z fastest).  Geometry
    only."""
    n0 = tuple(int(r) for r in root)
    L = maxlevel
    nf = tuple(r << L for r in n0)
    lev = np.zeros(nf, dtype=np.int64)

    def blocks(l):
        s = 1 << (L - l)
        return lev.reshape(n0[0] << l, s, n0[1] << l, s, n0[2] << l, s)

    def uniform_at(l):
        bl = blocks(l)
        return (bl.min(axis=(1, 3, 5)) == l) & (bl.max(axis=(1, 3, 5)) == l)

    def split(l, mask):
        s = 1 << (L - l)
        up = mask.repeat(s, axis=0).repeat(s, axis=1).repeat(s, axis=2)
        lev[up] = l + 1

    h0 = [(hi[a] - lo[a]) / n0[a] for a in range(3)]
    for l in range(L):
        c = [lo[a] + (np.arange(n0[a] << l) + 0.5) * h0[a] * 2.0 ** -l for a in range(3)]
        X, Y, Z = np.meshgrid(*c, indexing="ij")
        near = np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2) <= radii[l]
        split(l, uniform_at(l) & near)
    changed = True
    while changed:
        changed = False
        for l in range(L):
            s = 1 << (L - l)
            nl = tuple(r << l for r in n0)
            big = np.zeros(nl, dtype=bool)
            for a in range(3):
                # the largest level in the slab of finest cells on each side of every block
                first = np.take(lev, np.arange(0, nf[a], s), axis=a)
                last = np.take(lev, np.arange(s - 1, nf[a], s), axis=a)
                shp = [nl[0], s, nl[1], s, nl[2], s]
                shp[2 * a + 1] = 1
                fmax = first.reshape(shp).max(axis=(1, 3, 5))
                lmax = last.reshape(shp).max(axis=(1, 3, 5))
                lo_sl = [slice(None)] * 3
                hi_sl = [slice(None)] * 3
                lo_sl[a], hi_sl[a] = slice(1, None), slice(None, -1)
                big[tuple(lo_sl)] |= lmax[tuple(hi_sl)] >= l + 2
                big[tuple(hi_sl)] |= fmax[tuple(lo_sl)] >= l + 2
            m = uniform_at(l) & big
            if m.any():
                split(l, m)
                changed = True
    level, ix, iy, iz = [], [], [], []

    def visit(l, i, j, k):
        s = 1 << (L - l)
        if lev[i * s, j * s, k * s] == l:
            level.append(l)
            ix.append(i)
            iy.append(j)
            iz.append(k)
            return
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    visit(l + 1, 2 * i + di, 2 * j + dj, 2 * k + dk)

    for k in range(n0[2]):
        for j in range(n0[1]):
            for i in range(n0[0]):
                visit(0, i, j, k)
    return {"maxlevel": L, "level": level, "ix": ix, "iy": iy, "iz": iz}


def tree_case_3d(root=8, maxlevel=2, L=2.0, nv=6, V=4.5, Kn=0.1, Ma=0.3, radii=None, center=(0.0, 0.0, 0.0),
                 precision="fp64", steps=20, body=None):
    """A 3D case on an octree: root^3 cells on [-L, L]^3 refined about
    `center` (by default to level 1 within 0.6 L and to level 2 within 0.3 L),
    freestream domain faces, no body unless given (in the finest level)."""
    if radii is None:
        radii = [0.6 * L, 0.3 * L] + [0.3 * L * 0.5 ** i for i in range(1, maxlevel)]
    d = _case(3, root, L, nv, V, Kn, Ma, body or {"kind": "none"}, precision=precision, steps=steps)
    d["tree"] = tree_leaves_3d((root, root, root), maxlevel, d["lo"], d["hi"], center, radii)
    return d


def tree_centres(case):
    """Centres (nleaf, dim) of the leaves of a tree case (geometry only)."""
    tr = case["tree"]
    D = int(case["dim"])
    lev = np.asarray(tr["level"], dtype=np.float64)
    h = np.array([(case["hi"][a] - case["lo"][a]) / case["n"][a] for a in range(D)])
    size = h[None, :] * (0.5 ** lev)[:, None]
    ij = np.stack([np.asarray(tr[k], dtype=np.float64) for k in ("ix", "iy", "iz")[:D]], axis=1)
    return np.asarray(case["lo"][:D])[None, :] + (ij + 0.5) * size


def tree_case(root=16, maxlevel=2, L=2.0, nv=12, V=4.5, Kn=0.1, Ma=0.3, radii=None, center=(0.0, 0.0),
              precision="fp64", steps=20, metric="point", body=None):
    """A 2D case on a quadtree: root^2 cells on [-L, L]^2 refined around
    `center` (by default to level 1 within 0.6 L and to level 2 within 0.3 L),
    freestream domain faces, no body unless given (it must lie in the finest
    level)."""
    if radii is None:
        radii = [0.6 * L, 0.3 * L] + [0.3 * L * 0.5 ** i for i in range(1, maxlevel)]
    d = _case(2, root, L, nv, V, Kn, Ma, body or {"kind": "none"}, precision=precision, steps=steps)
    d["tree"] = tree_leaves((root, root), maxlevel, d["lo"], d["hi"], center, radii, metric)
    return d


def tree_2d(precision="mixed", steps=200, root=128):
    """A tree-refined 2D grid at GB300 size: a root grid of 128^2 cells on
    [-8,8]^2 refined around the origin to level 1 within 4, level 2 within 2
    and level 3 within 1 (finest edge 1/64: the 1024^2 uniform grid's), 2:1
    balanced (45,436 leaves), 48^2 velocities on [-6,6]^2, Kn 0.1, Ma 0.5, no
    body (the tree's transport, relaxation and moments alone)."""
    d = _case(2, root, 8.0, 48, 6.0, 0.1, 0.5, {"kind": "none"}, precision=precision, steps=steps)
    d["tree"] = tree_leaves((root, root), 3, d["lo"], d["hi"], (0.0, 0.0), [4.0, 2.0, 1.0])
    d["tree_spec"] = {"center": [0.0, 0.0], "radii": [4.0, 2.0, 1.0],
                      "sample": {"root": [16, 16], "maxlevel": 3, "radii": [4.0, 2.0, 1.0]}}
    return d
