"""Plain FP64 CPU oracle of the ghost-cell immersed-boundary DVM step.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
solver product (``paper_2512_20252_gb300``) never imports it and shares no code
with it: the oracle is a separate C file (``ibdvm_oracle.c``) compiled with gcc
and driven here through ctypes.

The oracle follows Ge, Cai, Zhang and Xiao, "An immersed boundary method for
the discrete velocity model of the Boltzmann equation" (arXiv 2512.20252):
Sec. 2 (Shakhov model, quadrature, finite volume with van Leer reconstruction,
Maxwell wall), Sec. 3.2 (ghost cells, shifted point, upwind-weighted compact
interpolation, intersect point, ghost construction, velocity-space cut cells)
and Sec. 4 (reduced distributions, non-dimensional equilibria, VHS viscosity,
residual, forward Euler).  The header of ``ibdvm_oracle.c`` lists every reading
taken where the paper is silent and the parts whose parity is unpinned.

Case descriptions are plain dicts (see ``paper_2512_20252_gb300.workloads``
for the presets); this module only marshals them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibdvm_oracle.c")
_SO = os.path.join(_HERE, "_build", "libibdvm_oracle.so")
_lock = threading.Lock()
_lib = None

BODY_KINDS = {"none": 0, "circle": 1, "ellipse": 2, "sphere": 3, "polygon": 4, "halfspace": 5}
FLUID, GHOST, SOLID = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (portable C11, -O2)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ibdvm_oracle.h"))
    ):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("nv", ctypes.c_int * 3),
        ("vlo", ctypes.c_double * 3),
        ("vhi", ctypes.c_double * 3),
        ("rule", ctypes.c_int),
        ("Kn", ctypes.c_double),
        ("Ma", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("omega_vhs", ctypes.c_double),
        ("alpha_vhs", ctypes.c_double),
        ("rho_inf", ctypes.c_double),
        ("T_inf", ctypes.c_double),
        ("dir", ctypes.c_double * 3),
        ("cfl", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("kind", ctypes.c_int),
        ("center", ctypes.c_double * 3),
        ("radii", ctypes.c_double * 3),
        ("angle", ctypes.c_double),
        ("verts", ctypes.POINTER(ctypes.c_double)),
        ("nverts", ctypes.c_int),
        ("accom", ctypes.c_double),
        ("Tw", ctypes.c_double),
        ("Uw", ctypes.c_double * 3),
        ("Lref", ctypes.c_double),
        ("cutcell", ctypes.c_int),
        ("upwind", ctypes.c_int),
        ("wall", ctypes.c_int * 6),
        ("wall_T", ctypes.c_double * 6),
        ("wall_U", (ctypes.c_double * 3) * 6),
        ("vnodes", ctypes.POINTER(ctypes.c_double) * 3),
        ("ghost_nonneg", ctypes.c_int),
    ]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_LL = ctypes.POINTER(ctypes.c_longlong)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            V = ctypes.c_void_p
            sig = {
                "or_create": ([P], V),
                "or_destroy": ([V], None),
                "or_set_threads": ([V, ctypes.c_int], None),
                "or_sizes": ([V, _LL], None),
                "or_dt": ([V], ctypes.c_double),
                "or_velocities": ([V, _D, _D], None),
                "or_cell_types": ([V, _U8], None),
                "or_links": ([V, _I, _I, _I, _I, _I, _D, _D], None),
                "or_cut_table": ([V, _D], None),
                "or_upwind_weights": ([V, ctypes.c_int, _D], None),
                "or_surface_count": ([V], ctypes.c_int),
                "or_surface_cells": ([V, _I, _I, _I], None),
                "or_get_f": ([V, _D], None),
                "or_set_f": ([V, _D], None),
                "or_freestream": ([V, _D], None),
                "or_step": ([V, ctypes.c_int, _D], ctypes.c_int),
                "or_moments": ([V, _D, _D], None),
                "or_forces": ([V, _D, _D, _D, _D], None),
                "or_ghost_band": ([V, _D, _D, _D, _D, _D, _D, _D], None),
                "or_domain_wall_density": ([V, _D, _D], None),
                "or_mu0": ([ctypes.c_double] * 3, ctypes.c_double),
                "or_vanleer": ([ctypes.c_double] * 2, ctypes.c_double),
                "or_cell_moments": ([V, _D, _D], None),
                "or_shakhov": ([V, ctypes.c_double, _D, ctypes.c_double, _D, _D], None),
                "or_maxwellian": ([V, ctypes.c_double, _D, ctypes.c_double, _D], None),
                "or_cut_fraction_2d": ([_D, _D, _D], ctypes.c_double),
                "or_cut_fraction_3d": ([_D, _D, _D], ctypes.c_double),
                "or_residual": ([V, _D, _D], ctypes.c_double),
                "or_tree_create": ([P, ctypes.c_long, ctypes.c_int, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_int)], V),
                "or_tree_destroy": ([V], None),
                "or_tree_set_threads": ([V, ctypes.c_int], None),
                "or_tree_sizes": ([V, _LL], None),
                "or_tree_dt": ([V], ctypes.c_double),
                "or_tree_neighbours": ([V, _LL], None),
                "or_tree_get_f": ([V, _D], None),
                "or_tree_set_f": ([V, _D], None),
                "or_tree_step": ([V, ctypes.c_int, _D], ctypes.c_int),
                "or_tree_moments": ([V, _D, _D], None),
                "or_tree_cell_types": ([V, ctypes.POINTER(ctypes.c_ubyte)], None),
                "or_tree_forces": ([V, _D, _D, _D, _D], None),
                "or_tree_finest": ([V], V),
            }
            for name, (args, res) in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _arr3(v, fill=0.0):
    v = list(v) + [fill] * (3 - len(v))
    return v[:3]


def _params(cfg: dict) -> tuple[_Params, object]:
    p = _Params()
    dim = int(cfg["dim"])
    p.dim = dim
    p.n[:] = [int(x) for x in _arr3(cfg["n"], 1)]
    p.lo[:] = _arr3(cfg["lo"])
    p.hi[:] = _arr3(cfg["hi"], 1.0)
    p.nv[:] = [int(x) for x in _arr3(cfg["nv"], 1)]
    p.vlo[:] = _arr3(cfg["vlo"])
    p.vhi[:] = _arr3(cfg["vhi"], 1.0)
    p.rule = {"trapezoid": 0, "midpoint": 1, "nodes": 2}[cfg.get("rule", "trapezoid")]
    p.Kn = cfg["Kn"]
    p.Ma = cfg["Ma"]
    p.Pr = cfg.get("Pr", 2.0 / 3.0)
    p.gamma = cfg.get("gamma", 5.0 / 3.0)
    p.omega_vhs = cfg.get("omega_vhs", 0.81)
    p.alpha_vhs = cfg.get("alpha_vhs", 1.0)
    p.rho_inf = cfg.get("rho_inf", 1.0)
    p.T_inf = cfg.get("T_inf", 1.0)
    p.dir[:] = _arr3(cfg.get("dir", [1.0, 0.0, 0.0]))
    p.cfl = cfg.get("cfl", 0.5)
    p.dt = cfg.get("dt", 0.0)
    body = cfg.get("body") or {"kind": "none"}
    p.kind = BODY_KINDS[body["kind"]]
    p.center[:] = _arr3(body.get("center", [0.0, 0.0, 0.0]))
    p.radii[:] = _arr3(body.get("radii", [0.0, 0.0, 0.0]))
    p.angle = body.get("angle", 0.0)
    keep = []
    if body["kind"] == "polygon":
        verts = np.ascontiguousarray(np.asarray(body["verts"], dtype=np.float64).reshape(-1))
        keep.append(verts)
        p.verts = _dp(verts)
        p.nverts = verts.size // 2
    if p.rule == 2:
        # explicit velocity nodes per axis (C25): nv and the interval follow them
        for a in range(dim):
            nodes = np.ascontiguousarray(np.asarray(cfg["vnodes"][a], dtype=np.float64))
            keep.append(nodes)
            p.vnodes[a] = _dp(nodes)
            p.nv[a] = nodes.size
            p.vlo[a] = float(nodes[0])
            p.vhi[a] = float(nodes[-1])
    p.accom = body.get("accom", 1.0)
    p.Tw = body.get("Tw", 1.0)
    p.Uw[:] = _arr3(body.get("Uw", [0.0, 0.0, 0.0]))
    p.Lref = body.get("Lref", 0.0)
    p.cutcell = int(cfg.get("cutcell", 1))
    p.upwind = int(cfg.get("upwind", 1))
    p.ghost_nonneg = int(cfg.get("ghost_nonneg", 0))
    # domain faces (x-, x+, y-, y+, z-, z+): None = freestream halo, or a
    # diffuse wall {"Tw": T, "Uw": [u, v, w]}
    for i, wall in enumerate(cfg.get("domain_walls") or [None] * 6):
        if wall:
            p.wall[i] = 1
            p.wall_T[i] = float(wall.get("Tw", 1.0))
            p.wall_U[i][:] = _arr3(list(wall.get("Uw", [0.0, 0.0, 0.0])))
    return p, keep


class OracleCase:
    """One case of the oracle: geometry, velocity grid and state f[cell][k][comp]."""

    def __init__(self, cfg: dict, threads: int = 1):
        self.lib = _load()
        self.cfg = dict(cfg)
        self._p, self._keep = _params(cfg)
        self.h = self.lib.or_create(ctypes.byref(self._p))
        self.set_threads(threads)
        s = np.zeros(6, dtype=np.int64)
        self.lib.or_sizes(self.h, s.ctypes.data_as(_LL))
        self.ncell, self.nvel, self.ncomp, self.nlink, self.nghost, self.nfluid = (int(x) for x in s)
        self.dim = int(cfg["dim"])

    def __del__(self):
        h = getattr(self, "h", None)
        if h and not getattr(self, "_owner", None):
            self.lib.or_destroy(h)
        self.h = None

    @classmethod
    def _view(cls, lib, h, cfg: dict, owner):
        """A case whose handle another object owns (the finest grid of a tree)."""
        c = cls.__new__(cls)
        c.lib, c.h, c.cfg, c._owner = lib, h, dict(cfg), owner
        s = np.zeros(6, dtype=np.int64)
        lib.or_sizes(h, s.ctypes.data_as(_LL))
        c.ncell, c.nvel, c.ncomp, c.nlink, c.nghost, c.nfluid = (int(x) for x in s)
        c.dim = int(cfg["dim"])
        return c

    def set_threads(self, threads: int) -> None:
        """Host threads of the per-ghost and per-cell loops (bitwise the same
        results for any count)."""
        self.threads = max(1, int(threads))
        self.lib.or_set_threads(self.h, self.threads)

    # geometry and grids -------------------------------------------------
    @property
    def dt(self) -> float:
        return float(self.lib.or_dt(self.h))

    def velocities(self):
        xi = np.zeros((self.nvel, 3))
        w = np.zeros(self.nvel)
        self.lib.or_velocities(self.h, _dp(xi), _dp(w))
        return xi, w

    def cell_types(self) -> np.ndarray:
        t = np.zeros(self.ncell, dtype=np.uint8)
        self.lib.or_cell_types(self.h, t.ctypes.data_as(_U8))
        return t

    def links(self) -> dict:
        n = self.nlink
        ints = [np.zeros(n, dtype=np.int32) for _ in range(5)]
        xw = np.zeros((n, 3))
        nw = np.zeros((n, 3))
        self.lib.or_links(self.h, *[a.ctypes.data_as(_I) for a in ints], _dp(xw), _dp(nw))
        keys = ["ghost", "donor", "aux", "axis", "side"]
        out = {k: v for k, v in zip(keys, ints)}
        out["xw"] = xw
        out["nw"] = nw
        return out

    def cut_table(self) -> np.ndarray:
        wg = np.zeros((self.nlink, self.nvel))
        self.lib.or_cut_table(self.h, _dp(wg))
        return wg

    def surface_cells(self):
        tot = self.lib.or_surface_count(self.h)
        g = np.zeros(self.nghost, dtype=np.int32)
        off = np.zeros(self.nghost + 1, dtype=np.int32)
        cells = np.zeros(max(tot, 1), dtype=np.int32)
        self.lib.or_surface_cells(
            self.h, g.ctypes.data_as(_I), off.ctypes.data_as(_I), cells.ctypes.data_as(_I)
        )
        return g, off, cells[:tot]

    def upwind_weights(self, gi: int) -> np.ndarray:
        """Weights of Eq. upwind of ghost gi over its surface cells, [j][k]."""
        _, off, _ = self.surface_cells()
        ns = int(off[gi + 1] - off[gi])
        out = np.zeros((ns, self.nvel))
        self.lib.or_upwind_weights(self.h, int(gi), _dp(out))
        return out

    # state --------------------------------------------------------------
    def shape(self):
        return (self.ncell, self.nvel, self.ncomp)

    def get_f(self) -> np.ndarray:
        f = np.zeros(self.shape())
        self.lib.or_get_f(self.h, _dp(f))
        return f

    def set_f(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape())
        self.lib.or_set_f(self.h, _dp(f))

    def freestream(self) -> np.ndarray:
        g = np.zeros((self.nvel, self.ncomp))
        self.lib.or_freestream(self.h, _dp(g))
        return g

    def step(self, nsteps: int = 1) -> float:
        r = ctypes.c_double(0.0)
        self.lib.or_step(self.h, int(nsteps), ctypes.byref(r))
        return r.value

    def moments(self):
        W = np.zeros((self.ncell, self.dim + 2))
        q = np.zeros((self.ncell, self.dim))
        self.lib.or_moments(self.h, _dp(W), _dp(q))
        return W, q

    def forces(self):
        F = np.zeros(3)
        Q = ctypes.c_double()
        CD = ctypes.c_double()
        CL = ctypes.c_double()
        self.lib.or_forces(self.h, _dp(F), ctypes.byref(Q), ctypes.byref(CD), ctypes.byref(CL))
        return F, Q.value, CD.value, CL.value

    def ghost_band(self, f: np.ndarray | None = None) -> dict:
        if f is None:
            f = self.get_f()
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape())
        shp = (self.nlink, self.nvel, self.ncomp)
        out = {k: np.zeros(shp) for k in ["fgc", "fsp", "fiw", "fstarw", "fstargc"]}
        rhow = np.zeros(max(self.nlink, 1))
        self.lib.or_ghost_band(
            self.h, _dp(f), *[_dp(out[k]) for k in ["fgc", "fsp", "fiw", "fstarw", "fstargc"]],
            _dp(rhow),
        )
        out["rhow"] = rhow[: self.nlink]
        return out

    def domain_wall_density(self, f: np.ndarray | None = None) -> np.ndarray:
        """rho_w of every diffuse domain face, [cell][6] (faces 2a + (s > 0));
        0 where the face is not a diffuse wall of a fluid cell."""
        if f is None:
            f = self.get_f()
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape())
        out = np.zeros((self.ncell, 6))
        self.lib.or_domain_wall_density(self.h, _dp(f), _dp(out))
        return out

    # wall points ------------------------------------------------------------
    WALL_COLUMNS = ("rho", "slip_x", "slip_y", "slip_z", "T", "T_jump", "p", "tau_x", "tau_y", "tau_z",
                    "q_n", "Cp")

    def wall_quantities(self, f: np.ndarray | None = None) -> np.ndarray:
        """Per link, the gas at its wall point (intersect point x_w, normal n
        into the gas): the moments (Sec. 2.1, Eqs. moments1-3) of the wall
        distribution f*_w of Eqs. general bc / Maxwell BC / fwc, whose cut
        boxes already hold the blend of the incident and reflected parts, so
        the plain quadrature weights give the cut-corrected moments.  Columns
        (WALL_COLUMNS), with h the mass-carrying component (f in 3D) and b the
        second reduced one (0 in 3D):
          rho     sum w h
          slip    U - U_w, with U = sum w xi h / rho
          T       three translational degrees of freedom (Sec. 4):
                  3/2 rho T = sum w (|c|^2 h + b), c = xi - U
          T_jump  T - T_w
          p       n.P.n with P_ab = sum w c_a c_b h (the normal stress)
          tau     P.n - p n (the tangential stress)
          q_n     n.q with q = 1/2 sum w c (|c|^2 h + b) (Eq. moments3)
          Cp      2 (p - p_0) / (rho_0 |U_0|^2), p_0 = rho_0 T_0 / 2
                  (Sec. 4.3); NaN without a free stream velocity
        The paper plots these along the wall without stating how they are
        taken from the wall distribution: this is the reading."""
        gb = self.ghost_band(f)
        fs = gb["fstarw"]
        xi, w = self.velocities()
        nw = self.links()["nw"]
        body = self.cfg.get("body") or {}
        Tw = float(body.get("Tw", 1.0))
        Uw = np.array(_arr3(list(body.get("Uw", [0.0, 0.0, 0.0]))))
        rho0 = float(self.cfg.get("rho_inf", 1.0))
        T0 = float(self.cfg.get("T_inf", 1.0))
        U0 = float(self.cfg["Ma"]) * np.sqrt(float(self.cfg.get("gamma", 5.0 / 3.0)) / 2.0)
        out = np.zeros((self.nlink, len(self.WALL_COLUMNS)))
        for l in range(self.nlink):
            h = fs[l, :, 0]
            b = fs[l, :, 1] if self.ncomp == 2 else np.zeros_like(h)
            n = nw[l]
            rho = np.sum(w * h)
            U = np.array([np.sum(w * xi[:, a] * h) for a in range(3)]) / rho
            c = xi - U
            e = np.sum(c * c, axis=1) * h + b
            T = 2.0 * np.sum(w * e) / (3.0 * rho)
            P = np.array([[np.sum(w * c[:, a] * c[:, bb] * h) for bb in range(3)] for a in range(3)])
            p = n @ P @ n
            tau = P @ n - p * n
            q = np.array([0.5 * np.sum(w * c[:, a] * e) for a in range(3)])
            cp = 2.0 * (p - 0.5 * rho0 * T0) / (rho0 * U0 * U0) if U0 > 0.0 else np.nan
            out[l] = [rho, *(U - Uw), T, T - Tw, p, *tau, q @ n, cp]
        return out

    # building blocks ------------------------------------------------------
    def cell_moments(self, fcell: np.ndarray) -> dict:
        fcell = np.ascontiguousarray(fcell, dtype=np.float64).reshape(self.nvel, self.ncomp)
        out = np.zeros(16)
        self.lib.or_cell_moments(self.h, _dp(fcell), _dp(out))
        D = self.dim
        return {
            "rho": out[0],
            "rhoU": out[1 : 1 + D].copy(),
            "rhoE": out[D + 1],
            "T": out[D + 2],
            "p": out[D + 3],
            "q": out[D + 4 : D + 4 + D].copy(),
        }

    def shakhov(self, rho, U, T, q) -> np.ndarray:
        U = np.asarray(_arr3(list(U)), dtype=np.float64)
        q = np.asarray(_arr3(list(q)), dtype=np.float64)
        g = np.zeros((self.nvel, self.ncomp))
        self.lib.or_shakhov(self.h, float(rho), _dp(U), float(T), _dp(q), _dp(g))
        return g

    def maxwellian(self, rho, U, T) -> np.ndarray:
        U = np.asarray(_arr3(list(U)), dtype=np.float64)
        g = np.zeros((self.nvel, self.ncomp))
        self.lib.or_maxwellian(self.h, float(rho), _dp(U), float(T), _dp(g))
        return g

    def residual(self, Wold: np.ndarray, Wnew: np.ndarray) -> float:
        Wold = np.ascontiguousarray(Wold, dtype=np.float64)
        Wnew = np.ascontiguousarray(Wnew, dtype=np.float64)
        return float(self.lib.or_residual(self.h, _dp(Wold), _dp(Wnew)))


def mu0(Kn: float, alpha: float = 1.0, omega: float = 0.81) -> float:
    return float(_load().or_mu0(Kn, alpha, omega))


def vanleer(s1: float, s2: float) -> float:
    return float(_load().or_vanleer(s1, s2))


def cut_fraction_2d(blo, bhi, n) -> float:
    a = [np.asarray(_arr3(list(v)), dtype=np.float64) for v in (blo, bhi, n)]
    return float(_load().or_cut_fraction_2d(*[_dp(x) for x in a]))


def cut_fraction_3d(blo, bhi, n) -> float:
    a = [np.asarray(_arr3(list(v)), dtype=np.float64) for v in (blo, bhi, n)]
    return float(_load().or_cut_fraction_3d(*[_dp(x) for x in a]))


class OracleTree:
    """A case on a tree-refined grid (reading C28; a quadtree in 2D, an octree
    in 3D): the leaves of ``cfg["tree"]`` (level, ix, iy, and iz in 3D, over
    the root grid ``cfg["n"]``) and the state f[leaf][k][comp]; freestream
    domain faces; a body in the finest level (reading C29)."""

    def __init__(self, cfg: dict, threads: int = 1):
        self.lib = _load()
        self.cfg = dict(cfg)
        self._p, self._keep = _params(cfg)
        tree = cfg["tree"]
        self.dim = int(cfg["dim"])
        self._lev = np.ascontiguousarray(np.asarray(tree["level"], dtype=np.int32))
        self._ix = np.ascontiguousarray(np.asarray(tree["ix"], dtype=np.int32))
        self._iy = np.ascontiguousarray(np.asarray(tree["iy"], dtype=np.int32))
        self._iz = np.ascontiguousarray(np.asarray(tree["iz"], dtype=np.int32)) if self.dim == 3 else None
        why = ctypes.c_int(0)
        self.h = self.lib.or_tree_create(ctypes.byref(self._p), self._lev.size, int(tree["maxlevel"]),
                                         self._lev.ctypes.data_as(_I), self._ix.ctypes.data_as(_I),
                                         self._iy.ctypes.data_as(_I),
                                         self._iz.ctypes.data_as(_I) if self._iz is not None else None,
                                         ctypes.byref(why))
        if not self.h:
            if why.value == 2:
                raise ValueError("the body must lie in the finest level of the tree")
            raise ValueError("invalid tree: the leaves must tile the domain with face neighbours at most one level apart")
        self.lib.or_tree_set_threads(self.h, max(1, int(threads)))
        s = np.zeros(3, dtype=np.int64)
        self.lib.or_tree_sizes(self.h, s.ctypes.data_as(_LL))
        self.nleaf, self.nvel, self.ncomp = (int(x) for x in s)
        self.ncell = self.nleaf
        self.nfluid = int(np.count_nonzero(self.cell_types() == 0))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_tree_destroy(h)
            self.h = None

    @property
    def dt(self) -> float:
        return float(self.lib.or_tree_dt(self.h))

    def shape(self):
        return (self.nleaf, self.nvel, self.ncomp)

    def neighbours(self) -> np.ndarray:
        nb = np.zeros((self.nleaf, 2 * self.dim, 1 << (self.dim - 1)), dtype=np.int64)
        self.lib.or_tree_neighbours(self.h, nb.ctypes.data_as(_LL))
        return nb

    def get_f(self) -> np.ndarray:
        f = np.zeros(self.shape())
        self.lib.or_tree_get_f(self.h, _dp(f))
        return f

    def set_f(self, f) -> None:
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.shape()))
        self.lib.or_tree_set_f(self.h, _dp(f))

    def step(self, n: int = 1) -> float:
        r = ctypes.c_double()
        self.lib.or_tree_step(self.h, int(n), ctypes.byref(r))
        return r.value

    def moments(self):
        W = np.zeros((self.nleaf, self.dim + 2))
        q = np.zeros((self.nleaf, self.dim))
        self.lib.or_tree_moments(self.h, _dp(W), _dp(q))
        return W, q

    def cell_types(self) -> np.ndarray:
        t = np.zeros(self.nleaf, dtype=np.uint8)
        self.lib.or_tree_cell_types(self.h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
        return t

    def forces(self):
        F = np.zeros(3)
        Q = ctypes.c_double()
        CD = ctypes.c_double()
        CL = ctypes.c_double()
        self.lib.or_tree_forces(self.h, _dp(F), ctypes.byref(Q), ctypes.byref(CD), ctypes.byref(CL))
        return F, Q.value, CD.value, CL.value

    def finest_case(self) -> "OracleCase":
        """The finest uniform grid under the tree with the finest leaves'
        current values (C29): its links are the tree's, so its ghost band and
        wall quantities are the tree's.  Valid while this tree lives."""
        fine = dict(self.cfg, n=[int(x) << int(self.cfg["tree"]["maxlevel"]) for x in self.cfg["n"][:self.dim]])
        fine.pop("tree", None)
        return OracleCase._view(self.lib, self.lib.or_tree_finest(self.h), fine, self)

    def sizes(self) -> np.ndarray:
        """Edge length of every leaf along each axis."""
        lev = self._lev.astype(np.float64)
        H = [(self.cfg["hi"][a] - self.cfg["lo"][a]) / self.cfg["n"][a] for a in range(self.dim)]
        return np.stack([H[a] * 0.5 ** lev for a in range(self.dim)], axis=1)

    def centres(self) -> np.ndarray:
        hs = self.sizes()
        idx = [self._ix, self._iy] + ([self._iz] if self.dim == 3 else [])
        return np.stack([self.cfg["lo"][a] + (idx[a] + 0.5) * hs[:, a] for a in range(self.dim)], axis=1)
