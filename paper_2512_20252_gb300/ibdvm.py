"""Thin ctypes binding of libibdvm.so (the C-ABI declared in include/ibdvm.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  The binding raises when the library is missing; there is no CPU or
PyTorch fallback.

Case descriptions are plain dicts (see ``workloads``): dim, n, lo, hi, nv, vlo,
vhi, rule, Kn, Ma, Pr, gamma, omega_vhs, alpha_vhs, rho_inf, T_inf, dir, cfl,
dt, precision ("fp64" | "mixed"), cutcell, upwind (1 upwind weights, 2 the
reverse unit vector, 0 plain average, 3 the linear extrapolation without
interpolation of Sec. 3.3.4), ghost_nonneg (1: ghost values below
zero set to zero), body = {kind, center, radii, angle,
verts, accom, Tw, Uw, Lref} and domain_walls (six entries for the faces x-,
x+, y-, y+, z-, z+: None for a freestream face, {Tw, Uw} for a diffuse wall).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libibdvm.so")

OK = 0
STATUS = {0: "OK", 1: "E_INVAL", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_UNSTABLE", 5: "E_NONFINITE",
          6: "E_NOTCONVERGED", 7: "E_TIMEOUT", 8: "E_STATE"}
BODY = {"none": 0, "circle": 1, "ellipse": 2, "sphere": 3, "polygon": 4, "halfspace": 5}
FLUID, GHOST, SOLID = 0, 1, 2
NO_CUTCELL, PLAIN_AVERAGE, RHAT_GHOST_TO_FLUID, GHOST_NONNEG, NAIVE_EXTRAPOLATION = 1, 2, 4, 8, 16


class IbdvmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class TreeDesc(ctypes.Structure):
    _fields_ = [("nleaf", ctypes.c_int), ("maxlevel", ctypes.c_int), ("level", ctypes.POINTER(ctypes.c_int)),
                ("ix", ctypes.POINTER(ctypes.c_int)), ("iy", ctypes.POINTER(ctypes.c_int)),
                ("iz", ctypes.POINTER(ctypes.c_int))]


class VGridDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("rule", ctypes.c_int), ("nodes", ctypes.POINTER(ctypes.c_double) * 3)]


class GasDesc(ctypes.Structure):
    _fields_ = [("Kn", ctypes.c_double), ("Ma", ctypes.c_double), ("Pr", ctypes.c_double),
                ("gamma", ctypes.c_double), ("omega_vhs", ctypes.c_double),
                ("alpha_vhs", ctypes.c_double), ("rho_inf", ctypes.c_double),
                ("T_inf", ctypes.c_double), ("dir", ctypes.c_double * 3), ("cfl", ctypes.c_double),
                ("dt", ctypes.c_double), ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


class BodyDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3),
                ("radii", ctypes.c_double * 3), ("angle", ctypes.c_double),
                ("verts", ctypes.POINTER(ctypes.c_double)), ("nverts", ctypes.c_int),
                ("accom_alpha", ctypes.c_double), ("T_w", ctypes.c_double),
                ("U_w", ctypes.c_double * 3), ("L_ref", ctypes.c_double)]


class DomainDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 6), ("T_w", ctypes.c_double * 6), ("U_w", (ctypes.c_double * 3) * 6)]


def domain_descriptor(walls) -> DomainDesc:
    """The faces x-, x+, y-, y+, z-, z+: None = freestream, {Tw, Uw} = diffuse wall."""
    d = DomainDesc()
    for i, wall in enumerate(walls or []):
        d.T_w[i] = 1.0
        if wall:
            d.kind[i] = 1
            d.T_w[i] = float(wall.get("Tw", 1.0))
            u = list(wall.get("Uw", [0.0, 0.0, 0.0])) + [0.0] * 3
            d.U_w[i][:] = [float(x) for x in u[:3]]
    return d


class ServerDesc(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_steps", ctypes.c_longlong), ("steps_per_round", ctypes.c_int),
                ("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int), ("sequential_fp64", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("done", ctypes.c_int), ("status", ctypes.c_int),
                ("steps", ctypes.c_longlong), ("residual", ctypes.c_double), ("F", ctypes.c_double * 3),
                ("Q", ctypes.c_double), ("CD", ctypes.c_double), ("CL", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t)]


class BatchTiling(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int), ("kpt", ctypes.c_int), ("nitems", ctypes.c_int),
                ("grid", ctypes.c_int), ("graphs", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("ncomp", ctypes.c_int), ("ncell", ctypes.c_longlong),
                ("nfluid", ctypes.c_longlong), ("nvel", ctypes.c_int), ("nvel_padded", ctypes.c_int),
                ("nlink", ctypes.c_int), ("nghost", ctypes.c_int), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("steps_done", ctypes.c_longlong),
                ("device_bytes", ctypes.c_size_t), ("sweep_variant", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_LL = ctypes.POINTER(ctypes.c_longlong)
_U8 = ctypes.POINTER(ctypes.c_ubyte)
_V = ctypes.c_void_p
_S = ctypes.c_int

SIGNATURES = {
    "ibdvm_create_grid": ([ctypes.POINTER(GridDesc), ctypes.POINTER(VGridDesc),
                           ctypes.POINTER(GasDesc), _V, ctypes.POINTER(_V)], _S),
    "ibdvm_create_tree": ([ctypes.POINTER(GridDesc), ctypes.POINTER(TreeDesc), ctypes.POINTER(VGridDesc),
                           ctypes.POINTER(GasDesc), _V, ctypes.POINTER(_V)], _S),
    "ibdvm_tree_neighbours": ([_V, _LL], _S),
    "ibdvm_set_body": ([_V, ctypes.POINTER(BodyDesc)], _S),
    "ibdvm_step": ([_V, ctypes.c_int, _D], _S),
    "ibdvm_moments": ([_V, _D, _D, _U8], _S),
    "ibdvm_forces": ([_V, _D, _D, _D, _D], _S),
    "ibdvm_step_forces": ([_V, _D, _D, _D, _D], _S),
    "ibdvm_set_profiling": ([_V, ctypes.c_int], _S),
    "ibdvm_get_kernel_times": ([_V, _D, _LL], _S),
    "ibdvm_reset_kernel_times": ([_V], _S),
    "ibdvm_get_f": ([_V, _D], _S),
    "ibdvm_set_f": ([_V, _D], _S),
    "ibdvm_get_f_native": ([_V, _V, ctypes.c_size_t], _S),
    "ibdvm_set_f_native": ([_V, _V, ctypes.c_size_t], _S),
    "ibdvm_fp64_fma_rate": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _V], _S),
    "ibdvm_velocity_positions": ([_V, ctypes.POINTER(ctypes.c_int)], _S),
    "ibdvm_ghost_band": ([_V, _D, _D, _D, _D], _S),
    "ibdvm_wall": ([_V, _D], _S),
    "ibdvm_set_domain": ([_V, _V], _S),
    "ibdvm_residual_noalloc": ([_V, _V, _V, ctypes.c_longlong, ctypes.c_int, _V, _V], _S),
    "ibdvm_get_info": ([_V, ctypes.POINTER(Info)], _S),
    "ibdvm_selftest_bounded_wait": ([ctypes.c_int, ctypes.c_int, _D, _V], _S),
    "ibdvm_set_stream": ([_V, _V], _S),
    "ibdvm_get_geom": ([_V], _V),
    "ibdvm_destroy": ([_V], None),
    "ibdvm_last_error": ([_V], ctypes.c_char_p),
    "ibdvm_status_string": ([_S], ctypes.c_char_p),
    "ibdvm_geom_build": ([ctypes.POINTER(GridDesc), ctypes.POINTER(VGridDesc), ctypes.POINTER(GasDesc),
                          ctypes.POINTER(BodyDesc), ctypes.POINTER(_V)], _S),
    "ibdvm_geom_sizes": ([_V, _LL], _S),
    "ibdvm_geom_cells": ([_V, _U8], _S),
    "ibdvm_geom_links": ([_V, _I, _I, _I, _I, _I, _D, _D], _S),
    "ibdvm_geom_cut_table": ([_V, _D], _S),
    "ibdvm_geom_velocities": ([_V, _D, _D], _S),
    "ibdvm_geom_surface": ([_V, _I, _I, _I], _S),
    "ibdvm_geom_dt": ([_V], ctypes.c_double),
    "ibdvm_geom_destroy": ([_V], None),
    "ibdvm_geom_last_error": ([], ctypes.c_char_p),
    "ibdvm_batch_create": ([_V, ctypes.POINTER(_V)], _S),
    "ibdvm_batch_add": ([_V, _V], _S),
    "ibdvm_batch_remove": ([_V, _V], _S),
    "ibdvm_batch_size": ([_V], ctypes.c_int),
    "ibdvm_batch_member": ([_V, ctypes.c_int], _V),
    "ibdvm_batch_step": ([_V, ctypes.c_int, _D, _I], _S),
    "ibdvm_batch_forces": ([_V, _D, _D, _D, _D], _S),
    "ibdvm_batch_set_tiling": ([_V, ctypes.c_int, ctypes.c_int], _S),
    "ibdvm_batch_get_tiling": ([_V, ctypes.POINTER(BatchTiling)], _S),
    "ibdvm_batch_tune": ([_V, ctypes.c_int, _D], _S),
    "ibdvm_batch_set_profiling": ([_V, ctypes.c_int], _S),
    "ibdvm_batch_get_kernel_times": ([_V, _D, _LL], _S),
    "ibdvm_batch_reset_kernel_times": ([_V], _S),
    "ibdvm_batch_destroy": ([_V], None),
    "ibdvm_batch_last_error": ([_V], ctypes.c_char_p),
    "ibdvm_server_create": ([ctypes.POINTER(ServerDesc), ctypes.POINTER(_V)], _S),
    "ibdvm_server_submit": ([_V, ctypes.POINTER(GridDesc), ctypes.POINTER(VGridDesc), ctypes.POINTER(GasDesc),
                             ctypes.POINTER(BodyDesc), _LL], _S),
    "ibdvm_server_poll": ([_V, _I, _I, _I], _S),
    "ibdvm_server_result": ([_V, ctypes.c_longlong, ctypes.POINTER(Result)], _S),
    "ibdvm_server_cancel": ([_V, ctypes.c_longlong], _S),
    "ibdvm_server_clock": ([_V], ctypes.c_double),
    "ibdvm_server_destroy": ([_V], None),
    "ibdvm_server_last_error": ([_V], ctypes.c_char_p),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads libibdvm.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(
                    f"libibdvm.so not found at {p}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def fp64_fma_rate(iters: int = 20000, stream: int | None = None):
    """This GPU's FP64 FMA rate in TFLOP/s and the timed launch in ms
    (ibdvm_fp64_fma_rate)."""
    lib = load()
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib.ibdvm_fp64_fma_rate(int(iters), ctypes.byref(tf), ctypes.byref(ms), _V(stream or 0))
    if st != OK:
        raise IbdvmError(st, "fp64_fma_rate")
    return tf.value, ms.value


def _a3(v, fill=0.0):
    v = list(v) + [fill] * 3
    return v[:3]


def descriptors(case: dict):
    """Marshal a case dict into the four C descriptors (plus owners of arrays)."""
    dim = int(case["dim"])
    g = GridDesc()
    g.dim = dim
    g.n[:] = [int(x) for x in _a3(case["n"], 1)]
    g.lo[:] = _a3(case["lo"])
    g.hi[:] = _a3(case["hi"], 1.0)
    v = VGridDesc()
    v.n[:] = [int(x) for x in _a3(case["nv"], 1)]
    v.lo[:] = _a3(case["vlo"])
    v.hi[:] = _a3(case["vhi"], 1.0)
    v.rule = {"trapezoid": 0, "midpoint": 1, "nodes": 2}[case.get("rule", "trapezoid")]
    node_arrays = []
    if v.rule == 2:
        # explicit velocity nodes per axis: the node counts and the interval follow them
        for a in range(dim):
            nodes = np.ascontiguousarray(np.asarray(case["vnodes"][a], dtype=np.float64))
            node_arrays.append(nodes)
            v.nodes[a] = _dp(nodes)
            v.n[a] = nodes.size
            v.lo[a], v.hi[a] = float(nodes[0]), float(nodes[-1])
    s = GasDesc()
    s.Kn = case["Kn"]
    s.Ma = case["Ma"]
    s.Pr = case.get("Pr", 2.0 / 3.0)
    s.gamma = case.get("gamma", 5.0 / 3.0)
    s.omega_vhs = case.get("omega_vhs", 0.81)
    s.alpha_vhs = case.get("alpha_vhs", 1.0)
    s.rho_inf = case.get("rho_inf", 1.0)
    s.T_inf = case.get("T_inf", 1.0)
    s.dir[:] = _a3(case.get("dir", [1.0, 0.0, 0.0]))
    s.cfl = case.get("cfl", 0.5)
    s.dt = case.get("dt", 0.0)
    s.precision = {"fp64": 0, "mixed": 1}[case.get("precision", "fp64")]
    flags = 0
    if not int(case.get("cutcell", 1)):
        flags |= NO_CUTCELL
    up = int(case.get("upwind", 1))
    if up == 0:
        flags |= PLAIN_AVERAGE
    elif up == 2:
        flags |= RHAT_GHOST_TO_FLUID
    elif up == 3:
        flags |= NAIVE_EXTRAPOLATION
    if int(case.get("ghost_nonneg", 0)):
        flags |= GHOST_NONNEG
    s.flags = flags
    body = case.get("body") or {"kind": "none"}
    b = BodyDesc()
    b.kind = BODY[body["kind"]]
    b.center[:] = _a3(body.get("center", [0.0, 0.0, 0.0]))
    b.radii[:] = _a3(body.get("radii", [0.0, 0.0, 0.0]))
    b.angle = body.get("angle", 0.0)
    keep = None
    if body["kind"] == "polygon":
        keep = np.ascontiguousarray(np.asarray(body["verts"], dtype=np.float64).reshape(-1))
        b.verts = keep.ctypes.data_as(_D)
        b.nverts = keep.size // 2
    b.accom_alpha = body.get("accom", 1.0)
    b.T_w = body.get("Tw", 1.0)
    b.U_w[:] = _a3(body.get("Uw", [0.0, 0.0, 0.0]))
    b.L_ref = body.get("Lref", 0.0)
    return g, v, s, b, (keep, node_arrays)


def _dp(a):
    return a.ctypes.data_as(_D)


def selftest_bounded_wait(deliver: bool, spin_limit: int, stream: int | None = None):
    """Runs the bounded mbarrier wait of the TMA sweeps on a barrier whose
    bytes are delivered or never delivered; returns (status, seconds)."""
    lib = load()
    sec = ctypes.c_double(0.0)
    st = lib.ibdvm_selftest_bounded_wait(1 if deliver else 0, int(spin_limit), ctypes.byref(sec), _V(stream or 0))
    return st, sec.value


def residual_noalloc(W_old_ptr: int, W_new_ptr: int, celltype_ptr: int | None, ncell: int, dim: int,
                     out_ptr: int, stream: int | None = None) -> int:
    """Residual of two device fields [ncell][dim+2] into a caller-owned device
    double, without any device allocation (see include/ibdvm.h).  Returns the
    status; raises IbdvmError on failure."""
    lib = load()
    st = lib.ibdvm_residual_noalloc(_V(W_old_ptr), _V(W_new_ptr), _V(celltype_ptr or 0), int(ncell),
                                    int(dim), _V(out_ptr), _V(stream or 0))
    if st != OK:
        raise IbdvmError(st, lib.ibdvm_last_error(None).decode())
    return st


class Geometry:
    """Host-only geometry of a case (classification, links, cut table); no GPU."""

    def __init__(self, case: dict):
        self.lib = load()
        g, v, s, b, self._keep = descriptors(case)
        h = _V()
        st = self.lib.ibdvm_geom_build(ctypes.byref(g), ctypes.byref(v), ctypes.byref(s),
                                       ctypes.byref(b), ctypes.byref(h))
        if st != OK:
            raise IbdvmError(st, self.lib.ibdvm_geom_last_error().decode())
        self.h = h
        self._owned = True
        self._read_sizes()

    @classmethod
    def _borrow(cls, lib, handle):
        self = cls.__new__(cls)
        self.lib = lib
        self.h = _V(handle)
        self._owned = False
        self._read_sizes()
        return self

    def _read_sizes(self):
        sz = np.zeros(8, dtype=np.int64)
        self.lib.ibdvm_geom_sizes(self.h, sz.ctypes.data_as(_LL))
        (self.ncell, self.nvel, self.ncomp, self.nlink, self.nghost, self.nfluid, self.nsurf,
         self.nvel_padded) = (int(x) for x in sz)

    def __del__(self):
        if getattr(self, "_owned", False) and getattr(self, "h", None):
            self.lib.ibdvm_geom_destroy(self.h)
            self.h = None

    @property
    def dt(self):
        return float(self.lib.ibdvm_geom_dt(self.h))

    def cell_types(self):
        t = np.zeros(self.ncell, dtype=np.uint8)
        self.lib.ibdvm_geom_cells(self.h, t.ctypes.data_as(_U8))
        return t

    def links(self):
        n = self.nlink
        ints = [np.zeros(n, dtype=np.int32) for _ in range(5)]
        xw = np.zeros((n, 3))
        nw = np.zeros((n, 3))
        self.lib.ibdvm_geom_links(self.h, *[a.ctypes.data_as(_I) for a in ints], _dp(xw), _dp(nw))
        out = dict(zip(["ghost", "donor", "aux", "axis", "side"], ints))
        out["xw"] = xw
        out["nw"] = nw
        return out

    def cut_table(self):
        wg = np.zeros((self.nlink, self.nvel))
        self.lib.ibdvm_geom_cut_table(self.h, _dp(wg))
        return wg

    def velocities(self):
        xi = np.zeros((self.nvel, 3))
        w = np.zeros(self.nvel)
        self.lib.ibdvm_geom_velocities(self.h, _dp(xi), _dp(w))
        return xi, w

    def surface_cells(self):
        g = np.zeros(self.nghost, dtype=np.int32)
        off = np.zeros(self.nghost + 1, dtype=np.int32)
        cells = np.zeros(max(self.nsurf, 1), dtype=np.int32)
        self.lib.ibdvm_geom_surface(self.h, g.ctypes.data_as(_I), off.ctypes.data_as(_I),
                                    cells.ctypes.data_as(_I))
        return g, off, cells[: self.nsurf]


class Solver:
    """One solver context on the current CUDA device (C-ABI handle)."""

    def __init__(self, case: dict, stream: int | None = None):
        self.lib = load()
        self.case = dict(case)
        g, v, s, b, keep = descriptors(case)
        h = _V()
        tree = case.get("tree")
        if tree:
            # a tree-refined 2D grid over the root grid case["n"] (ibdvm_create_tree)
            keys = ("level", "ix", "iy", "iz") if int(case["dim"]) == 3 else ("level", "ix", "iy")
            arrs = [np.ascontiguousarray(np.asarray(tree[k], dtype=np.int32)) for k in keys]
            keep = list(keep) + arrs
            t = TreeDesc()
            t.nleaf = arrs[0].size
            t.maxlevel = int(tree["maxlevel"])
            ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for a in arrs]
            t.level, t.ix, t.iy = ptrs[:3]
            t.iz = ptrs[3] if len(ptrs) > 3 else None
            st = self.lib.ibdvm_create_tree(ctypes.byref(g), ctypes.byref(t), ctypes.byref(v), ctypes.byref(s),
                                            _V(stream or 0), ctypes.byref(h))
        else:
            st = self.lib.ibdvm_create_grid(ctypes.byref(g), ctypes.byref(v), ctypes.byref(s),
                                            _V(stream or 0), ctypes.byref(h))
        if st != OK:
            raise IbdvmError(st, self.lib.ibdvm_last_error(None).decode())
        self.h = h
        body = case.get("body") or {"kind": "none"}
        if body["kind"] != "none":
            self._check(self.lib.ibdvm_set_body(self.h, ctypes.byref(b)))
        if any(case.get("domain_walls") or []):
            self.set_domain(case["domain_walls"])
        self._keep = keep
        self.refresh_info()

    def tree_neighbours(self) -> np.ndarray:
        """Face neighbours [leaf][side 2a + (s > 0)][2^(dim-1)] of a tree context (-1: none)."""
        D = int(self.case["dim"])
        nb = np.zeros((self.ncell, 2 * D, 1 << (D - 1)), dtype=np.int64)
        self._check(self.lib.ibdvm_tree_neighbours(self.h, nb.ctypes.data_as(_LL)))
        return nb

    def set_domain(self, walls):
        """Domain faces x-, x+, y-, y+, z-, z+: None = freestream halo,
        {"Tw": T, "Uw": [u, v, w]} = diffuse wall (ibdvm_set_domain)."""
        d = domain_descriptor(walls)
        self._check(self.lib.ibdvm_set_domain(self.h, ctypes.byref(d)))
        self.case["domain_walls"] = list(walls)

    def _check(self, st):
        if st != OK:
            raise IbdvmError(st, self.lib.ibdvm_last_error(self.h).decode())
        return st

    def refresh_info(self):
        info = Info()
        self._check(self.lib.ibdvm_get_info(self.h, ctypes.byref(info)))
        self.info = info
        self.dim, self.ncomp = info.dim, info.ncomp
        self.ncell, self.nvel, self.nvel_padded = info.ncell, info.nvel, info.nvel_padded
        self.nlink, self.nghost, self.dt = info.nlink, info.nghost, info.dt
        self.precision = "fp64" if info.precision == 0 else "mixed"
        return info

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibdvm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_body(self, body: dict):
        c = dict(self.case)
        c["body"] = body
        _, _, _, b, keep = descriptors(c)
        self._check(self.lib.ibdvm_set_body(self.h, ctypes.byref(b)))
        self._keep = keep
        self.case = c
        self.refresh_info()

    def set_stream(self, stream: int | None):
        self._check(self.lib.ibdvm_set_stream(self.h, _V(stream or 0)))

    def step(self, nsteps: int = 1) -> float:
        r = ctypes.c_double(0.0)
        self._check(self.lib.ibdvm_step(self.h, int(nsteps), ctypes.byref(r)))
        return r.value

    def moments(self, W=None, q=None, with_types=True):
        """W^n [ncell][D + 2], q^n [ncell][D] and the cell types.  W and q may
        be caller-owned C-contiguous float64 arrays of those shapes, filled in
        place (in pinned host memory the read is one direct copy per array);
        with_types=False skips the cell types (None is returned for them)."""
        W = self._out(W, (self.ncell, self.dim + 2), "W")
        q = self._out(q, (self.ncell, self.dim), "q")
        t = np.zeros(self.ncell, dtype=np.uint8) if with_types else None
        self._check(self.lib.ibdvm_moments(self.h, _dp(W), _dp(q),
                                           t.ctypes.data_as(_U8) if with_types else None))
        return W, q, t

    @staticmethod
    def _out(a, shape, name):
        if a is None:
            return np.zeros(shape)
        if a.dtype != np.float64 or tuple(a.shape) != shape or not a.flags["C_CONTIGUOUS"] \
                or not a.flags["WRITEABLE"]:
            raise ValueError(f"{name} must be a writeable C-contiguous float64 array of shape {shape}")
        return a

    def forces(self):
        F = np.zeros(3)
        Q, CD, CL = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.ibdvm_forces(self.h, _dp(F), ctypes.byref(Q), ctypes.byref(CD),
                                          ctypes.byref(CL)))
        return F, Q.value, CD.value, CL.value

    def step_forces(self):
        F = np.zeros(3)
        Q, CD, CL = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.ibdvm_step_forces(self.h, _dp(F), ctypes.byref(Q), ctypes.byref(CD),
                                               ctypes.byref(CL)))
        return F, Q.value, CD.value, CL.value

    KERNEL_CLASSES = ("ghost_band", "sweep", "moments", "forces")

    def set_profiling(self, on: bool = True):
        self._check(self.lib.ibdvm_set_profiling(self.h, 1 if on else 0))

    def kernel_times(self):
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        self._check(self.lib.ibdvm_get_kernel_times(self.h, _dp(ms), n.ctypes.data_as(_LL)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNEL_CLASSES)}

    def reset_kernel_times(self):
        self._check(self.lib.ibdvm_reset_kernel_times(self.h))

    def shape(self):
        return (self.ncell, self.nvel, self.ncomp)

    def get_f(self) -> np.ndarray:
        f = np.zeros(self.shape())
        self._check(self.lib.ibdvm_get_f(self.h, _dp(f)))
        return f

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(self.shape())
        self._check(self.lib.ibdvm_set_f(self.h, _dp(f)))

    def native_shape(self):
        return (self.ncell, self.nvel_padded, self.ncomp)

    def velocity_positions(self) -> np.ndarray:
        """Index along the velocity axis of the native layout of every velocity
        in its natural order (ibdvm_velocity_positions)."""
        pos = np.zeros(self.nvel, dtype=np.int32)
        self._check(self.lib.ibdvm_velocity_positions(self.h, pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return pos

    def native_dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32

    def get_f_native(self, out_ptr: int, nbytes: int):
        self._check(self.lib.ibdvm_get_f_native(self.h, _V(out_ptr), ctypes.c_size_t(nbytes)))

    def set_f_native(self, in_ptr: int, nbytes: int):
        self._check(self.lib.ibdvm_set_f_native(self.h, _V(in_ptr), ctypes.c_size_t(nbytes)))

    def ghost_band(self):
        shp = (self.nlink, self.nvel, self.ncomp)
        out = {k: np.zeros(shp) for k in ("fiw", "fstarw", "fstargc")}
        rhow = np.zeros(max(self.nlink, 1))
        self._check(self.lib.ibdvm_ghost_band(self.h, _dp(out["fiw"]), _dp(out["fstarw"]),
                                              _dp(out["fstargc"]), _dp(rhow)))
        out["rhow"] = rhow[: self.nlink]
        return out

    WALL_COLUMNS = ("rho", "slip_x", "slip_y", "slip_z", "T", "T_jump", "p", "tau_x", "tau_y", "tau_z",
                    "q_n", "Cp")

    def wall(self) -> np.ndarray:
        """Wall-point quantities per link ([nlink][12], columns WALL_COLUMNS):
        density, slip velocity, temperature and its jump, normal and
        tangential stress, normal heat flux and C_p from the moments of the
        wall distribution at each link's intersect point (geometry().links()
        gives the points and normals)."""
        out = np.zeros((max(self.nlink, 1), len(self.WALL_COLUMNS)))
        self._check(self.lib.ibdvm_wall(self.h, _dp(out)))
        return out[: self.nlink]

    def geometry(self) -> Geometry:
        return Geometry._borrow(self.lib, self.lib.ibdvm_get_geom(self.h))


class Batch:
    """A batch of 2D FP32 solvers advanced by grouped launches (C-ABI handle).

    Holds references to its member Solvers; members join and leave between
    steps (continuous batching)."""

    KERNEL_CLASSES = Solver.KERNEL_CLASSES

    def __init__(self, stream: int | None = None):
        self.lib = load()
        h = _V()
        st = self.lib.ibdvm_batch_create(_V(stream or 0), ctypes.byref(h))
        if st != OK:
            raise IbdvmError(st, "ibdvm_batch_create failed")
        self.h = h
        self.members: list[Solver] = []

    def _check(self, st):
        if st != OK:
            raise IbdvmError(st, self.lib.ibdvm_batch_last_error(self.h).decode())
        return st

    def add(self, solver: Solver):
        self._check(self.lib.ibdvm_batch_add(self.h, solver.h))
        self.members.append(solver)

    def remove(self, solver: Solver):
        self._check(self.lib.ibdvm_batch_remove(self.h, solver.h))
        self.members = [m for m in self.members if m is not solver]

    def __len__(self):
        return len(self.members)

    def step(self, nsteps: int = 1, check: bool = True):
        """Advances every member; returns (residuals, statuses) per member."""
        n = len(self.members)
        res = np.zeros(max(n, 1))
        sts = np.zeros(max(n, 1), dtype=np.int32)
        st = self.lib.ibdvm_batch_step(self.h, int(nsteps), _dp(res), sts.ctypes.data_as(_I))
        if check:
            self._check(st)
        return res[:n], sts[:n]

    def forces(self):
        n = max(len(self.members), 1)
        F, Q, CD, CL = np.zeros((n, 3)), np.zeros(n), np.zeros(n), np.zeros(n)
        self._check(self.lib.ibdvm_batch_forces(self.h, _dp(F), _dp(Q), _dp(CD), _dp(CL)))
        m = len(self.members)
        return F[:m], Q[:m], CD[:m], CL[:m]

    def set_tiling(self, rows: int = 0, kpt: int = 0):
        self._check(self.lib.ibdvm_batch_set_tiling(self.h, int(rows), int(kpt)))

    def tiling(self):
        t = BatchTiling()
        self._check(self.lib.ibdvm_batch_get_tiling(self.h, ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in BatchTiling._fields_}

    def tune(self, steps_per_trial: int = 4) -> float:
        best = ctypes.c_double(0.0)
        self._check(self.lib.ibdvm_batch_tune(self.h, int(steps_per_trial), ctypes.byref(best)))
        return best.value

    def set_profiling(self, on: bool = True):
        self._check(self.lib.ibdvm_batch_set_profiling(self.h, 1 if on else 0))

    def kernel_times(self):
        ms = np.zeros(8)
        n = np.zeros(8, dtype=np.int64)
        self._check(self.lib.ibdvm_batch_get_kernel_times(self.h, _dp(ms), n.ctypes.data_as(_LL)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.KERNEL_CLASSES)}

    def reset_kernel_times(self):
        self._check(self.lib.ibdvm_batch_reset_kernel_times(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibdvm_batch_destroy(self.h)
            self.h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop (C-ABI handle): requests are queued, admitted by HBM
    budget into a 2D and a 3D batch, advanced a round per poll and retired
    when converged, failed or capped.  sequential_fp64=True is the plain form:
    one request at a time in the FP64 path."""

    def __init__(self, tol=1e-6, max_steps=20000, steps_per_round=50, hbm_budget=0, max_active=0,
                 sequential_fp64=False):
        self.lib = load()
        d = ServerDesc(float(tol), int(max_steps), int(steps_per_round), int(hbm_budget), int(max_active),
                       1 if sequential_fp64 else 0)
        h = _V()
        st = self.lib.ibdvm_server_create(ctypes.byref(d), ctypes.byref(h))
        if st != OK:
            raise IbdvmError(st, "ibdvm_server_create failed")
        self.h = h

    def _check(self, st):
        if st != OK:
            raise IbdvmError(st, self.lib.ibdvm_server_last_error(self.h).decode())
        return st

    def submit(self, case: dict) -> int:
        g, v, s, b, keep = descriptors(case)
        body = case.get("body") or {"kind": "none"}
        rid = ctypes.c_longlong(-1)
        self._check(self.lib.ibdvm_server_submit(self.h, ctypes.byref(g), ctypes.byref(v), ctypes.byref(s),
                                                 ctypes.byref(b) if body["kind"] != "none" else None,
                                                 ctypes.byref(rid)))
        return rid.value

    def poll(self):
        a, q, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.ibdvm_server_poll(self.h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(f)))
        return a.value, q.value, f.value

    def cancel(self, rid: int):
        self._check(self.lib.ibdvm_server_cancel(self.h, int(rid)))

    def result(self, rid: int) -> dict:
        r = Result()
        self._check(self.lib.ibdvm_server_result(self.h, int(rid), ctypes.byref(r)))
        d = {k: getattr(r, k) for k, _ in Result._fields_}
        d["F"] = list(r.F)
        return d

    def clock(self) -> float:
        return self.lib.ibdvm_server_clock(self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.ibdvm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
