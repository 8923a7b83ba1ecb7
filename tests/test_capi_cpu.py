"""C-ABI library checks that need no GPU: the library loads, exports every
function that include/ibdvm.h declares, and its host-only geometry agrees with
the oracle's independent geometry."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2512_20252_gb300 import build as libbuild
from paper_2512_20252_gb300 import ibdvm
from paper_2512_20252_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ibdvm.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ibdvm_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(ibdvm.SIGNATURES), set(names) - set(ibdvm.SIGNATURES)


def test_status_strings(lib):
    assert lib.ibdvm_status_string(0) == b"ok"
    assert lib.ibdvm_status_string(4) == b"unstable time step"


def _cases():
    out = {
        "circle48": wl.cylinder_48(),
        "ellipse": wl.small_2d("ellipse", n=32, nv=10),
        "naca": wl.small_2d("naca", n=48, nv=8),
        "circle_midpoint": wl.small_2d("circle", n=20, nv=9, rule="midpoint"),
        "nocut": wl.small_2d("circle", n=20, nv=10, cutcell=0),
        "sphere": wl.sphere_24(),
        "halfspace3d": wl._case(3, 10, 1.0, 6, 4.0, 0.1, 0.3,
                                {"kind": "halfspace", "center": [0.05, 0.02, 0.0],
                                 "radii": [0.6, 0.48, 0.64], "accom": 0.7, "Tw": 1.2}),
        "naca_aoa": wl._case(2, 96, 2.0, 6, 4.0, 0.1, 0.5, wl.naca0012(2.0, 8.0, 80)),
        # non-uniform (stretched) velocity grids
        "stretched2d": wl.stretched(wl._case(2, 24, 2.0, 16, 5.0, 0.1, 0.4, wl.circle(0.6)), 0.3),
        "stretched3d": wl.stretched(wl._case(3, 10, 2.0, 10, 4.5, 0.1, 0.3, wl.sphere(0.7)), 0.4),
    }
    return out


@pytest.mark.parametrize("name", list(_cases()))
def test_geometry_matches_oracle(lib, name):
    case = _cases()[name]
    g = ibdvm.Geometry(case)
    o = oracle.OracleCase(case)
    assert (g.ncell, g.nvel, g.ncomp, g.nlink, g.nghost, g.nfluid) == (
        o.ncell, o.nvel, o.ncomp, o.nlink, o.nghost, o.nfluid)
    np.testing.assert_array_equal(g.cell_types(), o.cell_types())
    xg, wg_ = g.velocities()
    xo, wo = o.velocities()
    np.testing.assert_array_equal(xg, xo)
    np.testing.assert_allclose(wg_, wo, rtol=1e-15)
    assert g.dt == pytest.approx(o.dt, rel=1e-15)
    Lg, Lo = g.links(), o.links()
    for k in ("ghost", "donor", "aux", "axis", "side"):
        np.testing.assert_array_equal(Lg[k], Lo[k], err_msg=k)
    np.testing.assert_allclose(Lg["xw"], Lo["xw"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(Lg["nw"], Lo["nw"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(g.cut_table(), o.cut_table(), rtol=0, atol=1e-14 * wo.max())
    gg, go_, gc = g.surface_cells()
    og, oo, oc = o.surface_cells()
    np.testing.assert_array_equal(gg, og)
    np.testing.assert_array_equal(go_, oo)
    np.testing.assert_array_equal(gc, oc)


def test_geometry_rejects_bad_velocity_nodes(lib):
    base = wl.stretched(wl.small_2d("circle"), 0.4)
    for nodes in ([0.0, 1.0, 1.0, 2.0], [0.0, float("nan"), 1.0, 2.0], [2.0, 1.0, 0.0, -1.0]):
        bad = dict(base, vnodes=[nodes, base["vnodes"][1]])
        with pytest.raises(ibdvm.IbdvmError) as e:
            ibdvm.Geometry(bad)
        assert e.value.status == 1


def test_geometry_rejects_bad_input(lib):
    bad = wl.small_2d("circle")
    bad["n"] = [2, 2]
    with pytest.raises(ibdvm.IbdvmError) as e:
        ibdvm.Geometry(bad)
    assert e.value.status == 1
    bad = wl.small_2d("circle")
    bad["body"]["accom"] = 1.5
    with pytest.raises(ibdvm.IbdvmError):
        ibdvm.Geometry(bad)
    bad = wl.small_2d("circle")
    bad["body"] = wl.sphere(0.3)
    with pytest.raises(ibdvm.IbdvmError):
        ibdvm.Geometry(bad)


def test_product_cut_measures_closed_forms(lib):
    """The product's cut-cell measures (through the geometry of a half-space
    wall) against the oracle's independent clipping on every velocity box."""
    for nrm in ([0.6, 0.8, 0.0], [1.0, 0.0, 0.0], [0.28, -0.96, 0.0]):
        case = wl._case(2, 8, 1.0, 13, 4.0, 0.1, 0.0,
                        {"kind": "halfspace", "center": [0.031, 0.0, 0.0], "radii": nrm, "Tw": 1.0})
        g = ibdvm.Geometry(case)
        o = oracle.OracleCase(case)
        np.testing.assert_allclose(g.cut_table(), o.cut_table(), rtol=0, atol=1e-14)


def test_caller_owned_moment_outputs_are_checked():
    """Solver.moments fills caller-owned arrays only when they are writeable,
    C-contiguous float64 arrays of the right shape (checked before any call)."""
    ok = np.zeros((10, 4))
    assert ibdvm.Solver._out(ok, (10, 4), "W") is ok
    assert ibdvm.Solver._out(None, (10, 2), "q").shape == (10, 2)
    for bad in (np.zeros((10, 3)), np.zeros((10, 4), dtype=np.float32), np.zeros((4, 10)).T):
        with pytest.raises(ValueError):
            ibdvm.Solver._out(bad, (10, 4), "W")
    ro = np.zeros((10, 4))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        ibdvm.Solver._out(ro, (10, 4), "W")
