"""GPU path (through the C-ABI) against the CPU oracle, element by element.

Tolerances: the FP64 path must match the oracle within 1e-11 relative on f and
W (max |difference| over fluid cells divided by the largest |value|); the
mixed path (FP32 storage and transport) within 1e-5 on W and 1e-4 on C_D.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2512_20252_gb300 import ibdvm
from paper_2512_20252_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-11


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


def compare(g, o, tol=TOL, wtol=None, forces=True, q=True):
    t = o.cell_types()
    fl = t == oracle.FLUID
    fe = rel_err(g.get_f()[fl], o.get_f()[fl])
    Wg, qg, tg = g.moments()
    Wo, qo = o.moments()
    np.testing.assert_array_equal(tg, t)
    we = max(rel_err(Wg[fl, i], Wo[fl, i]) for i in range(Wo.shape[1]) if np.abs(Wo[fl, i]).max() > 1e-9)
    assert fe < tol, fe
    assert we < (wtol or tol), we
    if q:
        qe = float(np.abs(qg[fl] - qo[fl]).max() / max(np.abs(qo[fl]).max(), 1e-3))
        assert qe < 1e3 * (wtol or tol), qe
    if forces and o.nlink:
        Fg, Qg, CDg, CLg = g.forces()
        Fo, Qo, CDo, CLo = o.forces()
        scale = np.abs(Fo).max()
        assert np.abs(Fg - Fo).max() < 10 * (wtol or tol) * scale, (Fg, Fo)
        assert abs(Qg - Qo) < 10 * (wtol or tol) * max(abs(Qo), 1e-6), (Qg, Qo)
        assert abs(CDg - CDo) < 10 * (wtol or tol) * max(abs(CDo), 1e-6), (CDg, CDo)
    return fe, we


def pair(case, steps, f0=None):
    g = ibdvm.Solver(case)
    o = oracle.OracleCase(case)
    if f0 is not None:
        o.set_f(f0)
        g.set_f(f0)
    rg = g.step(steps)
    ro = o.step(steps)
    return g, o, rg, ro


def perturbed(o, seed, amp=0.3):
    rng = np.random.default_rng(seed)
    return o.get_f() * (1.0 + amp * rng.uniform(-1.0, 1.0, size=o.shape()))


def test_cylinder_48_fp64_parity():
    """2D cylinder, 48^2 cells, 24^2 trapezoid velocities, Kn 0.1, Ma 0.3."""
    case = wl.cylinder_48()
    g, o, rg, ro = pair(case, 10)
    compare(g, o)
    assert rg == pytest.approx(ro, rel=1e-9)
    g.close()


@pytest.mark.parametrize("body", ["circle", "ellipse", "naca"])
def test_perturbed_state_parity(body):
    case = wl.small_2d(body, n=40 if body == "naca" else 24, nv=11, Kn=0.05, Ma=0.4)
    o0 = oracle.OracleCase(case)
    f0 = perturbed(o0, 11)
    g, o, rg, ro = pair(case, 4, f0)
    compare(g, o)
    assert rg == pytest.approx(ro, rel=1e-9)


@pytest.mark.parametrize("variant", ["midpoint", "nocut", "plain_average", "rhat_reverse", "naive",
                                     "accom_0.6", "hot_moving_wall", "bgk", "odd_grid", "naive_3d"])
def test_method_variants_parity(variant):
    case = wl.small_2d("ellipse", n=24, nv=10, Kn=0.08, Ma=0.5)
    if variant == "midpoint":
        case["rule"] = "midpoint"
    elif variant == "nocut":
        case["cutcell"] = 0
    elif variant == "plain_average":
        case["upwind"] = 0
    elif variant == "rhat_reverse":
        case["upwind"] = 2
    elif variant == "naive":
        case["upwind"] = 3  # no interpolation: 2 f_d - f_ac (Sec. 3.3.4)
    elif variant == "naive_3d":
        case = wl._case(3, 10, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6), upwind=3)
    elif variant == "accom_0.6":
        case["body"]["accom"] = 0.6
    elif variant == "hot_moving_wall":
        case["body"]["Tw"] = 1.4
        case["body"]["Uw"] = [0.1, -0.05, 0.0]
    elif variant == "bgk":
        case["Pr"] = 1.0
    elif variant == "odd_grid":
        case["n"] = [27, 19]
        case["nv"] = [13, 9]
        case["hi"] = [2.0, 1.6]
        case["lo"] = [-2.2, -1.6]
    o0 = oracle.OracleCase(case)
    g, o, rg, ro = pair(case, 3, perturbed(o0, 5, 0.2))
    compare(g, o)


def test_ghost_band_parity():
    case = wl.small_2d("naca", n=40, nv=12, Ma=0.6)
    case["body"]["accom"] = 0.7
    o = oracle.OracleCase(case)
    f0 = perturbed(o, 9, 0.25)
    o.set_f(f0)
    g = ibdvm.Solver(case)
    g.set_f(f0)
    gb, ob = g.ghost_band(), o.ghost_band()
    for k in ("fiw", "fstarw", "fstargc"):
        assert rel_err(gb[k], ob[k]) < TOL, k
    np.testing.assert_allclose(gb["rhow"], ob["rhow"], rtol=1e-12)


def test_sphere_3d_parity():
    case = wl._case(3, 14, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6))
    o0 = oracle.OracleCase(case)
    g, o, rg, ro = pair(case, 3, perturbed(o0, 3, 0.2))
    compare(g, o)
    assert rg == pytest.approx(ro, rel=1e-9)


@pytest.mark.slow
def test_sphere_24_downscale_parity():
    """The 3D sphere case downscaled to 24^3 cells and 12^3 velocities."""
    case = wl.sphere_24()
    g, o, rg, ro = pair(case, 2)
    compare(g, o)


def test_halfspace_3d_wall_at_domain_edge():
    body = {"kind": "halfspace", "center": [-0.45, 0.0, 0.0], "radii": [0.8, 0.6, 0.0],
            "accom": 0.5, "Tw": 1.2}
    case = wl._case(3, 10, 1.0, 6, 4.0, 0.1, 0.3, body)
    o0 = oracle.OracleCase(case)
    g, o, _, _ = pair(case, 2, perturbed(o0, 4, 0.1))
    compare(g, o)


def test_no_body_and_tiny_grid():
    case = wl._case(2, 4, 1.0, 2, 3.0, 0.2, 0.2, {"kind": "none"})
    o0 = oracle.OracleCase(case)
    g, o, _, _ = pair(case, 3, perturbed(o0, 2, 0.2))
    compare(g, o, forces=False)


def test_mixed_precision_against_fp64_oracle():
    case = wl.cylinder_48()
    case["precision"] = "mixed"
    g, o, rg, ro = pair(case, 10)
    t = o.cell_types()
    fl = t == oracle.FLUID
    Wg, _, _ = g.moments()
    Wo, _ = o.moments()
    for i in range(4):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    CDg = g.forces()[2]
    CDo = o.forces()[2]
    assert abs(CDg - CDo) < 1e-4 * abs(CDo)
    assert rg == pytest.approx(ro, rel=1e-3)


@pytest.mark.parametrize("Kn", [0.01, 1.0])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_knudsen_sweep_against_the_oracle(Kn, precision):
    """The Knudsen numbers of the 512^2 cylinder sweep other than 0.1 (Sec. 4:
    tau = mu / p with the VHS viscosity mu0 T^omega, mu0 proportional to Kn) on a
    small cylinder with the sweep's velocity box and Ma, 20 steps.  Kn 0.01 is
    the stiffest relaxation (dt / tau about 0.09 here); Kn 1 nearly free
    transport.  FP64 at 1e-11 on f and W; the mixed path at 1e-5 on W and 1e-4
    on C_D."""
    case = wl._case(2, 40, 4.0, 16, 6.0, Kn, 0.5, wl.circle(0.5), precision=precision)
    g, o, rg, ro = pair(case, 20)
    if precision == "fp64":
        compare(g, o)
        assert rg == pytest.approx(ro, rel=1e-9)
        return
    fl = o.cell_types() == oracle.FLUID
    Wg, _, _ = g.moments()
    Wo, _ = o.moments()
    for i in range(4):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    CDg, CDo = g.forces()[2], o.forces()[2]
    assert abs(CDg - CDo) < 1e-4 * abs(CDo)
    assert rg == pytest.approx(ro, rel=1e-3)


def test_state_roundtrip_and_errors():
    case = wl.small_2d("circle", n=12, nv=6)
    g = ibdvm.Solver(case)
    o = oracle.OracleCase(case)
    f0 = perturbed(o, 1)
    g.set_f(f0)
    np.testing.assert_array_equal(g.get_f(), f0)
    with pytest.raises(ibdvm.IbdvmError) as e:
        g.step(-1)
    assert e.value.status == 1
    # dt far beyond the relaxation time: forward Euler relaxation is refused
    bad = dict(case)
    bad["dt"] = 5.0
    with pytest.raises(ibdvm.IbdvmError) as e:
        ibdvm.Solver(bad)
    assert e.value.status == 4


def test_native_state_transfer():
    torch = pytest.importorskip("torch")
    case = wl.small_2d("circle", n=16, nv=8, precision="mixed")
    g = ibdvm.Solver(case)
    shp = g.native_shape()
    buf = torch.empty(shp, dtype=torch.float32, pin_memory=True)
    g.get_f_native(buf.data_ptr(), buf.numel() * 4)
    f = g.get_f()
    pos = g.velocity_positions()
    np.testing.assert_allclose(buf.numpy()[:, pos], f, rtol=1e-7)
    buf.mul_(1.01)
    g.set_f_native(buf.data_ptr(), buf.numel() * 4)
    np.testing.assert_allclose(g.get_f(), buf.numpy()[:, pos].astype(np.float64), rtol=1e-7)
    # the moments into caller-owned pinned arrays equal those into fresh ones
    W, q, t = g.moments()
    Wp = torch.empty(W.shape, dtype=torch.float64, pin_memory=True).numpy()
    qp = torch.empty(q.shape, dtype=torch.float64, pin_memory=True).numpy()
    W2, q2, t2 = g.moments(Wp, qp, with_types=False)
    assert W2 is Wp and q2 is qp and t2 is None
    np.testing.assert_array_equal(Wp, W)
    np.testing.assert_array_equal(qp, q)


@pytest.mark.parametrize("kind", ["2d_mixed", "3d_mixed", "2d_fp64"])
def test_pipelined_state_upload(kind):
    """A state of 64 MiB or more is uploaded in cell ranges, the moments of each
    range taken as soon as its bytes arrive: W and q equal those of the
    one-copy path (ibdvm_set_f, the same kernels over all cells at once) and
    the oracle's moments of the same f."""
    torch = pytest.importorskip("torch")
    if kind == "2d_mixed":
        case = wl.small_2d("circle", n=128, nv=32, precision="mixed")
    elif kind == "2d_fp64":
        case = wl.small_2d("ellipse", n=96, nv=32)
    else:
        case = wl._case(3, 36, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6), precision="mixed")
    g = ibdvm.Solver(case)
    g.step(3)
    esize = 4 if g.precision == "mixed" else 8
    buf = torch.empty(g.native_shape(), dtype=torch.float32 if esize == 4 else torch.float64, pin_memory=True)
    assert buf.numel() * esize >= 64 << 20
    g.get_f_native(buf.data_ptr(), buf.numel() * esize)
    rng = np.random.default_rng(7)
    scale = torch.from_numpy(1.0 + 0.02 * rng.random(buf.shape[0])).to(buf.dtype)
    buf.mul_(scale[:, None, None])
    g.set_f_native(buf.data_ptr(), buf.numel() * esize)
    W1, q1, t = g.moments()
    f = buf.numpy()[:, g.velocity_positions()].astype(np.float64)
    g.set_f(f)
    W2, q2, _ = g.moments()
    np.testing.assert_array_equal(W1, W2)
    np.testing.assert_array_equal(q1, q2)
    o = oracle.OracleCase(case)
    o.set_f(f)
    Wo, qo = o.moments()
    fl = t == ibdvm.FLUID
    tol = TOL if esize == 8 else 1e-5
    for i in range(g.dim + 2):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(W1[fl, i], Wo[fl, i]) < tol, i
    qe = float(np.abs(q1[fl] - qo[fl]).max() / max(np.abs(qo[fl]).max(), 1e-3))
    assert qe < 1e3 * tol, qe


WALL = {k: i for i, k in enumerate(ibdvm.Solver.WALL_COLUMNS)}


def _no_flow_through_the_wall(wq, nw):
    """The wall density balance leaves no mass flux through any wall point:
    the gas velocity there is tangential, as is the tangential stress."""
    slip = wq[:, WALL["slip_x"]:WALL["slip_z"] + 1]
    tau = wq[:, WALL["tau_x"]:WALL["tau_z"] + 1]
    assert np.all(wq[:, WALL["rho"]] > 0) and np.all(wq[:, WALL["T"]] > 0)
    assert np.abs(np.sum(slip * nw, axis=1)).max() < 1e-10 * max(np.abs(slip).max(), 1e-3)
    assert np.abs(np.sum(tau * nw, axis=1)).max() < 1e-12 * np.abs(wq[:, WALL["p"]]).max()


@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (3, "fp64"), (2, "mixed"), (3, "mixed")])
def test_wall_quantities_against_the_oracle(dim, precision):
    """Wall-point quantities (moments of f*_w per link) through the C-ABI
    against the oracle, after a few steps of a flow past the body."""
    if dim == 2:
        case = wl.small_2d("circle", n=24, nv=12, Ma=0.5, precision=precision)
    else:
        case = wl._case(3, 12, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6), precision=precision)
    g = ibdvm.Solver(case)
    o = oracle.OracleCase(case)
    g.step(4)
    o.step(4)
    wg = g.wall()
    wo = o.wall_quantities()
    assert wg.shape == wo.shape == (o.nlink, len(ibdvm.Solver.WALL_COLUMNS)) and o.nlink > 8
    assert list(ibdvm.Solver.WALL_COLUMNS) == list(o.WALL_COLUMNS)
    tol = TOL if precision == "fp64" else 1e-4
    for i, c in enumerate(o.WALL_COLUMNS):
        err = np.abs(wg[:, i] - wo[:, i]).max() / max(np.abs(wo[:, i]).max(), 1e-3)
        assert err < tol, (c, err)
    _no_flow_through_the_wall(wg, g.geometry().links()["nw"])
    g.close()


def test_wall_quantities_without_a_body_or_a_free_stream():
    """No links: nothing to report.  Ma = 0: C_p is undefined (NaN), the rest
    is the equilibrium of a gas at rest at the wall temperature."""
    g = ibdvm.Solver(wl._case(2, 12, 1.0, 8, 4.0, 0.1, 0.3, {"kind": "none"}))
    assert g.wall().shape == (0, 12)
    g.close()
    g = ibdvm.Solver(wl.small_2d("circle", n=16, nv=16, Ma=0.0))
    wq = g.wall()
    assert np.all(np.isnan(wq[:, WALL["Cp"]]))
    # to the truncated tails of the Maxwellian on [-4.5, 4.5] (exp(-4.5^2) =
    # 1.6e-9 for the mass, a few times more for the second moment)
    np.testing.assert_allclose(wq[:, WALL["rho"]], 1.0, rtol=1e-8)
    np.testing.assert_allclose(wq[:, WALL["p"]], 0.5, rtol=1e-7)
    assert np.abs(wq[:, WALL["slip_x"]:WALL["slip_z"] + 1]).max() < 1e-12
    g.close()


# ---------------------------------------------------------------------------
# optional nonnegative ghost values (reading C26)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,precision", [(2, "fp64"), (2, "mixed"), (3, "fp64")])
def test_nonnegative_ghost_values_against_the_oracle(dim, precision):
    """A supersonic cylinder (sphere in 3D) at the hot wall of Sec. 4.4, where
    many ghost values would be negative: with the option, against the oracle."""
    if dim == 2:
        case = wl._case(2, 48, 4.0, 16, 7.29, 0.03, 3.834, wl.circle(0.5, Tw=5.9), precision=precision,
                        ghost_nonneg=1)
    else:
        case = wl._case(3, 14, 2.0, 8, 7.29, 0.03, 3.834, wl.sphere(0.6, Tw=5.9), precision=precision,
                        ghost_nonneg=1)
    g, o, _, _ = pair(case, 4)
    if precision == "fp64":
        compare(g, o)
    else:
        compare(g, o, tol=1e-5, wtol=1e-5)
    assert g.ghost_band()["fstargc"].min() >= 0.0


def test_supersonic_sphere_stays_positive():
    """The supersonic sphere of Sec. 4.4 (Ma 3.834, T_w = 5.9) started from
    the freestream on 64^3 cells, stretched 24^3 velocities: with
    nonnegative ghost values 100 steps keep a positive density and
    temperature everywhere (without them the first 10 steps fail)."""
    s = ibdvm.Solver(wl.sphere_supersonic())
    s.step(100)
    W, _, t = s.moments()
    fl = t == ibdvm.FLUID
    assert np.all(np.isfinite(W[fl])) and W[fl, 0].min() > 0.0
    wq = s.wall()
    assert np.all(wq[:, WALL["T"]] > 0) and np.all(wq[:, WALL["rho"]] > 0)
    s.close()


# ---------------------------------------------------------------------------
# non-uniform (stretched) velocity grids (reading C25)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,precision,accom", [(2, "fp64", 1.0), (2, "fp64", 0.6), (3, "fp64", 1.0),
                                                 (2, "mixed", 1.0), (3, "mixed", 1.0)])
def test_stretched_velocity_grid_against_the_oracle(dim, precision, accom):
    """Velocity nodes clustered about 0 (spacing growing geometrically toward
    the ends); alpha < 1 exercises the bisection of the specular part."""
    if dim == 2:
        base = wl._case(2, 24, 2.0, 16, 5.0, 0.1, 0.4, wl.circle(0.6, accom=accom), precision=precision)
        case = wl.stretched(base, 0.3)
    else:
        base = wl._case(3, 10, 2.0, 10, 4.5, 0.1, 0.3, wl.sphere(0.7, accom=accom), precision=precision)
        case = wl.stretched(base, 0.4)
    g, o, rg, ro = pair(case, 6)
    if precision == "fp64":
        compare(g, o)
        assert rg == pytest.approx(ro, rel=1e-9)
    else:
        compare(g, o, tol=1e-5, wtol=1e-5)


# ---------------------------------------------------------------------------
# diffuse domain walls (the lid-driven cavity of Sec. 4.1; reading C24)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", 1e-5)])
def test_cavity_against_the_oracle(precision, tol):
    """Lid-driven cavity with the cylinder at its centre: walls on all four
    faces, the lid moving, against the oracle."""
    case = wl.cavity(n=24, nv=16, precision=precision)
    g, o, rg, ro = pair(case, 12)
    if precision == "fp64":
        compare(g, o, tol=tol, wtol=tol, forces=False)  # no free stream: no C_D
    else:
        # W against its scale: the momentum of a flow the lid drives is of
        # order rho_0 U_w = 0.15 (after 12 steps it is still much smaller)
        fl = o.cell_types() == oracle.FLUID
        assert rel_err(g.get_f()[fl], o.get_f()[fl]) < tol
        Wg, _, _ = g.moments()
        Wo, _ = o.moments()
        for i in range(4):
            scale = max(np.abs(Wo[fl, i]).max(), 0.15)
            assert np.abs(Wg[fl, i] - Wo[fl, i]).max() < tol * scale, i
    _compare_force_and_heat(g, o, tol)
    # the residual is the change of W over one step, early in the cavity about
    # 1e-4 of W, so the FP32 rounding of both states shows at the 1e-3 level
    assert rg == pytest.approx(ro, rel=1e-9 if precision == "fp64" else 3e-3)
    # the 2D TMA sweep reads the wall halo; FP64 runs the generic sweep
    assert g.info.sweep_variant == (1 if precision == "mixed" else 0)


def _compare_force_and_heat(g, o, tol, scale=0.1):
    """Force and heat flux on the body, relative to their largest value and at
    least to scale (about p L: before the lid's disturbance reaches the body
    both are rounding noise)."""
    Fg, Qg, _, _ = g.forces()
    Fo, Qo, _, _ = o.forces()
    assert np.abs(Fg - Fo).max() < 10 * tol * max(np.abs(Fo).max(), scale), (Fg, Fo)
    assert abs(Qg - Qo) < 10 * tol * max(abs(Qo), scale), (Qg, Qo)


@pytest.mark.parametrize("precision,tol", [("fp64", TOL), ("mixed", 1e-5)])
def test_box_with_walls_3d_against_the_oracle(precision, tol):
    """3D: walls on all six faces, the top one moving; the mixed case runs
    the 3D TMA sweep, which reads the walls' halo values at the domain faces."""
    case = wl._case(3, 10, ([0.0] * 3, [1.0] * 3), 8, 4.5, 0.1, 0.0, wl.sphere(0.2, center=(0.5, 0.5, 0.5)),
                    domain_walls=wl.box_walls(3, 1.0, lid=(0.2, 0.0)), precision=precision)
    g, o, _, _ = pair(case, 6)
    if precision == "fp64":
        compare(g, o, forces=False)
    else:
        fl = o.cell_types() == oracle.FLUID
        assert rel_err(g.get_f()[fl], o.get_f()[fl]) < tol
        Wg, _, _ = g.moments()
        Wo, _ = o.moments()
        for i in range(5):
            scale = max(np.abs(Wo[fl, i]).max(), 0.2)
            assert np.abs(Wg[fl, i] - Wo[fl, i]).max() < tol * scale, i
    _compare_force_and_heat(g, o, tol)
    assert g.info.sweep_variant == (2 if precision == "mixed" else 0)


def test_closed_box_keeps_its_mass():
    """No mass crosses a diffuse wall: a collisionless closed box with a moving
    lid and walls at two temperatures keeps its mass to rounding."""
    case = wl._case(2, 32, ([0.0, 0.0], [1.0, 1.0]), 16, 5.0, 1e12, 0.0, {"kind": "none"},
                    domain_walls=wl.box_walls(2, 0.8, lid=(0.3, 0.0), lid_T=1.3))
    g = ibdvm.Solver(case)
    W0, _, _ = g.moments()
    g.step(40)
    W1, _, _ = g.moments()
    assert abs(W1[:, 0].sum() - W0[:, 0].sum()) < 1e-13 * W0[:, 0].sum()
    assert np.abs(W1[:, 1]).max() > 1e-3
    g.close()


def test_domain_descriptor_errors_and_batches():
    torch = pytest.importorskip("torch")
    stream = torch.cuda.Stream()
    case = wl.small_2d("circle", n=16, nv=8, precision="mixed")
    g = ibdvm.Solver(case, stream=stream.cuda_stream)
    assert g.info.sweep_variant != 0
    for bad in ([{"Tw": 0.0}] + [None] * 5,                       # T_w <= 0
                [None] * 4 + [{"Tw": 1.0}, None],                 # a z wall in 2D
                [{"Tw": 1.0, "Uw": [float("nan"), 0.0, 0.0]}] + [None] * 5):
        with pytest.raises(ibdvm.IbdvmError) as e:
            g.set_domain(bad)
        assert e.value.status == 1
    d = ibdvm.domain_descriptor([None] * 6)
    d.kind[0] = 7
    assert g.lib.ibdvm_set_domain(g.h, ctypes.byref(d)) == 1
    # walls: the 2D TMA sweep reads their halo; no batch membership
    g.set_domain(wl.box_walls(2, 1.0, lid=(0.1, 0.0)))
    g.refresh_info()
    assert g.info.sweep_variant == 1
    b = ibdvm.Batch(stream=stream.cuda_stream)
    with pytest.raises(ibdvm.IbdvmError):
        b.add(g)
    # no walls again: bit-identical to a case that never had walls
    g.set_domain([None] * 6)
    g.refresh_info()
    assert g.info.sweep_variant == 1
    twin = ibdvm.Solver(case, stream=stream.cuda_stream)
    twin.set_f(g.get_f())
    g.step(5)
    twin.step(5)
    np.testing.assert_array_equal(g.get_f(), twin.get_f())
    b.add(g)
    with pytest.raises(ibdvm.IbdvmError) as e:
        g.set_domain(wl.box_walls(2, 1.0))
    assert e.value.status == 8
    b.close()
    g.close()
    twin.close()


def test_runs_on_a_torch_stream():
    torch = pytest.importorskip("torch")
    case = wl.small_2d("circle", n=16, nv=8)
    s = torch.cuda.Stream()
    g = ibdvm.Solver(case, stream=s.cuda_stream)
    o = oracle.OracleCase(case)
    g.step(2)
    o.step(2)
    compare(g, o)


# ---------------------------------------------------------------------------
# full-size workloads in the launch configuration the benchmark times:
# properties that hold at any size (the oracle cannot run these sizes)
# ---------------------------------------------------------------------------

def _momentum_balance(g, steps=1):
    W0, _, t = g.moments()
    F, Q, _, _ = g.forces()
    g.step(steps)
    W1, _, _ = g.moments()
    fl = t == ibdvm.FLUID
    dV = np.prod([(g.case["hi"][a] - g.case["lo"][a]) / g.case["n"][a] for a in range(g.dim)])
    dP = (W1[fl, 1:1 + g.dim] - W0[fl, 1:1 + g.dim]).sum(axis=0) * dV / g.dt
    return dP, F[: g.dim], W1, t


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-7), ("mixed", 2e-2)])
def test_cylinder_512_full_size_properties(precision, tol):
    case = wl.cylinder_512(Kn=0.1, precision=precision)
    g = ibdvm.Solver(case)
    dP, F, W1, t = _momentum_balance(g)
    # conservative face fluxes: the gas loses the momentum the body receives
    np.testing.assert_allclose(dP, -F, rtol=tol, atol=tol * np.abs(F).max())
    # mirror symmetry about y = 0
    n = case["n"][0]
    Wm = W1.reshape(n, n, -1)
    sym = np.abs(Wm[::-1, :, 0] - Wm[:, :, 0]).max()
    assert sym < (1e-12 if precision == "fp64" else 1e-5)
    assert np.abs(Wm[::-1, :, 2] + Wm[:, :, 2]).max() < (1e-12 if precision == "fp64" else 1e-5)
    # far from the body the freestream is untouched after one step
    U = 0.5 * np.sqrt(5.0 / 6.0)
    far = W1.reshape(n, n, -1)[:40, :40]
    np.testing.assert_allclose(far[..., 0], 1.0, rtol=1e-5)
    np.testing.assert_allclose(far[..., 1], U, rtol=1e-4)
    # wall points: no flow through the wall, and mirror links agree
    wq = g.wall()
    lk = g.geometry().links()
    _no_flow_through_the_wall(wq, lk["nw"])
    key = {(round(x, 9), round(y, 9)): i for i, (x, y, _) in enumerate(lk["xw"])}
    mir = np.array([key[(round(x, 9), round(-y, 9))] for x, y, _ in lk["xw"]])
    stol = 1e-11 if precision == "fp64" else 1e-5
    for c in ("rho", "T", "p", "slip_x", "tau_x"):
        i = WALL[c]
        assert np.abs(wq[mir, i] - wq[:, i]).max() < stol * np.abs(wq[:, i]).max(), c
    for c in ("slip_y", "tau_y"):
        i = WALL[c]
        assert np.abs(wq[mir, i] + wq[:, i]).max() < stol * np.abs(wq[:, i]).max(), c
    g.close()


@pytest.mark.parametrize("workload,steps", [("cylinder_512", 5), ("sphere_96", 3)])
def test_full_size_mixed_against_fp64(workload, steps):
    """The mixed path at the benchmark's full size and launch shape (the TMA
    sweep, the FP32 ghost values, the chunked moment sums) against the FP64
    path (which matches the oracle to 1e-11 on the smaller cases) after a few
    steps: W within 1e-5 of its largest magnitude per component, C_D within
    1e-4."""
    out = {}
    for prec in ("fp64", "mixed"):
        case = getattr(wl, workload)(precision=prec)
        g = ibdvm.Solver(case)
        g.step(steps)
        W, q, t = g.moments()
        _, _, CD, _ = g.forces()
        out[prec] = (W, t, CD)
        g.close()
    (Wd, t, CDd), (Wm, _, CDm) = out["fp64"], out["mixed"]
    fl = t == ibdvm.FLUID
    for i in range(Wd.shape[1]):
        scale = np.abs(Wd[fl, i]).max()
        assert np.abs(Wm[fl, i] - Wd[fl, i]).max() < 1e-5 * scale, i
    assert abs(CDm - CDd) < 1e-4 * abs(CDd)


def test_cylinder_512_axis_exchange():
    """The TMA sweep treats x (faces exchanged through shared memory) and y
    (the march, faces in registers) by different code: a stream along y must
    still be the stream along x with the axes exchanged, at the workload's
    full size, to FP32 rounding."""
    ca = wl.cylinder_512(Kn=0.1, precision="mixed")
    cb = dict(ca, dir=[0.0, 1.0, 0.0])
    a = ibdvm.Solver(ca)
    a.step(20)
    Wa = a.moments()[0].reshape(512, 512, 4)
    a.close()
    b = ibdvm.Solver(cb)
    b.step(20)
    Wb = b.moments()[0].reshape(512, 512, 4)
    b.close()
    swapped = Wa.transpose(1, 0, 2)[:, :, [0, 2, 1, 3]]
    for i in range(4):
        assert np.abs(Wb[:, :, i] - swapped[:, :, i]).max() < 1e-5 * np.abs(swapped[:, :, i]).max(), i


def test_sphere_96_axis_exchange():
    """The 3D TMA sweep marches along z and exchanges x and y faces through
    shared memory: a stream along z must be the stream along x with x and z
    exchanged, at full size, to FP32 rounding."""
    ca = wl.sphere_96(precision="mixed")
    cb = dict(ca, dir=[0.0, 0.0, 1.0])
    out = []
    for c in (ca, cb):
        s = ibdvm.Solver(c)
        s.step(6)
        out.append(s.moments()[0].reshape(96, 96, 96, 5))
        s.close()
    Wa, Wb = out
    swapped = Wa.transpose(2, 1, 0, 3)[..., [0, 3, 2, 1, 4]]
    for i in range(5):
        assert np.abs(Wb[..., i] - swapped[..., i]).max() < 1e-5 * np.abs(swapped[..., i]).max(), i


def test_sphere_96_full_size_properties():
    case = wl.sphere_96(precision="mixed")
    g = ibdvm.Solver(case)
    dP, F, W1, t = _momentum_balance(g)
    np.testing.assert_allclose(dP, -F, rtol=3e-2, atol=3e-2 * np.abs(F).max())
    n = case["n"][0]
    Wm = W1.reshape(n, n, n, -1)
    assert np.abs(Wm[:, ::-1, :, 0] - Wm[:, :, :, 0]).max() < 1e-5
    assert np.abs(Wm[::-1, :, :, 0] - Wm[:, :, :, 0]).max() < 1e-5
    _no_flow_through_the_wall(g.wall(), g.geometry().links()["nw"])
    g.close()


# ---------------------------------------------------------------------------
# the TMA-staged sweep of 2D FP32 cases
# ---------------------------------------------------------------------------

def _solver_env(case, no_tma: bool):
    import os

    old = os.environ.get("IBDVM_NO_TMA")
    os.environ["IBDVM_NO_TMA"] = "1" if no_tma else "0"
    try:
        return ibdvm.Solver(case)
    finally:
        if old is None:
            del os.environ["IBDVM_NO_TMA"]
        else:
            os.environ["IBDVM_NO_TMA"] = old


@pytest.mark.parametrize("shape", ["square_256v", "ragged_64v", "short_rows", "naca_256v", "odd_nv", "asym_padded"])
def test_tma_sweep_against_oracle_and_plain_sweep(shape):
    if shape == "square_256v":
        case = wl.small_2d("circle", n=40, nv=16, Ma=0.4)           # 256 velocities, 64 per quadrant
    elif shape == "ragged_64v":
        case = wl.small_2d("ellipse", n=24, nv=8, Ma=0.6)           # 64 velocities, quadrants padded to 64
        case["n"] = [27, 21]
        case["lo"], case["hi"] = [-2.2, -1.7], [2.0, 1.9]
    elif shape == "short_rows":
        case = wl.small_2d("circle", n=20, nv=12, Ma=0.3)
        case["n"] = [36, 9]
        case["lo"], case["hi"] = [-3.0, -0.75], [3.0, 0.75]
        case["body"] = wl.circle(0.4)
    elif shape == "naca_256v":
        case = wl.small_2d("naca", n=48, nv=16, Ma=0.5)
    elif shape == "odd_nv":
        case = wl.small_2d("circle", n=32, nv=11, Ma=0.5)           # 121 velocities: quadrants of 36, 30, 30, 25
    else:
        # 24^2 velocities on [-4,8] x [-6,6]: quadrants of 192, 96, 192, 96 in
        # 192-velocity chunks, two of them half padding (the cost model's choice)
        case = wl.small_2d("circle", n=36, nv=24, Ma=0.5)
        case["vlo"], case["vhi"] = [-4.0, -6.0], [8.0, 6.0]
    case["precision"] = "mixed"
    o = oracle.OracleCase(case)
    f0 = perturbed(o, 21, 0.2)
    o.set_f(f0)
    g = _solver_env(case, False)
    p = _solver_env(case, True)
    if shape == "asym_padded":
        assert g.nvel_padded == 4 * 192
    g.set_f(f0)
    p.set_f(f0)
    rg = g.step(4)
    rp = p.step(4)
    ro = o.step(4)
    t = o.cell_types()
    fl = t == oracle.FLUID
    fo = o.get_f()[fl]
    assert rel_err(g.get_f()[fl], fo) < 2e-5
    assert rel_err(g.get_f()[fl], p.get_f()[fl]) < 2e-5
    Wg, _, _ = g.moments()
    Wo, _ = o.moments()
    for i in range(4):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    assert rg == pytest.approx(ro, rel=1e-3)
    kt = g.kernel_times()
    assert kt["sweep"][1] == 4


def test_graph_replay_matches_direct_launches():
    """Pairs of steps replayed from a captured CUDA graph give bit-identical
    results to launching every kernel directly."""
    torch = pytest.importorskip("torch")
    case = wl.small_2d("naca", n=40, nv=12, Ma=0.5, precision="mixed")
    s = torch.cuda.Stream()
    g = ibdvm.Solver(case, stream=s.cuda_stream)   # captured graphs
    d = ibdvm.Solver(case)                          # legacy stream: direct launches
    rg = g.step(7)
    rd = d.step(7)
    np.testing.assert_array_equal(g.get_f(), d.get_f())
    assert rg == rd
    rg = g.step(4)
    rd = d.step(4)
    np.testing.assert_array_equal(g.get_f(), d.get_f())
    Fg, Fd = g.step_forces(), d.step_forces()
    assert Fg[2] == Fd[2]


@pytest.mark.parametrize("shape", ["cube", "ragged", "thin_z"])
def test_tma3_sweep_against_oracle_and_plain_sweep(shape):
    """The TMA-staged 3D FP32 sweep against the CPU oracle and the plain sweep."""
    if shape == "cube":
        case = wl._case(3, 12, 2.0, 8, 4.5, 0.1, 0.5, wl.sphere(0.6), precision="mixed")      # 512 velocities
    elif shape == "ragged":
        case = wl._case(3, 12, 2.0, 6, 4.0, 0.08, 0.6, wl.sphere(0.55, center=(0.1, -0.05, 0.07)),
                        precision="mixed")
        case["n"] = [13, 10, 11]
        case["lo"], case["hi"] = [-2.1, -1.6, -1.8], [2.0, 1.7, 1.9]                          # 216 -> 256 padded
    else:
        case = wl._case(3, 12, 2.0, 6, 4.0, 0.1, 0.4, {"kind": "halfspace", "center": [-0.3, 0.0, 0.0],
                                                        "radii": [0.6, 0.0, 0.8], "accom": 0.8, "Tw": 1.1},
                        precision="mixed")
        case["n"] = [9, 7, 6]
    o = oracle.OracleCase(case)
    f0 = perturbed(o, 31, 0.2)
    o.set_f(f0)
    g = _solver_env(case, False)
    p = _solver_env(case, True)
    assert g.info.sweep_variant == 2 and p.info.sweep_variant == 0
    g.set_f(f0)
    p.set_f(f0)
    rg = g.step(3)
    p.step(3)
    ro = o.step(3)
    fl = o.cell_types() == oracle.FLUID
    assert rel_err(g.get_f()[fl], o.get_f()[fl]) < 2e-5
    assert rel_err(g.get_f()[fl], p.get_f()[fl]) < 2e-5
    Wg, _, _ = g.moments()
    Wo, _ = o.moments()
    for i in range(5):
        if np.abs(Wo[fl, i]).max() > 1e-9:
            assert rel_err(Wg[fl, i], Wo[fl, i]) < 1e-5, i
    assert rg == pytest.approx(ro, rel=1e-3)


# ---------------------------------------------------------------------------
# full step counts of the FP64 configurations, against the oracle's stored
# state (tests/golden/make_oracle_goldens.py runs only the oracle)
# ---------------------------------------------------------------------------

def _golden(name):
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    out = {"cells": [], "W": []}
    for line in open(path):
        if line.startswith("#"):
            continue
        key, *vals = line.split()
        if key in ("residual", "Q", "CD", "CL"):
            out[key] = float(vals[0])
        elif key == "F":
            out["F"] = np.array([float(v) for v in vals])
        else:
            out["cells"].append(int(key))
            out["W"].append([float(v) for v in vals])
    out["cells"] = np.array(out["cells"])
    out["W"] = np.array(out["W"])
    return out


@pytest.mark.slow
@pytest.mark.parametrize("name,make,steps", [("cylinder48_fp64_200steps.txt", wl.cylinder_48, 200),
                                             ("sphere24_fp64_50steps.txt", wl.sphere_24, 50)])
def test_full_configuration_fp64_against_the_oracle(name, make, steps):
    gold = _golden(name)
    g = ibdvm.Solver(make())
    res = g.step(steps)
    W, _, _ = g.moments()
    Wg = W[gold["cells"]]
    Wo = gold["W"]
    for i in range(Wo.shape[1]):
        if np.abs(Wo[:, i]).max() > 1e-9:
            assert rel_err(Wg[:, i], Wo[:, i]) < TOL, i
    assert res == pytest.approx(gold["residual"], rel=1e-8)
    F, Q, CD, CL = g.forces()
    scale = np.abs(gold["F"]).max()
    assert np.abs(F - gold["F"]).max() < 10 * TOL * scale
    assert abs(Q - gold["Q"]) < 10 * TOL * max(abs(gold["Q"]), 1e-6)
    assert abs(CD - gold["CD"]) < 10 * TOL * abs(gold["CD"])
    g.close()
