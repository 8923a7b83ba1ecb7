"""Sec. 4.2, the comparison of wall slip with and without the upwind-weighted
interpolation of Eq. upwind: on the hypersonic cylinder (Ma 5, Kn 0.1, radius
1, T_w = 1) the construction without it (the linear extrapolation 2 f_d - f_ac
of Sec. 3.3.4) gives a slip velocity that oscillates along the wall, most of
all on top of the cylinder where the staircase runs along the grid lines; the
upwind-weighted construction smooths it.  The paper plots the two slips; here
the oscillation is measured as the total variation of the tangential slip
along the wall (links ordered by the angle of their intersect point), on a
uniform 256^2 grid over [-8,8]^2 with 40^2 velocities on [-10,10]^2, after
3000 steps from the free stream (ghost values kept nonnegative, reading C26,
as the uniform grid needs for this impulsive start)."""
import numpy as np
import pytest

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


def _tangential_slip(upwind):
    case = wl._case(2, 256, 8.0, 40, 10.0, 0.1, 5.0, wl.circle(1.0), precision="mixed", ghost_nonneg=1,
                    upwind=upwind)
    s = ibdvm.Solver(case)
    res = s.step(3000)
    wq = s.wall()
    lk = s.geometry().links()
    s.close()
    xw, nw = lk["xw"][:, :2], lk["nw"][:, :2]
    th = np.arctan2(xw[:, 1], xw[:, 0])
    tangent = np.stack([-nw[:, 1], nw[:, 0]], axis=1)
    ut = np.sum(wq[:, 1:3] * tangent, axis=1)
    order = np.argsort(th)
    return th[order], ut[order], res


def test_upwind_weighting_smooths_the_wall_slip():
    th_u, ut_u, res_u = _tangential_slip(1)
    th_n, ut_n, res_n = _tangential_slip(3)
    assert np.all(np.isfinite(ut_u)) and np.all(np.isfinite(ut_n))
    assert res_u < 1e-4 and res_n < 1e-4  # both near steady
    tv_u, tv_n = np.abs(np.diff(ut_u)).sum(), np.abs(np.diff(ut_n)).sum()
    top_u = (th_u > np.pi / 3) & (th_u < 2 * np.pi / 3)
    top_n = (th_n > np.pi / 3) & (th_n < 2 * np.pi / 3)
    ttv_u, ttv_n = np.abs(np.diff(ut_u[top_u])).sum(), np.abs(np.diff(ut_n[top_n])).sum()
    # measured on GB300: 3.33 against 4.78 along the whole wall, 0.45 against
    # 0.82 on top of the cylinder
    assert tv_u < 0.85 * tv_n, (tv_u, tv_n)
    assert ttv_u < 0.75 * ttv_n, (ttv_u, ttv_n)
