"""Pins of the oracle's redistribution beyond the worked two-cell and 2x2
examples (Sec. 5.1): a neighbourhood grown to 2x2x2, the defining property
of the Barth-Jespersen-style limiter, the least-squares fallbacks, and the
sign rule of the merging direction.  Each test names, in its docstring, a
plausible mistake in the oracle that makes it fail.  CPU only."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# the permutations of the neighbourhood code (include/eb.h): xyz, xzy, yxz, yzx, zxy, zyx
PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def synth(oracle, shape, cells, normals=None, cents=None):
    """A c-grid of shape (nx, ny, nz) whose geometry is set by hand: every CV
    covered except ``cells`` {(i,j,k): alpha}; unit EB normals and volume
    centroid offsets (cell units) per CV where given, else zero."""
    nx, ny, nz = shape
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, np.zeros((ny + 1, nx + 1)))
    s = dom.shape(0)
    G = dict(alpha=np.zeros(s), cent=np.zeros((3,) + s), beta=np.zeros((3,) + s), fcent=np.zeros((6,) + s),
             aeb=np.zeros(s), nrm=np.zeros((3,) + s), ebc=np.zeros((3,) + s), ebv=np.zeros((3,) + s),
             flag=np.zeros(s, np.uint8))
    for (i, j, k), a in cells.items():
        G["alpha"][k, j, i] = a
        G["flag"][k, j, i] = 1 if a == 1.0 else 2
    for (i, j, k), n in (normals or {}).items():
        G["nrm"][:, k, j, i] = n
    for (i, j, k), c in (cents or {}).items():
        G["cent"][:, k, j, i] = c
    geom = {0: G}
    for g in (1, 2, 3):   # the other grids are not used: covered everywhere
        sg = dom.shape(g)
        geom[g] = {key: np.zeros(((3,) if key in ("cent", "beta", "nrm", "ebc", "ebv") else (6,) if key == "fcent"
                                  else ()) + sg, np.uint8 if key == "flag" else np.float64) for key in G}
    return dom, geom


def at(a, c):
    return a[..., c[2], c[1], c[0]]


def field(dom, values):
    arr = np.zeros(dom.shape(0))
    for (i, j, k), v in values.items():
        arr[k, j, i] = float(v)
    return arr


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


# ---------------------------------------------------------------------------
# 2x2x2 neighbourhood, worked by hand (tests/golden/wsrd_2x2x2.txt)
# ---------------------------------------------------------------------------
def test_two_by_two_by_two_worked_example(oracle):
    """The neighbourhood of i grows to level 3 past two covered candidates of
    level 2; i and its z neighbour are small, and each holds the extreme
    neighbourhood average of its least-squares stencil, so the limiter zeroes
    both slopes (phi = 0) and every value follows in closed form.  Fails if
    the growth stops at 2x2 (a dropped level), if covered candidates are
    counted in the volume sum, if N or kappa / N is taken per neighbourhood
    instead of per CV, or if the limiter does not bound the reconstruction
    by the stencil's extreme values."""
    gold = read_golden("wsrd_2x2x2.txt")
    i = (1, 1, 1)
    iz, ix, ixz, ixyz, i2z = (1, 1, 2), (2, 1, 1), (2, 1, 2), (2, 2, 2), (1, 1, 3)
    V = {i: Fr(1, 10), iz: Fr(3, 20), ix: Fr(3, 5), ixz: Fr(1), ixyz: Fr(7, 10), i2z: Fr(1)}
    dom, geom = synth(oracle, (5, 5, 6), {c: float(v) for c, v in V.items()},
                      normals={i: (0.48, 0.6, 0.64), iz: (0.0, 0.0, 1.0)})
    T = oracle.wsrd_setup(dom, geom)[0]
    assert at(T["code"], i) == gold["code_i"] and at(T["code"], iz) == gold["code_iz"]
    # the same quantities in exact fractions, from Eqs. kappa .. nbhd_vol
    ki = (Fr(1, 2) - V[i]) / (V[iz] + V[ix] + V[ixz] + V[ixyz])
    kz = (Fr(1, 2) - V[iz]) / V[i2z]
    N = {i: 1, iz: 2, ix: 2, ixz: 2, ixyz: 2, i2z: 2}
    om = {c: 1 - ki / 2 for c in (iz, ix, ixz, ixyz)}
    om[i], om[i2z] = Fr(1), 1 - kz / 2
    vhi = om[i] * V[i] + ki * sum(V[m] / N[m] for m in (iz, ix, ixz, ixyz))
    vhz = om[iz] * V[iz] + kz * V[i2z] / N[i2z]
    for want, got in ((ki, gold["kappa_i"]), (kz, gold["kappa_iz"]), (vhi, gold["vhat_i"]), (vhz, gold["vhat_iz"])):
        assert float(want) == pytest.approx(got, abs=1e-15)
    assert at(T["kappa"], i) == pytest.approx(gold["kappa_i"], abs=1e-15)
    assert at(T["kappa"], iz) == pytest.approx(gold["kappa_iz"], abs=1e-15)
    assert at(T["vhat"], i) == pytest.approx(gold["vhat_i"], abs=1e-15)
    assert at(T["vhat"], iz) == pytest.approx(gold["vhat_iz"], abs=1e-15)
    for c, n in N.items():
        assert at(T["nnb"], c) == n, c
        assert at(T["omega"], c) == pytest.approx(float(om[c]), abs=1e-15), c
    Uh = {i: Fr(10), iz: Fr(-10), ix: Fr(1), ixz: Fr(2), ixyz: Fr(3), i2z: Fr(0)}
    U, sig, phi, qh = oracle.wsrd(dom, geom, {0: T}, 0, field(dom, Uh), diag=True)
    assert at(qh, i) == pytest.approx(gold["Qhat_i"], abs=1e-14)
    assert at(qh, iz) == pytest.approx(gold["Qhat_iz"], abs=1e-14)
    assert at(phi, i) == 0.0 and at(phi, iz) == 0.0
    assert np.all(at(sig, i) == 0.0) and np.all(at(sig, iz) == 0.0)
    names = {i: "U_i", iz: "U_iz", ix: "U_ix", ixz: "U_ixz", ixyz: "U_ixyz", i2z: "U_i2z"}
    for c, key in names.items():
        assert at(U, c) == pytest.approx(gold[key], abs=1e-14), key
    assert sum(float(V[c]) * at(U, c) for c in V) == pytest.approx(float(sum(V[c] * Uh[c] for c in V)), abs=1e-14)


# ---------------------------------------------------------------------------
# the limiter's defining property, on a rough field over a hill
# ---------------------------------------------------------------------------
def decode(code):
    c = int(code) - 1
    L = c % 3 + 1
    c //= 3
    sb, p = c % 8, c // 8
    return PERMS[p], [(-1 if (sb >> d) & 1 else 1) for d in range(3)], L


def member_offsets(code):
    ax, s, L = decode(code)
    out = []
    for c in range((2, 4, 8)[L - 1]):
        off = [0, 0, 0]
        for bit, a in enumerate(ax):
            if (c >> bit) & 1:
                off[a] += s[a]
        out.append(tuple(off))
    return out


@pytest.fixture(scope="module")
def hill(oracle):
    from paper_2604_11959_gb300 import inputs
    nx, ny, nz = 24, 20, 16
    h = inputs.gaussian_hill(nx, ny, h0=0.2, sigma=0.12, centre=(0.43, 0.57))
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, h)
    G = oracle.geometry(dom)
    return dom, G, oracle.wsrd_setup(dom, G)


def test_limiter_keeps_member_reconstructions_within_the_stencil_range(hill, oracle):
    """For every small CV r with a fitted slope, the limited reconstruction
    q_r(x) = Qhat_r + sigma_r . (x - xhat_r) at the centroid of every member
    of M_r lies in [Qmin, Qmax] of Qhat over the least-squares stencil and r
    (the stencil rebuilt here: the non-covered CVs of the 3x3x3 box, an axis
    widened to 5 where the centroid spread is below half a cell); where the
    limiter acted (phi < 1) one of those reconstructions reaches Qmin or Qmax
    (phi is the largest factor that keeps them in range); and on this rough
    field the limiter does act.  Fails if the limiter is left out or takes
    the largest instead of the smallest factor (points leave the range), if
    its bounds come from the members of M_r only (no point reaches the
    stencil's bounds), or if the stencil used for the bounds is always the
    widened one."""
    dom, G, T = hill
    nx, ny = dom.WX, dom.WY
    rng = np.random.default_rng(17)
    limited = free = 0
    for g in range(4):
        nzg = dom.nzg(g)
        alpha = G[g]["alpha"]

        def active(i, j, k):
            if k < 0 or k >= nzg or (g == 3 and (k == 0 or k == dom.nz)):
                return False
            return alpha[k, j % ny, i % nx] > 0

        Uh = rng.uniform(-1, 1, dom.shape(g))
        U, sig, phi, qh = oracle.wsrd(dom, G, T, g, Uh, diag=True)
        xh, cent, code = T[g]["xhat"], G[g]["cent"], T[g]["code"]
        for k, j, i in zip(*np.nonzero(code)):
            if not active(i, j, k):
                continue
            mem = [o for o in member_offsets(code[k, j, i]) if active(i + o[0], j + o[1], k + o[2])]
            if len(mem) < 2:
                continue
            xr = xh[:, k, j, i]
            width = [1, 1, 1]
            for rnd in range(2):
                pts = []
                for dk in range(-width[2], width[2] + 1):
                    for dj in range(-width[1], width[1] + 1):
                        for di in range(-width[0], width[0] + 1):
                            if (di, dj, dk) != (0, 0, 0) and active(i + di, j + dj, k + dk):
                                m = (k + dk, (j + dj) % ny, (i + di) % nx)
                                pts.append((np.array([di, dj, dk]) + xh[(slice(None),) + m] - xr, qh[m]))
                spread = np.max(np.abs(np.array([p for p, _ in pts])), axis=0) if pts else np.zeros(3)
                narrow = spread < 0.5
                if rnd == 0 and narrow.any():
                    width = [2 if n else 1 for n in narrow]
                    continue
                break
            s = sig[:, k, j, i]
            if narrow.any() or len(pts) < 4:
                assert np.all(s == 0.0), (g, (i, j, k))
                continue
            q = [qh[k, j, i] + s @ (np.array(o) + cent[:, k + o[2], (j + o[1]) % ny, (i + o[0]) % nx] - xr)
                 for o in mem]
            vals = [v for _, v in pts] + [qh[k, j, i]]
            qmax, qmin = max(vals), min(vals)
            tol = 1e-13
            assert qmin - tol <= min(q) and max(q) <= qmax + tol, (g, (i, j, k), q, qmin, qmax)
            if phi[k, j, i] < 1.0:
                limited += 1
                assert min(abs(max(q) - qmax), abs(min(q) - qmin)) <= 1e-12, (g, (i, j, k), q, qmin, qmax)
            elif np.any(s != 0.0):
                free += 1
    assert limited > 20 and free > 5, (limited, free)


# ---------------------------------------------------------------------------
# least-squares fallbacks
# ---------------------------------------------------------------------------
def _small_pair(extra, cents=None, normal=(1.0, 0.0, 0.0)):
    """Small CV r = (3,3,3) (V = 0.2) merged with r + x (V = 1); ``extra`` are
    further non-covered CVs (offsets from r, V = 1)."""
    r = (3, 3, 3)
    cells = {r: 0.2, (4, 3, 3): 1.0}
    for o in extra:
        cells[(r[0] + o[0], r[1] + o[1], r[2] + o[2])] = 1.0
    cc = {(r[0] + o[0], r[1] + o[1], r[2] + o[2]): c for o, c in (cents or {}).items()}
    return r, cells, {r: normal}, cc


def _linear(dom, geom, g=(0.3, -0.7, 1.1), a=2.0):
    s = dom.shape(0)
    k, j, i = np.meshgrid(np.arange(s[0]), np.arange(s[1]), np.arange(s[2]), indexing="ij")
    pos = np.stack([i, j, k]).astype(float) + geom[0]["cent"]
    return a + np.tensordot(np.array(g), pos, axes=1)


def test_lsq_widens_a_narrow_axis(oracle):
    """No CV of the 3x3x3 box is offset in y, but two CVs at y +- 2 are: the
    y axis is widened to 5 and the slope of a linear field is recovered in
    all three components (the limiter stays inactive).  Fails if the
    widening is left out (the y slope comes out zero or the fit is refused)."""
    r, cells, nrm, _ = _small_pair([(-1, 0, 0), (0, 0, 1), (0, 0, -1), (1, 0, 1), (0, 2, 0), (0, -2, 0)])
    dom, geom = synth(oracle, (8, 8, 8), cells, normals=nrm)
    T = oracle.wsrd_setup(dom, geom)[0]
    U, sig, phi, qh = oracle.wsrd(dom, geom, {0: T}, 0, _linear(dom, geom), diag=True)
    assert at(phi, r) == 1.0
    assert np.allclose(at(sig, r), [0.3, -0.7, 1.1], rtol=0, atol=1e-13), at(sig, r)
    assert at(U, r) == pytest.approx(_linear(dom, geom)[r[2], r[1], r[0]], abs=1e-13)


def test_lsq_slope_is_zero_when_an_axis_stays_narrow(oracle):
    """The CVs of the box are offset in y only by their centroids (0.2 and
    -0.2 of a cell) and nothing lies at y +- 2: the y spread stays below half
    a cell after widening, so the slope is zero, although the normal matrix
    is regular.  Fails if the spread test after widening is left out (a
    slope is fitted)."""
    r, cells, nrm, cc = _small_pair([(-1, 0, 0), (0, 0, 1), (0, 0, -1), (1, 0, 1)],
                                    cents={(1, 0, 0): (0.0, 0.2, 0.0), (0, 0, -1): (0.0, -0.2, 0.0)})
    dom, geom = synth(oracle, (8, 8, 8), cells, normals=nrm, cents=cc)
    T = oracle.wsrd_setup(dom, geom)[0]
    U, sig, phi, qh = oracle.wsrd(dom, geom, {0: T}, 0, _linear(dom, geom), diag=True)
    assert np.all(at(sig, r) == 0.0)
    # the neighbourhood average itself is untouched by the fallback
    assert at(U, r) == pytest.approx(at(qh, r), abs=1e-15)


def test_lsq_slope_is_zero_for_a_coplanar_stencil(oracle):
    """Every CV of the box (and the neighbourhood centroid) lies in the plane
    x + y + z = 0 through r, with a spread of a whole cell along every axis:
    the normal matrix is singular (det <= 1e-12 (tr/3)^3) and the slope is
    zero.  The neighbourhood {r, r + x - y} reaches its member past the two
    covered candidates r + x and r - y.  Fails if the determinant test is
    left out (Cramer's rule divides by a vanishing determinant)."""
    r = (3, 3, 3)
    plane = [(1, -1, 0), (-1, 1, 0), (1, 0, -1), (-1, 0, 1), (0, 1, -1), (0, -1, 1)]
    cells = {r: 0.2}
    for o in plane:
        cells[(r[0] + o[0], r[1] + o[1], r[2] + o[2])] = 1.0
    dom, geom = synth(oracle, (8, 8, 8), cells, normals={r: (0.8, -0.6, 0.0)})
    T = oracle.wsrd_setup(dom, geom)[0]
    assert member_offsets(at(T["code"], r))[:4] == [(0, 0, 0), (1, 0, 0), (0, -1, 0), (1, -1, 0)]
    Uh = field(dom, {c: v for c, v in zip(cells, (0.5, 1.0, -2.0, 3.0, 0.25, -1.5, 2.5))})
    U, sig, phi, qh = oracle.wsrd(dom, geom, {0: T}, 0, Uh, diag=True)
    assert np.all(at(sig, r) == 0.0), at(sig, r)
    assert np.all(np.isfinite(U))


def test_lsq_slope_is_zero_with_fewer_than_four_points(oracle):
    """Three CVs in the box, spread along every axis and in general position:
    a slope would be determined, but fewer than four points give none.  Fails
    if the point-count test is left out or lowered to three."""
    r, cells, nrm, _ = _small_pair([(0, 1, 0), (0, 0, 1)])
    dom, geom = synth(oracle, (8, 8, 8), cells, normals=nrm)
    T = oracle.wsrd_setup(dom, geom)[0]
    U, sig, phi, qh = oracle.wsrd(dom, geom, {0: T}, 0, _linear(dom, geom), diag=True)
    assert np.all(at(sig, r) == 0.0)


# ---------------------------------------------------------------------------
# merging direction: the sign of a normal component that is rounding noise
# ---------------------------------------------------------------------------
def test_merging_signs_ignore_rounding_noise_in_the_normal(oracle):
    """A small CV under a flat EB whose unit normal carries rounding noise in
    x and y (-3e-14, -1e-15) merges as if the normal were exactly +z: axes
    z, x, y with positive signs, so its 2x2 neighbourhood takes r + x (open)
    and not r - x (covered).  A normal with a real negative x component
    (-0.3) keeps its sign.  Fails if the sign test compares with 0 instead of
    -1e-12 (the noisy normal merges toward -x: other code, other kappa)."""
    r, rz, rx, rxz = (3, 3, 3), (3, 3, 4), (4, 3, 3), (4, 3, 4)
    cells = {r: 0.1, rz: 0.2, rx: 1.0, rxz: 1.0}
    dom, geom = synth(oracle, (8, 8, 8), cells, normals={r: (-3e-14, -1e-15, 1.0), rz: (0.0, 0.0, 1.0)})
    T = oracle.wsrd_setup(dom, geom)[0]
    # axes (z, x, y): permutation 4; no sign bits; level 2
    assert at(T["code"], r) == 1 + (8 * 4 + 0) * 3 + 1
    assert at(T["kappa"], r) == pytest.approx((0.5 - 0.1) / (0.2 + 1.0 + 1.0), abs=1e-15)
    dom2, geom2 = synth(oracle, (8, 8, 8), {r: 0.1, (3, 3, 4): 1.0}, normals={r: (-0.3, 0.0, 0.953939201416946)})
    T2 = oracle.wsrd_setup(dom2, geom2)[0]
    # axes (z, x, y), sign bit of x set, level 1
    assert at(T2["code"], r) == 1 + (8 * 4 + 1) * 3 + 0
