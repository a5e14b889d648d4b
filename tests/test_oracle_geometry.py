"""Pins of the oracle's geometry (Sec. 3.2) against closed forms, brute-force
quadrature and exact invariants.  CPU only."""
import numpy as np
import pytest

GRIDS = range(4)


def make_dom(oracle, h, nx, ny, nz, L=(1.0, 1.0, 0.5)):
    return oracle.Domain(nx, ny, nz, L[0], L[1], L[2], h)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("c_over_dz", [2.3, 2.5, 3.0, 0.0])
def test_flat_terrain_closed_form(oracle, c_over_dz):
    """Flat cut h = c: alpha = clamp(top - max(c, bottom)), vertical face
    fractions the same, horizontal ones 0 or 1, EB area dx*dy in the cut cell,
    normal e_z (Sec. 3.1 definitions of alpha and beta)."""
    nx, ny, nz = 6, 5, 8
    dz = 0.5 / nz
    h = np.full((ny + 1, nx + 1), c_over_dz * dz)
    G = oracle.geometry(make_dom(oracle, h, nx, ny, nz))
    H = c_over_dz
    for g in GRIDS:
        nzg = nz + (g == 3)
        for k in range(nzg):
            lo, hi = (k - 0.5, k + 0.5) if g == 3 else (k, k + 1)
            lo_d, hi_d = max(lo, 0.0), min(hi, float(nz))
            alpha = np.clip(hi_d - max(H, lo_d), 0.0, hi_d - lo_d)
            a = G[g]["alpha"][k]
            assert np.all(a == alpha), (g, k, a[0, 0], alpha)
            if g != 3 or 1 <= k <= nz - 1:
                # vertical faces (x, y) carry the same fraction
                assert np.allclose(G[g]["beta"][0][k], alpha, atol=1e-15, rtol=0)
                assert np.allclose(G[g]["beta"][1][k], alpha, atol=1e-15, rtol=0)
                # low horizontal face at level lo is open iff c < lo
                assert np.all(G[g]["beta"][2][k] == (1.0 if H < lo else 0.0))
            # EB: present iff lo <= c < hi (inside the CV), area dx*dy, normal e_z
            has_eb = lo_d <= H < hi_d
            assert np.allclose(G[g]["aeb"][k], 1.0 if has_eb else 0.0, atol=1e-15)
            if has_eb:
                assert np.allclose(G[g]["nrm"][2][k], 1.0) and np.allclose(G[g]["nrm"][:2, k], 0.0)


def _pos3(L):
    return np.maximum(L, 0.0) ** 3


def rect_int_pos(a, b, c, x0, x1, y0, y1, power=1):
    """Exact integral over [x0,x1]x[y0,y1] of max(a x + b y + c, 0)^power
    (power 0: the measure of L > 0) by inclusion-exclusion of the double
    antiderivative (L+)^(p+2) / ((p+1)(p+2) a b)."""
    def F(x, y):
        L = a * x + b * y + c
        return np.maximum(L, 0.0) ** (power + 2) / ((power + 1) * (power + 2) * a * b)
    return F(x1, y1) - F(x0, y1) - F(x1, y0) + F(x0, y0)


def test_planar_terrain_closed_form(oracle):
    """Tilted plane h = h0 + sx x + sy y: the diagonal split is invisible, cell
    volumes follow from the exact integral of the clamped linear height, the
    vertical face areas from its 1D analogue, and the EB area is
    sqrt(1 + sx^2 + sy^2) times the covered-footprint change."""
    nx, ny, nz = 8, 8, 16
    Lx, Ly, Lz = 1.0, 1.0, 0.5
    dx, dy, dz = Lx / nx, Ly / ny, Lz / nz
    h0, sx, sy = 0.0731, 0.213, -0.117
    X = np.arange(nx + 1) * dx
    Y = np.arange(ny + 1) * dy
    h = h0 + 0.4 + sx * X[None, :] + sy * Y[:, None]   # no periodic wrap: every square is planar
    G = oracle.geometry(make_dom(oracle, h, nx, ny, nz))
    # height in grid units over lattice square (I, J): H = A + a xi + b eta
    a, b = sx * dx / dz, sy * dy / dz
    checked = 0
    for k in range(nz):
        for J in range(ny):
            for I in range(nx):
                A = (h0 + 0.4 + sx * I * dx + sy * J * dy) / dz
                # fluid height clamp(k+1 - H, 0, 1) = (k+1-H)+ - (k-H)+
                vol = (rect_int_pos(-a, -b, k + 1 - A, 0, 1, 0, 1) - rect_int_pos(-a, -b, k - A, 0, 1, 0, 1))
                assert abs(G[0]["alpha"][k, J, I] - vol) < 1e-13, (k, J, I)
                # low x face: xi = 0, H = A + b eta, area of clamp over eta in [0,1]
                def seg(c0, slope):
                    f = lambda e: np.maximum(slope * e + c0, 0.0) ** 2 / (2 * slope)
                    return f(1.0) - f(0.0)
                fx = seg(k + 1 - A, -b) - seg(k - A, -b)
                assert abs(G[0]["beta"][0][k, J, I] - fx) < 1e-13
                fy = seg(k + 1 - A, -a) - seg(k - A, -a)
                assert abs(G[0]["beta"][1][k, J, I] - fy) < 1e-13
                # EB footprint = area{H < k+1} - area{H < k}
                foot = (rect_int_pos(-a, -b, k + 1 - A, 0, 1, 0, 1, power=0)
                        - rect_int_pos(-a, -b, k - A, 0, 1, 0, 1, power=0))
                el = np.sqrt(1 + sx * sx + sy * sy)
                assert abs(G[0]["aeb"][k, J, I] - el * foot) < 1e-12
                if foot > 1e-10:
                    n = np.array([-sx, -sy, 1.0]) / el
                    assert np.allclose(G[0]["nrm"][:, k, J, I], n, atol=1e-14)
                checked += 1
    assert checked == nx * ny * nz


def test_divergence_theorem_planar(oracle):
    """V = 1/3 closed-surface integral of x.n (grid units), with the faces'
    fractions and the EB centroid and area vector: a pin on centroids."""
    nx, ny, nz = 6, 6, 12
    dx, dy, dz = 1.0 / nx, 1.0 / ny, 0.5 / nz
    X = np.arange(nx + 1) * dx
    Y = np.arange(ny + 1) * dy
    h = 0.21 + 0.19 * X[None, :] - 0.08 * Y[:, None]
    G = oracle.geometry(make_dom(oracle, h, nx, ny, nz))
    g = G[0]
    n_ok = 0
    for k in range(nz - 1):
        for j in range(ny - 1):
            for i in range(nx - 1):
                if g["flag"][k, j, i] != 2:
                    continue
                bl = [g["beta"][0][k, j, i], g["beta"][1][k, j, i], g["beta"][2][k, j, i]]
                bh = [g["beta"][0][k, j, i + 1], g["beta"][1][k, j + 1, i], g["beta"][2][k + 1, j, i]]
                faces = sum(0.5 * (bl[d] + bh[d]) for d in range(3))
                eb = -np.dot(g["ebc"][:, k, j, i], g["ebv"][:, k, j, i])
                assert abs(g["alpha"][k, j, i] - (faces + eb) / 3.0) < 1e-13
                n_ok += 1
    assert n_ok > 20


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------

def h_lin(h, dx, dy, X, Y):
    """Piecewise-linear interpolant of nodal heights on the lattice split
    along each square's (0,0)-(1,1) diagonal; X, Y in grid units."""
    I = np.floor(X).astype(int)
    J = np.floor(Y).astype(int)
    xi, eta = X - I, Y - J
    nx, ny = h.shape[1] - 1, h.shape[0] - 1
    I %= nx
    J %= ny
    h00, h10, h01, h11 = h[J, I], h[J, I + 1], h[J + 1, I], h[J + 1, I + 1]
    low = xi >= eta
    return np.where(low, h00 + (h10 - h00) * xi + (h11 - h10) * eta, h00 + (h11 - h01) * xi + (h01 - h00) * eta)


def brute_box(h, dx, dy, dz, x0, x1, y0, y1, z0, z1, m):
    """Midpoint quadrature (m x m columns) of the fluid height in a box given
    in grid units; returns volume (grid units) and centroid."""
    xs = x0 + (np.arange(m) + 0.5) * (x1 - x0) / m
    ys = y0 + (np.arange(m) + 0.5) * (y1 - y0) / m
    XX, YY = np.meshgrid(xs, ys)
    H = h_lin(h, dx, dy, XX, YY) / dz
    base = np.maximum(H, z0)
    g = np.clip(z1 - base, 0.0, z1 - z0)
    w = (x1 - x0) * (y1 - y0) / (m * m)
    V = g.sum() * w
    if V == 0:
        return 0.0, np.zeros(3)
    zm = np.where(g > 0, 0.5 * (z1 * z1 - np.minimum(base, z1) ** 2), 0.0)
    c = np.array([(XX * g).sum() * w, (YY * g).sum() * w, zm.sum() * w]) / V
    return V, c


@pytest.fixture(scope="module")
def rough(oracle):
    rng = np.random.default_rng(11)
    nx, ny, nz = 4, 4, 6
    dz = 0.5 / nz
    core = rng.uniform(0.4, 4.6, (ny, nx)) * dz
    h = np.zeros((ny + 1, nx + 1))
    h[:ny, :nx] = core
    h[:ny, nx] = core[:, 0]
    h[ny] = h[0]
    dom = make_dom(oracle, h, nx, ny, nz)
    return dom, h, oracle.geometry(dom)


def test_bruteforce_volumes_converge(rough):
    """Sub-cell quadrature converges to the oracle's volume fractions and
    centroids on all four grids at second order."""
    dom, h, G = rough
    dx, dy, dz = dom.dx, dom.dy, dom.dz
    boxes = {0: (0.0, 1.0, 0.0, 1.0, 0.0, 1.0), 1: (-0.5, 0.5, 0.0, 1.0, 0.0, 1.0),
             2: (0.0, 1.0, -0.5, 0.5, 0.0, 1.0), 3: (0.0, 1.0, 0.0, 1.0, -0.5, 0.5)}
    worst = {64: 0.0, 256: 0.0}
    n_cut = 0
    for g in range(4):
        ox0, ox1, oy0, oy1, oz0, oz1 = boxes[g]
        for k in range(1, dom.nz - 1):
            for j in range(dom.NY):
                for i in range(dom.NX):
                    if G[g]["flag"][k, j, i] != 2:
                        continue
                    n_cut += 1
                    errs = {}
                    for m in (64, 256):
                        V, c = brute_box(h, dx, dy, dz, i + ox0, i + ox1, j + oy0, j + oy1, k + oz0, k + oz1, m)
                        errs[m] = abs(V - G[g]["alpha"][k, j, i])
                        worst[m] = max(worst[m], errs[m])
                        if m == 256 and V > 0.05:
                            centre = np.array([i + 0.5 * (ox0 + ox1), j + 0.5 * (oy0 + oy1), k + 0.5 * (oz0 + oz1)])
                            assert np.allclose(c - centre, G[g]["cent"][:, k, j, i], atol=3e-4), (g, k, j, i)
    assert n_cut > 50
    assert worst[256] < 2e-5
    assert worst[256] < worst[64] / 8.0


def test_bruteforce_face_fractions(rough):
    """Vertical and horizontal face fractions against 1D / 2D midpoint sums."""
    dom, h, G = rough
    dx, dy, dz = dom.dx, dom.dy, dom.dz
    m = 4000
    s = (np.arange(m) + 0.5) / m
    for k in range(1, dom.nz - 1):
        for j in range(dom.NY):
            for i in range(dom.NX):
                # c-grid low x face at X = i, Y in [j, j+1], Z in [k, k+1]
                H = h_lin(h, dx, dy, np.full(m, float(i)), j + s) / dz
                bx = np.clip(k + 1 - np.maximum(H, k), 0, 1).mean()
                assert abs(bx - G[0]["beta"][0][k, j, i]) < 1e-6
                # u-grid low x face: mid-plane X = i - 1/2
                H = h_lin(h, dx, dy, np.full(m, i - 0.5), j + s) / dz
                bu = np.clip(k + 1 - np.maximum(H, k), 0, 1).mean()
                assert abs(bu - G[1]["beta"][0][k, j, i]) < 1e-6
                # w-grid low z face: plane Z = k - 1/2 over the square
                mm = 400
                ss = (np.arange(mm) + 0.5) / mm
                XX, YY = np.meshgrid(i + ss, j + ss)
                bw = (h_lin(h, dx, dy, XX, YY) / dz < k - 0.5).mean()
                assert abs(bw - G[3]["beta"][2][k, j, i]) < 2e-2 / mm * 10


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def hill(oracle):
    from paper_2604_11959_gb300 import inputs
    nx, ny, nz = 24, 20, 16
    h = inputs.gaussian_hill(nx, ny, h0=0.2, sigma=0.12, centre=(0.43, 0.57))
    dom = make_dom(oracle, h, nx, ny, nz)
    return dom, oracle.geometry(dom)


def test_closure(hill):
    """Discrete divergence theorem of a closed surface: on every CV,
    beta_hi - beta_lo equals the EB area vector, per axis (grid units)."""
    dom, G = hill
    for g in range(4):
        gg = G[g]
        k0, k1 = (1, dom.nz) if g == 3 else (0, dom.nz - 1)
        b = gg["beta"]
        for d in range(3):
            lo = b[d][k0:k1]
            if d == 0:
                hi = np.roll(b[0], -1, axis=2)[k0:k1]
            elif d == 1:
                hi = np.roll(b[1], -1, axis=1)[k0:k1]
            else:
                hi = b[2][k0 + 1:k1 + 1]
            assert np.allclose(hi - lo, gg["ebv"][d][k0:k1], atol=1e-13, rtol=0), (g, d)


def test_additivity_and_flags(hill):
    """Half-cell assembly: total fluid volume is the same on all four grids;
    covered iff alpha = 0; regular CVs are full; an open face has fluid on both
    sides."""
    dom, G = hill
    tot = [G[g]["alpha"].sum() for g in range(4)]
    assert np.allclose(tot, tot[0], rtol=1e-14, atol=0)
    for g in range(4):
        a, f = G[g]["alpha"], G[g]["flag"]
        inner = slice(1, dom.nz) if g == 3 else slice(0, dom.nz)
        assert np.all((a[inner] == 0) == (f[inner] == 0))
        reg = np.zeros_like(f, dtype=bool)
        reg[inner] = f[inner] == 1   # the truncated wall levels of w are excluded
        assert np.all(a[reg] == 1.0)
        assert np.all(G[g]["beta"][:, reg] == 1.0) and np.all(G[g]["aeb"][reg] == 0.0)
        for d, ax in ((0, 2), (1, 1)):
            open_ = G[g]["beta"][d] > 0
            assert np.all(a[open_] > 0) and np.all(np.roll(a, 1, axis=ax)[open_] > 0)
        assert np.all((a >= 0) & (a <= 1 + 1e-15))
        assert np.all((G[g]["beta"] >= 0) & (G[g]["beta"] <= 1 + 1e-15))


def test_ridge_is_y_invariant(oracle):
    """A ridge uniform in y gives bit-identical geometry in every row (the
    diagonal split leaves no trace when h does not depend on y)."""
    from paper_2604_11959_gb300 import inputs
    h = inputs.woa_ridge(32, 32)
    G = oracle.geometry(make_dom(oracle, h, 32, 32, 16))
    for g in range(4):
        for key in ("alpha", "beta", "fcent", "cent", "nrm", "aeb"):
            a = G[g][key]
            assert np.array_equal(a, np.broadcast_to(a[..., :1, :], a.shape)), (g, key)
        assert np.all(G[g]["nrm"][1] == 0.0)
