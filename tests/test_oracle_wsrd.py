"""Pins of the oracle's weighted state redistribution (Sec. 5.1): worked
examples evaluated by hand, exact identities, uniform and linear
preservation, conservation.  CPU only."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def synthetic(oracle, nx, ny, nz, alpha_cells, normals):
    """A c-grid whose geometry is set by hand: every CV covered except
    ``alpha_cells`` {(i,j,k): alpha}; unit normals {(i,j,k): n}."""
    h = np.zeros((ny + 1, nx + 1))
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, h)
    s = dom.shape(0)
    G = dict(alpha=np.zeros(s), cent=np.zeros((3,) + s), beta=np.zeros((3,) + s), fcent=np.zeros((6,) + s),
             aeb=np.zeros(s), nrm=np.zeros((3,) + s), ebc=np.zeros((3,) + s), ebv=np.zeros((3,) + s),
             flag=np.zeros(s, np.uint8))
    for (i, j, k), a in alpha_cells.items():
        G["alpha"][k, j, i] = a
        G["flag"][k, j, i] = 1 if a == 1.0 else 2
    for (i, j, k), n in normals.items():
        G["nrm"][:, k, j, i] = n
    geom = {0: G}
    for g in (1, 2, 3):   # other grids unused: covered everywhere
        sg = dom.shape(g)
        geom[g] = {key: np.zeros(((3,) if key in ("cent", "beta", "nrm", "ebc", "ebv") else (6,) if key == "fcent"
                                  else ()) + sg, np.uint8 if key == "flag" else np.float64) for key in G}
    return dom, geom


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_two_cell_worked_example(oracle):
    gold = read_golden("wsrd_two_cell.txt")
    i, n = (1, 0, 1), (2, 0, 1)
    dom, geom = synthetic(oracle, 4, 1, 4, {i: 0.1, n: 1.0}, {i: (1.0, 0.0, 0.0)})
    T = oracle.wsrd_setup(dom, geom)[0]
    at = lambda a, c: a[c[2], c[1], c[0]]
    assert at(T["kappa"], i) == pytest.approx(gold["kappa_i"], abs=1e-15)
    assert at(T["nnb"], i) == gold["N_i"] and at(T["nnb"], n) == gold["N_n"]
    assert at(T["omega"], i) == gold["omega_i"]
    assert at(T["omega"], n) == pytest.approx(gold["omega_n"], abs=1e-15)
    assert at(T["vhat"], i) == pytest.approx(gold["vhat_i"], abs=1e-15)
    Uh = np.zeros(dom.shape(0))
    Uh[i[2], i[1], i[0]] = 2.0
    Uh[n[2], n[1], n[0]] = 1.0
    U = oracle.wsrd(dom, geom, {0: T}, 0, Uh)
    assert at(U, i) == pytest.approx(gold["U_i"], abs=1e-15)
    assert at(U, n) == pytest.approx(gold["U_n"], abs=1e-15)
    assert 0.1 * at(U, i) + at(U, n) == pytest.approx(0.1 * 2.0 + 1.0, abs=1e-15)


def test_two_by_two_worked_example(oracle):
    """Small cell i (V = 0.1, normal (0.8, 0, 0.6)) whose x neighbour a is small
    too (V = 0.2, normal +z): M_i grows to the 2x2 square {i, a, i+z, a+z};
    M_a = {a, a+z}.  Expected values evaluated by hand in exact fractions."""
    i, a, iz, az = (1, 0, 1), (2, 0, 1), (1, 0, 2), (2, 0, 2)
    dom, geom = synthetic(oracle, 5, 1, 5, {i: 0.1, a: 0.2, iz: 1.0, az: 1.0},
                          {i: (0.8, 0.0, 0.6), a: (0.0, 0.0, 1.0)})
    T = oracle.wsrd_setup(dom, geom)[0]
    at = lambda arr, c: arr[c[2], c[1], c[0]]
    Vi, Va = Fr(1, 10), Fr(2, 10)
    ki = (Fr(1, 2) - Vi) / (Va + 1 + 1)           # 2/11
    ka = (Fr(1, 2) - Va) / 1                      # 3/10
    N = {i: 1, a: 2, iz: 2, az: 3}
    om = {i: Fr(1), a: 1 - ki / 2, iz: 1 - ki / 2, az: 1 - (ki + ka) / 3}
    vhi = om[i] * Vi + ki * (Va / 2 + Fr(1, 2) + Fr(1, 3))
    vha = om[a] * Va + ka * Fr(1, 3)
    assert at(T["kappa"], i) == pytest.approx(float(ki), abs=1e-15)
    assert at(T["kappa"], a) == pytest.approx(float(ka), abs=1e-15)
    for c, nn in N.items():
        assert at(T["nnb"], c) == nn
        assert at(T["omega"], c) == pytest.approx(float(om[c]), abs=1e-15)
    assert at(T["vhat"], i) == pytest.approx(float(vhi), abs=1e-15)
    assert at(T["vhat"], a) == pytest.approx(float(vha), abs=1e-15)
    Uh = {i: Fr(3), a: Fr(-1), iz: Fr(2), az: Fr(5)}
    Qi = (om[i] * Vi * Uh[i] + ki * (Va / 2 * Uh[a] + Fr(1, 2) * Uh[iz] + Fr(1, 3) * Uh[az])) / vhi
    Qa = (om[a] * Va * Uh[a] + ka * Fr(1, 3) * Uh[az]) / vha
    expect = {i: Qi, a: om[a] * Qa + ki * Qi / 2, iz: om[iz] * Uh[iz] + ki * Qi / 2,
              az: om[az] * Uh[az] + (ki * Qi + ka * Qa) / 3}
    arr = np.zeros(dom.shape(0))
    for c, v in Uh.items():
        arr[c[2], c[1], c[0]] = float(v)
    U = oracle.wsrd(dom, geom, {0: T}, 0, arr)
    for c, v in expect.items():
        assert at(U, c) == pytest.approx(float(v), abs=1e-14), c
    V = {i: Vi, a: Va, iz: Fr(1), az: Fr(1)}
    assert sum(float(V[c]) * at(U, c) for c in V) == pytest.approx(float(sum(V[c] * Uh[c] for c in V)), abs=1e-14)


@pytest.fixture(scope="module")
def hill(oracle):
    from paper_2604_11959_gb300 import inputs
    nx, ny, nz = 24, 20, 16
    h = inputs.gaussian_hill(nx, ny, h0=0.2, sigma=0.12, centre=(0.43, 0.57))
    dom = oracle.Domain(nx, ny, nz, 1.0, 1.0, 0.5, h)
    G = oracle.geometry(dom)
    return dom, G, oracle.wsrd_setup(dom, G)


def active_mask(dom, G, g):
    m = G[g]["alpha"] > 0
    if g == 3:
        m[0] = m[dom.nz] = False
    return m


def test_weights_bounds_and_identities(hill):
    """0 <= kappa, omega <= 1; omega + sum(kappa_r)/N = 1 makes the final
    update a convex combination; non-small CVs have V_hat = omega V."""
    dom, G, T = hill
    for g in range(4):
        act = active_mask(dom, G, g)
        t = T[g]
        assert (t["code"][act] > 0).sum() > 10
        assert np.all((t["kappa"][act] >= 0) & (t["kappa"][act] <= 1))
        assert np.all((t["omega"][act] > 0) & (t["omega"][act] <= 1))
        assert np.all(t["omega"][act] >= 1.0 / t["nnb"][act] - 1e-15)
        big = act & (t["code"] == 0)
        assert np.allclose(t["vhat"][big], t["omega"][big] * G[g]["alpha"][big], rtol=1e-15, atol=0)
        assert np.all(t["code"][~act] == 0)
        assert np.all(t["code"][act & (G[g]["alpha"] >= 0.5)] == 0)


def test_uniform_and_untouched(hill, oracle):
    """A uniform field is preserved bit for bit (pivoted deviation form); a CV
    that is neither small nor
    in another CV's neighbourhood keeps U_hat bit for bit (its own
    neighbourhood is itself, Sec. 5.1)."""
    dom, G, T = hill
    rng = np.random.default_rng(3)
    for g in range(4):
        c = 1.2345
        U = oracle.wsrd(dom, G, T, g, np.full(dom.shape(g), c))
        act = active_mask(dom, G, g)
        assert np.all(U[act] == c)
        Uh = rng.uniform(-1, 1, dom.shape(g))
        U = oracle.wsrd(dom, G, T, g, Uh)
        alone = act & (T[g]["nnb"] == 1) & (T[g]["code"] == 0)
        assert alone.sum() > 100
        assert np.array_equal(U[alone], Uh[alone])
        assert np.array_equal(U[~act], Uh[~act])


def test_conservation(hill, oracle):
    """sum V U is unchanged by redistribution, for any field."""
    dom, G, T = hill
    rng = np.random.default_rng(4)
    for g in range(4):
        act = active_mask(dom, G, g)
        Uh = rng.uniform(0.5, 2.0, dom.shape(g))
        U = oracle.wsrd(dom, G, T, g, Uh)
        V = G[g]["alpha"] * act
        assert abs((V * U).sum() - (V * Uh).sum()) <= 1e-14 * (V * Uh).sum()


def test_linearity_preserved(hill, oracle):
    """A field linear in the CV centroids is reproduced wherever no limiter or
    degenerate-stencil fallback acted in any neighbourhood the CV belongs to
    (linearity preservation of WSRD)."""
    dom, G, T = hill
    grad = np.array([0.3, -0.7, 1.1])
    for g in range(4):
        s = dom.shape(g)
        k, j, i = np.meshgrid(np.arange(s[0]), np.arange(s[1]), np.arange(s[2]), indexing="ij")
        pos = np.stack([i, j, k]).astype(float) + G[g]["cent"]
        f = 2.0 + np.tensordot(grad, pos, axes=1)
        U, sig, phi, _ = oracle.wsrd(dom, G, T, g, f, diag=True)
        act = active_mask(dom, G, g)
        small = act & (T[g]["code"] > 0)
        exact = small & np.all(np.abs(sig - grad[:, None, None, None]) < 1e-10, axis=0)
        assert exact.sum() > 0.5 * small.sum()
        # a CV is clean when every small CV in its 3x3x3 box that may hold it fits exactly
        bad = small & ~exact
        dirty = np.zeros_like(bad)
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    sh = np.roll(np.roll(bad, dj, axis=1), di, axis=2)
                    if dk > 0:
                        sh = np.concatenate([np.zeros_like(sh[:dk]), sh[:-dk]])
                    elif dk < 0:
                        sh = np.concatenate([sh[-dk:], np.zeros_like(sh[:-dk])])
                    dirty |= sh
        clean = act & ~dirty
        assert clean.sum() > 0.9 * act.sum()
        assert np.max(np.abs(U[clean] - f[clean])) < 1e-12


def test_small_cell_alone(hill, oracle):
    """A small CV that is in no other neighbourhood gets q_i at its own
    centroid: U_i = Q_i + sigma . (x_i - x_hat_i)."""
    dom, G, T = hill
    rng = np.random.default_rng(5)
    for g in range(4):
        Uh = rng.uniform(0, 1, dom.shape(g))
        U, sig, phi, _ = oracle.wsrd(dom, G, T, g, Uh, diag=True)
        t = T[g]
        act = active_mask(dom, G, g)
        sel = act & (t["code"] > 0) & (t["nnb"] == 1)
        assert sel.sum() > 0
        assert np.all(t["omega"][sel] == 1.0)
        # U - sigma.(x - xhat) is the neighbourhood average; it lies within the range of U_hat
        Q = U - np.sum(sig * (G[g]["cent"] - t["xhat"]), axis=0)
        assert np.all(Q[sel] >= Uh.min() - 1e-12) and np.all(Q[sel] <= Uh.max() + 1e-12)
