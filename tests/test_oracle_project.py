"""Pins of the projection oracle (oracle/eb_project.py) against what the
mathematics fixes: the closed-form spectrum of the discrete Neumann /
periodic Laplacian on flat terrain, summation by parts between the
divergence and the gradient, the constant null space, symmetry and sign of
the operator, a divergence-free result, the discrete Pythagoras identity of
an orthogonal projection, and idempotence.  CPU only."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs


@pytest.fixture(scope="module")
def proj():
    from oracle import eb_project
    return eb_project


def _domain(oracle, nx, ny, nz, h, Lz=0.5):
    return oracle.Domain(nx, ny, nz, 1.0, 1.0, Lz, h)


@pytest.fixture(scope="module")
def rough(oracle):
    w = inputs.Workload("grf-24x20x12", 24, 20, 12, 1, terrain="grf", seed=11, hmax=0.2, tiny=2)
    dom = _domain(oracle, w.nx, w.ny, w.nz, w.heights())
    return dom, oracle.geometry(dom)


def _random_momenta(dom, geom, seed):
    rng = np.random.default_rng(seed)
    m = []
    for g in (1, 2, 3):
        a = rng.standard_normal(dom.shape(g))
        a[geom[g]["alpha"] == 0] = 0.0
        if g == 3:
            a[0] = a[-1] = 0.0
        m.append(a)
    return m


def test_flat_terrain_operator_has_the_discrete_laplacian_spectrum(oracle, proj):
    """h = 0: every face open but the walls, so L is the 7-point Laplacian,
    periodic in x, y and Neumann in z, whose eigenvectors are products of
    cosines with eigenvalue -sum 4 sin^2(theta / 2) / delta^2."""
    nx, ny, nz = 16, 12, 10
    dom = _domain(oracle, nx, ny, nz, np.zeros((ny + 1, nx + 1)))
    geom = oracle.geometry(dom)
    b = proj.face_weights(dom, geom)
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    for p, q, r in ((1, 0, 0), (2, 3, 1), (0, 1, 4), (5, 5, 9)):
        tx, ty, tz = 2 * np.pi * p / nx, 2 * np.pi * q / ny, np.pi * r / nz
        phi = np.cos(tx * (i + 0.3)) * np.cos(ty * (j + 0.1)) * np.cos(tz * (k + 0.5))
        lam = -(4 * np.sin(tx / 2) ** 2 / dom.dx ** 2 + 4 * np.sin(ty / 2) ** 2 / dom.dy ** 2 +
                4 * np.sin(tz / 2) ** 2 / dom.dz ** 2)
        Lphi = proj.laplacian(dom, b, phi)
        assert np.max(np.abs(Lphi - lam * phi)) <= 1e-9 * max(1.0, abs(lam))


def test_divergence_and_gradient_are_adjoint(oracle, proj, rough):
    """sum_c phi_c D(m)_c = - sum_f beta_f m_f G(phi)_f (periodic sides,
    closed walls): a sign, index or weight slip in either breaks it."""
    dom, geom = rough
    b = proj.face_weights(dom, geom)
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(dom.shape(0))
    mu, mv, mw = _random_momenta(dom, geom, 4)
    lhs = np.sum(phi * proj.divergence(dom, b, mu, mv, mw))
    gu, gv, gw = proj.gradient(dom, b, phi)
    bw = np.zeros(dom.shape(3))
    bw[:-1] = b[2]
    rhs = -(np.sum(b[0] * mu * gu) + np.sum(b[1] * mv * gv) + np.sum(bw * mw * gw))
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs) + 1.0)


def test_operator_null_space_symmetry_and_sign(oracle, proj, rough):
    dom, geom = rough
    b = proj.face_weights(dom, geom)
    d = proj.diagonal(dom, b)
    one = np.where(d > 0, 1.0, 0.0)
    assert np.max(np.abs(proj.laplacian(dom, b, one))) <= 1e-12 * np.max(d)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(dom.shape(0)) * (d > 0)
    y = rng.standard_normal(dom.shape(0)) * (d > 0)
    xLy = np.sum(x * proj.laplacian(dom, b, y))
    yLx = np.sum(y * proj.laplacian(dom, b, x))
    assert abs(xLy - yLx) <= 1e-12 * (abs(xLy) + abs(yLx))
    assert np.sum(x * proj.laplacian(dom, b, x)) < 0.0


def test_projection_is_divergence_free_orthogonal_and_idempotent(oracle, proj, rough):
    dom, geom = rough
    b = proj.face_weights(dom, geom)
    mu, mv, mw = _random_momenta(dom, geom, 6)
    dt = 0.01
    nu, nv, nw, phi, it, res = proj.project(dom, geom, mu, mv, mw, dt, rtol=1e-12)
    assert res <= 1e-12 and it > 0
    d0 = np.linalg.norm(proj.divergence(dom, b, mu, mv, mw))
    d1 = np.linalg.norm(proj.divergence(dom, b, nu, nv, nw))
    assert d1 <= 1e-11 * d0
    # Pythagoras in the beta-weighted face norm: the correction dt G(phi) is
    # orthogonal to the projected field
    bw = np.zeros(dom.shape(3))
    bw[:-1] = b[2]
    wts = (b[0], b[1], bw)
    before = sum(np.sum(w * m * m) for w, m in zip(wts, (mu, mv, mw)))
    after = sum(np.sum(w * m * m) for w, m in zip(wts, (nu, nv, nw)))
    corr = sum(np.sum(w * (m - n) ** 2) for w, m, n in zip(wts, (mu, mv, mw), (nu, nv, nw)))
    assert abs(before - (after + corr)) <= 1e-9 * before
    assert after < before
    # projecting again changes nothing on the open faces (its divergence is
    # rounding, so the solve stops at the first projection's residual)
    qu, qv, qw, _, it2, _ = proj.project(dom, geom, nu, nv, nw, dt, rtol=1e-12, atol=1e-12 * d0 / dt)
    scale = max(np.max(np.abs(nu)), np.max(np.abs(nv)), np.max(np.abs(nw)))
    for w, a, c in zip(wts, (nu, nv, nw), (qu, qv, qw)):
        assert np.max(np.abs(np.where(w > 0, a - c, 0.0))) <= 1e-9 * scale


def test_warm_start_from_the_solution_needs_no_iterations(oracle, proj, rough):
    dom, geom = rough
    mu, mv, mw = _random_momenta(dom, geom, 8)
    _, _, _, phi, it, _ = proj.project(dom, geom, mu, mv, mw, 0.02, rtol=1e-10)
    _, _, _, _, it0, res0 = proj.project(dom, geom, mu, mv, mw, 0.02, rtol=1e-10, phi0=phi)
    assert it0 == 0 and res0 <= 1e-10 and it > 10
