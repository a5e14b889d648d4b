"""The warm-start network (eb_unet_*) against the FP64 oracle
(oracle/unet.py) with the same BF16-rounded weights: forward pass, the
gradient of every parameter, and the Adam step; and its use as the
projection's initial guess (eb_project_sample, eb_project_warm)."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import make_geometry, refs_for

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import eb as _eb
    _eb.load(build_if_missing=True)
    return _eb


@pytest.fixture(scope="module")
def un():
    from oracle import unet
    return unet


def bf16_weights(un, p32):
    """The parameters the kernels compute with: BF16-rounded weights (round to
    nearest even) and FP32 biases, as float64."""
    q = p32.astype(np.float32).copy()
    bits = q.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    wq = rounded.astype(np.uint32).view(np.float32)
    out, o = q.astype(np.float64), 0
    for ci, co, k in un.LAYERS:
        n = co * ci * k ** 3
        out[o:o + n] = wq[o:o + n]
        o += n + co
    return out


def _problem(un, shape, seed):
    rng = np.random.default_rng(seed)
    p = (un.init_params(seed) * 0.7).astype(np.float32)
    p += (0.02 * rng.standard_normal(p.size)).astype(np.float32)
    x = rng.standard_normal((2,) + shape)
    t = rng.standard_normal((1,) + shape)
    mask = (rng.uniform(size=(1,) + shape) > 0.25).astype(np.float64)
    return p, x, t, mask


def test_forward_matches_oracle(eb, un):
    shape = (8, 16, 20)
    p, x, _, _ = _problem(un, shape, 1)
    net = eb.UNet(shape[2], shape[1], shape[0])
    net.set_params(p)
    y = net.forward(torch.from_numpy(x).float().cuda()).double().cpu().numpy()
    want, _ = un.forward(bf16_weights(un, p), x.astype(np.float32).astype(np.float64))
    err = np.max(np.abs(y - want[0])) / np.max(np.abs(want))
    assert err <= 1e-4, err
    net.close()


def test_gradient_matches_oracle(eb, un):
    shape = (8, 12, 16)
    p, x, t, mask = _problem(un, shape, 2)
    net = eb.UNet(shape[2], shape[1], shape[0])
    net.set_params(p)
    xs = torch.from_numpy(x).float().cuda()
    ts = torch.from_numpy(t[0]).float().cuda()
    ms = torch.from_numpy(mask[0]).float().cuda()
    loss, g = net.gradient(xs, ts, ms)
    pw = bf16_weights(un, p)
    y, a = un.forward(pw, x.astype(np.float32).astype(np.float64))
    L, dy = un.loss(y, t.astype(np.float32).astype(np.float64), mask)
    gw, _ = un.backward(pw, a, dy)
    assert abs(loss - L) <= 1e-4 * L
    assert np.linalg.norm(g - gw) <= 1e-3 * np.linalg.norm(gw)
    o = 0
    for ci, co, k in un.LAYERS:   # every layer's weights and biases on their own
        for n in (co * ci * k ** 3, co):
            a_, b_ = g[o:o + n], gw[o:o + n]
            assert np.linalg.norm(a_ - b_) <= 5e-3 * np.linalg.norm(b_) + 1e-12, (ci, co, n)
            o += n
    net.close()


def test_adam_step_and_training_reduce_the_loss(eb, un):
    shape = (8, 12, 16)
    p, x, t, mask = _problem(un, shape, 3)
    net = eb.UNet(shape[2], shape[1], shape[0])
    net.set_params(p)
    xs = torch.from_numpy(x).float().cuda()
    ts = torch.from_numpy(t[0]).float().cuda()
    ms = torch.from_numpy(mask[0]).float().cuda()
    _, g = net.gradient(xs, ts, ms)
    lr = 1e-3
    l0 = net.train_step(xs, ts, ms, lr, want_loss=True)
    p1 = net.get_params()
    q, _, _ = un.adam(p.astype(np.float64), np.zeros(p.size), np.zeros(p.size), g.astype(np.float64), 1, lr)
    big = np.abs(g) > 1e-3 * np.max(np.abs(g))
    assert np.max(np.abs(p1 - q)[big]) <= 1e-3 * lr
    for _ in range(40):
        last = net.train_step(xs, ts, ms, lr, want_loss=True)
    assert last < 0.5 * l0, (l0, last)
    net.close()


def _flow(w, seed):
    return inputs.anelastic_state(w, seed=seed)


def test_warm_started_projection_is_the_same_projection(eb):
    """With any network (here untrained) the warm-started solve reaches the
    same tolerance and the same corrected momenta as the cold solve."""
    w = inputs.Workload("grf-32x32x16", 32, 32, 16, 1, terrain="grf", seed=21, hmax=0.15)
    refs = refs_for(w.nz, w.Lz)
    geo = make_geometry(eb, w, w.heights(), "f64", refs)
    U = eb.device_state(_flow(w, 1), "f64", refs)
    dt = w.dt()
    net = eb.UNet(w.nx, w.ny, w.nz)
    from oracle import unet as un
    net.set_params(un.init_params(5).astype(np.float32) * 0.1)
    A = {f: U[f].clone() for f in U}
    B = {f: U[f].clone() for f in U}
    it0, r0 = eb.project(geo, A, dt, rtol=1e-12)
    it1, r1 = eb.project_warm(geo, net, B, dt, scale=10.0, rtol=1e-12)
    assert r0 <= 1e-12 and r1 <= 1e-12
    scale = max(float(A[f].abs().max()) for f in ("rhou", "rhov", "rhow"))
    for f in ("rhou", "rhov", "rhow"):
        assert float((A[f] - B[f]).abs().max()) <= 1e-9 * scale
    x, t, m, its = eb.project_sample(geo, U, dt, scale=10.0, rtol=1e-10)
    assert its > 0 and float(m.sum()) > 0 and torch.isfinite(t).all()
    net.close()
    geo.close()


def test_trained_network_saves_iterations(eb):
    """Train the network briefly on small random terrains with the library's
    own samples and kernels, then compare cold and warm starts on held-out
    terrains: the warm start saves iterations at a loose tolerance and never
    costs more than a few at 1e-10, with the same converged result."""
    from paper_2604_11959_gb300 import warmstart as ws
    r = ws.Recipe(nx=32, ny=32, nz=16, dx=1.0 / 64.0, terrains=12, states_per_terrain=6, epochs=6, lr=2e-3,
                  seed=300)
    scale = ws.target_scale(r)
    data, _ = ws.make_dataset(r, scale)
    net = ws.train(r, data)
    params = net.get_params()
    net.close()
    cold_l, warm_l, cold_t, warm_t = [], [], [], []
    for q in range(4):
        w = ws.workload(r, 900 + q)
        g, refs = ws.geometry(w)
        c, h, rc, rw, d = ws.compare(g, params, w, refs, 5 + q, scale, rtol=1e-4)
        cold_l.append(c)
        warm_l.append(h)
        c, h, rc, rw, d = ws.compare(g, params, w, refs, 5 + q, scale, rtol=1e-10)
        cold_t.append(c)
        warm_t.append(h)
        assert rw <= 1e-10 and d <= 1e-7
        g.close()
    assert np.mean(warm_l) < np.mean(cold_l), (cold_l, warm_l)
    assert np.mean(warm_t) <= np.mean(cold_t) + 5, (cold_t, warm_t)


def test_many_tiles_per_cta_match_oracle(eb, un):
    """A 64 x 64 x 32 grid: the persistent convolution kernels then walk
    several tiles per CTA (the forward 512 tiles of 8 x 16 x 2 voxels over
    at most two CTAs per SM; the weight gradient 1024 tiles of 8 x 8 x 2 over
    about 100 to 300 CTAs per layer), carrying halo prefetches and tensor-
    memory accumulators from tile to tile.  Forward pass and gradient against
    the oracle with the tolerances above."""
    shape = (32, 64, 64)
    p, x, t, mask = _problem(un, shape, 4)
    net = eb.UNet(shape[2], shape[1], shape[0])
    net.set_params(p)
    xs = torch.from_numpy(x).float().cuda()
    y = net.forward(xs).double().cpu().numpy()
    pw = bf16_weights(un, p)
    want, a = un.forward(pw, x.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(y - want[0])) <= 1e-4 * np.max(np.abs(want))
    loss, g = net.gradient(xs, torch.from_numpy(t[0]).float().cuda(), torch.from_numpy(mask[0]).float().cuda())
    L, dy = un.loss(want, t.astype(np.float32).astype(np.float64), mask)
    gw, _ = un.backward(pw, a, dy)
    assert abs(loss - L) <= 1e-4 * L
    assert np.linalg.norm(g - gw) <= 1e-3 * np.linalg.norm(gw)
    net.sync_status()
    net.close()


def test_a_wait_that_runs_out_reports_a_timeout(eb, un):
    """The bounded waits of the convolution kernels, tested without a GPU
    fault: one convolution launch issues its products without signalling
    their completion, every CTA's wait runs out (about one second, twice) and
    the CTAs return; eb_unet_sync_status reports EB_ERR_TIMEOUT once, and the
    next forward pass on the same context matches the oracle."""
    shape = (8, 16, 16)
    p, x, _, _ = _problem(un, shape, 5)
    net = eb.UNet(shape[2], shape[1], shape[0])
    net.set_params(p)
    xs = torch.from_numpy(x).float().cuda()
    net.inject_wait_fault()
    net.forward(xs)
    with pytest.raises(eb.EbError) as e:
        net.sync_status()
    assert e.value.code == 5
    net.sync_status()   # reported once
    y = net.forward(xs).double().cpu().numpy()
    want, _ = un.forward(bf16_weights(un, p), x.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(y - want[0])) <= 1e-4 * np.max(np.abs(want))
    net.close()
