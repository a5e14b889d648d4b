"""eb_wsrd_noalloc (redistribution with the library's fixed device scratch)
against eb_wsrd, the entry point with handle-owned scratch.  Collected last
so that it also runs after every other test has used the library."""
import numpy as np
import pytest

from _gpu_helpers import FIELDS, make_geometry, refs_for, rel_linf, to_device

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import eb as _eb
    _eb.load(build_if_missing=True)
    return _eb


def _rough_case():
    from paper_2604_11959_gb300 import inputs
    w = inputs.Workload("grf-64x48x24", 64, 48, 24, 1, terrain="grf", seed=7, hmax=0.25, tiny=6)
    return w, w.heights()


def _provisional(w, seed):
    rng = np.random.default_rng(seed)
    U = w.state("uniform", pert=0.05, seed=seed)
    return {f: U[f] * (1.0 + 0.3 * rng.uniform(-1, 1, U[f].shape)) for f in FIELDS}


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_noalloc_matches_wsrd_on_two_calls_in_a_row(eb, precision):
    w, h = _rough_case()
    refs = refs_for(w.nz, w.Lz)
    geom = make_geometry(eb, w, h, precision, refs)
    assert min(geom.info()["small_cvs"]) > 0
    for seed in (21, 22):  # two different inputs, so a stale scratch would show
        dev = to_device(_provisional(w, seed), precision, refs)
        for f in FIELDS:
            want = eb.wsrd(geom, f, dev[f])
            first = torch.empty_like(dev[f])
            eb.wsrd_noalloc(geom, f, dev[f], first)
            second = dev[f].clone()
            eb.wsrd_noalloc(geom, f, second, second)  # in place, right after the first call
            eb.sync_status(geom)
            # the same kernels on the same inputs: any difference, even in the
            # last bit, is a scratch-layout or stale-scratch fault
            for got in (first, second):
                assert torch.equal(got, want), (precision, seed, f,
                                                rel_linf(got.double().cpu().numpy(), want.double().cpu().numpy()))


def test_noalloc_rejects_a_field_beyond_the_fixed_scratch(eb):
    """A flat terrain 0.8 dz below a level makes every c-grid column hold one
    small CV: 512 x 512 of them need 10.5 MB of scratch in double (rejected)
    and 5.2 MB in float (accepted, and equal to eb_wsrd)."""
    from paper_2604_11959_gb300 import inputs
    nz, Lz = 8, 0.5
    dz = Lz / nz
    w = inputs.Workload("flat-512x512x8", 512, 512, nz, 1, Lz=Lz, terrain="flat", hmax=2.8 * dz)
    h = w.heights()
    refs = refs_for(w.nz, w.Lz)
    U = _provisional(w, 5)

    g64 = make_geometry(eb, w, h, "f64", refs)
    assert g64.info()["small_cvs"][0] == 512 * 512
    dev = to_device(U, "f64", refs)
    out = dev["rho"].clone()
    with pytest.raises(eb.EbError) as ei:
        eb.wsrd_noalloc(g64, "rho", dev["rho"], out)
    assert "scratch" in str(ei.value)
    assert torch.equal(out, dev["rho"])  # nothing was launched
    del g64, dev, out

    g32 = make_geometry(eb, w, h, "mixed", refs)
    dev = to_device(U, "mixed", refs)
    want = eb.wsrd(g32, "rho", dev["rho"])
    got = torch.empty_like(dev["rho"])
    eb.wsrd_noalloc(g32, "rho", dev["rho"], got)
    eb.sync_status(g32)
    assert torch.equal(got, want)
