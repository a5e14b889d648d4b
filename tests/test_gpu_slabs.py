"""The x-slab decomposition on the GPU: two ranks held by one process (the
run has one GPU; their steps run one after the other and never wait on one
another), each with the geometry handle of its slab (owned columns plus halo,
built from the true nodal heights) and the library's eb_step, the halos
exchanged by copies before every step.  The owned columns must equal the
single-domain eb_step bit for bit, in both precisions, for forward Euler and
the three-stage form."""
import numpy as np
import pytest

from paper_2604_11959_gb300 import inputs

from _gpu_helpers import FIELDS, make_geometry, to_device, wind_refs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_11959_gb300 import build, eb as ebmod
    build.build()
    ebmod.load()
    return ebmod


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("stages", [1, 3])
def test_two_slabs_equal_the_single_domain(eb, precision, stages):
    from paper_2604_11959_gb300 import slabs as S
    nx = 64 if stages == 1 else 112
    w = inputs.Workload(f"grf-{nx}x16x12", nx, 16, 12, 3 if stages == 1 else 2, terrain="grf", seed=21, hmax=0.22,
                        tiny=2)
    h = w.heights()
    refs = wind_refs(w, "sheltered")
    U = w.state("sheltered", seed=3)
    whole = make_geometry(eb, w, h, precision, refs)
    want = eb.step(whole, to_device(U, precision, refs), w.dt(), w.steps, stages)
    sl = [S.Slabs(w.nx, 2, r, S.HALO_EULER if stages == 1 else S.HALO_RK3) for r in range(2)]
    geoms, held = [], []
    for s in sl:
        ws = inputs.Workload("slab", s.ext, w.ny, w.nz, 1, Lx=s.ext * w.Lx / w.nx, Ly=w.Ly, Lz=w.Lz)
        geoms.append(make_geometry(eb, ws, s.heights(h), precision, refs))
        held.append(to_device({f: np.ascontiguousarray(s.scatter(U[f])) for f in FIELDS}, precision, refs))
    for _ in range(w.steps):
        S.exchange_local(sl, held)
        held = [eb.step(g, Uq, w.dt(), 1, stages) for g, Uq in zip(geoms, held)]
    for f in FIELDS:
        got = torch.cat([s.interior(Uq[f]) for s, Uq in zip(sl, held)], dim=-1)
        assert torch.equal(got, want[f]), (precision, stages, f, float((got - want[f]).abs().max()))
    for g in geoms + [whole]:
        eb.sync_status(g)
        g.close()
