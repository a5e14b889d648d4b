"""The x-slab decomposition (paper_2604_11959_gb300/slabs.py) on CPU: two
gloo ranks, each advancing its slab (owned columns plus halo) with the FP64
oracle run on that column window, the halos exchanged through
torch.distributed before every step.  The owned columns must equal the
oracle's single-domain result bit for bit: the decomposition changes where
CVs are computed, never how.  The oracle stands in for the GPU library as the
per-rank stepper (the GPU form is tests/test_gpu_slabs.py); the module
itself imports neither."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = ("rho", "rhotheta", "rhou", "rhov", "rhow")


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(stages):
    from paper_2604_11959_gb300 import inputs
    nx = 64 if stages == 1 else 112
    return inputs.Workload(f"grf-{nx}x16x12", nx, 16, 12, 3 if stages == 1 else 2, terrain="grf", seed=21,
                           hmax=0.22, tiny=2)


def _rank_main(rank, world, port, stages, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import eb_oracle as O
    from paper_2604_11959_gb300 import slabs as S
    dist.init_process_group("gloo")
    try:
        O.set_threads(1)
        w = _case(stages)
        h = w.heights()
        U = w.state("sheltered", seed=3)
        sl = S.Slabs(w.nx, world, rank, S.HALO_EULER if stages == 1 else S.HALO_RK3)
        x0 = (sl.x0 - sl.halo) % w.nx
        dom = O.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, h, window=(x0, 0, sl.ext, w.ny))
        G = O.geometry(dom)
        T = O.wsrd_setup(dom, G)
        held = {f: torch.from_numpy(np.ascontiguousarray(sl.scatter(U[f]))) for f in FIELDS}

        def step_one(Ut):
            R = O.step(dom, G, T, {f: Ut[f].numpy() for f in FIELDS}, w.dt(), 1, stages)
            return {f: torch.from_numpy(R[f]) for f in FIELDS}

        held = S.advance(sl, held, w.steps, step_one, dist)
        out.put((rank, sl.x0, sl.x1, {f: sl.interior(held[f].numpy()).copy() for f in FIELDS}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("stages", [1, 3])
def test_two_ranks_equal_the_single_domain(oracle, stages):
    """Forward Euler (halo 12, three steps) and the three-stage form (halo
    24, two steps) on a random terrain with planted tiny cells."""
    w = _case(stages)
    dom = oracle.Domain(w.nx, w.ny, w.nz, w.Lx, w.Ly, w.Lz, w.heights())
    G = oracle.geometry(dom)
    want = oracle.step(dom, G, oracle.wsrd_setup(dom, G), w.state("sheltered", seed=3), w.dt(), w.steps, stages)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, stages, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for f in FIELDS:
        got = np.concatenate([r[3][f] for r in res], axis=-1)
        assert np.array_equal(got, want[f]), (stages, f, float(np.abs(got - want[f]).max()))


def test_slab_bounds_heights_and_local_exchange():
    """Owned ranges tile the domain; the held nodal heights are the true ones
    (the last node column is the slab's right edge); the in-process exchange
    fills each halo with the neighbours' edge columns."""
    from paper_2604_11959_gb300 import slabs as S
    nx, ny, world, H = 50, 3, 3, 4
    sl = [S.Slabs(nx, world, r, H) for r in range(world)]
    assert [s.x0 for s in sl] == [0, 16, 33] and [s.x1 for s in sl] == [16, 33, 50]
    h = np.arange((ny + 1) * (nx + 1), dtype=float).reshape(ny + 1, nx + 1)
    h[:, nx] = h[:, 0]
    hs = sl[1].heights(h)
    assert hs.shape == (ny + 1, sl[1].ext + 1)
    assert np.array_equal(hs[:, 0], h[:, 16 - H]) and np.array_equal(hs[:, -1], h[:, 33 + H])
    glob = {f: np.arange(2 * ny * nx, dtype=float).reshape(2, ny, nx) + 1000 * q for q, f in enumerate(S.FIELDS)}
    states = [{f: s.scatter(glob[f]).copy() for f in S.FIELDS} for s in sl]
    for st in states:           # spoil the halos, then exchange them back
        for f in S.FIELDS:
            st[f][..., :H] = -1
            st[f][..., -H:] = -1
    S.exchange_local(sl, states)
    for s, st in zip(sl, states):
        for f in S.FIELDS:
            assert np.array_equal(st[f], s.scatter(glob[f]))
    with pytest.raises(ValueError):
        S.Slabs(10, 4, 0, 4)
