"""Host logic of the two-level step (paper_2604_11959_gb300/amr.py) on CPU,
with a stand-in for the binding that records the calls: the patch is held
with its halo as an x-window whose first column wraps around the periodic
domain, its nodal heights are the true fine ones, and every step fills the
halo from the coarse state at time n, advances both levels, then restricts
the owned columns onto the new coarse state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


class _Geom:
    def __init__(self, log, nx, ny, nz, Lx, Ly, Lz, h, **kw):
        self.log, self.nx, self.ny, self.nz = log, nx, ny, nz
        self.Lx, self.h = Lx, h.cpu().numpy() if h is not None else None
        log.append(("build", nx, ny, nz, Lx))

    def coarse(self, **kw):
        self.log.append(("coarse", self.nx // 2))
        return _Geom(self.log, self.nx // 2, self.ny // 2, self.nz // 2, self.Lx, 0, 0, None)

    def set_wind_reference(self, *a):
        self.log.append(("wind",))

    def close(self):
        self.log.append(("close", self.nx))


class _Eb:
    def __init__(self):
        self.log = []

    def Geometry(self, *a, **kw):
        return _Geom(self.log, *a, **kw)

    def prolong(self, coarse, Uc, fine, Uf, fine_x0, owned):
        self.log.append(("prolong", fine_x0, tuple(owned), Uc))
        return Uf

    def step(self, geom, U, dt, n, stages):
        self.log.append(("step", geom.nx, U, stages))
        return U + "'"

    def restrict(self, fine, coarse, Uf, Uc, fine_x0, cols):
        self.log.append(("restrict", fine_x0, tuple(cols), Uf, Uc))
        return Uc


def test_two_level_host_sequence():
    from paper_2604_11959_gb300 import amr
    eb = _Eb()
    nx, ny = 40, 8
    h = np.arange((ny + 1) * (nx + 1), dtype=float).reshape(ny + 1, nx + 1)
    two = amr.TwoLevel(eb, nx, ny, 8, 2.0, 1.0, 1.0, h, 4, 12, 6, "f64", device="cpu")
    assert two.fine_x0 == 38 and two.owned == (6, 14)           # the window starts at column -2
    builds = [e for e in eb.log if e[0] == "build"]
    assert builds[0][1:] == (40, 8, 8, 2.0)                       # the whole fine level, then its coarse level
    assert builds[1][1] == 20 and builds[2][1] == 20              # the patch: 8 owned + 2 x 6 halo columns
    assert builds[2][4] == pytest.approx(20 * 2.0 / 40)
    patch_h = two.patch.h
    assert np.array_equal(patch_h[:, 0], h[:, 38]) and np.array_equal(patch_h[:, -1], h[:, 18])
    eb.log.clear()
    Uc, Uf = two.step("C", "F", 0.1, 3)
    assert (Uc, Uf) == ("C'", "F'")
    kinds = [e[0] for e in eb.log]
    assert kinds == ["prolong", "step", "step", "restrict"]
    assert eb.log[0][1:] == (38, (6, 14), "C")                    # halo from the coarse state at time n
    assert eb.log[1][1:] == (20, "C", 3) and eb.log[2][1:] == (20, "F", 3)
    assert eb.log[3][1:] == (38, (6, 14), "F'", "C'")              # owned columns onto the new coarse state
    with pytest.raises(ValueError):
        amr.TwoLevel(eb, nx, ny, 8, 2.0, 1.0, 1.0, h, 3, 12, 6, "f64", device="cpu")
