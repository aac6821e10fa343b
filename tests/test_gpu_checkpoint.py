"""Checkpoints (lb_save / lb_load): a run saved and restored continues bit
for bit in every storage format, and foreign, truncated or corrupt files
are refused without touching the context."""
import os

import numpy as np
import pytest

from paper_0707_1299_gb300 import workloads as W
from _harness import gpu_lattice

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0707_1299_gb300 import build, lb
    build.build()
    lb.load()
    torch.cuda.set_device(0)
    yield


def _state(g):
    pos, _ = g.particles()
    df = torch.empty((19,) + tuple(reversed(g.grid)), dtype=torch.float64, device="cuda")
    from paper_0707_1299_gb300 import lb
    lb.lb_get_populations(g.ctx, df)
    return pos.cpu().numpy(), df.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_restart_is_bit_exact(prec, tmp_path):
    from paper_0707_1299_gb300 import lb
    # eight colloids 8 apart: no two stencils overlap, so the spreading
    # atomics add in a fixed order and the continuation is bit for bit
    prob = W.colloids(L=24, n=8, seed=8, force=1e-5, a_L=1.5)
    prob.points[0].pos = np.array([[4.3 + 8 * i, 4.6 + 8 * j, 4.45 + 8 * k]
                                   for i in range(2) for j in range(2) for k in range(2)])
    prob.g = (1e-6, 0.0, 0.0)
    a = gpu_lattice(prob, prec)
    a.set_walls_z(0, 23)
    a.step(30)
    path = str(tmp_path / "run.ckpt")
    a.save(path)
    a.step(25)
    want = _state(a)
    b = lb.Lattice(prob.grid, 1.0, 2.0, prec)  # other parameters: the checkpoint restores them
    b.load(path)
    b.step(25)
    got = _state(b)
    assert np.array_equal(want[0], got[0]) and np.array_equal(want[1], got[1])
    a.close()
    b.close()


def test_bad_checkpoints_are_refused(tmp_path):
    from paper_0707_1299_gb300 import lb
    g = lb.Lattice((16, 16, 16), 0.5, 0.5, lb.LB_F32)
    g.add_point_forces(lb.LB_STOKESLET, [[8.2, 8.3, 8.4]], [[0.0, 0.0, 1e-5]])
    g.step(3)
    path = str(tmp_path / "a.ckpt")
    g.save(path)
    before = _state(g)
    other = lb.Lattice((16, 16, 18), 0.5, 0.5, lb.LB_F32)
    with pytest.raises(lb.LBError) as e:
        other.load(path)
    assert e.value.status == lb.LB_ERR_ARG
    other.close()
    f64 = lb.Lattice((16, 16, 16), 0.5, 0.5, lb.LB_F64)
    with pytest.raises(lb.LBError):
        f64.load(path)
    f64.close()
    data = open(path, "rb").read()
    bad = str(tmp_path / "bad.ckpt")
    open(bad, "wb").write(data[:-100])  # truncated
    with pytest.raises(lb.LBError):
        g.load(bad)
    flipped = bytearray(data)
    flipped[len(flipped) // 2] ^= 0x40  # one bit of a population
    open(bad, "wb").write(bytes(flipped))
    with pytest.raises(lb.LBError):
        g.load(bad)
    with pytest.raises(lb.LBError):
        g.load(str(tmp_path / "missing.ckpt"))
    after = _state(g)
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[0], after[0])
    g.close()


def _fnv1a(data):
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _reseal(body):
    """A checkpoint body with a valid digest appended (the file another tool
    could write)."""
    return bytes(body) + int(_fnv1a(body)).to_bytes(8, "little")


def test_intact_but_out_of_range_checkpoints_are_refused(tmp_path):
    """A file whose digest is valid but whose header or point block holds
    values the kernels would index with (a position outside the box, a wall
    plane outside the lattice) is refused, and the context is unchanged."""
    import struct
    from paper_0707_1299_gb300 import lb
    g = lb.Lattice((16, 16, 16), 0.5, 0.5, lb.LB_F32)
    g.add_point_forces(lb.LB_STOKESLET, [[8.2, 8.3, 8.4]], [[0.0, 0.0, 1e-5]])
    g.step(3)
    path = str(tmp_path / "a.ckpt")
    g.save(path)
    before = _state(g)
    body = bytearray(open(path, "rb").read()[:-8])
    assert _reseal(body) == open(path, "rb").read()  # the digest is FNV-1a over the body
    hdr = 112  # magic, grid, prec, tau_s, tau_b, g, a_L, counter, walls, seed, scales, counts, pop_bytes
    cases = {}
    far = bytearray(body)
    far[hdr:hdr + 8] = struct.pack("<d", 1.0e6)  # x of the first point
    cases["position"] = far
    nan = bytearray(body)
    nan[hdr + 24:hdr + 32] = struct.pack("<d", float("nan"))  # F_x of the first point
    cases["force"] = nan
    wall = bytearray(body)
    wall[76:80] = struct.pack("<i", 99)  # wall_lo beyond nz
    cases["wall"] = wall
    for name, b in cases.items():
        bad = str(tmp_path / f"{name}.ckpt")
        open(bad, "wb").write(_reseal(b))
        with pytest.raises(lb.LBError) as e:
            g.load(bad)
        assert e.value.status == lb.LB_ERR_ARG, name
    after = _state(g)
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[0], after[0])
    g.load(path)  # the genuine file still loads
    g.close()
