"""Batched replicas (one persistent cooperative launch per step over all
members, graph-replayed steps, tuned grid) against the oracle and against
stepping each member on its own; the bounded grid-barrier wait."""
import numpy as np
import pytest

import oracle
from paper_0707_1299_gb300 import workloads as W
from _harness import TOL, gpu_lattice, oracle_lattice, rel_err, periodic_diff

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


def _lb():
    from paper_0707_1299_gb300 import lb
    return lb


# Member sets: "uneven" takes the tiled collide (an nx that is not a multiple
# of 8); "x8" (every nx a multiple of 8) the flat 32-site-window collide.
GRIDS = {"uneven": [(12, 12, 12), (20, 16, 8), (9, 13, 11), (33, 5, 7), (16, 16, 16)],
         "x8": [(16, 12, 12), (24, 16, 8), (8, 13, 11), (40, 5, 7), (16, 9, 10)]}


def _uneven_members(kind="uneven"):
    r = W.rng(77)
    grids = GRIDS[kind]
    probs = []
    for k, n in enumerate(grids):
        m = [3, 0, 5, 2, 8][k]
        pts = []
        if m:
            pos = r.uniform(0, 1, size=(m, 3)) * np.asarray(n, float)
            F = r.normal(0, 1e-5, size=(m, 3))
            pts.append(W.PointSet(W.COLLOID, pos, F, np.full(m, 0.117)))
        if k == 2:
            pts.append(W.PointSet(W.ROTLET, [[4.5, 6.1, 5.5]], [[0, 0, 1e-4]], [2.0]))
        walls = (0, 6) if k == 3 else None
        probs.append(W.Problem(f"m{k}", n, 0.5 + 0.1 * k, 0.5 + 0.05 * k, g=(1e-6 * k, 0, 0), walls=walls,
                               a_L=1.6 + 0.1 * k, points=pts))
    return probs


@pytest.mark.parametrize("kind,steps", [("uneven", 31), ("uneven", 30), ("x8", 31)])
def test_batch_matches_oracle_fp64(kind, steps):
    # Each member of the batch advances exactly as the method does on its
    # own lattice: velocity field and colloid positions against the oracle.
    lb = _lb()
    probs = _uneven_members(kind)
    gs = [gpu_lattice(p, lb.LB_F64) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in gs])
    if kind == "x8":  # the untuned persistent grid: 6 blocks per SM
        assert lb.lb_batch_info(batch)["blocks"] == 152 * 6
    lb.lb_batch_step(batch, steps)
    for p, g in zip(probs, gs):
        _, u, _ = g.moments()
        o = oracle_lattice(p)
        p0 = o.pos.copy()
        o.step(steps)
        ref = o.observe()
        assert rel_err(u.cpu().numpy(), ref["u"]) < TOL["f64"], p.name
        if len(o.pos):
            pos, _ = g.particles()
            d = periodic_diff(pos.cpu().numpy(), p0, p.grid)
            dr = periodic_diff(o.pos, p0, p.grid)
            assert rel_err(d, dr) < TOL["f64"], p.name
    lb.lb_batch_destroy(batch)
    for g in gs:
        g.close()


@pytest.mark.parametrize("prec", ["f32", "bf16s"])
def test_batch_matches_members_stepped_alone(prec):
    # The sedimenting-replica recipe (uneven boxes, 20-60 colloids each) in
    # one batch with a tuned grid, against the same members stepped one by
    # one with lb_step: FP32 within the FP32 tolerance (atomic order differs),
    # bfloat16 (different rounding draws) within its stated tolerance.
    lb = _lb()
    pid = {"f32": lb.LB_F32, "bf16s": lb.LB_BF16S}[prec]
    probs = W.replicas(n=8, L_min=16, L_max=40, n_min=20, n_max=60, force=1e-5)
    for p in probs:
        p.a_L = 1.7
    a = [gpu_lattice(p, pid) for p in probs]
    b = [gpu_lattice(p, pid) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in a])
    blocks = lb.lb_batch_tune(batch)
    assert blocks > 0
    steps = 101
    lb.lb_batch_step(batch, 50)
    lb.lb_batch_step(batch, 51)
    for g in b:
        g.step(steps)
    for ga, gb, p in zip(a, b, probs):
        _, ua, _ = ga.moments()
        _, ub, _ = gb.moments()
        assert rel_err(ua.cpu().numpy(), ub.cpu().numpy()) < TOL[prec], p.name
        pa, _ = ga.particles()
        pb, _ = gb.particles()
        p0 = np.concatenate([ps.pos for ps in p.points])
        da = periodic_diff(pa.cpu().numpy(), p0, p.grid)
        db = periodic_diff(pb.cpu().numpy(), p0, p.grid)
        assert rel_err(da, db) < TOL[prec], p.name
    info = lb.lb_batch_info(batch)
    assert info["sites"] == sum(int(np.prod(p.grid)) for p in probs)
    lb.lb_batch_destroy(batch)
    for g in a + b:
        g.close()


def test_batch_refuses_stale_members():
    lb = _lb()
    probs = _uneven_members()[:2]
    gs = [gpu_lattice(p, lb.LB_F32) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in gs])
    lb.lb_batch_step(batch, 3)
    gs[0].set_body_force([0.0, 1e-6, 0.0])
    with pytest.raises(lb.LBError) as e:
        lb.lb_batch_step(batch, 1)
    assert e.value.status == lb.LB_ERR_STATE
    lb.lb_batch_destroy(batch)
    batch = lb.lb_batch_create([g.ctx for g in gs])
    gs[1].step(1)
    with pytest.raises(lb.LBError):
        lb.lb_batch_step(batch, 1)
    lb.lb_batch_destroy(batch)
    for g in gs:
        g.close()


def test_batch_one_launch_per_step_and_barrier_timeout():
    # Every batch step is one kernel launch.  A barrier wait bounded to zero
    # polls gives up at once: the call reports LB_ERR_TIMEOUT through
    # lb_batch_synchronize (the context stays usable), and with the default
    # bound restored a fresh batch of fresh members steps correctly again.
    lb = _lb()
    probs = _uneven_members("x8")
    gs = [gpu_lattice(p, lb.LB_F64) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in gs])
    l0 = lb.lb_batch_info(batch)["launches"]
    lb.lb_batch_step(batch, 6)
    lb.lb_batch_synchronize(batch)
    assert lb.lb_batch_info(batch)["launches"] - l0 == 6
    lb.lb_batch_set_wait_limit(batch, 0)
    lb.lb_batch_step(batch, 2)
    with pytest.raises(lb.LBError) as e:
        lb.lb_batch_synchronize(batch)
    assert e.value.status == lb.LB_ERR_TIMEOUT
    lb.lb_batch_synchronize(batch)  # reported once
    lb.lb_batch_destroy(batch)
    for g in gs:
        g.close()
    gs = [gpu_lattice(p, lb.LB_F64) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in gs])
    lb.lb_batch_step(batch, 5)
    lb.lb_batch_synchronize(batch)
    for p, g in zip(probs, gs):
        _, u, _ = g.moments()
        o = oracle_lattice(p)
        o.step(5)
        assert rel_err(u.cpu().numpy(), o.observe()["u"]) < TOL["f64"], p.name
    lb.lb_batch_destroy(batch)
    for g in gs:
        g.close()


def test_members_step_on_after_the_batch():
    # A batch leaves each member's force field spread at the new positions
    # and its own stencil rows stale: stepping the members alone afterwards
    # (the batch destroyed) continues the same trajectories as the oracle.
    lb = _lb()
    probs = _uneven_members("x8")
    gs = [gpu_lattice(p, lb.LB_F64) for p in probs]
    batch = lb.lb_batch_create([g.ctx for g in gs])
    lb.lb_batch_step(batch, 10)
    lb.lb_batch_synchronize(batch)
    lb.lb_batch_destroy(batch)
    for g in gs:
        g.step(7)
    for p, g in zip(probs, gs):
        _, u, _ = g.moments()
        o = oracle_lattice(p)
        p0 = o.pos.copy()
        o.step(17)
        assert rel_err(u.cpu().numpy(), o.observe()["u"]) < TOL["f64"], p.name
        if len(o.pos):
            pos, _ = g.particles()
            d = periodic_diff(pos.cpu().numpy(), p0, p.grid)
            assert rel_err(d, periodic_diff(o.pos, p0, p.grid)) < TOL["f64"], p.name
    for g in gs:
        g.close()
