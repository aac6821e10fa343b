"""The learned-correction kernels (features, bfloat16 forward, fused
backward, Adam) against the oracle MLP, and what the trained network gains
over the plain method on held-out 1x/2x run pairs."""
import numpy as np
import pytest

from oracle import mlp
from _harness import periodic_diff

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


def test_features_match_brute_force():
    lb = _lb()
    rng = np.random.default_rng(5)
    for box, n in (((20, 24, 30), 300), ((9, 9, 9), 40), ((40, 17, 33), 700)):
        pos = rng.uniform(0, 1, (n, 3)) * np.asarray(box, float)
        pos[:5] = np.asarray(box) - 1e-3 * rng.uniform(size=(5, 3))  # near the periodic boundary
        net = lb.lb_mlp_create(np.zeros(lb.lb_mlp_num_params(), dtype=np.float32))
        P = torch.as_tensor(pos, device="cuda").contiguous()
        f = torch.empty((n, 27), dtype=torch.float32, device="cuda")
        lb.lb_mlp_features(net, n, P, box, f)
        ref = mlp.features(pos, box)
        assert np.abs(f.cpu().numpy() - ref).max() < 1e-6
        lb.lb_mlp_destroy(net)


def _features(lb, pos, box):
    n = len(pos)
    net = lb.lb_mlp_create(np.zeros(lb.lb_mlp_num_params(), dtype=np.float32))
    P = torch.as_tensor(pos, device="cuda").contiguous()
    f = torch.empty((n, 27), dtype=torch.float32, device="cuda")
    lb.lb_mlp_features(net, n, P, box, f)
    lb.lb_mlp_destroy(net)
    return f.cpu().numpy()


def test_features_dense_and_near_ties():
    # (a) the number density of the 2e5-colloid 256^3 workload in a 64^3
    # box: about 25 others within the cutoff, so the kept list of the
    # float pass is full and the FP64 window decides;
    # (b) points on a grid of spacing (2, 2.5, 3) jittered by 1e-9, far
    # below float resolution: the four next-nearest at sqrt(10.25) tie in
    # float and the FP64 distances decide which two enter, by lower index
    # on an exact tie;
    # (c) a cubic grid of spacing 2 (exact ties everywhere): 18 entries
    # share the window, more than the float pass keeps, so the FP64
    # search repeats for every point.
    lb = _lb()
    rng = np.random.default_rng(21)
    box = (64, 64, 64)
    pos = rng.uniform(0, 64, (int(round(2e5 / 256 ** 3 * 64 ** 3)), 3))
    assert np.abs(_features(lb, pos, box) - mlp.features(pos, box)).max() < 1e-6
    g = np.stack(np.meshgrid(np.arange(8) * 2.0, np.arange(8) * 2.5, np.arange(8) * 3.0, indexing="ij"), -1)
    pos = g.reshape(-1, 3) + 0.25 + rng.uniform(-1e-9, 1e-9, (512, 3))
    box = (16, 20, 24)
    assert np.abs(_features(lb, pos, box) - mlp.features(pos, box)).max() < 1e-6
    g = np.stack(np.meshgrid(*[np.arange(8) * 2.0] * 3, indexing="ij"), -1)
    pos = g.reshape(-1, 3) + 0.5
    box = (16, 16, 16)
    assert np.abs(_features(lb, pos, box) - mlp.features(pos, box)).max() < 1e-6


def test_forward_many_tiles():
    # the tensor-core forward over 157 tiles of 128 samples (ragged last
    # tile) at the scale of the corrected step's inputs
    lb = _lb()
    n = 128 * 156 + 37
    P, x, _ = _random_problem(n, 4)
    v = mlp.flatten(P).astype(np.float32)
    net = lb.lb_mlp_create(v)
    X = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    y = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    lb.lb_mlp_forward(net, n, X, y)
    yref, _ = mlp.forward(mlp.unflatten(v.astype(np.float64)), x.astype(np.float32).astype(np.float64), bf16_round=True)
    err = np.abs(y.cpu().numpy() - yref).max(axis=1) / np.abs(yref).max()
    assert np.quantile(err, 0.98) < 1e-5 and err.max() < 2e-2
    lb.lb_mlp_destroy(net)


def test_forward_timeout_is_reported_and_recovers():
    # Every wait of the tensor-core forward is bounded.  A bound of 0 polls
    # makes the first one run out: the call returns LB_ERR_TIMEOUT (the
    # kernel drained the work it issued and freed its tensor memory), and
    # with the default bound restored the same network computes correctly.
    lb = _lb()
    n = 1000
    P, x, _ = _random_problem(n, 6)
    v = mlp.flatten(P).astype(np.float32)
    net = lb.lb_mlp_create(v)
    X = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    y = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    lb.lb_mlp_set_wait_limit(net, 0)
    with pytest.raises(lb.LBError) as e:
        lb.lb_mlp_forward(net, n, X, y)
    assert e.value.status == lb.LB_ERR_TIMEOUT
    lb.lb_mlp_set_wait_limit(net, 1 << 26)
    lb.lb_mlp_forward(net, n, X, y)
    yref, _ = mlp.forward(mlp.unflatten(v.astype(np.float64)), x.astype(np.float32).astype(np.float64), bf16_round=True)
    err = np.abs(y.cpu().numpy() - yref).max(axis=1) / np.abs(yref).max()
    assert np.quantile(err, 0.98) < 1e-5 and err.max() < 2e-2
    with pytest.raises(lb.LBError):
        lb.lb_mlp_set_wait_limit(net, -1)
    lb.lb_mlp_destroy(net)


def _random_problem(n, seed):
    rng = np.random.default_rng(seed)
    P = mlp.init_params(seed)
    for k in P:
        P[k] = P[k] + rng.normal(0, 0.05, P[k].shape)
    x = rng.normal(0, 1, (n, 27))
    t = rng.normal(0, 0.5, (n, 3))
    return P, x, t


def test_forward_and_gradient_match_oracle():
    # bfloat16 rounding points as in the kernels; FP32 accumulation on the
    # GPU against FP64 in the oracle.  A pre-activation that lies within the
    # FP32 error of a bfloat16 rounding boundary may round the other way, so
    # single outputs may differ by one bfloat16 unit of an activation; the
    # bulk agrees to FP32 accuracy.
    lb = _lb()
    for n in (200, 64, 1):
        P, x, t = _random_problem(n, 11 + n)
        v = mlp.flatten(P).astype(np.float32)
        P32 = mlp.unflatten(v.astype(np.float64))
        net = lb.lb_mlp_create(v)
        X = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
        T = torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
        y = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        lb.lb_mlp_forward(net, n, X, y)
        xr = x.astype(np.float32).astype(np.float64)
        tr = t.astype(np.float32).astype(np.float64)
        yref, _ = mlp.forward(P32, xr, bf16_round=True)
        err = np.abs(y.cpu().numpy() - yref).max(axis=1) / np.abs(yref).max()
        assert np.quantile(err, 0.98) < 1e-5 and err.max() < 2e-2
        g = np.zeros(lb.lb_mlp_num_params(), dtype=np.float32)
        sse = np.zeros(1, dtype=np.float32)
        lb.lb_mlp_grad(net, n, X, T, g, sse)
        gref = mlp.flatten(mlp.backward(P32, xr, tr, bf16_round=True))
        assert np.abs(g - gref).max() < 3e-3 * np.abs(gref).max()
        assert abs(sse[0] / (3 * n) - np.mean((yref - tr) ** 2)) < 1e-3 * np.mean((yref - tr) ** 2)
        lb.lb_mlp_destroy(net)


def test_adam_steps_match_oracle():
    lb = _lb()
    n, lr = 256, 1e-3
    P, x, t = _random_problem(n, 3)
    v = mlp.flatten(P).astype(np.float32)
    net = lb.lb_mlp_create(v)
    X = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    T = torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
    xr = x.astype(np.float32).astype(np.float64)
    tr = t.astype(np.float32).astype(np.float64)
    vr = v.astype(np.float64)
    m = np.zeros_like(vr)
    s = np.zeros_like(vr)
    for step in range(1, 4):
        g = mlp.flatten(mlp.backward(mlp.unflatten(vr), xr, tr, bf16_round=True))
        vr, m, s = mlp.adam(vr, g, m, s, step, lr)
        lb.lb_mlp_train_step(net, n, X, T, lr)
    out = np.zeros_like(v)
    lb.lb_mlp_get_params(net, out)
    moved = np.abs(vr - v) > 0.5 * lr  # entries whose gradient sign is not in doubt
    assert moved.mean() > 0.5
    assert np.abs(out - vr)[moved].max() < 0.05 * lr
    lb.lb_mlp_destroy(net)


def _splitmix64_rows(seed, s, batch, n):
    # SplitMix64 (Steele, Lea and Flood) of seed + (s batch + b + 1) * 0x9E3779B97F4A7C15,
    # shifted right by 11, mod n: the rows lb_mlp_train documents for minibatch s
    M = (1 << 64) - 1
    rows = []
    for b in range(batch):
        x = (seed + ((s * batch + b + 1) * 0x9E3779B97F4A7C15)) & M
        x ^= x >> 30
        x = (x * 0xBF58476D1CE4E5B9) & M
        x ^= x >> 27
        x = (x * 0x94D049BB133111EB) & M
        x ^= x >> 31
        rows.append((x >> 11) % n)
    return np.array(rows)


def test_native_training_draws_the_documented_minibatches():
    # Two steps of lb_mlp_train against lb_mlp_train_step on the minibatches
    # its documented draw selects (rows from SplitMix64 of seed, step and
    # slot; targets divided by the scale), with the cosine-decayed rate; the
    # recorded losses are the minibatch mean squared errors before each step.
    lb = _lb()
    n, batch, steps, lr, seed, scale = 700, 256, 2, 1e-3, 12345, 0.7
    P, x, t = _random_problem(n, 8)
    v = mlp.flatten(P).astype(np.float32)
    X = torch.as_tensor(x, dtype=torch.float32, device="cuda").contiguous()
    T = torch.as_tensor(t, dtype=torch.float32, device="cuda").contiguous()
    a = lb.lb_mlp_create(v)
    loss = np.zeros(3, dtype=np.float32)
    lb.lb_mlp_train(a, n, X, T, scale, batch, steps, lr, seed, 1, loss)
    b = lb.lb_mlp_create(v)
    sse = np.zeros(1, dtype=np.float32)
    ref_loss = []
    x32, t32 = x.astype(np.float32), t.astype(np.float32)
    for s in range(steps):
        rows = _splitmix64_rows(seed, s, batch, n)
        fb = torch.as_tensor(x32[rows], device="cuda").contiguous()
        tb = torch.as_tensor(t32[rows] * np.float32(1 / scale), device="cuda").contiguous()
        lr_s = max(lr * 0.5 * (1 + np.cos(np.pi * s / steps)), 1e-6)
        lb.lb_mlp_train_step(b, batch, fb, tb, lr_s, sse)
        torch.cuda.synchronize()
        ref_loss.append(sse[0] / (3 * batch))
    pa = np.zeros_like(v)
    pb = np.zeros_like(v)
    lb.lb_mlp_get_params(a, pa)
    lb.lb_mlp_get_params(b, pb)
    assert np.abs(pa - v).max() > 0.5 * lr  # the steps moved the parameters
    # same draws, same steps: equal up to the order of the gradient's FP32
    # sums across CTAs, which can flip the sign of a near-zero gradient
    # component and with it that entry's Adam step
    differ = np.abs(pa - pb) > 1e-3 * lr
    assert differ.mean() < 0.01 and np.abs(pa - pb).max() <= 2.5 * lr
    assert np.allclose(loss[:2], ref_loss, rtol=1e-4)
    lb.lb_mlp_destroy(a)
    lb.lb_mlp_destroy(b)
    c = lb.lb_mlp_create(v)
    with pytest.raises(lb.LBError):
        lb.lb_mlp_train(c, n, X, T, 0.0, batch, 1, lr)  # a target scale must be positive
    lb.lb_mlp_destroy(c)


def test_trained_network_reduces_subgrid_error():
    # Pairs of runs of the method at 1x and 2x resolution (48^3 boxes at the
    # number density of the 2e5-colloids-in-256^3 workload): train on 10
    # boxes, judge on 3 held-out boxes.  The corrected colloid velocity is
    # closer to the resolved one than the plain method's.
    from paper_0707_1299_gb300 import learned
    data = [learned.pair_samples(L=48, seed=s, T=400) for s in range(13)]
    ftr = torch.cat([d[0] for d in data[:10]]).contiguous()
    ltr = torch.cat([d[1] for d in data[:10]]).contiguous()
    fte = torch.cat([d[0] for d in data[10:]]).contiguous()
    lte = torch.cat([d[1] for d in data[10:]]).contiguous()
    net, hist = learned.train(ftr, ltr, steps=1500, batch=2048, lr=2e-3)
    assert hist[-1] < 0.9
    ev = learned.evaluate(net, fte, lte)
    assert ev["rms_corrected"] < 0.9 * ev["rms_plain"], ev


def test_corrected_step_moves_colloids_by_network_output():
    # With a network attached, one lb_step moves each colloid by
    # U + y |F| / (6 pi eta a): rebuild that from the pieces (interpolated
    # velocity, features, forward) and compare; detached, the plain update.
    lb = _lb()
    from paper_0707_1299_gb300 import learned, workloads as W
    prob = W.colloids(L=20, n=30, seed=9, force=1e-5, a_L=1.6)
    rng = np.random.default_rng(4)
    params = (learned.initial_params(7) * 0.3).astype(np.float32)
    net = lb.lb_mlp_create(params)
    g = lb.Lattice(prob.grid, 0.6, 0.6, lb.LB_F64)
    g.set_colloid_aL(1.6)
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    g.step(3)
    lb.lb_set_colloid_correction(g.ctx, net)
    R0, F = g.particles()
    n = R0.shape[0]
    v = g.velocity_at(R0)
    feat = torch.empty((n, 27), dtype=torch.float32, device="cuda")
    lb.lb_mlp_features(net, n, R0, prob.grid, feat)
    y = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    lb.lb_mlp_forward(net, n, feat, y)
    torch.cuda.synchronize()
    g.step(1)
    R1, _ = g.particles()
    eta = 0.6 / 3
    a = 0.117
    Fn = F.cpu().numpy()
    c = (1 / a - 1 / 1.6) / (6 * np.pi * eta)
    v0 = np.linalg.norm(Fn, axis=1, keepdims=True) / (6 * np.pi * eta * a)
    expect = R0.cpu().numpy() + v.cpu().numpy() + Fn * c + y.cpu().numpy().astype(np.float64) * v0
    expect %= np.asarray(prob.grid, float)
    assert np.abs(periodic_diff(R1.cpu().numpy(), expect, prob.grid)).max() < 1e-12
    assert np.abs(y.cpu().numpy()).max() > 1e-3  # the correction did move them
    # detached: the plain Faxen update of Sec. IV
    lb.lb_set_colloid_correction(g.ctx, None)
    v = g.velocity_at(R1)
    torch.cuda.synchronize()
    g.step(1)
    R2, _ = g.particles()
    expect = (R1.cpu().numpy() + v.cpu().numpy() + Fn * c) % np.asarray(prob.grid, float)
    assert np.abs(periodic_diff(R2.cpu().numpy(), expect, prob.grid)).max() < 1e-12
    g.close()
    lb.lb_mlp_destroy(net)


def _jitter(rng, R, delta, box):
    d = rng.normal(size=R.shape)
    d *= delta / np.linalg.norm(d, axis=1, keepdims=True)
    return (R + d) % box


@pytest.mark.parametrize("L,n", [(32, 90), (48, 300)])
def test_kept_candidate_lists_match_a_full_search(L, n):
    # lb_step keeps each colloid's candidates (others within 8.5 lattice
    # units) from step to step and rebuilds them on the device once some
    # colloid has moved more than 0.234 since the last rebuild.  Drive it
    # through reuse, rebuilds, lists that overflow their slots (a cluster of
    # 45 colloids within radius 3, more than their 40 slots) and an
    # unchanged configuration; every step the update must equal the one
    # rebuilt from the stateless full-search features (lb_mlp_features).
    lb = _lb()
    from paper_0707_1299_gb300 import learned, workloads as W
    prob = W.colloids(L=L, n=n, seed=21, force=1e-5, a_L=1.6)
    box = np.asarray(prob.grid, float)
    rng = np.random.default_rng(8)
    params = (learned.initial_params(3) * 0.3).astype(np.float32)
    net = lb.lb_mlp_create(params)
    g = lb.Lattice(prob.grid, 0.6, 0.6, lb.LB_F64)
    g.set_colloid_aL(1.6)
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    lb.lb_set_colloid_correction(g.ctx, net)
    eta, a = 0.6 / 3, 0.117
    R, F = g.particles()
    R = R.cpu().numpy()
    Fn = F.cpu().numpy()
    c = (1 / a - 1 / 1.6) / (6 * np.pi * eta)
    v0 = np.linalg.norm(Fn, axis=1, keepdims=True) / (6 * np.pi * eta * a)
    schedule = [0.01, 0.01, 0.01, 0.2, 0.02, 0.02, "cluster", 0.01, 0.01, 0.3, 0.0, 0.0, "redraw", 0.05]
    for move in schedule:
        if move == "cluster":
            centre = rng.uniform(0, 1, 3) * box
            R = R.copy()
            R[:45] = _jitter(rng, np.tile(centre, (45, 1)), 1.0, box) + rng.uniform(-1, 1, (45, 3))
            R %= box
        elif move == "redraw":
            R = rng.uniform(0, 1, R.shape) * box
        else:
            R = _jitter(rng, R, move, box)
        lb.lb_set_positions(g.ctx, np.ascontiguousarray(R))
        Rd = torch.as_tensor(R, device="cuda").contiguous()
        v = g.velocity_at(Rd)
        feat = torch.empty((n, 27), dtype=torch.float32, device="cuda")
        lb.lb_mlp_features(net, n, Rd, prob.grid, feat)
        y = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        lb.lb_mlp_forward(net, n, feat, y)
        torch.cuda.synchronize()
        g.step(1)
        R1, _ = g.particles()
        R1 = R1.cpu().numpy()
        expect = (R + v.cpu().numpy() + Fn * c + y.cpu().numpy().astype(np.float64) * v0) % box
        assert np.abs(periodic_diff(R1, expect, prob.grid)).max() < 1e-12, move
        R = R1
    lb.lb_set_colloid_correction(g.ctx, None)
    g.close()
    lb.lb_mlp_destroy(net)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_corrected_step_matches_oracle(prec):
    # Reading L4 end to end: lb_step with a network attached against the
    # oracle stepping the same colloids with its own features and its own
    # bfloat16-operand forward (oracle.OracleLB.step(net=...)), 120 steps,
    # trajectories compared.  The method's bar holds for the fluid part of
    # the update; the network's own output is FP32-accumulated on the GPU
    # (FP64 in the oracle, bfloat16 operands on both sides), so for the FP64
    # lattice its share of the displacement -- measured on the oracle as
    # corrected minus plain run -- is held to 1e-5 of itself (FP32 sums and
    # an operand that a near-boundary pre-activation rounds the other way).
    lb = _lb()
    import oracle
    from paper_0707_1299_gb300 import learned, workloads as W
    from _harness import TOL, disp_tol
    pid = {"f64": lb.LB_F64, "f32": lb.LB_F32}[prec]
    steps = 120
    prob = W.colloids(L=32, n=90, seed=12, force=1e-5, a_L=1.6)  # ~3 others within the cutoff
    params = learned.initial_params(11)
    params[-(3 * 64 + 3):] *= 0.1  # y ~ 0.1: the correction moves colloids by ~10 % of v0
    params = params.astype(np.float32)
    net = lb.lb_mlp_create(params)
    P = mlp.unflatten(params.astype(np.float64))
    g = lb.Lattice(prob.grid, prob.tau_s, prob.tau_b, pid)
    g.set_colloid_aL(1.6)
    ps = prob.points[0]
    g.add_point_forces(ps.kind, ps.pos, ps.F, ps.param)
    lb.lb_set_colloid_correction(g.ctx, net)
    p0, _ = g.particles()
    p0 = p0.cpu().numpy()
    g.step(steps)
    p1, _ = g.particles()
    _, u, _ = g.moments()
    torch.cuda.synchronize()
    corr = oracle.OracleLB(prob.grid, prob.tau_s, prob.tau_b, a_L=1.6)
    plain = oracle.OracleLB(prob.grid, prob.tau_s, prob.tau_b, a_L=1.6)
    for o in (corr, plain):
        o.add_points(ps.kind, ps.pos, ps.F, ps.param)
    corr.step(steps, net=P)
    plain.step(steps)
    d_gpu = periodic_diff(p1.cpu().numpy(), p0, prob.grid)
    d_ref = periodic_diff(corr.pos, p0, prob.grid)
    d_net = periodic_diff(corr.pos, plain.pos, prob.grid)  # the network's share
    dmax = np.abs(d_ref).max()
    assert np.abs(d_net).max() > 0.05 * dmax  # the correction matters
    err = np.abs(d_gpu - d_ref).max()
    bar = disp_tol(prec, prob.grid, steps, dmax) * dmax
    allow = bar + (1e-5 * np.abs(d_net).max() if prec == "f64" else 0.0)
    assert err <= allow, (err / dmax, allow / dmax)
    # the fluid is driven by the colloids: a position that differs by err
    # (lattice units) moves the spread force by ~err of its own size, so the
    # field may differ relatively by about err beyond the format's bar
    ref_u = corr.observe()["u"]
    err_u = np.abs(u.cpu().numpy() - ref_u).max() / np.abs(ref_u).max()
    assert err_u <= TOL[prec] + 10 * err, (err_u, err)
    lb.lb_set_colloid_correction(g.ctx, None)
    g.close()
    lb.lb_mlp_destroy(net)
