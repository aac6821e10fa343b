"""Pins of the oracle MLP of the learned correction: analytic gradients
against central finite differences of the loss, the bfloat16 rounding
against its definition, and the neighbour features on configurations whose
answer is known by construction."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    P = mlp.init_params(3)
    for k in P:
        P[k] = P[k] + rng.normal(0, 0.05, P[k].shape)
    x = rng.normal(0, 1, (7, 27))
    t = rng.normal(0, 0.1, (7, 3))
    G = mlp.backward(P, x, t)
    v = mlp.flatten(P)
    g = mlp.flatten(G)
    h = 1e-6
    idx = rng.choice(len(v), 60, replace=False)
    for i in idx:
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd = (mlp.loss(mlp.unflatten(vp), x, t) - mlp.loss(mlp.unflatten(vm), x, t)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])) + 1e-9


def test_silu_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.dsilu(z)).max() < 1e-8


def test_bf16_rounding():
    # bfloat16 keeps the top 16 bits of a float32; round to nearest, ties to even
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0            # tie -> even (mantissa ...0)
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (mantissa ...10)
    assert mlp.bf16(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7
    x = np.random.default_rng(2).normal(size=1000)
    r = mlp.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8 + 1e-300)
    assert np.array_equal(mlp.bf16(r), r)


def test_features_decide_in_float32():
    # The selection distances are float32: a neighbour 2 + 1e-9 away (index
    # 1) and one 2 away (index 2) tie in float32, so the lower index comes
    # first although it is the farther one in exact arithmetic; the vectors
    # are the float32 differences (12 + 1e-9 rounds to 12).
    box = (40, 40, 40)
    pos = np.array([[10.0, 10.0, 10.0], [12.0 + 1e-9, 10.0, 10.0], [8.0, 10.0, 10.0]])
    f = mlp.features(pos, box)
    nb = f[0, 3:9].reshape(2, 3) * mlp.FEAT_LENGTH
    assert np.array_equal(nb, [[2.0, 0.0, 0.0], [-2.0, 0.0, 0.0]])
    # a separation that float32 rounds to exactly R_CUT is kept
    pos = np.array([[1.0, 1.0, 1.0], [9.0 + 1e-8, 1.0, 1.0]])
    assert mlp.features(pos, box)[0, 3] * mlp.FEAT_LENGTH == 8.0


def test_features_known_geometry():
    # a colloid at the centre of a cube of 8 others: its 8 neighbours are the
    # corners, distance sqrt(3); the far colloid is never among them
    box = (40, 40, 40)
    c = np.array([20.25, 19.5, 21.75])
    corners = [c + np.array([sx, sy, sz]) for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]
    pos = np.array([c] + corners + [[2.0, 2.0, 2.0]])
    f = mlp.features(pos, box)
    assert np.allclose(f[0, :3], [0.25, 0.5, 0.75])
    nb = f[0, 3:].reshape(8, 3) * mlp.FEAT_LENGTH
    assert np.allclose(np.sort(np.abs(nb), axis=0), 1.0)
    assert np.allclose((nb ** 2).sum(1), 3.0)
    # minimum image across the periodic boundary; the cutoff
    pos = np.array([[0.5, 10.0, 10.0], [39.5, 10.0, 10.0], [0.5, 10.0, 18.6]])
    f = mlp.features(pos, box)
    assert np.allclose(f[0, 3:6] * mlp.FEAT_LENGTH, [-1.0, 0.0, 0.0])
    assert np.allclose(f[0, 6:], 0.0)  # the third colloid is beyond R_CUT: zero vectors


# ------------------------------------------------------------------ Adam
# Adam as Kingma & Ba define it (Algorithm 1 of "Adam: a method for
# stochastic optimization"): m_t = b1 m + (1 - b1) g, s_t = b2 s + (1 - b2) g^2,
# m^ = m_t / (1 - b1^t), s^ = s_t / (1 - b2^t), v -= lr m^ / (sqrt(s^) + eps).

def test_adam_first_step_moves_by_lr_sign():
    # t = 1: m^ = g and s^ = g^2 exactly, so every parameter moves by
    # -lr g / (|g| + eps), whatever the size of g
    rng = np.random.default_rng(5)
    g = rng.normal(size=200) * 10.0 ** rng.uniform(-6, 3, size=200)
    v = rng.normal(size=200)
    lr = 1e-3
    v1, m, s = mlp.adam(v, g, np.zeros(200), np.zeros(200), 1, lr)
    assert np.allclose(v1 - v, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-18)
    assert np.allclose(m, 0.1 * g, rtol=1e-15) and np.allclose(s, 0.001 * g * g, rtol=1e-15)


def test_adam_eps_outside_the_square_root():
    # g = 1e-9 at t = 1: |step| = lr 1e-9 / (1e-9 + 1e-8) = lr / 11 (eps added
    # after the square root; inside it the step would be ~lr 1e-5)
    v1, _, _ = mlp.adam(np.zeros(1), np.array([1e-9]), np.zeros(1), np.zeros(1), 1, 0.1)
    assert abs(v1[0] + 0.1 / 11) < 1e-15


def test_adam_two_steps_worked_by_hand():
    # v0 = 1, lr = 0.1, default b1, b2, eps; g1 = 0.5, g2 = -1:
    #   t = 1: m = 0.05, s = 0.00025, m^ = 0.5, s^ = 0.25, v1 = 1 - 0.1 * 0.5 / 0.50000001
    #   t = 2: m = -0.055, s = 0.00124975, m^ = -0.055 / 0.19, s^ = 0.00124975 / 0.001999,
    #          sqrt(s^) = 0.79068805087524779745, v2 = v1 + 0.1 * 0.28947368421052631579 / (0.79068805087524779745 + 1e-8)
    v, m, s = mlp.adam(np.array([1.0]), np.array([0.5]), np.zeros(1), np.zeros(1), 1, 0.1)
    assert abs(m[0] / 0.05 - 1) < 1e-14 and abs(s[0] / 0.00025 - 1) < 1e-14
    assert abs(v[0] - 0.90000000199999996) < 1e-15
    v, m, s = mlp.adam(v, np.array([-1.0]), m, s, 2, 0.1)
    assert abs(m[0] / -0.055 - 1) < 1e-14 and abs(s[0] / 0.00124975 - 1) < 1e-14
    assert abs(v[0] - 0.93661035424056560) < 1e-14


def test_adam_constant_gradient_is_bias_free():
    # a constant gradient g: m_t = (1 - b1^t) g and s_t = (1 - b2^t) g^2, so the
    # bias-corrected moments are g and g^2 at every step and each step moves
    # by exactly -lr g / (|g| + eps) (a missing or swapped bias correction
    # makes the steps drift)
    g = np.array([3e-4, -2.0, 7.0])
    v = np.zeros(3)
    m = np.zeros(3)
    s = np.zeros(3)
    for t in range(1, 60):
        v_new, m, s = mlp.adam(v, g, m, s, t, 1e-2)
        assert np.allclose(v_new - v, -1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        v = v_new


# ---------------------------------------------------- bfloat16 backward
# Reading L3: with bf16_round the products take bfloat16 operands -- the
# input x, the weights, h1, h2, dL/dy in the layer-3 gradients, gz2 and gz1
# where they enter the weight and bias gradients and gh1 = gz2 W2 -- while
# gh2 = (dL/dy) W3 takes the unrounded dL/dy.  The FP64 path is pinned by
# finite differences above; these pins fix where the rounding sits.

def _problem(seed, B=24):
    rng = np.random.default_rng(seed)
    P = mlp.init_params(seed)
    for k in P:
        P[k] = P[k] + rng.normal(0, 0.05, P[k].shape)
    x = rng.normal(0, 1, (B, 27))
    t = rng.normal(0, 0.3, (B, 3))
    return P, x, t


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in a)


def _nudge_within_cell(v, rng, frac=2 ** -12):
    """v moved by ~frac relative where that keeps its bfloat16 rounding."""
    w = v * (1 + frac * rng.choice([-1.0, 1.0], size=np.shape(v)))
    return np.where(mlp.bf16(w) == mlp.bf16(v), w, v)


def test_bf16_backward_close_to_fp64_backward():
    # every rounding point perturbs by at most 2^-9 relative: the rounded
    # gradients stay within a few percent of the finite-difference-pinned
    # FP64 ones (a wrong sign, index or transposed operand would not)
    P, x, t = _problem(3)
    G = mlp.backward(P, x, t)
    Gb = mlp.backward(P, x, t, bf16_round=True)
    for k in G:
        assert np.linalg.norm(Gb[k] - G[k]) <= 0.03 * np.linalg.norm(G[k]), k


def test_bf16_operands_enter_only_rounded():
    # x, W1, W2, W3 moved inside their bfloat16 rounding cells: the rounded
    # forward and every rounded gradient are unchanged bit for bit (the FP64
    # path, the control, changes)
    rng = np.random.default_rng(7)
    P, x, t = _problem(4)
    y0, _ = mlp.forward(P, x, bf16_round=True)
    G0 = mlp.backward(P, x, t, bf16_round=True)
    F0 = mlp.backward(P, x, t)
    for key in ("x", "W1", "W2", "W3"):
        Q = dict(P)
        xq = x
        if key == "x":
            xq = _nudge_within_cell(x, rng)
        else:
            Q[key] = _nudge_within_cell(P[key], rng)
        y1, _ = mlp.forward(Q, xq, bf16_round=True)
        assert np.array_equal(y0, y1), key
        assert _same(G0, mlp.backward(Q, xq, t, bf16_round=True)), key
        assert not _same(F0, mlp.backward(Q, xq, t)), key


def test_bf16_hidden_activations_and_their_gradients_are_rounded():
    # b1 (or b2) moved by 1e-13 relative changes z1 (z2) in FP64 only; z
    # reaches the outputs through h = bf16(silu(z)) and gz = bf16(gh
    # silu'(z)) alone, so nothing rounded changes (the FP64 control does)
    P, x, t = _problem(5)
    y0, c0 = mlp.forward(P, x, bf16_round=True)
    G0 = mlp.backward(P, x, t, bf16_round=True)
    F0 = mlp.backward(P, x, t)
    for key in ("b1", "b2"):
        Q = dict(P)
        Q[key] = P[key] * (1 + 1e-13) + 1e-15
        y1, c1 = mlp.forward(Q, x, bf16_round=True)
        assert np.array_equal(c0[2], c1[2]) and np.array_equal(c0[4], c1[4])  # h1, h2
        assert not np.array_equal(c0[1 if key == "b1" else 3], c1[1 if key == "b1" else 3])  # z moved
        assert np.array_equal(y0, y1), key
        assert _same(G0, mlp.backward(Q, x, t, bf16_round=True)), key
        assert not _same(F0, mlp.backward(Q, x, t)), key


def test_bf16_output_gradient_rounded_for_layer3_only():
    # targets moved so that dL/dy stays in its bfloat16 rounding cell but
    # moves by ~0.4 of half a cell: dW3 and db3 (which take bf16(dL/dy)) do
    # not change, while gh2 = (dL/dy) W3 (unrounded dL/dy) does, and with it
    # some of the rounded gz2 and the gradients of layers 1 and 2
    P, x, t = _problem(6)
    y, _ = mlp.forward(P, x, bf16_round=True)
    B = x.shape[0]
    gy = 2.0 * (y - t) / (3 * B)
    r = mlp.bf16(gy)
    ulp = np.abs(r) * 2.0 ** -7  # bfloat16 spacing near r (8 significant bits), conservative
    gy2 = r + 0.4 * 0.5 * ulp * np.where(gy >= r, -1.0, 1.0)
    assert np.array_equal(mlp.bf16(gy2), r)
    t2 = y - gy2 * (3 * B) / 2.0
    G0 = mlp.backward(P, x, t, bf16_round=True)
    G1 = mlp.backward(P, x, t2, bf16_round=True)
    assert np.array_equal(G0["W3"], G1["W3"]) and np.array_equal(G0["b3"], G1["b3"])
    assert not np.array_equal(G0["W2"], G1["W2"]) and not np.array_equal(G0["W1"], G1["W1"])


# ---------------------------------------------- corrected colloid update
# Reading L4: with a network attached a colloid moves by its Sec. IV
# velocity plus y |F| / (6 pi eta a), y evaluated at the step's start.

def _colloid_oracle():
    import oracle
    o = oracle.OracleLB((14, 12, 11), 0.6, 0.6, a_L=1.6)
    o.add_points(oracle.COLLOID, [[3.3, 4.4, 5.5], [7.1, 2.2, 3.3], [9.6, 8.1, 2.4]],
                 [[0.0, 0.0, -1e-5], [1e-5, 0.0, 0.0], [3e-6, -4e-6, 2e-6]], [0.117, 0.117, 0.2])
    o.step(4)
    return o


def test_corrected_step_with_zero_network_is_the_plain_step():
    P = mlp.init_params(2)
    P["W3"] = np.zeros_like(P["W3"])
    a, b = _colloid_oracle(), _colloid_oracle()
    a.step(3)
    b.step(3, net=P)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.df, b.df)


def test_corrected_step_adds_y_times_v0():
    # a network with W3 = 0 outputs y = b3 exactly: after one step from the
    # same state the corrected colloids sit y |F| / (6 pi eta a) beyond the
    # plain ones (the fluid, spread before the move, is the same)
    P = mlp.init_params(2)
    P["W3"] = np.zeros_like(P["W3"])
    P["b3"] = np.array([0.25, -0.5, 1.0])
    a, b = _colloid_oracle(), _colloid_oracle()
    a.step(1)
    b.step(1, net=P)
    eta = 0.6 / 3
    v0 = np.linalg.norm(a.f, axis=1) / (6 * np.pi * eta * a.radius)
    assert np.allclose(b.pos - a.pos, P["b3"][None, :] * v0[:, None], rtol=1e-9, atol=1e-18)
    assert np.array_equal(a.df, b.df)
