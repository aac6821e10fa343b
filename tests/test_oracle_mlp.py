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
