"""Learned correction of the point-colloid velocity (the paper's method stays
the reference it is judged against).

Training pairs come from the method itself at two lattice resolutions.  A
periodic box of side L with n colloids held in place (force F each, radius
a) is run for T steps; the same physical configuration on a lattice twice
as fine (side 2L, positions 2R, the same lattice force, radius 2a) is run
for 4T steps.  Under diffusive scaling at equal tau the fine run's lattice
velocities are half the coarse run's, so 2 U_2x is the coarse-unit colloid
velocity the finer lattice resolves; the label of a colloid is
(2 U_2x - U_1x) / v0 with v0 = |F| / (6 pi eta a), U the colloid velocity
of Sec. IV (interpolated fluid velocity plus the Faxen term with the a_L
subtraction) from `lb_colloid_velocity`.  Features come from
`lb_mlp_features` (fractional offset, 8 nearest neighbours).

Everything runs through the C ABI (`lb`); torch only holds device memory.
"""
from __future__ import annotations

import math

import numpy as np

from . import lb
from . import workloads as W

NUMBER_DENSITY = 2e5 / 256 ** 3  # colloids per lattice site of the 256^3, 2e5-colloid workload


def pair_samples(L: int = 64, seed: int = 0, T: int = 1000, force: float = 1e-6, a: float = W.A_TABLE1,
                 density: float = NUMBER_DENSITY, tau: float = 0.5, precision: int = lb.LB_F32):
    """One 1x/2x run pair: returns (features, labels, U1, U2x): features
    (n, 27) and labels (n, 3) as float32 torch tensors on the current device,
    and the two colloid velocities (n, 3) as float64 numpy arrays in coarse
    lattice units."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    r = W.rng(1000 + seed)
    n = max(2, int(round(density * L ** 3)))
    R = r.uniform(0, L, size=(n, 3))
    F = np.tile([0.0, 0.0, -force], (n, 1))
    eta = tau / 3.0
    v0 = force / (6 * math.pi * eta * a)
    out = {}
    for k, (Lk, Rk, ak, steps) in enumerate(((L, R, a, T), (2 * L, 2 * R, 2 * a, 4 * T))):
        g = lb.Lattice((Lk, Lk, Lk), tau, tau, precision)
        g.set_colloid_aL(lb.lb_compute_aL((Lk, Lk, Lk), [Lk / 2 + 0.5] * 3, [0, 0, 1]))
        g.add_point_forces(lb.LB_STOKESLET, Rk, F)
        g.step(steps)
        pos = torch.as_tensor(Rk, dtype=torch.float64, device=dev).contiguous()
        Ft = torch.as_tensor(F, dtype=torch.float64, device=dev).contiguous()
        rad = torch.full((n,), ak, dtype=torch.float64, device=dev)
        U = torch.empty((n, 3), dtype=torch.float64, device=dev)
        lb.lb_colloid_velocity(g.ctx, n, pos, Ft, rad, U)
        out[k] = U
        g.close()
    U1 = out[0].cpu().numpy()
    U2x = 2.0 * out[1].cpu().numpy()
    labels = torch.as_tensor(((U2x - U1) / v0).astype(np.float32), device=dev).contiguous()
    return features(R, (L, L, L)), labels, U1, U2x


_feature_net = None


def features(R, box):
    """(n, 27) float32 device tensor of `lb_mlp_features` for positions R."""
    import torch
    global _feature_net
    if _feature_net is None:
        _feature_net = lb.lb_mlp_create(np.zeros(lb.lb_mlp_num_params(), dtype=np.float32))
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.as_tensor(np.asarray(R), dtype=torch.float64, device=dev).contiguous()
    feat = torch.empty((len(pos), 27), dtype=torch.float32, device=dev)
    lb.lb_mlp_features(_feature_net, len(pos), pos, box, feat)
    return feat


def initial_params(seed: int = 0) -> np.ndarray:
    """Seeded initial weights: uniform with fan-in scaling, biases zero
    (float32, the layout of lb_mlp)."""
    r = W.rng(seed)
    parts = []
    for a, b in ((27, 64), (64, 64), (64, 3)):
        lim = math.sqrt(6.0 / a)
        parts += [r.uniform(-lim, lim, size=a * b), np.zeros(b)]
    return np.concatenate(parts).astype(np.float32)


def train(feat, labels, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 0):
    """Adam on minibatches drawn on the device (`lb_mlp_train`: seeded
    draws with replacement, cosine-decayed learning rate), with the labels
    divided by their RMS (folded back into the last layer at the end);
    returns the lb_mlp handle and the loss history (mean squared error of the
    minibatch every 50 steps and at the last, in units of the label RMS
    squared)."""
    net = lb.lb_mlp_create(initial_params(seed))
    lab = labels.cpu().numpy().astype(np.float64)
    scale = float(np.sqrt(np.mean(lab * lab)))
    scale = scale if scale > 0 else 1.0
    every = 50
    hist = np.zeros((steps - 1) // every + 2, dtype=np.float32)
    lb.lb_mlp_train(net, feat.shape[0], feat, labels, scale, min(batch, feat.shape[0]), steps, lr, seed, every, hist)
    k = (steps - 1) // every + 1 + (1 if (steps - 1) % every else 0)
    p = np.zeros(lb.lb_mlp_num_params(), dtype=np.float32)
    lb.lb_mlp_get_params(net, p)
    p[-(3 * 64 + 3):] *= scale  # W3, b3 predict the unscaled label
    lb.lb_mlp_set_params(net, p)
    return net, [float(h) for h in hist[:k]]


def predict(net, feat):
    import torch
    out = torch.empty((feat.shape[0], 3), dtype=torch.float32, device=feat.device)
    lb.lb_mlp_forward(net, feat.shape[0], feat, out)
    return out


def evaluate(net, feat, labels):
    """RMS error of the plain method (the label itself: 2 U_2x - U_1x in
    units of v0) and of the corrected velocity (label - prediction)."""
    p = predict(net, feat).cpu().numpy().astype(np.float64)
    lab = labels.cpu().numpy().astype(np.float64)
    plain = float(np.sqrt(np.mean(lab * lab)))
    corr = float(np.sqrt(np.mean((lab - p) ** 2)))
    return {"rms_plain": plain, "rms_corrected": corr, "gain": plain / corr if corr > 0 else float("inf")}


__all__ = ["pair_samples", "features", "initial_params", "train", "predict", "evaluate", "NUMBER_DENSITY"]
