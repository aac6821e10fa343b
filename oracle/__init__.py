"""Plain CPU oracle for the forced D3Q19 MRT lattice Boltzmann method with
off-lattice singular point forces (Nash, Adhikari & Cates).

TEST INFRASTRUCTURE.  Only ``tests/``, the package smoke check and the CPU
baseline of ``bench.py`` import this package.  It shares no code with the
CUDA library and never imports it.

Layout of the oracle:
  * ``lb_oracle.c``   -- the time stepper, one-site collision, Peskin kernel
    and lattice tables, in plain C (FP64, and a long-double self-check
    build), see its header for the step-by-step definition.
  * ``points.py``     -- expansion of stresslets and rotlets into point
    forces (Sec. III, Figs. stresslet/rotlet) and the uniform counter-force.
  * ``alattice.py``   -- the lattice offset parameter a_L of Appendix A.
  * this module       -- a small driver class around the C stepper.

Populations are stored as df[i, z, y, x] = fbar_i - w_i (rho0 = 1), i in the
D3Q19 order of ``lattice()``; vector fields as u[a, z, y, x].
"""
from __future__ import annotations

import numpy as np

from . import _lib
from .points import STOKESLET, STRESSLET, ROTLET, COLLOID, expand_points, counter_force
from .alattice import inv_aL_tensor, aL_along

NQ = 19

__all__ = ["NQ", "build", "lattice", "phi", "collide_site", "macro_site", "OracleLB",
           "STOKESLET", "STRESSLET", "ROTLET", "COLLOID", "expand_points",
           "counter_force", "inv_aL_tensor", "aL_along", "force_field", "num_threads"]


def build(force: bool = False) -> None:
    """Compile the C part of the oracle (both precisions)."""
    _lib.build(force)


def num_threads() -> int:
    """Host threads the oracle's site loops use (OpenMP)."""
    lib, _, pre = _lib.load("double")
    return int(getattr(lib, pre + "num_threads")())


def _real(precision):
    return np.float64 if precision == "double" else np.longdouble


def lattice(precision: str = "double"):
    """D3Q19 velocities c (19, 3) int and weights w (19,)."""
    lib, _, pre = _lib.load(precision)
    c = np.zeros((NQ, 3), dtype=np.int32)
    w = np.zeros(NQ, dtype=_real(precision))
    getattr(lib, pre + "lattice")(_lib.ptr(c), _lib.ptr(w, precision))
    return c, w


def phi(r, precision: str = "double"):
    """Peskin's 4-point kernel, Eq. (deltadef); vectorised over r."""
    lib, _, pre = _lib.load(precision)
    f = getattr(lib, pre + "phi")
    r = np.asarray(r, dtype=_real(precision))
    out = np.array([f(x) for x in r.ravel()], dtype=_real(precision))
    return out.reshape(r.shape)


def collide_site(df, F, tau_s, tau_b, precision: str = "double"):
    """Post-collision df* at one site (Eq. fiexp with the stress update read
    from Eq. mrtlbe); df is fbar - w."""
    lib, _, pre = _lib.load(precision)
    R = _real(precision)
    d = np.ascontiguousarray(df, dtype=R)
    Fv = np.ascontiguousarray(F, dtype=R)
    out = np.zeros(NQ, dtype=R)
    getattr(lib, pre + "collide_site")(_lib.ptr(d, precision), _lib.ptr(Fv, precision),
                                       tau_s, tau_b, _lib.ptr(out, precision))
    return out


def macro_site(df, F, precision: str = "double"):
    """(rho, v) at one site from Eq. (macrovariables2)."""
    lib, _, pre = _lib.load(precision)
    R = _real(precision)
    d = np.ascontiguousarray(df, dtype=R)
    Fv = np.ascontiguousarray(F, dtype=R)
    rho = np.zeros(1, dtype=R)
    v = np.zeros(3, dtype=R)
    getattr(lib, pre + "macro_site")(_lib.ptr(d, precision), _lib.ptr(Fv, precision),
                                     _lib.ptr(rho, precision), _lib.ptr(v, precision))
    return rho[0], v


class OracleLB:
    """A periodic (optionally z-walled) lattice advanced by the C oracle.

    n        -- (nx, ny, nz)
    tau_s    -- shear relaxation time, eta = cs^2 tau_s (rho0 = 1)
    tau_b    -- bulk relaxation time
    g        -- uniform body-force density on fluid nodes
    walls    -- (z_lo, z_hi) solid planes with halfway bounce-back, or None
    counter  -- balance the net point force with a uniform force density
    a_L      -- lattice offset parameter of the colloid update (inf = none)
    fc       -- explicit uniform force density on fluid nodes, used instead
                of the counter-force (e.g. a sub-box of a larger lattice)
    """

    def __init__(self, n, tau_s, tau_b, g=(0.0, 0.0, 0.0), walls=None, counter=True,
                 a_L=np.inf, precision: str = "double", fc=None):
        self.precision = precision
        self.R = _real(precision)
        self.n = tuple(int(v) for v in n)
        self.V = self.n[0] * self.n[1] * self.n[2]
        self.tau_s, self.tau_b = tau_s, tau_b
        self.g = np.asarray(g, dtype=np.float64)
        self.walls = walls
        self.counter = counter
        self.a_L = a_L
        self.fc = None if fc is None else np.asarray(fc, dtype=np.float64)
        self.df = np.zeros((NQ, self.n[2], self.n[1], self.n[0]), dtype=self.R)
        self.pos = np.zeros((0, 3), dtype=self.R)
        self.f = np.zeros((0, 3), dtype=self.R)
        self.mobile = np.zeros(0, dtype=np.int32)
        self.radius = np.zeros(0, dtype=self.R)

    @property
    def n_fluid(self):
        nz_fluid = self.n[2] - (0 if self.walls is None else
                                len({w for w in self.walls if 0 <= w < self.n[2]}))
        return self.n[0] * self.n[1] * nz_fluid

    def add_points(self, kind, pos, F, param=None):
        """Append points of one kind (expanded as in Sec. III)."""
        p, f, mob, rad = expand_points(kind, pos, F, param)
        self.pos = np.concatenate([self.pos, p.astype(self.R)])
        self.f = np.concatenate([self.f, f.astype(self.R)])
        self.mobile = np.concatenate([self.mobile, mob.astype(np.int32)])
        self.radius = np.concatenate([self.radius, rad.astype(self.R)])

    def _params(self):
        _, Params, _ = _lib.load(self.precision)
        p = Params()
        for a in range(3):
            p.n[a] = self.n[a]
            p.g[a] = float(self.g[a])
        if self.fc is not None:
            fc = self.fc
        else:
            fc = counter_force(self.f, self.n_fluid) if self.counter else np.zeros(3)
        for a in range(3):
            p.fc[a] = fc[a]
        p.tau_s, p.tau_b = self.tau_s, self.tau_b
        p.wall_lo, p.wall_hi = (-1, -1) if self.walls is None else self.walls
        p.a_L = self.a_L
        return p

    def step(self, nsteps: int = 1, net=None):
        """Advance nsteps.  With `net` (parameters of the correction network,
        the dict of ``mlp.unflatten``) every step first evaluates the
        network on the features of the positions at the start of the step
        (``mlp.features``, ``mlp.forward`` with bfloat16 operands) and moves
        each colloid by its Sec. IV velocity plus y |F| / (6 pi eta a)."""
        lib, _, pre = _lib.load(self.precision)
        p = self._params()
        run = getattr(lib, pre + "run")
        args = lambda y, k: (p, _lib.ptr(self.df, self.precision), len(self.mobile),
                             _lib.ptr(self.pos, self.precision), _lib.ptr(self.f, self.precision),
                             _lib.ptr(self.mobile), _lib.ptr(self.radius, self.precision),
                             _lib.ptr(y, self.precision), int(k))
        if net is None:
            if run(*args(None, nsteps)) != 0:
                raise MemoryError("oracle run failed to allocate")
            return
        from . import mlp
        for _ in range(int(nsteps)):
            y, _ = mlp.forward(net, mlp.features(np.asarray(self.pos, dtype=np.float64), self.n), bf16_round=True)
            y = np.ascontiguousarray(y, dtype=self.R)
            if run(*args(y, 1)) != 0:
                raise MemoryError("oracle run failed to allocate")

    def observe(self, qpos=None, fields=True):
        """rho (nz,ny,nx), u (3,nz,ny,nx), velocities at qpos (m,3) and
        totals [M, Px, Py, Pz] over fluid sites, at the current time."""
        lib, _, pre = _lib.load(self.precision)
        p = self._params()
        rho = np.zeros((self.n[2], self.n[1], self.n[0]), dtype=self.R) if fields else None
        u = np.zeros((3, self.n[2], self.n[1], self.n[0]), dtype=self.R) if fields else None
        q = np.zeros((0, 3), dtype=self.R) if qpos is None else np.ascontiguousarray(qpos, dtype=self.R)
        qv = np.zeros_like(q)
        tot = np.zeros(4, dtype=self.R)
        rc = getattr(lib, pre + "observe")(
            p, _lib.ptr(self.df, self.precision), len(self.mobile),
            _lib.ptr(self.pos, self.precision), _lib.ptr(self.f, self.precision),
            _lib.ptr(rho, self.precision), _lib.ptr(u, self.precision), len(q),
            _lib.ptr(q, self.precision), _lib.ptr(qv, self.precision),
            _lib.ptr(tot, self.precision))
        if rc != 0:
            raise MemoryError("oracle observe failed to allocate")
        return {"rho": rho, "u": u, "qv": qv, "totals": tot}


def force_field(n, pos, f, g=(0.0, 0.0, 0.0), fc=(0.0, 0.0, 0.0), walls=None,
                precision: str = "double"):
    """F (3, nz, ny, nx) = [fluid](g + fc) + sum_a f_a delta^P(x - R_a)."""
    lib, Params, pre = _lib.load(precision)
    R = _real(precision)
    p = Params()
    for a in range(3):
        p.n[a] = int(n[a])
        p.g[a] = float(g[a])
        p.fc[a] = float(fc[a])
    p.wall_lo, p.wall_hi = (-1, -1) if walls is None else walls
    pos = np.ascontiguousarray(pos, dtype=R).reshape(-1, 3)
    f = np.ascontiguousarray(f, dtype=R).reshape(-1, 3)
    F = np.zeros((3, n[2], n[1], n[0]), dtype=R)
    getattr(lib, pre + "force_field")(p, len(pos), _lib.ptr(pos, precision),
                                      _lib.ptr(f, precision), _lib.ptr(F, precision))
    return F
