"""Python binding of the C ABI in include/lb.h (ctypes).

The functions carry the C names and only marshal arguments: tensors and
arrays become pointers, a non-OK status becomes an ``LBError`` carrying
``lb_last_error``.  All arithmetic runs in libgb300lb.so; if the library
is missing this module raises instead of falling back to anything else.
PyTorch supplies device memory and the stream.

``Lattice`` is a small convenience wrapper that allocates outputs as torch
tensors on the lattice's device.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from .build import LIB

LB_OK, LB_ERR_ARG, LB_ERR_CUDA, LB_ERR_OOM, LB_ERR_NONFINITE, LB_ERR_STATE, LB_ERR_TIMEOUT = range(7)
LB_F64, LB_F32, LB_F16S, LB_BF16S = range(4)
LB_STOKESLET, LB_STRESSLET, LB_ROTLET, LB_COLLOID = range(4)
NQ = 19

EXPORTS = ["lb_create", "lb_destroy", "lb_last_error", "lb_set_body_force", "lb_set_walls_z",
           "lb_set_counterforce", "lb_set_colloid_aL", "lb_add_point_forces", "lb_clear_point_forces",
           "lb_num_points", "lb_set_positions", "lb_step", "lb_velocity_at", "lb_moments",
           "lb_particles", "lb_get_populations", "lb_set_populations", "lb_kernel_launches",
           "lb_synchronize", "lb_compute_aL", "lb_totals_noalloc", "lb_batch_create",
           "lb_batch_destroy", "lb_batch_last_error", "lb_batch_tune", "lb_batch_step", "lb_batch_info",
           "lb_colloid_velocity", "lb_mlp_num_params", "lb_mlp_create", "lb_mlp_destroy", "lb_mlp_last_error",
           "lb_mlp_get_params", "lb_mlp_set_params", "lb_mlp_features", "lb_mlp_forward", "lb_mlp_grad",
           "lb_mlp_train_step", "lb_set_colloid_correction", "lb_save", "lb_load",
           "lb_mlp_set_wait_limit", "lb_set_host_async", "lb_set_phase_timing", "lb_phase_times",
           "lb_batch_synchronize", "lb_batch_set_wait_limit", "lb_mlp_train"]

_lib = None


class LBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lb status {status}: {msg}")
        self.status = status


def load():
    """Load libgb300lb.so (built by ``paper_0707_1299_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with paper_0707_1299_gb300.build.build()")
    lib = ctypes.CDLL(LIB)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p
    sig = {
        "lb_create": ([ctypes.POINTER(ctypes.c_void_p), ip, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp],
                      ctypes.c_int),
        "lb_destroy": ([vp], None),
        "lb_last_error": ([vp], ctypes.c_char_p),
        "lb_set_body_force": ([vp, dp], ctypes.c_int),
        "lb_set_walls_z": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "lb_set_counterforce": ([vp, ctypes.c_int], ctypes.c_int),
        "lb_set_colloid_aL": ([vp, ctypes.c_double], ctypes.c_int),
        "lb_add_point_forces": ([vp, ctypes.c_int, dp, dp, ctypes.c_int, dp], ctypes.c_int),
        "lb_clear_point_forces": ([vp], ctypes.c_int),
        "lb_num_points": ([vp, ip], ctypes.c_int),
        "lb_set_positions": ([vp, dp], ctypes.c_int),
        "lb_step": ([vp, ctypes.c_int], ctypes.c_int),
        "lb_set_host_async": ([vp, ctypes.c_int], ctypes.c_int),
        "lb_velocity_at": ([vp, ctypes.c_int, dp, dp], ctypes.c_int),
        "lb_moments": ([vp, dp, dp, dp], ctypes.c_int),
        "lb_particles": ([vp, dp, dp], ctypes.c_int),
        "lb_get_populations": ([vp, dp], ctypes.c_int),
        "lb_set_populations": ([vp, dp], ctypes.c_int),
        "lb_kernel_launches": ([vp, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "lb_set_phase_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "lb_phase_times": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
        "lb_synchronize": ([vp], ctypes.c_int),
        "lb_save": ([vp, ctypes.c_char_p], ctypes.c_int),
        "lb_load": ([vp, ctypes.c_char_p], ctypes.c_int),
        "lb_compute_aL": ([ip, dp, dp, dp], ctypes.c_int),
        "lb_totals_noalloc": ([vp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int, dp, dp, vp], ctypes.c_int),
        "lb_colloid_velocity": ([vp, ctypes.c_int, dp, dp, dp, dp], ctypes.c_int),
        "lb_mlp_num_params": ([], ctypes.c_int),
        "lb_set_colloid_correction": ([vp, vp], ctypes.c_int),
        "lb_mlp_create": ([ctypes.POINTER(ctypes.c_void_p), vp, vp], ctypes.c_int),
        "lb_mlp_destroy": ([vp], None),
        "lb_mlp_last_error": ([vp], ctypes.c_char_p),
        "lb_mlp_get_params": ([vp, vp], ctypes.c_int),
        "lb_mlp_set_params": ([vp, vp], ctypes.c_int),
        "lb_mlp_features": ([vp, ctypes.c_longlong, vp, ip, vp], ctypes.c_int),
        "lb_mlp_forward": ([vp, ctypes.c_longlong, vp, vp], ctypes.c_int),
        "lb_mlp_set_wait_limit": ([vp, ctypes.c_longlong], ctypes.c_int),
        "lb_mlp_grad": ([vp, ctypes.c_longlong, vp, vp, vp, vp], ctypes.c_int),
        "lb_mlp_train_step": ([vp, ctypes.c_longlong, vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "lb_mlp_train": ([vp, ctypes.c_longlong, vp, vp, ctypes.c_float, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                          ctypes.c_ulonglong, ctypes.c_int, vp], ctypes.c_int),
        "lb_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), vp],
                            ctypes.c_int),
        "lb_batch_destroy": ([vp], None),
        "lb_batch_last_error": ([vp], ctypes.c_char_p),
        "lb_batch_tune": ([vp, ip], ctypes.c_int),
        "lb_batch_step": ([vp, ctypes.c_int], ctypes.c_int),
        "lb_batch_synchronize": ([vp], ctypes.c_int),
        "lb_batch_set_wait_limit": ([vp, ctypes.c_longlong], ctypes.c_int),
        "lb_batch_info": ([vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), ip,
                           ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


# ----------------------------------------------------------- marshalling
def _ptr(x):
    """Address of a float64 tensor/array (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):  # torch.Tensor
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        return x.data_ptr()
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data


def _check(ctx, status):
    if status != LB_OK:
        msg = load().lb_last_error(ctx)
        raise LBError(status, msg.decode() if msg else "")


# ----------------------------------------------------------- the C names
def lb_create(grid, tau_shear, tau_bulk, precision=LB_F32, stream=None):
    lib = load()
    out = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(None, lib.lb_create(ctypes.byref(out), g, float(tau_shear), float(tau_bulk), int(precision),
                               ctypes.c_void_p(stream)))
    return out.value


def lb_destroy(ctx):
    load().lb_destroy(ctx)


def lb_last_error(ctx):
    return load().lb_last_error(ctx).decode()


def lb_set_body_force(ctx, g):
    a = np.ascontiguousarray(g, dtype=np.float64)
    _check(ctx, load().lb_set_body_force(ctx, a.ctypes.data))


def lb_set_walls_z(ctx, z_lo, z_hi):
    _check(ctx, load().lb_set_walls_z(ctx, int(z_lo), int(z_hi)))


def lb_set_counterforce(ctx, enabled):
    _check(ctx, load().lb_set_counterforce(ctx, 1 if enabled else 0))


def lb_set_colloid_aL(ctx, a_L):
    _check(ctx, load().lb_set_colloid_aL(ctx, float(a_L)))


def lb_add_point_forces(ctx, n, pos, F, kind, param=None):
    _check(ctx, load().lb_add_point_forces(ctx, int(n), _ptr(pos), _ptr(F), int(kind), _ptr(param)))


def lb_clear_point_forces(ctx):
    _check(ctx, load().lb_clear_point_forces(ctx))


def lb_num_points(ctx):
    n = ctypes.c_int()
    _check(ctx, load().lb_num_points(ctx, ctypes.byref(n)))
    return n.value


def lb_set_positions(ctx, pos):
    _check(ctx, load().lb_set_positions(ctx, _ptr(pos)))


def lb_step(ctx, nsteps):
    _check(ctx, load().lb_step(ctx, int(nsteps)))


def lb_set_host_async(ctx, on):
    _check(ctx, load().lb_set_host_async(ctx, int(bool(on))))


def lb_velocity_at(ctx, n, pos, v_out):
    _check(ctx, load().lb_velocity_at(ctx, int(n), _ptr(pos), _ptr(v_out)))


def lb_moments(ctx, rho, u, totals):
    _check(ctx, load().lb_moments(ctx, _ptr(rho), _ptr(u), _ptr(totals)))


def lb_particles(ctx, pos_out, f_out):
    _check(ctx, load().lb_particles(ctx, _ptr(pos_out), _ptr(f_out)))


def lb_get_populations(ctx, df):
    _check(ctx, load().lb_get_populations(ctx, _ptr(df)))


def lb_set_populations(ctx, df):
    _check(ctx, load().lb_set_populations(ctx, _ptr(df)))


def lb_kernel_launches(ctx):
    n = ctypes.c_longlong()
    _check(ctx, load().lb_kernel_launches(ctx, ctypes.byref(n)))
    return n.value


PHASES = ("spread", "collide", "points", "sort", "correction")


def lb_set_phase_timing(ctx, on):
    _check(ctx, load().lb_set_phase_timing(ctx, int(bool(on))))


def lb_phase_times(ctx):
    """{phase: (total ms, occurrences)} since the last call (waits for the stream)."""
    ms = (ctypes.c_double * 5)()
    cnt = (ctypes.c_longlong * 5)()
    _check(ctx, load().lb_phase_times(ctx, ms, cnt))
    return {name: (ms[k], cnt[k]) for k, name in enumerate(PHASES)}


def lb_synchronize(ctx):
    _check(ctx, load().lb_synchronize(ctx))


def lb_save(ctx, path):
    _check(ctx, load().lb_save(ctx, os.fsencode(path)))


def lb_load(ctx, path):
    _check(ctx, load().lb_load(ctx, os.fsencode(path)))


def lb_compute_aL(grid, R, direction=None):
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    r = np.ascontiguousarray(R, dtype=np.float64)
    d = None if direction is None else np.ascontiguousarray(direction, dtype=np.float64)
    out = np.zeros(1)
    _check(None, load().lb_compute_aL(g, r.ctypes.data, None if d is None else d.ctypes.data, out.ctypes.data))
    return float(out[0])


def lb_totals_noalloc(df, precision, grid, z_lo, z_hi, F, totals, stream=None):
    """Totals of a caller-owned device population array without any device
    allocation (see include/lb.h).  df: contiguous CUDA tensor of the
    storage type of `precision` (float64, float32, float16 holding df * 2^20,
    bfloat16) with at least 19 * nx * ny * nz elements; totals: contiguous
    CUDA float64 tensor of at least 4 elements; F: None or 3 numbers.  The
    C call trusts its pointers, so they are checked here: a host array or a
    short buffer would make its kernels read or write out of bounds."""
    import torch
    storage = {LB_F64: torch.float64, LB_F32: torch.float32, LB_F16S: torch.float16, LB_BF16S: torch.bfloat16}
    if int(precision) not in storage:
        raise ValueError(f"lb_totals_noalloc: unknown precision {precision}")
    dims = [int(v) for v in grid]
    if len(dims) != 3 or min(dims) < 1:
        raise ValueError("lb_totals_noalloc: grid must be three sizes >= 1")
    V = dims[0] * dims[1] * dims[2]
    if not isinstance(df, torch.Tensor) or not df.is_cuda or not df.is_contiguous():
        raise TypeError("lb_totals_noalloc: df must be a contiguous CUDA tensor")
    if df.dtype != storage[int(precision)]:
        raise TypeError(f"lb_totals_noalloc: df is {df.dtype}, the format stores {storage[int(precision)]}")
    if df.numel() < NQ * V:
        raise ValueError(f"lb_totals_noalloc: df holds {df.numel()} elements, the grid needs {NQ * V}")
    if (not isinstance(totals, torch.Tensor) or not totals.is_cuda or totals.dtype != torch.float64
            or not totals.is_contiguous() or totals.numel() < 4):
        raise TypeError("lb_totals_noalloc: totals must be a contiguous CUDA float64 tensor of >= 4 elements")
    if totals.device != df.device:
        raise ValueError("lb_totals_noalloc: df and totals are on different devices")
    f = None
    if F is not None:
        f = np.ascontiguousarray(F, dtype=np.float64).ravel()
        if f.shape != (3,):
            raise ValueError("lb_totals_noalloc: F must hold exactly 3 numbers")
    g = (ctypes.c_int * 3)(*dims)
    if stream is None:
        stream = torch.cuda.current_stream(df.device).cuda_stream
    with torch.cuda.device(df.device):  # the C call works on the current device
        status = load().lb_totals_noalloc(df.data_ptr(), int(precision), g, int(z_lo), int(z_hi),
                                          None if f is None else f.ctypes.data, totals.data_ptr(),
                                          ctypes.c_void_p(stream))
    if status != LB_OK:
        raise LBError(status, "lb_totals_noalloc failed")


def lb_colloid_velocity(ctx, n, pos, F, radius, U_out):
    _check(ctx, load().lb_colloid_velocity(ctx, int(n), _ptr(pos), _ptr(F), _ptr(radius), _ptr(U_out)))


# ---------------------------------------------------------- learned part
def _addr(x):
    """Address of a tensor/array of any dtype (device or host)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    assert isinstance(x, np.ndarray) and x.flags["C_CONTIGUOUS"]
    return x.ctypes.data


def _mcheck(net, status):
    if status != LB_OK:
        msg = load().lb_mlp_last_error(net)
        raise LBError(status, msg.decode() if msg else "")


def lb_set_colloid_correction(ctx, net):
    _check(ctx, load().lb_set_colloid_correction(ctx, net))


def lb_mlp_num_params():
    return load().lb_mlp_num_params()


def lb_mlp_create(init_params, stream=None):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    _mcheck(None, load().lb_mlp_create(ctypes.byref(out), _addr(init_params), ctypes.c_void_p(stream)))
    return out.value


def lb_mlp_destroy(net):
    load().lb_mlp_destroy(net)


def lb_mlp_last_error(net):
    return load().lb_mlp_last_error(net).decode()


def lb_mlp_get_params(net, out):
    _mcheck(net, load().lb_mlp_get_params(net, _addr(out)))


def lb_mlp_set_params(net, params):
    _mcheck(net, load().lb_mlp_set_params(net, _addr(params)))


def lb_mlp_features(net, n, pos, box, feat):
    b = (ctypes.c_int * 3)(*[int(v) for v in box])
    _mcheck(net, load().lb_mlp_features(net, int(n), _addr(pos), b, _addr(feat)))


def lb_mlp_forward(net, n, feat, out):
    _mcheck(net, load().lb_mlp_forward(net, int(n), _addr(feat), _addr(out)))


def lb_mlp_set_wait_limit(net, polls):
    _mcheck(net, load().lb_mlp_set_wait_limit(net, int(polls)))


def lb_mlp_grad(net, n, feat, target, grad=None, sse=None):
    _mcheck(net, load().lb_mlp_grad(net, int(n), _addr(feat), _addr(target), _addr(grad), _addr(sse)))


def lb_mlp_train_step(net, n, feat, target, lr, sse=None):
    _mcheck(net, load().lb_mlp_train_step(net, int(n), _addr(feat), _addr(target), float(lr), _addr(sse)))


def lb_mlp_train(net, n, feat, target, target_scale, batch, steps, lr, seed=0, loss_every=50, loss=None):
    _mcheck(net, load().lb_mlp_train(net, int(n), _addr(feat), _addr(target), float(target_scale), int(batch),
                                     int(steps), float(lr), int(seed) & (2 ** 64 - 1), int(loss_every), _addr(loss)))


def _bcheck(batch, status):
    if status != LB_OK:
        msg = load().lb_batch_last_error(batch)
        raise LBError(status, msg.decode() if msg else "")


def lb_batch_create(ctxs, stream=None):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    arr = (ctypes.c_void_p * len(ctxs))(*ctxs)
    out = ctypes.c_void_p()
    _bcheck(None, load().lb_batch_create(ctypes.byref(out), len(ctxs), arr, ctypes.c_void_p(stream)))
    return out.value


def lb_batch_destroy(batch):
    load().lb_batch_destroy(batch)


def lb_batch_last_error(batch):
    return load().lb_batch_last_error(batch).decode()


def lb_batch_tune(batch):
    n = ctypes.c_int()
    _bcheck(batch, load().lb_batch_tune(batch, ctypes.byref(n)))
    return n.value


def lb_batch_step(batch, nsteps):
    _bcheck(batch, load().lb_batch_step(batch, int(nsteps)))


def lb_batch_synchronize(batch):
    _bcheck(batch, load().lb_batch_synchronize(batch))


def lb_batch_set_wait_limit(batch, polls):
    _bcheck(batch, load().lb_batch_set_wait_limit(batch, int(polls)))


def lb_batch_info(batch):
    s, p, l = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    b = ctypes.c_int()
    _bcheck(batch, load().lb_batch_info(batch, ctypes.byref(s), ctypes.byref(p), ctypes.byref(b), ctypes.byref(l)))
    return {"sites": s.value, "points": p.value, "blocks": b.value, "launches": l.value}


# ------------------------------------------------------------- wrapper
class Lattice:
    """An lb_ctx with torch-allocated outputs on the current CUDA device."""

    def __init__(self, grid, tau_shear, tau_bulk, precision=LB_F32, stream=None):
        import torch
        self.grid = tuple(int(v) for v in grid)
        self.V = self.grid[0] * self.grid[1] * self.grid[2]
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = lb_create(self.grid, tau_shear, tau_bulk, precision, self.stream.cuda_stream)

    def close(self):
        if self.ctx:
            lb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x, shape=None):
        import torch
        t = torch.as_tensor(x, dtype=torch.float64, device=self.device).contiguous()
        return t if shape is None else t.reshape(shape)

    def set_body_force(self, g):
        lb_set_body_force(self.ctx, g)

    def set_walls_z(self, z_lo, z_hi):
        lb_set_walls_z(self.ctx, z_lo, z_hi)

    def set_counterforce(self, enabled):
        lb_set_counterforce(self.ctx, enabled)

    def set_colloid_aL(self, a_L):
        lb_set_colloid_aL(self.ctx, a_L if math.isfinite(a_L) else float("inf"))

    def add_point_forces(self, kind, pos, F, param=None):
        p = self._dev(pos, (-1, 3))
        f = self._dev(F, (-1, 3))
        prm = None if param is None else self._dev(param, (-1,))
        lb_add_point_forces(self.ctx, p.shape[0], p, f, kind, prm)

    def clear_point_forces(self):
        lb_clear_point_forces(self.ctx)

    def num_points(self):
        return lb_num_points(self.ctx)

    def set_positions(self, pos):
        lb_set_positions(self.ctx, self._dev(pos, (-1, 3)))

    def save(self, path):
        lb_save(self.ctx, path)

    def load(self, path):
        lb_load(self.ctx, path)

    def step(self, nsteps=1):
        lb_step(self.ctx, nsteps)

    def velocity_at(self, pos):
        import torch
        p = self._dev(pos, (-1, 3))
        v = torch.empty_like(p)
        lb_velocity_at(self.ctx, p.shape[0], p, v)
        return v

    def moments(self, fields=True):
        import torch
        nx, ny, nz = self.grid
        rho = torch.empty((nz, ny, nx), dtype=torch.float64, device=self.device) if fields else None
        u = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=self.device) if fields else None
        tot = torch.empty(4, dtype=torch.float64, device=self.device)
        lb_moments(self.ctx, rho, u, tot)
        return rho, u, tot

    def particles(self):
        import torch
        n = self.num_points()
        pos = torch.empty((n, 3), dtype=torch.float64, device=self.device)
        f = torch.empty((n, 3), dtype=torch.float64, device=self.device)
        if n:
            lb_particles(self.ctx, pos, f)
        return pos, f

    def get_populations(self):
        import torch
        nx, ny, nz = self.grid
        df = torch.empty((NQ, nz, ny, nx), dtype=torch.float64, device=self.device)
        lb_get_populations(self.ctx, df)
        return df

    def set_populations(self, df):
        lb_set_populations(self.ctx, self._dev(df))

    def kernel_launches(self):
        return lb_kernel_launches(self.ctx)

    def synchronize(self):
        lb_synchronize(self.ctx)
