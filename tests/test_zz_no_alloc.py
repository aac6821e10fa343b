"""lb_totals_noalloc -- the totals reduction for callers that cannot allocate
device memory (their memory is owned by their own pool or arena, or they
cannot afford cudaFree's device-wide wait or a mid-run out-of-memory) --
must give the same totals as lb_moments, the call that uses the context's
own scratch buffers, on two calls in a row (its static scratch keeps the
previous call's contents)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_totals_noalloc_matches_lb_moments(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0707_1299_gb300 import build, lb
    from paper_0707_1299_gb300 import workloads as W
    build.build()
    lb.load()
    torch.cuda.set_device(0)
    pid = lb.LB_F64 if prec == "f64" else lb.LB_F32
    grid = (45, 19, 23)
    g = lb.Lattice(grid, 0.6, 0.8, pid)
    g.set_body_force([2e-6, -1e-6, 5e-7])
    g.set_walls_z(0, 22)
    df0 = W.random_state(grid, 5, amp=1e-4)
    df0[:, 0] = 0.0
    df0[:, 22] = 0.0
    g.set_populations(df0)
    g.step(7)
    _, _, ref = g.moments(fields=False)
    ref = ref.cpu().numpy()
    pops = g.get_populations()              # float64 copy of the stored state
    raw = pops if prec == "f64" else pops.float().contiguous()   # exact for float storage
    scale = max(1.0, np.abs(ref[1:]).max())
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        lb.lb_totals_noalloc(raw, pid, grid, 0, 22, [2e-6, -1e-6, 5e-7], out)
        torch.cuda.synchronize()
        t = out.cpu().numpy()
        assert abs(t[0] / ref[0] - 1) < TOL[prec]
        assert np.abs(t[1:] - ref[1:]).max() <= TOL[prec] * np.abs(ref[1:]).max()
    g.close()
