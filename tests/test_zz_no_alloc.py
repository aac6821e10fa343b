"""lb_totals_noalloc -- the totals reduction for callers that cannot allocate
device memory (their memory is owned by their own pool or arena, or they
cannot afford cudaFree's device-wide wait or a mid-run out-of-memory) --
must give the same totals as lb_moments, the call that uses the context's
own scratch buffers, and as the FP64 oracle on the same stored populations,
on two calls in a row (its static scratch keeps the previous call's
contents), in every storage format, with and without solid planes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# all formats are compared on the same stored values, so only the float
# arithmetic of the reduction separates them from the FP64 oracle
TOL = {"f64": 1e-12, "f32": 1e-5, "f16s": 1e-5, "bf16s": 1e-5}
F_UNIFORM = [2e-6, -1e-6, 5e-7]


def _raw(pops, prec):
    """The stored representation of the float64 populations the context
    reports (exact: they are the stored values converted)."""
    if prec == "f64":
        return pops.contiguous()
    if prec == "f32":
        return pops.float().contiguous()
    if prec == "f16s":
        return (pops * 2.0 ** 20).half().contiguous()
    return pops.bfloat16().contiguous()


@pytest.mark.parametrize("walls", [True, False], ids=["walls", "periodic"])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16s", "bf16s"])
def test_totals_noalloc_matches_lb_moments_and_oracle(prec, walls):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_0707_1299_gb300 import build, lb
    from paper_0707_1299_gb300 import workloads as W
    build.build()
    lb.load()
    oracle.build()
    torch.cuda.set_device(0)
    pid = {"f64": lb.LB_F64, "f32": lb.LB_F32, "f16s": lb.LB_F16S, "bf16s": lb.LB_BF16S}[prec]
    grid = (45, 19, 23)
    planes = (0, 22) if walls else (-1, -1)
    g = lb.Lattice(grid, 0.6, 0.8, pid)
    g.set_body_force(F_UNIFORM)
    if walls:
        g.set_walls_z(*planes)
    df0 = W.random_state(grid, 5, amp=1e-4)
    if walls:
        df0[:, 0] = 0.0
        df0[:, 22] = 0.0
    g.set_populations(df0)
    g.step(7)
    _, _, ref = g.moments(fields=False)
    ref = ref.cpu().numpy()
    pops = g.get_populations()              # float64 copy of the stored state
    raw = _raw(pops, prec)
    # the oracle's totals of the same populations (pulled with the same
    # planes, the same uniform force)
    o = oracle.OracleLB(grid, 0.6, 0.8, g=F_UNIFORM, walls=planes if walls else None, counter=False)
    o.df[...] = pops.cpu().numpy()
    want = o.observe(fields=False)["totals"]
    for _ in range(2):
        out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
        lb.lb_totals_noalloc(raw, pid, grid, planes[0], planes[1], F_UNIFORM, out)
        torch.cuda.synchronize()
        t = out.cpu().numpy()
        for r in (ref, want):
            assert abs(t[0] / r[0] - 1) < TOL[prec]
            assert np.abs(t[1:] - r[1:]).max() <= TOL[prec] * np.abs(r[1:]).max()
    g.close()


def test_totals_noalloc_binding_rejects_bad_buffers():
    """The binding checks what the C call trusts: device residence, storage
    dtype, length and the totals buffer."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0707_1299_gb300 import build, lb
    build.build()
    lb.load()
    torch.cuda.set_device(0)
    grid = (8, 4, 4)
    V = 8 * 4 * 4
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    good = torch.zeros(19 * V, dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        lb.lb_totals_noalloc(good.cpu(), lb.LB_F32, grid, -1, -1, None, out)
    with pytest.raises(TypeError):
        lb.lb_totals_noalloc(good.double(), lb.LB_F32, grid, -1, -1, None, out)
    with pytest.raises(ValueError):
        lb.lb_totals_noalloc(good[: 19 * V - 1], lb.LB_F32, grid, -1, -1, None, out)
    with pytest.raises(TypeError):
        lb.lb_totals_noalloc(good, lb.LB_F32, grid, -1, -1, None, out.cpu())
    with pytest.raises(ValueError):
        lb.lb_totals_noalloc(good, lb.LB_F32, grid, -1, -1, [1.0, 2.0], out)
    lb.lb_totals_noalloc(good, lb.LB_F32, grid, -1, -1, None, out)
    torch.cuda.synchronize()
    assert out.cpu().numpy()[0] == V and not out.cpu().numpy()[1:].any()
