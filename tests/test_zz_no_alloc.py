"""vp_potential_eval_noalloc against vp_potential_eval.

The allocation-free entry point serves callers that cannot allocate device
memory while they evaluate (memory owned by another allocator, or a serving
loop that cannot take cudaMalloc's device-wide synchronisation).  It must
give the results of the allocating entry point, on two calls in a row (its
fixed scratch keeps the previous call's contents), leave the device's free
memory and the context's own workspace untouched, and refuse requests that
need more than its fixed scratch.  This file is collected last so that a run
stopping at the first failure has run every other test before it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(u, ref):
    return float((np.abs(u - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04401_gb300 import inputs, vp
    ctx = vp.Context(0)
    mesh = inputs.star_mesh(n_tri=1024, seed=91, relax_iters=4)
    extra = inputs.random_interior_points(mesh, 200, 92)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, m, node_targets=True, txy=torch.from_numpy(extra).cuda())
    y, _ = vp.mesh_nodes(m)
    yn = y.cpu().numpy()
    rng = np.random.default_rng(93)
    f = np.stack([np.exp(-((yn - c) ** 2).sum(1) / 0.1) for c in rng.uniform(-0.5, 0.5, (3, 2))])
    return vp, ctx, m, nf, torch.from_numpy(f).cuda()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_allocating_entry_point_twice(setup, prec):
    vp, ctx, m, nf, f = setup
    ref = vp.potential_eval(ctx, nf, f, precision=prec).cpu().numpy()
    for _ in range(2):
        out = torch.full((f.shape[0], nf.M), float("nan"), dtype=torch.float64, device="cuda")
        vp.potential_eval_noalloc(ctx, nf, f, precision=prec, out=out)
        u = out.cpu().numpy()
        assert np.isfinite(u).all()
        assert _rel(u, ref) <= 1e-12
    # a single density after a wider call (the scratch keeps old contents)
    out1 = vp.potential_eval_noalloc(ctx, nf, f[1:2].contiguous(), precision=prec).cpu().numpy()
    assert _rel(out1, ref[1:2]) <= 1e-12


def test_noalloc_allocates_nothing():
    """A fresh context whose first evaluations are the allocation-free ones:
    neither the device's free memory nor the context's workspace changes
    across two rounds of calls at d = 3 in FP64 and in mixed precision."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04401_gb300 import inputs, vp
    ctx = vp.Context(0)
    mesh = inputs.star_mesh(n_tri=512, seed=95, relax_iters=4)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, m, node_targets=True)
    y, _ = vp.mesh_nodes(m)
    yn = y.cpu().numpy()
    f = torch.from_numpy(np.stack([np.cos(k * yn[:, 0]) * np.exp(-yn[:, 1] ** 2) for k in (1, 2, 3)])).cuda()
    outs = {p: torch.empty((3, nf.M), dtype=torch.float64, device="cuda") for p in (vp.VP_FP64, vp.VP_MIXED)}
    torch.cuda.synchronize()
    # measured before the first call: vp_create did the set-up (module,
    # symbol address, log tables), so even the first call allocates nothing
    free0, _ = torch.cuda.mem_get_info()
    ws0 = ctx.memory()
    assert ws0["workspace_bytes"] == 0     # no allocating evaluation has run on this context
    for _ in range(2):
        for p in (vp.VP_FP64, vp.VP_MIXED):
            vp.potential_eval_noalloc(ctx, nf, f, precision=p, out=outs[p])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert ctx.memory() == ws0
    assert free1 == free0
    # and the results are those of the allocating entry point
    for p in (vp.VP_FP64, vp.VP_MIXED):
        ref = vp.potential_eval(ctx, nf, f, precision=p).cpu().numpy()
        assert _rel(outs[p].cpu().numpy(), ref) <= 1e-12
    nf.release()
    m.release()
    ctx.close()


def test_noalloc_rejects_requests_beyond_its_scratch(setup):
    vp, ctx, m, nf, f = setup
    big = torch.zeros((256, m.N), dtype=torch.float64, device="cuda")
    with pytest.raises(vp.VPError) as e:
        vp.potential_eval_noalloc(ctx, nf, big, precision=vp.VP_FP64)
    assert e.value.code == -1 and "scratch" in str(e.value)
