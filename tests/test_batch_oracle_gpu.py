"""Batched evaluation (persistent far-sum launch, CUDA graph, autotuned tile)
against the FP64 oracle, item by item (Section 3.6's far sum plus
corrections), and the symmetric far sum above its scratch cap.

Bars: FP64 path <= 1e-12, mixed path <= 1e-10 per density against the
oracle on sampled targets; results of the batched far sum identical, bit for
bit, whatever targets-per-thread tile it runs with (each target's sources
are summed in the same order); the symmetric far sum cut into bands matches
the oracle and the single-band result.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2205_04401_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04401_gb300 import vp as _vp
    return _vp


def rel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return float((np.abs(u - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


@pytest.fixture(scope="module")
def batch_items(vp, tables):
    """Uneven items: the 256-triangle disk (16-node rule, every target
    checked), an L-shape, an annulus and a 12,288-triangle star large enough
    that the persistent kernel takes several work units per SM; 1, 2, 5 and
    11 densities (chunk widths 1, 2, 4 + 1, 8 + 2 + 1)."""
    ctx = vp.Context(0)
    specs = [("disk", inputs.config1()[0], 16, 1), ("lshape", inputs.lshape_mesh(900, 7, 2), 19, 2),
             ("annulus", inputs.annulus_mesh(1500, 8, 0.4, 2), 19, 5),
             ("star", inputs.star_mesh(n_tri=12288, seed=301, relax_iters=2), 19, 11)]
    items = []
    rng = np.random.default_rng(304)
    for name, mesh, rule, d in specs:
        o = Oracle("far16" if rule == 16 else "far19", tables=tables)
        s = o.setup(mesh.vxy, mesh.tri)
        fs = [inputs.gaussian_mix(mesh, 310 + k) for k in range(d - 1)] + [inputs.manufactured_sin_cos(2.0)]
        f = np.ascontiguousarray(np.stack([fn(s["yxy"]) for fn in fs]))
        sample = np.arange(s["N"]) if s["N"] <= 4096 else np.sort(rng.choice(s["N"], 160, replace=False))
        u_or, _ = o.potential(s, f, targets=sample)
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
        nf = vp.nearfield_build(ctx, m, node_targets=True)
        items.append(dict(name=name, mesh=m, nf=nf, f=torch.from_numpy(f).cuda(), sample=sample, u_or=u_or))
    yield ctx, items
    for it in items:
        it["nf"].release()
        it["mesh"].release()
    ctx.close()


def _run_batch(vp, ctx, items, prec):
    outs = [torch.full((it["f"].shape[0], it["nf"].M), float("nan"), dtype=torch.float64, device="cuda")
            for it in items]
    b = vp.Batch(ctx, [(it["nf"], it["f"], u) for it, u in zip(items, outs)], precision=prec)
    b.launch()
    torch.cuda.synchronize()
    info = b.info()
    b.release()
    return [u.cpu().numpy() for u in outs], info


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-10)])
def test_batch_items_against_oracle(vp, batch_items, prec, tol):
    ctx, items = batch_items
    outs, info = _run_batch(vp, ctx, items, prec)
    for it, u in zip(items, outs):
        assert np.isfinite(u).all(), it["name"]
        assert rel(u[:, it["sample"]], it["u_or"]) <= tol, it["name"]
    if prec == 1:
        # the large item alone: several persistent work units per SM
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        tpt = info[1][0]
        star = items[-1]
        assert tpt in (1, 2, 4)
        assert (star["nf"].M + 128 * tpt - 1) // (128 * tpt) >= 2 * sms


def test_batch_tile_is_result_neutral(vp, tables):
    """The autotuner's tile and every fixed tile give the same results, bit
    for bit (a fresh context, so that the autotuner runs)."""
    ctx = vp.Context(0)
    mesh = inputs.lobed_mesh(3000, 41, 4, 0.2, 2)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 19)
    nf = vp.nearfield_build(ctx, m, node_targets=True)
    y, _ = vp.mesh_nodes(m)
    yn = y.cpu().numpy()
    f = torch.from_numpy(np.stack([inputs.gaussian_mix(mesh, 42 + k)(yn) for k in range(3)])).cuda()
    items = [dict(nf=nf, f=f[:1].contiguous()), dict(nf=nf, f=f[1:3].contiguous())]
    auto, info = _run_batch(vp, ctx, items, 1)
    assert info[1][0] in (1, 2, 4) and info[2][0] in (1, 2, 4)
    for tpt in (1, 2, 4):
        for w in (1, 2):
            ctx.set_batch_tile(w, tpt)
        fixed, finfo = _run_batch(vp, ctx, items, 1)
        assert finfo[1][0] == tpt and finfo[2][0] == tpt
        for a, b in zip(auto, fixed):
            assert np.array_equal(a, b)
    with pytest.raises(vp.VPError):
        ctx.set_batch_tile(3, 2)
    nf.release()
    m.release()
    ctx.close()


def test_symmetric_far_sum_above_the_scratch_cap(vp, tables):
    """A 12,288-triangle star (233,472 nodes): its symmetric far sum needs
    N^2/1024 = 53 M column values, above the default cap of 256 MiB (33.5 M),
    so it runs in bands.  Against the oracle on sampled nodes (mixed bar),
    against a one-band run (a cap above the whole column layout) and a
    many-band run (1 MiB cap: one tile per band) to rounding, and the
    context's workspace stays near the cap instead of growing with N^2."""
    mesh = inputs.star_mesh(n_tri=12288, seed=301, relax_iters=2)
    o = Oracle("far19", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri)
    f = np.stack([inputs.gaussian_mix(mesh, 320)(s["yxy"])])
    sample = np.sort(np.random.default_rng(321).choice(s["N"], 200, replace=False))
    u_or, _ = o.potential(s, f, targets=sample)
    N = s["N"]
    res = {}
    for cap in (256 << 20, 1 << 20, 1 << 30):
        ctx = vp.Context(0)
        ctx.set_far_sym_cap(cap)
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 19)
        nf = vp.nearfield_build(ctx, m, node_targets=True)
        u = vp.potential_eval(ctx, nf, torch.from_numpy(f).cuda(), precision=vp.VP_MIXED).cpu().numpy()
        res[cap] = (u, ctx.memory()["workspace_bytes"])
        nf.release()
        m.release()
        ctx.close()
    u_def, ws_def = res[256 << 20]
    assert rel(u_def[:, sample], u_or) <= 1e-10
    for cap in (1 << 20, 1 << 30):
        assert rel(res[cap][0], u_def) <= 1e-13
    assert N * N // 1024 * 8 > (256 << 20)                 # above the cap: more than one band
    assert ws_def <= 1.25 * (256 << 20) + 64 * N + (8 << 20)
    assert res[1 << 30][1] > ws_def                         # one band holds every column
