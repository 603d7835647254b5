"""GPU parity of the fast multipole far sum (VP_MIXED_FMM): the far sum of
Section 3.6 by a quadtree FMM (40-term complex expansions, float-float direct
part), followed by the mixed-precision corrections.

Bars: within 1e-12 (relative to the largest |u|) of the FP64 oracle on the
unit disk (all nodes) and on sampled targets of a graded star with extra
targets, and of the GPU FP64 path; several densities at once; results
bit-identical between two evaluations (fixed summation order).
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


@pytest.fixture(scope="module")
def ctx(vp):
    return vp.Context(0)


def rel(u, ref):
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return float((np.abs(u - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


def test_fmm_disk_all_nodes(vp, ctx, tables):
    mesh, dens = inputs.config1()
    o = Oracle("far16", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri)
    f = np.stack([d(s["yxy"]) for d in dens])
    u_or, _ = o.potential(s, f)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 16)
    nf = vp.nearfield_build(ctx, m, node_targets=True)
    fd = torch.from_numpy(f).cuda()
    u = vp.potential_eval(ctx, nf, fd, precision=vp.VP_MIXED_FMM).cpu().numpy()
    assert rel(u, u_or) <= 1e-12
    u2 = vp.potential_eval(ctx, nf, fd, precision=vp.VP_MIXED_FMM).cpu().numpy()
    assert np.array_equal(u, u2)
    nf.release()
    m.release()


def test_fmm_star_with_extra_targets(vp, ctx, tables):
    mesh = inputs.star_mesh(n_tri=2048, seed=77, relax_iters=6)
    extra = inputs.random_interior_points(mesh, 300, 78)
    o = Oracle("far19", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    fs = [inputs.gaussian_mix(mesh, 79), inputs.manufactured_sin_cos(3.0), lambda p: np.ones(len(p))]
    f = np.ascontiguousarray(np.stack([fn(s["yxy"]) for fn in fs]))
    rng = np.random.default_rng(80)
    sample = np.unique(np.concatenate([rng.choice(s["N"], 400, replace=False), s["N"] + np.arange(len(extra))]))
    u_or, _ = o.potential(s, f, targets=sample)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 19)
    nf = vp.nearfield_build(ctx, m, node_targets=True, txy=torch.from_numpy(extra).cuda())
    fd = torch.from_numpy(f).cuda()
    u = vp.potential_eval(ctx, nf, fd, precision=vp.VP_MIXED_FMM).cpu().numpy()
    u64 = vp.potential_eval(ctx, nf, fd, precision=vp.VP_FP64).cpu().numpy()
    assert rel(u[:, sample], u_or) <= 1e-12
    assert rel(u, u64) <= 1e-12
    # one density at a time gives the same values
    u1 = vp.potential_eval(ctx, nf, fd[1:2].contiguous(), precision=vp.VP_MIXED_FMM).cpu().numpy()
    assert rel(u1, u[1:2]) <= 1e-14
    nf.release()
    m.release()


def test_fmm_curved_annulus_closed_form(vp, ctx):
    r0 = 0.45
    circles = [(0.0, 0.0, 1.0), (0.0, 0.0, r0)]
    mesh = inputs.snap_to_circles(inputs.annulus_mesh(1200, 41, r0), circles)
    tri, cur = inputs.curved_boundary(mesh, circles)
    m = vp.mesh_upload_curved(ctx, mesh.vxy, tri, cur, 19)
    nf = vp.nearfield_build(ctx, m, node_targets=True)
    y, _ = vp.mesh_nodes(m)
    f = torch.ones((1, m.N), dtype=torch.float64, device="cuda")
    u = vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED_FMM).cpu().numpy()[0]
    r = np.hypot(*y.cpu().numpy().T)
    ex = (r ** 2 - 1) / 4 - 0.5 * r0 ** 2 * np.log(r)
    assert np.abs(u - ex).max() / np.abs(ex).max() <= 1e-11
    nf.release()
    m.release()


def test_fmm_batch_matches_single_evaluations(vp, ctx, tables):
    """A graph-captured batch of uneven meshes with VP_MIXED_FMM gives each
    item's single VP_MIXED_FMM evaluation bit for bit (same kernels, same
    order), stays within 1e-12 of the direct mixed result, and within 1e-12
    of the FP64 oracle on sampled targets of every item."""
    meshes = [inputs.disk_uniform_mesh(600, 5, 2), inputs.lobed_mesh(1500, 6, 5, 0.25, 2),
              inputs.lshape_mesh(900, 7, 2)]
    o = Oracle("far19", tables=tables)
    rng = np.random.default_rng(95)
    items, refs = [], []
    for k, mesh in enumerate(meshes):
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 19)
        nf = vp.nearfield_build(ctx, m, node_targets=True)
        y, _ = vp.mesh_nodes(m)
        yn = y.cpu().numpy()
        d = k + 1
        fn = np.stack([inputs.gaussian_mix(mesh, 90 + 7 * k + j)(yn) for j in range(d)])
        f = torch.from_numpy(fn).cuda()
        u = torch.full((d, nf.M), float("nan"), dtype=torch.float64, device="cuda")
        s = o.setup(mesh.vxy, mesh.tri)
        sample = np.sort(rng.choice(s["N"], 150, replace=False))
        u_or, _ = o.potential(s, fn, targets=sample)
        items.append((nf, f, u))
        refs.append((vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED_FMM).cpu().numpy(),
                     vp.potential_eval(ctx, nf, f, precision=vp.VP_MIXED).cpu().numpy(), m, sample, u_or))
    batch = vp.Batch(ctx, items, precision=vp.VP_MIXED_FMM)
    for _ in range(2):
        batch.launch()
        torch.cuda.synchronize()
        for (nf, f, u), (uf, um, _, sample, u_or) in zip(items, refs):
            ub = u.cpu().numpy()
            assert np.array_equal(ub, uf)
            assert rel(ub, um) <= 1e-12
            assert rel(ub[:, sample], u_or) <= 1e-12
    batch.release()
    for (nf, _, _), ref in zip(items, refs):
        nf.release()
        ref[2].release()


def test_fmm_far_outside_targets(vp, ctx, tables):
    """Targets far outside the mesh stretch the tree's square (most leaves
    empty, the nodes in a few of them): the FMM still matches the oracle."""
    mesh, dens = inputs.config1()
    extra = np.array([[30.0, -20.0], [-25.0, 40.0], [0.3, 0.2], [1.5, 0.0], [0.999, 0.001]])
    o = Oracle("far16", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    f = np.stack([d(s["yxy"]) for d in dens])
    u_or, _ = o.potential(s, f)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 16)
    nf = vp.nearfield_build(ctx, m, node_targets=True, txy=torch.from_numpy(extra).cuda())
    u = vp.potential_eval(ctx, nf, torch.from_numpy(f).cuda(), precision=vp.VP_MIXED_FMM).cpu().numpy()
    assert rel(u, u_or) <= 1e-12
    assert np.abs(u[:, -5:] - u_or[:, -5:]).max() <= 1e-12 * np.abs(u_or).max()
    nf.release()
    m.release()
