"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bars (stated per result):
* nodes, point location and near/self lists: bit-exact (integer output of
  FP64 predicates evaluated without fused multiply-add on both sides);
* FP64 potential: max_t |u - u_ref| / max_t |u_ref| <= 1e-12 per density;
* mixed potential (compensated FP32 far sum): <= 1e-10 per density;
* correction weights: |dC| <= 1e-12 max|C| of the pair plus 1e-15 |J_T|
  with FP64 node quadratures (VP_NF_FP64_WEIGHTS), plus 1e-13 |J_T| with the
  default float-float ones (~2^-48 per operation): an order of magnitude
  below the method's own per-pair quadrature error, eps |J_T| with
  eps = 1e-12 (Eq. precise_far, Section 4.1).  Same subdivision trees on
  both sides (identical leaf and panel counts), so only rounding differs.
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


def rel_err(u, ref):
    u = np.atleast_2d(u)
    ref = np.atleast_2d(ref)
    return np.max(np.abs(u - ref), axis=1) / np.max(np.abs(ref), axis=1)


def gpu_run(vp, ctx, vxy, tri, rule, extra=None, node_targets=True, f=None, precisions=(0,), fp64_weights=False):
    mesh = vp.mesh_upload(ctx, vxy, tri, rule)
    txy = None if extra is None or len(extra) == 0 else torch.from_numpy(np.ascontiguousarray(extra)).cuda()
    nf = vp.nearfield_build(ctx, mesh, node_targets=node_targets, txy=txy, fp64_weights=fp64_weights)
    y, w = vp.mesh_nodes(mesh)
    row, ptri, kind, tself = vp.nf_lists(nf)
    C = vp.nf_weights(nf)
    out = dict(mesh=mesh, nf=nf, y=y.cpu().numpy(), w=w.cpu().numpy(), row=row.cpu().numpy(),
               ptri=ptri.cpu().numpy(), kind=kind.cpu().numpy(), tself=tself.cpu().numpy(), C=C.cpu().numpy(),
               stats=vp.nf_stats(nf))
    if f is not None:
        fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        for p in precisions:
            out[f"u{p}"] = vp.potential_eval(ctx, nf, fd, precision=p).cpu().numpy()
    torch.cuda.synchronize()
    return out


def compare_weights(Cg, Co, J, ptri, jtol=1e-13):
    scale = np.maximum(np.abs(Co).max(axis=1), 1e-300)
    err = np.abs(Cg - Co).max(axis=1)
    bound = 1e-12 * scale + jtol * J[ptri]
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float((err / scale).max()))


# ------------------------------------------------------------------ config 1
@pytest.fixture(scope="module")
def disk(vp, ctx, tables):
    mesh, dens = inputs.config1()
    o = Oracle("far16", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri)
    f = np.stack([d(s["yxy"]) for d in dens])
    u_or, info = o.potential(s, f)
    g = gpu_run(vp, ctx, mesh.vxy, mesh.tri, 16, f=f, precisions=(0, 1))
    g64 = gpu_run(vp, ctx, mesh.vxy, mesh.tri, 16, f=f, precisions=(0,), fp64_weights=True)
    g["fp64_weights"] = g64
    return s, f, u_or, info, g


def test_config1_nodes_bit_exact(disk):
    s, _, _, _, g = disk
    assert np.array_equal(g["y"], s["yxy"]) and np.array_equal(g["w"], s["W"])


def test_config1_lists_bit_exact(disk):
    s, _, _, info, g = disk
    assert np.array_equal(g["tself"], s["tself"])
    assert np.array_equal(g["row"], info["row"])
    assert np.array_equal(g["ptri"], info["ptri"])
    assert np.array_equal(g["kind"], info["pkind"])


@pytest.mark.parametrize("fp64", [False, True])
def test_config1_weights(disk, fp64):
    s, _, u_or, info, g = disk
    if fp64:
        g = g["fp64_weights"]
        assert rel_err(g["u0"], u_or).max() <= 1e-12
    compare_weights(g["C"], info["C"], s["J"], info["ptri"], jtol=1e-15 if fp64 else 1e-13)
    st = g["stats"]
    assert st["near_leaves"] == int(info["stats"][info["pkind"] == 0].sum())
    assert st["self_panels"] == int(info["stats"][info["pkind"] == 1].sum())
    assert st["depth_capped"] == 0


def test_config1_potential_fp64(disk):
    _, _, u_or, _, g = disk
    assert rel_err(g["u0"], u_or).max() <= 1e-12


def test_config1_potential_mixed(disk):
    _, _, u_or, _, g = disk
    assert rel_err(g["u1"], u_or).max() <= 1e-10


# ------------------------------------------------- graded star, 19-pt rule
@pytest.fixture(scope="module")
def star(vp, ctx, tables):
    mesh = inputs.star_mesh(n_tri=2048, seed=77, relax_iters=6)
    extra = inputs.random_interior_points(mesh, 300, 78)
    o = Oracle("far19", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    fs = [inputs.gaussian_mix(mesh, 79), inputs.manufactured_sin_cos(3.0), lambda p: np.ones(len(p))]
    f = np.stack([d(s["yxy"]) for d in fs])
    rng = np.random.default_rng(80)
    sample = np.unique(np.concatenate([rng.choice(s["N"], 500, replace=False), s["N"] + np.arange(len(extra))]))
    u_or, info = o.potential(s, f, targets=sample)
    row_all, ptri_all, kind_all = o.lists(s["vxy"], s["tri"], s["J"], s["txy"], s["tself"])
    g = gpu_run(vp, ctx, mesh.vxy, mesh.tri, 19, extra=extra, f=f, precisions=(0, 1))
    return s, f, sample, u_or, info, (row_all, ptri_all, kind_all), g


def test_star_lists_bit_exact(star):
    s, _, _, _, _, (row, ptri, kind), g = star
    assert np.array_equal(g["tself"], s["tself"])
    assert np.array_equal(g["row"], row) and np.array_equal(g["ptri"], ptri) and np.array_equal(g["kind"], kind)


def test_star_weights_sampled(star):
    s, _, sample, _, info, _, g = star
    rows = [np.arange(g["row"][t], g["row"][t + 1]) for t in sample]
    sel = np.concatenate(rows)
    compare_weights(g["C"][sel], info["C"], s["J"], info["ptri"])


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-10)])
def test_star_potential_sampled(star, prec, tol):
    _, _, sample, u_or, _, _, g = star
    assert rel_err(g[f"u{prec}"][:, sample], u_or).max() <= tol


# ----------------------------------------------------------------- edge cases
def test_single_triangle_with_outside_edge_and_vertex_targets(vp, ctx, tables):
    vxy = np.array([[0.0, 0.0], [0.3, 0.05], [0.1, 0.25]])
    tri = np.array([[0, 2, 1]], np.int32)          # clockwise on purpose
    extra = np.array([[0.12, 0.1], [0.5, 0.5], [0.15, 0.025], [0.0, 0.0], [-0.02, 0.01], [2.0, -1.0]])
    o = Oracle("far19", tables=tables)
    s = o.setup(vxy, tri, node_targets=True, extra=extra)
    f = np.stack([np.ones(s["N"]), np.cos(3 * s["yxy"][:, 0]) * s["yxy"][:, 1]])
    u_or, info = o.potential(s, f)
    g = gpu_run(vp, ctx, vxy, tri, 19, extra=extra, f=f)
    assert np.array_equal(g["tself"], s["tself"])
    assert np.array_equal(g["row"], info["row"]) and np.array_equal(g["ptri"], info["ptri"])
    assert g["stats"]["outside"] == int((s["tself"] < 0).sum()) >= 3
    compare_weights(g["C"], info["C"], s["J"], info["ptri"])
    assert rel_err(g["u0"], u_or).max() <= 1e-12
    assert g["stats"]["depth_capped"] == info["capped"]


def test_many_densities_and_extra_only(vp, ctx, tables, cfg1):
    """d = 11 exercises the density chunking (8 + 2 + 1); targets are only
    extra points (node_targets = False)."""
    mesh, _ = cfg1
    extra = inputs.random_interior_points(mesh, 333, 5)
    o = Oracle("far16", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=False, extra=extra)
    rng = np.random.default_rng(6)
    f = rng.normal(size=(11, s["N"]))
    u_or, _ = o.potential(s, f)
    g = gpu_run(vp, ctx, mesh.vxy, mesh.tri, 16, extra=extra, node_targets=False, f=f, precisions=(0, 1))
    assert rel_err(g["u0"], u_or).max() <= 1e-12
    assert rel_err(g["u1"], u_or).max() <= 1e-10


def test_forty_densities_on_the_star_mesh(vp, ctx, tables, star):
    """d = 40 takes the densities-across-lanes correction kernel (d >= 16):
    the oracle on sampled targets, and each density evaluated alone (which
    takes the entry-parallel kernel) to the FP64 bar."""
    s, _, sample, _, _, _, g = star
    mesh = inputs.star_mesh(n_tri=2048, seed=77, relax_iters=6)
    fs = [inputs.gaussian_mix(mesh, 900 + i) for i in range(32)]
    fs += [inputs.manufactured_sin_cos(float(k)) for k in range(1, 9)]
    f = np.ascontiguousarray(np.stack([fn(s["yxy"]) for fn in fs]))
    o = Oracle("far19", tables=tables)
    sub = sample[::4]
    u_or, _ = o.potential(s, f, targets=sub)
    fd = torch.from_numpy(f).cuda()
    for prec, tol in ((0, 1e-12), (1, 1e-10)):
        u = vp.potential_eval(ctx, g["nf"], fd, precision=prec).cpu().numpy()
        assert rel_err(u[:, sub], u_or).max() <= tol
        for k in (0, 17, 39):
            # alone, a mixed density takes the symmetric far sum, which groups
            # the float-float partial sums differently: rounding differences
            # of order 2^-41 sum|q log r^2| / max|u| (the far logarithm's
            # unnormalised tail leaves its products 41 bits), far below the
            # 1e-10 bar
            alone = vp.potential_eval(ctx, g["nf"], fd[k:k + 1].contiguous(), precision=prec).cpu().numpy()
            assert rel_err(u[k:k + 1], alone).max() <= (1e-13 if prec == 0 else 1e-11)


@pytest.mark.parametrize("which", ["star", "lshape"])
def test_symmetric_far_sum_single_density(vp, ctx, tables, star, which):
    """One density with node targets takes the symmetric far sum (each pair
    of nodes in different tiles evaluated once, used both ways): equal to
    the one-sided batch kernel within the FP64 parity bar (the same pair
    values summed in another order) and to the oracle within the mixed bar.  The L-shape has N = 13,300 nodes (ragged last tile) and
    extra targets."""
    if which == "star":
        s, f3, sample, u_or3, _, _, g = star
        f = f3[:1]
        u_or = u_or3[:1]
        nf = g["nf"]
    else:
        mesh = inputs.lshape_mesh(700, 91, relax_iters=2)
        extra = inputs.random_interior_points(mesh, 257, 92)
        o = Oracle("far19", tables=tables)
        s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
        f = np.stack([inputs.gaussian_mix(mesh, 93)(s["yxy"])])
        sample = np.unique(np.concatenate([np.arange(0, s["N"], 97), s["N"] + np.arange(257)]))
        u_or, _ = o.potential(s, f, targets=sample)
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 19)
        nf = vp.nearfield_build(ctx, m, node_targets=True, txy=torch.from_numpy(extra).cuda())
        assert s["N"] % 512 != 0
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    u = vp.potential_eval(ctx, nf, fd, precision=1).cpu().numpy()
    ub = torch.empty((1, nf.M), dtype=torch.float64, device="cuda")
    vp.potential_eval_batch(ctx, [(nf, fd, ub)], precision=1)
    # same pair values, FP64 partial sums in another order: the FP64 parity bar
    assert rel_err(u, ub.cpu().numpy()).max() <= 1e-12
    assert rel_err(u[:, sample], u_or).max() <= 1e-10


def test_host_entry_point_matches_device(vp, ctx, disk):
    s, f, _, _, g = disk
    for p in (0, 1):
        uh = vp.potential_eval_host(ctx, g["nf"], f, precision=p)
        assert np.array_equal(uh, g[f"u{p}"])


def test_batch_matches_single(vp, ctx, disk, star):
    _, f1, _, _, g1 = disk
    _, f2, _, _, _, _, g2 = star
    items = []
    outs = []
    for g, f in ((g1, f1), (g2, f2), (g1, f1[:1])):
        fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        u = torch.empty((f.shape[0], g["nf"].M), dtype=torch.float64, device="cuda")
        items.append((g["nf"], fd, u))
        outs.append(u)
    for prec in (0, 1):
        vp.potential_eval_batch(ctx, items, precision=prec)
        torch.cuda.synchronize()
        # the batch sums each target's sources in one pass where a single
        # evaluation may split them (other float-float tile boundaries):
        # rounding-level differences, held to the FP64 parity bar
        assert rel_err(outs[0].cpu().numpy(), g1[f"u{prec}"]).max() <= 1e-12
        assert rel_err(outs[1].cpu().numpy(), g2[f"u{prec}"]).max() <= 1e-12
        assert rel_err(outs[2].cpu().numpy(), g1[f"u{prec}"][:1]).max() <= 1e-12


def test_batch_graph_relaunch_with_new_densities(vp, ctx, disk, star):
    """A captured batch re-reads its density buffers at every launch."""
    _, f1, _, _, g1 = disk
    _, f2, _, _, _, _, g2 = star
    fd1 = torch.from_numpy(np.ascontiguousarray(f1)).cuda()
    fd2 = torch.from_numpy(np.ascontiguousarray(f2[:1])).cuda()
    u1 = torch.empty((f1.shape[0], g1["nf"].M), dtype=torch.float64, device="cuda")
    u2 = torch.empty((1, g2["nf"].M), dtype=torch.float64, device="cuda")
    b = vp.Batch(ctx, [(g1["nf"], fd1, u1), (g2["nf"], fd2, u2)], precision=1)
    b.launch()
    torch.cuda.synchronize()
    a1 = u1.cpu().numpy().copy()
    assert rel_err(a1, g1["u1"]).max() <= 1e-12
    fd1.mul_(2.0)                      # new densities in place, same buffers
    b.launch()
    torch.cuda.synchronize()
    assert rel_err(u1.cpu().numpy(), 2.0 * a1).max() <= 1e-13
    assert rel_err(u2.cpu().numpy(), g2["u1"][:1]).max() <= 1e-12
    b.release()


def test_errors_are_reported(vp, ctx):
    with pytest.raises(vp.VPError) as e:
        vp.mesh_upload(ctx, np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0]]), np.array([[0, 1, 2]], np.int32))
    assert e.value.code == -2
    with pytest.raises(vp.VPError) as e:
        vp.mesh_upload(ctx, np.array([[0.0, 0.0], [1.0, np.nan], [0.0, 1.0]]), np.array([[0, 1, 2]], np.int32))
    assert e.value.code == -3
    with pytest.raises(vp.VPError) as e:
        vp.mesh_upload(ctx, np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 3]], np.int32))
    assert e.value.code == -1


@pytest.mark.parametrize("cap", [0, 1, 2])
def test_depth_cap_trees_match_oracle(vp, ctx, tables, cfg1, cap):
    """Shallow depth caps (Section 3.3's subdivision stopped at depth `cap`):
    cap 0 makes every near pair a root leaf (the root classifier's capped
    branch), caps 1 and 2 stop the traversal kernel early; the capped counts,
    leaf counts and weights match the oracle's for the same cap."""
    mesh, dens = cfg1
    o = Oracle("far16", tables=tables, depth_cap=cap)
    s = o.setup(mesh.vxy, mesh.tri)
    f = np.stack([d(s["yxy"]) for d in dens])
    u_or, info = o.potential(s, f)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, 16)
    nf = vp.nearfield_build(ctx, m, node_targets=True, depth_cap=cap)
    st = vp.nf_stats(nf)
    C = vp.nf_weights(nf).cpu().numpy()
    u = vp.potential_eval(ctx, nf, torch.from_numpy(f).cuda(), precision=0).cpu().numpy()
    assert st["depth_capped"] == info["capped"]
    if cap == 0:
        assert info["capped"] > 0
    assert st["near_leaves"] == int(info["stats"][info["pkind"] == 0].sum())
    compare_weights(C, info["C"], s["J"], info["ptri"])
    assert rel_err(u, u_or).max() <= 1e-12


@pytest.mark.parametrize("rule", [16, 19])
def test_streamed_apply_rows_across_many_tiles(vp, ctx, tables, rule):
    """The streamed apply of one density (mixed path) cuts the pairs into
    tiles of 32; a target whose row spans several tiles takes the per-tile
    slots and the fix-up kernel, a row inside one tile a single update.  At
    eps = 1e-14 the targets inside the disk have rows of 100-250 pairs, the
    ones outside rows of 0-50 (one has none): against the oracle with the
    same eps (mixed bar) and against the GPU FP64 path (FP64 bar)."""
    mesh, _ = inputs.config1()
    extra = np.array([[0.013, 0.021], [1.08, 0.02], [-0.41, 0.33], [1.6, 0.0], [3.0, 0.1], [0.0, -1.15],
                      [0.2, -0.6]])
    o = Oracle("far16" if rule == 16 else "far19", tables=tables, eps=1e-14)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=False, extra=extra)
    f = np.stack([np.exp(-((s["yxy"][:, 0] - 0.1) ** 2 + s["yxy"][:, 1] ** 2) / 0.2)])
    u_or, info = o.potential(s, f)
    rows = np.diff(info["row"])
    assert rows.max() > 96 and rows.min() == 0
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
    nf = vp.nearfield_build(ctx, m, node_targets=False, txy=torch.from_numpy(extra).cuda(), eps=1e-14)
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    u1 = vp.potential_eval(ctx, nf, fd, precision=1).cpu().numpy()
    u0 = vp.potential_eval(ctx, nf, fd, precision=0).cpu().numpy()
    assert rel_err(u0, u_or).max() <= 1e-12
    assert rel_err(u1, u_or).max() <= 1e-10
    assert rel_err(u1, u0).max() <= 1e-12
    nf.release()
    m.release()
