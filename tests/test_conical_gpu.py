"""GPU parity with the higher-order far rules of the far-order sweep
(Section 4.2: raising the far order N_f offloads near-field work to the far
sum), through the C ABI against the FP64 oracle: the conical-product rules
and the S3-symmetric ones (about half the nodes).

The rules are generated independently on both sides (conical: host long
double in the library, 60-digit arithmetic in the oracle, equal to one unit
in the last place; symmetric: two Newton solvers in 90 digits, equal bit for
bit), so node coordinates are compared to a few units in the last place;
everything else keeps the bars of the built-in rules: lists bit-exact,
weights within 1e-12 max|C| + 1e-13 |J_T| (1e-15 |J_T| with FP64 node
quadratures), FP64 potential 1e-12, mixed and FMM potentials 1e-10.  Rules
with more than 32 nodes exercise the node-group loop of the moment-to-weight
step and the run-time node count of the correction apply.
"""
import numpy as np
import pytest

from oracle import gen_rules
from oracle.oracle import Oracle
from paper_2205_04401_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# C_N of Table "C_N values" for the far orders of the sweep
CN_TABLE = {12: 12.0, 20: 6.8, 25: 3.0, 30: 2.5, 40: 2.0, 50: 1.0}


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
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return np.max(np.abs(u - ref), axis=1) / np.max(np.abs(ref), axis=1)


def run(vp, ctx, mesh, rule, c_far, f, extra=None, node_targets=True, fp64_weights=False, precisions=(0, 1, 3)):
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
    txy = None if extra is None else torch.from_numpy(np.ascontiguousarray(extra)).cuda()
    nf = vp.nearfield_build(ctx, m, node_targets=node_targets, txy=txy, c_far=c_far, fp64_weights=fp64_weights)
    y, w = vp.mesh_nodes(m)
    row, ptri, kind, tself = vp.nf_lists(nf)
    out = dict(y=y.cpu().numpy(), w=w.cpu().numpy(), row=row.cpu().numpy(), ptri=ptri.cpu().numpy(),
               kind=kind.cpu().numpy(), tself=tself.cpu().numpy(), C=vp.nf_weights(nf).cpu().numpy(),
               stats=vp.nf_stats(nf))
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    for p in precisions:
        out[f"u{p}"] = vp.potential_eval(ctx, nf, fd, precision=p).cpu().numpy()
    torch.cuda.synchronize()
    return out


def check_nodes(g, s):
    assert g["y"].shape == s["yxy"].shape
    assert np.abs(g["y"] - s["yxy"]).max() <= 4 * np.spacing(np.abs(s["yxy"]).max())
    assert np.all(np.abs(g["w"] - s["W"]) <= 4 * np.spacing(np.abs(s["W"])))


def check_lists(g, s, info):
    assert np.array_equal(g["tself"], s["tself"])
    assert np.array_equal(g["row"], info["row"])
    assert np.array_equal(g["ptri"], info["ptri"])
    assert np.array_equal(g["kind"], info["pkind"])


def check_weights(Cg, Co, J, ptri, jtol):
    scale = np.maximum(np.abs(Co).max(axis=1), 1e-300)
    err = np.abs(Cg - Co).max(axis=1)
    bad = err > 1e-12 * scale + jtol * J[ptri]
    assert not bad.any(), (int(bad.sum()), float((err / scale).max()))


# 256-triangle disk, extra targets (interior, near vertices and edges, outside)
def far_rule(vp, tables, family, deg):
    """(oracle rule, library rule code) of a sweep rule."""
    if family == "sym":
        return f"sym{deg}", vp.VP_RULE_SYM(deg)
    return gen_rules.conical_rule(deg), vp.VP_RULE_CONICAL(deg)


@pytest.fixture(scope="module", params=[("conical", 12), ("conical", 30), ("sym", 20), ("sym", 40)],
                ids=lambda p: f"{p[0]}{p[1]}")
def disk_extra(request, vp, ctx, tables):
    family, deg = request.param
    mesh, dens = inputs.config1()
    extra = np.concatenate([inputs.random_interior_points(mesh, 300, 11),
                            mesh.vxy[::7] + 1e-9, [[1.01, 0.02], [0.0, -1.2]]])
    orule, rule = far_rule(vp, tables, family, deg)
    o = Oracle(orule, tables=tables, far_cn=CN_TABLE[deg])
    s = o.setup(mesh.vxy, mesh.tri, node_targets=False, extra=extra)
    f = np.stack([d(s["yxy"]) for d in dens])
    u_or, info = o.potential(s, f)
    g = run(vp, ctx, mesh, rule, CN_TABLE[deg], f, extra=extra, node_targets=False)
    g64 = run(vp, ctx, mesh, rule, CN_TABLE[deg], f, extra=extra, node_targets=False, fp64_weights=True,
              precisions=(0,))
    return deg, s, u_or, info, g, g64


def test_conical_nodes(disk_extra):
    _, s, _, _, g, _ = disk_extra
    check_nodes(g, s)


def test_conical_lists_bit_exact(disk_extra):
    _, s, _, info, g, _ = disk_extra
    check_lists(g, s, info)


@pytest.mark.parametrize("fp64", [False, True])
def test_conical_weights(disk_extra, fp64):
    _, s, _, info, g, g64 = disk_extra
    h = g64 if fp64 else g
    check_weights(h["C"], info["C"], s["J"], info["ptri"], 1e-15 if fp64 else 1e-13)
    assert h["stats"]["near_leaves"] == int(info["stats"][info["pkind"] == 0].sum())
    assert h["stats"]["self_panels"] == int(info["stats"][info["pkind"] == 1].sum())


def test_conical_potentials(disk_extra):
    _, _, u_or, _, g, g64 = disk_extra
    assert rel_err(g["u0"], u_or).max() <= 1e-12
    assert rel_err(g64["u0"], u_or).max() <= 1e-12
    assert rel_err(g["u1"], u_or).max() <= 1e-10
    assert rel_err(g["u3"], u_or).max() <= 1e-10


# 18-triangle disk, node targets, the degree-50 rules (676 / 453 nodes per
# triangle): own-node skipping in the far sum and the subtraction, the
# symmetric far sum and 22 / 15 node groups per pair in the moment-to-weight
# step
@pytest.fixture(scope="module", params=[("conical", 50), ("sym", 50)], ids=lambda p: f"{p[0]}{p[1]}")
def tiny_nodes(request, vp, ctx, tables):
    mesh = inputs.disk_mesh(n_b=10, n_i=5)
    family, deg = request.param
    orule, rule = far_rule(vp, tables, family, deg)
    o = Oracle(orule, tables=tables, far_cn=CN_TABLE[deg])
    s = o.setup(mesh.vxy, mesh.tri)
    y = s["yxy"]
    f = np.stack([1.0 + 0.0 * y[:, 0], np.exp(-4.0 * ((y[:, 0] - 0.2) ** 2 + (y[:, 1] + 0.1) ** 2))])
    u_or, info = o.potential(s, f)
    g = run(vp, ctx, mesh, rule, CN_TABLE[deg], f)
    one = run(vp, ctx, mesh, rule, CN_TABLE[deg], f[1:])   # d = 1: symmetric far sum
    return family, s, u_or, info, g, one


def test_high_order_node_targets(tiny_nodes):
    family, s, u_or, info, g, one = tiny_nodes
    assert s["N"] == 18 * (676 if family == "conical" else 453)
    check_nodes(g, s)
    check_lists(g, s, info)
    check_weights(g["C"], info["C"], s["J"], info["ptri"], 1e-13)
    assert rel_err(g["u0"], u_or).max() <= 1e-12
    assert rel_err(g["u1"], u_or).max() <= 1e-10
    assert rel_err(g["u3"], u_or).max() <= 1e-10
    assert rel_err(one["u1"], u_or[1:]).max() <= 1e-10


@pytest.mark.parametrize("family", ["conical", "sym"])
def test_higher_order_rules_refused_where_unsupported(vp, ctx, family):
    """The tensor-core apply takes the built-in rules only; rule codes outside
    the tabulated or generated ranges are refused at upload."""
    mesh = inputs.disk_mesh(n_b=10, n_i=5)
    code = vp.VP_RULE_CONICAL(12) if family == "conical" else vp.VP_RULE_SYM(12)
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, code)
    nf = vp.nearfield_build(ctx, m)
    with pytest.raises(vp.VPError):
        vp.nf_prepare_tc(nf)
    bad = vp.VP_RULE_CONICAL(51) if family == "conical" else vp.VP_RULE_SYM(13)
    with pytest.raises(vp.VPError):
        vp.mesh_upload(ctx, mesh.vxy, mesh.tri, bad)
    nf.release()
    m.release()


@pytest.mark.parametrize("prec", [1, 3])
def test_conical_rules_in_a_batch(vp, ctx, prec):
    """Meshes on different far rules (a conical rule of degree 20 and a
    symmetric one of degree 30 beside a built-in one) in one graph-captured batch, direct (run-time node count
    in the batched apply) and with the FMM: each item equals its single
    evaluation (FMM: bit for bit; direct: to 1e-12, the FP64 parity bar: the
    batched far sum is one-sided where the single evaluation is symmetric, so
    its FP64 partial sums are added in another order)."""
    meshes = [(inputs.disk_uniform_mesh(300, 11, 2), vp.VP_RULE_CONICAL(20)),
              (inputs.lshape_mesh(400, 12, 2), 19), (inputs.disk_mesh(n_b=10, n_i=5), vp.VP_RULE_SYM(30))]
    items, refs, keep = [], [], []
    for k, (mesh, rule) in enumerate(meshes):
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
        nf = vp.nearfield_build(ctx, m, node_targets=True, c_far=CN_TABLE.get(rule % 1000, 1.0) if rule > 1000 else 1.0)
        y, _ = vp.mesh_nodes(m)
        yn = y.cpu().numpy()
        f = torch.from_numpy(np.stack([np.cos(2 * yn[:, 0] + k) * yn[:, 1] + 1.0])).cuda()
        u = torch.full((1, nf.M), float("nan"), dtype=torch.float64, device="cuda")
        items.append((nf, f, u))
        refs.append(vp.potential_eval(ctx, nf, f, precision=prec).cpu().numpy())
        keep.append(m)
    batch = vp.Batch(ctx, items, precision=prec)
    batch.launch()
    torch.cuda.synchronize()
    for (nf, f, u), ref in zip(items, refs):
        ub = u.cpu().numpy()
        if prec == 3:
            assert np.array_equal(ub, ref)
        else:
            assert rel_err(ub, ref).max() <= 1e-12
    batch.release()
    for (nf, _, _), m in zip(items, keep):
        nf.release()
        m.release()


def test_conical_rule_on_curved_disk(vp, ctx, tables):
    """A degree-12 conical far rule (49 nodes) on the curved unit disk: the
    blending-map nodes, the curved near and self weights (node-group loop of
    the FP64 curved kernels) and the closed form (|x|^2 - 1)/4 of f = 1."""
    mesh = inputs.disk_mesh()
    tri, cur = inputs.curved_boundary(mesh, [(0.0, 0.0, 1.0)])
    rng = np.random.default_rng(21)
    r = np.sqrt(rng.random(200)) * 0.999
    th = rng.random(200) * 2 * np.pi
    extra = np.concatenate([np.stack([r * np.cos(th), r * np.sin(th)], 1),
                            [[0.999999, 0.0], [0.0, -0.9999], [0.70710678, 0.70710677]]])
    o = Oracle(gen_rules.conical_rule(12), tables=tables, far_cn=CN_TABLE[12])
    s = o.setup(mesh.vxy, tri, node_targets=False, extra=extra, curves=cur)
    f = np.ones((1, s["N"]))
    u_or, info = o.potential(s, f)
    m = vp.mesh_upload_curved(ctx, mesh.vxy, tri, cur, vp.VP_RULE_CONICAL(12))
    nf = vp.nearfield_build(ctx, m, node_targets=False, txy=torch.from_numpy(extra).cuda(), c_far=CN_TABLE[12])
    y, w = vp.mesh_nodes(m)
    row, ptri, kind, tself = vp.nf_lists(nf)
    C = vp.nf_weights(nf).cpu().numpy()
    fd = torch.from_numpy(f).cuda()
    u0 = vp.potential_eval(ctx, nf, fd, precision=vp.VP_FP64).cpu().numpy()
    u1 = vp.potential_eval(ctx, nf, fd, precision=vp.VP_MIXED).cpu().numpy()
    yy = y.cpu().numpy()
    assert np.abs(yy - s["yxy"]).max() <= 16 * np.spacing(1.0)
    assert np.array_equal(tself.cpu().numpy(), s["tself"])
    assert np.array_equal(row.cpu().numpy(), info["row"]) and np.array_equal(ptri.cpu().numpy(), info["ptri"])
    check_weights(C, info["C"], s["J"], info["ptri"], 1e-13)
    assert rel_err(u0, u_or).max() <= 1e-12
    assert rel_err(u1, u_or).max() <= 1e-10
    ex = (np.sum(extra ** 2, 1) - 1) / 4
    for u in (u0[0], u1[0]):
        assert np.abs(u - ex).max() / np.abs(ex).max() <= 1e-11
    nf.release()
    m.release()
