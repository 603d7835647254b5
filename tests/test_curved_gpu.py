"""GPU parity for curved boundary elements (Section 3.1, blending map of Eq.
for:blend): the CUDA path through the C ABI against the FP64 oracle, and
against closed forms that only hold when the circle is represented exactly.

Bars:
* nodes and weights W (Theorem 3.1 with det J_rho), point location (Newton
  preimage on curved elements) and near/self lists: bit-exact;
* subdivision trees and panel counts: identical (leaf and panel totals);
* correction weights: |dC| <= 1e-12 max|C| of the pair + 1e-13 |J_T|;
* potentials: FP64 <= 1e-12, mixed <= 1e-10 per density against the oracle;
* closed forms with f = 1: unit disk (|x|^2 - 1)/4 and the annulus
  r0 < |x| < 1, (|x|^2 - 1)/4 - (r0^2/2) log|x|, to 1e-11 relative.
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
    u, ref = np.atleast_2d(u), np.atleast_2d(ref)
    return np.max(np.abs(u - ref), axis=1) / np.max(np.abs(ref), axis=1)


def ring_points(rng, n, r_lo, r_hi, gaps):
    """Points near the circles |x| = r_hi (inside) and |x| = r_lo (outside),
    at the given relative gaps, plus uniform points of the ring."""
    out = []
    for g in gaps:
        th = rng.random(n) * 2 * np.pi
        out.append(np.stack([(1 - g) * r_hi * np.cos(th), (1 - g) * r_hi * np.sin(th)], 1))
        if r_lo > 0:
            th = rng.random(n) * 2 * np.pi
            out.append(np.stack([(1 + g) * r_lo * np.cos(th), (1 + g) * r_lo * np.sin(th)], 1))
    r = np.sqrt(rng.uniform(r_lo ** 2, r_hi ** 2, n))
    th = rng.random(n) * 2 * np.pi
    out.append(np.stack([r * np.cos(th), r * np.sin(th)], 1))
    return np.ascontiguousarray(np.vstack(out))


def run_both(vp, ctx, tables, vxy, tri, cur, rule, extra, f_fns, sample=None):
    name = {16: "far16", 19: "far19"}[rule]
    o = Oracle(name, tables=tables)
    s = o.setup(vxy, tri, node_targets=True, extra=extra, curves=cur)
    f = np.ascontiguousarray(np.stack([fn(s["yxy"]) for fn in f_fns]))
    u_or, info = o.potential(s, f, targets=sample)
    mesh = vp.mesh_upload_curved(ctx, vxy, tri, cur, rule)
    nf = vp.nearfield_build(ctx, mesh, node_targets=True, txy=torch.from_numpy(extra).cuda())
    y, w = vp.mesh_nodes(mesh)
    row, ptri, kind, tself = vp.nf_lists(nf)
    fd = torch.from_numpy(f).cuda()
    g = dict(y=y.cpu().numpy(), w=w.cpu().numpy(), row=row.cpu().numpy(), ptri=ptri.cpu().numpy(),
             kind=kind.cpu().numpy(), tself=tself.cpu().numpy(), C=vp.nf_weights(nf).cpu().numpy(),
             stats=vp.nf_stats(nf), u0=vp.potential_eval(ctx, nf, fd, precision=vp.VP_FP64).cpu().numpy(),
             u1=vp.potential_eval(ctx, nf, fd, precision=vp.VP_MIXED).cpu().numpy())
    torch.cuda.synchronize()
    nf.release()
    mesh.release()
    return s, f, u_or, info, g


def check_parity(s, u_or, info, g, sample=None):
    assert np.array_equal(g["y"], s["yxy"]) and np.array_equal(g["w"], s["W"])
    assert np.array_equal(g["tself"], s["tself"])
    if sample is None:
        assert np.array_equal(g["row"], info["row"])
        assert np.array_equal(g["ptri"], info["ptri"]) and np.array_equal(g["kind"], info["pkind"])
        sel = np.arange(len(g["ptri"]))
        st = g["stats"]
        assert st["near_leaves"] == int(info["stats"][info["pkind"] == 0].sum())
        assert st["self_panels"] == int(info["stats"][info["pkind"] == 1].sum())
        assert st["depth_capped"] == info["capped"] == 0
    else:
        sel = np.concatenate([np.arange(g["row"][t], g["row"][t + 1]) for t in sample])
        assert np.array_equal(g["ptri"][sel], info["ptri"]) and np.array_equal(g["kind"][sel], info["pkind"])
    Cg, Co = g["C"][sel], info["C"]
    scale = np.maximum(np.abs(Co).max(axis=1), 1e-300)
    err = np.abs(Cg - Co).max(axis=1)
    bad = err > 1e-12 * scale + 1e-13 * s["J"][info["ptri"]]
    assert not bad.any(), (int(bad.sum()), float((err / scale).max()))
    cols = slice(None) if sample is None else sample
    assert rel_err(g["u0"][:, cols], u_or).max() <= 1e-12
    assert rel_err(g["u1"][:, cols], u_or).max() <= 1e-10


@pytest.mark.parametrize("rule", [16, 19])
def test_curved_unit_disk_parity_and_closed_form(vp, ctx, tables, rule):
    mesh = inputs.disk_mesh()
    tri, cur = inputs.curved_boundary(mesh, [(0.0, 0.0, 1.0)])
    extra = ring_points(np.random.default_rng(11), 40, 0.0, 1.0, (1e-2, 1e-4, 1e-7))
    gauss, _ = inputs.gaussian_bump(12)
    s, f, u_or, info, g = run_both(vp, ctx, tables, mesh.vxy, tri, cur, rule, extra,
                                   [lambda p: np.ones(len(p)), gauss])
    assert (s["tself"] >= 0).all()
    check_parity(s, u_or, info, g)
    # curved pairs are present among both kinds
    curved = cur["cidx"][info["ptri"]] >= 0
    assert (curved & (info["pkind"] == 1)).any() and (curved & (info["pkind"] == 0)).any()
    ex = (np.sum(s["txy"] ** 2, 1) - 1) / 4
    for u in (g["u0"][0], g["u1"][0]):
        assert np.abs(u - ex).max() / np.abs(ex).max() <= 1e-11


def test_curved_annulus_hole_side_and_closed_form(vp, ctx, tables):
    """Both circles curved; on the hole the curved side lies outside its
    chord triangle's interior side (the element is smaller than the chord
    triangle), on the outer circle inside (larger)."""
    r0 = 0.45
    circles = [(0.0, 0.0, 1.0), (0.0, 0.0, r0)]
    mesh = inputs.snap_to_circles(inputs.annulus_mesh(600, 21, r0), circles)
    tri, cur = inputs.curved_boundary(mesh, circles)
    extra = ring_points(np.random.default_rng(22), 30, r0, 1.0, (1e-2, 1e-5))
    s, f, u_or, info, g = run_both(vp, ctx, tables, mesh.vxy, tri, cur, 19, extra,
                                   [lambda p: np.ones(len(p)), inputs.gaussian_mix(mesh, 23)])
    assert (s["tself"] >= 0).all()
    check_parity(s, u_or, info, g)
    r = np.hypot(s["txy"][:, 0], s["txy"][:, 1])
    ex = (r ** 2 - 1) / 4 - 0.5 * r0 ** 2 * np.log(r)
    for u in (g["u0"][0], g["u1"][0]):
        assert np.abs(u - ex).max() / np.abs(ex).max() <= 1e-11


def test_curved_points_outside_the_domain(vp, ctx, tables):
    """Points just outside the circle (beyond the bulge) are in no element;
    points in the bulge (between chord and circle) are in the curved one."""
    mesh = inputs.disk_mesh()
    tri, cur = inputs.curved_boundary(mesh, [(0.0, 0.0, 1.0)])
    th = np.linspace(0, 2 * np.pi, 500, endpoint=False) + 0.003
    pts = np.vstack([np.stack([(1 + g) * np.cos(th), (1 + g) * np.sin(th)], 1) for g in (1e-3, 1e-8)] +
                    [np.stack([(1 - g) * np.cos(th), (1 - g) * np.sin(th)], 1) for g in (1e-3, 1e-8)])
    pts = np.ascontiguousarray(pts)
    o = Oracle("far16", tables=tables)
    tri_ccw, _, _, _ = o.nodes_curved(mesh.vxy, tri, cur)
    ref = o.locate_curved(mesh.vxy, tri_ccw, cur, pts)
    m = vp.mesh_upload_curved(ctx, mesh.vxy, tri, cur, 16)
    nf = vp.nearfield_build(ctx, m, node_targets=False, txy=torch.from_numpy(pts).cuda())
    _, _, _, tself = vp.nf_lists(nf)
    tself = tself.cpu().numpy()
    assert np.array_equal(tself, ref)
    assert (tself[:1000] < 0).all() and (tself[1000:] >= 0).all()
    assert vp.nf_stats(nf)["outside"] == 1000
    nf.release()
    m.release()


def test_curved_annulus_sampled(vp, ctx, tables):
    """A larger mesh (graded annulus, 2,400 triangles, 19-point rule) on
    sampled targets: lists and weights of the sampled rows, potentials."""
    r0 = 0.3
    circles = [(0.0, 0.0, 1.0), (0.0, 0.0, r0)]
    mesh = inputs.snap_to_circles(inputs.annulus_mesh(2400, 31, r0), circles)
    tri, cur = inputs.curved_boundary(mesh, circles)
    extra = ring_points(np.random.default_rng(32), 50, r0, 1.0, (1e-3, 1e-6))
    o = Oracle("far19", tables=tables)
    N = mesh.nt * 19
    rng = np.random.default_rng(33)
    sample = np.unique(np.concatenate([rng.choice(N, 300, replace=False), N + np.arange(len(extra))]))
    s, f, u_or, info, g = run_both(vp, ctx, tables, mesh.vxy, tri, cur, 19, extra,
                                   [inputs.gaussian_mix(mesh, 34), inputs.manufactured_sin_cos(2.0)], sample=sample)
    check_parity(s, u_or, info, g, sample=sample)


def test_curved_clockwise_rejected(vp, ctx):
    mesh = inputs.disk_mesh()
    tri, cur = inputs.curved_boundary(mesh, [(0.0, 0.0, 1.0)])
    bad = tri.copy()
    T = int(np.where(cur["cidx"] >= 0)[0][0])
    bad[T, 1], bad[T, 2] = bad[T, 2], bad[T, 1]
    with pytest.raises(vp.VPError) as e:
        vp.mesh_upload_curved(ctx, mesh.vxy, bad, cur, 16)
    assert e.value.code == -1
    c2 = {"cidx": cur["cidx"].copy(), "coef": cur["coef"]}
    c2["cidx"][0] = len(cur["coef"])
    with pytest.raises(vp.VPError):
        vp.mesh_upload_curved(ctx, mesh.vxy, tri, c2, 16)
