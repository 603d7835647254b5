"""GPU parity for interpolation over mesh elements (Section 3.5) through the
C ABI (vp_interp_*), against the oracle's interpolator, and end to end on a
staggered interpolation mesh (Section 4.3).

Bars: node coordinates within 4e-16 of the oracle's (the reference nodes are
computed independently, in long double here and numpy there); coefficients
and interpolated values within 1e-12 of the oracle's, relative to the
largest; elements of the located points identical (same exact predicates);
points outside the mesh give NaN and -1.  End to end (curved unit disk,
f = 1, staggered curved interpolation mesh): interpolated potential within
1e-12 of the oracle's interpolant of its own potential, and within 1e-10 of
(|x|^2 - 1)/4.
"""
import numpy as np
import pytest

from oracle.interp import Interpolator
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


def test_interp_parity_straight_and_curved(vp, ctx, tables):
    circ = [(0.0, 0.0, 1.0)]
    mesh = inputs.disk_mesh(stagger=True)
    tri_c, cur = inputs.curved_boundary(mesh, circ)
    o = Oracle("far16", tables=tables)
    rng = np.random.default_rng(5)
    r = np.sqrt(rng.random(800)) * 1.02
    th = rng.random(800) * 2 * np.pi
    pts = np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th)], 1))
    for N, tri, curves in ((12, mesh.tri, None), (12, tri_c, cur), (20, tri_c, cur), (3, mesh.tri, None)):
        it_o = Interpolator(o, mesh.vxy, tri, N, curves=curves)
        it_g = vp.Interp(ctx, mesh.vxy, tri, N, curves=curves)
        assert it_g.nn == it_o.nn and it_g.nt == it_o.nt
        nodes_g = it_g.nodes().cpu().numpy()
        assert np.abs(nodes_g - it_o.nodes()).max() <= 4e-16
        u = rng.normal(size=(2, it_g.n_nodes))
        cg = it_g.coeffs(torch.from_numpy(u).cuda())
        co = it_o.coeffs(u)
        assert np.abs(cg.cpu().numpy() - co).max() <= 1e-12 * np.abs(co).max()
        vg, eg = it_g.eval(cg, torch.from_numpy(pts).cuda())
        vo, eo = it_o.evaluate(co, pts)
        eg = eg.cpu().numpy()
        vg = vg.cpu().numpy()
        assert np.array_equal(eg, eo)
        inside = eo >= 0
        assert (~inside).any() and inside.any()
        assert np.isnan(vg[:, ~inside]).all()
        assert np.abs(vg[:, inside] - vo[:, inside]).max() <= 1e-12 * np.abs(vo[:, inside]).max()
        it_g.release()


@pytest.mark.parametrize("prec", [0, 1])
def test_staggered_interpolation_end_to_end(vp, ctx, tables, prec):
    circ = [(0.0, 0.0, 1.0)]
    q = inputs.disk_mesh()
    tq, cq = inputs.curved_boundary(q, circ)
    st = inputs.disk_mesh(stagger=True)
    ts, cs = inputs.curved_boundary(st, circ)
    N = 12
    it_g = vp.Interp(ctx, st.vxy, ts, N, curves=cs)
    nodes = it_g.nodes()
    mesh = vp.mesh_upload_curved(ctx, q.vxy, tq, cq, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, mesh, node_targets=False, txy=nodes)
    f = torch.ones((1, mesh.N), dtype=torch.float64, device="cuda")
    u_nodes = vp.potential_eval(ctx, nf, f, precision=prec)
    coef = it_g.coeffs(u_nodes)
    rng = np.random.default_rng(7)
    r = np.sqrt(rng.random(2000)) * (1 - 1e-9)
    th = rng.random(2000) * 2 * np.pi
    pts = np.ascontiguousarray(np.stack([r * np.cos(th), r * np.sin(th)], 1))
    ug, eg = it_g.eval(coef, torch.from_numpy(pts).cuda())
    ug = ug.cpu().numpy()[0]
    assert (eg.cpu().numpy() >= 0).all()
    ex = (np.sum(pts ** 2, 1) - 1) / 4
    assert np.abs(ug - ex).max() / np.abs(ex).max() <= 1e-10
    # the oracle's potential at the same nodes, interpolated by the oracle
    o = Oracle("far19", tables=tables)
    s = o.setup(q.vxy, tq, node_targets=False, extra=nodes.cpu().numpy(), curves=cq)
    uo, _ = o.potential(s, np.ones((1, s["N"])))
    it_o = Interpolator(o, st.vxy, ts, N, curves=cs)
    vo, _ = it_o.evaluate(it_o.coeffs(uo), pts)
    assert np.abs(ug - vo[0]).max() / np.abs(vo[0]).max() <= (1e-12 if prec == 0 else 1e-10)
    nf.release()
    mesh.release()
    it_g.release()
