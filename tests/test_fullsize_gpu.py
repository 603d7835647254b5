"""Parity at full size: the 16,384-triangle graded star (r = 1 + 0.3 cos 5t,
8:1 grading toward the boundary), 19-node rule (311,296 nodes), targets =
the nodes plus 10,000 uniform interior points, density a sum of four
Gaussians -- evaluated exactly as the benchmark times one step (device mesh
upload, near-field build with float-float node quadratures, mixed-precision
evaluation: symmetric float-float far sum in bands, streamed apply), and
checked against the FP64 oracle (Section 3) on sampled targets it computes
one by one.

Bars, stated per result:
* nodes and weights of all 311,296 nodes, and the containing triangle of
  all 321,296 targets: bit-exact;
* near/self lists of the sampled targets: bit-exact;
* their correction weights: the bars of the smaller parity tests (1e-12 of
  the pair's max|C| plus 1e-13 |J_T|);
* potentials: max over the sample of |u - u_ref| / max |u_ref| within 1e-10
  (mixed) and 1e-12 (FP64 path);
* over all targets: mixed within 1e-10 of the FP64 path (max norm).

The sample: 240 random nodes, 60 random interior points, both ends of
every 512-node tile boundary the symmetric sum cuts at five places, the
first and last node and interior point, and the target with the longest
near-field list.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2205_04401_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NQ = 19
TILE = 512


@pytest.fixture(scope="module")
def full(tables):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04401_gb300 import vp
    ctx = vp.Context(0)
    mesh, fun, extra = inputs.config2()
    dev = torch.device("cuda", 0)
    vxy_d = torch.from_numpy(mesh.vxy).to(dev)
    tri_d = torch.from_numpy(mesh.tri).to(dev)
    extra_d = torch.from_numpy(extra).to(dev)
    mh = vp.mesh_upload_dev(ctx, vxy_d, tri_d, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, mh, node_targets=True, txy=extra_d)
    y, w = vp.mesh_nodes(mh)
    y, w = y.cpu().numpy(), w.cpu().numpy()
    f = fun(y)[None, :]
    f_d = torch.from_numpy(np.ascontiguousarray(f)).to(dev)
    u_mixed = vp.potential_eval(ctx, nf, f_d, precision=vp.VP_MIXED).cpu().numpy()
    u_fp64 = vp.potential_eval(ctx, nf, f_d, precision=vp.VP_FP64).cpu().numpy()
    row, ptri, kind, tself = (a.cpu().numpy() for a in vp.nf_lists(nf))
    C = vp.nf_weights(nf).cpu().numpy()
    torch.cuda.synchronize()
    nf.release()
    mh.release()

    o = Oracle("far19", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    N, M = s["N"], len(s["txy"])
    assert N == mesh.nt * NQ and M == N + len(extra)
    rng = np.random.default_rng(2205)
    cuts = np.linspace(1, N // TILE - 1, 5).astype(np.int64) * TILE
    sample = np.unique(np.concatenate([
        rng.choice(N, 240, replace=False), N + rng.choice(len(extra), 60, replace=False),
        cuts - 1, cuts, [0, N - 1, N, M - 1, int(np.argmax(np.diff(row)))]]))
    fo = fun(s["yxy"])[None, :]
    u_or, info = o.potential(s, fo, targets=sample)
    return dict(s=s, y=y, w=w, row=row, ptri=ptri, kind=kind, tself=tself, C=C, u_mixed=u_mixed,
                u_fp64=u_fp64, sample=sample, u_or=u_or, info=info)


def rel(u, ref):
    return float(np.abs(u - ref).max() / np.abs(ref).max())


def test_fullsize_nodes_and_located_triangles_bit_exact(full):
    s = full["s"]
    assert np.array_equal(full["y"], s["yxy"]) and np.array_equal(full["w"], s["W"])
    assert np.array_equal(full["tself"], s["tself"])


def test_fullsize_sampled_lists_bit_exact(full):
    row, info = full["row"], full["info"]
    sel = [np.arange(row[t], row[t + 1]) for t in full["sample"]]
    assert np.array_equal(np.array([len(r) for r in sel]), np.diff(info["row"]))
    sel = np.concatenate(sel)
    assert np.array_equal(full["ptri"][sel], info["ptri"]) and np.array_equal(full["kind"][sel], info["pkind"])


def test_fullsize_sampled_weights(full):
    row, info, s = full["row"], full["info"], full["s"]
    sel = np.concatenate([np.arange(row[t], row[t + 1]) for t in full["sample"]])
    Cg, Co = full["C"][sel], info["C"]
    scale = np.maximum(np.abs(Co).max(axis=1), 1e-300)
    bad = np.abs(Cg - Co).max(axis=1) > 1e-12 * scale + 1e-13 * s["J"][info["ptri"]]
    assert not bad.any(), int(bad.sum())


@pytest.mark.parametrize("which,tol", [("u_mixed", 1e-10), ("u_fp64", 1e-12)])
def test_fullsize_sampled_potentials(full, which, tol):
    smp = full["sample"]
    assert rel(full[which][0, smp], full["u_or"][0]) <= tol


def test_fullsize_mixed_against_fp64_at_every_target(full):
    assert rel(full["u_mixed"][0], full["u_fp64"][0]) <= 1e-10
