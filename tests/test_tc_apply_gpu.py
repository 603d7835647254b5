"""Tensor-core correction apply (VP_MIXED_TC) through the C ABI.

The path splits every weight C[t,e] and density value f[n,e] into L balanced
base-128 digits held as bf16 and sums the digit products on the tensor cores
with exact FP32 accumulation.  Its only error is the rounding of C to 7L - 1
bits below the largest weight of its kind (near or self) in its target row and
of f to 7L - 1 bits below the largest value of its density.  So, with the
same far sum,

    u_tc - u_mixed = sum_e (C~ f~ - C f)        (C~, f~: those roundings)

must hold to FP64 rounding (2e-15 of max|u| + max_t sum_e |C f|): this pins
the digit split, the level/column bookkeeping of the MMAs and the exactness
of the accumulation (an FP32-rounded accumulation would be off by some 1e-8
of sum_e |C f|).  Against the
oracle the stated bar is 1e-10 per density for L = 5.
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
    return np.max(np.abs(u - ref), axis=1) / np.max(np.abs(ref), axis=1)


def rounded(x, e, L):
    """x rounded to the grid 2^(e - 7L + 1) (round half to even)."""
    return np.ldexp(np.rint(np.ldexp(x, 7 * L - 1 - e)), e - 7 * L + 1)


def emulated_delta(C, row, ptri, kind, nq, f, L):
    """sum_e (C~ f~ - C f) per density and target, in FP64, and per density
    the largest sum_e |C f| over the targets."""
    M = len(row) - 1
    tgt = np.repeat(np.arange(M), np.diff(row))
    Ct = np.empty_like(C)
    for k in (0, 1):
        sel = kind == k
        rmax = np.zeros(M)
        np.maximum.at(rmax, tgt[sel], np.abs(C[sel]).max(axis=1) if sel.any() else np.zeros(0))
        et = np.where(rmax > 0, np.frexp(rmax)[1], 0)
        Ct[sel] = rounded(C[sel], et[tgt[sel]][:, None], L)
    fmax = np.abs(f).max(axis=1)
    tau = np.where(fmax > 0, np.frexp(fmax)[1], 0)
    ft = rounded(f, tau[:, None], L)
    src = (ptri[:, None].astype(np.int64) * nq + np.arange(nq)[None, :])      # [P][nq]
    out = np.zeros((f.shape[0], M))
    mag = np.zeros(f.shape[0])
    for n in range(f.shape[0]):
        contrib = (Ct * ft[n][src] - C * f[n][src]).sum(axis=1)
        np.add.at(out[n], tgt, contrib)
        a = np.zeros(M)
        np.add.at(a, tgt, np.abs(C * f[n][src]).sum(axis=1))
        mag[n] = a.max()
    return out, mag


def check_exact(um, ut, delta, mag):
    """The tensor-core result equals the FP64 apply plus the emulated digit
    rounding, up to the rounding of the two FP64 evaluations themselves: the
    FP64 apply sums a row of up to ~10^3 weight-density products (rounding
    ~sqrt(n) 2^-53 of sum |C f|), the emulation sums the same number of
    differences and the tensor-core path combines its exact FP32 level sums
    in float-float (~2^-48 per level): together a few 1e-15 of sum |C f|."""
    scale = np.abs(um).max(axis=1) + mag
    err = np.max(np.abs((ut - um) - delta), axis=1) / np.maximum(scale, 1e-300)
    assert err.max() <= 4e-15, err.max()


def build(vp, ctx, mesh, rule, extra=None):
    m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
    txy = None if extra is None else torch.from_numpy(np.ascontiguousarray(extra)).cuda()
    nf = vp.nearfield_build(ctx, m, node_targets=True, txy=txy)
    y, _ = vp.mesh_nodes(m)
    row, ptri, kind, _ = vp.nf_lists(nf)
    C = vp.nf_weights(nf)
    return dict(mesh=m, nf=nf, y=y.cpu().numpy(), row=row.cpu().numpy(), ptri=ptri.cpu().numpy(),
                kind=kind.cpu().numpy(), C=C.cpu().numpy())


def eval_pair(vp, ctx, g, f, levels):
    fd = torch.from_numpy(np.ascontiguousarray(f)).cuda()
    um = vp.potential_eval(ctx, g["nf"], fd, precision=vp.VP_MIXED).cpu().numpy()
    vp.nf_prepare_tc(g["nf"], levels)
    ut = vp.potential_eval(ctx, g["nf"], fd, precision=vp.VP_MIXED_TC).cpu().numpy()
    assert vp.device_status(ctx) == 0
    return um, ut


@pytest.fixture(scope="module")
def star(vp, ctx):
    mesh = inputs.star_mesh(n_tri=2048, seed=77, relax_iters=6)
    extra = inputs.random_interior_points(mesh, 300, 78)
    g = build(vp, ctx, mesh, 19, extra)
    fs = [inputs.gaussian_mix(mesh, 900 + i) for i in range(32)]
    fs += [inputs.manufactured_sin_cos(float(k)) for k in range(1, 9)]
    f = np.stack([fn(g["y"]) for fn in fs])
    return mesh, extra, g, f


@pytest.mark.parametrize("levels", [5, 4, 3])
def test_tc_apply_is_the_exact_product_of_the_rounded_operands(vp, ctx, star, levels):
    _, _, g, f = star
    um, ut = eval_pair(vp, ctx, g, f, levels)
    info = vp.nf_tc_info(g["nf"])
    assert info["levels"] == levels and info["n_tiles"] == (g["nf"].M + 127) // 128 and info["n_chunks"] > 0
    delta, mag = emulated_delta(g["C"], g["row"], g["ptri"], g["kind"], 19, f, levels)
    check_exact(um, ut, delta, mag)
    # the rounding is visible at all (the comparison is not vacuous)
    assert np.max(np.abs(delta).max(axis=1) / mag) > 1e-13


def test_tc_apply_against_the_oracle(vp, ctx, star, tables):
    mesh, extra, g, f = star
    o = Oracle("far19", tables=tables)
    s = o.setup(mesh.vxy, mesh.tri, node_targets=True, extra=extra)
    rng = np.random.default_rng(81)
    sample = np.unique(np.concatenate([rng.choice(s["N"], 200, replace=False), s["N"] + np.arange(0, 300, 7)]))
    u_or, _ = o.potential(s, f, targets=sample)
    _, ut = eval_pair(vp, ctx, g, f, 5)
    err = rel_err(ut[:, sample], u_or)
    assert err.max() <= 1e-10, err.max()


def test_tc_apply_sixteen_node_rule_two_density_passes(vp, ctx):
    """16-node rule (K columns 16 + 8 zeros per triangle) and d = 70 (passes
    of 32 + 32 + 6 densities with 5 digits)."""
    mesh = inputs.disk_mesh(seed=5)
    g = build(vp, ctx, mesh, 16)
    rng = np.random.default_rng(12)
    f = rng.normal(size=(70, g["nf"].mesh.N))
    um, ut = eval_pair(vp, ctx, g, f, 5)
    delta, mag = emulated_delta(g["C"], g["row"], g["ptri"], g["kind"], 16, f, 5)
    check_exact(um, ut, delta, mag)


def test_tc_apply_targets_without_pairs_and_odd_unions(vp, ctx):
    """One triangle, targets outside it (rows without pairs), a union of one
    triangle (its chunk repeats it with zero weights)."""
    vxy = np.array([[0.0, 0.0], [0.3, 0.05], [0.1, 0.25]])
    tri = np.array([[0, 1, 2]], np.int32)
    extra = np.array([[0.12, 0.1], [0.5, 0.5], [0.15, 0.025], [2.0, -1.0], [-3.0, 4.0]])

    class _M:
        pass
    mesh = _M()
    mesh.vxy, mesh.tri = vxy, tri
    g = build(vp, ctx, mesh, 19, extra)
    f = np.stack([np.ones(19), np.cos(3 * g["y"][:, 0]) * g["y"][:, 1], np.zeros(19)])
    um, ut = eval_pair(vp, ctx, g, f, 4)
    delta, mag = emulated_delta(g["C"], g["row"], g["ptri"], g["kind"], 19, f, 4)
    check_exact(um, ut, delta, mag)
    assert np.all(ut[2] == 0.0)


def test_tc_levels_out_of_range_are_rejected(vp, ctx, star):
    _, _, g, _ = star
    for bad in (2, 6):
        with pytest.raises(vp.VPError):
            vp.nf_prepare_tc(g["nf"], bad)
