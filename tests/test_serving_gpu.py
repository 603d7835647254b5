"""Serving loop (vp_server_*): continuous batching over resident meshes.

Each request's result must be the one vp_potential_eval gives for it alone,
whatever else is in flight (FP64 parity bar, 1e-12 relative), requests must
overlap when slots and memory allow, a budget must serialise them, cold
meshes must be built on first use, and oversized requests must fail cleanly.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(u, ref):
    return float((np.abs(u - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


@pytest.fixture(scope="module")
def pool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2205_04401_gb300 import inputs, vp
    ctx = vp.Context(0)
    specs = [(inputs.star_mesh(n_tri=800, seed=501, relax_iters=3), 19),
             (inputs.disk_mesh(seed=502), 16),
             (inputs.lshape_mesh(600, 503, relax_iters=2), 19)]
    res = []
    for mesh, rule in specs:
        m = vp.mesh_upload(ctx, mesh.vxy, mesh.tri, rule)
        nf = vp.nearfield_build(ctx, m, node_targets=True)
        y, _ = vp.mesh_nodes(m)
        res.append((mesh, m, nf, y.cpu().numpy()))
    cold = inputs.annulus_mesh(700, 504, 0.4, relax_iters=2)
    return vp, ctx, res, cold


def _densities(y, d, seed):
    rng = np.random.default_rng(seed)
    cs = rng.uniform(-0.6, 0.6, (d, 2))
    return np.ascontiguousarray(np.stack([np.exp(-((y - c) ** 2).sum(1) / 0.08) + 0.1 for c in cs]))


@pytest.mark.parametrize("prec", [0, 1])
def test_results_alone_equal_results_in_the_mix(pool, prec):
    vp, ctx, res, _ = pool
    srv = vp.Server(ctx, slots=3, hbm_budget_bytes=4 << 30, precision=prec)
    for k, (_, _, nf, _) in enumerate(res):
        srv.register(k, nf)
    reqs = []
    for i, d in enumerate([1, 3, 8, 2, 5, 1, 4, 8, 2, 1, 6, 3]):
        k = i % len(res)
        _, m, nf, y = res[k]
        f = _densities(y, d, 1000 + i)
        u = vp.pinned_empty((d, nf.M))
        reqs.append((k, f, u, srv.submit(k, f, u)))
    for k, f, u, t in reqs:
        st, lat = srv.wait(t)
        assert st == 0 and lat > 0
    for k, f, u, t in reqs:
        nf = res[k][2]
        alone = vp.potential_eval(ctx, nf, torch.from_numpy(f).cuda(), precision=prec).cpu().numpy()
        assert _rel(u, alone) <= 1e-12
    s = srv.stats()
    assert s["completed"] == len(reqs) and s["failed"] == 0 and s["queued"] == 0
    assert s["max_concurrent"] >= 2                 # requests overlapped on the device
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["evals_per_s"] > 0
    srv.close()


def test_budget_serialises_and_oversized_requests_fail(pool):
    vp, ctx, res, _ = pool
    _, m, nf, y = res[0]
    f1 = _densities(y, 2, 7)
    # footprint of one request, measured by a first server
    probe = vp.Server(ctx, slots=1, hbm_budget_bytes=4 << 30, precision=1)
    probe.register(0, nf)
    u0 = vp.pinned_empty((2, nf.M))
    assert probe.wait(probe.submit(0, f1, u0))[0] == 0
    need = probe.stats()["peak_bytes"]
    probe.close()
    srv = vp.Server(ctx, slots=4, hbm_budget_bytes=need + need // 2, precision=1)
    srv.register(0, nf)
    outs = []
    for i in range(4):
        u = vp.pinned_empty((2, nf.M))
        outs.append((u, srv.submit(0, f1, u)))
    big = _densities(y, 64, 8)
    ubig = vp.pinned_empty((64, nf.M))
    tb = srv.submit(0, big, ubig)
    for u, t in outs:
        assert srv.wait(t)[0] == 0
    assert srv.wait(tb)[0] == -4                    # VP_ERR_OOM: larger than the whole budget
    alone = vp.potential_eval(ctx, nf, torch.from_numpy(f1).cuda(), precision=1).cpu().numpy()
    for u, _ in outs:
        assert _rel(u, alone) <= 1e-12
    s = srv.stats()
    assert s["max_concurrent"] == 1 and s["failed"] == 1
    srv.close()


def test_cold_mesh_is_built_on_first_request(pool):
    vp, ctx, res, cold = pool
    srv = vp.Server(ctx, slots=2, hbm_budget_bytes=2 << 30, precision=1)
    srv.register_cold(7, cold.vxy, cold.tri, vp.VP_RULE_19_D9)
    N, M = srv.mesh_size(7)
    m = vp.mesh_upload(ctx, cold.vxy, cold.tri, vp.VP_RULE_19_D9)
    nf = vp.nearfield_build(ctx, m, node_targets=True)
    y, _ = vp.mesh_nodes(m)
    assert (N, M) == (m.N, nf.M)
    f = _densities(y.cpu().numpy(), 3, 9)
    u = vp.pinned_empty((3, M))
    t = srv.submit(7, f, u)
    assert srv.wait(t)[0] == 0
    alone = vp.potential_eval(ctx, nf, torch.from_numpy(f).cuda(), precision=1).cpu().numpy()
    assert _rel(u, alone) <= 1e-12
    assert srv.stats()["cold_builds"] == 1
    srv.close()
