"""GPU refinement (objective, analytic gradient, ascent, autograd) against
the FP64 oracle objective (oracle/refine.py)."""
import numpy as np
import pytest

from oracle import refine as ORF
from paper_1912_12807_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_12807_gb300 import pss
    pss.lib()
    return pss


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(0)
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small_case(L, ctx):
    wl = synth.workload_small(nsamp=1 << 14)
    stages = [synth.Stage(40.0, 1.0, 21, 1)]
    plan = L.Plan(L.FilDesc.of(wl.fil), stages)
    cfg = L.cfg_of(wl.cfg)
    data = _dev(wl.fil.data)
    L.pss_refine_prepare(ctx, plan, data, cfg, 0)
    obj = ORF.Objective(wl.fil, stages, wl.cfg, dm_idx=10)
    return wl, stages, plan, cfg, data, obj


def _pt(L, dm_idx, n, dm, r, z):
    p = np.zeros(1, dtype=L.REFINE_DTYPE)
    p["dm_idx"], p["numharm"], p["dm"], p["r"], p["z"] = dm_idx, n, dm, r, z
    return p


def test_objective_matches_oracle(L, ctx, small_case):
    wl, stages, plan, cfg, data, obj = small_case
    r0 = (1 / 0.0333) * obj.T
    pts = np.concatenate([_pt(L, 10, n, dm, r0 + dr, 0.0)
                          for n in (1, 4, 8) for dm in (47.3, 50.0, 52.9) for dr in (-0.71, 0.0, 0.37)])
    P, G = L.pss_refine_eval(ctx, plan, pts)
    for i, p in enumerate(pts):
        ref = obj(float(p["dm"]), float(p["r"]), float(p["z"]), int(p["numharm"]))
        assert abs(P[i] - ref) <= 2e-4 * max(ref, 1.0), (p, P[i], ref)


def _fd_grad(obj, dm, r, z, n, cells):
    g = []
    for d, h in zip(range(3), cells):
        e = [0.0, 0.0, 0.0]
        e[d] = h
        up = obj(dm + e[0], r + e[1], z + e[2], n)
        dn = obj(dm - e[0], r - e[1], z - e[2], n)
        g.append((up - dn) / (2 * h))
    return np.array(g)


def test_gradient_matches_oracle_finite_differences(L, ctx, small_case):
    wl, stages, plan, cfg, data, obj = small_case
    r0 = (1 / 0.0333) * obj.T
    for n, dm, dr in ((1, 49.3, 0.31), (4, 50.6, -0.22), (8, 51.1, 0.13)):
        p = _pt(L, 10, n, dm, r0 + dr, 0.0)
        _, G = L.pss_refine_eval(ctx, plan, p)
        fd = _fd_grad(obj, dm, r0 + dr, 0.0, n, (1e-3 * 1.0, 1e-3, 1e-3))
        fd[2] = G[0, 2]  # z: compared in the acceleration test
        err = np.linalg.norm(G[0] - fd) / np.linalg.norm(fd)
        assert err < 1e-3, (n, G[0], fd)


def test_gradient_in_z_matches_oracle():
    pytest.importorskip("torch")
    from paper_1912_12807_gb300 import pss as L
    ctx = L.Context(0)
    fil = synth.make_8bit(32, 1 << 13, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.6, z_direct=6.0)], seed=3)
    stages = [synth.Stage(10.0, 5.0, 4, 1)]
    cfgp = synth.SearchCfg(zmax=10, dz=2.0, numharm=2, whiten_block=128)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    L.pss_refine_prepare(ctx, plan, _dev(fil.data), L.cfg_of(cfgp), 0)
    obj = ORF.Objective(fil, stages, cfgp, dm_idx=2)
    r0 = 100.0 * obj.T  # the injected 100 Hz pulsar, in bins of the span T
    for n, dm, r, z in ((1, 20.4, r0 + 0.2, 5.3), (2, 19.1, r0 - 0.35, 6.7)):
        p = _pt(L, 2, n, dm, r, z)
        P, G = L.pss_refine_eval(ctx, plan, p)
        ref = obj(dm, r, z, n)
        assert abs(P[0] - ref) <= 2e-4 * max(ref, 1.0)
        fd = _fd_grad(obj, dm, r, z, n, (5e-3, 1e-3, 2e-3))
        err = np.linalg.norm(G[0] - fd) / np.linalg.norm(fd)
        assert err < 1e-3, (G[0], fd)
    ctx.close()


def test_ascent_reaches_oracle_grid_maximum(L, ctx, small_case):
    wl, stages, plan, cfg, data, obj = small_case
    cands = L.pss_search_dm_batch(ctx, plan, data, cfg, 0, plan.ndm)
    top = cands[np.argsort(-cands["sigma"])[:3]]
    ref_cfg = L.cfg_of(wl.cfg)
    out = L.pss_refine_candidates(ctx, plan, data, ref_cfg, top, iters=60, lr=0.05)
    for c0, c1 in zip(top, out):
        assert c1["power"] >= c0["power"] * (1 - 1e-3)
        o = ORF.Objective(wl.fil, stages, wl.cfg, dm_idx=int(c0["dm_idx"]))
        gmax, gdm, gr, gz = o.grid_max(float(c0["dm"]), float(c0["r"]), 0.0, int(c0["numharm"]), 1.0, 0.0)
        assert c1["power"] >= gmax * (1 - 1e-3), (c1, gmax)
        assert abs(c1["dm"] - gdm) <= 1.0 / 8 + 1e-9 or c1["power"] > gmax
        assert abs(c1["r"] - gr) <= 1.0 / 16 + 1e-9 or c1["power"] > gmax


def test_autograd_function(L, ctx, small_case):
    import torch
    wl, stages, plan, cfg, data, obj = small_case
    RP = L.refine_power_function()
    r0 = (1 / 0.0333) * obj.T
    dm = torch.tensor([49.7, 50.2], dtype=torch.float64, requires_grad=True)
    r = torch.tensor([r0 + 0.2, r0 - 0.1], dtype=torch.float64, requires_grad=True)
    z = torch.zeros(2, dtype=torch.float64, requires_grad=True)
    P = RP.apply(dm, r, z, ctx, plan, [10, 10], [4, 4])
    P.sum().backward()
    pts = np.concatenate([_pt(L, 10, 4, 49.7, r0 + 0.2, 0.0), _pt(L, 10, 4, 50.2, r0 - 0.1, 0.0)])
    _, G = L.pss_refine_eval(ctx, plan, pts)
    np.testing.assert_allclose(dm.grad.numpy(), G[:, 0], rtol=1e-12)
    np.testing.assert_allclose(r.grad.numpy(), G[:, 1], rtol=1e-12)
