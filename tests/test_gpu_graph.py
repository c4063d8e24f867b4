"""cd_eval_graph: one evaluation step (density update + evaluation) captured as
a CUDA graph.  Replays must give the eager calls' results bit for bit on the
densities the graph's buffer holds at launch, count their kernels, and be
refused (without launching) once a buffer the capture named may be gone."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _launches():
    return sum(colden.stats_get(k)[0] for k in range(len(colden.KERNEL_KINDS)))


def _outs(tree, geom):
    nd = tree.n_leaf * geom.n_dir
    return (torch.full((nd,), -1.0, device="cuda"), torch.full((nd,), -1.0, device="cuda"),
            torch.full((tree.n_leaf,), -1.0, device="cuda"))


def _eager(tree, geom, rho, precision, net=None):
    n_h, a_v, sh = _outs(tree, geom)
    colden.tree_update(tree, rho)
    colden.column_density(tree, geom, n_h=n_h, a_v=a_v, shield=sh, precision=precision, net=net)
    torch.cuda.synchronize()
    colden.device_status()
    return n_h, a_v, sh


def _uniform_field(L, seed):
    return torch.from_numpy(synth.lognormal_grf(1 << L, 30.0, 2.0, seed)).cuda().reshape(-1)


@pytest.mark.parametrize("L,precision", [(5, colden.FP32), (6, colden.BF16), (8, colden.BF16)])
def test_uniform_graph_replays_match_eager_and_oracle(L, precision):
    rho0 = _uniform_field(L, 1)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 2)
    buf = rho0.clone()
    n_h, a_v, sh = _outs(tree, geom)
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    assert g.kernels() > 0
    for seed in (2, 3):
        new = _uniform_field(L, seed)
        buf.copy_(new)
        n_h.fill_(-1.0)
        sh.fill_(-1.0)
        colden.stats_reset(timing=False)
        g.launch()
        torch.cuda.synchronize()
        colden.device_status()
        assert _launches() == g.kernels()
        got = (n_h.clone(), a_v.clone(), sh.clone())
        want = _eager(tree, geom, new, precision)
        for x, y in zip(got, want):
            assert torch.equal(x, y)
    if L <= 6:
        # the replayed columns of the last field against the FP64 oracle on sampled leaves
        T = oracle.Tree.uniform(new.reshape((1 << L,) * 3).cpu().numpy(), 10 * PC)
        m = np.sort(np.random.default_rng(L).choice(tree.n_leaf, 64, replace=False))
        lvl, ijk = tree.leaves()
        ref = T.column_density(geom.dirs, lvl[m], ijk[m])
        nd = geom.n_dir
        gg = got[0].reshape(-1, nd)[torch.from_numpy(m).cuda()].double().cpu().numpy()
        tol = 1e-5 if precision == colden.FP32 else 1e-2
        assert np.max(np.abs(gg - ref) / ref) < tol
    g.free()


def test_graph_without_update_sees_eager_updates():
    L = 6
    tree = colden.build_tree_uniform(_uniform_field(L, 4).reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 1)
    n_h, a_v, sh = _outs(tree, geom)
    g = colden.EvalGraph(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16)
    new = _uniform_field(L, 5)
    colden.tree_update(tree, new)
    g.launch()
    torch.cuda.synchronize()
    want = _eager(tree, geom, new, colden.BF16)
    assert torch.equal(n_h, want[0]) and torch.equal(sh, want[2])


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
def test_amr_graph_replays_match_eager(precision):
    fine = synth.lognormal_grf(128, 30.0, 2.0, seed=12)
    lv = synth.amr_leaves(fine, 5, [40.0, 80.0])
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], 20 * PC, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry("healpix", 2)
    buf = torch.from_numpy(lv["rho"]).cuda()
    n_h, a_v, sh = _outs(tree, geom)
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    scale = torch.from_numpy(np.random.default_rng(3).uniform(0.5, 2.0, size=tree.n_leaf).astype(np.float32)).cuda()
    new = buf * scale
    buf.copy_(new)
    colden.stats_reset(timing=False)
    g.launch()
    torch.cuda.synchronize()
    colden.device_status()
    assert _launches() == g.kernels()
    got = (n_h.clone(), a_v.clone(), sh.clone())
    want = _eager(tree, geom, new, precision)
    for x, y in zip(got, want):
        assert torch.equal(x, y)


def test_learned_graph_replays_match_eager_and_are_refused_after_training():
    L, nd, H = 5, 48, 128
    rho0 = _uniform_field(L, 6)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 2)
    net = colden.Net(nd, H, synth.mlp_init(nd, H, 6, out_scale=0.2))
    x = torch.empty((2048, 8 * nd + 1), device="cuda")
    colden.learned_features(tree, geom, x, leaves=torch.arange(2048, device="cuda"))
    net.fit_normaliser(x)
    n_h, a_v, sh = _outs(tree, geom)
    with pytest.raises(colden.ColdenError):
        colden.EvalGraph(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16, net=net)
    buf = rho0.clone()
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, a_v=a_v, shield=sh, precision=colden.BF16, net=net)
    new = _uniform_field(L, 7)
    buf.copy_(new)
    g.launch()
    torch.cuda.synchronize()
    colden.device_status()
    got = (n_h.clone(), a_v.clone(), sh.clone())
    want = _eager(tree, geom, new, colden.BF16, net=net)
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    # a changed trusted range or new parameters: refused, nothing launched
    net.set_delta_range(-1.0, 1.0)
    with pytest.raises(colden.ColdenError):
        g.launch()
    net.set_delta_range(float("-inf"), float("inf"))
    g.launch()
    st = net.state()
    net.load_state(st)
    with pytest.raises(colden.ColdenError):
        g.launch()
    torch.cuda.synchronize()
    colden.device_status()


def test_graph_is_refused_after_a_free_and_can_be_recreated():
    L = 6
    rho0 = _uniform_field(L, 8)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 2)
    buf = rho0.clone()
    n_h, a_v, sh = _outs(tree, geom)
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, shield=sh, precision=colden.BF16)
    g.launch()
    # another direction count reallocates the tree's workspace under the graph
    g12 = colden.precompute_geometry("healpix", 1)
    o12 = _outs(tree, g12)
    colden.column_density(tree, g12, n_h=o12[0], precision=colden.BF16)
    colden.stats_reset(timing=False)
    with pytest.raises(colden.ColdenError):
        g.launch()
    assert _launches() == 0
    g.free()
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, shield=sh, precision=colden.BF16)
    g.launch()
    torch.cuda.synchronize()
    want = _eager(tree, geom, rho0, colden.BF16)
    assert torch.equal(n_h, want[0]) and torch.equal(sh, want[2])
    # freeing any library object (here a geometry) also retires the graph
    g12.free()
    with pytest.raises(colden.ColdenError):
        g.launch()
    g.free()
    torch.cuda.synchronize()
    colden.device_status()


@pytest.mark.parametrize("mode,precision", [(colden.MODE_CONE, colden.BF16), (colden.MODE_INSITU, colden.FP32)])
def test_graph_of_the_cone_and_insitu_forms(mode, precision):
    L = 6
    rho0 = _uniform_field(L, 9)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 1, mode=mode)
    buf = rho0.clone()
    n_h, a_v, sh = _outs(tree, geom)
    g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    new = _uniform_field(L, 10)
    buf.copy_(new)
    g.launch()
    torch.cuda.synchronize()
    got = (n_h.clone(), a_v.clone(), sh.clone())
    want = _eager(tree, geom, new, precision)
    for x, y in zip(got, want):
        assert torch.equal(x, y)


def test_graph_captured_while_per_launch_timing_is_on():
    """With per-launch timing on the evaluation runs in order on one stream;
    its capture holds no timing events and replays match the eager step."""
    L = 6
    rho0 = _uniform_field(L, 11)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 2)
    buf = rho0.clone()
    n_h, a_v, sh = _outs(tree, geom)
    colden.stats_reset(timing=True)
    try:
        g = colden.EvalGraph(tree, geom, rho=buf, n_h=n_h, shield=sh, precision=colden.BF16)
        new = _uniform_field(L, 12)
        buf.copy_(new)
        g.launch()
        torch.cuda.synchronize()
        assert colden.stats_get(colden.K_LEAF)[0] >= 2      # the eager first step and the replay
    finally:
        colden.stats_reset(timing=False)
    got = (n_h.clone(), sh.clone())
    want = _eager(tree, geom, new, colden.BF16)
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[2])


def test_graph_creation_on_a_capturing_stream_is_refused():
    L = 5
    rho0 = _uniform_field(L, 13)
    tree = colden.build_tree_uniform(rho0.reshape((1 << L,) * 3), 10 * PC)
    geom = colden.precompute_geometry("healpix", 1)
    n_h, a_v, sh = _outs(tree, geom)
    colden.column_density(tree, geom, n_h=n_h, precision=colden.FP32)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    outer = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(outer, stream=s):
        try:
            colden.EvalGraph(tree, geom, n_h=n_h, precision=colden.FP32, stream=torch.cuda.current_stream())
        except colden.ColdenError as e:
            err = e
        colden.column_density(tree, geom, n_h=n_h, precision=colden.FP32, stream=torch.cuda.current_stream())
    assert err is not None and "capturing" in str(err)
    outer.replay()
    torch.cuda.synchronize()
    colden.device_status()
