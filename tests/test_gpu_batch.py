"""Batched evaluation (many independent boxes per call).

Every box of a mixed batch (uniform and AMR meshes, 12 and 48 HEALPix
directions) is compared with the FP64 oracle of the tree method (§3.2, §3.3,
Eqs. N_discret1 and N_discret) on seeded samples of its leaves, for the
per-box launches and for the captured graph, in FP32 (1e-5 relative on N_H,
1e-5 absolute on the screening factor) and BF16 (1e-2 relative, 5e-3 absolute;
the tolerances of the single-box parity tests).  The batch paths must also be
bitwise equal to per-box cd_column_density calls (the same kernels on the same
data), see density updates between graph replays, and refuse the requests that
would leave a captured graph pointing at reallocated scratch."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
BOX = 10 * PC
pytestmark = pytest.mark.gpu
TOL = {colden.FP32: (1e-5, 1e-5), colden.BF16: (1e-2, 5e-3)}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


# (kind, size, directions): uniform boxes of 2^size per axis, AMR boxes on a
# base of size / 4 per axis with two refined levels
SPECS = [("u", 3, 48), ("u", 4, 12), ("a", 16, 12), ("u", 5, 48), ("a", 32, 48), ("u", 6, 12), ("u", 4, 48)]


def _boxes(seed=0):
    """Uneven boxes; returns trees, geometries, flat leaf densities (the
    caller's order) and the oracle's view of each box."""
    rng = np.random.default_rng(seed)
    trees, geoms, rhos, srcs = [], [], [], []
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    for kind, size, nd in SPECS:
        sig = float(rng.uniform(1.0, 2.5))
        if kind == "u":
            rho = synth.lognormal_grf(1 << size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            trees.append(colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX))
            rhos.append(rho.reshape(-1))
            srcs.append(("u", rho))
        else:
            fine = synth.lognormal_grf(size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            lv = synth.amr_leaves(fine, int(np.log2(size)) - 2, [60.0, 120.0])
            trees.append(colden.build_tree_amr(lv["base"], lv["lmax"], BOX, lv["level"], lv["ijk"], lv["rho"]))
            rhos.append(lv["rho"])
            srcs.append(("a", lv))
        geoms.append(g12 if nd == 12 else g48)
    return trees, geoms, rhos, srcs


def _outs(trees, geoms):
    nh = [torch.full((t.n_leaf * g.n_dir,), -1.0, device="cuda") for t, g in zip(trees, geoms)]
    sh = [torch.full((t.n_leaf,), -1.0, device="cuda") for t in trees]
    return nh, sh


def _ref(trees, geoms, precision):
    nh, sh = _outs(trees, geoms)
    for t, g, a, b in zip(trees, geoms, nh, sh):
        colden.column_density(t, g, n_h=a, shield=b, precision=precision)
    torch.cuda.synchronize()
    return [x.cpu() for x in nh], [x.cpu() for x in sh]


def _sample(tree, rng, n=48):
    """Leaf rows to check: the first and last, every level's first leaf and a
    seeded random set."""
    lv, ijk = tree.leaves()
    rows = {0, tree.n_leaf - 1}
    for l in np.unique(lv):
        rows.add(int(np.flatnonzero(lv == l)[0]))
    rows.update(int(r) for r in rng.choice(tree.n_leaf, size=min(n, tree.n_leaf), replace=False))
    rows = np.array(sorted(rows))
    return rows, lv[rows], ijk[rows]


def _oracle_rows(src, trees, geoms, rng):
    """Oracle N_H of sampled leaves of every box: [(rows, N_H [rows, nd])]."""
    out = []
    for (kind, data), t, g in zip(src, trees, geoms):
        T = oracle.Tree.uniform(data, BOX) if kind == "u" else \
            oracle.Tree.amr(data["base"], data["lmax"], BOX, data["level"], data["ijk"], data["rho"])
        rows, lv, ijk = _sample(t, rng)
        dirs = oracle.dirs_healpix(1 if g.n_dir == 12 else 2)
        out.append((rows, T.column_density(dirs, lv, ijk)))
    return out


def _check_oracle(nh, sh, ref_rows, geoms, precision, what):
    rtol, satol = TOL[precision]
    for b, ((rows, ref), a, s, g) in enumerate(zip(ref_rows, nh, sh, geoms)):
        got = a.cpu().numpy().reshape(-1, g.n_dir)[rows].astype(np.float64)
        rel = np.max(np.abs(got - ref) / ref)
        dsh = np.max(np.abs(s.cpu().numpy()[rows] - oracle.shield(ref)))
        assert rel <= rtol, "%s box %d (%s): max rel N_H error %.3g" % (what, b, SPECS[b], rel)
        assert dsh <= satol, "%s box %d (%s): max shield error %.3g" % (what, b, SPECS[b], dsh)


# boxes the persistent form serves: uniform trees of 32^3 and more, AMR trees
# on a 32^3 base with two refined levels
PSPECS = [("u", 5, 48), ("a", 128, 12), ("u", 6, 12), ("a", 128, 48), ("u", 5, 12), ("u", 6, 48)]


def _pboxes(seed=0):
    rng = np.random.default_rng(seed)
    trees, geoms, rhos, srcs = [], [], [], []
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    for kind, size, nd in PSPECS:
        sig = float(rng.uniform(1.0, 2.5))
        if kind == "u":
            rho = synth.lognormal_grf(1 << size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            trees.append(colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX))
            rhos.append(rho.reshape(-1))
            srcs.append(("u", rho))
        else:
            fine = synth.lognormal_grf(size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            lv = synth.amr_leaves(fine, int(np.log2(size)) - 2, [60.0, 120.0])
            trees.append(colden.build_tree_amr(lv["base"], lv["lmax"], BOX, lv["level"], lv["ijk"], lv["rho"]))
            rhos.append(lv["rho"])
            srcs.append(("a", lv))
        geoms.append(g12 if nd == 12 else g48)
    return trees, geoms, rhos, srcs


def test_persistent_batch_matches_oracle_and_per_box():
    """BF16 batch of boxes the persistent form serves: the graph holds a few
    persistent launches (level-3 lists, one shell launch over every box,
    level and tile, one leaf launch per direction set), the autotuner tried
    both tile shapes and CTA counts, and every box matches the FP64 oracle at
    the BF16 tolerance and the per-box evaluation within it; a replay after a
    density update matches the oracle too."""
    trees, geoms, rhos, srcs = _pboxes()
    ref_rows = _oracle_rows(srcs, trees, geoms, np.random.default_rng(11))
    rn, rs = _ref(trees, geoms, colden.BF16)
    nh, sh = _outs(trees, geoms)
    colden.debug_batch_form(1)
    try:
        batch = colden.Batch(trees, geoms, n_h=nh, shield=sh, precision=colden.BF16)
    finally:
        colden.debug_batch_form(-1)
    info = batch.info()
    assert info["persistent"], info
    assert set(info["plan_ms"]) == {"half/1", "half/2", "full/1", "full/2"}, info
    assert not info["ms_tried"], info
    assert info["kernel_nodes"] <= 2 + 2 * len(geoms), info
    for x in nh + sh:
        x.fill_(-1.0)
    for _ in range(2):          # two replays in a row (the counters are reset by the graph)
        batch.run()
    torch.cuda.synchronize()
    colden.device_status()
    _check_oracle(nh, sh, ref_rows, geoms, colden.BF16, "persistent replay")
    for a, b in zip(nh, rn):
        a, b = a.double().cpu(), b.double().cpu()
        assert torch.max((a - b).abs() / b).item() <= 1e-2
    for a, b in zip(sh, rs):
        assert torch.max((a.cpu() - b).abs()).item() <= 5e-3
    # a density update between replays is seen
    rng = np.random.default_rng(6)
    new = [(r * rng.uniform(0.5, 2.0, size=r.shape)).astype(np.float32) for r in rhos]
    for t, r in zip(trees, new):
        colden.tree_update(t, torch.from_numpy(r).cuda())
    batch.run()
    torch.cuda.synchronize()
    src_new = []
    for (kind, data), r in zip(srcs, new):
        if kind == "u":
            src_new.append(("u", r.reshape(data.shape)))
        else:
            d = dict(data)
            d["rho"] = r
            src_new.append(("a", d))
    _check_oracle(nh, sh, _oracle_rows(src_new, trees, geoms, np.random.default_rng(12)), geoms, colden.BF16,
                  "persistent replay after update")
    colden.device_status()
    batch.free()


def test_batch_autotuner_keeps_the_fastest_form():
    """Without a forced form the autotuner times the graph replay of every
    persistent tile shape and every per-box fan-out and keeps the fastest;
    the kept graph's results match per-box evaluation at the BF16 tolerance."""
    trees, geoms, rhos, srcs = _pboxes(seed=3)
    rn, rs = _ref(trees, geoms, colden.BF16)
    nh, sh = _outs(trees, geoms)
    batch = colden.Batch(trees, geoms, n_h=nh, shield=sh, precision=colden.BF16)
    info = batch.info()
    assert set(info["plan_ms"]) == {"half/1", "half/2", "full/1", "full/2"}, info
    assert set(info["ms_tried"]) == {1, 2, 4}, info        # W <= number of boxes
    best_plan, best_w = min(info["plan_ms"].values()), min(info["ms_tried"].values())
    if info["persistent"]:
        assert best_plan <= best_w, info
    else:
        assert best_w < best_plan and info["ms_tried"][info["width"]] == best_w, info
    for x in nh + sh:
        x.fill_(-1.0)
    batch.run()
    torch.cuda.synchronize()
    colden.device_status()
    for a, b in zip(nh, rn):
        a, b = a.double().cpu(), b.double().cpu()
        assert torch.max((a - b).abs() / b).item() <= 1e-2
    for a, b in zip(sh, rs):
        assert torch.max((a.cpu() - b).abs()).item() <= 5e-3
    batch.free()


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
def test_batch_eager_and_graph_match_oracle_and_per_box(precision):
    trees, geoms, rhos, srcs = _boxes()
    ref_rows = _oracle_rows(srcs, trees, geoms, np.random.default_rng(7))
    rn, rs = _ref(trees, geoms, precision)
    nh, sh = _outs(trees, geoms)
    colden.column_density_batch(trees, geoms, n_h=nh, shield=sh, precision=precision)
    torch.cuda.synchronize()
    _check_oracle(nh, sh, ref_rows, geoms, precision, "per-box launches")
    for a, b in zip(nh + sh, rn + rs):
        assert torch.equal(a.cpu(), b)
    nh2, sh2 = _outs(trees, geoms)
    batch = colden.Batch(trees, geoms, n_h=nh2, shield=sh2, precision=precision)
    info = batch.info()
    # these boxes include small and shallow trees: every box's own kernels in the graph
    assert not info["persistent"]
    assert info["width"] in (1, 2, 4, 8) and info["kernel_nodes"] > len(trees)
    for x in nh2 + sh2:
        x.fill_(-1.0)
    batch.run()
    torch.cuda.synchronize()
    _check_oracle(nh2, sh2, ref_rows, geoms, precision, "graph replay")
    for a, b in zip(nh2 + sh2, rn + rs):
        assert torch.equal(a.cpu(), b)
    colden.device_status()
    batch.free()


def test_graph_replay_sees_updated_densities():
    trees, geoms, rhos, srcs = _boxes(seed=1)
    nh, sh = _outs(trees, geoms)
    batch = colden.Batch(trees, geoms, n_h=nh, shield=sh)
    rng = np.random.default_rng(5)
    new = [(r * rng.uniform(0.5, 2.0, size=r.shape)).astype(np.float32) for r in rhos]
    for t, r in zip(trees, new):
        colden.tree_update(t, torch.from_numpy(r).cuda())
    batch.run()
    torch.cuda.synchronize()
    got = [x.cpu() for x in nh + sh]
    rn, rs = _ref(trees, geoms, colden.FP32)
    for a, b in zip(got, rn + rs):
        assert torch.equal(a, b)
    # the replayed columns are those of the new densities, per the oracle
    src_new = []
    for (kind, data), r in zip(srcs, new):
        if kind == "u":
            src_new.append(("u", r.reshape(data.shape)))
        else:
            d = dict(data)
            d["rho"] = r
            src_new.append(("a", d))
    ref_rows = _oracle_rows(src_new, trees, geoms, np.random.default_rng(8))
    _check_oracle(nh, sh, ref_rows, geoms, colden.FP32, "replay after update")
    batch.free()


def test_batched_tree_scratch_is_pinned_while_the_batch_lives():
    """A tree held by a live batch graph must not have its scratch reallocated
    (another direction count): the call is refused, the batch still replays
    correctly, and after the batch is freed the evaluation goes through."""
    rho = synth.lognormal_grf(32, 30.0, 2.0, seed=3)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    nh = torch.empty(tree.n_leaf * 48, device="cuda")
    ref = torch.empty_like(nh)
    colden.column_density(tree, g48, n_h=ref)
    batch = colden.Batch([tree], [g48], n_h=[nh])
    other = torch.empty(tree.n_leaf * 12, device="cuda")
    with pytest.raises(colden.ColdenError) as e:
        colden.column_density(tree, g12, n_h=other)
    assert e.value.code == colden.CD_EINVAL and "batch" in str(e.value)
    # same direction count: no reallocation, allowed
    colden.column_density(tree, g48, n_h=ref)
    nh.fill_(-1.0)
    batch.run()
    torch.cuda.synchronize()
    assert torch.equal(nh, ref)
    batch.free()
    colden.column_density(tree, g12, n_h=other)
    torch.cuda.synchronize()
    assert torch.all(other > 0)


def test_batch_rejects_shared_tree_with_two_direction_counts_and_learned_form():
    rho = synth.lognormal_grf(16, 30.0, 2.0, seed=4)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    with pytest.raises(colden.ColdenError) as e:
        colden.Batch([tree, tree], [g12, g48],
                     shield=[torch.empty(tree.n_leaf, device="cuda") for _ in range(2)])
    assert e.value.code == colden.CD_EINVAL
    # one tree twice with the same geometry is fine
    b = colden.Batch([tree, tree], [g48, g48], shield=[torch.empty(tree.n_leaf, device="cuda") for _ in range(2)])
    b.free()
    params = synth.mlp_init(48, 128, seed=0)
    net = colden.Net(48, 128, params)
    L = colden.load()
    o = colden.opts_default()
    o.net = net.handle.value
    trees = (colden.ctypes.c_void_p * 1)(tree.handle.value)
    geoms = (colden.ctypes.c_void_p * 1)(g48.handle.value)
    sh = torch.empty(tree.n_leaf, device="cuda")
    shp = (colden.ctypes.c_void_p * 1)(sh.data_ptr())
    h = colden.ctypes.c_void_p()
    rc = L.cd_batch_create(1, trees, geoms, colden.ctypes.byref(o), None, None, shp, None, colden.ctypes.byref(h))
    assert rc == colden.CD_EUNSUPPORTED and not h.value


def test_batch_outputs_checked_before_launch():
    rho = synth.lognormal_grf(16, 30.0, 2.0, seed=5)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    g48 = colden.precompute_geometry("healpix", 2)
    short = torch.empty(tree.n_leaf * 48 - 1, device="cuda")
    colden.stats_reset()
    with pytest.raises(ValueError):
        colden.column_density_batch([tree], [g48], n_h=[short])
    with pytest.raises(ValueError):
        colden.Batch([tree], [g48], n_h=[short])
    with pytest.raises(ValueError):
        colden.column_density(tree, g48, shield=torch.empty(tree.n_leaf - 1, device="cuda"))
    assert all(colden.stats_get(k)[0] == 0 for k in range(len(colden.KERNEL_KINDS)))
