"""Bounds-checked build (libcolden_checked.so, -DCOLDEN_CHECKED).  The probe
shows that an index outside its array is recorded (site and index) and not
read; small grids of every kernel family (uniform FP32 and BF16, AMR lists,
the persistent and per-box batch forms) run with no check firing and give
results bit-identical to the normal library's."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import _build, colden, synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BOX = 10 * synth.PC_CM

# the workloads: run in this process with the normal library and in a child
# process with the checked one, outputs compared bitwise
RUN = r'''
import json, os, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1410_0624_gb300 import colden, synth

def run(out_dir):
    box = 10 * synth.PC_CM
    res, status = {}, []
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    trees = []
    for L, seed in ((4, 1), (5, 2)):
        rho = synth.lognormal_grf(1 << L, 30.0, 1.8, seed=seed)
        trees.append(("u%d" % L, colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)))
    lv = synth.amr_leaves(synth.lognormal_grf(128, 30.0, 2.0, seed=3), 5, [60.0, 120.0])
    trees.append(("amr", colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])))
    for name, t in trees:
        for gname, g in (("12", g12), ("48", g48)):
            for prec in (colden.FP32, colden.BF16):
                nh = torch.empty(t.n_leaf * g.n_dir, device="cuda")
                sh = torch.empty(t.n_leaf, device="cuda")
                colden.column_density(t, g, n_h=nh, shield=sh, precision=prec)
                torch.cuda.synchronize()
                key = "%s_%s_%d" % (name, gname, prec)
                np.save(os.path.join(out_dir, key + "_nh.npy"), nh.cpu().numpy())
                np.save(os.path.join(out_dir, key + "_sh.npy"), sh.cpu().numpy())
                status.append((key, colden.checked_status() if checked else (0, 0)))
    # batches: the persistent form, then per-box graphs
    bt = [t for _, t in trees[1:]]
    bg = [g48, g12]
    for form in (1, 0):
        colden.debug_batch_form(form)
        outs = [torch.empty(t.n_leaf * g.n_dir, device="cuda") for t, g in zip(bt, bg)]
        b = colden.Batch(bt, bg, n_h=outs, precision=colden.BF16)
        b.run()
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            np.save(os.path.join(out_dir, "batch%d_%d_nh.npy" % (form, i)), o.cpu().numpy())
        status.append(("batch%d" % form, colden.checked_status() if checked else (0, 0)))
        status.append(("persistent%d" % form, (int(b.info()["persistent"]), 0)))
        b.free()
    colden.debug_batch_form(-1)
    return status

checked = os.environ.get("COLDEN_CHECKED") == "1"
colden.load()
probes = []
if checked:
    for i in (2, 7, -3):
        colden.debug_check_probe(i)
        probes.append((i, colden.checked_status()))
print(json.dumps({"probes": probes, "status": run(sys.argv[2])}))
'''


def _run(env_checked, out_dir):
    env = dict(os.environ)
    env.pop("COLDEN_CHECKED", None)
    if env_checked:
        env["COLDEN_CHECKED"] = "1"
    r = subprocess.run([sys.executable, "-c", RUN, ROOT, str(out_dir)], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_records_out_of_bounds_and_is_clean_and_identical_on_every_kernel(tmp_path):
    _build.build(checked=True)
    (tmp_path / "plain").mkdir()
    (tmp_path / "checked").mkdir()
    chk = _run(True, tmp_path / "checked")
    # the probe: in bounds nothing is recorded; outside, the site and index are
    assert [tuple(p[1]) for p in chk["probes"]] == [(0, 0), (1, 7), (1, -3)], chk["probes"]
    forms = {k: s[0] for k, s in chk["status"] if k.startswith("persistent")}
    assert forms == {"persistent1": 1, "persistent0": 0}, forms
    bad = [(k, s) for k, s in chk["status"] if not k.startswith("persistent") and tuple(s) != (0, 0)]
    assert not bad, bad
    _run(False, tmp_path / "plain")
    files = sorted(os.listdir(tmp_path / "plain"))
    assert len(files) == 3 * 2 * 2 * 2 + 2 * 2
    for f in files:
        a, b = np.load(tmp_path / "plain" / f), np.load(tmp_path / "checked" / f)
        assert np.array_equal(a, b), f
