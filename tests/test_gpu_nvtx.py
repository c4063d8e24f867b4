"""NVTX ranges: an evaluation run with an NVTX injection library attached
(tests/nvtx_record.c, built here with gcc) records a "colden:<entry point>"
range around each entry point and a "colden:<kernel kind>" range around
every kernel launch (restriction, shells, leaves), properly nested."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_1410_0624_gb300 import colden, synth
colden.load()
g = colden.precompute_geometry("healpix", 2)
rho = synth.lognormal_grf(64, 30.0, 1.5, seed=1)
t = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), 10 * synth.PC_CM)
sh = torch.empty(t.n_leaf, device="cuda")
for prec in (colden.FP32, colden.BF16):
    colden.column_density(t, g, shield=sh, precision=prec)
colden.tree_update(t, torch.from_numpy(rho * 2).cuda())
torch.cuda.synchronize()
'''


def test_entry_points_and_kernel_kinds_open_nested_ranges(tmp_path):
    lib = tmp_path / "nvtx_record.so"
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["gcc", "-shared", "-fPIC", "-O1", "-I" + cuda_inc, os.path.join(ROOT, "tests", "nvtx_record.c"),
                    "-o", str(lib)], check=True)
    log = tmp_path / "ranges.txt"
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(lib), COLDEN_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", SCRIPT, ROOT], check=True, env=env, timeout=600)
    stack, seen = [], []
    for line in log.read_text().splitlines():
        if line.startswith("push "):
            stack.append(line[5:])
            seen.append((line[5:], tuple(stack[:-1])))
        else:
            assert line == "pop" and stack, line
            stack.pop()
    assert not stack, stack
    names = {n for n, _ in seen}
    for want in ("colden:precompute_geometry", "colden:build_tree_uniform", "colden:column_density",
                 "colden:tree_update", "colden:restrict", "colden:shell", "colden:leaf"):
        assert want in names, (want, sorted(names))
    # kernel-kind ranges of an evaluation sit inside its entry-point range
    inside = [p for n, p in seen if n in ("colden:shell", "colden:leaf")]
    assert inside and all("colden:column_density" in p for p in inside), inside[:3]
    assert all("colden:tree_update" in p or "colden:build_tree_uniform" in p
               for n, p in seen if n == "colden:restrict")
