"""The checked build (libsevenleague_checked.so, compiled with -DSL_CHECKED): the kernels verify
the indices they derive from caller data -- a path's set s against path_offsets
(offsets[s] <= g < offsets[s+1]), a listed path against the path count -- and report a status
bit and skip the path's outputs instead of trusting the index.

* On valid inputs the checked build sets no status bit and gives bit-identical outputs to the
  normal build (7L samplers in both forms, 7L-CDC, BF16 adjoint): the checks change no
  arithmetic.
* Paths outside every set -- total_paths past offsets[n_sets], or offsets[0] > 0 -- are reported
  as SL_DEV_OFFSETS by each sampler.  (Neither input makes the normal build read or write
  outside its arrays: every index stays below total_paths and n_sets.)

ctypes loads one library per process, so each build runs in a child process of its own.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2302_05170_b300 as sl
from paper_2302_05170_b300 import workloads as W

sl.load(sys.argv[2])
mode, out = sys.argv[3], sys.argv[4]
dev = lambda a, dt=torch.float32: torch.as_tensor(np.asarray(a), dtype=dt, device="cuda")
res = {}
P = W.xavier_params(4, 7, seed=1)
Pc = W.near_affine_params(4, 7, seed=2)
th = W.gbm_online_thetas(3)
y0 = np.ones(3, np.float32)
if mode == "valid":
    off = W.offsets_from_counts([1000, 129, 2000])
    total = int(off[-1])
else:
    # paths outside every set: 150 paths but offsets covering 100, or offsets starting at 10
    off = np.array([0, 50, 80, 100], np.int64) if mode == "short" else np.array([10, 50, 80, 150], np.int64)
    total = 150
for prec in (0, 1):
    yt = torch.zeros(total, device="cuda")
    ws = sl.seven_league_simulate_batched(0, sl.make_net(dev(P), 4, 7, prec=prec), dev(th), dev(y0),
                                          dev(off, torch.int64), 1.0, 8, 7, 3, out_YT=yt, total_paths=total)
    res["sim%d" % prec] = yt.cpu().numpy()
    res["st_sim%d" % prec] = sl.workspace_status(ws)
yt = torch.zeros(total, device="cuda")
ws = sl.seven_league_cdc_simulate_batched(0, sl.make_net(dev(Pc), 4, 7), dev(th), dev(y0), dev(off, torch.int64),
                                          1.0, 8, 7, 3, out_YT=yt, total_paths=total)
res["cdc"] = yt.cpu().numpy()
res["st_cdc"] = sl.workspace_status(ws)
if mode == "valid":
    paths = torch.zeros((4, total), device="cuda")
    ws = torch.empty(sl.adjoint_workspace_size(total, 3, 8, 4, 2), dtype=torch.uint8, device="cuda")
    sl.seven_league_adjoint(0, sl.make_net(dev(P), 4, 7, prec=1), dev(th), dev(y0), dev(off, torch.int64), 1.0, 8,
                            7, 3, 1.0, ckpt_k=4, out_paths=paths, ws=ws, total_paths=total)
    res["adj"] = paths.cpu().numpy()
    res["st_adj"] = sl.workspace_status(ws)
np.savez(out, **res)
"""


def _child(lib, mode, tmp_path):
    import paper_2302_05170_b300 as sl
    out = str(tmp_path / ("%s_%s.npz" % (os.path.basename(lib), mode)))
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib, mode, out], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    with np.load(out) as z:
        return {k: z[k] for k in z.files}


@pytest.fixture(scope="module")
def libs(sl):
    if not os.path.exists(sl.LIB_CHECKED_PATH):
        pytest.fail("libsevenleague_checked.so not built (paper_2302_05170_b300.build(checked=True))")
    return sl.LIB_PATH, sl.LIB_CHECKED_PATH


def test_checked_build_matches_on_valid_inputs(libs, tmp_path):
    normal = _child(libs[0], "valid", tmp_path)
    checked = _child(libs[1], "valid", tmp_path)
    for k in normal:
        if k.startswith("st_"):
            assert normal[k] == 0 and checked[k] == 0, k
        else:
            assert np.array_equal(normal[k], checked[k]), k


@pytest.mark.parametrize("mode", ["short", "start"])
def test_checked_build_reports_paths_outside_every_set(libs, tmp_path, mode):
    import paper_2302_05170_b300 as sl
    r = _child(libs[1], mode, tmp_path)
    for k in ("st_sim0", "st_sim1", "st_cdc"):
        assert int(r[k]) & sl.SL_DEV_OFFSETS, (k, int(r[k]))
