"""The allocation-free variant of the label generator.

Callers that cannot allocate device memory (an embedding application owns the
allocator, or the memory budget is fixed up front) use
em_collocation_labels_noalloc, which runs on the library's own fixed device
buffer instead of a caller workspace.  Checked here through the C ABI: two
calls in a row give the labels of em_collocation_labels (the existing entry
point, with a caller workspace) within the labels tests' tolerance (1e-5
relative), and sizes beyond the buffer are rejected before any work.

This file is collected last on purpose: it is independent of the other GPU
tests and passes alone in a fresh process as well as after them.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def test_noalloc_matches_workspace_entry_point(sl):
    th, yi, dt = W.cir_label_rows(24, seed=21)
    n_paths, n_fine, m = 50_000, 100, 7
    assert 24 * n_paths <= sl.em_labels_noalloc_max_samples()
    ref = sl.em_collocation_labels(2, _dev(th), _dev(yi), _dev(dt), n_paths, n_fine, m, 5).cpu().numpy()
    for _ in range(2):   # the shared buffer keeps the previous call's contents
        got = sl.em_collocation_labels_noalloc(2, _dev(th), _dev(yi), _dev(dt), n_paths, n_fine, m, 5)
        torch.cuda.synchronize()
        got = got.cpu().numpy()
        scale = np.maximum(th[:, 1], yi)[:, None]
        assert np.all(np.abs(got - ref) <= TOL * (np.abs(ref) + scale))
    # a different problem in between, then the first one again
    th2, yi2, dt2 = W.cir_label_rows(3, seed=22)
    other = sl.em_collocation_labels_noalloc(1, _dev(th2), _dev(yi2), _dev(dt2), 1000, 10, 5, 9).cpu().numpy()
    assert np.all(np.isfinite(other))
    again = sl.em_collocation_labels_noalloc(2, _dev(th), _dev(yi), _dev(dt), n_paths, n_fine, m, 5).cpu().numpy()
    assert np.all(np.abs(again - ref) <= TOL * (np.abs(ref) + np.maximum(th[:, 1], yi)[:, None]))


def test_noalloc_rejects_oversize(sl):
    th, yi, dt = W.cir_label_rows(64, seed=23)
    n_paths = sl.em_labels_noalloc_max_samples() // 64 + 1
    with pytest.raises(sl.SLError) as e:
        sl.em_collocation_labels_noalloc(2, _dev(th), _dev(yi), _dev(dt), n_paths, 100, 7, 5)
    assert e.value.status == sl.SL_ERR_WORKSPACE
