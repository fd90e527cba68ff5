"""The allocation-free variant of the label generator.

Callers that cannot allocate device memory (an embedding application owns the
allocator, or the memory budget is fixed up front) use
em_collocation_labels_noalloc, which runs on the library's own fixed device
buffer instead of a caller workspace.  Checked here through the C ABI: two
calls in a row give the labels of em_collocation_labels (the existing entry
point, with a caller workspace) bit for bit -- the same kernels on the same
inputs -- and so does a third call after a call of the same size with another
seed has overwritten every sample of the shared buffer; sizes beyond the
buffer are rejected before any work, and bad arguments with the argument
errors of em_collocation_labels, not with the size error.

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
    args = (_dev(th), _dev(yi), _dev(dt), n_paths, n_fine, m)
    ref = sl.em_collocation_labels(2, *args, 5).cpu().numpy()
    for _ in range(2):   # the shared buffer keeps the previous call's contents
        got = sl.em_collocation_labels_noalloc(2, *args, 5)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), ref)
    # the same rows with another seed overwrite every sample of the buffer, then the first again
    other = sl.em_collocation_labels_noalloc(2, *args, 6).cpu().numpy()
    ref6 = sl.em_collocation_labels(2, *args, 6).cpu().numpy()
    assert np.array_equal(other, ref6) and not np.array_equal(other, ref)
    again = sl.em_collocation_labels_noalloc(2, *args, 5).cpu().numpy()
    assert np.array_equal(again, ref)


def test_noalloc_rejects_oversize(sl):
    th, yi, dt = W.cir_label_rows(64, seed=23)
    n_paths = sl.em_labels_noalloc_max_samples() // 64 + 1
    with pytest.raises(sl.SLError) as e:
        sl.em_collocation_labels_noalloc(2, _dev(th), _dev(yi), _dev(dt), n_paths, 100, 7, 5)
    assert e.value.status == sl.SL_ERR_WORKSPACE
    # argument errors come first, even for sizes beyond the buffer
    with pytest.raises(sl.SLError) as e:
        sl.em_collocation_labels_noalloc(7, _dev(th), _dev(yi), _dev(dt), n_paths, 100, 7, 5)
    assert e.value.status == sl.SL_ERR_ARG
    with pytest.raises(sl.SLError) as e:
        sl.em_collocation_labels_noalloc(2, _dev(th), _dev(yi), _dev(dt), n_paths, 100, 11, 5)
    assert e.value.status == sl.SL_ERR_UNSUPPORTED
