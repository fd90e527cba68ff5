"""GPU parity of the offline stage (Algorithm I step 1) against the oracle.

* Euler-Maruyama terminal samples (Eq. 6.2) for GBM, OU and CIR (full
  truncation): FP32 against FP64 on the same Philox normals, per path within
  1e-5 of |a - b| / (|b| + s) (s = the row's start value or long-run level).
* Segmented order statistics: bit-exact against the oracle's sort on ragged
  segments (empty, length 1, ties, NaN for ranks past the end), short segments at
  every alignment and a base pointer off a 16-byte boundary.
* Labels: the GPU's empirical quantiles differ from the oracle's by at most
  the largest per-path sample difference of the row (order statistics are
  1-Lipschitz in the sup norm), and equal the select of the GPU's own samples.
* Full-size CIR workload (1024 rows x 1e5 paths x 100 fine steps): sampled
  rows against the oracle.
"""
import numpy as np
import pytest
import torch

from paper_2302_05170_b300 import workloads as W
from tests.helpers import rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _dev(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda")


def _scale(sde, th, yi):
    if sde == 2:
        return np.maximum(th[:, 1], np.abs(yi))[:, None]
    return np.abs(yi)[:, None] + 0.1


@pytest.mark.parametrize("sde", [0, 1, 2])
def test_em_terminal(sl, orc, sde):
    if sde == 0:
        th = np.array([[0.1, 0.3], [0.0, 0.5], [0.2, 0.1]], np.float32)
        yi = np.array([1.0, 0.5, 3.0], np.float32)
    elif sde == 1:
        th = np.array([[0.4, 0.3, 1.5], [-0.2, 0.6, 0.3], [1.0, 0.1, 2.0]], np.float32)
        yi = np.array([1.0, 0.0, -1.0], np.float32)
    else:
        th, yi, _ = W.cir_label_rows(3)
    dt = np.array([0.5, 1.0, 0.1], np.float32)
    n, nf = 3001, 100
    got = sl.em_terminal(sde, _dev(th), _dev(yi), _dev(dt), n, nf, 5).cpu().numpy()
    want = orc.em_terminal(sde, th, yi, dt, n, nf, 5)
    err = rel_err(got, want, _scale(sde, th, yi))
    assert err.max() <= TOL, err.max()
    if sde == 2:
        assert got.min() >= 0.0


def test_em_ragged_fine_steps(sl, orc):
    th, yi, dt = W.cir_label_rows(2)
    for nf in (1, 3, 7, 101):
        got = sl.em_terminal(2, _dev(th), _dev(yi), _dev(dt), 300, nf, 8).cpu().numpy()
        want = orc.em_terminal(2, th, yi, dt, 300, nf, 8)
        assert rel_err(got, want, _scale(2, th, yi)).max() <= TOL


@pytest.mark.parametrize("ties", [False, True])
def test_select_bit_exact(sl, orc, ties):
    v, off = W.random_segments(300, 5000, seed=12, ties=ties)
    v[:50] = -0.0 if ties else v[:50]
    ranks = np.array([0, 1, 7, 100, 2499, 4999])
    got = sl.segmented_select(_dev(v), _dev(off, torch.int64), ranks).cpu().numpy()
    want = orc.order_statistics(v, off, ranks)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert np.array_equal(got[fin], want[fin].astype(np.float32))


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
def test_select_short_and_misaligned(sl, orc, shift):
    """Segments of every length 0..41 at every 4-value alignment, read from a base pointer
    `shift` values past a 16-byte boundary: the select's unaligned head and tail, the aligned
    float4 body and segments with no body at all."""
    rng = np.random.default_rng(7 + shift)
    lens = np.concatenate([np.arange(42), np.arange(42)[::-1], rng.integers(0, 9, 40)])
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    v = rng.standard_normal(int(off[-1])).astype(np.float32)
    v[rng.integers(0, v.size, 30)] = 0.5                      # ties
    ranks = np.array([0, 1, 2, 3, 5, 8, 20, 40])
    buf = torch.zeros(v.size + 8, dtype=torch.float32, device="cuda")
    view = buf[shift:shift + v.size]
    view.copy_(_dev(v))
    got = sl.segmented_select(view, _dev(off, torch.int64), ranks).cpu().numpy()
    want = orc.order_statistics(v, off, ranks)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    fin = ~np.isnan(want)
    assert np.array_equal(got[fin], want[fin].astype(np.float32))


def test_select_large_segment(sl, orc):
    rng = np.random.default_rng(3)
    n = 1_000_003
    v = (rng.standard_normal(n) ** 3).astype(np.float32)
    v[::97] = 0.0
    off = np.array([0, 17, n], np.int64)
    ranks = orc.quantile_ranks(7, n - 17)
    got = sl.segmented_select(_dev(v), _dev(off, torch.int64), ranks).cpu().numpy()
    want = orc.order_statistics(v, off, ranks)
    assert np.array_equal(got[1], want[1].astype(np.float32))


@pytest.mark.parametrize("kind", ["atom", "atom_denormal", "narrow", "spread", "mixed"])
def test_select_value_distributions(sl, orc, kind):
    """Value distributions that stress a radix select's digit histograms.  atom: half of each
    segment exactly 0 (CIR's full truncation makes such atoms), ranks inside and outside it;
    atom_denormal: the atom (+0 and -0) shares its first-digit bin with positive denormals, and
    ranks fall on both sides of the zeros' count inside that bin; narrow: every value in
    [1, 1 + 2^-10), so the keys share their top 11 bits; spread: lognormal values; mixed: segments
    of each kind in one call.  Bit for bit against the oracle's sort."""
    rng = np.random.default_rng({"atom": 1, "narrow": 2, "spread": 3, "mixed": 4, "atom_denormal": 5}[kind])
    n, n_seg = 100_000, 6
    segs = []
    for k in range(n_seg):
        sk = kind if kind != "mixed" else ("atom", "narrow", "spread")[k % 3]
        if sk == "atom_denormal":
            v = rng.lognormal(-2, 1, n).astype(np.float32)
            z = rng.random(n)
            v[z < 0.3] = 0.0
            v[(z >= 0.3) & (z < 0.35)] = -0.0
            den = (z >= 0.35) & (z < 0.36)            # ~1000 positive denormals in the +0 bin
            v[den] = (rng.integers(1, 1 << 18, int(den.sum())).astype(np.uint32)).view(np.float32)
            segs.append(v)
            continue
        if sk == "atom":
            v = rng.lognormal(-2, 1, n)
            v[rng.random(n) < 0.5] = 0.0
        elif sk == "narrow":
            v = 1.0 + rng.random(n) * 2.0 ** -10
        else:
            v = rng.lognormal(0, 0.5, n)
        segs.append(v.astype(np.float32))
    v = np.concatenate(segs)
    off = W.offsets_from_counts([n] * n_seg)
    ranks = np.concatenate([orc.quantile_ranks(7, n), [0, n - 1, n // 2 - 1, n // 2]])
    if kind == "atom_denormal":   # around the end of the zeros, inside the denormals, just above them
        nz = int(np.sum(v[:n] == 0.0))
        ranks = np.concatenate([ranks, [nz - 1, nz, nz + 1, nz + 500, 36_500]])
    got = sl.segmented_select(_dev(v), _dev(off, torch.int64), ranks).cpu().numpy()
    want = orc.order_statistics(v, off, ranks)
    assert np.array_equal(got, want.astype(np.float32))
    if kind == "atom_denormal":
        assert np.any((want > 0) & (want < 1.2e-38))          # some ranks landed on denormals


@pytest.mark.parametrize("c", [22528, 40959, 40960, 40961, 60000])
def test_select_candidate_capacity(sl, orc, c):
    """A segment whose requested ranks sit in one narrow cluster of c values (1 + k 2^-22, many of
    them repeated) among values spread over many binades: the cluster's first-digit bin holds c
    values.  The select copies the ranks' bins to shared memory when they hold at most 40,960
    values together, so c up to 40960 takes its shared-memory finish and 40961, 60000 its
    refining passes (with ranks outside the cluster too, every c from 40960 on refines).  Bit for
    bit against the oracle's sort, ranks at both ends of the cluster."""
    rng = np.random.default_rng(c)
    far = np.concatenate([rng.uniform(2.0 ** -40, 2.0 ** -20, 30_000), rng.uniform(4.0, 2.0 ** 40, 30_000)])
    cl = 1.0 + rng.integers(0, 300, c) * 2.0 ** -22
    v = rng.permutation(np.concatenate([far, cl])).astype(np.float32)
    n = v.size
    lo = 30_000
    off = np.array([0, n, 2 * n], np.int64)
    v2 = np.concatenate([v, v[::-1]])
    inside = [lo, lo + 1, lo + c // 3, lo + c // 2, lo + c - 2, lo + c - 1]   # the cluster's bin alone
    for ranks in (np.array(inside), np.array(inside + [lo - 1, lo + c, 0, n - 1])):
        got = sl.segmented_select(_dev(v2), _dev(off, torch.int64), ranks).cpu().numpy()
        want = orc.order_statistics(v2, off, ranks)
        assert np.array_equal(got, want.astype(np.float32))


def test_labels_small(sl, orc):
    th, yi, dt = W.cir_label_rows(6)
    n, nf, m = 4000, 100, 7
    lab = sl.em_collocation_labels(2, _dev(th), _dev(yi), _dev(dt), n, nf, m, 3).cpu().numpy()
    got_t = sl.em_terminal(2, _dev(th), _dev(yi), _dev(dt), n, nf, 3)
    want_t = orc.em_terminal(2, th, yi, dt, n, nf, 3)
    want = orc.em_labels(2, th, yi, dt, n, nf, m, 3)
    bound = np.abs(got_t.cpu().numpy() - want_t).max(axis=1)
    assert np.all(np.abs(lab - want) <= bound[:, None] + 1e-12)
    # labels are the select of the GPU's own samples at the oracle's ranks
    ranks = orc.quantile_ranks(m, n)
    offs = torch.arange(0, (len(yi) + 1) * n, n, dtype=torch.int64, device="cuda")
    sel = sl.segmented_select(got_t.reshape(-1), offs, ranks).cpu().numpy()
    assert np.array_equal(sel, lab)
    assert np.array_equal(ranks, sl.quantile_ranks(m, n))


@pytest.mark.parametrize("sde,m", [(0, 5), (1, 7)])
def test_labels_gbm_ou(sl, orc, sde, m):
    if sde == 0:
        th = np.array([[0.1, 0.3], [0.05, 0.2]], np.float32)
        yi = np.array([1.0, 0.4], np.float32)
    else:
        th = np.array([[0.4, 0.3, 1.5], [0.0, 0.5, 0.7]], np.float32)
        yi = np.array([1.0, -0.3], np.float32)
    dt = np.array([0.25, 0.5], np.float32)
    lab = sl.em_collocation_labels(sde, _dev(th), _dev(yi), _dev(dt), 5000, 100, m, 11).cpu().numpy()
    want = orc.em_labels(sde, th, yi, dt, 5000, 100, m, 11)
    assert rel_err(lab, want, _scale(sde, th, yi)).max() <= TOL


def test_full_size_cir_labels_sampled(sl, orc):
    th, yi, dt = W.cir_label_rows(1024)
    n, nf, m = 100_000, 100, 7
    lab = sl.em_collocation_labels(2, _dev(th), _dev(yi), _dev(dt), n, nf, m, 1).cpu().numpy()
    assert np.all(np.isfinite(lab)) and np.all(np.diff(lab, axis=1) >= 0) and lab.min() >= 0
    for r in (0, 511, 1023):
        want = orc.em_labels(2, th, yi, dt, n, nf, m, 1, row0=r, n_rows=1)[0]
        assert rel_err(lab[r], want, max(th[r, 1], yi[r])).max() <= TOL
