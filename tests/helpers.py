"""Small helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel_err(a, b, scale):
    """|a - b| / (|b| + scale): relative error with an absolute floor `scale`
    (the size of the state, e.g. Y0), so values near zero are not amplified."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) / (np.abs(b) + scale)


def max_abs_normals(orc, seed, tag, sets, paths, n_steps):
    """max_i |X_i| of each (set, path) stream, from the oracle's generator."""
    out = np.empty(len(paths))
    for k, (s, q) in enumerate(zip(sets, paths)):
        out[k] = np.abs(orc.normals(seed, tag, int(s), int(q), 0, n_steps)).max()
    return out


def gate(err, maxabs_x, tol, x_cut=4.0, pct=99.99):
    """The per-path gate: max error over paths whose normals all satisfy
    |X| <= x_cut must be <= tol, and so must the pct-th percentile over all
    paths (g_m extrapolates beyond the outer nodes, where the Lebesgue function
    amplifies rounding).  Returns (ok, max_in, pct_all, max_all)."""
    inside = maxabs_x <= x_cut
    max_in = float(err[inside].max()) if inside.any() else 0.0
    p = float(np.percentile(err, pct))
    return (max_in <= tol and p <= tol), max_in, p, float(err.max())


def flat_sets(offsets, idx):
    offsets = np.asarray(offsets)
    s = np.searchsorted(offsets, idx, side="right") - 1
    return s, idx - offsets[s]


def with_biases(P, shapes, scale, seed):
    """Flat parameters P (per layer W [out][in], then b; `shapes` the layers' (out, in)) with every
    bias drawn from U(-scale, scale): Xavier parameters have zero biases."""
    P = P.copy()
    rng = np.random.default_rng(seed)
    o = 0
    for fo, fi in shapes:
        o += fo * fi
        P[o:o + fo] = rng.uniform(-scale, scale, fo)
        o += fo
    assert o == len(P)
    return P
