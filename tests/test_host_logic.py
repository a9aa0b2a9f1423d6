"""Host logic of the staged kernel, on the CPU (no GPU needed).

The fast pass (the staged kernel's prefilter) tests each level group of Eq. 2
only at its last level, against a bound below every threshold of the group,
and carries the bounds inside its FP32 sums.  It may mark too much, never too
little: a point whose FP32 level sum (ascending m, the order of Eq. 2) exceeds
its threshold must be marked.  These tests take the bounds the library
computes (hs_prefilter_bounds), redo the fast pass's FP32 arithmetic in numpy
in the kernel's order (each group's bound difference added to its last
level, each group summed as a pairwise tree, the groups chained), and check
that promise on inputs built to sit within a few ulps above a threshold; for
16-bit planes the fast pass sees the rounded values and the truth is the
FP32 copy.  The tile orders are checked as permutations with their sort keys.
"""
import math

import numpy as np
import pytest

from paper_1805_12258_gb300 import build as hsbuild
from paper_1805_12258_gb300 import hs, synth


@pytest.fixture(scope="module", autouse=True)
def _library():
    hsbuild.build()  # no-op when libhs.so is up to date


def group_ranges(ends):
    lo = 1
    out = []
    for e in ends:
        out.append((lo, int(e)))
        lo = int(e) + 1
    return out


def tree_sum(cur, lo, hi):
    """Pairwise sum of cur[:, lo..hi] (0-based, inclusive), split at the
    midpoint like the kernel's tree, in float32."""
    if lo == hi:
        return cur[:, lo]
    mid = (lo + hi) // 2
    return (tree_sum(cur, lo, mid) + tree_sum(cur, mid + 1, hi)).astype(np.float32)


def fast_pass_marks(v, ends, bounds):
    """Per row and group: True when the group's folded sign test passes.
    v: [rows, H] float32 values as the kernel loads them."""
    v = v.astype(np.float32)
    groups = group_ranges(ends)
    b = bounds.astype(np.float32)
    cur = v.copy()
    for g, (_, hi) in enumerate(groups):
        c = -b[0] if g == 0 else np.float32(b[g - 1] - b[g])
        cur[:, hi - 1] = (cur[:, hi - 1] + c).astype(np.float32)
    marks = np.zeros((v.shape[0], len(groups)), bool)
    acc = None
    for g, (lo, hi) in enumerate(groups):
        gs = tree_sum(cur, lo - 1, hi - 1)
        acc = gs if acc is None else (acc + gs).astype(np.float32)
        marks[:, g] = ~np.signbit(acc)
    return marks


def true_hits(v32, ta_rows, ends):
    """Per row and group: True when some level of the group has its FP32
    ascending sum above the row's threshold.  ta_rows: [rows, H]."""
    acc = np.zeros(v32.shape[0], np.float32)
    hit_level = np.zeros(v32.shape, bool)
    for m in range(v32.shape[1]):
        acc = v32[:, 0].copy() if m == 0 else (acc + v32[:, m]).astype(np.float32)
        hit_level[:, m] = acc > ta_rows[:, m]
    return np.stack([hit_level[:, lo - 1:hi].any(axis=1) for lo, hi in group_ranges(ends)],
                    axis=1)


def to_bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even), back as float32."""
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def stored(v32, dtype):
    if dtype == "f32":
        return v32
    if dtype == "bf16":
        return to_bf16(v32)
    return v32.astype(np.float16).astype(np.float32)


def near_threshold_rows(rng, ta_rows, n, H, tiny_frac=0.0):
    """Rows of non-negative float32 values whose FP32 ascending sum at a
    random level k sits on the smallest float32 above TA(k, row)."""
    v = rng.exponential(size=(n, H)).astype(np.float32)
    # mixed magnitudes: some values much smaller than the rest
    small = rng.random((n, H)) < 0.3
    v[small] *= np.float32(1e-3)
    if tiny_frac:
        tiny = rng.random((n, H)) < tiny_frac
        v[tiny] = rng.uniform(0, 6e-5, size=tiny.sum()).astype(np.float32)
    k = rng.integers(1, H + 1, size=n)
    acc = np.cumsum(v.astype(np.float64), axis=1)
    t = ta_rows[np.arange(n), k - 1].astype(np.float64)
    scale = t / acc[np.arange(n), k - 1]
    v = (v.astype(np.float64) * scale[:, None]).astype(np.float32)
    # a value above every threshold is a hit wherever it lands; keep it inside
    # the FP16 range
    v = np.minimum(v, np.float32(1000.0))

    def chain_at_k(v):
        a = v[:, 0].copy()
        out = np.where(k == 1, a, np.float32(0))
        for m in range(1, H):
            a = (a + v[:, m]).astype(np.float32)
            out = np.where(k == m + 1, a, out)
        return out

    rows = np.arange(n)
    tk = ta_rows[rows, k - 1]
    # steps of v_k that move the chain by about one ulp of the threshold (for
    # k = 1 the chain is v_1 itself: step to the next float)
    half = (np.spacing(tk) / 2).astype(np.float32)

    def step(sel, up):
        # at least to the next float of v_k, so every step moves it
        i, m = rows[sel], k[sel] - 1
        if up:
            nxt = np.maximum(np.nextafter(v[i, m], np.float32(np.inf)),
                             (v[i, m] + half[sel]).astype(np.float32))
            nxt = np.where(k[sel] == 1, np.nextafter(v[i, m], np.float32(np.inf)), nxt)
        else:
            nxt = np.minimum(np.nextafter(v[i, m], np.float32(0)),
                             (v[i, m] - half[sel]).astype(np.float32))
            nxt = np.where(k[sel] == 1, np.nextafter(v[i, m], np.float32(0)), nxt)
        v[i, m] = np.maximum(nxt, np.float32(0))

    # walk v_k down until the chain is at or below TA, then up until just above
    for _ in range(200):
        hi = chain_at_k(v) > tk
        if not hi.any():
            break
        step(hi, up=False)
    for _ in range(200):
        lo = chain_at_k(v) <= tk
        if not lo.any():
            break
        step(lo, up=True)
    c = chain_at_k(v)
    assert (c > tk).all()
    assert (c <= tk + 4 * np.spacing(tk)).all()  # within a few ulps above
    return v


@pytest.mark.parametrize("H,ends", [(16, [2, 4, 8, 12, 16]), (8, [2, 4, 8]),
                                    (13, [2, 4, 8, 12, 13]), (2, [2]), (5, [2, 4, 5])])
def test_group_ends(H, ends):
    ta = synth.thresholds(1e-6, H, 21)
    got, bounds = hs.hs_prefilter_bounds(ta)
    assert list(got) == ends and len(bounds) == len(ends)


@pytest.mark.parametrize("dtype,slack", [("f32", 2.0 ** -12), ("bf16", 2.0 ** -7),
                                         ("f16", 2.0 ** -10)])
def test_bounds_lie_just_below_the_group_minimum(dtype, slack):
    rng = np.random.default_rng(5)
    H, nt = 16, 85
    ta = synth.thresholds(1e-8, H, nt) * rng.uniform(1.0, 1.3, size=(1, nt)).astype(np.float32)
    ends, bounds = hs.hs_prefilter_bounds(ta, dtype)
    for (lo, hi), b in zip(group_ranges(ends), bounds):
        gmin = float(ta[lo - 1:hi, :].min())
        assert b < gmin
        assert b >= gmin * (1 - slack)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("H", [16, 8])
def test_fast_pass_never_drops_a_hit(dtype, H):
    rng = np.random.default_rng(11 + H)
    nt, n = 85, 60000
    # thresholds differ by row, so a group's bound is below most rows' values
    ta = synth.thresholds(1e-8, H, nt) * rng.uniform(1.0, 1.05, size=(1, nt)).astype(np.float32)
    ends, bounds = hs.hs_prefilter_bounds(ta, dtype)
    row = rng.integers(0, nt, size=n)
    ta_rows = np.ascontiguousarray(ta[:, row].T)
    v32 = near_threshold_rows(rng, ta_rows, n, H, tiny_frac=0.2 if dtype == "f16" else 0.0)
    hits = true_hits(v32, ta_rows, ends)
    assert hits.any(axis=1).all()  # every row holds a hit at its level k
    marks = fast_pass_marks(stored(v32, dtype), ends, bounds)
    missed = hits & ~marks
    assert not missed.any(), np.argwhere(missed)[:5]


def test_the_check_sees_an_unlowered_bound():
    # the same check with the bounds left at the plain group minimum misses
    # hits of BF16 planes: the lowering is what the promise rests on
    rng = np.random.default_rng(3)
    H, nt, n = 16, 85, 20000
    ta = synth.thresholds(1e-8, H, nt)
    ends, _ = hs.hs_prefilter_bounds(ta, "bf16")
    plain = np.array([ta[lo - 1:hi, :].min() for lo, hi in group_ranges(ends)], np.float32)
    row = rng.integers(0, nt, size=n)
    ta_rows = np.ascontiguousarray(ta[:, row].T)
    v32 = near_threshold_rows(rng, ta_rows, n, H)
    hits = true_hits(v32, ta_rows, ends)
    marks = fast_pass_marks(stored(v32, "bf16"), ends, plain)
    assert (hits & ~marks).any()


def test_prefilter_bounds_validation():
    ta = synth.thresholds(1e-6, 16, 85)
    with pytest.raises(hs.HsError):
        hs.hs_prefilter_bounds(ta[:, :84])  # even template count
    with pytest.raises(hs.HsError):
        hs.hs_prefilter_bounds(np.ones((17, 85), np.float32))  # H > 16


def octave_key(t):
    if t == 0:
        return (1.0, -1)
    e = int(t).bit_length() - 1
    return (t / 2.0 ** e, e)


def semitone_key(t, steps=12.0):
    if t == 0:
        return -1.0
    x = steps * math.log2(t)
    return x - math.floor(x)


def step53_key(t):
    return semitone_key(t, 53.0)


@pytest.mark.parametrize("n", [0, 1, 2, 7, 1000, 16384])
def test_tile_orders(n):
    lin = hs.hs_tile_order(n, 1)
    assert np.array_equal(lin, np.arange(n, dtype=np.uint32))
    for order, key in ((2, octave_key), (3, semitone_key), (4, step53_key)):
        o = hs.hs_tile_order(n, order)
        assert np.array_equal(np.sort(o), np.arange(n, dtype=np.uint32))
        keys = [key(int(t)) for t in o]
        assert all(a <= b for a, b in zip(keys, keys[1:]))
    assert np.array_equal(hs.hs_tile_order(n, 0), hs.hs_tile_order(n, 4))


def test_semitone_order_keeps_thirds_close():
    # tiles t and 3t (the span of m = 3 of tile 3t is tile t's level 1) are
    # visited within a small fraction of the plane of each other; in the
    # octave order they are far apart
    n = 16384
    pos = {}
    for order in (2, 3):
        o = hs.hs_tile_order(n, order)
        p = np.empty(n, np.int64)
        p[o] = np.arange(n)
        t = np.arange(n // 8, n // 3)
        pos[order] = np.abs(p[3 * t] - p[t]) / n
    assert np.median(pos[3]) < 0.05 < np.median(pos[2])


def test_53_step_order_keeps_fifths_closer():
    # tiles t and 5t (the span of m = 5 of tile 5t is tile t's level 1):
    # 2^(123/53) = 4.99 against 2^(28/12) = 5.04, so the 53-step order visits
    # them nearer together than the semitone order does
    n = 16384
    pos = {}
    for order in (3, 4):
        o = hs.hs_tile_order(n, order)
        p = np.empty(n, np.int64)
        p[o] = np.arange(n)
        t = np.arange(n // 16, n // 5)
        pos[order] = np.abs(p[5 * t] - p[t]) / n
    assert np.median(pos[4]) < np.median(pos[3])


def test_tile_order_validation():
    with pytest.raises(hs.HsError):
        hs.hs_tile_order(10, 5)
    with pytest.raises(hs.HsError):
        hs.hs_tile_order(-1, 1)
