"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test pins the oracle to something other than itself: values printed in
the paper (tests/golden/), closed forms, invariants, or an independent
brute-force.  The comment on each test names the mistake it would catch.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_12258_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                parts = line.split()
                out[parts[0]] = parts[1]
    return out


def _rand(nt, n, seed, lo=0.0, hi=1.0):
    return synth.random_plane(nt, n, seed, lo=lo, hi=hi)


MODES = [(oracle.STRETCH, oracle.ZSYM), (oracle.STRETCH, oracle.ZFLOOR),
         (oracle.HFRAC, oracle.ZSYM), (oracle.HFRAC, oracle.ZFLOOR)]


# --- Eq. 2 base case and constants ------------------------------------------

@pytest.mark.parametrize("index,zround", MODES)
def test_hp1_is_fop(index, zround):
    # Eq. 2: HP_1 = SP_1 = FOP.  Catches an off-by-one in the level index.
    p = _rand(9, 40, 1)
    hp = oracle.planes(p, 5, index=index, zround=zround)
    assert np.array_equal(hp[0], p.astype(np.float64))


@pytest.mark.parametrize("index,zround", MODES)
def test_constant_plane(index, zround):
    # A constant plane c gives level value k*c at every point (exact in fp64
    # for c = 0.75).  Catches a dropped or doubled term at any level.
    p = np.full((11, 37), 0.75, np.float32)
    hp = oracle.planes(p, 7, index=index, zround=zround)
    for k in range(1, 8):
        assert np.all(hp[k - 1] == 0.75 * k)


def test_origin_point():
    # Every stretch maps (0, 0) to itself: HP_k(0, 0) = k * FOP(0, 0).
    p = _rand(13, 50, 2)
    hp = oracle.planes(p, 9)
    Z = 6
    for k in range(1, 10):
        assert hp[k - 1, Z, 0] == pytest.approx(k * float(p[Z, 0]), rel=1e-15)


# --- linearity and adjointness -----------------------------------------------

@pytest.mark.parametrize("index,zround", MODES)
def test_linearity(index, zround):
    # HS(aP + bQ) = a HS(P) + b HS(Q).  Catches any non-linear slip
    # (a threshold or max mixed into the sums, a stale accumulator).
    P, Q = _rand(9, 64, 3).astype(np.float64), _rand(9, 64, 4).astype(np.float64)
    a, b = 1.75, -0.5
    lhs = oracle.planes(a * P + b * Q, 6, index=index, zround=zround)
    rhs = a * oracle.planes(P, 6, index=index, zround=zround) + \
        b * oracle.planes(Q, 6, index=index, zround=zround)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("zround", [oracle.ZSYM, oracle.ZFLOOR])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8, 16])
def test_stretch_adjoint(zround, k):
    # <SP_k(P), W> = <P, SP_k^T(W)>.  The gather follows Eq. 1 forward; the
    # scatter is written from preimage intervals.  A wrong rounding of negative
    # rows, a transposed operand or an off-by-one in a range breaks equality.
    P = _rand(15, 97, 5 + k, -1.0, 1.0).astype(np.float64)
    W = _rand(15, 97, 50 + k, -1.0, 1.0).astype(np.float64)
    lhs = float(np.sum(oracle.stretch(P, k, zround=zround) * W))
    rhs = float(np.sum(P * oracle.stretch_adjoint(W, k, zround=zround)))
    assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)


def test_zround_readings_differ_only_on_negative_rows():
    # Symmetric and floor rounding agree for rows >= 0 and differ below.
    p = _rand(9, 30, 7)
    s = oracle.planes(p, 4, zround=oracle.ZSYM)
    f = oracle.planes(p, 4, zround=oracle.ZFLOOR)
    Z = 4
    assert np.array_equal(s[:, Z:], f[:, Z:])
    assert not np.array_equal(s[:, :Z], f[:, :Z])


def test_hfrac_matches_stretch_for_k_le_2():
    # The two index maps coincide for k = 1, 2 ({f} and {f/2, f}) and differ
    # for k = 3 ({f, f/2, f/3} against {f/3, 2f/3, f}).
    p = _rand(9, 60, 8)
    a = oracle.planes(p, 3, index=oracle.STRETCH)
    b = oracle.planes(p, 3, index=oracle.HFRAC)
    np.testing.assert_allclose(a[:2], b[:2], rtol=1e-15)
    assert not np.allclose(a[2], b[2])


# --- independent brute force ---------------------------------------------------

def _brute(p, H, index, zround):
    """Pure-Python restatement on tiny planes, from the paper's wording."""
    nt, n = p.shape
    Z = (nt - 1) // 2

    def rnd(x_num, den):
        # round the (possibly negative) rational x_num/den to a row index
        if zround == oracle.ZFLOOR or x_num >= 0:
            return x_num // den          # Python's // is floor division
        return -((-x_num) // den)

    out = np.zeros((H, nt, n))
    for zi in range(-Z, Z + 1):
        for f in range(n):
            for k in range(1, H + 1):
                if index == oracle.STRETCH:
                    terms = [(rnd(zi, m), f // m) for m in range(1, k + 1)]
                else:
                    terms = [(rnd(zi * h, k), (f * h) // k) for h in range(1, k + 1)]
                out[k - 1, zi + Z, f] = sum(float(p[r + Z, b]) for r, b in terms)
    return out


@pytest.mark.parametrize("index,zround", MODES)
def test_brute_force_tiny(index, zround):
    p = _rand(7, 23, 9)
    ref = _brute(p, 6, index, zround)
    got = oracle.planes(p, 6, index=index, zround=zround)
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=0)


# --- injected harmonic signals: closed forms ----------------------------------

def _divisor_sum(amps, n, k):
    return sum(float(amps[n // m - 1]) for m in range(1, k + 1)
               if n % m == 0 and n // m <= len(amps))


@pytest.mark.parametrize("zround", [oracle.ZSYM, oracle.ZFLOOR])
@pytest.mark.parametrize("z0,f0", [(1, 37), (-1, 53), (2, 41), (0, 29), (-3, 19)])
def test_injected_signal_stretch(zround, z0, f0):
    # Noise-free plane with A_h at (h z0, h f0), f0 > H.  Under Eq. 1-2,
    # HP_k(n z0, n f0) = sum of A_{n/m} over m <= k dividing n: a stretch by
    # a non-divisor m lands on floor(n f0/m), never a multiple of f0.
    H = 8
    nt = 2 * max(1, abs(z0)) * H + 1
    n = f0 * H + 5
    amps = np.arange(1, H + 1, dtype=np.float32) * 1.25 + 2.0
    plane = np.zeros((nt, n), np.float32)
    synth.inject(plane, [synth.Signal(z0, f0, amps)])
    Z = (nt - 1) // 2
    hp = oracle.planes(plane, H, zround=zround)
    for nn in range(1, H + 1):
        for k in range(1, H + 1):
            assert hp[k - 1, nn * z0 + Z, nn * f0] == _divisor_sum(amps, nn, k)


@pytest.mark.parametrize("z0,f0", [(1, 37), (-2, 41), (0, 29)])
def test_injected_signal_hfrac(z0, f0):
    # Harmonic-fraction map: S_k(k z0, k f0) = A_1 + ... + A_k.
    H = 8
    nt = 2 * max(1, abs(z0)) * H + 1
    n = f0 * H + 3
    amps = np.linspace(3.0, 8.0, H).astype(np.float32)
    plane = np.zeros((nt, n), np.float32)
    synth.inject(plane, [synth.Signal(z0, f0, amps)])
    Z = (nt - 1) // 2
    for k in range(1, H + 1):
        v = oracle.sample(plane, H, [k * z0], [k * f0], index=oracle.HFRAC)[0, k - 1]
        assert v == sum(float(a) for a in amps[:k])


def test_delta_response_counts():
    # A unit delta at (r0, p0): HP_k(z, f) counts the m <= k whose stretch
    # reads (r0, p0).  Summed over the plane this is the number of output
    # points mapped onto (r0, p0), i.e. sum_m |preimage_m|.
    nt, n, H = 17, 64, 6
    Z = 8
    r0, p0 = 2, 5
    plane = np.zeros((nt, n), np.float32)
    plane[r0 + Z, p0] = 1.0
    hp = oracle.planes(plane, H)
    # preimage sizes for r0 > 0 (symmetric rounding): m rows x m bins
    expect_total = sum(min(m, Z - m * r0 + 1 if m * r0 <= Z else 0) * m
                       for m in range(1, H + 1))
    assert hp[-1].sum() == expect_total


# --- touch counts printed in Section IV-A ----------------------------------------

def _touch_counts():
    """Per-point touch counts of a 64 x 4096 plane (rows from 0), SP_1..SP_8."""
    rows, n, H = 64, 4096, 8
    nt = 2 * rows - 1            # symmetric plane whose top half is rows 0..63
    Z = rows - 1
    w = np.zeros((nt, n))
    w[Z:, :] = 1.0               # only outputs of the top half
    touch = np.zeros((nt, n))
    for m in range(1, H + 1):
        touch += oracle.stretch_adjoint(w, m)
    return touch[Z:, :]


def test_touch_counts_section_iv_a():
    g = _golden_kv("touch_counts.txt")
    t = _touch_counts()
    assert t.max() == float(g["max_touches"])
    zr, zb = int(g["zoom_rows"]), int(g["zoom_bins"])
    share = t[:zr, :zb].sum() / t.sum() * 100
    assert round(share, 1) == float(g["zoom_share_percent"])
    srt = np.sort(t.ravel())[::-1]
    cum = np.cumsum(srt) / srt.sum() * 100
    top = int(round(float(g["top_share_points_percent"]) / 100 * srt.size))
    assert abs(cum[top - 1] - float(g["top_share_touch_percent"])) < 0.5
    q = int(round(float(g["quarter_points_percent"]) / 100 * srt.size))
    assert abs(cum[q - 1] - float(g["quarter_touch_percent"])) < 1.0
    # the max-touch area under Eq. 1 is 8 x 512 points (the paper says 1.7%)
    assert np.count_nonzero(t == t.max()) == 8 * 512


# --- Table II and the necessary-points figures of Section IV-C -------------------

def _needed_points(rows, cols, m, c0, H_rows_from_zero=True):
    """Distinct plane points read at level m by output rows 0..rows-1 and
    output columns [c0, c0+cols), via the oracle's Eq. 1 adjoint."""
    n = c0 + cols + 1
    nt = 2 * rows + 1
    Z = rows
    w = np.zeros((nt, n))
    w[Z:Z + rows, c0:c0 + cols] = 1.0
    return int(np.count_nonzero(oracle.stretch_adjoint(w, m)))


def _needed_rows_cols(rows, cols, m, c0):
    n = c0 + cols + 1
    nt = 2 * rows + 1
    Z = rows
    w = np.zeros((nt, n))
    w[Z:Z + rows, c0:c0 + cols] = 1.0
    a = oracle.stretch_adjoint(w, m) != 0
    return int(a.any(axis=1).sum()), int(a.any(axis=0).sum())


def test_table_ii_loaded_points():
    rows_half, H = 42, 8
    table = {}
    with open(os.path.join(GOLDEN, "table2_loaded_points.txt")) as fh:
        for line in fh:
            line = line.split("#", 1)[0].split()
            if line:
                table[(int(line[0]), line[1])] = ([int(x) for x in line[2:6]],
                                                  [float(x) for x in line[6:10]])
    for cols in (1, 4, 16, 64):
        total = 0
        for m in range(1, H + 1):
            # aligned work-groups: c0 a multiple of cols; m positions cover
            # every residue of c0 modulo m
            total += max(_needed_points(rows_half, cols, m, cols * t) for t in range(m))
        plain, plain_ratio = table[(cols, "plain")]
        opt, opt_ratio = table[(cols, "opt")]
        for i, p in enumerate((1, 2, 4, 8)):
            lp = math.ceil(total * p / (rows_half * cols))
            assert lp == plain[i], (cols, p, lp)
            assert round(lp / p, 1) == plain_ratio[i]
            lp2 = 1 << (lp - 1).bit_length()
            assert lp2 == opt[i]
            assert round(lp2 / p, 1) == opt_ratio[i]


def test_necessary_points_section_iv_c():
    g = _golden_kv("necessary_points.txt")
    # a work-group of 8 aligned columns needs 3 or 4 FOP columns for HP_3
    widths = {_needed_rows_cols(42, 8, 3, 8 * t)[1] for t in range(3)}
    assert widths == {int(x) for x in g["hp3_columns_for_8_columns"].split(",")}
    # 16 columns per work-group, any start column, full plane as the paper
    # counts it: both template groups (rows from 0) plus the shared row 0
    total = 0
    for m in range(1, 9):
        r_half = max(_needed_rows_cols(42, 16, m, c)[0] for c in range(m))
        c_max = max(_needed_rows_cols(42, 16, m, c)[1] for c in range(m))
        total += (2 * r_half + 1) * c_max
    avg = total / 16
    assert abs(avg - float(g["avg_points_per_column_16_cols"])) < 0.1
    assert round(avg / 85, 2) == float(g["rfop_size_ratio_16_cols"])


# --- Algorithm 1 and Algorithm 2 orders agree --------------------------------

@pytest.mark.parametrize("index,zround", MODES)
def test_alg1_alg2_same_candidates(index, zround):
    nt, n, H = 11, 300, 6
    p = synth.noise(nt, n, 11)
    ta = synth.thresholds(1e-2, H, nt)
    hp = oracle.planes(p, H, index=index, zround=zround)
    cands, near = oracle.detect(p, H, ta, index=index, zround=zround)
    k, zi, f = np.nonzero(hp > ta.astype(np.float64)[:, :, None])
    assert len(cands) == len(k) > 0
    Z = (nt - 1) // 2
    ref = np.zeros(len(k), oracle.CAND_DTYPE)
    ref["k"], ref["z"], ref["f"] = k + 1, zi - Z, f
    ref["power"] = hp[k, zi, f]
    ref = oracle.sort_cands(ref)
    for key in ("k", "z", "f", "power"):
        assert np.array_equal(cands[key], ref[key])


def test_detect_threads_and_ranges_agree():
    nt, n, H = 9, 1000, 5
    p = synth.noise(nt, n, 12)
    ta = synth.thresholds(1e-2, H, nt)
    a, _ = oracle.detect(p, H, ta)
    b, _ = oracle.detect(p, H, ta, threads=4)
    assert np.array_equal(a, b)


def test_detection_is_strict():
    # Candidates need HP_k > TA(k, i): equality is not a hit (reading of
    # Section III, which does not name the comparison).
    nt, n, H = 5, 20, 4
    p = np.full((nt, n), 0.5, np.float32)
    ta = np.array([[0.5 * k] * nt for k in range(1, H + 1)], np.float32)
    c, near = oracle.detect(p, H, ta)
    assert len(c) == 0 and len(near) == nt * n * H
    c2, _ = oracle.detect(p, H, ta - np.float32(0.125))
    assert len(c2) == nt * n * H


def test_low_precision_inputs_convert_exactly():
    # bf16 and fp16 planes reach the oracle as their exact values.
    x = np.array([[0.5, 1.5, 3.0, 65504.0, 2.0 ** -24, -7.25]], np.float32)
    h = x.astype(np.float16)
    assert np.array_equal(oracle.stretch(h, 1), h.astype(np.float64))
    bits = (x.view(np.uint32) >> 16).astype(np.uint16)       # truncation is exact here
    bf = oracle.stretch(bits, 1, dtype_code=oracle.DT_BF16)
    assert np.array_equal(bf, (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64))


# --- thresholds of the synthetic recipe ---------------------------------------

def test_thresholds_closed_forms():
    p = 1e-6
    t = synth.level_thresholds(p, 16)
    assert t[0] == pytest.approx(-math.log(p), rel=1e-12)          # Q(1,T) = e^-T
    assert math.exp(-t[1]) * (1 + t[1]) == pytest.approx(p, rel=1e-10)  # Q(2,T)
    from scipy.special import gammaincc
    for k in range(1, 17):
        assert gammaincc(k, t[k - 1]) == pytest.approx(p, rel=1e-9)
    assert np.all(np.diff(t) > 0)
