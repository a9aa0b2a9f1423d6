"""The input recipe on the CPU: the seeded generators that both the CUDA path
and the oracle are given draw what the recipe says, reproducibly."""
import numpy as np
import pytest

from paper_1805_12258_gb300 import synth


def test_noise_is_seeded_and_row_addressable():
    a = synth.noise(9, 5000, seed=7)
    b = synth.noise(9, 5000, seed=7)
    assert a.dtype == np.float32 and a.shape == (9, 5000)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.noise(9, 5000, seed=8))
    # any row can be drawn on its own (row r uses the stream of (seed, r))
    for r in (0, 4, 8):
        assert np.array_equal(a[r], synth.noise(1, 5000, seed=7, row_offset=r)[0])
    # a preallocated output receives the same values
    out = np.empty((9, 5000), np.float32)
    assert synth.noise(9, 5000, seed=7, out=out) is out and np.array_equal(out, a)


def test_noise_is_unit_mean_exponential():
    x = synth.noise(5, 200000, seed=1).astype(np.float64).ravel()
    assert x.min() >= 0.0
    assert abs(x.mean() - 1.0) < 0.01 and abs(x.var() - 1.0) < 0.02
    # P(X > 3) = e^-3 for Exponential(1)
    assert abs((x > 3).mean() - np.exp(-3)) < 0.002


def test_workload_shapes():
    s, k = synth.small_plane(), synth.ska_plane()
    assert (s.n_templates, s.n_bins, s.H, s.p_fa, s.n_signals) == (21, 65536, 8, 1e-6, 5)
    assert (k.n_templates, k.n_bins, k.H, k.p_fa, k.n_signals) == (85, 1 << 21, 16, 1e-8, 50)


@pytest.mark.parametrize("make", [synth.small_plane, synth.ska_plane])
def test_signals_stay_inside_the_rows(make):
    wl = make()
    sigs = synth.draw_signals(wl)
    assert len(sigs) == wl.n_signals
    Z = (wl.n_templates - 1) // 2
    for s in sigs:
        assert wl.f0_range[0] <= s.f0 < wl.f0_range[1]
        assert wl.z0_range[0] <= s.z0 <= wl.z0_range[1]
        assert abs(s.z0) * wl.H <= Z  # every harmonic row exists
        assert s.amps.shape == (wl.H,) and (s.amps >= 3).all() and (s.amps <= 8).all()
    assert [(s.z0, s.f0) for s in sigs] == [(s.z0, s.f0) for s in synth.draw_signals(wl)]


def test_inject_adds_each_harmonic_once_where_it_fits():
    plane = np.zeros((21, 1000), np.float32)
    sig = synth.Signal(z0=1, f0=150, amps=np.arange(1, 9, dtype=np.float32))
    synth.inject(plane, [sig])
    Z = 10
    for h in range(1, 9):
        f = h * 150
        expect = float(h) if f < 1000 and h <= Z else 0.0
        if f < 1000:
            assert plane[h + Z, f] == expect
    assert plane.sum() == sum(h for h in range(1, 9) if h * 150 < 1000)


def test_beam_lengths():
    n = synth.beam_lengths()
    assert n.shape == (64,) and n.dtype == np.int64
    assert (n >= 2 ** 18).all() and (n <= 2 ** 22).all()
    assert np.array_equal(n, synth.beam_lengths())
    # log-uniform: about half the beams below 2^20
    assert 16 <= (n < 2 ** 20).sum() <= 48


def test_thresholds_are_per_level_and_row_independent():
    ta = synth.thresholds(1e-8, 16, 85)
    assert ta.shape == (16, 85) and ta.dtype == np.float32
    assert (ta == ta[:, :1]).all()
    assert (np.diff(ta[:, 0]) > 0).all()
    # level 1: Q(1, T) = e^-T
    assert ta[0, 0] == np.float32(-np.log(1e-8))


def test_random_plane_range():
    p = synth.random_plane(5, 1000, seed=2, lo=-1.0, hi=1.0)
    assert p.dtype == np.float32 and p.min() >= -1.0 and p.max() < 1.0 and p.min() < 0


def test_sparse_plane_holds_its_points_and_zeros_elsewhere():
    rows, bins, vals = synth.sparse_points(7, 1000, 300, seed=3)
    assert len(set(zip(rows.tolist(), bins.tolist()))) == 300  # distinct positions
    assert (rows >= 0).all() and (rows < 7).all() and (bins >= 0).all() and (bins < 1000).all()
    assert vals.dtype == np.float32 and (vals >= 0).all()
    p = synth.sparse(7, 1000, 300, seed=3, ld=1004)
    assert p.shape == (7, 1004) and p.dtype == np.float32
    assert np.array_equal(p[rows, bins], vals)
    assert np.count_nonzero(p) == np.count_nonzero(vals) and not p[:, 1000:].any()
    assert np.array_equal(p, synth.sparse(7, 1000, 300, seed=3, ld=1004))
    with pytest.raises(ValueError):
        synth.sparse(7, 1000, 3, seed=3, ld=999)
