"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance: FP32 level sums within 1e-6 relative of the oracle (the FP32
rounding bound of at most 15 ascending additions of non-negative terms is
below 9e-7); candidate sets identical except for points the oracle lists
within 1e-5 relative of their threshold.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1805_12258_gb300 import hs, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-6
NEAR = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1805_12258_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def run_gpu(plane, H, ta, *, cap=1 << 20, fop32=None, **plan_kw):
    nt, n = plane.shape
    if plane.dtype == np.uint16:  # bf16 bit patterns
        fop = torch.from_numpy(plane.view(np.int16)).cuda().view(torch.bfloat16)
    else:
        fop = torch.from_numpy(np.ascontiguousarray(plane)).cuda()
    cands = hs.CandBuffer(cap)
    with hs.Plan(nt, n, H, ta, **plan_kw) as plan:
        f32 = None if fop32 is None else torch.from_numpy(fop32).cuda()
        plan.run(fop, cands, fop_f32=f32)
        recs, count, st = cands.fetch()
        kernel = plan.kernel
    return recs, count, st, kernel


def assert_matches_oracle(recs, ref, near, *, rtol=RTOL):
    near_keys = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in near}
    g = {(int(r["k"]), int(r["z"]), int(r["bin"])): float(r["power"]) for r in recs}
    o = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in ref}
    assert len(g) == len(recs), "duplicate candidate records"
    only_gpu = set(g) - set(o) - near_keys
    only_ora = set(o) - set(g) - near_keys
    assert not only_gpu and not only_ora, (sorted(only_gpu)[:5], sorted(only_ora)[:5])
    common = sorted(set(g) & set(o))
    if common:
        gv = np.array([g[k] for k in common])
        ov = np.array([o[k] for k in common])
        err = np.abs(gv - ov) / np.maximum(np.abs(ov), 1e-30)
        assert err.max() <= rtol, (err.max(), common[int(err.argmax())])


# --- the small plane (21 x 65,536, H = 8) -------------------------------------

@pytest.mark.parametrize("kernel", ["staged", "generic"])
def test_small_plane_candidates(kernel):
    wl = synth.small_plane(seed=0)
    plane = synth.make_plane(wl)
    ta = synth.thresholds(wl.p_fa, wl.H, wl.n_templates)
    recs, n, st, used = run_gpu(plane, wl.H, ta, kernel=kernel)
    assert used == kernel and st == hs.HS_OK
    ref, near = oracle.detect(plane, wl.H, ta, threads=8)
    assert n == len(recs) and n > 0
    assert_matches_oracle(recs, ref, near)


# --- every level sum, by thresholds below every value --------------------------

def _all_sums(plane, H, **kw):
    nt, n = plane.shape
    ta = np.full((H, nt), -1e30, np.float32)
    recs, cnt, st, used = run_gpu(plane, H, ta, cap=nt * n * H, **kw)
    assert st == hs.HS_OK and cnt == nt * n * H
    Z = (nt - 1) // 2
    got = np.empty((H, nt, n), np.float64)
    got[recs["k"].astype(int) - 1, recs["z"].astype(int) + Z, recs["bin"].astype(int)] = \
        recs["power"]
    return got, used


@pytest.mark.parametrize("nt,n,H,kernel", [
    (21, 4096, 8, "staged"), (85, 2048, 16, "staged"), (21, 1000, 8, "staged"),
    (85, 300, 16, "staged"), (21, 4096, 8, "generic"), (85, 1000, 16, "generic"),
    (7, 333, 5, "generic"), (3, 5, 8, "generic"), (1, 17, 3, "generic"), (1, 1, 1, "generic"),
    (33, 129, 32, "generic")])
def test_every_level_sum(nt, n, H, kernel):
    plane = synth.noise(nt, n, seed=nt * 1000 + n)
    got, used = _all_sums(plane, H, kernel=kernel)
    assert used == kernel
    ref = oracle.planes(plane, H)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


@pytest.mark.parametrize("nt,n,H", [(21, 777, 8), (85, 1000, 16), (33, 500, 13)])
@pytest.mark.parametrize("index,zround", [("hfrac", "symmetric"), ("stretch", "floor"),
                                          ("hfrac", "floor")])
def test_other_index_maps(index, zround, nt, n, H):
    # The harmonic-fraction map with symmetric rounding at H = 8 or 16 runs
    # the staged kernel when rows are a multiple of 16 bytes and the gather
    # pair kernel otherwise (21 x 777); H = 13 and floor rounding run the
    # generic kernel
    plane = synth.noise(nt, n, seed=5)
    got, used = _all_sums(plane, H, index=index, zround=zround)
    staged = index == "hfrac" and zround == "symmetric" and H in (8, 16) and n % 4 == 0
    assert used == ("staged" if staged else "generic")
    ref = oracle.planes(plane, H, index=oracle.HFRAC if index == "hfrac" else oracle.STRETCH,
                        zround=oracle.ZFLOOR if zround == "floor" else oracle.ZSYM)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


# --- the harmonic-fraction map: staged (TMA) and gather kernels ------------------

@pytest.mark.parametrize("nt,n,H,tb", [(85, 1000, 16, 128), (85, 1000, 16, 64),
                                       (21, 776, 8, 128), (21, 776, 8, 64),
                                       (127, 520, 16, 128), (1, 300, 16, 128), (3, 64, 8, 64),
                                       (9, 4, 16, 128), (33, 2052, 8, 128), (43, 1300, 16, 64)])
def test_hfrac_staged_every_level_sum(nt, n, H, tb):
    # Row blocks of K pairs (the last one partial for every family head K
    # that does not divide the pair count), ragged last tiles, one template,
    # a plane narrower than a box
    plane = synth.noise(nt, n, seed=nt * 31 + n + tb)
    got, used = _all_sums(plane, H, index="hfrac", tile_bins=tb)
    assert used == "staged"
    ref = oracle.planes(plane, H, index=oracle.HFRAC)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


@pytest.mark.parametrize("nt,n,H", [(3, 200004, 16), (3, 200004, 8), (1, 300004, 16)])
def test_hfrac_large_plane_every_level_sum(nt, n, H):
    # thousands of tiles, the last one ragged
    plane = synth.noise(nt, n, seed=nt * 13 + n + H)
    got, used = _all_sums(plane, H, index="hfrac")
    assert used == "staged"
    ref = oracle.planes(plane, H, index=oracle.HFRAC)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_hfrac_candidates_equal_oracle_and_gather():
    nt, n, H = 85, 200004, 16
    plane = synth.noise(nt, n, seed=77)
    wl = synth.Workload("t", nt, n, H, 5, 1e-4, 12, (2000, 12000), (-2, 2))
    synth.inject(plane, synth.draw_signals(wl))
    ta = synth.thresholds(1e-5, H, nt)
    recs, cnt, st, used = run_gpu(plane, H, ta, index="hfrac")
    assert used == "staged" and st == hs.HS_OK and cnt > 0
    ref, near = oracle.detect(plane, H, ta, index=oracle.HFRAC, threads=16)
    assert_matches_oracle(recs, ref, near)
    g, _, st2, _ = run_gpu(plane, H, ta, index="hfrac", kernel="generic")
    assert st2 == hs.HS_OK and np.array_equal(np.sort(g, order=["k", "z", "bin"]),
                                               np.sort(recs, order=["k", "z", "bin"]))


def test_hfrac_padded_rows_never_read_the_pad():
    # a ragged plane in padded rows runs the staged kernel (its boxes end at
    # the last bin, so the pad -- NaN here -- is never read) and gives the
    # gather kernel's records on the unpadded plane, which are the oracle's
    nt, n, H = 85, 30011, 16
    plane = synth.noise(nt, n, seed=43)
    ta = synth.thresholds(1e-4, H, nt)
    ld = n + 5  # 30016: rows a multiple of 16 bytes
    padded = np.full((nt, ld), np.nan, np.float32)
    padded[:, :n] = plane
    dev = torch.from_numpy(padded).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(nt, n, H, ta, index="hfrac", row_pitch=ld) as plan:
        assert plan.kernel == "staged"
        plan.run(dev, cands)
        got, cnt, st = cands.fetch()
    assert st == hs.HS_OK and cnt > 0 and not np.isnan(got["power"]).any()
    ref, nref, _, used = run_gpu(plane, H, ta, index="hfrac")
    assert used == "generic" and np.array_equal(got, ref)
    o, near = oracle.detect(plane, H, ta, index=oracle.HFRAC, threads=8)
    assert_matches_oracle(got, o, near)


def test_hfrac_staged_at_the_largest_template_count():
    # 32,767 templates (Z = 16,383): thousands of row blocks per family, the
    # largest z a record holds; every level sum against the oracle
    nt, n, H = 32767, 64, 8
    plane = synth.noise(nt, n, seed=29)
    got, used = _all_sums(plane, H, index="hfrac")
    assert used == "staged"
    ref = oracle.planes(plane, H, index=oracle.HFRAC)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


@pytest.mark.parametrize("nt,n,H", [(85, 1000, 16), (21, 777, 8), (127, 333, 16), (1, 50, 8)])
def test_hfrac_gather_every_level_sum(nt, n, H):
    # the gather pair kernel: forced, or for rows that are not 16-byte multiples
    plane = synth.noise(nt, n, seed=nt * 37 + n)
    got, used = _all_sums(plane, H, index="hfrac", kernel="generic")
    assert used == "generic"
    ref = oracle.planes(plane, H, index=oracle.HFRAC)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_hfrac_kernels_orders_and_ranges_agree():
    # staged (linear and semitone tile order, 64 and 128 bins), gather and a
    # run split into two tile-aligned ranges give the same records, which
    # are the oracle's candidates
    nt, n, H = 85, 30000, 16
    plane = synth.noise(nt, n, seed=71)
    ta = synth.thresholds(1e-4, H, nt)
    runs = [dict(index="hfrac"), dict(index="hfrac", order=3), dict(index="hfrac", tile_bins=64),
            dict(index="hfrac", kernel="generic")]
    results = []
    for kw in runs:
        recs, cnt, st, _ = run_gpu(plane, H, ta, **kw)
        assert st == hs.HS_OK and cnt > 0
        results.append(np.sort(recs, order=["k", "z", "bin"]))
    fop = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(nt, n, H, ta, index="hfrac") as plan:
        plan.run_range(fop, cands, 0, 128 * 100)
        plan.run_range(fop, cands, 128 * 100, n, append=True)
        recs, cnt, st = cands.fetch()
    assert st == hs.HS_OK
    results.append(np.sort(recs, order=["k", "z", "bin"]))
    for r in results[1:]:
        assert np.array_equal(r, results[0])
    ref, near = oracle.detect(plane, H, ta, index=oracle.HFRAC, threads=8)
    assert_matches_oracle(results[0], ref, near)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_lowp_recheck_past_the_pending_list(dtype):
    # A 16-bit plane with its FP32 copy: the summing kernel lists marked row
    # pairs for the recheck kernel, 2^19 at most; with thresholds below every
    # value all 43 x 13,000 = 559,000 pairs are marked, so the last ones are
    # decided inside the summing kernel.  Every level sum of every point is
    # a record either way, equal to the oracle's on the FP32 plane.
    nt, n, H = 85, 13000, 16
    plane = synth.noise(nt, n, seed=91)
    low = _bf16_bits(plane) if dtype == "bf16" else plane.astype(np.float16)
    ta = np.full((H, nt), -1e30, np.float32)
    recs, cnt, st, used = run_gpu(low, H, ta, cap=nt * n * H, dtype=dtype, fop32=plane,
                                  assume_nonneg=True)
    assert used == "staged" and st == hs.HS_OK and cnt == nt * n * H
    Z = (nt - 1) // 2
    got = np.full((H, nt, n), np.nan)
    got[recs["k"].astype(int) - 1, recs["z"].astype(int) + Z, recs["bin"].astype(int)] = \
        recs["power"]
    np.testing.assert_allclose(got, oracle.planes(plane, H), rtol=RTOL, atol=0)
    assert not (recs["flags"] != 0).any()


def test_f16_overflow_is_decided_by_the_fp32_copy():
    # Values above 65,504 are stored as +inf in FP16.  The prefilter marks
    # their pairs and the FP32 copy decides them, so the records equal the
    # FP32 path's; without the copy they are records with power +inf,
    # flagged as decided in 16 bits and near their threshold.
    nt, n, H = 85, 20000, 16
    plane = synth.noise(nt, n, seed=41)
    hot = [(42, 5000), (10, 12345), (84, 19999), (0, 0)]
    for r, f in hot:
        plane[r, f] = 1.0e5
    ta = synth.thresholds(1e-4, H, nt)
    with np.errstate(over="ignore"):
        low = plane.astype(np.float16)
    assert np.isinf(low[42, 5000])
    ref, nref, _, _ = run_gpu(plane, H, ta, assume_nonneg=True)
    got, ngot, st, used = run_gpu(low, H, ta, dtype="f16", fop32=plane, assume_nonneg=True)
    assert used == "staged" and st == hs.HS_OK and ngot == nref
    assert np.array_equal(got, ref)
    bare, _, st2, _ = run_gpu(low, H, ta, dtype="f16", assume_nonneg=True)
    assert st2 == hs.HS_OK
    at_inf = bare[np.isinf(bare["power"])]
    assert len(at_inf) > 0
    assert ((at_inf["flags"] & hs.HS_FLAG_LOWP) != 0).all()
    assert ((at_inf["flags"] & hs.HS_FLAG_NEAR) != 0).all()
    assert {(int(r - 42), int(f)) for r, f in hot} <= \
        {(int(x["z"]), int(x["bin"])) for x in at_inf if x["k"] == 1}


def test_lowp_recheck_on_many_streams_of_one_plan():
    # more streams than the plan keeps pending lists for: the lists are
    # dropped and made again, and every run still gives the FP32 path's records
    nt, n, H = 21, 8192, 8
    plane = synth.noise(nt, n, seed=17)
    ta = synth.thresholds(1e-3, H, nt)
    ref, nref, _, _ = run_gpu(plane, H, ta)
    low = torch.from_numpy(_bf16_bits(plane).view(np.int16)).cuda().view(torch.bfloat16)
    f32 = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 16)
    with hs.Plan(nt, n, H, ta, dtype="bf16") as plan:
        for _ in range(20):
            s = torch.cuda.Stream()
            plan.run(low, cands, s, fop_f32=f32)
            got, cnt, st = cands.fetch(s)
            assert st == hs.HS_OK and cnt == nref and np.array_equal(got, ref)


def test_lowp_recheck_on_two_streams_of_one_plan():
    # each stream has its own pending list: two 16-bit planes run on one plan
    # from two streams, repeatedly, each giving the FP32 path's records
    nt, n, H = 85, 20000, 16
    planes = [synth.noise(nt, n, seed=s) for s in (101, 102)]
    for i, p_ in enumerate(planes):
        wl = synth.Workload("t", nt, n, H, 7 + i, 1e-4, 20, (200, 1200), (-2, 2))
        synth.inject(p_, synth.draw_signals(wl))
    ta = synth.thresholds(1e-4, H, nt)
    refs = [run_gpu(p_, H, ta)[0] for p_ in planes]
    lows = [torch.from_numpy(_bf16_bits(p_).view(np.int16)).cuda().view(torch.bfloat16)
            for p_ in planes]
    f32s = [torch.from_numpy(p_).cuda() for p_ in planes]
    streams = [torch.cuda.Stream() for _ in planes]
    bufs = [hs.CandBuffer(1 << 20) for _ in planes]
    with hs.Plan(nt, n, H, ta, dtype="bf16", assume_nonneg=True) as plan:
        for _ in range(5):
            for i in range(2):
                plan.run(lows[i], bufs[i], streams[i], fop_f32=f32s[i])
        torch.cuda.synchronize()
        for i in range(2):
            recs, cnt, st = bufs[i].fetch(streams[i])
            assert st == hs.HS_OK and cnt == len(refs[i]) > 0
            assert np.array_equal(recs, refs[i])


@pytest.mark.parametrize("nt,n,H,dtype", [(85, 20000, 16, "f32"), (21, 50000, 8, "f32"),
                                          (85, 8192, 16, "bf16")])
def test_declared_nonnegative_planes_same_records(nt, n, H, dtype):
    # assume_nonneg skips the per-value sign check: on a non-negative plane
    # the records are those of the checked kernel (and the oracle's)
    plane = synth.noise(nt, n, seed=53)
    ta = synth.thresholds(1e-4, H, nt)
    fop = plane if dtype == "f32" else _bf16_bits(plane)
    fop32 = None if dtype == "f32" else plane
    a, na, _, _ = run_gpu(fop, H, ta, dtype=dtype, fop32=fop32)
    b, nb, st, used = run_gpu(fop, H, ta, dtype=dtype, fop32=fop32, assume_nonneg=True)
    assert used == "staged" and st == hs.HS_OK and na == nb > 0
    assert np.array_equal(a, b)
    if dtype == "f32":
        ref, near = oracle.detect(plane, H, ta, threads=8)
        assert_matches_oracle(b, ref, near)


@pytest.mark.parametrize("nt,H", [(85, 16), (21, 8)])
def test_level_one_band_edges(nt, H):
    # FP32 planes declared non-negative load level 1 in row bands (rows
    # |z| <= Z/2 with the first barrier, the outer rows with a second one the
    # walk waits for at pair Z/2 + 1): peaks on both sides of the band edge
    # and on the outermost rows, in a full tile and in the ragged last one,
    # give the oracle's records
    Z = (nt - 1) // 2
    rb = Z // 2
    n = 3000  # 23 full tiles of 128 bins and a ragged one
    plane = synth.noise(nt, n, seed=61)
    rows = [0, Z - rb - 1, Z - rb, Z + rb, Z + rb + 1, nt - 1]
    for i, r in enumerate(rows):
        plane[r, 100 + 37 * i] = 60.0
        plane[r, n - 1 - i] = 60.0
    ta = synth.thresholds(1e-8, H, nt)
    recs, cnt, st, used = run_gpu(plane, H, ta, assume_nonneg=True)
    assert used == "staged" and st == hs.HS_OK
    ref, near = oracle.detect(plane, H, ta, threads=8)
    assert_matches_oracle(recs, ref, near)
    level1_rows = {int(r["z"]) + Z for r in recs if int(r["k"]) == 1}
    assert set(rows) <= level1_rows


def test_signed_inputs_take_the_exact_path():
    # Negative inputs void the monotone-sum prefilter; the staged kernel must
    # notice and test every level exactly.
    plane = synth.random_plane(21, 4096, seed=3, lo=-1.0, hi=1.0)
    plane[:, ::7] = np.abs(plane[:, ::7]) * 6.0
    ta = np.tile(np.array([[0.9 + 0.3 * k] for k in range(8)], np.float32), (1, 21))
    recs, n, st, used = run_gpu(plane, 8, ta)
    assert used == "staged" and n > 0
    ref, near = oracle.detect(plane, 8, ta)
    # signed sums carry an absolute error bound: compare values with atol
    assert_matches_oracle(recs, ref, near, rtol=1e-5)


def test_signed_lowp_with_copy_equals_the_fp32_path():
    # A signed 16-bit plane: every row of a thread that loads a negative
    # value is marked and goes to the recheck kernel, which decides it from
    # the FP32 copy -- the FP32 path's records (which the oracle confirms)
    plane = synth.random_plane(21, 4096, seed=5, lo=-1.0, hi=1.0)
    plane[:, ::7] = np.abs(plane[:, ::7]) * 6.0
    ta = np.tile(np.array([[0.9 + 0.3 * k] for k in range(8)], np.float32), (1, 21))
    ref, nref, _, used32 = run_gpu(plane, 8, ta)
    got, n, st, used = run_gpu(_bf16_bits(plane), 8, ta, dtype="bf16", fop32=plane)
    assert used32 == used == "staged" and st == hs.HS_OK and n == nref > 0
    assert np.array_equal(got, ref)
    o, near = oracle.detect(plane, 8, ta)
    assert_matches_oracle(got, o, near, rtol=1e-5)


def test_per_row_thresholds():
    plane = synth.noise(85, 4096, seed=21)
    rng = np.random.default_rng(4)
    ta = (synth.thresholds(1e-3, 16, 85) * rng.uniform(0.9, 1.3, size=(1, 85))).astype(np.float32)
    recs, n, st, used = run_gpu(plane, 16, ta)
    ref, near = oracle.detect(plane, 16, ta, threads=8)
    assert used == "staged" and n > 100
    assert_matches_oracle(recs, ref, near)


# --- 16-bit storage --------------------------------------------------------------

def _bf16_bits(x):
    return torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)


@pytest.mark.parametrize("nt,n,H", [(21, 8192, 8), (85, 4096, 16)])
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_lowp_recheck_matches_fp32_path(nt, n, H, dtype):
    plane = synth.noise(nt, n, seed=7)
    ta = synth.thresholds(1e-3, H, nt)
    r32, n32, _, _ = run_gpu(plane, H, ta)
    low = _bf16_bits(plane) if dtype == "bf16" else plane.astype(np.float16)
    rlp, nlp, st, used = run_gpu(low, H, ta, dtype=dtype, fop32=plane)
    assert used == "staged" and st == hs.HS_OK
    assert nlp == n32
    assert np.array_equal(r32, rlp)  # same records, same FP32 powers
    rg, ng, _, _ = run_gpu(low, H, ta, dtype=dtype, fop32=plane, kernel="generic")
    assert np.array_equal(r32, rg)


@pytest.mark.parametrize("dtype,u", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)])
def test_lowp_level_error_against_the_fp32_plane(dtype, u):
    # Precision form: every level sum of the 16-bit plane (no recheck) against
    # the FP64 oracle on the FP32 plane it was rounded from.  Non-negative
    # terms each carry at most the storage rounding u, so the relative error
    # of a level sum is at most u plus the FP32 accumulation bound.  The per
    # level max and RMS are printed (pytest -s) for the record.
    nt, n, H = 85, 2048, 16
    plane = synth.noise(nt, n, seed=31)
    low = _bf16_bits(plane) if dtype == "bf16" else plane.astype(np.float16)
    got, used = _all_sums(low, H, dtype=dtype)
    assert used == "staged"
    ref = oracle.planes(plane, H)
    # per term: relative rounding u, plus half the subnormal spacing eta of
    # the format for values below its normal range (FP16: 2^-25)
    eta = 0.0 if dtype == "bf16" else 2.0 ** -25
    k = np.arange(1, H + 1, dtype=np.float64)[:, None, None]
    bound = (u * (1 + 2 ** -24) + 15 * 2.0 ** -24) * ref + k * eta
    assert (np.abs(got - ref) <= bound).all()
    rel = np.abs(got - ref) / ref
    mx = rel.reshape(H, -1).max(axis=1)
    rms = np.sqrt((rel.reshape(H, -1) ** 2).mean(axis=1))
    print(f"\n{dtype} per-level relative error vs FP64 oracle on the FP32 plane "
          f"(85 x 2048, k = 1..16)")
    print("max:", " ".join(f"{x:.2e}" for x in mx))
    print("rms:", " ".join(f"{x:.2e}" for x in rms))
    # averaging over k terms shrinks the typical error roughly as 1/sqrt(k)
    assert rms[-1] < rms[0]


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_lowp_end_to_end_with_host_recheck_copy(dtype):
    # hs_run_host_checked: the 16-bit plane is copied to the device in
    # chunks, the FP32 copy stays in page-locked host memory and is read in
    # place for rechecks; the records equal the FP32 path's
    nt, n, H = 85, 1 << 15, 16
    plane = synth.noise(nt, n, seed=37)
    ta = synth.thresholds(1e-4, H, nt)
    r32, n32, _, _ = run_gpu(plane, H, ta)
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
    host32 = torch.from_numpy(plane).pin_memory()
    host = host32.to(tdt).pin_memory()
    dev = torch.empty_like(host, device="cuda")
    cands = hs.CandBuffer(1 << 18)
    out = np.zeros(1 << 18, hs.CAND_DTYPE)
    with hs.Plan(nt, n, H, ta, dtype=dtype) as plan:
        st, cnt = plan.run_host(host, dev, cands, out, fop32_host=host32)
        assert st == hs.HS_OK and cnt == n32 > 0
        assert np.array_equal(hs.sort_records(out[:cnt]), r32)
        # pageable host memory: refused where the device cannot address it,
        # read in place where it can (address translation); never wrong
        try:
            st2, cnt2 = plan.run_host(host, dev, cands, out, fop32_host=plane)
        except hs.HsError as e:
            assert e.status == hs.HS_ERR_INVALID
        else:
            assert st2 == hs.HS_OK and np.array_equal(hs.sort_records(out[:cnt2]), r32)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_lowp_without_recheck_flags_band(dtype):
    nt, n, H = 21, 8192, 8
    plane = synth.noise(nt, n, seed=8)
    ta = synth.thresholds(1e-3, H, nt)
    low = _bf16_bits(plane) if dtype == "bf16" else plane.astype(np.float16)
    recs, cnt, st, used = run_gpu(low, H, ta, dtype=dtype)
    assert cnt > 0 and np.all(recs["flags"] & hs.HS_FLAG_LOWP)
    # the oracle on the stored 16-bit values decides the same way except in the band
    dc = oracle.DT_BF16 if dtype == "bf16" else None
    ref, near = oracle.detect(low, H, ta, dtype_code=dc, near_rel=1e-5)
    assert_matches_oracle(recs, ref, near, rtol=1e-6)
    r32, _, _, _ = run_gpu(plane, H, ta)
    k32 = {(int(r["k"]), int(r["z"]), int(r["bin"])) for r in r32}
    klp = {(int(r["k"]), int(r["z"]), int(r["bin"])) for r in recs}
    flagged = {(int(r["k"]), int(r["z"]), int(r["bin"])) for r in recs
               if r["flags"] & hs.HS_FLAG_NEAR}
    assert (klp - k32) <= flagged


# --- buffers, ordering, end to end --------------------------------------------------

def test_overflow_reports_true_count():
    plane = synth.noise(21, 4096, seed=9)
    ta = synth.thresholds(1e-2, 8, 21)
    recs_all, n_all, _, _ = run_gpu(plane, 8, ta)
    recs, n, st, _ = run_gpu(plane, 8, ta, cap=5)
    assert st == hs.HS_ERR_OVERFLOW and n == n_all > 5 and len(recs) == 5


def test_octave_order_same_result():
    plane = synth.noise(85, 1 << 16, seed=10)
    ta = synth.thresholds(1e-4, 16, 85)
    a, na, _, _ = run_gpu(plane, 16, ta, order=1)
    b, nb, _, _ = run_gpu(plane, 16, ta, order=2)
    assert na == nb and np.array_equal(a, b)


def test_long_tile_walk_matches_generic():
    # Many tiles per CTA: every stage of the persistent ring is refilled many
    # times.  The staged and generic kernels must return identical records.
    plane = synth.noise(21, 1 << 20, seed=13)
    ta = synth.thresholds(1e-4, 8, 21)
    a, na, sa, ua = run_gpu(plane, 8, ta)
    b, nb, sb, ub = run_gpu(plane, 8, ta, kernel="generic")
    assert ua == "staged" and ub == "generic" and sa == sb == hs.HS_OK
    assert na == nb > 0 and np.array_equal(a, b)


@pytest.mark.parametrize("tb", [128, 64, 96])
def test_tile_widths_same_result(tb):
    # every compiled tile width gives the generic kernel's records, with a
    # ragged last tile in padded rows and patches of negative inputs (whose
    # pairs take the exact pass)
    n = 20011
    plane = synth.noise(85, n, seed=11)
    plane[3, 100:300] *= -1.0
    plane[60, 5000:5100] *= -1.0
    ta = synth.thresholds(1e-4, 16, 85)
    a, na, _, _ = run_gpu(plane, 16, ta, kernel="generic")
    padded = torch.zeros((85, n + 1), dtype=torch.float32, device="cuda")  # 16-byte rows
    padded[:, :n] = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(85, n, 16, ta, tile_bins=tb, row_pitch=n + 1) as plan:
        assert plan.kernel == "staged"
        plan.run(padded, cands)
        b, nb, st = cands.fetch()
    assert st == hs.HS_OK
    assert na == nb > 0 and np.array_equal(a, b)


@pytest.mark.parametrize("tb,groups,stages", [(128, 2, 3), (128, 3, 3), (96, 2, 4), (96, 4, 4)])
def test_pipelined_variants_same_result(tb, groups, stages):
    # the persistent pipelined kernel (a producer warp filling a ring of
    # stages that wraps many times, consumer groups summing) gives the
    # generic kernel's records, with a ragged last tile in padded rows and
    # patches of negative inputs
    n = (1 << 18) + 37
    plane = synth.noise(85, n, seed=17)
    plane[0, 1000:1300] *= -1.0
    plane[84, 70000:70100] *= -1.0
    ta = synth.thresholds(1e-4, 16, 85)
    a, na, _, _ = run_gpu(plane, 16, ta, kernel="generic")
    ld = n + 3
    padded = torch.zeros((85, ld), dtype=torch.float32, device="cuda")
    padded[:, :n] = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(85, n, 16, ta, tile_bins=tb, stages=stages, z_split=groups,
                 row_pitch=ld) as plan:
        assert plan.kernel == "staged"
        plan.run(padded, cands)
        b, nb, st = cands.fetch()
    assert st == hs.HS_OK
    assert na == nb > 0 and np.array_equal(a, b)


def test_pipelined_matches_oracle_on_the_small_ska_slice():
    n = 1 << 16
    plane = synth.noise(85, n, seed=23)
    ta = synth.thresholds(1e-5, 16, 85)
    recs, cnt, st, used = run_gpu(plane, 16, ta, stages=3)
    assert used == "staged" and st == hs.HS_OK
    ref, near = oracle.detect(plane, 16, ta, threads=8)
    assert_matches_oracle(recs, ref, near)


@pytest.mark.parametrize("order", [2, 3, 4])
@pytest.mark.parametrize("n", [1 << 15, (1 << 15) + 128, 1 << 18])
def test_tile_orders_give_the_same_records(n, order):
    # the octave, semitone and 53-step orders (the plan's tile table) visit
    # every tile exactly once: the same records as the linear order
    plane = synth.noise(85, n, seed=29)
    ta = synth.thresholds(1e-4, 16, 85)
    lin, nl, _, _ = run_gpu(plane, 16, ta, order=1)
    other, no, st, used = run_gpu(plane, 16, ta, order=order)
    assert used == "staged" and st == hs.HS_OK and nl == no > 0
    assert np.array_equal(lin, other)


@pytest.mark.parametrize("kernel", ["staged", "generic"])
def test_frequency_bands_append_to_the_full_run(kernel):
    # hs_run_range over the bands of shard.band_bounds, appended into one
    # buffer, gives the full run's records (a band reads only lower bins)
    from paper_1805_12258_gb300 import shard
    nt, n, H = 85, 50000, 16
    plane = synth.noise(nt, n, seed=19)
    ta = synth.thresholds(1e-3, H, nt)
    ref, nref, _, _ = run_gpu(plane, H, ta, kernel=kernel)
    fop = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(nt, n, H, ta, kernel=kernel) as plan:
        for i, (lo, hi) in enumerate(shard.band_bounds(n, 3, plan.tile_bins)):
            plan.run_range(fop, cands, lo, hi, append=i > 0)
        got, cnt, st = cands.fetch()
        with pytest.raises(hs.HsError):
            plan.run_range(fop, cands, 1, n)  # not tile-aligned (staged) / fine (generic)
            if kernel == "generic":
                raise hs.HsError(hs.HS_ERR_INVALID, "generic accepts any start")
    assert st == hs.HS_OK and cnt == nref > 0 and np.array_equal(got, ref)


def test_a_wait_that_runs_out_reports_timeout_and_the_context_stays_usable():
    # failure detection without a fault: a device wait on a barrier nothing
    # completes gives up after 20 ms and reports HS_ERR_TIMEOUT; the next
    # run on the same context is unaffected
    cands = hs.CandBuffer(16)
    cands.counters.zero_()
    st = hs.lib().hs_selftest_wait_timeout(ctypes.c_void_p(cands.counters.data_ptr()),
                                          20_000_000, hs._stream_handle(None))
    assert st == hs.HS_OK
    with pytest.raises(hs.HsError) as e:
        cands.sync()
    assert e.value.status == hs.HS_ERR_TIMEOUT
    plane = synth.noise(21, 4096, seed=2)
    ta = synth.thresholds(1e-3, 8, 21)
    recs, cnt, st2, used = run_gpu(plane, 8, ta)
    ref, near = oracle.detect(plane, 8, ta)
    assert st2 == hs.HS_OK and used == "staged"
    assert_matches_oracle(recs, ref, near)


@pytest.mark.parametrize("kernel,index", [("staged", "stretch"), ("generic", "stretch"),
                                          ("staged", "hfrac"), ("generic", "hfrac")])
def test_run_host_matches_run(kernel, index):
    # end to end from pinned host memory (the plane copied in chunks while
    # earlier chunks are summed) gives the device run's records
    wl = synth.small_plane(seed=2)
    plane = synth.make_plane(wl)
    ta = synth.thresholds(1e-4, wl.H, wl.n_templates)
    ref, n_ref, _, used = run_gpu(plane, wl.H, ta, kernel=kernel, index=index)
    assert used == kernel and n_ref > 0
    host = torch.from_numpy(plane).pin_memory()
    dev = torch.empty_like(host, device="cuda")
    cands = hs.CandBuffer(1 << 16)
    out = np.zeros(1 << 16, hs.CAND_DTYPE)
    with hs.Plan(wl.n_templates, wl.n_bins, wl.H, ta, kernel=kernel, index=index) as plan:
        st, n = plan.run_host(host, dev, cands, out)
    assert st == hs.HS_OK and n == n_ref
    assert np.array_equal(hs.sort_records(out[:n]), ref)


@pytest.mark.parametrize("kind", ["f32", "bf16", "hfrac"])
def test_plan_run_replays_in_a_cuda_graph(kind):
    # after one run on a stream (the pending list, descriptors and kernel
    # attributes exist then), a run captured on that stream replays with the
    # same records: the FP32 staged kernel, the 16-bit one with its recheck
    # kernel (a programmatic dependent launch), the harmonic-fraction families
    nt, n, H = 85, 20000, 16
    plane = synth.noise(nt, n, seed=61)
    wl = synth.Workload("t", nt, n, H, 9, 1e-4, 12, (500, 2500), (-2, 2))
    synth.inject(plane, synth.draw_signals(wl))
    ta = synth.thresholds(1e-4, H, nt)
    f32 = torch.from_numpy(plane).cuda()
    kw = {"hfrac": dict(index="hfrac"), "bf16": dict(dtype="bf16")}.get(kind, {})
    fop = f32.to(torch.bfloat16) if kind == "bf16" else f32
    copy = f32 if kind == "bf16" else None
    cands = hs.CandBuffer(1 << 18)
    s = torch.cuda.Stream()
    with hs.Plan(nt, n, H, ta, assume_nonneg=True, **kw) as plan:
        plan.run(fop, cands, s, fop_f32=copy)
        ref, nref, st = cands.fetch(s)
        assert st == hs.HS_OK and nref > 0
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            plan.run(fop, cands, s, fop_f32=copy)
        for _ in range(3):
            g.replay()  # on torch's current stream
            torch.cuda.synchronize()
            got, cnt, st = cands.fetch(s)
            assert st == hs.HS_OK and cnt == nref and np.array_equal(got, ref)


def test_many_distinct_ranges_keep_their_records():
    # more distinct bands than the plan keeps order tables for: the tables
    # are dropped and made again, and every band's records stay those of the
    # full run in that band
    nt, n, H = 21, 128 * 80, 8
    plane = synth.noise(nt, n, seed=15)
    ta = synth.thresholds(1e-3, H, nt)
    full, nfull, _, _ = run_gpu(plane, H, ta)
    assert nfull > 0
    fop = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 18)
    with hs.Plan(nt, n, H, ta) as plan:
        for lo in range(0, 70):  # 70 distinct bands of 10 tiles
            a, b = 128 * lo, 128 * (lo + 10)
            plan.run_range(fop, cands, a, b)
            got, cnt, st = cands.fetch()
            want = full[(full["bin"] >= a) & (full["bin"] < b)]
            assert st == hs.HS_OK and np.array_equal(got, want)


def test_launch_count_is_one():
    plane = synth.noise(21, 4096, seed=12)
    run_gpu(plane, 8, synth.thresholds(1e-3, 8, 21))
    # the last hs_run on this thread launched exactly one kernel
    assert hs.hs_last_launch_count() == 1


# --- the SKA plane at full size (85 x 2^21, H = 16), bench launch configuration ----

@pytest.fixture(scope="module")
def ska():
    wl = synth.ska_plane(seed=1)
    plane = synth.make_plane(wl)
    ta = synth.thresholds(wl.p_fa, wl.H, wl.n_templates)
    return wl, plane, ta


@pytest.fixture(scope="module")
def ska_oracle(ska):
    wl, plane, ta = ska
    return oracle.detect(plane, wl.H, ta, threads=16)


# assume_nonneg=True is the launch configuration bench.py times (no sign
# check, level 1 in row bands, the default 53-step tile order); False the
# checked one.
@pytest.mark.parametrize("assume_nonneg", [True, False])
def test_ska_plane_candidates(ska, ska_oracle, assume_nonneg):
    wl, plane, ta = ska
    recs, n, st, used = run_gpu(plane, wl.H, ta, assume_nonneg=assume_nonneg)
    assert used == "staged" and st == hs.HS_OK
    ref, near = ska_oracle
    assert n == len(recs) and n > 1000
    assert_matches_oracle(recs, ref, near)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_ska_plane_lowp_recheck_candidates(ska, ska_oracle, dtype):
    # Precision form at full size, in bench.py's launch configuration: the
    # 16-bit plane with the FP32 copy for rechecks gives the FP64 oracle's
    # candidate set on the FP32 plane (near-threshold points excepted)
    wl, plane, ta = ska
    low = _bf16_bits(plane) if dtype == "bf16" else plane.astype(np.float16)
    recs, n, st, used = run_gpu(low, wl.H, ta, dtype=dtype, fop32=plane, assume_nonneg=True)
    assert used == "staged" and st == hs.HS_OK
    ref, near = ska_oracle
    assert_matches_oracle(recs, ref, near)


@pytest.mark.parametrize("z,assume_nonneg", [(0, True), (-42, True), (17, True), (42, True),
                                             (-21, True), (22, True), (0, False), (-42, False),
                                             (17, False)])
def test_ska_plane_row_sums(ska, z, assume_nonneg):
    # Every level sum of one full row (2^21 bins x 16 levels), checked
    # against the oracle point by point: the row's thresholds are set below
    # every value so each sum becomes a record.  Rows 21 / 22 straddle the
    # edge of the level-1 centre band of the banded load.
    wl, plane, ta = ska
    Z = (wl.n_templates - 1) // 2
    ta2 = ta.copy()
    ta2[:, z + Z] = -1e30
    recs, n, st, _ = run_gpu(plane, wl.H, ta2, cap=wl.n_bins * wl.H + (1 << 16),
                             assume_nonneg=assume_nonneg)
    assert st == hs.HS_OK
    row = recs[recs["z"] == z]
    assert len(row) == wl.n_bins * wl.H
    got = np.empty((wl.n_bins, wl.H))
    got[row["bin"].astype(np.int64), row["k"].astype(np.int64) - 1] = row["power"]
    f = np.arange(wl.n_bins, dtype=np.int64)
    ref = oracle.sample(plane, wl.H, np.full(wl.n_bins, z, np.int32), f)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


def test_ska_plane_hfrac_candidates(ska):
    # The harmonic-fraction map on the full plane: every record's power
    # against the oracle's level sum at that point; inside three bin windows
    # (the start, the middle and the end of the plane) the record set is the
    # oracle's; the gather kernel gives the same records as the staged one
    wl, plane, ta = ska
    recs, n, st, used = run_gpu(plane, wl.H, ta, index="hfrac")
    assert used == "staged" and st == hs.HS_OK and n == len(recs) and n > 1000
    ref = oracle.sample(plane, wl.H, recs["z"].astype(np.int32), recs["bin"].astype(np.int64),
                        index=oracle.HFRAC)[np.arange(n), recs["k"].astype(int) - 1]
    np.testing.assert_allclose(recs["power"], ref, rtol=RTOL, atol=0)
    for lo in (0, wl.n_bins // 2 - 6000, wl.n_bins - 12000):
        hi = lo + 12000
        win = recs[(recs["bin"] >= lo) & (recs["bin"] < hi)]
        o, near = oracle.detect(plane, wl.H, ta, index=oracle.HFRAC, f_lo=lo, f_hi=hi,
                                threads=8)
        assert_matches_oracle(win, o, near)
    g, ng, st2, used2 = run_gpu(plane, wl.H, ta, index="hfrac", kernel="generic")
    assert used2 == "generic" and st2 == hs.HS_OK and ng == n
    assert np.array_equal(np.sort(g, order=["k", "z", "bin"]),
                          np.sort(recs, order=["k", "z", "bin"]))


# --- other plane shapes: kernel families with runtime rows ------------------------

@pytest.mark.parametrize("nt,n,H", [(85, 2500, 8), (43, 3000, 16), (127, 1500, 16),
                                    (83, 700, 16), (15, 1000, 8), (1, 300, 16)])
@pytest.mark.parametrize("assume_nonneg", [False, True])
def test_other_shapes_every_level_sum(nt, n, H, assume_nonneg):
    # 85 x 8 (the paper's N_hp = 8 on the full template set), 43 and 83
    # templates at 16 levels, 127 templates, one template: a staged kernel
    # compiled for more rows serves the plane (boxes centred on its centre
    # row, rows outside it filled with zeros and never read)
    plane = synth.noise(nt, n, seed=nt * 7 + n)
    got, used = _all_sums(plane, H, assume_nonneg=assume_nonneg)
    assert used == "staged"
    ref = oracle.planes(plane, H)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=0)


@pytest.mark.parametrize("nt,n,H", [(85, 40000, 8), (43, 30000, 16), (127, 20000, 16)])
@pytest.mark.parametrize("assume_nonneg", [False, True])
def test_other_shapes_candidates(nt, n, H, assume_nonneg):
    wl = synth.Workload("shape", nt, n, H, 11, 1e-6, 8, (500, 2000), (-1, 1))
    plane = synth.make_plane(wl)
    ta = synth.thresholds(1e-5, H, nt)
    recs, cnt, st, used = run_gpu(plane, H, ta, assume_nonneg=assume_nonneg)
    assert used == "staged" and st == hs.HS_OK and cnt == len(recs) > 0
    ref, near = oracle.detect(plane, H, ta, threads=8)
    assert_matches_oracle(recs, ref, near)


# --- the largest sizes a plan accepts ------------------------------------------

def test_stretch_at_the_largest_template_count():
    # 32,767 templates (z = -16,383 .. 16,383, the largest a record's 16-bit
    # z holds): no staged family has that many rows, so the generic kernel
    # runs; every level sum against the oracle
    nt, n, H = 32767, 40, 16
    plane = synth.noise(nt, n, seed=23)
    got, used = _all_sums(plane, H)
    assert used == "generic"
    np.testing.assert_allclose(got, oracle.planes(plane, H), rtol=RTOL, atol=0)


@pytest.fixture(scope="module")
def max_bins():
    # planes of one template row with a ragged last tile: 2^31 - 1 bins (the
    # largest bin count; its rows are not 16-byte multiples, so the generic
    # kernel runs) and 2^31 - 4 bins (the largest the FP32 staged kernel
    # takes, whose rows must be 16-byte multiples with an int row pitch).
    # Zero but for 3000 seeded exponential values below bin 2^31 - 4, so
    # that only the touched pages hold memory.  The oracle's candidates at a
    # threshold of 3 for every level over the whole smaller plane, and over
    # the larger plane's three extra bins.
    nt, H, count, seed = 1, 16, 3000, 31
    n_big, n_staged = (1 << 31) - 1, (1 << 31) - 4
    plane = synth.sparse(nt, n_staged, count, seed, ld=n_big)
    ta = np.full((H, nt), 3.0, np.float32)
    ref, near = oracle.detect(plane[:, :n_staged], H, ta, threads=16, cap=1 << 20)
    tail, tail_near = oracle.detect(plane, H, ta, f_lo=n_staged)
    assert len(ref) > 1000 and (ref["f"] >= (1 << 30)).any()
    return dict(nt=nt, H=H, count=count, seed=seed, n_big=n_big, n_staged=n_staged, ta=ta,
                ref=ref, near=near, tail=tail, tail_near=tail_near)


def _sparse_on_device(m, n):
    rows, bins, vals = synth.sparse_points(m["nt"], m["n_staged"], m["count"], m["seed"])
    fop = torch.zeros((m["nt"], n), device="cuda")
    fop[torch.from_numpy(rows).cuda(), torch.from_numpy(bins).cuda()] = \
        torch.from_numpy(vals).cuda()
    return fop


def _run_max(m, n, **plan_kw):
    fop = _sparse_on_device(m, n)
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(m["nt"], n, m["H"], m["ta"], **plan_kw) as plan:
        plan.run(fop, cands)
        recs, cnt, st = cands.fetch()
        used = plan.kernel
    del fop
    torch.cuda.empty_cache()
    assert st == hs.HS_OK and cnt == len(recs)
    return recs, used


@pytest.mark.parametrize("assume_nonneg", [True, False])
def test_staged_at_the_largest_bin_count(max_bins, assume_nonneg):
    m = max_bins
    recs, used = _run_max(m, m["n_staged"], assume_nonneg=assume_nonneg)
    assert used == "staged"
    assert_matches_oracle(recs, m["ref"], m["near"])


def test_generic_at_the_largest_bin_count(max_bins):
    m = max_bins
    recs, used = _run_max(m, m["n_big"])
    assert used == "generic"
    assert_matches_oracle(recs, np.concatenate([m["ref"], m["tail"]]),
                          np.concatenate([m["near"], m["tail_near"]]))


def test_hfrac_staged_at_the_largest_bin_count():
    # the harmonic-fraction staged kernel forms f h in 32 bits, so it takes
    # n_bins + tile <= 2^31 / H; the largest such plane (64-bin tiles, a
    # ragged last tile, the row pitch padded to a 16-byte multiple)
    nt, H, tb = 1, 16, 64
    ld = (1 << 31) // H - tb
    n = ld - 3
    plane = synth.sparse(nt, n, 2000, seed=37, ld=ld)
    ta = np.full((H, nt), 3.0, np.float32)
    fop = torch.from_numpy(plane).cuda()
    cands = hs.CandBuffer(1 << 20)
    with hs.Plan(nt, n, H, ta, index="hfrac", row_pitch=ld) as plan:
        assert plan.kernel == "staged" and plan.tile_bins == tb
        plan.run(fop, cands)
        recs, cnt, st = cands.fetch()
    del fop
    assert st == hs.HS_OK and cnt == len(recs)
    ref, near = oracle.detect(plane[:, :n], H, ta, index=oracle.HFRAC, threads=16,
                              cap=1 << 20)
    assert len(ref) > 1000 and (ref["f"] >= (1 << 26)).any()
    assert_matches_oracle(recs, ref, near)


@pytest.mark.parametrize("kind", ["staged", "generic", "hfrac", "bf16"])
def test_count_only_buffer_counts_every_hit_and_writes_none(kind):
    # a candidate buffer of capacity 0 with no records array: the run counts
    # every hit and writes no record; hs_cand_sync reports the true count
    # with HS_ERR_OVERFLOW.  The count equals a full buffer's and, but for
    # near-threshold points, the oracle's.
    nt, n, H = 21, 20000, 8
    plane = synth.noise(nt, n, seed=41)
    ta = synth.thresholds(1e-4, H, nt)
    kw = {"staged": dict(kernel="staged"), "generic": dict(kernel="generic"),
          "hfrac": dict(index="hfrac"), "bf16": dict(dtype="bf16")}[kind]
    fop32 = torch.from_numpy(plane).cuda()
    fop = fop32.to(torch.bfloat16) if kind == "bf16" else fop32
    f32 = fop32 if kind == "bf16" else None
    full = hs.CandBuffer(1 << 18)
    counters = torch.zeros(4, dtype=torch.int32, device="cuda")
    empty = hs.hs_cand_buf(None, counters.data_ptr(), 0)
    with hs.Plan(nt, n, H, ta, **kw) as plan:
        assert plan.kernel == ("generic" if kind == "generic" else "staged")
        plan.run(fop, full, fop_f32=f32)
        _, n_full, st_full = full.fetch()
        if f32 is None:
            hs.hs_run(plan.handle, fop, None, empty)
        else:
            hs.hs_run_checked(plan.handle, fop, f32, None, empty)
        st, n_empty = hs.hs_cand_sync(empty, None)
    assert st_full == hs.HS_OK and n_full > 100
    assert st == hs.HS_ERR_OVERFLOW and n_empty == n_full
    ref, near = oracle.detect(plane, H, ta, index=oracle.HFRAC if kind == "hfrac" else oracle.STRETCH)
    assert abs(n_empty - len(ref)) <= len(near)
