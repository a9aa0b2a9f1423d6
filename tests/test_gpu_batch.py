"""GPU: the batched form (many ragged beams in one launch, graph replay) and
the persistent mode of the plane kernel give the same records as per-plane
runs, and the per-plane runs agree with the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_12258_gb300 import autotune, hs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1805_12258_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _beam(nt, n, seed):
    """A plane of n bins stored with a row pitch rounded up to 16 bytes."""
    ld = (n + 3) // 4 * 4
    plane = synth.noise(nt, n, seed=seed)
    dev = torch.zeros((nt, ld), dtype=torch.float32, device="cuda")
    dev[:, :n] = torch.from_numpy(plane).cuda()
    return plane, dev


def _plan_records(plane, H, ta):
    nt, n = plane.shape
    cands = hs.CandBuffer(1 << 18)
    with hs.Plan(nt, n, H, ta) as plan:
        plan.run(torch.from_numpy(plane).cuda(), cands)
        recs, cnt, st = cands.fetch()
    assert st == hs.HS_OK
    return recs


@pytest.mark.parametrize("nt,H,gps,nonneg", [(85, 16, 0, False), (85, 16, 3, False),
                                             (21, 8, 0, False), (85, 16, 0, True),
                                             (21, 8, 0, True)])
def test_batch_matches_per_plane_runs_and_graph_replay(nt, H, gps, nonneg):
    rng = np.random.default_rng(nt)
    ta = synth.thresholds(1e-4, H, nt)
    sizes_a = [int(x) for x in rng.integers(1000, 40000, size=5)] + [129, 7]
    sizes_b = [int(x) for x in rng.integers(500, 60000, size=3)]
    with hs.Batch(nt, H, ta, max_beams=16, grid_per_sm=gps, assume_nonneg=nonneg) as batch:
        for rnd, sizes in enumerate((sizes_a, sizes_b, sizes_a)):
            beams, planes, bufs = [], [], []
            for i, n in enumerate(sizes):
                plane, dev = _beam(nt, n, seed=100 * rnd + i)
                cb = hs.CandBuffer(1 << 16)
                planes.append(plane)
                bufs.append(cb)
                beams.append((dev, n, cb))
            batch.set_beams(beams)
            assert batch.tiles == sum((n + 127) // 128 for n in sizes)
            batch.graph_run() if rnd else batch.run()
            for plane, cb in zip(planes, bufs):
                got, cnt, st = cb.fetch()
                assert st == hs.HS_OK
                assert np.array_equal(got, _plan_records(plane, H, ta))


@pytest.mark.parametrize("nt,H,order", [(85, 16, 0), (21, 8, 0), (85, 16, 1), (85, 16, 3),
                                        (85, 16, 2)])
def test_batch_spanning_several_launches(nt, H, order):
    # more beams than one launch's parameter block holds: the run splits them
    # over launches; graph replays, and re-captures after the beam set
    # changes, give the same records
    rng = np.random.default_rng(7 + nt + order)
    ta = synth.thresholds(1e-3, H, nt)
    sizes = [int(x) for x in rng.integers(100, 6000, size=37)]
    items = []
    for i, n in enumerate(sizes):
        plane, dev = _beam(nt, n, seed=500 + i)
        items.append((plane, dev, n, hs.CandBuffer(1 << 14)))
    refs = [_plan_records(plane, H, ta) for plane, _, _, _ in items]
    with hs.Batch(nt, H, ta, max_beams=64, order=order) as batch:
        for subset in (range(37), range(5, 25), range(37)):
            sel = list(subset)
            batch.set_beams([(items[i][1], items[i][2], items[i][3]) for i in sel])
            assert batch.launches >= (2 if len(sel) > 30 else 1)
            for rep in range(2):
                batch.graph_run()
                for i in sel:
                    got, cnt, st = items[i][3].fetch()
                    assert st == hs.HS_OK
                    assert np.array_equal(got, refs[i]), (i, rep)


def test_batch_beam_against_oracle():
    nt, H, n = 85, 16, 30011
    ta = synth.thresholds(1e-4, H, nt)
    plane, dev = _beam(nt, n, seed=7)
    cb = hs.CandBuffer(1 << 16)
    with hs.Batch(nt, H, ta, max_beams=4) as batch:
        batch.set_beams([(dev, n, cb)])
        batch.run()
        got, cnt, st = cb.fetch()
    ref, near = oracle.detect(plane, H, ta, threads=8)
    near_keys = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in near}
    g = {(int(r["k"]), int(r["z"]), int(r["bin"])): float(r["power"]) for r in got}
    o = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in ref}
    assert not ((set(g) ^ set(o)) - near_keys)
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= 1e-6 * abs(o[k])


def test_row_pitch_plane_same_records():
    # a ragged plane stored with padded rows runs on the staged kernel and
    # matches the unpadded plane (generic kernel for its odd row length)
    nt, n, H = 85, 30011, 16
    plane, dev = _beam(nt, n, seed=41)
    ta = synth.thresholds(1e-4, H, nt)
    ref = _plan_records(plane, H, ta)
    cands = hs.CandBuffer(1 << 16)
    with hs.Plan(nt, n, H, ta, row_pitch=dev.shape[1]) as plan:
        assert plan.kernel == "staged"
        plan.run(dev, cands)
        got, cnt, st = cands.fetch()
    assert st == hs.HS_OK and np.array_equal(got, ref)


@pytest.mark.parametrize("gps", [1, 3])
def test_persistent_plane_mode_same_records(gps):
    nt, n, H = 85, 1 << 18, 16
    plane = synth.noise(nt, n, seed=31)
    ta = synth.thresholds(1e-4, H, nt)
    ref = _plan_records(plane, H, ta)
    cands = hs.CandBuffer(1 << 18)
    with hs.Plan(nt, n, H, ta, grid_per_sm=gps) as plan:
        plan.run(torch.from_numpy(plane).cuda(), cands)
        got, cnt, st = cands.fetch()
    assert st == hs.HS_OK and np.array_equal(got, ref)


def test_autotuner_picks_a_measured_option(tmp_path, monkeypatch):
    monkeypatch.setenv("HS_TUNE_CACHE", str(tmp_path / "tune.json"))
    ta = synth.thresholds(1e-8, 16, 85)
    best, table = autotune.tune_plane(85, 1 << 16, 16, ta, reps=2,
                                      space={"tile_bins": (64, 128), "order": (2,),
                                             "grid_per_sm": (0, 3)})
    assert best in [t[0] for t in table] and len(table) == 4
    assert min(t[1] for t in table) < float("inf")
    best2, _ = autotune.tune_plane(85, 1 << 16, 16, ta)  # cached
    assert best2 == best
    # the default space also times the pipelined ring (staging depth, groups)
    best3, table3 = autotune.tune_plane(85, 1 << 16, 16, ta, reps=2, use_cache=False)
    assert any(t[0].get("stages") == 3 and t[1] < float("inf") for t in table3)
    assert best3 in [t[0] for t in table3]


# --- packed batch: beams side by side in one plane, one summing launch ----------

def _packed(nt, sizes, seed, align=4, gap=0, dtype=torch.float32):
    """Beams laid side by side along the bins of one plane (offsets a
    multiple of 16 bytes, optional unused gap between beams)."""
    offs, at = [], 0
    for n in sizes:
        offs.append(at)
        at = (at + n + gap + align - 1) // align * align
    pitch = (at + align - 1) // align * align
    planes = [synth.noise(nt, n, seed=seed + i) for i, n in enumerate(sizes)]
    host = np.full((nt, pitch), 1e4, np.float32)  # bins outside every beam: large
    for off, n, pl in zip(offs, sizes, planes):
        host[:, off:off + n] = pl
    return planes, offs, pitch, torch.from_numpy(host).cuda()


@pytest.mark.parametrize("nt,H,nonneg,gps,order", [(85, 16, True, 0, 0), (85, 16, False, 0, 0),
                                                   (21, 8, True, 0, 1), (85, 16, True, 3, 2)])
def test_packed_batch_one_launch_matches_per_plane_runs(nt, H, nonneg, gps, order):
    rng = np.random.default_rng(41 + nt)
    ta = synth.thresholds(1e-4, H, nt)
    sizes = [int(x) for x in rng.integers(200, 30000, size=9)] + [129, 7, 4096]
    planes, offs, pitch, dev = _packed(nt, sizes, seed=700, gap=13)
    bufs = [hs.CandBuffer(1 << 16) for _ in sizes]
    with hs.Batch(nt, H, ta, max_beams=len(sizes), assume_nonneg=nonneg, grid_per_sm=gps,
                  order=order) as batch:
        batch.set_packed(dev, [(o, n, cb) for o, n, cb in zip(offs, sizes, bufs)])
        assert batch.launches == 1
        assert batch.tiles == sum((n + 127) // 128 for n in sizes)
        for rnd in range(3):  # run, then graph replays (records reset each time)
            batch.graph_run() if rnd else batch.run()
            for plane, cb in zip(planes, bufs):
                got, cnt, st = cb.fetch()
                assert st == hs.HS_OK
                assert np.array_equal(got, _plan_records(plane, H, ta))


def test_packed_batch_beam_against_oracle():
    # a ragged beam in the middle of the packed plane and the last one, which
    # ends at the plane's edge, against the FP64 oracle
    nt, H = 85, 16
    ta = synth.thresholds(1e-4, H, nt)
    sizes = [5000, 12345, 3001]
    planes, offs, pitch, dev = _packed(nt, sizes, seed=900)
    assert offs[-1] + sizes[-1] <= pitch
    bufs = [hs.CandBuffer(1 << 16) for _ in sizes]
    with hs.Batch(nt, H, ta, max_beams=4, assume_nonneg=True) as batch:
        batch.set_packed(dev, [(o, n, cb) for o, n, cb in zip(offs, sizes, bufs)])
        batch.run()
    for plane, cb in zip(planes[1:], bufs[1:]):
        got, cnt, st = cb.fetch()
        ref, near = oracle.detect(plane, H, ta, threads=8)
        assert st == hs.HS_OK and cnt > 0
        near_keys = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in near}
        g = {(int(r["k"]), int(r["z"]), int(r["bin"])): float(r["power"]) for r in got}
        o = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in ref}
        assert not ((set(g) ^ set(o)) - near_keys)
        for k in set(g) & set(o):
            assert abs(g[k] - o[k]) <= 1e-6 * abs(o[k])


def test_packed_batch_bf16_with_recheck_equals_fp32_records():
    nt, H = 85, 16
    ta = synth.thresholds(1e-4, H, nt)
    sizes = [7000, 2500, 9999]
    planes, offs, pitch, dev32 = _packed(nt, sizes, seed=950, align=8)
    dev16 = dev32.to(torch.bfloat16)
    bufs = [hs.CandBuffer(1 << 16) for _ in sizes]
    with hs.Batch(nt, H, ta, dtype="bf16", max_beams=4, assume_nonneg=True) as batch:
        batch.set_packed(dev16, [(o, n, cb) for o, n, cb in zip(offs, sizes, bufs)],
                         fop32=dev32)
        batch.graph_run()
    for plane, cb in zip(planes, bufs):
        got, cnt, st = cb.fetch()
        assert st == hs.HS_OK
        assert np.array_equal(got, _plan_records(plane, H, ta))


def test_packed_batch_rejects_bad_layouts():
    nt, H = 85, 16
    ta = synth.thresholds(1e-4, H, nt)
    dev = torch.zeros((nt, 1024), device="cuda")
    cb = hs.CandBuffer(16)
    with hs.Batch(nt, H, ta, max_beams=4) as batch:
        for beams in ([(2, 100, cb)],          # offset not a multiple of 16 bytes
                      [(1000, 100, cb)],       # beyond the pitch
                      [(0, 0, cb)]):           # empty beam
            with pytest.raises(hs.HsError) as e:
                batch.set_packed(dev, beams)
            assert e.value.status == hs.HS_ERR_INVALID
        with pytest.raises(hs.HsError):
            batch.set_packed(dev[:, 1:], [(0, 100, cb)])  # misaligned plane / pitch
