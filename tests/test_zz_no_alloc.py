"""hs_run_noalloc: harmonic summing for callers that may not allocate device
memory (a host framework that owns all device memory, or latency-critical
loops that cannot afford cudaMalloc/cudaFree).  Its results must equal
hs_run's on the same plane, call after call, although it keeps its threshold
table in a static device array and runs tiles in linear order.

Collected last on purpose, and self-contained, so it passes both alone in a
fresh process and after the rest of the suite."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_12258_gb300 import hs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1805_12258_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _with_plan(plane_d, ta, nt, n, H):
    cands = hs.CandBuffer(1 << 18)
    with hs.Plan(nt, n, H, ta) as plan:
        plan.run(plane_d, cands)
        recs, cnt, st = cands.fetch()
    return recs, cnt, st


def _noalloc(plane_d, ta, nt, n, H, cands):
    hs.hs_run_noalloc(nt, n, H, ta, plane_d, None, cands.c)
    return cands.fetch()


@pytest.mark.parametrize("nt,n,H,p_fa", [(21, 65536, 8, 1e-4), (85, 1 << 17, 16, 1e-5),
                                         (9, 3001, 6, 1e-3)])
def test_noalloc_matches_plan_twice(nt, n, H, p_fa):
    plane = synth.noise(nt, n, seed=nt + n)
    ta = synth.thresholds(p_fa, H, nt)
    plane_d = torch.from_numpy(plane).cuda()
    ref, n_ref, st_ref = _with_plan(plane_d, ta, nt, n, H)
    assert st_ref == hs.HS_OK and n_ref > 0
    cands = hs.CandBuffer(1 << 18)
    for _ in range(2):  # the static table keeps the last call's contents
        got, n_got, st = _noalloc(plane_d, ta, nt, n, H, cands)
        assert st == hs.HS_OK and n_got == n_ref
        assert np.array_equal(got, ref)


def test_noalloc_second_call_uses_its_own_thresholds():
    nt, n, H = 21, 8192, 8
    plane_d = torch.from_numpy(synth.noise(nt, n, seed=5)).cuda()
    lo, hi = synth.thresholds(1e-2, H, nt), synth.thresholds(1e-4, H, nt)
    cands = hs.CandBuffer(1 << 18)
    a, na, _ = _noalloc(plane_d, lo, nt, n, H, cands)
    b, nb, _ = _noalloc(plane_d, hi, nt, n, H, cands)
    ra, _, _ = _with_plan(plane_d, lo, nt, n, H)
    rb, _, _ = _with_plan(plane_d, hi, nt, n, H)
    assert na > nb and np.array_equal(a, ra) and np.array_equal(b, rb)


def test_noalloc_rejects_tables_beyond_its_limit():
    nt, H = 1025, 16  # 16400 thresholds > 16384
    plane_d = torch.zeros((nt, 64), device="cuda")
    cands = hs.CandBuffer(16)
    with pytest.raises(hs.HsError, match="16384"):
        hs.hs_run_noalloc(nt, 64, H, np.ones((H, nt), np.float32), plane_d, None, cands.c)


def test_noalloc_leaves_free_device_memory_unchanged():
    # the property the entry point exists for: after a first call on each
    # path (staged and generic), further calls change no device allocation
    cases = [(21, 65536, 8), (9, 3001, 6)]  # staged kernel; generic fallback
    planes = {c: torch.from_numpy(synth.noise(c[0], c[1], seed=77)).cuda() for c in cases}
    tas = {c: synth.thresholds(1e-3, c[2], c[0]) for c in cases}
    cands = hs.CandBuffer(1 << 16)
    for c in cases:
        _noalloc(planes[c], tas[c], c[0], c[1], c[2], cands)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        for c in cases:
            hs.hs_run_noalloc(c[0], c[1], c[2], tas[c], planes[c], None, cands.c)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


@pytest.mark.parametrize("nt,n,H,p_fa", [(21, 65536, 8, 1e-4), (9, 3001, 6, 1e-3)])
def test_noalloc_matches_the_oracle(nt, n, H, p_fa):
    # against the FP64 oracle directly (staged kernel; generic kernel): the
    # same candidate set except points within 1e-5 of their threshold, powers
    # within 1e-6 relative
    plane = synth.noise(nt, n, seed=nt * 3 + n)
    ta = synth.thresholds(p_fa, H, nt)
    cands = hs.CandBuffer(1 << 18)
    got, cnt, st = _noalloc(torch.from_numpy(plane).cuda(), ta, nt, n, H, cands)
    assert st == hs.HS_OK and cnt == len(got) > 0
    ref, near = oracle.detect(plane, H, ta, threads=8)
    near_keys = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in near}
    g = {(int(r["k"]), int(r["z"]), int(r["bin"])): float(r["power"]) for r in got}
    o = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in ref}
    assert len(g) == len(got)
    assert not (set(g) - set(o) - near_keys) and not (set(o) - set(g) - near_keys)
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= 1e-6 * abs(o[k])
