"""GPU: the serving engine and its plane generator.  A served request's
candidates equal the FP64 oracle's on the same plane (bytes copied back from
the device) and an hs_run of that plane; they do not change when the request
runs alone or amid a mix of other requests; admission control answers busy
instead of queueing without bound."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_12258_gb300 import hs, synth

pytestmark = pytest.mark.gpu

NT, H = 85, 16


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1805_12258_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _ld(n):
    return (n + 7) // 8 * 8


def _plane(seed, n, dtype="f32", n_signals=0):
    """The generator's plane as (FP32 device tensor [NT][ld], BF16 tensor or None)."""
    ld = _ld(n)
    f32 = torch.empty((NT, ld), dtype=torch.float32, device="cuda")
    if dtype == "f32":
        hs.hs_synth_fop(f32, None, "f32", NT, n, ld, seed, n_signals)
        torch.cuda.synchronize()
        return f32, None
    bf = torch.empty((NT, ld), dtype=torch.bfloat16, device="cuda")
    hs.hs_synth_fop(bf, f32, "bf16", NT, n, ld, seed, n_signals)
    torch.cuda.synchronize()
    return f32, bf


def test_generator_is_deterministic_exponential_noise():
    n = (1 << 16) + 3
    a, _ = _plane(5, n)
    b, _ = _plane(5, n)
    c, _ = _plane(6, n)
    assert torch.equal(a, b) and not torch.equal(a, c)
    x = a[:, :n].double()
    assert (a[:, n:] == 0).all()
    assert (x >= 0).all() and not torch.signbit(a).any()
    assert abs(x.mean().item() - 1.0) < 0.01
    for t in (1.0, 3.0, 6.0):  # Exponential(1) tail P(x > t) = e^-t
        frac = (x > t).double().mean().item()
        assert abs(frac / np.exp(-t) - 1.0) < 0.05, (t, frac)


def test_generator_bf16_plane_rounds_the_fp32_copy():
    n = 40000
    f32, _ = _plane(9, n, "f32", n_signals=4)
    g32, bf = _plane(9, n, "bf16", n_signals=4)
    assert torch.equal(f32, g32)
    assert torch.equal(bf, g32.to(torch.bfloat16))


def test_generator_injects_signals_at_harmonics():
    n = 200000
    base, _ = _plane(21, n)
    sig, _ = _plane(21, n, n_signals=3)
    diff = (sig - base).cpu().numpy()
    rows, bins = np.nonzero(diff)
    assert 3 <= len(rows) <= 3 * 16
    assert (diff[rows, bins] >= 3.0 - 1e-3).all()
    # each touched point (z, f) is a harmonic (h z0, h f0), h <= 16, of a
    # fundamental (z0, f0) that is itself touched, |z0| <= 2, f0 in [1e4, 1e5)
    Z = (NT - 1) // 2
    fund = {(int(r) - Z, int(b)) for r, b in zip(rows, bins)
            if 10000 <= b < 100000 and abs(int(r) - Z) <= 2}

    def explained(z, f):
        return any(f % f0 == 0 and f // f0 <= 16 and z == (f // f0) * z0 for z0, f0 in fund)

    assert fund and all(explained(int(r) - Z, int(b)) for r, b in zip(rows, bins))


def _served(server, seed, n, dtype, n_signals, timeout_ms=60000):
    t = server.submit(seed, n, dtype, n_signals)
    assert t is not None
    out = server.wait(t, timeout_ms)
    assert out is not None, "request did not finish"
    res, recs = out
    assert res["status"] == hs.HS_OK, res
    return res, recs


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_served_request_matches_oracle_and_hs_run(dtype):
    n, seed = 60001, 11
    ta = synth.thresholds(1e-5, H, NT)
    with hs.Server(NT, H, ta, n_slots=4, slot_bins=1 << 17, cand_capacity=1 << 14) as srv:
        res, got = _served(srv, seed, n, dtype, 6)
    assert res["n_cands"] == len(got) > 0
    f32, _ = _plane(seed, n, "f32", 6)
    # the same plane through hs_run (FP32 path)
    cands = hs.CandBuffer(1 << 14)
    with hs.Plan(NT, n, H, ta, row_pitch=_ld(n)) as plan:
        plan.run(f32, cands)
        ref, cnt, st = cands.fetch()
    assert st == hs.HS_OK and np.array_equal(got, ref)
    # and the FP64 oracle on the bytes copied back
    plane = np.ascontiguousarray(f32[:, :n].cpu().numpy())
    o, near = oracle.detect(plane, H, ta, threads=8)
    near_keys = {(int(c["k"]), int(c["z"]), int(c["f"])) for c in near}
    g = {(int(r["k"]), int(r["z"]), int(r["bin"])): float(r["power"]) for r in got}
    w = {(int(c["k"]), int(c["z"]), int(c["f"])): float(c["power"]) for c in o}
    assert not ((set(g) ^ set(w)) - near_keys)
    for k in set(g) & set(w):
        assert abs(g[k] - w[k]) <= 1e-6 * abs(w[k])


def test_alone_equals_in_mix():
    ta = synth.thresholds(1e-5, H, NT)
    rng = np.random.default_rng(4)
    with hs.Server(NT, H, ta, n_slots=6, slot_bins=1 << 17, cand_capacity=1 << 14,
                   max_group=4) as srv:
        _, alone = _served(srv, 77, 90001, "bf16", 5)
        tickets = []
        for i in range(24):
            if i == 11:
                tickets.append(("R", srv.submit(77, 90001, "bf16", 5)))
            n = int(rng.integers(1000, 1 << 17))
            dt = "bf16" if rng.random() < 0.5 else "f32"
            tickets.append((i, srv.submit(1000 + i, n, dt, int(rng.integers(0, 11)))))
        results = {}
        for name, t in tickets:
            assert t is not None
            out = srv.wait(t, 120000)
            assert out is not None
            results[name] = out
        st = srv.stats()
    res, mixed = results["R"]
    assert res["status"] == hs.HS_OK
    assert np.array_equal(mixed, alone)
    assert all(r[0]["status"] == hs.HS_OK for r in results.values())
    assert st["completed"] == 26 and st["rejected"] == 0
    assert max(r[0]["group_size"] for r in results.values()) > 1  # groups did form


@pytest.mark.parametrize("nonneg", [False, True])
def test_resident_planes_are_summed_in_place(nonneg):
    # requests that bring a plane already in device memory (made upstream),
    # FP32 and BF16 with its FP32 copy, mixed with generated ones: each gives
    # the records of an hs_run of its plane
    ta = synth.thresholds(1e-5, H, NT)
    planes = []
    for i, (n, dt) in enumerate([(70001, "f32"), (50000, "bf16"), (123457, "f32")]):
        f32, bf = _plane(300 + i, n, dt, n_signals=4)
        planes.append((n, dt, f32, bf))
    with hs.Server(NT, H, ta, n_slots=4, slot_bins=1 << 17, cand_capacity=1 << 14,
                   assume_nonneg=nonneg) as srv:
        tickets = []
        for i, (n, dt, f32, bf) in enumerate(planes):
            tickets.append(srv.submit(0, n, dt, 0, fop=f32 if dt == "f32" else bf,
                                      fop32=None if dt == "f32" else f32))
            tickets.append(srv.submit(900 + i, 40000, "bf16", 3))  # generated, in the mix
        results = [srv.wait(t, 60000) for t in tickets]
    for (n, dt, f32, bf), (res, got) in zip(planes, results[0::2]):
        assert res["status"] == hs.HS_OK
        cands = hs.CandBuffer(1 << 14)
        with hs.Plan(NT, n, H, ta, row_pitch=f32.shape[1]) as plan:
            plan.run(f32, cands)
            ref, cnt, st = cands.fetch()
        assert np.array_equal(got, ref) and len(ref) > 0
    assert all(r[0]["status"] == hs.HS_OK for r in results[1::2])


def test_admission_answers_busy_when_the_queue_is_full():
    ta = synth.thresholds(1e-8, H, NT)
    with hs.Server(NT, H, ta, n_slots=1, slot_bins=1 << 20, cand_capacity=256,
                   queue_limit=2) as srv:
        tickets = [srv.submit(i, 1 << 20, "f32", 0) for i in range(40)]
        accepted = [t for t in tickets if t is not None]
        assert len(accepted) < len(tickets)
        for t in accepted:
            res, _ = srv.wait(t, 120000)
            assert res["status"] == hs.HS_OK and res["group_size"] == 1
        assert srv.drain(10000)
        st = srv.stats()
    assert st["rejected"] == len(tickets) - len(accepted)
    assert st["completed"] == len(accepted) and st["peak_queue"] <= 2 + 1


def test_server_rejects_bad_requests():
    ta = synth.thresholds(1e-8, H, NT)
    with hs.Server(NT, H, ta, n_slots=1, slot_bins=1000, cand_capacity=16) as srv:
        with pytest.raises(hs.HsError):
            srv.submit(1, 1001, "f32")
        with pytest.raises(hs.HsError):
            srv.submit(1, 100, "f16")
        with pytest.raises(hs.HsError):
            srv.wait(12345, 0)
