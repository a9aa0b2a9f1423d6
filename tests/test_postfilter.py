"""The paper's per-plane candidate cap (Section IV-A: first, last or largest
N_cand of a harmonic plane) as the library's host post-step, checked on the
oracle's candidate list: the selection follows Algorithm 2's visiting order
(bins, then templates), does not depend on the order the records arrive in,
and keeps every candidate of a plane that has at most N_cand of them."""
import numpy as np
import pytest

import oracle
from paper_1805_12258_gb300 import hs, synth


@pytest.fixture(scope="module")
def records():
    oracle.build()
    plane = synth.noise(21, 3000, seed=12)
    plane[:, 1000] = 9.0  # a bright column: ties in power at one bin
    ta = synth.thresholds(2e-3, 8, 21)
    cands, _ = oracle.detect(plane, 8, ta)
    r = np.zeros(len(cands), hs.CAND_DTYPE)
    r["bin"], r["z"], r["k"], r["power"] = cands["f"], cands["z"], cands["k"], cands["power"]
    return r


def _expected(r, policy, n_keep):
    out = []
    for k in np.unique(r["k"]):
        g = r[r["k"] == k]
        g = g[np.lexsort((g["z"], g["bin"]))]  # Algorithm 2: bin outer, z inner
        if policy == "first":
            g = g[:n_keep]
        elif policy == "last":
            g = g[len(g) - min(n_keep, len(g)):]
        else:
            pos = np.arange(len(g))
            order = np.lexsort((-pos, -g["power"].astype(np.float64)))[:n_keep]
            g = g[np.sort(order)]
        out.append(g)
    return np.concatenate(out) if out else r[:0]


@pytest.mark.parametrize("policy", ["first", "last", "largest"])
@pytest.mark.parametrize("n_keep", [0, 1, 7, 200, 10 ** 6])
def test_policy_matches_the_visiting_order(records, policy, n_keep):
    got = hs.hs_postfilter(records, policy, n_keep)
    assert np.array_equal(got, _expected(records, policy, n_keep))


@pytest.mark.parametrize("policy", ["first", "last", "largest"])
def test_independent_of_arrival_order(records, policy):
    rng = np.random.default_rng(5)
    a = hs.hs_postfilter(records, policy, 5)
    b = hs.hs_postfilter(records[rng.permutation(len(records))], policy, 5)
    assert np.array_equal(a, b)


def test_planes_under_the_cap_keep_everything(records):
    counts = np.bincount(records["k"])
    cap = int(counts.max())
    got = hs.hs_postfilter(records, "last", cap)
    assert len(got) == len(records)
    assert len(records) > 0 and counts[1:].min() > 5  # every level has several


def test_largest_keeps_the_top_powers(records):
    got = hs.hs_postfilter(records, "largest", 3)
    for k in np.unique(records["k"]):
        g = records[records["k"] == k]["power"]
        kept = got[got["k"] == k]["power"]
        assert len(kept) == min(3, len(g))
        assert kept.min() >= np.sort(g)[::-1][len(kept) - 1]


def test_rejects_bad_arguments():
    with pytest.raises(hs.HsError):
        hs.hs_postfilter(np.zeros(3, hs.CAND_DTYPE), policy=7)
    assert len(hs.hs_postfilter(np.zeros(0, hs.CAND_DTYPE), "last", 5)) == 0
