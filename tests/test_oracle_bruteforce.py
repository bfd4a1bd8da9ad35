"""The oracle's left-to-right clusterizer against two independent statements.

1. ``oracle/bruteforce.py``: the candidate rule written as a predicate over every
   interval of the module (arXiv 2101.11489 section 2: each cluster is bounded left
   and right around its seeds), exhaustively over all strip states of modules of up
   to 5 strips for several hole / bad-strip limits, over all 6-strip modules for the
   default limits, and over random 6-strip modules.
2. A textbook special case: with no bad strips and no holes allowed, candidates are
   exactly the maximal runs of consecutive active strips (found with numpy.diff).
"""
import itertools

import numpy as np
import pytest

import oracle as orc
from oracle import Params
from oracle import bruteforce as bf

# noise 4: channel limit 8, seed limit 12, single-strip cluster limit 20
STATES = [(0, 0), (6, 0), (10, 0), (14, 0), (40, 0), (0, 1), (40, 1)]  # (adc, bad)
PARAMS = [Params(), Params(max_seq_bad=0), Params(max_seq_holes=1, max_seq_bad=1),
          Params(max_seq_holes=1, max_seq_bad=0, max_adj_bad=1), Params(max_seq_holes=2, max_seq_bad=2, max_adj_bad=1),
          Params(t_cluster=1.0)]


def run_both(states, p, gain=1.0):
    adc = [a for a, _ in states]
    bad = [b for _, b in states]
    n = len(states)
    noise = np.full(n, 4.0, np.float32)
    g = np.full(n, gain, np.float32)
    r = orc.cluster_module(np.array(adc, np.uint8), noise, np.array(bad, np.uint8), g, p)
    got = list(zip(r["first"].tolist(), r["width"].tolist(), r["charge"].tolist(), r["barycenter"].tolist()))
    want = bf.cluster_module(adc, noise.tolist(), bad, g.tolist(), p)
    return got, want


@pytest.mark.parametrize("p", PARAMS, ids=lambda p: f"h{p.max_seq_holes}b{p.max_seq_bad}a{p.max_adj_bad}t{p.t_cluster}")
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_exhaustive_small_modules(n, p):
    for states in itertools.product(STATES, repeat=n):
        got, want = run_both(states, p)
        assert got == want, (states, got, want)


@pytest.mark.parametrize("p", PARAMS[:3], ids=["default", "b0", "h1b1"])
def test_random_six_strip_modules(p):
    r = np.random.default_rng(1234)
    for _ in range(3000):
        states = [STATES[i] for i in r.integers(0, len(STATES), 6)]
        got, want = run_both(states, p, gain=float(np.float32(r.uniform(0.8, 1.2))))
        assert got == want, (states, got, want)


def test_random_adc_six_strip_modules():
    r = np.random.default_rng(99)
    p = Params()
    for _ in range(3000):
        adc = r.integers(0, 256, 6)
        adc[r.random(6) < 0.4] = 0
        bad = (r.random(6) < 0.15).astype(int)
        got, want = run_both(list(zip(adc.tolist(), bad.tolist())), p)
        assert got == want


def test_runs_of_consecutive_actives_without_bad_strips():
    r = np.random.default_rng(42)
    p = Params(max_seq_holes=0, max_seq_bad=0, t_cluster=0.0)
    for _ in range(300):
        adc = r.integers(0, 60, 256).astype(np.uint8)
        adc[r.random(256) < 0.5] = 0
        noise = np.full(256, 4.0, np.float32)
        act = (adc > 8).astype(np.int8)
        seed = adc > 12
        edges = np.diff(np.concatenate([[0], act, [0]]))
        starts = np.flatnonzero(edges == 1)
        ends = np.flatnonzero(edges == -1)
        want = [(s, e - s) for s, e in zip(starts, ends) if seed[s:e].any()]
        got = orc.cluster_module(adc, noise, np.zeros(256, np.uint8), np.ones(256, np.float32), p)
        assert list(zip(got["first"].tolist(), got["width"].tolist())) == want


def test_exhaustive_six_strip_modules_default_parameters():
    """Every pattern of the 7 strip states over 6-strip modules (7^6 = 117,649),
    default thresholds and limits (section 2; channel 2, seed 3, cluster 5, no
    holes, one bad strip): the oracle's scan equals the interval predicate."""
    p = Params()
    for states in itertools.product(STATES, repeat=6):
        got, want = run_both(states, p)
        assert got == want, (states, got, want)
