"""The linking-gap table the device builds at calibration upload, checked against
the oracle's hole / bad-strip rule on the CPU.

The batched and per-event cluster kernels decide whether two successive active
strips a < t of a module are linked (same candidate) by one compare,
t - a - 1 <= G(t), where G(t) is the longest run of strips just below t in which
every maximal run of bad strips is at most max_seq_bad long and every maximal run
of good strips at most max_seq_holes long (k_gapmax builds it by walking down from
t).  That is exact because a valid gap stays valid when shortened from below.  Here
G is rebuilt the same way from random bad-strip maps and compared, for pairs of
strips, with the oracle clustering a module whose only active strips are a and t:
one cluster [a, t] when they are linked, two single-strip clusters otherwise.

The kernels store L(t) = min(G(t) + 1, t) and compare tile keys (channel << 8 |
strip) once: key(t) - key(prev) - 1 >= L(t), unsigned, starts a new candidate.
test_key_compare_matches_the_link_rule checks that this one compare gives the same
decision as "another channel, or t - a - 1 > G(t)" for every strip pair, every
G(t) <= t and previous active strips in the same, an earlier or no channel.
"""
import numpy as np
import pytest

import oracle as orc

N = 256


def gap_table(bad: np.ndarray, max_holes: int, max_bad: int) -> np.ndarray:
    g = np.zeros(N, np.int64)
    for t in range(N):
        run, prev, n = 0, -1, 0
        for u in range(t - 1, -1, -1):
            b = int(bad[u])
            run = run + 1 if b == prev else 1
            prev = b
            if run > (max_bad if b else max_holes):
                break
            n += 1
        g[t] = n
    return g


def linked_by_oracle(a: int, t: int, bad: np.ndarray, p: orc.Params) -> bool:
    adc = np.zeros(N, np.uint8)
    adc[a] = adc[t] = 100
    noise = np.ones(N, np.float32)
    gain = np.ones(N, np.float32)
    c = orc.cluster_module(adc, noise, bad, gain, p)
    if c["first"].size == 1:
        assert int(c["first"][0]) == a and int(c["width"][0]) == t - a + 1
        return True
    assert c["first"].tolist() == [a, t] and c["width"].tolist() == [1, 1]
    return False


@pytest.mark.parametrize("holes,bad_lim,p_bad", [(0, 1, 0.3), (0, 0, 0.3), (1, 1, 0.4), (2, 3, 0.5),
                                                 (3, 0, 0.2), (0, 3, 0.6), (4, 2, 0.5)])
def test_gap_table_matches_the_link_rule(holes, bad_lim, p_bad):
    rng = np.random.default_rng(1000 + 17 * holes + bad_lim)
    bad = (rng.random(N) < p_bad).astype(np.uint8)
    p = orc.Params(max_seq_holes=holes, max_seq_bad=bad_lim, max_adj_bad=0)
    g = gap_table(bad, holes, bad_lim)
    good = np.flatnonzero(bad == 0)
    pairs = [(int(a), int(t)) for i, a in enumerate(good) for t in good[i + 1:i + 12]]
    pairs += [(int(a), int(t)) for a, t in rng.choice(good, size=(200, 2)) if a < t]
    checked = linked = 0
    for a, t in pairs:
        expect = t - a - 1 <= g[t]
        assert linked_by_oracle(a, t, bad, p) == expect, (a, t, g[t])
        checked += 1
        linked += expect
    assert checked > 300 and 0 < linked < checked  # both outcomes occur


def test_gap_table_special_cases():
    bad = np.zeros(N, np.uint8)
    # no bad strips: only adjacent strips link with max_seq_holes = 0, and every
    # gap of up to max_seq_holes good strips links otherwise
    assert np.all(gap_table(bad, 0, 1) == 0)
    g = gap_table(bad, 3, 1)
    assert g.tolist() == [min(t, 3) for t in range(N)]
    # one bad strip between two good ones links with max_seq_bad >= 1 only
    bad[10] = 1
    assert gap_table(bad, 0, 1)[11] == 1 and gap_table(bad, 0, 0)[11] == 0
    # below strip 11 two bad strips in a row: max_seq_bad = 1 links only over strip 10
    bad[9] = 1
    assert gap_table(bad, 0, 1)[11] == 1 and gap_table(bad, 0, 2)[11] == 2
    # hole, bad, hole below strip 22 (bad strip 20) is one valid gap of 3 with
    # limits (1, 1); the strip below it would make a run of two holes
    bad[:] = 0
    bad[20] = 1
    assert gap_table(bad, 1, 1)[22] == 3 and gap_table(bad, 0, 1)[22] == 0
    p11 = orc.Params(max_seq_holes=1, max_seq_bad=1, max_adj_bad=0)
    assert linked_by_oracle(18, 22, bad, p11) and not linked_by_oracle(17, 22, bad, p11)


def starts_by_key_compare(key: int, prev: int, lim: int) -> bool:
    """The kernels' test for a new candidate: one unsigned 32-bit compare."""
    return ((key - prev - 1) % (1 << 32)) >= lim


def test_key_compare_matches_the_link_rule():
    none = 0x1FFF  # the scan's "no previous active digi": channel 31, above every key
    c = 7
    for t in range(N):
        key = (c << 8) | t
        for g in range(t + 1):  # G(t) <= t: the walk down from t - 1 stops at strip 0
            lim = min(g + 1, t)
            assert 0 <= lim <= 255
            assert starts_by_key_compare(key, none, lim)
            for a in range(N):
                # same channel: a new candidate unless a < t is linked; a repeated or
                # unsorted strip (a >= t) always starts one
                same = (c << 8) | a
                assert starts_by_key_compare(key, same, lim) == (a >= t or t - a - 1 > g), (t, g, a)
                # an earlier channel: always a new candidate
                for pc in (0, c - 1):
                    assert starts_by_key_compare(key, (pc << 8) | a, lim), (t, g, a, pc)


def test_key_compare_on_random_bad_maps():
    rng = np.random.default_rng(77)
    for holes, bad_lim, p_bad in [(0, 1, 0.3), (2, 3, 0.5), (4, 2, 0.5)]:
        bad = (rng.random(N) < p_bad).astype(np.uint8)
        g = gap_table(bad, holes, bad_lim)
        lim = np.minimum(g + 1, np.arange(N))
        assert lim.max() <= 255
        for a in range(N):
            for t in range(a + 1, min(N, a + 40)):
                key, prev = (3 << 8) | t, (3 << 8) | a
                assert starts_by_key_compare(key, prev, int(lim[t])) == (t - a - 1 > g[t])
