"""The batched and per-event cluster kernels pick the owner of every candidate (its
leftmost seed, arXiv 2101.11489 section 2: a cluster grows from a seed) 32 digis at a
time from two warp-wide masks: S (digis above the seed threshold) and B (digis that
start a candidate).  A seed owns its candidate when no other seed lies between the
candidate's start and it.  The kernels decide this for all 32 lanes with one 32-bit
addition: a seed generates a carry, a digi that is neither a seed nor a start passes
it on, a start stops it, and the carry into a digi then says that a seed of its
candidate lies before it; the carry out of the window goes into the next one.

Checked here on the CPU against the rule written per lane, on random masks and on
the degenerate ones (no seed, every digi a seed, every digi a start, the first and
last lanes alone).
"""
import random

M = 0xFFFFFFFF


def owners_per_lane(S: int, B: int, seen_in: bool):
    """Each seed looks back to its candidate's start (or into the open candidate of
    the windows before when no start lies at or below it)."""
    O = 0
    for lane in range(32):
        if not (S >> lane) & 1:
            continue
        below = S & ((1 << lane) - 1)
        starts = B & ((2 << lane) - 1)
        if starts:
            ls = starts.bit_length() - 1
            seen = (below >> ls) != 0
        else:
            seen = seen_in or below != 0
        if not seen:
            O |= 1 << lane
    if B:
        seen_out = (S >> (B.bit_length() - 1)) != 0
    else:
        seen_out = seen_in or S != 0
    return O, seen_out


def owners_by_addition(S: int, B: int, seen_in: bool):
    """The kernels' form (32-bit unsigned arithmetic)."""
    x = (S | ~B) & M
    total = (x + S + (1 if seen_in else 0)) & M
    O = S & ((~(total ^ x ^ S) & M) | B)
    seen_out = ((x & S) | ((x | S) & ~total & M)) >> 31
    return O, bool(seen_out)


def test_owner_masks_on_random_windows():
    rng = random.Random(2101)
    for _ in range(50000):
        # sparse and dense masks alike
        S = rng.getrandbits(32) & rng.getrandbits(32)
        B = rng.getrandbits(32) & rng.getrandbits(32) & rng.getrandbits(32)
        if rng.random() < 0.3:
            B |= S & rng.getrandbits(32)  # seeds that start their own candidate
        seen = rng.random() < 0.5
        assert owners_by_addition(S, B, seen) == owners_per_lane(S, B, seen), (hex(S), hex(B), seen)


def test_owner_masks_degenerate_windows():
    special = [0, M, 1, 1 << 31, 0x55555555, 0xAAAAAAAA, 0x80000001]
    for S in special:
        for B in special:
            for seen in (False, True):
                assert owners_by_addition(S, B, seen) == owners_per_lane(S, B, seen), (hex(S), hex(B), seen)


def test_owner_masks_across_windows():
    # a long module cut into windows: the carry out of one window is the carry in of
    # the next, and the owners match the rule applied to the whole module at once
    rng = random.Random(7)
    for _ in range(300):
        n = 32 * rng.randint(2, 6)
        seeds = [rng.random() < 0.2 for _ in range(n)]
        starts = [rng.random() < 0.15 for _ in range(n)]
        starts[0] = True
        whole = []
        last_start_seen = False
        for i in range(n):
            if starts[i]:
                last_start_seen = False
            if seeds[i] and not last_start_seen:
                whole.append(i)
            if seeds[i]:
                last_start_seen = True
        got, seen = [], False
        for base in range(0, n, 32):
            S = sum(1 << k for k in range(32) if seeds[base + k])
            B = sum(1 << k for k in range(32) if starts[base + k])
            O, seen = owners_by_addition(S, B, seen)
            got += [base + k for k in range(32) if (O >> k) & 1]
        assert got == whole
