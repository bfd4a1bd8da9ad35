"""FED records from explicit run lists (test infrastructure).

The canonical packers (the oracle's and eventgen's) always cut runs at the APV
boundary and never let runs touch.  The byte format (include/sst.h) allows more:
a run may cross strip 128, two runs may touch (first == previous first + width),
and a width may be anything from 1 to 255 as long as first + width <= 256.  This
builder writes such payloads as they are given, run by run, so that tests can feed
valid but non-canonical data to both sides.
"""
from __future__ import annotations

import numpy as np

CH_PER_FED, FE_PER_FED, CH_PER_FE = 96, 8, 12
FED_MAGIC, ZS_CODE, HDR = 0x46545353, 0x5A, 32


def channel_record(runs) -> bytes:
    """runs: [(first strip, [ADC, ...]), ...] in the order they are written."""
    body = bytearray()
    for first, adcs in runs:
        assert 1 <= len(adcs) <= 255
        body += bytes([first, len(adcs)]) + bytes(adcs)
    n = 3 + len(body)
    return bytes([n & 0xFF, n >> 8, ZS_CODE]) + bytes(body)


def fed_record(fed_id: int, channels: dict) -> bytes:
    """channels: {channel (0..95): runs}; channels not given are empty."""
    units, fe_len = [], []
    for u in range(FE_PER_FED):
        rec = b"".join(channel_record(channels.get(u * CH_PER_FE + k, [])) for k in range(CH_PER_FE))
        fe_len.append(len(rec))
        units.append(rec + bytes(-len(rec) % 8))
    body = b"".join(units)
    total = HDR + len(body)
    total += -total % 16
    hdr = np.zeros(1, dtype=[("magic", "<u4"), ("fed_id", "<u2"), ("n_ch", "u1"), ("n_fe", "u1"),
                             ("fed_bytes", "<u4"), ("reserved", "<u4"), ("fe_len", "<u2", (8,))])
    hdr["magic"], hdr["fed_id"], hdr["n_ch"], hdr["n_fe"], hdr["fed_bytes"] = FED_MAGIC, fed_id, 96, 8, total
    hdr["fe_len"] = fe_len
    out = hdr.tobytes() + body
    return out + bytes(total - len(out))


def event(feds: list) -> tuple[np.ndarray, np.ndarray]:
    """feds: one channels dict per FED -> (raw u8, fed_len u32)."""
    recs = [fed_record(f, ch) for f, ch in enumerate(feds)]
    raw = np.frombuffer(b"".join(recs), dtype=np.uint8).copy()
    return raw, np.array([len(r) for r in recs], dtype=np.uint32)


def expected_digis(feds: list) -> tuple[np.ndarray, np.ndarray]:
    """(global strip, ADC) of every digi, in strip order, straight from the runs."""
    strips, adcs = [], []
    for f, chans in enumerate(feds):
        for c in sorted(chans):
            for first, a in chans[c]:
                for k, v in enumerate(a):
                    strips.append((f * CH_PER_FED + c) * 256 + first + k)
                    adcs.append(v)
    return np.array(strips, dtype=np.uint32), np.array(adcs, dtype=np.uint8)


def non_canonical_feds(rng: np.random.Generator, n_feds: int) -> list:
    """Channels of valid runs the canonical packers never write: runs across strip
    128, touching runs, widths up to 255, every strip of a channel in one run."""
    feds = []
    for f in range(n_feds):
        ch = {}
        a = lambda n: rng.integers(1, 256, n).tolist()  # noqa: E731
        ch[0] = [(120, a(20))]                                  # crosses the APV boundary 127 | 128
        ch[1] = [(50, a(3)), (53, a(2)), (55, a(1))]            # three touching runs: strips 50..55
        ch[2] = [(0, a(255))]                                   # width 255, strips 0..254
        ch[3] = [(1, a(255))]                                   # width 255, strips 1..255
        ch[4] = [(0, a(128)), (128, a(128))]                    # two touching half-channel runs
        ch[5] = [(s, a(1)) for s in range(100, 140)]            # 40 touching single-strip runs across 128
        ch[6] = [(127, a(2)), (200, a(56))]                     # a 2-strip run across 128; a run to strip 255
        ch[7] = [(255, a(1))]                                   # the last strip alone
        ch[12 + (f % 12)] = [(3, a(7)), (10, a(9)), (40, a(129))]  # touching runs, width 129
        ch[95] = [(64, a(192))]                                 # a run from mid-APV to the module end
        # FE units 2 and 3: the same kinds of runs, few enough digis for one tile
        ch[24] = [(121, a(14))]
        ch[25] = [(60, a(2)), (62, a(3)), (65, a(1)), (66, a(4))]
        ch[26] = [(s, a(1)) for s in range(120, 136)]
        ch[30] = [(0, a(2)), (254, a(2))]
        ch[41] = [(126, a(5)), (131, a(1))]
        feds.append(ch)
    return feds
