"""Oracle packer / unpacker against the FED byte format.

The paper (arXiv 2101.11489 section 2) fixes the readout geometry (96 channels x 256
strips per FED) and that zero-suppressed data sit in a CSR-like layout with the
channel as row and the strip as column.  The byte layout itself is this project's
(the paper's Figure 1 is lost).  Pins:
  * a hand-written FED record (tests/golden/two_channel_fed.txt) with digis worked
    out by hand;
  * round trip: seeded digis -> pack -> unpack gives the same digis, and
    pack(unpack(b)) == b for canonical buffers;
  * two independent packers (the oracle's C packer and the event generator's numpy
    packer) write identical bytes;
  * corrupt records set the documented status bit and leave other channels alone.
"""
import os

import numpy as np
import pytest

import eventgen as eg
import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden_fed(name):
    data, digis = [], []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        if tok[0] == "hex":
            data += [int(t, 16) for t in tok[1:]]
        elif tok[0] == "repeat":
            data += [int(t, 16) for t in tok[2:]] * int(tok[1])
        elif tok[0] == "digi":
            digis.append((int(tok[1]), int(tok[2])))
    return np.array(data, np.uint8), digis


def test_golden_fed_unpacks_to_hand_digis():
    raw, want = read_golden_fed("two_channel_fed.txt")
    assert raw.size == 368
    d = orc.unpack_event(raw, np.array([368], np.uint32), 1)
    assert list(zip(d["strip"].tolist(), d["adc"].tolist())) == want
    assert not d["chan_status"].any()
    assert d["chan_off"][:3].tolist() == [0, 3, 6]
    assert d["chan_off"][-1] == 6


def test_golden_fed_is_what_both_packers_write():
    raw, want = read_golden_fed("two_channel_fed.txt")
    n = 96 * 256
    adc = np.zeros(n, np.uint8)
    rec = np.zeros(n, np.uint8)
    for g, a in want:
        adc[g] = a
        rec[g] = 1
    r1, f1 = orc.pack_event(adc, rec, 1)
    r2, f2 = eg.pack_event(adc, rec, 1)
    assert np.array_equal(r1, raw) and np.array_equal(r2, raw)
    assert f1.tolist() == f2.tolist() == [368]


def random_dense(n_feds, occ, seed):
    r = np.random.default_rng(seed)
    n = n_feds * 96 * 256
    rec = (r.random(n) < occ).astype(np.uint8)
    # some long runs and full channels too
    for _ in range(3):
        c = int(r.integers(0, n_feds * 96))
        rec[c * 256:(c + 1) * 256] = 1
    adc = np.where(rec != 0, r.integers(0, 256, n), 0).astype(np.uint8)
    return adc, rec


@pytest.mark.parametrize("occ,seed", [(0.0, 0), (0.01, 1), (0.3, 2), (0.9, 3)])
def test_round_trip(occ, seed):
    adc, rec = random_dense(3, occ, seed)
    raw, fl = orc.pack_event(adc, rec, 3)
    assert all(x % 16 == 0 for x in fl)
    d = orc.unpack_event(raw, fl, 3)
    idx = np.flatnonzero(rec)
    assert np.array_equal(d["strip"], idx)
    assert np.array_equal(d["adc"], adc[idx])
    assert not d["chan_status"].any()
    # pack(unpack(b)) == b
    adc2 = np.zeros_like(adc)
    rec2 = np.zeros_like(rec)
    adc2[d["strip"]] = d["adc"]
    rec2[d["strip"]] = 1
    raw2, fl2 = orc.pack_event(adc2, rec2, 3)
    assert np.array_equal(raw2, raw) and np.array_equal(fl2, fl)
    # the generator's packer writes the same bytes
    raw3, fl3 = eg.pack_event(adc, rec, 3)
    assert np.array_equal(raw3, raw) and np.array_equal(fl3, fl)
    # CSR row pointers agree with the strips
    co = d["chan_off"]
    assert np.array_equal(np.diff(co), np.bincount(idx >> 8, minlength=3 * 96))


def test_round_trip_generated_event():
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    adc, rec = eg.make_event_strips(w, calib, 0)
    raw, fl = eg.pack_event(adc, rec, w.n_feds)
    raw_o, fl_o = orc.pack_event(adc, rec, w.n_feds)
    assert np.array_equal(raw, raw_o) and np.array_equal(fl, fl_o)
    d = orc.unpack_event(raw, fl, w.n_feds)
    idx = np.flatnonzero(rec)
    assert np.array_equal(d["strip"], idx) and np.array_equal(d["adc"], adc[idx])


# ---- corrupt records ---------------------------------------------------------

def base_event():
    adc, rec = random_dense(2, 0.05, 17)
    raw, fl = orc.pack_event(adc, rec, 2)
    return raw, fl, orc.unpack_event(raw, fl, 2)


def channel_record_pos(raw, fed_start, ch):
    """Byte offset of channel ch's record in the FED starting at fed_start."""
    fe_len = [int(raw[fed_start + 16 + 2 * u]) | (int(raw[fed_start + 17 + 2 * u]) << 8) for u in range(8)]
    u, k = divmod(ch, 12)
    p = fed_start + 32 + sum((l + 7) // 8 * 8 for l in fe_len[:u])
    for _ in range(k):
        p += int(raw[p]) | (int(raw[p + 1]) << 8)
    return p


def check_only(d0, d1, bad_channels, bit):
    cs = d1["chan_status"]
    for c in range(cs.size):
        if c in bad_channels:
            assert cs[c] == bit, (c, cs[c])
            assert d1["chan_off"][c + 1] == d1["chan_off"][c]
        else:
            assert cs[c] == 0
            a0 = d0["strip"][d0["chan_off"][c]:d0["chan_off"][c + 1]]
            a1 = d1["strip"][d1["chan_off"][c]:d1["chan_off"][c + 1]]
            assert np.array_equal(a0, a1)


def runs_of(raw, p):
    """[(header offset, first, width)] of the channel record at p."""
    ln = int(raw[p]) | (int(raw[p + 1]) << 8)
    out, q = [], p + 3
    while q < p + ln:
        out.append((q, int(raw[q]), int(raw[q + 1])))
        q += 2 + int(raw[q + 1])
    return out


def pick(raw, fed_start, cond):
    for ch in range(96):
        p = channel_record_pos(raw, fed_start, ch)
        rs = runs_of(raw, p)
        if cond(rs):
            return ch, p, rs
    raise AssertionError("no suitable channel")


def test_bad_packet_code():
    raw, fl, d0 = base_event()
    ch, p, _ = pick(raw, 0, lambda rs: len(rs) >= 1)
    r = raw.copy()
    r[p + 2] = 0x11
    check_only(d0, orc.unpack_event(r, fl, 2), {ch}, orc.ST_BAD_CODE)


def test_zero_width_run():
    raw, fl, d0 = base_event()
    ch, p, rs = pick(raw, 0, lambda rs: len(rs) >= 1)
    r = raw.copy()
    r[rs[0][0] + 1] = 0
    check_only(d0, orc.unpack_event(r, fl, 2), {ch}, orc.ST_RUN_RANGE)


def test_run_past_strip_255():
    raw, fl, d0 = base_event()
    ch, p, rs = pick(raw, 0, lambda rs: len(rs) >= 1 and rs[0][2] >= 2)
    r = raw.copy()
    r[rs[0][0]] = 255
    check_only(d0, orc.unpack_event(r, fl, 2), {ch}, orc.ST_RUN_RANGE)


def test_overlapping_runs():
    raw, fl, d0 = base_event()
    ch, p, rs = pick(raw, 0, lambda rs: len(rs) >= 2)
    r = raw.copy()
    r[rs[1][0]] = rs[0][1]  # second run starts where the first started
    check_only(d0, orc.unpack_event(r, fl, 2), {ch}, orc.ST_RUN_ORDER)


def test_truncated_run():
    raw, fl, d0 = base_event()
    ch, p, rs = pick(raw, int(fl[0]), lambda rs: len(rs) >= 1 and rs[-1][1] + rs[-1][2] < 256)
    r = raw.copy()
    r[rs[-1][0] + 1] = rs[-1][2] + 1  # last run one byte longer than the record holds
    check_only(d0, orc.unpack_event(r, fl, 2), {96 + ch}, orc.ST_TRUNC)


def test_dangling_run_header_byte():
    # a record whose last run leaves one byte: shrink the last run by one strip
    # while keeping the record length -> one stray byte after it
    raw, fl, d0 = base_event()
    ch, p, rs = pick(raw, 0, lambda rs: len(rs) >= 1 and rs[-1][2] >= 2)
    r = raw.copy()
    r[rs[-1][0] + 1] = rs[-1][2] - 1
    check_only(d0, orc.unpack_event(r, fl, 2), {ch}, orc.ST_TRUNC)


def test_channel_length_breaks_fe_framing():
    raw, fl, d0 = base_event()
    p = channel_record_pos(raw, 0, 14)  # FE unit 1, channel 2
    r = raw.copy()
    r[p] = (int(raw[p]) + 1) & 0xFF
    check_only(d0, orc.unpack_event(r, fl, 2), set(range(12, 24)), orc.ST_FRAMING)


def test_short_channel_length_breaks_fe_framing():
    raw, fl, d0 = base_event()
    p = channel_record_pos(raw, 0, 30)  # FE unit 2
    r = raw.copy()
    r[p] = 2
    r[p + 1] = 0
    check_only(d0, orc.unpack_event(r, fl, 2), set(range(24, 36)), orc.ST_FRAMING)


@pytest.mark.parametrize("byte,val", [(0, 0x00), (4, 0x07), (6, 95), (7, 9), (8, 0x01)])
def test_fed_header_errors(byte, val):
    raw, fl, d0 = base_event()
    r = raw.copy()
    r[byte] = val if r[byte] != val else val ^ 1
    check_only(d0, orc.unpack_event(r, fl, 2), set(range(96)), orc.ST_FED_HDR)


def test_fe_length_inconsistent_with_fed_length():
    raw, fl, d0 = base_event()
    r = raw.copy()
    v = (int(r[16]) | (int(r[17]) << 8)) + 16  # FE 0 grows by 16: padded total no longer fed_bytes
    r[16], r[17] = v & 0xFF, v >> 8
    check_only(d0, orc.unpack_event(r, fl, 2), set(range(96)), orc.ST_FED_HDR)


def test_fed_len_disagrees_with_header():
    raw, fl, d0 = base_event()
    fl2 = fl.copy()
    fl2[1] = 16  # too short for a header
    d1 = orc.unpack_event(raw[: int(fl[0]) + 16], fl2, 2)
    assert (d1["chan_status"][96:] == orc.ST_FED_HDR).all()
    assert not d1["chan_status"][:96].any()


def test_absent_fed():
    raw, fl, d0 = base_event()
    fl2 = fl.copy()
    fl2[0] = 0
    d1 = orc.unpack_event(raw[int(fl[0]):], fl2, 2)
    assert not d1["chan_status"].any()
    assert d1["chan_off"][96] == 0
    assert np.array_equal(d1["strip"], d0["strip"][d0["chan_off"][96]:])


def test_fed_ranges_give_the_whole_event():
    """Processing an event as independent FED ranges (the inner level of the
    nested CPU scheme) gives exactly the whole event's digis and clusters."""
    w = eg.WORKLOADS[0]
    calib = eg.make_calibration(w.n_feds, w.seed, w.p_bad)
    e = eg.make_event(w, calib, 3)
    d, c = orc.process_event(e.raw, e.fed_len, w.n_feds, calib.noise, calib.gain, calib.bad, orc.Params())
    off = np.concatenate([[0], np.cumsum(e.fed_len)]).astype(np.int64)
    parts = []
    for f0, f1 in ((0, 7), (7, 8), (8, 31), (31, 50)):
        parts.append(orc.process_feds(e.raw[off[f0]:off[f1]], e.fed_len[f0:f1], f0, f1 - f0, calib.noise,
                                      calib.gain, calib.bad, orc.Params()))
    assert sum(p["n_digi"] for p in parts) == d["strip"].size
    for k in ("det", "first", "width", "charge", "barycenter"):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), c[k]), k


def test_valid_non_canonical_payloads_unpack_run_by_run():
    """Runs across strip 128, touching runs and widths up to 255 are valid (the
    format in include/sst.h); the oracle unpacks them to exactly the digis the
    runs list, and repacking those digis canonically gives the same digis back."""
    import _fedbuild as fb
    feds = fb.non_canonical_feds(np.random.default_rng(5), 3)
    raw, fl = fb.event(feds)
    d = orc.unpack_event(raw, fl, 3)
    strips, adcs = fb.expected_digis(feds)
    assert np.array_equal(d["strip"], strips) and np.array_equal(d["adc"], adcs)
    assert not d["chan_status"].any()
    dense = np.zeros(3 * 96 * 256, np.uint8)
    rec = np.zeros(3 * 96 * 256, np.uint8)
    dense[strips] = adcs
    rec[strips] = 1
    raw2, fl2 = orc.pack_event(dense, rec, 3)
    assert raw2.size != raw.size  # canonical runs are cut at strip 128 and merged where they touch
    d2 = orc.unpack_event(raw2, fl2, 3)
    assert np.array_equal(d2["strip"], strips) and np.array_equal(d2["adc"], adcs)


def test_touching_runs_and_the_apv_boundary_do_not_split_clusters():
    """A cluster is a chain of linked active strips of one module: where the runs
    of the payload start or end, or the APV boundary, plays no part."""
    import _fedbuild as fb
    p = orc.Params()
    noise = np.full(96 * 256, 4.0, np.float32)
    gain = np.ones(96 * 2, np.float32)
    bad = np.zeros(96 * 256, np.uint8)
    split = {0: [(126, [20, 30]), (128, [30, 20])], 1: [(10, [20]), (11, [30]), (12, [20])]}
    whole = {0: [(126, [20, 30, 30, 20])], 1: [(10, [20, 30, 20])]}
    for feds in ([split], [whole]):
        raw, fl = fb.event(feds)
        d, c = orc.process_event(raw, fl, 1, noise, gain, bad, p)
        assert list(zip(c["det"].tolist(), c["first"].tolist(), c["width"].tolist())) == [(0, 126, 4), (1, 10, 3)]
