// sst_fe.cuh -- warp-level unpacking and clustering of two adjacent FE units (24
// consecutive channels of one FED), the work item of the batched and per-event
// cluster kernels.
//
// FE units are independent of one another: their channel records sit back to back
// in the FED record, and clusters never cross a channel (arXiv 2101.11489, section
// 2: channel = module of 256 strips).  One warp handles one work item from the raw
// bytes to staged clusters with no block-wide barrier, so that a GB300 SM keeps
// dozens of independent items in flight and hides the latency of each item's
// serial steps (the run chains, the L2 gathers of calibration).  Two FE units per
// warp rather than one: the serial per-channel run walks then occupy 24 lanes
// instead of 12, and the fixed cost of an item is paid once per pair.
//
// Phases of an item (batched kernel):
//   parse_unit  one lane per FE unit walks the unit's 12 channel lengths; then one
//               lane per channel walks the channel's runs once: validates them,
//               counts digis and, for a staged pair, leaves a descriptor of every
//               run in a slot indexed by the byte position of its header / 3
//               (headers are at least 3 bytes apart, so slots never collide and
//               ascend in (channel, strip) order);
//   mark_slots  the tile is cleared, then each lane takes four slots and puts each
//               run's descriptor at the tile position of its first digi (channel
//               base + digis of the channel before the run): a nonzero tile word
//               marks a run start (no atomics);
//   scan_unit   32 digis at a time: each lane finds its digi's run (the last
//               nonzero tile word at or below it, by a ballot), reads its ADC byte,
//               and applies the thresholds, the gain correction, the candidate rule
//               and the leftmost-seed rule (warp ballots, carries across windows);
//   form_unit   one lane per owned candidate: sums, cluster threshold, centroid.
// Pairs whose digis exceed the tile, or whose bytes exceed the slot area, walk
// their runs a second time per chunk of channels (mark_walk) instead of using slots.
//
// Included by sst_kernels.cu only, inside its namespace, after the mask helper it
// uses (bit).
#pragma once

namespace fe {

// Per-warp shared memory of a work item of U adjacent FE units (U = 1 or 2; the
// work-item width is a launch knob of the batched kernel).  Tile and staging sizes
// share the shared memory that 8 warps of a CTA may use at 4 CTAs per SM: a larger
// tile sends fewer work items through the chunked (two-pass) path, a larger
// staging buffer fewer through in-place global reads.
template <int U>
struct __align__(16) WarpT {
  static constexpr int kUnits = U;                  // FE units per work item
  static constexpr int kChW = U * kChPerFe;         // consecutive channels per work item
  static constexpr int kTile = U == 2 ? 448 : 256;  // digis per warp tile (a chunk of whole channels)
  static constexpr int kBuf = U == 2 ? 1376 : 704;  // bytes of the units staged per warp (larger ones are read in place)
  static constexpr int kSlots = (kTile * 2 + kChW * kMaskWords * 4) / 4;  // run-header slots in own[] + bad[]
  uint8_t fe[kBuf];                      // staged bytes of the FE units
  float qmul[kChW * 2];                  // per APV of the channels: certified multiplier, or -gain
  uint32_t kf[kTile + 4];  // before scan_unit: run descriptors at run starts (ADC byte position << 13 |
                           // channel << 8 | first strip), 0 elsewhere, or, in the per-event kernel,
                           // key | ADC << 16 per digi; after: one word per digi: key (channel in the
                           // work item << 8 | strip, 13 bits; sorted) | flags << 13 (1 active,
                           // 4 first strip of a candidate) | ADC << 16 | gain-corrected charge << 24
                           // (ADC and charge 0 for an inactive digi), then a candidate-start sentinel
  float nsq[kTile];     // noise^2 of each digi
  uint16_t own[kTile];  // first digi of every seeded candidate (run slots, with bad[], until scan_unit)
  uint32_t bad[kChW * kMaskWords];       // bad-strip masks of the channels (only when max_adj > 0)
  uint32_t chan_pos[kChW];               // channel record offset from the first unit's start
  uint32_t chan_cnt[kChW + 1];           // digis per channel, then exclusive prefix
  uint16_t chan_len[kChW];
  uint8_t chan_st[kChW];
  static_assert(kTile % 32 == 0, "whole windows of 32 digis");
};
using Warp = WarpT<2>;  // the per-event cluster kernel's warp (it uses 12 of the 24 channels)

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Exclusive prefix sum of one value per lane; *total (when given) receives the sum.
__device__ __forceinline__ uint32_t warp_excl_sum(uint32_t v, uint32_t* total) {
  const int lane = threadIdx.x & 31;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (total) *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// Where the work item's two FE units are and what the FED header says about them.
struct Unit {
  uint32_t fed, u;         // FED index, first FE unit (0, 2, 4, 6)
  const uint8_t* src;      // first byte of the first unit's records (shared or global), or null
  uint32_t off1;           // byte offset of the second unit's records from src
  uint32_t len;            // bytes of the first unit's records
  uint32_t len1;           // bytes of the second unit's records
  uint8_t fed_status;      // SST_CH_FED_HDR when the FED record is corrupt or out of range, else 0
  bool staged;             // src is the warp's staging buffer
};

// Slots of a staged pair (one per 3 bytes), and whether they fit the slot area.
__device__ __forceinline__ uint32_t n_slots(const Unit& un) { return (un.off1 + un.len1 + 2u) / 3u; }
template <class W>
__device__ __forceinline__ bool use_slots(const Unit& un) { return un.staged && n_slots(un) <= (uint32_t)W::kSlots; }
template <class W>
__device__ __forceinline__ uint32_t* slot_area(W& w) { return reinterpret_cast<uint32_t*>(w.own); }

// Run descriptor in a slot: the run's tile descriptor (ADC byte position, 11 bits,
// << 13 | channel << 8 | first strip) << 8 | digis of the channel before the run.
// Never 0: the ADC bytes of a run start at least 5 bytes into the pair.  An empty
// slot is 0.
__device__ __forceinline__ uint32_t slot_desc(uint32_t adc_pos, uint32_t first, uint32_t c, uint32_t toff) {
  return (adc_pos << 21) | (c << 16) | (first << 8) | toff;
}

// One lane's walk over its channel's runs (record r, len bytes, the record at
// byte `pos` of the pair): validates every run in order and counts the digis; with
// SLOTS, writes each valid run's descriptor to slots[(pos + header) / 3].  The
// first error found decides the status (SST_CH_RUN_RANGE: width 0 or past strip
// 256; SST_CH_RUN_ORDER: starts before the previous run's end; SST_CH_TRUNC: a
// header or ADC bytes past the record end); the channel then has no digis and
// its slots written so far are cleared again.
template <bool SLOTS>
__device__ __forceinline__ uint32_t walk_runs(const uint8_t* r, uint32_t len, uint32_t pos, uint32_t c,
                                              uint32_t* slots, uint8_t* st) {
  uint32_t p = 3, prev_end = 0, cnt = 0;
  uint8_t err = 0;
  while (p + 2 <= len) {
    const uint32_t first = r[p], wd = r[p + 1];
    const uint32_t end = first + wd, np = p + 2 + wd;
    const bool range = wd - 1u > (uint32_t)kStrips - 1u - first;  // width 0, or past strip 256
    if (range || first < prev_end || np > len) {
      err = range ? SST_CH_RUN_RANGE : first < prev_end ? SST_CH_RUN_ORDER : SST_CH_TRUNC;
      break;
    }
    if (SLOTS) slots[(pos + p) / 3u] = slot_desc(pos + p + 2, first, c, cnt);
    prev_end = end;
    cnt += wd;
    p = np;
  }
  if (!err && p != len) err = SST_CH_TRUNC;  // a header cut by the record end
  if (err) {
    if (SLOTS)  // the runs before p were valid: walk them again to clear their slots
      for (uint32_t q = 3; q < p; q += 2 + r[q + 1]) slots[(pos + q) / 3u] = 0u;
    *st = err;
    return 0;
  }
  return cnt;
}

// a1 + a2 for the work item's FE units.  Lane 16 h (h < U) walks unit h's chain of
// 12 channel lengths (the paper's map of channel locations): each length at
// least 3, within the unit, and all of them adding up to the unit's length;
// otherwise all 12 channels get SST_CH_FRAMING.  Then lane c < 12 U validates
// channel c's runs and counts its digis in one walk and, when the units are
// staged and their slots fit, writes a slot descriptor for every valid run.  The
// counts are prefix-summed into chan_cnt.  Returns the digi count; *flags / *nbad
// receive the OR of the channel statuses and the number of bad channels.  src is
// un.src, passed separately so that a caller that knows it is the staging buffer
// lets the compiler read it as shared memory.
template <class W>
__device__ uint32_t parse_unit(W& w, const Unit& un, const uint8_t* src, uint32_t* flags, uint32_t* nbad) {
  const int lane = threadIdx.x & 31;
  uint32_t* slots = slot_area(w);
  const bool sl = use_slots<W>(un);
  if (sl) {  // 16-byte stores: the slot area is a whole number of 16-byte vectors
    const uint32_t nv = (n_slots(un) + 3u) / 4u;
    for (uint32_t i = lane; i < nv; i += 32) reinterpret_cast<uint4*>(slots)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if ((lane & 15) == 0 && (lane >> 4) < W::kUnits) {
    const int h = lane >> 4;
    const uint32_t base = h ? un.off1 : 0u;
    const uint32_t end = h ? un.len1 : un.len;
    uint32_t p = 0;
    int k = 0;
    if (un.src != nullptr) {
      // a unit that breaks the chain is marked as a whole below; the positions and
      // lengths written for it are then never read
#pragma unroll
      for (; k < kChPerFe; k++) {
        if (p + 2 > end) break;
        const uint32_t l = (uint32_t)src[base + p] | ((uint32_t)src[base + p + 1] << 8);
        if (l < 3 || p + l > end) break;
        w.chan_pos[h * kChPerFe + k] = base + p;
        w.chan_len[h * kChPerFe + k] = (uint16_t)l;
        p += l;
      }
    }
    const bool good = k == kChPerFe && p == end;
    const uint32_t st = un.src == nullptr ? un.fed_status : (good ? 0u : (uint32_t)SST_CH_FRAMING);
    uint32_t* st4 = reinterpret_cast<uint32_t*>(w.chan_st + h * kChPerFe);  // 4-byte aligned
#pragma unroll
    for (int v = 0; v < kChPerFe / 4; v++) st4[v] = st * 0x01010101u;
    if (!good) {  // no data, or a broken chain: no channel of the unit is walked (its status may be 0)
      uint32_t* len2 = reinterpret_cast<uint32_t*>(w.chan_len + h * kChPerFe);  // 4-byte aligned
#pragma unroll
      for (int v = 0; v < kChPerFe / 2; v++) len2[v] = 0u;
    }
  }
  __syncwarp();
  uint32_t cnt = 0;
  uint8_t st = 0;
  if (lane < W::kChW) {
    st = w.chan_st[lane];
    const uint32_t len = st ? 0u : w.chan_len[lane];
    if (st == 0 && len >= 3) {
      const uint32_t pos = w.chan_pos[lane];
      const uint8_t* r = src + pos;
      if (r[2] != SST_ZS_CODE)
        st = SST_CH_BAD_CODE;
      else if (sl)
        cnt = walk_runs<true>(r, len, pos, (uint32_t)lane, slots, &st);
      else
        cnt = walk_runs<false>(r, len, pos, (uint32_t)lane, slots, &st);
    }
    w.chan_st[lane] = st;
    if (st) w.chan_len[lane] = 0;
  }
  uint32_t total = 0;
  const uint32_t x = warp_excl_sum(cnt, &total);
  if (lane < W::kChW) w.chan_cnt[lane] = x;
  if (lane == 0) w.chan_cnt[W::kChW] = total;
  *flags = __reduce_or_sync(0xffffffffu, lane < W::kChW ? (uint32_t)st : 0u);
  *nbad = __popc(__ballot_sync(0xffffffffu, lane < W::kChW && st != 0));
  __syncwarp();
  return total;
}

// Greedy chunk of whole channels [c0, c1) with at most W::kTile digis.
template <int NCH, class W>
__device__ __forceinline__ int chunk_end(const W& w, int c0) {
  int c1 = c0 + 1;
  while (c1 < NCH && w.chan_cnt[c1 + 1] - w.chan_cnt[c0] <= (uint32_t)W::kTile) ++c1;
  return c1;
}

// Tile word of digi k of a run: key (channel << 8 | strip) | ADC << 16.
__device__ __forceinline__ uint32_t tile_word(uint32_t c, uint32_t strip, uint32_t adc) {
  return (c << 8) | strip | (adc << 16);
}

// Tile descriptor of a run: ADC byte position << 13 | key of its first digi (channel << 8 | first strip).
__device__ __forceinline__ uint32_t tile_desc(uint32_t adc_pos, uint32_t first, uint32_t c) {
  return (adc_pos << 13) | (c << 8) | first;
}

// Clears the first n tile words (whole 16-byte vectors; n <= kTile), so that a
// tile position where no run starts reads 0.
template <class W>
__device__ __forceinline__ void clear_tile(W& w, int n) {
  const int lane = threadIdx.x & 31;
  for (int v = lane; v < (n + 3) / 4; v += 32) reinterpret_cast<uint4*>(w.kf)[v] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
}

// Single-chunk pair with slots (a2): every valid run's slot descriptor goes to the
// tile position of its first digi (channel base + digis of the channel before it);
// a run of a channel found invalid was cleared.  Each lane takes four consecutive
// slots, so that the lanes' stores spread over the tile.  n: the pair's digis.
template <class W>
__device__ void mark_slots(W& w, const Unit& un, int n) {
  const int lane = threadIdx.x & 31;
  clear_tile(w, n);  // tile positions that start no run read 0
  const uint4* slots = reinterpret_cast<const uint4*>(slot_area(w));
  const int nv = (int)(n_slots(un) + 3u) / 4;  // parse_unit cleared whole vectors: slots past the last are 0
  auto mark = [&](uint32_t d) {
    if (d) w.kf[w.chan_cnt[(d >> 16) & 31u] + (d & 255u)] = d >> 8;  // the run's tile descriptor (never 0)
  };
  for (int v = lane; v < nv; v += 32) {
    const uint4 q = slots[v];
    mark(q.x);
    mark(q.y);
    mark(q.z);
    mark(q.w);
  }
  __syncwarp();
}

// Chunk [c0, c1) (or a pair whose slots do not fit): the chunk's tile words are
// cleared, then lanes c0 .. c1-1 walk their channel's runs again (validated by
// parse_unit) and write each run's tile descriptor where it starts; the walk is
// bounded by the counted digis, so that it cannot leave the tile.
template <class W>
__device__ void mark_walk(W& w, const uint8_t* src, int c0, int c1) {
  const int lane = threadIdx.x & 31;
  clear_tile(w, (int)(w.chan_cnt[c1] - w.chan_cnt[c0]));
  const int c = c0 + lane;
  if (c < c1) {
    const uint32_t cnt = w.chan_cnt[c + 1] - w.chan_cnt[c];
    uint32_t o = w.chan_cnt[c] - w.chan_cnt[c0];
    const uint32_t pos = w.chan_pos[c];
    const uint8_t* r = src + pos;
    const uint32_t len_c = w.chan_len[c];
    uint32_t p = 3, left = cnt;
    while (p + 2 <= len_c && left > 0) {
      const uint32_t first = r[p], wd0 = r[p + 1];
      const uint32_t wd = wd0 < left ? wd0 : left;
      if (wd > 0) w.kf[o] = tile_desc(pos + p + 2, first, (uint32_t)c);
      o += wd;
      left -= wd;
      p += 2 + wd0;
    }
  }
  __syncwarp();
}

// a2 + a3 + a4 in one pass over the tile, 32 digis at a time in strip order; the
// next window's digis are expanded and their calibration gathered while the
// current window is processed.
//  - expansion (EXP): the digi's run is the last run start at or below it (the
//    highest lane up to this one whose tile word is nonzero, found by a ballot, or
//    the last run start of the windows before, carried with its descriptor); its
//    ADC byte is read from the pair's bytes.  Without EXP the tile already holds
//    key | ADC << 16 per digi (0 for a digi that takes no part).
//  - thresholds: the per-strip table holds the channel and seed limits as the
//    largest failing ADC (for an integer ADC, (float)adc > T x noise exactly when
//    adc > floor(T x noise); a bad strip has 255, so it is never active or a
//    seed), and the linking gap; the gain-corrected charge of active digis
//    (saturation codes 254/255 kept) uses the APV's certified multiplier (a
//    division, when the work item has an APV without one); noise^2 comes from the
//    per-strip table;
//  - candidate starts: an active digi whose previous active digi in the tile lies
//    in another channel (the tile is sorted by channel, then strip) or is not
//    linked to it by the hole / bad-strip rules.  One unsigned compare of tile
//    keys decides both: key - prev - 1 >= lim[strip], where lim = min(G + 1, strip)
//    and G is the longest linking gap below the strip (a previous active digi of
//    the same channel is linked when strip - its strip <= G + 1; one of an earlier
//    channel lies at least strip + 1 keys below, and an unsorted or repeated
//    strip wraps the difference);
//  - owners, the leftmost seed of every candidate: two ballots (seeds, candidate
//    starts) and one 32-bit addition over them, with a carry across windows,
//    decide whether another seed lies between a seed's candidate start and it.
// The first digis of owned candidates are compacted in strip order into own[];
// returns their number.  src / src_end: the pair's bytes (EXP).
template <int NCH, bool EXP, class W>
__device__ int scan_unit(W& w, const KParams& kp, const uint2* __restrict__ calq, const uint8_t* src,
                         uint32_t src_end, int n) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt(lane);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  // whether an APV of the work item has no certified multiplier (the scan then divides)
  static_assert(NCH * 2 <= 64, "two multipliers per lane");
  const bool any_div = __any_sync(0xffffffffu, (lane < NCH * 2 && w.qmul[lane] < 0.f) ||
                                                  (lane + 32 < NCH * 2 && w.qmul[lane + 32] < 0.f));
  int n_own = 0, carry_start = -1;
  uint32_t carry_seen = 0u;  // 1: the open candidate of the windows before has a seed
  uint32_t carry_key = 0x1FFFu;  // key of the last active digi of the windows before (none: channel 31)
  int run_s = 0;               // expansion: last run start of the windows before, and its descriptor
  uint32_t run_d = 0;
  // key | ADC << 16 of digi base + lane; 0 beyond n (ADC 0: never active, never a seed)
  auto word_at = [&](int base) -> uint32_t {
    const int i = base + lane;
    if (!EXP) return i < n ? w.kf[i] : 0u;
    const uint32_t v = w.kf[i];  // a run's descriptor where it starts, else 0
    const uint32_t m = __ballot_sync(0xffffffffu, v != 0u);
    const uint32_t le = m & upto;
    const uint32_t dl = __shfl_sync(0xffffffffu, v, 31 - __clz(le));  // (lane 31 when le is 0: not used)
    int s = run_s;
    uint32_t d = run_d;
    if (le) {
      s = base + 31 - __clz(le);
      d = dl;
    }
    if (m) {
      const int l = 31 - __clz(m);
      run_s = base + l;
      run_d = __shfl_sync(0xffffffffu, v, l);
    }
    if (i >= n) return 0u;
    const uint32_t k = (uint32_t)(i - s);
    const uint32_t b = (d >> 13) + k;
    const uint32_t adc = b < src_end ? (uint32_t)src[b] : 0u;
    return ((d & 0x1FFFu) + k) | (adc << 16);  // a valid run ends at strip 256 at most: no carry into the channel
  };
  uint32_t wn = word_at(0);
  uint2 vn = __ldg(calq + (wn & 0x1FFFu));
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint32_t word = wn;
    const uint32_t cv = vn.x;
    const float nq = __uint_as_float(vn.y);
    if (base + 32 < n) {
      wn = word_at(base + 32);
      vn = __ldg(calq + (wn & 0x1FFFu));
    }
    const uint32_t key = word & 0x1FFFu;
    const uint32_t adc = word >> 16;
    const bool act = adc > (cv & 255u);
    const bool sd = adc > ((cv >> 8) & 255u);
    const uint32_t gm = (cv >> 16) & 255u;
    // gain-corrected charge with the APV's multiplier; an APV without a certified
    // multiplier (rq < 0) divides, in a branch taken only for a work item with one
    const float a = __uint2float_rn(adc);
    const float rq = w.qmul[key >> 7];  // the APV of strip st of channel c: 2 c + (st >> 7)
    float xq = __fmul_rn(a, rq);
    if (any_div)
      if (rq < 0.f) xq = __fdiv_rn(a, -rq);
    const int ci = __float2int_rz(__fadd_rn(xq, 0.5f));
    const uint32_t q = !act ? 0u : (adc >= 254u ? adc : (ci > 253 ? 254u : (uint32_t)ci));
    const unsigned A = __ballot_sync(0xffffffffu, act);
    const unsigned Al = A & lt;
    const uint32_t pk_l = __shfl_sync(0xffffffffu, key, 31 - __clz(Al));  // (lane 31 when Al is 0: not used)
    const uint32_t pk = Al ? pk_l : carry_key;
    const bool start = act && key - pk - 1u >= gm;
    const unsigned S = __ballot_sync(0xffffffffu, sd);
    const unsigned B = __ballot_sync(0xffffffffu, start);
    // owners, the first seed of each candidate, by one addition over the window's
    // masks: a seed generates a carry, a digi that is neither a seed nor a candidate
    // start passes it on, a candidate start stops it; so the carry into a digi says
    // that a seed lies between its candidate's start and it (the carry in: the open
    // candidate of the windows before has one)
    const unsigned x = S | ~B;
    const unsigned sum = x + S + carry_seen;
    const unsigned O = S & (~(sum ^ x ^ S) | B);
    carry_seen = ((x & S) | ((x | S) & ~sum)) >> 31;  // the carry out
    const unsigned mb = B & upto;
    const int cs = mb ? base + 31 - __clz(mb) : carry_start;
    if ((O >> lane) & 1u) w.own[n_own + __popc(O & lt)] = (uint16_t)cs;
    n_own += __popc(O);
    carry_start = __shfl_sync(0xffffffffu, cs, 31);  // lane 31's candidate: the open one at the window's end
    carry_key = __shfl_sync(0xffffffffu, act ? key : pk, 31);  // the last active digi up to the window's end
    if (i < n) {
      // an inactive digi keeps its key only (ADC, charge and noise^2 0), so that
      // form_unit sums every digi of a candidate without a test
      w.kf[i] = (act ? word | (1u << 13) : key) | ((start ? 4u : 0u) << 13) | (q << 24);
      w.nsq[i] = act ? nq : 0.f;
    }
  }
  if (lane == 0) w.kf[n] = 4u << 13;  // a candidate start after the last digi ends every walk of form_unit
  __syncwarp();
  return n_own;
}

// Staged cluster record (16 bytes): det | first, width | charge | barycenter.
__device__ __forceinline__ uint4 pack_cluster(uint32_t det, uint32_t first, uint32_t width, uint32_t charge,
                                              float bary) {
  return make_uint4(det, first | (width << 16), charge, __float_as_uint(bary));
}

// Where a kept cluster's amplitudes go during the write pass: the unit's region of
// the amplitude staging buffer (null: no amplitudes) and the running position in
// it (clusters' amplitudes follow each other in strip order).
struct AmpPos {
  uint8_t* amp;   // staging slice of the event, or null
  uint64_t cap;   // bytes in that slice
  uint64_t pos;   // next free byte of the unit's region
};

// a5 + a6: one lane per owned candidate walks it from its first strip to the
// digi before the next candidate start (or the sentinel after the last digi; the
// right boundary is its last active strip), summing in strip order raw ADC,
// noise^2 (binary32, left to right), gain-corrected charge and first moment
// (inactive digis, including those of a following channel before its first
// candidate, add 0 to each); the candidate is widened over up to
// max_adj adjacent bad strips; the cluster threshold decides.  Returns the number
// kept among owners [k_begin, n_own); when `stage` is given the kept clusters are
// written, in strip order, to stage[base + rank] for base + rank < cap.  With
// `keep`, the first window's records are returned to the caller instead; with
// `wsum`, the kept clusters' widths are added to it; with `ap` (write pass), the
// kept clusters' amplitudes are written at ap->pos onwards: 0 for every strip of
// the cluster, then the gain-corrected charge of its active strips.
template <bool AMP, class W>
__device__ uint32_t form_unit(W& w, const KParams& kp, int n, int k_begin, int n_own, uint32_t det0, uint4* stage,
                              uint64_t cap, uint64_t base, uint4* keep = nullptr, bool* keep_pass = nullptr,
                              uint32_t* wsum = nullptr, AmpPos* ap = nullptr) {
  const int lane = threadIdx.x & 31;
  uint32_t kept = 0;
  for (int k0 = k_begin; k0 < n_own; k0 += 32) {
    const int k = k0 + lane;
    bool pass = false;
    uint32_t c = 0, lo = 0, wd = 0, q_sum = 0;
    float bary = 0.f;
    if (k < n_own) {
      int j = w.own[k];
      uint32_t kj = w.kf[j];
      c = (kj >> 8) & 31u;
      const int l = (int)(kj & 255u);
      const uint32_t* B = w.bad + c * kMaskWords;
      int lo_i = l;
      for (int m = 0; m < kp.max_adj && lo_i - 1 >= 0 && bit(B, lo_i - 1); m++) lo_i--;
      uint32_t s16 = 0, mom = 0;  // sums of ADC | q << 8 and of strip x q over the active digis
      float n2 = 0.f;
      int r = l;
      for (;;) {  // an inactive digi adds 0 to every sum (and +0 to noise^2, which leaves it unchanged)
        const uint32_t q = kj >> 24;
        s16 += kj >> 16;
        n2 = __fadd_rn(n2, w.nsq[j]);
        q_sum += q;
        mom += (kj & 255u) * q;
        if (kj & (1u << 13)) r = (int)(kj & 255u);
        kj = w.kf[++j];
        if (kj & (4u << 13)) break;  // the next candidate (or the sentinel after the last digi)
      }
      const uint32_t s_raw = s16 - (q_sum << 8);
      const uint32_t moment = mom - (uint32_t)lo_i * q_sum;
      pass = __uint2float_rn(s_raw) > __fmul_rn(kp.t_cluster, __fsqrt_rn(n2));
      int hi = r;
      for (int m = 0; m < kp.max_adj && hi + 1 < kStrips && bit(B, hi + 1); m++) hi++;
      lo = (uint32_t)lo_i;
      wd = (uint32_t)(hi - lo_i + 1);
      if (pass && (stage || keep))
        bary = q_sum == 0 ? __fadd_rn((float)lo_i, __fmul_rn(0.5f, (float)wd))
                          : __fadd_rn(__fadd_rn((float)lo_i, 0.5f),
                                      __fdiv_rn(__uint2float_rn(moment), __uint2float_rn(q_sum)));
    }
    const unsigned b = __ballot_sync(0xffffffffu, pass);
    if (keep && k0 == k_begin) {
      *keep = pack_cluster(det0 + c, lo, wd, q_sum, bary);
      *keep_pass = pass;
    } else if (pass && stage) {
      const uint64_t pos = base + kept + __popc(b & lanemask_lt(lane));
      if (pos < cap) stage[pos] = pack_cluster(det0 + c, lo, wd, q_sum, bary);
    }
    if (AMP && wsum) *wsum += __reduce_add_sync(0xffffffffu, pass ? wd : 0u);
    if (AMP && ap) {
      // this lane's place among the window's kept clusters' amplitudes
      const uint32_t x = pass ? wd : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      const uint64_t a = ap->pos + incl - x;
      if (pass && ap->amp && a + wd <= ap->cap) {
        uint8_t* dst = ap->amp + a;
        for (uint32_t i = 0; i < wd; i++) dst[i] = 0;
        int j = w.own[k];
        do {
          const uint32_t kj = w.kf[j];
          if (kj & (1u << 13)) dst[(kj & 255u) - lo] = (uint8_t)(kj >> 24);
          ++j;
        } while (j < n && ((w.kf[j] >> 8) & 31u) == c && !(w.kf[j] & (4u << 13)));
      }
      ap->pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    kept += __popc(b);
  }
  return kept;
}

// Loads the APV multipliers (2 per channel) of channels ch0 .. ch0 + NCH - 1 with
// 16-byte loads (the table starts on a 16-byte boundary: ch0 is a multiple of 12).
template <int NCH, class W>
__device__ __forceinline__ void load_calib(W& w, const KParams& kp, uint32_t ch0) {
  const int lane = threadIdx.x & 31;
  constexpr int kG = NCH * 2 / 4;  // vectors of multipliers
  static_assert(kG <= 32, "one multiplier vector per lane");
  if (lane < kG)
    reinterpret_cast<uint4*>(w.qmul)[lane] = __ldg(reinterpret_cast<const uint4*>(kp.qmul + (size_t)ch0 * 2) + lane);
}

// Loads the bad-strip masks (8 words per channel) of the same channels when
// widening over bad strips is enabled (max_adj > 0); otherwise no cluster is
// widened and the masks are never read.  Called once the run slots, which share
// their space, are no longer needed.
template <int NCH, class W>
__device__ __forceinline__ void load_masks(W& w, const KParams& kp, uint32_t ch0) {
  const int lane = threadIdx.x & 31;
  constexpr int kB = NCH * kMaskWords / 4;  // vectors of masks
  if (kp.max_adj > 0) {
    for (int i = lane; i < kB; i += 32)
      reinterpret_cast<uint4*>(w.bad)[i] = __ldg(reinterpret_cast<const uint4*>(kp.badmask + (size_t)ch0 * kMaskWords) + i);
    __syncwarp();
  }
}

// Where one unit's clusters go: its event's staging slice (records allocated unit
// by unit with one atomic each) and the unit's segment bookkeeping; the same for
// its amplitudes when they are wanted (amp non-null).
struct SegOut {
  uint4* stage;         // the event's slice of the staging buffer
  uint64_t cap;         // records in that slice
  uint32_t* ev_alloc;   // the event's allocation counter
  uint32_t* seg_cnt;    // this unit's cluster count
  uint32_t* seg_start;  // this unit's offset in the slice
  uint8_t* amp = nullptr;           // the event's slice of the amplitude staging buffer
  uint64_t amp_cap = 0;             // bytes in that slice
  uint32_t* amp_alloc = nullptr;    // the event's amplitude allocation counter
  uint32_t* seg_amp_cnt = nullptr;  // this unit's amplitude count (0 when they did not fit)
  uint32_t* seg_amp_start = nullptr;  // their offset in the slice, or kNoAmp
};

// The warp's index in the grid, which selects its spill area.
__device__ __forceinline__ uint32_t spill_warp() { return blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); }

// Clusters the `total` digis of one unit and stages its clusters.  `fill(c0, c1,
// single)` prepares the tile for channel chunk [c0, c1) (single: the whole unit
// fits one chunk) and `scan(nn, single)` runs scan_unit over its nn digis.  det0 is
// the module id of the unit's first channel (its first channel in the calibration
// tables).  The kept
// clusters are first counted, then their region is allocated in one piece, then
// they are written.  Without amplitudes, the records of the first 64 candidates
// (two per lane) are kept in registers from the counting pass, so that only
// candidates beyond them are formed twice (a work item of a full event has about
// 49); a unit whose digis exceed the tile is processed chunk by chunk once, its
// records spilled to the warp's area in global memory and copied to their region
// (when they do not fit the area, or with amplitudes, it goes through its chunks
// twice).
// NCH: channels of the work item (12 or 24); AMP: amplitudes are wanted (so.amp
// is then non-null).
template <int NCH, bool AMP, class W, typename Fill, typename Scan>
__device__ void cluster_unit(W& w, const KParams& kp, uint32_t det0, uint32_t total, Fill& fill, Scan& scan,
                             const SegOut& so, sst_event_status* status) {
  const uint32_t ch0 = det0;
  const int lane = threadIdx.x & 31;
  const bool single = total <= (uint32_t)W::kTile;
  constexpr bool amps = AMP;
  uint32_t found = 0, found0 = 0, found1 = 0, wsum = 0;
  int n = 0, n_own = 0;
  uint4 rec0 = make_uint4(0u, 0u, 0u, 0u);  // this lane's records of the first 64 candidates
  uint4 rec1 = make_uint4(0u, 0u, 0u, 0u);
  bool pass0 = false, pass1 = false;
  if (single) {
    n = (int)total;
    if (n > 0) {
      fill(0, NCH, true);
      n_own = scan(n, true);
      load_masks<NCH>(w, kp, ch0);
      if (n_own > 0) {
        if (amps) {
          found = form_unit<AMP>(w, kp, n, 0, n_own, det0, nullptr, 0, 0, nullptr, nullptr, &wsum);
        } else {
          found0 = form_unit<AMP>(w, kp, n, 0, n_own < 32 ? n_own : 32, det0, nullptr, 0, 0, &rec0, &pass0);
          if (n_own > 32)
            found1 = form_unit<AMP>(w, kp, n, 32, n_own < 64 ? n_own : 64, det0, nullptr, 0, 0, &rec1, &pass1);
          found = found0 + found1;
          if (n_own > 64) found += form_unit<AMP>(w, kp, n, 64, n_own, det0, nullptr, 0, 0);
        }
      }
    }
  } else {
    // chunks of whole channels; without amplitudes the kept records go to the
    // warp's spill area as they are formed (one pass), else they are counted now
    // and formed again once their region is allocated
    load_masks<NCH>(w, kp, ch0);
    uint4* spill = amps || !kp.spill || spill_warp() >= kp.spill_warps ? nullptr
                                                                        : kp.spill + (size_t)spill_warp() * kSpillRecords;
    for (int c0 = 0; c0 < NCH;) {
      const int c1 = chunk_end<NCH>(w, c0);
      const int nn = (int)(w.chan_cnt[c1] - w.chan_cnt[c0]);
      if (nn > 0) {
        fill(c0, c1, false);
        const int no = scan(nn, false);
        if (no > 0)
          found += form_unit<AMP>(w, kp, nn, 0, no, det0, spill, spill ? kSpillRecords : 0u, found, nullptr, nullptr,
                                  amps ? &wsum : nullptr);
      }
      c0 = c1;
    }
  }
  uint32_t start = 0, astart = kNoAmp;
  if (lane == 0) {
    start = found ? atomicAdd(so.ev_alloc, found) : 0u;
    uint32_t fits = 0;
    if ((uint64_t)start < so.cap) fits = (uint64_t)start + found <= so.cap ? found : (uint32_t)(so.cap - start);
    if (fits < found) atomicOr(&status->flags, SST_EV_CLUSTER_CAPACITY);
    *so.seg_cnt = fits;
    *so.seg_start = start;
    if (amps) {
      uint32_t acnt = 0;
      if (wsum) {
        const uint32_t a = atomicAdd(so.amp_alloc, wsum);
        if ((uint64_t)a + wsum <= so.amp_cap) {
          astart = a;
          acnt = wsum;
        } else {
          atomicOr(&status->flags, SST_EV_AMP_CAPACITY);
        }
      }
      *so.seg_amp_cnt = acnt;
      *so.seg_amp_start = astart;
    }
  }
  start = __shfl_sync(0xffffffffu, start, 0);
  astart = __shfl_sync(0xffffffffu, astart, 0);
  if (found == 0) return;
  AmpPos ap{astart != kNoAmp ? so.amp : nullptr, so.amp_cap, astart != kNoAmp ? (uint64_t)astart : 0u};
  if (single && !amps) {
    const unsigned b0 = __ballot_sync(0xffffffffu, pass0), b1 = __ballot_sync(0xffffffffu, pass1);
    if (pass0) {
      const uint64_t pos = (uint64_t)start + __popc(b0 & lanemask_lt(lane));
      if (pos < so.cap) so.stage[pos] = rec0;
    }
    if (pass1) {
      const uint64_t pos = (uint64_t)start + found0 + __popc(b1 & lanemask_lt(lane));
      if (pos < so.cap) so.stage[pos] = rec1;
    }
    if (n_own > 64) form_unit<AMP>(w, kp, n, 64, n_own, det0, so.stage, so.cap, (uint64_t)start + found0 + found1);
  } else if (single) {
    form_unit<AMP>(w, kp, n, 0, n_own, det0, so.stage, so.cap, start, nullptr, nullptr, nullptr, &ap);
  } else if (!amps && kp.spill && spill_warp() < kp.spill_warps && found <= kSpillRecords) {
    // every record of the chunked unit is in the warp's spill area
    const uint4* spill = kp.spill + (size_t)spill_warp() * kSpillRecords;
    __syncwarp();  // the lanes' spilled records are visible to the whole warp
    for (uint32_t i = lane; i < found; i += 32)
      if ((uint64_t)start + i < so.cap) so.stage[(uint64_t)start + i] = spill[i];
  } else {
    uint64_t base = start;
    for (int c0 = 0; c0 < NCH;) {
      const int c1 = chunk_end<NCH>(w, c0);
      const int nn = (int)(w.chan_cnt[c1] - w.chan_cnt[c0]);
      if (nn > 0) {
        fill(c0, c1, false);
        const int no = scan(nn, false);
        if (no > 0)
          base += form_unit<AMP>(w, kp, nn, 0, no, det0, so.stage, so.cap, base, nullptr, nullptr, nullptr,
                                 amps ? &ap : nullptr);
      }
      c0 = c1;
    }
  }
}

// FE units u and u + 1 (only u when the work item has one unit; dB is then unused)
// of FED `fed` as described by dA and dB (k_fed_scan checked
// the FED header and wrote, per FE unit, its byte offset in the FED record, its
// length, the FED's status and whether the record holds data).  The units' bytes
// (the first unit, its padding, the second unit) are staged in the warp's buffer
// when they fit, else read in place.  g is the FED record.
template <class W>
__device__ Unit locate(W& w, const uint8_t* g, uint2 dA, uint2 dB, uint32_t fed, uint32_t u) {
  const int lane = threadIdx.x & 31;
  Unit r{fed, u, nullptr, 0, 0, 0, (uint8_t)((dA.y >> 16) & 255u), false};
  if (!(dA.y >> 24)) return r;
  r.len = dA.y & 0xFFFFu;
  if (W::kUnits == 2) {
    r.len1 = dB.y & 0xFFFFu;
    r.off1 = dB.x - dA.x;
  } else {  // one unit: no second unit, span = its length
    r.len1 = 0;
    r.off1 = r.len;
  }
  const uint32_t span = r.off1 + r.len1;
  const uint8_t* a = g + dA.x;
  if (span <= (uint32_t)W::kBuf) {
    if ((((uintptr_t)a) & 7u) == 0) {
      const uint32_t nv = (span + 7u) >> 3;  // whole 8-byte words; padding bytes exist up to the next 8
      for (uint32_t i = lane; i < nv; i += 32)
        *reinterpret_cast<uint2*>(w.fe + 8 * i) = __ldg(reinterpret_cast<const uint2*>(a) + i);
    } else {
      for (uint32_t i = lane; i < span; i += 32) w.fe[i] = __ldg(a + i);
    }
    r.src = w.fe;
    r.staged = true;
  } else {
    r.src = a;
  }
  __syncwarp();
  return r;
}

template <class W>
constexpr bool layout_ok() {
  return 8 * sizeof(W) + 1024 <= 233472 / 4 &&  // 8 warps per CTA fit 4 CTAs per SM
         offsetof(W, bad) % 16 == 0 && offsetof(W, qmul) % 16 == 0 && sizeof(W) % 16 == 0 &&  // vector loads
         offsetof(W, bad) == offsetof(W, own) + sizeof(uint16_t) * W::kTile && offsetof(W, own) % 16 == 0 &&
         W::kSlots % 4 == 0 &&  // the slot area is cleared with 16-byte stores
         W::kSlots * 4 <= sizeof(uint16_t) * W::kTile + sizeof(uint32_t) * W::kChW * kMaskWords &&  // slots
         W::kBuf % 8 == 0 && W::kBuf < 2048 &&  // staging in 8-byte words; ADC positions take 11 bits of a slot
         offsetof(W, chan_st) % 4 == 0 && offsetof(W, chan_len) % 4 == 0 && kChPerFe % 4 == 0;  // word stores
}
static_assert(layout_ok<WarpT<1>>() && layout_ok<WarpT<2>>(), "per-warp shared memory layout");

}  // namespace fe
