// sst_fe.cuh -- warp-level unpacking and clustering of two adjacent FE units (24
// consecutive channels of one FED), the work item of the batched and per-event
// cluster kernels.
//
// FE units are independent of one another: their channel records sit back to back
// in the FED record, and clusters never cross a channel (arXiv 2101.11489, section
// 2: channel = module of 256 strips).  One warp handles one work item from the raw
// bytes to staged clusters with no block-wide barrier, so that a GB300 SM keeps
// dozens of independent items in flight and hides the latency of each item's
// serial steps (the FE length chains, the run chains, the L2 gathers of noise).
// Two FE units per warp rather than one: the serial per-channel steps (length
// chains, run walks) then occupy 24 lanes instead of 12, and the fixed cost of an
// item is paid once per pair.
//
// Included by sst_kernels.cu only, inside its namespace, after the mask helper it
// uses (bit).
#pragma once

namespace fe {

// Tile and staging sizes share the 56 KB of shared memory that 8 warps of a CTA
// may use at 4 CTAs per SM: a larger tile sends fewer work items through the
// chunked (two-pass) path, a larger staging buffer fewer through in-place global
// reads.  With one 32-bit word per digi (10 bytes of tile per digi in all), 448
// digis and 1,376 bytes measured fastest on the 64-event batch (448 / 960: +1.1%,
// 480 / 960: +1.1%).
constexpr int kTile = 448;    // digis per warp tile (a chunk of whole channels)
constexpr int kBuf = 1376;    // bytes of the two FE units staged per warp (larger pairs are read in place)
constexpr int kUnits = 2;     // FE units per work item: two adjacent units of one FED
constexpr int kChW = kUnits * kChPerFe;  // 24 consecutive channels per work item

// Per-warp shared memory.
struct __align__(16) Warp {
  uint8_t fe[kBuf];                      // staged bytes of the two FE units
  uint32_t bad[kChW * kMaskWords];       // bad-strip masks of the 24 channels
  float gain[kChW * 2];                  // APV gains of the 24 channels
  float nsq[kTile];                      // noise^2 of active digis
  uint32_t chan_pos[kChW];               // channel record offset from the first unit's start
  uint32_t chan_cnt[kChW + 1];           // digis per channel, then exclusive prefix
  uint16_t chan_len[kChW];
  uint8_t chan_st[kChW];
  uint32_t kf[kTile];   // one word per digi: key (channel in the work item << 8 | strip, 13 bits; sorted) |
                        // flags << 13 (1 active, 2 seed, 4 first strip of a candidate) | ADC << 16 |
                        // gain-corrected charge of active digis << 24
  uint16_t own[kTile];  // first digi of every seeded candidate; run-start marks (bytes) while the tile fills
};

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Byte b (0..31) of a 32-byte block held one byte per lane.
__device__ __forceinline__ uint32_t byte_at(uint32_t v, int b) { return __shfl_sync(0xffffffffu, v, b) & 0xFFu; }
__device__ __forceinline__ uint32_t u16_at(uint32_t v, int b) { return byte_at(v, b) | (byte_at(v, b + 1) << 8); }
__device__ __forceinline__ uint32_t u32_at(uint32_t v, int b) { return u16_at(v, b) | (u16_at(v, b + 2) << 16); }

// Where the work item's two FE units are and what the FED header says about them.
struct Unit {
  uint32_t fed, u;         // FED index, first FE unit (0, 2, 4, 6)
  const uint8_t* src;      // first byte of the first unit's records (shared or global), or null
  uint32_t off1;           // byte offset of the second unit's records from src
  uint32_t len;            // bytes of the first unit's records
  uint32_t len1;           // bytes of the second unit's records
  uint8_t fed_status;      // SST_CH_FED_HDR when the FED record is corrupt or out of range, else 0
};

// a1 + a2 for the two FE units: lanes 0 and 16 each walk one unit's 12 channel
// lengths (the location map); lanes 0..23 then validate their channel's runs and
// count its digis; the counts are prefix-summed.  A broken length chain
// invalidates the 12 channels of its unit.  Returns the digi count; *flags /
// *nbad receive the OR of the channel statuses and the number of bad channels.
__device__ uint32_t parse_unit(Warp& w, const Unit& un, uint32_t* flags, uint32_t* nbad) {
  const int lane = threadIdx.x & 31;
  if ((lane & 15) == 0) {
    const int h = lane >> 4;
    const uint32_t base = h ? un.off1 : 0u;
    const uint32_t end = h ? un.len1 : un.len;
    bool good = un.src != nullptr;
    uint32_t p = 0;
    for (int k = 0; k < kChPerFe; k++) {
      uint32_t l = 0;
      if (good) {
        if (p + 2 > end) {
          good = false;
        } else {
          l = (uint32_t)un.src[base + p] | ((uint32_t)un.src[base + p + 1] << 8);
          if (l < 3 || p + l > end) good = false;
        }
      }
      w.chan_pos[h * kChPerFe + k] = good ? base + p : 0u;
      w.chan_len[h * kChPerFe + k] = good ? (uint16_t)l : (uint16_t)0;
      if (good) p += l;
    }
    if (good && p != end) good = false;
    uint8_t st = 0;
    if (un.src == nullptr)
      st = un.fed_status;
    else if (!good)
      st = SST_CH_FRAMING;
    for (int k = 0; k < kChPerFe; k++) {
      w.chan_st[h * kChPerFe + k] = st;
      if (st) w.chan_len[h * kChPerFe + k] = 0;
    }
  }
  __syncwarp();
  uint32_t cnt = 0;
  uint8_t st = 0;
  if (lane < kChW) {
    st = w.chan_st[lane];
    const uint32_t len_c = w.chan_len[lane];
    if (st == 0 && len_c >= 3) {
      const uint8_t* r = un.src + w.chan_pos[lane];
      if (r[2] != SST_ZS_CODE) {
        st = SST_CH_BAD_CODE;
      } else {
        uint32_t p = 3, prev_end = 0;
        while (p < len_c) {
          if (p + 2 > len_c) { st = SST_CH_TRUNC; break; }
          const uint32_t first = r[p], wd = r[p + 1];
          if (wd == 0 || first + wd > (uint32_t)kStrips) { st = SST_CH_RUN_RANGE; break; }
          if (first < prev_end) { st = SST_CH_RUN_ORDER; break; }
          if (p + 2 + wd > len_c) { st = SST_CH_TRUNC; break; }
          prev_end = first + wd;
          cnt += wd;
          p += 2 + wd;
        }
      }
      if (st) cnt = 0;
      w.chan_st[lane] = st;
    }
  }
  uint32_t x = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane < kChW) w.chan_cnt[lane] = x - cnt;
  const uint32_t total = __shfl_sync(0xffffffffu, x, kChW - 1);
  if (lane == 0) w.chan_cnt[kChW] = total;
  *flags = __reduce_or_sync(0xffffffffu, lane < kChW ? (uint32_t)st : 0u);
  *nbad = __popc(__ballot_sync(0xffffffffu, lane < kChW && st != 0));
  __syncwarp();
  return total;
}

// Greedy chunk of whole channels [c0, c1) with at most kTile digis.
template <int NCH>
__device__ __forceinline__ int chunk_end(const Warp& w, int c0) {
  int c1 = c0 + 1;
  while (c1 < NCH && w.chan_cnt[c1 + 1] - w.chan_cnt[c0] <= (uint32_t)kTile) ++c1;
  return c1;
}

// a2: the digis of channels [c0, c1) into the tile, all lanes at once.  Lanes
// c0 .. c1-1 walk their channel's runs (validated by parse_unit) and leave, at the
// tile position of each run's first digi, a descriptor (byte position of its ADCs,
// first strip, channel) and a run-start flag.  Then every lane takes one digi at a
// time and finds its run as the last run start at or before it: the highest set
// bit at or below the lane in the ballot of its 32-digi window, or the last run
// start of the windows before, and writes the digi's tile word (key and ADC).
// Descriptors live in nsq[] and run-start flags in the bytes of own[], which
// scan_unit overwrites afterwards.
__device__ void copy_runs(Warp& w, const Unit& un, int c0, int c1) {
  const int lane = threadIdx.x & 31;
  uint32_t* desc = reinterpret_cast<uint32_t*>(w.nsq);
  const int n = (int)(w.chan_cnt[c1] - w.chan_cnt[c0]);
  uint8_t* rs = reinterpret_cast<uint8_t*>(w.own);  // run-start marks
  uint32_t* rs32 = reinterpret_cast<uint32_t*>(w.own);
  for (int i = lane; i < (n + 3) / 4; i += 32) rs32[i] = 0;
  __syncwarp();
  const int c = c0 + lane;
  if (c < c1) {
    const uint32_t cnt = w.chan_cnt[c + 1] - w.chan_cnt[c];
    uint32_t o = w.chan_cnt[c] - w.chan_cnt[c0];
    const uint32_t pos = w.chan_pos[c];
    const uint8_t* r = un.src + pos;
    const uint32_t len_c = w.chan_len[c];
    uint32_t p = 3, left = cnt;
    while (p + 2 <= len_c && left > 0) {
      const uint32_t first = r[p], wd0 = r[p + 1];
      const uint32_t wd = wd0 < left ? wd0 : left;
      if (wd > 0) {
        desc[o] = ((pos + p + 2) << 13) | (first << 5) | (uint32_t)c;
        rs[o] = 1;
      }
      o += wd;
      left -= wd;
      p += 2 + wd0;
    }
  }
  __syncwarp();
  int carry = 0;
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint32_t m = __ballot_sync(0xffffffffu, i < n && rs[i] != 0);
    const uint32_t le = m & (lane == 31 ? 0xffffffffu : ((2u << lane) - 1u));
    const int s = le ? base + 31 - __clz(le) : carry;
    if (i < n) {
      const uint32_t d = desc[s];
      const uint32_t k = (uint32_t)(i - s);
      const uint32_t b = (d >> 13) + k;
      const uint32_t adc = b < un.off1 + un.len1 ? un.src[b] : 0u;
      w.kf[i] = ((d & 31u) << 8) | ((((d >> 5) & 255u) + k) & 255u) | (adc << 16);
    }
    if (m) carry = base + 31 - __clz(m);
  }
  __syncwarp();
}

// a3 + a4 in one pass over the tile, 32 digis at a time in strip order, with the
// next window's noise gather in flight:
//  - thresholds (binary32 product threshold x noise, strict "larger than"; a bad
//    strip, 255 in the linking-gap table, is never active), the gain-corrected
//    charge (saturation codes 254/255 kept) and noise^2 of active digis;
//  - candidate starts: an active digi whose previous active digi in the tile lies
//    in another channel (the tile is sorted by channel, then strip) or is not
//    linked to it by the hole / bad-strip rules, i.e. is more than gapmax[strip]
//    strips below it (the longest linking gap, built from the bad-strip mask
//    when the calibration is uploaded);
//  - owners, the leftmost seed of every candidate: two ballots (seeds, candidate
//    starts) and a carry across windows decide whether another seed lies between
//    a seed's candidate start and it.
// The first digis of owned candidates are compacted in strip order into own[];
// returns their number.
template <int NCH>
__device__ int scan_unit(Warp& w, const KParams& kp, const float* noise, const uint8_t* gapmax, int n) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = lanemask_lt(lane);
  const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  constexpr uint32_t kNone = 0x1FFFu;  // no digi: channel 31, out of range
  int n_own = 0, carry_start = -1;
  bool carry_seen = false;
  uint32_t carry_key = kNone;  // key of the last active digi of the windows before
  uint32_t wn = lane < n ? w.kf[lane] : kNone;  // key | ADC << 16
  uint32_t xn = ((wn >> 8) & 31u) < (uint32_t)NCH ? (wn & 0x1FFFu) : 0u;
  float zn = __ldg(noise + xn);
  uint32_t gn = __ldg(gapmax + xn);
  for (int base = 0; base < n; base += 32) {
    const int i = base + lane;
    const uint32_t word = wn;
    const float nz = zn;
    const uint32_t gmax = gn;
    if (base + 32 < n) {
      wn = i + 32 < n ? w.kf[i + 32] : kNone;
      xn = ((wn >> 8) & 31u) < (uint32_t)NCH ? (wn & 0x1FFFu) : 0u;
      zn = __ldg(noise + xn);
      gn = __ldg(gapmax + xn);
    }
    const uint32_t key = word & 0x1FFFu;
    const uint32_t c = key >> 8, st = key & 255u;
    bool act = false, sd = false;
    uint32_t q = 0;
    float nsq = 0.f;
    if (c < (uint32_t)NCH) {
      const bool isbad = gmax == kGapBad;
      const uint32_t adc = (word >> 16) & 255u;
      const float a = __uint2float_rn(adc);
      act = !isbad && a > __fmul_rn(kp.t_channel, nz);
      sd = !isbad && a > __fmul_rn(kp.t_seed, nz);
      if (act) {
        if (adc >= 254u) {
          q = adc;  // saturation codes are kept
        } else {
          const float x = __fdiv_rn(a, w.gain[c * 2 + (st >> 7)]);
          const int ci = __float2int_rz(__fadd_rn(x, 0.5f));
          q = ci > 253 ? 254u : (uint32_t)ci;
        }
        nsq = __fmul_rn(nz, nz);
      }
    }
    const unsigned A = __ballot_sync(0xffffffffu, act);
    const unsigned Al = A & lt;
    const uint32_t pk_l = __shfl_sync(0xffffffffu, key, Al ? 31 - __clz(Al) : lane);
    const uint32_t pk = Al ? pk_l : carry_key;
    const bool start = act && ((pk >> 8) != c || st - (pk & 255u) - 1u > gmax);
    const unsigned S = __ballot_sync(0xffffffffu, sd);
    const unsigned B = __ballot_sync(0xffffffffu, start);
    const unsigned mb = B & upto;
    bool seen;
    int cs;
    if (mb) {
      const int ls = 31 - __clz(mb);
      seen = (S & lt & ~lanemask_lt(ls)) != 0;
      cs = base + ls;
    } else {
      seen = carry_seen || (S & lt) != 0;
      cs = carry_start;
    }
    const bool owner = sd && !seen;
    const unsigned O = __ballot_sync(0xffffffffu, owner);
    if (owner) w.own[n_own + __popc(O & lt)] = (uint16_t)cs;
    n_own += __popc(O);
    if (B) {
      const int lw = 31 - __clz(B);
      carry_start = base + lw;
      carry_seen = (S >> lw) != 0;
    } else {
      carry_seen = carry_seen || S != 0;
    }
    if (A) carry_key = __shfl_sync(0xffffffffu, key, 31 - __clz(A));
    if (i < n) {
      w.kf[i] = (word & 0x00FF1FFFu) | ((act ? 1u : 0u) << 13) | ((sd ? 2u : 0u) << 13) | ((start ? 4u : 0u) << 13) |
                (q << 24);
      w.nsq[i] = nsq;
    }
  }
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
// digi before the next candidate start (the right boundary is its last active
// strip), summing in strip order raw ADC, noise^2 (binary32, left to right),
// gain-corrected charge and first moment; the candidate is widened over up to
// max_adj adjacent bad strips; the cluster threshold decides.  Returns the number
// kept among owners [k_begin, n_own); when `stage` is given the kept clusters are
// written, in strip order, to stage[base + rank] for base + rank < cap.  With
// `keep`, the first window's records are returned to the caller instead; with
// `wsum`, the kept clusters' widths are added to it; with `ap` (write pass), the
// kept clusters' amplitudes are written at ap->pos onwards: 0 for every strip of
// the cluster, then the gain-corrected charge of its active strips.
template <bool AMP>
__device__ uint32_t form_unit(Warp& w, const KParams& kp, int n, int k_begin, int n_own, uint32_t det0, uint4* stage,
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
      const uint32_t key0 = w.kf[j] & 0x1FFFu;
      c = key0 >> 8;
      const int l = (int)(key0 & 255u);
      const uint32_t* B = w.bad + c * kMaskWords;
      int lo_i = l;
      for (int m = 0; m < kp.max_adj && lo_i - 1 >= 0 && bit(B, lo_i - 1); m++) lo_i--;
      uint32_t s_raw = 0, moment = 0;
      float n2 = 0.f;
      int r = l;
      do {
        const uint32_t kj = w.kf[j];
        if (kj & (1u << 13)) {
          const uint32_t q = kj >> 24;
          const int st = (int)(kj & 255u);
          s_raw += (kj >> 16) & 255u;
          n2 = __fadd_rn(n2, w.nsq[j]);
          q_sum += q;
          moment += (uint32_t)(st - lo_i) * q;
          r = st;
        }
        ++j;
      } while (j < n && ((w.kf[j] >> 8) & 31u) == c && !(w.kf[j] & (4u << 13)));
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

// Clusters the `total` digis of one unit (placed in the tile by `fill(c0, c1)`,
// channel chunk [c0, c1)) and stages its clusters.  The kept clusters are first
// counted, then their region is allocated in one piece, then they are written; a
// unit whose digis exceed the tile goes through its channel chunks twice.  Without
// amplitudes, the records of the first 64 candidates (two per lane) are kept in
// registers from the counting pass, so that only candidates beyond them are
// formed twice (a work item of a full event has about 49).  s0: the work item's first strip in the per-strip
// calibration tables; NCH: channels of the work item (12 or 24); AMP: amplitudes
// are wanted (so.amp is then non-null).
template <int NCH, bool AMP, typename Fill>
__device__ void cluster_unit(Warp& w, const KParams& kp, size_t s0, uint32_t det0, uint32_t total,
                             Fill& fill, const SegOut& so, sst_event_status* status) {
  const int lane = threadIdx.x & 31;
  const bool single = total <= (uint32_t)kTile;
  const float* noise = kp.noise + s0;
  const uint8_t* gapmax = kp.gapmax + s0;
  constexpr bool amps = AMP;
  uint32_t found = 0, found0 = 0, found1 = 0, wsum = 0;
  int n = 0, n_own = 0;
  uint4 rec0 = make_uint4(0u, 0u, 0u, 0u);  // this lane's records of the first 64 candidates
  uint4 rec1 = make_uint4(0u, 0u, 0u, 0u);
  bool pass0 = false, pass1 = false;
  if (single) {
    n = (int)total;
    if (n > 0) {
      fill(0, NCH);
      n_own = scan_unit<NCH>(w, kp, noise, gapmax, n);
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
    for (int c0 = 0; c0 < NCH;) {
      const int c1 = chunk_end<NCH>(w, c0);
      const int nn = (int)(w.chan_cnt[c1] - w.chan_cnt[c0]);
      if (nn > 0) {
        fill(c0, c1);
        const int no = scan_unit<NCH>(w, kp, noise, gapmax, nn);
        if (no > 0) found += form_unit<AMP>(w, kp, nn, 0, no, det0, nullptr, 0, 0, nullptr, nullptr, amps ? &wsum : nullptr);
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
  } else {
    uint64_t base = start;
    for (int c0 = 0; c0 < NCH;) {
      const int c1 = chunk_end<NCH>(w, c0);
      const int nn = (int)(w.chan_cnt[c1] - w.chan_cnt[c0]);
      if (nn > 0) {
        fill(c0, c1);
        const int no = scan_unit<NCH>(w, kp, noise, gapmax, nn);
        if (no > 0)
          base += form_unit<AMP>(w, kp, nn, 0, no, det0, so.stage, so.cap, base, nullptr, nullptr, nullptr,
                            amps ? &ap : nullptr);
      }
      c0 = c1;
    }
  }
}

// Loads the bad-strip masks (8 words per channel) and APV gains (2 per channel)
// of channels ch0 .. ch0 + NCH - 1 with 16-byte loads (both tables start on a
// 16-byte boundary: ch0 is a multiple of 12).
template <int NCH>
__device__ __forceinline__ void load_calib(Warp& w, const KParams& kp, uint32_t ch0) {
  const int lane = threadIdx.x & 31;
  constexpr int kB = NCH * kMaskWords / 4, kG = NCH * 2 / 4;  // vectors of masks, of gains
  for (int i = lane; i < kB + kG; i += 32) {
    if (i < kB)
      reinterpret_cast<uint4*>(w.bad)[i] = __ldg(reinterpret_cast<const uint4*>(kp.badmask + (size_t)ch0 * kMaskWords) + i);
    else
      reinterpret_cast<uint4*>(w.gain)[i - kB] = __ldg(reinterpret_cast<const uint4*>(kp.gain + (size_t)ch0 * 2) + (i - kB));
  }
}

// FE units u and u + 1 of FED `fed` as described by dA and dB (k_fed_scan checked
// the FED header and wrote, per FE unit, its byte offset in the FED record, its
// length, the FED's status and whether the record holds data).  The units' bytes
// (the first unit, its padding, the second unit) are staged in the warp's buffer
// when they fit, else read in place.  g is the FED record.
__device__ Unit locate(Warp& w, const uint8_t* g, uint2 dA, uint2 dB, uint32_t fed, uint32_t u) {
  const int lane = threadIdx.x & 31;
  Unit r{fed, u, nullptr, 0, 0, 0, (uint8_t)((dA.y >> 16) & 255u)};
  if (!(dA.y >> 24)) return r;
  r.len = dA.y & 0xFFFFu;
  r.len1 = dB.y & 0xFFFFu;
  r.off1 = dB.x - dA.x;
  const uint32_t span = r.off1 + r.len1;
  const uint8_t* a = g + dA.x;
  if (span <= (uint32_t)kBuf) {
    if ((((uintptr_t)a) & 7u) == 0) {
      const uint32_t nv = (span + 7u) >> 3;  // whole 8-byte words; padding bytes exist up to the next 8
      for (uint32_t i = lane; i < nv; i += 32)
        *reinterpret_cast<uint2*>(w.fe + 8 * i) = __ldg(reinterpret_cast<const uint2*>(a) + i);
    } else {
      for (uint32_t i = lane; i < span; i += 32) w.fe[i] = __ldg(a + i);
    }
    r.src = w.fe;
  } else {
    r.src = a;
  }
  __syncwarp();
  return r;
}

static_assert(8 * sizeof(Warp) + 1024 <= 233472 / 4, "8 warps per CTA must fit 4 CTAs per SM");
static_assert(offsetof(Warp, bad) % 16 == 0 && offsetof(Warp, gain) % 16 == 0 && sizeof(Warp) % 16 == 0,
              "vector calibration loads need 16-byte aligned tables");

}  // namespace fe
