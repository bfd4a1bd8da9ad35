// sst_kernels.cu -- sm_103a kernels for unpacking zero-suppressed FED data and
// three-threshold clustering (arXiv 2101.11489, section 2), per event and batched
// (section 3).
//
// Clustering work item: two adjacent FE units (24 channels; one unit as a launch
// option) of one FED of one event, handled by one warp end to end (sst_fe.cuh):
// run validation and counts (one lane per channel, one walk), expansion of the runs into an on-chip digi
// tile sorted by strip fused with thresholds, candidate boundaries and the
// leftmost seed of each candidate (one lane per digi, warp ballots; the paper's
// array of seed strips), and cluster forming (one lane per kept candidate).  No
// block-wide barrier: a GB300 SM keeps 32 independent items in flight.  The FED
// headers are checked once per FED by the prologue kernel (k_fed_scan), which
// hands every FE unit its byte range; the FE units' channel length chains (the
// paper's "map of channel locations", here on the device) are walked from the
// staged bytes by the warp that owns the units.
//
// Output order without device-side waits: every unit allocates an exact-size
// staging region with one atomic per event; k_order prefix-sums the units' counts
// per event and copies the staged records into each event's sorted cluster SoA
// (with amplitudes: k_clu_scan scans, k_compact copies).  Placing each unit's
// clusters directly with a look-back over the units before it, in the batched
// kernel, measured slower: the look-back's L2 round trips and the waits for
// units still being counted cost more than the ordering pass.
//
// Per-event unpacking (k_unpack) keeps one CTA per FED and places the FED's digis
// with a warp-parallel decoupled look-back over the FEDs before it.
//
// Floating point in the threshold tests and sums uses explicit round-to-nearest
// intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn): no multiply-add is
// contracted and results equal a sequential binary32 evaluation bit for bit.
//
// Every device wait (the look-back) has an iteration limit; when it runs out the
// event is flagged SST_EV_TIMEOUT and the CTA carries on without the value.
#include <cstddef>
#include <utility>

#include "sst_internal.h"

namespace sst {

namespace {

// ---------------------------------------------------------------- constants

constexpr unsigned long long kLbAgg = 1ull << 62;  // state carries this FED's own count
constexpr unsigned long long kLbPre = 2ull << 62;  // state carries the inclusive prefix
constexpr unsigned long long kLbMask = 3ull << 62;
constexpr uint32_t kLbSpinLimit = 1u << 20;         // polls before giving up (about a second)
constexpr uint64_t kBadOff = ~0ull;                // fed_off marker: record outside the event
constexpr int kFedBufMin = 16384;                  // bytes of FED record staged on chip (at least)
constexpr int kFedScanThreads = 128;               // FEDs per k_fed_scan CTA

// Shared scalars.
enum {
  S_TICKET = 0, S_FEDOK, S_TOTAL, S_BASE, S_FLAGS, S_NBAD, S_TIMEOUT, S_SLOTS, S_NOWN,
  S_NEXT_T, S_NEXT_LEN, S_NEXT_OFF_LO, S_NEXT_OFF_HI, S_SCAL_N = 16
};

// ---------------------------------------------------------------- shared memory

// What one CTA of the per-event unpack kernel keeps on chip for one FED.
// TILE = digis per tile.
template <int TILE>
struct __align__(16) Shm {
  static constexpr int kRegion = (8 * TILE > kFedBufMin) ? 8 * TILE : kFedBufMin;
  uint32_t scal[S_SCAL_N];
  uint32_t wsum[32];
  uint32_t chan_pos[kCh];       // byte offset of the channel record within the FED
  uint32_t chan_cnt[kCh + 1];   // digis per channel, then exclusive prefix (in place)
  uint32_t chan_slot[kCh + 1];  // first run slot of each channel
  uint32_t fe_len[kFe];
  uint16_t chan_len[kCh];
  uint8_t chan_st[kCh];
  uint16_t t_key[TILE];  // (channel << 8) | strip, sorted
  uint8_t t_adc[TILE];
  alignas(16) uint2 runs[TILE];  // run records
  alignas(16) uint8_t fedbuf[kRegion];  // the staged FED record
};

// Fields written with 8- or 16-byte accesses must be aligned to that width.
template <int TILE>
constexpr bool shm_aligned() {
  return offsetof(Shm<TILE>, runs) % 16 == 0 && offsetof(Shm<TILE>, fedbuf) % 16 == 0 &&
         sizeof(Shm<TILE>) % 16 == 0;
}
static_assert(shm_aligned<1024>() && shm_aligned<2048>() && shm_aligned<4096>(), "shared layout misaligned");

// Run record: x = byte offset of the run's first ADC byte in the FED record;
// y = tile offset within the channel (9 bits) | first strip << 9 | width << 17 |
// channel << 25.  Width 0 marks an unused slot.
__device__ __forceinline__ uint32_t run_y(uint32_t toff, uint32_t first, uint32_t width, uint32_t ch) {
  return toff | (first << 9) | (width << 17) | (ch << 25);
}

// ---------------------------------------------------------------- small helpers

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before the kernel ahead of it on the stream has
// finished; pdl_wait() returns once that kernel has completed and its writes are
// visible (at once for a kernel launched the ordinary way).  pdl_release() lets
// the next such kernel be launched before this one ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t rd16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
__device__ __forceinline__ uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// Exclusive block-wide scan of one value per thread (blockDim.x <= 1024).
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  const uint32_t pre = warp > 0 ? wsum[warp - 1] : 0u;
  *total = wsum[nw - 1];
  __syncthreads();
  return pre + x - v;
}

// Warp-wide exclusive scan, in place, of 96 entries (three consecutive per lane);
// a[96] receives the total, which is also returned.
__device__ __forceinline__ uint32_t warp_scan96(uint32_t* a, int lane) {
  const uint32_t v0 = a[lane * 3], v1 = a[lane * 3 + 1], v2 = a[lane * 3 + 2];
  const uint32_t local = v0 + v1 + v2;
  uint32_t x = local;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  const uint32_t e = x - local;
  a[lane * 3] = e;
  a[lane * 3 + 1] = e + v0;
  a[lane * 3 + 2] = e + v0 + v1;
  const uint32_t total = __shfl_sync(0xffffffffu, x, 31);
  if (lane == 31) a[kCh] = total;
  return total;
}

// Decoupled look-back over items lo .. idx-1 of one event, by one warp: each
// round reads 32 predecessors at once and sums back to the nearest inclusive
// prefix.  Returns the sum of the counts of all earlier items (on every lane).
// After spin_limit polls without progress it gives up: *timed_out is set and the
// partial sum is returned.
__device__ uint32_t lookback_warp(unsigned long long* lb, long long idx, long long lo, uint32_t spin_limit,
                              bool* timed_out) {
  const int lane = threadIdx.x & 31;
  uint32_t excl = 0;
  long long j = idx - 1;
  uint32_t spins = 0;
  unsigned ns = 32;
  while (j >= lo) {
    const long long jj = j - lane;
    const unsigned long long v = jj >= lo ? ld_acquire(lb + jj) : kLbPre;
    const unsigned pre = __ballot_sync(0xffffffffu, (v & kLbMask) == kLbPre);
    const unsigned rdy = __ballot_sync(0xffffffffu, (v & kLbMask) != 0);
    const int stop = pre ? __ffs(pre) - 1 : 31;
    const unsigned need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
    if ((rdy & need) != need) {
      if (++spins > spin_limit) {
        *timed_out = true;
        return excl;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
      continue;
    }
    excl += __reduce_add_sync(0xffffffffu, lane <= stop ? (uint32_t)v : 0u);
    if (pre) break;
    j -= 32;
  }
  return excl;
}

// ---------------------------------------------------------------- FED parsing (a1, a2)

// Copies a FED record into shared memory (16-byte loads when aligned).
__device__ void stage_fed(const uint8_t* g, uint32_t len, uint8_t* dst) {
  if ((((uintptr_t)g) & 15u) == 0) {
    const uint32_t nv = len >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(g);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (uint32_t i = threadIdx.x; i < nv; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (uint32_t i = (nv << 4) + threadIdx.x; i < len; i += blockDim.x) dst[i] = __ldg(g + i);
  } else {
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) dst[i] = __ldg(g + i);
  }
}

// Header, FE-unit walk, per-channel validation and digi counts (a1 + a2).  `src`
// points at the record (shared or global memory).  On return (after a barrier):
// chan_* describe each channel, chan_cnt holds the exclusive prefix of the digi
// counts, scal[S_TOTAL] the FED's digis, scal[S_FLAGS] / scal[S_NBAD] the OR of
// channel statuses and the number of bad channels, and - when the run slots
// fitted (scal[S_SLOTS] != 0) - runs[] one record per run.
template <int TILE>
__device__ void parse_body(Shm<TILE>& s, const uint8_t* src, uint32_t len, uint32_t fed_id, bool in_range) {
  const int tid = threadIdx.x, lane = tid & 31;
  const bool present = in_range && len > 0;
  if (tid < 32) {
    // header and FE-unit lengths: lanes 0..7 hold one FE unit each
    bool ok = present && len >= (uint32_t)kHdr;
    uint32_t fl = 0, start = 0;
    if (ok) {
      fl = lane < kFe ? rd16(src + 16 + 2 * lane) : 0u;
      const uint32_t padded = (fl + 7u) & ~7u;
      uint32_t x = padded;
#pragma unroll
      for (int d = 1; d < 8; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
      }
      start = kHdr + x - padded;
      const uint32_t body = __shfl_sync(0xffffffffu, x, kFe - 1);
      const uint32_t total = (kHdr + body + 15u) & ~15u;
      bool hdr = true;
      if (lane == 0)
        hdr = rd32(src) == SST_FED_MAGIC && rd16(src + 4) == fed_id && src[6] == (uint8_t)kCh &&
              src[7] == (uint8_t)kFe && rd32(src + 8) == len && total == len;
      ok = __shfl_sync(0xffffffffu, hdr, 0);
    }
    const uint8_t fed_status = (!in_range || (present && !ok)) ? (uint8_t)SST_CH_FED_HDR : (uint8_t)0;
    if (lane < kFe) {
      // walk the 12 channel lengths of FE unit `lane`
      if (ok) {
        const uint32_t end = start + fl;
        uint32_t p = start;
        bool good = true;
        for (int k = 0; k < kChPerFe; k++) {
          const int c = lane * kChPerFe + k;
          uint32_t l = 0;
          if (good) {
            if (p + 2 > end) {
              good = false;
            } else {
              l = rd16(src + p);
              if (l < 3 || p + l > end) good = false;
            }
          }
          s.chan_pos[c] = good ? p : 0u;
          s.chan_len[c] = good ? (uint16_t)l : (uint16_t)0;
          if (good) p += l;
        }
        if (good && p != end) good = false;
        for (int k = 0; k < kChPerFe; k++) s.chan_st[lane * kChPerFe + k] = good ? 0 : (uint8_t)SST_CH_FRAMING;
      } else {
        for (int k = 0; k < kChPerFe; k++) {
          const int c = lane * kChPerFe + k;
          s.chan_pos[c] = 0;
          s.chan_len[c] = 0;
          s.chan_st[c] = fed_status;
        }
      }
    }
    __syncwarp();
    // run slots: a run takes at least 3 bytes, so (len - 3) / 3 slots per channel
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int c = lane * 3 + k;
      s.chan_slot[c] = s.chan_st[c] == 0 && s.chan_len[c] >= 3 ? (s.chan_len[c] - 3u) / 3u : 0u;
    }
    __syncwarp();
    const uint32_t slots = warp_scan96(s.chan_slot, lane);
    if (lane == 0) {
      s.scal[S_FEDOK] = ok ? 1u : 0u;
      s.scal[S_SLOTS] = slots <= (uint32_t)TILE ? 1u : 0u;
    }
  }
  __syncthreads();
  const bool use_slots = s.scal[S_SLOTS] != 0;

  // one thread per channel: validate every run, count digis, record run headers
  if (tid < kCh) {
    const int c = tid;
    uint32_t cnt = 0, nrun = 0;
    uint8_t st = s.chan_st[c];
    const uint32_t slot0 = s.chan_slot[c], slot1 = s.chan_slot[c + 1];
    if (st == 0 && s.chan_len[c] >= 3) {
      const uint32_t pos = s.chan_pos[c];
      const uint8_t* r = src + pos;
      const uint32_t len_c = s.chan_len[c];
      if (r[2] != SST_ZS_CODE) {
        st = SST_CH_BAD_CODE;
      } else {
        uint32_t p = 3, prev_end = 0;
        while (p < len_c) {
          if (p + 2 > len_c) { st = SST_CH_TRUNC; break; }
          const uint32_t first = r[p], w = r[p + 1];
          if (w == 0 || first + w > (uint32_t)kStrips) { st = SST_CH_RUN_RANGE; break; }
          if (first < prev_end) { st = SST_CH_RUN_ORDER; break; }
          if (p + 2 + w > len_c) { st = SST_CH_TRUNC; break; }
          if (use_slots && slot0 + nrun < slot1)
            s.runs[slot0 + nrun] = make_uint2(pos + p + 2, run_y(cnt, first, w, c));
          prev_end = first + w;
          cnt += w;
          nrun++;
          p += 2 + w;
        }
      }
      if (st) {
        cnt = 0;
        nrun = 0;
      }
      s.chan_st[c] = st;
    }
    if (use_slots)
      for (uint32_t k = slot0 + nrun; k < slot1; k++) s.runs[k] = make_uint2(0u, 0u);
    s.chan_cnt[c] = cnt;
  }
  __syncthreads();

  // exclusive prefix over the 96 channel counts, plus the status summary
  if (tid < 32) {
    uint32_t fl = 0, nb = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint8_t st = s.chan_st[lane * 3 + k];
      fl |= st;
      nb += st ? 1u : 0u;
    }
    const uint32_t total = warp_scan96(s.chan_cnt, lane);
    fl = __reduce_or_sync(0xffffffffu, fl);
    nb = __reduce_add_sync(0xffffffffu, nb);
    if (lane == 0) {
      s.scal[S_TOTAL] = total;
      s.scal[S_FLAGS] = fl;
      s.scal[S_NBAD] = nb;
    }
  }
  __syncthreads();
}

// Stages the FED record when it fits and parses it.  Returns true when the
// record was staged in shared memory.
template <int TILE>
__device__ bool parse_fed(Shm<TILE>& s, const uint8_t* gfed, uint32_t len, uint32_t fed_id, bool in_range) {
  const bool staged = in_range && len > 0 && len <= (uint32_t)Shm<TILE>::kRegion;
  if (staged) {
    stage_fed(gfed, len, s.fedbuf);
    __syncthreads();
    parse_body(s, s.fedbuf, len, fed_id, in_range);
  } else {
    parse_body(s, gfed, len, fed_id, in_range);
  }
  return staged;
}

// Copies all runs into the tile, one thread per run slot (single-chunk FEDs whose
// run slots fitted).
template <int TILE>
__device__ void emit_slots(Shm<TILE>& s, const uint8_t* src) {
  const uint32_t nslots = s.chan_slot[kCh];
  for (uint32_t k = threadIdx.x; k < nslots; k += blockDim.x) {
    const uint2 rr = s.runs[k];
    const uint32_t w = (rr.y >> 17) & 0xFFu;
    if (w == 0) continue;
    const uint32_t c = rr.y >> 25, first = (rr.y >> 9) & 0xFFu;
    const uint32_t o = s.chan_cnt[c] + (rr.y & 0x1FFu);
    const uint8_t* a = src + rr.x;
    for (uint32_t m = 0; m < w; m++) {
      s.t_key[o + m] = (uint16_t)((c << 8) | (first + m));
      s.t_adc[o + m] = a[m];
    }
  }
}

// Copies the runs of channels [c0, c1) into the tile: groups of `lanes` threads
// share a channel, all walk its run headers, each copies every lanes-th ADC byte.
// Records were validated by parse_body; the copy is still bounded by the counted
// digis so that it cannot leave the tile.
template <int TILE>
__device__ void emit_channels(Shm<TILE>& s, const uint8_t* src, int c0, int c1, int lanes) {
  const int gid = threadIdx.x / lanes, li = threadIdx.x % lanes, ng = blockDim.x / lanes;
  const uint32_t base = s.chan_cnt[c0];
  for (int c = c0 + gid; c < c1; c += ng) {
    const uint32_t o0 = s.chan_cnt[c] - base;
    const uint32_t n = s.chan_cnt[c + 1] - s.chan_cnt[c];
    if (n == 0) continue;
    const uint8_t* r = src + s.chan_pos[c];
    const uint32_t len_c = s.chan_len[c];
    uint32_t p = 3, o = 0;
    while (p + 2 <= len_c && o < n) {
      const uint32_t first = r[p];
      uint32_t w = r[p + 1];
      if (w > n - o) w = n - o;
      for (uint32_t k = li; k < w; k += lanes) {
        s.t_key[o0 + o + k] = (uint16_t)((c << 8) | ((first + k) & 255u));
        s.t_adc[o0 + o + k] = r[p + 2 + k];
      }
      o += w;
      p += 2 + w;
    }
  }
}

// ---------------------------------------------------------------- clustering (a3 - a6)

__device__ __forceinline__ bool bit(const uint32_t* m, int t) { return (m[t >> 5] >> (t & 31)) & 1u; }

#include "sst_fe.cuh"

// Greedy channel-aligned chunk [c0, c1) holding at most TILE digis.
template <int TILE>
__device__ int chunk_end(Shm<TILE>& s, int c0) {
  int c1 = c0 + 1;
  while (c1 < kCh && s.chan_cnt[c1 + 1] - s.chan_cnt[c0] <= (uint32_t)TILE) ++c1;
  return c1;
}

// ---------------------------------------------------------------- kernels

// Optional cluster amplitudes: the staging buffer and per-unit bookkeeping
// (context scratch) and the caller's output arrays; stage == nullptr: none.
struct AmpArgs {
  uint8_t* stage = nullptr;       // staged amplitudes, sliced per event like the output
  const uint64_t* off = nullptr;  // [n_events + 1] event slices (batch), or null (one event at 0)
  uint64_t cap = 0;               // bytes of staging and of output
  uint32_t* alloc = nullptr;      // allocation counter per event
  uint32_t* cnt = nullptr;        // per work item: amplitudes stored (0 when they did not fit)
  uint32_t* start = nullptr;      // per work item: offset in the event's staging slice, or kNoAmp
  uint32_t* dest = nullptr;       // per work item: offset in the event's output slice
  uint8_t* out = nullptr;         // caller's amp
  uint32_t* first = nullptr;      // caller's amp_first
};

// The event's slice [a, b) of the amplitude arrays.
__device__ __forceinline__ void amp_slice(const AmpArgs& am, uint32_t e, uint64_t* a, uint64_t* b) {
  uint64_t lo = am.off ? am.off[e] : 0, hi = am.off ? am.off[e + 1] : am.cap;
  if (hi > am.cap) hi = am.cap;
  if (lo > hi) lo = hi;
  *a = lo;
  *b = hi;
}

// a1, FED level: checks FED `fed`'s header (record at raw + fo, len bytes;
// fo == kBadOff when the record lies outside its event) and describes its 8 FE
// units for the batched kernel: d[v] = (byte offset of FE unit v in the record,
// its length | FED status << 16 | has data << 24).  A header is valid when the
// magic, FED id, channel and FE-unit counts and fed_bytes match and the padded FE
// lengths add up to the record length; otherwise every channel of the FED gets
// SST_CH_FED_HDR.  An absent FED (len 0) has no data and no error.
// Unit descriptor bit: the work item starting at this unit is too large to stage.
constexpr uint32_t kBigItem = 1u << 25;

__device__ uint32_t describe_fed(const uint8_t* __restrict__ raw, uint64_t fo, uint32_t len, uint32_t fed, uint2* d,
                                 uint32_t stage_max, uint32_t units) {
  uint32_t st = 0, data = 0;
  uint32_t fe_len[kFe], start[kFe];
#pragma unroll
  for (int v = 0; v < kFe; v++) fe_len[v] = start[v] = 0;
  if (fo == kBadOff) {
    st = SST_CH_FED_HDR;
  } else if (len > 0 && len < (uint32_t)kHdr) {
    st = SST_CH_FED_HDR;
  } else if (len > 0) {
    const uint8_t* g = raw + fo;
    uint32_t h[8];
    if ((fo & 15u) == 0) {
      const uint4 a = __ldg(reinterpret_cast<const uint4*>(g)), b = __ldg(reinterpret_cast<const uint4*>(g) + 1);
      h[0] = a.x; h[1] = a.y; h[2] = a.z; h[3] = a.w; h[4] = b.x; h[5] = b.y; h[6] = b.z; h[7] = b.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; i++) h[i] = rd32(g + 4 * i);
    }
    uint32_t body = 0;
#pragma unroll
    for (int v = 0; v < kFe; v++) {
      fe_len[v] = (h[4 + v / 2] >> (16 * (v & 1))) & 0xFFFFu;
      start[v] = kHdr + body;
      body += (fe_len[v] + 7u) & ~7u;
    }
    const uint32_t total = (kHdr + body + 15u) & ~15u;
    const bool ok = h[0] == SST_FED_MAGIC && (h[1] & 0xFFFFu) == fed && ((h[1] >> 16) & 0xFFu) == (uint32_t)kCh &&
                    (h[1] >> 24) == (uint32_t)kFe && h[2] == len && total == len;
    if (ok) data = 1;
    else st = SST_CH_FED_HDR;
  }
#pragma unroll
  for (int v = 0; v < kFe; v++)
    d[v] = make_uint2(data ? start[v] : 0u, (data ? fe_len[v] : 0u) | (st << 16) | (data << 24));
  // work items of `units` FE units whose bytes (first unit to the end of the last)
  // exceed the batched kernel's staging buffer: bit p of the result for item p,
  // and kBigItem in the descriptor of the item's first unit
  uint32_t big = 0;
  if (data)
    for (uint32_t v = 0; v + units <= (uint32_t)kFe; v += units)
      if (start[v + units - 1] - start[v] + fe_len[v + units - 1] > stage_max) {
        big |= 1u << (v / units);
        d[v].y |= kBigItem;
      }
  return big;
}

// a1, outer level: byte offset of every FED record (exclusive scan of fed_len per
// event, plus the event's start).  A record that would end past its event is
// marked kBadOff; a size mismatch sets SST_EV_SIZE.  `cpe` CTAs per event, CTA c
// taking the event's FEDs [c * blockDim.x, (c + 1) * blockDim.x) and summing the
// lengths of the FEDs before them itself.  With unit_desc (batched path) every
// FED's header is checked and its FE units described (describe_fed).  It is also
// the launch sequence's prologue: the event's last CTA writes its status (zero but
// SST_EV_SIZE), its first clears the staging counters (ev_alloc, amp_alloc, when
// given), the very first clears the work tickets, and every event's n_lb
// look-back states (lb[e * n_lb ..]) are cleared.  Event e's bytes are
// [event_off[e], event_end[e]) when event_end is given (events that do not follow
// one another, e.g. read in place from host memory), else [event_off[e],
// event_off[e + 1]).  With big_list, the work items of `units` FE units too large
// for the batched kernel's staging buffer (stage_max bytes) are appended to it by
// their ticket-order index (FED, then event, then item), counted in tickets[2],
// which the launch clears before this kernel (so it is not cleared here).
__global__ void k_fed_scan(const uint64_t* __restrict__ event_off, uint64_t raw_bytes,
                           const uint32_t* __restrict__ fed_len, uint32_t n_feds, uint32_t cpe,
                           uint64_t* __restrict__ fed_off, sst_event_status* status, uint32_t* ev_alloc,
                           uint32_t* tickets, unsigned long long* lb, uint32_t n_lb, const uint8_t* __restrict__ raw,
                           uint2* unit_desc, uint32_t* amp_alloc, uint32_t* big_list, uint32_t stage_max,
                           uint32_t units, const uint64_t* __restrict__ event_end) {
  __shared__ uint32_t wsum[32];
  __shared__ unsigned long long psum[32];
  pdl_release();
  const uint32_t e = blockIdx.x / cpe, c = blockIdx.x % cpe;
  const uint32_t f0 = c * blockDim.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t ev0 = event_off ? event_off[e] : 0;
  const uint64_t ev1 = event_end ? event_end[e] : event_off ? event_off[e + 1] : raw_bytes;
  if (c == 0 && threadIdx.x == 0) {
    if (ev_alloc) ev_alloc[e] = 0;
    if (amp_alloc) amp_alloc[e] = 0;
  }
  if (e == 0 && c == 0 && threadIdx.x < 16 && threadIdx.x != 2) tickets[threadIdx.x] = 0;
  if (lb)
    for (uint32_t i = f0 + threadIdx.x; i < n_lb; i += cpe * blockDim.x) lb[(size_t)e * n_lb + i] = 0;
  const uint32_t* len_e = fed_len + (size_t)e * n_feds;
  // bytes of the event's FEDs before this CTA's
  unsigned long long part = 0;
  for (uint32_t i = threadIdx.x; i < f0 && i < n_feds; i += blockDim.x) part += len_e[i];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) part += __shfl_down_sync(0xffffffffu, part, d);
  if (lane == 0) psum[warp] = part;
  __syncthreads();
  uint64_t pre = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) pre += psum[k];
  const uint32_t f = f0 + threadIdx.x;
  const uint32_t len = f < n_feds ? len_e[f] : 0u;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(len, wsum, &tot);
  if (f < n_feds) {
    const uint64_t o = ev0 + pre + ex;
    const uint64_t fo = (ev1 >= ev0 && o + len <= ev1) ? o : kBadOff;
    fed_off[(size_t)e * n_feds + f] = fo;
    if (unit_desc) {
      const uint32_t big = describe_fed(raw, fo, len, f, unit_desc + ((size_t)e * n_feds + f) * kFe, stage_max, units);
      if (big && big_list) {
        const uint32_t items = kFe / units, n_events = gridDim.x / cpe;
        uint32_t at = atomicAdd(&tickets[2], (uint32_t)__popc(big));
        for (uint32_t b = big; b; b &= b - 1)
          big_list[at++] = (f * n_events + e) * items + (uint32_t)(__ffs(b) - 1);
      }
    }
  }
  if (c == cpe - 1 && threadIdx.x == 0)
    status[e] = sst_event_status{0u, 0u, ev0 + pre + tot != ev1 ? SST_EV_SIZE : 0u, 0u};
}

// a6, ordering: per event, the exclusive scan of its work items' cluster counts
// gives every item's position in the event's sorted cluster SoA; the event's
// total is its cluster count.  One CTA of 1024 threads per event (1,760 items of a
// full event in two block scans).  With pack_off (events packed back to back),
// the CTA that finishes last (counted in *done, which the prologue cleared; no
// CTA waits for another) also scans the events' counts: pack_off[e] = clusters
// of the events before e, pack_off[n_events] = all clusters.
__global__ void __launch_bounds__(1024) k_clu_scan(const uint32_t* __restrict__ fed_cnt, uint32_t n_feds,
                                                   uint32_t* __restrict__ fed_dest, sst_event_status* status,
                                                   uint64_t* pack_off, uint32_t* done, AmpArgs am) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry_s, acarry_s;
  __shared__ uint64_t pcarry_s;
  __shared__ bool last_s;
  const uint32_t e = blockIdx.x;
  if (threadIdx.x == 0) carry_s = acarry_s = 0;
  __syncthreads();
  for (uint32_t b = 0; b < n_feds; b += blockDim.x) {
    const uint32_t f = b + threadIdx.x;
    const uint32_t n = f < n_feds ? fed_cnt[(size_t)e * n_feds + f] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(n, wsum, &tot);
    const uint32_t carry = carry_s;
    if (f < n_feds) fed_dest[(size_t)e * n_feds + f] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
    if (am.stage) {  // the units' amplitude counts, the same way
      const uint32_t na = f < n_feds ? am.cnt[(size_t)e * n_feds + f] : 0u;
      uint32_t atot;
      const uint32_t aex = block_excl_scan(na, wsum, &atot);
      const uint32_t acarry = acarry_s;
      if (f < n_feds) am.dest[(size_t)e * n_feds + f] = acarry + aex;
      __syncthreads();
      if (threadIdx.x == 0) acarry_s = acarry + atot;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) status[e].n_clusters = carry_s;
  if (!pack_off) return;
  if (threadIdx.x == 0) {
    __threadfence();  // this event's count is visible before it is counted as done
    last_s = atomicAdd(done, 1u) == gridDim.x - 1;
    pcarry_s = 0;
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  const uint32_t n_events = gridDim.x;
  for (uint32_t b = 0; b < n_events; b += blockDim.x) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t n = i < n_events ? __ldcg(&status[i].n_clusters) : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(n, wsum, &tot);
    const uint64_t carry = pcarry_s;
    if (i < n_events) pack_off[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) pcarry_s = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pack_off[n_events] = pcarry_s;
    *done = 0;
  }
}

// a6, output with amplitudes: copies every segment's staged clusters (one segment
// per work item) to its place in the event's sorted cluster SoA, one warp per
// segment (16-byte loads, coalesced stores), k_clu_scan having scanned the
// segments' cluster and amplitude counts.  The event's clusters start at
// clu_off[e] (its slice), or at pack_off[e] when pack_off is given (events packed
// back to back).  Each cluster's amp_first is the segment's output offset plus the
// widths of the segment's clusters before it, and the segment's amplitude bytes
// are copied after its clusters.
__global__ void __launch_bounds__(256) k_compact(const uint4* __restrict__ stage, const uint64_t* __restrict__ clu_off,
                                                 const uint64_t* __restrict__ pack_off,
                                                 const uint32_t* __restrict__ seg_cnt,
                                                 const uint32_t* __restrict__ seg_start,
                                                 const uint32_t* __restrict__ seg_dest, uint32_t n_events,
                                                 uint32_t n_segs, sst_clusters out, AmpArgs am) {
  const uint64_t items = (uint64_t)n_events * n_segs;
  const uint64_t it = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (it >= items) return;
  const uint32_t n = seg_cnt[it];
  if (n == 0) return;
  const int lane = threadIdx.x & 31;
  const uint32_t e = (uint32_t)(it / n_segs);
  const uint64_t off = clu_off ? clu_off[e] : 0;
  const uint4* src = stage + off + seg_start[it];
  const uint64_t dst = (pack_off ? pack_off[e] : off) + seg_dest[it];
  uint64_t a0 = 0, a1 = 0;
  amp_slice(am, e, &a0, &a1);
  const bool amps = am.start[it] != kNoAmp;
  uint64_t acarry = a0 + am.dest[it];
  for (uint32_t k0 = 0; k0 < n; k0 += 32) {
    const uint32_t k = k0 + lane;
    uint4 r = make_uint4(0u, 0u, 0u, 0u);
    if (k < n) {
      r = __ldg(src + k);
      const uint64_t o = dst + k;
      out.det[o] = r.x;
      out.first[o] = (uint16_t)(r.y & 0xFFFFu);
      out.width[o] = (uint16_t)(r.y >> 16);
      out.charge[o] = r.z;
      out.barycenter[o] = __uint_as_float(r.w);
    }
    {
      const uint32_t x = k < n ? (r.y >> 16) : 0u;
      uint32_t incl = x;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      if (k < n) am.first[dst + k] = amps ? (uint32_t)(acarry + incl - x) : kNoAmp;
      acarry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (amps) {
    const uint32_t na = am.cnt[it];
    const uint8_t* as = am.stage + a0 + am.start[it];
    uint8_t* ad = am.out + a0 + am.dest[it];
    for (uint32_t i = lane; i < na; i += 32) ad[i] = as[i];
  }
}

// a6, output without amplitudes: orders and copies the staged clusters in one
// pass.  CTA c of event e takes the event's segments [c * SEGS, (c + 1) * SEGS):
// it sums the counts of the event's segments before them (its place in the
// event), scans its own counts in shared memory, and copies its clusters to one
// contiguous range of the output, thread t taking output records t, t + 256, ...
// (four loads in flight per thread) and finding each one's segment by binary
// search over the scanned counts (coalesced stores; each segment's staged records
// are contiguous).  The event's
// clusters start at clu_off[e] (its slice; 0 without clu_off), or at pack_off[e]
// when pack_off is given (k_clu_scan computed it and the events' counts); the
// event's last CTA otherwise stores its cluster count.
template <int SEGS>
__global__ void __launch_bounds__(256) k_order(const uint4* __restrict__ stage, const uint64_t* __restrict__ clu_off,
                                               const uint64_t* __restrict__ pack_off,
                                               const uint32_t* __restrict__ seg_cnt,
                                               const uint32_t* __restrict__ seg_start, uint32_t n_segs, uint32_t cpe,
                                               sst_clusters out, sst_event_status* status) {
  static_assert(SEGS <= 256 && (SEGS & (SEGS - 1)) == 0, "one scan entry per thread, binary search");
  __shared__ uint32_t s_dest[SEGS + 1], s_start[SEGS];
  __shared__ uint32_t wsum[32];
  pdl_wait();  // the staged clusters and counts
  const uint32_t e = blockIdx.x / cpe, c = blockIdx.x % cpe;
  const uint32_t seg0 = c * SEGS;
  const uint32_t nseg = n_segs - seg0 < (uint32_t)SEGS ? n_segs - seg0 : (uint32_t)SEGS;
  const uint32_t* cnt_e = seg_cnt + (size_t)e * n_segs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // clusters of the event's segments before this CTA's
  uint32_t part = 0;
  for (uint32_t i = tid; i < seg0; i += blockDim.x) part += __ldg(cnt_e + i);
  part = __reduce_add_sync(0xffffffffu, part);
  if (lane == 0) wsum[warp] = part;
  __syncthreads();
  uint32_t pre = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) pre += wsum[k];
  __syncthreads();
  // this CTA's segments: exclusive scan of their counts
  const uint32_t v = tid < (int)nseg ? __ldg(cnt_e + seg0 + tid) : 0u;
  if (tid < SEGS) s_start[tid] = tid < (int)nseg ? __ldg(seg_start + (size_t)e * n_segs + seg0 + tid) : 0u;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(v, wsum, &tot);
  if (tid < SEGS) s_dest[tid] = ex;
  if (tid == 0) s_dest[SEGS] = tot;
  __syncthreads();
  const uint64_t off = clu_off ? clu_off[e] : 0;
  const uint4* src = stage + off;
  const uint64_t dst = (pack_off ? pack_off[e] : off) + pre;
  constexpr int kU = 4;  // records per thread in flight
  for (uint32_t d0 = tid; d0 < tot; d0 += kU * blockDim.x) {
    uint4 r[kU];
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const uint32_t d = d0 + u * blockDim.x;
      if (d < tot) {
        int lo = 0;  // the last segment starting at or before d: it holds d
#pragma unroll
        for (int step = SEGS / 2; step > 0; step >>= 1)
          if (s_dest[lo + step] <= d) lo += step;
        r[u] = __ldg(src + s_start[lo] + (d - s_dest[lo]));
      }
    }
#pragma unroll
    for (int u = 0; u < kU; u++) {
      const uint32_t d = d0 + u * blockDim.x;
      if (d < tot) {
        const uint64_t o = dst + d;
        out.det[o] = r[u].x;
        out.first[o] = (uint16_t)(r[u].y & 0xFFFFu);
        out.width[o] = (uint16_t)(r[u].y >> 16);
        out.charge[o] = r[u].z;
        out.barycenter[o] = __uint_as_float(r[u].w);
      }
    }
  }
  if (!pack_off && c == cpe - 1 && tid == 0) status[e].n_clusters = pre + tot;
}

// a1 + a2 per event: one CTA per FED (ticket order), digis written to the global
// digi SoA at the FED's offset from the look-back over FED digi counts.
template <int TILE>
__global__ void __launch_bounds__(256, 4) k_unpack(const uint8_t* __restrict__ raw,
                                                const uint32_t* __restrict__ fed_len,
                                                const uint64_t* __restrict__ fed_off, uint32_t n_feds,
                                                sst_digis out, unsigned long long* lb, uint32_t* ticket, int lanes,
                                                uint32_t spin_limit, int32_t withhold) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shm<TILE>& s = *reinterpret_cast<Shm<TILE>*>(smem_raw);
  const int tid = threadIdx.x;
  if (tid == 0) s.scal[S_TICKET] = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t f = s.scal[S_TICKET];
  if (f >= n_feds) return;
  const uint64_t fo = fed_off[f];
  const bool in_range = fo != kBadOff;
  const uint32_t len = in_range ? fed_len[f] : 0u;
  const uint8_t* gfed = in_range ? raw + fo : raw;
  const bool staged = parse_fed(s, gfed, len, f, in_range);
  const uint32_t total = s.scal[S_TOTAL];
  if (tid < 32) {
    bool to = false;
    uint32_t excl = 0;
    const bool publish = (int64_t)f != (int64_t)withhold;  // a FED withheld by the failure tests never publishes
    if (f > 0) {
      if (tid == 0 && publish) st_release(lb + f, kLbAgg | total);
      excl = lookback_warp(lb, f, 0, spin_limit, &to);
    }
    if (tid == 0) {
      if (publish) st_release(lb + f, kLbPre | (excl + total));
      s.scal[S_BASE] = excl;
      uint32_t fl = s.scal[S_FLAGS];
      if (to) fl |= SST_EV_TIMEOUT;
      if ((uint64_t)excl + total > out.capacity) fl |= SST_EV_DIGI_CAPACITY;
      if (fl) atomicOr(&out.status->flags, fl);
      if (s.scal[S_NBAD]) atomicAdd(&out.status->n_bad_channels, s.scal[S_NBAD]);
      const uint64_t end = (uint64_t)excl + total;
      const uint32_t written =
          end <= out.capacity ? total : ((uint64_t)excl < out.capacity ? (uint32_t)(out.capacity - excl) : 0u);
      if (written) atomicAdd(&out.status->n_digi, written);
    }
  }
  __syncthreads();
  const uint32_t base = s.scal[S_BASE];
  const uint64_t cap = out.capacity;
  for (int c = tid; c <= kCh; c += blockDim.x) {
    if (c == kCh && f != n_feds - 1) continue;
    const uint64_t v = (uint64_t)base + s.chan_cnt[c];
    out.chan_off[(size_t)f * kCh + c] = (uint32_t)(v < cap ? v : cap);
    if (c < kCh) out.chan_status[(size_t)f * kCh + c] = s.chan_st[c];
  }
  // digis, one tile-sized chunk at a time, copied out with coalesced stores
  const bool slots = total <= (uint32_t)TILE && s.scal[S_SLOTS] != 0;
  int c0 = 0;
  while (c0 < kCh) {
    const int c1 = slots ? kCh : chunk_end(s, c0);
    const int n = (int)(s.chan_cnt[c1] - s.chan_cnt[c0]);
    if (n > 0) {
      if (slots) {
        if (staged) emit_slots(s, s.fedbuf); else emit_slots(s, gfed);
      } else {
        if (staged) emit_channels(s, s.fedbuf, c0, c1, lanes); else emit_channels(s, gfed, c0, c1, lanes);
      }
      __syncthreads();
      const uint64_t o = (uint64_t)base + s.chan_cnt[c0];
      for (int i = tid; i < n; i += blockDim.x) {
        const uint64_t pos = o + i;
        if (pos < cap) {
          out.strip[pos] = f * (uint32_t)kFedStrips + s.t_key[i];
          out.adc[pos] = s.t_adc[i];
        }
      }
      __syncthreads();
    }
    c0 = c1;
  }
}

// a3 - a6 per event: one warp per FE unit over the global digi SoA (a single
// event has too few pairs of units to fill the GPU); clusters staged per unit.
template <bool AMP>
__global__ void __launch_bounds__(256, 4) k_cluster(sst_digis in, uint32_t n_feds, KParams kp, uint4* stage,
                                                    uint64_t cap, uint32_t* ev_alloc, uint32_t* seg_cnt,
                                                    uint32_t* seg_start, AmpArgs am) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  fe::Warp& w = reinterpret_cast<fe::Warp*>(smem_raw)[warp];
  const uint32_t unit = blockIdx.x * nw + warp;  // work item: one FE unit (12 channels)
  if (unit >= n_feds * kFe) return;
  const uint32_t ch0 = unit * kChPerFe;
  fe::load_calib<kChPerFe>(w, kp, ch0);
  // channel digi ranges from the CSR row pointers, clamped to the input capacity
  // and to 256 digis per channel, so that malformed input cannot leave the tile
  uint32_t cnt = 0;
  if (lane < kChPerFe) {
    uint64_t a = in.chan_off[ch0 + lane], b = in.chan_off[ch0 + lane + 1];
    if (a > in.capacity) a = in.capacity;
    if (b > in.capacity) b = in.capacity;
    const uint32_t n = b > a ? (uint32_t)(b - a) : 0u;
    cnt = n < (uint32_t)kStrips ? n : (uint32_t)kStrips;
    w.chan_pos[lane] = (uint32_t)a;
  }
  uint32_t x = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane < kChPerFe) w.chan_cnt[lane] = x - cnt;
  const uint32_t total = __shfl_sync(0xffffffffu, x, kChPerFe - 1);
  if (lane == 0) w.chan_cnt[kChPerFe] = total;
  __syncwarp();
  const uint32_t g0 = ch0 * (uint32_t)kStrips;
  auto fill = [&](int c0, int c1, bool) {
    for (int c = c0; c < c1; c++) {
      const uint32_t o = w.chan_cnt[c] - w.chan_cnt[c0];
      const uint32_t n = w.chan_cnt[c + 1] - w.chan_cnt[c];
      const size_t a = w.chan_pos[c];
      for (uint32_t k = lane; k < n; k += 32) {
        const uint32_t key = in.strip[a + k] - g0;
        // a digi that does not belong to channel c takes no part in clustering (ADC 0:
        // never active, never a seed)
        w.kf[o + k] = (key >> 8) == (uint32_t)c ? key | ((uint32_t)in.adc[a + k] << 16) : 0u;
      }
    }
    __syncwarp();
  };
  fe::SegOut so{stage, cap, ev_alloc, seg_cnt + unit, seg_start + unit};
  if (AMP) {
    so.amp = am.stage;
    so.amp_cap = am.cap;
    so.amp_alloc = am.alloc;
    so.seg_amp_cnt = am.cnt + unit;
    so.seg_amp_start = am.start + unit;
  }
  const uint2* calq = kp.calq + g0;
  auto scan = [&](int nn, bool) { return fe::scan_unit<kChPerFe, false>(w, kp, calq, nullptr, 0u, nn); };
  fe::cluster_unit<kChPerFe, AMP>(w, kp, ch0, total, fill, scan, so, in.status);
}

// The work-item loop of k_batch.  SPLIT: a staged item's code reads its bytes
// from the staging buffer as shared memory (a second inlined copy of the item
// code); otherwise every item reads them through a generic pointer (one copy).
// LIST: the prologue listed items too large to stage (n_big of them).
template <bool AMP, int U, bool SPLIT, bool LIST>
__device__ __forceinline__ void batch_items(fe::WarpT<U>& w, const uint8_t* __restrict__ raw,
                                            const uint64_t* __restrict__ fed_off, uint32_t n_events,
                                            uint32_t n_feds, const uint64_t* __restrict__ clu_off, uint64_t out_cap,
                                            sst_event_status* status, const KParams& kp, uint4* stage,
                                            uint32_t* ev_alloc, uint32_t* seg_cnt, uint32_t* seg_start,
                                            uint32_t* ticket, const uint2* __restrict__ unit_desc, const AmpArgs& am,
                                            uint32_t n_big) {
  const int lane = threadIdx.x & 31;
  using W = fe::WarpT<U>;
  constexpr uint32_t kItems = kFe / U;  // work items per FED
  const uint32_t per_fed = n_events * kItems;
  const uint32_t n_units = n_feds * per_fed;
  // Tickets: first the items too large to stage (the prologue's list; they take
  // several times longer than the others), then every item in ticket order (FED,
  // event, item), the listed ones skipped, so that the launch ends on small items.
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n_big + n_units) break;
    const bool listed = LIST && t < n_big;
    if (LIST) {
      if (listed) t = kp.big_list[t];
      else t -= n_big;
    }
    const uint32_t f = t / per_fed, r = t % per_fed, e = r / kItems, p = r % kItems, u = p * U;
    const size_t item = (size_t)e * n_feds + f;
    const uint2 dA = unit_desc[item * kFe + u];
    if (LIST && !listed && (dA.y & kBigItem)) continue;  // taken from the list
    const uint64_t fo = fed_off[item];
    const bool in_range = fo != kBadOff;
    const uint32_t ch0 = f * kCh + u * kChPerFe;
    fe::load_calib<W::kChW>(w, kp, ch0);
    const fe::Unit un = fe::locate(w, raw + (in_range ? fo : 0), dA, unit_desc[item * kFe + u + (U - 1)], f, u);
    // the rest of the item; src is the staging buffer for a staged item, so that
    // its bytes are read as shared memory there (two inlined copies)
    auto body = [&](const uint8_t* src) {
      uint32_t flags, nbad;
      const uint32_t total = fe::parse_unit(w, un, src, &flags, &nbad);
      if (lane == 0) {
        if (flags) atomicOr(&status[e].flags, flags);
        if (nbad) atomicAdd(&status[e].n_bad_channels, nbad);
        if (total) atomicAdd(&status[e].n_digi, total);
      }
      const uint64_t off = clu_off[e];
      const uint64_t end = clu_off[e + 1] < out_cap ? clu_off[e + 1] : out_cap;
      const uint64_t cap = end > off ? end - off : 0;
      fe::SegOut so{stage + (off < out_cap ? off : 0), cap, ev_alloc + e, seg_cnt + item * kItems + p,
                    seg_start + item * kItems + p};
      if (AMP) {
        uint64_t a0, a1;
        amp_slice(am, e, &a0, &a1);
        so.amp = am.stage + a0;
        so.amp_cap = a1 - a0;
        so.amp_alloc = am.alloc + e;
        so.seg_amp_cnt = am.cnt + item * kItems + p;
        so.seg_amp_start = am.start + item * kItems + p;
      }
      const bool slots = fe::use_slots<W>(un);
      auto fill = [&](int c0, int c1, bool single) {
        if (single && slots) fe::mark_slots(w, un, (int)total);
        else fe::mark_walk(w, src, c0, c1);
      };
      const uint2* calq = kp.calq + (size_t)ch0 * kStrips;
      const uint32_t src_end = un.off1 + un.len1;
      auto scan = [&](int nn, bool) { return fe::scan_unit<W::kChW, true>(w, kp, calq, src, src_end, nn); };
      fe::cluster_unit<W::kChW, AMP>(w, kp, ch0, total, fill, scan, so, &status[e]);
    };
    if (SPLIT && un.staged) body(w.fe);
    else body(un.src);
    __syncwarp();
  }
}

// a7: every FE unit of every FED of every event of a batch, unpacked and
// clustered on chip, one warp per work item of U adjacent FE units (U = 1 or 2).
// Persistent warps take tickets FED-major (FED, then event, then item), so that
// the warps working at any moment share the same FED's calibration in L2.
template <bool AMP, int U>
__global__ void __launch_bounds__(256, 4) k_batch(const uint8_t* __restrict__ raw,
                                                  const uint32_t* __restrict__ fed_len,
                                                  const uint64_t* __restrict__ fed_off, uint32_t n_events,
                                                  uint32_t n_feds, const uint64_t* __restrict__ clu_off,
                                                  uint64_t out_cap, sst_event_status* status, KParams kp,
                                                  uint4* stage, uint32_t* ev_alloc, uint32_t* seg_cnt,
                                                  uint32_t* seg_start, uint32_t* ticket,
                                                  const uint2* __restrict__ unit_desc, AmpArgs am) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  fe::WarpT<U>& w = reinterpret_cast<fe::WarpT<U>*>(smem_raw)[warp];
  pdl_wait();  // the prologue's tickets, offsets, unit descriptors and counts
  // Items whose bytes exceed the staging buffer (the prologue lists them) are read
  // in place from global memory, by a second inlined copy of the item code.  When
  // such items are common (more than 1 in 32, as in batches whose FED payloads
  // differ many times over) both copies would be hot at once and compete for the
  // instruction cache: every item then takes the in-place copy, with its staged
  // bytes read through a generic pointer.
  const uint32_t n_big = kp.big_list ? ticket[2] : 0u;
  const bool mixed = (uint64_t)n_big * 32u > (uint64_t)n_feds * n_events * (kFe / U);
  if (mixed)
    batch_items<AMP, U, false, true>(w, raw, fed_off, n_events, n_feds, clu_off, out_cap, status, kp, stage,
                                     ev_alloc, seg_cnt, seg_start, ticket, unit_desc, am, n_big);
  else if (n_big)
    batch_items<AMP, U, true, true>(w, raw, fed_off, n_events, n_feds, clu_off, out_cap, status, kp, stage, ev_alloc,
                                    seg_cnt, seg_start, ticket, unit_desc, am, n_big);
  else
    batch_items<AMP, U, true, false>(w, raw, fed_off, n_events, n_feds, clu_off, out_cap, status, kp, stage,
                                     ev_alloc, seg_cnt, seg_start, ticket, unit_desc, am, 0u);
  pdl_release();
}

// Host batches with amplitudes: the chunk's amp_first values index the chunk's
// amplitude arena; adding the chunk's first byte in the caller's array makes them
// absolute.  The first *count records are rebased (kNoAmp stays).
__global__ void k_rebase_amp(uint32_t* __restrict__ amp_first, const uint64_t* __restrict__ count, uint32_t base) {
  const uint64_t n = *count;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t a = amp_first[i];
    if (a != kNoAmp) amp_first[i] = a + base;
  }
}

__global__ void k_badmask(const uint8_t* __restrict__ bad, uint32_t* __restrict__ mask, uint64_t n_words) {
  const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_words) return;
  uint32_t m = 0;
  for (int b = 0; b < 32; b++) m |= (bad[w * 32 + b] != 0 ? 1u : 0u) << b;
  mask[w] = m;
}

// The per-strip calibration word the clusterizers read, built once per upload:
//   bits 0-7   thr_ch:   channel limit, the largest ADC that is NOT active;
//   bits 8-15  thr_seed: seed limit, the largest ADC that is NOT a seed;
//   bits 16-23 gap:      the longest linking gap below the strip;
// stored beside noise^2 of the strip (binary32, rounded once; summed by the
// cluster threshold), so that the scan gathers both with one 8-byte load.
//
// Limits (section 2: a strip is active / a seed when its ADC is larger than the
// channel / seed threshold times its noise): with P = T x noise rounded once in
// binary32 (P >= 0), an integer ADC satisfies (float)adc > P exactly when adc >
// floor(P), since every ADC is exactly representable; so the limit is floor(P),
// capped at 255 (no 8-bit ADC exceeds it).  A bad strip is never active nor a
// seed: both limits are 255.
//
// Linking gap (a candidate continues over at most max_seq_holes consecutive
// inactive good strips and at most max_seq_bad consecutive bad strips): G(t) is
// the largest g such that, among strips t-g .. t-1 of the channel, every maximal
// run of bad strips is at most max_bad long and every maximal run of good strips
// at most max_holes long.  The strips between successive active strips a < t are
// all inactive, so they are linked exactly when their gap t-a-1 is at most G(t): a
// gap that is valid stays valid when shortened from below, and one longer than
// G(t) contains the strip t-G(t)-1 that breaks a limit.  One thread per strip walks
// down from t-1.  The byte stored is min(G(t) + 1, t) <= 255 (G(t) <= t), the limit
// the clusterizers compare tile keys against (see the comment below).
__global__ void k_calib_pack(const float* __restrict__ noise, const uint32_t* __restrict__ mask,
                             uint2* __restrict__ calq, uint64_t n_strips, float t_ch,
                             float t_seed, int max_holes, int max_bad) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_strips) return;
  const int t = (int)(s % kStrips);
  const uint32_t* m = mask + (s - (uint64_t)t) / 32;  // the channel's 8 mask words
  int g = 0, run = 0, prev = -1;
  for (int u = t - 1; u >= 0; --u) {
    const int b = (int)((m[u >> 5] >> (u & 31)) & 1u);
    run = b == prev ? run + 1 : 1;
    prev = b;
    if (run > (b ? max_bad : max_holes)) break;
    ++g;
  }
  const bool bad = (m[t >> 5] >> (t & 31)) & 1u;
  const float nz = noise[s];
  auto limit = [&](float thr) -> uint32_t {
    const float p = __fmul_rn(thr, nz);
    return p >= 255.f ? 255u : (uint32_t)p;  // truncation = floor for p >= 0
  };
  // linking limit of the tile key difference: strip t is linked to the previous
  // active strip a of its channel when t - a <= g + 1 (<= t always holds); an active
  // strip of an earlier channel is at least t + 1 keys below, so with
  // lim = min(g + 1, t) one unsigned compare, key - prev - 1 >= lim, marks a new
  // candidate in both cases
  const uint32_t gap = (uint32_t)(g + 1 < t ? g + 1 : t);
  const uint32_t word = bad ? (255u | (255u << 8) | (gap << 16)) : (limit(t_ch) | (limit(t_seed) << 8) | (gap << 16));
  calq[s] = make_uint2(word, __float_as_uint(__fmul_rn(nz, nz)));
}

// ---------------------------------------------------------------- launch helpers

// Raises a kernel's dynamic shared memory limit to what a launch needs and
// returns its CTAs per SM.  The limit only grows (per device and kernel), and the
// occupancy is looked up once per device, kernel, block size and shared memory
// size, so that repeated launches make no driver calls for either.
struct Prep {
  int dev;
  const void* fn;
  int block;
  size_t smem;
  int per_sm;
};
struct Limit {
  int dev;
  const void* fn;
  size_t smem;
};
std::mutex g_prep_mu;
std::vector<Prep> g_prep;
std::vector<Limit> g_limit;

cudaError_t prepare(const void* fn, int block, size_t smem, int* per_sm) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  std::lock_guard<std::mutex> lock(g_prep_mu);
  Limit* lim = nullptr;
  for (Limit& l : g_limit)
    if (l.dev == dev && l.fn == fn) lim = &l;
  if (!lim) {
    g_limit.push_back(Limit{dev, fn, 0});
    lim = &g_limit.back();
  }
  if (smem > lim->smem) {
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) return e;
    lim->smem = smem;
  }
  for (const Prep& p : g_prep)
    if (p.dev == dev && p.fn == fn && p.block == block && p.smem == smem) {
      *per_sm = p.per_sm;
      return cudaSuccess;
    }
  int n = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem))) return e;
  g_prep.push_back(Prep{dev, fn, block, smem, n});
  *per_sm = n;
  return cudaSuccess;
}

template <int TILE>
cudaError_t launch_unpack_t(const uint8_t* raw, const uint32_t* fed_len, uint32_t n_feds, const sst_digis& out,
                            const Scratch& s, const Shape& sh, cudaStream_t st) {
  const size_t sm = sizeof(Shm<TILE>);
  int per_sm = 0;
  cudaError_t e = prepare((const void*)k_unpack<TILE>, sh.block, sm, &per_sm);
  if (e) return e;
  k_unpack<TILE><<<n_feds, sh.block, sm, st>>>(raw, fed_len, s.fed_off, n_feds, out, s.lb, s.tickets, sh.lanes,
                                                s.lb_spin_limit ? s.lb_spin_limit : kLbSpinLimit, s.lb_withhold);
  return cudaGetLastError();
}

// The kernels' parameters with the stream's spill areas.
KParams with_spill(const KParams& kp, const Scratch& s) {
  KParams k = kp;
  k.spill = s.spill;
  k.spill_warps = (uint32_t)s.spill_warps;
  return k;
}

// The amplitude arguments of a launch: none unless the caller asked for them.
AmpArgs amp_args(const sst_clusters& out, const Scratch& s) {
  AmpArgs a;
  if (!out.amp) return a;
  a.stage = s.amp_stage;
  a.off = out.amp_off;
  a.cap = out.amp_capacity;
  a.alloc = s.amp_alloc;
  a.cnt = s.seg_amp_cnt;
  a.start = s.seg_amp_start;
  a.dest = s.seg_amp_dest;
  a.out = out.amp;
  a.first = out.amp_first;
  return a;
}

// Launches `k` with programmatic stream serialization: it may start while the
// kernel before it on the stream drains, and waits for it with pdl_wait().
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

cudaError_t launch_cluster_fe(const sst_digis& in, uint32_t n_feds, const KParams& kp, const Scratch& s,
                              uint64_t cap, const Shape& sh, const AmpArgs& am, cudaStream_t st) {
  const int nw = sh.block / 32;
  const size_t sm = sizeof(fe::Warp) * nw;
  int per_sm = 0;
  const void* fn = am.stage ? (const void*)k_cluster<true> : (const void*)k_cluster<false>;
  cudaError_t e = prepare(fn, sh.block, sm, &per_sm);
  if (e) return e;
  const uint32_t units = n_feds * kFe;
  const KParams kps = with_spill(kp, s);
  if (am.stage)
    k_cluster<true><<<(units + nw - 1) / nw, sh.block, sm, st>>>(in, n_feds, kps, s.stage, cap, s.ev_alloc, s.fed_cnt,
                                                               s.fed_start, am);
  else
    k_cluster<false><<<(units + nw - 1) / nw, sh.block, sm, st>>>(in, n_feds, kps, s.stage, cap, s.ev_alloc,
                                                                s.fed_cnt, s.fed_start, am);
  return cudaGetLastError();
}

template <bool AMP, int U>
cudaError_t launch_batch_t(const uint8_t* raw, const uint32_t* fed_len, uint32_t n_events, uint32_t n_feds,
                           const uint64_t* clu_off, uint64_t out_cap, sst_event_status* status, const KParams& kp,
                           const Scratch& s, const Shape& sh, int n_sm, const AmpArgs& am, cudaStream_t st) {
  const int nw = sh.block / 32;
  const size_t sm = batch_smem(U, sh.block);
  const size_t units = (size_t)n_events * n_feds * (kFe / U);
  int per_sm = 0;
  cudaError_t e = prepare((const void*)k_batch<AMP, U>, sh.block, sm, &per_sm);
  if (e) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const size_t ctas = (size_t)n_sm * (sh.ctas_per_sm < per_sm ? sh.ctas_per_sm : per_sm);
  const size_t need = (units + nw - 1) / nw;
  const int grid = (int)(ctas < need ? ctas : need);
  KParams kps = with_spill(kp, s);
  kps.big_list = s.big_list;
  if (AMP) {
    k_batch<AMP, U><<<grid, sh.block, sm, st>>>(raw, fed_len, s.fed_off, n_events, n_feds, clu_off, out_cap, status, kps,
                                                s.stage, s.ev_alloc, s.fed_cnt, s.fed_start, s.tickets, s.unit_desc,
                                                am);
  } else if ((e = launch_pdl(k_batch<AMP, U>, (unsigned)grid, (unsigned)sh.block, sm, st, raw, fed_len,
                             (const uint64_t*)s.fed_off, n_events, n_feds, clu_off, out_cap, status, kps, s.stage,
                             s.ev_alloc, s.fed_cnt, s.fed_start, s.tickets, (const uint2*)s.unit_desc, am))) {
    return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_fe(const uint8_t* raw, const uint32_t* fed_len, uint32_t n_events, uint32_t n_feds,
                            const uint64_t* clu_off, uint64_t out_cap, sst_event_status* status, const KParams& kp,
                            const Scratch& s, const Shape& sh, int n_sm, const AmpArgs& am, cudaStream_t st,
                            cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  cudaError_t e;
  if (ev_begin && (e = cudaEventRecord(ev_begin, st))) return e;
  if (sh.units == 1)
    e = am.stage ? launch_batch_t<true, 1>(raw, fed_len, n_events, n_feds, clu_off, out_cap, status, kp, s, sh, n_sm, am, st)
                 : launch_batch_t<false, 1>(raw, fed_len, n_events, n_feds, clu_off, out_cap, status, kp, s, sh, n_sm, am, st);
  else
    e = am.stage ? launch_batch_t<true, 2>(raw, fed_len, n_events, n_feds, clu_off, out_cap, status, kp, s, sh, n_sm, am, st)
                 : launch_batch_t<false, 2>(raw, fed_len, n_events, n_feds, clu_off, out_cap, status, kp, s, sh, n_sm, am, st);
  if (e) return e;
  if (ev_end && (e = cudaEventRecord(ev_end, st))) return e;
  return cudaSuccess;
}

// Per-event cluster order and the copy into the caller's SoA.
cudaError_t launch_order(const uint64_t* clu_off, uint32_t n_events, uint32_t n_segs, const sst_clusters& out,
                         sst_event_status* status, const Scratch& s, uint64_t* pack_off, const AmpArgs& am,
                         cudaStream_t st) {
  cudaError_t e;
  if (am.stage || pack_off) {
    k_clu_scan<<<n_events, 1024, 0, st>>>(s.fed_cnt, n_segs, s.fed_dest, status, pack_off, s.tickets + 1, am);
    if ((e = cudaGetLastError())) return e;
  }
  if (am.stage) {
    const uint64_t items = (uint64_t)n_events * n_segs;
    k_compact<<<(unsigned)((items + 7) / 8), 256, 0, st>>>(s.stage, clu_off, pack_off, s.fed_cnt, s.fed_start,
                                                          s.fed_dest, n_events, n_segs, out, am);
  } else {
    // 64 segments per CTA for a batch; 16 when that would give a small grid (one
    // event, a short chunk), so that enough CTAs share the copy
    const uint32_t cpe64 = (n_segs + 63) / 64;
    const uint4* stage = s.stage;
    const uint64_t* pack = pack_off;
    const uint32_t* cnt = s.fed_cnt;
    const uint32_t* start = s.fed_start;
    if ((uint64_t)n_events * cpe64 >= 256) {
      e = launch_pdl(k_order<64>, (unsigned)((uint64_t)n_events * cpe64), 256u, 0, st, stage, clu_off, pack, cnt, start,
                     n_segs, cpe64, out, status);
    } else {
      const uint32_t cpe16 = (n_segs + 15) / 16;
      e = launch_pdl(k_order<16>, (unsigned)((uint64_t)n_events * cpe16), 256u, 0, st, stage, clu_off, pack, cnt, start,
                     n_segs, cpe16, out, status);
    }
    if (e) return e;
  }
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------- host side

size_t smem_bytes(int tile) {
  switch (tile) {
    case 1024: return sizeof(Shm<1024>);
    case 2048: return sizeof(Shm<2048>);
    case 4096: return sizeof(Shm<4096>);
    default: return 0;
  }
}

// Shared memory per CTA of the batched kernel for a work-item width and block size.
size_t batch_smem(int units, int block) {
  return (units == 1 ? sizeof(fe::WarpT<1>) : sizeof(fe::WarpT<2>)) * (size_t)(block / 32);
}

Shape default_shape() { return Shape{256, 2048, 2, 4, 0, 2}; }

bool shape_valid(const Shape& s) {
  const bool blk = s.block == 128 || s.block == 256;
  const bool til = s.tile == 1024 || s.tile == 2048 || s.tile == 4096;
  const bool ln = s.lanes == 1 || s.lanes == 2 || s.lanes == 4 || s.lanes == 8 || s.lanes == 16 || s.lanes == 32;
  return blk && til && ln && s.ctas_per_sm >= 1 && s.ctas_per_sm <= 8 && s.host_chunk >= 0 && s.host_chunk <= 4096 &&
         (s.units == 1 || s.units == 2);
}

cudaError_t batch_launch_info(const Shape& sh, uint32_t n_events, uint32_t n_feds, int n_sm, int* grid, size_t* smem,
                              int* items_per_fed) {
  const size_t sm = batch_smem(sh.units, sh.block);
  const void* fn = sh.units == 1 ? (const void*)k_batch<false, 1> : (const void*)k_batch<false, 2>;
  int per_sm = 0;
  cudaError_t e = prepare(fn, sh.block, sm, &per_sm);
  if (e) return e;
  const int nw = sh.block / 32;
  const size_t units = (size_t)n_events * n_feds * (kFe / sh.units);
  const size_t ctas = (size_t)n_sm * (sh.ctas_per_sm < per_sm ? sh.ctas_per_sm : per_sm);
  const size_t need = (units + nw - 1) / nw;
  *grid = (int)(ctas < need ? ctas : need);
  *smem = sm;
  *items_per_fed = kFe / sh.units;
  return cudaSuccess;
}

cudaError_t launch_unpack(const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len, uint32_t n_feds,
                          const sst_digis& out, const Scratch& s, const Shape& sh, cudaStream_t st) {
  cudaError_t e;
  const uint32_t cpe = (n_feds + kFedScanThreads - 1) / kFedScanThreads;
  k_fed_scan<<<cpe, kFedScanThreads, 0, st>>>(nullptr, raw_bytes, fed_len, n_feds, cpe, s.fed_off, out.status, nullptr,
                                              s.tickets, s.lb, n_feds, nullptr, nullptr, nullptr, nullptr, 0u, 1u,
                                              nullptr);
  if ((e = cudaGetLastError())) return e;
  switch (sh.tile) {
    case 1024: return launch_unpack_t<1024>(raw, fed_len, n_feds, out, s, sh, st);
    case 2048: return launch_unpack_t<2048>(raw, fed_len, n_feds, out, s, sh, st);
    case 4096: return launch_unpack_t<4096>(raw, fed_len, n_feds, out, s, sh, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cluster(const sst_digis& in, uint32_t n_feds, const sst_clusters& out, const KParams& kp,
                           const Scratch& s, const Shape& sh, cudaStream_t st) {
  cudaError_t e;
  const AmpArgs am = amp_args(out, s);
  if ((e = cudaMemsetAsync(s.ev_alloc, 0, sizeof(uint32_t), st))) return e;
  if (am.stage && (e = cudaMemsetAsync(s.amp_alloc, 0, sizeof(uint32_t), st))) return e;
  if ((e = launch_cluster_fe(in, n_feds, kp, s, out.capacity, sh, am, st))) return e;
  return launch_order(nullptr, 1, n_feds * kFe, out, in.status, s, nullptr, am, st);  // one event at offset 0
}

cudaError_t launch_batch(const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len, uint32_t n_events,
                         uint32_t n_feds, const uint64_t* clu_off, const sst_clusters& out, sst_event_status* status,
                         const KParams& kp, const Scratch& s, const Shape& sh, int n_sm, cudaStream_t st,
                         uint64_t* pack_off, cudaEvent_t ev_begin, cudaEvent_t ev_end, const uint64_t* event_end) {
  cudaError_t e;
  const AmpArgs am = amp_args(out, s);
  const uint32_t cpe = (n_feds + kFedScanThreads - 1) / kFedScanThreads;
  if ((e = cudaMemsetAsync(s.tickets + 2, 0, sizeof(uint32_t), st))) return e;  // the prologue's list of large items
  k_fed_scan<<<(unsigned)((uint64_t)n_events * cpe), kFedScanThreads, 0, st>>>(
      event_off, 0, fed_len, n_feds, cpe, s.fed_off, status, s.ev_alloc, s.tickets, nullptr, 0, raw, s.unit_desc,
      am.stage ? s.amp_alloc : nullptr, s.big_list, sh.units == 1 ? (uint32_t)fe::WarpT<1>::kBuf : (uint32_t)fe::WarpT<2>::kBuf,
      sh.units == 1 ? 1u : 2u, event_end);
  if ((e = cudaGetLastError())) return e;
  e = launch_batch_fe(raw, fed_len, n_events, n_feds, clu_off, out.capacity, status, kp, s, sh, n_sm, am, st,
                      ev_begin, ev_end);
  if (e) return e;
  return launch_order(clu_off, n_events, n_feds * (kFe / (sh.units == 1 ? 1 : 2)), out, status, s, pack_off, am, st);
}

cudaError_t rebase_amp_first(uint32_t* amp_first, const uint64_t* count, uint32_t base, int n_sm, cudaStream_t st) {
  k_rebase_amp<<<(unsigned)(n_sm > 0 ? n_sm * 2 : 128), 256, 0, st>>>(amp_first, count, base);
  return cudaGetLastError();
}

cudaError_t build_badmask(const uint8_t* bad_dev, uint32_t* mask_dev, uint64_t n_strips, cudaStream_t st) {
  const uint64_t words = n_strips / 32;
  k_badmask<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(bad_dev, mask_dev, words);
  return cudaGetLastError();
}

cudaError_t build_calib(const float* noise_dev, const uint32_t* mask_dev, uint2* calq_dev, uint64_t n_strips,
                        const sst_params& p, cudaStream_t st) {
  k_calib_pack<<<(unsigned)((n_strips + 255) / 256), 256, 0, st>>>(noise_dev, mask_dev, calq_dev, n_strips,
                                                                   p.t_channel, p.t_seed, p.max_seq_holes,
                                                                   p.max_seq_bad);
  return cudaGetLastError();
}

}  // namespace sst
