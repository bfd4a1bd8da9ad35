// sst_kernels.cu -- sm_103a kernels for unpacking zero-suppressed FED data and
// three-threshold clustering (arXiv 2101.11489, section 2), per event and batched
// (section 3).
//
// Work unit: one FED (96 channels x 256 strips) of one event, handled by one CTA.
// A CTA stages the FED's bytes in shared memory with 16-byte loads, walks the
// header and FE-unit lengths to locate the 96 channel records (the "map of channel
// locations"), validates and counts each channel's runs (one thread per channel),
// prefix-sums the counts, and copies the runs into an on-chip digi tile sorted by
// strip (groups of `lanes` threads per channel).  The clustering then works on the
// tile: flags against noise x threshold, per-channel 256-bit active / seed / bad
// masks in shared memory, a left scan from every seed that keeps only the leftmost
// seed of each candidate, a right scan, the charge / threshold / centroid sums in
// strip order, and a block scan that ranks the kept clusters.  The cluster (or
// digi) offset of a FED within its event comes from a decoupled look-back over the
// FEDs of that event, so that output is sorted without a second pass.  FEDs with
// more digis than one tile are processed in channel-aligned chunks.
//
// All floating point in the threshold tests and sums uses explicit round-to-nearest
// intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn), so no multiply-add is
// contracted and results match a sequential binary32 evaluation bit for bit.
//
// Every device wait (the look-back) has an iteration limit; when it runs out the
// event is flagged SST_EV_TIMEOUT and the CTA carries on without the value.
#include "sst_internal.h"

namespace sst {

namespace {

// ---------------------------------------------------------------- constants

constexpr unsigned long long kLbAgg = 1ull << 62;   // state carries this FED's own count
constexpr unsigned long long kLbPre = 2ull << 62;   // state carries the inclusive prefix
constexpr unsigned long long kLbMask = 3ull << 62;
constexpr int kLbSpinLimit = 1 << 21;               // polls before giving up (~seconds)
constexpr uint64_t kBadOff = ~0ull;                 // fed_off marker: record outside the event

// Shared-memory scalars (indices into s.scal).
enum {
  S_TICKET = 0, S_FEDOK, S_TOTAL, S_BASE, S_CHUNK_N, S_EMITS, S_FLAGS, S_NBAD, S_TIMEOUT, S_C1,
  S_SCAL_N = 16
};

constexpr int kFedBufMin = 16384;

// ---------------------------------------------------------------- shared layout

struct Smem {
  uint32_t* scal;      // [16]
  uint32_t* wsum;      // [32]
  uint32_t* chan_pos;  // [96] byte offset of the channel record within the FED
  uint32_t* chan_cnt;  // [97] digis per channel, then exclusive prefix (in place)
  uint16_t* chan_len;  // [96]
  uint8_t* chan_st;    // [96]
  uint32_t* fe_len;    // [8]
  uint32_t* bad;       // [96*8]
  uint32_t* act;       // [96*8]
  uint32_t* sed;       // [96*8]
  float* gain;         // [96*2]
  uint16_t* t_key;     // [tile] (channel << 8) | strip
  uint8_t* t_adc;      // [tile]
  uint8_t* t_flag;     // [tile] 1 active, 2 seed, 8 emits a cluster
  float* t_noise;      // [tile] noise; reused as the rank of emitting digis
  uint8_t* fedbuf;     // [fedbuf bytes]  union with the cluster staging below
  uint16_t* st_first;  // [tile]
  uint16_t* st_width;  // [tile]
  uint32_t* st_charge; // [tile]
  float* st_bary;      // [tile]
  int tile;
  int fedbuf_bytes;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

struct Layout {
  size_t scal, wsum, chan_pos, chan_cnt, chan_len, chan_st, fe_len, bad, act, sed, gain;
  size_t t_key, t_adc, t_flag, t_noise, uni, st_first, st_width, st_charge, st_bary, total;
  int fedbuf;
};

__host__ __device__ inline Layout make_layout(int tile) {
  Layout L{};
  size_t o = 0;
  L.scal = o; o = al16(o + S_SCAL_N * 4);
  L.wsum = o; o = al16(o + 32 * 4);
  L.chan_pos = o; o = al16(o + kCh * 4);
  L.chan_cnt = o; o = al16(o + (kCh + 1) * 4);
  L.chan_len = o; o = al16(o + kCh * 2);
  L.chan_st = o; o = al16(o + kCh);
  L.fe_len = o; o = al16(o + kFe * 4);
  L.bad = o; o = al16(o + kCh * kMaskWords * 4);
  L.act = o; o = al16(o + kCh * kMaskWords * 4);
  L.sed = o; o = al16(o + kCh * kMaskWords * 4);
  L.gain = o; o = al16(o + kCh * 2 * 4);
  L.t_noise = o; o = al16(o + (size_t)tile * 4);
  L.t_key = o; o = al16(o + (size_t)tile * 2);
  L.t_adc = o; o = al16(o + (size_t)tile);
  L.t_flag = o; o = al16(o + (size_t)tile);
  size_t staging = (size_t)tile * 12;
  size_t uni = staging > (size_t)kFedBufMin ? staging : (size_t)kFedBufMin;
  L.fedbuf = (int)uni;
  L.uni = o;
  L.st_charge = o;
  L.st_bary = o + (size_t)tile * 4;
  L.st_first = o + (size_t)tile * 8;
  L.st_width = o + (size_t)tile * 10;
  o = al16(o + uni);
  L.total = o;
  return L;
}

__device__ inline Smem bind_smem(unsigned char* base, int tile) {
  Layout L = make_layout(tile);
  Smem s;
  s.scal = (uint32_t*)(base + L.scal);
  s.wsum = (uint32_t*)(base + L.wsum);
  s.chan_pos = (uint32_t*)(base + L.chan_pos);
  s.chan_cnt = (uint32_t*)(base + L.chan_cnt);
  s.chan_len = (uint16_t*)(base + L.chan_len);
  s.chan_st = (uint8_t*)(base + L.chan_st);
  s.fe_len = (uint32_t*)(base + L.fe_len);
  s.bad = (uint32_t*)(base + L.bad);
  s.act = (uint32_t*)(base + L.act);
  s.sed = (uint32_t*)(base + L.sed);
  s.gain = (float*)(base + L.gain);
  s.t_key = (uint16_t*)(base + L.t_key);
  s.t_adc = (uint8_t*)(base + L.t_adc);
  s.t_flag = (uint8_t*)(base + L.t_flag);
  s.t_noise = (float*)(base + L.t_noise);
  s.fedbuf = (uint8_t*)(base + L.uni);
  s.st_first = (uint16_t*)(base + L.st_first);
  s.st_width = (uint16_t*)(base + L.st_width);
  s.st_charge = (uint32_t*)(base + L.st_charge);
  s.st_bary = (float*)(base + L.st_bary);
  s.tile = tile;
  s.fedbuf_bytes = L.fedbuf;
  return s;
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

__device__ __forceinline__ uint32_t rd8(const uint8_t* p) { return *p; }
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
    uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  uint32_t pre = warp > 0 ? wsum[warp - 1] : 0u;
  *total = wsum[nw - 1];
  __syncthreads();
  return pre + x - v;
}

// Decoupled look-back over items lo .. idx-1 of one event.  Returns the sum of the
// counts of all earlier items.  Called by one thread.
__device__ uint32_t lookback(unsigned long long* lb, long long idx, long long lo, bool* timed_out) {
  uint32_t excl = 0;
  for (long long j = idx - 1; j >= lo; --j) {
    unsigned long long v;
    int spins = 0;
    unsigned ns = 32;
    for (;;) {
      v = ld_acquire(lb + j);
      if (v & kLbMask) break;
      if (++spins > kLbSpinLimit) {
        *timed_out = true;
        return excl;
      }
      __nanosleep(ns);
      if (ns < 1024) ns <<= 1;
    }
    excl += (uint32_t)v;
    if ((v & kLbMask) == kLbPre) break;
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

// Parses one FED (a1 + the validating count of a2).  On return (after a barrier):
// chan_pos/len/st hold each channel's record, chan_cnt[0..96] the exclusive
// prefix of the per-channel digi counts, scal[S_TOTAL] the FED's digi count,
// scal[S_FLAGS] / scal[S_NBAD] the OR of channel statuses and the number of bad
// channels.  Returns the pointer the records are to be read from (shared or
// global).  `len` is the FED record length; `present` is false for an absent FED
// (fed_len 0) and `in_range` false when the record would leave the event.
__device__ const uint8_t* parse_fed(const Smem& s, const uint8_t* gfed, uint32_t len, uint32_t fed_id,
                                    bool in_range) {
  const int tid = threadIdx.x;
  const bool present = in_range && len > 0;
  const bool staged = present && len <= (uint32_t)s.fedbuf_bytes;
  if (staged) stage_fed(gfed, len, s.fedbuf);
  const uint8_t* src = staged ? s.fedbuf : gfed;
  __syncthreads();

  // FED header (thread 0).
  if (tid == 0) {
    uint32_t ok = 0;
    if (present && len >= (uint32_t)kHdr) {
      uint64_t body = 0;
      for (int u = 0; u < kFe; u++) {
        uint32_t l = rd16(src + 16 + 2 * u);
        s.fe_len[u] = l;
        body += (l + 7u) & ~7u;
      }
      uint64_t total = (kHdr + body + 15u) & ~uint64_t(15);
      ok = rd32(src) == SST_FED_MAGIC && rd16(src + 4) == fed_id && rd8(src + 6) == (uint32_t)kCh &&
           rd8(src + 7) == (uint32_t)kFe && rd32(src + 8) == len && total == len;
    }
    s.scal[S_FEDOK] = ok;
  }
  __syncthreads();
  const bool fed_ok = s.scal[S_FEDOK] != 0;
  const uint8_t fed_status = (!in_range || (present && !fed_ok)) ? (uint8_t)SST_CH_FED_HDR : (uint8_t)0;

  // FE-unit walk: one thread per FE unit locates its 12 channel records.
  if (tid < kFe) {
    const int u = tid;
    if (fed_ok) {
      uint32_t start = kHdr;
      for (int v = 0; v < u; v++) start += (s.fe_len[v] + 7u) & ~7u;
      const uint32_t end = start + s.fe_len[u];
      uint32_t p = start;
      bool ok = true;
      for (int k = 0; k < kChPerFe; k++) {
        const int c = u * kChPerFe + k;
        uint32_t l = 0;
        if (ok) {
          if (p + 2 > end) {
            ok = false;
          } else {
            l = rd16(src + p);
            if (l < 3 || p + l > end) ok = false;
          }
        }
        s.chan_pos[c] = ok ? p : 0;
        s.chan_len[c] = ok ? (uint16_t)l : 0;
        if (ok) p += l;
      }
      if (ok && p != end) ok = false;
      for (int k = 0; k < kChPerFe; k++) s.chan_st[u * kChPerFe + k] = ok ? 0 : (uint8_t)SST_CH_FRAMING;
    } else {
      for (int k = 0; k < kChPerFe; k++) {
        const int c = u * kChPerFe + k;
        s.chan_pos[c] = 0;
        s.chan_len[c] = 0;
        s.chan_st[c] = fed_status;
      }
    }
  }
  __syncthreads();

  // Channel records: validate every run and count digis (one thread per channel).
  if (tid < kCh) {
    const int c = tid;
    uint32_t cnt = 0;
    uint8_t st = s.chan_st[c];
    if (st == 0 && fed_ok) {
      const uint8_t* r = src + s.chan_pos[c];
      const uint32_t len_c = s.chan_len[c];
      if (rd8(r + 2) != SST_ZS_CODE) {
        st = SST_CH_BAD_CODE;
      } else {
        uint32_t p = 3, prev_end = 0;
        while (p < len_c) {
          if (p + 2 > len_c) { st = SST_CH_TRUNC; break; }
          const uint32_t first = rd8(r + p), w = rd8(r + p + 1);
          if (w == 0 || first + w > (uint32_t)kStrips) { st = SST_CH_RUN_RANGE; break; }
          if (first < prev_end) { st = SST_CH_RUN_ORDER; break; }
          if (p + 2 + w > len_c) { st = SST_CH_TRUNC; break; }
          prev_end = first + w;
          cnt += w;
          p += 2 + w;
        }
      }
      if (st) cnt = 0;
      s.chan_st[c] = st;
    }
    s.chan_cnt[c] = cnt;
  }
  __syncthreads();

  // Exclusive prefix over the 96 channel counts, plus status summary (warp 0).
  if (tid < 32) {
    uint32_t v[3], fl = 0, nb = 0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      v[k] = s.chan_cnt[tid * 3 + k];
      const uint8_t st = s.chan_st[tid * 3 + k];
      fl |= st;
      nb += st ? 1u : 0u;
    }
    const uint32_t local = v[0] + v[1] + v[2];
    uint32_t x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (tid >= d) x += y;
    }
    uint32_t e = x - local;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      s.chan_cnt[tid * 3 + k] = e;
      e += v[k];
    }
    if (tid == 31) {
      s.chan_cnt[kCh] = x;
      s.scal[S_TOTAL] = x;
    }
    fl = __reduce_or_sync(0xffffffffu, fl);
    nb = __reduce_add_sync(0xffffffffu, nb);
    if (tid == 0) {
      s.scal[S_FLAGS] = fl;
      s.scal[S_NBAD] = nb;
    }
  }
  __syncthreads();
  return src;
}

// Copies the runs of channels [c0, c1) into the tile (digis sorted by strip).
// Groups of `lanes` threads share a channel: all walk the run headers, each copies
// every lanes-th ADC byte.  Records were validated by parse_fed; the copy is still
// bounded by the counted digis so that it cannot leave the tile.
__device__ void emit_tile(const Smem& s, const uint8_t* src, int c0, int c1, int lanes) {
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
      const uint32_t first = rd8(r + p);
      uint32_t w = rd8(r + p + 1);
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

// Loads bad-strip masks and APV gains of the FED's 96 channels.
__device__ void load_fed_calib(const Smem& s, const KParams& kp, uint32_t fed) {
  const uint32_t* bm = kp.badmask + (size_t)fed * kCh * kMaskWords;
  for (int i = threadIdx.x; i < kCh * kMaskWords; i += blockDim.x) s.bad[i] = __ldg(bm + i);
  const float* gp = kp.gain + (size_t)fed * kCh * 2;
  for (int i = threadIdx.x; i < kCh * 2; i += blockDim.x) s.gain[i] = __ldg(gp + i);
}

// a3: active / seed flags of the n tile digis, and the per-channel masks.
__device__ void flag_tile(const Smem& s, const KParams& kp, uint32_t fed, int c0, int c1, int n) {
  for (int i = threadIdx.x; i < (c1 - c0) * kMaskWords; i += blockDim.x) {
    s.act[c0 * kMaskWords + i] = 0;
    s.sed[c0 * kMaskWords + i] = 0;
  }
  __syncthreads();
  const float* noise = kp.noise + (size_t)fed * kFedStrips;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const uint32_t key = s.t_key[i];
    const uint32_t c = key >> 8, st = key & 255u;
    uint8_t fl = 0;
    float nz = 0.f;
    if ((int)c >= c0 && (int)c < c1) {
      nz = __ldg(noise + key);
      const uint32_t w = c * kMaskWords + (st >> 5), m = 1u << (st & 31u);
      const bool isbad = (s.bad[w] & m) != 0;
      const float a = __uint2float_rn(s.t_adc[i]);
      const bool act = !isbad && a > __fmul_rn(kp.t_channel, nz);
      const bool sd = !isbad && a > __fmul_rn(kp.t_seed, nz);
      fl = (act ? 1 : 0) | (sd ? 2 : 0);
      if (act) atomicOr(&s.act[w], m);
      if (sd) atomicOr(&s.sed[w], m);
    }
    s.t_flag[i] = fl;
    s.t_noise[i] = nz;
  }
  __syncthreads();
}

__device__ __forceinline__ bool bit(const uint32_t* m, int t) { return (m[t >> 5] >> (t & 31)) & 1u; }

// a4 + a5 + a6: for every seed, scan left (stopping at another seed = not the
// leftmost seed of its candidate), scan right, widen over adjacent bad strips,
// sum in strip order, test against the cluster threshold, and stage the result.
__device__ void form_tile(const Smem& s, const KParams& kp, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (!(s.t_flag[i] & 2)) continue;
    const uint32_t key = s.t_key[i];
    const int c = key >> 8, sp = key & 255;
    const uint32_t* A = s.act + c * kMaskWords;
    const uint32_t* S = s.sed + c * kMaskWords;
    const uint32_t* B = s.bad + c * kMaskWords;
    // left boundary; ownership
    int l = sp, holes = 0, bads = 0;
    bool owner = true;
    for (int t = sp - 1; t >= 0; --t) {
      if (bit(A, t)) {
        if (bit(S, t)) { owner = false; break; }
        l = t; holes = 0; bads = 0;
      } else if (bit(B, t)) {
        if (++bads > kp.max_bad) break;
        holes = 0;
      } else {
        if (++holes > kp.max_holes) break;
        bads = 0;
      }
    }
    if (!owner) continue;
    // right boundary
    int r = sp;
    holes = 0; bads = 0;
    for (int t = sp + 1; t < kStrips; ++t) {
      if (bit(A, t)) {
        r = t; holes = 0; bads = 0;
      } else if (bit(B, t)) {
        if (++bads > kp.max_bad) break;
        holes = 0;
      } else {
        if (++holes > kp.max_holes) break;
        bads = 0;
      }
    }
    int lo = l, hi = r;
    for (int k = 0; k < kp.max_adj && lo - 1 >= 0 && bit(B, lo - 1); k++) lo--;
    for (int k = 0; k < kp.max_adj && hi + 1 < kStrips && bit(B, hi + 1); k++) hi++;
    // sums over the active strips of [l, r], left to right
    const uint32_t kl = ((uint32_t)c << 8) | (uint32_t)l, kr = ((uint32_t)c << 8) | (uint32_t)r;
    int j = i;
    while (j > 0 && s.t_key[j - 1] >= kl) --j;
    uint32_t s_raw = 0, q_sum = 0, moment = 0;
    float n2 = 0.f;
    const float g0 = s.gain[c * 2], g1 = s.gain[c * 2 + 1];
    for (; j < n && s.t_key[j] <= kr; ++j) {
      if (!(s.t_flag[j] & 1)) continue;
      const uint32_t a = s.t_adc[j];
      const int strip = s.t_key[j] & 255;
      const float nz = s.t_noise[j];
      s_raw += a;
      n2 = __fadd_rn(n2, __fmul_rn(nz, nz));
      uint32_t q;
      if (a >= 254u) {
        q = a;
      } else {
        const float x = __fdiv_rn(__uint2float_rn(a), strip < kApv ? g0 : g1);
        const int ci = __float2int_rz(__fadd_rn(x, 0.5f));
        q = ci > 253 ? 254u : (uint32_t)ci;
      }
      q_sum += q;
      moment += (uint32_t)(strip - lo) * q;
    }
    if (!(__uint2float_rn(s_raw) > __fmul_rn(kp.t_cluster, __fsqrt_rn(n2)))) continue;
    const int w = hi - lo + 1;
    float bary;
    if (q_sum == 0) {
      bary = __fadd_rn((float)lo, __fmul_rn(0.5f, (float)w));
    } else {
      bary = __fadd_rn(__fadd_rn((float)lo, 0.5f), __fdiv_rn(__uint2float_rn(moment), __uint2float_rn(q_sum)));
    }
    s.st_first[i] = (uint16_t)lo;
    s.st_width[i] = (uint16_t)w;
    s.st_charge[i] = q_sum;
    s.st_bary[i] = bary;
    s.t_flag[i] |= 8;
  }
  __syncthreads();
}

// Ranks the emitting digis of the tile in tile order; returns their number.
__device__ uint32_t rank_tile(const Smem& s, int n) {
  const int T = blockDim.x;
  const int k = (n + T - 1) / T;
  const int b0 = threadIdx.x * k;
  const int b1 = min(n, b0 + k);
  uint32_t cnt = 0;
  for (int i = b0; i < b1; i++) cnt += (s.t_flag[i] >> 3) & 1u;
  uint32_t total;
  uint32_t r = block_excl_scan(cnt, s.wsum, &total);
  uint32_t* rank = reinterpret_cast<uint32_t*>(s.t_noise);
  for (int i = b0; i < b1; i++)
    if (s.t_flag[i] & 8) rank[i] = r++;
  __syncthreads();
  return total;
}

// Writes the staged clusters of the tile to out[off + base + rank].
__device__ void write_tile(const Smem& s, const sst_clusters& out, uint64_t off, uint64_t cap, uint32_t base,
                           uint32_t fed, int n) {
  const uint32_t* rank = reinterpret_cast<const uint32_t*>(s.t_noise);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (!(s.t_flag[i] & 8)) continue;
    const uint64_t pos = (uint64_t)base + rank[i];
    if (pos >= cap) continue;
    const uint64_t o = off + pos;
    out.det[o] = fed * kCh + (s.t_key[i] >> 8);
    out.first[o] = s.st_first[i];
    out.width[o] = s.st_width[i];
    out.charge[o] = s.st_charge[i];
    out.barycenter[o] = s.st_bary[i];
  }
}

// Greedy channel-aligned chunk [c0, c1) holding at most `tile` digis.
__device__ int chunk_end(const Smem& s, int c0, int tile) {
  int c1 = c0 + 1;
  while (c1 < kCh && s.chan_cnt[c1 + 1] - s.chan_cnt[c0] <= (uint32_t)tile) ++c1;
  return c1;
}

// Clusters the digis of one FED (already parsed into chan_* or loaded by
// `load`), writing to out[off ...] with per-event capacity `cap`; the FED's
// cluster offset comes from the look-back over lb[lo .. idx-1].  `fill(c0, c1)`
// puts the digis of channels [c0, c1) into the tile.  Returns the clusters found.
template <typename Fill>
__device__ void cluster_fed(const Smem& s, const KParams& kp, uint32_t fed, Fill fill, const sst_clusters& out,
                            uint64_t off, uint64_t cap, unsigned long long* lb, long long idx, long long lo,
                            sst_event_status* status) {
  const int tid = threadIdx.x;
  const uint32_t total_digis = s.chan_cnt[kCh];
  const bool single = total_digis <= (uint32_t)s.tile;
  uint32_t base = 0, found = 0, written = 0;
  bool first_chunk = true;
  int c0 = 0;
  while (c0 < kCh) {
    const int c1 = single ? kCh : chunk_end(s, c0, s.tile);
    const int n = (int)(s.chan_cnt[c1] - s.chan_cnt[c0]);
    if (n > 0 || first_chunk) {
      if (n > 0) {
        fill(c0, c1);
        __syncthreads();
        flag_tile(s, kp, fed, c0, c1, n);
        form_tile(s, kp, n);
      }
      const uint32_t emits = n > 0 ? rank_tile(s, n) : 0u;
      if (first_chunk) {
        if (tid == 0) {
          bool to = false;
          uint32_t excl = 0;
          if (idx > lo) {
            if (single) st_release(lb + idx, kLbAgg | emits);
            excl = lookback(lb, idx, lo, &to);
          }
          if (single) st_release(lb + idx, kLbPre | (uint32_t)(excl + emits));
          s.scal[S_BASE] = excl;
          s.scal[S_TIMEOUT] = to ? 1u : 0u;
        }
        __syncthreads();
        base = s.scal[S_BASE];
        first_chunk = false;
      }
      if (n > 0) {
        write_tile(s, out, off, cap, base + found, fed, n);
        const uint64_t start = (uint64_t)base + found;
        const uint64_t end = start + emits;
        written += (uint32_t)(end <= cap ? emits : (start < cap ? cap - start : 0));
        found += emits;
        __syncthreads();
      }
    }
    c0 = c1;
  }
  if (tid == 0) {
    if (!single) st_release(lb + idx, kLbPre | (uint32_t)(base + found));
    uint32_t fl = 0;
    if ((uint64_t)base + found > cap) fl |= SST_EV_CLUSTER_CAPACITY;
    if (s.scal[S_TIMEOUT]) fl |= SST_EV_TIMEOUT;
    if (fl) atomicOr(&status->flags, fl);
    if (written) atomicAdd(&status->n_clusters, written);
  }
}

// ---------------------------------------------------------------- kernels

// a1, outer level: byte offset of every FED record (exclusive scan of fed_len per
// event, plus the event's start).  A record that would end past its event is
// marked kBadOff; a size mismatch sets SST_EV_SIZE.  One CTA per event.
__global__ void k_fed_scan(const uint64_t* __restrict__ event_off, uint64_t raw_bytes,
                           const uint32_t* __restrict__ fed_len, uint32_t n_feds, uint64_t* __restrict__ fed_off,
                           sst_event_status* status) {
  __shared__ uint32_t wsum[32];
  __shared__ uint64_t carry_s;
  const uint32_t e = blockIdx.x;
  const uint64_t ev0 = event_off ? event_off[e] : 0;
  const uint64_t ev1 = event_off ? event_off[e + 1] : raw_bytes;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint32_t b = 0; b < n_feds; b += blockDim.x) {
    const uint32_t f = b + threadIdx.x;
    const uint32_t len = f < n_feds ? fed_len[(size_t)e * n_feds + f] : 0u;
    uint32_t tot;
    // 32-bit scan of this chunk; carry kept in 64 bits
    const uint32_t ex = block_excl_scan(len, wsum, &tot);
    const uint64_t carry = carry_s;
    if (f < n_feds) {
      const uint64_t o = ev0 + carry + ex;
      fed_off[(size_t)e * n_feds + f] = (ev1 >= ev0 && o + len <= ev1 && o >= ev0) ? o : kBadOff;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_s = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && ev0 + carry_s != ev1) atomicOr(&status[e].flags, SST_EV_SIZE);
}

// a1 + a2 per event: one CTA per FED (ticket order), digis written to the global
// digi SoA at the FED's offset from the look-back over FED digi counts.
__global__ void __launch_bounds__(512) k_unpack(const uint8_t* __restrict__ raw,
                                                const uint32_t* __restrict__ fed_len,
                                                const uint64_t* __restrict__ fed_off, uint32_t n_feds,
                                                sst_digis out, unsigned long long* lb, uint32_t* ticket,
                                                int tile, int lanes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = bind_smem(smem, tile);
  const int tid = threadIdx.x;
  if (tid == 0) s.scal[S_TICKET] = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t f = s.scal[S_TICKET];
  if (f >= n_feds) return;
  const uint64_t fo = fed_off[f];
  const bool in_range = fo != kBadOff;
  const uint32_t len = in_range ? fed_len[f] : 0u;
  const uint8_t* src = parse_fed(s, in_range ? raw + fo : raw, len, f, in_range);
  const uint32_t total = s.scal[S_TOTAL];
  if (tid == 0) {
    bool to = false;
    uint32_t excl = 0;
    if (f > 0) {
      st_release(lb + f, kLbAgg | total);
      excl = lookback(lb, f, 0, &to);
    }
    st_release(lb + f, kLbPre | (excl + total));
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
  int c0 = 0;
  while (c0 < kCh) {
    const int c1 = chunk_end(s, c0, tile);
    const int n = (int)(s.chan_cnt[c1] - s.chan_cnt[c0]);
    if (n > 0) {
      emit_tile(s, src, c0, c1, lanes);
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

// a3 - a6 per event: one CTA per FED (ticket order) over the global digi SoA.
__global__ void __launch_bounds__(512) k_cluster(sst_digis in, uint32_t n_feds, sst_clusters out, KParams kp,
                                                 unsigned long long* lb, uint32_t* ticket, int tile) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = bind_smem(smem, tile);
  const int tid = threadIdx.x;
  if (tid == 0) s.scal[S_TICKET] = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t f = s.scal[S_TICKET];
  if (f >= n_feds) return;
  // Channel digi ranges from the CSR row pointers, clamped to the input capacity
  // and to 256 digis per channel, so that malformed input cannot leave the tile.
  if (tid < kCh) {
    const size_t c = (size_t)f * kCh + tid;
    uint64_t a = in.chan_off[c], b = in.chan_off[c + 1];
    if (a > in.capacity) a = in.capacity;
    if (b > in.capacity) b = in.capacity;
    const uint32_t n = b > a ? (uint32_t)(b - a) : 0u;
    s.chan_pos[tid] = (uint32_t)a;
    s.chan_cnt[tid] = n < (uint32_t)kStrips ? n : (uint32_t)kStrips;
  }
  load_fed_calib(s, kp, f);
  __syncthreads();
  if (tid < 32) {  // exclusive prefix of the 96 counts
    uint32_t v[3];
#pragma unroll
    for (int k = 0; k < 3; k++) v[k] = s.chan_cnt[tid * 3 + k];
    const uint32_t local = v[0] + v[1] + v[2];
    uint32_t x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (tid >= d) x += y;
    }
    uint32_t e = x - local;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      s.chan_cnt[tid * 3 + k] = e;
      e += v[k];
    }
    if (tid == 31) s.chan_cnt[kCh] = x;
  }
  __syncthreads();
  auto fill = [&](int c0, int c1) {
    const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const uint32_t g0 = f * (uint32_t)kFedStrips;
    for (int c = c0 + warp; c < c1; c += nw) {
      const uint32_t o = s.chan_cnt[c] - s.chan_cnt[c0];
      const uint32_t n = s.chan_cnt[c + 1] - s.chan_cnt[c];
      const size_t a = s.chan_pos[c];
      for (uint32_t k = lane; k < n; k += 32) {
        const uint32_t key = in.strip[a + k] - g0;
        // a digi that does not belong to channel c is ignored by flag_tile
        s.t_key[o + k] = (key >> 8) == (uint32_t)c ? (uint16_t)key : (uint16_t)0xFFFFu;
        s.t_adc[o + k] = in.adc[a + k];
      }
    }
  };
  cluster_fed(s, kp, f, fill, out, 0, out.capacity, lb, f, 0, in.status);
}

// a7: every FED of every event of a batch, unpacked and clustered on chip.  A
// persistent grid takes (FED, event) tickets FED-major, so that the CTAs working
// at any moment share the same FED's calibration in L2.
__global__ void __launch_bounds__(512) k_batch(const uint8_t* __restrict__ raw,
                                               const uint32_t* __restrict__ fed_len,
                                               const uint64_t* __restrict__ fed_off, uint32_t n_events,
                                               uint32_t n_feds, const uint64_t* __restrict__ clu_off,
                                               sst_clusters out, sst_event_status* status, KParams kp,
                                               unsigned long long* lb, uint32_t* ticket, int tile, int lanes) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Smem s = bind_smem(smem, tile);
  const int tid = threadIdx.x;
  const uint64_t n_items = (uint64_t)n_events * n_feds;
  for (;;) {
    if (tid == 0) s.scal[S_TICKET] = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t t = s.scal[S_TICKET];
    if (t >= n_items) break;
    const uint32_t f = t / n_events, e = t % n_events;
    const size_t item = (size_t)e * n_feds + f;
    const uint64_t fo = fed_off[item];
    const bool in_range = fo != kBadOff;
    const uint32_t len = in_range ? fed_len[item] : 0u;
    load_fed_calib(s, kp, f);
    const uint8_t* src = parse_fed(s, in_range ? raw + fo : raw, len, f, in_range);
    if (tid == 0) {
      if (s.scal[S_FLAGS]) atomicOr(&status[e].flags, s.scal[S_FLAGS]);
      if (s.scal[S_NBAD]) atomicAdd(&status[e].n_bad_channels, s.scal[S_NBAD]);
      if (s.scal[S_TOTAL]) atomicAdd(&status[e].n_digi, s.scal[S_TOTAL]);
    }
    const bool single = s.scal[S_TOTAL] <= (uint32_t)tile;
    // multi-chunk FEDs re-read their records from global memory: the staging
    // buffer is reused for cluster records after the first chunk
    const uint8_t* esrc = (single || src != s.fedbuf) ? src : raw + fo;
    auto fill = [&](int c0, int c1) { emit_tile(s, esrc, c0, c1, lanes); };
    const uint64_t off = clu_off[e];
    const uint64_t cap = clu_off[e + 1] - off;
    cluster_fed(s, kp, f, fill, out, off, cap, lb, (long long)item, (long long)e * n_feds, &status[e]);
    __syncthreads();
  }
}

__global__ void k_badmask(const uint8_t* __restrict__ bad, uint32_t* __restrict__ mask, uint64_t n_words) {
  const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_words) return;
  uint32_t m = 0;
  for (int b = 0; b < 32; b++) m |= (bad[w * 32 + b] != 0 ? 1u : 0u) << b;
  mask[w] = m;
}

}  // namespace

// ---------------------------------------------------------------- host side

size_t smem_bytes(int tile) { return make_layout(tile).total; }

Shape default_shape() { return Shape{256, 2048, 2, 3}; }

bool shape_valid(const Shape& s) {
  const bool blk = s.block == 128 || s.block == 256 || s.block == 512;
  const bool til = s.tile == 1024 || s.tile == 2048 || s.tile == 4096;
  const bool ln = s.lanes == 1 || s.lanes == 2 || s.lanes == 4 || s.lanes == 8 || s.lanes == 16 || s.lanes == 32;
  return blk && til && ln && s.ctas_per_sm >= 1 && s.ctas_per_sm <= 8;
}

static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_unpack(const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len, uint32_t n_feds,
                          const sst_digis& out, const Scratch& s, const Shape& sh, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(out.status, 0, sizeof(sst_event_status), st))) return e;
  if ((e = cudaMemsetAsync(s.lb, 0, sizeof(unsigned long long) * n_feds, st))) return e;
  if ((e = cudaMemsetAsync(s.tickets, 0, sizeof(uint32_t) * 4, st))) return e;
  k_fed_scan<<<1, 256, 0, st>>>(nullptr, raw_bytes, fed_len, n_feds, s.fed_off, out.status);
  const size_t sm = smem_bytes(sh.tile);
  if ((e = set_smem((const void*)k_unpack, sm))) return e;
  k_unpack<<<n_feds, sh.block, sm, st>>>(raw, fed_len, s.fed_off, n_feds, out, s.lb, s.tickets, sh.tile, sh.lanes);
  return cudaGetLastError();
}

cudaError_t launch_cluster(const sst_digis& in, uint32_t n_feds, const sst_clusters& out, const KParams& kp,
                           const Scratch& s, const Shape& sh, cudaStream_t st) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(&in.status->n_clusters, 0, sizeof(uint32_t), st))) return e;
  if ((e = cudaMemsetAsync(s.lb, 0, sizeof(unsigned long long) * n_feds, st))) return e;
  if ((e = cudaMemsetAsync(s.tickets, 0, sizeof(uint32_t) * 4, st))) return e;
  const size_t sm = smem_bytes(sh.tile);
  if ((e = set_smem((const void*)k_cluster, sm))) return e;
  k_cluster<<<n_feds, sh.block, sm, st>>>(in, n_feds, out, kp, s.lb, s.tickets, sh.tile);
  return cudaGetLastError();
}

cudaError_t launch_batch(const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len, uint32_t n_events,
                         uint32_t n_feds, const uint64_t* clu_off, const sst_clusters& out, sst_event_status* status,
                         const KParams& kp, const Scratch& s, const Shape& sh, int n_sm, cudaStream_t st) {
  cudaError_t e;
  const size_t items = (size_t)n_events * n_feds;
  if ((e = cudaMemsetAsync(status, 0, sizeof(sst_event_status) * n_events, st))) return e;
  if ((e = cudaMemsetAsync(s.lb, 0, sizeof(unsigned long long) * items, st))) return e;
  if ((e = cudaMemsetAsync(s.tickets, 0, sizeof(uint32_t) * 4, st))) return e;
  k_fed_scan<<<n_events, 256, 0, st>>>(event_off, 0, fed_len, n_feds, s.fed_off, status);
  const size_t sm = smem_bytes(sh.tile);
  if ((e = set_smem((const void*)k_batch, sm))) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, sh.block, sm))) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ctas = n_sm * (sh.ctas_per_sm < per_sm ? sh.ctas_per_sm : per_sm);
  const int grid = (size_t)ctas < items ? ctas : (int)items;
  k_batch<<<grid, sh.block, sm, st>>>(raw, fed_len, s.fed_off, n_events, n_feds, clu_off, out, status, kp, s.lb,
                                      s.tickets, sh.tile, sh.lanes);
  return cudaGetLastError();
}

cudaError_t build_badmask(const uint8_t* bad_dev, uint32_t* mask_dev, uint64_t n_strips, cudaStream_t st) {
  const uint64_t words = n_strips / 32;
  k_badmask<<<(unsigned)((words + 255) / 256), 256, 0, st>>>(bad_dev, mask_dev, words);
  return cudaGetLastError();
}

}  // namespace sst
