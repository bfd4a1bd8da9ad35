/*
 * sst_oracle.c -- plain sequential CPU oracle (test infrastructure only).
 *
 * Follows arXiv 2101.11489 section 2 ("Parallelization"):
 *   - the strip tracker is read out by FEDs of 96 channels x 256 strips, and in
 *     zero-suppression mode only strips above threshold are recorded, in a
 *     CSR-like layout where the channel is the row and the strip the column;
 *   - clustering is the "three thresholds" algorithm: a strip whose signal over
 *     noise exceeds the channel threshold is active, one that exceeds the seed
 *     threshold is a seed, every candidate cluster holds at least one seed, a
 *     cluster is bounded left and right around its seeds, and it is kept when
 *     its charge passes the cluster threshold; kept clusters report their
 *     boundaries and centroid.
 * Where the paper gives no detail (byte layout, the hole and bad-strip rules,
 * the gain rounding, the centroid convention) this file takes the readings that
 * the project's design notes list, and says so at each place.
 *
 * Floating point: every threshold and charge expression is evaluated in IEEE
 * binary32 with one rounding per operation.  Build with -ffp-contract=off and
 * without -ffast-math so that no multiply-add is fused.
 *
 * No part of this file is optimised: it walks FEDs, FE units, channels and
 * strips one at a time, in the order the definitions are stated.
 */
#include "sst_oracle.h"

#include <math.h>
#include <string.h>

/* ---- little-endian byte access ------------------------------------------ */

static uint32_t rd_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t rd_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static void wr_u16(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)(v & 0xFF);
  p[1] = (uint8_t)((v >> 8) & 0xFF);
}
static void wr_u32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)(v & 0xFF);
  p[1] = (uint8_t)((v >> 8) & 0xFF);
  p[2] = (uint8_t)((v >> 16) & 0xFF);
  p[3] = (uint8_t)((v >> 24) & 0xFF);
}
static uint64_t pad_to(uint64_t n, uint64_t a) { return (n + a - 1) / a * a; }

/* ---- packer --------------------------------------------------------------- */

/* Byte length of one channel record for channel `ch` of a dense row: the 3 header
 * bytes plus, for every run of consecutive recorded strips, 2 header bytes and one
 * ADC byte per strip.  A run never crosses the APV boundary at strip 128. */
static uint32_t channel_record_len(const uint8_t* rec_row) {
  uint32_t len = ORC_CH_HEADER_BYTES;
  int s = 0;
  while (s < ORC_STRIPS_PER_CH) {
    if (!rec_row[s]) {
      s++;
      continue;
    }
    int apv_end = (s / ORC_STRIPS_PER_APV + 1) * ORC_STRIPS_PER_APV;
    int e = s;
    while (e < apv_end && rec_row[e]) e++;
    len += 2u + (uint32_t)(e - s);
    s = e;
  }
  return len;
}

static uint8_t* write_channel_record(uint8_t* out, const uint8_t* adc_row, const uint8_t* rec_row) {
  uint32_t len = channel_record_len(rec_row);
  wr_u16(out, len);
  out[2] = (uint8_t)ORC_ZS_CODE;
  uint8_t* p = out + ORC_CH_HEADER_BYTES;
  int s = 0;
  while (s < ORC_STRIPS_PER_CH) {
    if (!rec_row[s]) {
      s++;
      continue;
    }
    int apv_end = (s / ORC_STRIPS_PER_APV + 1) * ORC_STRIPS_PER_APV;
    int e = s;
    while (e < apv_end && rec_row[e]) e++;
    *p++ = (uint8_t)s;
    *p++ = (uint8_t)(e - s);
    for (int k = s; k < e; k++) *p++ = adc_row[k];
    s = e;
  }
  return p;
}

int64_t orc_pack_event(const uint8_t* adc, const uint8_t* recorded, uint32_t n_feds,
                       uint8_t* out, uint64_t cap, uint32_t* fed_len) {
  uint64_t pos = 0;
  for (uint32_t f = 0; f < n_feds; f++) {
    uint32_t fe_len[ORC_FE_PER_FED];
    uint64_t body = 0;
    for (int u = 0; u < ORC_FE_PER_FED; u++) {
      uint32_t l = 0;
      for (int k = 0; k < ORC_CH_PER_FE; k++) {
        uint64_t ch = (uint64_t)f * ORC_CH_PER_FED + (uint64_t)(u * ORC_CH_PER_FE + k);
        l += channel_record_len(recorded + ch * ORC_STRIPS_PER_CH);
      }
      fe_len[u] = l;
      body += pad_to(l, 8);
    }
    uint64_t total = pad_to(ORC_FED_HEADER_BYTES + body, 16);
    if (pos + total > cap) return -1;
    uint8_t* fed = out + pos;
    memset(fed, 0, (size_t)total);
    wr_u32(fed + 0, ORC_FED_MAGIC);
    wr_u16(fed + 4, f);
    fed[6] = (uint8_t)ORC_CH_PER_FED;
    fed[7] = (uint8_t)ORC_FE_PER_FED;
    wr_u32(fed + 8, (uint32_t)total);
    wr_u32(fed + 12, 0);
    for (int u = 0; u < ORC_FE_PER_FED; u++) wr_u16(fed + 16 + 2 * u, fe_len[u]);
    uint8_t* fe = fed + ORC_FED_HEADER_BYTES;
    for (int u = 0; u < ORC_FE_PER_FED; u++) {
      uint8_t* p = fe;
      for (int k = 0; k < ORC_CH_PER_FE; k++) {
        uint64_t ch = (uint64_t)f * ORC_CH_PER_FED + (uint64_t)(u * ORC_CH_PER_FE + k);
        p = write_channel_record(p, adc + ch * ORC_STRIPS_PER_CH, recorded + ch * ORC_STRIPS_PER_CH);
      }
      fe += pad_to(fe_len[u], 8);
    }
    fed_len[f] = (uint32_t)total;
    pos += total;
  }
  return (int64_t)pos;
}

/* ---- unpacker ------------------------------------------------------------- */

/* Checks one channel record [rec, rec+len) and, when it is valid, appends its
 * digis.  Returns the status bit of the first error found (0 when valid).  A
 * channel with an error contributes no digis. */
static uint8_t unpack_channel(const uint8_t* rec, uint32_t len, uint32_t ch_global,
                              uint32_t* strip, uint8_t* adc, uint64_t* n, uint64_t cap,
                              int* overflow) {
  if (rec[2] != ORC_ZS_CODE) return ORC_ST_BAD_CODE;
  /* First pass: validate every run before emitting anything. */
  uint32_t p = ORC_CH_HEADER_BYTES;
  uint32_t prev_end = 0;
  while (p < len) {
    if (p + 2 > len) return ORC_ST_TRUNC;
    uint32_t first = rec[p];
    uint32_t width = rec[p + 1];
    if (width == 0 || first + width > ORC_STRIPS_PER_CH) return ORC_ST_RUN_RANGE;
    if (first < prev_end) return ORC_ST_RUN_ORDER;
    if (p + 2 + width > len) return ORC_ST_TRUNC;
    prev_end = first + width;
    p += 2 + width;
  }
  /* Second pass: emit (strip, adc) for every recorded strip, in strip order. */
  p = ORC_CH_HEADER_BYTES;
  while (p < len) {
    uint32_t first = rec[p];
    uint32_t width = rec[p + 1];
    for (uint32_t k = 0; k < width; k++) {
      if (*n >= cap) {
        *overflow = 1;
        return 0;
      }
      strip[*n] = ch_global * ORC_STRIPS_PER_CH + first + k;
      adc[*n] = rec[p + 2 + k];
      (*n)++;
    }
    p += 2 + width;
  }
  return 0;
}

int64_t orc_unpack_event(const uint8_t* raw, const uint32_t* fed_len, uint32_t n_feds,
                         uint32_t* strip, uint8_t* adc, uint64_t cap, uint32_t* chan_off,
                         uint8_t* chan_status) {
  return orc_unpack_feds(raw, fed_len, 0, n_feds, strip, adc, cap, chan_off, chan_status);
}

int64_t orc_unpack_feds(const uint8_t* raw, const uint32_t* fed_len, uint32_t fed_base, uint32_t n_feds,
                        uint32_t* strip, uint8_t* adc, uint64_t cap, uint32_t* chan_off,
                        uint8_t* chan_status) {
  uint64_t n = 0;
  uint64_t fed_pos = 0;
  int overflow = 0;
  for (uint32_t f = 0; f < n_feds; f++) {
    const uint8_t* fed = raw + fed_pos;
    uint32_t L = fed_len[f];
    fed_pos += L;
    uint32_t ch0 = f * ORC_CH_PER_FED;

    uint8_t fed_status = 0;
    uint32_t fe_len[ORC_FE_PER_FED];
    if (L == 0) {
      /* FED absent from this event: its channels are empty and valid. */
      for (int c = 0; c < ORC_CH_PER_FED; c++) {
        chan_off[ch0 + c] = (uint32_t)n;
        chan_status[ch0 + c] = 0;
      }
      continue;
    }
    if (L < ORC_FED_HEADER_BYTES) {
      fed_status = ORC_ST_FED_HDR;
    } else {
      uint64_t body = 0;
      for (int u = 0; u < ORC_FE_PER_FED; u++) {
        fe_len[u] = rd_u16(fed + 16 + 2 * u);
        body += pad_to(fe_len[u], 8);
      }
      if (rd_u32(fed) != ORC_FED_MAGIC || rd_u16(fed + 4) != fed_base + f || fed[6] != ORC_CH_PER_FED ||
          fed[7] != ORC_FE_PER_FED || rd_u32(fed + 8) != L ||
          pad_to(ORC_FED_HEADER_BYTES + body, 16) != L)
        fed_status = ORC_ST_FED_HDR;
    }
    if (fed_status) {
      for (int c = 0; c < ORC_CH_PER_FED; c++) {
        chan_off[ch0 + c] = (uint32_t)n;
        chan_status[ch0 + c] = fed_status;
      }
      continue;
    }

    uint64_t fe_start = ORC_FED_HEADER_BYTES;
    for (int u = 0; u < ORC_FE_PER_FED; u++) {
      /* Walk the 12 channel lengths of this FE unit.  Any inconsistency (a length
       * below the 3 header bytes, a record crossing the FE end, or bytes left over
       * after the 12th record) invalidates the framing of the whole FE unit. */
      uint64_t fe_end = fe_start + fe_len[u];
      uint32_t rec_pos[ORC_CH_PER_FE];
      uint32_t rec_len[ORC_CH_PER_FE];
      int framing_ok = 1;
      uint64_t p = fe_start;
      for (int k = 0; k < ORC_CH_PER_FE; k++) {
        if (p + 2 > fe_end) {
          framing_ok = 0;
          break;
        }
        uint32_t len = rd_u16(fed + p);
        if (len < ORC_CH_HEADER_BYTES || p + len > fe_end) {
          framing_ok = 0;
          break;
        }
        rec_pos[k] = (uint32_t)p;
        rec_len[k] = len;
        p += len;
      }
      if (framing_ok && p != fe_end) framing_ok = 0;

      for (int k = 0; k < ORC_CH_PER_FE; k++) {
        uint32_t c = ch0 + (uint32_t)(u * ORC_CH_PER_FE + k);
        chan_off[c] = (uint32_t)n;
        if (!framing_ok) {
          chan_status[c] = ORC_ST_FRAMING;
          continue;
        }
        uint64_t n_before = n;
        uint8_t st = unpack_channel(fed + rec_pos[k], rec_len[k], fed_base * ORC_CH_PER_FED + c, strip, adc, &n,
                                    cap, &overflow);
        if (overflow) return -1;
        if (st) n = n_before;
        chan_status[c] = st;
      }
      fe_start += pad_to(fe_len[u], 8);
    }
  }
  chan_off[(uint64_t)n_feds * ORC_CH_PER_FED] = (uint32_t)n;
  return (int64_t)n;
}

/* ---- three-threshold predicates (section 2) ------------------------------ */

/* "Larger than" is read as strict.  The product threshold * noise is rounded
 * once to binary32, and the integer ADC is compared with it exactly. */
int orc_is_active(uint8_t adc, float noise, uint8_t bad, const orc_params* p) {
  if (bad) return 0;
  float limit = p->t_channel * noise;
  return (float)adc > limit;
}

int orc_is_seed(uint8_t adc, float noise, uint8_t bad, const orc_params* p) {
  if (bad) return 0;
  float limit = p->t_seed * noise;
  return (float)adc > limit;
}

/* Cluster threshold: the summed raw ADC of the active strips must exceed
 * t_cluster times the quadrature sum of their noise. */
int orc_passes_cluster(uint32_t s_raw, float n2, const orc_params* p) {
  float limit = p->t_cluster * sqrtf(n2);
  return (float)s_raw > limit;
}

/* Gain correction: the saturation codes 254 and 255 pass through; any other
 * ADC is divided by its APV gain, rounded half up, and capped at 254. */
uint32_t orc_corrected_charge(uint8_t adc, float gain) {
  if (adc >= 254) return adc;
  float x = (float)adc / gain;
  float y = x + 0.5f;
  int c = (int)y;
  if (c > 253) return 254;
  return (uint32_t)c;
}

/* ---- clustering of one module --------------------------------------------- */

/* Two successive active strips a < b are linked when every maximal run of holes
 * (non-bad inactive strips) strictly between them is at most max_seq_holes long
 * and every maximal run of bad strips between them is at most max_seq_bad long. */
static int linked(int a, int b, const uint8_t* bad, const orc_params* p) {
  int holes = 0, bads = 0;
  for (int t = a + 1; t < b; t++) {
    if (bad[t]) {
      bads++;
      holes = 0;
      if (bads > p->max_seq_bad) return 0;
    } else {
      holes++;
      bads = 0;
      if (holes > p->max_seq_holes) return 0;
    }
  }
  return 1;
}

typedef struct {
  const uint8_t* adc;
  const float* noise;
  const uint8_t* bad;
  const float* gain;
  const uint8_t* active;
  int n;
  const orc_params* p;
  uint16_t* first;
  uint16_t* width;
  uint32_t* charge;
  float* barycenter;
  int cap;
  int count;
  int overflow;
} module_ctx;

/* Finishes the candidate [l, r]: keep it only when it holds a seed and passes
 * the cluster threshold; report first strip, width, corrected charge and the
 * charge-weighted centroid. */
static void finish_candidate(module_ctx* m, int l, int r, int has_seed) {
  if (!has_seed) return;
  const orc_params* p = m->p;

  /* Extend over up to max_adj_bad bad strips directly outside each end. */
  int lo = l, hi = r;
  for (int k = 0; k < p->max_adj_bad && lo - 1 >= 0 && m->bad[lo - 1]; k++) lo--;
  for (int k = 0; k < p->max_adj_bad && hi + 1 < m->n && m->bad[hi + 1]; k++) hi++;

  /* Raw ADC sum and noise quadrature sum over the active strips, strictly
   * left to right. */
  uint32_t s_raw = 0;
  float n2 = 0.0f;
  for (int i = l; i <= r; i++) {
    if (!m->active[i]) continue;
    s_raw += m->adc[i];
    float sq = m->noise[i] * m->noise[i];
    n2 = n2 + sq;
  }
  if (!orc_passes_cluster(s_raw, n2, p)) return;

  /* Gain-corrected charge and first moment about the first strip. */
  uint32_t q_sum = 0;
  uint32_t moment = 0;
  for (int i = l; i <= r; i++) {
    if (!m->active[i]) continue;
    uint32_t q = orc_corrected_charge(m->adc[i], m->gain[i]);
    q_sum += q;
    moment += (uint32_t)(i - lo) * q;
  }
  float bary;
  int w = hi - lo + 1;
  if (q_sum == 0) {
    bary = (float)lo + 0.5f * (float)w;
  } else {
    float centre = (float)lo + 0.5f;
    float offset = (float)moment / (float)q_sum;
    bary = centre + offset;
  }

  if (m->count >= m->cap) {
    m->overflow = 1;
    return;
  }
  m->first[m->count] = (uint16_t)lo;
  m->width[m->count] = (uint16_t)w;
  m->charge[m->count] = q_sum;
  m->barycenter[m->count] = bary;
  m->count++;
}

int orc_cluster_module(const uint8_t* adc, const float* noise, const uint8_t* bad,
                       const float* gain, int n, const orc_params* p, uint16_t* first,
                       uint16_t* width, uint32_t* charge, float* barycenter, int cap) {
  uint8_t active[ORC_STRIPS_PER_CH];
  uint8_t seed[ORC_STRIPS_PER_CH];
  if (n < 0 || n > ORC_STRIPS_PER_CH) return -1;
  for (int i = 0; i < n; i++) {
    active[i] = (uint8_t)orc_is_active(adc[i], noise[i], bad[i], p);
    seed[i] = (uint8_t)orc_is_seed(adc[i], noise[i], bad[i], p);
  }

  module_ctx m = {adc, noise, bad, gain, active, n, p, first, width, charge, barycenter, cap, 0, 0};

  /* Candidates are the maximal chains of linked active strips, found in one
   * left-to-right pass. */
  int open = 0, l = 0, last = 0, has_seed = 0;
  for (int s = 0; s < n; s++) {
    if (!active[s]) continue;
    if (open && linked(last, s, bad, p)) {
      last = s;
      has_seed |= seed[s];
    } else {
      if (open) finish_candidate(&m, l, last, has_seed);
      open = 1;
      l = s;
      last = s;
      has_seed = seed[s];
    }
  }
  if (open) finish_candidate(&m, l, last, has_seed);
  return m.overflow ? -1 : m.count;
}

/* ---- clustering of an event ----------------------------------------------- */

int64_t orc_cluster_event(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off,
                          uint32_t n_feds, const float* noise, const float* gain,
                          const uint8_t* bad, const orc_params* p, uint32_t* det,
                          uint16_t* first, uint16_t* width, uint32_t* charge,
                          float* barycenter, uint64_t cap) {
  return orc_cluster_feds(strip, adc, chan_off, 0, n_feds, noise, gain, bad, p, det, first, width, charge, barycenter,
                          cap);
}

int64_t orc_cluster_feds(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off, uint32_t fed_base,
                         uint32_t n_feds, const float* noise, const float* gain, const uint8_t* bad,
                         const orc_params* p, uint32_t* det, uint16_t* first, uint16_t* width, uint32_t* charge,
                         float* barycenter, uint64_t cap) {
  uint64_t out = 0;
  uint32_t n_ch = n_feds * ORC_CH_PER_FED;
  uint8_t row_adc[ORC_STRIPS_PER_CH];
  float row_gain[ORC_STRIPS_PER_CH];
  uint16_t f_first[ORC_STRIPS_PER_CH], f_width[ORC_STRIPS_PER_CH];
  uint32_t f_charge[ORC_STRIPS_PER_CH];
  float f_bary[ORC_STRIPS_PER_CH];
  for (uint32_t c = 0; c < n_ch; c++) {
    uint32_t d0 = chan_off[c], d1 = chan_off[c + 1];
    if (d0 == d1) continue; /* no recorded strip: no active strip, no cluster */
    uint64_t g0 = ((uint64_t)fed_base * ORC_CH_PER_FED + c) * ORC_STRIPS_PER_CH;
    memset(row_adc, 0, sizeof row_adc);
    for (uint32_t d = d0; d < d1; d++) row_adc[strip[d] - g0] = adc[d];
    for (int i = 0; i < ORC_STRIPS_PER_CH; i++)
      row_gain[i] = gain[(g0 + (uint64_t)i) / ORC_STRIPS_PER_APV];
    int k = orc_cluster_module(row_adc, noise + g0, bad + g0, row_gain, ORC_STRIPS_PER_CH, p,
                               f_first, f_width, f_charge, f_bary, ORC_STRIPS_PER_CH);
    if (k < 0) return -1;
    if (out + (uint64_t)k > cap) return -1;
    for (int j = 0; j < k; j++) {
      det[out] = fed_base * ORC_CH_PER_FED + c;
      first[out] = f_first[j];
      width[out] = f_width[j];
      charge[out] = f_charge[j];
      barycenter[out] = f_bary[j];
      out++;
    }
  }
  return (int64_t)out;
}

/* ---- per-strip amplitudes of clusters --------------------------------------- */

int64_t orc_cluster_amplitudes(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off,
                               const float* noise, const float* gain, const uint8_t* bad,
                               const orc_params* p, const uint32_t* det, const uint16_t* first,
                               const uint16_t* width, uint64_t n_clusters, uint32_t* amp_first,
                               uint8_t* amp, uint64_t cap) {
  uint64_t out = 0;
  uint8_t row_adc[ORC_STRIPS_PER_CH];
  for (uint64_t k = 0; k < n_clusters; k++) {
    uint32_t c = det[k];
    uint64_t g0 = (uint64_t)c * ORC_STRIPS_PER_CH;
    /* the module's ADC row: recorded strips from the digis, 0 elsewhere */
    memset(row_adc, 0, sizeof row_adc);
    for (uint32_t d = chan_off[c]; d < chan_off[c + 1]; d++) row_adc[strip[d] - g0] = adc[d];
    if (first[k] + width[k] > ORC_STRIPS_PER_CH) return -1;
    if (out + width[k] > cap) return -1;
    amp_first[k] = (uint32_t)out;
    for (int i = 0; i < width[k]; i++) {
      int s = first[k] + i;
      uint64_t g = g0 + (uint64_t)s;
      int act = orc_is_active(row_adc[s], noise[g], bad[g], p);
      amp[out++] = act ? (uint8_t)orc_corrected_charge(row_adc[s], gain[g / ORC_STRIPS_PER_APV]) : 0;
    }
  }
  return (int64_t)out;
}

/* ---- local positions ------------------------------------------------------- */

void orc_local_x(const uint32_t* det, const float* barycenter, uint64_t n, const float* pitch, float* x) {
  for (uint64_t k = 0; k < n; k++) {
    float from_centre = barycenter[k] - 128.0f;
    x[k] = from_centre * pitch[det[k]];
  }
}
