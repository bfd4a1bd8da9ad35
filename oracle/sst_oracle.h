/*
 * sst_oracle.h -- plain sequential CPU oracle for silicon-strip unpacking and
 * three-threshold clustering (arXiv 2101.11489, section 2 "Parallelization").
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to prove the CUDA path right.
 * Only the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it; the product library never includes, links or calls it, and it
 * includes nothing from the product.  It restates the byte format and the
 * clustering rules on its own, so that a mistake in one side does not hide in
 * shared code.
 *
 * Everything here is sequential and unoptimised on purpose: one FED, one FE unit,
 * one channel, one strip at a time, in the order the definitions are written.
 */
#ifndef SST_ORACLE_H
#define SST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Geometry of the readout (section 2: a FED has 96 optical channels of 256 strips;
 * a module is one 256-strip channel; an APV reads 128 strips). */
#define ORC_CH_PER_FED 96
#define ORC_STRIPS_PER_CH 256
#define ORC_FE_PER_FED 8
#define ORC_CH_PER_FE 12
#define ORC_STRIPS_PER_APV 128

/* Byte format (the paper's Figure 1 is lost; this is the format this project
 * defines for the zero-suppressed, CSR-like payload the paper describes). */
#define ORC_FED_HEADER_BYTES 32
#define ORC_FED_MAGIC 0x46545353u /* bytes 'S','S','T','F' */
#define ORC_ZS_CODE 0x5Au
#define ORC_CH_HEADER_BYTES 3

/* Channel status bits (one bit per invalid channel: the first error found). */
#define ORC_ST_FED_HDR 0x01u   /* FED header or FED length invalid */
#define ORC_ST_FRAMING 0x02u   /* channel lengths inconsistent in the FE unit */
#define ORC_ST_BAD_CODE 0x04u  /* unknown packet code */
#define ORC_ST_RUN_RANGE 0x08u /* width 0 or first + width > 256 */
#define ORC_ST_RUN_ORDER 0x10u /* run starts before the previous run ends */
#define ORC_ST_TRUNC 0x20u     /* run header or ADC bytes cross the channel end */

typedef struct {
  float t_channel;   /* channel threshold, in units of noise */
  float t_seed;      /* seed threshold, in units of noise */
  float t_cluster;   /* cluster threshold, in units of sqrt(sum noise^2) */
  int max_seq_holes; /* longest run of non-bad inactive strips allowed in a gap */
  int max_seq_bad;   /* longest run of bad strips allowed in a gap */
  int max_adj_bad;   /* bad strips added to each end of a cluster */
} orc_params;

/* Canonical packer: dense per-strip ADC plus a "recorded" mask (the front end's
 * zero suppression already applied) for FEDs 0..n_feds-1 -> raw FED records.
 * Returns the number of bytes written, or -1 when `cap` is too small. */
int64_t orc_pack_event(const uint8_t* adc, const uint8_t* recorded, uint32_t n_feds,
                       uint8_t* out, uint64_t cap, uint32_t* fed_len);

/* Unpacker: raw FED records (FED f at the running sum of fed_len) -> digis in
 * ascending global strip order g = (f*96 + ch)*256 + strip, CSR row pointers per
 * channel (chan_off[n_feds*96 + 1]) and one status byte per channel.
 * Returns the number of digis, or -1 when `cap` is too small. */
int64_t orc_unpack_event(const uint8_t* raw, const uint32_t* fed_len, uint32_t n_feds,
                         uint32_t* strip, uint8_t* adc, uint64_t cap, uint32_t* chan_off,
                         uint8_t* chan_status);

/* Clusterizer for one module of n strips (n <= 256).  adc[i] = 0 for strips that
 * were not recorded; gain[i] is the gain of strip i's APV.  Writes clusters in
 * strip order.  Returns their number, or -1 when `cap` is too small. */
int orc_cluster_module(const uint8_t* adc, const float* noise, const uint8_t* bad,
                       const float* gain, int n, const orc_params* p, uint16_t* first,
                       uint16_t* width, uint32_t* charge, float* barycenter, int cap);

/* Clusterizer for a whole event given its digis (as orc_unpack_event writes
 * them).  Calibration is indexed by global strip (noise, bad) and by global APV
 * (gain).  det[k] is the global module (channel) id.  Returns the number of
 * clusters, or -1 when `cap` is too small. */
/* The same for FEDs fed_base .. fed_base + n_feds - 1 of an event only (their
 * records back to back in `raw`, their lengths in fed_len[0 .. n_feds)): FED ids
 * in the headers, strip indices, module ids (det) and calibration indices are the
 * event's, channel arrays (chan_off, chan_status) are the range's.  Clusters
 * never cross a FED, so an event can be processed as independent FED ranges. */
int64_t orc_unpack_feds(const uint8_t* raw, const uint32_t* fed_len, uint32_t fed_base, uint32_t n_feds,
                        uint32_t* strip, uint8_t* adc, uint64_t cap, uint32_t* chan_off, uint8_t* chan_status);
int64_t orc_cluster_feds(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off, uint32_t fed_base,
                         uint32_t n_feds, const float* noise, const float* gain, const uint8_t* bad,
                         const orc_params* p, uint32_t* det, uint16_t* first, uint16_t* width, uint32_t* charge,
                         float* barycenter, uint64_t cap);

int64_t orc_cluster_event(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off,
                          uint32_t n_feds, const float* noise, const float* gain,
                          const uint8_t* bad, const orc_params* p, uint32_t* det,
                          uint16_t* first, uint16_t* width, uint32_t* charge,
                          float* barycenter, uint64_t cap);

/* The three threshold predicates, exposed for the pins (section 2). */
/* Optional per-strip amplitudes of clusters (section 2: a kept cluster reports
 * its boundaries, centroid "and optionally ADC values").  For cluster k (module
 * det[k], strips first[k] .. first[k] + width[k] - 1), the amplitude of a strip
 * is its gain-corrected charge (orc_corrected_charge) when the strip is active,
 * and 0 otherwise (a hole, a bad strip inside the cluster or a bad strip it was
 * widened over).  Clusters' amplitudes are written back to back:
 * amp_first[k] = sum of width[j] for j < k.  The digis and calibration are those
 * given to orc_cluster_event.  Returns the number of amplitudes written, or -1
 * when `cap` is too small. */
int64_t orc_cluster_amplitudes(const uint32_t* strip, const uint8_t* adc, const uint32_t* chan_off,
                               const float* noise, const float* gain, const uint8_t* bad,
                               const orc_params* p, const uint32_t* det, const uint16_t* first,
                               const uint16_t* width, uint64_t n_clusters, uint32_t* amp_first,
                               uint8_t* amp, uint64_t cap);

/* Local position of clusters on their module (CMS-style local x, here with a
 * synthetic per-module strip pitch; arXiv 2101.11489 section 4: the clusters are
 * turned into hits with positions for tracking).  The origin is the module's
 * centre, between strips 127 and 128, so x = (barycenter - 128) * pitch[det]:
 * one binary32 subtraction, then one binary32 multiplication. */
void orc_local_x(const uint32_t* det, const float* barycenter, uint64_t n, const float* pitch, float* x);

int orc_is_active(uint8_t adc, float noise, uint8_t bad, const orc_params* p);
int orc_is_seed(uint8_t adc, float noise, uint8_t bad, const orc_params* p);
int orc_passes_cluster(uint32_t s_raw, float n2, const orc_params* p);

/* Gain-corrected per-strip charge. */
uint32_t orc_corrected_charge(uint8_t adc, float gain);

#ifdef __cplusplus
}
#endif
#endif
