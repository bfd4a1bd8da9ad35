/*
 * sst.h -- C ABI of the GB300 silicon-strip unpacking and clustering library.
 *
 * The library implements the hot path of arXiv 2101.11489 ("Parallelizing the
 * Unpacking and Clustering of Detector Data for Reconstruction of Charged Particle
 * Tracks on Multi-core CPUs and Many-core GPUs"), section 2 "Parallelization":
 *   (1) unpack zero-suppressed FED raw data (96 channels x 256 strips per FED, a
 *       CSR-like layout with the channel as row and the strip as column) into a
 *       structure-of-arrays of digis, concurrently per channel;
 *   (2) cluster the digis with the "three thresholds" algorithm: channel threshold
 *       (active strips), seed threshold (seed strips), cluster forming around the
 *       seeds (left and right boundaries, charge) and the cluster threshold; kept
 *       clusters report boundaries, charge and centroid;
 * and section 3 "Optimization": many events processed concurrently on one GPU.
 *
 * Every entry point returns an sst_status.  Calls that take a `stream` enqueue
 * work on that CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 * stream) and return without waiting; their device outputs are valid once the
 * stream reaches that point.  Data errors in the raw buffers are NOT call errors:
 * they are reported per channel and per event in device status words (see
 * sst_event_status) and never make a kernel fault or trap.
 *
 * Ownership: inputs are owned by the caller and only read; the library copies
 * what it keeps (calibration).  Output buffers are owned by the caller.  A context
 * owns its device calibration tables and its internal scratch (look-back flags,
 * work tickets), which it sizes on first use; a call that has to grow scratch
 * synchronises the device, so make one warm-up call before capturing a stream
 * into a CUDA graph.  Contexts are independent; one context must not be used from
 * two host threads at once, except sst_submit / sst_poll, which are thread safe.
 */
#ifndef SST_H
#define SST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
typedef int32_t sst_status;
#define SST_OK 0
#define SST_ERR_INVALID_ARG 1 /* null pointer, bad size, bad alignment, bad parameter */
#define SST_ERR_NO_CALIB 2    /* sst_calib_upload has not been called */
#define SST_ERR_BUDGET 3      /* served: event does not fit the free budget now; retry */
#define SST_ERR_TOO_LARGE 4   /* served: event can never fit the budget / limits */
#define SST_ERR_BUSY 5        /* served: no free request slot; retry */
#define SST_ERR_NOT_READY 6   /* served: result not ready within the timeout */
#define SST_ERR_TIMEOUT 7     /* a device wait ran out of iterations (see flags) */
#define SST_ERR_CUDA 8        /* CUDA runtime error; text in sst_last_error() */
#define SST_ERR_STATE 9       /* call not valid in the context's current state */

/* ---- readout geometry (section 2) ----------------------------------------- */
#define SST_CH_PER_FED 96
#define SST_STRIPS_PER_CH 256 /* a module is one 256-strip channel */
#define SST_FE_PER_FED 8
#define SST_CH_PER_FE 12
#define SST_STRIPS_PER_APV 128

/* ---- FED byte format -------------------------------------------------------
 * The paper's Figure 1 (raw data format) is lost; section 2 states only the
 * geometry and that the zero-suppressed payload is CSR-like.  This library reads
 * the following little-endian format:
 *
 *   event  = FED record 0, FED record 1, ... back to back; FED f occupies
 *            fed_len[f] bytes (0 = FED absent: its channels are empty).
 *   FED    = 32-byte header | FE unit 0 | ... | FE unit 7 | zero padding to 16 B
 *   header = u32 magic (SST_FED_MAGIC) | u16 fed_id (== f) | u8 96 | u8 8 |
 *            u32 fed_bytes (== fed_len[f]) | u32 reserved | u16 fe_len[8]
 *   FE u   = 12 channel records back to back (fe_len[u] bytes), zero padding to 8 B
 *   channel record = u16 len (incl. these 3 bytes) | u8 packet code (SST_ZS_CODE) |
 *            runs: u8 first strip | u8 width (>= 1) | width x u8 ADC
 *            runs ascend and do not overlap (first >= previous first + width),
 *            first + width <= 256.
 * Global strip index of a digi: g = (fed * 96 + channel) * 256 + strip.
 */
#define SST_FED_HEADER_BYTES 32
#define SST_FED_MAGIC 0x46545353u /* bytes 'S','S','T','F' */
#define SST_ZS_CODE 0x5Au
#define SST_MAX_FEDS 65536u

/* ---- data status ------------------------------------------------------------
 * Each channel gets one status byte: 0 when valid, otherwise the bit of the first
 * error found.  An invalid channel yields no digis; its neighbours are unaffected,
 * except that a broken length chain invalidates all 12 channels of its FE unit and
 * a bad FED header all 96 channels of the FED. */
#define SST_CH_FED_HDR 0x01u   /* FED header / fed_len / FE lengths inconsistent */
#define SST_CH_FRAMING 0x02u   /* channel lengths inconsistent within the FE unit */
#define SST_CH_BAD_CODE 0x04u  /* packet code is not SST_ZS_CODE */
#define SST_CH_RUN_RANGE 0x08u /* run width 0, or first + width > 256 */
#define SST_CH_RUN_ORDER 0x10u /* run starts before the previous run ends */
#define SST_CH_TRUNC 0x20u     /* run header or ADC bytes cross the record end */
/* Event-level flags (ORed with the channel bits into sst_event_status.flags). */
#define SST_EV_DIGI_CAPACITY 0x100u    /* digi output capacity exceeded; digis dropped */
#define SST_EV_CLUSTER_CAPACITY 0x200u /* cluster output capacity exceeded; clusters dropped */
#define SST_EV_TIMEOUT 0x400u          /* a device wait gave up; the event's output is invalid */
#define SST_EV_SIZE 0x800u             /* batch: sum of fed_len != event_off[e+1] - event_off[e] */
#define SST_EV_AMP_CAPACITY 0x1000u    /* amplitude capacity exceeded; some clusters have no amplitudes */

/* Per-event status record, in device memory. */
typedef struct {
  uint32_t n_digi;         /* digis found (valid channels only) */
  uint32_t n_clusters;     /* clusters written (<= capacity) */
  uint32_t flags;          /* OR of channel status bits and SST_EV_* flags */
  uint32_t n_bad_channels; /* channels with a nonzero status */
} sst_event_status;

/* ---- clustering parameters (section 2, "three thresholds") ------------------
 * active(s)  = !bad[s] && (float)adc[s] > t_channel * noise[s]
 * seed(s)    = !bad[s] && (float)adc[s] > t_seed    * noise[s]
 * Two successive active strips are linked when every maximal run of non-bad
 * inactive strips between them is <= max_seq_holes long and every maximal run of
 * bad strips between them is <= max_seq_bad long.  A candidate is a maximal chain
 * of linked active strips; it is a cluster when it holds a seed and
 *   (float)sum(adc) > t_cluster * sqrt(sum noise^2)      (active strips only)
 * and it is then widened by up to max_adj_bad bad strips on each side.  Every
 * product, sum, quotient and square root is one binary32 operation rounded to
 * nearest, in strip order; "larger than" is strict.
 * Requirements: 0 < t_channel <= t_seed, t_cluster >= 0, all finite. */
typedef struct {
  float t_channel;
  float t_seed;
  float t_cluster;
  uint8_t max_seq_holes;
  uint8_t max_seq_bad;
  uint8_t max_adj_bad;
  uint8_t reserved; /* must be 0 */
} sst_params;

/* ---- outputs ---------------------------------------------------------------- */

/* Digi structure-of-arrays of one event (device memory, caller-owned).
 * Digis are in ascending global strip order; the digis of channel c are
 * [chan_off[c], chan_off[c+1]).  n_digi <= total raw bytes always holds (each
 * digi costs one payload byte), so capacity = raw bytes is always enough. */
typedef struct {
  uint32_t* strip;          /* [capacity] global strip index g */
  uint8_t* adc;             /* [capacity] 8-bit ADC */
  uint32_t* chan_off;       /* [n_feds*96 + 1] CSR row pointers */
  uint8_t* chan_status;     /* [n_feds*96] channel status byte */
  sst_event_status* status; /* [1] sst_unpack resets it and sets n_digi, flags, n_bad_channels */
  uint64_t capacity;        /* elements of strip[] and adc[] */
} sst_digis;

/* Cluster structure-of-arrays (device memory, caller-owned), sorted by
 * (det, first).  det = global module id = fed * 96 + channel; first = first strip
 * in the module; width in strips; charge = sum of gain-corrected ADC; barycenter =
 * charge-weighted centroid in module strip units (strip i spans [i, i+1)). */
typedef struct {
  uint32_t* det;
  uint16_t* first;
  uint16_t* width;
  uint32_t* charge;
  float* barycenter;
  uint64_t capacity; /* elements of each array; also sizes the context's staging scratch */
  /* Optional per-strip amplitudes (section 2: a cluster reports its boundaries,
   * centroid "and optionally ADC values"); amp == NULL: none are produced.
   * sst_cluster, sst_batch and sst_batch_host produce them (the served path does
   * not: sst_poll returns clusters only).  The amplitude of each strip of a cluster is its
   * gain-corrected charge when the strip is active, else 0 (a hole, a bad strip
   * inside, a bad strip the cluster was widened over): cluster k's width[k]
   * amplitudes are amp[amp_first[k] ..].  Within an event they follow the
   * cluster order.  Amplitudes are allocated per work item (one FE unit per
   * warp in sst_cluster, two in the batched paths); when an item's amplitudes do not
   * fit, none of them is stored, its clusters get amp_first = 0xFFFFFFFF and the
   * event SST_EV_AMP_CAPACITY (the clusters themselves are unaffected). */
  uint8_t* amp;            /* [amp_capacity] */
  uint32_t* amp_first;     /* [capacity], absolute index into amp */
  const uint64_t* amp_off; /* sst_batch: [n_events + 1] device, sst_batch_host: [n_events + 1]
                              host; event e's amplitudes lie in [amp_off[e], amp_off[e+1])
                              (bounded by amp_capacity); sst_cluster: unused, the event has
                              [0, amp_capacity) */
  uint64_t amp_capacity;   /* bytes of amp; also sizes the context's amplitude staging */
} sst_clusters;

/* ---- context ------------------------------------------------------------------ */
typedef struct sst_ctx sst_ctx;

/* Creates a context on CUDA device `device` for a detector of n_feds FEDs
 * (section 2's readout geometry: FEDs of 96 channels of 256 strips; calibration
 * covers n_feds * 96 * 256 strips).  INVALID_ARG if n_feds is 0 or above
 * SST_MAX_FEDS; CUDA if the device cannot be used. */
sst_status sst_create(sst_ctx** out, int device, uint32_t n_feds);

/* Waits for the context's work, stops the server if running, frees everything
 * (the device memory section 3 keeps resident across events: calibration and
 * scratch). */
sst_status sst_destroy(sst_ctx* ctx);

/* Text of the last error on this context (static storage, never NULL). */
const char* sst_last_error(const sst_ctx* ctx);

/* Uploads calibration (section 2: pre-measured gain and noise per strip, plus the
 * bad-strip list) from HOST memory, in global strip order:
 *   noise [n_feds*96*256] float, finite, >= 0   (ADC counts)
 *   gain  [n_feds*96*2]   float, finite, > 0    (one per 128-strip APV)
 *   bad   [n_feds*96*256] uint8, 0 = good, else bad
 * and the thresholds.  The tables are copied to device memory and stay resident;
 * a new upload replaces them after work already queued on `stream`, and returns
 * once they are in place.  From the bad-strip flags and the hole / bad-strip
 * limits the device also builds a bit mask and, per strip, a linking limit from
 * the longest gap below it that still links two successive active strips (one
 * byte per strip), which the clusterizers read instead of walking each gap.
 * INVALID_ARG on a null pointer, a non-finite or negative value, or parameters
 * outside their requirements; the previous calibration then stays in place. */
sst_status sst_calib_upload(sst_ctx* ctx, const float* noise, const float* gain, const uint8_t* bad,
                            const sst_params* params, void* stream);

/* ---- per-event path ----------------------------------------------------------- */

/* Unpacks one event (section 2: "unpack the data to SoA format ... concurrently
 * for each channel").  raw: device pointer, 16-byte aligned, raw_bytes bytes: the
 * event's FED records back to back; fed_len: device pointer, [n_feds] bytes per
 * FED record (the event builder's sizes); a FED whose record would end past
 * raw_bytes is treated as corrupt (SST_CH_FED_HDR) and SST_EV_SIZE is set when the
 * sizes do not add up to raw_bytes.  Writes `out` (device).  1 <= n_feds <=
 * context FEDs.  Digis beyond out->capacity are dropped and flagged
 * SST_EV_DIGI_CAPACITY (chan_off is then clamped to the capacity).  Does not need
 * calibration. */
sst_status sst_unpack(sst_ctx* ctx, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                      uint32_t n_feds, const sst_digis* out, void* stream);

/* Clusters one event's digis (as sst_unpack wrote them, for n_feds FEDs) with the
 * three-threshold algorithm (section 2).  Writes the cluster SoA and sets
 * in->status->n_clusters.  When the event has more clusters than out->capacity,
 * SST_EV_CLUSTER_CAPACITY is ORed into in->status->flags and the arrays hold a
 * sorted subset of the event's clusters (those of whole FE units, in allocation
 * order).  NO_CALIB before sst_calib_upload. */
sst_status sst_cluster(sst_ctx* ctx, const sst_digis* in, uint32_t n_feds, const sst_clusters* out,
                       void* stream);

/* ---- per-event unpacking without allocation ------------------------------------
 * The paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory once they run (a trigger or DAQ process whose device
 * memory is reserved up front by its own allocator; code that must not let
 * cudaMalloc synchronise the device under a real-time pipeline).  It needs no
 * context: it unpacks exactly as sst_unpack does (same arguments, same outputs,
 * same status semantics), on the current CUDA device, with its scratch in a fixed
 * device array of the library (SST_NOALLOC_MAX_FEDS look-back states and FED
 * offsets, about 16 KiB per device, held until the process exits).  It calls no
 * cudaMalloc, cudaFree or allocating routine.
 *   - n_feds > SST_NOALLOC_MAX_FEDS returns SST_ERR_TOO_LARGE; a null pointer, a
 *     misaligned raw buffer or n_feds == 0 returns SST_ERR_INVALID_ARG; a CUDA
 *     error returns SST_ERR_CUDA.
 *   - The first call on a device looks up the array's device address on that
 *     device (cudaGetSymbolAddress); make that first call before capturing any
 *     stream.
 *   - All calls on a device share the one array: calls whose work overlaps on the
 *     GPU (different streams, not ordered) race and give wrong results.  Every call
 *     clears what must start at zero on its own stream before its kernels run. */
#define SST_NOALLOC_MAX_FEDS 1024u
sst_status sst_unpack_noalloc(const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len, uint32_t n_feds,
                              const sst_digis* out, void* stream);

/* ---- batched path (section 3: many events concurrently on one GPU) -------------- */

/* Unpacks and clusters n_events events in one persistent launch; digis stay on
 * chip.  Each warp takes two adjacent FE units at a time; their clusters are
 * staged (context scratch of out->capacity records), then ordered and copied per
 * event by one more kernel (two with amplitudes).  The launch sequence allocates nothing once the context
 * has run one batch of this size, so it can be captured in a CUDA graph.  All
 * pointers are device memory:
 *   raw        events back to back; event e occupies [event_off[e], event_off[e+1]),
 *              every event_off[e] a multiple of 16
 *   event_off  [n_events + 1] uint64
 *   fed_len    [n_events * n_feds] uint32, event-major
 *   clu_off    [n_events + 1] uint64: event e's clusters go to
 *              [clu_off[e], clu_off[e+1]) of out's arrays (capacity per event);
 *              clu_off[n_events] <= out->capacity
 *   status     [n_events] per-event status records
 * Output is identical, event by event, to sst_unpack + sst_cluster on each event
 * alone.  NO_CALIB before sst_calib_upload. */
sst_status sst_batch(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                     uint32_t n_events, uint32_t n_feds, const uint64_t* clu_off, const sst_clusters* out,
                     sst_event_status* status, void* stream);

/* The batched path for events in HOST memory (section 3: transfers overlapped
 * with computation on CUDA streams).  Same computation as sst_batch, but every
 * pointer is host memory and the call is synchronous: it returns when all
 * results are in the caller's arrays.  The batch is cut into chunks of
 * consecutive events; the host->device copy, the kernels and the device->host
 * copy of successive chunks overlap on the context's streams (by default 4, 16,
 * ..., 16, 8, 4 events: short first and last chunks; sst_tune.host_chunk_events
 * sets equal chunks, best with the batch size when several batches are in
 * flight through sst_batch_host_submit).
 *   raw, event_off, fed_len  as for sst_batch, in host memory; event_off need
 *              not start at 0 (only [event_off[0], event_off[n_events]) is read)
 *   out        host arrays of out->capacity records; the events' clusters are
 *              stored back to back in event order, each event's sorted as in
 *              sst_batch
 *   event_first [n_events + 1] uint64, written: event e's clusters are records
 *              [event_first[e], event_first[e] + status[e].n_clusters);
 *              event_first[n_events] = records stored
 *   status     [n_events], written (host)
 * Clusters beyond out->capacity are not stored: the events cut set
 * SST_EV_CLUSTER_CAPACITY and their n_clusters counts what was stored.
 * Pinned host memory (cudaHostAlloc, cudaHostRegister) gives full copy speed;
 * pageable memory works, with copies staged by the CUDA driver.  Device arenas
 * grow on demand (cudaMalloc only when a call needs more than any call before it
 * on the context) and are freed by sst_destroy.  Calls from several threads are
 * processed one batch after another, in the order they were made.
 * Amplitudes (out->amp set): out->amp, out->amp_first and out->amp_off are host
 * arrays with sst_batch's meaning (event e's amplitudes in its slice
 * [amp_off[e], amp_off[e+1]) of amp, amp_first absolute indices into amp); each
 * chunk's slices are copied back whole.
 * Errors: INVALID_ARG (null pointer, n_events == 0, n_feds outside 1..context
 * FEDs, decreasing event_off; with amplitudes: amp_first or amp_off null,
 * amp_off decreasing or past amp_capacity, amp_capacity 0 or >= 2^32 - 1),
 * NO_CALIB, CUDA. */
sst_status sst_batch_host(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                          uint32_t n_events, uint32_t n_feds, const sst_clusters* out, uint64_t* event_first,
                          sst_event_status* status);

/* The same batch, submitted without waiting: the call checks the arguments,
 * queues the batch on the context's host pipeline and returns a ticket.  Batches
 * are processed in submission order as one stream of chunks, so the copies and
 * kernels of a batch overlap the end of the one before it.  Every buffer of the
 * batch (inputs and outputs) belongs to the library until sst_batch_host_wait
 * returns for its ticket: do not modify the inputs or read the outputs before.
 * Do not change the context's tune while batches are pending.  Thread safe with
 * respect to each other (submit and wait may come from different threads).
 * sst_batch_host_wait: blocks until the batch's results are in the caller's
 * arrays and releases the ticket; INVALID_ARG for an unknown ticket, CUDA when the
 * batch (or one before it) failed. */
sst_status sst_batch_host_submit(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off,
                                 const uint32_t* fed_len, uint32_t n_events, uint32_t n_feds,
                                 const sst_clusters* out, uint64_t* event_first, sst_event_status* status,
                                 uint64_t* ticket);
sst_status sst_batch_host_wait(sst_ctx* ctx, uint64_t ticket);

/* ---- local positions (section 4: clusters become hits for tracking) --------------
 * The detector geometry is not available: the caller gives every module a strip
 * pitch (a synthetic geometry).  The local x of a cluster is measured from its
 * module's centre, between strips 127 and 128:
 *   x = (barycenter - 128) * pitch[det]     (binary32, each operation rounded once)
 * in the pitch's length unit.
 * sst_pitch_upload: pitch = host [n_feds * 96] floats, finite and > 0 (copied;
 *   INVALID_ARG otherwise).
 * sst_local_x: det, barycenter = device [n] (a cluster SoA), x = device [n] output;
 *   a det outside the context's modules gives NaN.  STATE before sst_pitch_upload.
 *   Enqueued on `stream`. */
sst_status sst_pitch_upload(sst_ctx* ctx, const float* pitch);
sst_status sst_local_x(sst_ctx* ctx, const uint32_t* det, const float* barycenter, uint64_t n, float* x,
                       void* stream);

/* Launch knobs (section 3: the paper tunes the number of events processed
 * concurrently; here the batched kernel's launch shape and work-item width and
 * the host path's batch depth are picked by measurement, sst_autotune and
 * sst_autotune_host). */
typedef struct {
  uint32_t block;             /* batched kernel: threads per CTA, 128 or 256 */
  uint32_t ctas_per_sm;       /* batched kernel: persistent CTAs per SM, 1..8 (clamped to what fits) */
  uint32_t units_per_warp;    /* batched kernel: FE units per warp work item, 1 or 2 (12 or 24 channels) */
  uint32_t host_chunk_events; /* sst_batch_host: events per pipeline chunk (the batch depth of each
                                 launch), 0..4096; 0 = automatic (a quarter of the batch, at most 32) */
  uint32_t tile_digis;        /* per-event unpack (sst_unpack): digis per on-chip tile, 1024, 2048 or 4096 */
  uint32_t lanes_per_channel; /* per-event unpack: lanes that copy one channel's runs: 1, 2, 4, 8, 16 or 32 */
} sst_tune;

/* Sets / reads the context's knobs.  INVALID_ARG for a value outside its range. */
sst_status sst_set_tune(sst_ctx* ctx, const sst_tune* t);
sst_status sst_get_tune(const sst_ctx* ctx, sst_tune* t);

/* Times every candidate shape of the batched kernel on the given batch (same
 * arguments as sst_batch; the outputs are overwritten): block 128 / 256 x work
 * items of 1 / 2 FE units x 2..8 CTAs per SM (shapes that cannot be resident, or
 * that the occupancy clamps to a shape already timed, are skipped).  Each shape
 * runs one untimed and two timed launch sequences.  Keeps the fastest in the
 * context and returns it in *best with its time per launch sequence in *best_us.
 * Synchronises the stream. */
sst_status sst_autotune(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                        uint32_t n_events, uint32_t n_feds, const uint64_t* clu_off, const sst_clusters* out,
                        sst_event_status* status, void* stream, sst_tune* best, float* best_us);

/* Times sst_batch_host on the given HOST batch (same arguments; outputs are
 * overwritten) for events per chunk of 0 (automatic), 4, 8, 16, 32, 64 and 128
 * (those not above n_events), two calls each after one untimed call, keeps the
 * fastest in the context's host_chunk_events and returns it with its wall time
 * per call in microseconds.  Synchronous. */
sst_status sst_autotune_host(sst_ctx* ctx, const uint8_t* raw, const uint64_t* event_off, const uint32_t* fed_len,
                             uint32_t n_events, uint32_t n_feds, const sst_clusters* out, uint64_t* event_first,
                             sst_event_status* status, uint32_t* best_chunk, float* best_us);

/* What the context's knobs make of a batch of n_events x n_feds: the batched
 * kernel's grid (CTAs), threads per CTA, dynamic shared memory per CTA and work
 * items per FED, and the number of chunks sst_batch_host cuts the batch into.
 * Any output pointer may be NULL.  CUDA if the occupancy look-up fails. */
typedef struct {
  uint32_t grid;
  uint32_t block;
  uint32_t smem_bytes;
  uint32_t items_per_fed;
  uint32_t host_chunks;
} sst_launch_info;
sst_status sst_get_launch_info(sst_ctx* ctx, uint32_t n_events, uint32_t n_feds, sst_launch_info* info);

/* ---- kernel timing ------------------------------------------------------------
 * When enabled, the context brackets every launch of its batched kernel (the one
 * sst_batch and sst_autotune time) with CUDA events on the launching stream, so
 * that a caller can read the kernel's own device time apart from the memsets and
 * the FED-offset scan around it. */
sst_status sst_profile_enable(sst_ctx* ctx, int enable);
/* Waits for the recorded launches, returns their number and summed device time
 * in milliseconds, and (reset != 0) forgets them. */
sst_status sst_profile_read(sst_ctx* ctx, uint64_t* launches, double* total_ms, int reset);

/* ---- failure detection ----------------------------------------------------------
 * The per-event unpacker places each FED's digis after a device-side look-back over
 * the FEDs before it (section 2: the channel map, here built on the device).  Every
 * such wait gives up after a bounded number of polls (about a second by default),
 * flags the event SST_EV_TIMEOUT and lets the kernel finish; the event's output is
 * then invalid, but no access leaves its buffers.  For tests of that path:
 * spin_limit sets the polls (1 .. 2^20; 0 = the default) and withhold_fed >= 0
 * makes the FED of that index never publish its digi count, so that the FEDs after
 * it run out of polls; withhold_fed = -1 restores normal operation.  Nothing faults,
 * traps or waits without end.  INVALID_ARG for spin_limit above 2^20 or
 * withhold_fed below -1. */
sst_status sst_testing_set_wait(sst_ctx* ctx, uint32_t spin_limit, int32_t withhold_fed);

/* ---- served path: continuous batching ------------------------------------------ */

typedef struct {
  uint64_t mem_budget_bytes; /* device memory for in-flight events (admission budget) */
  uint32_t max_batch_events; /* events per launch */
  uint32_t max_inflight;     /* launches in flight at once (streams) */
  uint32_t max_requests;     /* request slots (admitted + finished-not-polled) */
  uint32_t n_feds;           /* FEDs per event */
  uint32_t zero_copy;        /* 0: sst_submit copies the event into the server's pinned pool, the
                                caller may reuse its buffer at once; 1: no copy, the server copies
                                from the caller's buffer to the device (pinned memory gives full
                                copy speed); 2: in place, the kernels read the event from the
                                caller's buffer over the host link, with no device copy: the buffer
                                must be one page-locked allocation (cudaHostAlloc, or memory
                                registered with cudaHostRegister), 16-byte aligned and a multiple of
                                16 bytes long (sst_submit checks the alignment and that its first
                                and last bytes are page-locked, else INVALID_ARG).  With 1 and 2
                                the buffer must stay unchanged until sst_poll returns for the
                                ticket.  In place saves the copy engine one transfer per event,
                                which dominates for events of about a megabyte */
} sst_server_opts;

/* Starts the request loop (one host thread, max_inflight streams): section 3's
 * events processed concurrently on one GPU as they arrive, with their transfers
 * overlapped with the computation and device memory taken once (the paper's
 * caching allocator), here carved from mem_budget_bytes at start.  A batch of the
 * pending events is launched whenever a slot is free; the batches' kernels run one
 * batch at a time (each launch fills the GPU) and each batch's copies overlap the
 * next one's kernels.  Requires calibration.  STATE if already running. */
sst_status sst_server_start(sst_ctx* ctx, const sst_server_opts* opts);

/* Stops the loop and frees the server; unpolled results are discarded.  Safe while
 * other threads are inside sst_submit / sst_poll: from the call on they get
 * STATE, pollers waiting without a timeout return, and the server is freed once
 * no such call is inside. */
sst_status sst_server_stop(sst_ctx* ctx);

/* Submits one event from HOST memory (raw: raw_bytes bytes, fed_len: [n_feds])
 * (section 3 and the served workload: events arrive one at a time and are
 * processed concurrently).  The bytes are copied before the call returns (unless
 * zero_copy).  Admission by memory: sst_server_start divides the device budget
 * into max_inflight batch slots of equal size, each holding a raw arena of
 * budget / (25 max_inflight) bytes and the cluster and staging arrays for it, so
 * that the device memory in use never exceeds the budget; admitted events wait
 * for a slot in a pinned host pool of max_inflight + 1 raw arenas (at most 2 GiB;
 * with zero_copy the event's size is reserved in it, its bytes stay with the
 * caller).
 * Returns OK and a ticket; BUSY when all max_requests request slots are taken;
 * BUDGET when the event does not fit the host pool now (retry after polling);
 * TOO_LARGE when it exceeds one raw arena (it never fits); STATE when no server
 * runs.  Thread safe. */
sst_status sst_submit(sst_ctx* ctx, const uint8_t* raw, uint64_t raw_bytes, const uint32_t* fed_len,
                      uint64_t* ticket);

typedef struct {
  sst_event_status status;
  double t_submit_us; /* host clock, microseconds, at sst_submit */
  double t_done_us;   /* host clock when the loop saw the event's launch complete */
} sst_result_info;

/* Waits up to timeout_us (0 = just check, < 0 = forever) for ticket's result
 * (section 3: the served events' results, in whatever order they finish).
 * On OK copies the status and up to `capacity` clusters to the HOST arrays (any
 * may be NULL to skip) and releases the request slot and the event's host bytes.
 * NOT_READY on timeout; INVALID_ARG for an unknown ticket (or one that another
 * caller collects meanwhile: a ticket's result is handed out once); STATE when
 * the server is (or gets) stopped.  Thread safe: the copy out runs without the
 * server's lock, so callers collecting different tickets do not wait for one
 * another, nor hold up sst_submit. */
sst_status sst_poll(sst_ctx* ctx, uint64_t ticket, int64_t timeout_us, sst_result_info* info, uint32_t* det,
                    uint16_t* first, uint16_t* width, uint32_t* charge, float* barycenter, uint64_t capacity);

/* ---- a native client for the served path ---------------------------------------
 * Measures the server as a stream of requests sees it (section 3: events processed
 * concurrently as they come), with no client of another language in the way.  The
 * server must be running.  Request i is event i mod n_events (raw[e], raw_bytes[e]
 * and fed_len[e] in HOST memory; with zero_copy they must stay unchanged until the
 * call returns) and is due at the i-th point of a Poisson process of `rate`
 * events/s (0: all at once, i.e. as fast as the server admits; seeded by `seed`).
 * `submitters` threads (1..64) submit the requests in turn, each at its due time,
 * retrying while the server answers BUSY or BUDGET; `pollers` threads (1..16)
 * collect them in admission order.  latency_us (NULL or [n_requests]) receives
 * each request's latency from its due time to its completion.  Returns when every
 * request is collected; INVALID_ARG for bad arguments, STATE without a server,
 * TIMEOUT when submissions are refused for a minute, or the first failing
 * submit / poll status. */
typedef struct {
  double offered_rate;    /* events/s asked for (0: saturating) */
  double throughput;      /* events/s: requests / (last completion - start) */
  double p50_us, p99_us;  /* latency from the due time to completion (host clock) */
  double mean_us, max_us;
  double p50_admitted_us, p99_admitted_us; /* latency from admission to completion */
  uint64_t requests;
  uint64_t retries;       /* submissions refused (BUSY or BUDGET) and retried */
} sst_load_result;
sst_status sst_serve_load(sst_ctx* ctx, const uint8_t* const* raw, const uint64_t* raw_bytes,
                          const uint32_t* const* fed_len, uint32_t n_events, uint64_t n_requests, double rate,
                          uint32_t submitters, uint32_t pollers, uint64_t seed, double* latency_us,
                          sst_load_result* out);

#ifdef __cplusplus
}
#endif
#endif
