/*
 * hs.h -- C ABI of libhs, a GB300 (sm_103a) harmonic summer for
 * Fourier-domain acceleration search.
 *
 * The operation (Wang, Thiagaraj & Sinnen, arXiv 1805.12258, Section III):
 * the filter-output plane (FOP) holds n_templates rows of detected power,
 * indexed by a signed template z in [-Z, Z] (Z = (n_templates-1)/2, row
 * r = z + Z), times n_bins frequency bins f.  For every point and every
 * harmonic level k = 1..H the library forms
 *
 *     HP_k(z, f) = sum_{m=1..k} FOP(rho(z, m), floor(f / m))        (Eq. 1-2)
 *
 * (the stretch planes SP_m of Eq. 1 summed cumulatively as in Eq. 2), tests
 * HP_k(z, f) > TA(k, z) against a per-level, per-row threshold, and appends
 * every hit to a candidate list.  Harmonic planes are never stored: all H
 * levels of a point are formed together and discarded after the test, the
 * MultipleHP loop order of Algorithm 2.
 *
 * rho(z, m) is sign(z) * floor(|z| / m) by default (the two template groups
 * stretched separately, Section III); HS_ZROUND_FLOOR selects floor(z / m).
 * HS_INDEX_HFRAC selects the harmonic-fraction sum
 * S_k(z, f) = sum_{h=1..k} FOP(rho(z*h/k), floor(f*h/k)) instead (not in the
 * paper; offered so that both readings of "sum over harmonics" exist).
 *
 * Conventions.
 *  - Device pointers are CUDA device (or managed) addresses on the current
 *    device.  Host pointers are ordinary CPU memory.
 *  - A stream argument is a cudaStream_t (NULL = legacy default stream).
 *  - Every call returns an hs_status; hs_last_error() gives a message for the
 *    last failure on the calling thread.
 *  - Calls that take a stream only enqueue work; they do not synchronise
 *    unless their comment says so.  Errors that only the device can see (a
 *    wait that timed out) are reported by hs_cand_sync().
 */
#ifndef HS_H
#define HS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define HS_API __attribute__((visibility("default")))
#else
#define HS_API
#endif

typedef struct CUstream_st *hs_stream_t; /* same type as cudaStream_t */

typedef enum {
    HS_OK = 0,
    HS_ERR_INVALID = 1,     /* bad argument (shape, pointer, alignment, option) */
    HS_ERR_CUDA = 2,        /* a CUDA runtime/driver call failed */
    HS_ERR_OOM = 3,         /* device or host allocation failed */
    HS_ERR_OVERFLOW = 4,    /* more candidates than the buffer holds */
    HS_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
    HS_ERR_UNSUPPORTED = 6, /* valid request this build does not implement */
    HS_ERR_BUSY = 7,        /* serving engine: queue full, or result not ready in time */
    HS_ERR_BOUNDS = 8       /* a library built with -DHS_CHECK_BOUNDS found an index outside
                               its buffer (the access was skipped); never in a normal build */
} hs_status;

typedef enum { HS_F32 = 0, HS_BF16 = 1, HS_F16 = 2 } hs_dtype;
typedef enum { HS_INDEX_STRETCH = 0, HS_INDEX_HFRAC = 1 } hs_index;
typedef enum { HS_ZROUND_SYMMETRIC = 0, HS_ZROUND_FLOOR = 1 } hs_zround;
typedef enum { HS_KERNEL_AUTO = 0, HS_KERNEL_GENERIC = 1, HS_KERNEL_STAGED = 2 } hs_kernel;

/* Plan options.  Zero-initialise for the defaults. */
typedef struct {
    int dtype;      /* hs_dtype of the stored plane (default HS_F32) */
    int index;      /* hs_index (default HS_INDEX_STRETCH, Eq. 1-2) */
    int zround;     /* hs_zround (default HS_ZROUND_SYMMETRIC) */
    int kernel;     /* hs_kernel: AUTO picks the staged kernel when it applies -- the
                       stretch map: a compiled shape family, symmetric rounding, rows a
                       multiple of 16 bytes; HS_INDEX_HFRAC: FP32, symmetric rounding,
                       H = 8 or 16, rows a multiple of 16 bytes (one launch per level
                       family).  Otherwise (or GENERIC) the generic kernel; for HFRAC at
                       H = 8 or 16 with symmetric rounding, its gather form. */
    int tile_bins;  /* bins per CTA of the staged kernel: 0 = default (128; 64 for
                       HS_INDEX_HFRAC, which takes 64 or 128) */
    int order;      /* tile order: 0 = default (4; linear for HS_INDEX_HFRAC),
                       1 = linear, 2 = octave (mantissa of the tile index), 3 = semitone
                       (fractional part of 12 log2 of the tile index), 4 = the same with
                       53 steps to the octave (fractional part of 53 log2) */
    int grid_per_sm;/* staged kernel: 0 = one CTA per tile; k > 0 = k resident CTAs per SM
                       that walk the tiles */
    int row_pitch;  /* elements between plane rows (0 = n_bins); >= n_bins.  The staged
                       kernel needs row_pitch * element size to be a multiple of 16 bytes
                       (so its largest FP32 plane has 2^31 - 4 bins; wider planes take the
                       generic kernel) */
    int stages;     /* staged kernel: 0 = one CTA per tile (or grid_per_sm); s > 0 = one
                       persistent CTA per SM with an s-stage ring of tiles, filled by a
                       producer warp while consumer groups sum (stretch map only) */
    int z_split;    /* with stages > 0: consumer groups of tile_bins threads (0 = 2) */
    int assume_nonneg; /* 1: the caller declares every plane value non-negative and not
                       NaN (detected power is); the staged kernel then skips its per-value
                       sign check (a few % faster; every compiled shape at 128 bins).  A
                       plane that breaks the promise may lose candidates.
                       0 (default): signed inputs are handled exactly. */
} hs_options;

/* Candidate record flags */
#define HS_FLAG_LOWP 0x1u /* decided on a 16-bit plane without an FP32 recheck */
#define HS_FLAG_NEAR 0x2u /* ... and within the 16-bit error band of its threshold */

/* One candidate, 16 bytes.  Section III packs (filter, plane, bin, amplitude)
 * into two 32-bit words; that packing cannot hold H = 16 with 2^22 bins, so
 * the record is widened (hs_pack_paper() gives the paper's form when it fits). */
typedef struct {
    uint32_t bin;      /* f */
    int16_t z;         /* signed template index */
    uint8_t k;         /* harmonic level, 1..H */
    uint8_t flags;     /* HS_FLAG_* */
    float power;       /* HP_k(z, f) as computed in FP32 */
    uint32_t reserved; /* 0 */
} hs_cand;

/* Caller-owned device candidate buffer.
 *  records : device array of `capacity` records (NULL with capacity 0: a
 *            count-only buffer; runs then count every hit and write none).
 *  count   : device array of 2 uint32: [0] = number of candidates found
 *            (may exceed capacity; records beyond it are dropped),
 *            [1] = device status (HS_OK or HS_ERR_TIMEOUT).
 * hs_run resets both words on its stream before its kernel. */
typedef struct {
    hs_cand *records;
    uint32_t *count;
    uint32_t capacity;
} hs_cand_buf;

typedef struct hs_plan hs_plan;

/* Create a plan (Section III, Table I parameters N_temp, N_chan, N_hp).
 *  n_templates : odd, 1..32767.   n_bins : 1..2^31-1.   H : 1..32.
 *  thresholds  : host array TA[H][n_templates] (level-major, binary32, all
 *                finite); copied, the caller keeps ownership.
 *  opt         : NULL for defaults.
 * Allocates the plan's device tables on the current device; the plan runs
 * only with that device current (any other gives HS_ERR_INVALID, and
 * hs_plan_destroy frees on the plan's device whatever device is current).
 * Errors: HS_ERR_INVALID, HS_ERR_UNSUPPORTED (kernel = STAGED, or stages > 0,
 *         where no such kernel applies), HS_ERR_OOM, HS_ERR_CUDA. */
HS_API hs_status hs_plan_create(hs_plan **out, int n_templates, int64_t n_bins, int H,
                         const float *thresholds, const hs_options *opt);

/* Enqueue harmonic summing + detection of one plane on `stream`: for every
 * point (z, f) of the plane and every level k = 1..H, the harmonic-plane
 * value HP_k(z, f) = sum over m = 1..k of FOP(rho(z, m), floor(f / m)) (the
 * stretch of Eq. 1 accumulated as in Eq. 2, Section III), tested against the
 * level's threshold TA(k, z) as Algorithms 1 and 2 detect; every point with
 * HP_k > TA(k, z) becomes a candidate record (Section III's F, H, B, A
 * fields), in no particular order.  All levels of a point are formed
 * together and never stored, the MultipleHP order of Algorithm 2.
 *  fop   : device plane [n_templates][row pitch], row-major, plan dtype,
 *          16-byte aligned; borrowed until the stream passes the kernel.
 *  cands : caller-owned buffer (see hs_cand_buf); its counters are reset on
 *          `stream` before the kernel.
 * A plan may serve several streams at once if each run has its own cands.
 * Errors (at enqueue): HS_ERR_INVALID (null/misaligned pointers),
 * HS_ERR_CUDA; device-side outcomes are read by hs_cand_sync. */
HS_API hs_status hs_run(hs_plan *plan, const void *fop, hs_stream_t stream,
                 const hs_cand_buf *cands);

/* As hs_run for a 16-bit plan, with an optional FP32 copy of the same plane.
 * When fop_f32 is given, every point whose 16-bit level sum could lie on
 * either side of its threshold is re-evaluated from the FP32 copy with the
 * FP32 path's arithmetic, so the candidate set (and each record) equals
 * hs_run on the FP32 plane: the summing kernel lists the row pairs it marks
 * in a plan-owned list (one per stream, allocated at the first such run on
 * it, 4 MiB -- make that first run outside stream capture; past 16 streams
 * the lists are freed after a device-wide wait and made again) and a second
 * kernel decides them from the copy (pairs past the list's 2^19 are decided
 * in the summing kernel).  When fop_f32 is NULL the 16-bit sums decide and
 * records carry HS_FLAG_LOWP (and HS_FLAG_NEAR inside the error band).  An
 * FP16 value above 65504 is stored as +inf: with the copy its pairs are
 * decided from the copy; without it their records carry power +inf and both
 * flags.  For an FP32 plan fop_f32 must be NULL. */
HS_API hs_status hs_run_checked(hs_plan *plan, const void *fop, const float *fop_f32,
                         hs_stream_t stream, const hs_cand_buf *cands);

/* Synchronise `stream`, read the candidate count and device status: the end
 * of one detection pass of Section III.  The paper keeps at most N_cand
 * candidates per harmonic plane and leaves open which (Section IV-A); here
 * every candidate is returned and the true count reported, and a cap can be
 * applied afterwards with hs_postfilter.
 *  cands : the buffer a run wrote (device counters, read on `stream`).
 *  n_out : receives the number of candidates found (the true count).
 * Returns HS_ERR_TIMEOUT if a device wait gave up, HS_ERR_OVERFLOW if
 * *n_out > capacity (the first `capacity` records are valid), HS_ERR_CUDA if
 * the copy or the synchronisation failed, else HS_OK. */
HS_API hs_status hs_cand_sync(const hs_cand_buf *cands, hs_stream_t stream, uint32_t *n_out);

/* End-to-end call on host memory: copies fop_host (the plane, plan dtype,
 * ideally page-locked) to fop_dev in frequency chunks and overlaps each copy
 * with the summing of the bins it completes, then copies the candidates back.
 * Synchronous.
 *  fop_dev      : device scratch plane of the same size (caller-owned).
 *  cands        : device candidate buffer (caller-owned).
 *  host_records : host array of host_capacity records (may be NULL if 0).
 *  n_out        : true candidate count.
 * Errors as hs_run and hs_cand_sync. */
HS_API hs_status hs_run_host(hs_plan *plan, const void *fop_host, void *fop_dev,
                      const hs_cand_buf *cands, hs_cand *host_records,
                      uint32_t host_capacity, hs_stream_t stream, uint32_t *n_out);

/* As hs_run_host for a 16-bit plan whose FP32 copy stays in page-locked host
 * memory: the few near-threshold points are re-added from fop32_host, read by
 * the kernel across the host link, so only the 16-bit plane crosses it in
 * bulk and the candidates equal the FP32 path's.  fop32_host: [n_templates]
 * [row pitch] FP32 host memory the device can address (page-locked, or any
 * host memory on systems with address translation), 16-byte aligned; NULL
 * behaves as hs_run_host.  Errors as hs_run_host, and HS_ERR_INVALID for an
 * FP32 plan or a copy the device cannot address. */
HS_API hs_status hs_run_host_checked(hs_plan *plan, const void *fop_host, void *fop_dev,
                                     const float *fop32_host, const hs_cand_buf *cands,
                                     hs_cand *host_records, uint32_t host_capacity,
                                     hs_stream_t stream, uint32_t *n_out);

/* ---- Batched form: many planes (beams) of one shape -------------------------
 * The paper processes one plane per DM trial and several planes on separate
 * boards (Section VI-C); a pipeline has thousands per observation.  A batch
 * sums many planes of the same template count, level count and thresholds,
 * each with its own number of bins and row pitch.  Each launch carries the
 * TMA descriptors of up to K beams in its parameter block (K = 13 for the
 * 85 x 16 shape, 24 for 21 x 8) and covers the concatenated tiles of its
 * beams; a run issues ceil(n_beams / K) launches after one counter reset.
 * Beams packed side by side in one plane (hs_batch_set_packed) are summed
 * by one launch whatever their number. */
typedef struct {
    const void *fop;     /* device plane [n_templates][ld], 16-byte aligned */
    const float *fop32;  /* FP32 copy for rechecks (16-bit batches), or NULL */
    int64_t n_bins;      /* bins of this beam */
    int64_t ld;          /* row pitch in elements (0 = n_bins); ld * elem a multiple of 16 */
    hs_cand_buf cands;   /* this beam's candidate buffer (reset by every run) */
} hs_beam;

typedef struct hs_batch hs_batch;

/* Create a batch for up to max_beams beams (1..65536) of n_templates rows and
 * H levels with thresholds TA[H][n_templates] (copied).  opt: dtype, order
 * (tile order inside each beam, as for a plan), grid_per_sm (0 = one CTA
 * per tile; k > 0 = k resident CTAs per SM) and assume_nonneg (as for a
 * plan).  Compiled shapes: 85 x 16 (FP32,
 * BF16) and 21 x 8 (FP32), stretch index map, symmetric rounding.  Like a
 * plan, a batch belongs to the device current at its creation: the other
 * hs_batch_* calls need that device current (else HS_ERR_INVALID), and
 * hs_batch_destroy frees on it.
 * Errors: HS_ERR_INVALID, HS_ERR_UNSUPPORTED, HS_ERR_OOM, HS_ERR_CUDA. */
HS_API hs_status hs_batch_create(hs_batch **out, int n_templates, int H, const float *thresholds,
                                 const hs_options *opt, int max_beams);

/* Describe the beams of the next runs (host array, copied): encodes their
 * descriptors on the host and uploads their tile order on `stream`.  The
 * planes and buffers are borrowed until the stream passes the runs that use
 * them.  On error the previous beam set stays in place.
 * Errors: HS_ERR_INVALID, HS_ERR_CUDA, HS_ERR_OOM. */
HS_API hs_status hs_batch_set_beams(hs_batch *b, const hs_beam *beams, int n_beams,
                                    hs_stream_t stream);

/* One beam of a packed batch: its bins are [offset, offset + n_bins) of
 * every row of the batch's packed plane. */
typedef struct {
    int64_t offset;      /* first bin of the beam; offset * element size a multiple of 16 */
    int64_t n_bins;      /* bins of this beam, >= 1; offset + n_bins <= the plane's pitch */
    hs_cand_buf cands;   /* this beam's candidate buffer (reset by every run) */
} hs_packed_beam;

/* Describe the beams of the next runs as one packed plane: `plane` is a
 * device array [n_templates][pitch] of the batch's dtype (16-byte aligned,
 * pitch * element size a multiple of 16) in which the beams lie side by
 * side along the bins (beams may share bins; bins outside every beam are
 * never read into a result).  fop32: the FP32 copy in the same layout for
 * 16-bit batches (NULL: records flagged HS_FLAG_LOWP), NULL for FP32.  The
 * beam table (host array, copied) and the tile order go to device memory on
 * `stream`.  One set of descriptors then serves every beam, so a run is one
 * summing launch over all their tiles, whatever the beam count, after one
 * kernel that clears every beam's counters.  The definition summed is that
 * of hs_run (Section III, Eq. 1-2) for each beam on its own bins.  Borrowed
 * and error rules as for hs_batch_set_beams; replaces any beam set.
 * Errors: HS_ERR_INVALID, HS_ERR_CUDA, HS_ERR_OOM. */
HS_API hs_status hs_batch_set_packed(hs_batch *b, const void *plane, const float *fop32,
                                     int64_t pitch, const hs_packed_beam *beams, int n_beams,
                                     hs_stream_t stream);

/* Enqueue one run over every beam set by hs_batch_set_beams (or
 * hs_batch_set_packed): one kernel clears each beam's counters, then
 * hs_batch_launches() launches sum the tiles.  Records go to each beam's
 * buffer in an unspecified order. */
HS_API hs_status hs_batch_run(hs_batch *b, hs_stream_t stream);

/* As hs_batch_run, through a CUDA graph of the same launches, captured (on
 * a private stream) on first use and again after hs_batch_set_beams, then
 * replayed on `stream`; a re-capture updates the instantiated graph in place
 * when the launch count is unchanged. */
HS_API hs_status hs_batch_graph_run(hs_batch *b, hs_stream_t stream);

/* Tiles of the current beam set, and the kernel launches a run issues to
 * sum them (the counter reset not included; 1 for a packed batch). */
HS_API int hs_batch_tiles(const hs_batch *b);
HS_API int hs_batch_launches(const hs_batch *b);

/* Destroy a batch (NULL is accepted); synchronises the device first. */
HS_API hs_status hs_batch_destroy(hs_batch *b);
HS_API const char *hs_batch_last_error(void);

/* ---- Serving form: a long-lived engine over resident plane slots ----------
 * The paper's pipeline feeds harmonic summing one plane per DM trial, as the
 * upstream Fourier-domain convolution produces them (Section II, Fig. 1), with
 * thousands of planes per observation (Section VI-C).  The engine keeps
 * n_slots plane slots resident in device memory (memory admission: a request
 * runs only when a slot is free; at most queue_limit wait, further submits
 * answer HS_ERR_BUSY), produces each admitted request's plane on the device
 * into its slot with hs_synth_fop (standing in for the upstream stage), and
 * sums every group of admitted requests with the batched kernels (FP32 and
 * BF16 requests mixed; BF16 planes keep an FP32 copy for rechecks, so their
 * candidates equal the FP32 path's).  A dispatcher thread admits and launches
 * groups while earlier groups run (continuous batching); a completion thread
 * copies each request's candidates to host memory and frees its slot.  One
 * request's candidates do not depend on what it ran with. */
typedef struct {
    int n_templates;          /* rows of every plane (odd; 85 or 21 compiled) */
    int H;                    /* levels (16 for 85 rows, 8 for 21) */
    const float *thresholds;  /* host TA[H][n_templates], copied */
    int n_slots;              /* resident slots (1..1024), reserved at create */
    int64_t slot_bins;        /* largest n_bins of a request */
    uint32_t cand_capacity;   /* records kept per request (1..2^20) */
    int queue_limit;          /* requests waiting for a slot (>= 0) */
    int max_group;            /* requests admitted into one group (0 = n_slots) */
    int assume_nonneg;        /* 1: resident planes brought by requests are non-negative
                                 (generated planes are); the kernels skip their per-value
                                 sign check, as hs_options.assume_nonneg */
} hs_server_config;

typedef struct {
    uint64_t seed;            /* generator seed of the plane (noise and signals) */
    int64_t n_bins;           /* 1..slot_bins */
    int dtype;                /* HS_F32 or HS_BF16 */
    int n_signals;            /* injected signals, 0..16 */
    /* A plane already resident in device memory (made upstream): when fop is
     * not NULL the engine sums it in place instead of generating one into the
     * slot (seed and n_signals unused).  Borrowed until the request is done;
     * 16-byte aligned rows of pitch ld (0 = n_bins; ld * element size a
     * multiple of 16).  BF16 planes need their FP32 copy fop32 (same pitch). */
    const void *fop;
    const float *fop32;
    int64_t ld;
} hs_request;

typedef struct {
    uint64_t ticket;
    hs_status status;         /* HS_OK, HS_ERR_OVERFLOW, HS_ERR_TIMEOUT or HS_ERR_CUDA */
    uint32_t n_cands;         /* true hit count; min(n_cands, cand_capacity) records kept */
    int32_t group;            /* admission group that ran the request */
    int32_t group_size;       /* requests in that group */
    int32_t slot;
    int64_t t_submit_ns;      /* steady clock: submit, admission, candidates on host */
    int64_t t_admit_ns;
    int64_t t_done_ns;
} hs_result;

typedef struct {
    uint64_t submitted, rejected, completed, groups;
    uint64_t points;          /* n_templates x n_bins summed over completed requests */
    uint64_t dispatch_ns;     /* host time the dispatcher spent enqueuing groups */
    int32_t queued, in_flight, free_slots, peak_queue;
} hs_server_stats;

typedef struct hs_server hs_server;

/* Create an engine on the current device: reserves n_slots slots of
 * n_templates x round_up(slot_bins, 8) elements at 6 bytes each (FP32 plane
 * or FP32 copy + BF16 plane; every request keeps the slot's row pitch, so
 * the slots' TMA descriptors are encoded once here) plus the candidate
 * buffers, and starts the dispatcher and completion threads.  Groups
 * alternate between two streams.
 * Errors: HS_ERR_INVALID, HS_ERR_UNSUPPORTED (no batched kernel for the
 * shape), HS_ERR_OOM, HS_ERR_CUDA. */
HS_API hs_status hs_server_create(hs_server **out, const hs_server_config *cfg);

/* Queue a request; *ticket identifies it.  HS_ERR_BUSY when queue_limit
 * requests already wait for a slot (nothing is queued), HS_ERR_INVALID for a
 * bad request. */
HS_API hs_status hs_server_submit(hs_server *s, const hs_request *r, uint64_t *ticket);

/* Wait up to timeout_ms (< 0: forever) for a request to finish; on success
 * fills *res, copies up to `capacity` records to host memory `records` (may
 * be NULL) and forgets the request.  Returns HS_ERR_BUSY if it did not finish
 * in time, HS_ERR_INVALID for an unknown ticket; otherwise HS_OK (the
 * request's own outcome is res->status). */
HS_API hs_status hs_server_wait(hs_server *s, uint64_t ticket, int timeout_ms, hs_result *res,
                                hs_cand *records, uint32_t capacity);

/* Wait up to timeout_ms (< 0: forever) until nothing is queued or running. */
HS_API hs_status hs_server_drain(hs_server *s, int timeout_ms);

HS_API hs_status hs_server_stats_get(hs_server *s, hs_server_stats *st);

/* Stop the threads (finishing admitted work) and free everything; NULL ok. */
HS_API hs_status hs_server_destroy(hs_server *s);
HS_API const char *hs_server_last_error(void);

/* The plane generator of the serving engine, standing in for the upstream
 * stage: writes iid Exponential(mean 1) noise -- Philox4x32-10 (Salmon et
 * al., SC'11) keyed by seed, counter (bin / 4, row) -- into the
 * n_templates x n_bins plane with row pitch ld (>= n_bins, multiple of 8;
 * pad bins are zeroed), then adds n_signals harmonic signals (amplitude
 * U[3, 8) at (h z0, h f0) for h = 1..16 inside the plane; z0 in [-2, 2], f0
 * drawn from the seed).  dtype HS_F32: fop is the FP32 plane, fop32 unused.
 * dtype HS_BF16: fop receives the BF16 plane (round to nearest even) and
 * fop32 the FP32 values.  Pointers 16-byte aligned.
 * Errors: HS_ERR_INVALID, HS_ERR_CUDA. */
HS_API hs_status hs_synth_fop(void *fop, float *fop32, int dtype, int n_templates,
                              int64_t n_bins, int64_t ld, uint64_t seed, int n_signals,
                              hs_stream_t stream);

/* Sum only the output bins [f_lo, f_hi) of the plane (all rows, all levels):
 * the unit of a frequency-band shard (each shard reads the bins
 * [f_lo / m, f_hi / m) of level m, all below f_hi, so a band needs no data
 * from higher bands).  f_lo, and f_hi unless it equals n_bins, must be
 * multiples of hs_plan_tile_bins().  append != 0 keeps the buffer's count and
 * appends, so several bands can share one buffer.  The band's tiles run in
 * the plan's tile order restricted to the band (the staged kernel; a table
 * the plan makes at the first run of each band -- make that run outside
 * stream capture).
 * fop32: FP32 recheck copy for 16-bit plans, or NULL.
 * Errors: as hs_run_checked, and HS_ERR_INVALID for a bad range. */
HS_API hs_status hs_run_range(hs_plan *p, const void *fop, const float *fop32, int64_t f_lo,
                              int64_t f_hi, hs_stream_t stream, const hs_cand_buf *cands,
                              int append);

/* Harmonic summing with no device allocation.  The paper has no counterpart:
 * this entry point is for callers that may not allocate device memory, such
 * as code inside a host framework that has reserved all device memory for its
 * own pool, or latency-critical loops that cannot afford cudaMalloc/cudaFree
 * (they may synchronise the device).  It does what hs_plan_create + hs_run +
 * hs_plan_destroy do for an FP32 plane with the default options, without a
 * plan and without allocating: the threshold table is copied into a fixed
 * array inside the library's device image, and tiles run in linear order.
 *  - Limit: H * n_templates <= 16384 (a 64 KiB table); larger requests fail
 *    with HS_ERR_INVALID.  Every GPU that loads the library holds the array
 *    until the process exits.
 *  - Every call looks up the array's device address with the caller's
 *    device current (cudaGetSymbolAddress), so a context made again after
 *    cudaDeviceReset gets the right one.  The first call on a device may load
 *    the library's module there.
 *  - All calls share the array and it keeps the last call's thresholds: two
 *    calls whose work overlaps on the GPU (different streams, or threads)
 *    race on it.  Serialise them, e.g. issue them on one stream.
 *  - fop, stream and cands as for hs_run (the counters are reset on stream).
 * Errors: HS_ERR_INVALID, HS_ERR_CUDA; device timeouts via hs_cand_sync. */
HS_API hs_status hs_run_noalloc(int n_templates, int64_t n_bins, int H, const float *thresholds,
                                const void *fop, hs_stream_t stream, const hs_cand_buf *cands);
HS_API const char *hs_noalloc_last_error(void);

/* Destroy a plan (NULL is accepted).  Synchronises the device first. */
HS_API hs_status hs_plan_destroy(hs_plan *plan);

/* Which kernel a plan runs: 1 = generic, 2 = staged (TMA). */
HS_API int hs_plan_kernel(const hs_plan *plan);

/* Bins per CTA of the plan's kernel. */
HS_API int hs_plan_tile_bins(const hs_plan *plan);

/* Kernel timing for profiling.  While enabled, the kernels of every run of the
 * plan are bracketed by one pair of CUDA events on its stream (not the
 * counter reset or copies; a run is one kernel, two for a 16-bit plane with
 * an FP32 copy, one per level family for the harmonic-fraction map).  A pair
 * costs a few microseconds of device time per run.  hs_plan_kernel_time
 * waits for the recorded runs, returns their summed device time in
 * milliseconds and their number, and clears the record (which grows by a
 * pair of events per run until then).  Errors: HS_ERR_INVALID (null plan),
 * HS_ERR_CUDA. */
HS_API hs_status hs_plan_set_timing(hs_plan *plan, int enable);
HS_API hs_status hs_plan_kernel_time(hs_plan *plan, double *total_ms, int *launches);

/* Kernels launched by the last hs_run* call on this thread. */
HS_API int hs_last_launch_count(void);

/* Self-test of the bounded device waits (failure detection without a GPU
 * fault): one CTA waits on an mbarrier phase that nothing completes, gives up
 * after limit_ns (1 ns .. 10 s) and writes HS_ERR_TIMEOUT into counters[1]
 * (device memory, the status word of an hs_cand_buf), as a summing kernel
 * does when a tile's copies never arrive.  Asynchronous on `stream`; read the
 * status with hs_cand_sync.  Errors: HS_ERR_INVALID, HS_ERR_CUDA. */
HS_API hs_status hs_selftest_wait_timeout(uint32_t *counters, uint64_t limit_ns,
                                          hs_stream_t stream);

/* The paper's packed candidate form (Section III): CL1 = F*2^24 + H*2^21 + B,
 * CL2 = A, with F the row r = z + Z (7 bits), H the 0-based level (3 bits),
 * B the bin (21 bits).  HS_ERR_INVALID when a field does not fit. */
HS_API hs_status hs_pack_paper(const hs_cand *c, int n_templates, uint32_t *cl1, float *cl2);

/* The paper's candidate cap per harmonic plane (Section IV-A): the policy is
 * left open there (first, last or largest N_cand), so all three are offered.
 * Host arrays.  For each level k keep at most n_keep of its records: FIRST /
 * LAST = the first / last n_keep in Algorithm 2's visiting order (bins
 * ascending, then z ascending), LARGEST = the n_keep largest powers (equal
 * powers: the later visited first).  out (capacity n, not aliasing in)
 * receives the kept records grouped by k ascending, each level in visiting
 * order; *n_out their number.  Errors: HS_ERR_INVALID. */
typedef enum { HS_KEEP_FIRST = 0, HS_KEEP_LAST = 1, HS_KEEP_LARGEST = 2 } hs_keep;
HS_API hs_status hs_postfilter(const hs_cand *in, uint32_t n, int policy, uint32_t n_keep,
                               hs_cand *out, uint32_t *n_out);
HS_API const char *hs_postfilter_last_error(void);

/* Host logic of the staged kernel, exposed for inspection and tests (no GPU
 * needed).
 *
 * hs_prefilter_bounds: the fast pass's bound of each level group (Eq. 2 sums
 * tested at the group ends 2, 4, 8, then every 4 levels, and H): the smallest
 * threshold TA(k, row) of the group's levels over all rows, lowered by the
 * storage error of dtype (BF16, FP16: relative error of the stored values,
 * plus the FP16 subnormal spacing) and by the rounding of the fast pass's
 * FP32 sums, so that the prefilter never drops a point whose FP32 level sum
 * (ascending m, Eq. 2 order) exceeds its threshold.  thresholds: host
 * [H][n_templates] float32.  ends[8] receives the last level of each group,
 * bounds[8] its bound, *n_groups the group count.  Errors: HS_ERR_INVALID
 * (null pointers, n_templates not odd in 1..127, H not in 2..16).
 *
 * hs_tile_order: the order in which a plan visits the tiles of a plane
 * (hs_options.order; 0 = the default), as tile indices: out[n_tiles] is a
 * permutation of 0 .. n_tiles-1.  Errors: HS_ERR_INVALID. */
HS_API hs_status hs_prefilter_bounds(const float *thresholds, int n_templates, int H, int dtype,
                                     int *ends, float *bounds, int *n_groups);
HS_API hs_status hs_tile_order(int n_tiles, int order, uint32_t *out);

HS_API const char *hs_status_str(hs_status s);
HS_API const char *hs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HS_H */
