/*
 * ddsp.h -- C ABI of the B300 (sm_103a) brute-force dedispersion and boxcar
 * single-pulse search library (libddsp.so).
 *
 * The method is the hot path of a radio transient / pulsar search:
 *   1. the dispersion delay of every (trial DM, channel) pair from the cold-
 *      plasma law of Ch.1 Eq.1, dt = 4148.808 s MHz^2 * DM * (f^-2 - f_ref^-2),
 *      rounded to the nearest sample (ties away from zero);
 *   2. brute-force incoherent dedispersion (Sec.3.2): every trial is the sum
 *      over channels of the channel's samples shifted by its delay;
 *   3. the single-pulse search (Sec.2.1): time-domain boxcar filtering of
 *      every dedispersed series, normalised by a robust median / MAD noise
 *      estimate (Sec.3.3), keeping the samples whose S/N reaches a user
 *      threshold.
 *
 * Conventions shared by every call
 *   - All pointers named d_* are DEVICE pointers owned by the caller (for
 *     example the data_ptr() of a CUDA tensor); all others are host pointers
 *     owned by the caller.  The plan owns its own workspaces.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     take a stream are asynchronous and stream-ordered: they return once the
 *     work is enqueued.  ddsp_candidates_fetch and the *_get_* calls
 *     synchronise: reads of a search's results wait for that search only
 *     (an event recorded after it), not for work queued behind it on the
 *     same stream, and copy through a plan-owned non-blocking stream, so a
 *     pipeline can fetch block k's candidates while block k+1 is being
 *     dedispersed.
 *   - Every call returns DDSP_OK (0) or a negative DDSP_E_* code; no C++
 *     exception crosses this boundary.  A plan is not thread-safe: use one
 *     plan per host thread / stream.
 *   - Frequencies are in MHz, times in seconds, DMs in pc cm^-3.
 */
#ifndef DDSP_H
#define DDSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ddsp_stream_t; /* same type as cudaStream_t */
typedef struct ddsp_plan ddsp_plan;        /* opaque; owned by the library */

/* One single-pulse candidate (Sec.2.1): DM-trial index into the plan's DM
 * list, output sample t (sample of arrival at the highest channel
 * frequency), index of the best boxcar width into the plan's width list, and
 * that width's S/N in FP32. */
typedef struct {
    uint32_t dm_idx;
    uint32_t t;
    uint32_t w_idx;
    float snr;
} ddsp_cand;

enum {
    DDSP_OK = 0,
    DDSP_E_INVALID_ARG = -1, /* bad argument (see each call)                     */
    DDSP_E_SHAPE = -2,       /* input too short / too long for the plan          */
    DDSP_E_CUDA = -3,        /* a CUDA runtime call or kernel launch failed      */
    DDSP_E_NOMEM = -4,       /* device or host allocation failed                 */
    DDSP_E_TIMEOUT = -5,     /* a bounded device wait expired (kernel returned)  */
    DDSP_E_TRUNCATED = -6,   /* more candidates than capacity; count still exact */
    DDSP_E_RANGE = -7,       /* a series window spans >= 2^31 (MAD undefined)    */
    DDSP_E_STATE = -8        /* call out of order (e.g. fetch before a search)   */
};

/*
 * ddsp_plan_create -- validate the search parameters and build the plan.
 *
 *   nchan        channels (> 0); channel c is centred at f_top + c*chan_bw
 *   f_top_mhz    frequency of channel 0 (> 0)
 *   chan_bw_mhz  channel spacing, non-zero, either sign
 *   tsamp_s      sampling time (> 0)
 *   dm_list      ndm trial DMs (finite, >= 0), any order; host array, copied
 *   widths       nwidths boxcar widths, each a power of two in [1, 1024],
 *                strictly increasing; host array, copied
 *   nbits        8 or 16: sample type of the filterbank (uint8 / uint16)
 *   norm_window  L, samples per median/MAD window (0 = one window over the
 *                whole series); windows are [jL,(j+1)L), the last one
 *                extended to the end of the series
 *   cand_capacity  candidate records kept per search (> 0)
 *
 * The delay table d[k][c] = round_half_away(4148.808*DM_k*(f_c^-2 -
 * f_ref^-2)/tsamp) (Ch.1 Eq.1, f_ref the highest channel frequency) is built
 * on the host in FP64 and copied to the device.  Returns DDSP_E_INVALID_ARG
 * for any bad argument, DDSP_E_NOMEM / DDSP_E_CUDA on allocation failure.
 * On success *out owns every plan resource until ddsp_plan_destroy.
 */
int ddsp_plan_create(ddsp_plan **out, int nchan, double f_top_mhz,
                     double chan_bw_mhz, double tsamp_s, const double *dm_list,
                     int ndm, const int *widths, int nwidths, int nbits,
                     int64_t norm_window, size_t cand_capacity);

/* The delay table alone, on the host, without a plan or a GPU: the same
 * FP64 expression ddsp_plan_create uses (Ch.1 Eq.1).  host_out[ndm*nchan]
 * receives d[k][c]; *max_delay (may be NULL) receives D.  Arguments are
 * checked as in ddsp_plan_create. */
int ddsp_delay_table(int nchan, double f_top_mhz, double chan_bw_mhz,
                     double tsamp_s, const double *dm_list, int ndm,
                     int32_t *host_out, int32_t *max_delay);

/* Output samples per trial for nsamp_in input samples: N_out = N_in - D,
 * D the largest delay of the plan.  DDSP_E_SHAPE if N_out <= 0. */
int ddsp_plan_nsamp_out(const ddsp_plan *plan, int64_t nsamp_in, int64_t *nsamp_out);

/* Largest delay D (samples) over the whole (DM, channel) grid. */
int ddsp_plan_max_delay(const ddsp_plan *plan, int32_t *max_delay);

/* Copy the plan's delay table into host_out[ndm*nchan], row k = DM trial k in
 * the order given to ddsp_plan_create. */
int ddsp_plan_get_delays(const ddsp_plan *plan, int32_t *host_out);

/* Unpack (step 2 of the path): time-major spectra d_in[nsamp_in][nchan]
 * (uint8 or uint16 as the plan's nbits, the block layout of Sec.2.2) into
 * channel-major rows d_out[nchan][pitch] of the same type; samples
 * nsamp_in..pitch-1 of every row are written as zero.  pitch >= nsamp_in and
 * a multiple of 128; d_in and d_out 16-byte aligned. */
int ddsp_unpack(ddsp_plan *plan, const void *d_in, int64_t nsamp_in,
                void *d_out, int64_t pitch, ddsp_stream_t stream);

/* Dedisperse (Sec.3.2): d_out[k][t] = sum_c in[t + d[k][c]][c] for every DM
 * trial k (plan order) and t in [0, N_out), N_out = nsamp_in - D, exact in
 * int32.  d_in: time-major spectra [nsamp_in][nchan] (uint8/uint16), 16-byte
 * aligned.  d_out: int32 [ndm][N_out], rows contiguous.  Stages the block
 * into plan-owned rows (ddsp_stage; the workspace grows on demand with
 * cudaMalloc, so the first call for a new size synchronises) and then runs
 * the dedispersion kernel (ddsp_dedisperse_staged).  DDSP_E_SHAPE if
 * N_out <= 0. */
int ddsp_dedisperse(ddsp_plan *plan, const void *d_in, int64_t nsamp_in,
                    int32_t *d_out, ddsp_stream_t stream);

/* The two halves of ddsp_dedisperse, so that a block can be staged on one
 * stream position and dedispersed on the next (and each timed alone).
 * ddsp_stage: unpack the time-major block d_in[nsamp_in][nchan] (as in
 * ddsp_dedisperse) into the plan-owned staging rows of the current tile
 * shape: channel-major rows, or for DDSP_TILE_INTERLEAVED the interleaved
 * rows that tile reads (4 bytes per uint8 sample, 2 per uint16 sample;
 * uint8 plans with nchan % 16 == 0 write them in one pass straight from
 * d_in).  DDSP_E_SHAPE if N_out <= 0.  ddsp_dedisperse_staged: dedisperse
 * the staged block into d_out[ndm][nsamp_out]; nsamp_out must equal the
 * staged block's N_out (DDSP_E_SHAPE otherwise); DDSP_E_STATE if nothing
 * is staged (a tile change drops the staged block).  Both are stream-
 * ordered: a stage must not be overwritten by the next ddsp_stage before
 * the dedispersion that reads it has run (same stream, or an event). */
int ddsp_stage(ddsp_plan *plan, const void *d_in, int64_t nsamp_in,
               ddsp_stream_t stream);
int ddsp_dedisperse_staged(ddsp_plan *plan, int64_t nsamp_out, int32_t *d_out,
                           ddsp_stream_t stream);

/* Dedisperse from channel-major rows already on the device (for example
 * the output of ddsp_unpack, or a per-beam ring kept in that layout):
 * d_cm[nchan][pitch] of the plan's sample type, 16-byte aligned; pitch a
 * multiple of 128 and at least ddsp_plan_cm_pitch(nsamp_out); samples
 * beyond nsamp_out + D of every row must be readable (they are read but do
 * not reach any stored output).  d_out as in ddsp_dedisperse.  With
 * DDSP_TILE_INTERLEAVED the rows are first interleaved into the plan's
 * staging rows (one extra streaming kernel). */
int ddsp_dedisperse_cm(ddsp_plan *plan, const void *d_cm, int64_t pitch,
                       int64_t nsamp_out, int32_t *d_out, ddsp_stream_t stream);

/* Smallest channel-major row pitch (samples) ddsp_dedisperse_cm accepts for
 * nsamp_out output samples with the plan's current tile shape. */
int ddsp_plan_cm_pitch(const ddsp_plan *plan, int64_t nsamp_out, int64_t *pitch);

/* Single-pulse search (Sec.2.1 with the Sec.3.3 median noise estimate) over
 * d_series[ndm][nsamp_out] (int32, e.g. the output of ddsp_dedisperse):
 *   per (k, window j): m = median, MAD = median |x - m| (exact integers),
 *     sigma = 1.482602218505602 * MAD;
 *   per (k, t) and width w with t + w <= nsamp_out:
 *     B_w(t) = sum_{i<w} x[t+i] (exact), S/N_w = (B_w - w*m)/(sigma*sqrt(w))
 *     in FP32 (0 when MAD = 0), best = first width reaching the maximum;
 *   a candidate is every (k, t) whose best S/N >= threshold (> 0).
 * Candidates go to a plan-owned device buffer (capacity from plan creation);
 * read them with ddsp_candidates_fetch.  A window of up to 49152 samples
 * (with the max width - 1 samples after it) is searched on chip in one
 * pass; longer windows (norm_window = 0 over a long series, or a long L)
 * take two: an exact median / MAD pass over global memory, then the search
 * in segments of 8192 start times.  Boxcar sums must fit in int32. */
int ddsp_single_pulse_search(ddsp_plan *plan, const int32_t *d_series,
                             int64_t nsamp_out, float threshold,
                             ddsp_stream_t stream);

/* Same search without the threshold, for checking: per (k, t) writes the
 * best width index (-1 where no width fits), its FP32 S/N and its boxcar sum
 * B to d_best_w / d_best_snr / d_best_sum, each [ndm][nsamp_out]. */
int ddsp_single_pulse_search_dense(ddsp_plan *plan, const int32_t *d_series,
                                   int64_t nsamp_out, int32_t *d_best_w,
                                   float *d_best_snr, int32_t *d_best_sum,
                                   ddsp_stream_t stream);

/* The single-pulse search of ddsp_single_pulse_search for callers that
 * cannot allocate device memory (a fixed device-memory budget, a real-time
 * loop that must not stall on an allocation, or a host that only hands out
 * pre-allocated buffers).  There is no counterpart in the paper: it is the
 * same search, only without a plan.  Nothing is allocated: the scratch
 * (per-(DM trial, window) statistics, the width table, an error word) is a
 * static device array of the library of a little over 4 MiB, which every
 * GPU that loads the library holds until exit.
 *   d_series   int32 [ndm][nsamp_out] on the current device
 *   widths     nwidths boxcar widths (host array, as in ddsp_plan_create);
 *              they reach the device as a kernel argument of a small
 *              set-up launch (no host-to-device copy), which also zeroes
 *              *d_count and the error word
 *   norm_window, threshold  as in ddsp_plan_create / the plan search
 *   d_cands    caller's device buffer of cand_capacity records; the
 *              candidates come back unsorted
 *   d_count    caller's device uint32: the true number of candidates (may
 *              exceed cand_capacity; only that many records are written)
 * Rejects ndm * (number of windows) > 262144 and windows longer than the
 * plan search allows with DDSP_E_SHAPE, bad arguments with
 * DDSP_E_INVALID_ARG.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress); make it before any stream
 * capture.  Every call uses the same array: calls whose work overlaps on a
 * GPU (different streams, or different host threads) race and must be
 * serialised by the caller.  A window whose values span 2^31 or more gives
 * no candidates (its MAD is taken as 0) and sets the error word, which
 * ddsp_single_pulse_search_noalloc_check reports.  Asynchronous on
 * `stream`. */
int ddsp_single_pulse_search_noalloc(const int32_t *d_series, int ndm,
                                     int64_t nsamp_out, const int *widths,
                                     int nwidths, int64_t norm_window,
                                     float threshold, ddsp_cand *d_cands,
                                     uint32_t cand_capacity,
                                     uint32_t *d_count, ddsp_stream_t stream);

/* Synchronise `stream` and report the error word the last allocation-free
 * search on the current device left in the shared static scratch:
 * DDSP_E_RANGE if a window's values spanned 2^31 or more (its candidates
 * were dropped), DDSP_OK otherwise; the word is then cleared.  No
 * counterpart in the paper; allocates nothing.  The word is shared like the
 * rest of the scratch, so it belongs to whichever call ran last. */
int ddsp_single_pulse_search_noalloc_check(ddsp_stream_t stream);

/* Copy the per-(DM, window) statistics of the last search to the host:
 * m2[k*nwin + j] = 2*median, mad4[k*nwin + j] = 4*MAD (both exact).  *nwin
 * receives the window count.  Waits for the last search.
 * host arrays may be NULL to query *nwin only. */
int ddsp_plan_get_stats(ddsp_plan *plan, int64_t *m2, int64_t *mad4,
                        int64_t cap, int64_t *nwin);

/* Wait for the last search, copy up to min(cap, capacity) candidates to
 * host_buf sorted by (dm_idx, t), and set *n_total to the true number found.
 * Returns DDSP_E_TRUNCATED when *n_total exceeds what was copied (the copied
 * records are then the first ones the device stored, sorted),
 * DDSP_E_TIMEOUT / DDSP_E_RANGE if a kernel reported one, DDSP_E_STATE if no
 * search ran. */
int ddsp_candidates_fetch(ddsp_plan *plan, ddsp_cand *host_buf, size_t cap,
                          size_t *n_total);

/* Wait for the last search and report only the number of candidates it
 * found (no records are copied).  Error codes as ddsp_candidates_fetch. */
int ddsp_candidates_count(ddsp_plan *plan, size_t *n_total);

/* Like ddsp_candidates_fetch, restricted to DM-trial indices in
 * [dm_lo, dm_hi): the stored records are streamed to the host in bounded
 * pieces and filtered there, so a caller can inspect a few DM rows of a very
 * large candidate set without a host buffer for all of it.  *n_range gets
 * the number of stored records in the range, *n_total the device count.
 * DDSP_E_TRUNCATED if *n_range > cap or the device count exceeded the
 * capacity (some records of the range may then be missing). */
int ddsp_candidates_fetch_dm_range(ddsp_plan *plan, uint32_t dm_lo,
                                   uint32_t dm_hi, ddsp_cand *host_buf,
                                   size_t cap, size_t *n_range,
                                   size_t *n_total);

/* Synchronise `stream` and report any error a kernel of this plan recorded
 * on the device (DDSP_E_TIMEOUT, DDSP_E_RANGE), then clear it. */
int ddsp_plan_check(ddsp_plan *plan, ddsp_stream_t stream);

/* Release every resource of the plan (NULL is ignored). */
void ddsp_plan_destroy(ddsp_plan *plan);

/* Static, human-readable text for a DDSP_* code. */
const char *ddsp_error_string(int code);

/* ---------------------------------------------------------------------
 * Batches: many beams of uneven shape (channel counts, block lengths, DM
 * grids) searched together.  One step = a batched unpack launch, ONE
 * persistent dedispersion launch whose blocks take (beam, DM tile, time
 * tile) work items from a device queue, and a batched search launch; the
 * step can be replayed from a captured CUDA graph.  Every beam's results are
 * the same as its plan would give alone (same exact sums).
 * --------------------------------------------------------------------- */
typedef struct ddsp_batch ddsp_batch;

/* Create a batch over `nbeams` plans (uint8, nchan a multiple of 16, all on
 * the current device); nsamp_in[b] input samples per beam.  The batch owns
 * each beam's channel-major input rows (filled by ddsp_batch_ingest from a
 * time-major block, or written directly: see ddsp_batch_input).  Output
 * series [ndm][nsamp_out] go to d_series[b] (caller-owned device buffers
 * that must outlive the batch) or, where d_series or d_series[b] is NULL, to
 * buffers the batch allocates (ddsp_batch_series); candidates go to each
 * plan's own buffer (read them with ddsp_candidates_fetch on that plan
 * after ddsp_batch_run).  The plans must outlive the batch.  Chooses a
 * common tile shape that fits every beam.  DDSP_E_SHAPE if a block is
 * shorter than its plan's largest delay. */
int ddsp_batch_create(ddsp_batch **out, ddsp_plan *const *plans, int nbeams,
                      const int64_t *nsamp_in, int32_t *const *d_series);
void ddsp_batch_destroy(ddsp_batch *batch);

/* Unpack (step 2 of the path) a beam's time-major block d_in[nsamp_in]
 * [nchan] (16-byte aligned, the caller's) into the batch's channel-major
 * rows of that beam.  Asynchronous on `stream`. */
int ddsp_batch_ingest(ddsp_batch *batch, int beam, const void *d_in,
                      ddsp_stream_t stream);

/* Device pointer and row pitch (samples) of a beam's channel-major rows
 * [nchan][pitch] (rows past nsamp_in must hold zeros or any readable
 * bytes), and of its output series [ndm][nsamp_out]. */
int ddsp_batch_input(ddsp_batch *batch, int beam, void **d_cm, int64_t *pitch,
                     int64_t *nsamp_in);
int ddsp_batch_series(ddsp_batch *batch, int beam, int32_t **d_series,
                      int64_t *nsamp_out);

/* One batch step on `stream` (asynchronous): persistent dedispersion and
 * single-pulse search (threshold > 0) of every beam's ingested rows.  With
 * use_graph != 0 the step is captured once into a CUDA graph (on an
 * internal stream) and replayed on `stream` afterwards; the first call
 * after creation or a tile change runs directly.  Synchronises only when it
 * (re)captures. */
int ddsp_batch_run(ddsp_batch *batch, float threshold, int use_graph,
                   ddsp_stream_t stream);

/* Synchronise `stream` and report a device-side timeout or range error of
 * the last batch step (DDSP_E_TIMEOUT / DDSP_E_RANGE), then clear it. */
int ddsp_batch_check(ddsp_batch *batch, ddsp_stream_t stream);

/* The batch's main warp-specialised tile (see ddsp_plan_set_tile) and its
 * persistent grid size.  All beams share dm_tile, dm_per_thread and stages;
 * chan_chunk (1..32) is an upper limit: each beam stages the largest chunk
 * up to it whose buffers (which grow with the beam's delay span inside a
 * DM tile) fit two blocks per SM, or one block per SM if some beam fits
 * only that way.  set_tile returns DDSP_E_INVALID_ARG if the shape does not
 * fit every beam on chip.  Both synchronise. */
int ddsp_batch_set_tile(ddsp_batch *batch, int dm_tile, int dm_per_thread,
                        int chan_chunk, int stages);
int ddsp_batch_get_tile(const ddsp_batch *batch, int *dm_tile,
                        int *dm_per_thread, int *time_tile, int *chan_chunk,
                        int *stages, int *grid);

/* The channel chunk beam `beam` stages under the current tile. */
int ddsp_batch_get_beam_chunk(const ddsp_batch *batch, int beam,
                              int *chan_chunk);

/* The shape beam `beam` is dedispersed with: beams whose DM grid is coarse
 * for the main shape (fewer than 2 channels per chunk, or a narrower-DM
 * shape relayouts at least 30 % fewer bytes per add) go to a second
 * persistent launch of the same step with that narrower shape; *group is 0
 * (main) or 1 (that launch).  Any pointer may be NULL. */
int ddsp_batch_get_beam_tile(const ddsp_batch *batch, int beam, int *dm_tile,
                             int *dm_per_thread, int *time_tile,
                             int *chan_chunk, int *group);

/* Autotuner: for each tile shape of the library's candidate list, time the
 * persistent dedispersion of every 16th work item of the cost-ordered work
 * list (the same share of each beam's work; best of `reps` runs after one
 * warm-up, on the current input buffers) and keep the fastest; then time
 * one whole pass of the per-beam interleaved mode (DDSP_BATCH_PER_BEAM,
 * when every beam fits an interleaved shape) and take it if it is
 * faster.  ms_out[i] (up to cap entries, may be NULL) receives candidate
 * i's time scaled to the full work list, or -1 if the shape does not fit;
 * the last candidate is the per-beam mode; *ntried the number of
 * candidates, *best the chosen index.  The runs overwrite the output
 * series. */
int ddsp_batch_autotune(ddsp_batch *batch, int reps, ddsp_stream_t stream,
                        float *ms_out, int cap, int *ntried, int *best);

/* Execution mode of ddsp_batch_run.  DDSP_BATCH_PERSISTENT: persistent
 * launches of the warp-specialised relayout kernel over a device work
 * queue of every beam's (DM tile, time tile) items (the tile from
 * ddsp_batch_set_tile or the autotuner).  DDSP_BATCH_PER_BEAM: beam after
 * beam, its channel-major rows interleaved into one staging area the
 * batch owns (4 bytes per sample of the largest beam; allocated on the
 * first switch) and dedispersed by the interleaved kernel (per beam the
 * first of the 16-trial wide, 16-trial, 8-trial and 4-trial interleaved
 * shapes whose staging fits: coarse DM grids take the narrower ones), then
 * the same batched search.  set_mode returns DDSP_E_INVALID_ARG for an
 * unknown mode or if some beam fits none of those shapes, DDSP_E_NOMEM if
 * the staging area cannot be allocated;
 * ddsp_batch_set_tile switches back to DDSP_BATCH_PERSISTENT.  Both modes
 * compute the same exact sums. */
#define DDSP_BATCH_PERSISTENT 0
#define DDSP_BATCH_PER_BEAM 1
int ddsp_batch_set_mode(ddsp_batch *batch, int mode);
int ddsp_batch_get_mode(const ddsp_batch *batch, int *mode);

/* ---- Streaming server (the real-time ring-buffer design of Sec.2.1 and
 * Ch.3: every beam delivers blocks of B new spectra, each block is
 * dedispersed and searched once the GPU is free, together with the blocks
 * other beams have waiting).
 *
 * All beams have the shape of `plan` (channels, band, DM trials, widths,
 * normalisation window, candidate capacity per block; uint8 samples,
 * nchan a multiple of 16).  Per admitted beam the server owns a
 * channel-major ring of ceil(D16/B) + 1 blocks (D16 = the largest delay
 * rounded up to 16 samples) whose rows end in a copy of their first bytes,
 * the carry [ndm][C] (C = widest boxcar - 1 rounded up to 4: the last C
 * outputs of the previous block), per-window statistics and two candidate
 * buffers.  Block j (0, 1, ...) is dedispersed for output samples s_j ..
 * s_j + B - 1 with s_j = j*B - D16 (input before the stream's first sample
 * reads as 0) into a series [ndm][C + B] whose first C columns are the
 * carry, and searched for start times 0 .. B - 1 of the series, normalised
 * per window of the C + B columns as ddsp_single_pulse_search does:
 * candidate t is global output sample s_j - C + t.  The results equal those
 * of ddsp_dedisperse and ddsp_single_pulse_search on the same input
 * window.  The series live in G series slots the server shares among the
 * beams: a step runs its beam-blocks in groups of G (16 in the relayout
 * mode, the staging slot count in the interleaved mode), each group's
 * dedispersion, search and carry in turn. */
typedef struct ddsp_server ddsp_server;

/* Create a server for up to max_beams beams of plan's shape receiving
 * blocks of block_samples (a multiple of 16 and of the tile's time tile,
 * >= C) spectra.  hbm_reserve_bytes: device memory admission leaves free.
 * dm_tile = 0 lets the server choose the warp-specialised tile (see
 * ddsp_plan_set_tile; chan_chunk is an upper limit), else the given shape.
 * The plan must outlive the server; its own buffers are not used.
 * DDSP_E_SHAPE if the block is too short for the tile or the search window
 * (see ddsp_single_pulse_search), DDSP_E_INVALID_ARG for a shape the kernel
 * does not implement. */
int ddsp_server_create(ddsp_server **out, ddsp_plan *plan,
                       int64_t block_samples, int max_beams,
                       int64_t hbm_reserve_bytes, int dm_tile,
                       int dm_per_thread, int chan_chunk, int stages);
void ddsp_server_destroy(ddsp_server *server);

/* Device bytes one admitted beam holds, ring length (samples), series
 * columns (C + B), carry C and the output lag D16 (any pointer may be
 * NULL). */
int ddsp_server_info(const ddsp_server *server, int64_t *beam_bytes,
                     int64_t *ring_samples, int64_t *series_cols,
                     int64_t *carry, int64_t *first_delay);
int ddsp_server_get_tile(const ddsp_server *server, int *dm_tile,
                         int *dm_per_thread, int *time_tile, int *chan_chunk,
                         int *stages, int *grid);

/* Admission: allocate and zero a new beam's ring and buffers if the device's
 * free memory, less the reserve, holds them; *beam = its index.
 * DDSP_E_NOMEM if it does not fit, DDSP_E_RANGE if max_beams are admitted.
 * Synchronises.  Evict frees a beam (synchronises the device first). */
int ddsp_server_admit(ddsp_server *server, int *beam);
int ddsp_server_evict(ddsp_server *server, int beam);

/* Ingest the beam's next block: d_block is time-major uint8 [B][nchan] in
 * device memory (16-byte aligned), read by kernels on `stream` (the caller
 * keeps it unchanged until they ran).  The block's ring slot last served the
 * step of block j - 1, which `stream` waits for.  DDSP_E_STATE if block j - 1
 * has not been given to a step yet (one block per beam waits for a step):
 * run a step first (the caller holds the block meanwhile). */
int ddsp_server_push(ddsp_server *server, int beam, const void *d_block,
                     ddsp_stream_t stream);

/* One step on `stream` (asynchronous): every admitted beam with a pushed,
 * unsearched block contributes its oldest such block (max_beams_in_step > 0:
 * only that many beams, those whose block was pushed first); each group of
 * G of them is carried in, dedispersed (one persistent launch, or the
 * interleaves and one interleaved launch), searched (one batched launch)
 * and carried out.
 * *nbeams = the number of beams in the step (0: nothing was launched),
 * their indices in beams_out (up to cap entries, may be NULL), *step_id its
 * number for ddsp_server_query.  Waits on the host for the step before the
 * previous one, whose descriptor staging it reuses. */
int ddsp_server_step(ddsp_server *server, float threshold,
                     int max_beams_in_step, ddsp_stream_t stream,
                     int64_t *step_id, int *beams_out, int cap, int *nbeams);

/* 1 if step step_id has completed, 0 if it is still running; negative on
 * error. */
int ddsp_server_query(ddsp_server *server, int64_t step_id);

/* Candidates of block `block` of a beam (one of its two most recently
 * stepped blocks; DDSP_E_STATE otherwise), after waiting for its step:
 * records sorted by (dm_idx, t), t relative to series column 0, *t_start =
 * that column's global output sample (s_j - C).  As ddsp_candidates_fetch for cap,
 * *n_found and DDSP_E_TRUNCATED. */
int ddsp_server_fetch(ddsp_server *server, int beam, int64_t block,
                      ddsp_cand *host_buf, size_t cap, size_t *n_found,
                      int64_t *t_start);

/* Device pointer of the series [ndm][ncols] of a beam's last stepped block
 * (valid once its step completed, until the next step): its series slot (a
 * step runs its beam-blocks in groups of G, the k-th in slot k mod G), which
 * is reported only if the block was in the latest step's last group;
 * DDSP_E_STATE otherwise. */
int ddsp_server_series(ddsp_server *server, int beam, int32_t **d_series,
                       int64_t *ncols);

/* Synchronise `stream` and report a device-side timeout or range error of
 * the server's steps, then clear it. */
int ddsp_server_check(ddsp_server *server, ddsp_stream_t stream);

/* Dedispersion mode of the server's steps.  DDSP_SERVER_RELAYOUT (the
 * default): one persistent launch of the warp-specialised relayout kernel
 * over every waiting beam-block's work items, staging straight from the
 * rings.  DDSP_SERVER_INTERLEAVED: each waiting beam-block's window of its
 * ring is interleaved into one of `staging_slots` (1..16) staging slots
 * the server allocates (4 * nchan * (B + D16 + 64, rounded up to 128)
 * bytes each; set the mode before admitting beams, so admission sees the
 * memory), and each group of slots is dedispersed by one launch of the
 * interleaved kernel; the search is the same.  The mode also sets the
 * series slots (16 for the relayout mode, staging_slots for the
 * interleaved one; 4 * ndm * (C + B) bytes each).  Synchronises the device.
 * DDSP_E_INVALID_ARG for an unknown mode, a slot count outside 1..16 or a
 * shape no interleaved tile fits (the time tile must divide the block);
 * DDSP_E_NOMEM if the slots cannot be allocated.  Both modes compute the
 * same exact sums. */
#define DDSP_SERVER_RELAYOUT 0
#define DDSP_SERVER_INTERLEAVED 1
int ddsp_server_set_mode(ddsp_server *server, int mode, int staging_slots);
int ddsp_server_get_mode(const ddsp_server *server, int *mode,
                         int *staging_slots);

/* Name and text of the last CUDA error this library saw on the calling
 * host thread (empty if none); the storage is the library's. */
const char *ddsp_last_error_detail(void);

/* Tile shape of the dedispersion kernel.  A block of 8 (consumer) warps
 * computes dm_tile DM trials x time_tile output samples; each thread owns
 * dm_per_thread (2, 4 or 8) trials x 16 samples; chan_chunk channels (1..32)
 * are staged per pipeline step with `stages` (2..4) raw-window buffers.
 * dm_tile must be dm_per_thread x {1, 2, 4}; time_tile follows from it.
 * flags: DDSP_TILE_SINGLE_ELEM_BUFFER (one relayout buffer, two barriers
 * per chunk, less shared memory), DDSP_TILE_REGISTER_TOTALS (int32 totals
 * kept in registers instead of being accumulated in the output array every
 * <= 256 channels; uint8 plans accept it only together with
 * DDSP_TILE_SINGLE_ELEM_BUFFER, uint16 plans always keep their totals in
 * registers and accept 0 or DDSP_TILE_SINGLE_ELEM_BUFFER), or
 * DDSP_TILE_WARP_SPECIALIZED alone (producer warps stage and relayout,
 * consumer warps accumulate, no block-wide barrier in the main loop;
 * dm_per_thread 4, or 8 for uint8; stages 2 or 4, since each of the two
 * producer warps owns every other chunk and half the stages), or
 * DDSP_TILE_INTERLEAVED alone (the default where it fits: rows interleaved
 * once per block of data in HBM, element i = {x[i], x[i+S], x[i+2S],
 * x[i+3S]} for the tile's segment S, are copied by TMA straight into a
 * ring of `stages` (2..8) element stages of chan_chunk channels each; one
 * producer warp, eight consumer warps; dm_per_thread 4, or 8 for uint8),
 * optionally with DDSP_TILE_WIDE (sixteen consumer warps and one block per
 * SM: time_tile doubles for the same dm_tile).  Every variant computes the
 * same exact sums.  dm_tile = 0 restores the library's choice, dm_tile = -1
 * selects the direct (unstaged) kernel.  DDSP_E_INVALID_ARG for a shape the
 * kernel does not implement or whose staging does not fit on chip.
 * Synchronises. */
#define DDSP_TILE_SINGLE_ELEM_BUFFER 1
#define DDSP_TILE_REGISTER_TOTALS 4
#define DDSP_TILE_WARP_SPECIALIZED 8
#define DDSP_TILE_INTERLEAVED 16
#define DDSP_TILE_WIDE 32
int ddsp_plan_set_tile(ddsp_plan *plan, int dm_tile, int dm_per_thread,
                       int chan_chunk, int stages, int flags);
int ddsp_plan_get_tile(const ddsp_plan *plan, int *dm_tile,
                       int *dm_per_thread, int *time_tile, int *chan_chunk,
                       int *stages, int *flags);

/* Tile autotuning of a single-beam plan, with a cache (no counterpart in
 * the paper: which dedispersion tile shape runs fastest depends on the
 * channel count, the DM grid's delay spans and the GPU).
 * ddsp_plan_autotune: time the candidate tiles the plan's shape fits (the
 * interleaved kernel with 16 or 8 consumer warps and 4..32 DM trials per
 * tile, the relayout kernel), each the best of `reps` passes of
 * ddsp_stage + ddsp_dedisperse_staged over the caller's block d_in (as in
 * ddsp_dedisperse), keep the fastest on the plan, and, if cache_path is
 * not NULL, record it in that JSON file under the plan's key, replacing an
 * older entry of the key.  ms (cap entries, may be NULL) receives each
 * candidate's best time in ms (-1: does not fit), *best (may be NULL) the
 * winner's index.  Allocates a scratch output of ndm * N_out int32 for the
 * time of the call; synchronises.  DDSP_E_SHAPE if N_out <= 0.
 * ddsp_plan_tile_key: the key ("<GPU name>/nchan=.../nbits=.../ndm=.../
 * D=.../span16=...", the largest delay span inside a 16-trial DM tile) into
 * buf (cap bytes with the terminating 0; DDSP_E_INVALID_ARG if too short).
 * ddsp_plan_create uses the tile cached under the new plan's key in the
 * file named by the environment variable DDSP_TILE_CACHE, if there is one
 * that fits, instead of its built-in choice.
 * ddsp_tile_cache_get / _put: read or write one entry of a cache file on
 * the host (tile = dm_tile, dm_per_thread, chan_chunk, stages, flags as
 * ddsp_plan_set_tile takes them; keys without '"', '\\' or control
 * characters); get returns DDSP_E_STATE when the key is absent and
 * DDSP_E_INVALID_ARG for a file that does not parse; a missing file is an
 * empty cache. */
int ddsp_plan_autotune(ddsp_plan *plan, const void *d_in, int64_t nsamp_in,
                       const char *cache_path, int reps,
                       ddsp_stream_t stream, float *ms, int cap, int *best);
int ddsp_plan_tile_key(const ddsp_plan *plan, char *buf, size_t cap);
int ddsp_tile_cache_get(const char *path, const char *key, int *tile,
                        float *ms);
int ddsp_tile_cache_put(const char *path, const char *key, const int *tile,
                        float ms);

/* Failure detection of the dedispersion (no counterpart in the paper).
 * Every device wait of the staged kernels is bounded: when a bound runs out
 * the kernel records DDSP_E_TIMEOUT in the plan's error word, lets the
 * copies it already issued land, and returns, so the context stays usable
 * and ddsp_plan_check / ddsp_candidates_fetch report the error.
 * ddsp_plan_set_wait_limit: the bound of the copy/compute hand-off waits of
 * the interleaved kernel (DDSP_TILE_INTERLEAVED, the default tile), in SM
 * clock cycles; 0 restores the default of 4e9 (about 2 s at 2 GHz).  The
 * waits a block makes for its own copies in flight before it exits keep
 * the default bound.  ddsp_plan_withhold_copy: a switch for testing that
 * path without a fault: chunk >= 0 makes the copy-issuing warp of every
 * block of the interleaved kernel stop before that chunk of channels, so
 * the computing warps' bounded wait for it runs out; -1 (the default)
 * turns it off.  Neither call synchronises; both apply from the next
 * dedispersion on.  DDSP_E_INVALID_ARG for a negative limit or a chunk
 * below -1. */
int ddsp_plan_set_wait_limit(ddsp_plan *plan, int64_t cycles);
int ddsp_plan_withhold_copy(ddsp_plan *plan, int chunk);

/* Bounds-checked build (no counterpart in the paper): the library compiled
 * with -DDDSP_BOUNDS_CHECK (libddsp_bounds.so, for tests) checks the index
 * of every shared- and global-memory access of the staging, interleave,
 * dedispersion and search kernels against its buffer before making it; a
 * failing check skips the access and records the first violation as
 * (site << 32 | low 32 bits of the index) in one device word.  Synchronises
 * the device, sets *enabled (1 in the checked build, 0 otherwise) and
 * *violation (0: none), then clears the word. */
int ddsp_bounds_check_status(int *enabled, uint64_t *violation);

/* ------------------------------------------------------------------------
 * Unit peaks (measurement): microbenchmarks of the on-chip units the
 * dedispersion is bound by, per SM and SM clock, each over one full wave of
 * identical blocks timed by clock64 (an SM's rate = the work of its blocks
 * over the span from their first start to their last end; the median SM):
 *   smem_bytes_per_clk  conflict-free 32-bit shared-memory loads;
 *   iadd3_per_clk       3-input integer adds (lane operations);
 *   prmt_per_clk        byte permutes (lane operations);
 *   swar_adds_per_clk   the dedispersion inner loop as the default tile
 *                       runs it (4 DM trials x 32 samples per thread, two
 *                       channels per step, B's adds on the FMA pipe) on
 *                       channels resident in shared memory: sample adds.
 * blocks_per_sm: the resident blocks of each probe, in that order.
 * Allocates and frees a few MB on `device`; synchronises.  Returns
 * DDSP_E_INVALID_ARG for a bad device or out == NULL.
 * ------------------------------------------------------------------------ */
typedef struct {
    int sms;
    int blocks_per_sm[4];
    double smem_bytes_per_clk;
    double iadd3_per_clk;
    double prmt_per_clk;
    double swar_adds_per_clk;
} ddsp_unit_peaks;
int ddsp_probe_unit_peaks(int device, ddsp_unit_peaks *out);

/* ------------------------------------------------------------------------
 * Peaks filtering and DM-time clustering of candidates (Sec.2.1: the
 * candidate list is thinned with square stencils of different sizes in the
 * DM-time plane, the survivors are clustered with DBSCAN in that plane, and
 * the highest-S/N candidate of each cluster is kept).
 *
 *   peaks:  candidate i stays unless a stronger candidate j -- snr_j >
 *           snr_i, or equal S/N and (dm_idx_j, t_j) before (dm_idx_i, t_i)
 *           -- lies in its square stencil |dm_idx_j - dm_idx_i| <= h,
 *           |t_j - t_i| <= h, h = half[w_idx_i] (trials and samples);
 *   DBSCAN: the peaks in (dm_idx, t) order; the neighbourhood of a peak is
 *           every peak with |d dm_idx| <= eps_dm and |d t| <= eps_t, itself
 *           included; core peaks have >= min_pts neighbours; a cluster (the
 *           core peaks connected through neighbourhoods, plus the non-core
 *           peaks next to them) is labelled by the index, in the sorted peak
 *           list, of its first core peak; a non-core peak next to several
 *           clusters takes the smallest label; the rest are noise (-1);
 *   reps:   the strongest member of each cluster (ties to the earlier peak),
 *           clusters in increasing label order.
 * S/N values are compared exactly as given (FP32).
 * --------------------------------------------------------------------- */
typedef struct ddsp_cluster ddsp_cluster;

/* Workspace on `device` for planes of ndm trials x nsamp samples and up to
 * `capacity` candidates per call: two plane bitmaps with their prefix sums
 * and the largest S/N of every 32 cells of a row (about 5/8 byte per plane
 * cell) plus 72 bytes per candidate, owned by the library.  DDSP_E_INVALID_ARG if a size is <= 0, capacity >= 2^31,
 * nsamp >= 2^32 or the device does not exist; DDSP_E_NOMEM / DDSP_E_CUDA on
 * allocation failure. */
int ddsp_cluster_create(ddsp_cluster **out, int device, int ndm,
                        int64_t nsamp, int64_t capacity);
void ddsp_cluster_destroy(ddsp_cluster *cluster);

/* Filter and cluster the records d_cands[0 .. m) (device, any order, each
 * (dm_idx, t) at most once), m = n, or m = min(*d_count, n) when d_count (a
 * device counter, such as the search's own: ddsp_plan_candidates_device) is
 * given.  half: host array of nwidths (1..32) stencil half-sizes >= 0,
 * indexed by w_idx; it is read before the call returns.  Stream-ordered
 * and asynchronous.  DDSP_E_INVALID_ARG for n > capacity, a bad parameter,
 * or a negative half-size.  Records outside the plane or with w_idx >=
 * nwidths, and repeated (dm_idx, t), are found on the device and reported
 * by the fetch calls as DDSP_E_INVALID_ARG. */
int ddsp_peaks_cluster(ddsp_cluster *cluster, const ddsp_cand *d_cands,
                       const uint32_t *d_count, int64_t n,
                       const int32_t *half, int nwidths, int eps_dm,
                       int eps_t, int min_pts, ddsp_stream_t stream);

/* The peaks of the last call sorted by (dm_idx, t), and (host_labels may be
 * NULL) their cluster labels.  Synchronises with that call's stream.
 * *n_peaks is the true count; DDSP_E_TRUNCATED if it exceeds cap (cap
 * records copied); DDSP_E_STATE before any call; DDSP_E_INVALID_ARG for a
 * bad record (see ddsp_peaks_cluster); DDSP_E_TIMEOUT if a bounded device
 * loop gave up. */
int ddsp_cluster_fetch_peaks(ddsp_cluster *cluster, ddsp_cand *host_peaks,
                             int32_t *host_labels, size_t cap,
                             size_t *n_peaks);

/* The strongest member of every cluster of the last call, in increasing
 * label order, and (host_idx may be NULL) its index in the sorted peak
 * list.  Same synchronisation and error codes as ddsp_cluster_fetch_peaks. */
int ddsp_cluster_fetch_reps(ddsp_cluster *cluster, ddsp_cand *host_reps,
                            uint32_t *host_idx, size_t cap, size_t *n_reps);

/* The plan's device candidate buffer (records of the last search, in no
 * particular order), its device counter (the true count, possibly above
 * the capacity) and the capacity; valid until the plan is destroyed. */
int ddsp_plan_candidates_device(ddsp_plan *plan, const ddsp_cand **d_cands,
                                const uint32_t **d_count, size_t *capacity);

/* ------------------------------------------------------------------------
 * Downsampling and de-reddening of dedispersed series, between the
 * dedispersion and the search.  Rows of int32 series in the caller's
 * device buffers, row pitches in samples; overflow of int32 is reported
 * through the plan's error word (ddsp_plan_check returns DDSP_E_RANGE).
 * --------------------------------------------------------------------- */

/* Downsampling by a user factor (Sec.3.2): out[r][j] = sum over
 * i < factor of in[r][j*factor + i], j < nsamp / factor (a trailing partial
 * group is dropped), r < nrows; nothing is written (and d_out may be NULL)
 * when nsamp < factor.  Stream-ordered.  DDSP_E_INVALID_ARG for a NULL
 * pointer, nrows or nsamp <= 0, factor < 1, in_pitch < nsamp or
 * out_pitch < nsamp / factor. */
int ddsp_downsample(ddsp_plan *plan, const int32_t *d_in, int64_t nrows,
                    int64_t nsamp, int64_t in_pitch, int64_t factor,
                    int32_t *d_out, int64_t out_pitch, ddsp_stream_t stream);

/* Running-median de-reddening (Sec.3.3): out[r][t] = in[r][t] - m, with m
 * the median of in[r] over [t - h, t + h] clamped to [0, nsamp); a window
 * cut by an end may hold an even count, and m is then the lower of the two
 * middle values, so m is always a sample and out is exact.  h =
 * half_window, 0 .. 6700 (a chunk of outputs with its 2h-sample halo is
 * processed on chip).  Stream-ordered.  DDSP_E_INVALID_ARG for a NULL
 * pointer, d_in == d_out, nrows outside 1 .. 65535, nsamp <= 0 or >= 2^31,
 * h out of range, or a pitch < nsamp. */
int ddsp_dered(ddsp_plan *plan, const int32_t *d_in, int64_t nrows,
               int64_t nsamp, int64_t in_pitch, int64_t half_window,
               int32_t *d_out, int64_t out_pitch, ddsp_stream_t stream);

/* ------------------------------------------------------------------------
 * Folding transform and folded-profile search (Sec.3.5), for periodicity
 * searches of dedispersed (typically downsampled and de-reddened) series.
 * A series of nsamp samples is cut into m rows of p samples, m the largest
 * power of two with m*p <= nsamp (whole rows; the rest is unused), and
 * folded by the fast folding algorithm: the profile of trial s = 0 .. m-1
 * drifts by s samples over the m - 1 row steps (trial period p + s/(m-1)
 * samples), with the classic binary recursion
 *   F[s][j] = A[s/2][j] + B[s/2][(j + (s+1)/2) mod p]
 * (A, B the transforms of the two halves of a group of rows).  Sums are
 * int32; an overflow sets the plan's error word (ddsp_plan_check returns
 * DDSP_E_RANGE).  m*p <= 16384: one row's stack is folded on chip.
 * --------------------------------------------------------------------- */

/* The transform of every row at base period p: d_out[r][s][j] (nrows x m x
 * p int32, the caller's), *m set on return.  Stream-ordered.
 * DDSP_E_INVALID_ARG for a NULL pointer, nrows <= 0, pitch < nsamp,
 * p < 1, nsamp < p or m*p > 16384. */
int ddsp_ffa(ddsp_plan *plan, const int32_t *d_series, int64_t nrows,
             int64_t nsamp, int64_t pitch, int p, int32_t *d_out, int *m,
             ddsp_stream_t stream);

/* For every row r and base period p in [p_lo, p_hi): the transform, then
 * per trial s the best cyclic boxcar of the folded profile P (length p):
 *   B_w(j) = sum_{i<w} P[(j+i) mod p],
 *   S/N = (B_w(j) - w*sum(P)/p) / (sigma_r * sqrt(m*w)),
 * sigma_r = d_sigma[r] the noise of one sample of row r; widths: host list
 * of 1..16 increasing values (those > p are skipped); the best is the
 * largest S/N, ties to the smaller width index, then the smaller phase j.
 * Outputs d_snr (FP32), d_widx, d_phase, each [nrows][p_hi - p_lo][mmax]
 * (the caller's), mmax >= m(p_lo); trials s >= m(p) hold -inf, -1, -1.
 * Stream-ordered.  DDSP_E_INVALID_ARG for a NULL pointer, nrows outside
 * 1 .. 65535, pitch < nsamp, an empty or unsorted width list, p_lo < 1,
 * p_hi <= p_lo, nsamp < p_hi - 1, mmax < m(p_lo), or m*p > 16384. */
int ddsp_ffa_search(ddsp_plan *plan, const int32_t *d_series, int64_t nrows,
                    int64_t nsamp, int64_t pitch, int p_lo, int p_hi,
                    const int32_t *widths, int nwidths, const float *d_sigma,
                    float *d_snr, int32_t *d_widx, int32_t *d_phase,
                    int64_t mmax, ddsp_stream_t stream);

/* ------------------------------------------------------------------------
 * Resampling for frequency derivatives (Sec.3.4): a periodic signal of
 * frequency f0 + f1 t + f2 t^2/2 (t from the first sample, tsamp seconds per
 * sample) is brought to a constant frequency.  Output bin k lasts
 * tau_k = tsamp (1 + f' t/F + f'' t^2/(2F)) at t = k tsamp, with F = f0,
 * f' = -f1, f'' = -f2 when f1 <= 0; when f1 > 0 the series is reversed,
 * transformed with F = f0 + f1 T + f2 T^2/2, f' = f1 + f2 T, f'' = -f2
 * (T = nsamp tsamp) and the result reversed, so the signal ends at
 * frequency F.  out[k] sums the input samples the bin overlaps, each
 * weighted by the overlap in samples (FP64 arithmetic, FP32 output); the
 * bins kept are those ending within the series.
 * --------------------------------------------------------------------- */

/* The number of output bins for these parameters.  DDSP_E_INVALID_ARG for
 * nsamp < 1, tsamp <= 0, f0 <= 0 (or F <= 0), non-finite derivatives, a
 * bin width <= 0 before the end of the series, or widths averaging below
 * about one half of a sample. */
int ddsp_resample_length(int64_t nsamp, double tsamp, double f0, double f1,
                         double f2, int64_t *nout);

/* Resample every row: d_out[r][k], k < *nout (out_pitch >= *nout, the
 * caller's FP32 buffer).  Stream-ordered.  Errors as ddsp_resample_length,
 * plus DDSP_E_INVALID_ARG for a NULL pointer, nrows <= 0, in_pitch < nsamp
 * or out_pitch < *nout. */
int ddsp_resample(ddsp_plan *plan, const int32_t *d_in, int64_t nrows,
                  int64_t nsamp, int64_t in_pitch, double tsamp, double f0,
                  double f1, double f2, float *d_out, int64_t out_pitch,
                  int64_t *nout, ddsp_stream_t stream);

/* ------------------------------------------------------------------------
 * RFI mitigation of a block of 8-bit spectra, gptool style (Sec.2.1: a
 * bandpass from the mean spectrum median-filtered over 21 channels,
 * channels beyond 4 sigma of the corrected mean spectrum and time samples
 * beyond 3 sigma of the frequency-averaged series flagged, both twice).
 * Exact integer arithmetic, per round: s[c] = sum of x[t][c] over unflagged
 * samples; b[c] = lower median of s over [c - hw, c + hw] (clamped);
 * R = lower median of b; e[c] = round(s[c] R / b[c]) (0 if b[c] = 0);
 * among unflagged channels, c is flagged when |e - median| > kc 1.4826 MAD
 * (evaluated as 20000 |2e - 2median| > kc 14826 (4 MAD)) and MAD > 0;
 * y[t][c] = min(255, round(x[t][c] R / b[c])); u[t] = sum of y[t][c] over
 * unflagged channels; among unflagged samples, t is flagged when
 * |u - median| > kt 1.4826 MAD (same form).  Flags accumulate.  The output
 * is y of the last round with flagged channels and samples set to the fill
 * level min(255, round(R / T')), T' the unflagged samples of that round.
 * round(a/b) = floor((2a + b) / (2b)).
 * --------------------------------------------------------------------- */
typedef struct ddsp_rfi ddsp_rfi;

/* Workspace for blocks of up to max_nsamp (<= 2^22) spectra of up to
 * max_nchan (<= 8192) channels: about 17 bytes per sample and 273 per
 * channel.  DDSP_E_INVALID_ARG for sizes out of range or a missing device,
 * DDSP_E_NOMEM / DDSP_E_CUDA on allocation failure. */
int ddsp_rfi_create(ddsp_rfi **out, int device, int64_t max_nsamp,
                    int max_nchan);
void ddsp_rfi_destroy(ddsp_rfi *rfi);

/* Clean the time-major block d_in[nsamp][nchan] into d_out (same layout;
 * d_out may be d_in).  half_window 0..32 (10 for 21 channels), kc and kt
 * 0..100 (4 and 3), rounds 1..16 (2).  Stream-ordered.
 * DDSP_E_INVALID_ARG for a NULL pointer or an argument out of range. */
int ddsp_rfi_clean(ddsp_rfi *rfi, const uint8_t *d_in, int64_t nsamp,
                   int nchan, int half_window, int kc, int kt, int rounds,
                   uint8_t *d_out, ddsp_stream_t stream);

/* The flags of the last clean (host_chan_flags[nchan], host_time_flags
 * [nsamp], either may be NULL; 1 = flagged) and the fill level.
 * Synchronises.  DDSP_E_STATE before any clean. */
int ddsp_rfi_flags(ddsp_rfi *rfi, uint8_t *host_chan_flags,
                   uint8_t *host_time_flags, int64_t *fill);

#ifdef __cplusplus
}
#endif

#endif /* DDSP_H */
