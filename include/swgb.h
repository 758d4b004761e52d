/*
 * swgb.h -- C ABI of the GB300 (sm_103a) exact affine-gap Smith-Waterman library.
 *
 * Method: Korpar & Sikic, "SW# - GPU enabled exact alignments on genome scale".
 *   Sec. 2, wavefront paragraph    forward local pass -> best score S and end point
 *   Sec. 2, pruning paragraph      cells that cannot reach the running best are skipped
 *   Sec. 2, start-point paragraph  reverse pass from the end point, borders at -inf,
 *                                  no zero floor -> start point
 *   Sec. 2, reconstruction para.   linear-space divide and conquer between start and
 *                                  end point -> the alignment
 *
 * Scoring.  Rows index sequence A (length n), columns sequence B (length m).
 *   H[i][j] = max(0, H[i-1][j-1] + s(a_i, b_j), E[i][j], F[i][j])
 *   E[i][j] = max(E[i][j-1] - ge, H[i][j-1] - go)      (horizontal gap, consumes B)
 *   F[i][j] = max(F[i-1][j] - ge, H[i-1][j] - go)      (vertical gap, consumes A)
 *   so a gap of length k costs go + ge*(k-1)  (the paper's affine model).
 *
 * Results are exact and deterministic (the paper fixes no tie rule; these are the
 * library's):
 *   end point   first cell with H = S in row-major order of (A, B);
 *   start point among cells of the reverse pass reaching S, the first in row-major
 *               order of the reversed sequences (the largest start, shortest alignment);
 *   alignment   greedy traceback from the end point: at a full cell diagonal >
 *               vertical (I) > horizontal (D); inside a gap, open > extend.
 *   Coordinates are 0-based, end exclusive.  S = 0 gives score 0, coordinates -1
 *   and an empty CIGAR.
 *
 * CIGAR ops: '=' identical codes, 'X' different codes, 'I' consumes A only,
 * 'D' consumes B only; runs are written as <length><op>.
 *
 * Memory.  Every call runs on the context's CUDA stream and takes its device
 * scratch (boundary rows, band flags, checkpoint rows) from the context's
 * workspace, a caller-provided device buffer or one the context allocated.
 * Host buffers passed in are read before the call returns; device buffers
 * (SW_FLAG_DEVICE_INPUT) must stay valid until it returns.
 *
 * Errors.  Every entry point returns an sw_status; nothing is thrown across the
 * ABI.  SW_ECUDA leaves the reason in sw_ctx_last_error().  SW_ETIMEOUT means an
 * inter-band wait inside a kernel ran past its limit: the kernel stopped itself
 * and the context remains usable.
 *
 * Threading.  A context may be used by one host thread at a time.
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SW_OK = 0,
    SW_EINVAL = 1,     /* bad argument: lengths, codes >= alphabet, scheme out of range */
    SW_ENOMEM = 2,     /* workspace too small for this call (or host allocation failed) */
    SW_ECUDA = 3,      /* CUDA runtime error; see sw_ctx_last_error() */
    SW_ETIMEOUT = 4,   /* a bounded device-side wait expired */
    SW_EBUSY = 5,      /* serving: request refused by admission (memory budget / slots) */
    SW_ENOTIMPL = 6,
    SW_EPENDING = 7    /* serving: result not ready yet */
} sw_status;

/* call flags */
#define SW_FLAG_DEVICE_INPUT  0x1   /* a, b are device pointers (else host) */
#define SW_FLAG_SCORE_ONLY    0x2   /* batch / serving: score and end point only */
#define SW_FLAG_NO_PRUNE      0x4   /* disable block pruning (results are identical) */
#define SW_FLAG_FORCE_INT32   0x8   /* batch: never use int16x2 lanes */
#define SW_FLAG_FORCE_INT16   0x10  /* batch: int16x2 lanes even when the static bound
                                       does not rule out overflow (overflow is detected
                                       and the pair re-run in int32) */
#define SW_FLAG_BOTH_STRANDS  0x20  /* batch: align every pair against B and against its
                                       reverse complement in the same batch; keep the
                                       strand with the higher score (forward on a tie) */

/* Substitution scores and gap costs.  Codes are 0..alphabet-1 (DNA: A0 C1 G2 T3,
 * N4).  matrix == NULL uses match on identical codes below 4 and mismatch
 * elsewhere (so N mismatches everything).  Limits: 1 <= alphabet <= 8, scores in
 * [-127, 127], gap_open >= gap_extend >= 1, gap_open <= 65535. */
typedef struct {
    int32_t alphabet;
    const int8_t *matrix;       /* host, alphabet*alphabet row-major, or NULL */
    int32_t match, mismatch;
    int32_t gap_open, gap_extend;
} sw_scheme;

typedef struct {
    int64_t cells;             /* n*m of the forward pass */
    int64_t cells_computed;    /* cells actually computed by all passes */
    int64_t tiles_total;       /* forward-pass 32-column band tiles */
    int64_t tiles_pruned;      /* of which skipped by the pruning bound */
    int32_t int16_reruns;      /* batch: pairs re-run in int32 after int16 overflow */
    int32_t levels;            /* reconstruction: divide-and-conquer levels */
    float ms_forward, ms_start, ms_align;   /* device time per phase */
    int64_t fwd_cells;         /* cells computed by the forward-pass kernel alone */
    int64_t kernel_launches;   /* kernels this call launched */
    int64_t start_cells;       /* cells computed by the start-point pass */
    int64_t align_cells;       /* cells computed by the reconstruction label passes */
    int32_t band_rows;         /* rows per band of the forward pass (int16x2 batch: as tuned) */
    int32_t tuned;             /* batch: 1 when this call timed the candidate band heights */
    int32_t cta_warps;         /* warps per CTA of the local forward pass: 4, or 12-20 when one
                                  CTA per SM runs consecutive bands on each scheduler */
} sw_stats;

typedef struct {
    int64_t score;
    int64_t a_begin, a_end, b_begin, b_end;   /* -1 when score == 0 or score-only start */
    char *cigar;                              /* library-owned; free with sw_result_free */
    int64_t cigar_len;
    sw_stats stats;
    int32_t strand;       /* 0: B as given; 1 (SW_FLAG_BOTH_STRANDS only): the reverse
                             complement of B scored higher, and b_begin, b_end and the
                             CIGAR refer to revcomp(B) */
    int32_t reserved;
} sw_result;

typedef struct {
    const uint8_t *a; int64_t n;
    const uint8_t *b; int64_t m;
} sw_pair;

typedef struct sw_ctx sw_ctx;

/* Create a context on `device` using CUDA stream `stream` (cudaStream_t, NULL =
 * legacy default stream).  `workspace` is a device buffer of `workspace_bytes`
 * that the library sub-allocates and never frees (the caller owns it); pass
 * NULL to let the context cudaMalloc `workspace_bytes` itself (freed by
 * sw_ctx_destroy).  Returns SW_EINVAL, SW_ECUDA or SW_OK. */
int sw_ctx_create(int device, void *stream, void *workspace, uint64_t workspace_bytes,
                  sw_ctx **out);
void sw_ctx_destroy(sw_ctx *ctx);
const char *sw_ctx_last_error(const sw_ctx *ctx);
const char *sw_strerror(int status);

/* Tuning / testing knobs (values persist on the context):
 *   SW_OPT_ROWS_PER_THREAD  forward pass rows per thread: 8, 16, 24 or 32 (0 = by size)
 *   SW_OPT_WARPS_PER_SM     resident warps per SM for the persistent kernels
 *   SW_OPT_TIMEOUT_MS       limit of every device-side inter-band wait
 *   SW_OPT_FAULT_BAND       testing: this forward-pass band never publishes its
 *                           progress (-1 = off), so the next band's bounded wait
 *                           expires and the call returns SW_ETIMEOUT
 *   SW_OPT_CKPT_BANDS       reconstruction: bands between checkpoint rows at level 0
 *   SW_OPT_LEAF_CELLS       reconstruction: largest sub-problem solved by full traceback
 *   SW_OPT_FORWARD_LANES    single-pair forward and start passes: 0 = int16x2 lanes
 *                           with per-warp offsets when the scheme allows, else int32;
 *                           16 = always try int16x2; 32 = int32 lanes only.  The
 *                           result is identical either way.
 *   SW_OPT_TRACE            1 = print one line per device pass to stderr (kernel
 *                           time, cells computed, chunks visited and pruned); also
 *                           switched on at context creation by the environment
 *                           variable SWGB_TRACE=1.
 *   SW_OPT_AUTOTUNE         sw_align_batch: 1 (default) = the first call of a batch
 *                           shape (pair count, mean and largest length, rounded to
 *                           powers of two) times each band height of the int16x2
 *                           forward pass on the whole batch and keeps the fastest
 *                           for later calls of that shape; 0 = chosen by size.
 *                           The results are identical either way. */
enum {
    SW_OPT_ROWS_PER_THREAD = 1,
    SW_OPT_WARPS_PER_SM = 2,
    SW_OPT_TIMEOUT_MS = 3,
    SW_OPT_FAULT_BAND = 4,
    SW_OPT_CKPT_BANDS = 5,
    SW_OPT_LEAF_CELLS = 6,
    SW_OPT_FORWARD_LANES = 7,
    SW_OPT_TRACE = 8,
    SW_OPT_AUTOTUNE = 9
};
int sw_ctx_set_option(sw_ctx *ctx, int option, int64_t value);

/* The SW_OPT_AUTOTUNE table (batch shape -> int16x2 band height) as text, so a
 * later process on the same GPU model can skip the timing runs (the paper has no
 * autotuner; this is a deployment aid).  The text is a header line naming the
 * format and the device model, then one "<shape key, hex> <rows per lane>" line
 * per batch shape.
 * sw_ctx_tuning_export: writes the text and its NUL into buf[0..cap) and the
 * text's length into *len; SW_ENOMEM (with *len set) when cap is too small.
 * sw_ctx_tuning_import: merges such a text into the context's table; SW_EINVAL,
 * leaving the table unchanged, when the text is malformed, names a band height
 * the library does not have, or was written on another GPU model.  Either call
 * takes the context's call lock; neither touches the GPU. */
int sw_ctx_tuning_export(sw_ctx *ctx, char *buf, uint64_t cap, uint64_t *len);
int sw_ctx_tuning_import(sw_ctx *ctx, const char *text);

/* Score and end point (Sec. 2, wavefront and pruning paragraphs).  a[0..n),
 * b[0..m) are codes below scheme->alphabet, host memory unless
 * SW_FLAG_DEVICE_INPUT.  Fills score, a_end, b_end; a_begin = b_begin = -1;
 * cigar = NULL.  n, m up to 2^31-1 (and max score * min(n, m) < 2^30). */
int sw_score(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const sw_scheme *scheme, int32_t flags, sw_result *out);

/* Full alignment: score + end point, start point (Sec. 2, start-point paragraph)
 * and the canonical alignment as a CIGAR (Sec. 2, reconstruction paragraph),
 * in device memory linear in n + m plus the checkpoint rows.  The CIGAR is
 * allocated by the library: release it with sw_result_free. */
int sw_align(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const sw_scheme *scheme, int32_t flags, sw_result *out);

/* Many independent pairs in one persistent launch (device work queue over all
 * pairs' row bands).  outs[count] receives one result per pair, in input order.
 * With SW_FLAG_SCORE_ONLY only score and end point are produced; otherwise each
 * pair is also aligned.  Pairs whose score bound fits int16 run on int16x2
 * lanes unless SW_FLAG_FORCE_INT32.
 *
 * SW_FLAG_BOTH_STRANDS (Sec. 3 runs each pair against both strands of B; DNA
 * codes, alphabet 4 or 5): the batch holds every pair twice, with B and with
 * revcomp(B) (A0 C1 G2 T3 complement as c <-> 3 - c, N stays), and outs[p] is
 * the strand with the higher score, the forward one on a tie; outs[p].strand
 * says which.  Each result's stats.cells counts both strands.  count may be
 * at most 2^30 - 1 with this flag. */
int sw_align_batch(sw_ctx *ctx, const sw_pair *pairs, int32_t count,
                   const sw_scheme *scheme, int32_t flags, sw_result *outs);

/* ---- Checkpointable score pass ------------------------------------------------
 * The paper has no checkpoints; these calls let a chromosome-scale score pass
 * stop and resume.  A job runs sw_score's forward pass (same lanes, band height,
 * pruning and results) in segments of row bands.  Between segments its whole
 * state is the boundary row (H and F of the last finished band's bottom row,
 * the paper's O(n + 9m) memory; Sec. 2), the per-band results and the running
 * best: sw_score_job_snapshot copies it to host memory, and
 * sw_score_job_resume rebuilds a job from a snapshot, in this or another process
 * on a GPU of the same model.  Each segment boundary drains and refills the band
 * pipeline, so segments should be long (thousands of bands at 5 Mbp).
 *
 * sw_score_job_create: a, b and flags as for sw_score (SW_FLAG_DEVICE_INPUT,
 *   SW_FLAG_NO_PRUNE); both sequences non-empty.  The job copies the sequences
 *   and holds its device state in ctx's workspace until sw_score_job_destroy
 *   (about 16 B per column of b plus 24 B per band).
 * sw_score_job_run: runs up to `bands` more bands as one launch (bands < 0: all
 *   that are left; 0: none, progress only) and reports the bands done, the total
 *   and the wave: how many bands the GPU runs at once.  A launch ends when its
 *   last band has crossed every column, with the GPU ever less busy meanwhile,
 *   so segments that are whole waves add the least time (a segment shorter
 *   than a wave leaves SMs idle throughout).  If the int16x2 lanes
 *   overflow, the job restarts from band 0 on int32 lanes (bands_done drops to 0;
 *   results are unchanged).
 * sw_score_job_snapshot: writes the state into buf[0..cap) and its size into
 *   *len; SW_ENOMEM (with *len set) when cap is too small.  Call with cap = 0 to
 *   learn the size.  The snapshot is a header naming the inputs (sizes,
 *   FNV-1a 64 fingerprints of both sequences, scheme, pruning, lanes, band
 *   height) followed by raw device bytes.
 * sw_score_job_resume: SW_EINVAL when the snapshot is malformed, of another
 *   library version, or was taken for other sequences, scheme or pruning flag.
 * sw_score_job_result: score, a_end, b_end and statistics once every band has
 *   run; SW_EPENDING before.
 * Every call takes the context's call lock; ctx must outlive the job. */
typedef struct sw_score_job sw_score_job;
int sw_score_job_create(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const sw_scheme *scheme, int32_t flags, sw_score_job **out);
int sw_score_job_run(sw_score_job *job, int64_t bands, int64_t *bands_done, int64_t *bands_total,
                     int64_t *wave_bands);
int sw_score_job_snapshot(sw_score_job *job, void *buf, uint64_t cap, uint64_t *len);
int sw_score_job_resume(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const sw_scheme *scheme, int32_t flags, const void *snapshot, uint64_t len,
                        sw_score_job **out);
int sw_score_job_result(sw_score_job *job, sw_result *out);
void sw_score_job_destroy(sw_score_job *job);

/* The plain GPU path used as the comparison baseline: one thread per cell of
 * each anti-diagonal, int32, no pruning, one launch per anti-diagonal.  Same
 * score and end point as sw_score. */
int sw_score_plain(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                   const sw_scheme *scheme, int32_t flags, sw_result *out);

void sw_result_free(sw_result *r);

/* ---- Serving: continuous batching of requests -------------------------------
 * A server owns `workers` worker threads, each with its own CUDA stream and a
 * slice of `ctx`'s workspace (device_budget bytes in total, 0 = all that is
 * free; the slices stay reserved until sw_server_destroy).  Requests are host
 * sequences, copied at submit.  A free worker takes every queued request that
 * fits its slice (same scheme, first come first served) and runs them as one
 * batch; requests arriving meanwhile go to the next free worker, whose kernels
 * overlap the running ones on the device.  Each result is identical to the
 * same request run alone.  flags: SW_FLAG_SCORE_ONLY (else full alignment),
 * SW_FLAG_NO_PRUNE.  `ctx` must outlive the server and not be used for other
 * calls while the server exists. */
typedef struct sw_server sw_server;
int sw_server_create(sw_ctx *ctx, int32_t workers, uint64_t device_budget, sw_server **out);
/* SW_EBUSY: refused by admission (the request's device footprint exceeds a
 * worker's slice, or the queued footprint would exceed four times the budget). */
int sw_server_submit(sw_server *srv, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                     const sw_scheme *scheme, int32_t flags, uint64_t *ticket);
/* Waits up to timeout_us (-1: forever) for the result.  SW_EPENDING if not done
 * (the ticket stays valid); otherwise the request's status, `out` filled (the
 * caller owns out->cigar: sw_result_free) and the ticket retired. */
int sw_server_poll(sw_server *srv, uint64_t ticket, sw_result *out, int64_t timeout_us);
/* Removes a request that has not started (SW_OK); SW_EBUSY once it is running. */
int sw_server_cancel(sw_server *srv, uint64_t ticket);
/* Finishes the queued work, then releases the workers and their slices. */
void sw_server_destroy(sw_server *srv);

/* Score and end point, like sw_score, for callers that cannot allocate device
 * memory at call time: processes whose device memory is all reserved up front by
 * their framework's caching allocator, or latency-bound pipelines that forbid
 * cudaMalloc/cudaFree (and the synchronisation they imply) on the hot path.  The
 * paper has no counterpart; this is a deployment variant of the forward pass.
 *
 * a[0..n) and b[0..m) are codes in DEVICE memory; `stream` is the cudaStream_t to
 * run on (NULL = legacy default stream) and the call returns after synchronising
 * it; `out` is host memory (score, a_end, b_end and stats; no CIGAR).  No device
 * memory is allocated or freed and no context is needed: the scratch (boundary
 * row, flags, band records, counters) is one library-wide static device array of
 * 10 MiB that every GPU loading the library keeps until the process exits.
 * Limits: n <= 16,777,216 and m <= 1,048,576; larger inputs return SW_ENOMEM
 * (the static scratch cannot hold them; use sw_score).  Codes >= alphabet return
 * SW_EINVAL, an expired inter-band wait SW_ETIMEOUT.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array, which keeps the previous call's
 * contents (each call re-initialises what it needs): calls that overlap on the
 * GPU -- from several host threads or streams at once -- race and give wrong
 * results, so serialise them. */
int sw_score_static(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                    const sw_scheme *scheme, void *stream, sw_result *out);

/* Diagnostics: measured issue rate on `device`, per SM clock, with independent
 * chains at full occupancy.  Kinds 0-5, 7, 8, 10 give lane operations per clock
 * per SM of one instruction: 0 IADD+LOP pair, 1 IMNMX+IADD pair, 2 DPX
 * viaddmax, 3 viaddmax relu, 4 PRMT, 5 viaddmax 16x2, 7 vimax3, 8 vimax3 relu,
 * 10 vimax relu + IADD pair.  Kinds 6, 9, 11 give cells per clock per SM of a
 * whole cell update: 6 the forward pass's form, 9 a vimax3-relu form, 11 the
 * 16x2 form (two cells per lane).  Used for the forward pass's issue-rate
 * roofline; allocates its own buffers. */
int sw_probe_issue_rate(int device, int kind, double *ops_per_clk_per_sm);

#ifdef __cplusplus
}
#endif
#endif /* SWGB_H */
