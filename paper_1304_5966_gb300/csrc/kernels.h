// kernels.h -- host/device structures and launchers of the library's kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

// ----------------------------------------------------------------------------
// Forward band pass (local score + end point; or the biased anchored reverse pass)
// ----------------------------------------------------------------------------
enum FwdMode : int32_t { FWD_LOCAL = 0, FWD_ANCHORED = 1 };

struct FwdProblem {          // one alignment problem, device resident
    const uint8_t *a;        // row sequence (codes), n entries
    const uint8_t *b;        // column sequence, m entries
    int32_t n, m;
    int32_t nbands;          // ceil(n / rows-per-band)
    int32_t mode;            // FwdMode
    int32_t target;          // FWD_ANCHORED: biased value sought (BIAS + S)
    int32_t transposed;      // 1: rows are the user's B (tie rule column-first)
    int2 *bus;               // m entries: {H, F} of the row above the current band (int32 lanes),
                             // one self-validating 64-bit word each (int16x2 lanes)
    int32_t *flags;          // ceil(m/32): 2 * (last band that released chunk c) + useful bit
    int2 *span;              // nbands: {first, last} useful chunk of each band's bottom row
    int32_t *best;           // running best for pruning (FWD_LOCAL)
    int32_t *stop_band;      // FWD_ANCHORED: smallest band that reached the target
    int4 *band_res;          // per band {score, row(1-based), col(1-based), valid}
    int32_t *ovf;            // int16 lanes: set when a value reached the overflow guard
    // Row record (int16x2 offset lanes only): for every band b with
    // (b + 1) % gstride == 0, row (b + 1) / gstride - 1 of gout (gnch + 2
    // entries) receives, per 32-column chunk q, the maximum H of the band's
    // bottom row over columns 0 .. 32q + 31 (absolute; biased in anchored
    // mode), then the first and last chunk written (read with rec_at).  Null:
    // no record.
    int32_t *gout;
    int32_t gstride, gnch;
    // Anchored mode: the forward pass's record of the same pair, used to bound
    // what a path can still gain before its start (null: none).  Record row k
    // is forward DP row (k + 1) * gin_step; this problem's DP row i and column
    // j are forward DP row gin_i0 - i and column gin_j0 - j.
    const int32_t *gin;
    int32_t gin_step, gin_rows, gin_nch;
    int32_t gin_i0, gin_j0;
};

struct FwdParams {
    const FwdProblem *probs;
    const int2 *tickets;     // ticket -> {problem, band}, in issue order
    int32_t ntickets;
    int32_t *ticket_ctr;
    int32_t *err;            // device error word (0 = ok)
    unsigned long long *stats;   // [0] cells computed, [1] tiles, [2] tiles pruned
    uint32_t prof_lo[8];     // per a-code: s(a, c) for c = 0..3 as signed bytes
    uint32_t prof_hi[8];     // per a-code: s(a, c) for c = 4..7
    uint32_t prof_lo_t[8];   // the same for transposed problems: s(c, a)
    uint32_t prof_hi_t[8];
    int32_t go, ge, max_sub;
    int32_t slack;           // max(go, -min_sub): what splitting a path at one cell can under-count
    int32_t prune;
    int32_t fault_band;      // testing: this band never publishes (-1 = off)
    unsigned long long timeout_ns;
};

// rows per thread supported by the forward kernel
bool fwd_rpt_supported(int rpt);
// int16x2 forward kernel (local mode, alphabet <= 4): 64*rpt rows per band
bool fwd16_rpt_supported(int rpt);
// rel: values relative to a per-warp offset (long pairs, local and anchored modes)
// anch: every problem of the launch is anchored (offset lanes only)
// wide: one CTA per SM whose schedulers each run consecutive bands (local mode
// with offset lanes only); fwd16_cta_warps gives its warps per CTA
cudaError_t fwd16_launch(const FwdParams &p, int rpt, bool rel, bool anch, bool wide, int ctas, cudaStream_t s);
cudaError_t fwd16_occupancy(int rpt, bool rel, bool anch, bool wide, int *ctas_per_sm);
int fwd16_cta_warps(int rpt, bool wide);
cudaError_t fwd_launch(const FwdParams &p, int rpt, bool two_word_profile, int ctas,
                       int threads, cudaStream_t s);
cudaError_t fwd_occupancy(int rpt, bool two_word_profile, int threads, int *ctas_per_sm);
// fills bus with {h0, f0} and flags with -1 etc. for a set of problems
// packed: 0 for {H, F} pairs (int32 lanes); the int16x2 kernel's
// self-validating words in the local (1) or anchored (2) layout (BusWord)
cudaError_t fwd_init_launch(FwdProblem *probs_dev, int nprobs, const FwdProblem *probs_host,
                            int h0, int f0, int packed, cudaStream_t s);
// per-problem reduction of band results -> out[p] = {score, row, col, found}
cudaError_t fwd_reduce_launch(const FwdProblem *probs_dev, int nprobs, int4 *out,
                              cudaStream_t s);

// ----------------------------------------------------------------------------
// Plain anti-diagonal baseline (one thread per cell, one launch per diagonal)
// ----------------------------------------------------------------------------
cudaError_t plain_score(const uint8_t *a, int n, const uint8_t *b, int m,
                        const int32_t *subtab_dev, int alph, int go, int ge,
                        int32_t *diag_bufs, unsigned long long *best_key,
                        cudaStream_t s);

// ----------------------------------------------------------------------------
// small utilities
// ----------------------------------------------------------------------------
cudaError_t reverse_copy_launch(const uint8_t *src, uint8_t *dst, int64_t len, cudaStream_t s);
cudaError_t fill_i32_launch(int32_t *p, int32_t v, int64_t count, cudaStream_t s);
cudaError_t check_codes_launch(const uint8_t *p, int64_t len, int alph, int32_t *bad, cudaStream_t s);

}  // namespace swgb
