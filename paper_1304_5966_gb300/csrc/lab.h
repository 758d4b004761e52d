// lab.h -- structures of the reconstruction kernels (label pass, walk, leaves).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

// node states (same numbering in every kernel): H full cell, E horizontal gap
// (consumes the column sequence), F vertical gap (consumes the row sequence)
constexpr int ST_H = 0, ST_E = 1, ST_F = 2;
// crossing-edge label = (source column << 2) | type
constexpr int LAB_DIAG = 0, LAB_OPEN = 1, LAB_EXT = 2, LAB_INIT = 3;
constexpr int LAB_RPT = 8;            // rows per thread of the label pass
// Rows per thread of a label pass bounded by the reverse record.  Its bands
// form a chain along a narrow band around the path; measured on the 5 Mbp
// pair, each chunk of that chain is dominated by the hand-over between bands
// rather than by the rows, so thinner lanes (2 or 4 rows) only add bands.
constexpr int LAB_RPT_GUIDED = LAB_RPT;

struct LabProblem {
    const uint8_t *a;      // kernel rows, n codes
    const uint8_t *b;      // kernel columns, m codes
    int32_t n, m;
    int32_t nbands;
    int32_t src, snk;      // source / sink states in kernel orientation
    int32_t ck;            // bands per checkpoint (0: none)
    int32_t target;        // biased optimum at the sink (BIAS + S) or 0 when unknown
    int4 *bus;             // m x {H, F, labH, labF}
    int32_t *flags;        // ceil(m/32): 2 * (last band that released the chunk) + useful bit
    int2 *span;            // nbands: {first, last} useful chunk of each band's bottom row
    int4 *ckpt;            // nck x m x {H, F, labH, labF}
    int4 *sink;            // [0] {H, F, E, done}  [1] {labH, labF, labE, done}
    // Row record of the reverse anchored pass from this problem's sink (null:
    // none): row k holds, per 32-column chunk c of the reversed matrix, the
    // largest biased H of reversed columns 0 .. 32c + 31 on reversed row
    // (k + 1) * gin_step, which is this problem's row gin_i0 - (k + 1) * gin_step;
    // this problem's column j is reversed column gin_j0 - j.
    const int32_t *gin;
    int32_t gin_step, gin_rows, gin_nch, gin_i0, gin_j0;
};

struct LabParams {
    const LabProblem *probs;
    const int2 *tickets;
    int32_t ntickets;
    int32_t *ticket_ctr;
    int32_t *err;
    unsigned long long *stats;
    uint32_t prof_lo[8], prof_hi[8];
    int32_t go, ge, max_sub;
    int32_t slack;         // max(go, -min_sub)
    int32_t prune;
    unsigned long long timeout_ns;
};

// rpt: LAB_RPT or LAB_RPT_GUIDED
cudaError_t lab_launch(const LabParams &p, int rpt, bool pref_vert, bool p2, int ctas, cudaStream_t s);
cudaError_t lab_occupancy(int rpt, bool pref_vert, bool p2, int *n);
cudaError_t lab_init_launch(LabProblem *probs, int nprobs, int go, int ge, cudaStream_t s);
cudaError_t lab_walk_launch(const LabProblem *probs, int nprobs, int R, int go, int ge, int4 *out, int stride,
                            int4 *res, cudaStream_t s);

// full-matrix leaves: one CTA each, pointers in shared memory, greedy traceback
struct LeafProblem {
    const uint8_t *a;      // user rows (A), n codes
    const uint8_t *b;      // user columns (B), m codes
    int32_t n, m;
    int32_t src, snk;      // user states
    int64_t out_off;       // offset of this leaf's op buffer (n + m + 2 chars)
};
constexpr int LEAF_MAX_DIM = 1024;
cudaError_t leaf_launch(const LeafProblem *probs, int nprobs, const int8_t *table8, int go, int ge,
                        int max_cells, char *ops, int32_t *ops_len, cudaStream_t s);

}  // namespace swgb
