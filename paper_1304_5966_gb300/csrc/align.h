// align.h -- host-side reconstruction and staging helpers shared by the
// single-pair (align.cu), batch (batch.cu) and serving (server.cpp) drivers.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "ctx.h"

namespace swgb {

struct Sub {
    int64_t a0, b0;    // offsets into the A and B arrays the driver passes
    int64_t n, m;      // rows (A) and columns (B)
    int src, snk;      // node states (ST_H / ST_E / ST_F)
    int64_t S;         // optimum from source to sink
};

// Reverse-pass row record for a root whose sink is the reverse pass's anchor
// (forward DP cell (e_i, e_j)); rows of reversed row index (k + 1) * step.
struct RootGuide {
    const Guide *g = nullptr;
    int64_t e_i = 0, e_j = 0;
};

int stage_seq(sw_ctx *ctx, Scope &sc, const uint8_t *p, int64_t len, int alph, bool dev_in,
              const uint8_t **out);
int validate_lengths(sw_ctx *ctx, int64_t n, int64_t m, const SchemeDev &sc);
// canonical alignments of many (source H, sink H) rectangles in one recursion
int reconstruct_many(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                     const uint8_t *hA, const uint8_t *hB, const std::vector<Sub> &roots, bool prune,
                     std::vector<std::string> &ops_out, sw_stats *stats, const RootGuide *rg = nullptr);
char *make_cigar(const std::string &ops, const uint8_t *a, const uint8_t *b, int64_t *len_out);
// forward pass on int16x2 lanes (local mode); ovf[p] = 1 when problem p must be re-run
int run_forward16(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                  int rpt, std::vector<int4> &res, std::vector<int> &ovf, sw_stats *stats, float *ms);
cudaError_t reverse_segments_launch(const uint8_t *src, uint8_t *dst, const int64_t *src_off,
                                    const int64_t *dst_off, const int32_t *len, int count, cudaStream_t s);

// reverse complement of count segments (same offsets in src and dst), one block each
cudaError_t revcomp_segments_launch(const uint8_t *src, uint8_t *dst, const int64_t *off, const int32_t *len,
                                    int count, cudaStream_t s);
// DNA complement of one code (A0 C1 G2 T3: c <-> 3 - c); N (4) and other codes stay
inline uint8_t complement_code(uint8_t c) { return c < 4 ? (uint8_t)(3 - c) : c; }

}  // namespace swgb
