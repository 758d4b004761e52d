// batch.cu -- sw_align_batch: many independent pairs per launch.
//
// All pairs' row bands go into one ordered ticket queue of a persistent kernel
// (fwd.cu / fwd16.cu), so thousands of pairs of very different lengths share the
// GPU without a launch per pair; within a pair the bands still form the
// wavefront pipeline.  Each pair is oriented so that its longer sequence indexes
// the rows (fewer column steps on the critical path; the tie rule follows the
// orientation so results are in the user's row-major order).  Pairs whose score
// bound fits int16 run on int16x2 lanes (two cells per instruction); a pair
// whose values reach the int16 guard is re-run on int32 lanes.  Alignment
// requests then run their start-point passes as one batched anchored launch and
// their reconstructions as one recursion over all pairs.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "align.h"
#include "common.cuh"
#include "lab.h"

using namespace swgb;

namespace swgb {

// batch shape for the band-height table: pair count, mean and largest row
// count, each rounded down to a power of two
static uint64_t batch_shape_key(const std::vector<FwdJob> &jobs)
{
    int64_t sum = 0, mx = 0;
    for (const FwdJob &j : jobs) { sum += j.n; mx = std::max<int64_t>(mx, j.n); }
    auto lg = [](int64_t x) { uint64_t b = 0; while (x > 1) { x >>= 1; ++b; } return b; };
    return lg((int64_t)jobs.size()) << 40 | lg(sum / (int64_t)jobs.size()) << 20 | lg(mx);
}

// can this pair run on int16x2 lanes without possible overflow?
static bool fits_int16(const SchemeDev &sc, int64_t n, int64_t m)
{
    if (sc.alphabet > 4) return false;
    if (sc.go + sc.ge + 128 >= 32768) return false;
    const int64_t bound = (int64_t)sc.max_sub * std::min(n, m);
    return bound < 32767 - 2 * sc.max_sub;
}

int batch_forward(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                  const std::vector<int64_t> &aoff, const std::vector<int64_t> &boff,
                  const std::vector<int64_t> &len_a, const std::vector<int64_t> &len_b, int32_t flags,
                  std::vector<int4> &score_end, sw_stats *stats, float *ms_total)
{
    const int count = (int)len_a.size();
    score_end.assign(count, make_int4(0, -1, -1, 0));
    const bool prune = !(flags & SW_FLAG_NO_PRUNE);
    std::vector<FwdJob> j16, j32;
    std::vector<int> id16, id32;
    std::vector<int> trans(count, 0);
    for (int p = 0; p < count; ++p) {
        const int64_t n = len_a[p], m = len_b[p];
        if (n == 0 || m == 0) continue;
        const int t = m > n ? 1 : 0;
        trans[p] = t;
        FwdJob j;
        j.a = t ? dB + boff[p] : dA + aoff[p];
        j.b = t ? dA + aoff[p] : dB + boff[p];
        j.n = (int32_t)(t ? m : n);
        j.m = (int32_t)(t ? n : m);
        j.mode = FWD_LOCAL; j.target = 0; j.transposed = t;
        const bool use16 = !(flags & SW_FLAG_FORCE_INT32) && sc.alphabet <= 4 &&
                           ((flags & SW_FLAG_FORCE_INT16) || fits_int16(sc, n, m));
        if (use16) { j16.push_back(j); id16.push_back(p); }
        else { j32.push_back(j); id32.push_back(p); }
    }
    auto store = [&](int p, const int4 &r) {
        if (!r.w || r.x <= 0) { score_end[p] = make_int4(0, -1, -1, 1); return; }
        // kernel (row, col) -> user (a_end, b_end)
        if (trans[p]) score_end[p] = make_int4(r.x, r.z, r.y, 1);
        else score_end[p] = make_int4(r.x, r.y, r.z, 1);
    };
    float ms = 0, ms2 = 0;
    int st;
    if (!j16.empty()) {
        std::vector<int4> res;
        std::vector<int> ovf;
        // Band height of the int16x2 pass: taken from the context's table for this
        // batch shape, or found by timing each candidate on this batch (every
        // candidate gives the same results; the fastest run's are kept).
        int rpt = 0;
        bool timed = false;
        if (ctx->opt.autotune && j16.size() > 1) {
            const uint64_t key = batch_shape_key(j16);
            auto it = ctx->tuned_rpt16.find(key);
            if (it != ctx->tuned_rpt16.end()) {
                rpt = it->second;
            } else {
                float best = 0;
                sw_stats sbest{};
                for (int cand : {4, 8, 16}) {
                    std::vector<int4> r;
                    std::vector<int> o;
                    sw_stats sc_{};
                    float ms_c = 0;
                    if ((st = run_forward16(ctx, sc, j16, prune, cand, r, o, &sc_, &ms_c))) return st;
                    if (!timed || ms_c < best) {
                        best = ms_c; rpt = cand; res.swap(r); ovf.swap(o); sbest = sc_; timed = true;
                    }
                }
                ctx->tuned_rpt16[key] = rpt;
                ms = best;
                if (stats) {
                    stats->fwd_cells += sbest.fwd_cells; stats->cells_computed += sbest.cells_computed;
                    stats->tiles_total += sbest.tiles_total; stats->tiles_pruned += sbest.tiles_pruned;
                    stats->band_rows = sbest.band_rows; stats->tuned = 1;
                }
            }
        }
        if (!timed && (st = run_forward16(ctx, sc, j16, prune, rpt, res, ovf, stats, &ms))) return st;
        for (size_t k = 0; k < j16.size(); ++k) {
            if (ovf[k]) { j32.push_back(j16[k]); id32.push_back(id16[k]); if (stats) stats->int16_reruns++; }
            else store(id16[k], res[k]);
        }
    }
    if (!j32.empty()) {
        std::vector<int4> res;
        if ((st = run_forward32(ctx, sc, j32, prune, 0, res, stats, &ms2))) return st;
        for (size_t k = 0; k < j32.size(); ++k) store(id32[k], res[k]);
    }
    if (ms_total) *ms_total = ms + ms2;
    return SW_OK;
}

}  // namespace swgb

// One strand: every pair as given.
static int align_batch_strand(sw_ctx *ctx, const sw_pair *pairs, int32_t count, const sw_scheme *scheme,
                              int32_t flags, sw_result *outs)
{
    if (!ctx || !outs || count < 0 || (count > 0 && !pairs)) return SW_EINVAL;
    for (int p = 0; p < count; ++p) {
        std::memset(&outs[p], 0, sizeof(sw_result));
        outs[p].a_begin = outs[p].a_end = outs[p].b_begin = outs[p].b_end = -1;
    }
    if (count == 0) return SW_OK;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_align_batch");
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) { ctx->last_error = "invalid scheme"; return st; }
    const bool dev = (flags & SW_FLAG_DEVICE_INPUT) != 0;
    const bool score_only = (flags & SW_FLAG_SCORE_ONLY) != 0;
    std::vector<int64_t> la(count), lb(count), aoff(count), boff(count);
    int64_t ta = 0, tb = 0;
    for (int p = 0; p < count; ++p) {
        if ((st = validate_lengths(ctx, pairs[p].n, pairs[p].m, sc))) return st;
        if ((pairs[p].n && !pairs[p].a) || (pairs[p].m && !pairs[p].b)) return SW_EINVAL;
        la[p] = pairs[p].n; lb[p] = pairs[p].m;
        aoff[p] = ta; boff[p] = tb;
        ta += la[p]; tb += lb[p];
        outs[p].stats.cells = la[p] * lb[p];
    }
    cudaSetDevice(ctx->device);
    const int64_t l0 = ctx->launches;
    Scope s(ctx->arena);
    uint8_t *dA = s.get<uint8_t>((size_t)ta + 16), *dB = s.get<uint8_t>((size_t)tb + 16);
    if (s.failed()) { ctx->last_error = "workspace too small for the batch sequences"; return SW_ENOMEM; }
    std::vector<uint8_t> hA((size_t)ta), hB((size_t)tb);
    cudaError_t e;
    if (!dev) {
        for (int p = 0; p < count; ++p) {
            if (la[p]) std::memcpy(hA.data() + aoff[p], pairs[p].a, (size_t)la[p]);
            if (lb[p]) std::memcpy(hB.data() + boff[p], pairs[p].b, (size_t)lb[p]);
        }
        if ((e = cudaMemcpyAsync(dA, hA.data(), (size_t)ta, cudaMemcpyHostToDevice, ctx->stream)) ||
            (e = cudaMemcpyAsync(dB, hB.data(), (size_t)tb, cudaMemcpyHostToDevice, ctx->stream)))
            return set_cuda_error(ctx, e, "batch upload");
        // the code check runs on the device copies (one kernel per arena)
        const uint8_t *chk;
        if ((st = stage_seq(ctx, s, dA, ta, sc.alphabet, true, &chk))) return st;
        if ((st = stage_seq(ctx, s, dB, tb, sc.alphabet, true, &chk))) return st;
    } else {
        for (int p = 0; p < count; ++p) {
            if ((la[p] && (e = cudaMemcpyAsync(dA + aoff[p], pairs[p].a, (size_t)la[p], cudaMemcpyDeviceToDevice, ctx->stream))) ||
                (lb[p] && (e = cudaMemcpyAsync(dB + boff[p], pairs[p].b, (size_t)lb[p], cudaMemcpyDeviceToDevice, ctx->stream))))
                return set_cuda_error(ctx, e, "batch gather");
        }
        const uint8_t *chk;
        if ((st = stage_seq(ctx, s, dA, ta, sc.alphabet, true, &chk))) return st;
        if ((st = stage_seq(ctx, s, dB, tb, sc.alphabet, true, &chk))) return st;
        if (!score_only) {
            if ((e = cudaMemcpyAsync(hA.data(), dA, (size_t)ta, cudaMemcpyDeviceToHost, ctx->stream)) ||
                (e = cudaMemcpyAsync(hB.data(), dB, (size_t)tb, cudaMemcpyDeviceToHost, ctx->stream)) ||
                (e = cudaStreamSynchronize(ctx->stream)))
                return set_cuda_error(ctx, e, "batch readback");
        }
    }
    sw_stats agg{};
    std::vector<int4> se;
    float ms = 0;
    if ((st = batch_forward(ctx, sc, dA, dB, aoff, boff, la, lb, flags, se, &agg, &ms))) return st;
    for (int p = 0; p < count; ++p) {
        if (se[p].x > 0) { outs[p].score = se[p].x; outs[p].a_end = se[p].y; outs[p].b_end = se[p].z; }
        outs[p].stats.int16_reruns = 0;
    }
    outs[0].stats.ms_forward = ms;
    outs[0].stats.fwd_cells = agg.fwd_cells;
    outs[0].stats.cells_computed = agg.cells_computed;
    outs[0].stats.tiles_total = agg.tiles_total;
    outs[0].stats.tiles_pruned = agg.tiles_pruned;
    outs[0].stats.int16_reruns = agg.int16_reruns;
    outs[0].stats.band_rows = agg.band_rows;
    outs[0].stats.tuned = agg.tuned;
    if (!score_only) {
        const bool prune = !(flags & SW_FLAG_NO_PRUNE);
        // start points: one anchored launch over all reversed prefixes
        std::vector<int> ids;
        int64_t ra = 0, rbt = 0;
        for (int p = 0; p < count; ++p)
            if (se[p].x > 0) { ids.push_back(p); ra += se[p].y; rbt += se[p].z; }
        if (!ids.empty()) {
            const int k = (int)ids.size();
            Scope s2(ctx->arena);
            uint8_t *rA = s2.get<uint8_t>((size_t)ra + 16), *rB = s2.get<uint8_t>((size_t)rbt + 16);
            int64_t *offs = s2.get<int64_t>(4 * (size_t)k);
            int32_t *lens = s2.get<int32_t>(2 * (size_t)k);
            if (s2.failed()) { ctx->last_error = "workspace too small for the start passes"; return SW_ENOMEM; }
            std::vector<int64_t> ho(4 * (size_t)k);
            std::vector<int32_t> hl(2 * (size_t)k);
            int64_t pa = 0, pb = 0;
            for (int x = 0; x < k; ++x) {
                const int p = ids[x];
                ho[x] = aoff[p]; ho[k + x] = pa; hl[x] = se[p].y;
                ho[2 * k + x] = boff[p]; ho[3 * k + x] = pb; hl[k + x] = se[p].z;
                pa += se[p].y; pb += se[p].z;
            }
            if ((e = cudaMemcpyAsync(offs, ho.data(), sizeof(int64_t) * ho.size(), cudaMemcpyHostToDevice, ctx->stream)) ||
                (e = cudaMemcpyAsync(lens, hl.data(), sizeof(int32_t) * hl.size(), cudaMemcpyHostToDevice, ctx->stream)) ||
                (e = reverse_segments_launch(dA, rA, offs, offs + k, lens, k, ctx->stream)) ||
                (e = reverse_segments_launch(dB, rB, offs + 2 * k, offs + 3 * k, lens + k, k, ctx->stream)))
                return set_cuda_error(ctx, e, "batch reverse");
            ctx->launches += 2;
            std::vector<FwdJob> jobs(k);
            for (int x = 0; x < k; ++x) {
                const int p = ids[x];
                jobs[x] = {rA + ho[k + x], rB + ho[3 * k + x], se[p].y, se[p].z, FWD_ANCHORED, BIAS + se[p].x, 0};
            }
            std::vector<int4> res;
            float ms_s = 0;
            sw_stats tmp{};
            if ((st = run_forward(ctx, sc, jobs, prune, 0, res, &tmp, &ms_s))) return st;
            outs[0].stats.ms_start = ms_s;
            std::vector<Sub> roots(k);
            for (int x = 0; x < k; ++x) {
                const int p = ids[x];
                if (!res[x].w || res[x].x != BIAS + se[p].x) { ctx->last_error = "internal: start point not found"; return SW_ECUDA; }
                outs[p].a_begin = se[p].y - res[x].y;
                outs[p].b_begin = se[p].z - res[x].z;
                roots[x] = Sub{aoff[p] + outs[p].a_begin, boff[p] + outs[p].b_begin,
                               outs[p].a_end - outs[p].a_begin, outs[p].b_end - outs[p].b_begin, ST_H, ST_H,
                               (int64_t)se[p].x};
            }
            std::vector<std::string> ops;
            cudaEventRecord(ctx->ev[5], ctx->stream);
            if ((st = reconstruct_many(ctx, sc, dA, dB, hA.data(), hB.data(), roots, prune, ops, &outs[0].stats)))
                return st;
            cudaEventRecord(ctx->ev[6], ctx->stream);
            cudaEventSynchronize(ctx->ev[6]);
            cudaEventElapsedTime(&outs[0].stats.ms_align, ctx->ev[5], ctx->ev[6]);
            for (int x = 0; x < k; ++x) {
                const int p = ids[x];
                int64_t cl = 0;
                outs[p].cigar = make_cigar(ops[x], hA.data() + roots[x].a0, hB.data() + roots[x].b0, &cl);
                if (!outs[p].cigar) return SW_ENOMEM;
                outs[p].cigar_len = cl;
            }
        }
    }
    outs[0].stats.kernel_launches = ctx->launches - l0;
    return SW_OK;
}

// Both strands (Sec. 3 runs each chromosome pair against B and its reverse
// complement): the batch holds every pair twice, once with B and once with
// revcomp(B), and each pair keeps the strand with the higher score (the
// forward strand on a tie).  The reverse complements are made on the host for
// host inputs and by one kernel over all pairs for device inputs.
static int align_batch_both(sw_ctx *ctx, const sw_pair *pairs, int32_t count, const sw_scheme *scheme,
                            int32_t flags, sw_result *outs)
{
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) { ctx->last_error = "invalid scheme"; return st; }
    if (sc.alphabet > 5) { ctx->last_error = "both strands need DNA codes (alphabet 4 or 5)"; return SW_EINVAL; }
    if (count > INT32_MAX / 2) return SW_EINVAL;
    const bool dev = (flags & SW_FLAG_DEVICE_INPUT) != 0;
    std::vector<int64_t> off(count);
    int64_t tb = 0;
    for (int p = 0; p < count; ++p) {
        if (pairs[p].m < 0 || pairs[p].n < 0 || (pairs[p].m && !pairs[p].b)) return SW_EINVAL;
        if (pairs[p].m > INT32_MAX) return SW_EINVAL;
        off[p] = tb;
        tb += pairs[p].m;
    }
    std::vector<sw_pair> ext(2 * (size_t)count);
    std::vector<uint8_t> hrc;
    Scope s(ctx->arena);
    const uint8_t *rc = nullptr;
    if (!dev) {
        hrc.resize((size_t)tb + 1);
        for (int p = 0; p < count; ++p) {
            const uint8_t *b = pairs[p].b;
            uint8_t *d = hrc.data() + off[p];
            const int64_t m = pairs[p].m;
            for (int64_t i = 0; i < m; ++i) d[i] = complement_code(b[m - 1 - i]);
        }
        rc = hrc.data();
    } else {
        uint8_t *dg = s.get<uint8_t>((size_t)tb + 16), *drc = s.get<uint8_t>((size_t)tb + 16);
        int64_t *doff = s.get<int64_t>((size_t)count);
        int32_t *dlen = s.get<int32_t>((size_t)count);
        if (s.failed()) { ctx->last_error = "workspace too small for the reverse complements"; return SW_ENOMEM; }
        std::vector<int32_t> len(count);
        cudaError_t e;
        cudaSetDevice(ctx->device);
        for (int p = 0; p < count; ++p) {
            len[p] = (int32_t)pairs[p].m;
            if (len[p] && (e = cudaMemcpyAsync(dg + off[p], pairs[p].b, (size_t)len[p], cudaMemcpyDeviceToDevice,
                                               ctx->stream)))
                return set_cuda_error(ctx, e, "both strands gather");
        }
        if ((e = cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, ctx->stream)) ||
            (e = cudaMemcpyAsync(dlen, len.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, ctx->stream)) ||
            (e = revcomp_segments_launch(dg, drc, doff, dlen, count, ctx->stream)))
            return set_cuda_error(ctx, e, "both strands reverse complement");
        ctx->launches += 1;
        rc = drc;
    }
    for (int p = 0; p < count; ++p) {
        ext[p] = pairs[p];
        ext[(size_t)count + p] = sw_pair{pairs[p].a, pairs[p].n, rc + off[p], pairs[p].m};
    }
    std::vector<sw_result> tmp(2 * (size_t)count);
    st = align_batch_strand(ctx, ext.data(), 2 * count, scheme, flags & ~SW_FLAG_BOTH_STRANDS, tmp.data());
    if (st) {
        for (sw_result &r : tmp) sw_result_free(&r);
        return st;
    }
    const sw_stats call_stats = tmp[0].stats;
    for (int p = 0; p < count; ++p) {
        sw_result &f = tmp[p], &r = tmp[(size_t)count + p];
        const bool rev = r.score > f.score;
        sw_result &win = rev ? r : f, &lose = rev ? f : r;
        outs[p] = win;                  // takes over the winner's CIGAR
        win.cigar = nullptr;
        sw_result_free(&lose);
        outs[p].strand = rev ? 1 : 0;
        outs[p].stats = sw_stats{};
        outs[p].stats.cells = 2 * pairs[p].n * pairs[p].m;
    }
    outs[0].stats = call_stats;
    outs[0].stats.cells = 2 * pairs[0].n * pairs[0].m;
    return SW_OK;
}

extern "C" int sw_align_batch(sw_ctx *ctx, const sw_pair *pairs, int32_t count, const sw_scheme *scheme,
                              int32_t flags, sw_result *outs)
{
    if (!(flags & SW_FLAG_BOTH_STRANDS)) return align_batch_strand(ctx, pairs, count, scheme, flags, outs);
    if (!ctx || !outs || count < 0 || (count > 0 && !pairs)) return SW_EINVAL;
    for (int p = 0; p < count; ++p) {
        std::memset(&outs[p], 0, sizeof(sw_result));
        outs[p].a_begin = outs[p].a_end = outs[p].b_begin = outs[p].b_end = -1;
    }
    if (count == 0) return SW_OK;
    return align_batch_both(ctx, pairs, count, scheme, flags, outs);
}

// The autotuner's table as text: a header line with the device model, then one
// "shape-key band-height" line per batch shape (keys as written by
// batch_shape_key, in hexadecimal).
static const char *kTuneHeader = "swgb-tuning 1 ";

extern "C" int sw_ctx_tuning_export(sw_ctx *ctx, char *buf, uint64_t cap, uint64_t *len)
{
    if (!ctx || !len || (cap && !buf)) return SW_EINVAL;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    std::string out = std::string(kTuneHeader) + ctx->gpu_name + "\n";
    char line[64];
    for (const auto &kv : ctx->tuned_rpt16) {
        snprintf(line, sizeof line, "%llx %d\n", (unsigned long long)kv.first, kv.second);
        out += line;
    }
    *len = out.size();
    if (out.size() + 1 > cap) return SW_ENOMEM;
    std::memcpy(buf, out.c_str(), out.size() + 1);
    return SW_OK;
}

extern "C" int sw_ctx_tuning_import(sw_ctx *ctx, const char *text)
{
    if (!ctx || !text) return SW_EINVAL;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    const std::string t(text);
    const std::string head = std::string(kTuneHeader) + ctx->gpu_name + "\n";
    if (t.compare(0, head.size(), head) != 0) {
        ctx->last_error = "tuning table from another format or GPU model";
        return SW_EINVAL;
    }
    std::map<uint64_t, int> add;
    size_t pos = head.size();
    while (pos < t.size()) {
        size_t eol = t.find('\n', pos);
        if (eol == std::string::npos) eol = t.size();
        const std::string ln = t.substr(pos, eol - pos);
        pos = eol + 1;
        if (ln.empty()) continue;
        unsigned long long key = 0;
        int rpt = 0;
        char extra = 0;
        if (sscanf(ln.c_str(), "%llx %d %c", &key, &rpt, &extra) != 2 || !fwd16_rpt_supported(rpt)) {
            ctx->last_error = "malformed tuning line: " + ln;
            return SW_EINVAL;
        }
        add[(uint64_t)key] = rpt;
    }
    for (const auto &kv : add) ctx->tuned_rpt16[kv.first] = kv.second;
    return SW_OK;
}
