// job.cu -- sw_score_job_*: the score pass in segments of bands, with its state
// copied to and restored from host memory between segments (checkpoint/resume).
//
// The forward pass (Sec. 2, wavefront and pruning paragraphs) carries, from one
// band of rows to the next, only the boundary row (H and F of the band's bottom
// row, the paper's O(n + 9m) state), the per-band results and the running best.
// A job runs the bands [done, done + k) as one persistent launch; when the
// launch returns every band below done + k has written its bottom row, so that
// row, the band results and the best are the whole state.  A snapshot is that
// state plus a header naming the inputs; resuming writes it back and continues
// with band done + k.  Scores, end points and statistics are those of sw_score
// (pruning reads the running best, which the snapshot keeps).  Each segment
// boundary drains and refills the band pipeline, so segments should be long
// (thousands of bands at chromosome scale).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/swgb.h"
#include "align.h"
#include "common.cuh"
#include "ctx.h"

using namespace swgb;

namespace {

constexpr uint64_t kSnapMagic = 0x31424f4a42475753ull;   // "SWGBJOB1"
constexpr uint32_t kSnapVersion = 1;

// Snapshot layout: this header, then the boundary row (bus_bytes), the chunk
// flags (flags_bytes) and the band results (res_bytes), all raw device bytes.
struct SnapHeader {
    uint64_t magic;
    uint32_t version, header_bytes;
    int64_t n, m;
    uint64_t fp_a, fp_b;                  // FNV-1a 64 of the two code sequences
    int32_t alphabet, match, mismatch, gap_open, gap_extend, has_matrix;
    int8_t matrix[64];
    int32_t prune, lane16, rpt, nbands;
    int64_t bands_done;
    uint64_t cells, tiles, pruned;        // statistics of the bands done
    int32_t int16_reruns, best;
    uint64_t bus_bytes, flags_bytes, res_bytes;
};

uint64_t fnv1a(const uint8_t *p, int64_t len)
{
    uint64_t h = 0xcbf29ce484222325ull;
    for (int64_t i = 0; i < len; ++i) { h ^= p[i]; h *= 0x100000001b3ull; }
    return h;
}

}  // namespace

struct sw_score_job {
    sw_ctx *ctx = nullptr;
    SchemeDev sc;
    SnapHeader h{};
    Scope *seqs = nullptr;        // device copies of the sequences
    Scope *state = nullptr;       // boundary row, flags, band results, counters, tickets
    const uint8_t *da = nullptr, *db = nullptr;
    FwdProblem hp{};
    FwdProblem *dprob = nullptr;
    int2 *dtk = nullptr;
    int32_t *ctrs = nullptr;      // [0] ticket, [1] error word, [8] best, [9] stop band, [10] overflow
    unsigned long long *dstats = nullptr;
    int4 *dres = nullptr;
    float ms = 0;
    int64_t launches = 0;

    ~sw_score_job() { delete state; delete seqs; }
};

namespace {

int64_t bus_bytes(const sw_score_job *j) { return j->h.m * (int64_t)sizeof(int2); }
int64_t flags_bytes(const sw_score_job *j) { return (j->h.m + CH - 1) / CH * (int64_t)sizeof(int32_t); }
int64_t res_bytes(const sw_score_job *j) { return (int64_t)j->h.nbands * (int64_t)sizeof(int4); }

// Header fields that name the inputs: sizes, fingerprints, scheme, pruning.
int describe(sw_score_job *j, const sw_scheme *scheme, const uint8_t *ha, int64_t n, const uint8_t *hb, int64_t m,
             int32_t flags)
{
    SnapHeader &h = j->h;
    h.magic = kSnapMagic;
    h.version = kSnapVersion;
    h.header_bytes = (uint32_t)sizeof(SnapHeader);
    h.n = n; h.m = m;
    h.fp_a = fnv1a(ha, n);
    h.fp_b = fnv1a(hb, m);
    h.alphabet = scheme->alphabet; h.match = scheme->match; h.mismatch = scheme->mismatch;
    h.gap_open = scheme->gap_open; h.gap_extend = scheme->gap_extend;
    h.has_matrix = scheme->matrix != nullptr;
    std::memset(h.matrix, 0, sizeof h.matrix);
    if (scheme->matrix) std::memcpy(h.matrix, scheme->matrix, (size_t)scheme->alphabet * scheme->alphabet);
    h.prune = (flags & SW_FLAG_NO_PRUNE) ? 0 : 1;
    return SW_OK;
}

// Device state for the header's lanes and band height; the initial row when
// `fresh`, else left for the caller to fill.
int setup_state(sw_score_job *j, bool fresh)
{
    sw_ctx *ctx = j->ctx;
    delete j->state;
    j->state = new Scope(ctx->arena);
    Scope &s = *j->state;
    SnapHeader &h = j->h;
    const int R = (h.lane16 ? 64 : 32) * h.rpt;
    h.nbands = (int32_t)((h.n + R - 1) / R);
    FwdProblem &q = j->hp;
    std::memset(&q, 0, sizeof q);
    q.a = j->da; q.b = j->db; q.n = (int32_t)h.n; q.m = (int32_t)h.m;
    q.nbands = h.nbands;
    q.mode = FWD_LOCAL;
    q.bus = s.get<int2>((size_t)h.m);
    q.flags = s.get<int32_t>((size_t)((h.m + CH - 1) / CH));
    q.band_res = s.get<int4>((size_t)h.nbands);
    q.span = s.get<int2>((size_t)h.nbands);
    q.gstride = 1; q.gin_step = 1;
    j->ctrs = s.get<int32_t>(16);
    j->dstats = s.get<unsigned long long>(4);
    j->dprob = s.get<FwdProblem>(1);
    j->dtk = s.get<int2>((size_t)h.nbands);
    j->dres = s.get<int4>(1);
    if (s.failed()) { ctx->last_error = "workspace too small for the score job"; return SW_ENOMEM; }
    q.best = j->ctrs + 8;
    q.stop_band = j->ctrs + 9;
    q.ovf = j->ctrs + 10;
    std::vector<int2> tk((size_t)h.nbands);
    for (int b = 0; b < h.nbands; ++b) tk[b] = make_int2(0, b);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(j->dprob, &q, sizeof q, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(j->dtk, tk.data(), sizeof(int2) * tk.size(), cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemsetAsync(j->ctrs, 0, 16 * sizeof(int32_t), ctx->stream)))
        return set_cuda_error(ctx, e, "score job setup");
    if (fresh) {
        if ((e = fwd_init_launch(j->dprob, 1, &q, 0, -j->sc.go, h.lane16 ? 1 : 0, ctx->stream)))
            return set_cuda_error(ctx, e, "score job init");
        ++j->launches;
        h.bands_done = 0;
        h.cells = h.tiles = h.pruned = 0;
        h.best = 0;
    }
    // the host's FwdProblem is copied before `tk` goes out of scope
    if ((e = cudaStreamSynchronize(ctx->stream))) return set_cuda_error(ctx, e, "score job setup");
    return SW_OK;
}

// Sequences: device copies (checked codes) and host copies for the fingerprints.
int stage(sw_score_job *j, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, bool dev,
          std::vector<uint8_t> &ha, std::vector<uint8_t> &hb)
{
    sw_ctx *ctx = j->ctx;
    j->seqs = new Scope(ctx->arena);
    Scope &s = *j->seqs;
    uint8_t *da = s.get<uint8_t>((size_t)n), *db = s.get<uint8_t>((size_t)m);
    if (s.failed()) { ctx->last_error = "workspace too small for the sequences"; return SW_ENOMEM; }
    ha.resize((size_t)n);
    hb.resize((size_t)m);
    cudaError_t e;
    const cudaMemcpyKind in = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if ((e = cudaMemcpyAsync(da, a, (size_t)n, in, ctx->stream)) ||
        (e = cudaMemcpyAsync(db, b, (size_t)m, in, ctx->stream)))
        return set_cuda_error(ctx, e, "score job sequences");
    if (dev) {
        if ((e = cudaMemcpyAsync(ha.data(), da, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(hb.data(), db, (size_t)m, cudaMemcpyDeviceToHost, ctx->stream)))
            return set_cuda_error(ctx, e, "score job sequences");
    } else {
        std::memcpy(ha.data(), a, (size_t)n);
        std::memcpy(hb.data(), b, (size_t)m);
    }
    if ((e = cudaStreamSynchronize(ctx->stream))) return set_cuda_error(ctx, e, "score job sequences");
    for (int64_t i = 0; i < n; ++i)
        if (ha[i] >= j->sc.alphabet) { ctx->last_error = "sequence code >= alphabet"; return SW_EINVAL; }
    for (int64_t i = 0; i < m; ++i)
        if (hb[i] >= j->sc.alphabet) { ctx->last_error = "sequence code >= alphabet"; return SW_EINVAL; }
    j->da = da;
    j->db = db;
    return SW_OK;
}

// Validated job for (a, b, scheme, flags) with sequences staged; lanes not set.
int make_job(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m, const sw_scheme *scheme,
             int32_t flags, sw_score_job **out)
{
    *out = nullptr;
    sw_score_job *j = new (std::nothrow) sw_score_job();
    if (!j) return SW_ENOMEM;
    j->ctx = ctx;
    int st = build_scheme(scheme, &j->sc);
    if (st) { ctx->last_error = "invalid scheme"; delete j; return st; }
    if ((st = validate_lengths(ctx, n, m, j->sc)) || n == 0 || m == 0 || (n && !a) || (m && !b)) {
        if (!st) ctx->last_error = "score jobs need two non-empty sequences";
        delete j;
        return st ? st : SW_EINVAL;
    }
    cudaSetDevice(ctx->device);
    std::vector<uint8_t> ha, hb;
    if ((st = stage(j, a, n, b, m, (flags & SW_FLAG_DEVICE_INPUT) != 0, ha, hb))) { delete j; return st; }
    describe(j, scheme, ha.data(), n, hb.data(), m, flags);
    *out = j;
    return SW_OK;
}

}  // namespace

extern "C" {

int sw_score_job_create(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const sw_scheme *scheme, int32_t flags, sw_score_job **out)
{
    if (!ctx || !out) return SW_EINVAL;
    *out = nullptr;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_score_job_create");
    sw_score_job *j;
    int st = make_job(ctx, a, n, b, m, scheme, flags, &j);
    if (st) return st;
    FwdJob fj{j->da, j->db, (int32_t)n, (int32_t)m, FWD_LOCAL, 0, 0};
    bool lane16 = false;
    int rpt = 0;
    forward_plan(ctx, j->sc, fj, true, &lane16, &rpt);
    j->h.lane16 = lane16 ? 1 : 0;
    j->h.rpt = rpt;
    if ((st = setup_state(j, true))) { delete j; return st; }
    *out = j;
    return SW_OK;
}

int sw_score_job_run(sw_score_job *j, int64_t bands, int64_t *bands_done, int64_t *bands_total,
                     int64_t *wave_bands)
{
    if (!j) return SW_EINVAL;
    sw_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_score_job_run");
    cudaSetDevice(ctx->device);
    SnapHeader &h = j->h;
    const int64_t left = h.nbands - h.bands_done;
    const int64_t seg = bands < 0 ? left : std::min(bands, left);
    if (seg > 0) {
        cudaError_t e;
        if ((e = cudaMemsetAsync(j->ctrs, 0, 2 * sizeof(int32_t), ctx->stream)) ||
            (e = cudaMemsetAsync(j->dstats, 0, 4 * sizeof(unsigned long long), ctx->stream)))
            return set_cuda_error(ctx, e, "score job segment");
        FwdParams P;
        fwd_params(ctx, j->sc, h.prune != 0, j->dprob, j->dtk + h.bands_done, seg, j->ctrs, j->dstats, P);
        cudaEventRecord(ctx->ev[0], ctx->stream);
        // every segment keeps the launch shape of the whole pass
        if ((e = fwd_launch_pass(ctx, j->sc, P, h.rpt, h.lane16 != 0, h.lane16 != 0, false, nullptr, h.nbands)))
            return set_cuda_error(ctx, e, "score job launch");
        cudaEventRecord(ctx->ev[1], ctx->stream);
        ++j->launches;
        int32_t hc[16];
        unsigned long long hs[4];
        if ((e = cudaMemcpyAsync(hc, j->ctrs, sizeof hc, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(hs, j->dstats, sizeof hs, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaStreamSynchronize(ctx->stream)))
            return set_cuda_error(ctx, e, "score job segment");
        float ms = 0;
        cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
        j->ms += ms;
        if (hc[1] == DEV_ETIMEOUT) { ctx->last_error = "device-side inter-band wait timed out"; return SW_ETIMEOUT; }
        if (hc[1]) { ctx->last_error = "device error word set"; return SW_ECUDA; }
        if (h.lane16 && hc[10]) {
            // a value left the int16 window: start over on int32 lanes (same results)
            FwdJob fj{j->da, j->db, (int32_t)h.n, (int32_t)h.m, FWD_LOCAL, 0, 0};
            bool lane16 = false;
            int rpt = 0;
            forward_plan(ctx, j->sc, fj, false, &lane16, &rpt);
            h.lane16 = 0;
            h.rpt = rpt;
            h.int16_reruns += 1;
            int st = setup_state(j, true);
            if (st) return st;
        } else {
            h.bands_done += seg;
            h.cells += hs[0]; h.tiles += hs[1]; h.pruned += hs[2];
            h.best = hc[8];
        }
    }
    if (bands_done) *bands_done = h.bands_done;
    if (bands_total) *bands_total = h.nbands;
    if (wave_bands) {
        // bands resident at once in the pass's launch shape
        int ctas = 0, cta_warps = 4;
        bool wide = false;
        fwd_launch_shape(ctx, j->sc, h.nbands, h.rpt, h.lane16 != 0, h.lane16 != 0, false, &ctas, &cta_warps, &wide);
        *wave_bands = (int64_t)ctas * cta_warps;
    }
    return SW_OK;
}

int sw_score_job_snapshot(sw_score_job *j, void *buf, uint64_t cap, uint64_t *len)
{
    if (!j || !len || (cap && !buf)) return SW_EINVAL;
    sw_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    SnapHeader h = j->h;
    h.bus_bytes = (uint64_t)bus_bytes(j);
    h.flags_bytes = (uint64_t)flags_bytes(j);
    h.res_bytes = (uint64_t)res_bytes(j);
    const uint64_t total = sizeof h + h.bus_bytes + h.flags_bytes + h.res_bytes;
    *len = total;
    if (cap < total) return SW_ENOMEM;
    cudaSetDevice(ctx->device);
    char *p = (char *)buf;
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p, j->hp.bus, h.bus_bytes, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaMemcpyAsync(p + h.bus_bytes, j->hp.flags, h.flags_bytes, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaMemcpyAsync(p + h.bus_bytes + h.flags_bytes, j->hp.band_res, h.res_bytes, cudaMemcpyDeviceToHost,
                             ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return set_cuda_error(ctx, e, "score job snapshot");
    return SW_OK;
}

int sw_score_job_resume(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const sw_scheme *scheme, int32_t flags, const void *snap, uint64_t len,
                        sw_score_job **out)
{
    if (!ctx || !out || !snap) return SW_EINVAL;
    *out = nullptr;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_score_job_resume");
    SnapHeader s;
    if (len < sizeof s) { ctx->last_error = "snapshot too short"; return SW_EINVAL; }
    std::memcpy(&s, snap, sizeof s);
    if (s.magic != kSnapMagic || s.version != kSnapVersion || s.header_bytes != sizeof s) {
        ctx->last_error = "not a score-job snapshot of this library version";
        return SW_EINVAL;
    }
    sw_score_job *j;
    int st = make_job(ctx, a, n, b, m, scheme, flags, &j);
    if (st) return st;
    const SnapHeader &h = j->h;
    const bool same = s.n == h.n && s.m == h.m && s.fp_a == h.fp_a && s.fp_b == h.fp_b &&
                      s.alphabet == h.alphabet && s.match == h.match && s.mismatch == h.mismatch &&
                      s.gap_open == h.gap_open && s.gap_extend == h.gap_extend && s.has_matrix == h.has_matrix &&
                      std::memcmp(s.matrix, h.matrix, sizeof s.matrix) == 0 && s.prune == h.prune;
    const bool lanes_ok = s.lane16 ? fwd16_rpt_supported(s.rpt) : fwd_rpt_supported(s.rpt);
    if (!same || !lanes_ok) {
        ctx->last_error = same ? "snapshot names an unsupported band height"
                               : "snapshot was taken for other sequences, scheme or flags";
        delete j;
        return SW_EINVAL;
    }
    j->h.lane16 = s.lane16;
    j->h.rpt = s.rpt;
    if ((st = setup_state(j, false))) { delete j; return st; }
    const uint64_t want = sizeof s + (uint64_t)bus_bytes(j) + (uint64_t)flags_bytes(j) + (uint64_t)res_bytes(j);
    if (s.nbands != j->h.nbands || s.bus_bytes != (uint64_t)bus_bytes(j) ||
        s.flags_bytes != (uint64_t)flags_bytes(j) || s.res_bytes != (uint64_t)res_bytes(j) || len != want ||
        s.bands_done < 0 || s.bands_done > s.nbands) {
        ctx->last_error = "snapshot sizes do not match its header";
        delete j;
        return SW_EINVAL;
    }
    const char *p = (const char *)snap + sizeof s;
    int32_t counters[3] = {s.best, 0x7fffffff, 0};          // best, stop band, overflow
    cudaError_t e;
    if ((e = cudaMemcpyAsync(j->hp.bus, p, s.bus_bytes, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(j->hp.flags, p + s.bus_bytes, s.flags_bytes, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaMemcpyAsync(j->hp.band_res, p + s.bus_bytes + s.flags_bytes, s.res_bytes, cudaMemcpyHostToDevice,
                             ctx->stream)) ||
        (e = cudaMemcpyAsync(j->ctrs + 8, counters, sizeof counters, cudaMemcpyHostToDevice, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream))) {
        delete j;
        return set_cuda_error(ctx, e, "score job resume");
    }
    j->h.bands_done = s.bands_done;
    j->h.cells = s.cells; j->h.tiles = s.tiles; j->h.pruned = s.pruned;
    j->h.int16_reruns = s.int16_reruns;
    j->h.best = s.best;
    *out = j;
    return SW_OK;
}

int sw_score_job_result(sw_score_job *j, sw_result *out)
{
    if (!j || !out) return SW_EINVAL;
    sw_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    std::memset(out, 0, sizeof *out);
    out->a_begin = out->a_end = out->b_begin = out->b_end = -1;
    const SnapHeader &h = j->h;
    if (h.bands_done < h.nbands) { ctx->last_error = "score job has bands left to run"; return SW_EPENDING; }
    cudaSetDevice(ctx->device);
    int4 r;
    cudaError_t e;
    if ((e = fwd_reduce_launch(j->dprob, 1, j->dres, ctx->stream)) ||
        (e = cudaMemcpyAsync(&r, j->dres, sizeof r, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return set_cuda_error(ctx, e, "score job result");
    ++j->launches;
    out->stats.cells = h.n * h.m;
    out->stats.cells_computed = out->stats.fwd_cells = (int64_t)h.cells;
    out->stats.tiles_total = (int64_t)h.tiles;
    out->stats.tiles_pruned = (int64_t)h.pruned;
    out->stats.int16_reruns = h.int16_reruns;
    out->stats.ms_forward = j->ms;
    out->stats.kernel_launches = j->launches;
    out->stats.band_rows = (h.lane16 ? 64 : 32) * h.rpt;
    if (r.w && r.x > 0) { out->score = r.x; out->a_end = r.y; out->b_end = r.z; }
    return SW_OK;
}

void sw_score_job_destroy(sw_score_job *j)
{
    if (!j) return;
    sw_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete j;
}

}  // extern "C"
