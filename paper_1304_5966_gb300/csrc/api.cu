// api.cu -- the C ABI (include/swgb.h): context, validation, forward-pass driver,
// sw_score and the plain baseline.  sw_align lives in align.cu, the batch path in
// batch.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "align.h"
#include "ctx.h"

using namespace swgb;

namespace swgb {

int set_cuda_error(sw_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) {
        char buf[256];
        snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
        ctx->last_error = buf;
    }
    cudaGetLastError();   // clear sticky-free errors
    return SW_ECUDA;
}

int build_scheme(const sw_scheme *s, SchemeDev *out)
{
    if (!s) return SW_EINVAL;
    if (s->alphabet < 1 || s->alphabet > 8) return SW_EINVAL;
    if (s->gap_extend < 1 || s->gap_open < s->gap_extend || s->gap_open > 65535) return SW_EINVAL;
    SchemeDev d;
    d.alphabet = s->alphabet;
    d.go = s->gap_open;
    d.ge = s->gap_extend;
    std::memset(d.table, 0, sizeof d.table);
    int mx = -1000, mn = 1000;
    for (int x = 0; x < s->alphabet; ++x)
        for (int y = 0; y < s->alphabet; ++y) {
            int v;
            if (s->matrix) v = s->matrix[x * s->alphabet + y];
            else v = (x == y && x < 4) ? s->match : s->mismatch;
            if (v < -127 || v > 127) return SW_EINVAL;
            d.table[x * 8 + y] = (int8_t)v;
            mx = std::max(mx, v);
            mn = std::min(mn, v);
        }
    if (mx <= 0) return SW_EINVAL;          // a local alignment needs a positive score
    d.max_sub = mx;
    d.min_sub = mn;
    for (int x = 0; x < 8; ++x) {
        uint32_t lo = 0, hi = 0;
        for (int y = 0; y < 4; ++y) lo |= (uint32_t)(uint8_t)d.table[x * 8 + y] << (8 * y);
        for (int y = 0; y < 4; ++y) hi |= (uint32_t)(uint8_t)d.table[x * 8 + 4 + y] << (8 * y);
        d.prof_lo[x] = lo;
        d.prof_hi[x] = hi;
        uint32_t tlo = 0, thi = 0;
        for (int y = 0; y < 4; ++y) tlo |= (uint32_t)(uint8_t)d.table[y * 8 + x] << (8 * y);
        for (int y = 0; y < 4; ++y) thi |= (uint32_t)(uint8_t)d.table[(4 + y) * 8 + x] << (8 * y);
        d.prof_lo_t[x] = tlo;
        d.prof_hi_t[x] = thi;
    }
    *out = d;
    return SW_OK;
}

static int occupancy_ctas(sw_ctx *ctx, int rpt, bool p2)
{
    int per_sm = 0;
    if (fwd_occupancy(rpt, p2, 128, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    if (ctx->opt.warps_per_sm > 0) per_sm = std::max(1, std::min(per_sm, ctx->opt.warps_per_sm / 4));
    return per_sm * ctx->sms;
}

// rows per thread when the context leaves it to the library (option 0): the
// largest band height that still leaves a few bands per resident warp, so the
// band pipeline stays full; smaller problems get thinner bands.
static int auto_rpt(sw_ctx *ctx, const std::vector<FwdJob> &jobs, bool p2)
{
    int64_t rows = 0;
    for (auto &j : jobs) rows += j.n;
    const int cands[4] = {32, 24, 16, 8};
    const double need[4] = {2.5, 2.5, 1.0, 0.0};
    for (int k = 0; k < 4; ++k) {
        int per_sm = 1;
        if (fwd_occupancy(cands[k], p2, 128, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
        const double warps = 4.0 * per_sm * ctx->sms;
        if ((double)rows / (32.0 * cands[k]) >= need[k] * warps) return cands[k];
    }
    return 8;
}

// int16x2 lanes with per-warp offsets: all true values of a band's window
// (64*rpt rows x 96 columns) lie within (64*rpt + 96)(go + max_sub) of each other;
// they must stay between the offset's sentinel floor and the top of int16.
static bool rel16_fits(const SchemeDev &sc, int rpt)
{
    if (sc.alphabet > 4) return false;
    if (sc.go + sc.ge - sc.min_sub > 255 || sc.max_sub > 127) return false;
    if (sc.go - sc.ge > 255) return false;      // the anchored passes' boundary words keep 8 bits of F
    const int64_t spread = (int64_t)(64 * rpt + 96) * (sc.go + sc.max_sub) + 64 * sc.max_sub;
    return spread <= 44000;
}

static int auto_rpt16(sw_ctx *ctx, const std::vector<FwdJob> &jobs, bool rel, const SchemeDev &sc)
{
    const int cands[3] = {16, 8, 4};
    for (int k = 0; k < 3; ++k) {
        if (rel && !rel16_fits(sc, cands[k])) continue;
        int per_sm = 1;
        if (fwd16_occupancy(cands[k], rel, rel && jobs[0].mode == FWD_ANCHORED, false, &per_sm) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        const double warps = 4.0 * per_sm * ctx->sms;
        int64_t bands = 0, rows = 0;
        for (auto &j : jobs) { bands += (j.n + 64 * cands[k] - 1) / (64 * cands[k]); rows += j.n; }
        // enough bands to fill the GPU, and not mostly empty rows in the bands
        if (bands >= 2.0 * warps && (double)rows >= 0.6 * (double)bands * 64 * cands[k]) return cands[k];
    }
    return 4;
}

void fwd_params(sw_ctx *ctx, const SchemeDev &sc, bool prune, const FwdProblem *dprobs, const int2 *dtk,
                int64_t ntk, int32_t *ctrs, unsigned long long *dstats, FwdParams &P)
{
    std::memset(&P, 0, sizeof P);
    P.probs = dprobs;
    P.tickets = dtk;
    P.ntickets = (int32_t)ntk;
    P.ticket_ctr = ctrs;
    P.err = ctrs + 1;
    P.stats = dstats;
    for (int x = 0; x < 8; ++x) {
        P.prof_lo[x] = sc.prof_lo[x]; P.prof_hi[x] = sc.prof_hi[x];
        P.prof_lo_t[x] = sc.prof_lo_t[x]; P.prof_hi_t[x] = sc.prof_hi_t[x];
    }
    P.go = sc.go; P.ge = sc.ge; P.max_sub = sc.max_sub;
    P.slack = std::max(sc.go, -sc.min_sub);
    P.prune = prune ? 1 : 0;
    P.fault_band = ctx->opt.fault_band;
    P.timeout_ns = (unsigned long long)ctx->opt.timeout_ms * 1000000ull;
}

void fwd_launch_shape(sw_ctx *ctx, const SchemeDev &sc, int64_t ntk, int rpt, bool lane16, bool rel, bool anch,
                      int *ctas_out, int *cta_warps_out, bool *wide_out)
{
    const bool p2 = sc.alphabet > 4;
    int ctas, cta_warps = 4;
    // local pass with offset lanes and bands enough to fill every SM twice over:
    // one CTA per SM, each scheduler on consecutive bands
    const bool wide = lane16 && rel && !anch && ctx->opt.warps_per_sm <= 0 &&
                      ntk >= 2 * (int64_t)ctx->sms * fwd16_cta_warps(rpt, true);
    if (lane16) {
        int per_sm = 1;
        cta_warps = fwd16_cta_warps(rpt, wide);
        if (fwd16_occupancy(rpt, rel, rel && anch, wide, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
        if (ctx->opt.warps_per_sm > 0) per_sm = std::max(1, std::min(per_sm, ctx->opt.warps_per_sm / 4));
        ctas = per_sm * ctx->sms;
    } else {
        ctas = occupancy_ctas(ctx, rpt, p2);
    }
    ctas = (int)std::min<int64_t>(ctas, (ntk + cta_warps - 1) / cta_warps);
    *ctas_out = ctas;
    *cta_warps_out = cta_warps;
    *wide_out = wide;
}

cudaError_t fwd_launch_pass(sw_ctx *ctx, const SchemeDev &sc, const FwdParams &P, int rpt, bool lane16, bool rel,
                            bool anch, int *cta_warps_out, int64_t shape_ntk)
{
    int ctas = 0, cta_warps = 4;
    bool wide = false;
    fwd_launch_shape(ctx, sc, shape_ntk > 0 ? shape_ntk : P.ntickets, rpt, lane16, rel, anch, &ctas, &cta_warps,
                     &wide);
    if (cta_warps_out) *cta_warps_out = cta_warps;
    return lane16 ? fwd16_launch(P, rpt, rel, rel && anch, wide, ctas, ctx->stream)
                  : fwd_launch(P, rpt, sc.alphabet > 4, ctas, 128, ctx->stream);
}

void forward_plan(sw_ctx *ctx, const SchemeDev &sc, const FwdJob &job, bool allow16, bool *lane16, int *rpt)
{
    const std::vector<FwdJob> jobs(1, job);
    const int opt = ctx->opt.rows_per_thread;
    const bool rel_ok = allow16 && ctx->opt.forward_lanes != 32 && rel16_fits(sc, 4) &&
                        (ctx->opt.forward_lanes == 16 || opt <= 0);
    if (rel_ok) {
        *lane16 = true;
        *rpt = (ctx->opt.forward_lanes == 16 && fwd16_rpt_supported(opt) && rel16_fits(sc, opt))
                   ? opt : auto_rpt16(ctx, jobs, true, sc);
    } else {
        *lane16 = false;
        *rpt = fwd_rpt_supported(opt) ? opt : auto_rpt(ctx, jobs, sc.alphabet > 4);
    }
}

static int run_forward_impl(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                            int rpt, bool lane16, bool rel, std::vector<int4> &res, std::vector<int> *ovf,
                            sw_stats *stats, float *ms)
{
    const int np = (int)jobs.size();
    Range nv(np && jobs[0].mode == FWD_ANCHORED ? "swgb start-point pass" : "swgb forward pass");
    res.assign(np, make_int4(0, 0, 0, 0));
    if (ovf) ovf->assign(np, 0);
    if (np == 0) return SW_OK;
    if (rpt <= 0) rpt = lane16 ? auto_rpt16(ctx, jobs, rel, sc) : auto_rpt(ctx, jobs, sc.alphabet > 4);
    const int R = (lane16 ? 64 : 32) * rpt;
    Scope sc_(ctx->arena);
    std::vector<FwdProblem> hp(np);
    int64_t ntk = 0;
    for (int p = 0; p < np; ++p) {
        const FwdJob &j = jobs[p];
        FwdProblem &q = hp[p];
        q.a = j.a; q.b = j.b; q.n = j.n; q.m = j.m;
        q.nbands = (j.n + R - 1) / R;
        q.mode = j.mode; q.target = j.target; q.transposed = j.transposed;
        q.bus = sc_.get<int2>((size_t)j.m);
        q.flags = sc_.get<int32_t>((size_t)(j.m + CH - 1) / CH);
        q.band_res = sc_.get<int4>((size_t)q.nbands);
        q.span = sc_.get<int2>((size_t)q.nbands);
        q.gout = nullptr; q.gstride = 1; q.gnch = 0;
        q.gin = nullptr; q.gin_step = 1; q.gin_rows = 0; q.gin_nch = 0; q.gin_i0 = 0; q.gin_j0 = 0;
        if (lane16 && rel && j.gout && j.gout->scope) {
            // every band's row when the budget allows, else every stride-th
            Guide &g = *j.gout;
            g.valid = false;
            const int64_t nch = (j.m + CH - 1) / CH;
            int64_t stride = 1;
            while (stride < q.nbands && (q.nbands / stride) * (nch + 2) * 4 > (int64_t)g.budget) ++stride;
            const int64_t rows = q.nbands / stride;
            if (rows > 0 && rows * (nch + 2) * 4 <= (int64_t)g.budget) {
                g.buf = g.scope->get<int32_t>((size_t)(rows * (nch + 2)));
                if (g.buf) {
                    g.step = (int32_t)(stride * R); g.rows = (int32_t)rows; g.nch = (int32_t)nch;
                    q.gout = g.buf; q.gstride = (int32_t)stride; q.gnch = (int32_t)nch;
                }
            }
        }
        if (lane16 && rel && j.gin && j.gin->valid && j.mode == FWD_ANCHORED) {
            q.gin = j.gin->buf; q.gin_step = j.gin->step; q.gin_rows = j.gin->rows; q.gin_nch = j.gin->nch;
            q.gin_i0 = j.gin_i0; q.gin_j0 = j.gin_j0;
        }
        ntk += q.nbands;
    }
    int32_t *ctrs = sc_.get<int32_t>(4 * (size_t)np + 8);      // best, stop, ovf per problem + globals
    unsigned long long *dstats = sc_.get<unsigned long long>(4);
    FwdProblem *dprobs = sc_.get<FwdProblem>(np);
    int2 *dtk = sc_.get<int2>((size_t)ntk);
    int4 *dres = sc_.get<int4>(np);
    if (sc_.failed()) { ctx->last_error = "workspace too small for the forward pass"; return SW_ENOMEM; }
    for (int p = 0; p < np; ++p) {
        hp[p].best = ctrs + 8 + 3 * p;
        hp[p].stop_band = ctrs + 8 + 3 * p + 1;
        hp[p].ovf = ctrs + 8 + 3 * p + 2;
    }
    // ticket order: by band index first (every problem's band b after its band b-1),
    // larger problems first within a band index
    std::vector<int> order(np);
    for (int p = 0; p < np; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (int64_t)hp[x].n * hp[x].m > (int64_t)hp[y].n * hp[y].m;
    });
    std::vector<int2> tk;
    tk.reserve((size_t)ntk);
    if (np == 1) {
        for (int b = 0; b < hp[0].nbands; ++b) tk.push_back(make_int2(0, b));
    } else {
        // priority = remaining chain (bands left * lag + own width), larger first
        struct T { int64_t key; int p, b; };
        std::vector<T> all;
        all.reserve((size_t)ntk);
        for (int p = 0; p < np; ++p)
            for (int b = 0; b < hp[p].nbands; ++b)
                all.push_back({(int64_t)(hp[p].nbands - b) * 96 + hp[p].m, p, b});
        std::stable_sort(all.begin(), all.end(), [](const T &x, const T &y) {
            return x.key > y.key || (x.key == y.key && (x.p < y.p || (x.p == y.p && x.b < y.b)));
        });
        for (auto &t : all) tk.push_back(make_int2(t.p, t.b));
    }
    cudaStream_t s = ctx->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dprobs, hp.data(), sizeof(FwdProblem) * np, cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemcpyAsync(dtk, tk.data(), sizeof(int2) * tk.size(), cudaMemcpyHostToDevice, s)) ||
        (e = cudaMemsetAsync(ctrs, 0, sizeof(int32_t) * 8, s)) ||
        (e = cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * 4, s)))
        return set_cuda_error(ctx, e, "forward setup");
    // local: bus row 0 = {0, -go}; anchored: -inf everywhere (biased 0)
    const bool anch = jobs[0].mode == FWD_ANCHORED;
    if ((e = fwd_init_launch(dprobs, np, hp.data(), 0, anch ? 0 : -sc.go, lane16 ? (rel && anch ? 2 : 1) : 0, s)))
        return set_cuda_error(ctx, e, "forward init");
    FwdParams P;
    fwd_params(ctx, sc, prune, dprobs, dtk, ntk, ctrs, dstats, P);
    int cta_warps = 4;
    cudaEventRecord(ctx->ev[0], s);
    if ((e = fwd_launch_pass(ctx, sc, P, rpt, lane16, rel, anch, &cta_warps)))
        return set_cuda_error(ctx, e, "forward launch");
    cudaEventRecord(ctx->ev[1], s);
    if ((e = fwd_reduce_launch(dprobs, np, dres, s))) return set_cuda_error(ctx, e, "forward reduce");
    int32_t herr = 0;
    unsigned long long hst[4];
    std::vector<int32_t> hctr;
    if (ovf) {
        hctr.resize(3 * (size_t)np);
        if ((e = cudaMemcpyAsync(hctr.data(), ctrs + 8, sizeof(int32_t) * 3 * np, cudaMemcpyDeviceToHost, s)))
            return set_cuda_error(ctx, e, "forward overflow words");
    }
    if ((e = cudaMemcpyAsync(res.data(), dres, sizeof(int4) * np, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(&herr, ctrs + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(hst, dstats, sizeof hst, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return set_cuda_error(ctx, e, "forward pass");
    ctx->launches += 3;
    if (ms) cudaEventElapsedTime(ms, ctx->ev[0], ctx->ev[1]);
    if (ctx->opt.trace) {
        float kms = 0;
        cudaEventElapsedTime(&kms, ctx->ev[0], ctx->ev[1]);
        fprintf(stderr, "swgb: %s pass: %d problem(s), %s lanes, %d rows/band, %d warps/CTA, %.2f ms, cells %.4g, chunks %llu pruned %llu%s%s\n",
                anch ? "anchored" : "local", np, lane16 ? (rel ? "int16x2 offset" : "int16x2") : "int32", R, cta_warps, kms,
                (double)hst[0], hst[1], hst[2], hp[0].gout ? ", recording rows" : "",
                hp[0].gin ? ", bounded by the forward record" : "");
    }
    if (stats) {
        stats->band_rows = R;
        if (jobs[0].mode == FWD_LOCAL) { stats->fwd_cells += (int64_t)hst[0]; stats->cta_warps = cta_warps; }
        stats->cells_computed += (int64_t)hst[0];
        stats->tiles_total += (int64_t)hst[1];
        stats->tiles_pruned += (int64_t)hst[2];
    }
    if (herr == DEV_ETIMEOUT) { ctx->last_error = "device-side inter-band wait timed out"; return SW_ETIMEOUT; }
    if (herr) { ctx->last_error = "device error word set"; return SW_ECUDA; }
    if (ovf)
        for (int p = 0; p < np; ++p) (*ovf)[p] = hctr[3 * (size_t)p + 2] != 0;
    for (int p = 0; p < np; ++p)
        if (hp[p].gout) jobs[p].gout->valid = !(ovf && (*ovf)[p]);
    return SW_OK;
}

int run_forward32(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                  int rpt, std::vector<int4> &res, sw_stats *stats, float *ms)
{
    return run_forward_impl(ctx, sc, jobs, prune, rpt, false, false, res, nullptr, stats, ms);
}

// Forward pass of long problems: int16x2 lanes with per-warp offsets when the
// scheme's value spread allows (and the context does not force int32 lanes),
// int32 lanes otherwise or for any problem whose offset could not absorb a jump.
int run_forward(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                int rpt, std::vector<int4> &res, sw_stats *stats, float *ms)
{
    const bool rel_ok = ctx->opt.forward_lanes != 32 && rel16_fits(sc, 4) &&
                        (ctx->opt.forward_lanes == 16 || rpt <= 0);
    if (!rel_ok) return run_forward32(ctx, sc, jobs, prune, rpt, res, stats, ms);
    std::vector<int> ovf;
    int rpt16 = (ctx->opt.forward_lanes == 16 && fwd16_rpt_supported(rpt) && rel16_fits(sc, rpt)) ? rpt : 0;
    if (rpt16 == 0 && fwd16_rpt_supported(jobs[0].rpt16) && rel16_fits(sc, jobs[0].rpt16)) rpt16 = jobs[0].rpt16;
    int st = run_forward_impl(ctx, sc, jobs, prune, rpt16, true, true, res, &ovf, stats, ms);
    if (st) return st;
    std::vector<FwdJob> redo;
    std::vector<int> idx;
    for (size_t p = 0; p < jobs.size(); ++p)
        if (ovf[p]) { redo.push_back(jobs[p]); idx.push_back((int)p); }
    if (redo.empty()) return SW_OK;
    if (stats) stats->int16_reruns += (int32_t)redo.size();
    std::vector<int4> r2;
    float ms2 = 0;
    if ((st = run_forward32(ctx, sc, redo, prune, fwd_rpt_supported(rpt) ? rpt : 0, r2, stats, &ms2))) return st;
    for (size_t k = 0; k < idx.size(); ++k) res[idx[k]] = r2[k];
    if (ms) *ms += ms2;
    return SW_OK;
}

int run_forward16(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                  int rpt, std::vector<int4> &res, std::vector<int> &ovf, sw_stats *stats, float *ms)
{
    return run_forward_impl(ctx, sc, jobs, prune, rpt, true, false, res, &ovf, stats, ms);
}

// copy (or borrow) a sequence to the device and check its codes
int stage_seq(sw_ctx *ctx, Scope &sc, const uint8_t *p, int64_t len, int alph, bool dev_in,
              const uint8_t **out)
{
    if (len == 0) { *out = nullptr; return SW_OK; }
    if (!p) return SW_EINVAL;
    if (!dev_in) {
        for (int64_t i = 0; i < len; ++i)
            if (p[i] >= alph) { ctx->last_error = "sequence code >= alphabet"; return SW_EINVAL; }
        uint8_t *d = sc.get<uint8_t>((size_t)len);
        if (!d) { ctx->last_error = "workspace too small for the sequences"; return SW_ENOMEM; }
        cudaError_t e = cudaMemcpyAsync(d, p, (size_t)len, cudaMemcpyHostToDevice, ctx->stream);
        if (e) return set_cuda_error(ctx, e, "sequence copy");
        *out = d;
        return SW_OK;
    }
    int32_t *bad = sc.get<int32_t>(1);
    if (!bad) return SW_ENOMEM;
    int32_t hbad = 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(bad, 0, 4, ctx->stream)) ||
        (e = (++ctx->launches, check_codes_launch(p, len, alph, bad, ctx->stream))) ||
        (e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, ctx->stream)) ||
        (e = cudaStreamSynchronize(ctx->stream)))
        return set_cuda_error(ctx, e, "sequence check");
    if (hbad) { ctx->last_error = "sequence code >= alphabet"; return SW_EINVAL; }
    *out = p;
    return SW_OK;
}

int validate_lengths(sw_ctx *ctx, int64_t n, int64_t m, const SchemeDev &sc)
{
    if (n < 0 || m < 0 || n > 0x7fffffff - 1024 || m > 0x7fffffff - 1024) {
        ctx->last_error = "sequence length out of range";
        return SW_EINVAL;
    }
    const int64_t mn = std::min(n, m);
    const int64_t worst = (int64_t)sc.max_sub * mn + (int64_t)std::max(-sc.min_sub, sc.go) * (n + m) +
                          (int64_t)sc.go;
    if (worst >= (int64_t)1 << 29) {
        ctx->last_error = "score range exceeds the int32 kernels (max score * length too large)";
        return SW_EINVAL;
    }
    return SW_OK;
}

}  // namespace swgb

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char *sw_strerror(int st)
{
    switch (st) {
    case SW_OK: return "ok";
    case SW_EINVAL: return "invalid argument";
    case SW_ENOMEM: return "workspace too small";
    case SW_ECUDA: return "CUDA error";
    case SW_ETIMEOUT: return "device-side wait timed out";
    case SW_EBUSY: return "request refused by admission";
    case SW_ENOTIMPL: return "not implemented";
    case SW_EPENDING: return "result pending";
    default: return "unknown status";
    }
}

int sw_ctx_create(int device, void *stream, void *workspace, uint64_t workspace_bytes, sw_ctx **out)
{
    if (!out) return SW_EINVAL;
    *out = nullptr;
    if (workspace_bytes < (1u << 20)) return SW_EINVAL;
    cudaError_t e = cudaSetDevice(device);
    if (e) return set_cuda_error(nullptr, e, "cudaSetDevice");
    sw_ctx *c = new (std::nothrow) sw_ctx();
    if (!c) return SW_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)stream;
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device))) { delete c; return set_cuda_error(nullptr, e, "props"); }
    c->sms = prop.multiProcessorCount;
    c->gpu_name = prop.name;
    if (workspace) {
        c->ws = (char *)workspace;
    } else {
        if ((e = cudaMalloc((void **)&c->ws, workspace_bytes))) { delete c; return set_cuda_error(nullptr, e, "cudaMalloc"); }
        c->owns_ws = true;
    }
    c->ws_bytes = workspace_bytes;
    c->arena.reset(c->ws, workspace_bytes);
    for (auto &ev : c->ev) cudaEventCreate(&ev);
    if (const char *t = getenv("SWGB_TRACE")) c->opt.trace = (t[0] == '1');
    *out = c;
    return SW_OK;
}

void sw_ctx_destroy(sw_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream); else cudaDeviceSynchronize();
    for (auto &ev : ctx->ev) if (ev) cudaEventDestroy(ev);
    if (ctx->owns_ws && ctx->ws) cudaFree(ctx->ws);
    delete ctx;
}

const char *sw_ctx_last_error(const sw_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int sw_ctx_set_option(sw_ctx *ctx, int option, int64_t value)
{
    if (!ctx) return SW_EINVAL;
    switch (option) {
    case SW_OPT_ROWS_PER_THREAD:
        if (value != 0 && !fwd_rpt_supported((int)value) && !fwd16_rpt_supported((int)value)) return SW_EINVAL;
        ctx->opt.rows_per_thread = (int)value; return SW_OK;
    case SW_OPT_WARPS_PER_SM:
        if (value < 0 || value > 64) return SW_EINVAL;
        ctx->opt.warps_per_sm = (int)value; return SW_OK;
    case SW_OPT_TIMEOUT_MS:
        if (value < 1 || value > 600000) return SW_EINVAL;
        ctx->opt.timeout_ms = value; return SW_OK;
    case SW_OPT_FAULT_BAND:
        if (value < -1 || value > 0x7fffffff) return SW_EINVAL;
        ctx->opt.fault_band = (int)value; return SW_OK;
    case SW_OPT_CKPT_BANDS:
        if (value < 0 || value > 1000000) return SW_EINVAL;
        ctx->opt.ckpt_bands = (int)value; return SW_OK;
    case SW_OPT_FORWARD_LANES:
        if (value != 0 && value != 16 && value != 32) return SW_EINVAL;
        ctx->opt.forward_lanes = (int)value; return SW_OK;
    case SW_OPT_AUTOTUNE:
        if (value != 0 && value != 1) return SW_EINVAL;
        ctx->opt.autotune = (int)value; return SW_OK;
    case SW_OPT_TRACE:
        if (value != 0 && value != 1) return SW_EINVAL;
        ctx->opt.trace = (int)value; return SW_OK;
    case SW_OPT_LEAF_CELLS:
        if (value < 256 || value > (1 << 18)) return SW_EINVAL;
        ctx->opt.leaf_cells = value; return SW_OK;
    default: return SW_EINVAL;
    }
}

static void clear_result(sw_result *out)
{
    std::memset(out, 0, sizeof *out);
    out->a_begin = out->a_end = out->b_begin = out->b_end = -1;
}

int sw_score(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
             const sw_scheme *scheme, int32_t flags, sw_result *out)
{
    if (!ctx || !out) return SW_EINVAL;
    clear_result(out);
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_score");
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) { ctx->last_error = "invalid scheme"; return st; }
    if ((st = validate_lengths(ctx, n, m, sc))) return st;
    out->stats.cells = n * m;
    if (n == 0 || m == 0) return SW_OK;
    cudaSetDevice(ctx->device);
    Scope s(ctx->arena);
    const uint8_t *da = nullptr, *db = nullptr;
    const bool dev = (flags & SW_FLAG_DEVICE_INPUT) != 0;
    if ((st = stage_seq(ctx, s, a, n, sc.alphabet, dev, &da))) return st;
    if ((st = stage_seq(ctx, s, b, m, sc.alphabet, dev, &db))) return st;
    std::vector<FwdJob> jobs(1);
    jobs[0] = {da, db, (int32_t)n, (int32_t)m, FWD_LOCAL, 0, 0};
    std::vector<int4> res;
    float ms = 0;
    const int64_t l0 = ctx->launches;
    st = run_forward(ctx, sc, jobs, !(flags & SW_FLAG_NO_PRUNE), ctx->opt.rows_per_thread, res,
                     &out->stats, &ms);
    out->stats.ms_forward = ms;
    out->stats.kernel_launches = ctx->launches - l0;
    if (st) return st;
    if (res[0].w && res[0].x > 0) {
        out->score = res[0].x;
        out->a_end = res[0].y;
        out->b_end = res[0].z;
    }
    return SW_OK;
}

int sw_score_plain(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                   const sw_scheme *scheme, int32_t flags, sw_result *out)
{
    if (!ctx || !out) return SW_EINVAL;
    clear_result(out);
    std::lock_guard<std::mutex> g(ctx->call_mu);
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) return st;
    if ((st = validate_lengths(ctx, n, m, sc))) return st;
    if (n >= (1 << 20) - 1 || m >= (1 << 20) - 1) { ctx->last_error = "plain path limited to 2^20"; return SW_EINVAL; }
    out->stats.cells = n * m;
    if (n == 0 || m == 0) return SW_OK;
    cudaSetDevice(ctx->device);
    Scope s(ctx->arena);
    const uint8_t *da = nullptr, *db = nullptr;
    const bool dev = (flags & SW_FLAG_DEVICE_INPUT) != 0;
    if ((st = stage_seq(ctx, s, a, n, sc.alphabet, dev, &da))) return st;
    if ((st = stage_seq(ctx, s, b, m, sc.alphabet, dev, &db))) return st;
    int32_t *tab = s.get<int32_t>(64);
    int32_t *bufs = s.get<int32_t>(9 * (size_t)(n + 2));
    unsigned long long *key = s.get<unsigned long long>(1);
    if (s.failed()) return SW_ENOMEM;
    int32_t htab[64];
    for (int x = 0; x < sc.alphabet; ++x)
        for (int y = 0; y < sc.alphabet; ++y) htab[x * sc.alphabet + y] = sc.table[x * 8 + y];
    cudaError_t e;
    cudaStream_t strm = ctx->stream;
    if ((e = cudaMemcpyAsync(tab, htab, sizeof htab, cudaMemcpyHostToDevice, strm)) ||
        (e = cudaMemsetAsync(key, 0, 8, strm)) ||
        (e = cudaMemsetAsync(bufs, 0, sizeof(int32_t) * 9 * (size_t)(n + 2), strm)))
        return set_cuda_error(ctx, e, "plain setup");
    cudaEventRecord(ctx->ev[0], strm);
    if ((e = plain_score(da, (int)n, db, (int)m, tab, sc.alphabet, sc.go, sc.ge, bufs, key, strm)))
        return set_cuda_error(ctx, e, "plain launch");
    out->stats.kernel_launches = n + m - 1;
    ctx->launches += n + m - 1;
    cudaEventRecord(ctx->ev[1], strm);
    unsigned long long hk = 0;
    if ((e = cudaMemcpyAsync(&hk, key, 8, cudaMemcpyDeviceToHost, strm)) || (e = cudaStreamSynchronize(strm)))
        return set_cuda_error(ctx, e, "plain pass");
    float ms = 0;
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]);
    out->stats.ms_forward = ms;
    out->stats.cells_computed = n * m;
    if (hk) {
        out->score = (int64_t)(hk >> 40);
        out->a_end = (1 << 20) - 1 - (int64_t)((hk >> 20) & 0xFFFFF);
        out->b_end = (1 << 20) - 1 - (int64_t)(hk & 0xFFFFF);
    }
    return SW_OK;
}

void sw_result_free(sw_result *r)
{
    if (!r) return;
    free(r->cigar);
    r->cigar = nullptr;
    r->cigar_len = 0;
}

}  // extern "C"
