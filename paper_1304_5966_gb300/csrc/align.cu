// align.cu -- sw_align: start point (reverse anchored pass) and the linear-space
// reconstruction driver (label passes + leaves), CIGAR assembly.
//
// Paper, Sec. 2: after the forward pass gives the score S and the end point,
// "the modified Smith-Waterman algorithm on reverse subsequences which start
// from the found endpoint" gives the start point, and a modified Myers-Miller
// divide and conquer gives the alignment between them, each part solved by the
// wavefront method and small parts by a plain full-matrix alignment.
//
// Reconstruction here (exact under the tie rule; see lab.cu): each pending
// sub-problem, a rectangle with a source node and a sink node on the canonical
// path plus its optimum value, is either a leaf (full-matrix traceback, leaf.cu)
// or is split by one label pass into strips between consecutive checkpoint rows.
// A wide sub-problem is transposed first so that its rows are the longer side.
// All sub-problems of one level run in one launch per kind.  The path segments
// come back in order and are joined into the CIGAR on the host.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "align.h"
#include "lab.h"

using namespace swgb;

namespace swgb {

struct Seg {
    bool pending;
    Sub sub;
    std::string ops;   // resolved ops, user orientation: 'M', 'I' (A only), 'D' (B only)
};

static inline int swap_state(int st) { return st == ST_E ? ST_F : (st == ST_F ? ST_E : st); }

struct Crossing { int c, type, v, r; };

// One level of label passes over `subs` (all split).  For each sub-problem
// returns its crossings (kernel orientation) and sink value, or an error.
static int run_label_level(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                           const std::vector<Sub> &subs, const std::vector<int> &trans, bool prune,
                           std::vector<std::vector<Crossing>> &cross, std::vector<int> &sinkv,
                           sw_stats *stats, const std::vector<const RootGuide *> &guides)
{
    const int np = (int)subs.size();
    Range nv("swgb label pass");
    cross.assign(np, {});
    sinkv.assign(np, 0);
    if (np == 0) return SW_OK;
    // a level bounded by the reverse record runs on thin lanes
    bool guided_level = false;
    for (auto *g : guides) guided_level |= g != nullptr;
    const int rpt = guided_level ? LAB_RPT_GUIDED : LAB_RPT;
    const int R = 32 * rpt;
    Scope s(ctx->arena);
    std::vector<LabProblem> hp(np);
    int64_t ntk = 0;
    size_t fixed = 0, ckbytes_ck1 = 0;
    for (int p = 0; p < np; ++p) {
        const Sub &u = subs[p];
        const int64_t kn = trans[p] ? u.m : u.n, km = trans[p] ? u.n : u.m;
        const int64_t nb = (kn + R - 1) / R;
        fixed += (size_t)km * 16 + (size_t)((km + CH - 1) / CH) * 4 + 1024;
        ckbytes_ck1 += (size_t)std::max<int64_t>(0, nb - 1) * (size_t)km * 16;
    }
    // checkpoint spacing: one value per level, as small as the workspace allows
    const size_t avail = ctx->arena.largest_free();
    const size_t reserve = fixed + (size_t)np * 64 + (32u << 20);
    int ck = ctx->opt.ckpt_bands;
    if (ck <= 0) {
        if (avail <= reserve) { ctx->last_error = "workspace too small for the label pass"; return SW_ENOMEM; }
        const size_t budget = (avail - reserve) * 9 / 10;
        ck = (int)std::max<size_t>(1, (ckbytes_ck1 + budget - 1) / std::max<size_t>(budget, 1));
    }
    int maxnck = 0;
    for (int p = 0; p < np; ++p) {
        const Sub &u = subs[p];
        const int64_t kn = trans[p] ? u.m : u.n, km = trans[p] ? u.n : u.m;
        LabProblem &q = hp[p];
        const int64_t a_off = trans[p] ? u.b0 : u.a0, b_off = trans[p] ? u.a0 : u.b0;
        q.a = (trans[p] ? dB : dA) + a_off;
        q.b = (trans[p] ? dA : dB) + b_off;
        q.n = (int32_t)kn; q.m = (int32_t)km;
        q.nbands = (int32_t)((kn + R - 1) / R);
        q.src = trans[p] ? swap_state(u.src) : u.src;
        q.snk = trans[p] ? swap_state(u.snk) : u.snk;
        q.ck = std::max(1, std::min(ck, q.nbands - 1));
        q.target = (u.S >= 0 && prune) ? (int32_t)(BIAS + u.S) : 0;
        const int nck = (q.nbands - 1) / q.ck;
        if (nck < 1) { ctx->last_error = "workspace too small to split a sub-problem"; return SW_ENOMEM; }
        maxnck = std::max(maxnck, nck);
        q.bus = s.get<int4>((size_t)km);
        q.flags = s.get<int32_t>((size_t)(km + CH - 1) / CH);
        q.span = s.get<int2>((size_t)q.nbands);
        q.ckpt = s.get<int4>((size_t)nck * (size_t)km);
        q.sink = s.get<int4>(2);
        q.gin = nullptr;
        const RootGuide *rg = guides.empty() ? nullptr : guides[p];
        if (rg && rg->g && rg->g->valid && !trans[p] && rg->g->step > 0) {
            // rows recorded by bands that ended before the start point's band
            const int64_t rows = std::min<int64_t>(rg->g->rows, (rg->e_i - u.a0) / rg->g->step);
            if (rows > 0) {
                q.gin = rg->g->buf; q.gin_step = rg->g->step; q.gin_rows = (int32_t)rows;
                q.gin_nch = rg->g->nch;
                q.gin_i0 = (int32_t)(rg->e_i + 1 - u.a0); q.gin_j0 = (int32_t)(rg->e_j + 1 - u.b0);
            }
        }
        ntk += q.nbands;
    }
    LabProblem *dprobs = s.get<LabProblem>(np);
    int2 *dtk = s.get<int2>((size_t)ntk);
    int32_t *ctrs = s.get<int32_t>(8);
    unsigned long long *dstats = s.get<unsigned long long>(4);
    int4 *dcross = s.get<int4>((size_t)np * maxnck);
    int4 *dres = s.get<int4>(np);
    if (s.failed()) { ctx->last_error = "workspace too small for the label pass"; return SW_ENOMEM; }
    std::vector<int2> tk;
    tk.reserve((size_t)ntk);
    {
        struct T { int64_t key; int p, b; };
        std::vector<T> all;
        all.reserve((size_t)ntk);
        for (int p = 0; p < np; ++p)
            for (int b = 0; b < hp[p].nbands; ++b)
                all.push_back({(int64_t)(hp[p].nbands - b) * 96 + hp[p].m, p, b});
        std::stable_sort(all.begin(), all.end(), [](const T &x, const T &y) { return x.key > y.key; });
        for (auto &t : all) tk.push_back(make_int2(t.p, t.b));
    }
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dprobs, hp.data(), sizeof(LabProblem) * np, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dtk, tk.data(), sizeof(int2) * tk.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemsetAsync(ctrs, 0, sizeof(int32_t) * 8, st)) ||
        (e = cudaMemsetAsync(dstats, 0, sizeof(unsigned long long) * 4, st)) ||
        (e = lab_init_launch(dprobs, np, sc.go, sc.ge, st)))
        return set_cuda_error(ctx, e, "label setup");
    LabParams P;
    std::memset(&P, 0, sizeof P);
    P.probs = dprobs; P.tickets = dtk; P.ntickets = (int32_t)ntk; P.ticket_ctr = ctrs; P.err = ctrs + 1;
    P.stats = dstats;
    const bool tr_launch = np > 0 && trans[0];
    for (int x = 0; x < 8; ++x) {
        P.prof_lo[x] = tr_launch ? sc.prof_lo_t[x] : sc.prof_lo[x];
        P.prof_hi[x] = tr_launch ? sc.prof_hi_t[x] : sc.prof_hi[x];
    }
    P.go = sc.go; P.ge = sc.ge; P.max_sub = sc.max_sub; P.prune = prune ? 1 : 0;
    P.slack = std::max(sc.go, -sc.min_sub);
    P.timeout_ns = (unsigned long long)ctx->opt.timeout_ms * 1000000ull;
    const bool p2 = sc.alphabet > 4;
    // problems of both orientations: two launches sharing the ticket counter
    // would break ticket order, so split tickets by orientation
    bool any_t = false, any_n = false;
    for (int p = 0; p < np; ++p) (trans[p] ? any_t : any_n) = true;
    if (any_t && any_n) { ctx->last_error = "internal: mixed orientations in one level"; return SW_ECUDA; }
    int per_sm = 1;
    cudaEvent_t t0 = ctx->ev[8], t1 = ctx->ev[9];
    if (ctx->opt.trace) cudaEventRecord(t0, st);
    lab_occupancy(rpt, !any_t, p2, &per_sm);
    int ctas = std::max(1, per_sm) * ctx->sms;
    ctas = (int)std::min<int64_t>(ctas, (ntk + 3) / 4);
    if ((e = lab_launch(P, rpt, !any_t, p2, ctas, st))) return set_cuda_error(ctx, e, "label launch");
    if ((e = lab_walk_launch(dprobs, np, R, sc.go, sc.ge, dcross, maxnck, dres, st)))
        return set_cuda_error(ctx, e, "label walk");
    ctx->launches += 3;
    std::vector<int4> hc((size_t)np * maxnck), hr(np);
    int32_t herr = 0;
    unsigned long long hst[4];
    if ((e = cudaMemcpyAsync(hc.data(), dcross, sizeof(int4) * hc.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hr.data(), dres, sizeof(int4) * np, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(&herr, ctrs + 1, 4, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hst, dstats, sizeof hst, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return set_cuda_error(ctx, e, "label pass");
    if (stats) { stats->cells_computed += (int64_t)hst[0]; stats->align_cells += (int64_t)hst[0]; }
    if (ctx->opt.trace) {
        cudaEventRecord(t1, st);
        cudaEventSynchronize(t1);
        float kms = 0;
        cudaEventElapsedTime(&kms, t0, t1);
        int64_t rows = 0, guided = 0;
        for (auto &q : hp) { rows += q.n; guided += q.gin != nullptr; }
        fprintf(stderr, "swgb: label pass: %d problem(s)%s, %lld rows, checkpoint every %d bands, %.2f ms, cells %.4g, chunks %llu pruned %llu%s\n",
                np, any_t ? " (transposed)" : "", (long long)rows, ck, kms, (double)hst[0], hst[1], hst[2],
                guided ? ", bounded by the reverse record" : "");
    }
    if (herr == DEV_ETIMEOUT) { ctx->last_error = "label pass: device-side wait timed out"; return SW_ETIMEOUT; }
    if (herr) { ctx->last_error = "label pass: device error"; return SW_ECUDA; }
    for (int p = 0; p < np; ++p) {
        if (!hr[p].y) { ctx->last_error = "internal: label walk failed"; return SW_ECUDA; }
        sinkv[p] = hr[p].x;
        const int nck = hr[p].z;
        cross[p].resize(nck);
        for (int t = 0; t < nck; ++t) {
            const int4 c = hc[(size_t)p * maxnck + t];
            cross[p][t] = {c.x, c.y, c.z, c.w};
        }
    }
    return SW_OK;
}

// Split sub-problem u (solved in kernel orientation tr) at its crossings into
// child segments (user orientation) appended to out.
static int split_sub(const Sub &u, int tr, const std::vector<Crossing> &cr, int sink_v,
                     const uint8_t *hA, const uint8_t *hB, const SchemeDev &sc, std::vector<Seg> &out)
{
    const int64_t kn = tr ? u.m : u.n, km = tr ? u.n : u.m;
    const uint8_t *ka = tr ? hB + u.b0 : hA + u.a0;     // kernel row sequence
    const uint8_t *kb = tr ? hA + u.a0 : hB + u.b0;     // kernel column sequence
    const int ksrc = tr ? swap_state(u.src) : u.src;
    const int ksnk = tr ? swap_state(u.snk) : u.snk;
    const char vert_op = tr ? 'D' : 'I';
    // nodes in kernel coordinates: (row, col, state, value)
    int64_t pr_ = 0, pc = 0;
    int pst = ksrc;
    int64_t pv = BIAS;
    auto emit_child = [&](int64_t r1, int64_t c1, int st1, int64_t v1) -> int {
        Sub c;
        const int64_t nr = r1 - pr_, nc = c1 - pc;
        if (nr < 0 || nc < 0) return SW_ECUDA;
        if (!tr) { c.a0 = u.a0 + pr_; c.b0 = u.b0 + pc; c.n = nr; c.m = nc; c.src = pst; c.snk = st1; }
        else { c.a0 = u.a0 + pc; c.b0 = u.b0 + pr_; c.n = nc; c.m = nr; c.src = swap_state(pst); c.snk = swap_state(st1); }
        c.S = v1 - pv;
        out.push_back({true, c, std::string()});
        return SW_OK;
    };
    for (const Crossing &x : cr) {
        const int st_u = (x.type == LAB_EXT) ? ST_F : ST_H;
        if (emit_child(x.r, x.c, st_u, x.v)) return SW_ECUDA;
        // the crossing edge into row r + 1
        int64_t w;
        Seg e{false, Sub{}, std::string()};
        if (x.type == LAB_DIAG) {
            if (x.r >= kn || x.c >= km) return SW_ECUDA;
            w = tr ? sc.table[kb[x.c] * 8 + ka[x.r]] : sc.table[ka[x.r] * 8 + kb[x.c]];
            e.ops = "M";
            pr_ = x.r + 1; pc = x.c + 1; pst = ST_H;
        } else {
            w = (x.type == LAB_OPEN) ? -sc.go : -sc.ge;
            e.ops = std::string(1, vert_op);
            pr_ = x.r + 1; pc = x.c; pst = ST_F;
        }
        out.push_back(e);
        pv = (int64_t)x.v + w;
    }
    return emit_child(kn, km, ksnk, sink_v);
}

static int run_leaves(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                      const std::vector<Sub> &subs, int max_cells, std::vector<std::string> &ops)
{
    const int np = (int)subs.size();
    Range nv("swgb leaves");
    ops.assign(np, std::string());
    if (np == 0) return SW_OK;
    Scope s(ctx->arena);
    std::vector<LeafProblem> hp(np);
    int64_t off = 0;
    for (int p = 0; p < np; ++p) {
        const Sub &u = subs[p];
        hp[p] = LeafProblem{dA + u.a0, dB + u.b0, (int32_t)u.n, (int32_t)u.m, u.src, u.snk, off};
        off += u.n + u.m + 2;
    }
    LeafProblem *dp = s.get<LeafProblem>(np);
    char *dops = s.get<char>((size_t)off);
    int32_t *dlen = s.get<int32_t>(np);
    int8_t *dtab = s.get<int8_t>(64);
    if (s.failed()) { ctx->last_error = "workspace too small for the leaves"; return SW_ENOMEM; }
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    cudaEvent_t t0 = ctx->ev[8], t1 = ctx->ev[9];
    if (ctx->opt.trace) cudaEventRecord(t0, st);
    if ((e = cudaMemcpyAsync(dp, hp.data(), sizeof(LeafProblem) * np, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dtab, sc.table, 64, cudaMemcpyHostToDevice, st)) ||
        (e = leaf_launch(dp, np, dtab, sc.go, sc.ge, max_cells, dops, dlen, st)))
        return set_cuda_error(ctx, e, "leaf launch");
    ctx->launches += 1;
    std::vector<char> hops((size_t)off);
    std::vector<int32_t> hlen(np);
    if ((e = cudaMemcpyAsync(hops.data(), dops, (size_t)off, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(hlen.data(), dlen, sizeof(int32_t) * np, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return set_cuda_error(ctx, e, "leaf pass");
    if (ctx->opt.trace) {
        cudaEventRecord(t1, st);
        cudaEventSynchronize(t1);
        float kms = 0;
        cudaEventElapsedTime(&kms, t0, t1);
        int64_t cells = 0;
        for (auto &u : subs) cells += (u.n + 1) * (u.m + 1);
        fprintf(stderr, "swgb: leaves: %d problem(s), %.4g cells, %.2f ms\n", np, (double)cells, kms);
    }
    for (int p = 0; p < np; ++p) {
        if (hlen[p] < 0) { ctx->last_error = "internal: leaf traceback failed"; return SW_ECUDA; }
        ops[p].assign(hops.data() + hp[p].out_off, (size_t)hlen[p]);
    }
    return SW_OK;
}

// Reconstruct the canonical alignment of A[a0, a0+n) x B[b0, b0+m) between
// H(0,0) and H(n,m) with optimum S.  dA/dB device, hA/hB host copies.
int reconstruct_many(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                     const uint8_t *hA, const uint8_t *hB, const std::vector<Sub> &roots, bool prune,
                     std::vector<std::string> &ops_out, sw_stats *stats, const RootGuide *rg)
{
    std::vector<Seg> segs;
    std::vector<int> owner;                 // root index of every segment
    for (size_t r = 0; r < roots.size(); ++r) {
        segs.push_back({true, roots[r], std::string()});
        owner.push_back((int)r);
    }
    const int64_t leaf_cells = ctx->opt.leaf_cells;
    int levels = 0;
    for (;;) {
        std::vector<int> leaf_idx, split_idx;
        for (int k = 0; k < (int)segs.size(); ++k) {
            if (!segs[k].pending) continue;
            Sub &u = segs[k].sub;
            if (u.n == 0 || u.m == 0) {
                // a path inside one row or one column: only gap ops, with the
                // zero-cost state changes at its ends
                segs[k].pending = false;
                segs[k].ops = u.n == 0 ? std::string((size_t)u.m, 'D') : std::string((size_t)u.n, 'I');
                continue;
            }
            // a leaf: small enough for the full matrix, or inside one band of the
            // label pass (which could not split it)
            const int64_t R = 32 * LAB_RPT;
            if ((u.n <= LEAF_MAX_DIM && u.m <= LEAF_MAX_DIM && (u.n + 1) * (u.m + 1) <= leaf_cells) ||
                (u.n <= R && u.m <= R))
                leaf_idx.push_back(k);
            else
                split_idx.push_back(k);
        }
        if (leaf_idx.empty() && split_idx.empty()) break;
        ++levels;
        if (!leaf_idx.empty()) {
            std::vector<Sub> ls;
            for (int k : leaf_idx) ls.push_back(segs[k].sub);
            std::vector<std::string> lops;
            const int64_t R = 32 * LAB_RPT;
            const int cap = (int)std::max<int64_t>(leaf_cells, (R + 1) * (R + 1));
            int st = run_leaves(ctx, sc, dA, dB, ls, cap, lops);
            if (st) return st;
            for (size_t x = 0; x < leaf_idx.size(); ++x) {
                segs[leaf_idx[x]].pending = false;
                segs[leaf_idx[x]].ops = std::move(lops[x]);
            }
        }
        if (!split_idx.empty()) {
            // one launch per orientation
            std::vector<Seg> next;
            std::vector<std::vector<Seg>> children(segs.size());
            for (int orient = 0; orient < 2; ++orient) {
                std::vector<Sub> ss;
                std::vector<int> idx, tr;
                std::vector<const RootGuide *> gd;
                for (int k : split_idx) {
                    const Sub &u = segs[k].sub;
                    // the first root keeps the reverse record while it is whole; it
                    // is solved in the record's orientation unless that would leave
                    // too few row bands to fill the GPU
                    const bool guided = levels == 1 && k == 0 && rg && rg->g && rg->g->valid &&
                                        (u.m <= u.n || u.n >= 65536);
                    const int t = (u.m > u.n && !guided) ? 1 : 0;
                    if (t != orient) continue;
                    ss.push_back(u); idx.push_back(k); tr.push_back(t);
                    gd.push_back(guided ? rg : nullptr);
                }
                if (ss.empty()) continue;
                std::vector<std::vector<Crossing>> cross;
                std::vector<int> sinkv;
                int st = run_label_level(ctx, sc, dA, dB, ss, tr, prune, cross, sinkv, stats, gd);
                if (st) return st;
                for (size_t x = 0; x < ss.size(); ++x) {
                    if (ss[x].S >= 0 && (int64_t)sinkv[x] != BIAS + ss[x].S) {
                        ctx->last_error = "internal: label pass optimum differs from the expected value";
                        return SW_ECUDA;
                    }
                    if (split_sub(ss[x], tr[x], cross[x], sinkv[x], hA, hB, sc, children[idx[x]])) {
                        ctx->last_error = "internal: inconsistent crossings";
                        return SW_ECUDA;
                    }
                }
            }
            std::vector<int> next_owner;
            for (int k = 0; k < (int)segs.size(); ++k) {
                if (!children[k].empty()) {
                    for (auto &c : children[k]) { next.push_back(std::move(c)); next_owner.push_back(owner[k]); }
                } else {
                    next.push_back(std::move(segs[k]));
                    next_owner.push_back(owner[k]);
                }
            }
            segs.swap(next);
            owner.swap(next_owner);
        }
        if (levels > 200) { ctx->last_error = "internal: reconstruction does not converge"; return SW_ECUDA; }
    }
    ops_out.assign(roots.size(), std::string());
    for (size_t k = 0; k < segs.size(); ++k) ops_out[owner[k]] += segs[k].ops;
    if (stats) stats->levels = std::max(stats->levels, levels);
    return SW_OK;
}

int reconstruct(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB,
                const uint8_t *hA, const uint8_t *hB, int64_t a0, int64_t n, int64_t b0, int64_t m,
                int64_t S, bool prune, std::string &ops_out, sw_stats *stats, const RootGuide *rg)
{
    std::vector<Sub> roots(1, Sub{a0, b0, n, m, ST_H, ST_H, S});
    std::vector<std::string> ops;
    const int st = reconstruct_many(ctx, sc, dA, dB, hA, hB, roots, prune, ops, stats, rg);
    if (st == SW_OK) ops_out.swap(ops[0]);
    return st;
}

char *make_cigar(const std::string &ops, const uint8_t *a, const uint8_t *b, int64_t *len_out)
{
    std::string out;
    out.reserve(ops.size() / 2 + 16);
    int64_t i = 0, j = 0;
    char cur = 0;
    int64_t run = 0;
    char buf[32];
    auto flush = [&]() {
        if (run) { snprintf(buf, sizeof buf, "%lld%c", (long long)run, cur); out += buf; }
    };
    for (char o : ops) {
        char c;
        if (o == 'M') { c = (a[i] == b[j]) ? '=' : 'X'; ++i; ++j; }
        else if (o == 'I') { c = 'I'; ++i; }
        else { c = 'D'; ++j; }
        if (c != cur) { flush(); cur = c; run = 0; }
        ++run;
    }
    flush();
    char *r = (char *)malloc(out.size() + 1);
    if (!r) return nullptr;
    memcpy(r, out.c_str(), out.size() + 1);
    *len_out = (int64_t)out.size();
    return r;
}

// Start point: reverse anchored pass on A[0, a_end) and B[0, b_end) reversed.
int find_start(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB, int64_t a_end,
               int64_t b_end, int64_t S, bool prune, int64_t *a_begin, int64_t *b_begin, sw_stats *stats,
               float *ms, const Guide *fwd_rec, Guide *rev_rec)
{
    Scope s(ctx->arena);
    uint8_t *rA = s.get<uint8_t>((size_t)a_end), *rB = s.get<uint8_t>((size_t)b_end);
    if (s.failed()) { ctx->last_error = "workspace too small for the reverse pass"; return SW_ENOMEM; }
    cudaError_t e;
    if ((e = reverse_copy_launch(dA, rA, a_end, ctx->stream)) || (e = reverse_copy_launch(dB, rB, b_end, ctx->stream)))
        return set_cuda_error(ctx, e, "reverse copy");
    ctx->launches += 2;
    std::vector<FwdJob> jobs(1);
    jobs[0] = {rA, rB, (int32_t)a_end, (int32_t)b_end, FWD_ANCHORED, (int32_t)(BIAS + S), 0};
    if (prune) {
        jobs[0].gout = rev_rec;
        jobs[0].gin = fwd_rec;
        // Bounded by the forward record, the pass follows a narrow band around
        // the path; its bands form a chain whose length is the band height
        // times the rows per thread, so thin lanes finish first.
        if (fwd_rec && fwd_rec->valid) jobs[0].rpt16 = 4;
        jobs[0].gin_i0 = (int32_t)(a_end + 1);
        jobs[0].gin_j0 = (int32_t)(b_end + 1);
    }
    std::vector<int4> res;
    sw_stats tmp{};
    int st = run_forward(ctx, sc, jobs, prune, ctx->opt.rows_per_thread, res, &tmp, ms);
    if (stats) { stats->cells_computed += tmp.cells_computed; stats->start_cells += tmp.cells_computed; }
    if (st) return st;
    if (!res[0].w || res[0].x != BIAS + S) { ctx->last_error = "internal: start point not found"; return SW_ECUDA; }
    *a_begin = a_end - res[0].y;
    *b_begin = b_end - res[0].z;
    return SW_OK;
}

int align_one(sw_ctx *ctx, const SchemeDev &sc, const uint8_t *dA, const uint8_t *dB, const uint8_t *hA,
              const uint8_t *hB, int64_t n, int64_t m, bool prune, bool have_score, int64_t S_in,
              int64_t ei_in, int64_t ej_in, sw_result *out)
{
    int64_t S = S_in, ei = ei_in, ej = ej_in;
    int st;
    // Row records: the forward pass's bounds the start pass's pruning, the start
    // pass's bounds the first reconstruction level's.  Each may take a sixth
    // of the free workspace; without room a pass runs without its record.
    Scope keep(ctx->arena);
    Guide fwd_rec, rev_rec;
    fwd_rec.scope = &keep; fwd_rec.budget = ctx->arena.largest_free() / 6;
    rev_rec.scope = &keep;
    if (!have_score) {
        std::vector<FwdJob> jobs(1);
        jobs[0] = {dA, dB, (int32_t)n, (int32_t)m, FWD_LOCAL, 0, 0};
        if (prune) jobs[0].gout = &fwd_rec;
        std::vector<int4> res;
        float ms = 0;
        st = run_forward(ctx, sc, jobs, prune, ctx->opt.rows_per_thread, res, &out->stats, &ms);
        out->stats.ms_forward = ms;
        if (st) return st;
        S = (res[0].w && res[0].x > 0) ? res[0].x : 0;
        ei = res[0].y; ej = res[0].z;
    }
    if (S == 0) return SW_OK;
    out->score = S; out->a_end = ei; out->b_end = ej;
    cudaEvent_t e0 = ctx->ev[2], e1 = ctx->ev[3], e2 = ctx->ev[4];
    cudaEventRecord(e0, ctx->stream);
    int64_t ab = -1, bb = -1;
    float ms_start = 0;
    rev_rec.budget = ctx->arena.largest_free() / 6;
    if ((st = find_start(ctx, sc, dA, dB, ei, ej, S, prune, &ab, &bb, &out->stats, &ms_start, &fwd_rec,
                         &rev_rec)))
        return st;
    cudaEventRecord(e1, ctx->stream);
    out->a_begin = ab; out->b_begin = bb;
    std::string ops;
    RootGuide rg;
    rg.g = &rev_rec; rg.e_i = ei; rg.e_j = ej;
    if ((st = reconstruct(ctx, sc, dA, dB, hA, hB, ab, ei - ab, bb, ej - bb, S, prune, ops, &out->stats,
                          prune ? &rg : nullptr)))
        return st;
    cudaEventRecord(e2, ctx->stream);
    cudaEventSynchronize(e2);
    cudaEventElapsedTime(&out->stats.ms_start, e0, e1);
    cudaEventElapsedTime(&out->stats.ms_align, e1, e2);
    int64_t cl = 0;
    out->cigar = make_cigar(ops, hA + ab, hB + bb, &cl);
    if (!out->cigar) return SW_ENOMEM;
    out->cigar_len = cl;
    return SW_OK;
}

}  // namespace swgb

extern "C" int sw_align(sw_ctx *ctx, const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const sw_scheme *scheme, int32_t flags, sw_result *out)
{
    if (!ctx || !out) return SW_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->a_begin = out->a_end = out->b_begin = out->b_end = -1;
    std::lock_guard<std::mutex> g(ctx->call_mu);
    Range nv("swgb sw_align");
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) { ctx->last_error = "invalid scheme"; return st; }
    if ((st = validate_lengths(ctx, n, m, sc))) return st;
    out->stats.cells = n * m;
    if (n == 0 || m == 0) return SW_OK;
    cudaSetDevice(ctx->device);
    Scope s(ctx->arena);
    const bool dev = (flags & SW_FLAG_DEVICE_INPUT) != 0;
    const uint8_t *da = nullptr, *db = nullptr;
    if ((st = stage_seq(ctx, s, a, n, sc.alphabet, dev, &da))) return st;
    if ((st = stage_seq(ctx, s, b, m, sc.alphabet, dev, &db))) return st;
    std::vector<uint8_t> ha, hb;
    const uint8_t *pa = a, *pb = b;
    if (dev) {
        ha.resize((size_t)n); hb.resize((size_t)m);
        cudaError_t e;
        if ((e = cudaMemcpyAsync(ha.data(), a, (size_t)n, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaMemcpyAsync(hb.data(), b, (size_t)m, cudaMemcpyDeviceToHost, ctx->stream)) ||
            (e = cudaStreamSynchronize(ctx->stream)))
            return set_cuda_error(ctx, e, "sequence readback");
        pa = ha.data(); pb = hb.data();
    }
    const int64_t l0 = ctx->launches;
    st = align_one(ctx, sc, da, db, pa, pb, n, m, !(flags & SW_FLAG_NO_PRUNE), false, 0, 0, 0, out);
    out->stats.kernel_launches = ctx->launches - l0;
    return st;
}
