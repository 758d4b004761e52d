// lab.cu -- the reconstruction pass: global affine alignment between two path
// nodes with crossing labels (sm_103a).
//
// The paper reconstructs the alignment between start and end point with a
// modified Myers-Miller divide and conquer whose parts are solved by the same
// wavefront method (Sec. 2, reconstruction paragraph).  A Myers-Miller midpoint
// has no tie rule, so this pass splits the problem differently: every node
// (cell x state) takes, during the forward sweep, the predecessor the greedy
// traceback would take (diagonal > vertical > horizontal; open > extend) and
// inherits that predecessor's label.  Rows at the bottom of every ck-th band are
// checkpoints: the next band starts fresh labels that name the edge crossing
// from the checkpoint row, and the checkpoint row's values and labels are saved.
// The sink's label names the last crossing; the saved label of that crossing's
// source names the one before, and so on (walk kernel below).  The path segment
// between two consecutive crossings is itself the greedy traceback of that
// strip (both end nodes lie on the path), so strips recurse independently.
//
// Values are biased by BIAS (biased 0 = minus infinity), no zero floor.  The
// band pipeline, ticket queue, bounded waits and pruning follow fwd.cu; the
// pruning bound here also charges ge per unavoidable gap column, since the sink
// is fixed, and compares with the known optimum at the sink.
#include "common.cuh"
#include "lab.h"

namespace swgb {

__device__ __forceinline__ int border_cost(int k, bool cont, int go, int ge)
{
    // cost of k >= 1 gap columns leaving the source: a continued gap pays ge each
    return cont ? ge * k : go + ge * (k - 1);
}

// Upper bound of the best path value from the source (0,0) through cell (i, j)
// to the sink (n, m): at most a per diagonal step and at least g per gap column
// on each side.  Concave and piecewise linear in j (breakpoints j = i and
// j = i + m - n), so the cells of row i that can still reach the optimum S form
// one interval, and its ends never decrease from one row to the next.
__device__ __forceinline__ long long env_bound(long long i, long long j, long long n, long long m,
                                               long long a, long long g)
{
    const long long dr = n - i, dc = m - j;
    return a * min(i, j) - g * (i > j ? i - j : j - i) + a * min(dr, dc) - g * (dr > dc ? dr - dc : dc - dr);
}

// First (hi = false) or last (hi = true) DP column of row i whose bound reaches
// S, or -1 when none does.  The bound peaks at one of j = 0, m, i, i + m - n.
__device__ __forceinline__ long long env_end(long long i, long long n, long long m, long long a, long long g,
                                             long long S, bool hi)
{
    const long long cand[4] = {0, m, i, i + m - n};
    long long pj = 0, pv = LLONG_MIN;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long j = max(0LL, min(m, cand[k]));
        const long long v = env_bound(i, j, n, m, a, g);
        if (v > pv) { pv = v; pj = j; }
    }
    if (pv < S) return -1;
    long long lo = hi ? pj : 0, up = hi ? m : pj;
    while (lo < up) {
        const long long md = hi ? (lo + up + 1) >> 1 : (lo + up) >> 1;
        const bool in = env_bound(i, md, n, m, a, g) >= S;
        if (hi) { if (in) lo = md; else up = md - 1; }
        else { if (in) up = md; else lo = md + 1; }
    }
    return lo;
}

// Chunks [first, last] that band b (DP rows bR+1 .. min(n, bR+R)) visits: from
// the first live column of its first row to the last live column of its last
// row, one chunk of margin on each side.  Every band's range is computed the
// same way by the band and by its successor, and both ends are non-decreasing
// in b, so a chunk a band skips is never overwritten by an earlier band later.
__device__ __forceinline__ int2 env_band(int b, int R, int n, int m, long long a, long long g, long long S)
{
    const int nch = (m + CH - 1) / CH;
    const long long lo = env_end((long long)b * R + 1, n, m, a, g, S, false);
    const long long hi = env_end(min((long long)n, (long long)b * R + R), n, m, a, g, S, true);
    if (lo < 0 || hi < 0) return make_int2(0, nch - 1);
    // DP column j >= 1 is kernel column j - 1
    const int qlo = (int)((max(lo, 1LL) - 1) / CH) - 1, qhi = (int)((max(hi, 1LL) - 1) / CH) + 1;
    return make_int2(max(0, qlo), min(nch - 1, qhi));
}

// Reverse-pass record row that bounds band `band`: a path through a cell of
// the band reaches the sink through a recorded row r at or below the band, so
// beyond the band's frontier (its rows and the row above) it gains at most
// max_sub per row down to r plus the largest reverse value of row r right of
// the cell's column, plus the slack of the split cell.  gain holds the row
// part (minus BIAS, the reverse values being biased).
struct LabGuide {
    const int32_t *row = nullptr;
    long long gain = 0;
    int lo = 1, hi = 0, nch = 0, j0 = 0;     // written chunk range, chunks, column map
    // record entry for block q: the largest reverse value right of the block's
    // smallest column (0, minus infinity biased, below the written range)
    __device__ __forceinline__ int entry(int q) const {
        if (!row) return 0;
        const int jr = j0 - max(0, q * CH - 31);          // as a reversed column
        const int c = max(0, min(nch - 1, (jr - 1) / CH));
        if (hi < lo || c < lo) return 0;
        return row[min(c, hi)];
    }
};

__device__ __forceinline__ LabGuide lab_guide(const LabProblem &pr, const LabParams &P, int band, int R)
{
    LabGuide g;
    if (!(P.prune && pr.target > 0 && pr.gin) || band >= pr.nbands) return g;
    const long long T = min((long long)pr.n, (long long)(band + 1) * R);
    if ((long long)pr.gin_i0 - T < 0) return g;
    long long k = ((long long)pr.gin_i0 - T) / pr.gin_step - 1;
    if (k > pr.gin_rows - 1) k = pr.gin_rows - 1;
    if (k < 0) return g;
    const long long r = (long long)pr.gin_i0 - (k + 1) * (long long)pr.gin_step;
    g.row = pr.gin + (size_t)k * (size_t)(pr.gin_nch + 2);
    g.gain = (long long)P.max_sub * (r - (long long)band * R) + P.slack - BIAS;
    g.nch = pr.gin_nch;
    g.j0 = pr.gin_j0;
    g.lo = g.row[pr.gin_nch];
    g.hi = g.row[pr.gin_nch + 1];
    return g;
}

// What a path can still gain, up to the sink, after a frontier node of block q
// of `band` (every cell the block or a later block of the band computes): the
// smaller of max_sub per remaining diagonal step less the unavoidable gap
// columns, and the reverse-record bound (entry = g.entry(q), loaded ahead).
// Non-increasing in q.
__device__ __forceinline__ long long lab_gain(const LabProblem &pr, const LabParams &P, const LabGuide &g,
                                              int band, int q, int R, int entry)
{
    const long long dr_hi = (long long)pr.n - (long long)band * R, dr_lo = max(0LL, dr_hi - R);
    const long long jlo = max(0, q * CH - CH), jhi = min(pr.m, q * CH + CH);
    const long long dc_hi = pr.m - jlo, dc_lo = pr.m - jhi;
    long long gapmin = 0;
    if (dr_lo > dc_hi) gapmin = dr_lo - dc_hi;
    if (dc_lo > dr_hi) gapmin = dc_lo - dr_hi;
    long long gain = (long long)P.max_sub * min(dr_hi, dc_hi) - (long long)P.ge * gapmin;
    if (g.row) gain = min(gain, g.gain + entry);
    return gain;
}

template <int RPT, bool PREF_VERT, bool PROF2>
__global__ void __launch_bounds__(128) lab_kernel(const LabParams P)
{
    __shared__ int4 s_in_all[4][2][CH];      // {H, F, labH, labF} of the row above
    __shared__ int4 s_out_all[4][2 * CH];    // bottom row ring
    __shared__ uint32_t s_sel_all[4][2][CH]; // column selectors
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    int4 (*s_in)[CH] = s_in_all[wid];
    int4 *s_out = s_out_all[wid];
    uint32_t (*s_sel)[CH] = s_sel_all[wid];
    const int go = P.go, ge = P.ge;
    constexpr int R = 32 * RPT;

    for (;;) {
        int tk = 0, stop_now = 0;
        if (lane == 0) { tk = atomicAdd(P.ticket_ctr, 1); stop_now = ld_volatile(P.err); }
        tk = __shfl_sync(FULL, tk, 0);
        stop_now = __shfl_sync(FULL, stop_now, 0);
        if (tk >= P.ntickets || stop_now) return;
        const int2 tb = P.tickets[tk];
        const LabProblem &pr = P.probs[tb.x];
        const int band = tb.y;
        const int n = pr.n, m = pr.m, ck = pr.ck;
        const uint8_t *__restrict__ bseq = pr.b;
        int4 *__restrict__ bus = pr.bus;
        int *__restrict__ flags = pr.flags;
        const int need = band - 1;
        const bool fresh = ck > 0 && band > 0 && (band % ck) == 0;
        const bool ckpt_band = ck > 0 && ((band + 1) % ck) == 0 && band + 1 < pr.nbands;
        int4 *ck_row = ckpt_band ? pr.ckpt + (size_t)((band + 1) / ck - 1) * (size_t)m : nullptr;
        const bool src_f = pr.src == ST_F;
        const int blab = (ck > 0 && band >= ck) ? ((0 << 2) | (go == ge ? LAB_OPEN : LAB_EXT)) : LAB_INIT;
        const int prev_blab = (ck > 0 && band - 1 >= ck) ? ((0 << 2) | (go == ge ? LAB_OPEN : LAB_EXT)) : LAB_INIT;

        const int rowbase = band * R + lane * RPT;   // 0-based row index of the lane's first row
        uint32_t plo[RPT], phi[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = rowbase + k;
            uint32_t lo = VIRTUAL_PROF, hi = VIRTUAL_PROF;
            if (r < n) {
                const int c = pr.a[r] & 7;
                lo = P.prof_lo[c];
                if (PROF2) hi = P.prof_hi[c];
            }
            plo[k] = lo;
            phi[k] = PROF2 ? hi : 0u;
        }
        // column 0 border: H(i,0) = F(i,0) = BIAS - cost(i); E(i,0) = -inf
        int Hl[RPT], E[RPT], lHl[RPT], lE[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int i = rowbase + k + 1;
            Hl[k] = max(0, BIAS - border_cost(i, src_f, go, ge));
            E[k] = 0;
            lHl[k] = blab;
            lE[k] = LAB_INIT;
        }
        int Hlast = Hl[RPT - 1], Flast = 0, lHlast = blab, lFlast = LAB_INIT;
        // a valid selector for the cells left of the band's first column
        uint32_t sellast = code_selector(0);
        int updiag, lupdiag;
        if (band == 0) { updiag = (lane == 0) ? BIAS : Hl[0]; lupdiag = LAB_INIT; }
        else { updiag = max(0, BIAS - border_cost(rowbase, src_f, go, ge)); lupdiag = lane ? blab : prev_blab; }
        if (lane > 0) {
            // H(row above the lane, 0): the previous lane's last row
            updiag = max(0, BIAS - border_cost(rowbase, src_f, go, ge));
            lupdiag = blab;
        }
        // sink bookkeeping
        const int sink_k = n - 1 - rowbase;            // row n lives at k = sink_k in this lane
        const bool has_sink = sink_k >= 0 && sink_k < RPT;
        bool aborted = false;
        unsigned tiles = 0, pruned = 0;

        const int nch = (m + CH - 1) / CH;
        const int rows_left = n - band * R;
        const bool dyn = P.prune && pr.target > 0;
        const long long target = pr.target;
        // Static envelope: only cells whose best source-to-sink bound reaches
        // the target can lie on an optimal path, and such a cell's optimal
        // predecessors are such cells too, so chunks outside the band's range
        // are never computed and inputs outside the predecessor's range are
        // taken as -infinity without waiting for them.
        int q_lo = 0, q_hi = nch - 1, p_lo = 0, p_hi = nch - 1;
        {
            const long long S = target - BIAS;
            const long long a_sub = P.max_sub, g_min = ge;
            if (dyn && a_sub * min(n, m) - g_min * (n > m ? n - m : m - n) >= S) {
                const int2 own = env_band(band, R, n, m, a_sub, g_min, S);
                q_lo = own.x; q_hi = own.y;
                if (band > 0) {
                    const int2 pre = env_band(band - 1, R, n, m, a_sub, g_min, S);
                    p_lo = pre.x; p_hi = pre.y;
                }
            }
        }
        const LabGuide gd = lab_guide(pr, P, band, R), gd_next = lab_guide(pr, P, band + 1, R);
        const bool has_next_band = band + 1 < pr.nbands;
        // Dynamic range: every band marks each chunk it releases as useful or
        // not (low bit of the flag: can a value of the chunk still reach the
        // target from the next band?) and publishes its first and last useful
        // chunk.  The next band takes everything else as -infinity: it starts
        // at the first useful chunk (unless the column-0 border itself can
        // still reach the target), never waits for chunks outside the range and
        // stops once a pruned block has nothing useful left from its column on.
        int pfirst = 0;
        const int *pred_last = nullptr;
        if (dyn && band > 0) {
            int pf = 0, ok = 1;
            if (lane == 0) ok = wait_published(&pr.span[band - 1].x, P.err, P.timeout_ns, &pf);
            ok = __shfl_sync(FULL, ok, 0);
            pf = __shfl_sync(FULL, pf, 0);
            if (!ok) continue;                // the error word is set: every band stops
            pfirst = pf;
            pred_last = &pr.span[band - 1].y;
        }
        int L = q_lo;
        if (dyn) {
            const long long bh = band == 0 ? BIAS : max(0, BIAS - border_cost(band * R, src_f, go, ge));
            if (bh + lab_gain(pr, P, gd, band, 0, R, gd.entry(0)) < target) L = max(L, pfirst);
        }
        if (L > q_hi) {
            // nothing of this band can reach the target
            if (lane == 0) {
                st_release(&pr.span[band].x, SPAN_NONE);
                st_release(&pr.span[band].y, -1);
            }
            continue;
        }
        if (L > 0) {
            // the band enters at chunk L with everything to its left dead
#pragma unroll
            for (int k = 0; k < RPT; ++k) { Hl[k] = 0; E[k] = 0; lHl[k] = LAB_INIT; lE[k] = LAB_INIT; }
            Hlast = 0; lHlast = LAB_INIT;
            updiag = 0; lupdiag = LAB_INIT;
        }
        // input chunk c: 1 useful (read the bus), 0 dead, 2 not released yet
        auto in_status = [&](int c) -> int {
            if (c < p_lo || c > p_hi || c < pfirst) return 0;
            const int v = ld_acquire(&flags[c]);
            if (v >= 2 * need) return v & 1;
            if (pred_last) {
                const int y = ld_acquire(pred_last);
                if (y != SPAN_UNPUB && c > y) return 0;
            }
            return 2;
        };
        // the same, waiting (bounded) for the release; -1 when the band must stop
        auto wait_status = [&](int c) -> int {
            int st = in_status(c);
            if (st != 2) return st;
            const unsigned long long t0 = globaltimer();
            unsigned ns = 64;
            for (;;) {
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
                st = in_status(c);
                if (st != 2) return st;
                if (ld_volatile(P.err)) return -1;
                if (globaltimer() - t0 > P.timeout_ns) { atomicCAS(P.err, 0, DEV_ETIMEOUT); return -1; }
            }
        };
        {
            int st = 0;
            if (lane == 0) st = wait_status(L);
            st = __shfl_sync(FULL, st, 0);
            if (st < 0) aborted = true;
            else {
                int4 v = make_int4(0, 0, LAB_INIT, LAB_INIT);
                uint32_t sel = 0;
                const int col = L * CH + lane;
                if (col < m) {
                    if (st == 1) v = bus[col];
                    sel = code_selector(bseq[col]);
                }
                s_in[L & 1][lane] = v;
                s_sel[L & 1][lane] = sel;
            }
            __syncwarp();
        }
        bool first_pub = false;
        int last_useful = -1;
        for (int q = L; q <= q_hi + 1 && !aborted; ++q) {
            const int buf = q & 1;
            // record entries for this block and for the chunk flushed at its end,
            // loaded first so that their latency overlaps the block's work
            const int e_own = gd.entry(q), e_nx = gd_next.entry(q - 1);
            const bool has_next = q + 1 <= q_hi;
            int nst = 0;
            int4 nv = make_int4(0, 0, LAB_INIT, LAB_INIT);
            uint32_t nsel = 0;
            const int ncol = (q + 1) * CH + lane;
            if (has_next) {
                if (lane == 0) nst = in_status(q + 1);
                nst = __shfl_sync(FULL, nst, 0);
                if (nst != 2 && ncol < m) {
                    if (nst == 1) nv = bus[ncol];
                    nsel = code_selector(bseq[ncol]);
                }
            }
            bool skip = false;
            if (dyn) {
                int mx = 0;
#pragma unroll
                for (int k = 0; k < RPT; ++k) mx = max(mx, Hl[k]);
                mx = max(mx, max(Hlast, updiag));
                if (q <= q_hi) mx = max(mx, s_in[buf][lane].x);
                mx = __reduce_max_sync(FULL, mx);
                skip = (long long)mx + lab_gain(pr, P, gd, band, q, R, e_own) < target;
            }
            ++tiles;
            if (skip) {
                ++pruned;
#pragma unroll
                for (int k = 0; k < RPT; ++k) { Hl[k] = 0; E[k] = 0; }
                Hlast = 0; Flast = 0;
                if (q <= q_hi) {
                    sellast = s_sel[buf][31 - lane];
                    updiag = (lane == 0) ? s_in[buf][31].x : 0;
                    lupdiag = (lane == 0) ? s_in[buf][31].z : 0;
                } else { updiag = 0; }
                const int oc = q * CH - 31 + lane;
                if (oc >= 0 && oc < m) s_out[oc & 63] = make_int4(0, 0, LAB_INIT, LAB_INIT);
            } else {
#pragma unroll 1
                for (int u = 0; u < CH; ++u) {
                    const int4 in = s_in[buf][u];
                    const uint32_t insel = s_sel[buf][u];
                    const int rH = __shfl_up_sync(FULL, Hlast, 1);
                    const int rF = __shfl_up_sync(FULL, Flast, 1);
                    const int rlH = __shfl_up_sync(FULL, lHlast, 1);
                    const int rlF = __shfl_up_sync(FULL, lFlast, 1);
                    const uint32_t rS = __shfl_up_sync(FULL, sellast, 1);
                    const int j = q * CH + u - lane;       // 0-based column; DP column j + 1
                    int upH, upF, lupH, lupF, ldiag;
                    const uint32_t sel = lane ? rS : insel;
                    int diag = updiag;
                    if (lane) {
                        upH = rH; upF = rF; lupH = rlH; lupF = rlF; ldiag = lupdiag;
                    } else {
                        upH = in.x; upF = in.y;
                        if (fresh) {
                            ldiag = (j << 2) | LAB_DIAG;
                            lupH = ((j + 1) << 2) | LAB_OPEN;
                            lupF = ((j + 1) << 2) | LAB_EXT;
                        } else {
                            ldiag = lupdiag; lupH = in.z; lupF = in.w;
                        }
                    }
                    updiag = upH;
                    lupdiag = lupH;
                    sellast = sel;
                    if ((unsigned)j < (unsigned)m) {
                        int hgo = upH - go;
                        int F = upF, lF = lupF, lH = lupH;
                        const bool sink_step = has_sink && j == m - 1;
                        int sH = 0, sF = 0, sE = 0, slH = 0, slF = 0, slE = 0;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            const int s = sub_lookup(plo[k], phi[k], sel);
                            bool pv, pt, pd, pe;
                            // F(i,j): open from H(i-1,j) preferred on ties
                            F = __vibmax_s32(hgo, F - ge, &pv);
                            lF = pv ? lH : lF;
                            const int Ein = E[k], lEin = lE[k];
                            int t, lt;
                            if (PREF_VERT) { t = __vibmax_s32(F, Ein, &pt); lt = pt ? lF : lEin; }
                            else { t = __vibmax_s32(Ein, F, &pt); lt = pt ? lEin : lF; }
                            const int h = __vibmax_s32(diag + s, t, &pd);
                            const int lh = pd ? ldiag : lt;
                            diag = Hl[k];
                            ldiag = lHl[k];
                            Hl[k] = h;
                            lHl[k] = lh;
                            hgo = h - go;
                            E[k] = __vibmax_s32(hgo, Ein - ge, &pe);   // E(i, j+1)
                            lE[k] = pe ? lh : lEin;
                            lH = lh;
                            if (sink_step && k == sink_k) {
                                sH = h; sF = F; sE = Ein; slH = lh; slF = lF; slE = lEin;
                            }
                        }
                        Hlast = Hl[RPT - 1]; lHlast = lH;
                        Flast = F; lFlast = lF;
                        if (sink_step) {
                            pr.sink[0] = make_int4(sH, sF, sE, 1);
                            pr.sink[1] = make_int4(slH, slF, slE, 1);
                        }
                        if (lane == 31) s_out[j & 63] = make_int4(Hlast, Flast, lHlast, lFlast);
                    }
                }
            }
            if (has_next) {
                if (nst == 2) {
                    int st = 0;
                    if (lane == 0) st = wait_status(q + 1);
                    st = __shfl_sync(FULL, st, 0);
                    if (st < 0) { aborted = true; break; }
                    if (ncol < m) {
                        if (st == 1) nv = bus[ncol];
                        nsel = code_selector(bseq[ncol]);
                    }
                }
                s_in[buf ^ 1][lane] = nv;
                s_sel[buf ^ 1][lane] = nsel;
            }
            __syncwarp();
            if (q > L) {
                const int c = q - 1;
                const int col = c * CH + lane;
                int hmax = 0;
                if (col < m) {
                    const int4 o = s_out[col & 63];
                    bus[col] = o;
                    if (ck_row) ck_row[col] = o;
                    hmax = o.x;
                }
                bool useful = true;
                if (dyn && has_next_band) {
                    hmax = __reduce_max_sync(FULL, hmax);
                    useful = (long long)hmax + lab_gain(pr, P, gd_next, band + 1, c, R, e_nx) >= target;
                }
                __syncwarp();
                if (lane == 0) {
                    st_release(&flags[c], 2 * band + (useful ? 1 : 0));
                    if (useful && dyn && !first_pub) st_release(&pr.span[band].x, c);
                }
                if (useful) { first_pub = true; last_useful = c; }
            }
            if (dyn && skip && q <= q_hi) {
                // a pruned block leaves only dead state behind; the band is done
                // when nothing useful arrives from chunk q on
                int done = q > p_hi;
                if (!done && pred_last) {
                    int y = SPAN_UNPUB;
                    if (lane == 0) y = ld_acquire(pred_last);
                    y = __shfl_sync(FULL, y, 0);
                    done = y != SPAN_UNPUB && q > y;
                }
                if (done) break;
            }
        }
        if (!aborted) {
            if (dyn && lane == 0) {
                if (!first_pub) st_release(&pr.span[band].x, SPAN_NONE);
                st_release(&pr.span[band].y, last_useful);
            }
            if (lane == 0) {
                atomicAdd(&P.stats[1], (unsigned long long)tiles);
                atomicAdd(&P.stats[2], (unsigned long long)pruned);
                atomicAdd(&P.stats[0], (unsigned long long)(tiles - pruned) * CH *
                                           (unsigned long long)min(R, rows_left));
            }
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void lab_init_kernel(LabProblem *probs, int nprobs, int go, int ge)
{
    const int p = blockIdx.x;
    if (p >= nprobs) return;
    const LabProblem pr = probs[p];
    const bool src_e = pr.src == ST_E;
    for (int j = threadIdx.x; j < pr.m; j += blockDim.x) {
        // row 0: H(0, j+1) = E(0, j+1) = BIAS - cost(j+1); F = -inf
        const int c = src_e ? ge * (j + 1) : go + ge * j;
        pr.bus[j] = make_int4(max(0, BIAS - c), 0, LAB_INIT, LAB_INIT);
    }
    const int nch = (pr.m + CH - 1) / CH;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) pr.flags[c] = -1;   // row 0: released, useful
    for (int b = threadIdx.x; b < pr.nbands; b += blockDim.x) pr.span[b] = make_int2(SPAN_UNPUB, SPAN_UNPUB);
    if (threadIdx.x == 0) {
        pr.sink[0] = make_int4(0, 0, 0, 0);
        pr.sink[1] = make_int4(0, 0, 0, 0);
    }
}

// one thread per problem: follow the labels from the sink back through the
// checkpoint rows.  out[p*stride + t-1] = {col, type, value of the crossing's
// source node, 0} for checkpoint t = 1..nck; res[p] = {sink value, ok, 0, 0}.
__global__ void lab_walk_kernel(const LabProblem *probs, int nprobs, int R, int go, int ge,
                                int4 *out, int stride, int4 *res)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprobs) return;
    const LabProblem pr = probs[p];
    const int4 sv = pr.sink[0], sl = pr.sink[1];
    int v = pr.snk == ST_H ? sv.x : (pr.snk == ST_F ? sv.y : sv.z);
    int L = pr.snk == ST_H ? sl.x : (pr.snk == ST_F ? sl.y : sl.z);
    int ok = sv.w == 1;
    const int nck = pr.ck > 0 ? (pr.nbands - 1) / pr.ck : 0;
    const bool src_f = pr.src == ST_F;
    for (int t = nck; t >= 1 && ok; --t) {
        const int type = L & 3, c = L >> 2;
        if (type == LAB_INIT || c < 0 || c > pr.m) { ok = 0; break; }
        const int st = (type == LAB_EXT) ? ST_F : ST_H;
        const int r = t * pr.ck * R;         // DP row of checkpoint t
        int vu, Lp;
        if (c == 0) {
            vu = max(0, BIAS - border_cost(r, src_f, go, ge));
            Lp = (t >= 2) ? ((0 << 2) | (go == ge ? LAB_OPEN : LAB_EXT)) : LAB_INIT;
        } else {
            const int4 e = pr.ckpt[(size_t)(t - 1) * pr.m + (c - 1)];
            vu = st == ST_H ? e.x : e.y;
            Lp = st == ST_H ? e.z : e.w;
        }
        out[(size_t)p * stride + (t - 1)] = make_int4(c, type, vu, r);
        L = Lp;
    }
    res[p] = make_int4(v, ok, nck, 0);
}

// ---------------------------------------------------------------------------
template <int RPT, bool PV, bool P2>
static cudaError_t lab_one(const LabParams &p, int ctas, cudaStream_t s)
{
    lab_kernel<RPT, PV, P2><<<ctas, 128, 0, s>>>(p);
    return cudaGetLastError();
}

template <int RPT>
static cudaError_t lab_launch_rpt(const LabParams &p, bool pref_vert, bool p2, int ctas, cudaStream_t s)
{
    if (pref_vert) return p2 ? lab_one<RPT, true, true>(p, ctas, s) : lab_one<RPT, true, false>(p, ctas, s);
    return p2 ? lab_one<RPT, false, true>(p, ctas, s) : lab_one<RPT, false, false>(p, ctas, s);
}

cudaError_t lab_launch(const LabParams &p, int rpt, bool pref_vert, bool p2, int ctas, cudaStream_t s)
{
    if (rpt == LAB_RPT) return lab_launch_rpt<LAB_RPT>(p, pref_vert, p2, ctas, s);
    if (LAB_RPT_GUIDED != LAB_RPT && rpt == LAB_RPT_GUIDED) return lab_launch_rpt<LAB_RPT_GUIDED>(p, pref_vert, p2, ctas, s);
    return cudaErrorInvalidValue;
}

template <int RPT>
static cudaError_t lab_occupancy_rpt(bool pref_vert, bool p2, int *n)
{
    if (pref_vert)
        return p2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lab_kernel<RPT, true, true>, 128, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lab_kernel<RPT, true, false>, 128, 0);
    return p2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lab_kernel<RPT, false, true>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, lab_kernel<RPT, false, false>, 128, 0);
}

cudaError_t lab_occupancy(int rpt, bool pref_vert, bool p2, int *n)
{
    if (rpt == LAB_RPT) return lab_occupancy_rpt<LAB_RPT>(pref_vert, p2, n);
    if (LAB_RPT_GUIDED != LAB_RPT && rpt == LAB_RPT_GUIDED) return lab_occupancy_rpt<LAB_RPT_GUIDED>(pref_vert, p2, n);
    return cudaErrorInvalidValue;
}

cudaError_t lab_init_launch(LabProblem *probs, int nprobs, int go, int ge, cudaStream_t s)
{
    if (nprobs <= 0) return cudaSuccess;
    lab_init_kernel<<<nprobs, 256, 0, s>>>(probs, nprobs, go, ge);
    return cudaGetLastError();
}

cudaError_t lab_walk_launch(const LabProblem *probs, int nprobs, int R, int go, int ge, int4 *out, int stride,
                            int4 *res, cudaStream_t s)
{
    if (nprobs <= 0) return cudaSuccess;
    lab_walk_kernel<<<(nprobs + 127) / 128, 128, 0, s>>>(probs, nprobs, R, go, ge, out, stride, res);
    return cudaGetLastError();
}

}  // namespace swgb
