// fwd16.cu -- forward pass on int16x2 lanes (sm_103a DPX 16x2 forms).
//
// Same computation and tie rule as fwd.cu, with two cells per register: a warp
// owns a band of 64*RPT rows, lane t holds the rows of "virtual lane" t in the
// low halfword and of virtual lane t+32 in the high halfword of every state
// register.  Virtual lane v processes column j at step j + v, so the high half
// runs 32 columns behind the low half.  Each step the bottom row of every
// virtual lane moves to the next one by a rotating shuffle (lane 0's high half
// receives lane 31's low half); lane 0's low half reads the row above the band
// from the shared-memory chunk, lane 31's high half writes the band's bottom row.
//
// Two value encodings (template REL):
//  * absolute (REL = false, local mode, batches): int16 scores; the host routes
//    a pair here only when its score bound fits, and a value reaching the guard
//    (32767 - max_sub) sets the problem's overflow word so the pair is re-run on
//    int32 lanes (the first value reaching the guard is computed before anything
//    can wrap, since H grows by at most max_sub per step).
//  * relative (REL = true, local and anchored modes, single long pairs): every
//    value is stored minus a warp-wide offset O, re-chosen at each 32-step block
//    so the largest live value sits at 16384.  Horizontally or vertically
//    adjacent cells differ by at most go + max_sub, so all true values of a
//    band's window (64*RPT rows x 96 columns) lie within (64*RPT + 96) *
//    (go + max_sub) of each other; the host uses this encoding only when that
//    spread fits.  Minus infinity (anchored borders) and skipped cells are the
//    sentinel FLOOR = -32512, which lies below every true value of the window
//    and above anything an add can wrap from.  The local zero floor is the
//    register fl2 = max(-O, FLOOR).  The boundary row in HBM stays absolute
//    int32 (converted when a chunk enters shared memory / leaves lane 31).
//
// Per cell pair: prmt (both substitution scores), viaddmax16x2 (F),
// viaddmax16x2 (diag + s vs E), vimax3_16x2 (with F and the floor),
// viaddmax16x2 (H - go), viaddmax16x2 (E), vimax16x2 for the running maximum.
#include "common.cuh"
#include "kernels.h"

namespace swgb {

__device__ __forceinline__ uint32_t p16(int lo, int hi) {
    return ((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ int lo16(uint32_t x) { return (int)(int16_t)(x & 0xffffu); }
__device__ __forceinline__ int hi16(uint32_t x) { return (int)(int16_t)(x >> 16); }
__device__ __forceinline__ uint32_t perm(uint32_t a, uint32_t b, uint32_t s) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(s));
    return r;
}
// selector of a column code for the low half (bytes 0-3 of the profile pair);
// the high half's selector is the same plus 0x44 (bytes 4-7)
__device__ __forceinline__ uint32_t sel_lo8(uint32_t c) { return c | ((c | 8u) << 4); }

// a valid selector pair (code 0 for both halves)
constexpr uint32_t SEL_NEUTRAL = (0u | (8u << 4)) | (((0u | (8u << 4)) + 0x44u) << 8);

// per-halfword max of two (DPX three-input form with a repeated operand)
__device__ __forceinline__ uint32_t vmax16(uint32_t a, uint32_t b) { return __vimax3_s16x2(a, b, b); }

// A step's detection value: max(thr1, H of every row of the lane) per half,
// in three-way maxima over pairs of rows (RPT / 2 operations), so it differs
// from thr1 exactly when some cell of the step exceeds the threshold.
template <int RPT>
__device__ __forceinline__ uint32_t rows_max(const uint32_t (&Hl)[RPT], uint32_t thr1)
{
    uint32_t m = __vimax3_s16x2(thr1, Hl[0], Hl[RPT > 1 ? 1 : 0]);
#pragma unroll
    for (int k = 2; k + 1 < RPT; k += 2) m = __vimax3_s16x2(m, Hl[k], Hl[k + 1]);
    if (RPT > 2 && (RPT & 1)) m = vmax16(m, Hl[RPT - 1]);
    return m;
}

constexpr int REL_FLOOR = -32768 + 256;
constexpr int REL_TOP = 16384;

// absolute int32 -> relative int16 range; anchored minus infinity (biased values
// below BIAS/2) and anything below the window become FLOOR
__device__ __forceinline__ int to_rel(int v, int O, bool anch)
{
    if (anch && v < BIAS / 2) return REL_FLOOR;
    const long long r = (long long)v - O;
    return (int)(r < REL_FLOOR ? REL_FLOOR : (r > 32767 ? 32767 : r));
}

// Anchored with the forward record: any path through a cell of band `band`
// that reaches the start crosses a recorded forward row r at or above the band
// (or starts below it), so what it gains beyond the band's frontier (its rows
// and the row above) is at most max_sub per row from the frontier up to r, plus
// the largest forward H of row r left of the cell's column, plus the slack of
// the split cell.  Row 0 of the forward matrix is all zero.
struct GinRow {
    const int32_t *row = nullptr;
    long long gain = 0;            // max_sub * rows + slack (add the record entry)
    int lo = 1, hi = 0, nch = 0;   // written chunk range of the row
    bool valid = false;
    // record entry bounding forward columns up to jf (0 below the written range)
    __device__ __forceinline__ int at(int jf) const {
        if (!row || jf < 1) return 0;
        const int c = min(nch - 1, (jf - 1) / CH);
        if (hi < lo || c < lo) return 0;
        return row[min(c, hi)];
    }
};

__device__ __forceinline__ GinRow gin_for_band(const FwdProblem &pr, const FwdParams &P, int band, int R)
{
    GinRow g;
    if (!pr.gin) return g;
    const long long T = max(1LL, (long long)pr.gin_i0 - (long long)(band + 1) * R);
    long long k = T / pr.gin_step - 1;
    if (k > pr.gin_rows - 1) k = pr.gin_rows - 1;
    const long long r = k >= 0 ? (k + 1) * (long long)pr.gin_step : 0;
    if (k >= 0) {
        g.row = pr.gin + (size_t)k * (size_t)(pr.gin_nch + 2);
        g.nch = pr.gin_nch;
        g.lo = g.row[pr.gin_nch];
        g.hi = g.row[pr.gin_nch + 1];
    }
    g.gain = (long long)P.max_sub * ((long long)pr.gin_i0 - (long long)band * R - r) + P.slack;
    g.valid = true;
    return g;
}

// row of the record this band writes (null: none)
__device__ __forceinline__ int32_t *rec_row(const FwdProblem &pr, int band)
{
    if (!pr.gout || (band + 1) % pr.gstride != 0) return nullptr;
    return pr.gout + (size_t)((band + 1) / pr.gstride - 1) * (size_t)(pr.gnch + 2);
}

template <int RPT, bool REL, bool ANCH, int NW>
__global__ void __launch_bounds__(NW * 32) fwd16_kernel(const FwdParams P)
{
    // NW warps per CTA.  Four: every warp claims its own band.  More (one CTA
    // per SM, the full-width local pass): the CTA claims NW consecutive bands
    // and gives each scheduler (warp slots s, s + 4, s + 8, ...) NW / 4
    // consecutive ones, slot order = band order.  A scheduler favours its
    // older warps; with bands of unrelated parts of the chain on one
    // scheduler, the band that loses holds up every band after it, while here
    // the favoured warp is the one the others wait for.
    static_assert(NW % 4 == 0 && (NW == 4 || !ANCH), "grouped hand-over uses four-warp CTAs");
    __shared__ int4 s_in_all[NW][3][CH];   // {H, F, selector8, 0} per column, three chunks
    __shared__ uint32_t s_out_all[NW][2 * CH];   // bottom row, packed int16 (H | F << 16)
    // Grouped launch (anchored): a CTA takes four consecutive tickets, and a band
    // whose successor runs in the same CTA hands its bottom row over through a
    // ring of GK chunks in shared memory instead of the boundary row in HBM and
    // its flags.  The anchored pass follows a narrow band around the path, where
    // the bands form a chain and hand-over latency is part of the pass's time;
    // the full-width local pass runs faster with its producers decoupled.
    constexpr bool GROUP = ANCH;
    constexpr int GW = 4, GK = 8;
    __shared__ int2 s_ring[GROUP ? GW : 1][GROUP ? GK : 1][CH];   // absolute {H, F}
    __shared__ int s_tag[GROUP ? GW : 1][GROUP ? GK : 1];         // 2 * chunk + useful
    __shared__ int s_need[GW], s_spx[GW], s_spy[GW];              // reader's next chunk; span
    __shared__ int s_base, s_err;
    __shared__ int s_grun[NW];                                    // record row's running maximum
    __shared__ int32_t *s_grow[NW];                               // record row of the warp's band
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    int4 (*s_in)[CH] = s_in_all[wid];
    uint32_t *s_out = s_out_all[wid];
    const uint32_t pk_in = lane ? 0x3210u : 0x1054u;  // lane 0 splices the band's input in
    const int go = P.go, ge = P.ge;
    const uint32_t go2 = p16(-go, -go), ge2 = p16(-ge, -ge);
    const uint32_t NEG2 = REL ? p16(REL_FLOOR, REL_FLOOR) : p16(-32768, -32768);
    const uint32_t ZERO2 = 0u;
    const int src_lane = (lane + 31) & 31;
    constexpr int R = 64 * RPT;

    for (;;) {
        int tk = 0, stop_now = 0, gbase = 0;
        if (GROUP) {
            __syncthreads();                               // the previous group is done
            if (threadIdx.x == 0) { s_base = atomicAdd(P.ticket_ctr, GW); s_err = ld_volatile(P.err); }
            if (lane == 0) {
                for (int k = 0; k < GK; ++k) s_tag[wid][k] = -1;
                s_need[wid] = INT_MIN; s_spx[wid] = SPAN_UNPUB; s_spy[wid] = SPAN_UNPUB;
            }
            __syncthreads();
            gbase = s_base;
            if (gbase >= P.ntickets || s_err) return;      // the whole CTA leaves together
            tk = gbase + wid;
            if (tk >= P.ntickets) continue;
        } else if (NW > 4) {
            __syncthreads();                               // the previous claim is done
            if (threadIdx.x == 0) { s_base = atomicAdd(P.ticket_ctr, NW); s_err = ld_volatile(P.err); }
            __syncthreads();
            gbase = s_base;
            if (gbase >= P.ntickets || s_err) return;      // the whole CTA leaves together
            tk = gbase + (wid & 3) * (NW / 4) + (wid >> 2);
            if (tk >= P.ntickets) continue;
        } else {
            if (lane == 0) { tk = atomicAdd(P.ticket_ctr, 1); stop_now = ld_volatile(P.err); }
            tk = __shfl_sync(FULL, tk, 0);
            stop_now = __shfl_sync(FULL, stop_now, 0);
            if (tk >= P.ntickets || stop_now) return;
        }
        const int2 tb = P.tickets[tk];
        const FwdProblem &pr = P.probs[tb.x];
        const int band = tb.y;
        const int n = pr.n, m = pr.m;
        const bool transposed = pr.transposed != 0;
        constexpr bool anch = REL && ANCH;    // every problem of an anchored launch is anchored
        const uint8_t *__restrict__ bseq = pr.b;
        unsigned long long *__restrict__ busw = (unsigned long long *)pr.bus;
        int *stop = anch ? pr.stop_band : nullptr;
        using BW = BusWord<anch>;
        const unsigned want_tag = BW::band_tag(band - 1);           // tag of the row above
        const int guard = 32767 - P.max_sub;
        const int target = pr.target;
        // dead values of skipped cells, absolute (what the boundary row carries)
        const int DEAD_H = 0, DEAD_F = anch ? 0 : -go;

        const int rb_lo = band * R + lane * RPT;           // first row of the low half
        const int rb_hi = rb_lo + 32 * RPT;                // first row of the high half
        uint32_t plo[RPT], phi[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r0 = rb_lo + k, r1 = rb_hi + k;
            const uint32_t *prof = transposed ? P.prof_lo_t : P.prof_lo;
            plo[k] = (r0 < n) ? prof[pr.a[r0] & 7] : VIRTUAL_PROF;
            phi[k] = (r1 < n) ? prof[pr.a[r1] & 7] : VIRTUAL_PROF;
        }
        bool aborted = false;
        const int nch = (m + CH - 1) / CH;
        const int nblk = nch + 2;
        const int rows_left = n - band * R;
        // Dynamic range (anchored with pruning): every band marks each chunk it
        // releases as useful or not (low bit of the flag: can a value of the
        // chunk still reach the target from the next band?) and publishes its
        // first and last useful chunk.  Below the anchor the left border is
        // minus infinity, so the next band starts at the first useful chunk,
        // takes everything else as minus infinity without waiting for it and
        // stops once a pruned block has nothing useful left from its column on.
        const bool dyn = anch && P.prune;
        // neighbours in this CTA's group: the predecessor's row arrives through
        // its ring, this band's row leaves through its own ring
        const bool pred_in = GROUP && wid > 0 && P.tickets[tk - 1].x == tb.x && P.tickets[tk - 1].y == band - 1;
        const bool succ_in = GROUP && wid < GW - 1 && tk + 1 < P.ntickets && P.tickets[tk + 1].x == tb.x &&
                             P.tickets[tk + 1].y == band + 1;
        volatile int *vtag = GROUP && pred_in ? (volatile int *)s_tag[wid - 1] : nullptr;
        volatile int *vneed = (volatile int *)s_need;
        volatile int *vspx = (volatile int *)s_spx, *vspy = (volatile int *)s_spy;
        // the reader of this band's ring no longer needs anything (bands that end early)
        auto release_reader = [&]() {
            if (GROUP && lane == 0) { __threadfence_block(); vneed[wid] = INT_MAX; }
        };
        int pfirst = 0;
        const int *pred_last = nullptr;
        if (dyn && band > 0) {
            int pf = 0, ok = 1;
            if (lane == 0) {
                if (pred_in) {
                    const unsigned long long t0 = globaltimer();
                    for (;;) {
                        pf = vspx[wid - 1];
                        if (pf != SPAN_UNPUB) break;
                        __nanosleep(20);
                        if (ld_volatile(P.err) || (stop && ld_volatile(stop) < band)) { ok = 0; break; }
                        if (globaltimer() - t0 > P.timeout_ns) { atomicCAS(P.err, 0, DEV_ETIMEOUT); ok = 0; break; }
                    }
                    __threadfence_block();
                } else {
                    ok = wait_published(&pr.span[band - 1].x, P.err, P.timeout_ns, &pf, stop, band);
                }
            }
            ok = __shfl_sync(FULL, ok, 0);
            pf = __shfl_sync(FULL, pf, 0);
            if (!ok) { release_reader(); continue; }    // error, or the search already ended above
            pfirst = pf;
            pred_last = pred_in ? nullptr : &pr.span[band - 1].y;
        }
        const int L = pfirst;
        if (L >= nch) {
            // nothing from above can reach the target: neither can this band
            if (lane == 0) {
                if (succ_in) { vspx[wid] = SPAN_NONE; vspy[wid] = -1; }
                else { st_release(&pr.span[band].x, SPAN_NONE); st_release(&pr.span[band].y, -1); }
            }
            release_reader();
            continue;
        }
        // Input chunk c, called by the whole warp: returns 1 (useful; v holds the
        // lane's column), 0 (dead: minus infinity, no data needed) or 2 (not yet
        // written).  From the ring: the producer's tag for the chunk.  From the
        // boundary row: every word carries its writer's band, so the data load is
        // also the readiness test (no flag, no fence).
        auto in_status = [&](int c, int2 &v) -> int {
            if (c < pfirst) return 0;
            if (pred_in) {
                int st = 2;
                if (lane == 0) {
                    const int t = vtag[c % GK];
                    if ((t >> 1) == c) { __threadfence_block(); st = t & 1; }
                    else {
                        const int y = vspy[wid - 1];
                        if (y != SPAN_UNPUB && c > y) st = 0;
                    }
                }
                st = __shfl_sync(FULL, st, 0);
                if (st == 1) {
                    __syncwarp();      // orders the ring reads after lane 0's view of the tag
                    v = s_ring[GROUP ? wid - 1 : 0][GROUP ? c % GK : 0][lane];
                }
                return st;
            }
            const int col = c * CH + lane;
            unsigned long long w = 0;
            bool ok = true;
            if (col < m) {
                w = ld_relaxed_u64(&busw[col]);
                ok = (BW::tag_of(w) >> 1) == want_tag;
            }
            if (__all_sync(FULL, ok)) {
                v = make_int2(BW::h(w), BW::f(w));
                return __shfl_sync(FULL, (int)(BW::tag_of(w) & 1u), 0);   // column c * CH < m
            }
            if (pred_last) {
                int y = 0;
                if (lane == 0) y = ld_acquire(pred_last);
                y = __shfl_sync(FULL, y, 0);
                if (y != SPAN_UNPUB && c > y) return 0;
            }
            return 2;
        };
        // tell the predecessor that chunks before `next` have been read
        auto mark_read = [&](int next) {
            if (GROUP && pred_in) {
                __syncwarp();
                if (lane == 0) { __threadfence_block(); vneed[wid] = next; }
            }
        };
        // the same, waiting (bounded) for the chunk; -1 when the band must stop
        auto wait_status = [&](int c, int2 &v) -> int {
            int st = in_status(c, v);
            if (st != 2) return st;
            const unsigned long long t0 = globaltimer();
            unsigned ns = 64;
            for (;;) {
                if (!pred_in) {
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                } else {
                    __nanosleep(20);
                }
                st = in_status(c, v);
                if (st != 2) return st;
                int quit = 0;
                if (lane == 0) {
                    if (ld_volatile(P.err) || (stop && ld_volatile(stop) < band)) quit = 1;
                    else if (globaltimer() - t0 > P.timeout_ns) { atomicCAS(P.err, 0, DEV_ETIMEOUT); quit = 1; }
                }
                if (__shfl_sync(FULL, quit, 0)) return -1;
            }
        };
        {
            int2 v = make_int2(DEAD_H, DEAD_F);
            const int st = wait_status(L, v);
            if (st < 0) aborted = true;
            else {
                if (st != 1 || L * CH + lane >= m) v = make_int2(DEAD_H, DEAD_F);
                uint32_t sel = 0;
                const int col = L * CH + lane;
                if (col < m) sel = sel_lo8(bseq[col]);
                s_in[L % 3][lane] = make_int4(v.x, v.y, (int)sel, 0);
            }
            mark_read(L + 1);
            __syncwarp();
        }
        if (aborted) { release_reader(); continue; }
        // ---- offset, floor and initial state
        int O = 0;
        uint32_t fl2 = ZERO2;                              // the local zero floor (relative)
        if (REL) {
            int mx0 = INT_MIN;
            if (L * CH + lane < m) mx0 = (anch && s_in[L % 3][lane].x < BIAS / 2) ? INT_MIN : s_in[L % 3][lane].x;
            mx0 = __reduce_max_sync(FULL, mx0);
            const int border = anch ? (band == 0 ? BIAS : INT_MIN) : 0;
            const int base = max(mx0, border);
            // nothing finite yet (anchored, all inputs minus infinity): any offset
            // works, the first finite input re-centres it
            O = (base == INT_MIN) ? 0 : base - REL_TOP;
            const int z = anch ? REL_FLOOR : to_rel(0, O, false);
            fl2 = p16(z, z);
            // the chunk enters shared memory in relative form
            const int4 c = s_in[L % 3][lane];
            s_in[L % 3][lane] = make_int4(to_rel(c.x, O, anch), to_rel(c.y, O, anch), c.z, 0);
            __syncwarp();
        }
        const int hb = REL ? (anch ? REL_FLOOR : to_rel(0, O, false)) : 0;
        const int eb = REL ? (anch ? REL_FLOOR : to_rel(-go, O, false)) : -go;
        uint32_t Hl[RPT], E[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) { Hl[k] = p16(hb, hb); E[k] = p16(eb, eb); }
        // Selectors reach a lane from the one above it, so cells left of the
        // band's first column start from this one: any valid selector (sign
        // extension included) keeps their scores in the profile's range.
        uint32_t Hlast = p16(hb, hb), Flast = p16(eb, eb), sellast = SEL_NEUTRAL;
        uint32_t updiag = p16(hb, hb);
        if (REL && anch && band == 0 && lane == 0) updiag = p16(BIAS - O, REL_FLOOR);
        const int binit = anch ? target - 1 : 0;
        int best_lo = binit, bk_lo = RPT, bc_lo = -1, best_hi = binit, bk_hi = RPT, bc_hi = -1;
        auto thr_of = [&](int b) -> int {
            const long long t = (long long)max(b, binit + 1) - O;
            return (int)(t > 32767 ? 32767 : (t < -32768 ? -32768 : t));
        };
        // Detection threshold minus one per half (saturating): a step whose
        // running maximum exceeds it may hold a new best, ties included.  The
        // test is a per-half max and one compare; the DPX max-with-predicates
        // form produced missed maxima in this kernel under ptxas -O2 and above.
        auto thr_minus1 = [&](int bl, int bh) -> uint32_t {
            const int tl = REL ? thr_of(bl) : max(bl, 1), th = REL ? thr_of(bh) : max(bh, 1);
            return p16(max(tl - 1, -32768), max(th - 1, -32768));
        };
        uint32_t thr1 = thr_minus1(best_lo, best_hi);
        int published = 0;
        unsigned tiles = 0, pruned = 0;
        // row record of this band's bottom row (running maximum over chunks)
        // (its row pointer and running maximum live in shared memory rather than
        // in registers across the step loop, whose register budget they would
        // otherwise take)
        if (lane == 0) { s_grun[wid] = INT_MIN; s_grow[wid] = rec_row(pr, band); }
        __syncwarp();
        // Anchored with the forward record: any path through a cell of this band
        // that reaches the start crosses a recorded forward row r at or above the
        // band (or starts below it), so what it gains beyond the band's frontier
        // is at most max_sub per row from the frontier up to r, plus the largest
        // forward H of row r left of the cell's column (plus the slack of the
        // split cell).  Row 0 of the forward matrix is all zero.
        // The same bound for the next band decides which output chunks are
        // useful to it.  Both record rows' written ranges are read once.
        const GinRow gin_own = anch ? gin_for_band(pr, P, band, R) : GinRow{};
        const GinRow gin_nx = (anch && dyn && band + 1 < pr.nbands) ? gin_for_band(pr, P, band + 1, R) : GinRow{};
        unsigned long long cells = 0;
        const int rows_lo = max(0, min(RPT, n - rb_lo)), rows_hi = max(0, min(RPT, n - rb_hi));
        int O_even = O, O_odd = O;                         // offset used in each block (by parity)

        bool first_pub = false;
        int last_useful = -1, last_flushed = -1, ring_first = 0;
        int best_seen = 0;
        for (int q = L; q < nblk && !aborted; ++q) {
            const int buf = q % 3;
            // loads whose results are needed only later in the block, issued first
            // so that their latency overlaps the flag probe and the block's work:
            // the record entries for this block and for the chunk flushed at its
            // end, and the word that ends the search
            const int pm_own = gin_own.at(pr.gin_j0 - max(1, q * CH - 62));
            const int pm_nx = gin_nx.at(pr.gin_j0 - max(1, (q - 2) * CH - 62));
            const int stop_seen = (anch && stop && lane == 0) ? ld_volatile(stop) : INT_MAX;
            // local mode prunes against the running best read one block earlier
            // (the best only grows, so an older value prunes less, never wrongly)
            const int best_used = best_seen;
            if (!anch && lane == 0) best_seen = ld_volatile(pr.best);
            const bool has_next = (q + 1) < nch;
            int nst = 0;
            int2 nv = make_int2(DEAD_H, DEAD_F);
            uint32_t nsel = 0;
            const int ncol = (q + 1) * CH + lane;
            // Chunk q + 1: from the ring, test now; from the boundary row, issue the
            // word loads now and test their tags after the block's steps, so the
            // load latency overlaps the steps.
            unsigned long long wnext = 0;
            int cnext = 0;
            const bool from_bus = has_next && !pred_in && q + 1 >= pfirst;
            if (has_next && ncol < m) {
                cnext = bseq[ncol];
                if (from_bus) wnext = ld_relaxed_u64(&busw[ncol]);
            }
            nst = 2;
            if (has_next && !from_bus) {
                int2 v;
                nst = in_status(q + 1, v);
                if (nst != 2) {
                    if (ncol < m && nst == 1) nv = v;
                    mark_read(q + 2);
                }
            }
            // ---- relative mode: re-centre the offset on the window's largest value
            // (the first block keeps the offset chosen with its chunk, which is
            // already relative)
            if (REL && q > L) {
                uint32_t m2 = Hlast;
#pragma unroll
                for (int k = 0; k < RPT; ++k) m2 = vmax16(m2, Hl[k]);
                m2 = vmax16(m2, updiag);
                int mx = max(lo16(m2), hi16(m2));
                if (q < nch) {
                    // chunk q arrived in absolute form at the end of the last block
                    const int v = s_in[buf][lane].x;
                    if (!(anch && v < BIAS / 2)) {
                        const long long r = (long long)v - O;
                        mx = max(mx, (int)(r > (1 << 30) ? (1 << 30) : (r < -(1 << 30) ? -(1 << 30) : r)));
                    }
                }
                mx = __reduce_max_sync(FULL, mx);
                // Re-centre so the largest value sits at REL_TOP.  Every true value of
                // the window lies within the window spread of that maximum, so it
                // stays above FLOOR after the shift; whatever falls below FLOOR was a
                // sentinel (skipped or minus infinity) and stays FLOOR, a value no
                // larger than the cell's true one.
                const int d = (mx > REL_FLOOR + 4096) ? mx - REL_TOP : 0;
                if (d != 0) {
                    O += d;
                    if (d >= REL_TOP - REL_FLOOR) {
                        // everything held was a sentinel: all of it is FLOOR now
#pragma unroll
                        for (int k = 0; k < RPT; ++k) { Hl[k] = NEG2; E[k] = NEG2; }
                        Hlast = NEG2; Flast = NEG2; updiag = NEG2;
                    } else {
                        const int lf = max(REL_FLOOR + d, -32768);   // at most FLOOR when d < 0
                        const uint32_t lift = p16(lf, lf), md = p16(-d, -d);
                        // x - d, never below FLOOR and never wrapping
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            Hl[k] = __viaddmax_s16x2(vmax16(Hl[k], lift), md, NEG2);
                            E[k] = __viaddmax_s16x2(vmax16(E[k], lift), md, NEG2);
                        }
                        Hlast = __viaddmax_s16x2(vmax16(Hlast, lift), md, NEG2);
                        Flast = __viaddmax_s16x2(vmax16(Flast, lift), md, NEG2);
                        updiag = __viaddmax_s16x2(vmax16(updiag, lift), md, NEG2);
                    }
                    const int z = anch ? REL_FLOOR : to_rel(0, O, false);
                    fl2 = p16(z, z);
                    thr1 = thr_minus1(best_lo, best_hi);
                }
                if (q < nch) {
                    const int4 c = s_in[buf][lane];
                    s_in[buf][lane] = make_int4(to_rel(c.x, O, anch), to_rel(c.y, O, anch), c.z, 0);
                }
                __syncwarp();
            }
            if (q & 1) O_odd = O; else O_even = O;
            bool skip = false;
            if (P.prune) {
                int pthr = target;
                if (!anch) pthr = __shfl_sync(FULL, best_used, 0);
                uint32_t mx2 = Hlast;
#pragma unroll
                for (int k = 0; k < RPT; ++k) mx2 = REL ? vmax16(mx2, Hl[k]) : __vimax_s16x2_relu(mx2, Hl[k]);
                mx2 = REL ? vmax16(mx2, updiag) : __vimax_s16x2_relu(mx2, updiag);
                int mx = max(lo16(mx2), hi16(mx2));
                if (q < nch) mx = max(mx, s_in[buf][lane].x);
                mx = __reduce_max_sync(FULL, mx);
                long long mxa = (long long)mx + O;
                if (!anch) mxa = max(mxa, 0LL);                // a local path may start afresh
                const int jmin = max(0, q * CH - 2 * CH);
                const long long rem = (long long)min(rows_left, m - jmin) + 1;
                skip = mxa + (long long)P.max_sub * rem < (long long)pthr;
                if (!skip && gin_own.valid)
                    skip = mxa + gin_own.gain + pm_own < (long long)pthr;
            }
            ++tiles;
            const bool ramp = (q * CH < 2 * CH) || (q * CH + CH - 1 >= m);
            if (!skip) {
                int jl = max(0, q * CH - lane), jh = min(m, q * CH + CH - lane);
                if (jh > jl) cells += (unsigned long long)(jh - jl) * (unsigned)rows_lo;
                jl = max(0, q * CH - lane - 32); jh = min(m, q * CH + CH - lane - 32);
                if (jh > jl) cells += (unsigned long long)(jh - jl) * (unsigned)rows_hi;
            }
            if (skip) {
                ++pruned;
                const int dh = REL ? (anch ? REL_FLOOR : to_rel(0, O, false)) : 0;
                const int de = REL ? (anch ? REL_FLOOR : to_rel(-go, O, false)) : -go;
#pragma unroll
                for (int k = 0; k < RPT; ++k) { Hl[k] = p16(dh, dh); E[k] = p16(de, de); }
                Hlast = p16(dh, dh);
                Flast = p16(de, de);
                // selectors of the columns each half reaches at the end of the block
                const uint32_t s_lo = (q < nch) ? (uint32_t)s_in[buf][31 - lane].z : sel_lo8(0);
                const uint32_t s_hi = (q > L && q - 1 < nch) ? (uint32_t)s_in[(q + 2) % 3][31 - lane].z : sel_lo8(0);
                sellast = s_lo | ((s_hi + 0x44u) << 8);
                updiag = (lane == 0 && q < nch) ? p16(s_in[buf][31].x, dh) : p16(dh, dh);
                const int oc = q * CH - 63 + lane;
                if (oc >= 0 && oc < m) s_out[oc & 63] = p16(dh, de);
            } else if (!ramp) {
                // every lane's two columns are inside the matrix: no validity checks
#pragma unroll 1
                for (int u = 0; u < CH; ++u) {
                    const int s = q * CH + u;
                    const int4 in = s_in[buf][u];
                    const uint32_t rH = __shfl_sync(FULL, Hlast, src_lane);
                    const uint32_t rF = __shfl_sync(FULL, Flast, src_lane);
                    const uint32_t rS = __shfl_sync(FULL, sellast, src_lane);
                    const uint32_t upH = perm(rH, lane ? rH : (uint32_t)in.x, pk_in);
                    const uint32_t upF = perm(rF, lane ? rF : (uint32_t)in.y, pk_in);
                    const uint32_t sel = lane ? rS : (perm((uint32_t)in.z, rS, 0x0040u) + 0x4400u);
                    uint32_t diag = updiag;
                    updiag = upH;
                    uint32_t hgo = __viaddmax_s16x2(upH, go2, NEG2);       // H(i-1, j) - go
                    uint32_t F = upF;
#pragma unroll
                    for (int k = 0; k < RPT; ++k) {
                        const uint32_t sc = perm(plo[k], phi[k], sel);
                        F = __viaddmax_s16x2(F, ge2, hgo);                     // F(i, j)
                        const uint32_t t = __viaddmax_s16x2(diag, sc, E[k]);   // max(diag + s, E)
                        const uint32_t h = REL ? __vimax3_s16x2(t, F, fl2)     // H(i, j)
                                               : __vimax3_s16x2_relu(t, F, ZERO2);
                        diag = Hl[k];
                        Hl[k] = h;
                        hgo = __viaddmax_s16x2(h, go2, NEG2);
                        E[k] = __viaddmax_s16x2(E[k], ge2, hgo);               // E(i, j+1)
                    }
                    Hlast = Hl[RPT - 1];
                    Flast = F;
                    const uint32_t smax = rows_max<RPT>(Hl, thr1);
                    if (smax != thr1) {
                        const bool pl = lo16(smax) > lo16(thr1), ph = hi16(smax) > hi16(thr1);
                        const int jlo = s - lane, jhi = s - lane - 32;
                        const int sl = lo16(smax) + O, sh = hi16(smax) + O;
                        if (pl) {
                            int kf = RPT;
#pragma unroll
                            for (int k = RPT - 1; k >= 0; --k) if (lo16(Hl[k]) + O == sl) kf = k;
                            if (sl > best_lo || (!transposed && kf < bk_lo)) { best_lo = sl; bk_lo = kf; bc_lo = jlo; }
                        }
                        if (ph) {
                            int kf = RPT;
#pragma unroll
                            for (int k = RPT - 1; k >= 0; --k) if (hi16(Hl[k]) + O == sh) kf = k;
                            if (sh > best_hi || (!transposed && kf < bk_hi)) { best_hi = sh; bk_hi = kf; bc_hi = jhi; }
                        }
                        thr1 = thr_minus1(best_lo, best_hi);
                        if (!REL && max(best_lo, best_hi) >= guard && pr.ovf) atomicExch(pr.ovf, 1);
                    }
                    if (lane == 31) s_out[(s - 63) & 63] = perm(Hlast, Flast, 0x7632u);
                    sellast = sel;
                }
            } else {
#pragma unroll 1
                for (int u = 0; u < CH; ++u) {
                    const int s = q * CH + u;
                    const int4 in = s_in[buf][u];
                    const uint32_t rH = __shfl_sync(FULL, Hlast, src_lane);
                    const uint32_t rF = __shfl_sync(FULL, Flast, src_lane);
                    const uint32_t rS = __shfl_sync(FULL, sellast, src_lane);
                    uint32_t upH = rH, upF = rF, sel = rS;
                    if (lane == 0) {
                        upH = perm(rH, (uint32_t)in.x, 0x1054u);
                        upF = perm(rF, (uint32_t)in.y, 0x1054u);
                        // past the last input chunk the low half is outside the matrix
                        // (and merged back); mask so stale shared memory cannot reach the
                        // high half's selector
                        sel = ((uint32_t)in.z & 0xffu) | (((rS & 0xffu) + 0x44u) << 8);
                    }
                    uint32_t diag = updiag;
                    updiag = upH;
                    const int jlo = s - lane, jhi = s - lane - 32;
                    const bool vlo = (unsigned)jlo < (unsigned)m, vhi = (unsigned)jhi < (unsigned)m;
                    if (vlo || vhi) {
                        const bool partial = ramp && !(vlo && vhi);
                        // partial steps keep the half whose column is outside the matrix
                        const uint32_t ks = vlo ? 0x7610u : 0x3254u;
                        const uint32_t oFlast = Flast;
                        uint32_t hgo = __viaddmax_s16x2(upH, go2, NEG2);   // H(i-1, j) - go
                        uint32_t F = upF;
                        uint32_t smax;
                        if (!partial) {
#pragma unroll
                            for (int k = 0; k < RPT; ++k) {
                                const uint32_t sc = perm(plo[k], phi[k], sel);
                                F = __viaddmax_s16x2(F, ge2, hgo);                     // F(i, j)
                                const uint32_t t = __viaddmax_s16x2(diag, sc, E[k]);   // max(diag + s, E)
                                const uint32_t h = REL ? __vimax3_s16x2(t, F, fl2)     // H(i, j)
                                                       : __vimax3_s16x2_relu(t, F, ZERO2);
                                diag = Hl[k];
                                Hl[k] = h;
                                hgo = __viaddmax_s16x2(h, go2, NEG2);
                                E[k] = __viaddmax_s16x2(E[k], ge2, hgo);               // E(i, j+1)
                            }
                            smax = rows_max<RPT>(Hl, thr1);
                            Hlast = Hl[RPT - 1];
                            Flast = F;
                        } else {
#pragma unroll
                            for (int k = 0; k < RPT; ++k) {
                                const uint32_t sc = perm(plo[k], phi[k], sel);
                                F = __viaddmax_s16x2(F, ge2, hgo);
                                const uint32_t t = __viaddmax_s16x2(diag, sc, E[k]);
                                const uint32_t h = REL ? __vimax3_s16x2(t, F, fl2)
                                                       : __vimax3_s16x2_relu(t, F, ZERO2);
                                diag = Hl[k];
                                Hl[k] = perm(h, Hl[k], ks);
                                hgo = __viaddmax_s16x2(h, go2, NEG2);
                                E[k] = perm(__viaddmax_s16x2(E[k], ge2, hgo), E[k], ks);
                            }
                            // the half outside the matrix keeps older values: it takes thr1
                            smax = perm(rows_max<RPT>(Hl, thr1), thr1, ks);
                            Hlast = Hl[RPT - 1];
                            Flast = perm(F, oFlast, ks);
                        }
                        if (smax != thr1) {
                            const bool pl = lo16(smax) > lo16(thr1), ph = hi16(smax) > hi16(thr1);
                            const int sl = lo16(smax) + O, sh = hi16(smax) + O;
                            if (pl && vlo) {
                                int kf = RPT;
#pragma unroll
                                for (int k = RPT - 1; k >= 0; --k) if (lo16(Hl[k]) + O == sl) kf = k;
                                if (sl > best_lo || (!transposed && kf < bk_lo)) { best_lo = sl; bk_lo = kf; bc_lo = jlo; }
                            }
                            if (ph && vhi) {
                                int kf = RPT;
#pragma unroll
                                for (int k = RPT - 1; k >= 0; --k) if (hi16(Hl[k]) + O == sh) kf = k;
                                if (sh > best_hi || (!transposed && kf < bk_hi)) { best_hi = sh; bk_hi = kf; bc_hi = jhi; }
                            }
                            thr1 = thr_minus1(best_lo, best_hi);
                            if (!REL && max(best_lo, best_hi) >= guard && pr.ovf) atomicExch(pr.ovf, 1);
                        }
                        if (lane == 31 && vhi) s_out[jhi & 63] = perm(Hlast, Flast, 0x7632u);
                    }
                    sellast = sel;
                }
            }
            if (has_next) {
                if (from_bus) {
                    const bool ok = ncol >= m || (BW::tag_of(wnext) >> 1) == want_tag;
                    if (__all_sync(FULL, ok)) {
                        nst = __shfl_sync(FULL, (int)(BW::tag_of(wnext) & 1u), 0);
                        if (nst == 1 && ncol < m) nv = make_int2(BW::h(wnext), BW::f(wnext));
                    }
                }
                if (nst == 2) {
                    int2 v;
                    const int st = wait_status(q + 1, v);
                    if (st < 0) { aborted = true; break; }
                    if (ncol < m && st == 1) nv = v;
                    mark_read(q + 2);
                }
                if (ncol < m) nsel = sel_lo8((uint32_t)cnext);
                s_in[(q + 1) % 3][lane] = make_int4(nv.x, nv.y, (int)nsel, 0);
            }
            __syncwarp();
            if (q >= L + 2) {
                const int c = q - 2;
                const int col = c * CH + lane;
                int rec = INT_MIN;
                int2 outv = make_int2(DEAD_H, DEAD_F);
                if (col < m) {
                    // column col was written at step col + 63, in block (col + 63) / 32
                    const uint32_t v = s_out[col & 63];
                    int oh = lo16(v), of = hi16(v);
                    if (REL) {
                        const int Ou = (((col + 63) >> 5) & 1) ? O_odd : O_even;
                        oh = (oh <= REL_FLOOR) ? DEAD_H : oh + Ou;
                        of = (of <= REL_FLOOR) ? DEAD_F : of + Ou;
                    }
                    outv = make_int2(oh, of);
                    rec = oh;
                }
                int cmax = 0;
                int32_t *const grow = s_grow[wid];
                if (grow || dyn) cmax = __reduce_max_sync(FULL, rec);
                // can a value of this chunk still reach the target from the next band?
                bool useful = true;
                if (dyn && band + 1 < pr.nbands) {
                    const long long nrem = (long long)min(n - (band + 1) * R, m - max(0, c * CH - 2 * CH)) + 1;
                    long long gain = (long long)P.max_sub * nrem;
                    if (gin_nx.valid) gain = min(gain, gin_nx.gain + pm_nx);
                    useful = (long long)cmax + gain >= (long long)target;
                }
                if (succ_in) {
                    // The ring carries chunks from the first useful one on (the
                    // reader starts there); a slot is reused once the reader has
                    // moved GK chunks past it.
                    if (first_pub || useful) {
                        if (!first_pub) ring_first = c;
                        int ok = 1;
                        // slot c % GK last held chunk c - GK: wait until the reader is past it
                        if (lane == 0 && c - GK >= ring_first && c - GK >= vneed[wid + 1]) {
                            const unsigned long long t0 = globaltimer();
                            while (c - GK >= vneed[wid + 1]) {
                                __nanosleep(20);
                                if (ld_volatile(P.err)) { ok = 0; break; }
                                if (globaltimer() - t0 > P.timeout_ns) { atomicCAS(P.err, 0, DEV_ETIMEOUT); ok = 0; break; }
                            }
                            __threadfence_block();
                        }
                        if (!__shfl_sync(FULL, ok, 0)) { aborted = true; break; }
                        s_ring[GROUP ? wid : 0][GROUP ? c % GK : 0][lane] = outv;
                        __syncwarp();
                        if (lane == 0 && band != P.fault_band) {
                            __threadfence_block();
                            ((volatile int *)s_tag[GROUP ? wid : 0])[GROUP ? c % GK : 0] = 2 * c + (useful ? 1 : 0);
                            if (dyn && useful && !first_pub) vspx[wid] = c;
                        }
                    }
                } else {
                    // one self-validating word per column (a band that never
                    // publishes, for testing, writes nothing)
                    if (col < m && band != P.fault_band)
                        st_relaxed_u64(&busw[col], BW::pack(outv.x, outv.y, BW::tag(band, useful)));
                    __syncwarp();
                    if (lane == 0 && band != P.fault_band && dyn && useful && !first_pub)
                        st_release(&pr.span[band].x, c);
                }
                // the record entry goes out after the release, which then does not
                // wait for it
                if (grow && lane == 0) {
                    const int g = max(s_grun[wid], cmax);
                    s_grun[wid] = g;
                    grow[c] = g;
                }
                if (useful) { first_pub = true; last_useful = c; }
                if (ANCH) last_flushed = c;
            }
            if (!anch) {
                const int wb = __reduce_max_sync(FULL, max(best_lo, best_hi));
                if (lane == 0 && wb > published) { atomicMax(pr.best, wb); published = wb; }
            } else if (stop != nullptr) {
                if (__shfl_sync(FULL, stop_seen < band ? 1 : 0, 0)) aborted = true;
            }
            if (dyn && skip && q < nch && !aborted) {
                // A pruned block leaves only dead state behind (lane 0 keeps the
                // diagonal input of chunk q); the band is done when nothing useful
                // arrives from chunk q on.  Row 0 holds nothing but the anchor.
                int y = -1;
                if (pred_in || pred_last) {
                    if (lane == 0) y = pred_in ? vspy[wid - 1] : ld_acquire(pred_last);
                    y = __shfl_sync(FULL, y, 0);
                }
                if (y != SPAN_UNPUB && q > y) break;
            }
        }
        release_reader();
        if (aborted) continue;
        if (dyn && lane == 0) {
            if (succ_in) {
                __threadfence_block();
                if (!first_pub) vspx[wid] = SPAN_NONE;
                vspy[wid] = last_useful;
            } else {
                if (!first_pub) st_release(&pr.span[band].x, SPAN_NONE);
                st_release(&pr.span[band].y, last_useful);
            }
        }
        if (lane == 0) {
            int32_t *const grow = s_grow[wid];
            // a local band flushes every chunk; an anchored one may stop early
            if (grow) { grow[nch] = L; grow[nch + 1] = ANCH ? last_flushed : nch - 1; }
        }
        // band result over the 64 virtual lanes (low halves hold the smaller rows)
        int vs = best_lo, vr = rb_lo + (bk_lo < RPT ? bk_lo : 0) + 1, vc = bc_lo + 1, ok = best_lo > binit;
        {
            const int hs = best_hi, hr = rb_hi + (bk_hi < RPT ? bk_hi : 0) + 1, hc = bc_hi + 1, hok = best_hi > binit;
            bool take;
            if (!hok) take = false;
            else if (!ok) take = true;
            else if (hs != vs) take = hs > vs;
            else if (!transposed) take = (hr < vr) || (hr == vr && hc < vc);
            else take = (hc < vc) || (hc == vc && hr < vr);
            if (take) { vs = hs; vr = hr; vc = hc; ok = hok; }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            const int os = __shfl_xor_sync(FULL, vs, off);
            const int orr = __shfl_xor_sync(FULL, vr, off);
            const int oc = __shfl_xor_sync(FULL, vc, off);
            const int ook = __shfl_xor_sync(FULL, ok, off);
            bool take;
            if (!ook) take = false;
            else if (!ok) take = true;
            else if (os != vs) take = os > vs;
            else if (!transposed) take = (orr < vr) || (orr == vr && oc < vc);
            else take = (oc < vc) || (oc == vc && orr < vr);
            if (take) { vs = os; vr = orr; vc = oc; ok = ook; }
        }
        for (int off = 16; off >= 1; off >>= 1) cells += __shfl_xor_sync(FULL, cells, off);
        if (lane == 0) {
            pr.band_res[band] = make_int4(vs, vr, vc, ok);
            if (anch && ok && vs == target) atomicMin(pr.stop_band, band);
            atomicAdd(&P.stats[1], (unsigned long long)tiles);
            atomicAdd(&P.stats[2], (unsigned long long)pruned);
            atomicAdd(&P.stats[0], cells);
        }
    }
}

// warps per CTA of the one-CTA-per-SM layout: what the registers of each
// band height allow on one SM
static constexpr int wide_warps(int rpt) { return rpt == 16 ? 12 : rpt == 8 ? 16 : 20; }

int fwd16_cta_warps(int rpt, bool wide) { return wide ? wide_warps(rpt) : 4; }

template <int RPT, bool REL, bool ANCH, int NW>
static cudaError_t launch16(const FwdParams &p, int ctas, cudaStream_t s)
{
    fwd16_kernel<RPT, REL, ANCH, NW><<<ctas, NW * 32, 0, s>>>(p);
    return cudaGetLastError();
}

template <int RPT>
static cudaError_t launch16_rpt(const FwdParams &p, bool rel, bool anch, bool wide, int ctas, cudaStream_t s)
{
    if (!rel) return anch ? cudaErrorInvalidValue : launch16<RPT, false, false, 4>(p, ctas, s);
    if (anch) return launch16<RPT, true, true, 4>(p, ctas, s);
    return wide ? launch16<RPT, true, false, wide_warps(RPT)>(p, ctas, s) : launch16<RPT, true, false, 4>(p, ctas, s);
}

template <int RPT>
static cudaError_t occupancy16_rpt(bool rel, bool anch, bool wide, int *n)
{
    if (!rel) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fwd16_kernel<RPT, false, false, 4>, 128, 0);
    if (anch) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fwd16_kernel<RPT, true, true, 4>, 128, 0);
    return wide ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fwd16_kernel<RPT, true, false, wide_warps(RPT)>,
                                                                wide_warps(RPT) * 32, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fwd16_kernel<RPT, true, false, 4>, 128, 0);
}

bool fwd16_rpt_supported(int rpt) { return rpt == 4 || rpt == 8 || rpt == 16; }

cudaError_t fwd16_launch(const FwdParams &p, int rpt, bool rel, bool anch, bool wide, int ctas, cudaStream_t s)
{
    switch (rpt) {
    case 4: return launch16_rpt<4>(p, rel, anch, wide, ctas, s);
    case 8: return launch16_rpt<8>(p, rel, anch, wide, ctas, s);
    case 16: return launch16_rpt<16>(p, rel, anch, wide, ctas, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fwd16_occupancy(int rpt, bool rel, bool anch, bool wide, int *n)
{
    switch (rpt) {
    case 4: return occupancy16_rpt<4>(rel, anch, wide, n);
    case 8: return occupancy16_rpt<8>(rel, anch, wide, n);
    case 16: return occupancy16_rpt<16>(rel, anch, wide, n);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace swgb
