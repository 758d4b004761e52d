// fwd.cu -- forward wavefront pass over row bands (sm_103a).
//
// Computes the affine-gap Smith-Waterman matrix (Gotoh H/E/F) band by band and
// returns, per band, the best cell under the library's tie rule.  This is the
// paper's "solving" phase (Sec. 2, wavefront paragraph): cells of one
// anti-diagonal are computed at the same time, and only boundary rows are kept
// in memory, so device memory is linear in the sequence lengths.  The same
// kernel, in FWD_ANCHORED mode, is the start-point pass (Sec. 2, start-point
// paragraph): values are offset by BIAS so that the zero floor of the DPX
// "relu" forms acts as minus infinity, the borders are minus infinity except
// the origin, and the cell sought is the first one reaching the known score.
//
// GB300 design (not the paper's two-phase cell blocks):
//   * one warp owns a band of 32*RPT rows; lane t holds RPT consecutive rows in
//     registers and processes column j at step j + t (a skewed anti-diagonal);
//   * the vertical dependency (H and F of the lane above) moves one lane down
//     per step with __shfl_up_sync, together with the column's score selector;
//   * lane 0 reads the row above the band from a 32-column shared-memory chunk
//     that the warp fetched coalesced from the boundary row in HBM (8 bytes per
//     column: H and F); lane 31's bottom row goes to a shared ring and is written
//     back in place, coalesced, one chunk behind;
//   * bands are taken from an ordered ticket counter by a persistent grid, so a
//     band only ever waits (bounded, acquire/release flag per chunk) on a band
//     that a running warp already holds: no deadlock without co-residency;
//   * exact pruning (Sec. 2, pruning paragraph): a 32-step block is skipped when
//     the largest H on its entry edges plus max_sub times the remaining length
//     is strictly below the running best; skipped cells are set to values no
//     larger than their true ones, which leaves every cell that reaches the
//     final best, and the tie rule, unchanged.
//   * per cell: one prmt (substitution score), four DPX/int max ops, two adds.
#include "common.cuh"
#include "kernels.h"

namespace swgb {

template <int RPT, bool PROF2>
__global__ void __launch_bounds__(128) fwd_kernel(const FwdParams P)
{
    __shared__ int4 s_in_all[4][2][CH];
    __shared__ int2 s_out_all[4][2 * CH];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    int4 (*s_in)[CH] = s_in_all[wid];
    int2 *s_out = s_out_all[wid];
    const int go = P.go, ge = P.ge;
    constexpr int R = 32 * RPT;

    for (;;) {
        int tk = 0, stop_now = 0;
        if (lane == 0) {
            tk = atomicAdd(P.ticket_ctr, 1);
            stop_now = ld_volatile(P.err);
        }
        tk = __shfl_sync(FULL, tk, 0);
        stop_now = __shfl_sync(FULL, stop_now, 0);   // warp-uniform decisions only
        if (tk >= P.ntickets || stop_now) return;
        const int2 tb = P.tickets[tk];
        const FwdProblem &pr = P.probs[tb.x];
        const int band = tb.y;
        const int n = pr.n, m = pr.m;
        const bool anch = pr.mode == FWD_ANCHORED;
        const bool transposed = pr.transposed != 0;
        const uint8_t *__restrict__ bseq = pr.b;
        int2 *__restrict__ bus = pr.bus;
        int *__restrict__ flags = pr.flags;
        const int target = pr.target;
        int *stop = anch ? pr.stop_band : nullptr;
        const int need = band - 1;

        // ---- per-row substitution profiles
        const int rowbase = band * R + lane * RPT;   // 0-based first row of this lane
        uint32_t plo[RPT], phi[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) {
            const int r = rowbase + k;
            uint32_t lo = VIRTUAL_PROF, hi = VIRTUAL_PROF;
            if (r < n) {
                const int c = pr.a[r] & 7;
                lo = transposed ? P.prof_lo_t[c] : P.prof_lo[c];
                if (PROF2) hi = transposed ? P.prof_hi_t[c] : P.prof_hi[c];
            }
            plo[k] = lo;
            phi[k] = PROF2 ? hi : 0u;
        }
        // ---- border state (column 0): local H = 0, E = -go; anchored -inf (biased 0)
        const int EB = anch ? 0 : -go;
        const int FB = anch ? 0 : -go;
        int Hl[RPT], E[RPT];
#pragma unroll
        for (int k = 0; k < RPT; ++k) { Hl[k] = 0; E[k] = EB; }
        int Hlast = 0, Flast = FB;
        uint32_t sellast = 0;
        int updiag = (anch && band == 0 && lane == 0) ? BIAS : 0;   // H(row above, 0)
        const int binit = anch ? target - 1 : 0;
        int best = binit, bk = RPT, bc = -1;
        int published = 0;
        unsigned tiles = 0, pruned = 0;
        unsigned long long cells = 0;
        const int lane_rows = max(0, min(RPT, n - rowbase));
        bool aborted = false;

        const int nch = (m + CH - 1) / CH;
        const int nblk = nch + 1;
        const int rows_left = n - band * R;

        // ---- chunk 0 of the row above
        {
            int ok = 1;
            if (lane == 0) ok = wait_flag(&flags[0], need, P.err, stop, band, P.timeout_ns);
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) aborted = true;
            else {
                const int col = lane;
                int2 v = make_int2(0, FB);
                uint32_t sel = 0;
                if (col < m) { v = bus[col]; sel = code_selector(bseq[col]); }
                s_in[0][lane] = make_int4(v.x, v.y, (int)sel, 0);
            }
            __syncwarp();
        }

        for (int q = 0; q < nblk && !aborted; ++q) {
            const int buf = q & 1;
            // (a) opportunistic prefetch of chunk q+1
            const bool has_next = (q + 1) < nch;
            int ready = 0;
            int2 nv = make_int2(0, FB);
            uint32_t nsel = 0;
            const int ncol = (q + 1) * CH + lane;
            if (has_next) {
                if (lane == 0) ready = ld_acquire(&flags[q + 1]) >= need;
                ready = __shfl_sync(FULL, ready, 0);
                if (ready && ncol < m) { nv = bus[ncol]; nsel = code_selector(bseq[ncol]); }
            }
            // (b) pruning bound for this 32-step block
            bool skip = false;
            if (P.prune) {
                int pthr = target;
                if (!anch) {
                    if (lane == 0) pthr = ld_volatile(pr.best);
                    pthr = __shfl_sync(FULL, pthr, 0);
                }
                int mx = 0;
#pragma unroll
                for (int k = 0; k < RPT; ++k) mx = max(mx, Hl[k]);
                mx = max(mx, max(Hlast, updiag));
                if (q < nch) mx = max(mx, s_in[buf][lane].x);
                mx = __reduce_max_sync(FULL, mx);
                const int jmin = max(0, q * CH - CH);
                const long long rem = (long long)min(rows_left, m - jmin) + 1;
                const long long bound = (long long)mx + (long long)P.max_sub * rem;
                skip = bound < (long long)pthr;
            }
            ++tiles;
            if (!skip) {
                // cells this lane really computes in this block (columns in range x rows < n)
                const int jlo = max(0, q * CH - lane), jhi = min(m, q * CH + CH - lane);
                if (jhi > jlo) cells += (unsigned long long)(jhi - jlo) * (unsigned)lane_rows;
            }
            if (skip) {
                ++pruned;
#pragma unroll
                for (int k = 0; k < RPT; ++k) { Hl[k] = 0; E[k] = EB; }
                Hlast = 0;
                Flast = FB;
                if (q < nch) {
                    sellast = (uint32_t)s_in[buf][31 - lane].z;
                    updiag = (lane == 0) ? s_in[buf][31].x : 0;
                } else {
                    updiag = 0;
                }
                const int oc = q * CH - 31 + lane;
                if (oc >= 0 && oc < m) s_out[oc & 63] = make_int2(0, FB);
            } else {
#pragma unroll 1
                for (int u = 0; u < CH; ++u) {
                    const int4 in = s_in[buf][u];
                    const int rH = __shfl_up_sync(FULL, Hlast, 1);
                    const int rF = __shfl_up_sync(FULL, Flast, 1);
                    const uint32_t rS = __shfl_up_sync(FULL, sellast, 1);
                    const int upH = lane ? rH : in.x;
                    const int upF = lane ? rF : in.y;
                    const uint32_t sel = lane ? rS : (uint32_t)in.z;
                    int diag = updiag;
                    updiag = upH;
                    sellast = sel;
                    const int j = q * CH + u - lane;
                    if ((unsigned)j < (unsigned)m) {
                        int hgo = upH - go;          // H(i-1, j) - go
                        int F = upF;                 // F(i-1, j)
                        int smax = 0;
#pragma unroll
                        for (int k = 0; k < RPT; ++k) {
                            const int s = sub_lookup(plo[k], phi[k], sel);
                            F = addmax(F, -ge, hgo);                 // F(i, j)
                            const int t = addmax0(diag, s, E[k]);    // max(diag + s, E(i, j), 0)
                            const int h = max(t, F);                 // H(i, j)
                            diag = Hl[k];                            // H(i, j-1): diag of row i+1
                            Hl[k] = h;
                            hgo = h - go;
                            E[k] = addmax(E[k], -ge, hgo);           // E(i, j+1)
                            smax = max(smax, h);
                        }
                        Hlast = Hl[RPT - 1];
                        Flast = F;
                        if (smax >= best && smax > binit) {
                            int kf = RPT;
#pragma unroll
                            for (int k = RPT - 1; k >= 0; --k)
                                if (Hl[k] == smax) kf = k;
                            if (smax > best || (!transposed && kf < bk)) {
                                best = smax; bk = kf; bc = j;
                            }
                        }
                        if (lane == 31) s_out[j & 63] = make_int2(Hlast, Flast);
                    }
                }
            }
            // (c) complete the prefetch of chunk q+1
            if (has_next) {
                if (!ready) {
                    int ok = 1;
                    if (lane == 0) ok = wait_flag(&flags[q + 1], need, P.err, stop, band, P.timeout_ns);
                    ok = __shfl_sync(FULL, ok, 0);
                    if (!ok) { aborted = true; break; }
                    if (ncol < m) { nv = bus[ncol]; nsel = code_selector(bseq[ncol]); }
                }
                s_in[buf ^ 1][lane] = make_int4(nv.x, nv.y, (int)nsel, 0);
            }
            // (d) write back output chunk q-1 and publish it
            __syncwarp();
            if (q >= 1) {
                const int col = (q - 1) * CH + lane;
                if (col < m) bus[col] = s_out[col & 63];
                __syncwarp();
                if (lane == 0 && band != P.fault_band) st_release(&flags[q - 1], band);
            }
            // (e) share the running best (local mode) for pruning elsewhere
            if (!anch) {
                const int wb = __reduce_max_sync(FULL, best);
                if (lane == 0 && wb > published) { atomicMax(pr.best, wb); published = wb; }
            } else if (stop != nullptr) {
                int cancel = 0;
                if (lane == 0) cancel = ld_volatile(stop) < band;
                if (__shfl_sync(FULL, cancel, 0)) aborted = true;
            }
        }
        if (aborted) continue;

        // ---- band result: best value, then first in row-major order
        //      (column-major when the problem is transposed)
        int vs = best, vr = rowbase + (bk < RPT ? bk : 0) + 1, vc = bc + 1;
        int ok = best > binit;
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

// ---------------------------------------------------------------------------
__global__ void fwd_init_kernel(FwdProblem *probs, int nprobs, int h0, int f0, int packed)
{
    const int p = blockIdx.x;
    if (p >= nprobs) return;
    FwdProblem pr = probs[p];
    // row 0: {H, F} pairs (int32 lanes) or self-validating words tagged as
    // written by band -1 (int16x2 lanes; packed 2: the anchored passes' layout)
    if (packed) {
        const unsigned long long w = packed == 2 ? BusWord<true>::pack(h0, f0, BusWord<true>::tag(-1, true))
                                                 : BusWord<false>::pack(h0, f0, BusWord<false>::tag(-1, true));
        for (int j = threadIdx.x; j < pr.m; j += blockDim.x) ((unsigned long long *)pr.bus)[j] = w;
    } else {
        for (int j = threadIdx.x; j < pr.m; j += blockDim.x) pr.bus[j] = make_int2(h0, f0);
    }
    const int nch = (pr.m + CH - 1) / CH;
    for (int c = threadIdx.x; c < nch; c += blockDim.x) pr.flags[c] = -1;
    for (int b = threadIdx.x; b < pr.nbands; b += blockDim.x) {
        pr.band_res[b] = make_int4(0, 0, 0, 0);
        if (pr.span) pr.span[b] = make_int2(SPAN_UNPUB, SPAN_UNPUB);
    }
    if (threadIdx.x == 0) {
        if (pr.best) *pr.best = 0;
        if (pr.stop_band) *pr.stop_band = 0x7fffffff;
        if (pr.ovf) *pr.ovf = 0;
    }
}

// one warp per problem: pick the best band result under the problem's tie rule
__global__ void fwd_reduce_kernel(const FwdProblem *probs, int nprobs, int4 *out)
{
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= nprobs) return;
    const FwdProblem pr = probs[p];
    const bool tr = pr.transposed != 0;
    int vs = 0, vr = 0, vc = 0, ok = 0;
    for (int b = lane; b < pr.nbands; b += 32) {
        const int4 x = pr.band_res[b];
        bool take;
        if (!x.w) take = false;
        else if (!ok) take = true;
        else if (x.x != vs) take = x.x > vs;
        else if (!tr) take = (x.y < vr) || (x.y == vr && x.z < vc);
        else take = (x.z < vc) || (x.z == vc && x.y < vr);
        if (take) { vs = x.x; vr = x.y; vc = x.z; ok = 1; }
    }
    for (int off = 16; off >= 1; off >>= 1) {
        const int os = __shfl_xor_sync(FULL, vs, off);
        const int orr = __shfl_xor_sync(FULL, vr, off);
        const int oc = __shfl_xor_sync(FULL, vc, off);
        const int ook = __shfl_xor_sync(FULL, ok, off);
        bool take;
        if (!ook) take = false;
        else if (!ok) take = true;
        else if (os != vs) take = os > vs;
        else if (!tr) take = (orr < vr) || (orr == vr && oc < vc);
        else take = (oc < vc) || (oc == vc && orr < vr);
        if (take) { vs = os; vr = orr; vc = oc; ok = ook; }
    }
    if (lane == 0) out[p] = make_int4(vs, vr, vc, ok);
}

// ---------------------------------------------------------------------------
template <int RPT, bool P2>
static cudaError_t launch_one(const FwdParams &p, int ctas, int threads, cudaStream_t s)
{
    fwd_kernel<RPT, P2><<<ctas, threads, 0, s>>>(p);
    return cudaGetLastError();
}

bool fwd_rpt_supported(int rpt) { return rpt == 8 || rpt == 16 || rpt == 24 || rpt == 32; }

cudaError_t fwd_launch(const FwdParams &p, int rpt, bool p2, int ctas, int threads, cudaStream_t s)
{
    switch (rpt) {
    case 8:  return p2 ? launch_one<8, true>(p, ctas, threads, s) : launch_one<8, false>(p, ctas, threads, s);
    case 16: return p2 ? launch_one<16, true>(p, ctas, threads, s) : launch_one<16, false>(p, ctas, threads, s);
    case 24: return p2 ? launch_one<24, true>(p, ctas, threads, s) : launch_one<24, false>(p, ctas, threads, s);
    case 32: return p2 ? launch_one<32, true>(p, ctas, threads, s) : launch_one<32, false>(p, ctas, threads, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int RPT, bool P2>
static cudaError_t occ_one(int threads, int *n)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, fwd_kernel<RPT, P2>, threads, 0);
}

cudaError_t fwd_occupancy(int rpt, bool p2, int threads, int *n)
{
    switch (rpt) {
    case 8:  return p2 ? occ_one<8, true>(threads, n) : occ_one<8, false>(threads, n);
    case 16: return p2 ? occ_one<16, true>(threads, n) : occ_one<16, false>(threads, n);
    case 24: return p2 ? occ_one<24, true>(threads, n) : occ_one<24, false>(threads, n);
    case 32: return p2 ? occ_one<32, true>(threads, n) : occ_one<32, false>(threads, n);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t fwd_init_launch(FwdProblem *probs_dev, int nprobs, const FwdProblem *, int h0, int f0, int packed,
                            cudaStream_t s)
{
    if (nprobs <= 0) return cudaSuccess;
    fwd_init_kernel<<<nprobs, 256, 0, s>>>(probs_dev, nprobs, h0, f0, packed);
    return cudaGetLastError();
}

cudaError_t fwd_reduce_launch(const FwdProblem *probs_dev, int nprobs, int4 *out, cudaStream_t s)
{
    if (nprobs <= 0) return cudaSuccess;
    const int wpb = 4;
    fwd_reduce_kernel<<<(nprobs + wpb - 1) / wpb, 32 * wpb, 0, s>>>(probs_dev, nprobs, out);
    return cudaGetLastError();
}

}  // namespace swgb
