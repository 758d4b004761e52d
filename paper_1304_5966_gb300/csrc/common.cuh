// common.cuh -- device helpers shared by the sm_103a kernels of the library.
//
// Integer max-plus helpers (DPX: VIMNMX / VIADDMNMX on Hopper and later),
// the byte permute used to look up substitution scores, acquire/release
// accessors for the inter-band progress flags, and the bounded wait that
// every inter-warp dependency goes through.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace swgb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int CH = 32;                 // columns per boundary chunk (one per lane)
constexpr int BIAS = 1 << 30;          // global-mode offset: biased 0 is -infinity
constexpr uint32_t VIRTUAL_PROF = 0x80808080u;  // -128 for rows past the end

// error codes written to the device error word (mirror sw_status)
constexpr int DEV_ETIMEOUT = 4;

// ---------------------------------------------------------------- arithmetic
// max(a + b, c)
__device__ __forceinline__ int addmax(int a, int b, int c) { return __viaddmax_s32(a, b, c); }
// max(a + b, c, 0)
__device__ __forceinline__ int addmax0(int a, int b, int c) { return __viaddmax_s32_relu(a, b, c); }
__device__ __forceinline__ int imax(int a, int b) { return max(a, b); }
__device__ __forceinline__ int imax3(int a, int b, int c) { return __vimax3_s32(a, b, c); }

// Substitution score lookup: the profile word holds s(a_row, c) for b codes
// c = 0..3 as four signed bytes (a second word holds c = 4..7).  `sel` is the
// prmt selector of the column code: byte c, then three sign-replicating copies,
// so the result is the selected byte sign-extended to 32 bits.
__device__ __forceinline__ int sub_lookup(uint32_t lo, uint32_t hi, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(lo), "r"(hi), "r"(sel));
    return (int)r;
}
__host__ __device__ __forceinline__ uint32_t code_selector(uint32_t c) {
    uint32_t s = c | 8u;
    return c | (s << 4) | (s << 8) | (s << 12);
}

// ---------------------------------------------------------------- memory
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int *p) {
    return *(const volatile int *)p;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait until *flag >= need.  Called by one lane.  Returns 1 when the
// flag is reached, 0 when the call must abandon the band: the error word is
// set (by anyone), `*cancel` exceeds `cancel_above`, or the wait ran past
// `limit_ns`, in which case this wait records DEV_ETIMEOUT in the error word.
__device__ __forceinline__ int wait_flag(const int *flag, int need, int *err,
                                         const int *cancel, int cancel_above,
                                         unsigned long long limit_ns) {
    if (ld_acquire(flag) >= need) return 1;
    unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        if (ld_acquire(flag) >= need) return 1;
        if (ld_volatile(err)) return 0;
        if (cancel && ld_volatile(cancel) < cancel_above) return 0;
        if (globaltimer() - t0 > limit_ns) {
            atomicCAS(err, 0, DEV_ETIMEOUT);
            return 0;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;      // short naps: the awaited chunk is usually microseconds away
    }
}

// Self-validating boundary-row entry (int16x2 kernel): one 64-bit word per
// column, read and written whole, so a reader that finds its predecessor's tag
// has its data.  Bits 0-31 hold H as int32; then how far F lies below H, D bits
// clamped at 2^D - 1 (exact while go - ge < 2^D: farther below, F - ge stays
// under H - go, so F no longer matters); then the tag of the band that wrote
// it, (band mod P) << 1 | useful, where P = 2^(31 - D) - 1 and the all-ones
// band field P is reserved for row 0 (only band 0 reads it).
//  * WIDE = false (D = 16, P = 32767): the local passes, whose bands write
//    every column of the row, so a reader never meets a word older than its
//    predecessor's.
//  * WIDE = true (D = 8, P = 2^23 - 1): the anchored passes, whose bands write
//    only their live range, so a column can keep a word from any earlier band.
//    Their schemes have go - ge <= 255, and a band index stays below P (at
//    least 256 rows a band and fewer than 2^31 rows), so no two bands share a
//    tag.
template <bool WIDE> struct BusWord {
    static constexpr int DBITS = WIDE ? 8 : 16;
    static constexpr unsigned DMAX = (1u << DBITS) - 1u;
    static constexpr int TSHIFT = 32 + DBITS;
    static constexpr unsigned ROW0 = (1u << (31 - DBITS)) - 1u;   // reserved band field
    __host__ __device__ static unsigned band_tag(int band) {
        return band < 0 ? ROW0 : (unsigned)band % ROW0;
    }
    __host__ __device__ static unsigned tag(int band, bool useful) { return band_tag(band) << 1 | (useful ? 1u : 0u); }
    __host__ __device__ static unsigned long long pack(int h, int f, unsigned t) {
        const long long d = (long long)h - f;
        const unsigned dd = d > (long long)DMAX ? DMAX : (unsigned)d;
        return (unsigned long long)(unsigned)h | ((unsigned long long)dd << 32) | ((unsigned long long)t << TSHIFT);
    }
    __device__ static int h(unsigned long long w) { return (int)(unsigned)(w & 0xffffffffull); }
    __device__ static int f(unsigned long long w) { return h(w) - (int)((w >> 32) & DMAX); }
    __device__ static unsigned tag_of(unsigned long long w) { return (unsigned)(w >> TSHIFT); }
};
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// Published-range words (the first and last useful chunk of a band, see the
// label and anchored passes): not yet written, and "no useful chunk".
constexpr int SPAN_UNPUB = INT_MIN;
constexpr int SPAN_NONE = INT_MAX;

// Bounded wait until *p holds a published value (not SPAN_UNPUB).  Called by
// one lane; returns 1 with the value in *out, or 0 when the error word is set
// or the wait ran past limit_ns (then it records DEV_ETIMEOUT).
// Also returns 0 (without recording anything) when `*cancel` drops below
// cancel_above.
__device__ __forceinline__ int wait_published(const int *p, int *err, unsigned long long limit_ns, int *out,
                                              const int *cancel = nullptr, int cancel_above = 0) {
    int v = ld_acquire(p);
    if (v != SPAN_UNPUB) { *out = v; return 1; }
    const unsigned long long t0 = globaltimer();
    unsigned ns = 64;
    for (;;) {
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_acquire(p);
        if (v != SPAN_UNPUB) { *out = v; return 1; }
        if (ld_volatile(err)) return 0;
        if (cancel && ld_volatile(cancel) < cancel_above) return 0;
        if (globaltimer() - t0 > limit_ns) {
            atomicCAS(err, 0, DEV_ETIMEOUT);
            return 0;
        }
    }
}

// Record row of running maxima (see FwdProblem::gout): nch entries, then the
// first and last chunk the band wrote.  Chunks before the first hold nothing
// (0: minus infinity biased, or the local zero); chunks after the last hold
// the row's final maximum.
__device__ __forceinline__ int rec_at(const int32_t *row, int nch, int c) {
    const int lo = row[nch], hi = row[nch + 1];
    if (hi < lo || c < lo) return 0;
    return row[min(c, hi)];
}

}  // namespace swgb
