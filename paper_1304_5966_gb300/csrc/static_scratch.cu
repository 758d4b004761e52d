// static_scratch.cu -- sw_score_static: the forward score pass without any
// device allocation.
//
// Some callers cannot allocate device memory when they need a score: a process
// whose device memory is entirely reserved up front by its framework's caching
// allocator, or a latency-bound pipeline that forbids cudaMalloc/cudaFree (and
// their implicit synchronisation) on its hot path.  This entry point runs the
// same forward kernel as sw_score (fwd.cu, int32 lanes, 256-row bands) but takes
// its scratch -- the boundary row, the per-chunk flags, the per-band results, the
// ticket table and the counters -- from one file-scope __device__ array of
// SWGB_STATIC_SCRATCH_BYTES.  Every GPU that loads the library holds that array
// until the process exits.  The caller passes the sequences (device memory) and
// the result struct (host memory); nothing is allocated by this file.
//
// In host code `g_static_scratch` names a host-side stand-in, not device memory,
// so the device address is looked up with cudaGetSymbolAddress once per device
// (on that device's first call) and cached.
#include <cstring>
#include <mutex>

#include "../../include/swgb.h"
#include "common.cuh"
#include "ctx.h"
#include "kernels.h"

namespace swgb {

constexpr size_t STATIC_SCRATCH_BYTES = 10u << 20;
constexpr int STATIC_RPT = 8;                       // 256-row bands
constexpr int64_t STATIC_MAX_N = 16777216;          // 65,536 bands
constexpr int64_t STATIC_MAX_M = 1048576;
// layout (byte offsets inside the array)
constexpr size_t OFF_CTR = 0;                       // 64 ints: ticket, err, best, stop, ovf, bad code
constexpr size_t OFF_STATS = 256;                   // 4 x u64
constexpr size_t OFF_DESC = 512;                    // FwdProblem
constexpr size_t OFF_RES = 1024;                    // int4
constexpr size_t OFF_TICKETS = 4096;                // 65,536 x int2
constexpr size_t OFF_BANDRES = OFF_TICKETS + 65536 * sizeof(int2);
constexpr size_t OFF_FLAGS = OFF_BANDRES + 65536 * sizeof(int4);
constexpr size_t OFF_BUS = OFF_FLAGS + (STATIC_MAX_M / 32) * sizeof(int32_t);
static_assert(OFF_BUS + STATIC_MAX_M * sizeof(int2) <= STATIC_SCRATCH_BYTES, "static scratch too small");
static_assert(sizeof(FwdProblem) <= OFF_RES - OFF_DESC, "descriptor does not fit");

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Writes the problem descriptor and ticket table and resets everything the
// forward pass expects at its initial value (the array keeps the previous call's
// contents).
__global__ void static_setup_kernel(FwdProblem desc, int nbands, int nch, int f0)
{
    unsigned char *base = g_static_scratch;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (tid == 0) {
        *(FwdProblem *)(base + OFF_DESC) = desc;
        int32_t *ctr = (int32_t *)(base + OFF_CTR);
        for (int k = 0; k < 64; ++k) ctr[k] = 0;
        ctr[3] = 0x7fffffff;                               // stop band (unused in local mode)
        unsigned long long *st = (unsigned long long *)(base + OFF_STATS);
        for (int k = 0; k < 4; ++k) st[k] = 0;
    }
    int2 *tickets = (int2 *)(base + OFF_TICKETS);
    int4 *band_res = (int4 *)(base + OFF_BANDRES);
    for (int b = tid; b < nbands; b += stride) { tickets[b] = make_int2(0, b); band_res[b] = make_int4(0, 0, 0, 0); }
    int32_t *flags = (int32_t *)(base + OFF_FLAGS);
    for (int c = tid; c < nch; c += stride) flags[c] = -1;
    int2 *bus = (int2 *)(base + OFF_BUS);
    for (int j = tid; j < desc.m; j += stride) bus[j] = make_int2(0, f0);
}

__global__ void static_check_codes_kernel(const uint8_t *p, int64_t len, int alph)
{
    int32_t *bad = (int32_t *)(g_static_scratch + OFF_CTR) + 5;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x)
        if (p[i] >= alph) { atomicExch(bad, 1); return; }
}

}  // namespace swgb

using namespace swgb;

extern "C" int sw_score_static(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                               const sw_scheme *scheme, void *stream, sw_result *out)
{
    static std::mutex mu;
    static unsigned char *dev_base[64] = {};
    if (!out) return SW_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->a_begin = out->a_end = out->b_begin = out->b_end = -1;
    SchemeDev sc;
    int st = build_scheme(scheme, &sc);
    if (st) return st;
    if (n < 0 || m < 0 || (n && !a) || (m && !b)) return SW_EINVAL;
    if (n > STATIC_MAX_N || m > STATIC_MAX_M) return SW_ENOMEM;      // beyond the static scratch
    const int64_t worst = (int64_t)sc.max_sub * (n < m ? n : m) +
                          (int64_t)(sc.go > -sc.min_sub ? sc.go : -sc.min_sub) * (n + m) + sc.go;
    if (worst >= ((int64_t)1 << 29)) return SW_EINVAL;
    out->stats.cells = n * m;
    if (n == 0 || m == 0) return SW_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SW_ECUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!dev_base[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) { cudaGetLastError(); return SW_ECUDA; }
            dev_base[dev] = (unsigned char *)p;
        }
        base = dev_base[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *ctr = (int32_t *)(base + OFF_CTR);
    const int nbands = (int)((n + 32 * STATIC_RPT - 1) / (32 * STATIC_RPT));
    const int nch = (int)((m + CH - 1) / CH);
    FwdProblem d;
    std::memset(&d, 0, sizeof d);
    d.a = a; d.b = b; d.n = (int32_t)n; d.m = (int32_t)m; d.nbands = nbands;
    d.mode = FWD_LOCAL; d.target = 0; d.transposed = 0;
    d.bus = (int2 *)(base + OFF_BUS);
    d.flags = (int32_t *)(base + OFF_FLAGS);
    d.best = ctr + 2;
    d.stop_band = ctr + 3;
    d.ovf = ctr + 4;
    d.band_res = (int4 *)(base + OFF_BANDRES);
    static_setup_kernel<<<256, 256, 0, s>>>(d, nbands, nch, -sc.go);
    static_check_codes_kernel<<<128, 256, 0, s>>>(a, n, sc.alphabet);
    static_check_codes_kernel<<<128, 256, 0, s>>>(b, m, sc.alphabet);
    if (cudaGetLastError() != cudaSuccess) return SW_ECUDA;
    FwdParams P;
    std::memset(&P, 0, sizeof P);
    P.probs = (const FwdProblem *)(base + OFF_DESC);
    P.tickets = (const int2 *)(base + OFF_TICKETS);
    P.ntickets = nbands;
    P.ticket_ctr = ctr + 0;
    P.err = ctr + 1;
    P.stats = (unsigned long long *)(base + OFF_STATS);
    for (int x = 0; x < 8; ++x) {
        P.prof_lo[x] = sc.prof_lo[x]; P.prof_hi[x] = sc.prof_hi[x];
        P.prof_lo_t[x] = sc.prof_lo_t[x]; P.prof_hi_t[x] = sc.prof_hi_t[x];
    }
    P.go = sc.go; P.ge = sc.ge; P.max_sub = sc.max_sub;
    P.prune = 1;
    P.fault_band = -1;
    P.timeout_ns = 2000ull * 1000000ull;
    const bool p2 = sc.alphabet > 4;
    int per_sm = 1, sms = 1;
    if (fwd_occupancy(STATIC_RPT, p2, 128, &per_sm) != cudaSuccess || per_sm < 1) per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SW_ECUDA;
    int ctas = per_sm * sms;
    if (ctas > (nbands + 3) / 4) ctas = (nbands + 3) / 4;
    // a bad code makes the kernel read nothing out of range (codes are masked), but
    // the result would be meaningless: checked after the run, reported as EINVAL
    if (fwd_launch(P, STATIC_RPT, p2, ctas, 128, s) != cudaSuccess) return SW_ECUDA;
    if (fwd_reduce_launch(P.probs, 1, (int4 *)(base + OFF_RES), s) != cudaSuccess) return SW_ECUDA;
    int4 res;
    int32_t hctr[6];
    unsigned long long hst[4];
    if (cudaMemcpyAsync(&res, base + OFF_RES, sizeof res, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hctr, ctr, sizeof hctr, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hst, base + OFF_STATS, sizeof hst, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SW_ECUDA;
    if (hctr[5]) return SW_EINVAL;
    if (hctr[1] == DEV_ETIMEOUT) return SW_ETIMEOUT;
    if (hctr[1]) return SW_ECUDA;
    out->stats.fwd_cells = out->stats.cells_computed = (int64_t)hst[0];
    out->stats.tiles_total = (int64_t)hst[1];
    out->stats.tiles_pruned = (int64_t)hst[2];
    out->stats.kernel_launches = 5;
    if (res.w && res.x > 0) { out->score = res.x; out->a_end = res.y; out->b_end = res.z; }
    return SW_OK;
}
