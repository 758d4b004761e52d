// ctx.h -- host-side context, workspace arena and shared driver helpers.
#pragma once
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/swgb.h"
#include "kernels.h"

namespace swgb {

// NVTX range over the current scope, named after a library phase: shows the
// phases on the host timeline of Nsight Systems and filters Nsight Compute
// (--nvtx --nvtx-include).  NVTX v3 is header-only and does nothing unless a
// tool is attached.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// First-fit sub-allocator over the context's device workspace (256-byte aligned).
class Arena {
public:
    void reset(char *base, size_t bytes) {
        base_ = base; bytes_ = bytes; free_.clear(); used_.clear();
        if (bytes) free_[0] = bytes;
    }
    void *alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (bytes == 0) bytes = 256;
        std::lock_guard<std::mutex> g(mu_);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_[off] = bytes;
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(void *p) {
        if (!p) return;
        std::lock_guard<std::mutex> g(mu_);
        size_t off = (size_t)((char *)p - base_);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t sz = u->second;
        used_.erase(u);
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first == off + sz) { sz += nx->second; nx = free_.erase(nx); }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) { pv->second += sz; return; }
        }
        free_[off] = sz;
    }
    size_t largest_free() const {
        std::lock_guard<std::mutex> g(mu_);
        size_t best = 0;
        for (auto &f : free_) best = f.second > best ? f.second : best;
        return best;
    }
    size_t free_bytes() const {
        std::lock_guard<std::mutex> g(mu_);
        size_t t = 0;
        for (auto &f : free_) t += f.second;
        return t;
    }
    size_t capacity() const { return bytes_; }
private:
    char *base_ = nullptr;
    size_t bytes_ = 0;
    std::map<size_t, size_t> free_;
    std::map<size_t, size_t> used_;
    mutable std::mutex mu_;
};

// Allocations of one call, released together (RAII).
class Scope {
public:
    explicit Scope(Arena &a) : a_(a) {}
    ~Scope() { for (void *p : ptrs_) a_.release(p); }
    template <class T> T *get(size_t count) {
        void *p = a_.alloc(sizeof(T) * (count ? count : 1));
        if (!p) { failed_ = true; return nullptr; }
        ptrs_.push_back(p);
        return (T *)p;
    }
    bool failed() const { return failed_; }
private:
    Arena &a_;
    std::vector<void *> ptrs_;
    bool failed_ = false;
};

// Scheme as the kernels consume it.
struct SchemeDev {
    int alphabet = 4;
    int go = 5, ge = 2;
    int max_sub = 1;
    int min_sub = -3;
    int8_t table[64];          // 8 x 8 row-major (a code, b code)
    uint32_t prof_lo[8], prof_hi[8];
    uint32_t prof_lo_t[8], prof_hi_t[8];   // same for the transposed table
};

struct Options {
    int rows_per_thread = 0;       // 0 = chosen per call from the problem size
    int warps_per_sm = 0;          // 0 = occupancy limit
    int64_t timeout_ms = 2000;
    int fault_band = -1;
    int ckpt_bands = 0;            // 0 = choose from the workspace size
    int64_t leaf_cells = 1 << 16;
    int forward_lanes = 0;         // 0 auto, 16 int16x2 (offset) lanes, 32 int32 lanes
    int trace = 0;                 // 1: one stderr line per device pass
    int autotune = 1;              // 1: batch band height timed per batch shape
};

}  // namespace swgb

struct sw_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    bool owns_ws = false;
    int sms = 0;
    swgb::Arena arena;
    swgb::Options opt;
    std::string last_error;
    cudaEvent_t ev[10] = {};
    std::mutex call_mu;
    int64_t launches = 0;          // kernels launched by this context (all calls)
    std::map<uint64_t, int> tuned_rpt16;   // batch shape -> fastest int16x2 band height
    std::string gpu_name;                  // device model the tuned table was measured on
};

namespace swgb {

int set_cuda_error(sw_ctx *ctx, cudaError_t e, const char *where);
int build_scheme(const sw_scheme *s, SchemeDev *out);

// Forward pass over a set of problems (one persistent launch).  res[p] receives
// {score, row, col, found} (biased in anchored mode).  stats may be null.
// Row record of a forward or anchored pass (see FwdProblem::gout): running
// column maxima of every stride-th band's bottom row, kept by the caller for
// the next pass over the same pair.
struct Guide {
    Scope *scope = nullptr;    // where the pass allocates the record
    size_t budget = 0;         // bytes it may take there
    int32_t *buf = nullptr;    // rows x (nch + 2), rows read with rec_at
    int32_t step = 0;          // DP rows between recorded rows
    int32_t rows = 0, nch = 0;
    bool valid = false;        // set when the pass wrote it (int16x2 offset lanes, no re-run)
};

struct FwdJob {
    const uint8_t *a;      // device
    const uint8_t *b;      // device
    int32_t n, m;
    int32_t mode;          // FwdMode
    int32_t target;        // anchored: biased target
    int32_t transposed;
    int32_t rpt16 = 0;             // rows per thread on int16x2 lanes (0: chosen by size)
    Guide *gout = nullptr;         // record this pass's rows here
    const Guide *gin = nullptr;    // anchored: forward record to prune with
    int32_t gin_i0 = 0, gin_j0 = 0;
};
int run_forward(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                int rpt, std::vector<int4> &res, sw_stats *stats, float *ms);
// Kernel parameters of one forward launch over the problems dprobs[] and the
// tickets dtk[0, ntk) (counters: ctrs[0] ticket, ctrs[1] error word)
void fwd_params(sw_ctx *ctx, const SchemeDev &sc, bool prune, const FwdProblem *dprobs, const int2 *dtk,
                int64_t ntk, int32_t *ctrs, unsigned long long *dstats, FwdParams &P);
// launch shape of a forward pass over ntk tickets: CTAs, warps per CTA (one band
// each at a time) and whether it is the one-CTA-per-SM layout
void fwd_launch_shape(sw_ctx *ctx, const SchemeDev &sc, int64_t ntk, int rpt, bool lane16, bool rel, bool anch,
                      int *ctas, int *cta_warps, bool *wide);
// launches the forward kernel for P on the context's stream with the launch
// shape the library uses (one CTA per SM for long local passes on offset
// lanes), chosen for shape_ntk tickets (> 0; else P's own count)
cudaError_t fwd_launch_pass(sw_ctx *ctx, const SchemeDev &sc, const FwdParams &P, int rpt, bool lane16, bool rel,
                            bool anch, int *cta_warps, int64_t shape_ntk = -1);
// lanes (int16x2 offset lanes or int32) and band height that run_forward starts
// a single local problem with (int32 lanes only when allow16 is false)
void forward_plan(sw_ctx *ctx, const SchemeDev &sc, const FwdJob &job, bool allow16, bool *lane16, int *rpt);
int run_forward32(sw_ctx *ctx, const SchemeDev &sc, const std::vector<FwdJob> &jobs, bool prune,
                  int rpt, std::vector<int4> &res, sw_stats *stats, float *ms);

}  // namespace swgb
