// probe.cu -- issue-rate microbenchmark of the integer / DPX instructions the
// forward pass is built from, for its roofline (ops per clock per SM).
//
// Each thread runs 8 independent dependency chains of one instruction kind for
// `iters` iterations; clock64() around the loop gives SM cycles, so the result
// does not depend on the clock the GPU happened to run at.
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/swgb.h"
#include "common.cuh"

namespace swgb {

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(int iters, int seed, int *sink,
                                                     unsigned long long *cycles)
{
    int x0 = threadIdx.x ^ seed, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3;
    int x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    const int c = (seed | 1) + (int)(threadIdx.x & 1), d = seed >> 3, go = (seed >> 5) | 1;
    const uint32_t sel = code_selector((uint32_t)seed & 3u);
    const uint32_t pw = 0x01fdfdfdu ^ (uint32_t)(threadIdx.x & 0x10);
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            if (KIND == 0) {        // IADD (chains through xor so it cannot fold)
                x0 = (x0 + x7) ^ c; x1 = (x1 + x0) ^ c; x2 = (x2 + x1) ^ c; x3 = (x3 + x2) ^ c;
            } else if (KIND == 1) { // IMNMX
                x0 = max(x0, x7) - c; x1 = max(x1, x0) - c; x2 = max(x2, x1) - c; x3 = max(x3, x2) - c;
            } else if (KIND == 2) { // DPX viaddmax
                x0 = __viaddmax_s32(x0, c, x1); x1 = __viaddmax_s32(x1, c, x2);
                x2 = __viaddmax_s32(x2, c, x3); x3 = __viaddmax_s32(x3, c, x4);
                x4 = __viaddmax_s32(x4, c, x5); x5 = __viaddmax_s32(x5, c, x6);
                x6 = __viaddmax_s32(x6, c, x7); x7 = __viaddmax_s32(x7, c, x0);
            } else if (KIND == 3) { // DPX viaddmax relu
                x0 = __viaddmax_s32_relu(x0, d, x1); x1 = __viaddmax_s32_relu(x1, d, x2);
                x2 = __viaddmax_s32_relu(x2, d, x3); x3 = __viaddmax_s32_relu(x3, d, x4);
                x4 = __viaddmax_s32_relu(x4, d, x5); x5 = __viaddmax_s32_relu(x5, d, x6);
                x6 = __viaddmax_s32_relu(x6, d, x7); x7 = __viaddmax_s32_relu(x7, d, x0);
            } else if (KIND == 4) { // PRMT
                x0 = sub_lookup((uint32_t)x0, 0u, sel); x1 = sub_lookup((uint32_t)x1, 0u, sel);
                x2 = sub_lookup((uint32_t)x2, 0u, sel); x3 = sub_lookup((uint32_t)x3, 0u, sel);
                x4 = sub_lookup((uint32_t)x4, 0u, sel); x5 = sub_lookup((uint32_t)x5, 0u, sel);
                x6 = sub_lookup((uint32_t)x6, 0u, sel); x7 = sub_lookup((uint32_t)x7, 0u, sel);
            } else if (KIND == 5) { // 16x2 DPX viaddmax
                x0 = (int)__viaddmax_s16x2((unsigned)x0, (unsigned)c, (unsigned)x1);
                x1 = (int)__viaddmax_s16x2((unsigned)x1, (unsigned)c, (unsigned)x2);
                x2 = (int)__viaddmax_s16x2((unsigned)x2, (unsigned)c, (unsigned)x3);
                x3 = (int)__viaddmax_s16x2((unsigned)x3, (unsigned)c, (unsigned)x4);
                x4 = (int)__viaddmax_s16x2((unsigned)x4, (unsigned)c, (unsigned)x5);
                x5 = (int)__viaddmax_s16x2((unsigned)x5, (unsigned)c, (unsigned)x6);
                x6 = (int)__viaddmax_s16x2((unsigned)x6, (unsigned)c, (unsigned)x7);
                x7 = (int)__viaddmax_s16x2((unsigned)x7, (unsigned)c, (unsigned)x0);
            } else if (KIND == 6) { // the forward pass's cell (A): 7 ops
                const int s = sub_lookup(pw, 0u, sel ^ (uint32_t)(x7 & 3));
                x1 = __viaddmax_s32(x1, -d, x2);
                const int t = __viaddmax_s32_relu(x3, s, x4);
                x5 = max(t, x1);
                x2 = x5 - go;
                x4 = __viaddmax_s32(x4, -d, x2);
                x6 = max(x6, x5);
                x3 = x5; x7 ^= x6;
            } else if (KIND == 7) { // DPX vimax3
                x0 = __vimax3_s32(x0, x1, c); x1 = __vimax3_s32(x1, x2, c); x2 = __vimax3_s32(x2, x3, c);
                x3 = __vimax3_s32(x3, x4, c); x4 = __vimax3_s32(x4, x5, c); x5 = __vimax3_s32(x5, x6, c);
                x6 = __vimax3_s32(x6, x7, c); x7 = __vimax3_s32(x7, x0, c);
            } else if (KIND == 8) { // DPX vimax3 relu
                x0 = __vimax3_s32_relu(x0, x1, c); x1 = __vimax3_s32_relu(x1, x2, c);
                x2 = __vimax3_s32_relu(x2, x3, c); x3 = __vimax3_s32_relu(x3, x4, c);
                x4 = __vimax3_s32_relu(x4, x5, c); x5 = __vimax3_s32_relu(x5, x6, c);
                x6 = __vimax3_s32_relu(x6, x7, c); x7 = __vimax3_s32_relu(x7, x0, c);
            } else if (KIND == 9) { // cell form B: D by add, H by vimax3_relu
                const int s = sub_lookup(pw, 0u, sel ^ (uint32_t)(x7 & 3));
                x1 = __viaddmax_s32(x1, -d, x2);                 // F
                const int D = x3 + s;
                x5 = __vimax3_s32_relu(D, x4, x1);               // H
                x2 = x5 - go;
                x4 = __viaddmax_s32(x4, -d, x2);                 // E
                x6 = max(x6, x5);
                x3 = x5; x7 ^= x6;
            } else if (KIND == 10) { // DPX vimax relu (2 inputs)
                x0 = __vimax_s32_relu(x0, x1 - c); x1 = __vimax_s32_relu(x1, x2 - c);
                x2 = __vimax_s32_relu(x2, x3 - c); x3 = __vimax_s32_relu(x3, x0 - c);
            } else {                // 16x2 cell form (2 cells per op)
                const uint32_t s = (uint32_t)sub_lookup(pw, pw, sel ^ (uint32_t)(x7 & 3));
                x1 = (int)__viaddmax_s16x2((unsigned)x1, (unsigned)d, (unsigned)x2);
                const unsigned D = __vadd2((unsigned)x3, s);
                x5 = (int)__vimax3_s16x2_relu(D, (unsigned)x4, (unsigned)x1);
                x2 = (int)__vsub2((unsigned)x5, (unsigned)go);
                x4 = (int)__viaddmax_s16x2((unsigned)x4, (unsigned)d, (unsigned)x2);
                x6 = (int)__vmaxs2((unsigned)x6, (unsigned)x5);
                x3 = x5; x7 ^= x6;
            }
        }
    }
    const unsigned long long t1 = clock64();
    sink[blockIdx.x * blockDim.x + threadIdx.x] = x0 ^ x1 ^ x2 ^ x3 ^ x4 ^ x5 ^ x6 ^ x7;
    if (threadIdx.x == 0) atomicMax(cycles, t1 - t0);
}

}  // namespace swgb

using namespace swgb;

extern "C" int sw_probe_issue_rate(int device, int kind, double *ops_per_clk_per_sm)
{
    if (!ops_per_clk_per_sm || kind < 0 || kind > 11) return SW_EINVAL;
    if (cudaSetDevice(device)) return SW_ECUDA;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device)) return SW_ECUDA;
    const int threads = 256, per_sm = 4, iters = 4096;
    const int blocks = prop.multiProcessorCount * per_sm;
    int *sink = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(int) * blocks * threads) || cudaMalloc(&cyc, 8)) return SW_ECUDA;
    cudaMemset(cyc, 0, 8);
    void (*k)(int, int, int *, unsigned long long *) = nullptr;
    switch (kind) {
    case 0: k = probe_kernel<0>; break;
    case 1: k = probe_kernel<1>; break;
    case 2: k = probe_kernel<2>; break;
    case 3: k = probe_kernel<3>; break;
    case 4: k = probe_kernel<4>; break;
    case 5: k = probe_kernel<5>; break;
    case 6: k = probe_kernel<6>; break;
    case 7: k = probe_kernel<7>; break;
    case 8: k = probe_kernel<8>; break;
    case 9: k = probe_kernel<9>; break;
    case 10: k = probe_kernel<10>; break;
    default: k = probe_kernel<11>; break;
    }
    k<<<blocks, threads>>>(iters, 12345, sink, cyc);          // warm-up
    cudaMemset(cyc, 0, 8);
    k<<<blocks, threads>>>(iters, 12345, sink, cyc);
    unsigned long long c = 0;
    cudaError_t e = cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(cyc);
    if (e || c == 0) return SW_ECUDA;
    // lane operations per SM: the chains do 8 ops per inner step, except the
    // add / max probes (kinds 0, 1: 4 x 2 ops) and the 2-input relu max (4 ops);
    // for the cell mixes (6, 9, 11) one inner step is one cell (11: two cells)
    double per_step = 8.0;
    if (kind == 10) per_step = 4.0;
    if (kind == 6 || kind == 9) per_step = 1.0;
    if (kind == 11) per_step = 2.0;
    const double ops = (double)per_sm * threads * iters * 16.0 * per_step;
    *ops_per_clk_per_sm = ops / (double)c;
    return SW_OK;
}
