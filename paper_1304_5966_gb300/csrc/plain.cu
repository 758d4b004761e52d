// plain.cu -- the plain GPU path kept as the comparison baseline, plus small
// utility kernels.
//
// plain_score: the textbook wavefront (the paper's starting point, Sec. 2:
// "solving the elements on the matrix anti-diagonal at the same time"): one
// thread per cell of anti-diagonal d, one launch per anti-diagonal, three
// diagonal buffers of H, E, F in global memory, int32, no pruning, no register
// blocking.  The best cell is kept with a 64-bit atomicMax on a key ordered by
// (score, smallest row, smallest column), which gives the library's end-point
// tie rule.  Rows and columns must be below 2^20.
#include "common.cuh"
#include "kernels.h"

namespace swgb {

// diag_bufs holds 3 diagonals x 3 arrays (H, E, F) x (n + 2) ints
__global__ void plain_diag_kernel(const uint8_t *__restrict__ a, int n, const uint8_t *__restrict__ b,
                                  int m, const int32_t *__restrict__ sub, int alph, int go, int ge,
                                  int32_t *bufs, int d, unsigned long long *best_key)
{
    const int stride = n + 2;
    int32_t *Hc = bufs + ((d % 3) * 3 + 0) * stride;
    int32_t *Ec = bufs + ((d % 3) * 3 + 1) * stride;
    int32_t *Fc = bufs + ((d % 3) * 3 + 2) * stride;
    const int d1 = (d + 2) % 3, d2 = (d + 1) % 3;   // d-1, d-2
    const int32_t *H1 = bufs + (d1 * 3 + 0) * stride;
    const int32_t *E1 = bufs + (d1 * 3 + 1) * stride;
    const int32_t *F1 = bufs + (d1 * 3 + 2) * stride;
    const int32_t *H2 = bufs + (d2 * 3 + 0) * stride;
    const int ilo = max(1, d - m), ihi = min(n, d - 1);
    const int i = ilo + blockIdx.x * blockDim.x + threadIdx.x;
    if (i > ihi) return;
    const int j = d - i;
    // neighbours: (i, j-1) and (i-1, j) lie on diagonal d-1, (i-1, j-1) on d-2;
    // border cells (row 0 / column 0) hold H = 0, E = F = -inf
    const int NEG = -(1 << 29);
    const int hl = (j > 1) ? H1[i] : 0;
    const int el = (j > 1) ? E1[i] : NEG;
    const int hu = (i > 1) ? H1[i - 1] : 0;
    const int fu = (i > 1) ? F1[i - 1] : NEG;
    const int hd = (i > 1 && j > 1) ? H2[i - 1] : 0;
    const int e = max(el - ge, hl - go);
    const int f = max(fu - ge, hu - go);
    const int h = max(max(hd + sub[a[i - 1] * alph + b[j - 1]], 0), max(e, f));
    Hc[i] = h; Ec[i] = e; Fc[i] = f;
    if (h > 0) {
        const unsigned long long key = ((unsigned long long)h << 40) |
                                       ((unsigned long long)((1 << 20) - 1 - i) << 20) |
                                       (unsigned long long)((1 << 20) - 1 - j);
        if (key > *(volatile unsigned long long *)best_key) atomicMax(best_key, key);
    }
}

cudaError_t plain_score(const uint8_t *a, int n, const uint8_t *b, int m, const int32_t *sub,
                        int alph, int go, int ge, int32_t *bufs, unsigned long long *best_key,
                        cudaStream_t s)
{
    for (int d = 2; d <= n + m; ++d) {
        const int ilo = max(1, d - m), ihi = min(n, d - 1);
        const int cnt = ihi - ilo + 1;
        if (cnt <= 0) continue;
        const int th = 256;
        plain_diag_kernel<<<(cnt + th - 1) / th, th, 0, s>>>(a, n, b, m, sub, alph, go, ge, bufs, d,
                                                             best_key);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void reverse_copy_kernel(const uint8_t *src, uint8_t *dst, int64_t len)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[len - 1 - i];
}
cudaError_t reverse_copy_launch(const uint8_t *src, uint8_t *dst, int64_t len, cudaStream_t s)
{
    if (len <= 0) return cudaSuccess;
    const int64_t nb = (len + 255) / 256;
    const int blocks = (int)(nb < 4096 ? nb : 4096);
    reverse_copy_kernel<<<blocks, 256, 0, s>>>(src, dst, len);
    return cudaGetLastError();
}

// one block per segment: dst[dst_off + i] = src[src_off + len - 1 - i]
__global__ void reverse_segments_kernel(const uint8_t *src, uint8_t *dst, const int64_t *src_off,
                                        const int64_t *dst_off, const int32_t *len)
{
    const int k = blockIdx.x;
    const int64_t so = src_off[k], d0 = dst_off[k];
    const int L = len[k];
    for (int i = threadIdx.x; i < L; i += blockDim.x) dst[d0 + i] = src[so + L - 1 - i];
}
cudaError_t reverse_segments_launch(const uint8_t *src, uint8_t *dst, const int64_t *src_off,
                                    const int64_t *dst_off, const int32_t *len, int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    reverse_segments_kernel<<<count, 256, 0, s>>>(src, dst, src_off, dst_off, len);
    return cudaGetLastError();
}

// one block per segment: dst[off + i] = complement(src[off + len - 1 - i])
// (DNA codes A0 C1 G2 T3 pair as c <-> 3 - c; N and any other code stay)
__global__ void revcomp_segments_kernel(const uint8_t *src, uint8_t *dst, const int64_t *off, const int32_t *len)
{
    const int k = blockIdx.x;
    const int64_t o = off[k];
    const int L = len[k];
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const uint8_t c = src[o + L - 1 - i];
        dst[o + i] = c < 4 ? (uint8_t)(3 - c) : c;
    }
}
cudaError_t revcomp_segments_launch(const uint8_t *src, uint8_t *dst, const int64_t *off, const int32_t *len,
                                    int count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    revcomp_segments_kernel<<<count, 256, 0, s>>>(src, dst, off, len);
    return cudaGetLastError();
}

__global__ void fill_i32_kernel(int32_t *p, int32_t v, int64_t count)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}
cudaError_t fill_i32_launch(int32_t *p, int32_t v, int64_t count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int64_t nb = (count + 255) / 256;
    const int blocks = (int)(nb < 4096 ? nb : 4096);
    fill_i32_kernel<<<blocks, 256, 0, s>>>(p, v, count);
    return cudaGetLastError();
}

__global__ void check_codes_kernel(const uint8_t *p, int64_t len, int alph, int32_t *bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x)
        if (p[i] >= alph) { atomicExch(bad, 1); return; }
}
cudaError_t check_codes_launch(const uint8_t *p, int64_t len, int alph, int32_t *bad, cudaStream_t s)
{
    if (len <= 0) return cudaSuccess;
    const int64_t nb = (len + 255) / 256;
    const int blocks = (int)(nb < 2048 ? nb : 2048);
    check_codes_kernel<<<blocks, 256, 0, s>>>(p, len, alph, bad);
    return cudaGetLastError();
}

}  // namespace swgb
