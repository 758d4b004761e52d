// leaf.cu -- full-matrix traceback of small sub-problems (sm_103a).
//
// The paper stops its Myers-Miller recursion once a sub-matrix is small and
// solves that sub-matrix with a plain Needleman-Wunsch alignment (Sec. 2,
// reconstruction paragraph; on the CPU there).  Here every such leaf is one CTA:
// the global affine DP between the leaf's source node (0,0,src) and sink node
// (n,m,snk) runs anti-diagonal by anti-diagonal over rows held cyclically by the
// CTA's threads, one pointer byte per cell in shared memory (H source: diagonal
// / F / E, plus E-open and F-open bits), then thread 0 follows the greedy rule
// (diagonal > F > E; open > extend) back from the sink.  All leaves of one
// recursion level go in one launch.
#include "common.cuh"
#include "lab.h"

namespace swgb {

__global__ void __launch_bounds__(256) leaf_kernel(const LeafProblem *probs, const int8_t *tab8, int go,
                                                   int ge, char *ops, int32_t *ops_len)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int8_t tab[64];
    const LeafProblem pr = probs[blockIdx.x];
    const int n = pr.n, m = pr.m, W = m + 1;
    const int tid = threadIdx.x, bd = blockDim.x;
    const size_t cells = (size_t)(n + 1) * (size_t)W;
    const size_t pbytes = (cells + 15) & ~(size_t)15;
    unsigned char *ptr = sm;
    int *Hb = (int *)(sm + pbytes);          // 3 x (n+1): H on diagonals d, d-1, d-2
    int *Fb = Hb + 3 * (n + 1);              // 2 x (n+1): F on diagonals d, d-1
    int *Eb = Fb + 2 * (n + 1);              // (n+1): E(i, j) of the row's latest cell
    if (tid < 64) tab[tid] = tab8[tid];
    const int NEG = -(1 << 28);
    for (int d = 0; d <= n + m; ++d) {
        const int c0 = d % 3, c1 = (d + 2) % 3, c2 = (d + 1) % 3;
        for (int i = tid; i <= n; i += bd) {
            const int j = d - i;
            if (j < 0 || j > m) continue;
            int h, e, f, bits = 0;
            if (i == 0 && j == 0) {
                h = 0;
                e = pr.src == ST_E ? 0 : NEG;
                f = pr.src == ST_F ? 0 : NEG;
                bits = pr.src == ST_F ? 1 : (pr.src == ST_E ? 2 : 3);
            } else if (i == 0) {
                const int eo = Hb[c1 * (n + 1)] - go, ex = Eb[0] - ge;
                if (eo >= ex) { e = eo; bits |= 4; } else e = ex;
                h = e; f = NEG; bits |= 2;
            } else if (j == 0) {
                const int fo = Hb[c1 * (n + 1) + i - 1] - go, fx = Fb[((d - 1) & 1) * (n + 1) + i - 1] - ge;
                if (fo >= fx) { f = fo; bits |= 8; } else f = fx;
                h = f; e = NEG; bits |= 1;
            } else {
                const int eo = Hb[c1 * (n + 1) + i] - go, ex = Eb[i] - ge;
                if (eo >= ex) { e = eo; bits |= 4; } else e = ex;
                const int fo = Hb[c1 * (n + 1) + i - 1] - go, fx = Fb[((d - 1) & 1) * (n + 1) + i - 1] - ge;
                if (fo >= fx) { f = fo; bits |= 8; } else f = fx;
                const int dd = Hb[c2 * (n + 1) + i - 1] + tab[pr.a[i - 1] * 8 + pr.b[j - 1]];
                if (dd >= f && dd >= e) h = dd;
                else if (f >= e) { h = f; bits |= 1; }
                else { h = e; bits |= 2; }
            }
            h = max(h, NEG); e = max(e, NEG); f = max(f, NEG);
            Hb[c0 * (n + 1) + i] = h;
            Fb[(d & 1) * (n + 1) + i] = f;
            Eb[i] = e;
            ptr[(size_t)i * W + j] = (unsigned char)bits;
        }
        __syncthreads();
    }
    if (tid == 0) {
        char *o = ops + pr.out_off;
        int i = n, j = m, st = pr.snk, len = 0;
        const int cap = n + m + 2;
        int ok = 1;
        for (int guard = 0; guard < 2 * (n + m) + 8; ++guard) {
            if (i == 0 && j == 0 && st == pr.src) break;
            const int p = ptr[(size_t)i * W + j];
            if (st == ST_H) {
                const int hs = p & 3;
                if (hs == 0) { if (len >= cap || i == 0 || j == 0) { ok = 0; break; } o[len++] = 'M'; --i; --j; }
                else if (hs == 1) st = ST_F;
                else if (hs == 2) st = ST_E;
                else { ok = 0; break; }
            } else if (st == ST_F) {
                if (i == 0 || len >= cap) { ok = 0; break; }
                o[len++] = 'I';
                st = (p & 8) ? ST_H : ST_F;
                --i;
            } else {
                if (j == 0 || len >= cap) { ok = 0; break; }
                o[len++] = 'D';
                st = (p & 4) ? ST_H : ST_E;
                --j;
            }
        }
        if (!(i == 0 && j == 0 && st == pr.src)) ok = 0;
        for (int x = 0, y = len - 1; x < y; ++x, --y) { const char t = o[x]; o[x] = o[y]; o[y] = t; }
        ops_len[blockIdx.x] = ok ? len : -1;
    }
}

size_t leaf_smem_bytes(int n, int m)
{
    const size_t cells = (size_t)(n + 1) * (size_t)(m + 1);
    return ((cells + 15) & ~(size_t)15) + sizeof(int) * 6 * (size_t)(n + 1);
}

cudaError_t leaf_launch(const LeafProblem *probs, int nprobs, const int8_t *table8, int go, int ge,
                        int max_cells, char *ops, int32_t *ops_len, cudaStream_t s)
{
    if (nprobs <= 0) return cudaSuccess;
    const size_t smem = ((size_t)max_cells + 15 + 16) + sizeof(int) * 6 * (LEAF_MAX_DIM + 1);
    cudaError_t e = cudaFuncSetAttribute(leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    leaf_kernel<<<nprobs, 256, smem, s>>>(probs, table8, go, ge, ops, ops_len);
    return cudaGetLastError();
}

}  // namespace swgb
