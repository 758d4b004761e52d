/*
 * sw_oracle.c -- plain scalar CPU oracle for exact affine-gap Smith-Waterman.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Every function is the plain definition of what the paper computes, written
 * out cell by cell in 64-bit integers, with no blocking, banding, pruning or
 * reordering:
 *
 *   orc_local_score     Smith-Waterman with affine gaps (Gotoh H/E/F): best
 *                       local score S and the end point (paper: Abstract and
 *                       Sec. 2, wavefront paragraph: "output of this phase is
 *                       the score and the endpoint").
 *   orc_reverse_start   the start point: the modified Smith-Waterman run on the
 *                       reversed prefixes that end at the end point, borders at
 *                       minus infinity, no zero floor (Sec. 2, start-point
 *                       paragraph).
 *   orc_global_trace    Needleman-Wunsch with affine gaps between two nodes and
 *                       a full-matrix greedy traceback (Sec. 2, reconstruction
 *                       paragraph: the alignment between start and end point).
 *   orc_verify_path     streaming check, O(columns) memory, that a given path is
 *                       exactly the greedy traceback path of orc_global_trace.
 *   orc_rescore         score of an explicit alignment (op string).
 *
 * Conventions (the paper is silent on them; these are the readings used):
 *   - A has length n and indexes rows i = 1..n; B has length m, columns j.
 *   - A gap of length k costs go + ge*(k-1) (affine model, Abstract).
 *   - E is the horizontal gap state (consumes B only, op 'D'); F the vertical
 *     state (consumes A only, op 'I'); H the best of diagonal, E and F.
 *   - End point: among cells with H = S, the smallest row, then the smallest
 *     column.  Start point: among reverse-pass cells with value S, the smallest
 *     reversed row, then the smallest reversed column (largest original start).
 *   - Traceback preference: in H, diagonal > F > E; in E and F, open > extend.
 *   - Coordinates are 0-based, end exclusive.  S = 0 gives an empty result.
 *
 * States passed across this ABI: 0 = H, 1 = E, 2 = F.
 * Ops written: 'M' (diagonal), 'I' (consumes A), 'D' (consumes B).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NEG_INF (-(INT64_C(1) << 60))

static inline int64_t max2(int64_t x, int64_t y) { return x > y ? x : y; }

static inline int64_t subst(const int32_t *sub, int alph, uint8_t x, uint8_t y) {
    return (int64_t)sub[(int)x * alph + (int)y];
}

/* ------------------------------------------------------------------------ */
/* Local Gotoh: score and end point.                                         */
/* H[i][j] = max(0, H[i-1][j-1] + s(a_i, b_j), E[i][j], F[i][j])             */
/* E[i][j] = max(E[i][j-1] - ge, H[i][j-1] - go)                             */
/* F[i][j] = max(F[i-1][j] - ge, H[i-1][j] - go)                             */
/* with H = 0 on row 0 and column 0, E = F = -inf there.                     */
/* Row-major scan with a strict '>' keeps the first cell in row-major order.  */
/* ------------------------------------------------------------------------ */
int64_t orc_local_score(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                        const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                        int64_t *end_i, int64_t *end_j)
{
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -1; }
    for (int64_t j = 0; j <= m; ++j) { Hrow[j] = 0; Frow[j] = NEG_INF; }
    int64_t best = 0, bi = -1, bj = -1;
    for (int64_t i = 1; i <= n; ++i) {
        int64_t diag = Hrow[0];          /* H[i-1][0] = 0 */
        int64_t left = 0;                /* H[i][0] = 0 */
        int64_t e = NEG_INF;             /* E[i][0] */
        for (int64_t j = 1; j <= m; ++j) {
            e = max2(e - ge, left - go);
            Frow[j] = max2(Frow[j] - ge, Hrow[j] - go);
            int64_t h = diag + subst(sub, alph, a[i - 1], b[j - 1]);
            h = max2(h, e);
            h = max2(h, Frow[j]);
            h = max2(h, 0);
            diag = Hrow[j];
            Hrow[j] = h;
            left = h;
            if (h > best) { best = h; bi = i; bj = j; }
        }
    }
    free(Hrow); free(Frow);
    *end_i = bi; *end_j = bj;
    return best;
}

/* ------------------------------------------------------------------------ */
/* Start point (Sec. 2, start-point paragraph).  On A' = reverse(A[0..ei)),   */
/* B' = reverse(B[0..ej)): the same recurrences without the zero floor, with  */
/* every border at -inf except the origin H'[0][0] = 0, so every path starts  */
/* at the end point.  Start = first cell in row-major order with H' = S.      */
/* Also returns the largest H' seen (it never exceeds S); scan_all = 1 keeps */
/* scanning past the row of the start so that maximum covers the matrix.    */
/* ------------------------------------------------------------------------ */
int orc_reverse_start(const uint8_t *a, const uint8_t *b, int64_t ei, int64_t ej,
                      const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                      int64_t S, int32_t scan_all,
                      int64_t *begin_i, int64_t *begin_j, int64_t *max_seen)
{
    int64_t *Hrow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ej + 1));
    int64_t *Frow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ej + 1));
    if (!Hrow || !Frow) { free(Hrow); free(Frow); return -1; }
    for (int64_t j = 0; j <= ej; ++j) { Hrow[j] = NEG_INF; Frow[j] = NEG_INF; }
    Hrow[0] = 0;
    int64_t mx = NEG_INF;
    int found = 0;
    *begin_i = -1; *begin_j = -1;
    for (int64_t i = 1; i <= ei && (scan_all || !found); ++i) {
        uint8_t ai = a[ei - i];                /* A'[i-1] */
        int64_t diag = Hrow[0];                /* H'[i-1][0] */
        int64_t left = NEG_INF;                /* H'[i][0] */
        int64_t e = NEG_INF;
        Hrow[0] = NEG_INF;
        for (int64_t j = 1; j <= ej; ++j) {
            e = max2(e - ge, left - go);
            Frow[j] = max2(Frow[j] - ge, Hrow[j] - go);
            int64_t h = diag + subst(sub, alph, ai, b[ej - j]);
            h = max2(h, e);
            h = max2(h, Frow[j]);
            if (h < NEG_INF) h = NEG_INF;     /* keep -inf from drifting */
            diag = Hrow[j];
            Hrow[j] = h;
            left = h;
            if (h > mx) mx = h;
            if (h == S && !found) { found = 1; *begin_i = ei - i; *begin_j = ej - j; }
        }
    }
    free(Hrow); free(Frow);
    if (max_seen) *max_seen = mx;
    return found ? 0 : 1;
}

/* ------------------------------------------------------------------------ */
/* Global affine alignment between two nodes, full matrix, greedy traceback. */
/* Source node (0,0) in state src, value 0; sink (N,M) in state snk.         */
/* Borders: row 0 holds only horizontal gaps from the source, column 0 only  */
/* vertical ones.  Pointer nibble per cell: bits 0-1 = H source (0 diag,     */
/* 1 F, 2 E, 3 none), bit 2 = E opened from H, bit 3 = F opened from H.      */
/* ops receives the op string in forward order; returns its length, or -1   */
/* (allocation) / -2 (capacity) / -3 (sink unreachable).  *value = optimum.  */
/* ------------------------------------------------------------------------ */
int64_t orc_global_trace(const uint8_t *a, int64_t N, const uint8_t *b, int64_t M,
                         const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                         int32_t src, int32_t snk, char *ops, int64_t cap,
                         int64_t *value)
{
    size_t W = (size_t)(M + 1);
    size_t cells = (size_t)(N + 1) * W;
    uint8_t *ptr = (uint8_t *)calloc((cells + 1) / 2, 1);
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * W);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * W);
    if (!ptr || !H || !F) { free(ptr); free(H); free(F); return -1; }
#define SETP(i, j, v) do { size_t q_ = (size_t)(i) * W + (size_t)(j); \
        ptr[q_ >> 1] |= (uint8_t)(((v) & 15) << ((q_ & 1) * 4)); } while (0)
#define GETP(i, j) ((ptr[((size_t)(i) * W + (size_t)(j)) >> 1] >> ((((size_t)(i) * W + (size_t)(j)) & 1) * 4)) & 15)

    int64_t e_src = (src == 1) ? 0 : NEG_INF;
    int64_t f_src = (src == 2) ? 0 : NEG_INF;
    /* row 0 */
    H[0] = 0;
    F[0] = f_src;
    SETP(0, 0, src == 2 ? 1 : (src == 1 ? 2 : 3));
    int64_t e = e_src, left = 0;
    for (int64_t j = 1; j <= M; ++j) {
        int64_t ext = e - ge, opn = left - go;
        int bits = 2;                      /* H comes from E */
        if (opn >= ext) { e = opn; bits |= 4; } else e = ext;
        H[j] = e; F[j] = NEG_INF; left = e;
        SETP(0, j, bits);
    }
    int64_t lastE = e;                     /* E[0][M], used if N == 0 */
    for (int64_t i = 1; i <= N; ++i) {
        /* column 0 */
        int64_t fx = F[0] - ge, fo = H[0] - go;
        int bits0 = 1;                     /* H comes from F */
        if (fo >= fx) { F[0] = fo; bits0 |= 8; } else F[0] = fx;
        int64_t diag = H[0];
        H[0] = F[0];
        SETP(i, 0, bits0);
        e = NEG_INF; left = H[0];
        for (int64_t j = 1; j <= M; ++j) {
            int bits = 0;
            int64_t ex = e - ge, eo = left - go;
            if (eo >= ex) { e = eo; bits |= 4; } else e = ex;
            int64_t fx2 = F[j] - ge, fo2 = H[j] - go;
            int64_t f;
            if (fo2 >= fx2) { f = fo2; bits |= 8; } else f = fx2;
            int64_t d = diag + subst(sub, alph, a[i - 1], b[j - 1]);
            int64_t h;
            if (d >= f && d >= e) { h = d; /* bits |= 0 */ }
            else if (f >= e) { h = f; bits |= 1; }
            else { h = e; bits |= 2; }
            if (h < NEG_INF) h = NEG_INF;
            if (f < NEG_INF) f = NEG_INF;
            if (e < NEG_INF) e = NEG_INF;
            diag = H[j];
            H[j] = h; F[j] = f; left = h;
            SETP(i, j, bits);
        }
        lastE = e;
    }
    int64_t v = (snk == 0) ? H[M] : (snk == 2 ? F[M] : lastE);
    free(H); free(F);
    if (v <= NEG_INF / 2) { free(ptr); return -3; }
    *value = v;

    /* greedy traceback from the sink */
    int64_t i = N, j = M, len = 0;
    int st = snk;
    for (;;) {
        if (i == 0 && j == 0 && st == src) break;
        int p = GETP(i, j);
        if (st == 0) {
            int hs = p & 3;
            if (hs == 0) {
                if (len >= cap) { free(ptr); return -2; }
                ops[len++] = 'M'; --i; --j;
            } else if (hs == 1) st = 2;
            else if (hs == 2) st = 1;
            else { free(ptr); return -3; }
        } else if (st == 2) {
            if (i == 0) { free(ptr); return -3; }
            if (len >= cap) { free(ptr); return -2; }
            ops[len++] = 'I';
            st = (p & 8) ? 0 : 2;
            --i;
        } else {
            if (j == 0) { free(ptr); return -3; }
            if (len >= cap) { free(ptr); return -2; }
            ops[len++] = 'D';
            st = (p & 4) ? 0 : 1;
            --j;
        }
    }
    free(ptr);
    for (int64_t x = 0, y = len - 1; x < y; ++x, --y) { char t = ops[x]; ops[x] = ops[y]; ops[y] = t; }
    return len;
#undef SETP
#undef GETP
}

/* ------------------------------------------------------------------------ */
/* Score of an explicit path from node (0,0,src) to its end, affine gaps.    */
/* A run of gap ops opens once (go) then extends (ge); when go == ge every   */
/* gap op counts as its own opening, which costs the same.  A leading run of */
/* the source state's own gap op continues that gap (ge only).              */
/* ------------------------------------------------------------------------ */
int64_t orc_rescore(const uint8_t *a, const uint8_t *b, const char *ops, int64_t len,
                    const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                    int32_t src, int64_t *used_a, int64_t *used_b)
{
    int64_t i = 0, j = 0, score = 0;
    char prev = (src == 2) ? 'I' : (src == 1 ? 'D' : 'M');
    for (int64_t k = 0; k < len; ++k) {
        char o = ops[k];
        if (o == 'M' || o == '=' || o == 'X') {
            score += subst(sub, alph, a[i], b[j]); ++i; ++j; prev = 'M';
        } else if (o == 'I') {
            score -= (prev == 'I') ? ge : go; ++i; prev = 'I';
        } else if (o == 'D') {
            score -= (prev == 'D') ? ge : go; ++j; prev = 'D';
        } else return INT64_MIN;
    }
    *used_a = i; *used_b = j;
    return score;
}

/* ------------------------------------------------------------------------ */
/* Streaming canonicality check, O(M) memory.                                */
/* Recomputes the forward values of orc_global_trace row by row and checks   */
/* that every node of the given path was entered by its most preferred       */
/* optimal predecessor: the chosen one is optimal and every more preferred   */
/* one is not.  That is exactly the greedy traceback, so a path that passes  */
/* is the traceback path.  Gap runs are single gaps when go > ge; when       */
/* go == ge each gap op is its own opening (open wins that tie).             */
/* Returns 0 if canonical, else a positive code naming the first failure.   */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t i, j; int st; int how; } onode;
/* how: 0 source, 1 diag from H(i-1,j-1), 2 H from F(i,j), 3 H from E(i,j),
 *      4 F open from H(i-1,j), 5 F extend from F(i-1,j),
 *      6 E open from H(i,j-1), 7 E extend from E(i,j-1) */

int orc_verify_path(const uint8_t *a, int64_t N, const uint8_t *b, int64_t M,
                    const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                    int32_t src, int32_t snk, const char *ops, int64_t len)
{
    /* 1. expand ops into the node sequence */
    size_t cap = (size_t)(3 * len + 4);
    onode *P = (onode *)malloc(sizeof(onode) * cap);
    if (!P) return 100;
    size_t np = 0;
    int64_t i = 0, j = 0;
    int st = src;
    P[np++] = (onode){0, 0, src, 0};
    for (int64_t k = 0; k < len; ++k) {
        char o = ops[k];
        if (o == 'M' || o == '=' || o == 'X') {
            if (st != 0) P[np++] = (onode){i, j, 0, st == 2 ? 2 : 3};
            ++i; ++j; st = 0;
            P[np++] = (onode){i, j, 0, 1};
        } else if (o == 'I') {
            if (st == 2 && go > ge) {
                ++i; P[np++] = (onode){i, j, 2, 5};
            } else {
                if (st != 0) P[np++] = (onode){i, j, 0, st == 2 ? 2 : 3};
                ++i; st = 2; P[np++] = (onode){i, j, 2, 4};
            }
        } else if (o == 'D') {
            if (st == 1 && go > ge) {
                ++j; P[np++] = (onode){i, j, 1, 7};
            } else {
                if (st != 0) P[np++] = (onode){i, j, 0, st == 2 ? 2 : 3};
                ++j; st = 1; P[np++] = (onode){i, j, 1, 6};
            }
        } else { free(P); return 101; }
    }
    if (st != snk) {
        if (snk == 0) P[np++] = (onode){i, j, 0, st == 2 ? 2 : 3};
        else { free(P); return 102; }
    }
    if (i != N || j != M) { free(P); return 103; }

    /* 2. forward values, two rows, checking path nodes as rows complete */
    size_t W = (size_t)(M + 1);
    int64_t *Hp = malloc(sizeof(int64_t) * W), *Fp = malloc(sizeof(int64_t) * W);
    int64_t *Ep = malloc(sizeof(int64_t) * W);
    int64_t *Hc = malloc(sizeof(int64_t) * W), *Fc = malloc(sizeof(int64_t) * W);
    int64_t *Ec = malloc(sizeof(int64_t) * W);
    if (!Hp || !Fp || !Ep || !Hc || !Fc || !Ec) { free(P); return 100; }
    size_t q = 1;                    /* next path node to check (P[0] is the source) */
    int rc = 0;
    for (int64_t r = 0; r <= N && rc == 0; ++r) {
        /* fill row r into (Hc, Ec, Fc) */
        for (int64_t c = 0; c <= M; ++c) {
            int64_t e, f, h;
            if (r == 0 && c == 0) {
                e = (src == 1) ? 0 : NEG_INF; f = (src == 2) ? 0 : NEG_INF; h = 0;
            } else {
                e = (c == 0) ? NEG_INF : max2(Ec[c - 1] - ge, Hc[c - 1] - go);
                f = (r == 0) ? NEG_INF : max2(Fp[c] - ge, Hp[c] - go);
                int64_t d = (r == 0 || c == 0) ? NEG_INF
                          : Hp[c - 1] + subst(sub, alph, a[r - 1], b[c - 1]);
                h = max2(d, max2(e, f));
            }
            if (e < NEG_INF) e = NEG_INF;
            if (f < NEG_INF) f = NEG_INF;
            if (h < NEG_INF) h = NEG_INF;
            Ec[c] = e; Fc[c] = f; Hc[c] = h;
        }
        /* check the path nodes that lie in row r */
        while (q < np && P[q].i == r) {
            onode x = P[q];
            int64_t c = x.j;
            int64_t h = Hc[c], e = Ec[c], f = Fc[c];
            switch (x.how) {
            case 1: { int64_t d = Hp[c - 1] + subst(sub, alph, a[r - 1], b[c - 1]);
                      if (d != h) rc = 1; } break;
            case 2: { int64_t d = (r && c) ? Hp[c - 1] + subst(sub, alph, a[r - 1], b[c - 1]) : NEG_INF;
                      if (f != h || d >= h) rc = 2; } break;
            case 3: { int64_t d = (r && c) ? Hp[c - 1] + subst(sub, alph, a[r - 1], b[c - 1]) : NEG_INF;
                      if (e != h || d >= h || f >= h) rc = 3; } break;
            case 4: if (Hp[c] - go != f) rc = 4; break;
            case 5: if (Fp[c] - ge != f || Hp[c] - go >= f) rc = 5; break;
            case 6: if (Hc[c - 1] - go != e) rc = 6; break;
            case 7: if (Ec[c - 1] - ge != e || Hc[c - 1] - go >= e) rc = 7; break;
            default: rc = 8;
            }
            if (h <= NEG_INF / 2) rc = 9;
            ++q;
        }
        int64_t *t;
        t = Hp; Hp = Hc; Hc = t;
        t = Fp; Fp = Fc; Fc = t;
        t = Ep; Ep = Ec; Ec = t;
    }
    if (rc == 0 && q != np) rc = 10;
    free(P); free(Hp); free(Fp); free(Ep); free(Hc); free(Fc); free(Ec);
    return rc;
}

/* Full local H matrix ((n+1) x (m+1), row-major), for tiny cross-checks. */
int orc_local_matrix(const uint8_t *a, int64_t n, const uint8_t *b, int64_t m,
                     const int32_t *sub, int32_t alph, int32_t go, int32_t ge,
                     int64_t *Hout)
{
    size_t W = (size_t)(m + 1);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * W);
    if (!F) return -1;
    for (size_t j = 0; j < W; ++j) { Hout[j] = 0; F[j] = NEG_INF; }
    for (int64_t i = 1; i <= n; ++i) {
        int64_t e = NEG_INF;
        Hout[(size_t)i * W] = 0;
        for (int64_t j = 1; j <= m; ++j) {
            e = max2(e - ge, Hout[(size_t)i * W + j - 1] - go);
            F[j] = max2(F[j] - ge, Hout[(size_t)(i - 1) * W + j] - go);
            int64_t h = Hout[(size_t)(i - 1) * W + j - 1] + subst(sub, alph, a[i - 1], b[j - 1]);
            h = max2(max2(h, e), max2(F[j], 0));
            Hout[(size_t)i * W + j] = h;
        }
    }
    free(F);
    return 0;
}
