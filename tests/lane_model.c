/*
 * Host model of the packed lane words of the D->C Hungarian (test
 * infrastructure; the CUDA kernel is not compiled here).
 *
 * The device form solves each LAP (Sec. 4.1: one linear assignment problem
 * per concentration) with a warp: lane c % 32, slot c / 32 owns column c.
 * This model keeps the same words in arrays indexed by column and performs
 * the same word arithmetic modulo 2^32, step by step:
 *   key  = 64 (distance + D) + c        packed key, top bit set once labelled
 *   ruM  = 64 uM + rowOf + 1            matched row and its potential
 *   wv   = c - 64 v                     column potential
 *   z    = ruM - key + c                handed over by the winning column
 * with the sentinel column `sent` (outside the LAP) keyed at the largest
 * packed distance.  It is compared with the oracle's Hungarian method
 * (orc_lap) on random tiles: duals, assignment, steps and relaxations must be
 * equal; on tiles of arbitrary 32-bit entries it must stop (bounded).
 *
 * Usage: lane_model <trials> <seed>; prints one line and exits 0 when every
 * tile agreed and every run stopped.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int64_t orc_lap(int n, const int64_t *M, int64_t *u_out, int64_t *v_out, int32_t *col_of_row, int64_t *work,
                void *st);

#define MAXC 64

typedef struct {
    int rowOf[MAXC], u[MAXC], v[MAXC];
    unsigned steps, relax;
    int status;  /* 1 solved, 0 invariant failure reported, -1 did not stop */
} Result;

static Result model(const int *M, int ld, int n, int width, int dead0, int dead1, int sent, int NS)
{
    const unsigned kLab = 0x80000000u, kNone = 0x7fffffffu, kSentBase = ((1u << 25) - 1u) << 6;
    const int C = 32 * NS;
    Result R;
    memset(&R, 0, sizeof R);
    int valid[MAXC], way[MAXC];
    unsigned key[MAXC], key0[MAXC], ruM[MAXC], wv[MAXC];
    long long budget = 64LL * 64 * 64 * 8;  /* far above n (n + 1) steps and hops */
    for (int c = 0; c < C; ++c) {
        valid[c] = c < width && c != dead0 && c != dead1;
        key0[c] = c == sent ? (kSentBase | (unsigned)c) : kNone;
        ruM[c] = 0u;
        wv[c] = (unsigned)c;
        way[c] = -1;
    }
    int sumK = 0, sumK2 = 0;
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < C; ++c) key[c] = key0[c];
        unsigned r1 = (unsigned)r + 1u, q = 0u, mm = 0u;
        int j0 = -1;
        for (;;) {
            if (--budget < 0) { R.status = -1; return R; }
            const int *row = M + ((int)r1 - 1) * ld;
            for (int c = 0; c < C; ++c) {
                if (!valid[c]) continue;
                const unsigned ck = (unsigned)row[c] * 64u + (wv[c] - q);
                if ((int)ck < (int)key[c]) { key[c] = ck; way[c] = j0; }
            }
            /* each lane offers its smaller key and that slot's z; the warp's
               unsigned minimum picks the lane, the lane's word is handed over */
            unsigned lmin[32], z[32];
            for (int l = 0; l < 32; ++l) {
                int s = 0;
                if (NS == 2 && key[l + 32] < key[l]) s = 1;
                const int c = l + 32 * s;
                lmin[l] = key[c];
                z[l] = ruM[c] - key[c] + (unsigned)c;
            }
            mm = 0xffffffffu;
            for (int l = 0; l < 32; ++l) if (lmin[l] < mm) mm = lmin[l];
            const unsigned zw = z[mm & 31u];
            r1 = zw & 63u;
            if (r1 == 0u) break;
            for (int c = 0; c < C; ++c) if (key[c] == mm) key[c] |= kLab;
            q = zw & ~63u;
            j0 = (int)mm;
        }
        const int jf = (int)(mm & 63u);
        if (jf == sent) { R.status = 0; return R; }
        const unsigned Dend6 = mm & ~63u;
        int K = 1;
        for (int c = 0; c < C; ++c) {
            if ((int)key[c] >= 0) continue;
            ++K;
            const unsigned dd = Dend6 - (key[c] & (kLab - 64u));
            wv[c] += dd;
            ruM[c] += dd;
        }
        sumK += K;
        sumK2 += K * K;
        const unsigned root = Dend6 + (unsigned)r + 1u;
        int c = jf;
        for (int hop = 0;; ++hop) {
            if (hop > K) { R.status = 0; return R; }
            const int w = way[c];
            const int wc = (w & 31) + (NS == 2 ? 32 * ((w >> 5) & 1) : 0);  /* the lane and slot read */
            ruM[c] = w >= 0 ? ruM[wc] : root;
            if (w < 0) break;
            c = w & 63;
        }
    }
    for (int c = 0; c < C; ++c) {
        R.rowOf[c] = (int)(ruM[c] & 63u) - 1;
        R.u[c] = (int)(ruM[c] & ~63u) >> 6;
        R.v[c] = (int)((unsigned)c - wv[c]) >> 6;
    }
    R.steps = (unsigned)sumK;
    R.relax = (unsigned)(n * sumK - (sumK2 - sumK) / 2);
    R.status = 1;
    return R;
}

static uint64_t rng_state;
static uint64_t next(void)
{
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}

int main(int argc, char **argv)
{
    const long trials = argc > 1 ? atol(argv[1]) : 10000;
    rng_state = 0x9e3779b97f4a7c15ull ^ (uint64_t)(argc > 2 ? atol(argv[2]) : 1);
    static int M[64 * 64];
    static int64_t Mo[64 * 64];
    long checked = 0, garbage = 0, wrong = 0, unbounded = 0;
    const int limit = (1 << 25) / 3 - 1;  /* largest entry the packed keys take */
    for (long t = 0; t < trials; ++t) {
        const int kind = (int)(next() % 6);
        const int dead = (int)(next() % 2);  /* D->C tile with two dead columns, or a full LAP */
        int NS = 1 + (int)(next() % 2), width, n, d0 = -1, d1 = -1, sent;
        if (dead) {
            width = NS == 1 ? 3 + (int)(next() % 30) : 32 + (int)(next() % 33);  /* 3..32 / 32..64 */
            n = width - 2;
            d0 = (int)(next() % width);
            d1 = (int)(next() % width);
            if (d1 == d0) d1 = (d0 + 1) % width;
            sent = d0;
        } else {
            width = NS == 1 ? 1 + (int)(next() % 31) : 32 + (int)(next() % 32);  /* 1..31 / 32..63 */
            n = width;
            sent = 32 * NS - 1;
        }
        const int A = kind == 0 ? 2 : kind == 1 ? 100 : kind == 2 ? 100000 : limit;
        const int ld = 64;
        for (int e = 0; e < 64 * 64; ++e) M[e] = (int)(next() & 0x7fffffffu);  /* garbage outside the LAP */
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < width; ++c) {
                unsigned x = (unsigned)(next() % ((uint64_t)A + 1));
                if (kind == 4) x = (unsigned)limit - (unsigned)(next() % 4);
                if (kind == 5) x = (unsigned)next();
                M[r * ld + c] = (int)x;
            }
        const Result R = model(M, ld, n, width, d0, d1, sent, NS);
        if (R.status < 0) { ++unbounded; continue; }
        if (kind == 5) { ++garbage; continue; }
        int cols[64], k = 0;
        for (int c = 0; c < width; ++c) if (c != d0 && c != d1) cols[k++] = c;
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) Mo[r * n + c] = M[r * ld + cols[c]];
        int64_t u[64], v[64], work[3] = {0, 0, 0};
        int32_t col_of_row[64];
        orc_lap(n, Mo, u, v, col_of_row, work, NULL);
        int ok = R.status == 1 && (int64_t)R.steps == work[0] && (int64_t)R.relax == work[1];
        for (int c = 0; ok && c < n; ++c) {
            const int col = cols[c], row = R.rowOf[col];
            ok = row >= 0 && row < n && R.v[col] == v[c] && R.u[col] == u[row] && col_of_row[row] == c;
        }
        if (!ok && wrong < 5)
            fprintf(stderr, "disagrees: trial %ld, width %d, n %d, slots %d, kind %d\n", t, width, n, NS, kind);
        wrong += !ok;
        ++checked;
    }
    printf("checked %ld, garbage %ld, disagree %ld, unbounded %ld\n", checked, garbage, wrong, unbounded);
    return wrong || unbounded ? 1 : 0;
}
