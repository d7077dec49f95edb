/*
 * rlt2_oracle.c -- TEST INFRASTRUCTURE, not part of the product path.
 *
 * A plain, slow, single-threaded CPU restatement of the level-2 RLT (RLT2)
 * dual ascent for the Koopmans-Beckmann QAP (Algorithm 1 of Goncalves,
 * Pessoa, Drummond, Bentes, Farias, arXiv:1510.02065), in int64.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, header, table or helper with the
 * CUDA library: it is the independent definition the CUDA path is checked
 * against.
 *
 * Storage is the plainest possible: the reduced costs are dense arrays
 * indexed by the paper's own subscripts,
 *     b[i][j]               (matrix B, N x N)
 *     c[i][j][k][n]         (matrix C; only i!=k, j!=n are meaningful)
 *     d[i][j][k][n][p][q]   (matrix D; only distinct i,k,p and distinct j,n,q)
 * with every meaningless entry held at 0.
 *
 * Readings of passages the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   R1  rows and columns of every submatrix are taken in ascending index order;
 *   R2  one iteration runs the seven operations in the order of Algorithm 1;
 *   R3  a cost spread over m rows (Sec. 4.2 divides by N-1 and N-2) is split
 *       into integers: q = floor(x/m), r = x mod m, and the t-th row
 *       (ascending, t = 0..m-1) receives q + [t < r].  Every row of the
 *       submatrix gets the same increment on all its columns, so the cost of
 *       every feasible solution is kept exactly;
 *   R4  the transfer between complementary costs (Sec. 4.3) is the equal split
 *       of the class sum T: the member of lexicographic rank t (t = 0..s-1,
 *       s = 2 for C, 6 for D) receives floor(T/s) + [t < T mod s];
 *   R5  the "residual coefficients" of a concentration (Sec. 4.1) are the
 *       reduced costs M[r][s] - u[r] - v[s] under the duals of the Hungarian
 *       method below;
 *   R6  the Hungarian method is the shortest-augmenting-path form with row and
 *       column potentials: u = v = 0 at the start, rows inserted in ascending
 *       order, the next column is the unlabelled one of least reduced
 *       distance with ties going to the smallest column index, a distance
 *       label (and its predecessor) changes only on a strict improvement.
 *   R13 (paired mode, the complementary submatrices of Sec. 6) each
 *       coefficient (d_ijkn)_pq has the complementary coefficient
 *       (d_knij)_pq (the same variable by the symmetry constraints), so the
 *       pair is kept as one sum in the submatrix with i < k and the other is
 *       held at 0: spreading C -> D adds the shares of c_knij to D_ijkn
 *       (same rows p, same ranks); the transfer between complementary costs
 *       of D splits a class sum over its three members of that kind,
 *       d_ijknpq, d_ijpqkn, d_knpqij (i < k < p, lexicographic order), equally
 *       as in R4 with s = 3; and D -> C concentrates only the submatrices
 *       with i < k, adding S to c_ijkn.  Half of D and half of the D -> C LAPs
 *       remain; the bound differs from the full form (a LAP of a sum is at
 *       least the sum of the LAPs).
 *   R14 (FP64 form, the orf_* functions) the paper's real division: a cost x
 *       spread over m rows adds x/m (one IEEE double division, the same
 *       quotient for every row) to each coefficient of the submatrix; a class
 *       of s complementary costs is summed in lexicographic rank order and
 *       every member becomes T/s; costs, potentials and LB are doubles, and
 *       every sum is formed in the order written below (rows and columns
 *       ascending, left to right), so that the result is one defined double.
 *
 * Parity pins for every function live in tests/ (N!-enumeration and scipy for
 * the LAP, brute-force QAP optima, the conservation identity
 * Q(pi) = LB + sum of reduced costs along pi, non-negativity, monotone LB, and
 * the Gilmore-Lawler bound in RLT1 mode).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_INF INT64_MAX

typedef struct {
    int N;
    int rlt1_only;     /* strong-branching dual of Sec. 6: Algorithm 1 without D */
    int paired;        /* complementary submatrices of Sec. 6 kept as one (reading R13) */
    int64_t LB;
    int64_t iters;
    int64_t *b, *c, *d;
    /* work counters of the Hungarian method, summed over all LAPs solved */
    int64_t laps, steps, relaxations;
    int64_t max_abs;   /* largest |value| seen in a potential, label or cost */
} orc_state;

/* ---------------------------------------------------------------- indexing */

static inline size_t ix2(int N, int i, int j) { return (size_t)i * N + j; }
static inline size_t ix4(int N, int i, int j, int k, int n)
{
    return (((size_t)i * N + j) * N + k) * N + n;
}
static inline size_t ix6(int N, int i, int j, int k, int n, int p, int q)
{
    return (((((size_t)i * N + j) * N + k) * N + n) * N + p) * N + q;
}

static inline void track(orc_state *st, int64_t x)
{
    int64_t a = x < 0 ? -x : x;
    if (st && a > st->max_abs) st->max_abs = a;
}

/* ------------------------------------------------------- Hungarian method */

/*
 * Linear assignment by the Hungarian method (Sec. 4.1 names Munkres' method
 * for each concentration; the variant is fixed by reading R6).
 *
 *   n            size of the square cost matrix M (row-major, n*n, entries >= 0)
 *   u_out[n]     row potentials, v_out[n] column potentials (may be NULL)
 *   col_of_row   assignment sigma: row r -> column col_of_row[r] (may be NULL)
 *   work[3]      += {steps, relaxations, 1} (may be NULL)
 * Returns S = sum_r M[r][sigma(r)], the optimal assignment cost.
 *
 * Column index n is a virtual column that holds the row being inserted.  A
 * "step" labels one column; a "relaxation" is one evaluation of a reduced
 * distance M[i0][j] - u[i0] - v[j] for an unlabelled column j.
 */
int64_t orc_lap(int n, const int64_t *M, int64_t *u_out, int64_t *v_out,
                int32_t *col_of_row, int64_t *work, orc_state *st)
{
    int64_t *u = calloc((size_t)n + 1, sizeof(int64_t));   /* per row     */
    int64_t *v = calloc((size_t)n + 1, sizeof(int64_t));   /* per column  */
    int64_t *dist = malloc(((size_t)n + 1) * sizeof(int64_t));
    int *row_at = malloc(((size_t)n + 1) * sizeof(int));    /* row matched to column */
    int *pred = malloc(((size_t)n + 1) * sizeof(int));      /* previous column on path */
    char *labelled = malloc((size_t)n + 1);
    int64_t steps = 0, relax = 0;

    for (int j = 0; j <= n; j++) row_at[j] = -1;

    for (int r = 0; r < n; r++) {
        const int root = n;               /* virtual column carrying row r */
        row_at[root] = r;
        for (int j = 0; j <= n; j++) { dist[j] = ORC_INF; labelled[j] = 0; }
        int col = root;                   /* last labelled column */
        for (;;) {
            labelled[col] = 1;
            const int i0 = row_at[col];   /* its row is scanned once */
            int64_t delta = ORC_INF;
            int next = -1;
            steps++;
            for (int j = 0; j < n; j++) {
                if (labelled[j]) continue;
                relax++;
                int64_t red = M[(size_t)i0 * n + j] - u[i0] - v[j];
                track(st, red);
                if (red < dist[j]) { dist[j] = red; pred[j] = col; }
                if (dist[j] < delta) { delta = dist[j]; next = j; }
            }
            /* move the potentials by delta: labelled columns and their rows
             * (the tree) keep their reduced costs, the rest get closer */
            for (int j = 0; j <= n; j++) {
                if (labelled[j]) {
                    u[row_at[j]] += delta;
                    v[j] -= delta;
                    track(st, u[row_at[j]]);
                    track(st, v[j]);
                } else {
                    dist[j] -= delta;
                }
            }
            col = next;
            if (row_at[col] < 0) break;   /* free column: augmenting path found */
        }
        /* augment: every column on the path takes the row of its predecessor */
        while (col != root) {
            int p = pred[col];
            row_at[col] = row_at[p];
            col = p;
        }
    }

    int64_t S = 0;
    for (int j = 0; j < n; j++) {
        int r = row_at[j];
        S += M[(size_t)r * n + j];
        if (col_of_row) col_of_row[r] = j;
    }
    if (u_out) for (int r = 0; r < n; r++) u_out[r] = u[r];
    if (v_out) for (int j = 0; j < n; j++) v_out[j] = v[j];
    if (work) { work[0] += steps; work[1] += relax; work[2] += 1; }
    if (st) { st->steps += steps; st->relaxations += relax; st->laps += 1; }
    free(u); free(v); free(dist); free(row_at); free(pred); free(labelled);
    return S;
}

/* Batch form for tests: count matrices of n*n, outputs per matrix. */
void orc_lap_batch(int n, int count, const int64_t *M, int64_t *S,
                   int64_t *u, int64_t *v, int32_t *col_of_row, int64_t *work)
{
    for (int t = 0; t < count; t++)
        S[t] = orc_lap(n, M + (size_t)t * n * n, u ? u + (size_t)t * n : NULL,
                       v ? v + (size_t)t * n : NULL,
                       col_of_row ? col_of_row + (size_t)t * n : NULL,
                       work ? work + (size_t)t * 3 : NULL, NULL);
}

/* ------------------------------------------------------------ state setup */

/*
 * Initialisation of Algorithm 1: LB <- lb_const, b_ij <- linear cost (B_lin,
 * or 0), c_ijkn <- f_ik * d_jn for i != k and j != n, d <- 0.
 * F, D: N x N row-major flow and distance matrices (Eq. (1)).
 */
orc_state *orc_create(int N, const int32_t *F, const int32_t *Dist,
                      const int64_t *B_lin, int64_t lb_const, int rlt1_only)
{
    if (N < 3) return NULL;
    orc_state *st = calloc(1, sizeof(orc_state));
    st->N = N;
    st->rlt1_only = rlt1_only;
    st->paired = 0;
    st->LB = lb_const;
    size_t n2 = (size_t)N * N, n4 = n2 * n2;
    st->b = calloc(n2, sizeof(int64_t));
    st->c = calloc(n4, sizeof(int64_t));
    if (!rlt1_only) st->d = calloc(n4 * n2, sizeof(int64_t));
    if (!st->b || !st->c || (!rlt1_only && !st->d)) {
        free(st->b); free(st->c); free(st->d); free(st);
        return NULL;
    }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            st->b[ix2(N, i, j)] = B_lin ? B_lin[ix2(N, i, j)] : 0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++)
                for (int n = 0; n < N; n++)
                    if (k != i && n != j)
                        st->c[ix4(N, i, j, k, n)] =
                            (int64_t)F[ix2(N, i, k)] * (int64_t)Dist[ix2(N, j, n)];
    return st;
}

/* Switch a freshly created state to the paired form of reading R13. */
void orc_set_paired(orc_state *st, int paired) { st->paired = paired; }

void orc_destroy(orc_state *st)
{
    if (!st) return;
    free(st->b); free(st->c); free(st->d); free(st);
}

/* -------------------------------------------------------- cost spreading */

/* The t-th of m rows receives floor(x/m) + [t < x mod m]  (reading R3). */
static inline int64_t row_share(int64_t x, int m, int t)
{
    return x / m + (t < x % m ? 1 : 0);
}

/*
 * Costs spreading from B to C (Sec. 4.2): b_ij is spread over the N-1 rows
 * k != i of the submatrix C_ij, every c_ijkn (n != j) of a row receiving that
 * row's share; then b_ij = 0.
 */
void orc_spread_B_to_C(orc_state *st)
{
    const int N = st->N, m = N - 1;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int64_t x = st->b[ix2(N, i, j)];
            int t = 0;
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                int64_t sh = row_share(x, m, t++);
                for (int n = 0; n < N; n++)
                    if (n != j) st->c[ix4(N, i, j, k, n)] += sh;
            }
            st->b[ix2(N, i, j)] = 0;
        }
}

/*
 * Costs spreading from C to D (Sec. 4.2): c_ijkn is spread over the N-2 rows
 * p not in {i,k} of the submatrix D_ijkn, every d_ijknpq (q not in {j,n}) of
 * a row receiving that row's share; then c_ijkn = 0.
 * Only first indices i in [i_lo, i_hi) are processed (the whole operation is
 * [0, N)); the range exists so that a time-bounded sample can be measured.
 */
void orc_spread_C_to_D_range(orc_state *st, int i_lo, int i_hi)
{
    const int N = st->N, m = N - 2;
    for (int i = i_lo; i < i_hi; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    int64_t x = st->c[ix4(N, i, j, k, n)];
                    /* paired (R13): the shares of c_knij (k < i) go to D_ijkn's complement */
                    const int up = !st->paired || i < k;
                    int t = 0;
                    for (int p = 0; p < N; p++) {
                        if (p == i || p == k) continue;
                        int64_t sh = row_share(x, m, t++);
                        for (int q = 0; q < N; q++) {
                            if (q == j || q == n) continue;
                            if (up) st->d[ix6(N, i, j, k, n, p, q)] += sh;
                            else st->d[ix6(N, k, n, i, j, p, q)] += sh;
                        }
                    }
                    st->c[ix4(N, i, j, k, n)] = 0;
                }
            }
}

void orc_spread_C_to_D(orc_state *st) { orc_spread_C_to_D_range(st, 0, st->N); }

/* ------------------------------------------- complementary cost transfer */

/*
 * Transfer between complementary costs of D (Sec. 4.3, the six coefficients of
 * Eq. (11)).  A class is an unordered set of three pairs (i,j),(k,n),(p,q)
 * with distinct facilities and distinct locations; it is visited once, with
 * its facilities sorted i < k < p.  Its six members, in lexicographic order of
 * their index 6-tuples (the facilities are distinct, so the order is decided
 * by the first two facilities), are
 *   d_ijknpq < d_ijpqkn < d_knijpq < d_knpqij < d_pqijkn < d_pqknij.
 * The class sum T is re-split equally (reading R4).
 * Only smallest facilities i in [i_lo, i_hi) are processed.
 */
void orc_complementary_D_range(orc_state *st, int i_lo, int i_hi)
{
    const int N = st->N;
    int64_t *d = st->d;
    for (int i = i_lo; i < i_hi; i++)
        for (int k = i + 1; k < N; k++)
            for (int p = k + 1; p < N; p++)
                for (int j = 0; j < N; j++)
                    for (int n = 0; n < N; n++) {
                        if (n == j) continue;
                        for (int q = 0; q < N; q++) {
                            if (q == j || q == n) continue;
                            size_t mem[6] = {
                                ix6(N, i, j, k, n, p, q), ix6(N, i, j, p, q, k, n),
                                ix6(N, k, n, i, j, p, q), ix6(N, k, n, p, q, i, j),
                                ix6(N, p, q, i, j, k, n), ix6(N, p, q, k, n, i, j)};
                            int64_t T = 0;
                            for (int t = 0; t < 6; t++) T += d[mem[t]];
                            track(st, T);
                            if (!st->paired) {
                                for (int t = 0; t < 6; t++) d[mem[t]] = T / 6 + (t < T % 6 ? 1 : 0);
                            } else {
                                /* R13: the members with first facility below the second,
                                 * d_ijknpq, d_ijpqkn, d_knpqij, share T; the others stay 0 */
                                const int upper[3] = {0, 1, 3}, lower[3] = {2, 4, 5};
                                for (int t = 0; t < 3; t++) {
                                    d[mem[upper[t]]] = T / 3 + (t < T % 3 ? 1 : 0);
                                    d[mem[lower[t]]] = 0;
                                }
                            }
                        }
                    }
}

void orc_complementary_D(orc_state *st) { orc_complementary_D_range(st, 0, st->N); }

/*
 * Transfer between complementary costs of C (Sec. 4.3, Eq. (10)): the pair
 * c_ijkn, c_knij with i < k (the first in lexicographic order) is re-split
 * equally, the first member taking the odd unit (reading R4).
 */
void orc_complementary_C(orc_state *st)
{
    const int N = st->N;
    for (int i = 0; i < N; i++)
        for (int k = i + 1; k < N; k++)
            for (int j = 0; j < N; j++)
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    int64_t T = st->c[ix4(N, i, j, k, n)] + st->c[ix4(N, k, n, i, j)];
                    st->c[ix4(N, i, j, k, n)] = T / 2 + T % 2;
                    st->c[ix4(N, k, n, i, j)] = T / 2;
                }
}

/* ------------------------------------------------------ cost concentration */

/*
 * Cost concentration from D to C (Sec. 4.1): for each (i,j,k,n) with i != k,
 * j != n, M_rs = d_ijkn p_r q_s over the (N-2) x (N-2) submatrix D_ijkn
 * (p_r: r-th row not in {i,k}, q_s: s-th column not in {j,n}); S = LAP(M) is
 * added to c_ijkn and D_ijkn is replaced by M's residual coefficients
 * (reading R5).  Only first indices i in [i_lo, i_hi) are processed.
 */
void orc_concentrate_D_to_C_range(orc_state *st, int i_lo, int i_hi)
{
    const int N = st->N, m = N - 2;
    int64_t *M = malloc((size_t)m * m * sizeof(int64_t));
    int64_t *u = malloc((size_t)m * sizeof(int64_t));
    int64_t *v = malloc((size_t)m * sizeof(int64_t));
    int rows[64], cols[64];
    for (int i = i_lo; i < i_hi; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                if (st->paired && k < i) continue;  /* R13: the complement holds the pair */
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    int r = 0, s = 0;
                    for (int p = 0; p < N; p++) if (p != i && p != k) rows[r++] = p;
                    for (int q = 0; q < N; q++) if (q != j && q != n) cols[s++] = q;
                    for (r = 0; r < m; r++)
                        for (s = 0; s < m; s++)
                            M[r * m + s] = st->d[ix6(N, i, j, k, n, rows[r], cols[s])];
                    int64_t S = orc_lap(m, M, u, v, NULL, NULL, st);
                    st->c[ix4(N, i, j, k, n)] += S;
                    for (r = 0; r < m; r++)
                        for (s = 0; s < m; s++)
                            st->d[ix6(N, i, j, k, n, rows[r], cols[s])] = M[r * m + s] - u[r] - v[s];
                }
            }
    free(M); free(u); free(v);
}

void orc_concentrate_D_to_C(orc_state *st) { orc_concentrate_D_to_C_range(st, 0, st->N); }

/*
 * Cost concentration from C to B (Sec. 4.1): for each (i,j), the
 * (N-1) x (N-1) submatrix C_ij (rows k != i, columns n != j); b_ij += S and
 * C_ij is replaced by its residual coefficients.
 */
void orc_concentrate_C_to_B(orc_state *st)
{
    const int N = st->N, m = N - 1;
    int64_t *M = malloc((size_t)m * m * sizeof(int64_t));
    int64_t *u = malloc((size_t)m * sizeof(int64_t));
    int64_t *v = malloc((size_t)m * sizeof(int64_t));
    int rows[64], cols[64];
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int r = 0, s = 0;
            for (int k = 0; k < N; k++) if (k != i) rows[r++] = k;
            for (int n = 0; n < N; n++) if (n != j) cols[s++] = n;
            for (r = 0; r < m; r++)
                for (s = 0; s < m; s++)
                    M[r * m + s] = st->c[ix4(N, i, j, rows[r], cols[s])];
            int64_t S = orc_lap(m, M, u, v, NULL, NULL, st);
            st->b[ix2(N, i, j)] += S;
            for (r = 0; r < m; r++)
                for (s = 0; s < m; s++)
                    st->c[ix4(N, i, j, rows[r], cols[s])] = M[r * m + s] - u[r] - v[s];
        }
    free(M); free(u); free(v);
}

/*
 * Cost concentration from B to LB (Sec. 4.1): S = LAP(B) is the increment
 * LB' of Algorithm 1; B is replaced by its residual coefficients.
 */
int64_t orc_concentrate_B_to_LB(orc_state *st)
{
    const int N = st->N;
    int64_t *u = malloc((size_t)N * sizeof(int64_t));
    int64_t *v = malloc((size_t)N * sizeof(int64_t));
    int64_t *M = malloc((size_t)N * N * sizeof(int64_t));
    memcpy(M, st->b, (size_t)N * N * sizeof(int64_t));
    int64_t S = orc_lap(N, M, u, v, NULL, NULL, st);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            st->b[ix2(N, i, j)] = M[i * N + j] - u[i] - v[j];
    free(u); free(v); free(M);
    return S;
}

/* -------------------------------------------------------------- Algorithm 1 */

/*
 * One pass of the loop of Algorithm 1 (reading R2): spread B->C, spread C->D,
 * complementary D, concentrate D->C, complementary C, concentrate C->B,
 * concentrate B->LB, LB += LB'.  In RLT1 mode (Sec. 6, strong branching) the
 * three operations on D are skipped.  Returns LB after the pass.
 */
int64_t orc_iterate(orc_state *st)
{
    orc_spread_B_to_C(st);
    if (!st->rlt1_only) {
        orc_spread_C_to_D(st);
        orc_complementary_D(st);
        orc_concentrate_D_to_C(st);
    }
    orc_complementary_C(st);
    orc_concentrate_C_to_B(st);
    st->LB += orc_concentrate_B_to_LB(st);
    st->iters++;
    return st->LB;
}

/* Run k passes; hist (may be NULL) receives LB after each. */
void orc_run(orc_state *st, int k, int64_t *hist)
{
    for (int t = 0; t < k; t++) {
        int64_t lb = orc_iterate(st);
        if (hist) hist[t] = lb;
    }
}

/* ----------------------------------------------------------------- access */

int orc_N(const orc_state *st) { return st->N; }
int64_t orc_LB(const orc_state *st) { return st->LB; }
int64_t *orc_b(orc_state *st) { return st->b; }
int64_t *orc_c(orc_state *st) { return st->c; }
int64_t *orc_d(orc_state *st) { return st->d; }
void orc_work(const orc_state *st, int64_t *out4)
{
    out4[0] = st->laps; out4[1] = st->steps; out4[2] = st->relaxations; out4[3] = st->max_abs;
}

/* ----------------------------------------------- branch-and-bound subproblem */

/*
 * Residual instance of a branch-and-bound node (Sec. 6): facilities fac[t] are
 * fixed to locations loc[t], t < kfix.  The free facilities and free locations
 * are renumbered in ascending order (N' = N - kfix).  For any completion pi',
 *   Q(full pi) = const + sum_x Blin[x][pi'(x)] + sum_{x != y} F'[x][y] D'[pi'(x)][pi'(y)]
 * with
 *   F'[x][y]  = F[fx][fy],  D'[x][y] = D[lx][ly],
 *   Blin[x][y] = sum_t F[fx][a_t] D[ly][l_t] + F[a_t][fx] D[l_t][ly],
 *   const     = sum_{t != t'} F[a_t][a_t'] D[l_t][l_t'].
 * Outputs: Fp, Dp (N'*N' int32), Blin (N'*N' int64), *cst.  Returns N'.
 */
int orc_subproblem(int N, const int32_t *F, const int32_t *Dist, int kfix,
                   const int32_t *fac, const int32_t *loc,
                   int32_t *Fp, int32_t *Dp, int64_t *Blin, int64_t *cst)
{
    int ff[64], fl[64], nf = 0, nl = 0;
    for (int a = 0; a < N; a++) {
        int fixed = 0;
        for (int t = 0; t < kfix; t++) if (fac[t] == a) fixed = 1;
        if (!fixed) ff[nf++] = a;
    }
    for (int l = 0; l < N; l++) {
        int fixed = 0;
        for (int t = 0; t < kfix; t++) if (loc[t] == l) fixed = 1;
        if (!fixed) fl[nl++] = l;
    }
    const int Np = nf;
    for (int x = 0; x < Np; x++)
        for (int y = 0; y < Np; y++) {
            Fp[x * Np + y] = F[ix2(N, ff[x], ff[y])];
            Dp[x * Np + y] = Dist[ix2(N, fl[x], fl[y])];
            int64_t s = 0;
            for (int t = 0; t < kfix; t++)
                s += (int64_t)F[ix2(N, ff[x], fac[t])] * Dist[ix2(N, fl[y], loc[t])] +
                     (int64_t)F[ix2(N, fac[t], ff[x])] * Dist[ix2(N, loc[t], fl[y])];
            Blin[x * Np + y] = s;
        }
    int64_t c0 = 0;
    for (int t = 0; t < kfix; t++)
        for (int t2 = 0; t2 < kfix; t2++)
            if (t != t2) c0 += (int64_t)F[ix2(N, fac[t], fac[t2])] * Dist[ix2(N, loc[t], loc[t2])];
    *cst = c0;
    return Np;
}

/*
 * Warm start of a branch-and-bound child (the node of the parent fixing
 * facility f to location l).  The conservation identity of the parent,
 *   Q(pi) = LB + sum_i b_{i pi_i} + sum_{i!=k} c_{i pi_i k pi_k}
 *              + sum_{distinct i,k,p} d_{i pi_i k pi_k p pi_p},
 * restricted to the permutations with pi(f) = l splits into the child's terms
 * over the other facilities and locations (renumbered in ascending order):
 *   LB'      = LB + b_fl
 *   b'_kn    = b_kn + c_flkn + c_knfl
 *   c'_knpq  = c_knpq + d_flknpq + d_knflpq + d_knpqfl
 *   d'       = d over the free indices,
 * all sums of reduced costs, so >= 0, and the child's dual ascent starts from
 * LB' >= LB instead of from 0.  (The paper is silent on how a node's bound is
 * started; this is the warm-started variant of reading R10.)  The child keeps
 * the parent's paired flag (the pair sums stay in the tiles with i < k).
 * Returns NULL for N < 4 or on allocation failure.
 */
orc_state *orc_child(const orc_state *par, int f, int l)
{
    const int N = par->N, M = N - 1;
    if (M < 3 || f < 0 || f >= N || l < 0 || l >= N) return NULL;
    orc_state *st = calloc(1, sizeof(orc_state));
    if (!st) return NULL;
    st->N = M;
    st->rlt1_only = par->rlt1_only;
    st->paired = par->paired;
    size_t m2 = (size_t)M * M, m4 = m2 * m2;
    st->b = calloc(m2, sizeof(int64_t));
    st->c = calloc(m4, sizeof(int64_t));
    if (!par->rlt1_only) st->d = calloc(m4 * m2, sizeof(int64_t));
    if (!st->b || !st->c || (!par->rlt1_only && !st->d)) {
        free(st->b); free(st->c); free(st->d); free(st);
        return NULL;
    }
    int fa[64], lo[64];  /* child index -> parent index */
    for (int x = 0, a = 0; a < N; a++) if (a != f) fa[x++] = a;
    for (int x = 0, a = 0; a < N; a++) if (a != l) lo[x++] = a;
    st->LB = par->LB + par->b[ix2(N, f, l)];
    for (int x = 0; x < M; x++)
        for (int y = 0; y < M; y++) {
            const int k = fa[x], n = lo[y];
            st->b[ix2(M, x, y)] = par->b[ix2(N, k, n)] + par->c[ix4(N, f, l, k, n)] + par->c[ix4(N, k, n, f, l)];
        }
    for (int x = 0; x < M; x++)
        for (int y = 0; y < M; y++)
            for (int u = 0; u < M; u++)
                for (int w = 0; w < M; w++) {
                    if (u == x || w == y) continue;
                    const int k = fa[x], n = lo[y], p = fa[u], q = lo[w];
                    int64_t v = par->c[ix4(N, k, n, p, q)];
                    if (par->d)
                        v += par->d[ix6(N, f, l, k, n, p, q)] + par->d[ix6(N, k, n, f, l, p, q)] +
                             par->d[ix6(N, k, n, p, q, f, l)];
                    st->c[ix4(M, x, y, u, w)] = v;
                }
    if (st->d)
        for (int x = 0; x < M; x++)
            for (int y = 0; y < M; y++)
                for (int u = 0; u < M; u++)
                    for (int w = 0; w < M; w++)
                        for (int r = 0; r < M; r++)
                            for (int z = 0; z < M; z++)
                                st->d[ix6(M, x, y, u, w, r, z)] =
                                    par->d[ix6(N, fa[x], lo[y], fa[u], lo[w], fa[r], lo[z])];
    return st;
}

/* LB <- LB + x (the last line of the loop of Algorithm 1, for step-wise use). */
void orc_add_LB(orc_state *st, int64_t x) { st->LB += x; }

/* ====================================================== FP64 form (R14) */

/*
 * The same dual ascent with double costs and the paper's real division
 * (Sec. 4.2 divides a cost by N-1 or N-2; Sec. 4.3 re-splits a class sum).
 * Storage as in the int64 form: b[i][j], c[i][j][k][n], d[i][j][k][n][p][q].
 */
typedef struct {
    int N;
    int rlt1_only;
    double LB;
    int64_t iters;
    double *b, *c, *d;
    int64_t laps, steps, relaxations;
} orf_state;

/*
 * Hungarian method in doubles: the steps of orc_lap (reading R6), every
 * reduced distance formed as (M[i0][j] - u[i0]) - v[j], the potentials moved
 * by delta after every step.  Returns S = sum over columns j = 0..n-1 (in that
 * order, from 0) of M[row of j][j].
 */
double orf_lap(int n, const double *M, double *u_out, double *v_out,
               int32_t *col_of_row, int64_t *work, orf_state *st)
{
    double *u = calloc((size_t)n + 1, sizeof(double));
    double *v = calloc((size_t)n + 1, sizeof(double));
    double *dist = malloc(((size_t)n + 1) * sizeof(double));
    int *row_at = malloc(((size_t)n + 1) * sizeof(int));
    int *pred = malloc(((size_t)n + 1) * sizeof(int));
    char *labelled = malloc((size_t)n + 1);
    int64_t steps = 0, relax = 0;

    for (int j = 0; j <= n; j++) row_at[j] = -1;

    for (int r = 0; r < n; r++) {
        const int root = n;
        row_at[root] = r;
        for (int j = 0; j <= n; j++) { dist[j] = INFINITY; labelled[j] = 0; }
        int col = root;
        for (;;) {
            labelled[col] = 1;
            const int i0 = row_at[col];
            double delta = INFINITY;
            int next = -1;
            steps++;
            for (int j = 0; j < n; j++) {
                if (labelled[j]) continue;
                relax++;
                double red = M[(size_t)i0 * n + j] - u[i0] - v[j];
                if (red < dist[j]) { dist[j] = red; pred[j] = col; }
                if (dist[j] < delta) { delta = dist[j]; next = j; }
            }
            for (int j = 0; j <= n; j++) {
                if (labelled[j]) {
                    u[row_at[j]] += delta;
                    v[j] -= delta;
                } else {
                    dist[j] -= delta;
                }
            }
            col = next;
            if (row_at[col] < 0) break;
        }
        while (col != root) {
            int p = pred[col];
            row_at[col] = row_at[p];
            col = p;
        }
    }

    double S = 0.0;
    for (int j = 0; j < n; j++) {
        int r = row_at[j];
        S += M[(size_t)r * n + j];
        if (col_of_row) col_of_row[r] = j;
    }
    if (u_out) for (int r = 0; r < n; r++) u_out[r] = u[r];
    if (v_out) for (int j = 0; j < n; j++) v_out[j] = v[j];
    if (work) { work[0] += steps; work[1] += relax; work[2] += 1; }
    if (st) { st->steps += steps; st->relaxations += relax; st->laps += 1; }
    free(u); free(v); free(dist); free(row_at); free(pred); free(labelled);
    return S;
}

void orf_lap_batch(int n, int count, const double *M, double *S,
                   double *u, double *v, int32_t *col_of_row, int64_t *work)
{
    for (int t = 0; t < count; t++)
        S[t] = orf_lap(n, M + (size_t)t * n * n, u ? u + (size_t)t * n : NULL,
                       v ? v + (size_t)t * n : NULL,
                       col_of_row ? col_of_row + (size_t)t * n : NULL,
                       work ? work + (size_t)t * 3 : NULL, NULL);
}

/* Initialisation of Algorithm 1 in doubles (c_ijkn = f_ik d_jn exactly). */
orf_state *orf_create(int N, const int32_t *F, const int32_t *Dist,
                      const double *B_lin, double lb_const, int rlt1_only)
{
    if (N < 3) return NULL;
    orf_state *st = calloc(1, sizeof(orf_state));
    st->N = N;
    st->rlt1_only = rlt1_only;
    st->LB = lb_const;
    size_t n2 = (size_t)N * N, n4 = n2 * n2;
    st->b = calloc(n2, sizeof(double));
    st->c = calloc(n4, sizeof(double));
    if (!rlt1_only) st->d = calloc(n4 * n2, sizeof(double));
    if (!st->b || !st->c || (!rlt1_only && !st->d)) {
        free(st->b); free(st->c); free(st->d); free(st);
        return NULL;
    }
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            st->b[ix2(N, i, j)] = B_lin ? B_lin[ix2(N, i, j)] : 0.0;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++)
                for (int n = 0; n < N; n++)
                    if (k != i && n != j)
                        st->c[ix4(N, i, j, k, n)] =
                            (double)((int64_t)F[ix2(N, i, k)] * (int64_t)Dist[ix2(N, j, n)]);
    return st;
}

void orf_destroy(orf_state *st)
{
    if (!st) return;
    free(st->b); free(st->c); free(st->d); free(st);
}

/* Spreading B -> C (Sec. 4.2): every c_ijkn (k != i, n != j) += b_ij / (N-1). */
void orf_spread_B_to_C(orf_state *st)
{
    const int N = st->N;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            const double sh = st->b[ix2(N, i, j)] / (double)(N - 1);
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                for (int n = 0; n < N; n++)
                    if (n != j) st->c[ix4(N, i, j, k, n)] += sh;
            }
            st->b[ix2(N, i, j)] = 0.0;
        }
}

/* Spreading C -> D (Sec. 4.2): every d_ijknpq (p not in {i,k}, q not in {j,n})
 * += c_ijkn / (N-2).  First indices i in [i_lo, i_hi) only. */
void orf_spread_C_to_D_range(orf_state *st, int i_lo, int i_hi)
{
    const int N = st->N;
    for (int i = i_lo; i < i_hi; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    const double sh = st->c[ix4(N, i, j, k, n)] / (double)(N - 2);
                    for (int p = 0; p < N; p++) {
                        if (p == i || p == k) continue;
                        for (int q = 0; q < N; q++)
                            if (q != j && q != n) st->d[ix6(N, i, j, k, n, p, q)] += sh;
                    }
                    st->c[ix4(N, i, j, k, n)] = 0.0;
                }
            }
}

void orf_spread_C_to_D(orf_state *st) { orf_spread_C_to_D_range(st, 0, st->N); }

/* Complementary costs of D (Sec. 4.3): the six members of a class, in the
 * lexicographic order of orc_complementary_D, are summed in that order and
 * each becomes T / 6.  Smallest facilities i in [i_lo, i_hi) only. */
void orf_complementary_D_range(orf_state *st, int i_lo, int i_hi)
{
    const int N = st->N;
    double *d = st->d;
    for (int i = i_lo; i < i_hi; i++)
        for (int k = i + 1; k < N; k++)
            for (int p = k + 1; p < N; p++)
                for (int j = 0; j < N; j++)
                    for (int n = 0; n < N; n++) {
                        if (n == j) continue;
                        for (int q = 0; q < N; q++) {
                            if (q == j || q == n) continue;
                            size_t mem[6] = {
                                ix6(N, i, j, k, n, p, q), ix6(N, i, j, p, q, k, n),
                                ix6(N, k, n, i, j, p, q), ix6(N, k, n, p, q, i, j),
                                ix6(N, p, q, i, j, k, n), ix6(N, p, q, k, n, i, j)};
                            double T = 0.0;
                            for (int t = 0; t < 6; t++) T += d[mem[t]];
                            for (int t = 0; t < 6; t++) d[mem[t]] = T / 6.0;
                        }
                    }
}

void orf_complementary_D(orf_state *st) { orf_complementary_D_range(st, 0, st->N); }

/* Complementary costs of C (Sec. 4.3): T = c_ijkn + c_knij (i < k); both = T / 2. */
void orf_complementary_C(orf_state *st)
{
    const int N = st->N;
    for (int i = 0; i < N; i++)
        for (int k = i + 1; k < N; k++)
            for (int j = 0; j < N; j++)
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    const double T = st->c[ix4(N, i, j, k, n)] + st->c[ix4(N, k, n, i, j)];
                    st->c[ix4(N, i, j, k, n)] = T / 2.0;
                    st->c[ix4(N, k, n, i, j)] = T / 2.0;
                }
}

/* Concentration D -> C (Sec. 4.1): c_ijkn += LAP(D_ijkn); D_ijkn becomes
 * (M - u) - v.  First indices i in [i_lo, i_hi) only. */
void orf_concentrate_D_to_C_range(orf_state *st, int i_lo, int i_hi)
{
    const int N = st->N, m = N - 2;
    double *M = malloc((size_t)m * m * sizeof(double));
    double *u = malloc((size_t)m * sizeof(double));
    double *v = malloc((size_t)m * sizeof(double));
    int rows[64], cols[64];
    for (int i = i_lo; i < i_hi; i++)
        for (int j = 0; j < N; j++)
            for (int k = 0; k < N; k++) {
                if (k == i) continue;
                for (int n = 0; n < N; n++) {
                    if (n == j) continue;
                    int r = 0, s = 0;
                    for (int p = 0; p < N; p++) if (p != i && p != k) rows[r++] = p;
                    for (int q = 0; q < N; q++) if (q != j && q != n) cols[s++] = q;
                    for (r = 0; r < m; r++)
                        for (s = 0; s < m; s++)
                            M[r * m + s] = st->d[ix6(N, i, j, k, n, rows[r], cols[s])];
                    const double S = orf_lap(m, M, u, v, NULL, NULL, st);
                    st->c[ix4(N, i, j, k, n)] += S;
                    for (r = 0; r < m; r++)
                        for (s = 0; s < m; s++)
                            st->d[ix6(N, i, j, k, n, rows[r], cols[s])] = M[r * m + s] - u[r] - v[s];
                }
            }
    free(M); free(u); free(v);
}

void orf_concentrate_D_to_C(orf_state *st) { orf_concentrate_D_to_C_range(st, 0, st->N); }

/* Concentration C -> B (Sec. 4.1): b_ij += LAP(C_ij); C_ij becomes (M - u) - v. */
void orf_concentrate_C_to_B(orf_state *st)
{
    const int N = st->N, m = N - 1;
    double *M = malloc((size_t)m * m * sizeof(double));
    double *u = malloc((size_t)m * sizeof(double));
    double *v = malloc((size_t)m * sizeof(double));
    int rows[64], cols[64];
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int r = 0, s = 0;
            for (int k = 0; k < N; k++) if (k != i) rows[r++] = k;
            for (int n = 0; n < N; n++) if (n != j) cols[s++] = n;
            for (r = 0; r < m; r++)
                for (s = 0; s < m; s++)
                    M[r * m + s] = st->c[ix4(N, i, j, rows[r], cols[s])];
            const double S = orf_lap(m, M, u, v, NULL, NULL, st);
            st->b[ix2(N, i, j)] += S;
            for (r = 0; r < m; r++)
                for (s = 0; s < m; s++)
                    st->c[ix4(N, i, j, rows[r], cols[s])] = M[r * m + s] - u[r] - v[s];
        }
    free(M); free(u); free(v);
}

/* Concentration B -> LB (Sec. 4.1): returns LAP(B); B becomes (M - u) - v. */
double orf_concentrate_B_to_LB(orf_state *st)
{
    const int N = st->N;
    double *u = malloc((size_t)N * sizeof(double));
    double *v = malloc((size_t)N * sizeof(double));
    double *M = malloc((size_t)N * N * sizeof(double));
    memcpy(M, st->b, (size_t)N * N * sizeof(double));
    const double S = orf_lap(N, M, u, v, NULL, NULL, st);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++)
            st->b[ix2(N, i, j)] = M[i * N + j] - u[i] - v[j];
    free(u); free(v); free(M);
    return S;
}

/* One pass of Algorithm 1 in the FP64 form (order of reading R2). */
double orf_iterate(orf_state *st)
{
    orf_spread_B_to_C(st);
    if (!st->rlt1_only) {
        orf_spread_C_to_D(st);
        orf_complementary_D(st);
        orf_concentrate_D_to_C(st);
    }
    orf_complementary_C(st);
    orf_concentrate_C_to_B(st);
    st->LB += orf_concentrate_B_to_LB(st);
    st->iters++;
    return st->LB;
}

void orf_run(orf_state *st, int k, double *hist)
{
    for (int t = 0; t < k; t++) {
        double lb = orf_iterate(st);
        if (hist) hist[t] = lb;
    }
}

double orf_LB(const orf_state *st) { return st->LB; }
void orf_add_LB(orf_state *st, double x) { st->LB += x; }
double *orf_b(orf_state *st) { return st->b; }
double *orf_c(orf_state *st) { return st->c; }
double *orf_d(orf_state *st) { return st->d; }
void orf_work(const orf_state *st, int64_t *out3)
{
    out3[0] = st->laps; out3[1] = st->steps; out3[2] = st->relaxations;
}
