/*
 * CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, scalar int32 Smith-Waterman local alignment with Gotoh affine
 * gaps, written from the recurrences of Sec. 2.2 (Eqs. 1-3) and the
 * cell-update order of Algorithm 1 (Sec. 3.2.1): the score of a pair, of all
 * pairs of two sets, and one optimal alignment of a pair (traceback).  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load this library; the
 * product path never does.  It shares no code, header or table with the GPU
 * library.
 *
 * Notation (Sec. 2.2): query Q (rows i = 1..m), database sequence D (columns
 * j = 1..n), substitution matrix SM, gap-open Go and gap-extend Ge penalties.
 *
 *   H[i][j] = max(0, H[i-1][j-1] + SM(Q[i], D[j]), E[i][j], F[i][j])   (Eq. 1)
 *   E[i][j] = max(H[i][j-1] - Go, E[i][j-1] - Ge)                      (Eq. 2)
 *   F[i][j] = max(H[i-1][j] - Go, F[i-1][j] - Ge)                      (Eq. 3)
 *
 * H, E and F are 0 on row 0 and column 0, and the score S is the largest H
 * (Sec. 2.2, the paragraph after Eq. 3).
 *
 * Gap convention of this library's interface: a gap run of length k costs
 * gap_open + k * gap_extend.  In Eqs. 2-3 the first gap position costs Go and
 * every further one Ge, so Go = gap_open + gap_extend and Ge = gap_extend.
 * With the paper's "10/2" this gives 10 + 2k (12, 14, 16, ... for k = 1, 2, 3).
 *
 * SM is a row-major 20x20 int8 table, row = query residue, column = database
 * residue.  Residue codes are 0..19.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

#define ORACLE_ALPHABET 20

/* Boundary initialisation of E and F on row 0 / column 0.  ORACLE_INIT_ZERO is
 * the paper's rule (Sec. 2.2); ORACLE_INIT_NEGINF is the textbook -infinity,
 * kept so that a test can show the two give the same score. */
#define ORACLE_INIT_ZERO 0
#define ORACLE_INIT_NEGINF 1
#define ORACLE_NEG_INF (-(1 << 28))

static int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/* Score of one (query, database sequence) pair.  Returns -1 on invalid input
 * (a residue code >= 20, a negative length or negative penalties). */
int32_t oracle_sw_score_init(const uint8_t *Q, int64_t m, const uint8_t *D, int64_t n,
                             const int8_t *SM, int32_t gap_open, int32_t gap_extend,
                             int32_t init_mode) {
    if (m < 0 || n < 0 || gap_open < 0 || gap_extend < 0) return -1;
    for (int64_t i = 0; i < m; ++i) if (Q[i] >= ORACLE_ALPHABET) return -1;
    for (int64_t j = 0; j < n; ++j) if (D[j] >= ORACLE_ALPHABET) return -1;
    if (m == 0 || n == 0) return 0;

    const int32_t Go = gap_open + gap_extend;
    const int32_t Ge = gap_extend;
    const int32_t edge = (init_mode == ORACLE_INIT_NEGINF) ? ORACLE_NEG_INF : 0;

    /* Hup[j] = H[i-1][j], Fup[j] = F[i-1][j]; entry 0 is column 0. */
    int32_t *Hup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *Fup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!Hup || !Fup) { free(Hup); free(Fup); return -1; }
    for (int64_t j = 0; j <= n; ++j) { Hup[j] = 0; Fup[j] = edge; } /* row 0 */

    int32_t S = 0;
    for (int64_t i = 1; i <= m; ++i) {
        int32_t Hl = 0;       /* H[i][0] */
        int32_t El = edge;    /* E[i][0] */
        int32_t Hul = Hup[0]; /* H[i-1][0] */
        const int8_t *row = SM + (size_t)Q[i - 1] * ORACLE_ALPHABET;
        for (int64_t j = 1; j <= n; ++j) {
            /* Algorithm 1, in its order. */
            int32_t E1 = El - Ge;
            int32_t E2 = Hl - Go;
            int32_t E = max2(E1, E2);
            int32_t F1 = Fup[j] - Ge;
            int32_t F2 = Hup[j] - Go;
            int32_t F = max2(F1, F2);
            int32_t H = Hul + row[D[j - 1]];
            H = max2(H, E);
            H = max2(H, F);
            H = max2(H, 0);
            S = max2(H, S);
            /* shift the neighbours for the next column */
            Hul = Hup[j];
            Hup[j] = H;
            Fup[j] = F;
            Hl = H;
            El = E;
        }
    }
    free(Hup);
    free(Fup);
    return S;
}

int32_t oracle_sw_score(const uint8_t *Q, int64_t m, const uint8_t *D, int64_t n,
                        const int8_t *SM, int32_t gap_open, int32_t gap_extend) {
    return oracle_sw_score_init(Q, m, D, n, SM, gap_open, gap_extend, ORACLE_INIT_ZERO);
}

/* ---- many queries x many database sequences, threaded across pairs ---- */

typedef struct {
    const uint8_t *qres; const int64_t *qoff; int64_t nq;
    const uint8_t *dres; const int64_t *doff; int64_t nd;
    const int64_t *dsel; int64_t nsel; /* optional subset of database indices */
    const int8_t *SM; int32_t go, ge;
    int32_t *out;
    int64_t next;  /* shared work counter */
    pthread_mutex_t lock;
    int failed;
} oracle_job;

static void *oracle_worker(void *arg) {
    oracle_job *J = (oracle_job *)arg;
    const int64_t ncols = J->dsel ? J->nsel : J->nd;
    const int64_t total = J->nq * ncols;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int64_t t = J->next;
        J->next += 16;
        pthread_mutex_unlock(&J->lock);
        if (t >= total) break;
        int64_t e = t + 16 < total ? t + 16 : total;
        for (; t < e; ++t) {
            int64_t q = t / ncols, c = t % ncols;
            int64_t d = J->dsel ? J->dsel[c] : c;
            int32_t s = oracle_sw_score(J->qres + J->qoff[q], J->qoff[q + 1] - J->qoff[q],
                                        J->dres + J->doff[d], J->doff[d + 1] - J->doff[d],
                                        J->SM, J->go, J->ge);
            if (s < 0) J->failed = 1;
            J->out[q * ncols + c] = s;
        }
    }
    return NULL;
}

/* scores_out[q * ncols + c] for every query q and every database index c
 * (or dsel[c] when dsel is given, ncols = nsel).  Returns 0 on success. */
int32_t oracle_sw_batch(const uint8_t *qres, const int64_t *qoff, int64_t nq,
                        const uint8_t *dres, const int64_t *doff, int64_t nd,
                        const int64_t *dsel, int64_t nsel,
                        const int8_t *SM, int32_t gap_open, int32_t gap_extend,
                        int32_t *scores_out, int32_t nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 1024) nthreads = 1024;
    oracle_job J = {qres, qoff, nq, dres, doff, nd, dsel, nsel, SM, gap_open, gap_extend,
                    scores_out, 0, PTHREAD_MUTEX_INITIALIZER, 0};
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!th) return -1;
    int started = 0;
    for (int k = 0; k < nthreads; ++k)
        if (pthread_create(&th[k], NULL, oracle_worker, &J) == 0) started++;
        else break;
    if (started == 0) oracle_worker(&J);
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    free(th);
    return J.failed ? -1 : 0;
}

/* ---- one optimal local alignment (traceback), full matrices -------------
 *
 * The same recurrences (Eqs. 1-3, paper boundary values) kept for every cell,
 * then a walk back from the first cell (row-major order) that holds the
 * score S: in H, the diagonal move if H = H[i-1][j-1] + SM, else the E state
 * if H = E, else the F state (H = F); in E, a gap opening if E = H[i][j-1] -
 * Go, else an extension; in F likewise with H[i-1][j]; the walk ends in H on
 * a cell with H = 0.  Operations, from the first aligned position to the
 * last: 'M' aligns Q[i] with D[j], 'D' consumes a database residue (a gap in
 * the query, the E direction), 'I' consumes a query residue (the F
 * direction).  Coordinates are 0-based: the alignment covers Q[q_begin ..
 * q_end) and D[t_begin .. t_end).  ops must hold m + n bytes.  Returns the
 * number of operations, or -1 on invalid input or allocation failure. */
int64_t oracle_sw_align(const uint8_t *Q, int64_t m, const uint8_t *D, int64_t n,
                        const int8_t *SM, int32_t gap_open, int32_t gap_extend,
                        int32_t *score, int64_t *coords, uint8_t *ops) {
    if (m < 0 || n < 0 || gap_open < 0 || gap_extend < 0) return -1;
    for (int64_t i = 0; i < m; ++i) if (Q[i] >= ORACLE_ALPHABET) return -1;
    for (int64_t j = 0; j < n; ++j) if (D[j] >= ORACLE_ALPHABET) return -1;
    *score = 0;
    coords[0] = coords[1] = coords[2] = coords[3] = 0;
    if (m == 0 || n == 0) return 0;
    const int32_t Go = gap_open + gap_extend;
    const int32_t Ge = gap_extend;
    const int64_t W = n + 1;
    int32_t *H = (int32_t *)calloc((size_t)((m + 1) * W), sizeof(int32_t));
    int32_t *E = (int32_t *)calloc((size_t)((m + 1) * W), sizeof(int32_t));
    int32_t *F = (int32_t *)calloc((size_t)((m + 1) * W), sizeof(int32_t));
    if (!H || !E || !F) { free(H); free(E); free(F); return -1; }
    int32_t S = 0;
    int64_t bi = 0, bj = 0;
    for (int64_t i = 1; i <= m; ++i) {
        const int8_t *row = SM + (size_t)Q[i - 1] * ORACLE_ALPHABET;
        for (int64_t j = 1; j <= n; ++j) {
            const int64_t c = i * W + j;
            E[c] = max2(E[c - 1] - Ge, H[c - 1] - Go);
            F[c] = max2(F[c - W] - Ge, H[c - W] - Go);
            int32_t h = H[c - W - 1] + row[D[j - 1]];
            h = max2(h, E[c]);
            h = max2(h, F[c]);
            h = max2(h, 0);
            H[c] = h;
            if (h > S) { S = h; bi = i; bj = j; }
        }
    }
    *score = S;
    int64_t k = 0;  /* operations, written backwards */
    int64_t i = bi, j = bj;
    int state = 0;  /* 0 = H, 1 = E, 2 = F */
    while (i > 0 && j > 0) {
        const int64_t c = i * W + j;
        if (state == 0) {
            if (H[c] == 0) break;
            if (H[c] == H[c - W - 1] + SM[(size_t)Q[i - 1] * ORACLE_ALPHABET + D[j - 1]]) {
                ops[k++] = 'M'; --i; --j;
            } else if (H[c] == E[c]) {
                state = 1;
            } else {
                state = 2;
            }
        } else if (state == 1) {
            ops[k++] = 'D';
            state = (E[c] == H[c - 1] - Go) ? 0 : 1;
            --j;
        } else {
            ops[k++] = 'I';
            state = (F[c] == H[c - W] - Go) ? 0 : 2;
            --i;
        }
    }
    for (int64_t a = 0, b = k - 1; a < b; ++a, --b) { uint8_t t = ops[a]; ops[a] = ops[b]; ops[b] = t; }
    coords[0] = i; coords[1] = bi; coords[2] = j; coords[3] = bj;
    free(H); free(E); free(F);
    return k;
}
