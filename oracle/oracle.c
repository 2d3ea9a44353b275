/*
 * ORACLE -- test infrastructure only.
 *
 * A plain, slow, full-matrix int32 implementation of the alignment the
 * library computes.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the library itself never does.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (SOAP3-dp, Methods section 3, "GPU-accelerated dynamic
 * programming"):
 *   T = candidate window of length m (index i), R = read of length n (index j).
 *   M(i,j) is the best score of a suffix of T[1..i] against R[1..j];
 *   I(i,j) the same with R[j] against a space, D(i,j) with T[i] against a space.
 *     I(i,j) = max(M(i,j-1) + S_GO, I(i,j-1) + S_GE)
 *     D(i,j) = max(M(i-1,j) + S_GO, D(i-1,j) + S_GE)
 *     M(i,j) = max(M(i-1,j-1) + delta(T[i],R[j]), I(i,j), D(i,j))
 *   with base cases I(i,0) = D(0,j) = -inf, M(i,0) = 0, M(0,j) = S_GO + (j-1) S_GE,
 *   and result max_i M(i,n).  The paper's delta(R[i],T[j]) is read as
 *   delta(T[i],R[j]) because i indexes T and j indexes R.
 * This is the GLOCAL mode (whole read, free placement in the window).  LOCAL
 * mode is the Smith-Waterman variant the paper names: every cell is floored at
 * 0, M(0,j) = 0, and the result is the maximum over all cells.
 * The code calls I "E" and D "F" and M "H", as Gotoh's formulation does.
 *
 * Scoring is the BWA convention the paper adopts (Abstract; Results, "same
 * scoring scheme as BWA"): magnitudes match a, mismatch b, gap open o, gap
 * extend e, a gap of length L costs o + L*e.  In the paper's signed form:
 * S_MA = a, S_MI = -b, S_GO = -(o+e), S_GE = -e.
 *
 * Readings fixed here where the paper is silent (listed in the design notes):
 *  - best cell: scan i = 1..m outer, j = 1..n inner, update on strict '>';
 *    LOCAL starts from best = 0 (no alignment if nothing is positive).
 *  - traceback from the best cell in state H with priority
 *    stop (LOCAL and H == 0, or i == 0 or j == 0) > diagonal > D (F) > I (E);
 *    in a gap state, extend only if extending is strictly better than opening.
 *    GLOCAL: reaching i == 0 with j > 0 emits j insertions.
 *  - second best: colbest(i) = max_j H(i,j) (LOCAL) or H(i,n) (GLOCAL);
 *    second = max colbest(i) over |i - i*| >= n, smallest such i on ties.
 *  - CIGAR in BAM encoding (len << 4 | op), M=0 I=1 D=2 S=4; LOCAL soft-clips
 *    the unaligned read ends.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define NEG (INT32_MIN / 4)
#define NO_SCORE INT32_MIN

enum { OR_LOCAL = 0, OR_GLOCAL = 1 };
enum { OR_EMPTY = 1, OR_BELOW_MIN = 2 };
enum { OP_M = 0, OP_I = 1, OP_D = 2, OP_S = 4 };

typedef struct {
    int32_t score, second;
    int32_t read_begin, read_end;
    int64_t ref_begin, ref_end, second_ref_end;
    int32_t n_ops;
    uint32_t flags;
} oracle_result;

typedef struct {
    int32_t a, b, GO, GE;     /* signed: match, mismatch, gap open (first base), extension */
    int mode;
    int want_cigar;
    int32_t min_score;
} oracle_params;

static inline int32_t max2(int32_t x, int32_t y) { return x > y ? x : y; }

static int base_code(uint8_t c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    }
    return -1;
}

/* Fill H, E, F of size (m+1) x (n+1), row-major by i.  T and R hold codes 0..3. */
void oracle_fill(const uint8_t* T, int m, const uint8_t* R, int n, const oracle_params* p,
                 int32_t* H, int32_t* E, int32_t* F) {
    const int w = n + 1;
    for (int i = 0; i <= m; i++) {              /* M(i,0) = 0, I(i,0) = -inf */
        H[i * w] = 0;
        E[i * w] = NEG;
        F[i * w] = NEG;
    }
    for (int j = 1; j <= n; j++) {              /* M(0,j), D(0,j) = -inf */
        H[j] = p->mode == OR_GLOCAL ? p->GO + (j - 1) * p->GE : 0;
        F[j] = NEG;
        E[j] = NEG;
    }
    for (int i = 1; i <= m; i++) {
        for (int j = 1; j <= n; j++) {
            int32_t e = max2(H[i * w + j - 1] + p->GO, E[i * w + j - 1] + p->GE);
            int32_t f = max2(H[(i - 1) * w + j] + p->GO, F[(i - 1) * w + j] + p->GE);
            int32_t g = H[(i - 1) * w + j - 1] + (T[i - 1] == R[j - 1] ? p->a : p->b);
            int32_t h = max2(g, max2(e, f));
            if (p->mode == OR_LOCAL) h = max2(h, 0);
            E[i * w + j] = e;
            F[i * w + j] = f;
            H[i * w + j] = h;
        }
    }
}

/* colbest(i) for i = 1..m into cb[1..m] */
void oracle_colbest(const int32_t* H, int m, int n, int mode, int32_t* cb) {
    const int w = n + 1;
    for (int i = 1; i <= m; i++) {
        if (mode == OR_GLOCAL) { cb[i] = H[i * w + n]; continue; }
        int32_t c = H[i * w + 1];
        for (int j = 2; j <= n; j++) c = max2(c, H[i * w + j]);
        cb[i] = c;
    }
}

static void push_op(uint32_t* ops, int* n_ops, int op, int len) {
    if (len <= 0) return;
    if (*n_ops > 0 && (int)(ops[*n_ops - 1] & 15) == op) {
        ops[*n_ops - 1] += (uint32_t)len << 4;
    } else {
        ops[(*n_ops)++] = ((uint32_t)len << 4) | (uint32_t)op;
    }
}

/* Align one job.  T, R are codes.  ops must hold 2n+3 entries; work must hold
 * 3*(m+1)*(n+1) + (m+1) int32. */
void oracle_align_codes(const uint8_t* T, int m, const uint8_t* R, int n, int64_t ref_pos,
                        const oracle_params* p, int32_t* work, uint32_t* ops,
                        oracle_result* res) {
    const int w = n + 1;
    int32_t* H = work;
    int32_t* E = H + (size_t)(m + 1) * w;
    int32_t* F = E + (size_t)(m + 1) * w;
    int32_t* cb = F + (size_t)(m + 1) * w;
    oracle_fill(T, m, R, n, p, H, E, F);

    /* best cell */
    int32_t best;
    int bi = 0, bj = 0;
    if (p->mode == OR_GLOCAL) {
        best = H[1 * w + n]; bi = 1; bj = n;
        for (int i = 2; i <= m; i++)
            if (H[i * w + n] > best) { best = H[i * w + n]; bi = i; }
    } else {
        best = 0;
        for (int i = 1; i <= m; i++)
            for (int j = 1; j <= n; j++)
                if (H[i * w + j] > best) { best = H[i * w + j]; bi = i; bj = j; }
    }

    memset(res, 0, sizeof(*res));
    res->score = best;
    res->second = NO_SCORE;
    res->second_ref_end = -1;
    res->read_begin = res->read_end = -1;
    res->ref_begin = res->ref_end = -1;
    res->n_ops = 0;
    if (best < p->min_score) res->flags |= OR_BELOW_MIN;
    if (p->mode == OR_LOCAL && best == 0) {      /* nothing positive: no alignment */
        res->flags |= OR_EMPTY;
        return;
    }
    res->read_end = bj;
    res->ref_end = ref_pos + bi;

    /* second best at a distinct location */
    oracle_colbest(H, m, n, p->mode, cb);
    int si = 0;
    for (int i = 1; i <= m; i++) {
        int d = i > bi ? i - bi : bi - i;
        if (d < n) continue;
        if (si == 0 || cb[i] > res->second) { res->second = cb[i]; si = i; }
    }
    if (si) res->second_ref_end = ref_pos + si;

    if (!p->want_cigar || (res->flags & OR_BELOW_MIN)) return;

    /* traceback by re-comparing stored values; ops collected in reverse */
    uint32_t* rev = ops + (2 * n + 3);          /* scratch half of the ops buffer */
    int nrev = 0;
    int i = bi, j = bj;
    enum { ST_H, ST_E, ST_F } st = ST_H;
    for (;;) {
        if (st == ST_H) {
            if (i == 0 || j == 0) break;
            int32_t h = H[i * w + j];
            if (p->mode == OR_LOCAL && h == 0) break;
            int32_t g = H[(i - 1) * w + j - 1] + (T[i - 1] == R[j - 1] ? p->a : p->b);
            if (h == g) { push_op(rev, &nrev, OP_M, 1); i--; j--; }
            else if (h == F[i * w + j]) st = ST_F;
            else st = ST_E;
        } else if (st == ST_F) {                 /* T[i] against a space */
            push_op(rev, &nrev, OP_D, 1);
            int ext = F[(i - 1) * w + j] + p->GE > H[(i - 1) * w + j] + p->GO;
            i--;
            st = ext ? ST_F : ST_H;
        } else {                                 /* R[j] against a space */
            push_op(rev, &nrev, OP_I, 1);
            int ext = E[i * w + j - 1] + p->GE > H[i * w + j - 1] + p->GO;
            j--;
            st = ext ? ST_E : ST_H;
        }
    }
    if (p->mode == OR_GLOCAL && j > 0) { push_op(rev, &nrev, OP_I, j); j = 0; }
    res->read_begin = j;
    res->ref_begin = ref_pos + i;

    int n_ops = 0;
    if (p->mode == OR_LOCAL) push_op(ops, &n_ops, OP_S, res->read_begin);
    for (int k = nrev - 1; k >= 0; k--) push_op(ops, &n_ops, (int)(rev[k] & 15), (int)(rev[k] >> 4));
    if (p->mode == OR_LOCAL) push_op(ops, &n_ops, OP_S, n - res->read_end);
    res->n_ops = n_ops;
}

/* ------------------------------------------------------------------------ */
/* batch driver over ASCII inputs                                            */

typedef struct {
    const uint8_t* ref; uint64_t ref_len;
    const uint8_t* reads;
    const uint64_t* read_off; const uint32_t* read_len; const uint32_t* flags;
    const uint64_t* ref_pos; const uint32_t* win_len;
    const oracle_params* p;
    oracle_result* res; uint32_t* ops; uint64_t ops_stride;
    uint64_t lo, hi;
    int status;
} batch_task;

static void* batch_worker(void* arg) {
    batch_task* t = (batch_task*)arg;
    size_t work_cap = 0, code_cap = 0;
    int32_t* work = NULL;
    uint8_t *T = NULL, *R = NULL;
    uint32_t* ops_tmp = NULL;
    size_t ops_cap = 0;
    for (uint64_t k = t->lo; k < t->hi; k++) {
        int n = (int)t->read_len[k], m = (int)t->win_len[k];
        size_t need = (size_t)3 * (m + 1) * (n + 1) + (m + 1);
        if (need > work_cap) { free(work); work = (int32_t*)malloc(need * 4); work_cap = need; }
        if ((size_t)(m + n) > code_cap) {
            free(T); free(R);
            code_cap = (size_t)(m + n);
            T = (uint8_t*)malloc(code_cap); R = (uint8_t*)malloc(code_cap);
        }
        if ((size_t)(4 * n + 6) > ops_cap) { free(ops_tmp); ops_cap = 4 * n + 6; ops_tmp = (uint32_t*)malloc(ops_cap * 4); }
        if (!work || !T || !R || !ops_tmp) { t->status = -2; break; }
        if (t->ref_pos[k] + (uint64_t)m > t->ref_len || n < 1 || m < 1) { t->status = -1; break; }
        for (int i = 0; i < m; i++) {
            int c = base_code(t->ref[t->ref_pos[k] + i]);
            if (c < 0) { t->status = -1; break; }
            T[i] = (uint8_t)c;
        }
        const uint8_t* r = t->reads + t->read_off[k];
        int rc = t->flags[k] & 1;
        for (int j = 0; j < n; j++) {
            int c = base_code(rc ? r[n - 1 - j] : r[j]);
            if (c < 0) { t->status = -1; break; }
            R[j] = (uint8_t)(rc ? 3 - c : c);   /* complement: A<->T, C<->G */
        }
        if (t->status) break;
        oracle_align_codes(T, m, R, n, (int64_t)t->ref_pos[k], t->p, work, ops_tmp, &t->res[k]);
        if (t->ops) {
            uint64_t cap = t->ops_stride;
            if ((uint64_t)t->res[k].n_ops > cap) { t->status = -3; break; }
            memcpy(t->ops + k * cap, ops_tmp, (size_t)t->res[k].n_ops * 4);
        }
    }
    free(work); free(T); free(R); free(ops_tmp);
    return NULL;
}

/* Align jobs [0, n_jobs).  ops (optional) has ops_stride entries per job.
 * Returns 0, -1 (invalid input), -2 (out of memory) or -3 (ops stride too small). */
int oracle_align_batch(const uint8_t* ref, uint64_t ref_len, const uint8_t* reads,
                       const uint64_t* read_off, const uint32_t* read_len, const uint32_t* flags,
                       const uint64_t* ref_pos, const uint32_t* win_len, uint64_t n_jobs,
                       int32_t a, int32_t b, int32_t go, int32_t ge, int mode, int want_cigar,
                       int32_t min_score, oracle_result* res, uint32_t* ops, uint64_t ops_stride,
                       int n_threads) {
    oracle_params p = { a, b, go, ge, mode, want_cigar, min_score };
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    if ((uint64_t)n_threads > n_jobs) n_threads = n_jobs ? (int)n_jobs : 1;
    pthread_t th[512];
    batch_task tk[512];
    for (int t = 0; t < n_threads; t++) {
        tk[t] = (batch_task){ ref, ref_len, reads, read_off, read_len, flags, ref_pos, win_len,
                              &p, res, ops, ops_stride,
                              n_jobs * t / n_threads, n_jobs * (t + 1) / n_threads, 0 };
        pthread_create(&th[t], NULL, batch_worker, &tk[t]);
    }
    int st = 0;
    for (int t = 0; t < n_threads; t++) {
        pthread_join(th[t], NULL);
        if (tk[t].status && !st) st = tk[t].status;
    }
    return st;
}

/* Expose the matrices of one job (codes in, (m+1)x(n+1) int32 out) for tests. */
void oracle_matrices(const uint8_t* T, int m, const uint8_t* R, int n, int32_t a, int32_t b,
                     int32_t go, int32_t ge, int mode, int32_t* H, int32_t* E, int32_t* F) {
    oracle_params p = { a, b, go, ge, mode, 1, 0 };
    oracle_fill(T, m, R, n, &p, H, E, F);
}

int oracle_sizeof_result(void) { return (int)sizeof(oracle_result); }
