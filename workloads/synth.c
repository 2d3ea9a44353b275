/*
 * Seeded synthetic workloads for batched read-vs-window alignment.
 *
 * This module only draws random sequences and job descriptors; it holds none
 * of the alignment arithmetic.  Both the CPU oracle (oracle/) and the CUDA
 * library read the bytes it writes, so they see identical inputs.
 *
 * Randomness is counter based: every draw is splitmix64's output function
 * (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) applied to key + (counter + 1) * 0x9E3779B97F4A7C15, where the
 * key is derived from (workload, seed, stream, item).  Any item can therefore
 * be regenerated on its own, and multi-threaded generation is deterministic.
 * All probabilities are integer parts-per-million and all arithmetic is
 * integer, so x86-64 and aarch64 produce the same bytes.
 *
 * Shapes follow the paper's workloads (100/150 bp Illumina-like reads, 500 bp
 * inserts; Experiments and Methods sections) as restated in the workload
 * recipe of the design notes:
 *   W1  plain:          concatenated 400 bp windows, 100 bp reads
 *   W2  mate rescue:    100 Mbp GC-41% genome + 300 bp repeats, 150 bp mates
 *   W3  uneven:         n ~ U[50,250], m ~ U[ceil(1.5n), 6n]
 *   W4  low similarity: n = 250, m = 1000, divergence 0..40 %
 *   W5  serving:        requests of U[1, 50000] jobs, m ~ U[2n, 6n]
 *   W6  pairs:          paired 150 bp reads, several candidate windows per read
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t key, ctr; } rng_t;

static inline uint64_t draw(rng_t* r) { r->ctr++; return mix64(r->key + r->ctr * GOLDEN); }
static inline uint32_t draw32(rng_t* r) { return (uint32_t)(draw(r) >> 32); }
/* uniform integer in [lo, hi] (multiply-shift, bias < 2^-32 * range) */
static inline uint64_t uni(rng_t* r, uint64_t lo, uint64_t hi) {
    uint64_t span = hi - lo + 1;
    if (span <= 0xFFFFFFFFULL) return lo + (((uint64_t)draw32(r) * span) >> 32);
    return lo + draw(r) % span;
}
/* Bernoulli with probability ppm / 1e6 */
static inline int bern(rng_t* r, uint32_t ppm) {
    uint64_t thr = ((uint64_t)ppm << 32) / 1000000ULL;
    return (uint64_t)draw32(r) < thr;
}

static rng_t stream(uint32_t workload, uint64_t seed, uint32_t purpose, uint64_t item) {
    uint64_t k = mix64(((uint64_t)workload << 56) ^ (seed * 0xD1B54A32D192ED03ULL) ^ ((uint64_t)purpose << 32));
    rng_t r = { mix64(k ^ (item * GOLDEN + 0x632BE59BD9B4E019ULL)), 0 };
    return r;
}

static const char ACGT[4] = { 'A', 'C', 'G', 'T' };

static inline int code_of(char c) {
    switch (c) { case 'A': return 0; case 'C': return 1; case 'G': return 2; case 'T': return 3; }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* reference sequences                                                       */

typedef struct {
    char* out; uint64_t len; uint32_t workload; uint64_t seed; uint32_t gc_ppm;
    uint64_t lo, hi;
} ref_task;

#define REF_BLOCK (1ULL << 20)

static void* ref_worker(void* p) {
    ref_task* t = (ref_task*)p;
    /* G and C each with probability gc/2, A and T each (1-gc)/2 */
    uint64_t thr_gc = ((uint64_t)t->gc_ppm << 32) / 1000000ULL;
    for (uint64_t b = t->lo; b < t->hi; b++) {
        rng_t r = stream(t->workload, t->seed, 1, b);
        uint64_t s = b * REF_BLOCK, e = s + REF_BLOCK;
        if (e > t->len) e = t->len;
        for (uint64_t i = s; i < e; i++) {
            uint32_t u = draw32(&r);
            int half = u & 1;               /* low bit picks the member of the pair */
            uint32_t v = u >> 1;
            int gc = ((uint64_t)v << 1) < thr_gc;
            t->out[i] = gc ? (half ? 'C' : 'G') : (half ? 'A' : 'T');
        }
    }
    return NULL;
}

/* i.i.d. bases with GC fraction gc_ppm / 1e6; multi-threaded, deterministic */
void synth_reference(uint32_t workload, uint64_t seed, uint64_t len, uint32_t gc_ppm,
                     char* out, int n_threads) {
    uint64_t nblocks = (len + REF_BLOCK - 1) / REF_BLOCK;
    if (n_threads < 1) n_threads = 1;
    if ((uint64_t)n_threads > nblocks) n_threads = (int)(nblocks ? nblocks : 1);
    pthread_t th[256]; ref_task tk[256];
    if (n_threads > 256) n_threads = 256;
    for (int t = 0; t < n_threads; t++) {
        tk[t] = (ref_task){ out, len, workload, seed, gc_ppm,
                            nblocks * t / n_threads, nblocks * (t + 1) / n_threads };
        pthread_create(&th[t], NULL, ref_worker, &tk[t]);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}

/* Paste n_copies segments of seg_len bases, each copied from a uniform random
 * source position, to a uniform random destination, with div_ppm substitutions.
 * Sequential (copies may overlap, the order is part of the definition). */
void synth_paste_repeats(uint32_t workload, uint64_t seed, char* ref, uint64_t len,
                         uint32_t n_copies, uint32_t seg_len, uint32_t div_ppm) {
    if (len < 2ULL * seg_len) return;
    char* buf = (char*)malloc(seg_len);
    for (uint32_t c = 0; c < n_copies; c++) {
        rng_t r = stream(workload, seed, 2, c);
        uint64_t src = uni(&r, 0, len - seg_len);
        uint64_t dst = uni(&r, 0, len - seg_len);
        memcpy(buf, ref + src, seg_len);
        for (uint32_t k = 0; k < seg_len; k++) {
            if (bern(&r, div_ppm)) {
                int old = code_of(buf[k]);
                buf[k] = ACGT[(old + 1 + (int)uni(&r, 0, 2)) & 3];
            }
        }
        memcpy(ref + dst, buf, seg_len);
    }
    free(buf);
}

/* ------------------------------------------------------------------------ */
/* read mutation                                                              */

typedef struct {
    uint32_t sub_ppm;        /* per source base: substitution */
    uint32_t indel_ppm;      /* per source base: start of an indel event */
    uint32_t indel_min, indel_max;   /* uniform length, used when geo_ppm == 0 */
    uint32_t geo_ppm;        /* if > 0: length ~ geometric(p = geo_ppm/1e6), capped at indel_max */
} mut_model;

/* Walk the source from src_pos, emitting exactly target_len bases into out.
 * Per source base: an indel event with probability indel_ppm (insertion or
 * deletion 50/50; inserted bases uniform), else the base is copied and
 * substituted with probability sub_ppm to one of the 3 other bases.  Past the
 * reference end the source is uniform random bases. */
static void mutate(rng_t* r, const char* ref, uint64_t ref_len, uint64_t src_pos,
                   uint32_t target_len, const mut_model* mm, char* out) {
    uint32_t emitted = 0;
    uint64_t p = src_pos;
    while (emitted < target_len) {
        if (mm->indel_ppm && bern(r, mm->indel_ppm)) {
            uint32_t L;
            if (mm->geo_ppm) {
                L = 1;
                while (L < mm->indel_max && !bern(r, mm->geo_ppm)) L++;
            } else {
                L = (uint32_t)uni(r, mm->indel_min, mm->indel_max);
            }
            if (draw32(r) & 0x80000000u) {           /* insertion */
                for (uint32_t k = 0; k < L && emitted < target_len; k++)
                    out[emitted++] = ACGT[uni(r, 0, 3)];
            } else {                                  /* deletion */
                p += L;
            }
            continue;
        }
        char c = p < ref_len ? ref[p] : ACGT[uni(r, 0, 3)];
        p++;
        if (mm->sub_ppm && bern(r, mm->sub_ppm)) c = ACGT[(code_of(c) + 1 + (int)uni(r, 0, 2)) & 3];
        out[emitted++] = c;
    }
}

static void revcomp_inplace(char* s, uint32_t n) {
    for (uint32_t a = 0, b = n ? n - 1 : 0; a < b; a++, b--) { char t = s[a]; s[a] = s[b]; s[b] = t; }
    for (uint32_t k = 0; k < n; k++) {
        switch (s[k]) { case 'A': s[k] = 'T'; break; case 'C': s[k] = 'G'; break;
                        case 'G': s[k] = 'C'; break; case 'T': s[k] = 'A'; break; }
    }
}

/* ------------------------------------------------------------------------ */
/* job generation                                                             */

/* kinds of job recipes */
enum { J_PLAIN = 1, J_MATE = 2, J_UNEVEN = 3, J_LOWSIM = 4, J_SERVE = 5 };

typedef struct {
    uint32_t kind;
    uint32_t workload;
    uint64_t seed;
    const char* ref; uint64_t ref_len;
    /* plain */
    uint32_t win_len, read_len;
    /* uneven / serving: n ~ U[n_lo, n_hi], m ~ U[ceil(m_lo_x10 * n / 10), m_hi_x * n] */
    uint32_t n_lo, n_hi, m_lo_x10, m_hi_x;
    /* mate rescue */
    uint32_t insert_mean, insert_sd, win_before, win_total;
    uint32_t flip_rc;
} job_recipe;

typedef struct {
    const job_recipe* jr;
    uint64_t first_item;          /* global item id of job 0 of this call */
    uint64_t n_jobs;
    uint64_t* read_off; uint32_t* read_len; uint32_t* flags; uint64_t* ref_pos; uint32_t* win_len;
    char* reads; uint64_t* truth_pos;
    uint64_t lo, hi;
} job_task;

/* read length and window length of job item (no sequence work) */
static void job_shape(const job_recipe* jr, uint64_t item, uint32_t* n, uint32_t* m) {
    rng_t r = stream(jr->workload, jr->seed, 3, item);
    switch (jr->kind) {
    case J_PLAIN: case J_LOWSIM: case J_MATE:
        *n = jr->read_len; *m = jr->win_len; break;
    default: {
        uint32_t nn = (uint32_t)uni(&r, jr->n_lo, jr->n_hi);
        uint32_t mlo = (uint32_t)((jr->m_lo_x10 * (uint64_t)nn + 9) / 10);
        uint32_t mhi = jr->m_hi_x * nn;
        if (mlo < nn) mlo = nn;
        *n = nn; *m = (uint32_t)uni(&r, mlo, mhi);
        if (*m > jr->ref_len) *m = (uint32_t)jr->ref_len;
    } }
}

/* Irwin-Hall approximation of a standard normal, scaled: mean + sd * z,
 * rounded, integer only: z = (sum of 12 U16 - 6*65536) / 65536 */
static int64_t normal_int(rng_t* r, int64_t mean, int64_t sd) {
    int64_t s = 0;
    for (int k = 0; k < 12; k++) s += (int64_t)(draw32(r) >> 16);
    int64_t num = sd * (s - 6 * 65536);
    /* floor((num + 32768) / 65536) */
    int64_t q = (num + 32768) >= 0 ? (num + 32768) / 65536 : -((-(num + 32768) + 65535) / 65536);
    return mean + q;
}

static void* job_worker(void* p) {
    job_task* t = (job_task*)p;
    const job_recipe* jr = t->jr;
    for (uint64_t j = t->lo; j < t->hi; j++) {
        uint64_t item = t->first_item + j;
        uint32_t n, m;
        job_shape(jr, item, &n, &m);
        rng_t r = stream(jr->workload, jr->seed, 4, item);
        char* out = t->reads + t->read_off[j];
        uint64_t pos = 0, src = 0;
        uint32_t fl = 0;
        mut_model mm;
        memset(&mm, 0, sizeof(mm));
        switch (jr->kind) {
        case J_PLAIN:
            /* window j of the concatenated reference, read from a uniform offset */
            pos = (item * (uint64_t)jr->win_len) % (jr->ref_len - jr->win_len + 1);
            src = pos + uni(&r, 0, m - n);
            mm = (mut_model){ 20000, 2000, 1, 5, 0 };
            break;
        case J_UNEVEN: case J_SERVE:
            pos = uni(&r, 0, jr->ref_len - m);
            src = pos + uni(&r, 0, m - n);
            mm = (mut_model){ 20000, 2000, 1, 5, 0 };
            break;
        case J_LOWSIM: {
            static const uint32_t div_ppm[6] = { 0, 50000, 100000, 200000, 300000, 400000 };
            uint32_t d = div_ppm[item % 6];
            pos = uni(&r, 0, jr->ref_len - m);
            src = pos + uni(&r, 0, m - n);
            mm = (mut_model){ (uint32_t)(d * 9ULL / 10), d / 10, 1, 30, 300000 };
            break; }
        case J_MATE: {
            /* fragment start uniform; insert ~ round(N(mean, sd)); mate 2 is the
             * reverse complement of the fragment end; window placed from mate 1 */
            uint64_t span = (uint64_t)jr->insert_mean + 4ULL * jr->insert_sd + jr->win_total;
            uint64_t pos1 = uni(&r, 0, jr->ref_len > span ? jr->ref_len - span : 0);
            int64_t ins = normal_int(&r, jr->insert_mean, jr->insert_sd);
            if (ins < (int64_t)n) ins = n;
            src = pos1 + (uint64_t)ins - n;
            int64_t w0 = (int64_t)pos1 + jr->insert_mean - jr->win_before;
            if (w0 < 0) w0 = 0;
            int64_t w1 = w0 + jr->win_total;
            if ((uint64_t)w1 > jr->ref_len) { w1 = (int64_t)jr->ref_len; if (w1 - w0 < (int64_t)n) w0 = w1 - n; }
            pos = (uint64_t)w0;
            m = (uint32_t)(w1 - w0);
            mm = (mut_model){ 10000, 3000, 1, 10, 0 };
            fl = jr->flip_rc;
            break; }
        }
        mutate(&r, jr->ref, jr->ref_len, src, n, &mm, out);
        if (fl) revcomp_inplace(out, n);
        t->read_len[j] = n;
        t->win_len[j] = m;
        t->ref_pos[j] = pos;
        t->flags[j] = fl;
        if (t->truth_pos) t->truth_pos[j] = src;
    }
    return NULL;
}

static void run_jobs(const job_recipe* jr, uint64_t first_item, uint64_t n_jobs,
                     uint64_t* read_off, uint32_t* read_len, uint32_t* flags,
                     uint64_t* ref_pos, uint32_t* win_len, char* reads,
                     uint64_t* truth_pos, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if ((uint64_t)n_threads > n_jobs) n_threads = n_jobs ? (int)n_jobs : 1;
    pthread_t th[256]; job_task tk[256];
    for (int t = 0; t < n_threads; t++) {
        tk[t] = (job_task){ jr, first_item, n_jobs, read_off, read_len, flags, ref_pos, win_len,
                            reads, truth_pos, n_jobs * t / n_threads, n_jobs * (t + 1) / n_threads };
        pthread_create(&th[t], NULL, job_worker, &tk[t]);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}

/* Pass 1: read lengths of jobs [first_item, first_item + n_jobs) so the caller
 * can size the read buffer and fill read_off (exclusive prefix sum). */
void synth_job_read_lens(uint32_t kind, uint32_t workload, uint64_t seed, uint64_t ref_len,
                         uint32_t win_len, uint32_t read_len,
                         uint32_t n_lo, uint32_t n_hi, uint32_t m_lo_x10, uint32_t m_hi_x,
                         uint64_t first_item, uint64_t n_jobs, uint32_t* out_n) {
    job_recipe jr;
    memset(&jr, 0, sizeof(jr));
    jr.kind = kind; jr.workload = workload; jr.seed = seed; jr.ref_len = ref_len;
    jr.win_len = win_len; jr.read_len = read_len;
    jr.n_lo = n_lo; jr.n_hi = n_hi; jr.m_lo_x10 = m_lo_x10; jr.m_hi_x = m_hi_x;
    for (uint64_t j = 0; j < n_jobs; j++) {
        uint32_t n, m;
        job_shape(&jr, first_item + j, &n, &m);
        out_n[j] = n;
    }
}

/* Pass 2: sequences and descriptors.  read_off must be filled by the caller. */
void synth_jobs(uint32_t kind, uint32_t workload, uint64_t seed,
                const char* ref, uint64_t ref_len,
                uint32_t win_len, uint32_t read_len,
                uint32_t n_lo, uint32_t n_hi, uint32_t m_lo_x10, uint32_t m_hi_x,
                uint32_t insert_mean, uint32_t insert_sd, uint32_t win_before, uint32_t win_total,
                uint32_t flip_rc,
                uint64_t first_item, uint64_t n_jobs,
                uint64_t* read_off, uint32_t* out_read_len, uint32_t* flags,
                uint64_t* ref_pos, uint32_t* out_win_len, char* reads, uint64_t* truth_pos,
                int n_threads) {
    job_recipe jr;
    memset(&jr, 0, sizeof(jr));
    jr.kind = kind; jr.workload = workload; jr.seed = seed; jr.ref = ref; jr.ref_len = ref_len;
    jr.win_len = win_len; jr.read_len = read_len;
    jr.n_lo = n_lo; jr.n_hi = n_hi; jr.m_lo_x10 = m_lo_x10; jr.m_hi_x = m_hi_x;
    jr.insert_mean = insert_mean; jr.insert_sd = insert_sd;
    jr.win_before = win_before; jr.win_total = win_total; jr.flip_rc = flip_rc;
    run_jobs(&jr, first_item, n_jobs, read_off, out_read_len, flags, ref_pos, out_win_len,
             reads, truth_pos, n_threads);
}

/* Uniform draws for the serving harness: request sizes and exponential gaps.
 * out_u[k] = uniform in [lo, hi]; out_ppm[k] = uniform in [1, 1e6]. */
void synth_uniform(uint32_t workload, uint64_t seed, uint32_t purpose, uint64_t n,
                   uint64_t lo, uint64_t hi, uint64_t* out_u, uint32_t* out_ppm) {
    for (uint64_t k = 0; k < n; k++) {
        rng_t r = stream(workload, seed, purpose, k);
        if (out_u) out_u[k] = uni(&r, lo, hi);
        if (out_ppm) out_ppm[k] = (uint32_t)uni(&r, 1, 1000000);
    }
}

/* ------------------------------------------------------------------------ */
/* W6  paired reads with several candidate windows per read                  */
/*                                                                          */
/* Pair p: fragment start uniform, insert ~ round(N(mean, sd)); end 1 is the  */
/* fragment's first n bases (forward), end 2 the reverse complement of its   */
/* last n bases (flag SA_RC on its candidates), both mutated like the mate-   */
/* rescue mates.  Each read gets the window around its source (both sides    */
/* padded by U[8, 40]), with probability 20 % a second window around the     */
/* same source shifted by U[1, 20], U[0, decoy_max] decoy windows at uniform  */
/* positions (m = n + U[16, 80]).  For the pairs chosen with probability      */
/* dup_ppm a copy (0.5 % substitutions) is planted at a uniform position:     */
/* half of them copy end 2's source only, half the whole fragment (a          */
/* segmental duplication); the ends whose source was copied get a window      */
/* around the copy too.                                                       */
/* Candidates are shuffled; each carries a seed-support count (source and     */
/* planted copy U[6, 24], shifted U[3, 12], decoys U[1, 16]).                 */

#define W_PAIRS_PURPOSE_COUNT 8
#define W_PAIRS_PURPOSE_DUP   9
#define W_PAIRS_PURPOSE_PAIR  10
#define W_PAIRS_PURPOSE_CAND  11

typedef struct {
    uint32_t workload; uint64_t seed;
    uint64_t ref_len; uint32_t n;
    uint32_t insert_mean, insert_sd;
    uint32_t decoy_max; uint32_t dup_ppm;
} pair_recipe;

static void pair_sources(const pair_recipe* pr, uint64_t item, uint64_t* src1, uint64_t* src2) {
    rng_t r = stream(pr->workload, pr->seed, W_PAIRS_PURPOSE_PAIR, item);
    uint64_t span = (uint64_t)pr->insert_mean + 4ULL * pr->insert_sd + 200;
    uint64_t pos1 = uni(&r, 200, pr->ref_len > span + 200 ? pr->ref_len - span : 200);
    int64_t ins = normal_int(&r, pr->insert_mean, pr->insert_sd);
    if (ins < (int64_t)pr->n) ins = pr->n;
    *src1 = pos1;
    *src2 = pos1 + (uint64_t)ins - pr->n;
}

/* planted copy for pair item: 0 none, 1 end 2's source, 2 the whole fragment;
 * *dst is where the copied span starts */
static int pair_dup(const pair_recipe* pr, uint64_t item, uint64_t* dst) {
    rng_t r = stream(pr->workload, pr->seed, W_PAIRS_PURPOSE_DUP, item);
    if (!bern(&r, pr->dup_ppm)) return 0;
    const int kind = bern(&r, 500000) ? 2 : 1;
    const uint64_t room = (uint64_t)pr->insert_mean + 4ULL * pr->insert_sd + 400;
    *dst = uni(&r, 100, pr->ref_len > room + 100 ? pr->ref_len - room : 100);
    return kind;
}

/* candidate counts of read (2 item + end): source, shifted, decoys, planted copy */
static void read_counts(const pair_recipe* pr, uint64_t item, int end, uint32_t* shifted,
                        uint32_t* decoys, uint32_t* dup) {
    rng_t r = stream(pr->workload, pr->seed, W_PAIRS_PURPOSE_COUNT, 2 * item + (uint64_t)end);
    *decoys = (uint32_t)uni(&r, 0, pr->decoy_max);
    *shifted = (uint32_t)bern(&r, 200000);
    uint64_t dst;
    const int kind = pair_dup(pr, item, &dst);
    *dup = (kind == 2 || (kind == 1 && end == 1)) ? 1u : 0u;
}

/* Pass 0 (sequential; writes into ref): plant the copies. */
void synth_pairs_plant(uint32_t workload, uint64_t seed, char* ref, uint64_t ref_len, uint32_t n,
                       uint32_t insert_mean, uint32_t insert_sd, uint32_t dup_ppm,
                       uint64_t first_item, uint64_t n_pairs) {
    pair_recipe pr = { workload, seed, ref_len, n, insert_mean, insert_sd, 0, dup_ppm };
    for (uint64_t p = 0; p < n_pairs; p++) {
        uint64_t item = first_item + p, s1, s2, dst;
        const int kind = pair_dup(&pr, item, &dst);
        if (!kind) continue;
        pair_sources(&pr, item, &s1, &s2);
        const uint64_t from = kind == 2 ? s1 : s2;
        const uint64_t len = s2 + n + 40 - from;
        rng_t r = stream(workload, seed, W_PAIRS_PURPOSE_DUP + 100, item);
        for (uint64_t k = 0; k < len && from + k < ref_len && dst + k < ref_len; k++) {
            char c = ref[from + k];
            if (bern(&r, 5000)) c = ACGT[(code_of(c) + 1 + (int)uni(&r, 0, 2)) & 3];
            ref[dst + k] = c;
        }
    }
}

/* Pass 1: candidates per read (2 n_pairs reads). */
void synth_pairs_counts(uint32_t workload, uint64_t seed, uint64_t ref_len, uint32_t n,
                        uint32_t decoy_max, uint32_t dup_ppm, uint64_t first_item, uint64_t n_pairs,
                        uint32_t* out_count) {
    if (decoy_max > 61) decoy_max = 61;        /* at most 64 candidates a read */
    pair_recipe pr = { workload, seed, ref_len, n, 0, 0, decoy_max, dup_ppm };
    for (uint64_t p = 0; p < n_pairs; p++)
        for (int e = 0; e < 2; e++) {
            uint32_t sh, dc, du;
            read_counts(&pr, first_item + p, e, &sh, &dc, &du);
            out_count[2 * p + e] = 1 + sh + dc + du;
        }
}

typedef struct {
    const pair_recipe* pr; const char* ref; uint64_t first_item;
    const uint64_t* read_first;
    char* reads; uint64_t* truth;
    uint64_t* read_off; uint32_t* read_len; uint32_t* flags; uint64_t* ref_pos; uint32_t* win_len;
    uint32_t* support;
    uint64_t lo, hi;
} pair_task;

static void window_around(rng_t* r, uint64_t src, uint32_t n, uint64_t ref_len, uint64_t* pos, uint32_t* m) {
    uint64_t padl = uni(r, 8, 40), padr = uni(r, 8, 40);
    uint64_t a = src > padl ? src - padl : 0;
    uint64_t b = src + n + padr;
    if (b > ref_len) b = ref_len;
    *pos = a;
    *m = (uint32_t)(b - a);
}

static void* pair_worker(void* p) {
    pair_task* t = (pair_task*)p;
    const pair_recipe* pr = t->pr;
    const uint32_t n = pr->n;
    mut_model mm = { 10000, 3000, 1, 10, 0 };
    for (uint64_t q = t->lo; q < t->hi; q++) {
        uint64_t item = t->first_item + q, src[2], dst = 0;
        pair_sources(pr, item, &src[0], &src[1]);
        const int kind = pair_dup(pr, item, &dst);
        const uint64_t from = kind == 2 ? src[0] : src[1];
        for (int e = 0; e < 2; e++) {
            const uint64_t rd = 2 * q + (uint64_t)e;
            rng_t r = stream(pr->workload, pr->seed, W_PAIRS_PURPOSE_CAND, 2 * item + (uint64_t)e);
            char* out = t->reads + rd * n;
            mutate(&r, t->ref, pr->ref_len, src[e], n, &mm, out);
            if (e == 1) revcomp_inplace(out, n);
            t->truth[rd] = src[e];
            uint32_t sh, dc, du;
            read_counts(pr, item, e, &sh, &dc, &du);
            const uint32_t k_n = 1 + sh + dc + du;
            uint64_t pos[64]; uint32_t m[64], sup[64];
            uint32_t k = 0;
            window_around(&r, src[e], n, pr->ref_len, &pos[k], &m[k]); sup[k++] = (uint32_t)uni(&r, 6, 24);
            if (sh) {
                uint64_t s = src[e] + uni(&r, 1, 20);
                window_around(&r, s, n, pr->ref_len, &pos[k], &m[k]); sup[k++] = (uint32_t)uni(&r, 3, 12);
            }
            if (du) {
                window_around(&r, dst + (src[e] - from), n, pr->ref_len, &pos[k], &m[k]);
                sup[k++] = (uint32_t)uni(&r, 6, 24);
            }
            for (uint32_t d = 0; d < dc && k < 64; d++) {
                uint32_t mm_len = n + (uint32_t)uni(&r, 16, 80);
                pos[k] = uni(&r, 0, pr->ref_len - mm_len);
                m[k] = mm_len;
                sup[k++] = (uint32_t)uni(&r, 1, 16);
            }
            /* Fisher-Yates shuffle of the k_n candidates */
            for (uint32_t i = k_n; i > 1; i--) {
                uint32_t j = (uint32_t)uni(&r, 0, i - 1);
                uint64_t tp = pos[i - 1]; pos[i - 1] = pos[j]; pos[j] = tp;
                uint32_t tm = m[i - 1]; m[i - 1] = m[j]; m[j] = tm;
                uint32_t ts = sup[i - 1]; sup[i - 1] = sup[j]; sup[j] = ts;
            }
            const uint64_t c0 = t->read_first[rd];
            for (uint32_t c = 0; c < k_n; c++) {
                t->read_off[c0 + c] = rd * n;
                t->read_len[c0 + c] = n;
                t->flags[c0 + c] = e == 1 ? 1u : 0u;
                t->ref_pos[c0 + c] = pos[c];
                t->win_len[c0 + c] = m[c];
                t->support[c0 + c] = sup[c];
            }
        }
    }
    return NULL;
}

/* Pass 2: reads (n bases each, read r at r * n), per-read truth, candidates. */
void synth_pairs(uint32_t workload, uint64_t seed, const char* ref, uint64_t ref_len, uint32_t n,
                 uint32_t insert_mean, uint32_t insert_sd, uint32_t decoy_max, uint32_t dup_ppm,
                 uint64_t first_item, uint64_t n_pairs, const uint64_t* read_first,
                 char* reads, uint64_t* truth, uint64_t* read_off, uint32_t* read_len,
                 uint32_t* flags, uint64_t* ref_pos, uint32_t* win_len, uint32_t* support,
                 int n_threads) {
    if (decoy_max > 61) decoy_max = 61;
    pair_recipe pr = { workload, seed, ref_len, n, insert_mean, insert_sd, decoy_max, dup_ppm };
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if ((uint64_t)n_threads > n_pairs) n_threads = n_pairs ? (int)n_pairs : 1;
    pthread_t th[256]; pair_task tk[256];
    for (int t = 0; t < n_threads; t++) {
        tk[t] = (pair_task){ &pr, ref, first_item, read_first, reads, truth, read_off, read_len,
                             flags, ref_pos, win_len, support,
                             n_pairs * t / n_threads, n_pairs * (t + 1) / n_threads };
        pthread_create(&th[t], NULL, pair_worker, &tk[t]);
    }
    for (int t = 0; t < n_threads; t++) pthread_join(th[t], NULL);
}
