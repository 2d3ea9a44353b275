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
