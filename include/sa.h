/*
 * sa.h -- batched affine-gap alignment of short reads against candidate
 * reference windows on one GB300 (sm_103a).
 *
 * The operation is the dynamic programming of SOAP3-dp's gapped stage
 * (Luo et al., arXiv:1302.5507, Methods section 3 "GPU-accelerated dynamic
 * programming"): for a window T of length m and a read R of length n,
 *   I(i,j) = max(M(i,j-1) + S_GO, I(i,j-1) + S_GE)      read base against a space
 *   D(i,j) = max(M(i-1,j) + S_GO, D(i-1,j) + S_GE)      window base against a space
 *   M(i,j) = max(M(i-1,j-1) + delta(T[i],R[j]), I(i,j), D(i,j))
 * with I(i,0) = D(0,j) = -inf, M(i,0) = 0 and M(0,j) = S_GO + (j-1) S_GE.
 * SA_GLOCAL is exactly that recurrence (the whole read, placed anywhere in the
 * window, result max_i M(i,n)).  SA_LOCAL is Smith-Waterman: every cell is
 * floored at 0, M(0,j) = 0 and the result is the best cell.
 * The windows come from the candidate regions of the paper's steps 2 and 3
 * (Methods section 3 and "Paired-end alignment": the region next to a mapped
 * mate, inferred from the insert-size bounds); the library takes them as
 * (position, length) into a device-resident reference.
 *
 * Every result is exact integer arithmetic and identical, field by field, to
 * the plain full-matrix definition (including the tie rules below), whatever
 * the internal width (16-bit packed with exact overflow detection, or 32-bit).
 *
 * Conventions
 *  - Scores are BWA magnitudes (the paper adopts BWA's scoring scheme): match
 *    a, mismatch b, gap open o, gap extend e, all >= 0; a gap of length L costs
 *    o + L*e.  In the paper's signed form S_MA = a, S_MI = -b, S_GO = -(o+e),
 *    S_GE = -e.  Limits: a <= 2047 (a LOCAL best score then fits 21 bits),
 *    b, o + e <= 16383.
 *  - Best cell: the first maximum in window-major order (smallest reference
 *    end, then smallest read end).  LOCAL with no positive cell: no alignment
 *    (SA_RES_EMPTY, score 0, coordinates -1, second SA_NO_SCORE).
 *  - Traceback from the best cell: stop (LOCAL cell value 0, or a border) >
 *    diagonal > deletion > insertion; a gap run is extended only when that is
 *    strictly better than opening it.  GLOCAL reaching the window start with
 *    read bases left emits them as an insertion.
 *  - Second best: colbest(i) = max_j M(i,j) (LOCAL) or M(i,n) (GLOCAL); the
 *    largest colbest(i) over columns with |i - i*| >= n, smallest such i.
 *  - CIGAR: BAM encoding (length << 4 | op), M=0 I=1 D=2 S=4; LOCAL soft-clips
 *    the unaligned read ends.  At most 2n+3 ops per job.
 *
 * Ownership and errors
 *  - The caller owns every buffer it passes.  sa_create_reference and
 *    sa_submit copy their inputs before returning.  Handles are released only
 *    by the matching destroy call.  No C++ exception crosses this interface.
 *  - Every call returns SA_OK (0), SA_PENDING (1, sa_poll only) or a negative
 *    error code; sa_last_error() gives a message for the calling thread.
 *  - All GPU work runs on one device (the one the reference was created on).
 */
#ifndef SA_H
#define SA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define SA_OK         0
#define SA_PENDING    1     /* sa_poll: the request is not finished yet */
#define SA_EINVAL    -1     /* bad argument: non-ACGT base, n or m out of range, window past the reference end */
#define SA_ENOMEM    -2     /* device or host memory could not be obtained */
#define SA_ECUDA     -3     /* a CUDA call failed (message in sa_last_error) */
#define SA_ETIMEOUT  -4     /* sa_poll: timeout_ms elapsed */
#define SA_EOVERFLOW -5     /* the CIGAR buffer is too small; *cigar_used says how much is needed */
#define SA_ENOTFOUND -6     /* sa_poll: unknown or already collected ticket */
#define SA_EBUSY     -7     /* sa_submit: the request can never fit the server's memory budget */

#define SA_NO_SCORE  INT32_MIN   /* "no second-best location" */

#define SA_MAX_READ   1024u      /* longest read (n) */
#define SA_MAX_WINDOW 65536u     /* longest window (m) */

/* job flags */
#define SA_RC 1u                 /* align the reverse complement of the read */

/* result flags */
#define SA_RES_EMPTY     1u      /* LOCAL: no positive-scoring alignment */
#define SA_RES_BELOW_MIN 2u      /* score < min_score: no traceback was run */

typedef struct {
    int32_t match, mismatch, gap_open, gap_extend;   /* BWA magnitudes, >= 0 */
} sa_scoring;

typedef enum { SA_LOCAL = 0, SA_GLOCAL = 1 } sa_mode;

/* execution form (same results; see sa_align_batch) */
typedef enum {
    SA_FORM_BATCHED = 0,   /* length-bucketed persistent launches, score pass + reduced traceback */
    SA_FORM_PLAIN   = 1    /* fixed-size batches, one full-direction fill launch + one traceback each */
} sa_form;

typedef struct {
    sa_scoring sc;
    int32_t mode;          /* sa_mode */
    int32_t want_cigar;    /* 0: score, ends and second best only (begins -1, no CIGAR) */
    int32_t width;         /* 0 auto, 16 (packed 16-bit + exact int32 rerun), 32 */
    int32_t min_score;     /* results below it get SA_RES_BELOW_MIN and no traceback; INT32_MIN disables */
    int32_t form;          /* sa_form */
    int32_t profile;       /* nonzero: time each phase with CUDA events (sa_last_stats) */
    int32_t arena_mb;      /* cap on the traceback's rectangle direction arena in MiB (0: 60 % of
                              free device memory); a batch whose rectangles exceed it runs their
                              direction pass in waves (sa_stats.waves); results never depend on it */
    int32_t _reserved;
} sa_params;

typedef struct {           /* 32 bytes */
    uint64_t read_off;     /* offset of the read in the reads buffer */
    uint32_t read_len;     /* n, 1..SA_MAX_READ */
    uint32_t flags;        /* SA_RC */
    uint64_t ref_pos;      /* window start in the reference (0-based) */
    uint32_t win_len;      /* m, 1..SA_MAX_WINDOW, ref_pos + m <= reference length */
    uint32_t _pad;
} sa_job;

typedef struct {           /* 56 bytes */
    int32_t score;         /* best score (0 with SA_RES_EMPTY) */
    int32_t second;        /* second best at a distinct location, SA_NO_SCORE if none */
    int32_t read_begin;    /* 0-based in the (reverse-complemented if SA_RC) read; -1 if no traceback */
    int32_t read_end;      /* exclusive */
    int64_t ref_begin;     /* absolute reference coordinate; -1 if no traceback */
    int64_t ref_end;       /* exclusive */
    int64_t second_ref_end;/* exclusive end column of the second best; -1 if none */
    uint32_t cigar_off;    /* first op in the cigar buffer */
    uint32_t cigar_len;    /* number of ops */
    uint32_t flags;        /* SA_RES_* */
    uint32_t _pad;
} sa_result;

typedef struct {           /* statistics of the last call on a reference or server */
    uint64_t jobs, cells;          /* sum of n*m */
    uint64_t rect_cells;           /* cells of the direction-bit pass */
    uint32_t overflow_reruns;      /* jobs recomputed in 32-bit after a 16-bit overflow */
    uint32_t waves;                /* direction-arena waves */
    uint32_t fill_launches;        /* score-pass kernel launches */
    uint32_t kernel_launches;      /* all kernels launched by the call */
    float ms_stage, ms_fill, ms_rerun, ms_rect, ms_traceback, ms_finalize;  /* with profile != 0 */
    float ms_total;                /* device time of the whole call (profile != 0) */
    uint32_t diag_jobs;            /* traced jobs whose optimal path is all matches (no direction pass) */
    uint32_t band_jobs;            /* ... whose optimal paths fit a band of 8, 16, 32 or 64 diagonals */
    uint32_t rect_jobs;            /* ... neither: whole-rectangle direction pass */
    uint32_t jobs16;               /* jobs whose score pass ran in 16-bit packed pairs */
    uint32_t graph_replays;        /* 1 if the score segment ran as a replayed CUDA graph
                                      (graphs are used when profile == 0) */
    uint32_t rect_pairs;           /* rectangle jobs whose pass ran two to a lane group in
                                      16-bit halves (byte heights, buckets with many of them) */
} sa_stats;

typedef struct sa_reference sa_reference;
typedef struct sa_server sa_server;

/* Default parameters: scoring 1/2/2/1 (the BWA-form scheme consistent with the
 * paper's default tolerance of one gap up to 68 bp or 23 one-base gaps for a
 * 100 bp read), LOCAL, CIGAR on, width auto, min_score INT32_MIN, batched form. */
void sa_default_params(sa_params* p);

/* Pack len ACGT characters (case-insensitive; anything else is SA_EINVAL) to a
 * 2-bit device-resident reference on `device`.  The input is copied. */
int sa_create_reference(const char* acgt, uint64_t len, int device, sa_reference** out);
int sa_destroy_reference(sa_reference* ref);
uint64_t sa_reference_length(const sa_reference* ref);

/* Align n_jobs jobs.  Host buffers: jobs[n_jobs], reads[reads_len] (ASCII),
 * out[n_jobs], cigar[cigar_cap] (ops, compacted in job order; cigar_used, if
 * not NULL, receives the number of ops written or needed).  cuda_stream is a
 * cudaStream_t or NULL for a library-owned stream; the call returns when the
 * results are in `out`.  Inputs are validated; on an error nothing is written
 * to `out`.  Calls on the same reference are serialised. */
int sa_align_batch(sa_reference* ref, const sa_params* params, const sa_job* jobs, uint32_t n_jobs,
                   const char* reads, uint64_t reads_len, sa_result* out, uint32_t* cigar,
                   uint64_t cigar_cap, uint64_t* cigar_used, void* cuda_stream);

/* The same with every buffer in device memory of the reference's device
 * (d_jobs, d_reads, d_out, d_cigar); the work is queued on cuda_stream and the
 * call returns after it completes.  cigar_used is a host pointer. */
int sa_align_batch_dev(sa_reference* ref, const sa_params* params, const sa_job* d_jobs,
                       uint32_t n_jobs, const char* d_reads, uint64_t reads_len, sa_result* d_out,
                       uint32_t* d_cigar, uint64_t cigar_cap, uint64_t* cigar_used,
                       void* cuda_stream);

/* Allocation-free score pass.  This entry point has no counterpart in the
 * paper; it exists for callers that cannot let a library allocate device
 * memory: code inside a host framework that owns all device memory through its
 * own allocator, and latency-sensitive callers that cannot afford the
 * device-wide synchronisation cudaMalloc / cudaFree may imply.
 *
 * It computes what sa_align_batch_dev computes with want_cigar = 0 (score,
 * read/reference ends, second best and its end, flags; begins -1, no CIGAR;
 * params->want_cigar, width and form are ignored; the scores and mode are
 * checked with the same limits as sa_align_batch) on device buffers d_jobs,
 * d_reads and d_out of the reference's device, and calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its intermediate arrays live in one
 * file-scope device array of SA_NOALLOC_SCRATCH_BYTES that every device which
 * loads the library holds until the process exits.  A batch whose
 * intermediate arrays do not fit (about 30 + 4*ceil(max_n/16) bytes per job
 * plus 4*max_m bytes per resident lane group) is rejected with SA_EINVAL and a
 * message giving the size needed: split it.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the array and it keeps the previous call's
 * contents (the call clears what must start at zero), so calls whose work
 * overlaps on the GPU -- on different streams or from different host threads
 * -- race on it and must not be issued.  The work runs on cuda_stream (NULL:
 * the reference's own stream); the call reads the batch's validation status
 * back to the host between its kernels and returns only when all of its work
 * has completed. */
#define SA_NOALLOC_SCRATCH_BYTES (32u << 20)
int sa_align_batch_noalloc(sa_reference* ref, const sa_params* params, const sa_job* d_jobs,
                           uint32_t n_jobs, const char* d_reads, uint64_t reads_len,
                           sa_result* d_out, void* cuda_stream);

/* Statistics of the last sa_align_batch / sa_align_batch_dev call on ref. */
int sa_last_stats(const sa_reference* ref, sa_stats* out);

/* Tuned plan (SOAP3-dp classifies candidates by complexity before the DP,
 * Methods section 3; here the bucketing and lane-group choice are tuned on the
 * device).  Every reference holds a plan: the lane-group configuration serving
 * each read length and the width of each configuration's score pass.  The
 * default maps n to the smallest configuration with L*K >= n and picks 16-bit
 * where no job of a bucket can overflow.
 *
 * sa_tune times the score pass (CUDA events, second of two runs, CIGAR off) of
 * the sample `jobs` (host buffers, same layout as sa_align_batch; up to 65,536
 * jobs per length class, classes with fewer than 256 jobs are skipped) under
 * each candidate -- the default configuration, the next larger K with the same
 * lane count, the first 32-lane configuration that covers the class; 16- and
 * 32-bit where LOCAL 16-bit applies -- and keeps the fastest in the plan.
 * *classes_tuned (nullable) receives the number of length classes tuned.
 * Results never depend on the plan.  It must not run concurrently with other
 * calls on the same reference or with a server on it.
 *
 * sa_plan_get copies the plan (a fixed-size byte string, *needed bytes) to
 * out[size] (SA_EOVERFLOW if size is too small); sa_plan_set installs one
 * (SA_EINVAL if it is malformed or maps a read length to a configuration with
 * fewer rows); plan == NULL restores the default.  A saved plan is the plan
 * cache between runs on the same GPU type. */
int sa_tune(sa_reference* ref, const sa_params* params, const sa_job* jobs, uint32_t n_jobs,
            const char* reads, uint64_t reads_len, uint32_t* classes_tuned);
int sa_plan_get(const sa_reference* ref, void* out, uint64_t size, uint64_t* needed);
int sa_plan_set(sa_reference* ref, const void* plan, uint64_t size);

/* Serving: a background thread admits submitted requests while device memory
 * (hbm_budget bytes, 0 = 80% of free memory) and in-flight slots allow, and runs
 * them on a pool of streams, so requests overlap on the device.  The reference
 * stays device-resident.  max_inflight = 0 picks a default. */
int sa_server_create(sa_reference* ref, const sa_params* params, uint64_t hbm_budget,
                     uint32_t max_inflight, sa_server** out);
/* Queue one request; jobs and reads are copied before the call returns. */
int sa_submit(sa_server* srv, const sa_job* jobs, uint32_t n_jobs, const char* reads,
              uint64_t reads_len, uint64_t* ticket);
/* Wait up to timeout_ms (0 = just check, < 0 = forever) for a request.  On
 * SA_OK the results are copied to out/cigar and the ticket is released; on
 * SA_PENDING / SA_ETIMEOUT nothing is written.  SA_EOVERFLOW keeps the ticket. */
int sa_poll(sa_server* srv, uint64_t ticket, int timeout_ms, sa_result* out, uint32_t* cigar,
            uint64_t cigar_cap, uint64_t* cigar_used);
int sa_server_destroy(sa_server* srv);

/* Counters of a server since its creation (host side, exact). */
typedef struct {
    uint64_t submitted;         /* requests accepted by sa_submit */
    uint64_t completed;         /* requests finished with SA_OK */
    uint64_t failed;            /* requests finished with an error */
    uint64_t batches;           /* device batches run (a failed batch rerun request by request counts once) */
    uint64_t coalesced;         /* requests that joined the batch of an earlier queued request */
    uint64_t admission_stalls;  /* batches whose head request first waited for the memory budget */
    uint64_t max_queue;         /* longest queue seen at submit */
    uint64_t jobs;              /* jobs of all batches */
} sa_server_stats;
int sa_server_get_stats(sa_server* srv, sa_server_stats* out);

/* Message of the last error on the calling thread ("" if none). */
const char* sa_last_error(void);

/* ---------------------------------------------------------------------------
 * Reads with several candidate windows (Methods sections 4 "Effort limit for
 * dynamic programming" and 5 "Paired-end alignment"; mapping quality from the
 * Experiments section).
 *
 * A read's candidate windows are consecutive jobs of a batch: read r owns jobs
 * read_first[r] .. read_first[r+1]-1 (read_first: n_reads + 1 ascending uint32
 * offsets starting at 0; a read may have none).  With paired selection reads
 * 2p and 2p+1 are the two ends of fragment p.
 */
#define SA_NO_JOB   0xFFFFFFFFu
#define SA_MAPQ_MAX 60

/* sa_read_result.flags */
#define SA_READ_ALIGNED      1u   /* some candidate aligned (not SA_RES_EMPTY / SA_RES_BELOW_MIN) */
#define SA_READ_PAIRED       2u   /* selected as one end of a pair */
#define SA_READ_PROPER       4u   /* properly paired: orientation and fragment length as expected */
#define SA_READ_MATE_ALIGNED 8u   /* the other end aligned */
#define SA_READ_REVERSE     16u   /* the chosen job carries SA_RC */

/* orientations of properly paired ends */
#define SA_PAIR_FR 0   /* one end forward, the other SA_RC; the fragment runs from the forward
                          end's first reference base to the reverse end's last (Illumina) */
#define SA_PAIR_FF 1   /* both ends on one strand; forward: end 1 first, SA_RC: end 2 first (SOLiD) */

typedef struct {
    sa_scoring sc;          /* the scoring the jobs were aligned with (sets the MAPQ scale) */
    int32_t paired;         /* 0: every read alone; 1: reads 2p, 2p+1 are the ends of pair p */
    int32_t orientation;    /* SA_PAIR_FR or SA_PAIR_FF */
    int64_t frag_min;       /* proper fragment lengths, inclusive, 0 <= frag_min <= frag_max */
    int64_t frag_max;
} sa_select_params;

typedef struct {            /* 32 bytes, one per read */
    uint32_t job;           /* chosen job (batch index); SA_NO_JOB if no candidate aligned */
    int32_t score;          /* its score (0 without one) */
    int32_t second;         /* best other hit of the read at least n from the chosen reference end
                               (every aligned candidate's best and its own second), SA_NO_SCORE if none */
    int32_t mapq;           /* 0..SA_MAPQ_MAX */
    uint32_t flags;         /* SA_READ_* */
    uint32_t n_cand;        /* candidates of the read */
    int64_t frag_len;       /* properly paired: fragment length (both ends); else 0 */
} sa_read_result;

/* Effort limit: of each read's candidates keep the `ceiling` (>= 1) with the
 * most supporting seeds (support[j] per job); equal support goes to the
 * earlier candidate.  Kept jobs are written in their input order to kept
 * (capacity: all jobs), their batch indices to kept_from, and the per-read
 * offsets into them to kept_first (n_reads + 1 entries); *n_kept (host) gets
 * the total.  Device buffers; runs on cuda_stream (NULL: the reference's
 * stream) and returns when done.  SA_EINVAL for a read_first that is not
 * ascending from 0 or a zero ceiling.  `ref` only names the device. */
int sa_effort_limit_dev(sa_reference* ref, const sa_job* jobs, const uint32_t* support,
                        const uint32_t* read_first, uint32_t n_reads, uint32_t ceiling,
                        sa_job* kept, uint32_t* kept_from, uint32_t* kept_first,
                        uint32_t* n_kept, void* cuda_stream);
/* The same with host buffers (n_jobs = read_first[n_reads]). */
int sa_effort_limit(sa_reference* ref, const sa_job* jobs, const uint32_t* support,
                    const uint32_t* read_first, uint32_t n_reads, uint32_t ceiling,
                    sa_job* kept, uint32_t* kept_from, uint32_t* kept_first, uint32_t* n_kept);

/* Per-read selection from the results of the reads' candidate jobs (results
 * of sa_align_batch* on jobs[0 .. read_first[n_reads])):
 *  - best: the aligned candidate with the highest score, then the smallest
 *    reference end, then the earliest job;
 *  - second: as in sa_read_result;
 *  - mapq: SA_MAPQ_MAX without a second hit, 0 if second >= score, else
 *    20 * (score - second) / (match + mismatch) (integer), at most SA_MAPQ_MAX;
 *  - paired: among the proper (end 1, end 2) combinations of aligned
 *    candidates, the highest summed score (then the earliest end-1 job, then
 *    the earliest end-2 job) is chosen for both ends; the pair's second best is
 *    the highest proper combination that moves an end by its read length or
 *    more, and each end's mapq is the larger of the pair's and its own.
 *    Without a proper combination each end is selected on its own.
 * Results that ran without a traceback (ref_begin -1) are taken as ungapped:
 * first base ref_end - n.  Device buffers; runs on cuda_stream (NULL: the
 * reference's stream) and returns when done. */
int sa_select_dev(sa_reference* ref, const sa_select_params* sp, const sa_job* jobs,
                  const sa_result* results, const uint32_t* read_first, uint32_t n_reads,
                  sa_read_result* out, void* cuda_stream);
/* The same with host buffers. */
int sa_select(sa_reference* ref, const sa_select_params* sp, const sa_job* jobs,
              const sa_result* results, const uint32_t* read_first, uint32_t n_reads,
              sa_read_result* out);

/* ---------------------------------------------------------------------------
 * Seeding front end: candidate windows of whole reads (the paper's step 3:
 * Methods, "Implementation details of SOAP3-dp", and "Effort limit for
 * dynamic programming").  Seeds -- substrings of fixed length -- are taken at
 * regular intervals along each read and along its reverse complement and
 * matched exactly against the reference with an FM index on the device; the
 * regions their hits point to become candidate windows, each with its number
 * of supporting seeds, in the layout sa_effort_limit[_dev] takes.
 *
 * Definitions (the paper leaves these values to its supplementary material):
 *  - seeds of a read of length n, per strand (the read, then its reverse
 *    complement): offsets 0, seed_step, 2*seed_step, ... while offset +
 *    seed_len <= n; a seed occurring more than max_occ times is repetitive
 *    and contributes nothing;
 *  - a hit of the seed at offset o on reference position p implies the
 *    strand's sequence starts at d = p - o (its diagonal); a read strand's hits
 *    sorted by diagonal form one region while neighbouring diagonals differ by
 *    at most `join`;
 *  - a region's window is [max(0, d_min - pad), min(L, d_max + n + pad)), at
 *    most SA_MAX_WINDOW long; its support is the number of distinct seeds with
 *    a hit in it;
 *  - a read's candidates are its forward regions by d_min, then its
 *    reverse-complement regions (job flag SA_RC) by d_min.
 */
typedef struct {
    uint32_t seed_len;     /* 12..32 */
    uint32_t seed_step;    /* >= 1; at most 128 seeds per strand */
    uint32_t max_occ;      /* >= 1; seeds per strand x max_occ <= 8192 */
    uint32_t pad;          /* <= 65536 */
    uint32_t join;         /* <= 65536 */
    uint32_t _reserved;
} sa_seed_params;

typedef struct sa_seed_index sa_seed_index;

/* Defaults: seed_len 20, seed_step 10, max_occ 256, pad 24, join 16. */
void sa_default_seed_params(sa_seed_params* p);

/* Build the seed index of a reference (its packed bases are read back from the
 * device): the suffix order of the reference, its BWT in 64-byte chunks (the
 * counts of A, C, G, T before the chunk and 192 two-bit BWT entries, so one
 * backward-search step reads one chunk per interval end), the row interval of
 * every 12-base pattern, and the full suffix array (4 bytes a row) on the
 * reference's device.  Built on the host with all cores, once per reference;
 * about 12 bytes a base of host memory while it runs.  References of up to
 * 2^32 - 33 bases (SA_EINVAL beyond).  The reference must outlive the index. */
int sa_seed_index_create(sa_reference* ref, sa_seed_index** out);
int sa_seed_index_destroy(sa_seed_index* idx);
/* Reference length and device bytes the index holds (either pointer may be NULL). */
int sa_seed_index_info(const sa_seed_index* idx, uint64_t* ref_len, uint64_t* device_bytes);

/* Candidate windows of n_reads reads: read r is reads[read_off[r] ..
 * read_off[r] + read_len[r]) (ASCII A/C/G/T, 1..SA_MAX_READ bases; anything
 * else is SA_EINVAL).  Writes the candidates as jobs (read_off, read_len of the
 * read; flags 0 or SA_RC; ref_pos, win_len of the window) to cand and their
 * support to support (capacity cand_cap each), read r's candidates being
 * read_first[r] .. read_first[r+1]-1 (n_reads + 1 entries).  *n_cand (host)
 * receives the number of candidates; if it exceeds cand_cap the call returns
 * SA_EOVERFLOW and writes no candidate.  Device buffers; runs on cuda_stream
 * (NULL: the reference's stream) and returns when done.  Calls on one index
 * are serialised. */
int sa_seed_candidates_dev(sa_seed_index* idx, const sa_seed_params* params, const char* d_reads,
                           uint64_t reads_len, const uint64_t* d_read_off, const uint32_t* d_read_len,
                           uint32_t n_reads, sa_job* d_cand, uint32_t* d_support, uint32_t* d_read_first,
                           uint64_t cand_cap, uint64_t* n_cand, void* cuda_stream);
/* The same with host buffers. */
int sa_seed_candidates(sa_seed_index* idx, const sa_seed_params* params, const char* reads, uint64_t reads_len,
                       const uint64_t* read_off, const uint32_t* read_len, uint32_t n_reads, sa_job* cand,
                       uint32_t* support, uint32_t* read_first, uint64_t cand_cap, uint64_t* n_cand);

#ifdef __cplusplus
}
#endif

#endif /* SA_H */
