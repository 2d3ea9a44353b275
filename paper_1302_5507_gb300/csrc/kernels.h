// Host-side launch wrappers of the libsa kernels (stage.cu, fill_cfg*.cu).
#pragma once

#include "sa_internal.cuh"

namespace sa {

struct PlanStats {                 // filled by the plan kernel (device)
    uint32_t max_n, max_m;
    unsigned long long cells;
    uint32_t bad_job;              // first invalid job (UINT32_MAX: none)
    uint32_t bad_read;             // first job with a non-ACGT base (UINT32_MAX: none)
    uint32_t max_wave;             // last direction-arena wave with work
    uint32_t bad_walk;             // first job whose traceback left its rectangle (internal error)
    uint32_t dbg_site;             // SA_DEBUG builds: smallest store site that was out of range
    unsigned long long bad_ref_pos;
};

struct TbOut {                     // traceback result of one job
    int32_t n_rev;                 // ops written (reverse order) to the temporary slot
    int32_t read_begin;            // 0-based
    int32_t ref_begin_rel;         // 0-based, relative to the job's window start
};

struct BandArgs {                  // banded direction pass of one class
    const uint32_t* ref;
    int64_t ref_len;
    const sa_job* jobs;
    const uint32_t* rpack;
    uint32_t rw;
    const Rect* rect;
    const uint32_t* list;          // job ids of this class
    uint32_t count;
    uint32_t* arena;               // this class's region
    uint64_t warp_stride;          // words per 32 list entries (max_n * B/8 * 32)
    Score sc;
    // the walk from the best cell runs in the same thread right after the pass
    const JobState* state;
    uint32_t* tmp_ops;             // reversed ops, tmp_stride words per job
    uint32_t tmp_stride;
    TbOut* tb;
    unsigned* err_job;             // smallest job whose walk failed (internal error)
    uint64_t region_cap;           // words of this class's region (SA_DEBUG checks)
    uint32_t n_state;
    unsigned* dbg;
};

struct BandLayout {                // where the traceback finds band nibbles
    const uint32_t* arena;
    uint64_t base[kNumBand];       // word offset of the band 16 / 32 / 64 regions
    uint64_t warp_stride[kNumBand];
};



void launch_pack_ref(const uint8_t* ascii, uint64_t len, uint64_t base_off, uint32_t* words,
                     unsigned long long* bad_pos, cudaStream_t st);
void launch_plan(const sa_job* jobs, uint32_t n_jobs, uint64_t reads_len, int64_t ref_len,
                 const uint8_t* plan_cfg, uint16_t* key, uint32_t* hist, PlanStats* stats, cudaStream_t st);
void launch_plan_order(const uint16_t* key, uint32_t n_jobs, const uint32_t* hist,
                       uint32_t* key_off, uint32_t* cursor, uint32_t* order, cudaStream_t st);
void launch_collect_overflow(const uint32_t* order, uint32_t n_pos, const JobState* state,
                             const uint32_t* cfg_begin, uint32_t* list, uint32_t* cnt,
                             cudaStream_t st);
void launch_pack_reads(const sa_job* jobs, uint32_t n_jobs, const uint8_t* reads, uint32_t* rpack,
                       uint32_t rw, unsigned* bad_job, cudaStream_t st);
void launch_rect_plan(const sa_job* jobs, const uint32_t* order, uint32_t n_pos, const uint32_t* cfg_begin,
                      const JobState* state, const Score& sc, int32_t min_score, int allow_band,
                      Rect* rect, uint64_t* sizes, uint32_t* const* lists, uint32_t* cls_count,
                      uint32_t* rect_flag, int heights, const uint32_t* ref, const uint32_t* rpack, uint32_t rw,
                      cudaStream_t st);
// the rectangle-pass jobs compacted in bucketed order (rect_pos = exclusive scan of
// rect_flag, total its sum), their positions in that order (list_pos), and each
// bucket's first index in the list (rect_begin[kNumCfg + 1])
uint64_t rect_sort_bytes();        // scratch of launch_rect_list
void launch_rect_list(const uint32_t* order, uint32_t n_pos, const uint32_t* rect_flag, const Rect* rect,
                      void* sort_scratch, uint64_t* bsum, uint64_t* total, uint32_t* list, uint32_t* list_pos,
                      uint32_t* rect_begin, cudaStream_t st);
// heights: the byte-height form (LOCAL and every score below 255; the band
// regions then hold B/4 words a row instead of B/8)
// returns the number of kernels it launched
int launch_band(int cls, const BandArgs& a, bool heights, cudaStream_t st);
void launch_rect_assign(const uint32_t* order, const uint32_t* list_pos, uint32_t n, const uint64_t* offs,
                        uint64_t wave_words, Rect* rect, uint32_t* max_wave, cudaStream_t st);
void launch_plain_rect(const sa_job* jobs, uint32_t j0, uint32_t nb, uint64_t stride, Rect* rect,
                       cudaStream_t st);
void launch_scan_u64(const uint64_t* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* total,
                     cudaStream_t st);
void launch_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* total,
                     cudaStream_t st);
// rectangle jobs whose pass stored byte heights (LOCAL, every score below 255):
// the walk re-derives its decisions from the heights and the bases
struct HeightWalk {
    int on;
    const uint32_t* ref;           // padded packed reference
    const uint32_t* rpack;         // packed reads, rw words per job
    uint32_t rw;
    Score sc;
};
// part 0: every job of [job_begin, job_begin + n_jobs); part 1: the same jobs but the
// rectangle jobs' height walks; part 2: those walks for list[job_begin ..] (job ids)
void launch_traceback(const sa_job* jobs, uint32_t job_begin, uint32_t n_jobs, const JobState* state,
                      const Rect* rect, const uint32_t* arena, const BandLayout& band, int wave,
                      int mode, int plain, int cfg_force, int32_t min_score, uint32_t* tmp_ops,
                      uint32_t tmp_stride, TbOut* tb, unsigned* err_job, const HeightWalk& hw,
                      cudaStream_t st, const uint32_t* list = nullptr, int part = 0);
void launch_iota(uint32_t* p, uint32_t n, cudaStream_t st);
void launch_cigar_count(const sa_job* jobs, uint32_t n_jobs, const JobState* state, const TbOut* tb,
                        int mode, int want_cigar, int32_t min_score, uint32_t* count,
                        cudaStream_t st);
void launch_finalize(const sa_job* jobs, uint32_t n_jobs, const JobState* state, const TbOut* tb,
                     const uint32_t* count, const uint64_t* coff, const uint32_t* tmp_ops,
                     uint32_t tmp_stride, int mode, int want_cigar, int32_t min_score,
                     sa_result* out, uint32_t* cigar, cudaStream_t st);

// the wavefront kernels, dispatched by configuration index
void launch_fill_cfg(int cfg, const FillLaunch& fl);
int fill_max_blocks_per_sm(int cfg, int kind, int mode);

// what other translation units may read of a reference handle (api.cu)
struct RefView {
    const uint32_t* d_words;       // padded packed reference
    uint64_t len;                  // bases
    int device;
    int num_sms;
    cudaStream_t own;              // the reference's own stream
};
RefView ref_view(const sa_reference* R);
int set_error(int code, const char* msg);   // sets sa_last_error() for the calling thread
// validates params->sc and params->mode (SA_EINVAL with a message) and fills *sc
int check_scoring(const sa_params* p, Score* sc);

// scan scratch: number of uint64 block sums needed for n elements
inline uint64_t scan_bsum_len(uint64_t n) { return (n + 1023) / 1024 + 1; }

}  // namespace sa
