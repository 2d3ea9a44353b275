// One configuration's wavefront kernels (compiled once per configuration with
// -DSA_CFG=<index>, so the translation units build in parallel).
#include "rect16.cuh"
#include "kernels.h"

#ifndef SA_CFG
#error "compile with -DSA_CFG=<configuration index>"
#endif

namespace sa {

namespace {
constexpr int kL = kCfgs[SA_CFG].L;
constexpr int kK = kCfgs[SA_CFG].K;

// dynamic shared memory of a 128-thread block: the score pass's profile
template <bool DIR, bool BEST>
constexpr size_t smem_bytes() { return (BEST != DIR) ? 4 * prof_words_per_warp<kK>() * sizeof(int32_t) : 0; }

template <int MODE, bool DIR, bool BEST, bool HGT = false>
void prepare() {
    static bool done = false;   // attribute set once per process (same on every device)
    if (!done) {
        cudaFuncSetAttribute(k_fill32<kL, kK, MODE, DIR, BEST, HGT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes<DIR, BEST>());
        done = true;
    }
}

template <int MODE, bool DIR, bool BEST, bool HGT = false>
void launch_one(const FillLaunch& fl) {
    prepare<MODE, DIR, BEST, HGT>();
    k_fill32<kL, kK, MODE, DIR, BEST, HGT><<<fl.grid, fl.block, smem_bytes<DIR, BEST>(), fl.stream>>>(fl.args);
}

constexpr size_t smem16_bytes() { return 4 * prof16_words_per_warp<kK>() * sizeof(int32_t); }

void prepare16() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_fill16<kL, kK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem16_bytes());
        cudaFuncSetAttribute(k_fill16h<kL, kK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem16_bytes());
        done = true;
    }
}

template <int MODE, bool DIR, bool BEST, bool HGT = false>
int blocks_per_sm() {
    prepare<MODE, DIR, BEST, HGT>();
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill32<kL, kK, MODE, DIR, BEST, HGT>, 128,
                                                  smem_bytes<DIR, BEST>());
    return nb;
}
}  // namespace

template <>
void launch_fill<SA_CFG>(const FillLaunch& fl) {
    const bool local = fl.args.sc.mode == SA_LOCAL;
    switch (fl.kind) {
    case kFillScore:
        local ? launch_one<SA_LOCAL, false, true>(fl) : launch_one<SA_GLOCAL, false, true>(fl);
        break;
    case kFillRect:
        local ? launch_one<SA_LOCAL, true, false>(fl) : launch_one<SA_GLOCAL, true, false>(fl);
        break;
    case kFillPlain:
        local ? launch_one<SA_LOCAL, true, true>(fl) : launch_one<SA_GLOCAL, true, true>(fl);
        break;
    case kFillScore16:
        prepare16();
        k_fill16<kL, kK><<<fl.grid, fl.block, smem16_bytes(), fl.stream>>>(fl.args);
        break;
    case kFillRectH:            // byte heights: LOCAL only
        if (local) launch_one<SA_LOCAL, true, false, true>(fl);
        break;
    case kFillRectH16:          // byte heights, two jobs a lane group: LOCAL only
        prepare16();
        if (local) k_fill16h<kL, kK><<<fl.grid, fl.block, smem16_bytes(), fl.stream>>>(fl.args);
        break;
    default:
        break;
    }
}

template <>
int fill_blocks_per_sm<SA_CFG>(int kind, int mode) {
    const bool local = mode == SA_LOCAL;
    switch (kind) {
    case kFillScore:
        return local ? blocks_per_sm<SA_LOCAL, false, true>() : blocks_per_sm<SA_GLOCAL, false, true>();
    case kFillRect:
        return local ? blocks_per_sm<SA_LOCAL, true, false>() : blocks_per_sm<SA_GLOCAL, true, false>();
    case kFillPlain:
        return local ? blocks_per_sm<SA_LOCAL, true, true>() : blocks_per_sm<SA_GLOCAL, true, true>();
    case kFillRectH:
        return local ? blocks_per_sm<SA_LOCAL, true, false, true>() : 0;
    case kFillScore16: {
        prepare16();
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill16<kL, kK>, 128, smem16_bytes());
        return nb;
    }
    case kFillRectH16: {
        prepare16();
        int nb = 0;
        if (local) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fill16h<kL, kK>, 128, smem16_bytes());
        return nb;
    }
    }
    return 0;
}

}  // namespace sa
