// Dispatch from a configuration index to its translation unit.
#include <utility>

#include "kernels.h"

namespace sa {

namespace {

using LaunchFn = void (*)(const FillLaunch&);
using BlocksFn = int (*)(int, int);

template <int... C>
constexpr void fill_tables(std::integer_sequence<int, C...>, LaunchFn* launch, BlocksFn* blocks) {
    ((launch[C] = &launch_fill<C>), ...);
    ((blocks[C] = &fill_blocks_per_sm<C>), ...);
}

struct Tables {
    LaunchFn launch[kNumCfg];
    BlocksFn blocks[kNumCfg];
    Tables() { fill_tables(std::make_integer_sequence<int, kNumCfg>{}, launch, blocks); }
};

const Tables& tables() {
    static const Tables t;
    return t;
}

}  // namespace

void launch_fill_cfg(int cfg, const FillLaunch& fl) {
    if (cfg >= 0 && cfg < kNumCfg) tables().launch[cfg](fl);
}

int fill_max_blocks_per_sm(int cfg, int kind, int mode) {
    return cfg >= 0 && cfg < kNumCfg ? tables().blocks[cfg](kind, mode) : 0;
}

}  // namespace sa
