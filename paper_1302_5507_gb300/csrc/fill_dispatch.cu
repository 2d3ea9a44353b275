// Dispatch from a configuration index to its translation unit.
#include "kernels.h"

namespace sa {

void launch_fill_cfg(int cfg, const FillLaunch& fl) {
    switch (cfg) {
    case 0: launch_fill<0>(fl); break;
    case 1: launch_fill<1>(fl); break;
    case 2: launch_fill<2>(fl); break;
    case 3: launch_fill<3>(fl); break;
    case 4: launch_fill<4>(fl); break;
    case 5: launch_fill<5>(fl); break;
    case 6: launch_fill<6>(fl); break;
    case 7: launch_fill<7>(fl); break;
    case 8: launch_fill<8>(fl); break;
    case 9: launch_fill<9>(fl); break;
    case 10: launch_fill<10>(fl); break;
    case 11: launch_fill<11>(fl); break;
    case 12: launch_fill<12>(fl); break;
    case 13: launch_fill<13>(fl); break;
    default: break;
    }
}

int fill_max_blocks_per_sm(int cfg, int kind, int mode) {
    switch (cfg) {
    case 0: return fill_blocks_per_sm<0>(kind, mode);
    case 1: return fill_blocks_per_sm<1>(kind, mode);
    case 2: return fill_blocks_per_sm<2>(kind, mode);
    case 3: return fill_blocks_per_sm<3>(kind, mode);
    case 4: return fill_blocks_per_sm<4>(kind, mode);
    case 5: return fill_blocks_per_sm<5>(kind, mode);
    case 6: return fill_blocks_per_sm<6>(kind, mode);
    case 7: return fill_blocks_per_sm<7>(kind, mode);
    case 8: return fill_blocks_per_sm<8>(kind, mode);
    case 9: return fill_blocks_per_sm<9>(kind, mode);
    case 10: return fill_blocks_per_sm<10>(kind, mode);
    case 11: return fill_blocks_per_sm<11>(kind, mode);
    case 12: return fill_blocks_per_sm<12>(kind, mode);
    case 13: return fill_blocks_per_sm<13>(kind, mode);
    default: return 0;
    }
}

}  // namespace sa
