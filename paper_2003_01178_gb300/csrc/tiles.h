// Compiled tile shapes (threads per block x items per thread) of each operator.
// Section 3.3 sweeps block sizes 32..1024 and 1/2/4 items per thread and settles on
// 128 x 4 for its microbenchmarks and 256 x 8 for the full queries; the paper's
// 128 x 4 shape is kept as one variant of every scan operator next to wider tiles that
// suit bulk asynchronous copies on sm_103a.  Entry 0 is the default.
#pragma once

#include "crystal.h"

namespace crys {

struct TileShape {
  int threads;
  int items;
};

constexpr int kMaxVariants = 4;

constexpr TileShape kTiles[CRYS_NUM_OPS][kMaxVariants] = {
    /* SELECT      */ {{256, 16}, {128, 16}, {512, 8}, {128, 4}},
    /* PROJECT     */ {{256, 16}, {256, 8}, {512, 8}, {128, 4}},
    /* PROBE       */ {{256, 16}, {256, 8}, {512, 8}, {128, 4}},
    /* PLAN        */ {{256, 8}, {512, 8}, {512, 4}, {128, 4}},
    /* SHARED_SCAN */ {{256, 4}, {256, 8}, {128, 8}, {128, 4}},
    /* SORT        */ {{256, 32}, {256, 24}, {512, 16}, {256, 16}},
    /* TAGGED_SCAN */ {{1024, 4}, {256, 4}, {512, 4}, {256, 8}},
};

constexpr int kNumVariants[CRYS_NUM_OPS] = {4, 4, 4, 4, 4, 4, 4};

}  // namespace crys
