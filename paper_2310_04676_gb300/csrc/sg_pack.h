// Warp orders of the packings (sg_pack.cpp).
#pragma once

#include <cstdint>
#include <vector>

#include "sg_internal.h"

namespace sg {

// Warp order of a packing (SG_PACK_*): order[w] = the warp of the plan's
// class-grouped order that position w holds (the identity for SG_PACK_CLASS).
std::vector<int32_t> packing_order(const Plan& plan, int packing);

}  // namespace sg
