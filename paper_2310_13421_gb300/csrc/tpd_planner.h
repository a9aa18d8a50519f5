// Host-side pass planner (see tpd_plan.h for the plan structures).
#pragma once

#include <string>

#include "tpd_plan.h"

namespace tpd {

// Bytes of one element as the kernels hold it in registers / shared memory.
int arith_elem_bytes(int dtype, int precision);

// Split n levels into passes and lay out tiles and stages.  tile_bits_opt /
// max_levels_opt: 0 = defaults.  Returns false (with *err) if impossible.
bool build_plan(int n, int dtype, int precision, int tile_bits_opt, int max_levels_opt, Plan* plan,
                std::string* err);

std::string describe_plan(const Plan& plan);

}  // namespace tpd
