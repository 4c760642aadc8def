// Helpers of the host runtime shared with the other host entry points.
#pragma once

#include <string>

#include "../../include/densify.h"
#include "desc.cuh"

namespace dz {

// Filter constants of one stage (log2(e)-scaled Gaussian coefficients, spatial table).
void fill_stage_args(StageArgs &a, const densify_stage &st, int pool, int override_sparse);
// Empty when the parameters are valid, else the reason.
std::string check_params(const densify_params &p);
// The message densify_last_error(NULL) returns on this thread.
void set_thread_error(const std::string &m);

}  // namespace dz
