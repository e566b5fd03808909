// tuning.h -- process-wide tuning parameters (set through bp_set_tuning; the
// autotuner in the Python package measures candidates and installs the best).
#pragma once
#include "../../include/bp128.h"

namespace bp {

using Tuning = bp_tuning;

// Current parameters (defaults until bp_set_tuning is called).
const Tuning &tuning();

}  // namespace bp
