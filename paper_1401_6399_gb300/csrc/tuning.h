// tuning.h -- process-wide tuning parameters (set through bp_set_tuning; the
// autotuner in the Python package measures candidates and installs the best).
#pragma once
#include "../../include/bp128.h"

namespace bp {

using Tuning = bp_tuning;

// Current parameters (defaults until bp_set_tuning is called).
const Tuning &tuning();

// Polls of one look-back state word before a wait gives up (default).
constexpr uint32_t kLookbackSpinLimit = 1u << 22;

// The look-back wait limits in force: the spin limit (the tuning's, or the
// default when it is 0) and the tile that publishes nothing (UINT32_MAX:
// none).
void lookback_limits(uint32_t &spin_limit, uint32_t &withhold);

}  // namespace bp
