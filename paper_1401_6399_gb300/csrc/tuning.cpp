// tuning.cpp -- storage of the tuning parameters.
#include "tuning.h"

#include <mutex>

namespace bp {
namespace {
std::mutex g_mu;
Tuning g_tuning = {4u, 1u, 8u, 0u, 0u, 0u, {0, 0}};
}  // namespace

const Tuning &tuning() { return g_tuning; }

void lookback_limits(uint32_t &spin_limit, uint32_t &withhold) {
  std::lock_guard<std::mutex> g(g_mu);
  spin_limit = g_tuning.lookback_spin_limit ? g_tuning.lookback_spin_limit : kLookbackSpinLimit;
  withhold = g_tuning.withhold_tile ? g_tuning.withhold_tile - 1u : 0xFFFFFFFFu;
}

}  // namespace bp

extern "C" {

int bp_get_tuning(bp_tuning *out) {
  if (!out) return BP_ERR_ARG;
  std::lock_guard<std::mutex> g(bp::g_mu);
  *out = bp::g_tuning;
  return BP_OK;
}

int bp_set_tuning(const bp_tuning *in) {
  if (!in) return BP_ERR_ARG;
  if (in->dense_blocks < 1 || in->dense_blocks > 8) return BP_ERR_ARG;
  if (in->query_chunk_blocks < 1 || in->query_chunk_blocks > 8) return BP_ERR_ARG;
  if (in->query_warps != 4 && in->query_warps != 8) return BP_ERR_ARG;
  if (in->lookback_spin_limit > bp::kLookbackSpinLimit) return BP_ERR_ARG;
  if (in->merge_span > 64u) return BP_ERR_ARG;
  std::lock_guard<std::mutex> g(bp::g_mu);
  bp::g_tuning = *in;
  return BP_OK;
}

}  // extern "C"
