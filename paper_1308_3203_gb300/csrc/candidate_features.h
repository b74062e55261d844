// Feature extraction of candidate instances on the host cores, started
// asynchronously on the library's worker threads (features.cpp).
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>

#include "racecheck.h"

namespace rc {

struct FeatureJob;

// Validates every candidate (throws std::string on a bad one, before any
// work starts) and starts computing RC_N_FEATURES floats per candidate into
// out (which must stay valid until features_wait returns).  `participants`
// threads take part (0: as many as pay off); with caller_helps the calling
// thread is one of them, and does its share inside features_wait.
std::shared_ptr<FeatureJob> features_start(const rc_bytecode *const *bcs, const uint32_t *groups,
                                           const uint32_t *group_size, const rc_input *inputs, size_t n,
                                           float *out, unsigned participants, bool caller_helps);
bool features_finished(const FeatureJob &j);
// Candidates not yet started are skipped; features_wait still returns only
// once no thread works on the job.
void features_cancel(FeatureJob &j);
// Returns when the job is finished (or cancelled and idle); throws
// std::string if a candidate failed.
void features_wait(FeatureJob &j);

}  // namespace rc
