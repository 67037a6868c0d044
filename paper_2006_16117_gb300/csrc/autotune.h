// A small run-time autotuner: the first calls of a launch site with a given
// key try each candidate variant in turn, timed with CUDA events on the
// launching stream; once every candidate has its samples (the events are read
// when they have completed, never waited on) the fastest is used from then on.
// Only for candidates that compute bit-identical results, so the choice never
// changes an answer.
#pragma once

#include <cuda_runtime.h>

#include <string>

namespace sim {

// Candidate to launch for this call (0 .. ncand-1).  When it returns with
// *timing set, record the launch between autotune_end's events.
int autotune_begin(const std::string& key, int ncand, cudaStream_t st, bool* timing);
void autotune_end(const std::string& key, cudaStream_t st);
// The chosen candidate (-1 while still tuning); for reports.
int autotune_choice(const std::string& key);

}  // namespace sim
