// Host-side helpers shared by the translation units that implement the C ABI
// (bipm.cu and noalloc.cu): argument validation, option defaults, the error
// message of bipm_last_error and the layout of the per-call counters.
#pragma once

#include <string>

#include "../../include/bipm.h"
#include "common.cuh"

namespace bipm {

// Per-call device counters: [0] queue / slot counter, [1] spare-slot counter,
// [2] time-budget flag, [3] unused, [4..5] device start time of the call (ns).
constexpr int kCounterInts = 8;

// Points the launch record's time budget at the counters of its call.
inline void set_budget(Params& P, int* counter, int time_limit_ms) {
  P.time_limit_ns = (unsigned long long)time_limit_ms * 1000000ull;
  P.timeout_flag = counter + 2;
  P.t0 = reinterpret_cast<unsigned long long*>(counter + 4);
}

// Records the message bipm_last_error() returns.
void set_last_error(const std::string& msg);
// The documented defaults of bipm_options.
bipm_options default_options();
// Validated dims of one problem structure (0, or an error code with message).
int dims_from_desc(const bipm_problem_desc* desc, Dims* out);
// Options with defaults filled in and validated (o_out), and their device copy.
int options_from(const bipm_options* opt, bipm_options* o_out, Options* dev);
// The queue kernel of a precision form for problems of nq quadrotors.
void* queue_kernel_ptr(int precision, int nq);

}  // namespace bipm
