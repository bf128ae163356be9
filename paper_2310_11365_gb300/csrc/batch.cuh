// batch.cuh -- one persistent launch per Parareal sweep over the slices of
// many problems.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fine.cuh"

namespace mmp {

// One (problem, slice) task of a batched sweep.  Tasks are listed in the
// order seats are handed out; task t owns seats [seat0, seat0 + G) of the
// sweep, and its group's flags, tagged words and publication slots are
// those of its seats (flags + seat0, tags + kSlots seat0, partials +
// kSeatDoubles seat0).
struct BatchTask {
  int prob;     // index into the problem records
  int slice;    // slice n
  int src_buf;  // -1: every slice reads u0 (first sweep), else sweep buffer of slice n - 1
  int dst_buf;  // sweep buffer written
  int seat0;    // first seat
  int G;        // CTAs of the task (the problem's group size)
};

struct BatchArgs {
  const FineArgs* probs;   // per-problem records (slice fields unused)
  void* const* bufs;       // [2 * n_probs] sweep buffer bases (B0, B1 per problem)
  const BatchTask* tasks;  // [n_tasks] by ascending seat0
  const int* header;       // [0] n_tasks, [1] total seats
  unsigned* seat_counter;  // zeroed per sweep
  unsigned* flags;         // [total seats] epoch flags, zeroed per sweep
  unsigned long long* tags;  // [total seats] x kSlots tagged step words, zeroed per sweep
  double* partials;        // [total seats] x kSeatDoubles doubles
};

const void* fine_batch_kernel(int precision, bool mult);
cudaError_t launch_fine_batch(int precision, bool mult, int grid, size_t smem, const BatchArgs& args,
                              cudaStream_t stream);

}  // namespace mmp
