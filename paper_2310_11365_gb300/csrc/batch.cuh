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

// Device-side builder of a batched sweep's task list, so that sweeps can be
// enqueued back to back (and captured in a CUDA graph) without the host:
// every problem whose control block says "not done" contributes its slices
// k-1 .. N-1 (k = sweeps done + 1), problems in `order` (largest P n_f
// first), seats handed out in task order.  A sweep budget (`remaining`)
// stops the sweeps after the requested number.
struct BatchPlanArgs {
  const double* const* ctl;  // [n] control blocks: ctl[2] sweeps done, ctl[3] done
  const int* order;          // [n] problem indices, largest P n_f first (stable)
  const int* N;              // [n] slices
  const int* G;              // [n] CTAs per slice
  int n;
  BatchTask* tasks;          // out: task list
  int* header;               // out: [0] tasks, [1] seats, [2] problems swept
  int* sweep;                // out: [n] sweep index k of each problem, -1 if idle
  unsigned* seat_counter;    // zeroed
  int* remaining;            // sweeps still allowed (decremented when > 0)
};
cudaError_t launch_batch_plan(const BatchPlanArgs& args, cudaStream_t stream);

const void* fine_batch_kernel(int precision, bool mult);
cudaError_t launch_fine_batch(int precision, bool mult, int grid, size_t smem, const BatchArgs& args,
                              cudaStream_t stream);

}  // namespace mmp
