// batch.cu -- the batched fine sweep: all slices of all unconverged problems
// in one cooperative launch.
//
// Seats: task t needs G_t CTAs.  Every CTA of the launch repeatedly takes the
// next seat from a global counter; seat s belongs to the task t with
// seat0_t <= s < seat0_t + G_t and makes the CTA rank s - seat0_t of that
// task's group.  Seats are handed out in task order, so at most one group is
// incomplete at any time and its members only wait for CTAs that are busy
// with earlier, complete groups: every wait ends (and is bounded in time
// anyway).  Tasks come largest first, so small tasks fill the tail.  A rank
// works on the same particle range as in a per-problem launch with the same
// group size, so a batched sweep reproduces the per-problem results bit for
// bit.
#include "batch.cuh"
#include "fine_kernel.cuh"

namespace mmp {

// Two CTAs per SM, 128 registers a thread and four quads in flight, as the
// per-problem kernel: the batch sizes its shared memory for the largest
// quads-per-thread count of its problems, which at the measured caps (~27)
// leaves room for two CTAs per SM anyway (sized for four, the kernel spilled
// and ran config 5 11 % slower).
constexpr int kBatchOcc = 2;

template <typename R, bool MULT>
__global__ void __launch_bounds__(kTPB, kBatchOcc) k_fine_batch(const BatchArgs b) {
  __shared__ GroupShared sh;
  // the current task's arguments (raw storage: FineArgs has member
  // initialisers, which a __shared__ variable cannot run)
  __shared__ __align__(16) unsigned char sa_raw[sizeof(FineArgs)];
  FineArgs& sa = *reinterpret_cast<FineArgs*>(sa_raw);
  __shared__ int s_task, s_rank;
  const int tid = threadIdx.x;
  if (tid == 0) sh.abort = 0;
  QuadStore<R, 0> xs;
  xs.bind();
  const int n_tasks = b.header[0];
  const int total = b.header[1];
  for (;;) {
    if (tid == 0) {
      const int seat = (int)atomicAdd(b.seat_counter, 1u);
      int t = -1;
      if (seat < total) {
        int lo = 0, hi = n_tasks - 1;  // last task with seat0 <= seat
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (b.tasks[mid].seat0 <= seat) lo = mid;
          else hi = mid - 1;
        }
        t = lo;
        s_rank = seat - b.tasks[t].seat0;
      }
      s_task = t;
    }
    __syncthreads();
    const int t = s_task;
    if (t < 0) return;
    const BatchTask tk = b.tasks[t];
    if (tid == 0) {
      sa = b.probs[tk.prob];
      sa.src = tk.src_buf < 0 ? nullptr : b.bufs[2 * tk.prob + tk.src_buf];
      sa.dst = b.bufs[2 * tk.prob + tk.dst_buf];
      sa.dst_fixed = 0;
      sa.aff_fixed = 0;
      sa.stats_fixed = 0;
    }
    __syncthreads();
    Group grp;
    grp.part = b.partials + (size_t)tk.seat0 * kSeatDoubles;
    grp.flags = b.flags + tk.seat0;
    grp.tags = b.tags + (size_t)tk.seat0 * kSlots;
    grp.status = sa.status;
    grp.limit_ns = sa.wait_limit_ns;
    grp.G = tk.G;
    grp.g = s_rank;
    grp.epoch = 0;
    if (!fine_task<R, 0, MULT, kStepUnrollSmem>(sa, tk.slice, s_rank, grp, sh, xs)) return;
    __syncthreads();  // every thread is done with sa and s_task
  }
}

// One CTA: per-problem task and seat counts, a block-wide scan over the
// problems in order, then each thread writes the tasks of its problems.
constexpr int kPlanThreads = 1024;

__global__ void __launch_bounds__(kPlanThreads) k_batch_plan(const BatchPlanArgs a) {
  __shared__ int s_t[kPlanThreads], s_s[kPlanThreads];
  __shared__ int s_active;
  const int tid = threadIdx.x;
  if (tid == 0) s_active = 0;
  const bool go = *(volatile int*)a.remaining > 0;
  const int per = (a.n + kPlanThreads - 1) / kPlanThreads;
  const int r0 = min(a.n, tid * per), r1 = min(a.n, r0 + per);
  auto next_sweep = [&](int i) -> int {  // k of problem i, or 0 if it does not sweep
    const double* ctl = a.ctl[i];
    return (go && ctl[3] == 0.0) ? (int)ctl[2] + 1 : 0;
  };
  int nt = 0, ns = 0, na = 0;
  for (int r = r0; r < r1; ++r) {
    const int i = a.order[r];
    const int k = next_sweep(i);
    if (k > 0) {
      const int cnt = a.N[i] - k + 1;
      nt += cnt;
      ns += cnt * a.G[i];
      na += 1;
    }
  }
  s_t[tid] = nt;
  s_s[tid] = ns;
  __syncthreads();
  if (na > 0) atomicAdd(&s_active, na);
  for (int off = 1; off < kPlanThreads; off <<= 1) {  // inclusive scan
    const int vt = tid >= off ? s_t[tid - off] : 0;
    const int vs = tid >= off ? s_s[tid - off] : 0;
    __syncthreads();
    s_t[tid] += vt;
    s_s[tid] += vs;
    __syncthreads();
  }
  int t = s_t[tid] - nt, seat = s_s[tid] - ns;
  for (int r = r0; r < r1; ++r) {
    const int i = a.order[r];
    const int k = next_sweep(i);
    a.sweep[i] = k > 0 ? k : -1;
    if (k == 0) continue;
    for (int sl = k - 1; sl < a.N[i]; ++sl) {
      a.tasks[t++] = BatchTask{i, sl, k == 1 ? -1 : ((k - 1) & 1), k & 1, seat, a.G[i]};
      seat += a.G[i];
    }
  }
  __syncthreads();
  if (tid == kPlanThreads - 1) {
    a.header[0] = s_t[tid];
    a.header[1] = s_s[tid];
    a.header[2] = s_active;
    *a.seat_counter = 0u;
    if (go) *a.remaining -= 1;
  }
}

cudaError_t launch_batch_plan(const BatchPlanArgs& args, cudaStream_t stream) {
  k_batch_plan<<<1, kPlanThreads, 0, stream>>>(args);
  return cudaGetLastError();
}

const void* fine_batch_kernel(int precision, bool mult) {
  if (precision == MMP_MIXED)
    return mult ? (const void*)k_fine_batch<float, true> : (const void*)k_fine_batch<float, false>;
  return mult ? (const void*)k_fine_batch<double, true> : (const void*)k_fine_batch<double, false>;
}

// Cooperative launch through cudaLaunchKernelEx with the cooperative
// attribute: the form stream capture records as a cooperative kernel node
// (cudaLaunchCooperativeKernel itself cannot be captured).
cudaError_t launch_fine_batch(int precision, bool mult, int grid, size_t smem, const BatchArgs& args,
                              cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kTPB);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BatchArgs copy = args;
  void* params[] = {&copy};
  return cudaLaunchKernelExC(&cfg, fine_batch_kernel(precision, mult), params);
}

}  // namespace mmp
