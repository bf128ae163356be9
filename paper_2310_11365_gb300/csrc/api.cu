// api.cu -- the C-ABI of libmmp: descriptor validation, workspace layout,
// launch planning of the fine kernel, and the Parareal orchestration
// (Eq. mM_parareal_other_k_NEW) on one stream.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "adjoint.cuh"
#include <nvtx3/nvToolsExt.h>

#include "batch.cuh"
#include "driver.cuh"
#include "fine.cuh"
#include "misc.cuh"
#include "mmp_internal.cuh"
static_assert(mmp::kNGrad == MMP_N_THETA, "adjoint gradient length");

namespace mmp {
cudaError_t launch_fma_probe(int precision, void* sink, long long iters, int grid, cudaStream_t stream);
int step_probe_quads(int form);
cudaError_t prepare_step_probe(int form);
cudaError_t launch_step_probe(int form, float* sink, int steps, int grid, cudaStream_t stream);
cudaError_t launch_wait_probe(double* partials, unsigned* flags, unsigned long long* tags, unsigned* status, int G,
                              unsigned long long limit_ns, int channel, cudaStream_t stream);
const void* fine_kernel_f32(int nq, bool mult, int family);
const void* fine_kernel_f64(int nq, bool mult, int family);

const void* fine_kernel(int precision, int layout, int nq, bool mult, int family) {
  const int t = layout == kLayoutSmem ? 0 : nq;
  if (layout != kLayoutSmem && nq < 1) return nullptr;
  return precision == MMP_MIXED ? fine_kernel_f32(t, mult, family) : fine_kernel_f64(t, mult, family);
}

size_t fine_smem_bytes(int precision, int layout, int nq, int family) {
  if (layout != kLayoutSmem) return 0;
  // the plane rotator keeps sin x and cos x beside x
  const size_t per = family == MMP_FAMILY_ROTATOR ? 3 : 1;
  return per * (size_t)nq * kTPB * 4 * (precision == MMP_MIXED ? sizeof(float) : sizeof(double));
}

cudaError_t launch_fine(int precision, int layout, int nq, bool mult, int grid, const FineArgs& args,
                        cudaStream_t stream, int family) {
  const void* fn = fine_kernel(precision, layout, nq, mult, family);
  if (fn == nullptr) return cudaErrorInvalidValue;
  FineArgs copy = args;
  void* params[] = {&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTPB), params,
                                     fine_smem_bytes(precision, layout, nq, family), stream);
}
}  // namespace mmp

using namespace mmp;

namespace {

// An NVTX range over a library call (a tool such as Nsight Systems shows the
// phases of a run on its timeline; without a tool attached it costs a call).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

// written by any thread that sees a CUDA call fail
std::atomic<int> g_last_cuda_error{0};

// Records a failed CUDA call; MMP_DEBUG=1 also names it on stderr.
int cuda_fail(cudaError_t e, const char* what, int line) {
  g_last_cuda_error.store((int)e, std::memory_order_relaxed);
  static const bool debug = [] {
    const char* v = std::getenv("MMP_DEBUG");
    return v != nullptr && v[0] == '1';
  }();
  if (debug) std::fprintf(stderr, "libmmp: %s (api.cu:%d): %s\n", what, line, cudaGetErrorString(e));
  return MMP_ERR_CUDA;
}
#define MMP_CUDA(call)                         \
  do {                                         \
    cudaError_t e_ = (call);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call, __LINE__); \
  } while (0)

constexpr size_t kAlign = 256;

// Raises a kernel's dynamic shared-memory limit to what its static shared
// memory leaves of the per-block opt-in maximum; returns that limit.
int allow_dynamic_smem(const void* fn, int device, size_t* limit) {
  int optin = 0;
  MMP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  cudaFuncAttributes attr;
  MMP_CUDA(cudaFuncGetAttributes(&attr, fn));
  const int dyn = optin - (int)attr.sharedSizeBytes;
  if (dyn <= 0) return MMP_ERR_UNSUPPORTED;
  MMP_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
  *limit = (size_t)dyn;
  return MMP_OK;
}

struct Prob {
  mmp_problem_desc d;
  int I = 1, nf = 1, nc = 1, max_sweeps = 1;
  double h = 0, sqrt_h = 0, dT = 0, hc = 0;
  int Q = 0;
  long long pitch = 0;
  size_t esz = 8;
  bool mult = false;
  uint32_t key0 = 0, key1 = 0;
  // launch plan of the fine kernel
  int layout = kLayoutRegs, nq = 1, G = 1, slots_max = 1;
  // device memory inside the caller's workspace
  char* u0 = nullptr;
  char* B[2] = {nullptr, nullptr};
  char* S[2] = {nullptr, nullptr};
  double *stats = nullptr, *stats_u0 = nullptr, *ser_stats = nullptr, *tmp_stats = nullptr;
  double *rho = nullptr, *cache = nullptr, *aff = nullptr, *ctl = nullptr, *partials = nullptr;
  unsigned *flags = nullptr, *status = nullptr;
  unsigned long long* tags = nullptr;  // followed by flags: one block, cleared per launch
  // host view of the iteration
  int sweeps = 0;
  bool lifted = false, done = false, converged = false;
  double last_change = 0.0;
  std::vector<int> out_buf;  // which B buffer holds the latest F_n output of slice n
  int fine_pending = 0;      // sweep whose fine phase ran alone (mmp_sweep_fine), awaiting its driver
  // adjoint state: the forward run recorded into adj_ws
  bool adj_ready = false;
  void* adj_ws = nullptr;
  int adj_ckpt_every = 1;
};

struct Device {
  int dev = 0, sms = 0;
};

int query_device(Device& d) {
  MMP_CUDA(cudaGetDevice(&d.dev));
  MMP_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, d.dev));
  return MMP_OK;
}

bool finite_all(const mmp_problem_desc& d) {
  const double v[] = {d.c3, d.c1, d.kappa, d.c0, d.B, d.BE, d.B0, d.m0, d.s0, d.T, d.dt,
                      d.coarse_h, d.threshold, d.threshold2, d.threshold3, d.tol, d.K, d.g};
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

int validate(const mmp_problem_desc& d) {
  if (!finite_all(d)) return MMP_ERR_INVALID_ARG;
  if (!(d.T > 0) || !(d.dt > 0) || !(d.coarse_h > 0) || d.s0 < 0 || d.tol < 0) return MMP_ERR_INVALID_ARG;
  if (d.N < 1 || d.N > 65535) return MMP_ERR_INVALID_ARG;
  if (d.P < 1 || d.P > (1LL << 31) - 8) return MMP_ERR_INVALID_ARG;
  if (d.n_regions < 1 || d.n_regions > kMaxRegions) return MMP_ERR_INVALID_ARG;
  if (d.n_regions >= 3 && !(d.threshold2 > d.threshold)) return MMP_ERR_INVALID_ARG;
  if (d.n_regions >= 4 && !(d.threshold3 > d.threshold2)) return MMP_ERR_INVALID_ARG;
  if (d.variant < MMP_UNIMODAL || d.variant > MMP_LEARNING) return MMP_ERR_INVALID_ARG;
  if (d.precision != MMP_FP64 && d.precision != MMP_MIXED) return MMP_ERR_INVALID_ARG;
  if (d.coarse_model < MMP_COARSE_CLOSURE || d.coarse_model > MMP_COARSE_TAYLOR1) return MMP_ERR_INVALID_ARG;
  if (d.family != MMP_FAMILY_POLY && d.family != MMP_FAMILY_ROTATOR) return MMP_ERR_INVALID_ARG;
  if (d.family == MMP_FAMILY_ROTATOR) {
    // the plane rotator: additive noise, one region (Sec. 5's unimodal example)
    if (d.B != 0.0 || d.BE != 0.0) return MMP_ERR_INVALID_ARG;
    if (d.n_regions != 1) return MMP_ERR_UNSUPPORTED;
  }
  const double steps = std::ceil((d.T / d.N) / d.dt - 1e-9);
  if (!(steps >= 1) || steps > 2e9) return MMP_ERR_INVALID_ARG;
  const double csteps = std::ceil((d.T / d.N) / d.coarse_h - 1e-9);
  if (!(csteps >= 1) || csteps > 1e7) return MMP_ERR_INVALID_ARG;
  return MMP_OK;
}

void derive(Prob& p) {
  const mmp_problem_desc& d = p.d;
  p.I = d.n_regions;
  p.dT = d.T / d.N;
  p.nf = std::max(1, (int)std::ceil(p.dT / d.dt - 1e-9));
  p.h = p.dT / p.nf;
  p.sqrt_h = std::sqrt(p.h);
  p.nc = std::max(1, (int)std::ceil(p.dT / d.coarse_h - 1e-9));
  p.hc = p.dT / p.nc;
  p.Q = (int)((d.P + 3) / 4);
  p.pitch = 4LL * p.Q;
  p.esz = d.precision == MMP_MIXED ? 4 : 8;
  p.mult = d.family == MMP_FAMILY_POLY && (d.B != 0.0 || d.BE != 0.0);
  p.key0 = (uint32_t)(d.seed & 0xffffffffull);
  p.key1 = (uint32_t)(d.seed >> 32);
  const int mi = d.max_iter > 0 ? d.max_iter : d.N;
  p.max_sweeps = std::min(d.N, mi);
  p.out_buf.assign(d.N, -1);
}

// Measured launch shapes (mmp_set_tuning, usually filled by mmp_autotune):
// quads per thread for a precision and a range of P.  Later entries win.
struct TuneEntry {
  int precision;
  long long p_lo, p_hi;
  int nq;
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;

int tuned_nq(int precision, long long P) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (auto it = g_tune.rbegin(); it != g_tune.rend(); ++it)
    if (it->precision == precision && it->p_lo <= P && P <= it->p_hi) return it->nq;
  return 0;
}

// Launch plan of the fine kernel: particle layout (registers or shared
// memory), quads per thread (nq) and CTAs per slice (G).  The group size is
// fixed per problem so that every launch reduces in the same order (the
// serial reference then matches the sweeps bit for bit).  Among the shapes
// whose group fits in the co-resident CTAs, pick the smallest modelled sweep
// time: waves of concurrent slices times the per-step time, with the per-SM
// load in quad-steps and a fixed per-step latency for the group barrier.
// The layout is the shared-memory one unless MMP_FINE_LAYOUT=regs;
// MMP_FINE_NQ=<k>, else a tuning entry (mmp_set_tuning) for the problem's
// precision and P, selects the largest reachable count of at most k quads
// per thread.
int plan(Prob& p, const Device& dev, int batch_nq = 0) {
  int tuned = batch_nq > 0 ? 0 : tuned_nq(p.d.precision, p.d.P);
  if (batch_nq > 0) {
    // many problems share one launch: the most particles per thread (the
    // fewest CTAs, hence group barriers, per slice) within the cap
    p.layout = kLayoutSmem;
    p.nq = (int)std::min<long long>(batch_nq, std::max<long long>(1, ((long long)p.Q + kTPB - 1) / kTPB));
    p.G = (int)(((long long)p.Q + (long long)p.nq * kTPB - 1) / ((long long)p.nq * kTPB));
    p.slots_max = 1;
    // the per-problem kernel still serves lifting and serial runs
    const void* fn = fine_kernel(p.d.precision, kLayoutSmem, p.nq, p.mult, p.d.family);
    size_t limit = 0;
    const int rc = allow_dynamic_smem(fn, dev.dev, &limit);
    if (rc) return rc;
    if (fine_smem_bytes(p.d.precision, kLayoutSmem, p.nq, p.d.family) > limit) return MMP_ERR_UNSUPPORTED;
    int occ = 0;
    MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB,
                                                           fine_smem_bytes(p.d.precision, kLayoutSmem, p.nq, p.d.family)));
    if ((long long)occ * dev.sms < p.G) return MMP_ERR_UNSUPPORTED;
    return MMP_OK;
  }
  const char* env = std::getenv("MMP_FINE_LAYOUT");
  const int layout = (env != nullptr && std::strcmp(env, "regs") == 0 && p.d.family == MMP_FAMILY_POLY)
                         ? kLayoutRegs : kLayoutSmem;
  const char* env_nq = std::getenv("MMP_FINE_NQ");
  const int max_nq_l = layout == kLayoutSmem ? (p.esz == 4 ? 32 : 16) : (p.esz == 4 ? 8 : 4);
  if (tuned > 0 && (layout != kLayoutSmem || tuned > max_nq_l)) tuned = 0;
  if (tuned > 0) {
    // a measured shape is a saturated-throughput optimum: use it only if the
    // problem's slices fill the resident CTAs at that shape
    const void* fn = fine_kernel(p.d.precision, layout, tuned, p.mult, p.d.family);
    size_t limit = 0;
    int occ = 0;
    const size_t smem = fine_smem_bytes(p.d.precision, layout, tuned, p.d.family);
    const int rc = allow_dynamic_smem(fn, dev.dev, &limit);
    if (rc) return rc;
    if (smem <= limit) MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB, smem));
    const long long G = ((long long)p.Q + (long long)tuned * kTPB - 1) / ((long long)tuned * kTPB);
    if (occ < 1 || (long long)p.d.N * G < (long long)occ * dev.sms) tuned = 0;
  }
  const int force_nq = env_nq != nullptr ? std::atoi(env_nq) : tuned;
  const int max_nq = layout == kLayoutSmem ? (p.esz == 4 ? 32 : 16) : (p.esz == 4 ? 8 : 4);
  int occ_of[33] = {0};
  for (int nq = 1; nq <= max_nq; ++nq) {
    int occ = 0;
    const void* fn = fine_kernel(p.d.precision, layout, nq, p.mult, p.d.family);
    if (fn == nullptr) return MMP_ERR_UNSUPPORTED;
    const size_t smem = fine_smem_bytes(p.d.precision, layout, nq, p.d.family);
    if (layout == kLayoutSmem) {
      size_t limit = 0;
      const int rc = allow_dynamic_smem(fn, dev.dev, &limit);
      if (rc) return rc;
      if (smem > limit) break;
    }
    MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB, smem));
    occ_of[nq] = occ;
  }
  // quad-steps per cycle per SM (the rotator evaluates two sine-cosine pairs per particle-step)
  const double quad_rate = (p.esz == 4 ? 0.8 : 0.02) * (p.d.family == MMP_FAMILY_ROTATOR ? 0.4 : 1.0);
  double best = INFINITY;
  int best_nq = 0, best_G = 0, best_slots = 0;
  const int N = p.d.N;
  const int g_max = std::min<long long>((long long)dev.sms * 32, p.Q);
  for (int G = 1; G <= g_max; ++G) {
    const long long qpc = (p.Q + G - 1) / G;
    const int nq = (int)std::max<long long>(1, (qpc + kTPB - 1) / kTPB);
    if (nq > max_nq || occ_of[nq] < 1) continue;
    if (force_nq > 0 && nq > force_nq) continue;
    const int S = dev.sms * occ_of[nq];
    if (G > S) continue;
    const int slots = std::min(N, S / G);
    const int waves = (N + slots - 1) / slots;
    const int per_sm = (slots * G + dev.sms - 1) / dev.sms;
    // the rotator's step is latency-bound (a group exchange per step): an SM
    // with fewer than the two CTAs the kernel is built for runs them at their
    // own rate, not the SM's, so its throughput scales with the CTAs it holds
    // (also where its shared memory fits only one) (measured on
    // the Sec. 5 example: one CTA per SM ran 7 % (mixed) and 22 % (FP64)
    // slower than the best shape with two)
    const double fill = p.d.family == MMP_FAMILY_ROTATOR ? std::min(1.0, per_sm / 2.0) : 1.0;  // built for 2 per SM
    const double step = per_sm * (double)kTPB * nq / (quad_rate * fill) + (G > 1 ? 2500.0 : 400.0);
    const double cost = waves * step;
    // forced (MMP_FINE_NQ or a tuning entry): the largest reachable count
    // not above the forced one, else the cheapest by the cost model
    const bool better = force_nq > 0 ? (nq > best_nq || (nq == best_nq && cost < best * (1 - 1e-12)))
                                     : cost < best * (1 - 1e-12);
    if (better) {
      best = cost;
      best_nq = nq;
      best_G = G;
      best_slots = S / G;
    }
  }
  if (best_G == 0) return MMP_ERR_UNSUPPORTED;
  p.layout = layout;
  p.nq = best_nq;
  p.G = best_G;
  p.slots_max = best_slots;
  return MMP_OK;
}

struct Carver {
  char* base;
  size_t off = 0;
  size_t take(size_t bytes) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    const size_t at = off;
    off += bytes;
    return at;
  }
};

// Bytes of a problem's synchronisation block: tagged step words
// [slot][kSlots][G], then epoch flags [slot][G].
size_t sync_bytes(const Prob& p) {
  return (sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * (size_t)p.slots_max * p.G;
}

// Lays out (or, with base == nullptr, sizes) one problem's workspace.
size_t layout(Prob& p, char* base, size_t start) {
  Carver c{base, start};
  const int N = p.d.N;
  const size_t row = (size_t)p.pitch * p.esz;
  auto ptr = [&](size_t bytes) -> char* {
    const size_t at = c.take(bytes);
    return base ? base + at : nullptr;
  };
  p.u0 = ptr(row);
  p.B[0] = ptr(row * N);
  p.B[1] = ptr(row * N);
  p.S[0] = ptr(row);
  p.S[1] = ptr(row);
  p.stats = (double*)ptr(sizeof(double) * kStat * N);
  p.stats_u0 = (double*)ptr(sizeof(double) * kStat);
  p.ser_stats = (double*)ptr(sizeof(double) * kStat * (N + 1));
  p.tmp_stats = (double*)ptr(sizeof(double) * kStat);
  p.rho = (double*)ptr(sizeof(double) * kMom * (N + 1));
  p.cache = (double*)ptr(sizeof(double) * 2 * kMaxRegions * N);
  p.aff = (double*)ptr(sizeof(double) * kMaxRegions * kAff * (N + 1));
  p.ctl = (double*)ptr(sizeof(double) * 16);
  p.partials = (double*)ptr(sizeof(double) * kSeatDoubles * (size_t)p.slots_max * p.G);
  p.tags = (unsigned long long*)ptr(sync_bytes(p));
  p.flags = base ? (unsigned*)(p.tags + (size_t)p.slots_max * kSlots * p.G) : nullptr;
  p.status = (unsigned*)ptr(sizeof(unsigned) * 4);
  return c.off;
}

unsigned long long wait_limit_ns() {
  const char* e = std::getenv("MMP_WAIT_LIMIT_MS");
  const double ms = e ? std::atof(e) : 5000.0;
  return (unsigned long long)(std::max(1.0, ms) * 1e6);
}

}  // namespace

struct mmp_ctx {
  std::vector<Prob> probs;
  char* ws = nullptr;   // the caller's workspace and the bytes the layout uses
  size_t ws_used = 0;
  cudaStream_t stream = nullptr;
  Device dev;
  unsigned long long limit_ns = 0;
  std::vector<double> host_ctl;
  // device-time accounting of the fine kernel (events on `stream`)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  double fine_ms = 0.0, fine_steps = 0.0;
  long long fine_launches = 0, other_launches = 0;
  // batched sweeps (several problems of one precision and noise form)
  bool batch = false;
  int batch_grid = 0;
  size_t batch_smem = 0;
  FineArgs* b_probs = nullptr;
  void** b_bufs = nullptr;
  BatchTask* b_tasks = nullptr;
  int* b_header = nullptr;
  unsigned* b_seat = nullptr;
  unsigned* b_flags = nullptr;
  unsigned long long* b_tags = nullptr;
  double* b_partials = nullptr;
  DriverArgs* b_dargs = nullptr;
  int* b_sweep = nullptr;
  double* b_summary = nullptr;
  const double** b_ctlp = nullptr;  // device-side task builder inputs
  int* b_order = nullptr;
  int* b_N = nullptr;
  int* b_G = nullptr;
  int* b_remaining = nullptr;
  size_t b_seats_cap = 0;
  std::vector<double> h_summary;
  // a CUDA graph of kGraphSweeps batched sweeps (built on first use on a
  // private stream: the context stream may be the legacy default stream,
  // which cannot be captured)
  cudaGraphExec_t b_graph = nullptr;
  cudaStream_t cap_stream = nullptr;
  bool b_graph_failed = false;
  ~mmp_ctx() {
    if (b_graph != nullptr) cudaGraphExecDestroy(b_graph);
    if (cap_stream != nullptr) cudaStreamDestroy(cap_stream);
    for (auto& pr : pending) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }
};

namespace {

// Quads per thread of every problem when several problems are batched:
// MMP_BATCH_NQ overrides (launch-shape sweeps).
int g_batch_nq[2] = {0, 0};  // mmp_set_batch_nq, by precision (0: default)

int batch_nq_cap(int precision) {
  const char* e = std::getenv("MMP_BATCH_NQ");
  if (e != nullptr && std::atoi(e) > 0) return std::atoi(e);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const int set = g_batch_nq[precision == MMP_MIXED ? 1 : 0];
    if (set > 0) return set;
  }
  return precision == MMP_MIXED ? 26 : 13;
}

int prepare(const mmp_problem_desc* descs, int n, std::vector<Prob>& probs, Device& dev) {
  if (descs == nullptr || n < 1) return MMP_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const int v = validate(descs[i]);
    if (v) return v;
  }
  int rc = query_device(dev);
  if (rc) return rc;
  probs.resize(n);
  const int bnq = n > 1 ? batch_nq_cap(descs[0].precision) : 0;
  for (int i = 0; i < n; ++i) {
    probs[i].d = descs[i];
    derive(probs[i]);
    rc = plan(probs[i], dev, bnq);
    if (rc) return rc;
  }
  return MMP_OK;
}

// The problem-constant part of the fine kernel's arguments.
FineArgs fine_args_of(const Prob& p, unsigned long long limit_ns) {
  FineArgs a;
  const mmp_problem_desc& d = p.d;
  a.nc3 = -d.c3; a.c1 = d.c1; a.kappa = d.kappa; a.c0 = d.c0;
  a.B = d.B; a.BE = d.BE; a.B0 = d.B0;
  a.K = d.K; a.gpin = d.g;
  a.h = p.h; a.sqrt_h = p.sqrt_h; a.nf = p.nf;
  a.P = d.P; a.Q = p.Q; a.pitch = p.pitch;
  a.n_regions = p.I; a.thr = d.threshold; a.thr2 = d.threshold2; a.thr3 = d.threshold3;
  a.key0 = p.key0; a.key1 = p.key1; a.ptag = d.problem_tag;
  a.slice_begin = 0; a.n_tasks = 0;
  a.src0 = p.u0; a.src = nullptr; a.dst = nullptr; a.dst_fixed = 0;
  a.aff = p.aff; a.aff_fixed = 0;
  a.stats = p.stats; a.stats_fixed = 0;
  a.G = p.G;
  a.nq = p.nq;
  a.partials = p.partials; a.flags = p.flags; a.tags = p.tags; a.status = p.status;
  a.wait_limit_ns = limit_ns;
  return a;
}

FineArgs make_fine_args(mmp_ctx* c, const Prob& p) { return fine_args_of(p, c->limit_ns); }

DriverArgs make_driver_args(const Prob& p, int sweep) {
  DriverArgs a;
  const mmp_problem_desc& d = p.d;
  a.nc3 = -d.c3; a.c1 = d.c1; a.kappa = d.kappa; a.c0 = d.c0;
  a.B = d.B; a.BE = d.BE; a.B0 = d.B0;
  a.family = d.family; a.K = d.K; a.g = d.g;
  a.N = d.N; a.I = p.I; a.variant = d.variant; a.precision = d.precision;
  a.coarse_model = d.coarse_model;
  a.dT = p.dT; a.hc = p.hc; a.nc = p.nc; a.P = d.P;
  a.thr = d.threshold; a.thr2 = d.threshold2; a.thr3 = d.threshold3;
  a.tol = d.tol; a.max_sweeps = p.max_sweeps;
  a.stats = p.stats; a.stats_u0 = p.stats_u0; a.rho = p.rho; a.cache = p.cache; a.aff = p.aff;
  a.ctl = p.ctl; a.status = p.status; a.sweep = sweep;
  return a;
}

// Batch region of the workspace (several problems of one precision and
// noise form): per-problem kernel and driver records, the sweep's task
// list, and the epoch flags and publication slots of every seat.
struct BatchLayout {
  bool on = false;
  int grid = 0;
  size_t smem = 0, seats_cap = 0;
  int tasks_cap = 0;
};

int batch_plan(const std::vector<Prob>& probs, const Device& dev, BatchLayout& B) {
  B = BatchLayout();
  const int n = (int)probs.size();
  if (n < 2) return MMP_OK;
  const char* e = std::getenv("MMP_BATCH");
  if (e != nullptr && std::strcmp(e, "0") == 0) return MMP_OK;
  for (const Prob& p : probs)
    if (p.d.precision != probs[0].d.precision || p.mult != probs[0].mult || p.d.family != MMP_FAMILY_POLY)
      return MMP_OK;
  int nq_max = 1;
  for (const Prob& p : probs) {
    nq_max = std::max(nq_max, p.nq);
    B.tasks_cap += p.d.N;
    B.seats_cap += (size_t)p.d.N * p.G;
  }
  const void* fn = fine_batch_kernel(probs[0].d.precision, probs[0].mult);
  int occ = 0;
  B.smem = fine_smem_bytes(probs[0].d.precision, kLayoutSmem, nq_max);
  size_t limit = 0;
  const int rc = allow_dynamic_smem(fn, dev.dev, &limit);
  if (rc) return rc;
  if (B.smem > limit) return MMP_ERR_UNSUPPORTED;
  MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB, B.smem));
  if (occ < 1) return MMP_ERR_UNSUPPORTED;
  B.grid = occ * dev.sms;
  for (const Prob& p : probs)
    if (p.G > B.grid) return MMP_ERR_UNSUPPORTED;
  B.on = true;
  return MMP_OK;
}

size_t batch_layout(const std::vector<Prob>& probs, const BatchLayout& B, char* base, size_t start, mmp_ctx* c) {
  if (!B.on) return start;
  Carver cv{base, start};
  const int n = (int)probs.size();
  auto ptr = [&](size_t b) -> char* {
    const size_t at = cv.take(b);
    return base ? base + at : nullptr;
  };
  char* probs_p = ptr(sizeof(FineArgs) * n);
  char* bufs_p = ptr(sizeof(void*) * 2 * n);
  char* tasks_p = ptr(sizeof(BatchTask) * B.tasks_cap);
  char* header_p = ptr(sizeof(int) * 4);
  char* seat_p = ptr(sizeof(unsigned) * 4);
  char* flags_p = ptr(sizeof(unsigned) * B.seats_cap);
  char* tags_p = ptr(sizeof(unsigned long long) * kSlots * B.seats_cap);
  char* partials_p = ptr(sizeof(double) * kSeatDoubles * B.seats_cap);
  char* dargs_p = ptr(sizeof(DriverArgs) * n);
  char* sweep_p = ptr(sizeof(int) * n);
  char* summary_p = ptr(sizeof(double) * 5 * n);
  char* ctlp_p = ptr(sizeof(double*) * n);
  char* order_p = ptr(sizeof(int) * n);
  char* N_p = ptr(sizeof(int) * n);
  char* G_p = ptr(sizeof(int) * n);
  char* remaining_p = ptr(sizeof(int) * 4);
  if (c != nullptr) {
    c->b_probs = (FineArgs*)probs_p;
    c->b_bufs = (void**)bufs_p;
    c->b_tasks = (BatchTask*)tasks_p;
    c->b_header = (int*)header_p;
    c->b_seat = (unsigned*)seat_p;
    c->b_flags = (unsigned*)flags_p;
    c->b_tags = (unsigned long long*)tags_p;
    c->b_partials = (double*)partials_p;
    c->b_dargs = (DriverArgs*)dargs_p;
    c->b_sweep = (int*)sweep_p;
    c->b_summary = (double*)summary_p;
    c->b_ctlp = (const double**)ctlp_p;
    c->b_order = (int*)order_p;
    c->b_N = (int*)N_p;
    c->b_G = (int*)G_p;
    c->b_remaining = (int*)remaining_p;
    c->b_seats_cap = B.seats_cap;
  }
  return cv.off;
}

// One launch of the fused fine kernel over slices [slice_begin, slice_begin + n_tasks).
int run_fine(mmp_ctx* c, Prob& p, int slice_begin, int n_tasks, int nf, const void* src0, const void* src,
             void* dst, int dst_fixed, const double* aff, int aff_fixed, double* stats, int stats_fixed,
             void* rec_uni = nullptr, void* rec_ckpt = nullptr, int ckpt_every = 1, long long step_offset = 0) {
  if (n_tasks < 1) return MMP_OK;
  const mmp_problem_desc& d = p.d;
  FineArgs a = make_fine_args(c, p);
  a.nf = nf;
  a.slice_begin = slice_begin; a.n_tasks = n_tasks;
  a.src0 = src0; a.src = src; a.dst = dst; a.dst_fixed = dst_fixed;
  a.aff = aff; a.aff_fixed = aff_fixed;
  a.stats = stats; a.stats_fixed = stats_fixed;
  a.rec_uni = rec_uni;
  a.rec_ckpt = rec_ckpt;
  a.ckpt_every = ckpt_every;
  a.step_offset = step_offset;
  const int slots = std::min(n_tasks, p.slots_max);
  a.tight_polls = slots * p.G <= c->dev.sms ? kTightPolls : 0;
  MMP_CUDA(cudaMemsetAsync(p.tags, 0, sync_bytes(p), c->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    for (cudaEvent_t* e : {&e0, &e1}) {
      if (!c->ev_pool.empty()) {
        *e = c->ev_pool.back();
        c->ev_pool.pop_back();
      } else {
        MMP_CUDA(cudaEventCreate(e));
      }
    }
    MMP_CUDA(cudaEventRecord(e0, c->stream));
  }
  MMP_CUDA(launch_fine(d.precision, p.layout, p.nq, p.mult, slots * p.G, a, c->stream, d.family));
  if (c->timing) {
    MMP_CUDA(cudaEventRecord(e1, c->stream));
    c->pending.emplace_back(e0, e1);
  }
  c->fine_launches += 1;
  c->fine_steps += (double)n_tasks * (double)d.P * (double)nf;
  return MMP_OK;
}

// Folds finished event pairs into the fine-kernel time (after a stream sync).
int collect_timing(mmp_ctx* c) {
  for (auto& pr : c->pending) {
    float ms = 0.0f;
    MMP_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second));
    c->fine_ms += ms;
    c->ev_pool.push_back(pr.first);
    c->ev_pool.push_back(pr.second);
  }
  c->pending.clear();
  return MMP_OK;
}

int run_driver(mmp_ctx* c, Prob& p, int sweep) {
  MMP_CUDA(launch_driver(make_driver_args(p, sweep), c->stream));
  c->other_launches += 1;
  return MMP_OK;
}

// Device records of a batched context (after layout and before any sweep).
int batch_setup(mmp_ctx* c) {
  const int n = (int)c->probs.size();
  std::vector<FineArgs> fa(n);
  std::vector<void*> bufs(2 * n);
  std::vector<DriverArgs> da(n);
  std::vector<const double*> ctlp(n);
  std::vector<int> order(n), Ns(n), Gs(n);
  for (int i = 0; i < n; ++i) {
    fa[i] = make_fine_args(c, c->probs[i]);
    bufs[2 * i] = c->probs[i].B[0];
    bufs[2 * i + 1] = c->probs[i].B[1];
    da[i] = make_driver_args(c->probs[i], 0);
    ctlp[i] = c->probs[i].ctl;
    order[i] = i;
    Ns[i] = c->probs[i].d.N;
    Gs[i] = c->probs[i].G;
  }
  // tasks largest first: problems by P n_f, descending, ties by index
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const Prob& px = c->probs[x];
    const Prob& py = c->probs[y];
    return (double)px.d.P * px.nf > (double)py.d.P * py.nf;
  });
  MMP_CUDA(cudaMemcpyAsync(c->b_probs, fa.data(), sizeof(FineArgs) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_bufs, bufs.data(), sizeof(void*) * 2 * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_dargs, da.data(), sizeof(DriverArgs) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_ctlp, ctlp.data(), sizeof(double*) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_N, Ns.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaMemcpyAsync(c->b_G, Gs.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
  MMP_CUDA(cudaStreamSynchronize(c->stream));
  return MMP_OK;
}

// Enqueues one batched sweep, all on the device: clear the exchange words
// and flags of every seat, build the task list from the problems' control
// blocks, one cooperative launch over every unconverged problem's slices
// k-1..N-1 (largest tasks first), then every driver in one launch.  No host
// work depends on the sweep, so sweeps can be enqueued back to back and
// captured in a graph.
int batch_enqueue_sweep(mmp_ctx* c, cudaStream_t stream) {
  const int n = (int)c->probs.size();
  MMP_CUDA(cudaMemsetAsync(c->b_flags, 0, sizeof(unsigned) * c->b_seats_cap, stream));
  MMP_CUDA(cudaMemsetAsync(c->b_tags, 0, sizeof(unsigned long long) * kSlots * c->b_seats_cap, stream));
  BatchPlanArgs pa;
  pa.ctl = c->b_ctlp;
  pa.order = c->b_order;
  pa.N = c->b_N;
  pa.G = c->b_G;
  pa.n = n;
  pa.tasks = c->b_tasks;
  pa.header = c->b_header;
  pa.sweep = c->b_sweep;
  pa.seat_counter = c->b_seat;
  pa.remaining = c->b_remaining;
  MMP_CUDA(launch_batch_plan(pa, stream));
  BatchArgs b;
  b.probs = c->b_probs;
  b.bufs = c->b_bufs;
  b.tasks = c->b_tasks;
  b.header = c->b_header;
  b.seat_counter = c->b_seat;
  b.flags = c->b_flags;
  b.tags = c->b_tags;
  b.partials = c->b_partials;
  MMP_CUDA(launch_fine_batch(c->probs[0].d.precision, c->probs[0].mult, c->batch_grid, c->batch_smem, b, stream));
  MMP_CUDA(launch_driver_batch(c->b_dargs, c->b_sweep, c->b_summary, n, stream));
  return MMP_OK;
}

// Batched sweeps per graph launch.  A graph runs this many sweeps whatever
// the problems do; sweeps after the last problem finished (or after the
// requested count) build no task and cost a few microseconds.
constexpr int kGraphSweeps = 4;

// Enqueues kGraphSweeps batched sweeps: one launch of a graph captured on
// first use (MMP_BATCH_GRAPH=0, or a capture the runtime refuses, enqueues
// the same work directly).
int batch_enqueue_sweeps(mmp_ctx* c) {
  const char* e = std::getenv("MMP_BATCH_GRAPH");
  const bool want = !(e != nullptr && std::strcmp(e, "0") == 0);
  if (want && c->b_graph == nullptr && !c->b_graph_failed) {
    cudaGraph_t g = nullptr;
    int rc = MMP_OK;
    cudaError_t ce = cudaSuccess;
    if (c->cap_stream == nullptr) ce = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      for (int s = 0; s < kGraphSweeps && rc == MMP_OK; ++s) rc = batch_enqueue_sweep(c, c->cap_stream);
      ce = cudaStreamEndCapture(c->cap_stream, &g);
    }
    if (ce == cudaSuccess && rc == MMP_OK) ce = cudaGraphInstantiate(&c->b_graph, g, 0);
    if (g != nullptr) cudaGraphDestroy(g);
    if (ce != cudaSuccess || rc != MMP_OK) {
      // a refused capture is not an error of the run: enqueue directly
      if (ce != cudaSuccess) cuda_fail(ce, "batched sweep capture (falling back to direct enqueue)", __LINE__);
      cudaGetLastError();
      if (c->b_graph != nullptr) cudaGraphExecDestroy(c->b_graph);
      c->b_graph = nullptr;
      c->b_graph_failed = true;
    }
  }
  bool launched = false;
  if (want && c->b_graph != nullptr) {
    const cudaError_t ce = cudaGraphLaunch(c->b_graph, c->stream);
    if (ce == cudaSuccess) {
      launched = true;
    } else {
      cuda_fail(ce, "batched sweep graph launch (falling back to direct enqueue)", __LINE__);
      cudaGetLastError();
      cudaGraphExecDestroy(c->b_graph);
      c->b_graph = nullptr;
      c->b_graph_failed = true;
    }
  }
  if (!launched) {
    for (int s = 0; s < kGraphSweeps; ++s) {
      int rc = batch_enqueue_sweep(c, c->stream);
      if (rc) return rc;
    }
  }
  c->other_launches += 2 * kGraphSweeps;
  return MMP_OK;
}

int status_to_error(unsigned s) {
  if (s & kStatusTimeout) return MMP_ERR_TIMEOUT;
  if (s & kStatusNumeric) return MMP_ERR_NUMERIC;
  return MMP_OK;
}

// Layout of the adjoint workspace: checkpoint rows, recorded uniforms, the
// segment buffers, cotangents, gradient and the reverse kernel's group
// scratch; also the reverse kernel's launch shape (all particles in one
// co-resident group of at most one CTA per SM, the fewest quads per thread
// that fit, the particles spread over as many SMs as there are CTAs' worth
// of threads).
struct AdjLayout {
  size_t bytes = 0;
  int n_seg = 0, G = 1, nq = 1;
  int fG = 1, fnq = 1;  // the recording forward: one slice over the whole GPU
  double* fpartials = nullptr;
  unsigned long long* ftags = nullptr;  // followed by flags
  void *ckpt = nullptr, *uni = nullptr, *segx = nullptr, *segz = nullptr;
  double *gm = nullptr, *gv = nullptr, *grad = nullptr, *partials = nullptr;
  unsigned* flags = nullptr;
  unsigned long long* tags = nullptr;  // followed by flags
};

int adjoint_layout(mmp_ctx* c, Prob& p, int ckpt_every, char* base, AdjLayout& L) {
  if (p.d.family != MMP_FAMILY_POLY) return MMP_ERR_UNSUPPORTED;  // the adjoint is the polynomial drift's
  const long long J = (long long)p.d.N * p.nf;
  L.n_seg = (int)((J + ckpt_every - 1) / ckpt_every);
  const void* fn = adjoint_kernel(p.d.precision, p.mult);
  size_t limit = 0;
  const int arc = allow_dynamic_smem(fn, c->dev.dev, &limit);
  if (arc) return arc;
  const int max_nq = p.esz == 4 ? 32 : 16;
  L.G = 0;
  for (int nq = 1; nq <= max_nq; ++nq) {
    int occ = 0;
    const size_t smem = adjoint_smem_bytes(p.d.precision, nq);
    if (smem > limit) break;
    MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kAdjTPB, smem));
    const long long G = ((long long)p.Q + (long long)nq * kAdjTPB - 1) / ((long long)nq * kAdjTPB);
    if (occ >= 1 && G <= (long long)c->dev.sms) {  // about one CTA per SM (see the forward below)
      L.nq = nq;
      L.G = (int)std::min<long long>(c->dev.sms, std::max<long long>(G, ((long long)p.Q + kAdjTPB - 1) / kAdjTPB));
      break;
    }
  }
  if (L.G == 0) return MMP_ERR_UNSUPPORTED;
  // The recording forward runs the slices one after another, so it takes
  // its own shape rather than the Parareal plan's: about one CTA per SM
  // (the fewest quads per thread with G <= SMs).  More CTAs leave each with
  // too little work per step for the cross-CTA exchange they add.
  L.fG = 0;
  for (int nq = 1; nq <= max_nq; ++nq) {
    const void* ff = fine_kernel(p.d.precision, kLayoutSmem, nq, p.mult, p.d.family);
    size_t flimit = 0;
    const int frc = allow_dynamic_smem(ff, c->dev.dev, &flimit);
    if (frc) return frc;
    const size_t smem = fine_smem_bytes(p.d.precision, kLayoutSmem, nq, p.d.family);
    if (smem > flimit) break;
    int occ = 0;
    MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ff, kTPB, smem));
    const long long G = ((long long)p.Q + (long long)nq * kTPB - 1) / ((long long)nq * kTPB);
    if (occ >= 1 && G <= (long long)c->dev.sms) {
      L.fnq = nq;
      L.fG = (int)G;
      break;
    }
  }
  if (L.fG == 0) return MMP_ERR_UNSUPPORTED;
  Carver cv{base, 0};
  const size_t row = (size_t)p.pitch * p.esz;
  auto ptr = [&](size_t b) -> char* {
    const size_t at = cv.take(b);
    return base ? base + at : nullptr;
  };
  L.ckpt = ptr(row * L.n_seg);
  L.uni = ptr(p.esz * 3 * (size_t)J);
  // two buffers of c + 1 rows of replayed states (one segment is replayed
  // while the next is reversed)
  L.segx = ptr(row * 2 * (size_t)(ckpt_every + 1));
  // two buffers of c draw rows: used by the general diffusion form only (additive noise
  // regenerates its draws), carved for both so that the size does not change with the form
  // (mmp_set_params)
  L.segz = ptr(row * 2 * (size_t)ckpt_every);
  L.gm = (double*)ptr(sizeof(double) * p.d.N);
  L.gv = (double*)ptr(sizeof(double) * p.d.N);
  L.grad = (double*)ptr(sizeof(double) * 8);
  L.partials = (double*)ptr(sizeof(double) * kSeatDoubles * (size_t)L.G);
  L.tags = (unsigned long long*)ptr((sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * (size_t)L.G);
  L.flags = base ? (unsigned*)(L.tags + (size_t)kSlots * L.G) : nullptr;
  L.fpartials = (double*)ptr(sizeof(double) * kSeatDoubles * (size_t)L.fG);
  L.ftags = (unsigned long long*)ptr((sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * (size_t)L.fG);
  L.bytes = (cv.off + kAlign - 1) / kAlign * kAlign;
  return MMP_OK;
}

int check_prob(mmp_ctx* c, int prob) {
  if (c == nullptr || prob < 0 || prob >= (int)c->probs.size()) return MMP_ERR_INVALID_ARG;
  return MMP_OK;
}

}  // namespace

extern "C" {

const char* mmp_strerror(int code) {
  switch (code) {
    case MMP_OK: return "ok";
    case MMP_ERR_INVALID_ARG: return "invalid argument";
    case MMP_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case MMP_ERR_UNSUPPORTED: return "unsupported configuration";
    case MMP_ERR_CUDA: return "CUDA error";
    case MMP_ERR_NUMERIC: return "non-finite value or negative variance on the device";
    case MMP_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case MMP_ERR_STATE: return "call out of order";
    default: return "unknown error";
  }
}

int mmp_version(void) { return MMP_VERSION; }

int mmp_last_cuda_error(void) { return g_last_cuda_error.load(std::memory_order_relaxed); }

int mmp_workspace_size(const mmp_problem_desc* descs, int n_problems, size_t* bytes) {
  if (bytes == nullptr) return MMP_ERR_INVALID_ARG;
  std::vector<Prob> probs;
  Device dev;
  const int rc = prepare(descs, n_problems, probs, dev);
  if (rc) return rc;
  size_t off = 0;
  for (Prob& p : probs) off = layout(p, nullptr, off);
  BatchLayout B;
  const int brc = batch_plan(probs, dev, B);
  if (brc) return brc;
  off = batch_layout(probs, B, nullptr, off, nullptr);
  *bytes = (off + kAlign - 1) / kAlign * kAlign;
  return MMP_OK;
}

int mmp_create(mmp_ctx** out, const mmp_problem_desc* descs, int n_problems, void* workspace,
               size_t workspace_bytes, void* stream) {
  Range nvtx_range("mmp_create");
  if (out == nullptr) return MMP_ERR_INVALID_ARG;
  *out = nullptr;
  if (workspace == nullptr || ((uintptr_t)workspace % kAlign) != 0) return MMP_ERR_WORKSPACE;
  mmp_ctx* c = new (std::nothrow) mmp_ctx();
  if (c == nullptr) return MMP_ERR_INVALID_ARG;
  int rc = prepare(descs, n_problems, c->probs, c->dev);
  if (rc) {
    delete c;
    return rc;
  }
  size_t off = 0;
  for (Prob& p : c->probs) off = layout(p, (char*)workspace, off);
  BatchLayout B;
  rc = batch_plan(c->probs, c->dev, B);
  if (rc) {
    delete c;
    return rc;
  }
  off = batch_layout(c->probs, B, (char*)workspace, off, c);
  c->ws = (char*)workspace;
  c->ws_used = off;
  c->batch = B.on;
  c->batch_grid = B.grid;
  c->batch_smem = B.smem;
  if (off > workspace_bytes) {
    delete c;
    return MMP_ERR_WORKSPACE;
  }
  c->stream = (cudaStream_t)stream;
  c->limit_ns = wait_limit_ns();
  c->host_ctl.assign(16, 0.0);
  for (Prob& p : c->probs) {
    cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(unsigned) * 4, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.ctl, 0, sizeof(double) * 16, c->stream);
    if (e == cudaSuccess)
      e = launch_init_u0(p.d.precision, p.u0, p.d.P, p.Q, p.d.m0, p.d.s0, p.key0, p.key1,
                         p.d.problem_tag, p.d.family == MMP_FAMILY_ROTATOR, c->stream);
    c->other_launches += 1;
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "launch", __LINE__);
    }
  }
  if (c->batch) {
    rc = batch_setup(c);
    if (rc) {
      delete c;
      return rc;
    }
  }
  *out = c;
  return MMP_OK;
}

int mmp_destroy(mmp_ctx* ctx) {
  delete ctx;
  return MMP_OK;
}

int mmp_set_initial(mmp_ctx* ctx, int prob, const void* u0, int from_host) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (u0 == nullptr) return MMP_ERR_INVALID_ARG;
  Prob& p = ctx->probs[prob];
  const size_t bytes = (size_t)p.d.P * p.esz;
  MMP_CUDA(cudaMemcpyAsync(p.u0, u0, bytes, from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           ctx->stream));
  if (from_host) MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  p.lifted = false;
  p.sweeps = 0;
  p.done = false;
  return MMP_OK;
}

int mmp_lift(mmp_ctx* ctx) {
  Range nvtx_range("mmp_lift");
  if (ctx == nullptr) return MMP_ERR_INVALID_ARG;
  for (Prob& p : ctx->probs) {
    int rc = run_fine(ctx, p, 0, 1, 0, p.u0, nullptr, nullptr, 0, nullptr, 0, p.stats_u0, 1);
    if (rc) return rc;
    rc = run_driver(ctx, p, 0);
    if (rc) return rc;
    p.lifted = true;
    p.sweeps = 0;
    p.done = false;
    p.converged = false;
    p.last_change = 0.0;
    p.fine_pending = 0;
    std::fill(p.out_buf.begin(), p.out_buf.end(), -1);
  }
  if (ctx->batch)
    MMP_CUDA(cudaMemsetAsync(ctx->b_summary, 0, sizeof(double) * 5 * ctx->probs.size(), ctx->stream));
  return MMP_OK;
}

int mmp_iterate(mmp_ctx* ctx, int n_iter, int* all_converged) {
  Range nvtx_range("mmp_iterate");
  if (ctx == nullptr || n_iter < 0) return MMP_ERR_INVALID_ARG;
  for (Prob& p : ctx->probs)
    if (!p.lifted || p.fine_pending != 0) return MMP_ERR_STATE;
  if (ctx->batch) {
    // sweeps are built and run on the device, kGraphSweeps per graph launch;
    // the host reads the problems' summaries once per launch
    const int n = (int)ctx->probs.size();
    bool any = false;
    for (Prob& p : ctx->probs) any = any || !p.done;
    if (any && n_iter > 0) {
      MMP_CUDA(cudaMemcpyAsync(ctx->b_remaining, &n_iter, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
      ctx->h_summary.assign((size_t)5 * n, 0.0);
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      for (int done_sweeps = 0; done_sweeps < n_iter;) {
        if (ctx->timing) {
          for (cudaEvent_t* ev : {&e0, &e1}) {
            if (!ctx->ev_pool.empty()) {
              *ev = ctx->ev_pool.back();
              ctx->ev_pool.pop_back();
            } else {
              MMP_CUDA(cudaEventCreate(ev));
            }
          }
          MMP_CUDA(cudaEventRecord(e0, ctx->stream));
        }
        int rc = batch_enqueue_sweeps(ctx);
        if (rc) return rc;
        if (ctx->timing) {
          MMP_CUDA(cudaEventRecord(e1, ctx->stream));
          ctx->pending.emplace_back(e0, e1);
        }
        done_sweeps += kGraphSweeps;
        MMP_CUDA(cudaMemcpyAsync(ctx->h_summary.data(), ctx->b_summary, sizeof(double) * 5 * n,
                                 cudaMemcpyDeviceToHost, ctx->stream));
        MMP_CUDA(cudaStreamSynchronize(ctx->stream));
        rc = collect_timing(ctx);
        if (rc) return rc;
        int err = MMP_OK;
        bool all = true;
        int max_new = 0;
        for (int i = 0; i < n; ++i) {
          Prob& p = ctx->probs[i];
          const double* sm = &ctx->h_summary[(size_t)5 * i];
          const int K = (int)sm[2];
          if (K <= p.sweeps) {  // not swept since the last look
            all = all && p.done;
            continue;
          }
          for (int k = p.sweeps + 1; k <= K; ++k)
            ctx->fine_steps += (double)(p.d.N - k + 1) * (double)p.d.P * (double)p.nf;
          max_new = std::max(max_new, K - p.sweeps);
          p.sweeps = K;
          for (int sl = 0; sl < p.d.N; ++sl) p.out_buf[sl] = std::min(K, sl + 1) & 1;
          p.last_change = sm[0];
          p.converged = sm[1] != 0.0 || K == p.d.N;
          p.done = sm[3] != 0.0;
          all = all && p.done;
          const int e = status_to_error((unsigned)sm[4]);
          if (e && !err) err = e;
        }
        ctx->fine_launches += max_new;
        if (err) return err;
        if (all) break;
      }
    }
    if (all_converged) {
      bool all = true;
      for (Prob& p : ctx->probs) all = all && p.done;
      *all_converged = all ? 1 : 0;
    }
    return MMP_OK;
  }
  for (int it = 0; it < n_iter; ++it) {
    bool any = false;
    for (Prob& p : ctx->probs) {
      if (p.done) continue;
      const int k = p.sweeps + 1;
      const int first = k - 1;  // slices before k - 1 are exact (Property 3.3)
      const char* src = k == 1 ? nullptr : p.B[(k - 1) & 1];
      int rc = run_fine(ctx, p, first, p.d.N - first, p.nf, p.u0, src, p.B[k & 1], 0, p.aff, 0, p.stats, 0);
      if (rc) return rc;
      rc = run_driver(ctx, p, k);
      if (rc) return rc;
      any = true;
    }
    if (!any) break;
    // one host round trip per sweep: the driver leaves the status word in
    // ctl[15], and a copy to pageable host memory returns only once it (and
    // so all the stream's earlier work) has completed
    std::vector<double> ctls;
    ctls.reserve(16 * ctx->probs.size());
    for (Prob& p : ctx->probs) {
      if (p.done) continue;
      ctls.resize(ctls.size() + 16);
      MMP_CUDA(cudaMemcpyAsync(ctls.data() + ctls.size() - 16, p.ctl, sizeof(double) * 16, cudaMemcpyDeviceToHost,
                               ctx->stream));
    }
    MMP_CUDA(cudaStreamSynchronize(ctx->stream));
    {
      const int trc = collect_timing(ctx);
      if (trc) return trc;
    }
    size_t slot = 0;
    for (Prob& p : ctx->probs) {
      if (p.done) continue;
      const double* ctl = ctls.data() + 16 * slot++;
      const unsigned st0 = (unsigned)ctl[15];
      const int k = p.sweeps + 1;
      for (int n = k - 1; n < p.d.N; ++n) p.out_buf[n] = k & 1;
      p.sweeps = k;
      p.last_change = ctl[0];
      p.converged = ctl[1] != 0.0 || k == p.d.N;
      p.done = ctl[3] != 0.0;
      const int err = status_to_error(st0);
      if (err) return err;
    }
  }
  if (all_converged) {
    bool all = true;
    for (Prob& p : ctx->probs) all = all && p.done;
    *all_converged = all ? 1 : 0;
  }
  return MMP_OK;
}

// ---------------------------------------------------------------------------
// A sweep in two phases, for running one problem's slices on several GPUs
// (each rank propagates a contiguous block of slices; the restriction
// records are gathered on every rank, the driver runs redundantly, and the
// fine output at the end of a block is handed to the next rank).
// ---------------------------------------------------------------------------
int mmp_sweep_fine(mmp_ctx* ctx, int prob, int n_lo, int n_hi) {
  Range nvtx_range("mmp_sweep_fine");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (ctx->batch) return MMP_ERR_UNSUPPORTED;
  Prob& p = ctx->probs[prob];
  if (n_lo < 0 || n_hi > p.d.N || n_lo >= n_hi) return MMP_ERR_INVALID_ARG;
  if (!p.lifted || p.fine_pending != 0 || p.done) return MMP_ERR_STATE;
  const int k = p.sweeps + 1;
  const int first = std::max(k - 1, n_lo);  // slices before k - 1 are exact (Property 3.3)
  if (first < n_hi) {
    const char* src = k == 1 ? nullptr : p.B[(k - 1) & 1];
    rc = run_fine(ctx, p, first, n_hi - first, p.nf, p.u0, src, p.B[k & 1], 0, p.aff, 0, p.stats, 0);
    if (rc) return rc;
  }
  p.fine_pending = k;
  return MMP_OK;
}

int mmp_sweep_coarse(mmp_ctx* ctx, int prob, int* done) {
  Range nvtx_range("mmp_sweep_coarse");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (p.fine_pending != p.sweeps + 1 || p.fine_pending == 0) return MMP_ERR_STATE;
  const int k = p.fine_pending;
  rc = run_driver(ctx, p, k);
  if (rc) return rc;
  double ctl[16];
  MMP_CUDA(cudaMemcpyAsync(ctl, p.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  rc = collect_timing(ctx);
  if (rc) return rc;
  for (int n = k - 1; n < p.d.N; ++n) p.out_buf[n] = k & 1;
  p.sweeps = k;
  p.fine_pending = 0;
  p.last_change = ctl[0];
  p.converged = ctl[1] != 0.0 || k == p.d.N;
  p.done = ctl[3] != 0.0;
  if (done != nullptr) *done = p.done ? 1 : 0;
  return status_to_error((unsigned)ctl[15]);
}

int mmp_get_records(mmp_ctx* ctx, int prob, int n_lo, int n_hi, double* out) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (out == nullptr || n_lo < 0 || n_hi > p.d.N || n_lo > n_hi) return MMP_ERR_INVALID_ARG;
  if (!p.lifted) return MMP_ERR_STATE;
  if (n_hi == n_lo) return MMP_OK;
  MMP_CUDA(cudaMemcpyAsync(out, p.stats + (size_t)n_lo * kStat, sizeof(double) * kStat * (n_hi - n_lo),
                           cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

int mmp_set_records(mmp_ctx* ctx, int prob, int n_lo, int n_hi, const double* in) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (in == nullptr || n_lo < 0 || n_hi > p.d.N || n_lo > n_hi) return MMP_ERR_INVALID_ARG;
  if (!p.lifted) return MMP_ERR_STATE;
  if (n_hi == n_lo) return MMP_OK;
  MMP_CUDA(cudaMemcpyAsync(p.stats + (size_t)n_lo * kStat, in, sizeof(double) * kStat * (n_hi - n_lo),
                           cudaMemcpyHostToDevice, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

// Row n of the buffer the latest fine phase wrote (sweep fine_pending, or the
// last complete sweep), or nullptr before the first fine phase.
static char* output_row(Prob& p, int n) {
  const int k = p.fine_pending != 0 ? p.fine_pending : p.sweeps;
  if (k < 1) return nullptr;
  return p.B[k & 1] + (size_t)n * p.pitch * p.esz;
}

int mmp_get_output(mmp_ctx* ctx, int prob, int n, void* dst, int to_host) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (dst == nullptr || n < 0 || n >= p.d.N) return MMP_ERR_INVALID_ARG;
  if (ctx->batch) return MMP_ERR_UNSUPPORTED;
  char* row = output_row(p, n);
  if (!p.lifted || row == nullptr) return MMP_ERR_STATE;
  MMP_CUDA(cudaMemcpyAsync(dst, row, (size_t)p.d.P * p.esz, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                           ctx->stream));
  if (to_host) MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

int mmp_set_output(mmp_ctx* ctx, int prob, int n, const void* src, int from_host) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (src == nullptr || n < 0 || n >= p.d.N) return MMP_ERR_INVALID_ARG;
  if (ctx->batch) return MMP_ERR_UNSUPPORTED;
  char* row = output_row(p, n);
  if (!p.lifted || row == nullptr) return MMP_ERR_STATE;
  MMP_CUDA(cudaMemcpyAsync(row, src, (size_t)p.d.P * p.esz, from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                           ctx->stream));
  if (from_host) MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

int mmp_run(mmp_ctx* ctx, int* sweeps_out) {
  Range nvtx_range("mmp_run");
  int rc = mmp_lift(ctx);
  if (rc) return rc;
  int all = 0;
  int most = 0;
  for (Prob& p : ctx->probs) most = std::max(most, p.d.N);
  while (!all) {
    rc = mmp_iterate(ctx, most, &all);
    if (rc) return rc;
  }
  if (sweeps_out) {
    int m = 0;
    for (Prob& p : ctx->probs) m = std::max(m, p.sweeps);
    *sweeps_out = m;
  }
  return MMP_OK;
}

int mmp_status(mmp_ctx* ctx, int prob, int* sweeps, int* converged, double* last_change, int* dev_err) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  unsigned st[4] = {0, 0, 0, 0};
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  MMP_CUDA(cudaMemcpy(st, p.status, sizeof(st), cudaMemcpyDeviceToHost));
  if (sweeps) *sweeps = p.sweeps;
  if (converged) *converged = p.converged ? 1 : 0;
  if (last_change) *last_change = p.last_change;
  if (dev_err) *dev_err = status_to_error(st[0]);
  return MMP_OK;
}

int mmp_get_moments(mmp_ctx* ctx, int prob, double* out) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (out == nullptr) return MMP_ERR_INVALID_ARG;
  Prob& p = ctx->probs[prob];
  if (!p.lifted) return MMP_ERR_STATE;
  MMP_CUDA(cudaMemcpyAsync(out, p.rho, sizeof(double) * kMom * (p.d.N + 1), cudaMemcpyDeviceToHost,
                           ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

int mmp_get_particles(mmp_ctx* ctx, int prob, int n, void* dst, int to_host) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (dst == nullptr || n < 0 || n > p.d.N) return MMP_ERR_INVALID_ARG;
  const size_t bytes = (size_t)p.d.P * p.esz;
  const cudaMemcpyKind kind = to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (n == 0) {
    MMP_CUDA(cudaMemcpyAsync(dst, p.u0, bytes, kind, ctx->stream));
  } else {
    if (!p.lifted) return MMP_ERR_STATE;
    const int buf = p.sweeps == 0 ? -1 : p.out_buf[n - 1];
    const char* src = buf < 0 ? nullptr : p.B[buf];
    rc = run_fine(ctx, p, n, 1, 0, p.u0, src, p.S[0], 1, p.aff, 0, p.tmp_stats, 1);
    if (rc) return rc;
    MMP_CUDA(cudaMemcpyAsync(dst, p.S[0], bytes, kind, ctx->stream));
  }
  if (to_host) MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

int mmp_fine_serial(mmp_ctx* ctx, int prob, int n_end, double* stats_out, void* parts_dev) {
  Range nvtx_range("mmp_fine_serial");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  const int N = (n_end <= 0 || n_end > p.d.N) ? p.d.N : n_end;
  rc = run_fine(ctx, p, 0, 1, 0, p.u0, nullptr, nullptr, 0, nullptr, 0, p.ser_stats, 1);
  if (rc) return rc;
  for (int n = 0; n < N; ++n) {
    const void* in = n == 0 ? (const void*)p.u0 : (const void*)p.S[(n - 1) & 1];
    rc = run_fine(ctx, p, n, 1, p.nf, in, nullptr, p.S[n & 1], 1, nullptr, 0,
                  p.ser_stats + (size_t)(n + 1) * kStat, 1);
    if (rc) return rc;
  }
  if (parts_dev)
    MMP_CUDA(cudaMemcpyAsync(parts_dev, p.S[(N - 1) & 1], (size_t)p.d.P * p.esz, cudaMemcpyDeviceToDevice,
                             ctx->stream));
  if (stats_out)
    MMP_CUDA(cudaMemcpyAsync(stats_out, p.ser_stats, sizeof(double) * kStat * (N + 1), cudaMemcpyDeviceToHost,
                             ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  unsigned st[4];
  MMP_CUDA(cudaMemcpy(st, p.status, sizeof(st), cudaMemcpyDeviceToHost));
  return status_to_error(st[0]);
}

int mmp_set_params(mmp_ctx* ctx, int prob, const double* theta, int n_theta) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (theta == nullptr || (n_theta != 5 && n_theta != 7)) return MMP_ERR_INVALID_ARG;
  for (int k = 0; k < n_theta; ++k)
    if (!std::isfinite(theta[k])) return MMP_ERR_INVALID_ARG;
  Prob& p = ctx->probs[prob];
  if (p.d.family != MMP_FAMILY_POLY) return MMP_ERR_UNSUPPORTED;  // the coefficients are the polynomial drift's
  const double B = n_theta == 7 ? theta[5] : p.d.B;
  const double BE = n_theta == 7 ? theta[6] : p.d.BE;
  const bool mult = B != 0.0 || BE != 0.0;
  if (mult != p.mult) {
    // the fine kernel changes form: a batch shares one form, and a single
    // problem keeps its launch shape only if the other form fits it too
    if (ctx->batch) return MMP_ERR_UNSUPPORTED;
    const void* fn = fine_kernel(p.d.precision, p.layout, p.nq, mult, p.d.family);
    if (fn == nullptr) return MMP_ERR_UNSUPPORTED;
    const size_t smem = fine_smem_bytes(p.d.precision, p.layout, p.nq, p.d.family);
    if (p.layout == kLayoutSmem) {
      size_t limit = 0;
      rc = allow_dynamic_smem(fn, ctx->dev.dev, &limit);
      if (rc) return rc;
      if (smem > limit) return MMP_ERR_UNSUPPORTED;
    }
    int occ = 0;
    MMP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB, smem));
    if ((long long)occ * ctx->dev.sms < (long long)p.slots_max * p.G) return MMP_ERR_UNSUPPORTED;
  }
  p.d.c3 = theta[0];
  p.d.c1 = theta[1];
  p.d.kappa = theta[2];
  p.d.c0 = theta[3];
  p.d.B0 = theta[4];
  p.d.B = B;
  p.d.BE = BE;
  p.mult = mult;
  p.adj_ready = false;
  return MMP_OK;
}

int mmp_adjoint_workspace_size(mmp_ctx* ctx, int prob, int ckpt_every, size_t* bytes) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (bytes == nullptr || ckpt_every < 1) return MMP_ERR_INVALID_ARG;
  Prob& p = ctx->probs[prob];
  AdjLayout L;
  rc = adjoint_layout(ctx, p, ckpt_every, nullptr, L);
  if (rc) return rc;
  *bytes = L.bytes;
  return MMP_OK;
}

int mmp_adjoint_forward(mmp_ctx* ctx, int prob, int ckpt_every, void* ws, size_t ws_bytes, double* moments_out) {
  Range nvtx_range("mmp_adjoint_forward");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (ckpt_every < 1) return MMP_ERR_INVALID_ARG;
  if (ws == nullptr || ((uintptr_t)ws % kAlign) != 0) return MMP_ERR_WORKSPACE;
  Prob& p = ctx->probs[prob];
  AdjLayout L;
  rc = adjoint_layout(ctx, p, ckpt_every, (char*)ws, L);
  if (rc) return rc;
  if (L.bytes > ws_bytes) return MMP_ERR_WORKSPACE;
  const int N = p.d.N;
  // the serial fine run with recording, in the forward's own launch shape;
  // slice ends restricted into ser_stats
  Prob q = p;
  q.layout = kLayoutSmem;
  q.nq = L.fnq;
  q.G = L.fG;
  q.slots_max = 1;
  q.partials = L.fpartials;
  q.tags = L.ftags;
  q.flags = (unsigned*)(L.ftags + (size_t)kSlots * L.fG);
  rc = run_fine(ctx, q, 0, 1, 0, p.u0, nullptr, nullptr, 0, nullptr, 0, p.ser_stats, 1);
  if (rc) return rc;
  for (int n = 0; n < N; ++n) {
    const void* in = n == 0 ? (const void*)p.u0 : (const void*)p.S[(n - 1) & 1];
    rc = run_fine(ctx, q, n, 1, p.nf, in, nullptr, p.S[n & 1], 1, nullptr, 0,
                  p.ser_stats + (size_t)(n + 1) * kStat, 1, L.uni, L.ckpt, ckpt_every, (long long)n * p.nf);
    if (rc) return rc;
  }
  if (moments_out) {
    std::vector<double> st((size_t)kStat * (N + 1));
    MMP_CUDA(cudaMemcpyAsync(st.data(), p.ser_stats, sizeof(double) * st.size(), cudaMemcpyDeviceToHost,
                             ctx->stream));
    MMP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int n = 0; n <= N; ++n) {
      moments_out[2 * n] = st[(size_t)n * kStat + 10];
      moments_out[2 * n + 1] = st[(size_t)n * kStat + 11];
    }
  } else {
    MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  unsigned stw[4];
  MMP_CUDA(cudaMemcpy(stw, p.status, sizeof(stw), cudaMemcpyDeviceToHost));
  rc = status_to_error(stw[0]);
  if (rc) return rc;
  p.adj_ready = true;
  p.adj_ws = ws;
  p.adj_ckpt_every = ckpt_every;
  return MMP_OK;
}

int mmp_adjoint_backward(mmp_ctx* ctx, int prob, const double* gm, const double* gv, void* ws, size_t ws_bytes,
                         double* grad_out) {
  Range nvtx_range("mmp_adjoint_backward");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (gm == nullptr || gv == nullptr || grad_out == nullptr) return MMP_ERR_INVALID_ARG;
  if (ws == nullptr || ((uintptr_t)ws % kAlign) != 0) return MMP_ERR_WORKSPACE;
  Prob& p = ctx->probs[prob];
  if (!p.adj_ready || p.adj_ws != ws) return MMP_ERR_STATE;
  AdjLayout L;
  rc = adjoint_layout(ctx, p, p.adj_ckpt_every, (char*)ws, L);
  if (rc) return rc;
  if (L.bytes > ws_bytes) return MMP_ERR_WORKSPACE;
  const int N = p.d.N;
  MMP_CUDA(cudaMemcpyAsync(L.gm, gm, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
  MMP_CUDA(cudaMemcpyAsync(L.gv, gv, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
  MMP_CUDA(cudaMemsetAsync(L.tags, 0, (sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * L.G,
                           ctx->stream));
  AdjointArgs a;
  a.nc3 = -p.d.c3; a.c1 = p.d.c1; a.kappa = p.d.kappa; a.h = p.h; a.sqrt_h = p.sqrt_h;
  a.B = p.d.B; a.BE = p.d.BE;
  a.nf = p.nf; a.J = (long long)N * p.nf; a.c = p.adj_ckpt_every; a.n_seg = L.n_seg;
  a.P = p.d.P; a.Q = p.Q; a.pitch = p.pitch;
  a.key0 = p.key0; a.key1 = p.key1; a.ptag = p.d.problem_tag;
  a.G = L.G; a.nq = L.nq;
  a.ckpt = L.ckpt; a.uni = L.uni; a.segx = L.segx; a.segz = L.segz;
  a.mom = p.ser_stats; a.gm = L.gm; a.gv = L.gv; a.grad = L.grad;
  a.partials = L.partials; a.flags = L.flags; a.tags = L.tags; a.status = p.status;
  a.wait_limit_ns = ctx->limit_ns;
  a.sms = ctx->dev.sms;
  MMP_CUDA(launch_adjoint(p.d.precision, p.mult, a, ctx->stream));
  ctx->other_launches += 1;
  MMP_CUDA(cudaMemcpyAsync(grad_out, L.grad, sizeof(double) * kNGrad, cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  unsigned stw[4];
  MMP_CUDA(cudaMemcpy(stw, p.status, sizeof(stw), cudaMemcpyDeviceToHost));
  return status_to_error(stw[0]);
}

int mmp_adjoint(mmp_ctx* ctx, int prob, const double* m_tgt, const double* v_tgt, int ckpt_every, void* ws,
                size_t ws_bytes, double* grad_out, double* loss) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (m_tgt == nullptr || v_tgt == nullptr || grad_out == nullptr) return MMP_ERR_INVALID_ARG;
  const int N = ctx->probs[prob].d.N;
  std::vector<double> mom(2 * (size_t)(N + 1)), gm(N), gv(N);
  rc = mmp_adjoint_forward(ctx, prob, ckpt_every, ws, ws_bytes, mom.data());
  if (rc) return rc;
  double L = 0.0;
  for (int n = 1; n <= N; ++n) {
    const double dm = mom[2 * n] - m_tgt[n - 1], dv = mom[2 * n + 1] - v_tgt[n - 1];
    L += dm * dm + dv * dv;
    gm[n - 1] = 2.0 * dm;
    gv[n - 1] = 2.0 * dv;
  }
  if (loss) *loss = L;
  return mmp_adjoint_backward(ctx, prob, gm.data(), gv.data(), ws, ws_bytes, grad_out);
}

int mmp_set_timing(mmp_ctx* ctx, int on) {
  if (ctx == nullptr) return MMP_ERR_INVALID_ARG;
  ctx->timing = on != 0;
  return MMP_OK;
}

int mmp_timing(mmp_ctx* ctx, int reset, double* fine_ms, long long* fine_launches,
               double* fine_particle_steps, long long* other_launches) {
  if (ctx == nullptr) return MMP_ERR_INVALID_ARG;
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  const int rc = collect_timing(ctx);
  if (rc) return rc;
  if (fine_ms) *fine_ms = ctx->fine_ms;
  if (fine_launches) *fine_launches = ctx->fine_launches;
  if (fine_particle_steps) *fine_particle_steps = ctx->fine_steps;
  if (other_launches) *other_launches = ctx->other_launches;
  if (reset) {
    ctx->fine_ms = 0.0;
    ctx->fine_steps = 0.0;
    ctx->fine_launches = 0;
    ctx->other_launches = 0;
  }
  return MMP_OK;
}

int mmp_batch_info(mmp_ctx* ctx, int* batched, int* graph) {
  if (ctx == nullptr) return MMP_ERR_INVALID_ARG;
  if (batched) *batched = ctx->batch ? 1 : 0;
  if (graph) *graph = ctx->b_graph != nullptr ? 1 : 0;
  return MMP_OK;
}

int mmp_get_plan(mmp_ctx* ctx, int prob, int* quads_per_thread, int* ctas_per_slice,
                 int* max_concurrent_slices, int* particles_in_shared) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  const Prob& p = ctx->probs[prob];
  if (particles_in_shared) *particles_in_shared = p.layout == kLayoutSmem ? 1 : 0;
  if (quads_per_thread) *quads_per_thread = p.nq;
  if (ctas_per_slice) *ctas_per_slice = p.G;
  if (max_concurrent_slices) *max_concurrent_slices = p.slots_max;
  return MMP_OK;
}

int mmp_fine(mmp_ctx* ctx, int prob, int n, const void* u_in, void* u_out, double* stats_out) {
  Range nvtx_range("mmp_fine");
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  Prob& p = ctx->probs[prob];
  if (u_in == nullptr || u_out == nullptr || u_in == u_out || n < 0 || n >= p.d.N) return MMP_ERR_INVALID_ARG;
  if (((uintptr_t)u_in % 16) || ((uintptr_t)u_out % 16)) return MMP_ERR_INVALID_ARG;
  rc = run_fine(ctx, p, n, 1, p.nf, u_in, nullptr, u_out, 1, nullptr, 0, p.tmp_stats, 1);
  if (rc) return rc;
  if (stats_out)
    MMP_CUDA(cudaMemcpyAsync(stats_out, p.tmp_stats, sizeof(double) * kStat, cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  unsigned st[4];
  MMP_CUDA(cudaMemcpy(st, p.status, sizeof(st), cudaMemcpyDeviceToHost));
  return status_to_error(st[0]);
}

int mmp_philox(const unsigned int* ctr, const unsigned int* key, unsigned int* out, long long n, void* stream) {
  if (ctr == nullptr || key == nullptr || out == nullptr || n < 0) return MMP_ERR_INVALID_ARG;
  if (n == 0) return MMP_OK;
  if (((uintptr_t)ctr % 16) || ((uintptr_t)out % 16)) return MMP_ERR_INVALID_ARG;
  MMP_CUDA(launch_philox(ctr, key[0], key[1], out, n, (cudaStream_t)stream));
  return MMP_OK;
}

int mmp_normals(const mmp_problem_desc* desc, int tag, unsigned int j, unsigned int n, long long count,
                void* out, void* stream) {
  if (desc == nullptr || out == nullptr || count < 0 || tag < 0 || tag > 255 || n >= (1u << 24))
    return MMP_ERR_INVALID_ARG;
  if (desc->precision != MMP_FP64 && desc->precision != MMP_MIXED) return MMP_ERR_INVALID_ARG;
  // element-aligned output; particle quads are counted in 32 bits
  if ((uintptr_t)out % (desc->precision == MMP_MIXED ? sizeof(float) : sizeof(double)) != 0) return MMP_ERR_INVALID_ARG;
  if (count > (4LL << 32)) return MMP_ERR_INVALID_ARG;
  if (count == 0) return MMP_OK;
  MMP_CUDA(launch_normals(desc->precision, out, count, (uint32_t)tag, j, n, (uint32_t)(desc->seed & 0xffffffffull),
                          (uint32_t)(desc->seed >> 32), desc->problem_tag, (cudaStream_t)stream));
  return MMP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fine propagation without any device allocation (mmp_fine_static).
//
// Some callers cannot allocate device memory where they need a fine
// propagation: code issuing work while a stream is being captured into a
// CUDA graph (allocation calls are not allowed inside a capture), hosts that
// hand the whole device pool to another allocator and forbid allocations in
// their inner loop, and latency-bound loops where an allocation could stall.
// They own their ensembles; what they cannot provide is the scratch that the
// fine kernel's cross-CTA mean reduction needs (publication slots and
// epoch flags).  This entry point takes that scratch from one fixed array
// compiled into the library instead of a caller workspace.
// ---------------------------------------------------------------------------

// CTAs per slice the array serves: publication slots
// [MMP_STATIC_MAX_CTAS][kSlots][kNV] doubles, then the control block (the
// tagged step words [kSlots][MMP_STATIC_MAX_CTAS], one epoch flag per CTA
// and the status word) and one restriction row.
static_assert(MMP_STATIC_MAX_CTAS == 1216, "keep the header and the array in step");
constexpr size_t kStaticPartialDoubles = (size_t)MMP_STATIC_MAX_CTAS * kSeatDoubles;
constexpr size_t kStaticTagDoubles = (size_t)kSlots * MMP_STATIC_MAX_CTAS;
constexpr size_t kStaticCtlDoubles = kStaticTagDoubles + MMP_STATIC_MAX_CTAS / 2 + 8;
constexpr size_t kStaticDoubles = kStaticPartialDoubles + kStaticCtlDoubles + kStat;
static __device__ __align__(256) double mmp_static_scratch[kStaticDoubles];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_addr[kStaticMaxDevices] = {nullptr};

// The device address of the array on the current device, looked up once per
// device (the host-side name of a __device__ array is not a device address).
int static_scratch(double** out) {
  int dev = 0;
  MMP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return MMP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_addr[dev] == nullptr) {
    void* p = nullptr;
    MMP_CUDA(cudaGetSymbolAddress(&p, mmp_static_scratch));
    g_static_addr[dev] = (double*)p;
  }
  *out = g_static_addr[dev];
  return MMP_OK;
}

__global__ void k_status_to_stats(const unsigned* status, double* stats) {
  stats[14] = (double)status[0];
}

}  // namespace

extern "C" int mmp_fine_static(const mmp_problem_desc* desc, int n, const void* u_in, void* u_out,
                               double* stats_dev, void* stream) {
  if (desc == nullptr || u_in == nullptr || u_out == nullptr || u_in == u_out) return MMP_ERR_INVALID_ARG;
  if (((uintptr_t)u_in % 16) || ((uintptr_t)u_out % 16)) return MMP_ERR_INVALID_ARG;
  int rc = validate(*desc);
  if (rc) return rc;
  if (n < 0 || n >= desc->N) return MMP_ERR_INVALID_ARG;
  Prob p;
  p.d = *desc;
  derive(p);
  Device dev;
  rc = query_device(dev);
  if (rc) return rc;
  rc = plan(p, dev);
  if (rc) return rc;
  if (p.G > MMP_STATIC_MAX_CTAS) return MMP_ERR_UNSUPPORTED;
  double* base = nullptr;
  rc = static_scratch(&base);
  if (rc) return rc;
  unsigned long long* tags = (unsigned long long*)(base + kStaticPartialDoubles);
  unsigned* flags = (unsigned*)(base + kStaticPartialDoubles + kStaticTagDoubles);
  unsigned* status = flags + MMP_STATIC_MAX_CTAS;
  double* stats = stats_dev != nullptr ? stats_dev : base + kStaticPartialDoubles + kStaticCtlDoubles;
  cudaStream_t s = (cudaStream_t)stream;
  // every call shares the array: clear what must start at zero
  MMP_CUDA(cudaMemsetAsync(tags, 0, kStaticCtlDoubles * sizeof(double), s));
  // the problem's own arguments; only the buffers and the one task differ
  FineArgs a = fine_args_of(p, wait_limit_ns());
  a.slice_begin = n; a.n_tasks = 1;
  a.src0 = u_in; a.src = nullptr; a.dst = u_out; a.dst_fixed = 1;
  a.aff = nullptr; a.aff_fixed = 0;
  a.stats = stats; a.stats_fixed = 1;
  a.partials = base; a.flags = flags; a.tags = tags; a.status = status;
  a.tight_polls = p.G <= dev.sms ? kTightPolls : 0;
  MMP_CUDA(launch_fine(p.d.precision, p.layout, p.nq, p.mult, p.G, a, s, p.d.family));
  if (stats_dev != nullptr) {
    k_status_to_stats<<<1, 1, 0, s>>>(status, stats_dev);
    MMP_CUDA(cudaGetLastError());
  }
  return MMP_OK;
}

// ---------------------------------------------------------------------------
// Measured launch shapes (mmp_autotune, mmp_set_tuning).
//
// The planner's cost model ranks launch shapes by modelled time.  The
// autotuner measures instead: for each candidate count of quads per thread
// (shared-memory layout; it fixes the CTAs per slice G = ceil(Q / (256 nq))
// and the slices resident at once), one fine launch over all N slices of the
// problem, n_probe steps each, from the problem's own initial ensemble,
// timed with CUDA events after a warm-up launch.  Rates are particle-steps
// per second of that launch; the fastest candidate is returned, and
// mmp_set_tuning makes the planner use it for a range of P.
// ---------------------------------------------------------------------------

namespace {

struct TuneLayout {
  size_t bytes = 0;
  int seats = 0;
  char* u0 = nullptr;
  double* stats = nullptr;
  double* partials = nullptr;
  unsigned long long* tags = nullptr;  // followed by flags
  unsigned* flags = nullptr;
  unsigned* status = nullptr;
};

size_t tune_layout(const Prob& p, const Device& dev, char* base, TuneLayout& L) {
  Carver c{base, 0};
  auto ptr = [&](size_t b) -> char* {
    const size_t at = c.take(b);
    return base ? base + at : nullptr;
  };
  L.seats = 8 * dev.sms;  // at most 8 resident CTAs of 256 threads per SM
  L.u0 = ptr((size_t)p.pitch * p.esz);
  L.stats = (double*)ptr(sizeof(double) * kStat * (size_t)std::max(p.d.N, 2 * L.seats));
  L.partials = (double*)ptr(sizeof(double) * kSeatDoubles * (size_t)L.seats);
  L.tags = (unsigned long long*)ptr((sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * (size_t)L.seats);
  L.flags = base ? (unsigned*)(L.tags + (size_t)kSlots * L.seats) : nullptr;
  L.status = (unsigned*)ptr(sizeof(unsigned) * 4);
  L.bytes = (c.off + kAlign - 1) / kAlign * kAlign;
  return L.bytes;
}

}  // namespace

extern "C" int mmp_autotune_workspace_size(const mmp_problem_desc* desc, size_t* bytes) {
  if (desc == nullptr || bytes == nullptr) return MMP_ERR_INVALID_ARG;
  int rc = validate(*desc);
  if (rc) return rc;
  Prob p;
  p.d = *desc;
  derive(p);
  Device dev;
  rc = query_device(dev);
  if (rc) return rc;
  TuneLayout L;
  *bytes = tune_layout(p, dev, nullptr, L);
  return MMP_OK;
}

extern "C" int mmp_autotune(const mmp_problem_desc* desc, const int* candidates, int n_candidates, int probe_steps,
                            void* workspace, size_t bytes, void* stream, int* best_nq, double* rates) {
  Range nvtx_range("mmp_autotune");
  if (desc == nullptr || best_nq == nullptr) return MMP_ERR_INVALID_ARG;
  if (candidates != nullptr && n_candidates < 1) return MMP_ERR_INVALID_ARG;
  if (workspace == nullptr || ((uintptr_t)workspace % kAlign) != 0) return MMP_ERR_WORKSPACE;
  int rc = validate(*desc);
  if (rc) return rc;
  Prob p;
  p.d = *desc;
  derive(p);
  Device dev;
  rc = query_device(dev);
  if (rc) return rc;
  TuneLayout L;
  if (tune_layout(p, dev, (char*)workspace, L) > bytes) return MMP_ERR_WORKSPACE;
  const int max_nq = p.esz == 4 ? 32 : 16;
  std::vector<int> cand;
  if (candidates != nullptr) {
    cand.assign(candidates, candidates + n_candidates);
  } else {
    for (int k = 1; k <= max_nq; ++k) cand.push_back(k);
  }
  const int nf = probe_steps > 0 ? std::min(probe_steps, p.nf) : std::min(p.nf, 64);
  cudaStream_t s = (cudaStream_t)stream;
  MMP_CUDA(cudaMemsetAsync(L.status, 0, sizeof(unsigned) * 4, s));
  MMP_CUDA(launch_init_u0(p.d.precision, L.u0, p.d.P, p.Q, p.d.m0, p.d.s0, p.key0, p.key1, p.d.problem_tag,
                          p.d.family == MMP_FAMILY_ROTATOR, s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MMP_CUDA(cudaEventCreate(&e0));
  MMP_CUDA(cudaEventCreate(&e1));
  int best = 0;
  double best_rate = -1.0;
  int err = MMP_OK;
  for (size_t ci = 0; ci < cand.size() && err == MMP_OK; ++ci) {
    double rate = 0.0;
    const int nq = cand[ci];
    const void* fn = nq >= 1 && nq <= max_nq ? fine_kernel(p.d.precision, kLayoutSmem, nq, p.mult, p.d.family) : nullptr;
    size_t limit = 0;
    const size_t smem = fine_smem_bytes(p.d.precision, kLayoutSmem, nq, p.d.family);
    if (fn != nullptr && (err = allow_dynamic_smem(fn, dev.dev, &limit)) == MMP_OK && smem <= limit) {
      int occ = 0;
      cudaError_t ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTPB, smem);
      if (ce != cudaSuccess) {
        err = cuda_fail(ce, "occupancy", __LINE__);
        break;
      }
      const long long G = ((long long)p.Q + (long long)nq * kTPB - 1) / ((long long)nq * kTPB);
      if (occ >= 1 && G <= (long long)occ * dev.sms && G <= L.seats) {
        Prob t = p;
        t.layout = kLayoutSmem;
        t.nq = nq;
        t.G = (int)G;
        t.slots_max = (int)(std::min<long long>((long long)occ * dev.sms, L.seats) / G);
        t.u0 = L.u0;
        t.stats = L.stats;
        t.partials = L.partials;
        t.tags = L.tags;
        t.flags = L.flags;
        t.status = L.status;
        FineArgs a = fine_args_of(t, wait_limit_ns());
        // saturated: at least two full waves of resident slices (slice
        // indices past N only select other draws)
        const int n_tasks = std::max(p.d.N, 2 * t.slots_max);
        a.nf = nf;
        a.slice_begin = 0;
        a.n_tasks = n_tasks;
        a.aff = nullptr;
        const size_t sync = (sizeof(unsigned long long) * kSlots + sizeof(unsigned)) * (size_t)L.seats;
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && err == MMP_OK; ++rep) {  // warm-up, then timed
          ce = cudaMemsetAsync(L.tags, 0, sync, s);
          if (ce == cudaSuccess && rep == 1) ce = cudaEventRecord(e0, s);
          if (ce == cudaSuccess) ce = launch_fine(p.d.precision, kLayoutSmem, nq, p.mult, t.slots_max * t.G, a, s, p.d.family);
          if (ce == cudaSuccess && rep == 1) ce = cudaEventRecord(e1, s);
          if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
          if (ce != cudaSuccess) err = cuda_fail(ce, "autotune launch", __LINE__);
        }
        if (err == MMP_OK) {
          cudaError_t ce2 = cudaEventElapsedTime(&ms, e0, e1);
          unsigned stw = 0;
          if (ce2 == cudaSuccess) ce2 = cudaMemcpy(&stw, L.status, sizeof(unsigned), cudaMemcpyDeviceToHost);
          if (ce2 != cudaSuccess) {
            err = cuda_fail(ce2, "autotune timing", __LINE__);
          } else if (stw & kStatusTimeout) {
            err = MMP_ERR_TIMEOUT;
          } else if (ms > 0.0f) {
            rate = (double)n_tasks * (double)p.d.P * (double)nf / (ms * 1e-3);
          }
        }
      }
    }
    if (rates != nullptr) rates[ci] = rate;
    if (rate > best_rate) {
      best_rate = rate;
      best = nq;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err) return err;
  if (best_rate <= 0.0) return MMP_ERR_UNSUPPORTED;
  *best_nq = best;
  return MMP_OK;
}

extern "C" int mmp_set_tuning(int precision, long long p_lo, long long p_hi, int quads_per_thread) {
  if (precision != MMP_FP64 && precision != MMP_MIXED) return MMP_ERR_INVALID_ARG;
  if (quads_per_thread < 0 || quads_per_thread > (precision == MMP_MIXED ? 32 : 16)) return MMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (quads_per_thread == 0) {
    g_tune.erase(std::remove_if(g_tune.begin(), g_tune.end(),
                                [&](const TuneEntry& e) { return e.precision == precision; }),
                 g_tune.end());
    return MMP_OK;
  }
  if (p_lo < 1 || p_hi < p_lo) return MMP_ERR_INVALID_ARG;
  g_tune.push_back({precision, p_lo, p_hi, quads_per_thread});
  return MMP_OK;
}

extern "C" int mmp_set_batch_nq(int precision, int quads_per_thread) {
  if (precision != MMP_FP64 && precision != MMP_MIXED) return MMP_ERR_INVALID_ARG;
  if (quads_per_thread < 0 || quads_per_thread > (precision == MMP_MIXED ? 32 : 16)) return MMP_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_batch_nq[precision == MMP_MIXED ? 1 : 0] = quads_per_thread;
  return MMP_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint and resume (mmp_state_size, mmp_get_state, mmp_set_state).
//
// The state of a run is the contents of the workspace the layout uses (every
// particle buffer, macro state, matching record and control block lives
// there) plus each problem's host view of the iteration.  A blob starts with
// a header (library version, a hash of the problem descriptions and of each
// launch plan), so it is only restored into a context whose problems and
// plans are the same: the plan fixes the workspace layout and the order of
// every sum, so the resumed run continues bit for bit.  Restoring into a
// workspace at another address rewrites the batched records, which hold
// device pointers.
// ---------------------------------------------------------------------------

namespace {

constexpr unsigned long long kStateMagic = 0x6d6d702d73746174ull;  // "mmp-stat"

struct StateHeader {
  unsigned long long magic;
  int version, n;
  unsigned long long digest;
  unsigned long long ws_used;
};

struct ProbState {
  int sweeps, lifted, done, converged;
  double last_change;
};

unsigned long long fnv(unsigned long long h, const void* p, size_t n) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Digest of the problem descriptions (field by field: the struct's padding
// bytes carry no value) and of the launch plans.
unsigned long long state_digest(const mmp_ctx* c) {
  unsigned long long h = 1469598103934665603ull;
  for (const Prob& p : c->probs) {
    const mmp_problem_desc& d = p.d;
    const double dv[] = {d.c3, d.c1, d.kappa, d.c0, d.B, d.BE, d.B0, d.m0, d.s0, d.T, d.dt, d.coarse_h,
                         d.threshold, d.threshold2, d.threshold3, d.tol};
    const long long iv[] = {d.N, d.P, d.n_regions, d.variant, d.precision, (long long)d.seed,
                            (long long)d.problem_tag, d.max_iter, d.coarse_model, p.layout, p.nq, p.G,
                            p.slots_max};
    h = fnv(h, dv, sizeof(dv));
    h = fnv(h, iv, sizeof(iv));
  }
  return fnv(h, &c->ws_used, sizeof(c->ws_used));
}

size_t state_bytes(const mmp_ctx* c) {
  size_t b = sizeof(StateHeader);
  for (const Prob& p : c->probs) b += sizeof(ProbState) + sizeof(int) * (size_t)p.d.N;
  return b + c->ws_used;
}

}  // namespace

extern "C" int mmp_state_size(mmp_ctx* ctx, size_t* bytes) {
  if (ctx == nullptr || bytes == nullptr) return MMP_ERR_INVALID_ARG;
  *bytes = state_bytes(ctx);
  return MMP_OK;
}

extern "C" int mmp_get_state(mmp_ctx* ctx, void* dst) {
  Range nvtx_range("mmp_get_state");
  if (ctx != nullptr)
    for (const Prob& p : ctx->probs)
      if (p.fine_pending != 0) return MMP_ERR_STATE;  // a sweep half done is no resumable state
  if (ctx == nullptr || dst == nullptr) return MMP_ERR_INVALID_ARG;
  char* o = (char*)dst;
  StateHeader hd{kStateMagic, mmp_version(), (int)ctx->probs.size(), state_digest(ctx), ctx->ws_used};
  std::memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  for (const Prob& p : ctx->probs) {
    ProbState ps{p.sweeps, p.lifted ? 1 : 0, p.done ? 1 : 0, p.converged ? 1 : 0, p.last_change};
    std::memcpy(o, &ps, sizeof(ps));
    o += sizeof(ps);
    std::memcpy(o, p.out_buf.data(), sizeof(int) * (size_t)p.d.N);
    o += sizeof(int) * (size_t)p.d.N;
  }
  MMP_CUDA(cudaMemcpyAsync(o, ctx->ws, ctx->ws_used, cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  return MMP_OK;
}

extern "C" int mmp_set_state(mmp_ctx* ctx, const void* src) {
  Range nvtx_range("mmp_set_state");
  if (ctx == nullptr || src == nullptr) return MMP_ERR_INVALID_ARG;
  const char* i = (const char*)src;
  StateHeader hd;
  std::memcpy(&hd, i, sizeof(hd));
  i += sizeof(hd);
  if (hd.magic != kStateMagic || hd.version != mmp_version() || hd.n != (int)ctx->probs.size() ||
      hd.digest != state_digest(ctx) || hd.ws_used != ctx->ws_used)
    return MMP_ERR_STATE;
  // every host view must be one this context could have reached (the output
  // buffer indices select device buffers) before anything is changed
  const char* j = i;
  for (const Prob& p : ctx->probs) {
    ProbState ps;
    std::memcpy(&ps, j, sizeof(ps));
    j += sizeof(ps);
    if (ps.sweeps < 0 || ps.sweeps > p.d.N || (unsigned)ps.lifted > 1u || (unsigned)ps.done > 1u ||
        (unsigned)ps.converged > 1u)
      return MMP_ERR_STATE;
    for (int n = 0; n < p.d.N; ++n) {
      int b;
      std::memcpy(&b, j + sizeof(int) * (size_t)n, sizeof(b));
      if (b < -1 || b > 1) return MMP_ERR_STATE;
    }
    j += sizeof(int) * (size_t)p.d.N;
  }
  for (Prob& p : ctx->probs) {
    ProbState ps;
    std::memcpy(&ps, i, sizeof(ps));
    i += sizeof(ps);
    p.sweeps = ps.sweeps;
    p.lifted = ps.lifted != 0;
    p.done = ps.done != 0;
    p.converged = ps.converged != 0;
    p.last_change = ps.last_change;
    std::memcpy(p.out_buf.data(), i, sizeof(int) * (size_t)p.d.N);
    i += sizeof(int) * (size_t)p.d.N;
    p.adj_ready = false;
  }
  MMP_CUDA(cudaMemcpyAsync(ctx->ws, i, ctx->ws_used, cudaMemcpyHostToDevice, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ctx->batch) {
    const int rc = batch_setup(ctx);  // the batched records hold device pointers
    if (rc) return rc;
  }
  return MMP_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the failure detection (mmp_probe_wait): one CTA of a G-CTA
// group waits for peers that never publish; its bounded wait must run out.
// ---------------------------------------------------------------------------
int mmp_probe_wait(int channel, int G, double limit_ms, void* ws, size_t ws_bytes, void* stream,
                   unsigned* status_out) {
  if (channel != 0 && channel != 1) return MMP_ERR_INVALID_ARG;
  if (G < 1 || G > 1024 || !(limit_ms >= 1.0) || !(limit_ms <= 10000.0)) return MMP_ERR_INVALID_ARG;
  if (ws == nullptr || ((uintptr_t)ws % kAlign) != 0) return MMP_ERR_WORKSPACE;
  // partials [G][kSlots][kNV] doubles, tags [kSlots][G], flags [G], status
  const size_t part = sizeof(double) * (size_t)G * kSeatDoubles;
  const size_t tagb = sizeof(unsigned long long) * (size_t)kSlots * G;
  const size_t need = part + tagb + sizeof(unsigned) * ((size_t)G + 1);
  if (ws_bytes < need) return MMP_ERR_WORKSPACE;
  char* base = (char*)ws;
  double* partials = (double*)base;
  unsigned long long* tags = (unsigned long long*)(base + part);
  unsigned* flags = (unsigned*)(base + part + tagb);
  unsigned* status = flags + G;
  cudaStream_t s = (cudaStream_t)stream;
  MMP_CUDA(cudaMemsetAsync(tags, 0, need - part, s));
  MMP_CUDA(launch_wait_probe(partials, flags, tags, status, G, (unsigned long long)(limit_ms * 1e6), channel, s));
  unsigned st = 0;
  MMP_CUDA(cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MMP_CUDA(cudaStreamSynchronize(s));
  if (status_out != nullptr) *status_out = st;
  return (st & kStatusTimeout) ? MMP_ERR_TIMEOUT : MMP_OK;
}

// ---------------------------------------------------------------------------
// FMA throughput of the device in a precision (mmp_probe_fma): the peak the
// plain FP64 form is measured against.
// ---------------------------------------------------------------------------
int mmp_probe_fma(int precision, void* ws, size_t ws_bytes, void* stream, double* tflops) {
  if (precision != MMP_FP64 && precision != MMP_MIXED) return MMP_ERR_INVALID_ARG;
  if (tflops == nullptr) return MMP_ERR_INVALID_ARG;
  if (ws == nullptr || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < 8) return MMP_ERR_WORKSPACE;
  Device dev;
  int rc = query_device(dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = dev.sms * 4;
  const long long threads = (long long)grid * kTPB;
  // about 10^10 (FP64) or 3 x 10^11 (FP32) fused multiply-adds per timed launch
  const long long iters = std::max(1LL, (precision == MMP_FP64 ? 10000000000LL : 300000000000LL) / (threads * 8));
  MMP_CUDA(launch_fma_probe(precision, ws, iters / 10 + 1, grid, s));  // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MMP_CUDA(cudaEventCreate(&e0));
  MMP_CUDA(cudaEventCreate(&e1));
  MMP_CUDA(cudaEventRecord(e0, s));
  cudaError_t le = launch_fma_probe(precision, ws, iters, grid, s);
  cudaError_t re = cudaEventRecord(e1, s);
  cudaError_t se = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaError_t te = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MMP_CUDA(le);
  MMP_CUDA(re);
  MMP_CUDA(se);
  MMP_CUDA(te);
  *tflops = 2.0 * 8.0 * (double)threads * (double)iters / ((double)ms * 1e-3) / 1e12;
  return MMP_OK;
}

// ---------------------------------------------------------------------------
// The fine step's arithmetic without the cross-CTA exchange (mmp_probe_step):
// the ceiling the fused fine kernel's step loop is compared against.
// ---------------------------------------------------------------------------
int mmp_probe_step(int form, void* ws, size_t ws_bytes, void* stream, double* particle_steps_per_s) {
  if (form != 0 && form != 1) return MMP_ERR_INVALID_ARG;
  if (particle_steps_per_s == nullptr) return MMP_ERR_INVALID_ARG;
  if (ws == nullptr || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < 8) return MMP_ERR_WORKSPACE;
  Range nvtx_range("mmp_probe_step");
  Device dev;
  int rc = query_device(dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  MMP_CUDA(prepare_step_probe(form));
  const int grid = dev.sms * 2;  // two CTAs per SM, as the fine kernel runs
  const double particles = (double)grid * kTPB * 4.0 * step_probe_quads(form);
  const int steps = (int)std::max(1.0, 2.5e10 / particles);  // about 2.5e10 particle-steps per launch
  MMP_CUDA(launch_step_probe(form, (float*)ws, steps / 10 + 1, grid, s));  // warm-up
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MMP_CUDA(cudaEventCreate(&e0));
  MMP_CUDA(cudaEventCreate(&e1));
  MMP_CUDA(cudaEventRecord(e0, s));
  cudaError_t le = launch_step_probe(form, (float*)ws, steps, grid, s);
  cudaError_t re = cudaEventRecord(e1, s);
  cudaError_t se = cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaError_t te = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MMP_CUDA(le);
  MMP_CUDA(re);
  MMP_CUDA(se);
  MMP_CUDA(te);
  *particle_steps_per_s = particles * (double)steps / ((double)ms * 1e-3);
  return MMP_OK;
}

// Counters of the device-side iteration (mmp_sweep_info).
int mmp_sweep_info(mmp_ctx* ctx, int prob, double* out) {
  int rc = check_prob(ctx, prob);
  if (rc) return rc;
  if (out == nullptr) return MMP_ERR_INVALID_ARG;
  Prob& p = ctx->probs[prob];
  double ctl[16];
  MMP_CUDA(cudaMemcpyAsync(ctl, p.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, ctx->stream));
  MMP_CUDA(cudaStreamSynchronize(ctx->stream));
  out[0] = ctl[4];  // regions accepted, summed over slices and sweeps
  out[1] = ctl[5];  // regions rejected
  out[2] = ctl[8];  // the last sweep used learned fractions
  out[3] = ctl[6];  // two-region fit: alpha
  out[4] = ctl[7];  //                 beta
  out[5] = ctl[0];  // change of the last sweep
  return MMP_OK;
}
