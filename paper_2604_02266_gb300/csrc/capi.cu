// C ABI of the zotfs library: plans, argument validation and dispatch to the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace zotfs {

thread_local std::string g_err;
thread_local int g_launches = 0;

void set_error(const std::string& msg) { g_err = msg; }

zotfs_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? ZOTFS_ENOMEM : ZOTFS_ECUDA;
}

// Allocation countdown of zotfs_debug_fail_alloc: -1 off; n >= 0 lets n more allocations
// through and fails the next one, which switches it off again.
static std::atomic<int> g_fail_after{-1};

static bool injected_failure() {
  int n = g_fail_after.load();
  while (n >= 0)
    if (g_fail_after.compare_exchange_weak(n, n - 1)) return n == 0;
  return false;
}

cudaError_t dev_alloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();  // not sticky: keep it out of later launch checks
  return e;
}

cudaError_t host_alloc_bytes(void** p, size_t bytes, unsigned flags) {
  *p = nullptr;
  if (injected_failure()) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaHostAlloc(p, bytes, flags);
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();
  return e;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

static zotfs_status inval(const std::string& msg) {
  set_error(msg);
  return ZOTFS_EINVAL;
}

void fill_plan_args(const zotfs_plan_s* plan, FrameArgs& A) {
  std::memset(&A, 0, sizeof(A));
  A.M = plan->M;
  A.N = plan->N;
  A.logM = plan->logM;
  A.logN = plan->logN;
  A.nrx = plan->nrx;
  A.ntx = plan->ntx;
  A.K0 = plan->opt.K0;
  A.L0 = plan->opt.L0;
  A.pilot_mode = plan->opt.pilot_mode;
  A.guard = plan->opt.guard;
  A.p_max = plan->opt.p_max;
  A.in_dtype = plan->opt.in_dtype;
  A.tap_dtype = plan->opt.tap_dtype;
  A.qam = plan->qam;
  A.bps = plan->bps;
  A.a_pilot = plan->opt.a_pilot;
  A.inv_sqrtN = 1.0 / std::sqrt((double)plan->N);
  A.sqrtN = std::sqrt((double)plan->N);
  A.pam_d = std::sqrt(3.0 / (2.0 * (plan->qam - 1)));
  for (int hb = 1; hb <= 3; ++hb) A.pam_d_hb[hb] = std::sqrt(3.0 / (2.0 * ((1 << (2 * hb)) - 1)));
  A.eps2 = (double)plan->opt.cg_eps * (double)plan->opt.cg_eps;
  const bool fp64 = plan->opt.compute == ZOTFS_COMPUTE_FP64;
  A.W = fp64 ? (const void*)plan->d_W64 : (const void*)plan->d_W;
  A.Tab = fp64 ? (const void*)plan->d_Tab64 : (const void*)plan->d_Tab;
}

static int real_bytes_of(const zotfs_plan_s* plan) { return plan->opt.compute == ZOTFS_COMPUTE_FP64 ? 8 : 4; }

bool choose_frame_cfg(int M, int N, int nrx, int ntx, int p_max, int threads_override, FrameCfg& cfg,
                      int real_bytes) {
  const int MN = M * N, nb = nrx > ntx ? nrx : ntx;
  // coefficient-table variants first; each only where its tables still leave room for the
  // variant's designed CTAs per SM (228 KB of shared memory per SM, 1 KB reserved per CTA)
  static const int kPref[] = {8, 0, 9, 1, 10, 3, 2, 4, 5, 6, 7};
  const size_t kSmemCap = 227 * 1024;
  for (int idx : kPref) {
    int E, NB, TMAX, rb, minb, coef;
    if (!frame_variant_info(idx, E, NB, TMAX, rb, minb, coef)) continue;
    if (rb != real_bytes) continue;
    if (NB < nb || E > N || (N % E) != 0) continue;
    const int T = MN / E;
    if (T < 32 || (T % 32) != 0 || T > TMAX || (T % M) != 0) continue;
    if (threads_override > 0 && T != threads_override) continue;
    const size_t smem = frame_smem_bytes(M, N, E, nrx, ntx, p_max, real_bytes, coef != 0);
    if (smem > kSmemCap) continue;
    if (coef) {
      const size_t per_cta = 228 * 1024 / (size_t)minb - 1024;
      if (smem > per_cta) continue;
    }
    cfg.E = E;
    cfg.NB = NB;
    cfg.T = T;
    cfg.coef = coef != 0;
    cfg.variant = idx;
    cfg.smem = smem;
    return true;
  }
  return false;
}

namespace {

// One CTA of 1024 threads: keys are 31-bit (theta's bit pattern, or 2^30 - total paths),
// bucketed into 256 ranges between the smallest and largest key, counted, scanned and
// scattered (ascending key = decreasing expected work).
__global__ void __launch_bounds__(1024) frame_order_kernel(const float* theta, const int32_t* count,
                                                           const int32_t* ids, int n_sets, int nlists, int n,
                                                           int* order) {
  __shared__ unsigned lo_s, hi_s;
  __shared__ int hist[256];
  auto key = [&](int i) -> unsigned {
    if (theta) {
      const float t = theta[i];
      return (t > 0.f && isfinite(t)) ? __float_as_uint(t) : 0x7f800000u;
    }
    int tot = 0;
    const int s = ids ? ids[i] : i;  // the frame's list set
    if (s >= 0 && s < n_sets)
      for (int l = 0; l < nlists; ++l) tot += count[(size_t)s * nlists + l];
    return (1u << 30) - (unsigned)min(max(tot, 0), 1 << 29);
  };
  if (threadIdx.x == 0) {
    lo_s = 0xffffffffu;
    hi_s = 0u;
  }
  if (threadIdx.x < 256) hist[threadIdx.x] = 0;
  __syncthreads();
  unsigned lo = 0xffffffffu, hi = 0u;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned k = key(i);
    lo = min(lo, k);
    hi = max(hi, k);
  }
  atomicMin(&lo_s, lo);
  atomicMax(&hi_s, hi);
  __syncthreads();
  lo = lo_s;
  const unsigned range = hi_s - lo;
  const int shift = range < 256u ? 0 : 32 - __clz(range) - 8;
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[min(255u, (key(i) - lo) >> shift)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = 0; b < 256; ++b) {
      const int c = hist[b];
      hist[b] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&hist[min(255u, (key(i) - lo) >> shift)], 1)] = i;
}

}  // namespace

cudaError_t launch_frame_order(const float* theta, const int32_t* count, const int32_t* ids, int n_sets, int nlists,
                               int n, int* order, cudaStream_t stream) {
  frame_order_kernel<<<1, 1024, 0, stream>>>(theta, count, ids, n_sets, nlists, n, order);
  return cudaGetLastError();
}

// Frames are taken heaviest-first when a launch needs more than one round of resident CTAs
// (the last round then holds the lightest frames): returns the order array to use, or NULL.
static const int* maybe_order(zotfs_plan_s* plan, const FrameArgs& A, int resident, cudaStream_t stream) {
  if (A.descs || A.frame_ids || A.n_frames <= resident || A.n_frames > kOrderCap) return nullptr;
  const bool by_theta = (A.mode & kEstimate) && A.theta;
  const bool by_count = !(A.mode & kEstimate) && (A.mode & kLoadPaths) && A.pcount;
  if (!by_theta && !by_count) return nullptr;
  int* order = plan->d_order + (size_t)(plan->order_next++ % kOrderSlots) * kOrderCap;
  if (launch_frame_order(by_theta ? A.theta : nullptr, by_count ? A.pcount : nullptr, A.path_ids,
                         A.path_ids ? A.n_path_sets : A.n_frames, A.nrx * A.ntx, A.n_frames, order,
                         stream) != cudaSuccess)
    return nullptr;  // run in index order
  ++g_launches;
  return order;
}

int frames_per_cta_for(const FrameCfg& cfg, int want) {
  int E, NB, TMAX, rb, minb, coef;
  if (want <= 1 || !frame_variant_packs(cfg.variant) || !frame_variant_info(cfg.variant, E, NB, TMAX, rb, minb, coef))
    return 1;
  int f = want > kMaxFramesPerCta ? kMaxFramesPerCta : want;
  while (f > 1 && (cfg.T * f > TMAX || ((cfg.smem + 127) & ~size_t(127)) * (size_t)f > 227 * 1024)) --f;
  return f;
}

zotfs_status launch_frame_kernel(zotfs_plan_s* plan, const FrameCfg& cfg, FrameArgs& A, int radix, int ctas_per_sm,
                                 cudaStream_t stream, int frames_per_cta) {
  int* counter = plan->d_counters + (plan->counter_next++ & 63);
  A.work_counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work counter)");
  const int fpc = frames_per_cta_for(cfg, frames_per_cta);
  int blocks = 0;
  e = frame_variant_occupancy(cfg.variant, cfg.T, cfg.smem, blocks, fpc);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (blocks < 1) {
    set_error("frame kernel does not fit on an SM (registers or shared memory)");
    return ZOTFS_EUNSUPPORTED;
  }
  if (ctas_per_sm > 0 && ctas_per_sm < blocks) blocks = ctas_per_sm;
  long long grid = (long long)plan->sm_count * blocks;
  if (const int* order = maybe_order(plan, A, (int)(grid * fpc), stream)) A.frame_ids = order;
  if (grid * fpc > A.n_frames) grid = (A.n_frames + fpc - 1) / fpc;
  e = frame_variant_launch(cfg.variant, A, radix, (int)grid, cfg.T, cfg.smem, stream, fpc);
  if (e != cudaSuccess) return cuda_fail(e, "frame kernel launch");
  ++g_launches;
  return ZOTFS_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static zotfs_status check_paths(const zotfs_plan_s* plan, const zotfs_paths* paths, bool need_status_ok) {
  (void)need_status_ok;
  if (!paths) return inval("paths is NULL");
  if (!paths->count || !paths->dk || !paths->dl || !paths->h) return inval("paths: NULL device pointer");
  if (paths->p_max != plan->opt.p_max) return inval("paths.p_max differs from the plan's p_max");
  if (paths->tap_dtype != plan->opt.tap_dtype) return inval("paths.tap_dtype differs from the plan's tap_dtype");
  return ZOTFS_OK;
}

static int radix_of(const zotfs_plan_s* plan) { return plan->tune.fft_radix == 2 ? 2 : 4; }

// Launch the shared-memory frame kernel when the shape fits one CTA, else the large-frame
// kernel on the plan's scratch slots.
// The cluster receiver, where the plan asks for it and the call qualifies: FP32 SISO, the
// data frame in the time domain, a separate pilot frame, no single apply / DZT.
static bool cluster_applies(const zotfs_plan_s* plan, int nrx, int ntx, const FrameArgs& A, ClusterCfg& cc) {
  if (plan->tune.cluster == 1 || real_bytes_of(plan) != 4 || A.y_is_dd || (A.mode & (kApply | kDzt | kLoadX)))
    return false;
  // an embedded pilot is removed from the data grid before the CG, which the cluster
  // receiver does not do
  if (!(A.mode & kCG) || A.pilot_mode != ZOTFS_PILOT_SEPARATE) return false;
  if (plan->tune.cluster >= 2)
    return choose_cluster_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.cluster, cc);
  // automatic: only where the one-CTA shared-memory kernel does not fit, and while the call
  // leaves SMs idle
  FrameCfg fc;
  if (choose_frame_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.threads_per_frame, fc,
                       real_bytes_of(plan)))
    return false;
  if ((long long)A.n_frames * 2 > plan->sm_count) return false;
  return choose_cluster_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, 2, cc);
}

// The clustered large-frame kernel, for calls the one-CTA shared-memory kernel cannot take:
// FP32, equalisation with separate pilot frames (lists estimated or loaded; DD or time-domain
// data).  cluster = 2 or 4 asks for it; cluster = 0 takes it with 4 CTAs per frame while the
// call has at most one frame per four SMs (latency), and with 2 otherwise for MIMO frames
// (measured on 4x4 128x64 frames: about as fast per SM as one CTA per frame, with half the
// frame latency and a shorter tail).
static bool big_cluster_applies(const zotfs_plan_s* plan, int nrx, int ntx, const FrameArgs& A,
                                BigClusterCfg& bc) {
  if (plan->tune.cluster == 1 || real_bytes_of(plan) != 4 || !plan->d_big) return false;
  if (!(A.mode & kCG) || (A.mode & (kApply | kDzt | kLoadX))) return false;
  if (A.pilot_mode != ZOTFS_PILOT_SEPARATE) return false;  // as for the cluster receiver
  FrameCfg fc;
  if (choose_frame_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.threads_per_frame, fc,
                       real_bytes_of(plan)))
    return false;
  if (plan->tune.cluster >= 2)
    return choose_big_cluster_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.cluster, bc);
  const bool low_load = (long long)A.n_frames * 4 <= plan->sm_count;
  // a SISO frame's pilot and data transforms do not spread over the cluster's CTAs, which
  // costs throughput (128x64 in a loaded batch: 6.45 ms against 5.53 ms on one CTA per frame)
  if (!low_load && nrx * ntx == 1) return false;
  const int first = low_load ? 4 : 2;
  return choose_big_cluster_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, first, bc) ||
         choose_big_cluster_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, 6 - first, bc);
}

// Calls that use the plan's scratch run after the previous such call, on whatever stream it
// was issued (outside stream capture, where the caller's stream order applies).
static cudaError_t scratch_acquire(zotfs_plan_s* plan, cudaStream_t stream, bool& capturing) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cs);
  if (e != cudaSuccess) return e;
  capturing = cs != cudaStreamCaptureStatusNone;
  if (capturing || !plan->scratch_used) return cudaSuccess;
  return cudaStreamWaitEvent(stream, plan->scratch_done, 0);
}
static cudaError_t scratch_release(zotfs_plan_s* plan, cudaStream_t stream, bool capturing) {
  if (capturing) return cudaSuccess;
  plan->scratch_used = true;
  return cudaEventRecord(plan->scratch_done, stream);
}

static zotfs_status launch_kernels(zotfs_plan_s* plan, int nrx, int ntx, FrameArgs& A, cudaStream_t stream);

static zotfs_status launch_any(zotfs_plan_s* plan, int nrx, int ntx, FrameArgs& A, cudaStream_t stream) {
  // kernels without plan scratch: the cluster receiver and the shared-memory frame kernel
  ClusterCfg cc;
  FrameCfg fc;
  if (!plan->d_grid && (cluster_applies(plan, nrx, ntx, A, cc) ||
                        choose_frame_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.threads_per_frame,
                                         fc, real_bytes_of(plan))))
    return launch_kernels(plan, nrx, ntx, A, stream);
  bool capturing = false;
  cudaError_t e = scratch_acquire(plan, stream, capturing);
  if (e != cudaSuccess) return cuda_fail(e, "plan scratch ordering");
  const zotfs_status st = launch_kernels(plan, nrx, ntx, A, stream);
  e = scratch_release(plan, stream, capturing);
  if (st == ZOTFS_OK && e != cudaSuccess) return cuda_fail(e, "plan scratch ordering");
  return st;
}

static zotfs_status launch_kernels(zotfs_plan_s* plan, int nrx, int ntx, FrameArgs& A, cudaStream_t stream) {
  if (plan->d_grid) {  // paper-scale grid: one frame at a time on the whole GPU
    if (plan->opt.pilot_mode != ZOTFS_PILOT_SEPARATE) {
      set_error("grids with M > 256 or M*N > 16384 take separate pilot frames only");
      return ZOTFS_EUNSUPPORTED;
    }
    GridCfg gc;
    cudaError_t e = choose_grid_cfg(plan->M, plan->N, plan->opt.p_max, plan->sm_count, plan->tune.ctas_per_sm, gc);
    if (e != cudaSuccess) return cuda_fail(e, "grid receiver configuration");
    if (grid_scratch_size(plan->M, plan->N, plan->opt.p_max, gc.grid) > plan->grid_bytes) {
      set_error("grid receiver scratch too small");
      return ZOTFS_EUNSUPPORTED;
    }
    e = grid_launch(gc, A, plan->d_grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid receiver launch");
    ++g_launches;
    return ZOTFS_OK;
  }
  ClusterCfg cc;
  if (cluster_applies(plan, nrx, ntx, A, cc)) {
    int clusters = 0;
    cudaError_t e = cluster_max_active(cc, clusters);
    if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
    if (clusters < 1) {
      set_error("cluster receiver does not fit on the device");
      return ZOTFS_EUNSUPPORTED;
    }
    if (clusters > A.n_frames) clusters = A.n_frames;
    e = cluster_launch(cc, A, radix_of(plan), clusters, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cluster kernel launch");
    ++g_launches;
    return ZOTFS_OK;
  }
  FrameCfg cfg;
  if (choose_frame_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, plan->tune.threads_per_frame, cfg,
                       real_bytes_of(plan)))
    return launch_frame_kernel(plan, cfg, A, radix_of(plan), plan->tune.ctas_per_sm, stream,
                               plan->tune.frames_per_cta);
  BigClusterCfg bcc;
  if (big_cluster_applies(plan, nrx, ntx, A, bcc)) {
    int clusters = 0;
    cudaError_t e = big_cluster_max_active(bcc, clusters);
    if (e != cudaSuccess) return cuda_fail(e, "cluster occupancy query");
    clusters = big_cluster_count(bcc, clusters, plan->sm_count, plan->tune.ctas_per_sm);
    const long long room = (long long)(plan->big_bytes / bcc.slot_bytes);
    if (clusters > room) clusters = (int)room;
    if (clusters > A.n_frames) clusters = A.n_frames;
    if (clusters < 1) {
      set_error("clustered large-frame receiver does not fit on the device");
      return ZOTFS_EUNSUPPORTED;
    }
    int* counter = plan->d_counters + (plan->counter_next++ & 63);
    A.work_counter = counter;
    e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work counter)");
    e = big_cluster_launch(bcc, A, radix_of(plan), clusters, plan->d_big, stream);
    if (e != cudaSuccess) return cuda_fail(e, "clustered large-frame kernel launch");
    ++g_launches;
    return ZOTFS_OK;
  }
  BigCfg big;
  if (real_bytes_of(plan) != 4 || !plan->d_big || !choose_big_cfg(plan->M, plan->N, nrx, ntx, plan->opt.p_max, big)) {
    set_error("no kernel for this shape / antenna count / precision");
    return ZOTFS_EUNSUPPORTED;
  }
  int* counter = plan->d_counters + (plan->counter_next++ & 63);
  A.work_counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work counter)");
  int grid = plan->big_slots < A.n_frames ? plan->big_slots : A.n_frames;
  e = big_launch(big, A, radix_of(plan), grid, plan->d_big, stream);
  if (e != cudaSuccess) return cuda_fail(e, "large-frame kernel launch");
  ++g_launches;
  return ZOTFS_OK;
}

}  // namespace zotfs

using namespace zotfs;

// The ABI's struct sizes (mirrored by the Python binding's ctypes structures).
static_assert(sizeof(zotfs_options) == 40, "zotfs_options layout");
static_assert(sizeof(zotfs_tuning) == 20, "zotfs_tuning layout");
static_assert(sizeof(zotfs_frame_desc) == 16 * 4 + 9 * 8, "zotfs_frame_desc layout");
static_assert(sizeof(zotfs_batch_opts) == 32, "zotfs_batch_opts layout");
static_assert(sizeof(zotfs_request) == 10 * 4 + 3 * 8, "zotfs_request layout");

namespace zotfs {
namespace {
__global__ void cg_ratio_check_kernel(const double* a, const double* b, float* q, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (float)cg_ratio<float>(a[i], b[i]);
}
}  // namespace
cudaError_t launch_cg_ratio_check(const double* a, const double* b, float* q, int n, cudaStream_t stream) {
  cg_ratio_check_kernel<<<(n + 255) / 256, 256, 0, stream>>>(a, b, q, n);
  return cudaGetLastError();
}
}  // namespace zotfs

extern "C" {

const char* zotfs_last_error(void) { return g_err.c_str(); }
int zotfs_last_launch_count(void) { return g_launches; }

zotfs_status zotfs_plan_create(int M, int N, int n_rx, int n_tx, zotfs_pulse pulse, int qam, zotfs_plan* out) {
  g_launches = 0;
  if (!out) return inval("out is NULL");
  *out = nullptr;
  if (!is_pow2(M) || M < 16 || M > 16384) return inval("M must be a power of two in [16, 16384]");
  if (!is_pow2(N) || N < 8 || N > 64) return inval("N must be a power of two in [8, 64]");
  if (n_rx < 1 || n_rx > 4 || n_tx < 1 || n_tx > 4) return inval("n_rx, n_tx must be in [1, 4]");
  const bool paper_scale = M > 256 || M * N > 16384;  // the grid receiver
  if (paper_scale && (n_rx != 1 || n_tx != 1))
    return inval("grids with M > 256 or M*N > 16384 are SISO only (n_rx = n_tx = 1)");
  if (paper_scale && ((size_t)M * N > kGridMaxElems || M < 32))
    return inval("grids with M > 256 or M*N > 16384 need 32 <= M and M*N <= 524288");
  if (qam != 4 && qam != 16 && qam != 64) return inval("qam must be 4, 16 or 64");
  if (pulse != ZOTFS_PULSE_SINC && pulse != ZOTFS_PULSE_RECT) return inval("unknown pulse");

  zotfs_plan_s* p = new (std::nothrow) zotfs_plan_s();
  if (!p) {
    set_error("host allocation failed");
    return ZOTFS_ENOMEM;
  }
  std::memset(p, 0, sizeof(*p));
  p->M = M;
  p->N = N;
  p->logM = ilog2(M);
  p->logN = ilog2(N);
  p->nrx = n_rx;
  p->ntx = n_tx;
  p->qam = qam;
  p->bps = ilog2(qam);
  p->pulse = pulse;
  p->opt.pilot_mode = ZOTFS_PILOT_SEPARATE;
  p->opt.K0 = M / 2;
  p->opt.L0 = N / 2;
  p->opt.a_pilot = (float)std::sqrt((double)M * N);
  p->opt.guard = 2;
  p->opt.p_max = 64;
  p->opt.in_dtype = ZOTFS_C64;
  p->opt.tap_dtype = ZOTFS_C64;
  p->opt.compute = ZOTFS_COMPUTE_FP32;
  p->tune.threads_per_frame = 0;
  p->tune.fft_radix = kDefaultRadix;
  p->tune.ctas_per_sm = 0;
  p->tune.frames_per_cta = 0;

  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "device query");
  }
  const int MN = M * N;
  // root-of-unity tables: FP64 on the host, stored FP32
  std::vector<float2> W(MN), Tab(MN);
  std::vector<double2> W64(MN), Tab64(MN);
  const double two_pi = 6.283185307179586476925286766559;
  for (int t = 0; t < MN; ++t) {
    const double a = two_pi * (double)t / (double)MN;
    W64[t] = make_double2(std::cos(a), std::sin(a));
    W[t] = make_float2((float)W64[t].x, (float)W64[t].y);
  }
  for (int dl = -N / 2; dl < N / 2; ++dl)
    for (int k = 0; k < M; ++k) {
      const size_t src = (size_t)(((long long)dl * k) & (MN - 1));
      Tab[(size_t)(dl + N / 2) * M + k] = W[src];
      Tab64[(size_t)(dl + N / 2) * M + k] = W64[src];
    }
  p->plain_bytes = paper_scale ? 0 : plain_scratch_bytes(M, N, n_rx, n_tx, 256);
  e = dev_alloc(&p->d_W, sizeof(float2) * MN);
  if (e == cudaSuccess) e = dev_alloc(&p->d_Tab, sizeof(float2) * MN);
  if (e == cudaSuccess) e = dev_alloc(&p->d_W64, sizeof(double2) * MN);
  if (e == cudaSuccess) e = dev_alloc(&p->d_Tab64, sizeof(double2) * MN);
  if (e == cudaSuccess) e = dev_alloc(&p->d_counters, sizeof(int) * 64);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->scratch_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = dev_alloc(&p->d_order, sizeof(int) * kOrderCap * kOrderSlots);
  if (e == cudaSuccess && p->plain_bytes) e = dev_alloc(&p->d_plain, p->plain_bytes);
  if (e == cudaSuccess && paper_scale) {
    // scratch for the largest grid the receiver launches (kGridMaxCtasPerSm CTAs per SM) and p_max 256
    p->grid_bytes = grid_scratch_size(M, N, 256, kGridMaxCtasPerSm * p->sm_count);
    e = dev_alloc(&p->d_grid, p->grid_bytes);
  }
  {
    FrameCfg fc;
    BigCfg bc;
    if (e == cudaSuccess && !choose_frame_cfg(M, N, n_rx, n_tx, 256, 0, fc, 4) &&
        choose_big_cfg(M, N, n_rx, n_tx, 64, bc)) {
      int occ = 0;
      e = big_occupancy(bc, occ);
      if (e == cudaSuccess) {
        p->big_slots = p->sm_count * (occ > 0 ? occ : 1);
        p->big_slot_bytes = bc.slot_bytes;
        p->big_bytes = bc.slot_bytes * (size_t)p->big_slots;
      }
      // room for every resident cluster of the clustered kernel too
      for (int CL : {2, 4}) {
        BigClusterCfg cc;
        int clusters = 0;
        if (e == cudaSuccess && choose_big_cluster_cfg(M, N, n_rx, n_tx, 64, CL, cc)) {
          e = big_cluster_max_active(cc, clusters);
          p->big_bytes = std::max(p->big_bytes, cc.slot_bytes * (size_t)clusters);
        }
      }
      if (e == cudaSuccess) e = dev_alloc(&p->d_big, p->big_bytes);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(p->d_W, W.data(), sizeof(float2) * MN, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_Tab, Tab.data(), sizeof(float2) * MN, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_W64, W64.data(), sizeof(double2) * MN, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_Tab64, Tab64.data(), sizeof(double2) * MN, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_counters, 0, sizeof(int) * 64);
  if (e != cudaSuccess) {
    zotfs_plan_destroy(p);
    if (e == cudaErrorMemoryAllocation) {
      set_error("device allocation failed");
      return ZOTFS_ENOMEM;
    }
    return cuda_fail(e, "plan tables");
  }
  *out = p;
  return ZOTFS_OK;
}

zotfs_status zotfs_plan_destroy(zotfs_plan plan) {
  if (!plan) return ZOTFS_OK;
  if (plan->d_W) cudaFree(plan->d_W);
  if (plan->d_Tab) cudaFree(plan->d_Tab);
  if (plan->d_W64) cudaFree(plan->d_W64);
  if (plan->d_Tab64) cudaFree(plan->d_Tab64);
  if (plan->d_counters) cudaFree(plan->d_counters);
  if (plan->d_order) cudaFree(plan->d_order);
  if (plan->d_plain) cudaFree(plan->d_plain);
  if (plan->d_big) cudaFree(plan->d_big);
  if (plan->d_grid) cudaFree(plan->d_grid);
  if (plan->scratch_done) cudaEventDestroy(plan->scratch_done);
  delete plan;
  return ZOTFS_OK;
}

zotfs_status zotfs_plan_set_options(zotfs_plan plan, const zotfs_options* o) {
  if (!plan || !o) return inval("NULL argument");
  zotfs_options n = *o;
  if (n.pilot_mode != ZOTFS_PILOT_SEPARATE && n.pilot_mode != ZOTFS_PILOT_EMBEDDED) return inval("pilot_mode");
  if (n.K0 < 0) n.K0 = plan->M / 2;
  if (n.L0 < 0) n.L0 = plan->N / 2;
  if (n.K0 != plan->M / 2 || n.L0 != plan->N / 2)
    return inval("the pilot must sit at (M/2, N/2) (Sec. III-B 'Channel Estimation')");
  if (!(n.a_pilot > 0.f)) {
    const double s = std::sqrt((double)plan->M * plan->N);
    n.a_pilot = (float)(n.pilot_mode == ZOTFS_PILOT_EMBEDDED ? 0.5 * s : s);
  }
  if (!std::isfinite(n.a_pilot)) return inval("a_pilot must be finite");
  if (n.pilot_mode == ZOTFS_PILOT_EMBEDDED) {
    if (plan->nrx != 1 || plan->ntx != 1) return inval("embedded pilot: SISO plans only");
    if (n.guard < 0 || n.guard >= plan->M / 2) return inval("guard must be in [0, M/2)");
  }
  if (n.p_max < 1 || n.p_max > 256) return inval("p_max must be in [1, 256]");
  for (int d : {n.in_dtype, n.tap_dtype})
    if (d != ZOTFS_C64 && d != ZOTFS_C32_F16 && d != ZOTFS_C32_BF16 && d != ZOTFS_C128) return inval("unknown dtype");
  if (n.compute != ZOTFS_COMPUTE_FP32 && n.compute != ZOTFS_COMPUTE_FP64) return inval("compute must be FP32 or FP64");
  if (!std::isfinite(n.cg_eps) || n.cg_eps < 0.f) return inval("cg_eps must be finite and >= 0");
  if (n.compute == ZOTFS_COMPUTE_FP64) {
    FrameCfg cfg;
    if (!choose_frame_cfg(plan->M, plan->N, plan->nrx, plan->ntx, n.p_max, 0, cfg, 8))
      return inval("no FP64 frame kernel for this shape / antenna count");
  }
  plan->opt = n;
  return ZOTFS_OK;
}

zotfs_status zotfs_plan_get_options(zotfs_plan plan, zotfs_options* o) {
  if (!plan || !o) return inval("NULL argument");
  *o = plan->opt;
  return ZOTFS_OK;
}

zotfs_status zotfs_plan_set_tuning(zotfs_plan plan, const zotfs_tuning* t) {
  if (!plan || !t) return inval("NULL argument");
  if (t->fft_radix != 0 && t->fft_radix != 2 && t->fft_radix != 4) return inval("fft_radix must be 0, 2 or 4");
  if (t->threads_per_frame < 0 || t->threads_per_frame > 1024) return inval("threads_per_frame");
  if (t->ctas_per_sm < 0) return inval("ctas_per_sm");
  if (t->cluster < 0 || t->cluster == 3 || t->cluster > 4) return inval("cluster must be 0, 1, 2 or 4");
  if (t->frames_per_cta < 0 || t->frames_per_cta > kMaxFramesPerCta) return inval("frames_per_cta must be 0..8");
  zotfs_tuning n = *t;
  if (n.fft_radix == 0) n.fft_radix = kDefaultRadix;
  if (n.threads_per_frame > 0) {
    FrameCfg cfg;
    if (!choose_frame_cfg(plan->M, plan->N, plan->nrx, plan->ntx, plan->opt.p_max, n.threads_per_frame, cfg,
                          real_bytes_of(plan)))
      return inval("no frame kernel with that many threads per frame for this plan");
  }
  plan->tune = n;
  return ZOTFS_OK;
}

zotfs_status zotfs_plan_get_tuning(zotfs_plan plan, zotfs_tuning* t) {
  if (!plan || !t) return inval("NULL argument");
  *t = plan->tune;
  return ZOTFS_OK;
}

zotfs_status zotfs_dzt(zotfs_plan plan, const void* y_td, float* y_dd, int n_grids, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_grids < 0) return inval("n_grids < 0");
  if (n_grids == 0) return ZOTFS_OK;
  if (!y_td || !y_dd) return inval("NULL buffer");
  if (!aligned16(y_td)) return inval("y_td must be 16-byte aligned");
  FrameArgs A;
  fill_plan_args(plan, A);
  A.nrx = A.ntx = 1;
  A.mode = kDzt;
  A.n_frames = n_grids;
  A.y_data = y_td;
  A.u_out = y_dd;
  return launch_any(plan, 1, 1, A, stream);
}

zotfs_status zotfs_estimate(zotfs_plan plan, const void* y_pilot_td, const float* theta, int n_frames,
                            const zotfs_paths* paths, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0) return inval("n_frames < 0");
  zotfs_status s = check_paths(plan, paths, true);
  if (s) return s;
  if (n_frames == 0) return ZOTFS_OK;
  if (!y_pilot_td || !theta) return inval("NULL buffer");
  if (!aligned16(y_pilot_td)) return inval("y_pilot_td must be 16-byte aligned");
  const bool emb = plan->opt.pilot_mode == ZOTFS_PILOT_EMBEDDED;
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kEstimate | kWritePaths;
  A.n_frames = n_frames;
  if (emb) A.y_data = y_pilot_td;
  else A.y_pilot = y_pilot_td;
  A.theta = theta;
  A.pcount = paths->count;
  A.pstatus = paths->status;
  A.pdk = paths->dk;
  A.pdl = paths->dl;
  A.ph = paths->h;
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_ss_apply(zotfs_plan plan, const zotfs_paths* paths, const float* v, float* u, int adjoint,
                            int n_frames, int32_t* status, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0) return inval("n_frames < 0");
  zotfs_status s = check_paths(plan, paths, false);
  if (s) return s;
  if (n_frames == 0) return ZOTFS_OK;
  if (!v || !u) return inval("NULL buffer");
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kLoadPaths | kApply;
  A.n_frames = n_frames;
  A.adjoint = adjoint ? 1 : 0;
  A.v_in = v;
  A.u_out = u;
  A.status = status;
  A.pcount = paths->count;
  A.pdk = paths->dk;
  A.pdl = paths->dl;
  A.ph = paths->h;
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_equalize(zotfs_plan plan, const void* y, int y_is_dd, const zotfs_paths* paths,
                            const float* noise_var, int iters, float* x_hat, int n_frames, int32_t* status,
                            zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0 || iters < 0) return inval("n_frames and iters must be >= 0");
  zotfs_status s = check_paths(plan, paths, false);
  if (s) return s;
  if (n_frames == 0) return ZOTFS_OK;
  if (!y || !noise_var || !x_hat) return inval("NULL buffer");
  if (y_is_dd && plan->opt.pilot_mode == ZOTFS_PILOT_EMBEDDED)
    return inval("embedded pilot: equalize takes the TD frame (the pilot is removed after the Zak transform)");
  if (!y_is_dd && !aligned16(y)) return inval("y must be 16-byte aligned");
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kLoadPaths | kCG | kWriteX;
  A.n_frames = n_frames;
  A.y_data = y;
  A.y_is_dd = y_is_dd ? 1 : 0;
  A.noise_var = noise_var;
  A.iters = iters;
  A.x_hat = x_hat;
  A.status = status;
  A.pcount = paths->count;
  A.pdk = paths->dk;
  A.pdl = paths->dl;
  A.ph = paths->h;
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_demap(zotfs_plan plan, const float* x_hat, const float* noise_var, float* llr, uint8_t* bits,
                         int n_frames, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0) return inval("n_frames < 0");
  if (n_frames == 0) return ZOTFS_OK;
  if (!x_hat || !noise_var) return inval("NULL buffer");
  if (!llr && !bits) return ZOTFS_OK;
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kLoadX | kDemap;
  A.n_frames = n_frames;
  A.x_in = x_hat;
  A.noise_var = noise_var;
  A.llr = llr;
  A.bits = bits;
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_rx(zotfs_plan plan, const void* y_pilot_td, const void* y_data_td, const float* noise_var,
                      const float* theta, int iters, const zotfs_paths* paths, float* x_hat, float* llr, uint8_t* bits,
                      int32_t* status, int n_frames, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0 || iters < 0) return inval("n_frames and iters must be >= 0");
  if (n_frames == 0) return ZOTFS_OK;
  const bool emb = plan->opt.pilot_mode == ZOTFS_PILOT_EMBEDDED;
  if ((!emb && !y_pilot_td) || !y_data_td || !noise_var || !theta || !status) return inval("NULL buffer");
  if ((!emb && !aligned16(y_pilot_td)) || !aligned16(y_data_td)) return inval("TD frames must be 16-byte aligned");
  if (paths) {
    zotfs_status s = check_paths(plan, paths, true);
    if (s) return s;
  }
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kEstimate | kCG | kDemap | (paths ? kWritePaths : 0) | (x_hat ? kWriteX : 0);
  A.n_frames = n_frames;
  A.y_pilot = y_pilot_td;
  A.y_data = y_data_td;
  A.noise_var = noise_var;
  A.theta = theta;
  A.iters = iters;
  A.x_hat = x_hat;
  A.llr = llr;
  A.bits = bits;
  A.status = status;
  if (paths) {
    A.pcount = paths->count;
    A.pstatus = paths->status;
    A.pdk = paths->dk;
    A.pdl = paths->dl;
    A.ph = paths->h;
  }
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_rx_lists(zotfs_plan plan, const void* y_data_td, const zotfs_paths* paths,
                            const int32_t* path_ids, int n_sets, const float* noise_var, int iters,
                            float* x_hat, float* llr, uint8_t* bits, int32_t* status, int n_frames,
                            zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0 || iters < 0) return inval("n_frames and iters must be >= 0");
  zotfs_status s = check_paths(plan, paths, false);
  if (s) return s;
  if (n_sets < 1 || (!path_ids && n_sets < n_frames)) return inval("n_sets must cover the frames' list sets");
  if (n_frames == 0) return ZOTFS_OK;
  if (!y_data_td || !noise_var || !status) return inval("NULL buffer");
  if (!aligned16(y_data_td)) return inval("TD frames must be 16-byte aligned");
  FrameArgs A;
  fill_plan_args(plan, A);
  A.mode = kLoadPaths | kCG | kDemap | (x_hat ? kWriteX : 0);
  A.n_frames = n_frames;
  A.y_data = y_data_td;
  A.noise_var = noise_var;
  A.iters = iters;
  A.x_hat = x_hat;
  A.llr = llr;
  A.bits = bits;
  A.status = status;
  A.pcount = paths->count;
  A.pdk = paths->dk;
  A.pdl = paths->dl;
  A.ph = paths->h;
  A.path_ids = path_ids;
  A.n_path_sets = n_sets;
  return launch_any(plan, plan->nrx, plan->ntx, A, stream);
}

zotfs_status zotfs_check_bounded_wait(int which, uint32_t max_polls, int32_t* status, zotfs_stream stream) {
  g_launches = 0;
  if (which != 0 && which != 1) return inval("which must be 0 (mbarrier wait) or 1 (grid barrier)");
  if (max_polls < 1 || max_polls > (1u << 24)) return inval("max_polls must be in [1, 2^24]");
  if (!status) return inval("status is NULL");
  cudaError_t e = check_bounded_wait(which, max_polls, status, stream);
  if (e != cudaSuccess) return cuda_fail(e, "bounded-wait check launch");
  ++g_launches;
  return ZOTFS_OK;
}

zotfs_status zotfs_check_cg_ratio(const double* a, const double* b, float* q, int n, zotfs_stream stream) {
  g_launches = 0;
  if (n < 0) return inval("n < 0");
  if (n == 0) return ZOTFS_OK;
  if (!a || !b || !q) return inval("NULL buffer");
  cudaError_t e = launch_cg_ratio_check(a, b, q, n, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cg ratio check launch");
  ++g_launches;
  return ZOTFS_OK;
}

zotfs_status zotfs_debug_fail_alloc(int after) {
  if (after < -1) return inval("after must be >= -1");
  g_fail_after.store(after);
  return ZOTFS_OK;
}

zotfs_status zotfs_rx_plain(zotfs_plan plan, const void* y_pilot_td, const void* y_data_td, const float* noise_var,
                            const float* theta, int iters, const zotfs_paths* paths, float* x_hat, float* llr,
                            uint8_t* bits, int32_t* status, int n_frames, zotfs_stream stream) {
  g_launches = 0;
  if (!plan) return inval("plan is NULL");
  if (n_frames < 0 || iters < 0) return inval("n_frames and iters must be >= 0");
  if (n_frames == 0) return ZOTFS_OK;
  const bool emb = plan->opt.pilot_mode == ZOTFS_PILOT_EMBEDDED;
  if ((!emb && !y_pilot_td) || !y_data_td || !noise_var || !theta || !status) return inval("NULL buffer");
  if (plan->opt.compute != ZOTFS_COMPUTE_FP32) {
    set_error("the plain form runs in FP32 only");
    return ZOTFS_EUNSUPPORTED;
  }
  if (plan->d_grid) {
    set_error("the plain form runs grids with M <= 256 and M*N <= 16384 only");
    return ZOTFS_EUNSUPPORTED;
  }
  if (paths) {
    zotfs_status s = check_paths(plan, paths, true);
    if (s) return s;
  }
  bool capturing = false;
  cudaError_t e = scratch_acquire(plan, stream, capturing);
  if (e != cudaSuccess) return cuda_fail(e, "plan scratch ordering");
  const zotfs_status st = run_plain(plan, y_pilot_td, y_data_td, noise_var, theta, iters, paths, x_hat, llr, bits,
                                    status, n_frames, stream);
  e = scratch_release(plan, stream, capturing);
  if (st == ZOTFS_OK && e != cudaSuccess) return cuda_fail(e, "plan scratch ordering");
  return st;
}

}  // extern "C"
