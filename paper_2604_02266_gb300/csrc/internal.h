// Host-side internals shared by the zotfs translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/zotfs.h"
#include "frame_engine.cuh"

struct zotfs_plan_s {
  int M, N, logM, logN, nrx, ntx, qam, bps;
  zotfs_pulse pulse;
  zotfs_options opt;
  zotfs_tuning tune;
  int device, sm_count;
  float2* d_W;    // W[t] = exp(j 2 pi t / MN), FP32
  float2* d_Tab;  // Tab[(dl + N/2) M + k] = W[(dl k) mod MN], FP32
  double2* d_W64;   // the same tables in FP64 (FP64 plans)
  double2* d_Tab64;
  int* d_counters;
  int counter_next;
  // frame orders for multi-round launches (heaviest expected work first): a ring of
  // kOrderSlots arrays of kOrderCap frame indices
  int* d_order;
  int order_next;
  // plain-form scratch (one frame): y_dd, b/x/c/p/t/a vectors, scalars, paths
  void* d_plain;
  size_t plain_bytes;
  // large-frame kernel: one scratch slot per resident CTA (shapes that do not fit shared memory)
  char* d_big;
  size_t big_slot_bytes;
  int big_slots;
  size_t big_bytes;  // size of d_big (also the clustered large-frame kernel's slots)
  // paper-scale grids: the grid receiver's scratch (one frame at a time)
  char* d_grid;
  size_t grid_bytes;
  // orders the calls that use the plan's scratch (d_big, d_grid, d_plain) across streams
  cudaEvent_t scratch_done;
  bool scratch_used;
};

namespace zotfs {

using PathRec = PathRecT<float>;

void set_error(const std::string& msg);
// Records `what` and the CUDA error; returns ZOTFS_ENOMEM for an allocation failure, else
// ZOTFS_ECUDA.
zotfs_status cuda_fail(cudaError_t e, const char* what);

// Every device and pinned-host allocation of the library goes through these, so that
// zotfs_debug_fail_alloc can make a chosen one fail (cudaErrorMemoryAllocation, *p = NULL)
// without touching the device.
cudaError_t dev_alloc_bytes(void** p, size_t bytes);
cudaError_t host_alloc_bytes(void** p, size_t bytes, unsigned flags);
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_bytes(reinterpret_cast<void**>(p), bytes);
}
template <class T>
inline cudaError_t host_alloc(T** p, size_t bytes, unsigned flags) {
  return host_alloc_bytes(reinterpret_cast<void**>(p), bytes, flags);
}
int ilog2(int v);
bool is_pow2(int v);

// FFT radix of the in-shared-memory Zak transform when the caller leaves it open (radix 4
// with a closing radix-2 stage measured a few per cent faster than pure radix 2 at 64x32).
constexpr int kDefaultRadix = 4;

// Frame-order arrays rotate over kOrderSlots per plan, and work counters over 64: up to
// kOrderSlots calls of one plan may be in flight on different streams at once.
constexpr int kOrderCap = 16384, kOrderSlots = 16;

// Launch a kernel that writes into `order` a permutation of [0, n) listing frames by
// decreasing expected work: by increasing threshold theta (a lower threshold keeps more
// taps) when `theta` is given, else by decreasing total path count over the `nlists` lists
// of the frame's list set in `count` (set ids[i] of n_sets when ids is given, else set i;
// a set outside [0, n_sets) counts as empty).  Frames with equal keys keep no particular
// order.
cudaError_t launch_frame_order(const float* theta, const int32_t* count, const int32_t* ids, int n_sets, int nlists,
                               int n, int* order, cudaStream_t stream);

// Fill the constant parts of FrameArgs from a plan.
void fill_plan_args(const zotfs_plan_s* plan, FrameArgs& A);

// Choose the frame-kernel configuration for a shape; returns false if no SMEM-resident
// variant fits (the caller then reports ZOTFS_EUNSUPPORTED or uses the big-frame path).
struct FrameCfg {
  int E, NB, T;   // template rows/thread, blocks, threads per CTA
  bool coef;      // the variant keeps coefficient tables in shared memory
  int variant;    // index into the instantiation table
  size_t smem;
};
bool choose_frame_cfg(int M, int N, int nrx, int ntx, int p_max, int threads_override, FrameCfg& cfg,
                      int real_bytes = 4);

// Launch the persistent frame kernel (counter reset included).  n_frames > 0.  frames_per_cta
// frames are packed into each CTA (0 or 1: one), reduced to what the variant's thread limit
// and shared memory allow.
zotfs_status launch_frame_kernel(zotfs_plan_s* plan, const FrameCfg& cfg, FrameArgs& A, int radix,
                                 int ctas_per_sm, cudaStream_t stream, int frames_per_cta = 1);
// The frames per CTA a launch of `cfg` can take, at most `want`.
int frames_per_cta_for(const FrameCfg& cfg, int want);

// Variant table implemented in frame_variants.cu.  fpc: frames packed into one CTA (a (T, fpc)
// block, `smem` bytes of shared memory per frame; T * fpc <= the variant's TMAX, fpc <= 15).
int frame_variant_count();
bool frame_variant_info(int v, int& E, int& NB, int& TMAX, int& real_bytes, int& minb, int& coef);
cudaError_t frame_variant_launch(int v, const FrameArgs& A, int radix, int grid, int T, size_t smem,
                                 cudaStream_t stream, int fpc = 1);
cudaError_t frame_variant_occupancy(int v, int T, size_t smem, int& blocks, int fpc = 1);
// Whether variant v has an instantiation that packs frames (the small-frame variants).
bool frame_variant_packs(int v);
constexpr int kMaxFramesPerCta = 8;

// Large-frame kernel (big_variant.cu)
struct BigCfg {
  int T, EW;
  size_t smem, slot_bytes;
};
bool choose_big_cfg(int M, int N, int nrx, int ntx, int p_max, BigCfg& cfg);
cudaError_t big_launch(const BigCfg& cfg, const FrameArgs& A, int radix, int grid, char* scratch,
                       cudaStream_t stream);
cudaError_t big_occupancy(const BigCfg& cfg, int& blocks);

// Clustered large-frame kernel (big_cluster_variant.cu): one frame on CL CTAs of a cluster,
// its vectors in one global scratch slot per cluster.
struct BigClusterCfg {
  int CL, T, EQ;
  size_t smem, slot_bytes;
};
bool choose_big_cluster_cfg(int M, int N, int nrx, int ntx, int p_max, int CL, BigClusterCfg& cfg);
cudaError_t big_cluster_launch(const BigClusterCfg& cfg, const FrameArgs& A, int radix, int clusters, char* scratch,
                               cudaStream_t stream);
cudaError_t big_cluster_max_active(const BigClusterCfg& cfg, int& clusters);
// Clusters of one launch: the resident maximum, capped by `ctas_per_sm` CTAs per SM when it is
// positive.
int big_cluster_count(const BigClusterCfg& cfg, int max_active, int sm_count, int ctas_per_sm);

// Paper-scale grid receiver (grid_variant.cu): one SISO frame at a time on the whole GPU, a
// cooperative launch whose CTAs meet at grid barriers; frames with M > 256 or M N > 16384.
constexpr size_t kGridMaxElems = (size_t)1 << 19;  // M N up to 524288 (16384 x 32)
struct GridCfg {
  int T, EQ, E, grid, variant;
  size_t smem;
  int win_cols, win_dcap;  // the CG windows: columns per row (0: none), largest |dk| covered
  int tab_smem;            // the CG coefficient table in shared memory (else in global scratch)
};
bool grid_shape(int M, int N, int nrx, int ntx);
// ctas_per_sm: the plan's tuning, CTAs per SM of the cooperative launch (0: as many as fit, at
// most two).
cudaError_t choose_grid_cfg(int M, int N, int p_max, int sm_count, int ctas_per_sm, GridCfg& cfg);
size_t grid_scratch_size(int M, int N, int p_max, int grid);
cudaError_t grid_launch(const GridCfg& cfg, const FrameArgs& A, char* scratch, cudaStream_t stream);
// Runs one bounded device wait that nothing satisfies (0: an mbarrier wait, 1: the grid
// barrier with one CTA absent) and stores its outcome in *status.
cudaError_t check_bounded_wait(int which, uint32_t max_polls, int32_t* status, cudaStream_t stream);

// Cluster receiver (cluster_variant.cu): one SISO frame on C CTAs of a thread-block cluster.
struct ClusterCfg {
  int C, T;
  size_t smem;
};
bool choose_cluster_cfg(int M, int N, int nrx, int ntx, int p_max, int C, ClusterCfg& cfg);
cudaError_t cluster_launch(const ClusterCfg& cfg, const FrameArgs& A, int radix, int clusters, cudaStream_t stream);
cudaError_t cluster_max_active(const ClusterCfg& cfg, int& clusters);

// FrameArgs for a descriptor-driven launch over frames of one geometry (batch.cu); per-frame
// values (noise, threshold, QAM order, pilot amplitude, iterations, buffers) come from the
// descriptors.
void bucket_args(int M, int N, int nrx, int ntx, int pilot_mode, int guard, int p_max, int in_dtype, const float2* W,
                 const float2* Tab, FrameArgs& A);
// Work model of one frame (grid sizing of uneven batches; the autotuner's SM shares).
double frame_work(const zotfs_frame_desc& d);
// Root-of-unity tables of one (M, N) shape in FP32 (allocates).
zotfs_status make_shape_tables(int M, int N, float2** dW, float2** dTab);

// Plain form (plain.cu)
size_t plain_scratch_bytes(int M, int N, int nrx, int ntx, int p_max);
zotfs_status run_plain(zotfs_plan_s* plan, const void* y_pilot_td, const void* y_data_td, const float* noise_var,
                       const float* theta, int iters, const zotfs_paths* paths, float* x_hat, float* llr,
                       uint8_t* bits, int32_t* status, int n_frames, cudaStream_t stream);

// Self-check of cg_ratio<float> (capi.cu): q[i] = float(cg_ratio(a[i], b[i])).
cudaError_t launch_cg_ratio_check(const double* a, const double* b, float* q, int n, cudaStream_t stream);

extern thread_local int g_launches;

}  // namespace zotfs
