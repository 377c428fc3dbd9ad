// CUDA-graph capture of a batch run, and the launch-shape autotuner: both sit on top of the
// batch API (zotfs_batch_create / zotfs_rx_batch) and add no device code of their own.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

struct zotfs_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

using namespace zotfs;

zotfs_status tinval(const std::string& m) {
  set_error(m);
  return ZOTFS_EINVAL;
}

// Frames per SM (per unit of occupancy, times two) in the autotuner's timing sets.
constexpr int kTuneFramesPerSm = 4;

struct Candidate {
  int threads, radix, ctas, cluster, fpc;
};

// Launch shapes worth timing for one (M, N, n_rx, n_tx, p_max) group.
std::vector<Candidate> candidates(int M, int N, int nrx, int ntx, int p_max) {
  std::vector<Candidate> out;
  const int MN = M * N;
  bool any = false;
  for (int T = 32; T <= 1024 && T <= MN; T += 32) {
    FrameCfg cfg;
    if (!choose_frame_cfg(M, N, nrx, ntx, p_max, T, cfg) || cfg.T != T) continue;
    // frames per CTA: one, and packings of 2 and 4 small frames where the kernel takes them
    for (int fpc : {1, 2, 4}) {
      if (frames_per_cta_for(cfg, fpc) != fpc) continue;
      int occ = 0;
      if (frame_variant_occupancy(cfg.variant, cfg.T, cfg.smem, occ, fpc) != cudaSuccess || occ < 1) continue;
      any = true;
      for (int radix : {2, 4})
        for (int c = 1; c <= occ; ++c) out.push_back({T, radix, c, 0, fpc});
    }
  }
  if (!any) {  // the large-frame kernels: fixed threads and occupancy; radix, CTAs per frame
    BigCfg big;
    if (choose_big_cfg(M, N, nrx, ntx, p_max, big))
      for (int radix : {2, 4}) out.push_back({0, radix, 0, 1, 1});
    for (int cl : {2, 4}) {
      BigClusterCfg bc;
      if (choose_big_cluster_cfg(M, N, nrx, ntx, p_max, cl, bc))
        for (int radix : {2, 4}) out.push_back({0, radix, 0, cl, 1});
    }
  }
  return out;
}

// Mean milliseconds of one zotfs_rx_batch run of `D` with the given launch shape, or < 0 on
// failure (the error string is kept).
float time_shape(const std::vector<zotfs_frame_desc>& D, const Candidate& c, int max_sms, int warmup, int reps,
                 int32_t* d_status, cudaStream_t stream, cudaEvent_t e0, cudaEvent_t e1) {
  zotfs_batch_opts o{};
  o.threads_per_frame = c.threads;
  o.fft_radix = c.radix;
  o.ctas_per_sm = c.ctas;
  o.max_sms = max_sms;
  o.cluster = c.cluster;
  // frames per CTA travel in a tuning entry of the group's shape (the timing set is one shape)
  zotfs_tuning_entry te{};
  if (!D.empty()) {
    te.M = D[0].M;
    te.N = D[0].N;
    te.n_rx = D[0].n_rx;
    te.n_tx = D[0].n_tx;
    te.tuning.frames_per_cta = c.fpc;
    o.n_tuning = 1;
    o.tuning = &te;
  }
  zotfs_batch b = nullptr;
  if (zotfs_batch_create(D.data(), (int)D.size(), &o, &b) != ZOTFS_OK) return -1.f;
  float ms = -1.f;
  bool ok = true;
  for (int i = 0; i < warmup && ok; ++i) ok = zotfs_rx_batch(b, d_status, stream) == ZOTFS_OK;
  if (ok && cudaEventRecord(e0, stream) != cudaSuccess) ok = false;
  for (int i = 0; i < reps && ok; ++i) ok = zotfs_rx_batch(b, d_status, stream) == ZOTFS_OK;
  if (ok && cudaEventRecord(e1, stream) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / (float)reps;
  }
  zotfs_batch_destroy(b);
  return ms;
}

}  // namespace

extern "C" {

zotfs_status zotfs_batch_capture(zotfs_batch batch, int32_t* status, zotfs_graph* out) {
  if (!out) return tinval("out is NULL");
  *out = nullptr;
  if (!batch) return tinval("batch is NULL");
  if (!status) return tinval("status is NULL");
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "capture stream");
  zotfs_graph_s* g = new (std::nothrow) zotfs_graph_s();
  if (!g) {
    cudaStreamDestroy(s);
    set_error("host allocation failed");
    return ZOTFS_ENOMEM;
  }
  zotfs_status st = ZOTFS_OK;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    st = cuda_fail(e, "begin capture");
  } else {
    st = zotfs_rx_batch(batch, status, s);
    const std::string msg = st ? std::string(zotfs_last_error()) : std::string();
    e = cudaStreamEndCapture(s, &g->graph);  // always end the capture, even after an error
    if (st) {
      set_error(msg);
    } else if (e != cudaSuccess) {
      st = cuda_fail(e, "end capture");
    } else {
      e = cudaGraphInstantiate(&g->exec, g->graph, 0);
      if (e != cudaSuccess) st = cuda_fail(e, "graph instantiate");
    }
  }
  cudaStreamDestroy(s);
  if (st) {
    const std::string msg = zotfs_last_error();
    zotfs_graph_destroy(g);
    set_error(msg);
    return st;
  }
  *out = g;
  return ZOTFS_OK;
}

zotfs_status zotfs_graph_launch(zotfs_graph graph, zotfs_stream stream) {
  if (!graph || !graph->exec) return tinval("graph is NULL");
  g_launches = 0;
  cudaError_t e = cudaGraphLaunch(graph->exec, stream);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return ZOTFS_OK;
}

zotfs_status zotfs_graph_destroy(zotfs_graph graph) {
  if (!graph) return ZOTFS_OK;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  if (graph->graph) cudaGraphDestroy(graph->graph);
  delete graph;
  return ZOTFS_OK;
}

zotfs_status zotfs_autotune(const zotfs_frame_desc* descs, int n_frames, const zotfs_autotune_opts* opts,
                            zotfs_tuning_result* out, int max_out, int* n_out, zotfs_stream stream) {
  if (!n_out) return tinval("n_out is NULL");
  *n_out = 0;
  if (n_frames < 0 || (n_frames > 0 && !descs)) return tinval("descs / n_frames");
  if (max_out < 0 || (max_out > 0 && !out)) return tinval("out / max_out");
  zotfs_autotune_opts o{};
  if (opts) o = *opts;
  if (o.warmup < 0 || o.reps < 0 || o.max_frames < 0) return tinval("autotune options must be >= 0");
  const int warmup = o.warmup ? o.warmup : 2;
  const int reps = o.reps ? o.reps : 5;

  // groups in order of first appearance
  std::map<std::tuple<int, int, int, int>, int> key_to_group;
  std::vector<std::vector<zotfs_frame_desc>> groups;
  for (int i = 0; i < n_frames; ++i) {
    const zotfs_frame_desc& d = descs[i];
    auto key = std::make_tuple(d.M, d.N, d.n_rx, d.n_tx);
    auto it = key_to_group.find(key);
    if (it == key_to_group.end()) {
      it = key_to_group.emplace(key, (int)groups.size()).first;
      groups.emplace_back();
    }
    auto& G = groups[it->second];
    if (o.max_frames == 0 || (int)G.size() < o.max_frames) G.push_back(d);
  }
  if ((int)groups.size() > max_out) return tinval("more shape groups than max_out");
  int device = 0, sm_count = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_fail(e, "device query");

  // Each group is timed in the throughput regime it runs at inside a large batch: its sampled
  // frames are repeated until every SM holds several frames per resident CTA.  The repeats
  // read the same received frames but write hard bits to the tuner's own scratch (no x_hat,
  // LLR or path outputs), so the caller's outputs are left alone.
  const int target = 2 * kTuneFramesPerSm * sm_count;
  size_t most_bits = 0;
  for (auto& G : groups)
    for (const auto& d : G)
      most_bits = std::max(most_bits, (size_t)d.n_tx * d.M * d.N * 6 / 8);
  int32_t* d_status = nullptr;
  uint8_t* d_bits = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const size_t slot = (most_bits + 255) & ~size_t(255);
  e = dev_alloc(&d_status, sizeof(int32_t) * (size_t)target);
  if (e == cudaSuccess && !groups.empty()) e = dev_alloc(&d_bits, slot * (size_t)target);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  zotfs_status st = e == cudaSuccess ? ZOTFS_OK : cuda_fail(e, "autotune setup");

  for (size_t gi = 0; gi < groups.size() && st == ZOTFS_OK; ++gi) {
    const auto& G = groups[gi];
    const zotfs_frame_desc& d0 = G[0];
    int p_max = 0;
    for (const auto& d : G) p_max = std::max(p_max, d.p_max);
    std::vector<zotfs_frame_desc> T(target);
    for (int i = 0; i < target; ++i) {
      T[i] = G[(size_t)i % G.size()];
      T[i].x_hat = nullptr;
      T[i].llr = nullptr;
      T[i].path_count = nullptr;
      T[i].path_dk = T[i].path_dl = nullptr;
      T[i].path_h = nullptr;
      T[i].bits = d_bits + (size_t)i * slot;
    }
    zotfs_tuning_result R{};
    R.best.M = d0.M;
    R.best.N = d0.N;
    R.best.n_rx = d0.n_rx;
    R.best.n_tx = d0.n_tx;
    R.n_frames = target;
    R.ms_default = time_shape(T, Candidate{0, 0, 0, 0, 0}, 0, warmup, reps, d_status, stream, e0, e1);
    if (R.ms_default < 0.f) {
      st = ZOTFS_EINVAL;
      set_error(std::string("autotune: default launch shape failed: ") + zotfs_last_error());
      break;
    }
    R.ms_best = R.ms_default;
    for (const Candidate& c : candidates(d0.M, d0.N, d0.n_rx, d0.n_tx, p_max)) {
      const float ms = time_shape(T, c, 0, warmup, reps, d_status, stream, e0, e1);
      ++R.n_candidates;
      if (ms >= 0.f && ms < R.ms_best) {
        R.ms_best = ms;
        R.best.tuning.threads_per_frame = c.threads;
        R.best.tuning.fft_radix = c.radix;
        R.best.tuning.ctas_per_sm = c.ctas;
        R.best.tuning.cluster = c.cluster;
        R.best.tuning.frames_per_cta = c.fpc;
      }
    }
    R.sm_ms_per_frame = R.ms_best * (float)sm_count / (float)target;
    out[gi] = R;
    *n_out = (int)gi + 1;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_bits) cudaFree(d_bits);
  if (d_status) cudaFree(d_status);
  return st;
}

}  // extern "C"
