// Uneven persistent batches: frames of mixed shapes, antenna counts, QAM orders, noise levels
// and iteration counts in one call.  Frames are grouped into buckets of equal kernel
// geometry; each bucket runs one persistent frame kernel whose CTAs pull that bucket's frames
// from a device counter, and the buckets run side by side on the batch's own streams, each
// with a grid sized in proportion to its share of the batch's work.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

using zotfs::FrameArgs;
using zotfs::FrameCfg;

struct Bucket {
  int M, N, nrx, ntx, qam, pilot_mode, guard, p_max, in_dtype;
  float a_pilot;
  std::vector<int> ids;
  double work = 0.0;
  FrameCfg cfg{};
  int radix = 2;
  int ctas_per_sm = 0;
  int fpc = 1;  // frames packed into one CTA (shared-memory kernel)
  int grid = 0;
  int ids_off = 0;
  float2* d_W = nullptr;
  float2* d_Tab = nullptr;
  bool big = false;      // vectors too large for shared memory: the large-frame kernel
  zotfs::BigCfg bigcfg{};
  bool bigc = false;      // ... on clusters of bccfg.CL CTAs per frame (grid counts clusters)
  zotfs::BigClusterCfg bccfg{};
  char* d_big = nullptr;  // its scratch slots (one per CTA, or per cluster, of the grid)
};

}  // namespace

struct zotfs_batch_s {
  int n_frames = 0;
  int device = 0, sm_count = 0;
  std::vector<Bucket> buckets;
  zotfs_frame_desc* d_descs = nullptr;
  int* d_ids = nullptr;
  int* d_counters = nullptr;
  std::map<std::pair<int, int>, std::pair<float2*, float2*>> tables;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;  // [0] fork, [1..] joins
};

namespace zotfs {

static zotfs_status binval(const std::string& m) {
  set_error(m);
  return ZOTFS_EINVAL;
}

// Work model of one frame for sizing the buckets' grids: the gathers of the CG (two applies
// per iteration and one for b, over all antenna pairs and up to p_max paths) plus the
// transforms.
double frame_work(const zotfs_frame_desc& d) {
  return (double)d.M * d.N * d.n_rx * d.n_tx * d.p_max * (2.0 * d.iters + 1.0) + 8.0 * d.M * d.N;
}

zotfs_status make_shape_tables(int M, int N, float2** dW, float2** dTab) {
  const int MN = M * N;
  std::vector<float2> W(MN), Tab(MN);
  const double two_pi = 6.283185307179586476925286766559;
  for (int t = 0; t < MN; ++t) {
    const double a = two_pi * (double)t / (double)MN;
    W[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  for (int dl = -N / 2; dl < N / 2; ++dl)
    for (int k = 0; k < M; ++k) Tab[(size_t)(dl + N / 2) * M + k] = W[(size_t)(((long long)dl * k) & (MN - 1))];
  cudaError_t e = dev_alloc(dW, sizeof(float2) * MN);
  if (e == cudaSuccess) e = dev_alloc(dTab, sizeof(float2) * MN);
  if (e == cudaSuccess) e = cudaMemcpy(*dW, W.data(), sizeof(float2) * MN, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(*dTab, Tab.data(), sizeof(float2) * MN, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch tables");
  return ZOTFS_OK;
}

void bucket_args(int M, int N, int nrx, int ntx, int pilot_mode, int guard, int p_max, int in_dtype, const float2* W,
                 const float2* Tab, FrameArgs& A) {
  std::memset(&A, 0, sizeof(A));
  A.M = M;
  A.N = N;
  A.logM = ilog2(M);
  A.logN = ilog2(N);
  A.nrx = nrx;
  A.ntx = ntx;
  A.K0 = M / 2;
  A.L0 = N / 2;
  A.pilot_mode = pilot_mode;
  A.guard = guard;
  A.p_max = p_max;
  A.in_dtype = in_dtype;
  A.tap_dtype = ZOTFS_C64;
  A.qam = 4;
  A.bps = 2;
  A.a_pilot = std::sqrt((double)M * N);
  A.inv_sqrtN = 1.0 / std::sqrt((double)N);
  A.sqrtN = std::sqrt((double)N);
  A.pam_d = std::sqrt(3.0 / 6.0);
  for (int hb = 1; hb <= 3; ++hb) A.pam_d_hb[hb] = std::sqrt(3.0 / (2.0 * ((1 << (2 * hb)) - 1)));
  A.W = W;
  A.Tab = Tab;
  A.mode = kEstimate | kCG | kDemap | kWritePaths | kWriteX;
}

static zotfs_status validate_desc(const zotfs_frame_desc& d, int i) {
  auto bad = [&](const char* what) { return binval("frame " + std::to_string(i) + ": " + what); };
  if (!is_pow2(d.M) || d.M < 16 || d.M > 256) return bad("M must be a power of two in [16, 256]");
  if (!is_pow2(d.N) || d.N < 8 || d.N > 64) return bad("N must be a power of two in [8, 64]");
  if (d.M * d.N > 16384) return bad("M*N must be <= 16384");
  if (d.n_rx < 1 || d.n_rx > 4 || d.n_tx < 1 || d.n_tx > 4) return bad("n_rx, n_tx in [1, 4]");
  if (d.qam != 4 && d.qam != 16 && d.qam != 64) return bad("qam must be 4, 16 or 64");
  if (d.iters < 0) return bad("iters < 0");
  if (d.pilot_mode != ZOTFS_PILOT_SEPARATE && d.pilot_mode != ZOTFS_PILOT_EMBEDDED) return bad("pilot_mode");
  if (d.pilot_mode == ZOTFS_PILOT_EMBEDDED && (d.n_rx != 1 || d.n_tx != 1)) return bad("embedded pilot: SISO only");
  if (d.pilot_mode == ZOTFS_PILOT_EMBEDDED && (d.guard < 0 || d.guard >= d.M / 2)) return bad("guard");
  if (d.p_max < 1 || d.p_max > 256) return bad("p_max in [1, 256]");
  if (d.in_dtype != ZOTFS_C64 && d.in_dtype != ZOTFS_C32_F16 && d.in_dtype != ZOTFS_C32_BF16) return bad("in_dtype");
  if (!((d.K0 < 0 || d.K0 == d.M / 2) && (d.L0 < 0 || d.L0 == d.N / 2))) return bad("pilot must sit at (M/2, N/2)");
  if (!d.y_data) return bad("y_data is NULL");
  if (d.pilot_mode == ZOTFS_PILOT_SEPARATE && !d.y_pilot) return bad("y_pilot is NULL");
  if ((reinterpret_cast<uintptr_t>(d.y_data) & 15u) || (reinterpret_cast<uintptr_t>(d.y_pilot) & 15u))
    return bad("TD frames must be 16-byte aligned");
  if (!std::isfinite(d.noise_var) || d.noise_var < 0.f) return bad("noise_var must be finite and >= 0");
  if (!std::isfinite(d.theta)) return bad("theta must be finite");
  if (!std::isfinite(d.cg_eps) || d.cg_eps < 0.f) return bad("cg_eps must be finite and >= 0");
  if (d.path_count && (!d.path_dk || !d.path_dl || !d.path_h)) return bad("path outputs: all or none");
  return ZOTFS_OK;
}

}  // namespace zotfs

using namespace zotfs;

extern "C" {

zotfs_status zotfs_batch_create(const zotfs_frame_desc* descs, int n_frames, const zotfs_batch_opts* opts,
                                zotfs_batch* out) {
  g_launches = 0;
  if (!out) return binval("out is NULL");
  *out = nullptr;
  if (n_frames < 0 || (n_frames > 0 && !descs)) return binval("descs / n_frames");
  zotfs_batch_opts o{};
  if (opts) o = *opts;
  if (o.fft_radix != 0 && o.fft_radix != 2 && o.fft_radix != 4) return binval("fft_radix must be 0, 2 or 4");
  if (o.n_tuning < 0 || (o.n_tuning > 0 && !o.tuning)) return binval("tuning table");
  if (o.max_sms < 0) return binval("max_sms < 0");
  if (o.cluster != 0 && o.cluster != 1 && o.cluster != 2 && o.cluster != 4) return binval("cluster must be 0, 1, 2 or 4");

  std::vector<zotfs_frame_desc> D(descs, descs + n_frames);
  for (int i = 0; i < n_frames; ++i) {
    zotfs_status s = validate_desc(D[i], i);
    if (s) return s;
    if (D[i].K0 < 0) D[i].K0 = D[i].M / 2;
    if (D[i].L0 < 0) D[i].L0 = D[i].N / 2;
    if (!(D[i].a_pilot > 0.f)) {
      const double sq = std::sqrt((double)D[i].M * D[i].N);
      D[i].a_pilot = (float)(D[i].pilot_mode == ZOTFS_PILOT_EMBEDDED ? 0.5 * sq : sq);
    }
  }

  zotfs_batch_s* b = new (std::nothrow) zotfs_batch_s();
  if (!b) {
    set_error("host allocation failed");
    return ZOTFS_ENOMEM;
  }
  b->n_frames = n_frames;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess) {
    delete b;
    return cuda_fail(e, "device query");
  }

  // group frames into buckets of equal kernel geometry
  std::map<std::tuple<int, int, int, int, int, int, int, int>, int> key_to_bucket;
  for (int i = 0; i < n_frames; ++i) {
    const zotfs_frame_desc& d = D[i];
    // QAM order, pilot amplitude, noise, threshold and iteration count are per frame
    auto key = std::make_tuple(d.M, d.N, d.n_rx, d.n_tx, d.pilot_mode, d.guard, d.p_max, d.in_dtype);
    auto it = key_to_bucket.find(key);
    int bi;
    if (it == key_to_bucket.end()) {
      bi = (int)b->buckets.size();
      key_to_bucket[key] = bi;
      Bucket B;
      B.M = d.M;
      B.N = d.N;
      B.nrx = d.n_rx;
      B.ntx = d.n_tx;
      B.qam = d.qam;
      B.pilot_mode = d.pilot_mode;
      B.guard = d.guard;
      B.p_max = d.p_max;
      B.in_dtype = d.in_dtype;
      B.a_pilot = d.a_pilot;
      b->buckets.push_back(B);
    } else {
      bi = it->second;
    }
    Bucket& B = b->buckets[bi];
    B.ids.push_back(i);
    B.work += frame_work(d);
  }

  // per-bucket kernel configuration
  zotfs_status st = ZOTFS_OK;
  double total_work = 0.0;
  std::vector<int> occ(b->buckets.size(), 0);
  for (size_t bi = 0; bi < b->buckets.size() && st == ZOTFS_OK; ++bi) {
    Bucket& B = b->buckets[bi];
    int tpf = o.threads_per_frame, radix = o.fft_radix, cps = o.ctas_per_sm, cl = o.cluster, fpc = 0;
    for (int j = 0; j < o.n_tuning; ++j) {
      const zotfs_tuning_entry& te = o.tuning[j];
      if (te.M == B.M && te.N == B.N && te.n_rx == B.nrx && te.n_tx == B.ntx) {
        if (!o.threads_per_frame) tpf = te.tuning.threads_per_frame;
        if (!o.fft_radix) radix = te.tuning.fft_radix;
        if (!o.ctas_per_sm) cps = te.tuning.ctas_per_sm;
        if (!o.cluster) cl = te.tuning.cluster;
        fpc = te.tuning.frames_per_cta;
      }
    }
    B.radix = radix == 2 ? 2 : (radix == 4 ? 4 : kDefaultRadix);
    B.ctas_per_sm = cps;
    if (!choose_frame_cfg(B.M, B.N, B.nrx, B.ntx, B.p_max, tpf, B.cfg) &&
        !(tpf > 0 && choose_frame_cfg(B.M, B.N, B.nrx, B.ntx, B.p_max, 0, B.cfg))) {
      if (!choose_big_cfg(B.M, B.N, B.nrx, B.ntx, B.p_max, B.bigcfg)) {
        set_error("bucket " + std::to_string(B.M) + "x" + std::to_string(B.N) + " " + std::to_string(B.nrx) + "x" +
                  std::to_string(B.ntx) + ": no kernel for this shape");
        st = ZOTFS_EUNSUPPORTED;
        break;
      }
      B.big = true;
      // MIMO frames on 2-CTA clusters unless the caller asks otherwise (a SISO frame's pilot
      // and data transforms do not spread over the cluster's CTAs, which costs throughput);
      // separate pilot frames only: the clustered kernel does not remove an embedded pilot
      if ((cl >= 2 || (cl == 0 && B.nrx * B.ntx > 1)) && B.pilot_mode == ZOTFS_PILOT_SEPARATE)
        B.bigc = choose_big_cluster_cfg(B.M, B.N, B.nrx, B.ntx, B.p_max, cl >= 2 ? cl : 2, B.bccfg);
    }
    if (B.bigc) {
      int clusters = 0;
      e = big_cluster_max_active(B.bccfg, clusters);
      occ[bi] = std::max(1, clusters * B.bccfg.CL / std::max(1, b->sm_count));  // CTAs per SM
      if (e == cudaSuccess && clusters < 1) e = cudaErrorInvalidConfiguration;
    } else if (B.big) {
      e = big_occupancy(B.bigcfg, occ[bi]);
    } else {
      B.fpc = frames_per_cta_for(B.cfg, fpc);
      e = frame_variant_occupancy(B.cfg.variant, B.cfg.T, B.cfg.smem, occ[bi], B.fpc);
    }
    if (e != cudaSuccess) {
      st = cuda_fail(e, "occupancy query");
      break;
    }
    if (occ[bi] < 1) {
      set_error("frame kernel does not fit on an SM");
      st = ZOTFS_EUNSUPPORTED;
      break;
    }
    if (B.ctas_per_sm > 0 && B.ctas_per_sm < occ[bi]) occ[bi] = B.ctas_per_sm;
    total_work += B.work;
  }
  // grids: each bucket gets SMs in proportion to its work (at least one CTA)
  const int avail = o.max_sms > 0 ? std::min(o.max_sms, b->sm_count) : b->sm_count;
  for (size_t bi = 0; bi < b->buckets.size() && st == ZOTFS_OK; ++bi) {
    Bucket& B = b->buckets[bi];
    const double share = total_work > 0 ? B.work / total_work : 1.0;
    int sms = (int)std::ceil(share * avail);
    sms = std::max(1, std::min(sms, avail));
    B.grid = std::max(1, std::min(((int)B.ids.size() + B.fpc - 1) / B.fpc, sms * occ[bi]));
    if (B.bigc) B.grid = std::max(1, std::min((int)B.ids.size(), sms * occ[bi] / B.bccfg.CL));  // clusters
  }
  // each bucket's CTAs take its frames heaviest first (lowest threshold first: more taps pass
  // it; then more iterations), so the last frames to start are the lightest
  for (Bucket& B : b->buckets)
    std::stable_sort(B.ids.begin(), B.ids.end(), [&](int i, int j) {
      const float ti = std::isfinite(D[i].theta) ? D[i].theta : INFINITY;
      const float tj = std::isfinite(D[j].theta) ? D[j].theta : INFINITY;
      if (ti != tj) return ti < tj;
      return D[i].iters > D[j].iters;
    });
  // device copies: descriptors, frame ids per bucket, counters, per-shape tables
  std::vector<int> ids;
  for (Bucket& B : b->buckets) {
    B.ids_off = (int)ids.size();
    ids.insert(ids.end(), B.ids.begin(), B.ids.end());
  }
  if (st == ZOTFS_OK && n_frames > 0) {
    e = dev_alloc(&b->d_descs, sizeof(zotfs_frame_desc) * n_frames);
    if (e == cudaSuccess) e = dev_alloc(&b->d_ids, sizeof(int) * n_frames);
    if (e == cudaSuccess) e = dev_alloc(&b->d_counters, sizeof(int) * std::max<size_t>(1, b->buckets.size()));
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_descs, D.data(), sizeof(zotfs_frame_desc) * n_frames, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_ids, ids.data(), sizeof(int) * n_frames, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "batch allocation");
  }
  for (Bucket& B : b->buckets) {
    if (st) break;
    auto key = std::make_pair(B.M, B.N);
    auto it = b->tables.find(key);
    if (it == b->tables.end()) {
      float2 *W = nullptr, *T = nullptr;
      st = make_shape_tables(B.M, B.N, &W, &T);
      b->tables[key] = {W, T};
      it = b->tables.find(key);
    }
    B.d_W = it->second.first;
    B.d_Tab = it->second.second;
    if (B.big) {
      e = dev_alloc(&B.d_big, (B.bigc ? B.bccfg.slot_bytes : B.bigcfg.slot_bytes) * (size_t)B.grid);
      if (e != cudaSuccess) {
        st = e == cudaErrorMemoryAllocation ? ZOTFS_ENOMEM : cuda_fail(e, "large-frame scratch");
        if (st == ZOTFS_ENOMEM) set_error("large-frame scratch allocation failed");
      }
    }
  }
  // streams and fork/join events
  const size_t ns = b->buckets.size();
  for (size_t i = 0; i < ns && st == ZOTFS_OK; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "stream create");
      break;
    }
    b->streams.push_back(s);
  }
  for (size_t i = 0; i < ns + 1 && st == ZOTFS_OK; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "event create");
      break;
    }
    b->events.push_back(ev);
  }
  if (st != ZOTFS_OK) {
    std::string msg = zotfs_last_error();
    zotfs_batch_destroy(b);
    set_error(msg);
    return st;
  }
  *out = b;
  return ZOTFS_OK;
}

zotfs_status zotfs_rx_batch(zotfs_batch b, int32_t* status, zotfs_stream stream) {
  g_launches = 0;
  if (!b) return binval("batch is NULL");
  if (b->n_frames == 0) return ZOTFS_OK;
  if (!status) return binval("status is NULL");
  cudaStream_t caller = stream;
  cudaError_t e = cudaEventRecord(b->events[0], caller);
  if (e != cudaSuccess) return cuda_fail(e, "fork event");
  for (size_t bi = 0; bi < b->buckets.size(); ++bi) {
    Bucket& B = b->buckets[bi];
    cudaStream_t s = b->streams[bi];
    e = cudaStreamWaitEvent(s, b->events[0], 0);
    if (e != cudaSuccess) return cuda_fail(e, "fork wait");
    int* counter = b->d_counters + bi;
    e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    FrameArgs A;
    bucket_args(B.M, B.N, B.nrx, B.ntx, B.pilot_mode, B.guard, B.p_max, B.in_dtype, B.d_W, B.d_Tab, A);
    A.n_frames = (int)B.ids.size();
    A.work_counter = counter;
    A.status = status;
    A.descs = b->d_descs;
    A.frame_ids = b->d_ids + B.ids_off;
    e = B.bigc  ? big_cluster_launch(B.bccfg, A, B.radix, B.grid, B.d_big, s)
        : B.big ? big_launch(B.bigcfg, A, B.radix, B.grid, B.d_big, s)
                : frame_variant_launch(B.cfg.variant, A, B.radix, B.grid, B.cfg.T, B.cfg.smem, s, B.fpc);
    if (e != cudaSuccess) return cuda_fail(e, "bucket kernel launch");
    ++g_launches;
    e = cudaEventRecord(b->events[1 + bi], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, b->events[1 + bi], 0);
    if (e != cudaSuccess) return cuda_fail(e, "join");
  }
  return ZOTFS_OK;
}

zotfs_status zotfs_batch_destroy(zotfs_batch b) {
  if (!b) return ZOTFS_OK;
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t ev : b->events) cudaEventDestroy(ev);
  for (Bucket& B : b->buckets)
    if (B.d_big) cudaFree(B.d_big);
  for (auto& kv : b->tables) {
    cudaFree(kv.second.first);
    cudaFree(kv.second.second);
  }
  if (b->d_descs) cudaFree(b->d_descs);
  if (b->d_ids) cudaFree(b->d_ids);
  if (b->d_counters) cudaFree(b->d_counters);
  delete b;
  return ZOTFS_OK;
}

}  // extern "C"
