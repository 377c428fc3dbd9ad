// Serving: continuous batching of arriving frames on one GPU.
//
// Callers submit requests (frames already resident in device memory).  A scheduler thread
// owned by the server
//   * reaps finished waves (event queries) and publishes their completions,
//   * whenever a wave slot is free, admits pending requests in arrival order as long as the
//     device output arena can hold their results (memory-based admission; a frame that waits
//     is admitted as soon as earlier frames are released), and
//   * launches the wave: descriptors to the device, one persistent frame kernel per shape
//     bucket, forked onto the wave's worker streams and joined with events, statuses back.
// Waves in flight run concurrently, so frames admitted while others run overlap with them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "frame_big.cuh"
#include "internal.h"

namespace {

using namespace zotfs;
using Clock = std::chrono::steady_clock;

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

constexpr int kWorkers = 8;       // worker streams per wave
constexpr int kMaxBuckets = 128;  // shape buckets per wave
constexpr int kServerCluster = 2;  // CTAs per MIMO frame too large for one CTA's shared memory

struct Pending {
  zotfs_request r;
  int64_t arrival_ns;
};

struct Admitted {
  Pending p;
  size_t off, bytes;  // arena chunk
  size_t bits, llr, pc, pdk, pdl, ph;  // offsets within the arena
  int64_t admit_ns;
};

struct Wave {
  bool busy = false;
  int cls = -1;  // the queue it takes frames from: 0 light, 1 heavy, -1 either (one queue)
  std::vector<Admitted> frames;
  zotfs_frame_desc* h_desc = nullptr;  // pinned
  zotfs_frame_desc* d_desc = nullptr;
  int* h_ids = nullptr;  // pinned
  int* d_ids = nullptr;
  int* d_counters = nullptr;
  int32_t* h_status = nullptr;  // pinned, mapped: each frame's status, -1 until the kernel stores it
  int32_t* d_status = nullptr;  // the device's view of h_status
  std::vector<char> reported;   // completion already published
  int n_reported = 0;
  char* d_big = nullptr;        // large-frame scratch: big_slots slots of big_slot_bytes
  cudaStream_t main = nullptr;
  cudaStream_t work[kWorkers] = {};
  cudaEvent_t start = nullptr, done = nullptr, wdone[kWorkers] = {};
};

}  // namespace

struct zotfs_server_s {
  zotfs_server_opts o{};
  int device = 0, sm_count = 0;
  std::map<std::pair<int, int>, std::pair<float2*, float2*>> tables;
  char* arena = nullptr;
  size_t arena_bytes = 0, in_use = 0, high_water = 0;
  std::map<size_t, size_t> free_list;  // offset -> size
  std::unordered_map<uint64_t, std::pair<size_t, size_t>> live;  // tag -> arena chunk (completed, unreleased)
  std::unordered_map<uint64_t, zotfs_request> live_req;            // tag -> its request (shape of the outputs)
  std::vector<Wave> waves;
  size_t big_slot_bytes = 0;
  int big_slots = 0;
  std::deque<Pending> pending[2];  // light, heavy (one queue: everything is heavy)
  bool split = false;              // light frames have their own queue and wave slots
  std::deque<zotfs_completion> done;
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  std::string thread_error;
  zotfs_server_stats st{};
};

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int frame_class(const zotfs_server_s* s, const zotfs_request& r) {
  const long long work = (long long)r.M * r.N * r.n_rx * r.n_tx;
  return (s->split && work <= s->o.light_work) ? 0 : 1;
}

size_t pending_total(const zotfs_server_s* s) { return s->pending[0].size() + s->pending[1].size(); }

bool arena_alloc(zotfs_server_s* s, size_t bytes, size_t& off) {
  for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
    if (it->second >= bytes) {
      off = it->first;
      const size_t rest = it->second - bytes;
      s->free_list.erase(it);
      if (rest) s->free_list[off + bytes] = rest;
      s->in_use += bytes;
      s->high_water = std::max(s->high_water, s->in_use);
      return true;
    }
  }
  return false;
}

void arena_free(zotfs_server_s* s, size_t off, size_t bytes) {
  auto it = s->free_list.emplace(off, bytes).first;
  // merge with the next and previous free ranges
  auto nx = std::next(it);
  if (nx != s->free_list.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_list.erase(nx);
  }
  if (it != s->free_list.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_list.erase(it);
    }
  }
  s->in_use -= bytes;
}

// Arena bytes of one frame's outputs and their offsets inside its chunk.
size_t frame_bytes(const zotfs_server_s* s, const zotfs_request& r, Admitted* a) {
  const size_t MN = (size_t)r.M * r.N;
  const int bps = ilog2(r.qam), nl = r.n_rx * r.n_tx, pm = s->o.p_max;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t o = off;
    off += align256(b);
    return o;
  };
  const size_t bits = take((size_t)r.n_tx * MN * bps / 8);
  const size_t llr = s->o.keep_llr ? take((size_t)r.n_tx * MN * bps * sizeof(float)) : 0;
  const size_t pc = take((size_t)nl * sizeof(int32_t));
  const size_t pdk = take((size_t)nl * pm * sizeof(int16_t));
  const size_t pdl = take((size_t)nl * pm * sizeof(int16_t));
  const size_t ph = take((size_t)nl * pm * sizeof(float2));
  if (a) {
    a->bits = bits;
    a->llr = llr;
    a->pc = pc;
    a->pdk = pdk;
    a->pdl = pdl;
    a->ph = ph;
  }
  return off;
}

zotfs_status validate_request(const zotfs_server_s* s, const zotfs_request& r) {
  auto bad = [](const char* m) {
    set_error(std::string("zotfs_server_submit: ") + m);
    return ZOTFS_EINVAL;
  };
  if (!is_pow2(r.M) || r.M < 16 || r.M > s->o.max_M) return bad("M must be a power of two in [16, max_M]");
  if (!is_pow2(r.N) || r.N < 8 || r.N > s->o.max_N || r.M * r.N > 16384) return bad("N out of range");
  if (r.n_rx < 1 || r.n_tx < 1 || r.n_rx > s->o.max_ant || r.n_tx > s->o.max_ant) return bad("antennas out of range");
  if (r.qam != 4 && r.qam != 16 && r.qam != 64) return bad("qam must be 4, 16 or 64");
  if (r.iters < 0) return bad("iters < 0");
  if (!r.y_pilot || !r.y_data) return bad("NULL frame");
  if ((reinterpret_cast<uintptr_t>(r.y_pilot) | reinterpret_cast<uintptr_t>(r.y_data)) & 15u)
    return bad("frames must be 16-byte aligned");
  if (!std::isfinite(r.noise_var) || r.noise_var < 0.f || !std::isfinite(r.theta)) return bad("noise_var / theta");
  if (!std::isfinite(r.cg_eps) || r.cg_eps < 0.f) return bad("cg_eps must be finite and >= 0");
  return ZOTFS_OK;
}

// Launch one formed wave (scheduler thread; touches only the wave and read-only server state).
cudaError_t launch_wave(zotfs_server_s* s, Wave& w) {
  const int n = (int)w.frames.size();
  // bucket frames by geometry
  std::map<std::tuple<int, int, int, int>, std::vector<int>> buckets;
  for (int i = 0; i < n; ++i) {
    const zotfs_request& r = w.frames[i].p.r;
    buckets[std::make_tuple(r.M, r.N, r.n_rx, r.n_tx)].push_back(i);
  }
  int pos = 0;
  for (auto& kv : buckets)
    for (int i : kv.second) w.h_ids[pos++] = i;
  for (int i = 0; i < n; ++i) {
    const Admitted& a = w.frames[i];
    const zotfs_request& r = a.p.r;
    zotfs_frame_desc& d = w.h_desc[i];
    std::memset(&d, 0, sizeof(d));
    d.M = r.M;
    d.N = r.N;
    d.n_rx = r.n_rx;
    d.n_tx = r.n_tx;
    d.qam = r.qam;
    d.iters = r.iters;
    d.pilot_mode = ZOTFS_PILOT_SEPARATE;
    d.guard = 2;
    d.p_max = s->o.p_max;
    d.in_dtype = ZOTFS_C64;
    d.K0 = r.M / 2;
    d.L0 = r.N / 2;
    d.noise_var = r.noise_var;
    d.cg_eps = r.cg_eps;
    d.theta = r.theta;
    d.a_pilot = r.a_pilot > 0.f ? r.a_pilot : (float)std::sqrt((double)r.M * r.N);
    d.y_pilot = r.y_pilot;
    d.y_data = r.y_data;
    char* base = s->arena + a.off;
    d.bits = reinterpret_cast<uint8_t*>(base + a.bits);
    d.llr = s->o.keep_llr ? reinterpret_cast<float*>(base + a.llr) : nullptr;
    d.path_count = reinterpret_cast<int32_t*>(base + a.pc);
    d.path_dk = reinterpret_cast<int16_t*>(base + a.pdk);
    d.path_dl = reinterpret_cast<int16_t*>(base + a.pdl);
    d.path_h = reinterpret_cast<float*>(base + a.ph);
  }
  for (int i = 0; i < n; ++i) reinterpret_cast<volatile int32_t*>(w.h_status)[i] = -1;
  w.reported.assign(n, 0);
  w.n_reported = 0;
  cudaError_t e = cudaMemcpyAsync(w.d_desc, w.h_desc, sizeof(zotfs_frame_desc) * n, cudaMemcpyHostToDevice, w.main);
  if (e == cudaSuccess) e = cudaMemcpyAsync(w.d_ids, w.h_ids, sizeof(int) * n, cudaMemcpyHostToDevice, w.main);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.d_counters, 0, sizeof(int) * buckets.size(), w.main);
  if (e == cudaSuccess) e = cudaEventRecord(w.start, w.main);
  if (e != cudaSuccess) return e;
  int b = 0, off = 0, big_next = 0;
  bool used[kWorkers] = {false};
  // large-frame buckets get disjoint ranges of the wave's scratch slots: one each, the rest
  // in proportion to their frame counts (the ranges never overlap, so these kernels may run
  // side by side)
  std::vector<int> big_share;
  {
    std::vector<int> nfs;
    int big_frames = 0;
    for (auto& kv : buckets) {
      FrameCfg fc;
      const auto& key = kv.first;
      if (!choose_frame_cfg(std::get<0>(key), std::get<1>(key), std::get<2>(key), std::get<3>(key), s->o.p_max, 0,
                            fc)) {
        nfs.push_back((int)kv.second.size());
        big_frames += (int)kv.second.size();
      }
    }
    if ((int)nfs.size() > s->big_slots) return cudaErrorInvalidValue;
    const int extra = s->big_slots - (int)nfs.size();
    for (int nf : nfs) big_share.push_back(1 + (big_frames ? (int)((long long)extra * nf / big_frames) : 0));
  }
  int big_idx = 0;
  for (auto& kv : buckets) {
    const int M = std::get<0>(kv.first), N = std::get<1>(kv.first), nrx = std::get<2>(kv.first),
              ntx = std::get<3>(kv.first);
    const int nf = (int)kv.second.size();
    const int wi = b % kWorkers;
    cudaStream_t st = w.work[wi];
    if (!used[wi]) {
      e = cudaStreamWaitEvent(st, w.start, 0);
      if (e != cudaSuccess) return e;
      used[wi] = true;
    }
    const auto& tb = s->tables.at(std::make_pair(M, N));
    FrameArgs A;
    bucket_args(M, N, nrx, ntx, ZOTFS_PILOT_SEPARATE, 2, s->o.p_max, ZOTFS_C64, tb.first, tb.second, A);
    A.n_frames = nf;
    A.work_counter = w.d_counters + b;
    A.status = w.d_status;
    A.status_fence = 1;
    A.descs = w.d_desc;
    A.frame_ids = w.d_ids + off;
    FrameCfg fc;
    if (choose_frame_cfg(M, N, nrx, ntx, s->o.p_max, 0, fc)) {
      int occ = 1;
      frame_variant_occupancy(fc.variant, fc.T, fc.smem, occ);
      const int grid = std::max(1, std::min(nf, s->sm_count * std::max(occ, 1)));
      e = frame_variant_launch(fc.variant, A, kDefaultRadix, grid, fc.T, fc.smem, st);
    } else {
      // MIMO frames on 2-CTA clusters (half the frame latency of one CTA per frame at the
      // same cost per SM), one scratch slot per cluster; SISO frames on one CTA each
      const int share = big_share[big_idx++];
      char* slots = w.d_big + (size_t)big_next * s->big_slot_bytes;
      BigClusterCfg bcc;
      if (nrx * ntx > 1 && choose_big_cluster_cfg(M, N, nrx, ntx, s->o.p_max, kServerCluster, bcc)) {
        bcc.slot_bytes = s->big_slot_bytes;
        const int clusters = std::max(1, std::min(nf, share / kServerCluster));
        e = big_cluster_launch(bcc, A, kDefaultRadix, clusters, slots, st);
      } else {
        BigCfg bc;
        if (!choose_big_cfg(M, N, nrx, ntx, s->o.p_max, bc)) return cudaErrorInvalidValue;
        bc.slot_bytes = s->big_slot_bytes;
        e = big_launch(bc, A, kDefaultRadix, std::min(nf, share), slots, st);
      }
      big_next += share;
    }
    if (e != cudaSuccess) return e;
    off += nf;
    ++b;
  }
  for (int wi = 0; wi < kWorkers; ++wi)
    if (used[wi]) {
      e = cudaEventRecord(w.wdone[wi], w.work[wi]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(w.main, w.wdone[wi], 0);
      if (e != cudaSuccess) return e;
    }
  return cudaEventRecord(w.done, w.main);
}

void scheduler(zotfs_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // publish frames as their statuses appear in mapped memory; free waves whose work is done
    bool any_busy = false;
    for (Wave& w : s->waves) {
      if (!w.busy) continue;
      const cudaError_t q = cudaEventQuery(w.done);
      const bool finished = q != cudaErrorNotReady;
      const int64_t t = now_ns();
      for (size_t i = 0; i < w.frames.size(); ++i) {
        if (w.reported[i]) continue;
        const int32_t v = reinterpret_cast<volatile const int32_t*>(w.h_status)[i];
        if (v < 0 && !finished) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        const Admitted& a = w.frames[i];
        zotfs_completion c;
        std::memset(&c, 0, sizeof(c));
        c.tag = a.p.r.tag;
        c.status = (q == cudaSuccess || !finished) && v >= 0 ? v : ZOTFS_ECUDA;
        c.n_lists = a.p.r.n_rx * a.p.r.n_tx;
        c.arrival_ns = a.p.arrival_ns;
        c.admit_ns = a.admit_ns;
        c.done_ns = t;
        char* base = s->arena + a.off;
        c.bits = reinterpret_cast<const uint8_t*>(base + a.bits);
        c.llr = s->o.keep_llr ? reinterpret_cast<const float*>(base + a.llr) : nullptr;
        c.path_count = reinterpret_cast<const int32_t*>(base + a.pc);
        c.path_dk = reinterpret_cast<const int16_t*>(base + a.pdk);
        c.path_dl = reinterpret_cast<const int16_t*>(base + a.pdl);
        c.path_h = reinterpret_cast<const float*>(base + a.ph);
        s->live[c.tag] = std::make_pair(a.off, a.bytes);
        s->live_req[c.tag] = a.p.r;
        s->done.push_back(c);
        ++s->st.completed;
        w.reported[i] = 1;
        ++w.n_reported;
      }
      if (!finished) {
        any_busy = true;
        continue;
      }
      if (q != cudaSuccess) s->thread_error = cudaGetErrorString(q);
      w.frames.clear();
      w.busy = false;
    }
    if (s->stop && pending_total(s) == 0 && !any_busy) break;
    // admit pending frames into the free waves, each from its own queue
    bool launched = false;
    for (Wave& wv : s->waves) {
      if (wv.busy) continue;
      Wave* free_w = &wv;
      std::deque<Pending>& queue = s->pending[free_w->cls == 0 ? 0 : 1];
      if (queue.empty()) continue;
      const int64_t t = now_ns();
      while (!queue.empty() && (int)free_w->frames.size() < s->o.max_wave_frames) {
        Admitted a;
        a.p = queue.front();
        a.bytes = frame_bytes(s, a.p.r, &a);
        if (a.bytes > s->arena_bytes) {  // can never fit: fail the frame instead of blocking the queue
          zotfs_completion c;
          std::memset(&c, 0, sizeof(c));
          c.tag = a.p.r.tag;
          c.status = ZOTFS_ENOMEM;
          c.arrival_ns = a.p.arrival_ns;
          c.admit_ns = c.done_ns = t;
          s->done.push_back(c);
          ++s->st.rejected_too_large;
          ++s->st.completed;
          queue.pop_front();
          continue;
        }
        if (!arena_alloc(s, a.bytes, a.off)) break;  // wait for releases
        a.admit_ns = t;
        free_w->frames.push_back(a);
        queue.pop_front();
        ++s->st.admitted;
      }
      if (!free_w->frames.empty()) {
        free_w->busy = true;
        ++s->st.waves;
        const cudaError_t e = launch_wave(s, *free_w);
        if (e != cudaSuccess) s->thread_error = cudaGetErrorString(e);
        launched = true;
      }
    }
    if (!launched) {
      if (any_busy) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
      } else {
        s->cv.wait_for(lk, std::chrono::microseconds(200));
      }
    }
  }
}

void destroy_waves(zotfs_server_s* s) {
  for (Wave& w : s->waves) {
    if (w.main) cudaStreamSynchronize(w.main);
    if (w.h_desc) cudaFreeHost(w.h_desc);
    if (w.d_desc) cudaFree(w.d_desc);
    if (w.h_ids) cudaFreeHost(w.h_ids);
    if (w.d_ids) cudaFree(w.d_ids);
    if (w.d_counters) cudaFree(w.d_counters);
    if (w.h_status) cudaFreeHost(w.h_status);
    if (w.d_big) cudaFree(w.d_big);
    for (int i = 0; i < kWorkers; ++i) {
      if (w.work[i]) cudaStreamDestroy(w.work[i]);
      if (w.wdone[i]) cudaEventDestroy(w.wdone[i]);
    }
    if (w.main) cudaStreamDestroy(w.main);
    if (w.start) cudaEventDestroy(w.start);
    if (w.done) cudaEventDestroy(w.done);
  }
  s->waves.clear();
}

}  // namespace

extern "C" {

zotfs_status zotfs_server_create(const zotfs_server_opts* opts, zotfs_server* out) {
  g_launches = 0;
  if (!out || !opts) {
    set_error("NULL argument");
    return ZOTFS_EINVAL;
  }
  *out = nullptr;
  zotfs_server_opts o = *opts;
  if (o.p_max < 1 || o.p_max > 256 || o.max_wave_frames < 1 || o.max_wave_frames > 4096 ||
      o.waves_in_flight < 1 || o.waves_in_flight > 16 || o.arena_bytes < 4096 || !is_pow2(o.max_M) ||
      o.max_M < 16 || o.max_M > 256 || !is_pow2(o.max_N) || o.max_N < 8 || o.max_N > 64 || o.max_ant < 1 ||
      o.max_ant > 4 || o.light_work < 0) {
    set_error("zotfs_server_create: options out of range");
    return ZOTFS_EINVAL;
  }
  zotfs_server_s* s = new (std::nothrow) zotfs_server_s();
  if (!s) {
    set_error("host allocation failed");
    return ZOTFS_ENOMEM;
  }
  s->o = o;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device);
  zotfs_status st = ZOTFS_OK;
  // tables of every admissible shape; large-frame slot size of the largest shape that needs one
  for (int M = 16; M <= o.max_M && e == cudaSuccess && !st; M *= 2)
    for (int N = 8; N <= o.max_N && !st; N *= 2) {
      if (M * N > 16384) continue;
      float2 *W = nullptr, *T = nullptr;
      st = make_shape_tables(M, N, &W, &T);
      s->tables[std::make_pair(M, N)] = {W, T};
      FrameCfg fc;
      BigCfg bc;
      for (int nr = 1; nr <= o.max_ant && !st; ++nr)
        for (int nt = 1; nt <= o.max_ant; ++nt)
          if (!choose_frame_cfg(M, N, nr, nt, o.p_max, 0, fc)) {
            if (!choose_big_cfg(M, N, nr, nt, o.p_max, bc)) {
              set_error("zotfs_server_create: a shape up to max_M x max_N has no kernel");
              st = ZOTFS_EUNSUPPORTED;
              break;
            }
            s->big_slot_bytes = std::max(s->big_slot_bytes, bc.slot_bytes);
            BigClusterCfg bcc;
            if (nr * nt > 1 && choose_big_cluster_cfg(M, N, nr, nt, o.p_max, kServerCluster, bcc))
              s->big_slot_bytes = std::max(s->big_slot_bytes, bcc.slot_bytes);
          }
    }
  if (e != cudaSuccess && !st) st = cuda_fail(e, "server setup");
  s->big_slots = s->big_slot_bytes ? s->sm_count : 0;
  s->arena_bytes = (size_t)o.arena_bytes;
  if (!st) {
    e = dev_alloc(&s->arena, s->arena_bytes);
    if (e != cudaSuccess) st = cuda_fail(e, "server arena");
    else s->free_list[0] = s->arena_bytes;
  }
  s->waves.resize(o.waves_in_flight);
  s->split = o.light_work > 0 && o.waves_in_flight >= 2;
  if (s->split)  // the first half of the slots serve light frames
    for (int i = 0; i < o.waves_in_flight; ++i) s->waves[i].cls = i < o.waves_in_flight / 2 ? 0 : 1;
  // Light waves run on the device's highest-priority streams: when an SM frees up, their
  // waiting CTAs are placed before the heavy waves' (heavy CTAs run to the end of their frame;
  // nothing is preempted).
  int prio_least = 0, prio_greatest = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  for (Wave& w : s->waves) {
    if (st) break;
    const int n = o.max_wave_frames;
    e = host_alloc(&w.h_desc, sizeof(zotfs_frame_desc) * n, cudaHostAllocDefault);
    if (e == cudaSuccess) e = dev_alloc(&w.d_desc, sizeof(zotfs_frame_desc) * n);
    if (e == cudaSuccess) e = host_alloc(&w.h_ids, sizeof(int) * n, cudaHostAllocDefault);
    if (e == cudaSuccess) e = dev_alloc(&w.d_ids, sizeof(int) * n);
    if (e == cudaSuccess) e = dev_alloc(&w.d_counters, sizeof(int) * kMaxBuckets);
    if (e == cudaSuccess) e = host_alloc(&w.h_status, sizeof(int32_t) * n, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&w.d_status), w.h_status, 0);
    if (e == cudaSuccess && s->big_slots)
      e = dev_alloc(&w.d_big, s->big_slot_bytes * (size_t)s->big_slots);
    const int prio = w.cls == 0 ? prio_greatest : prio_least;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&w.main, cudaStreamNonBlocking, prio);
    for (int i = 0; i < kWorkers && e == cudaSuccess; ++i) {
      e = cudaStreamCreateWithPriority(&w.work[i], cudaStreamNonBlocking, prio);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.wdone[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) st = cuda_fail(e, "server wave resources");
  }
  s->st.arena_bytes = (int64_t)s->arena_bytes;
  if (st) {
    std::string msg = zotfs_last_error();
    destroy_waves(s);
    for (auto& kv : s->tables) {
      cudaFree(kv.second.first);
      cudaFree(kv.second.second);
    }
    if (s->arena) cudaFree(s->arena);
    delete s;
    set_error(msg);
    return st;
  }
  s->th = std::thread(scheduler, s);
  *out = s;
  return ZOTFS_OK;
}

zotfs_status zotfs_server_submit(zotfs_server s, const zotfs_request* reqs, int n) {
  if (!s || (n > 0 && !reqs) || n < 0) {
    set_error("zotfs_server_submit: bad arguments");
    return ZOTFS_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    zotfs_status v = validate_request(s, reqs[i]);
    if (v) return v;
  }
  const int64_t t = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      set_error("zotfs_server_submit: server is shutting down");
      return ZOTFS_EINVAL;
    }
    for (int i = 0; i < n; ++i) s->pending[frame_class(s, reqs[i])].push_back(Pending{reqs[i], t});
    s->st.submitted += n;
  }
  s->cv.notify_one();
  return ZOTFS_OK;
}

zotfs_status zotfs_server_replay(zotfs_server s, const zotfs_request* reqs, const double* arrival_s, int n) {
  if (!s || n < 0 || (n > 0 && (!reqs || !arrival_s))) {
    set_error("zotfs_server_replay: bad arguments");
    return ZOTFS_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    zotfs_status v = validate_request(s, reqs[i]);
    if (v) return v;
  }
  const int64_t t0 = now_ns();
  int i = 0;
  while (i < n) {
    const int64_t t = now_ns();
    int j = i;
    while (j < n && t0 + (int64_t)(arrival_s[j] * 1e9) <= t) ++j;
    if (j > i) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int q = i; q < j; ++q)
          s->pending[frame_class(s, reqs[q])].push_back(Pending{reqs[q], t0 + (int64_t)(arrival_s[q] * 1e9)});
        s->st.submitted += j - i;
      }
      s->cv.notify_one();
      i = j;
    }
  }
  return ZOTFS_OK;
}

int zotfs_server_poll(zotfs_server s, zotfs_completion* out, int max) {
  if (!s || !out || max <= 0) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

zotfs_status zotfs_server_release(zotfs_server s, uint64_t tag) {
  if (!s) {
    set_error("server is NULL");
    return ZOTFS_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(tag);
    if (it == s->live.end()) {
      set_error("zotfs_server_release: unknown or unfinished tag");
      return ZOTFS_EINVAL;
    }
    arena_free(s, it->second.first, it->second.second);
    s->live.erase(it);
    s->live_req.erase(tag);
    ++s->st.released;
  }
  s->cv.notify_one();
  return ZOTFS_OK;
}

zotfs_status zotfs_server_read(zotfs_server s, uint64_t tag, uint8_t* bits, float* llr, int32_t* path_count,
                               int16_t* path_dk, int16_t* path_dl, float* path_h) {
  if (!s) {
    set_error("server is NULL");
    return ZOTFS_EINVAL;
  }
  zotfs_request r;
  size_t off;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->live.find(tag);
    if (it == s->live.end()) {
      set_error("zotfs_server_read: unknown, unfinished or released tag");
      return ZOTFS_EINVAL;
    }
    off = it->second.first;
    r = s->live_req[tag];
  }
  Admitted a;
  frame_bytes(s, r, &a);
  const size_t MN = (size_t)r.M * r.N;
  const int bps = ilog2(r.qam), nl = r.n_rx * r.n_tx, pm = s->o.p_max;
  const char* base = s->arena + off;
  cudaError_t e = cudaSuccess;
  if (bits) e = cudaMemcpy(bits, base + a.bits, (size_t)r.n_tx * MN * bps / 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && llr) {
    if (!s->o.keep_llr) {
      set_error("zotfs_server_read: this server does not keep LLRs");
      return ZOTFS_EINVAL;
    }
    e = cudaMemcpy(llr, base + a.llr, (size_t)r.n_tx * MN * bps * sizeof(float), cudaMemcpyDeviceToHost);
  }
  if (e == cudaSuccess && path_count) e = cudaMemcpy(path_count, base + a.pc, (size_t)nl * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && path_dk) e = cudaMemcpy(path_dk, base + a.pdk, (size_t)nl * pm * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && path_dl) e = cudaMemcpy(path_dl, base + a.pdl, (size_t)nl * pm * 2, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && path_h) e = cudaMemcpy(path_h, base + a.ph, (size_t)nl * pm * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "zotfs_server_read");
  return ZOTFS_OK;
}

zotfs_status zotfs_server_get_stats(zotfs_server s, zotfs_server_stats* out) {
  if (!s || !out) {
    set_error("NULL argument");
    return ZOTFS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = (int64_t)pending_total(s);
  out->arena_in_use = (int64_t)s->in_use;
  out->arena_high_water = (int64_t)s->high_water;
  if (!s->thread_error.empty()) {
    set_error("scheduler: " + s->thread_error);
    return ZOTFS_ECUDA;
  }
  return ZOTFS_OK;
}

zotfs_status zotfs_server_destroy(zotfs_server s) {
  if (!s) return ZOTFS_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->pending[0].clear();
    s->pending[1].clear();
  }
  s->cv.notify_one();
  if (s->th.joinable()) s->th.join();
  destroy_waves(s);
  for (auto& kv : s->tables) {
    cudaFree(kv.second.first);
    cudaFree(kv.second.second);
  }
  if (s->arena) cudaFree(s->arena);
  delete s;
  return ZOTFS_OK;
}

}  // extern "C"
