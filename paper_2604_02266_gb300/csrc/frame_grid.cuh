// The receiver for paper-scale frames (M up to 16384, M N up to 524288: 4 MB per FP32
// vector), one frame at a time on the whole GPU.  A cooperative persistent kernel: its CTAs
// split every stage by delay columns (Zak transform tiles, operator gathers, CG updates,
// demapping) or by contiguous index ranges (read-off, bit packing) and meet at grid barriers.
// The frame's grid, the quasi-periodic extensions of p, t and c (row-major, as in the
// large-frame kernel) and the CG vectors live in global scratch that stays in L2 (about 58 MB
// at 16384 x 32).  In the CG each CTA owns a slab of delay columns over all rows; when every
// path's delay offset is within the launch's cap it gathers from shared-memory windows of the
// extensions (its columns and the offsets' reach on either side) with a per-CTA table of the
// paths' coefficients, and keeps p's window in shared memory across the iterations: three grid
// barriers per iteration.  The read-off happens inside the pilot's Zak transform: the taps
// that pass the threshold are appended as candidates and, after the transforms' barrier, every
// CTA selects the exact top-P_max (ties to the lowest q, list in ascending q) in shared memory;
// with too many candidates the threshold / stable-compaction / radix select runs over the
// grid with scans and histograms across the CTAs.  Algorithm 1's scalars are FP64 sums of per-CTA partials taken in CTA order, so
// every CTA derives the same alpha, beta and stopping decision.  SISO, separate pilot frames
// (or loaded lists), FP32.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoding is done through the runtime's driver entry point)

#include "frame_kernel.cuh"

namespace zotfs {

constexpr int kGridThreads = 256;
constexpr int kGridE = 8;         // most rows per work item (column k, rows j0 .. j0 + E - 1): sizes the scratch
constexpr int kGridDftCols = 32;  // delay columns per Zak-transform tile
constexpr uint32_t kGridMaxPolls = 1u << 22;

constexpr int kGridMaxCtas = 512;  // two CTAs per SM on up to 256 SMs
constexpr int kGridCandMax = 4096;  // passing taps the CTAs select among in shared memory

// Elements of one CG window (N + E + 3 rows of win_cols), rounded to 128 bytes.
__host__ __device__ __forceinline__ size_t grid_window_elems(int N, int win_cols) {
  return (((size_t)(N + kGridE + 3) * (size_t)win_cols * sizeof(float2) + 127) & ~size_t(127)) / sizeof(float2);
}

// A tap that passed the read-off threshold: its grid index, |h|^2 as an ordered bit pattern,
// and h.
struct GridCand {
  int q;
  uint32_t key;
  float2 h;
};
static_assert(sizeof(GridCand) == 16, "a candidate is read as one 16-byte vector");

// Delay columns per CTA in the CG stages (the last CTAs may hold fewer, or none).
// Even, so that the CTAs' column ranges start on 16-byte boundaries of the extensions' rows.
__host__ __device__ __forceinline__ int grid_cols_per_cta(int M, int grid) { return ((M + grid - 1) / grid + 1) & ~1; }

struct GridBarrier {
  unsigned long long count;  // CTA arrivals since the launch began (zeroed before each launch)
  int err;                   // a wait gave up: every CTA leaves at its next barrier
  int pad;
  int cand[2];               // read-off candidates appended, frames alternating (zeroed likewise)
  int pad2[2];
};

// The pilot read-off done inside the pilot's Zak transform: each output's h_eff (Eq.
// heff_hadamard) against the threshold, passing taps appended to cand (unordered) through the
// counter; beyond cap they are only counted.
struct GridReadoff {
  float scale, th2;
  GridCand* cand;
  int* counter;
  int cap;
};

// Global scratch of one grid receiver (one frame at a time).
struct GridScratch {
  float2* Y;                     // [MN] Zak-transformed grid (pilot, then data), q = l M + k
  float2* extP[2];               // extensions of p (row-major, ext_block_elems(M, N, 8)): the
                                 // iterations alternate, the previous p stays readable
  float2* extT;                  // extension of y, then of t = H p
  float2* extC;                  // extension of the residual c
  float2 *X, *Vv;                // [MN] the CG vectors x and a
  PathRecT<float>* list;         // [p_max] the frame's path list (read-offs with many taps)
  GridCand* cand;                // [kGridCandMax] the passing taps of a read-off (appended by
                                 // the pilot's transform; in ascending q on the ordered route)
  double* part;                  // [2 grid] per-CTA partial sums, two alternating sets
  int* icnt;                     // [2 grid] per-CTA counts of the read-off compaction
  int* hist;                     // [5 x 128] radix-select histograms (zeroed per frame)
  GridBarrier* bar;
  float2* ctab_g;                // [grid][p_max][cpc] the CG's coefficient tables when they do not
                                 // fit shared memory (large p_max at large M)
  // shared-memory windows of the CG gathers (set by the launch): columns per window row (0: no
  // windows) and the largest |dk| a window covers; tab_smem: the coefficient table in shared
  // memory (else ctab_g, and no windows)
  int win_cols, win_dcap, tab_smem;
};

// TMA descriptors of the extensions of c and t (row-major, rows N + E + 3 of 2 M 8-byte
// elements), with a box of the CG windows' size: win_cols columns by all rows.
struct GridMaps {
  CUtensorMap c, t;
};

// Rows of the extension and bytes of the scratch for one (M, N, p_max) at a given grid.
__host__ __device__ __forceinline__ size_t grid_scratch_bytes(int M, int N, int p_max, int grid) {
  const size_t MN = (size_t)M * N, ext = ext_block_elems(M, N, kGridE);
  size_t b = 0;
  auto take = [&](size_t n) { b += (n + 255) & ~size_t(255); };
  take(MN * 8);       // Y
  for (int i = 0; i < 4; ++i) take(ext * 8);  // extP[0], extP[1], extT, extC
  for (int i = 0; i < 2; ++i) take(MN * 8);   // X, Vv
  take((size_t)p_max * sizeof(PathRecT<float>));
  take((size_t)kGridCandMax * sizeof(GridCand));
  take((size_t)grid * 16);
  take((size_t)grid * 8);
  take(5 * 128 * 4);
  take(sizeof(GridBarrier));
  take((size_t)grid * grid_cols_per_cta(M, grid) * p_max * sizeof(float2));  // ctab_g
  return b;
}

__host__ __device__ __forceinline__ GridScratch grid_scratch_carve(char* base, int M, int N, int p_max, int grid) {
  const size_t MN = (size_t)M * N, ext = ext_block_elems(M, N, kGridE);
  GridScratch G;
  size_t off = 0;
  auto take = [&](size_t n) {
    char* p = base + off;
    off += (n + 255) & ~size_t(255);
    return p;
  };
  G.Y = reinterpret_cast<float2*>(take(MN * 8));
  G.extP[0] = reinterpret_cast<float2*>(take(ext * 8));
  G.extP[1] = reinterpret_cast<float2*>(take(ext * 8));
  G.extT = reinterpret_cast<float2*>(take(ext * 8));
  G.extC = reinterpret_cast<float2*>(take(ext * 8));
  G.X = reinterpret_cast<float2*>(take(MN * 8));
  G.Vv = reinterpret_cast<float2*>(take(MN * 8));
  G.list = reinterpret_cast<PathRecT<float>*>(take((size_t)p_max * sizeof(PathRecT<float>)));
  G.cand = reinterpret_cast<GridCand*>(take((size_t)kGridCandMax * sizeof(GridCand)));
  G.part = reinterpret_cast<double*>(take((size_t)grid * 16));
  G.icnt = reinterpret_cast<int*>(take((size_t)grid * 8));
  G.hist = reinterpret_cast<int*>(take(5 * 128 * 4));
  G.bar = reinterpret_cast<GridBarrier*>(take(sizeof(GridBarrier)));
  G.ctab_g = reinterpret_cast<float2*>(take((size_t)grid * grid_cols_per_cta(M, grid) * p_max * sizeof(float2)));
  G.win_cols = 0;
  G.win_dcap = -1;
  G.tab_smem = 1;
  return G;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_gpu_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Barrier over all CTAs of the cooperative grid (co-resident by construction of the launch).
// The arrival counter only grows: barrier g (0-based, counted per thread in `gen`) is complete
// once it holds (g + 1) gridDim.x arrivals, so an arriving CTA adds one with a release
// reduction (no round trip, no reset by a last arriver) and polls with acquire loads.
// Returns false in every thread of the CTA when this wait or an earlier one gave up (bounded
// polls): the caller abandons the frame.
__device__ __forceinline__ bool grid_sync(GridBarrier* b, unsigned& gen, uint32_t max_polls = kGridMaxPolls) {
  __syncthreads();
  const unsigned g = gen;
  gen = g + 1;
  int ok = 1;
  if (threadIdx.x == 0) {
    if (*reinterpret_cast<volatile int*>(&b->err) != 0) {
      ok = 0;
    } else {
      red_release_gpu_add(&b->count, 1ull);
      const unsigned long long target = (unsigned long long)(g + 1) * gridDim.x;
      uint32_t polls = 0;
      while (ld_acquire_gpu_u64(&b->count) < target) {
        if (++polls > max_polls) {
          atomicExch(&b->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
      __threadfence();
    }
  }
  return __syncthreads_and(ok) != 0;
}

// Store DD value v of (delay k, Doppler l) into a row-major quasi-periodic extension (element
// (A, r) at r 2M + A + M/2, rows N + E + 3): the main column, the halo column with its
// quasi-periodic phase W_N^{+-l} (from wn[l] = W_N^{-l} in shared memory), and the periodic
// halo rows.
template <int E>
__device__ __forceinline__ void ext_store_rm(float2* ext, const FrameArgs& A, int k, int l, float2 v, const float2* wn) {
  const int M = A.M, N = A.N, Hk = M >> 1;
  const bool low = k < Hk;
  const int mc = k + Hk, hc = (low ? k + M : k - M) + Hk;
  const float2 w = wn[l];
  const float2 hv = cmul(v, low ? conjf2(w) : w);
  for (int r = l; r < N + E + 3; r += N) {
    ext[(size_t)r * 2 * M + mc] = v;
    ext[(size_t)r * 2 * M + hc] = hv;
  }
}

// Store the E values of item (column k, rows j0 .. j0 + E - 1) into a row-major quasi-periodic
// extension: the main column and the periodic halo rows always, the halo column (with its
// quasi-periodic phase W_N^{+-l}, from wn[l] = W_N^{-l} in shared memory) when `halo` -- the
// windowed gathers read halo columns only within a few delays of the wrap, the global gathers
// anywhere.
template <int E>
__device__ __forceinline__ void grid_ext_store(float2* ext, const FrameArgs& A, int k, int j0, const float2 (&v)[E],
                                               bool halo, const float2* wn) {
  const int M = A.M, N = A.N, Hk = M >> 1, R = N + E + 3;
  const size_t RS = (size_t)(2 * M);
  const bool low = k < Hk;
  float2* mcol = ext + (k + Hk);
  float2* hcol = ext + ((low ? k + M : k - M) + Hk);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int l = j0 + i;
    for (int r = l; r < R; r += N) mcol[r * RS] = v[i];
    if (halo) {
      const float2 w = wn[l];
      const float2 hv = cmul(v[i], low ? conjf2(w) : w);
      for (int r = l; r < R; r += N) hcol[r * RS] = hv;
    }
  }
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// A bulk copy that completes on `bar` without arriving on it (the expected bytes were armed once).
__device__ __forceinline__ void bulk_g2s_tx(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Copy the box of the CG windows -- columns [A0, A0 + win_cols) of all rows of a row-major
// extension -- into the shared-memory window dst (row-major, rows win_cols elements apart) by
// one tiled bulk tensor copy, issued by thread 0 after arming the barrier with the box's bytes.
// A0 is even, so the copy's inner coordinate A0 + M/2 is a multiple of 16 bytes; columns past
// the extension read as zeros.  The extension was written by other CTAs before the grid barrier
// this CTA passed (generic stores): the issuing thread orders them before the async read with a
// proxy fence.  All threads call (`active` false: no copy); false, uniformly, if the bounded
// wait gave up.
__device__ __forceinline__ bool grid_window_load(float2* dst, const CUtensorMap* map, int M, int A0,
                                                 uint32_t box_bytes, bool active, uint64_t* bar, uint32_t& phase) {
  __syncthreads();  // earlier generic accesses to the window are complete
  bool ok = true;
  if (active) {
    if (threadIdx.x == 0) {
      fence_proxy_async_smem();
      asm volatile("fence.proxy.async.global;" ::: "memory");
      mbar_arrive_expect_tx(bar, box_bytes);
      const int x = A0 + (M >> 1), y = 0;
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              smem_u32(dst)),
          "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
          : "memory");
    }
    ok = mbar_wait_bounded(bar, phase, kMaxPolls);
    if (!ok) ok = mbar_wait_bounded(bar, phase, kMaxPolls);  // let an in-flight copy land
    phase ^= 1u;
  }
  return __syncthreads_and(ok) != 0;
}

// Y[l M + k] = N^-1/2 sum_n y[k + n M] W_N^{-n l} (Eq. zak) for all columns: tiles of
// kGridDftCols columns over all N rows staged in shared memory (coalesced along k), an
// in-place radix-2 decimation-in-frequency FFT along n per column (log2 N stages of N/2
// butterflies), and the outputs read back from bit-reversed rows.  The result goes to Y
// (q = l M + k) and/or straight into a row-major quasi-periodic extension `ext` (E rows per
// item), either may be NULL.  `tile` holds N kGridDftCols values, `wn` N twiddles.
template <int E>
__device__ __forceinline__ void grid_dzt(const char* src, int dtype, float2* Y, float2* ext, const FrameArgs& A,
                                         float2* tile, float2* wn, const GridReadoff* ro = nullptr) {
  const int M = A.M, N = A.N, logM = A.logM, logN = A.logN, MN = M * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) wn[i] = conjf2(tw<float>(A, (size_t)i << logM));
  const float s = (float)A.inv_sqrtN;
  const int ntiles = M / kGridDftCols;
  __syncthreads();
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int k0 = t * kGridDftCols;
    for (int e = threadIdx.x; e < N * kGridDftCols; e += blockDim.x) {
      const int n = e / kGridDftCols, kk = e - n * kGridDftCols;
      tile[e] = load_complex<float2>(src, (size_t)n * M + k0 + kk, dtype);
    }
    __syncthreads();
    for (int h = N >> 1; h >= 1; h >>= 1) {
      const int tws = N / (2 * h);
      for (int b = threadIdx.x; b < (N >> 1) * kGridDftCols; b += blockDim.x) {
        const int kk = b & (kGridDftCols - 1), g = b / kGridDftCols;
        const int gi = g & (h - 1);
        const int n = ((g - gi) << 1) + gi;
        float2* p0 = tile + n * kGridDftCols + kk;
        const float2 u = p0[0], v = p0[h * kGridDftCols];
        p0[0] = cadd(u, v);
        p0[h * kGridDftCols] = cmul(csub(u, v), wn[gi * tws]);
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < N * kGridDftCols; e += blockDim.x) {
      const int l = e / kGridDftCols, kk = e - l * kGridDftCols;
      const float2 v = cscale(tile[bitrev(l, logN) * kGridDftCols + kk], s);
      if (Y) Y[(size_t)l * M + k0 + kk] = v;
      if (ext) ext_store_rm<E>(ext, A, k0 + kk, l, v, wn);
      if (ro) {  // every lane of a warp runs the same number of elements
        const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
        const float2 h = cscale(cmul(v, tw<float>(A, (size_t)((-A.K0 * dl) & (MN - 1)))), ro->scale);
        const float m2 = h.x * h.x + h.y * h.y;
        const bool pass = m2 > ro->th2;
        const unsigned mask = __ballot_sync(0xffffffffu, pass);
        if (mask) {
          const int lane = threadIdx.x & 31, first = __ffs(mask) - 1;
          int base = 0;
          if (lane == first) base = atomicAdd(ro->counter, __popc(mask));
          base = __shfl_sync(0xffffffffu, base, first);
          const int pos = base + __popc(mask & ((1u << lane) - 1u));
          if (pass && pos < ro->cap) {
            GridCand c;
            c.q = l * M + k0 + kk;
            c.key = __float_as_uint(m2);
            c.h = h;
            ro->cand[pos] = c;
          }
        }
      }
    }
    __syncthreads();
  }
}

// Sum of the CTAs' partials (each CTA's thread 0 stored part[blockIdx.x] before the barrier),
// by warp 0 in a fixed order -- lane j loads CTAs j, j + 32, ..., j + 32 (kGridMaxCtas / 32 - 1)
// (zero past the grid) and adds them pairwise (a tree of depth 5 instead of a chain of up to
// 32 dependent FP64 additions, which cost ~56 cycles each on this part), then a butterfly over
// the lanes -- so every CTA gets the same value; valid in thread 0.  Consecutive reductions
// alternate between two sets of partials (part and part + gridDim.x): a CTA that has summed
// one set may store into the other while a slower CTA is still summing the first.
__device__ __forceinline__ double grid_partials(const double* part) {
  double s = 0.0;
  if (threadIdx.x < 32) {
    constexpr int kPer = kGridMaxCtas / 32;
    double v[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
      const int b = (int)threadIdx.x + 32 * i;
      v[i] = b < (int)gridDim.x ? __ldcg(part + b) : 0.0;
    }
#pragma unroll
    for (int w = 1; w < kPer; w <<= 1)
#pragma unroll
      for (int i = 0; i + w < kPer; i += 2 * w) v[i] += v[i + w];
    s = warp_sum_f64(v[0]);
  }
  return s;
}

// This CTA's exclusive prefix and the grid total of one count per CTA, by warp 0; stored in
// S->isc[2] (prefix) and S->isc[3] (total).
__device__ __forceinline__ void grid_prefix(const int* counts, SharedHdr* S) {
  if (threadIdx.x < 32) {
    int pre = 0, tot = 0;
#pragma unroll 4
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
      const int c = __ldcg(counts + b);
      tot += c;
      if (b < (int)blockIdx.x) pre += c;
    }
    pre = warp_sum_i(pre);
    tot = warp_sum_i(tot);
    if (threadIdx.x == 0) {
      S->isc[2] = pre;
      S->isc[3] = tot;
    }
  }
  __syncthreads();
}

// hist[bin] += 1 for every lane with `active`, one atomic per distinct counter of the warp (the
// read-off's magnitudes crowd into a few bins, where one atomic per tap serialises).  Every
// thread of the block calls (a warp may hold threads of two rows of a 2D block, each row with
// its own histogram: lanes group by the counter's address).
__device__ __forceinline__ void warp_hist_add(int* hist, unsigned bin, bool active) {
  const unsigned lin = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
  const unsigned base = lin & ~31u, lanes = nthr - base < 32u ? nthr - base : 32u;
  const unsigned mask = lanes == 32u ? 0xffffffffu : (1u << lanes) - 1u;
  const unsigned lane = lin & 31u;
  const unsigned key = active ? (unsigned)reinterpret_cast<uintptr_t>(hist + bin) : 0xffffffffu;
  const unsigned peers = __match_any_sync(mask, key);
  if (active && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&hist[bin], __popc(peers));
}

// The path list from the n <= kGridCandMax passing taps in cand (ascending q): all of them, or
// when n > K the exact K largest |h|^2, ties to the lower q (the same list the grid-wide
// selection gives), into out[0, P) in ascending q (Eq. heff_thres with the p_max cap).  Every
// CTA computes it alike from the same candidates: thread t holds candidates [t CPT, t CPT + CPT),
// a radix select of 7 bits per pass finds the K-th largest key from block histograms, and one
// block scan places the kept taps.  With gout (one CTA) the list is also stored there.
// All threads call; returns P and sets trunc.
template <int CPT>
__device__ __forceinline__ int grid_select(const GridCand* cand, int n, const FrameArgs& A, PathRecT<float>* out,
                                           SharedHdr* S, const PathIO* gout, int& trunc) {
  const int tid = threadIdx.x, K = A.p_max;
  const int M = A.M, N = A.N;
  const int b0 = tid * CPT;
  uint32_t key[CPT];
  uint32_t have = 0;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    key[j] = 0;
    if (b0 + j < n) {
      key[j] = __ldcg(&cand[b0 + j].key);
      have |= 1u << j;
    }
  }
  uint32_t keep = have;
  int total = n, base = b0;
  trunc = 0;
  if (n > K) {
    trunc = 1;
    uint32_t prefix = 0, fixed = 0;
    int kleft = K;  // rank of the wanted key among the candidates that match `prefix`
    const int lane = tid & 31;
    for (int b = tid; b < 128; b += blockDim.x) S->hist[b] = 0;
    __syncthreads();
    for (int hb = 31; hb > 0; hb -= 7) {
      const int w = hb < 7 ? hb : 7, sh = hb - w;
#pragma unroll
      for (int j = 0; j < CPT; ++j)
        warp_hist_add(S->hist, (key[j] >> sh) & 127u, ((have >> j) & 1u) && ((key[j] ^ prefix) & fixed) == 0);
      __syncthreads();
      if (tid < 32) {  // the bin holding the kleft-th largest, from the top (lane: 4 bins)
        int c[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          c[j] = S->hist[4 * lane + j];
          S->hist[4 * lane + j] = 0;
          sum += c[j];
        }
        int suf = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_down_sync(0xffffffffu, suf, o);
          if (lane + o < 32) suf += v;
        }
        int acc = suf - sum;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
          if (acc < kleft && acc + c[j] >= kleft) {
            S->isc[2] = 4 * lane + j;
            S->isc[3] = kleft - acc;
          }
          acc += c[j];
        }
      }
      __syncthreads();
      prefix |= (uint32_t)S->isc[2] << sh;
      kleft = S->isc[3];
      fixed |= ((1u << w) - 1u) << sh;
      __syncthreads();
    }
    const uint32_t vK = prefix;  // the K-th largest key
    const int need = kleft;      // keys equal to vK that are kept: the first `need` in ascending q
    uint32_t gt = 0, eq = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if ((have >> j) & 1u) {
        if (key[j] > vK) gt |= 1u << j;
        else if (key[j] == vK) eq |= 1u << j;
      }
    int both_total;
    const int both = block_exclusive_scan((__popc(gt) << 16) | __popc(eq), S->scan, both_total);
    (void)both_total;
    int eq_before = both & 0xffff;
    base = (both >> 16) + min(eq_before, need);
    keep = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      if ((gt >> j) & 1u) {
        keep |= 1u << j;
      } else if ((eq >> j) & 1u) {
        if (eq_before < need) keep |= 1u << j;
        ++eq_before;
      }
    }
    total = K;
  }
  int pos = base;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    if ((keep >> j) & 1u) {
      const GridCand c = cand[b0 + j];
      const int k = c.q & (M - 1), l = c.q >> A.logM;
      const int dk = ((k - A.K0 + (M >> 1)) & (M - 1)) - (M >> 1);
      const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
      PathRecT<float> rec;  // hf unused: the grid CG forms its factors from a table and phases
      rec.h = c.h;
      rec.dk = dk;
      rec.dl = dl;
      rec.hf = make_float2(0.f, 0.f);
      rec.pad0 = rec.pad1 = 0;
      out[pos] = rec;
      if (gout) {
        gout->dk[pos] = (int16_t)dk;
        gout->dl[pos] = (int16_t)dl;
        store_complex(gout->h, (size_t)pos, gout->tap_dtype, c.h);
      }
      ++pos;
    }
  }
  if (gout && tid == 0) {
    gout->count[0] = total;
    if (gout->status) gout->status[0] = trunc ? ZOTFS_ETRUNCATED : ZOTFS_OK;
  }
  __syncthreads();
  return total;
}

// As grid_select, for candidates in any order (appended by the pilot's transform): the same
// radix select gives the K-th largest key; the ties to it that are kept are those of the lowest
// q (each tie ranked by q among all ties, through tq: room for tie_cap indices), and the kept
// taps are placed in ascending q by ranking each against the others (kq, kh: room for K).
// Returns P, or -1 (uniformly) when more than tie_cap taps tie with the K-th largest -- the
// caller then takes the ordered route.
template <int CPT>
__device__ __forceinline__ int grid_select_q(const GridCand* cand, int n, const FrameArgs& A, PathRecT<float>* out,
                                             SharedHdr* S, const PathIO* gout, int* tq, int tie_cap, int* kq,
                                             float2* kh, int* whist, int nh, int& trunc) {
  const int tid = threadIdx.x, K = A.p_max;
  const int M = A.M, N = A.N;
  const int nw = nh, warp = (tid >> 5) % nh;  // nh histograms, warps sharing them round-robin
  // thread t holds candidates t + j blockDim (whole records, coalesced)
  uint32_t key[CPT];
  int qv[CPT];
  uint32_t have = 0;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int i = tid + j * kGridThreads;
    key[j] = 0;
    qv[j] = 0;
    if (i < n) {
      const int2 qk = __ldcg(reinterpret_cast<const int2*>(cand + i));  // q and key
      qv[j] = qk.x;
      key[j] = (uint32_t)qk.y;
      have |= 1u << j;
    }
  }
  uint32_t keep = have;
  int total = n;
  trunc = 0;
  if (n > K) {
    trunc = 1;
    uint32_t prefix = 0, fixed = 0;
    int kleft = K;
    const int lane = tid & 31;
    // 128-bin histograms, one per warp when nh covers the warps, so their increments do not contend
    for (int b = tid; b < 128 * nw; b += blockDim.x) whist[b] = 0;
    __syncthreads();
    for (int hb = 31; hb > 0; hb -= 7) {
      const int w = hb < 7 ? hb : 7, sh = hb - w;
#pragma unroll
      for (int j = 0; j < CPT; ++j)
        warp_hist_add(whist + 128 * warp, (key[j] >> sh) & 127u,
                      ((have >> j) & 1u) && ((key[j] ^ prefix) & fixed) == 0);
      __syncthreads();
      if (tid < 32) {
        int c[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          c[j] = 0;
          for (int u = 0; u < nw; ++u) {
            c[j] += whist[128 * u + 4 * lane + j];
            whist[128 * u + 4 * lane + j] = 0;
          }
          sum += c[j];
        }
        int suf = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_down_sync(0xffffffffu, suf, o);
          if (lane + o < 32) suf += v;
        }
        int acc = suf - sum;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
          if (acc < kleft && acc + c[j] >= kleft) {
            S->isc[2] = 4 * lane + j;
            S->isc[3] = kleft - acc;
            S->isc[0] = c[j];  // taps in that bin
          }
          acc += c[j];
        }
      }
      __syncthreads();
      prefix |= (uint32_t)S->isc[2] << sh;
      kleft = S->isc[3];
      fixed |= ((1u << w) - 1u) << sh;
      const int in_bin = S->isc[0];
      __syncthreads();
      if (sh > 0 && in_bin <= min(256, tie_cap)) {
        // Few taps share the bits fixed so far: rank them against each other directly (the
        // kleft-th largest among them is the K-th largest of all) instead of further passes.
        uint32_t match = 0;
#pragma unroll
        for (int j = 0; j < CPT; ++j)
          if (((have >> j) & 1u) && ((key[j] ^ prefix) & fixed) == 0) match |= 1u << j;
        int nm;
        int mpos = block_exclusive_scan(__popc(match), S->scan, nm);
        uint32_t* mk = reinterpret_cast<uint32_t*>(tq);
#pragma unroll
        for (int j = 0; j < CPT; ++j)
          if ((match >> j) & 1u) mk[mpos++] = key[j];
        __syncthreads();
        for (int i = tid; i < nm; i += blockDim.x) {
          const uint32_t x = mk[i];
          int gtc = 0, gec = 0;
          for (int t = 0; t < nm; ++t) {
            gtc += mk[t] > x;
            gec += mk[t] >= x;
          }
          if (gtc < kleft && kleft <= gec) {  // every writer stores the same pair
            S->isc[2] = (int)x;
            S->isc[3] = kleft - gtc;
          }
        }
        __syncthreads();
        prefix = (uint32_t)S->isc[2];
        kleft = S->isc[3];
        __syncthreads();
        break;
      }
    }
    const uint32_t vK = prefix;  // the K-th largest key (all 31 bits fixed, by passes or ranking)
    const int need = kleft;      // keys equal to vK that are kept
    uint32_t gt = 0, eq = 0;
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if ((have >> j) & 1u) {
        if (key[j] > vK) gt |= 1u << j;
        else if (key[j] == vK) eq |= 1u << j;
      }
    // the ties' indices, compacted, then each tie kept when fewer than `need` ties have a lower q
    int nties;
    int tpos = block_exclusive_scan(__popc(eq), S->scan, nties);
    if (nties > tie_cap) return -1;
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if ((eq >> j) & 1u) tq[tpos++] = qv[j];
    __syncthreads();
    keep = gt;
#pragma unroll
    for (int j = 0; j < CPT; ++j)
      if ((eq >> j) & 1u) {
        int r = 0;
        for (int t = 0; t < nties; ++t) r += tq[t] < qv[j];
        if (r < need) keep |= 1u << j;
      }
    total = K;
  }
  // the kept taps, compacted in any order, then each placed at its rank in q
  int nk;
  int kpos = block_exclusive_scan(__popc(keep), S->scan, nk);
#pragma unroll
  for (int j = 0; j < CPT; ++j)
    if ((keep >> j) & 1u) {
      kq[kpos] = qv[j];
      kh[kpos] = __ldcg(&cand[tid + j * kGridThreads].h);
      ++kpos;
    }
  __syncthreads();
  for (int i = tid; i < nk; i += blockDim.x) {
    const int q = kq[i];
    int r = 0;
    for (int t = 0; t < nk; ++t) r += kq[t] < q;
    const int k = q & (M - 1), l = q >> A.logM;
    const int dk = ((k - A.K0 + (M >> 1)) & (M - 1)) - (M >> 1);
    const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
    PathRecT<float> rec;  // hf unused: the grid CG forms its factors from a table and phases
    rec.h = kh[i];
    rec.dk = dk;
    rec.dl = dl;
    rec.hf = make_float2(0.f, 0.f);
    rec.pad0 = rec.pad1 = 0;
    out[r] = rec;
    if (gout) {
      gout->dk[r] = (int16_t)dk;
      gout->dl[r] = (int16_t)dl;
      store_complex(gout->h, (size_t)r, gout->tap_dtype, rec.h);
    }
  }
  if (gout && tid == 0) {
    gout->count[0] = total;
    if (gout->status) gout->status[0] = trunc ? ZOTFS_ETRUNCATED : ZOTFS_OK;
  }
  __syncthreads();
  return total;
}

// EQ: pilot-grid entries per thread in the read-off; E: rows per CG work item (column k, rows
// j0 .. j0 + E - 1); MINB: CTAs per SM the launch bounds are set for.
template <int EQ, int E, int MINB>
__global__ void __launch_bounds__(kGridThreads, MINB)
    grid_kernel(const __grid_constant__ FrameArgs A, GridScratch G, const __grid_constant__ GridMaps maps) {
  using R = float;
  using C = float2;
  using PathRec = PathRecT<R>;
  extern __shared__ __align__(128) unsigned char smem[];
  SharedHdr* S = reinterpret_cast<SharedHdr*>(smem);
  size_t off = (sizeof(SharedHdr) + 127) & ~size_t(127);
  PathRec* paths = reinterpret_cast<PathRec*>(smem + off);
  int* cnt = reinterpret_cast<int*>(paths + A.p_max);
  int* nruns = cnt + 1;
  off += ((size_t)A.p_max * sizeof(PathRec) + sizeof(int) * 2 + 127) & ~size_t(127);
  RunRec* runs = reinterpret_cast<RunRec*>(smem + off);
  off += ((size_t)A.p_max * sizeof(RunRec) + 127) & ~size_t(127);
  PathRec* sort_tmp = reinterpret_cast<PathRec*>(smem + off);
  off += ((size_t)A.p_max * sizeof(PathRec) + 127) & ~size_t(127);
  int* sort_keys = reinterpret_cast<int*>(smem + off);
  off += ((size_t)((A.p_max + 3) & ~3) * sizeof(int) + 127) & ~size_t(127);
  C* tile = reinterpret_cast<C*>(smem + off);
  off += (size_t)A.N * kGridDftCols * sizeof(C);
  C* wn = reinterpret_cast<C*>(smem + off);
  off += ((size_t)A.N * sizeof(C) + 127) & ~size_t(127);
  // the CG's coefficient table (p_max rows of the CTA's columns) with the paths' forward
  // phases, and windows (p and c / t: N + E + 3 rows of G.win_cols columns each)
  C* ctab = reinterpret_cast<C*>(smem + off);
  off += ((size_t)A.p_max * (G.tab_smem ? grid_cols_per_cta(A.M, (int)gridDim.x) : 0) * sizeof(C) + 127) &
         ~size_t(127);
  C* phi = reinterpret_cast<C*>(smem + off);
  off += ((size_t)A.p_max * sizeof(C) + 127) & ~size_t(127);
  C* bufP = reinterpret_cast<C*>(smem + off);
  C* bufX = bufP + grid_window_elems(A.N, G.win_cols);  // both 128-byte aligned, as the tensor copy needs

  const int M = A.M, N = A.N, MN = M * N, logM = A.logM, tid = threadIdx.x;
  const int gtid = blockIdx.x * blockDim.x + tid, nthr = gridDim.x * blockDim.x;
  const int items = MN / E;  // (column k, row group j0 / E), k fastest
  // CG work items are split evenly over the CTAs in contiguous ranges (consecutive columns,
  // coalesced): every SM then carries the same number of items, so no grid barrier waits for
  // SMs that hold twice the work of others
  const int ipc = (items + (int)gridDim.x - 1) / (int)gridDim.x;
  const int it_beg = min(items, (int)blockIdx.x * ipc), it_end = min(items, it_beg + ipc);
  // read-off: pilot-grid entries likewise, EQ consecutive q per thread, ranges in CTA order
  const int qpc = ((MN + (int)gridDim.x - 1) / (int)gridDim.x + EQ - 1) / EQ * EQ;
  const int q_beg = min(MN, (int)blockIdx.x * qpc), q_end = min(MN, q_beg + qpc);
  const size_t blk = ext_block_elems(M, N, E);
  const bool write_paths = (A.mode & kWritePaths) != 0;
  unsigned gen = 0;  // barriers passed
  uint32_t mph = 0;  // phase of the window barrier
  auto fail = [&](const FrameIO& io) {
    if (tid == 0 && io.status) *io.status = ZOTFS_ETIMEOUT;
  };
  if (tid == 0) mbar_init(&S->mbar, 1);
  __syncthreads();

  for (int f = 0; f < A.n_frames; ++f) {
    const FrameIO io = frame_io(A, f, (int)sizeof(C));
    int st = 0;
    if (blockIdx.x == 0)
      for (int i = tid; i < 5 * 128; i += blockDim.x) G.hist[i] = 0;

    // ------------------------------------------------ Zak transform only
    if (A.mode & kDzt) {
      grid_dzt<E>(io.y_data, A.in_dtype, reinterpret_cast<C*>(io.u_out), nullptr, A, tile, wn);
      if (!grid_sync(G.bar, gen)) return fail(io);
      if (blockIdx.x == 0 && tid == 0 && io.status) *io.status = ZOTFS_OK;
      continue;
    }

    // ------------------------------------------------ path list
    int P = 0;
    // the data frame's Zak transform goes with the pilot's when both run (no barrier of its own;
    // the read-off's barriers publish it): it writes the extension of y directly
    const bool y_early = (A.mode & kEstimate) && (A.mode & kCG) && !A.y_is_dd;
    if (A.mode & kEstimate) {
      // The pilot's transform reads the taps off as it writes them (Eq. heff_hadamard against the
      // threshold) and appends those that pass as candidates; after the one barrier every CTA
      // selects the list from them in shared memory.  When more taps pass than the candidates
      // hold, or too many tie with the p_max-th largest, the ordered route below runs from the
      // transformed grid Y.
      const R scale = (R)(1.0 / io.a_pilot);
      const R th2 = (R)io.theta * (R)io.theta;
      const GridReadoff ro{scale, th2, G.cand, &G.bar->cand[f & 1], kGridCandMax};
      grid_dzt<E>(io.y_pilot, A.in_dtype, G.Y, nullptr, A, tile, wn, &ro);
      if (y_early) grid_dzt<E>(io.y_data, A.in_dtype, nullptr, G.extT, A, tile, wn);
      if (!grid_sync(G.bar, gen)) return fail(io);
      if (blockIdx.x == 0 && tid == 0) G.bar->cand[(f + 1) & 1] = 0;  // the next frame's count
      const int ncand = *reinterpret_cast<volatile int*>(&G.bar->cand[f & 1]);
      P = -1;
      if (ncand <= kGridCandMax) {
        const PathIO* gout = (write_paths && io.paths.count && blockIdx.x == 0) ? &io.paths : nullptr;
        int trunc = 0;
        // scratch: the transform's tile for the ties' indices, the sort buffer for the kept taps
        float2* kh = reinterpret_cast<float2*>(sort_tmp);
        int* kq = reinterpret_cast<int*>(kh + A.p_max);
        // per-warp histograms in the (still unused) p window when it has room, else the header's
        const bool wh = (size_t)G.win_cols * (N + E + 3) * sizeof(C) >= (size_t)kGridThreads / 32 * 128 * sizeof(int);
        P = grid_select_q<kGridCandMax / kGridThreads>(G.cand, ncand, A, paths, S, gout,
                                                        reinterpret_cast<int*>(tile), 64 * N, kq, kh,
                                                        wh ? reinterpret_cast<int*>(bufP) : S->hist,
                                                        wh ? kGridThreads / 32 : 1, trunc);
        if (P >= 0 && trunc) st |= kStTrunc;
      }
      if (P < 0) {
        C hv[EQ];
        uint32_t mb[EQ];
        uint32_t pass = 0;
  #pragma unroll
        for (int i = 0; i < EQ; ++i) {
          const int q = q_beg + tid * EQ + i;
          hv[i] = make_float2(0.f, 0.f);
          mb[i] = 0;
          if (q < q_end) {
            const int l = q >> logM;
            const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
            const C h = cscale(cmul(G.Y[q], tw<R>(A, (size_t)((-A.K0 * dl) & (MN - 1)))), scale);
            const R m2 = h.x * h.x + h.y * h.y;
            hv[i] = h;
            mb[i] = __float_as_uint(m2);
            if (m2 > th2) pass |= 1u << i;
          }
        }
        int blk_total;
        const int in_blk = block_exclusive_scan(__popc(pass), S->scan, blk_total);
        if (tid == 0) G.icnt[blockIdx.x] = blk_total;
        if (!grid_sync(G.bar, gen)) return fail(io);
        grid_prefix(G.icnt, S);
        int total = S->isc[3];
        int base = S->isc[2] + in_blk;
        if (total <= kGridCandMax) {
          // The passing taps as candidates at their places in ascending q; then every CTA selects
          // the list from them alike in shared memory: one grid barrier instead of the grid-wide
          // radix select's and the list's.
          int pos = base;
  #pragma unroll
          for (int i = 0; i < EQ; ++i)
            if ((pass >> i) & 1u) {
              GridCand c;
              c.q = q_beg + tid * EQ + i;
              c.key = mb[i];
              c.h = hv[i];
              G.cand[pos++] = c;
            }
          if (!grid_sync(G.bar, gen)) return fail(io);
          const PathIO* gout = (write_paths && io.paths.count && blockIdx.x == 0) ? &io.paths : nullptr;
          int trunc = 0;
          P = grid_select<kGridCandMax / kGridThreads>(G.cand, total, A, paths, S, gout, trunc);
          if (trunc) st |= kStTrunc;
        } else {
          uint32_t keep = pass;
          int trunc = 0;
          if (total > A.p_max) {
            // the K-th largest |h|^2 among the passing taps, exactly: radix select on the bit
            // patterns, 7 bits per pass, histograms over the whole grid
            trunc = 1;
            const int K = A.p_max;
            uint32_t prefix = 0, fixed = 0;
            int kleft = K;
            int hp = 0;
            for (int hb = 31; hb > 0; hb -= 7, ++hp) {
              const int w = hb < 7 ? hb : 7, sh = hb - w;
              int* H = G.hist + hp * 128;
#pragma unroll
              for (int i = 0; i < EQ; ++i)
                warp_hist_add(H, (mb[i] >> sh) & 127u, ((pass >> i) & 1u) && ((mb[i] ^ prefix) & fixed) == 0);
              if (!grid_sync(G.bar, gen)) return fail(io);
              if (tid < 32) {  // the bin holding the kleft-th largest, from the top (lane: 4 bins)
                const int lane = tid;
                int c[4], sum = 0;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  c[j] = __ldcg(H + 4 * lane + j);
                  sum += c[j];
                }
                int suf = sum;  // inclusive suffix sum over lanes >= lane
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                  const int n = __shfl_down_sync(0xffffffffu, suf, o);
                  if (lane + o < 32) suf += n;
                }
                int acc = suf - sum;  // taps in the bins above this lane's four
#pragma unroll
                for (int j = 3; j >= 0; --j) {
                  if (acc < kleft && acc + c[j] >= kleft) {
                    S->isc[2] = 4 * lane + j;
                    S->isc[3] = kleft - acc;
                  }
                  acc += c[j];
                }
              }
              __syncthreads();
              prefix |= (uint32_t)S->isc[2] << sh;
              kleft = S->isc[3];
              fixed |= ((1u << w) - 1u) << sh;
              __syncthreads();
            }
            const uint32_t vK = prefix;  // the K-th largest value; `kleft` ties to it are kept
            const int need = kleft;
            uint32_t gt = 0, eq = 0;
#pragma unroll
            for (int i = 0; i < EQ; ++i)
              if ((pass >> i) & 1u) {
                if (mb[i] > vK) gt |= 1u << i;
                else if (mb[i] == vK) eq |= 1u << i;
              }
            int tg, te;
            const int gt_in = block_exclusive_scan(__popc(gt), S->scan, tg);
            const int eq_in = block_exclusive_scan(__popc(eq), S->scan, te);
            if (tid == 0) {
              G.icnt[blockIdx.x] = tg;
              G.icnt[gridDim.x + blockIdx.x] = te;
            }
            if (!grid_sync(G.bar, gen)) return fail(io);
            grid_prefix(G.icnt, S);
            const int gt_pre = S->isc[2];
            __syncthreads();
            grid_prefix(G.icnt + gridDim.x, S);
            int eq_before = S->isc[2] + eq_in;
            base = gt_pre + gt_in + min(eq_before, need);
            keep = 0;
#pragma unroll
            for (int i = 0; i < EQ; ++i) {
              if ((gt >> i) & 1u) {
                keep |= 1u << i;
              } else if ((eq >> i) & 1u) {
                if (eq_before < need) keep |= 1u << i;
                ++eq_before;
              }
            }
            total = K;
          }
          if (trunc) st |= kStTrunc;
          const PathIO* gout = (write_paths && io.paths.count) ? &io.paths : nullptr;
          int pos = base;
#pragma unroll
          for (int i = 0; i < EQ; ++i) {
            if ((keep >> i) & 1u) {
              const int q = q_beg + tid * EQ + i;
              const int k = q & (M - 1), l = q >> logM;
              const int dk = ((k - A.K0 + (M >> 1)) & (M - 1)) - (M >> 1);
              const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
              PathRec rec;
              rec.h = hv[i];
              rec.dk = dk;
              rec.dl = dl;
              rec.hf = cmul(hv[i], tw<R>(A, (size_t)((-dl * dk) & (MN - 1))));
              rec.pad0 = rec.pad1 = 0;
              G.list[pos] = rec;
              if (gout) {
                gout->dk[pos] = (int16_t)dk;
                gout->dl[pos] = (int16_t)dl;
                store_complex(gout->h, (size_t)pos, gout->tap_dtype, hv[i]);
              }
              ++pos;
            }
          }
          if (gout && blockIdx.x == 0 && tid == 0) {
            gout->count[0] = total;
            if (gout->status) gout->status[0] = trunc ? ZOTFS_ETRUNCATED : ZOTFS_OK;
          }
          if (!grid_sync(G.bar, gen)) return fail(io);
          P = total;
          for (int p = tid; p < P; p += blockDim.x) {
            PathRec rec;
            const float4* s4 = reinterpret_cast<const float4*>(G.list + p);
            const float4 a = __ldcg(s4), b = __ldcg(s4 + 1);
            rec.h = make_float2(a.x, a.y);
            rec.hf = make_float2(a.z, a.w);
            rec.dk = __float_as_int(b.x);
            rec.dl = __float_as_int(b.y);
            rec.pad0 = rec.pad1 = 0;
            paths[p] = rec;
          }
        }
      }
      if (tid == 0) cnt[0] = P;
      __syncthreads();
    } else if (A.mode & kLoadPaths) {
      int bad;
      P = load_paths<R>(A, io.paths, 0, paths, bad);
      if (tid == 0) cnt[0] = P;
      if (bad) st |= kStInval;
      __syncthreads();
    }
    if ((A.mode & (kEstimate | kLoadPaths)) && (A.mode & (kCG | kApply)))
      build_runs<R>(paths, P, runs, sort_tmp, sort_keys, nruns);

    C v[E];
    // ------------------------------------------------ one operator apply
    if (A.mode & kApply) {
      C* src = A.adjoint ? G.extT : G.extP[0];
      for (int it = it_beg + tid; it < it_end; it += blockDim.x) {
        const int k = it & (M - 1), j0 = (it >> logM) * E;
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = reinterpret_cast<const C*>(io.v_in)[(size_t)(j0 + i) * M + k];
        write_ext<R, E, true>(src, A, k, j0, v);
      }
      if (!grid_sync(G.bar, gen)) return fail(io);
      for (int it = it_beg + tid; it < it_end; it += blockDim.x) {
        const int k = it & (M - 1), j0 = (it >> logM) * E;
        if (A.adjoint) gather_adj<R, E, true>(src, blk, paths, runs, nruns, A, 0, k, j0, v);
        else gather_fwd<R, E, true>(src, blk, paths, runs, nruns, A, 0, k, j0, v);
#pragma unroll
        for (int i = 0; i < E; ++i) reinterpret_cast<C*>(io.u_out)[(size_t)(j0 + i) * M + k] = v[i];
      }
      if (!grid_sync(G.bar, gen)) return fail(io);
      if (blockIdx.x == 0 && tid == 0 && io.status) *io.status = status_from_bits(st);
      continue;
    }

    // ------------------------------------------------ equalisation (Algorithm 1)
    if (A.mode & kCG) {
      const R lam = (R)io.lam;
      // Work items (column k, rows j0 .. j0 + E - 1): this CTA owns the delay columns [k0, k1)
      // over all rows, column fastest.
      const int cpc = grid_cols_per_cta(M, (int)gridDim.x);
      const int k0 = min(M, (int)blockIdx.x * cpc), k1 = min(M, k0 + cpc), ncol = k1 - k0;
      // a row group's items on lanes of their own warps (gstride a power of two >= 32), so no warp
      // mixes two row groups in its shared-memory reads
      int gshift = 5;
      while ((1 << gshift) < ncol) ++gshift;
      const int nslots = (N / E) << gshift;
      // The per-(path, column) factors of Eq. sparse_mvm / Eq. sparse_herm_mvm on the CTA's
      // columns, h_p W[dl_p k] (the adjoint's, conjugated at use), and each path's phase
      // W[-dl_p dk_p] that turns one into the forward factor hf_p W[dl_p k] (paths in the
      // sorted order of the runs).  In shared memory, or when it does not fit there (large
      // p_max at large M) in the CTA's slice of global scratch, read by the global route only.
      C* const tabg = G.ctab_g + (size_t)blockIdx.x * A.p_max * cpc;
      C* const tabp = G.tab_smem ? ctab : tabg;
      for (int e = tid; e < P * ncol; e += blockDim.x) {
        const int p = e / ncol, c = e - p * ncol;
        const PathRec& rec = paths[p];
        tabp[p * cpc + c] = cmul(rec.h, tab<R>(A, (size_t)(rec.dl + (N >> 1)) * M + k0 + c));
      }
      for (int p = tid; p < P; p += blockDim.x)
        phi[p] = tw<R>(A, (size_t)((-paths[p].dl * paths[p].dk) & (MN - 1)));
      for (int i = tid; i < N; i += blockDim.x) wn[i] = conjf2(tw<R>(A, (size_t)i << logM));  // W_N^{-l}
      // Window mode, when every path's |dk| is within the launch's cap: the CTA keeps p over the
      // columns [A0, A0 + Wc) -- its own and dmax more on either side -- in shared memory, forming it
      // there from a window of c each iteration (so no grid barrier separates the p update from
      // the forward gather), and gathers t from a window of t.  Otherwise the gathers read the
      // global extensions, p included.
      if (tid < 32) {
        int m = 0;
        for (int p = tid; p < P; p += 32) m = max(m, abs(paths[p].dk));
        m = __reduce_max_sync(0xffffffffu, m);
        if (tid == 0) S->isc[5] = m;
      }
      __syncthreads();
      const int dmax = S->isc[5];
      const bool win = G.tab_smem && G.win_cols > 0 && dmax <= G.win_dcap;
      const int A0 = (k0 - dmax) & ~1, Wc = ((k1 + dmax + 1) & ~1) - A0, Wp = G.win_cols;
      const uint32_t box_bytes = (uint32_t)(N + E + 3) * (uint32_t)Wp * 8u;
      const int Rw = N + E + 3, colw = -A0;

      const int hw = win ? dmax + 2 : M;  // halo columns stored: k < hw or k >= M - hw
      const size_t RS = (size_t)(2 * M);
      auto main_at = [&](const C* ext, int k, int l) { return ext[(size_t)l * RS + (k + (M >> 1))]; };
      auto wfail = [&](const FrameIO& io) {
        if (tid == 0) atomicExch(&G.bar->err, 1);  // the other CTAs leave at their next barrier
        fail(io);
      };

      if (y_early) {
        // done with the pilot's
      } else if (!A.y_is_dd) {
        // the data frame's Zak transform writes the extension of y directly
        grid_dzt<E>(io.y_data, A.in_dtype, nullptr, G.extT, A, tile, wn);
      } else {
        const C* Yd = reinterpret_cast<const C*>(io.y_data);
        for (int s = tid; s < nslots; s += blockDim.x) {
          const int g = s >> gshift, kk = s - (g << gshift);
          if (kk >= ncol) continue;
          const int k = k0 + kk, j0 = g * E;
#pragma unroll
          for (int i = 0; i < E; ++i) v[i] = Yd[(size_t)(j0 + i) * M + k];
          grid_ext_store<E>(G.extT, A, k, j0, v, k < hw || k >= M - hw, wn);
        }
      }
      if (!y_early && !grid_sync(G.bar, gen)) return fail(io);

      // b = H^H y;  c = b, x = 0, c_n = ||c||^2  (p = c is formed by the first iteration)
      if (win && !grid_window_load(bufX, &maps.t, M, A0, box_bytes, ncol > 0, &S->mbar, mph)) return wfail(io);
      R part = 0;
      for (int s = tid; s < nslots; s += blockDim.x) {
        const int g = s >> gshift, kk = s - (g << gshift);
        if (kk >= ncol) continue;
        const int k = k0 + kk, j0 = g * E;
        if (win) gather_adj<R, E, true, 2, false>(bufX, 0, paths, runs, nruns, A, 0, k, j0, v, nullptr, Wp, colw, ctab, phi, cpc, k0);
        else gather_adj<R, E, true, 2, false>(G.extT, blk, paths, runs, nruns, A, 0, k, j0, v, nullptr, 0, kColHalf, tabp, phi, cpc, k0);
#pragma unroll
        for (int i = 0; i < E; ++i) {
          G.X[(size_t)(j0 + i) * M + k] = make_float2(0.f, 0.f);
          part = fma(v[i].x, v[i].x, fma(v[i].y, v[i].y, part));
        }
        grid_ext_store<E>(G.extC, A, k, j0, v, k < hw || k >= M - hw, wn);
      }
      double* const partA = G.part;               // Re(p^H a)
      double* const partC = G.part + gridDim.x;   // ||c||^2
      double d = block_sum_to_thread0(part, S);
      if (tid == 0) partC[blockIdx.x] = d;
      if (!grid_sync(G.bar, gen)) return fail(io);
      double cn = grid_partials(partC);  // thread 0; the same in every CTA
      const double stop_at = io.eps2 > 0.0 ? io.eps2 * cn : -1.0;
      if (tid == 0) {
        S->isc[1] = isfinite(cn) ? 0 : 1;
        S->isc[4] = cn <= stop_at ? 1 : 0;
      }
      __syncthreads();

      for (int iter = 0; iter < io.iters && !S->isc[4]; ++iter) {
        C* const extPc = G.extP[iter & 1];
        const C* const extPo = G.extP[(iter & 1) ^ 1];
        const R beta = iter ? (R)S->fsc[1] : (R)0;
        // p = c + beta p (p = c in the first iteration), then t = H p
        if (win) {
          if (!grid_window_load(bufX, &maps.c, M, A0, box_bytes, ncol > 0, &S->mbar, mph)) return wfail(io);
          // two columns per thread and step (rows are 16-byte aligned: Wp and A0 even); rows
          // split over blockDim / 64 thread groups
          for (int r = tid >> 6; r < (ncol > 0 ? Rw : 0); r += blockDim.x >> 6)
            for (int c = 2 * (tid & 63); c < Wc; c += 128) {
              const float4 cv = *reinterpret_cast<const float4*>(bufX + r * Wp + c);
              float4* pp = reinterpret_cast<float4*>(bufP + r * Wp + c);
              if (iter) {
                const float4 pv = *pp;
                *pp = make_float4(fma(beta, pv.x, cv.x), fma(beta, pv.y, cv.y), fma(beta, pv.z, cv.z),
                                  fma(beta, pv.w, cv.w));
              } else {
                *pp = cv;
              }
            }
          __syncthreads();
          for (int s = tid; s < nslots; s += blockDim.x) {
            const int g = s >> gshift, kk = s - (g << gshift);
            if (kk >= ncol) continue;
            const int k = k0 + kk, j0 = g * E;
            gather_fwd<R, E, true, 2, false>(bufP, 0, paths, runs, nruns, A, 0, k, j0, v, nullptr, Wp, colw, ctab, phi, cpc, k0);
            grid_ext_store<E>(G.extT, A, k, j0, v, k < hw || k >= M - hw, wn);
          }
        } else {
          // the main column of p from those of c and the previous p; the halo column likewise
          // from the stored halo columns (as a window forms it)
          for (int s = tid; s < nslots; s += blockDim.x) {
            const int g = s >> gshift, kk = s - (g << gshift);
            if (kk >= ncol) continue;
            const int k = k0 + kk, j0 = g * E;
            const int mc = k + (M >> 1), hc = (k < (M >> 1) ? k + M : k - M) + (M >> 1);
            C ph[E];
#pragma unroll
            for (int i = 0; i < E; ++i) {
              const size_t o = (size_t)(j0 + i) * RS;
              v[i] = G.extC[o + mc];
              ph[i] = G.extC[o + hc];
              if (iter) {
                const C po = extPo[o + mc], qo = extPo[o + hc];
                v[i] = make_float2(fma(beta, po.x, v[i].x), fma(beta, po.y, v[i].y));
                ph[i] = make_float2(fma(beta, qo.x, ph[i].x), fma(beta, qo.y, ph[i].y));
              }
            }
#pragma unroll
            for (int i = 0; i < E; ++i)
              for (int r = j0 + i; r < Rw; r += N) {
                extPc[(size_t)r * RS + mc] = v[i];
                extPc[(size_t)r * RS + hc] = ph[i];
              }
          }
          if (!grid_sync(G.bar, gen)) return fail(io);
          for (int s = tid; s < nslots; s += blockDim.x) {
            const int g = s >> gshift, kk = s - (g << gshift);
            if (kk >= ncol) continue;
            const int k = k0 + kk, j0 = g * E;
            gather_fwd<R, E, true, 2, false>(extPc, blk, paths, runs, nruns, A, 0, k, j0, v, nullptr, 0, kColHalf, tabp, phi, cpc, k0);
            grid_ext_store<E>(G.extT, A, k, j0, v, true, wn);
          }
        }
        if (!grid_sync(G.bar, gen)) return fail(io);
        // p of item (k, l): the window, else the global extension (written this iteration)
        auto p_at = [&](int k, int l) { return win ? bufP[l * Wp + (k - A0)] : main_at(extPc, k, l); };
        // a = H^H t + lambda p;  Re(p^H a)
        if (win && !grid_window_load(bufX, &maps.t, M, A0, box_bytes, ncol > 0, &S->mbar, mph)) return wfail(io);
        part = 0;
        for (int s = tid; s < nslots; s += blockDim.x) {
          const int g = s >> gshift, kk = s - (g << gshift);
          if (kk >= ncol) continue;
          const int k = k0 + kk, j0 = g * E;
          if (win) gather_adj<R, E, true, 2, false>(bufX, 0, paths, runs, nruns, A, 0, k, j0, v, nullptr, Wp, colw, ctab, phi, cpc, k0);
          else gather_adj<R, E, true, 2, false>(G.extT, blk, paths, runs, nruns, A, 0, k, j0, v, nullptr, 0, kColHalf, tabp, phi, cpc, k0);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const C pv = p_at(k, j0 + i);
            v[i].x = fma(lam, pv.x, v[i].x);
            v[i].y = fma(lam, pv.y, v[i].y);
            part = fma(pv.x, v[i].x, fma(pv.y, v[i].y, part));
            G.Vv[(size_t)(j0 + i) * M + k] = v[i];
          }
        }
        d = block_sum_to_thread0(part, S);
        if (tid == 0) partA[blockIdx.x] = d;
        if (!grid_sync(G.bar, gen)) return fail(io);
        const double pa = grid_partials(partA);
        if (tid == 0) S->fsc[0] = cg_ratio<R>(cn, pa);  // alpha, FP64
        __syncthreads();
        const R alpha = (R)S->fsc[0];
        // x += alpha p;  c -= alpha a;  c_n' = ||c||^2
        part = 0;
        for (int s = tid; s < nslots; s += blockDim.x) {
          const int g = s >> gshift, kk = s - (g << gshift);
          if (kk >= ncol) continue;
          const int k = k0 + kk, j0 = g * E;
          C xv[E], av[E];  // the global loads before the first store
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)(j0 + i) * M + k;
            av[i] = G.Vv[o];
            xv[i] = G.X[o];
            v[i] = main_at(G.extC, k, j0 + i);
          }
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const C pv = p_at(k, j0 + i);
            xv[i].x = fma(alpha, pv.x, xv[i].x);
            xv[i].y = fma(alpha, pv.y, xv[i].y);
            v[i].x = fma(-alpha, av[i].x, v[i].x);
            v[i].y = fma(-alpha, av[i].y, v[i].y);
            G.X[(size_t)(j0 + i) * M + k] = xv[i];
            part = fma(v[i].x, v[i].x, fma(v[i].y, v[i].y, part));
          }
          grid_ext_store<E>(G.extC, A, k, j0, v, k < hw || k >= M - hw, wn);
        }
        d = block_sum_to_thread0(part, S);
        if (tid == 0) partC[blockIdx.x] = d;
        if (!grid_sync(G.bar, gen)) return fail(io);
        const double cn_new = grid_partials(partC);
        if (tid == 0) {
          S->fsc[1] = cg_ratio<R>(cn_new, cn);  // beta, FP64
          if (!isfinite(cn_new)) S->isc[1] = 1;
          if (cn_new <= stop_at) S->isc[4] = 1;
          cn = cn_new;
        }
        __syncthreads();
      }
      if (S->isc[1]) st |= kStNonFinite;
      if ((A.mode & kWriteX) && io.x_hat)
        for (int s = tid; s < nslots; s += blockDim.x) {
          const int g = s >> gshift, kk = s - (g << gshift);
          if (kk >= ncol) continue;
          const int k = k0 + kk, j0 = g * E;
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)(j0 + i) * M + k;
            reinterpret_cast<C*>(io.x_hat)[o] = G.X[o];
          }
        }
    }

    // ------------------------------------------------ demapping
    if ((A.mode & kDemap) && (io.llr || io.bits)) {
      const C* xs = (A.mode & kLoadX) ? reinterpret_cast<const C*>(io.x_in) : G.X;
      const R inv_lam = (R)1 / (R)io.lam;
      const int bps = io.bps;
      // eight consecutive symbols per thread: their LLRs, and their hard bits packed into bps
      // bytes right away (bit j of a symbol's label = its bit j)
      for (int g = gtid; g < MN / 8; g += nthr) {
        unsigned long long w = 0;
#pragma unroll
        for (int s8 = 0; s8 < 8; ++s8) {
          const int q = 8 * g + s8;
          float2 l01, l23, l45;
          const int hard = qam_llr_regs<R>(xs[q], bps, (R)io.pam_d, inv_lam, l01, l23, l45);
          w |= (unsigned long long)(__brev((unsigned)hard) >> (32 - bps)) << (bps * s8);
          if (io.llr) {
            float2* ol = reinterpret_cast<float2*>(io.llr + (size_t)q * bps);
            ol[0] = l01;
            if (bps > 2) ol[1] = l23;
            if (bps > 4) ol[2] = l45;
          }
        }
        if (io.bits) {
          uint8_t* o = io.bits + (size_t)g * bps;
          for (int h = 0; h < bps; ++h) o[h] = (uint8_t)(w >> (8 * h));
        }
      }
    }
    // every CTA done with this frame's scratch before the next frame (or the status) moves on
    if (!grid_sync(G.bar, gen)) return fail(io);
    if (blockIdx.x == 0 && tid == 0 && io.status) *io.status = status_from_bits(st);
  }
}

// win_cols: columns per row of the two CG windows (0: none); tab_cols: delay columns of the
// coefficient table in shared memory (the CTA's columns; 0 when the table is in global memory).
__host__ __device__ __forceinline__ size_t grid_smem_bytes(int N, int p_max, int win_cols, int tab_cols) {
  size_t off = (sizeof(SharedHdr) + 127) & ~size_t(127);
  off += ((size_t)p_max * sizeof(PathRecT<float>) + sizeof(int) * 2 + 127) & ~size_t(127);
  off += ((size_t)p_max * sizeof(RunRec) + 127) & ~size_t(127);
  off += ((size_t)p_max * sizeof(PathRecT<float>) + 127) & ~size_t(127);
  off += ((size_t)((p_max + 3) & ~3) * sizeof(int) + 127) & ~size_t(127);
  off += (size_t)N * kGridDftCols * sizeof(float2);
  off += ((size_t)N * sizeof(float2) + 127) & ~size_t(127);
  off += ((size_t)p_max * tab_cols * sizeof(float2) + 127) & ~size_t(127);
  off += ((size_t)p_max * sizeof(float2) + 127) & ~size_t(127);
  off += 2 * grid_window_elems(N, win_cols) * sizeof(float2);
  return off;
}

}  // namespace zotfs
