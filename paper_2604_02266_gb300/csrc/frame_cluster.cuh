// The receiver for one frame on a thread-block cluster of C CTAs (C SMs), for latency: each
// CTA owns a band of N / C Doppler rows of the CG vectors, and every CTA keeps a full replica
// of the quasi-periodic extension being gathered, so all operator gathers read local shared
// memory.  After each operator step a CTA stores its rows into every replica (distributed
// shared memory), and the scalar reductions of Algorithm 1 combine the CTAs' FP64 partials
// in rank order, so every CTA derives the same alpha and beta.  The pilot and data Zak
// transforms and the read-off run redundantly in every CTA (the transform along the Doppler
// axis needs the whole grid), which keeps them at one CTA's latency without an exchange.
//
// SISO frames (separate pilot frame, or path lists loaded from global memory), E = 8 rows per
// thread; C in {2, 4}; T = M N / (8 C) threads per CTA.
#pragma once

#include <cooperative_groups.h>

#include "frame_kernel.cuh"

namespace zotfs {

namespace cgx = cooperative_groups;

constexpr int kClusterE = 8;

// Scalars exchanged between the CTAs of a cluster (after the frame kernel's layout).
struct ClusterScratch {
  double part[2][4];  // two alternating sets of per-rank partial sums
  int flag[2][4];     // two alternating sets of per-rank flags
};

__host__ __device__ __forceinline__ size_t cluster_smem_bytes(int M, int N, int p_max) {
  return frame_smem_bytes(M, N, kClusterE, 1, 1, p_max, 4, false) + ((sizeof(ClusterScratch) + 127) & ~size_t(127));
}

// OR of one flag per CTA over the cluster, the same in every CTA.  `set` alternates between
// calls: a set is written again only after a cluster barrier that every CTA reaches after
// reading it.
template <int C>
__device__ __forceinline__ bool cluster_any(cgx::cluster_group& cluster, ClusterScratch* cs, int& set, bool mine) {
  const int rank = (int)cluster.block_rank();
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < C; ++r) cluster.map_shared_rank(cs, r)->flag[set][rank] = mine ? 1 : 0;
  cluster.sync();
  bool any = false;
#pragma unroll
  for (int r = 0; r < C; ++r) any |= cs->flag[set][r] != 0;
  set ^= 1;
  return any;
}

// Sum over the cluster of the CTAs' partials (`local`, valid in thread 0), in rank order; the
// result is valid in thread 0 of every CTA.  `set` alternates so that a fast CTA's next
// reduction never overwrites a slot that a slow CTA has yet to read.
template <int C>
__device__ __forceinline__ double cluster_sum(cgx::cluster_group& cluster, ClusterScratch* cs, int set,
                                              double local) {
  const int rank = (int)cluster.block_rank();
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < C; ++r) cluster.map_shared_rank(cs, r)->part[set][rank] = local;
  cluster.sync();
  double s = 0.0;
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < C; ++r) s += cs->part[set][r];
  return s;
}

// Store this thread's E rows of one vector into the extension replica of every CTA.
template <int C>
__device__ __forceinline__ void broadcast_ext(cgx::cluster_group& cluster, float2* ext, const FrameArgs& A, int k,
                                              int j0, const float2 (&v)[kClusterE]) {
#pragma unroll
  for (int r = 0; r < C; ++r) write_ext<float, kClusterE>(cluster.map_shared_rank(ext, r), A, k, j0, v);
}

template <int C, int TMAX>
__global__ void __launch_bounds__(TMAX, 1) cluster_kernel(const __grid_constant__ FrameArgs A, int radix) {
  using R = float;
  using Cv = float2;
  using PathRec = PathRecT<R>;
  constexpr int E = kClusterE;
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = (int)(blockIdx.x / C), ncl = (int)(gridDim.x / C);
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
  Cv* ext = reinterpret_cast<Cv*>(smem + off);
  const size_t blk = ext_block_elems(A.M, A.N, E);
  ClusterScratch* cs = reinterpret_cast<ClusterScratch*>(smem + off + blk * sizeof(Cv));

  const int M = A.M, N = A.N, MN = M * N, logM = A.logM;
  const int tid = threadIdx.x, k = tid & (M - 1);
  const int band = N / C;  // rows per CTA
  const int j0 = rank * band + (tid >> logM) * E;
  const bool write_paths = (A.mode & kWritePaths) != 0 && rank == 0;

  if (tid == 0) mbar_init(&S->mbar, 1);
  __syncthreads();
  uint32_t phase = 0;
  int fset = 0;  // flag set of the next cluster_any

  for (int f = cid; f < A.n_frames; f += ncl) {
    const FrameIO io = frame_io(A, f, (int)sizeof(Cv));
    const PathIO* gout = (write_paths && io.paths.count) ? &io.paths : nullptr;
    int st = 0;

    // ------------------------------------------------ path list (every CTA the same)
    if (A.mode & kEstimate) {
      const bool ok = stage_grid<R, E * C>(ext, io.y_pilot, MN, A.in_dtype, &S->mbar, phase);
      if (cluster_any<C>(cluster, cs, fset, !ok)) {
        st |= kStTimeout;
      } else {
        dzt_inplace<R>(ext, A, radix);
        int trunc;
        const int P = readoff_compact<R, E * C>(ext, A, (R)io.theta, io.a_pilot, paths, S, gout, 0, trunc);
        if (tid == 0) cnt[0] = P;
        if (trunc) st |= kStTrunc;
      }
    } else {
      int bad;
      const int P = load_paths<R>(A, io.paths, 0, paths, bad);
      if (tid == 0) cnt[0] = P;
      if (bad) st |= kStInval;
    }
    __syncthreads();
    if (st & kStTimeout) {
      if (rank == 0) publish_status(A, io.status, st);
      break;  // every CTA of the cluster saw the failure: all stop together
    }
    build_runs<R>(paths, cnt[0], runs, sort_tmp, sort_keys, nruns);

    // ------------------------------------------------ data frame: y_ext in every replica
    Cv v[E];
    const bool ok = stage_grid<R, E * C>(ext, io.y_data, MN, A.in_dtype, &S->mbar, phase);
    if (cluster_any<C>(cluster, cs, fset, !ok)) {
      if (rank == 0) publish_status(A, io.status, st | kStTimeout);
      break;
    }
    dzt_inplace<R>(ext, A, radix);
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = cscale(ext[(size_t)bitrev(j0 + i, A.logN) * M + k], (R)A.inv_sqrtN);
    cluster.sync();  // every CTA has read its rows of the transformed grid
    broadcast_ext<C>(cluster, ext, A, k, j0, v);
    cluster.sync();

    // b = H^H y;  c = b, p = b, x = 0, c_n = ||c||^2   (Algorithm 1, initialisation)
    const R lam = (R)io.lam;
    Cv x[E], c[E], p[E];
    R part = 0;
    gather_adj<R, E>(ext, blk, paths, runs, nruns, A, 0, k, j0, c);
#pragma unroll
    for (int i = 0; i < E; ++i) {
      x[i] = make_float2(0.f, 0.f);
      p[i] = c[i];
      part = fma(c[i].x, c[i].x, fma(c[i].y, c[i].y, part));
    }
    int set = 0;
    double cn = cluster_sum<C>(cluster, cs, set, block_sum_to_thread0(part, S));  // all gathers of y_ext done
    set ^= 1;
    // every CTA's thread 0 holds the same rank-ordered sums, so all take the same decision
    const double stop_at = io.eps2 > 0.0 ? io.eps2 * cn : -1.0;
    if (tid == 0) {
      S->isc[1] = isfinite(cn) ? 0 : 1;
      S->isc[4] = cn <= stop_at ? 1 : 0;
    }
    broadcast_ext<C>(cluster, ext, A, k, j0, p);
    cluster.sync();

    for (int it = 0; it < io.iters && !S->isc[4]; ++it) {
      gather_fwd<R, E>(ext, blk, paths, runs, nruns, A, 0, k, j0, v);  // t = H p
      cluster.sync();                                                   // p_ext no longer read
      broadcast_ext<C>(cluster, ext, A, k, j0, v);
      cluster.sync();
      gather_adj<R, E>(ext, blk, paths, runs, nruns, A, 0, k, j0, v);  // a = H^H t + lambda p
      part = 0;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        v[i].x = fma(lam, p[i].x, v[i].x);
        v[i].y = fma(lam, p[i].y, v[i].y);
        part = fma(p[i].x, v[i].x, fma(p[i].y, v[i].y, part));
      }
      const double pa = cluster_sum<C>(cluster, cs, set, block_sum_to_thread0(part, S));
      set ^= 1;
      if (tid == 0) S->fsc[0] = cg_ratio<float>(cn, pa);  // alpha, FP64, the same in every CTA
      __syncthreads();
      const R alpha = (R)S->fsc[0];
      part = 0;
#pragma unroll
      for (int i = 0; i < E; ++i) {
        x[i].x = fma(alpha, p[i].x, x[i].x);
        x[i].y = fma(alpha, p[i].y, x[i].y);
        c[i].x = fma(-alpha, v[i].x, c[i].x);
        c[i].y = fma(-alpha, v[i].y, c[i].y);
        part = fma(c[i].x, c[i].x, fma(c[i].y, c[i].y, part));
      }
      const double cn_new = cluster_sum<C>(cluster, cs, set, block_sum_to_thread0(part, S));
      set ^= 1;
      if (tid == 0) {
        S->fsc[1] = cg_ratio<float>(cn_new, cn);  // beta, FP64
        if (!isfinite(cn_new)) S->isc[1] = 1;
        if (cn_new <= stop_at) S->isc[4] = 1;
        cn = cn_new;
      }
      __syncthreads();
      const R beta = (R)S->fsc[1];
#pragma unroll
      for (int i = 0; i < E; ++i) {
        p[i].x = fma(beta, p[i].x, c[i].x);
        p[i].y = fma(beta, p[i].y, c[i].y);
      }
      if (it + 1 < io.iters) {  // the t replicas are no longer read once every CTA passed the sum
        broadcast_ext<C>(cluster, ext, A, k, j0, p);
        cluster.sync();
      }
    }
    if (S->isc[1]) st |= kStNonFinite;
    if ((A.mode & kWriteX) && io.x_hat) {
#pragma unroll
      for (int i = 0; i < E; ++i) reinterpret_cast<Cv*>(io.x_hat)[(size_t)(j0 + i) * M + k] = x[i];
    }

    // ------------------------------------------------ demapping of this CTA's rows
    if ((A.mode & kDemap) && (io.llr || io.bits)) {
      const R inv_lam = (R)1 / (R)io.lam;
      const int bps = io.bps;
      const int q0 = rank * band * M, nq = band * M;  // this CTA's symbols: q0 .. q0 + nq - 1
      __syncthreads();                                // ext is read by no one any more
      uint8_t* lab = reinterpret_cast<uint8_t*>(ext);
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int q = (j0 + i) * M + k;
        float2 l01, l23, l45;
        const int hard = qam_llr_regs<R>(x[i], bps, (R)io.pam_d, inv_lam, l01, l23, l45);
        lab[q - q0] = (uint8_t)(__brev((unsigned)hard) >> (32 - bps));
        if (io.llr) {
          float2* o = reinterpret_cast<float2*>(io.llr + (size_t)q * bps);
          o[0] = l01;
          if (bps > 2) o[1] = l23;
          if (bps > 4) o[2] = l45;
        }
      }
      __syncthreads();
      if (io.bits) {
        for (int g = tid; g < nq / 8; g += blockDim.x) {
          const unsigned long long l8 = reinterpret_cast<const unsigned long long*>(lab)[g];
          unsigned long long w = 0;
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) w |= ((l8 >> (8 * s8)) & 0xffull) << (bps * s8);
          uint8_t* o = io.bits + (size_t)(q0 / 8 + g) * bps;
          if ((reinterpret_cast<uintptr_t>(o) & 1u) == 0) {
            uint16_t* o2 = reinterpret_cast<uint16_t*>(o);
            for (int h = 0; h < bps / 2; ++h) o2[h] = (uint16_t)(w >> (16 * h));
          } else {
            for (int h = 0; h < bps; ++h) o[h] = (uint8_t)(w >> (8 * h));
          }
        }
      }
    }
    // the frame's status after every CTA has written its rows (and before any CTA's next
    // frame overwrites a replica)
    const bool nonfinite = cluster_any<C>(cluster, cs, fset, (st & kStNonFinite) != 0);
    if (nonfinite) st |= kStNonFinite;
    if (rank == 0) publish_status(A, io.status, st);
  }
}

}  // namespace zotfs
