// The large-frame receiver on a thread-block cluster of CL CTAs per frame.  The frame's
// vectors live in one global-memory scratch slot per cluster (as in big_kernel, where one
// CTA owns a slot), and each CTA of the cluster owns a band of N / CL Doppler rows of every
// antenna block.  With CL CTAs per frame, CL times fewer slots are live at once (a higher L2
// hit rate for the gathers) and each frame finishes about CL times sooner.  The pilot read-offs and data-frame transforms are spread
// over the CTAs by antenna block; the path lists are then copied to every CTA through
// distributed shared memory.  Cluster barriers order the CTAs' global-memory vector updates,
// and Algorithm 1's scalars are rank-ordered FP64 sums of the CTAs' partials.
//
// Separate pilot frames (or lists loaded from global memory), time-domain or DD data frames,
// FP32.  EQ = M N / T elements per thread in the read-off (T threads per CTA); EW = EQ / CL
// rows per thread in the CG, walked in chunks of 8.
#pragma once

#include "frame_big.cuh"
#include "frame_cluster.cuh"

namespace zotfs {

// Complex elements of one cluster's slot: the p and t extensions (p itself is read from the
// main columns of its extension), x, and one region that holds c and a during the CG and the CL
// staging grids of the Zak transforms (and the demapper's labels) outside it.  Keeping the slot
// small keeps the live slots of a loaded GPU in L2.
__host__ __device__ __forceinline__ size_t big_cluster_union_elems(int M, int N, int ntx, int CL) {
  const size_t MN = (size_t)M * N, cv = (size_t)2 * ntx * MN, st = (size_t)CL * MN;
  return cv > st ? cv : st;
}
__host__ __device__ __forceinline__ size_t big_cluster_slot_elems(int M, int N, int nrx, int ntx, int CL) {
  const size_t MN = (size_t)M * N;
  return (size_t)(nrx + ntx) * ext_block_elems(M, N, kBigChunk) + (size_t)ntx * MN +
         big_cluster_union_elems(M, N, ntx, CL);
}

// OR of one status word per CTA over the cluster, the same in every CTA (the flag sets of
// cluster_any, which alternate the same way).
template <int CL>
__device__ __forceinline__ int cluster_or(cgx::cluster_group& cluster, ClusterScratch* cs, int& set, int mine) {
  const int rank = (int)cluster.block_rank();
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < CL; ++r) cluster.map_shared_rank(cs, r)->flag[set][rank] = mine;
  cluster.sync();
  int any = 0;
#pragma unroll
  for (int r = 0; r < CL; ++r) any |= cs->flag[set][r];
  set ^= 1;
  return any;
}

__host__ __device__ __forceinline__ size_t big_cluster_smem_bytes(int nrx, int ntx, int p_max) {
  return big_smem_bytes(nrx, ntx, p_max, 4) + ((sizeof(ClusterScratch) + 127) & ~size_t(127)) + 128;
}

struct BigClusterShared {  // after the path-list area
  int frame;               // the cluster's current frame (written by rank 0 into every CTA)
};

template <int EQ, int CL, int TMAX>
__global__ void __launch_bounds__(TMAX, 1)
    big_cluster_kernel(const __grid_constant__ FrameArgs A, int radix, char* scratch, size_t slot_bytes) {
  using R = float;
  using C = float2;
  using PathRec = PathRecT<R>;
  constexpr int E = kBigChunk;
  constexpr int EW = EQ / CL;
  constexpr int NCH = EW / E;
  static_assert(EW % E == 0, "rows per thread must be a multiple of the chunk");
  cgx::cluster_group cluster = cgx::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(128) unsigned char smem[];
  SharedHdr* S = reinterpret_cast<SharedHdr*>(smem);
  const int nlists = A.nrx * A.ntx;
  size_t off = (sizeof(SharedHdr) + 127) & ~size_t(127);
  PathRec* paths = reinterpret_cast<PathRec*>(smem + off);
  int* cnt = reinterpret_cast<int*>(paths + (size_t)nlists * A.p_max);
  int* nruns = cnt + nlists;
  off += ((size_t)nlists * A.p_max * sizeof(PathRec) + (size_t)nlists * sizeof(int) * 2 + 127) & ~size_t(127);
  RunRec* runs = reinterpret_cast<RunRec*>(smem + off);
  off += ((size_t)nlists * A.p_max * sizeof(RunRec) + 127) & ~size_t(127);
  PathRec* sort_tmp = reinterpret_cast<PathRec*>(smem + off);
  off += ((size_t)A.p_max * sizeof(PathRec) + 127) & ~size_t(127);
  int* sort_keys = reinterpret_cast<int*>(smem + off);
  off += ((size_t)((A.p_max + 3) & ~3) * sizeof(int) + 127) & ~size_t(127);
  ClusterScratch* cs = reinterpret_cast<ClusterScratch*>(smem + off);
  off += (sizeof(ClusterScratch) + 127) & ~size_t(127);
  BigClusterShared* bs = reinterpret_cast<BigClusterShared*>(smem + off);

  const int M = A.M, N = A.N, MN = M * N, logM = A.logM, T = blockDim.x;
  const size_t blk = ext_block_elems(M, N, E);
  char* slot = scratch + (size_t)(blockIdx.x / CL) * slot_bytes;
  C* extP = reinterpret_cast<C*>(slot);
  C* extT = extP + (size_t)A.ntx * blk;
  C* Xv = extT + (size_t)A.nrx * blk;
  C* Cv = Xv + (size_t)A.ntx * MN;    // c and a share their region with the staging grids:
  C* Vv = Cv + (size_t)A.ntx * MN;    // the grids are used only before b = H^H y and in the
  C* stage = Cv + (size_t)rank * MN;  // demapper (labels), when c and a are dead
  const int tid = threadIdx.x;
  const int k = tid & (M - 1);
  const int band = N / CL;
  const int jw = rank * band + (tid >> logM) * EW;  // first of this thread's EW rows
  const size_t in_bytes = (size_t)MN * dtype_bytes(A.in_dtype);
  const bool write_paths = (A.mode & kWritePaths) != 0;
  int fset = 0;

  auto own = [&](int c, int i) { return (size_t)(jw + c * E + i) * M + k; };
  // p's value at an own element: the main column of its extension
  auto p_at = [&](int t, int c, int i) -> C& {
    return extP[(size_t)t * blk + (size_t)(jw + c * E + i) * 2 * M + k + (M >> 1)];
  };
  auto load_grid = [&](const char* src) {  // TD grid -> this CTA's staging grid, all threads
    __syncthreads();
    for (int e = tid; e < MN; e += T) stage[e] = load_complex<C>(src, (size_t)e, A.in_dtype);
    __syncthreads();
  };

  for (;;) {
    // the next frame: rank 0 takes it from the work counter and hands it to every CTA
    if (rank == 0 && tid == 0) {
      const int f = atomicAdd(A.work_counter, 1);
#pragma unroll
      for (int r = 0; r < CL; ++r) cluster.map_shared_rank(bs, r)->frame = f;
    }
    cluster.sync();
    const int f = bs->frame;
    cluster.sync();  // every CTA has read it before rank 0 may overwrite it
    if (f >= A.n_frames) break;
    const FrameIO io = frame_io(A, f, (int)sizeof(C));
    int st = 0;

    // ------------------------------------------------ path lists: list li on CTA li mod CL
    if (A.mode & kEstimate) {
      for (int li = rank; li < nlists; li += CL) {
        const int r = li / A.ntx, t = li - r * A.ntx;
        load_grid(io.y_pilot + ((size_t)t * A.nrx + r) * in_bytes);
        dzt_inplace<R>(stage, A, radix);
        int trunc;
        const PathIO* gout = (write_paths && io.paths.count) ? &io.paths : nullptr;
        const int P = readoff_compact<R, EQ>(stage, A, (R)io.theta, io.a_pilot, paths + (size_t)li * A.p_max, S,
                                             gout, li, trunc);
        if (tid == 0) cnt[li] = P;
        if (trunc) st |= kStTrunc;
        __syncthreads();
        // copy the list to the other CTAs
        const uint32_t* src = reinterpret_cast<const uint32_t*>(paths + (size_t)li * A.p_max);
        const int words = P * (int)(sizeof(PathRec) / 4);
        for (int r2 = 0; r2 < CL; ++r2) {
          if (r2 == rank) continue;
          uint32_t* dst = reinterpret_cast<uint32_t*>(cluster.map_shared_rank(paths, r2) + (size_t)li * A.p_max);
          for (int w = tid; w < words; w += T) dst[w] = src[w];
          if (tid == 0) cluster.map_shared_rank(cnt, r2)[li] = P;
        }
      }
    } else {
      for (int li = 0; li < nlists; ++li) {
        int bad;
        const int P = load_paths<R>(A, io.paths, li, paths + (size_t)li * A.p_max, bad);
        if (tid == 0) cnt[li] = P;
        if (bad) st |= kStInval;
      }
    }
    cluster.sync();  // every CTA holds every list
    for (int li = 0; li < nlists; ++li)
      build_runs<R>(paths + (size_t)li * A.p_max, cnt[li], runs + (size_t)li * A.p_max, sort_tmp, sort_keys,
                    nruns + li);

    C v[E];
    const R lam = (R)io.lam;
    // ------------------------------------------------ y_r -> extT (block r on CTA r mod CL)
    if (A.y_is_dd) {
      for (int r = 0; r < A.nrx; ++r) {
        const C* yd = reinterpret_cast<const C*>(io.y_data) + (size_t)r * MN;
        for (int c = 0; c < NCH; ++c) {
#pragma unroll
          for (int i = 0; i < E; ++i) v[i] = yd[own(c, i)];
          write_ext<R, E, true>(extT + r * blk, A, k, jw + c * E, v);
        }
      }
    } else {
      for (int r = rank; r < A.nrx; r += CL) {
        load_grid(io.y_data + (size_t)r * in_bytes);
        dzt_inplace<R>(stage, A, radix);
        // the whole block from this CTA: EQ rows per thread over the full grid
        const int jf = (tid >> logM) * EQ;
        for (int c = 0; c < EQ / E; ++c) {
#pragma unroll
          for (int i = 0; i < E; ++i)
            v[i] = cscale(stage[(size_t)bitrev(jf + c * E + i, A.logN) * M + k], (R)A.inv_sqrtN);
          write_ext<R, E, true>(extT + r * blk, A, k, jf + c * E, v);
        }
      }
    }
    cluster.sync();  // extT holds every y_r

    // b = H^H y;  c = b, p = b, x = 0, c_n = ||c||^2  (this CTA's rows)
    R part = 0;
    for (int t = 0; t < A.ntx; ++t)
      for (int c = 0; c < NCH; ++c) {
        gather_adj<R, E, true>(extT, blk, paths, runs, nruns, A, t, k, jw + c * E, v);
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const size_t o = (size_t)t * MN + own(c, i);
          Cv[o] = v[i];
          Xv[o] = make_float2(0.f, 0.f);
          part = fma(v[i].x, v[i].x, fma(v[i].y, v[i].y, part));
        }
        write_ext<R, E, true>(extP + t * blk, A, k, jw + c * E, v);
      }
    int set = 0;
    double cn = cluster_sum<CL>(cluster, cs, set, block_sum_to_thread0(part, S));  // extP complete
    set ^= 1;
    // every CTA's thread 0 holds the same rank-ordered sums, so all take the same decision
    const double stop_at = io.eps2 > 0.0 ? io.eps2 * cn : -1.0;
    if (tid == 0) {
      S->isc[1] = isfinite(cn) ? 0 : 1;
      S->isc[4] = cn <= stop_at ? 1 : 0;
    }
    __syncthreads();

    for (int it = 0; it < io.iters && !S->isc[4]; ++it) {
      // t = H p  (extP -> extT)
      for (int r = 0; r < A.nrx; ++r)
        for (int c = 0; c < NCH; ++c) {
          gather_fwd<R, E, true>(extP, blk, paths, runs, nruns, A, r, k, jw + c * E, v);
          write_ext<R, E, true>(extT + r * blk, A, k, jw + c * E, v);
        }
      cluster.sync();  // extT complete
      // a = H^H t + lambda p;  Re(p^H a)
      part = 0;
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c) {
          gather_adj<R, E, true>(extT, blk, paths, runs, nruns, A, t, k, jw + c * E, v);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            const C pv = p_at(t, c, i);
            v[i].x = fma(lam, pv.x, v[i].x);
            v[i].y = fma(lam, pv.y, v[i].y);
            part = fma(pv.x, v[i].x, fma(pv.y, v[i].y, part));
            Vv[o] = v[i];
          }
        }
      const double pa = cluster_sum<CL>(cluster, cs, set, block_sum_to_thread0(part, S));
      set ^= 1;
      if (tid == 0) S->fsc[0] = cg_ratio<float>(cn, pa);
      __syncthreads();
      const R alpha = (R)S->fsc[0];
      part = 0;
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c) {
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            const C pv = p_at(t, c, i), av = Vv[o];
            C xv = Xv[o], cv = Cv[o];
            xv.x = fma(alpha, pv.x, xv.x);
            xv.y = fma(alpha, pv.y, xv.y);
            cv.x = fma(-alpha, av.x, cv.x);
            cv.y = fma(-alpha, av.y, cv.y);
            Xv[o] = xv;
            Cv[o] = cv;
            part = fma(cv.x, cv.x, fma(cv.y, cv.y, part));
          }
        }
      const double cn_new = cluster_sum<CL>(cluster, cs, set, block_sum_to_thread0(part, S));
      set ^= 1;
      if (tid == 0) {
        S->fsc[1] = cg_ratio<float>(cn_new, cn);
        if (!isfinite(cn_new)) S->isc[1] = 1;
        if (cn_new <= stop_at) S->isc[4] = 1;
        cn = cn_new;
      }
      __syncthreads();
      const R beta = (R)S->fsc[1];
      if (it + 1 < io.iters) {
        for (int t = 0; t < A.ntx; ++t)
          for (int c = 0; c < NCH; ++c) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
              const size_t o = (size_t)t * MN + own(c, i);
              const C cv = Cv[o];
              C pv = p_at(t, c, i);  // this thread's own element: no other thread writes it
              pv.x = fma(beta, pv.x, cv.x);
              pv.y = fma(beta, pv.y, cv.y);
              v[i] = pv;
            }
            write_ext<R, E, true>(extP + t * blk, A, k, jw + c * E, v);
          }
        cluster.sync();  // extP complete
      }
    }
    if (S->isc[1]) st |= kStNonFinite;
    if ((A.mode & kWriteX) && io.x_hat)
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            reinterpret_cast<C*>(io.x_hat)[o] = Xv[o];
          }

    // ------------------------------------------------ demapping of this CTA's rows
    if ((A.mode & kDemap) && (io.llr || io.bits)) {
      const R inv_lam = (R)1 / (R)io.lam;
      const int bps = io.bps;
      const int q0 = rank * band * M, nq = band * M;
      uint8_t* lab = reinterpret_cast<uint8_t*>(stage);  // [t][nq] labels, bit j at bit j
      __syncthreads();
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            const int q = (int)(o - (size_t)t * MN);
            float2 l01, l23, l45;
            const int hard = qam_llr_regs<R>(Xv[o], bps, (R)io.pam_d, inv_lam, l01, l23, l45);
            lab[(size_t)t * nq + (q - q0)] = (uint8_t)(__brev((unsigned)hard) >> (32 - bps));
            if (io.llr) {
              float2* ol = reinterpret_cast<float2*>(io.llr + ((size_t)t * MN + q) * bps);
              ol[0] = l01;
              if (bps > 2) ol[1] = l23;
              if (bps > 4) ol[2] = l45;
            }
          }
      __syncthreads();
      if (io.bits) {
        const int groups = nq / 8;
        for (int g = tid; g < A.ntx * groups; g += T) {
          const int t = g / groups, gl = g - t * groups;
          const unsigned long long l8 = reinterpret_cast<const unsigned long long*>(lab + (size_t)t * nq)[gl];
          unsigned long long w = 0;
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) w |= ((l8 >> (8 * s8)) & 0xffull) << (bps * s8);
          uint8_t* o = io.bits + ((size_t)t * MN + q0) / 8 * bps + (size_t)gl * bps;
          if ((reinterpret_cast<uintptr_t>(o) & 1u) == 0) {
            uint16_t* o2 = reinterpret_cast<uint16_t*>(o);
            for (int h = 0; h < bps / 2; ++h) o2[h] = (uint16_t)(w >> (16 * h));
          } else {
            for (int h = 0; h < bps; ++h) o[h] = (uint8_t)(w >> (8 * h));
          }
        }
      }
      __syncthreads();
    }
    st = cluster_or<CL>(cluster, cs, fset, st);
    if (rank == 0) publish_status(A, io.status, st);
  }
}

}  // namespace zotfs
