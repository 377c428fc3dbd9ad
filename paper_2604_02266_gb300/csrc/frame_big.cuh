// The receiver for frames whose CG vectors do not fit one CTA's shared memory (large grids,
// large MIMO stacks).  Same stages and the same device routines as frame_kernel; the
// difference is where the vectors live: each resident CTA owns a slice ("slot") of global
// scratch holding the Zak-transform staging grid, the quasi-periodic extensions of p and of
// t = H p (row-major, so a warp's 32 consecutive columns are one coalesced L1 access), and the
// per-element vectors x, c, p, a.  Shared memory holds the path lists and the reduction
// scratch.  A thread owns column k and EW = MN / T consecutive Doppler rows of every antenna
// block and walks them in chunks of 8 rows.
#pragma once

#include "frame_kernel.cuh"

namespace zotfs {

constexpr int kBigThreads = 512;
constexpr int kBigChunk = 8;

// Complex elements of one CTA's scratch slot.
__host__ __device__ __forceinline__ size_t big_slot_elems(int M, int N, int nrx, int ntx) {
  const size_t MN = (size_t)M * N;
  const int nb = nrx > ntx ? nrx : ntx;
  const size_t blk = ext_block_elems(M, N, kBigChunk);
  return MN + (size_t)(nrx + ntx) * blk + (size_t)3 * ntx * MN + (size_t)nb * MN;
}
__host__ __device__ __forceinline__ size_t big_smem_bytes(int nrx, int ntx, int p_max, int real_bytes) {
  size_t hdr = (sizeof(SharedHdr) + 127) & ~size_t(127);
  const size_t rec = (size_t)4 * real_bytes + 16;
  size_t paths = ((size_t)nrx * ntx * p_max * rec + (size_t)nrx * ntx * sizeof(int) * 2 + 127) & ~size_t(127);
  paths += ((size_t)nrx * ntx * p_max * sizeof(RunRec) + 127) & ~size_t(127);
  paths += ((size_t)p_max * rec + 127) & ~size_t(127);
  paths += ((size_t)((p_max + 3) & ~3) * sizeof(int) + 127) & ~size_t(127);
  return hdr + paths;
}

template <typename R, int EW>
__global__ void __launch_bounds__(kBigThreads, 1)
    big_kernel(const __grid_constant__ FrameArgs A, int radix, char* scratch, size_t slot_bytes) {
  using C = typename Cx<R>::C;
  using PathRec = PathRecT<R>;
  constexpr int E = kBigChunk;
  constexpr int NCH = EW / E;
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

  const int M = A.M, N = A.N, MN = M * N, logM = A.logM, T = blockDim.x;
  const int nb = A.nrx > A.ntx ? A.nrx : A.ntx;
  const size_t blk = ext_block_elems(M, N, E);
  C* stage = reinterpret_cast<C*>(scratch + (size_t)blockIdx.x * slot_bytes);
  C* extP = stage + MN;
  C* extT = extP + (size_t)A.ntx * blk;
  C* Xv = extT + (size_t)A.nrx * blk;
  C* Cv = Xv + (size_t)A.ntx * MN;
  C* Pv = Cv + (size_t)A.ntx * MN;
  C* Vv = Pv + (size_t)A.ntx * MN;
  const int tid = threadIdx.x;
  const int k = tid & (M - 1);
  const int jw = (tid >> logM) * EW;  // first of this thread's EW rows
  const size_t in_bytes = (size_t)MN * dtype_bytes(A.in_dtype);
  const bool write_paths = (A.mode & kWritePaths) != 0;
  (void)nb;

  auto own = [&](int c, int i) { return (size_t)(jw + c * E + i) * M + k; };
  auto load_grid = [&](const char* src) {  // TD grid -> stage (complex R), all threads
    __syncthreads();
    for (int e = tid; e < MN; e += T) stage[e] = load_complex<C>(src, (size_t)e, A.in_dtype);
    __syncthreads();
  };

  for (;;) {
    if (tid == 0) S->isc[0] = atomicAdd(A.work_counter, 1);
    __syncthreads();
    const int f = S->isc[0];
    __syncthreads();
    if (f >= A.n_frames) break;
    const FrameIO io = frame_io(A, f, (int)sizeof(C));
    const PathIO* gout = (write_paths && io.paths.count) ? &io.paths : nullptr;
    int st = 0;

    if (A.mode & kDzt) {
      load_grid(io.y_data);
      dzt_inplace<R>(stage, A, radix);
      for (int e = tid; e < MN; e += T) {
        const int kk = e & (M - 1), l = e >> logM;
        reinterpret_cast<C*>(io.u_out)[e] = cscale(stage[(size_t)bitrev(l, A.logN) * M + kk], (R)A.inv_sqrtN);
      }
      if (io.status && tid == 0) *io.status = status_from_bits(st);
      continue;
    }

    // ------------------------------------------------ path lists
    bool have_paths = false;
    if ((A.mode & kEstimate) && A.pilot_mode == ZOTFS_PILOT_SEPARATE) {
      for (int t = 0; t < A.ntx; ++t)
        for (int r = 0; r < A.nrx; ++r) {
          load_grid(io.y_pilot + ((size_t)t * A.nrx + r) * in_bytes);
          dzt_inplace<R>(stage, A, radix);
          const int li = r * A.ntx + t;
          int trunc;
          const int P = readoff_compact<R, EW>(stage, A, (R)io.theta, io.a_pilot, paths + (size_t)li * A.p_max, S, gout, li, trunc);
          if (tid == 0) cnt[li] = P;
          if (trunc) st |= kStTrunc;
        }
      have_paths = true;
    } else if ((A.mode & kEstimate) && A.pilot_mode == ZOTFS_PILOT_EMBEDDED && !(A.mode & kCG)) {
      load_grid(io.y_data);
      dzt_inplace<R>(stage, A, radix);
      int trunc;
      const int P = readoff_compact<R, EW>(stage, A, (R)io.theta, io.a_pilot, paths, S, gout, 0, trunc);
      if (tid == 0) cnt[0] = P;
      if (trunc) st |= kStTrunc;
      have_paths = true;
    } else if (A.mode & kLoadPaths) {
      for (int li = 0; li < nlists; ++li) {
        int bad;
        const int P = load_paths<R>(A, io.paths, li, paths + (size_t)li * A.p_max, bad);
        if (tid == 0) cnt[li] = P;
        if (bad) st |= kStInval;
      }
      have_paths = true;
    }
    __syncthreads();
    if (have_paths)
      for (int li = 0; li < nlists; ++li)
        build_runs<R>(paths + (size_t)li * A.p_max, cnt[li], runs + (size_t)li * A.p_max, sort_tmp, sort_keys, nruns + li);

    C v[E];
    // ------------------------------------------------ one operator apply
    if (A.mode & kApply) {
      const int nin = A.adjoint ? A.nrx : A.ntx, nout = A.adjoint ? A.ntx : A.nrx;
      C* src = A.adjoint ? extT : extP;
      for (int b = 0; b < nin; ++b)
        for (int c = 0; c < NCH; ++c) {
#pragma unroll
          for (int i = 0; i < E; ++i) v[i] = reinterpret_cast<const C*>(io.v_in)[(size_t)b * MN + own(c, i)];
          write_ext<R, E, true>(src + b * blk, A, k, jw + c * E, v);
        }
      __syncthreads();
      for (int b = 0; b < nout; ++b)
        for (int c = 0; c < NCH; ++c) {
          if (A.adjoint) gather_adj<R, E, true>(src, blk, paths, runs, nruns, A, b, k, jw + c * E, v);
          else gather_fwd<R, E, true>(src, blk, paths, runs, nruns, A, b, k, jw + c * E, v);
#pragma unroll
          for (int i = 0; i < E; ++i) reinterpret_cast<C*>(io.u_out)[(size_t)b * MN + own(c, i)] = v[i];
        }
      __syncthreads();
      if (io.status && tid == 0) *io.status = status_from_bits(st);
      continue;
    }

    // ------------------------------------------------ equalisation
    if (A.mode & kCG) {
      const R lam = (R)io.lam;
      // y_r -> extT (its quasi-periodic extension); embedded pilot read off and removed
      for (int r = 0; r < A.nrx; ++r) {
        if (A.y_is_dd) {
          const C* yd = reinterpret_cast<const C*>(io.y_data) + (size_t)r * MN;
          for (int c = 0; c < NCH; ++c) {
#pragma unroll
            for (int i = 0; i < E; ++i) v[i] = yd[own(c, i)];
            write_ext<R, E, true>(extT + r * blk, A, k, jw + c * E, v);
          }
          continue;
        }
        load_grid(io.y_data + (size_t)r * in_bytes);
        dzt_inplace<R>(stage, A, radix);
        if (A.pilot_mode == ZOTFS_PILOT_EMBEDDED) {
          if ((A.mode & kEstimate) && !have_paths) {
            int trunc;
            const int P = readoff_compact<R, EW>(stage, A, (R)io.theta, io.a_pilot, paths, S, gout, 0, trunc);
            if (tid == 0) cnt[0] = P;
            if (trunc) st |= kStTrunc;
            __syncthreads();
            build_runs<R>(paths, cnt[0], runs, sort_tmp, sort_keys, nruns);
          }
          for (int p = tid; p < cnt[0]; p += T) {
            const PathRec rec = paths[p];
            const int kr = (A.K0 + rec.dk) & (M - 1), lr = (A.L0 + rec.dl) & (N - 1);
            const int Acol = kr - rec.dk;
            const int nw = Acol >> logM;
            C val = cmul(rec.h, tw<R>(A, (size_t)((rec.dl * Acol) & (MN - 1))));
            val = cmul(val, tw<R>(A, (size_t)(((nw * A.L0) << logM) & (MN - 1))));
            val = cscale(val, (R)(io.a_pilot * A.sqrtN));
            C* y = stage + (size_t)bitrev(lr, A.logN) * M + kr;
            *y = csub(*y, val);
          }
          __syncthreads();
        }
        for (int c = 0; c < NCH; ++c) {
#pragma unroll
          for (int i = 0; i < E; ++i)
            v[i] = cscale(stage[(size_t)bitrev(jw + c * E + i, A.logN) * M + k], (R)A.inv_sqrtN);
          write_ext<R, E, true>(extT + r * blk, A, k, jw + c * E, v);
        }
      }
      __syncthreads();

      // b = H^H y;  c = b, p = b, x = 0, c_n = ||c||^2
      R part = 0;
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c) {
          gather_adj<R, E, true>(extT, blk, paths, runs, nruns, A, t, k, jw + c * E, v);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            Cv[o] = v[i];
            Pv[o] = v[i];
            Xv[o] = Cx<R>::make(0, 0);
            part = fma(v[i].x, v[i].x, fma(v[i].y, v[i].y, part));
          }
          write_ext<R, E, true>(extP + t * blk, A, k, jw + c * E, v);
        }
      double cn = block_sum_to_thread0(part, S);
      const double stop_at = io.eps2 > 0.0 ? io.eps2 * cn : -1.0;  // eps^2 ||b||^2 (thread 0)
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
        __syncthreads();
        // a = H^H t + lambda p;  Re(p^H a)
        part = 0;
        for (int t = 0; t < A.ntx; ++t)
          for (int c = 0; c < NCH; ++c) {
            gather_adj<R, E, true>(extT, blk, paths, runs, nruns, A, t, k, jw + c * E, v);
#pragma unroll
            for (int i = 0; i < E; ++i) {
              const size_t o = (size_t)t * MN + own(c, i);
              const C pv = Pv[o];
              v[i].x = fma(lam, pv.x, v[i].x);
              v[i].y = fma(lam, pv.y, v[i].y);
              part = fma(pv.x, v[i].x, fma(pv.y, v[i].y, part));
              Vv[o] = v[i];
            }
          }
        const double pa = block_sum_to_thread0(part, S);
        if (tid == 0) S->fsc[0] = cg_ratio<R>(cn, pa);
        __syncthreads();
        const R alpha = (R)S->fsc[0];
        part = 0;
        for (int t = 0; t < A.ntx; ++t)
          for (int c = 0; c < NCH; ++c) {
#pragma unroll
            for (int i = 0; i < E; ++i) {
              const size_t o = (size_t)t * MN + own(c, i);
              const C pv = Pv[o], av = Vv[o];
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
        const double cn_new = block_sum_to_thread0(part, S);
        if (tid == 0) {
          S->fsc[1] = cg_ratio<R>(cn_new, cn);
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
                C pv = Pv[o];
                pv.x = fma(beta, pv.x, cv.x);
                pv.y = fma(beta, pv.y, cv.y);
                Pv[o] = pv;
                v[i] = pv;
              }
              write_ext<R, E, true>(extP + t * blk, A, k, jw + c * E, v);
            }
          __syncthreads();
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
    } else if (A.mode & kLoadX) {
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            Xv[o] = reinterpret_cast<const C*>(io.x_in)[o];
          }
    }

    // ------------------------------------------------ demapping
    if ((A.mode & kDemap) && (io.llr || io.bits)) {
      const R inv_lam = (R)1 / (R)io.lam;
      const int bps = io.bps;
      uint8_t* lab = reinterpret_cast<uint8_t*>(stage);
      __syncthreads();
      for (int t = 0; t < A.ntx; ++t)
        for (int c = 0; c < NCH; ++c)
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const size_t o = (size_t)t * MN + own(c, i);
            const int q = (int)(o - (size_t)t * MN);
            float2 l01, l23, l45;
            const int hard = qam_llr_regs<R>(Xv[o], bps, (R)io.pam_d, inv_lam, l01, l23, l45);
            lab[o] = (uint8_t)hard;
            if (io.llr) {
              float2* ol = reinterpret_cast<float2*>(io.llr + ((size_t)t * MN + q) * bps);
              ol[0] = l01;
              if (bps > 2) ol[1] = l23;
              if (bps > 4) ol[2] = l45;
            }
          }
      __syncthreads();
      if (io.bits) {
        const int bytes_per_block = MN * bps / 8;
        const int total = A.ntx * bytes_per_block;
        for (int B = tid; B < total; B += T) {
          const int t = B / bytes_per_block;
          const int b0 = (B - t * bytes_per_block) * 8;
          int byte = 0;
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int bit = b0 + j;
            const int q = bit / bps, jj = bit - q * bps;
            byte |= ((lab[(size_t)t * MN + q] >> (bps - 1 - jj)) & 1) << j;
          }
          io.bits[B] = (uint8_t)byte;
        }
      }
      __syncthreads();
    }
    publish_status(A, io.status, st);
  }
}

}  // namespace zotfs
