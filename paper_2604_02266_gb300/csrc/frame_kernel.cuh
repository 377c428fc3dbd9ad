// The persistent frame kernel: CTAs pull frame indices from a device counter and run the
// requested stages of the receiver on each frame entirely in shared memory and registers.
//
// Template parameters: E = Doppler rows owned per thread and antenna block (MN = T E),
// NB = maximum antenna blocks (max(n_rx, n_tx)) the register arrays hold, TMAX / MINB =
// launch bounds.  Per thread the CG keeps x, c, p and one operator output for its NB*E
// elements in registers; the shared memory holds the path lists and one ext buffer that
// alternately carries p's and t = H p's quasi-periodic extension.
#pragma once

#include <type_traits>

#include "frame_engine.cuh"

namespace zotfs {

// Warp partials of `v` summed in FP64 by thread 0 (pairwise, eight partials at a time, in a
// fixed order); the total is valid in thread 0 only.  One barrier; the caller publishes
// results with another.
template <typename R>
__device__ __forceinline__ double block_sum_to_thread0(R v, SharedHdr* S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) S->red[warp] = (double)v;
  frame_sync();
  double d = 0.0;
  if (threadIdx.x == 0) {
    for (int b = 0; b < nwarps; b += 8) {
      double r[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) r[i] = b + i < nwarps ? S->red[b + i] : 0.0;
      d += ((r[0] + r[1]) + (r[2] + r[3])) + ((r[4] + r[5]) + (r[6] + r[7]));
    }
  }
  return d;
}

// Resolve frame f's buffers: strided views of the call's tensors, or its descriptor.
// csz = bytes of one complex element of the arithmetic precision.
__device__ __forceinline__ FrameIO frame_io(const FrameArgs& A, int f, int csz) {
  FrameIO io;
  const int MN = A.M * A.N, nl = A.nrx * A.ntx;
  const size_t in_bytes = (size_t)MN * dtype_bytes(A.in_dtype);
  if (A.descs) {
    const zotfs_frame_desc& d = A.descs[A.frame_ids[f]];
    io.y_pilot = static_cast<const char*>(d.y_pilot);
    io.y_data = static_cast<const char*>(d.y_data);
    io.v_in = nullptr;
    io.x_in = nullptr;
    io.lam = d.noise_var;
    io.theta = d.theta;
    io.iters = d.iters;
    io.eps2 = (double)d.cg_eps * (double)d.cg_eps;
    io.bps = 31 - __clz(d.qam);
    io.pam_d = A.pam_d_hb[(io.bps >> 1) & 3];  // filled on the host: no per-thread FP64 sqrt / divide
    io.a_pilot = d.a_pilot;
    io.x_hat = reinterpret_cast<char*>(d.x_hat);
    io.llr = d.llr;
    io.bits = d.bits;
    io.u_out = nullptr;
    io.paths.count = d.path_count;
    io.paths.status = nullptr;
    io.paths.dk = d.path_dk;
    io.paths.dl = d.path_dl;
    io.paths.h = d.path_h;
    io.paths.tap_dtype = ZOTFS_C64;
    io.paths.invalid = 0;
    io.status = A.status ? A.status + A.frame_ids[f] : nullptr;
    return io;
  }
  if (A.frame_ids) f = A.frame_ids[f];
  io.y_pilot = A.y_pilot ? static_cast<const char*>(A.y_pilot) + (size_t)f * A.ntx * A.nrx * in_bytes : nullptr;
  const size_t data_bytes = A.y_is_dd ? (size_t)MN * csz : in_bytes;
  io.y_data = A.y_data ? static_cast<const char*>(A.y_data) + (size_t)f * A.nrx * data_bytes : nullptr;
  const int nin = (A.mode & kApply) ? (A.adjoint ? A.nrx : A.ntx) : 0;
  const int nout = (A.mode & kApply) ? (A.adjoint ? A.ntx : A.nrx) : 1;
  io.v_in = A.v_in ? static_cast<const char*>(A.v_in) + (size_t)f * nin * MN * csz : nullptr;
  io.x_in = A.x_in ? static_cast<const char*>(A.x_in) + (size_t)f * A.ntx * MN * csz : nullptr;
  io.lam = A.noise_var ? A.noise_var[f] : 0.f;
  io.theta = A.theta ? A.theta[f] : 0.f;
  io.iters = A.iters;
  io.eps2 = A.eps2;
  io.bps = A.bps;
  io.pam_d = A.pam_d;
  io.a_pilot = A.a_pilot;
  io.x_hat = A.x_hat ? static_cast<char*>(A.x_hat) + (size_t)f * A.ntx * MN * csz : nullptr;
  io.llr = A.llr ? A.llr + (size_t)f * A.ntx * MN * A.bps : nullptr;
  io.bits = A.bits ? A.bits + (size_t)f * A.ntx * MN * A.bps / 8 : nullptr;
  io.u_out = A.u_out ? static_cast<char*>(A.u_out) + (size_t)f * nout * MN * csz : nullptr;
  int ls = f;  // the frame's list set
  io.paths.invalid = 0;
  if (A.path_ids) {
    ls = A.path_ids[f];
    if (ls < 0 || ls >= A.n_path_sets) {
      io.paths.invalid = 1;
      ls = 0;
    }
  }
  io.paths.count = A.pcount ? A.pcount + (size_t)ls * nl : nullptr;
  io.paths.status = A.pstatus ? A.pstatus + (size_t)ls * nl : nullptr;
  io.paths.dk = A.pdk ? A.pdk + (size_t)ls * nl * A.p_max : nullptr;
  io.paths.dl = A.pdl ? A.pdl + (size_t)ls * nl * A.p_max : nullptr;
  io.paths.h = A.ph ? static_cast<char*>(A.ph) + (size_t)ls * nl * A.p_max * dtype_bytes(A.tap_dtype) : nullptr;
  io.paths.tap_dtype = A.tap_dtype;
  io.status = A.status ? A.status + f : nullptr;
  return io;
}

// COEF: keep per-(path, column) coefficient tables in shared memory for the frame's lists
// (forward and adjoint forms), so the CG's gathers read one value per path instead of a path
// record, a twiddle-table entry and a complex product.
// PACK: the kernel may be launched with a two-dimensional block of blockDim.y frames per CTA;
// without it the block is one-dimensional, which the compiler is told (the frame-scope barriers
// and the shared-memory base then reduce to their one-frame forms at no register cost).
template <typename R, int E, int NB, int TMAX, int MINB, bool COEF, bool PACK>
__global__ void __launch_bounds__(TMAX, MINB) frame_kernel(const __grid_constant__ FrameArgs A, int radix) {
  using C = typename Cx<R>::C;
  using PathRec = PathRecT<R>;
  if constexpr (!PACK) {
    __builtin_assume(blockDim.y == 1);
    __builtin_assume(threadIdx.y == 0);
  }
  extern __shared__ __align__(128) unsigned char smem_all[];
  // frames packed into one CTA (2D block): row threadIdx.y owns its own slice of shared memory
  const size_t row_bytes =
      (frame_smem_bytes(A.M, A.N, E, A.nrx, A.ntx, A.p_max, (int)sizeof(R), COEF) + 127) & ~size_t(127);
  unsigned char* smem = smem_all + (size_t)threadIdx.y * row_bytes;
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
  C* coefF = nullptr;
  C* coefA = nullptr;
  if constexpr (COEF) {
    coefF = reinterpret_cast<C*>(smem + off);
    coefA = coefF + (size_t)nlists * A.p_max * A.M;
    off += coef_table_bytes(A.M, A.nrx, A.ntx, A.p_max, (int)sizeof(R));
  }
  // sorted path lists -> runs (and coefficient tables); all threads
  auto finalize_lists = [&]() {
    for (int li = 0; li < nlists; ++li) {
      PathRec* pl = paths + (size_t)li * A.p_max;
      const int P = cnt[li];
      if constexpr (COEF) {  // the coefficient tables are built while warp 0 cuts the runs
        const size_t o = (size_t)li * A.p_max * A.M;
        build_runs<R>(pl, P, runs + (size_t)li * A.p_max, sort_tmp, sort_keys, nruns + li,
                      [&](int first, int stride) { coef_tables<R>(pl, P, A, coefF + o, coefA + o, first, stride); });
      } else {
        build_runs<R>(pl, P, runs + (size_t)li * A.p_max, sort_tmp, sort_keys, nruns + li);
      }
    }
  };
  C* ext = reinterpret_cast<C*>(smem + off);

  const int M = A.M, N = A.N, MN = M * N, logM = A.logM;
  const size_t blk = ext_block_elems(M, N, E);
  const int tid = threadIdx.x;
  const int k = tid & (M - 1);
  const int j0 = (tid >> logM) * E;
  const size_t in_bytes = (size_t)MN * dtype_bytes(A.in_dtype);
  const bool write_paths = (A.mode & kWritePaths) != 0;

  if (tid == 0) mbar_init(&S->mbar, 1);
  frame_sync();
  uint32_t phase = 0;

  for (;;) {
    if (tid == 0) S->isc[0] = atomicAdd(A.work_counter, 1);
    frame_sync();
    const int f = S->isc[0];
    frame_sync();
    if (f >= A.n_frames) break;
    const FrameIO io = frame_io(A, f, (int)sizeof(C));
    const PathIO* gout = (write_paths && io.paths.count) ? &io.paths : nullptr;
    int st = 0;

    // ------------------------------------------------ Zak transform only
    if (A.mode & kDzt) {
      if (!stage_grid<R, E>(ext, io.y_data, MN, A.in_dtype, &S->mbar, phase)) {
        st |= kStTimeout;
      } else {
        dzt_inplace<R>(ext, A, radix);
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int l = j0 + i;
          reinterpret_cast<C*>(io.u_out)[(size_t)l * M + k] = cscale(ext[(size_t)bitrev(l, A.logN) * M + k], (R)A.inv_sqrtN);
        }
      }
      if (io.status && tid == 0) *io.status = status_from_bits(st);
      if (st & kStTimeout) break;
      continue;
    }

    // ------------------------------------------------ path lists (estimated or loaded)
    bool have_paths = false;
    if ((A.mode & kEstimate) && A.pilot_mode == ZOTFS_PILOT_SEPARATE) {
      for (int t = 0; t < A.ntx && !(st & kStTimeout); ++t) {
        for (int r = 0; r < A.nrx; ++r) {
          const char* src = io.y_pilot + ((size_t)t * A.nrx + r) * in_bytes;  // pilot frames [t][r]
          if (!stage_grid<R, E>(ext, src, MN, A.in_dtype, &S->mbar, phase)) {
            st |= kStTimeout;
            break;
          }
          dzt_inplace<R>(ext, A, radix);
          const int li = r * A.ntx + t;
          int trunc;
          const int P = readoff_compact<R, E>(ext, A, (R)io.theta, io.a_pilot, paths + (size_t)li * A.p_max, S, gout, li, trunc);
          if (tid == 0) cnt[li] = P;
          if (trunc) st |= kStTrunc;
        }
      }
      have_paths = true;
    } else if ((A.mode & kEstimate) && A.pilot_mode == ZOTFS_PILOT_EMBEDDED && !(A.mode & kCG)) {
      // estimation only, embedded pilot: read off the data frame itself
      if (!stage_grid<R, E>(ext, io.y_data, MN, A.in_dtype, &S->mbar, phase)) {
        st |= kStTimeout;
      } else {
        dzt_inplace<R>(ext, A, radix);
        int trunc;
        const int P = readoff_compact<R, E>(ext, A, (R)io.theta, io.a_pilot, paths, S, gout, 0, trunc);
        if (tid == 0) cnt[0] = P;
        if (trunc) st |= kStTrunc;
      }
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
    frame_sync();
    if (st & kStTimeout) {
      if (io.status && tid == 0) *io.status = status_from_bits(st);
      break;  // barrier phases are no longer trustworthy: stop this CTA
    }
    if (have_paths) finalize_lists();

    C v[NB][E];  // operator outputs / inputs per antenna block

    // ------------------------------------------------ one operator apply
    if (A.mode & kApply) {
      const int nin = A.adjoint ? A.nrx : A.ntx, nout = A.adjoint ? A.ntx : A.nrx;
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < nin) {
#pragma unroll
          for (int i = 0; i < E; ++i) v[b][i] = reinterpret_cast<const C*>(io.v_in)[(size_t)b * MN + (size_t)(j0 + i) * M + k];
          write_ext<R, E>(ext + b * blk, A, k, j0, v[b]);
        }
      frame_sync();
#pragma unroll
      for (int b = 0; b < NB; ++b)
        if (b < nout) {
          if (A.adjoint) gather_adj<R, E, false, COEF>(ext, blk, paths, runs, nruns, A, b, k, j0, v[b], coefA);
          else gather_fwd<R, E, false, COEF>(ext, blk, paths, runs, nruns, A, b, k, j0, v[b], coefF);
#pragma unroll
          for (int i = 0; i < E; ++i) reinterpret_cast<C*>(io.u_out)[(size_t)b * MN + (size_t)(j0 + i) * M + k] = v[b][i];
        }
      frame_sync();
      if (io.status && tid == 0) *io.status = status_from_bits(st);
      continue;
    }

    C x[NB][E];
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
      for (int i = 0; i < E; ++i) x[b][i] = Cx<R>::make(0, 0);

    // ------------------------------------------------ equalisation
    if (A.mode & kCG) {
      const R lam = (R)io.lam;
      // received DD grids y_r -> registers (and the embedded pilot's read-off)
      if (A.y_is_dd) {
        const C* yd = reinterpret_cast<const C*>(io.y_data);
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < A.nrx)
#pragma unroll
            for (int i = 0; i < E; ++i) v[r][i] = yd[(size_t)r * MN + (size_t)(j0 + i) * M + k];
      } else {
        for (int r = 0; r < A.nrx; ++r) {
          if (!stage_grid<R, E>(ext + r * blk, io.y_data + (size_t)r * in_bytes, MN, A.in_dtype, &S->mbar, phase)) {
            st |= kStTimeout;
            break;
          }
          dzt_inplace<R>(ext + r * blk, A, radix);
        }
        if (st & kStTimeout) {
          if (io.status && tid == 0) *io.status = status_from_bits(st);
          break;
        }
        if (A.pilot_mode == ZOTFS_PILOT_EMBEDDED) {
          if ((A.mode & kEstimate) && !have_paths) {
            int trunc;
            const int P = readoff_compact<R, E>(ext, A, (R)io.theta, io.a_pilot, paths, S, gout, 0, trunc);
            if (tid == 0) cnt[0] = P;
            if (trunc) st |= kStTrunc;
            frame_sync();
            finalize_lists();
          }
          // remove the pilot's response a_pilot H e_(K0,L0) (grid still scaled by sqrt(N))
          for (int p = tid; p < cnt[0]; p += blockDim.x) {
            const PathRec rec = paths[p];
            const int kr = (A.K0 + rec.dk) & (M - 1), lr = (A.L0 + rec.dl) & (N - 1);
            const int Acol = kr - rec.dk;
            const int nw = Acol >> logM;  // floor division by M
            C val = cmul(rec.h, tw<R>(A, (size_t)((rec.dl * Acol) & (MN - 1))));
            val = cmul(val, tw<R>(A, (size_t)(((nw * A.L0) << logM) & (MN - 1))));
            val = cscale(val, (R)(io.a_pilot * A.sqrtN));
            C* y = ext + (size_t)bitrev(lr, A.logN) * M + kr;
            *y = csub(*y, val);
          }
          frame_sync();
        }
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < A.nrx)
#pragma unroll
            for (int i = 0; i < E; ++i)
              v[r][i] = cscale(ext[r * blk + (size_t)bitrev(j0 + i, A.logN) * M + k], (R)A.inv_sqrtN);
        frame_sync();
      }
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < A.nrx) write_ext<R, E>(ext + r * blk, A, k, j0, v[r]);
      frame_sync();

      // b = H^H y;  c = b, p = b, x = 0, c_n = ||c||^2   (Algorithm 1, initialisation)
      C c[NB][E], p[NB][E];
      R part = 0;
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < A.ntx) {
          gather_adj<R, E, false, COEF>(ext, blk, paths, runs, nruns, A, t, k, j0, c[t], coefA);
#pragma unroll
          for (int i = 0; i < E; ++i) {
            p[t][i] = c[t][i];
            part = fma(c[t][i].x, c[t][i].x, fma(c[t][i].y, c[t][i].y, part));
          }
        }
      double cn = block_sum_to_thread0(part, S);  // valid in thread 0
      const double stop_at = io.eps2 > 0.0 ? io.eps2 * cn : -1.0;  // eps^2 ||b||^2 (thread 0)
      if (tid == 0) {
        S->isc[1] = isfinite(cn) ? 0 : 1;
        S->isc[4] = cn <= stop_at ? 1 : 0;
      }
      frame_sync();  // all gathers of y_ext done; flags published
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < A.ntx) write_ext<R, E>(ext + t * blk, A, k, j0, p[t]);
      frame_sync();

      // the stopping test's flag is read after the barrier that follows the p update
      for (int it = 0; it < io.iters && !S->isc[4]; ++it) {
        // t = H p
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < A.nrx) gather_fwd<R, E, false, COEF>(ext, blk, paths, runs, nruns, A, r, k, j0, v[r], coefF);
        frame_sync();
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < A.nrx) write_ext<R, E>(ext + r * blk, A, k, j0, v[r]);
        frame_sync();
        // a = H^H t + lambda p;  Re(p^H a)
        part = 0;
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < A.ntx) {
            gather_adj<R, E, false, COEF>(ext, blk, paths, runs, nruns, A, t, k, j0, v[t], coefA);
#pragma unroll
            for (int i = 0; i < E; ++i) {
              v[t][i].x = fma(lam, p[t][i].x, v[t][i].x);
              v[t][i].y = fma(lam, p[t][i].y, v[t][i].y);
              part = fma(p[t][i].x, v[t][i].x, fma(p[t][i].y, v[t][i].y, part));
            }
          }
        const double pa = block_sum_to_thread0(part, S);
        if (tid == 0) S->fsc[0] = cg_ratio<R>(cn, pa);  // alpha, FP64
        frame_sync();
        const R alpha = (R)S->fsc[0];
        // x += alpha p;  c -= alpha a;  c_n' = ||c||^2
        part = 0;
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < A.ntx)
#pragma unroll
            for (int i = 0; i < E; ++i) {
              x[t][i].x = fma(alpha, p[t][i].x, x[t][i].x);
              x[t][i].y = fma(alpha, p[t][i].y, x[t][i].y);
              c[t][i].x = fma(-alpha, v[t][i].x, c[t][i].x);
              c[t][i].y = fma(-alpha, v[t][i].y, c[t][i].y);
              part = fma(c[t][i].x, c[t][i].x, fma(c[t][i].y, c[t][i].y, part));
            }
        const double cn_new = block_sum_to_thread0(part, S);
        if (tid == 0) {
          S->fsc[1] = cg_ratio<R>(cn_new, cn);  // beta, FP64
          if (!isfinite(cn_new)) S->isc[1] = 1;
          if (cn_new <= stop_at) S->isc[4] = 1;
          cn = cn_new;
        }
        frame_sync();
        const R beta = (R)S->fsc[1];
        // p = c + beta p
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < A.ntx)
#pragma unroll
            for (int i = 0; i < E; ++i) {
              p[t][i].x = fma(beta, p[t][i].x, c[t][i].x);
              p[t][i].y = fma(beta, p[t][i].y, c[t][i].y);
            }
        if (it + 1 < io.iters) {
#pragma unroll
          for (int t = 0; t < NB; ++t)
            if (t < A.ntx) write_ext<R, E>(ext + t * blk, A, k, j0, p[t]);
          frame_sync();
        }
      }
      if (S->isc[1]) st |= kStNonFinite;
      if ((A.mode & kWriteX) && io.x_hat) {
#pragma unroll
        for (int t = 0; t < NB; ++t)
          if (t < A.ntx)
#pragma unroll
            for (int i = 0; i < E; ++i) reinterpret_cast<C*>(io.x_hat)[(size_t)t * MN + (size_t)(j0 + i) * M + k] = x[t][i];
      }
    } else if (A.mode & kLoadX) {
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < A.ntx)
#pragma unroll
          for (int i = 0; i < E; ++i) x[t][i] = reinterpret_cast<const C*>(io.x_in)[(size_t)t * MN + (size_t)(j0 + i) * M + k];
    }

    // ------------------------------------------------ demapping
    if ((A.mode & kDemap) && (io.llr || io.bits)) {
      const R inv_lam = (R)1 / (R)io.lam;
      const int bps = io.bps;
      // x_hat is staged in shared memory and demapped by a plain loop, so only one
      // constellation's unrolled code is live at a time
      uint8_t* lab = reinterpret_cast<uint8_t*>(ext);  // labels, bit j of the symbol at bit j
      C* xs = reinterpret_cast<C*>(ext) + (A.ntx * MN + sizeof(C) - 1) / sizeof(C);
      frame_sync();  // ext no longer read by anyone
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < A.ntx)
#pragma unroll
          for (int i = 0; i < E; ++i) xs[(size_t)t * MN + (j0 + i) * M + k] = x[t][i];
      frame_sync();
      const R pd = (R)io.pam_d;
      auto demap_all = [&](auto hb) {
        constexpr int HB = decltype(hb)::value;
#pragma unroll 1
        for (int e = tid; e < A.ntx * MN; e += blockDim.x) {
          float2 l01, l23, l45;
          const int hard = qam_llr_c<R, HB>(xs[e], pd, inv_lam, l01, l23, l45);
          lab[e] = (uint8_t)(__brev((unsigned)hard) >> (32 - 2 * HB));  // label bits LSB first
          if (io.llr) {
            float2* o = reinterpret_cast<float2*>(io.llr + (size_t)e * (2 * HB));
            o[0] = l01;
            if (HB > 1) o[1] = l23;
            if (HB > 2) o[2] = l45;
          }
        }
      };
      if (bps == 2) demap_all(std::integral_constant<int, 1>{});
      else if (bps == 4) demap_all(std::integral_constant<int, 2>{});
      else demap_all(std::integral_constant<int, 3>{});
      frame_sync();
      if (io.bits) {
        // 8 consecutive symbols fill exactly bps bytes (bits LSB first, symbol by symbol)
        const int groups = A.ntx * MN / 8;
        for (int g = tid; g < groups; g += blockDim.x) {
          const unsigned long long l8 = reinterpret_cast<const unsigned long long*>(lab)[g];
          unsigned long long w = 0;
#pragma unroll
          for (int s8 = 0; s8 < 8; ++s8) w |= ((l8 >> (8 * s8)) & 0xffull) << (bps * s8);
          uint8_t* o = io.bits + (size_t)g * bps;
          if ((reinterpret_cast<uintptr_t>(o) & 1u) == 0) {
            uint16_t* o2 = reinterpret_cast<uint16_t*>(o);
            for (int h = 0; h < bps / 2; ++h) o2[h] = (uint16_t)(w >> (16 * h));
          } else {
            for (int h = 0; h < bps; ++h) o[h] = (uint8_t)(w >> (8 * h));
          }
        }
      }
      frame_sync();
    }
    publish_status(A, io.status, st);
  }
}

}  // namespace zotfs
