// Frame-resident Zak-OTFS receiver engine: one CTA owns one frame at a time and keeps
// everything it needs in shared memory.
//
// Work split.  A CTA of T threads handles an M x N grid (times the antenna blocks); thread
// t owns column k = t mod M and the E = MN/T consecutive Doppler rows
// [j0, j0 + E), j0 = (t / M) E, of every block.  The per-element CG vectors (x, c, p and the
// operator outputs) live in that thread's registers.
//
// Shared-memory vector layout ("ext").  The vector an operator gathers from is stored as
// its quasi-periodic extension (footnote of Eq. y_channel_DD):
//     X_ext[A, r] = X[<A>_M, <r>_N] exp(j2pi floor(A/M) <r>_N / N)
// for columns A in [-M/2, 3M/2) and rows r in [0, N + E + 3), column-major: element (A, r)
// at (A + M/2) CS + r with column stride CS = N + E + 3 (odd, so the 32 consecutive columns
// a warp reads fall in distinct banks).
// With it, path p's contribution to output (k, l) -- the twisted shift of Sec. IV-B with
// map Eq. map_chMatDD_col, wrap count n and phase phi -- becomes a plain shifted read:
//     (H v)[k, l]   = sum_p h_p W[dl (k - dk)]      X_ext[k - dk, l - dl]
//     (H^H u)[k, l] = sum_p conj(h_p W[dl k])       U_ext[k + dk, l + dl]
// with W[t] = exp(j2pi t/(MN)) and (dk, dl) = (k_p - K0, l_p - L0).  The quasi-periodic
// phase exp(j2pi n l_{p,q} / N) of the paper's phi is carried by the stored halo columns,
// the term (l_p - L0) A by the per-(path, column) coefficient, so each gather is one
// shared load at a constant offset and two packed FMAs.  Rows are periodic (no phase), so
// E + 3 halo rows let a thread read a window of up to E + 3 consecutive source rows without a
// wrap.  Paths are applied in runs: paths with equal dk and consecutive dl read overlapping
// rows, so a run of L <= 4 such paths loads one (L + E - 1)-row window into registers and
// applies all L paths from it.
//
// Everything is templated on the arithmetic type R (float, or double for FP64 plans).
#pragma once

#include <type_traits>

#include "common.cuh"

namespace zotfs {

// A run of paths (indices start .. start + len - 1 of a list sorted by (dk, dl)) with equal
// dk and consecutive dl = dl0, dl0 + 1, ...
struct RunRec {
  short start, len, dk, dl0;
};
constexpr int kMaxRun = 4;

template <typename R>
struct PathRecT {             // one dominant path in shared memory
  typename Cx<R>::C h;        // h_p
  typename Cx<R>::C hf;       // h_p * W[-dl dk]: forward coefficient is hf * W[dl k]
  int dk, dl;                 // centred offsets k_p - K0, l_p - L0
  int pad0, pad1;
};

enum FrameMode : int {
  kEstimate = 1,     // pilots -> path lists in shared memory
  kLoadPaths = 2,    // path lists from global memory
  kCG = 4,           // data frame -> x_hat
  kDemap = 8,        // x_hat -> LLRs / bits
  kWriteX = 16,      // store x_hat
  kWritePaths = 32,  // store the estimated path lists
  kApply = 64,       // one operator apply u = H v or H^H v
  kLoadX = 128,      // x_hat from global memory (demap only)
  kDzt = 256         // Zak transform only (y_td -> y_dd)
};

// per-frame status bits, folded into one zotfs_status at the end (most severe wins)
enum StatusBit : int { kStTrunc = 1, kStInval = 2, kStNonFinite = 4, kStTimeout = 8 };
__device__ __forceinline__ int status_from_bits(int b) {
  if (b & kStTimeout) return ZOTFS_ETIMEOUT;
  if (b & kStNonFinite) return ZOTFS_ENONFINITE;
  if (b & kStInval) return ZOTFS_EINVAL;
  if (b & kStTrunc) return ZOTFS_ETRUNCATED;
  return ZOTFS_OK;
}

struct FrameArgs {
  // geometry (one shape per launch)
  int M, N, logM, logN, nrx, ntx, T;
  int K0, L0, pilot_mode, guard, p_max, in_dtype, tap_dtype, qam, bps;
  double a_pilot, inv_sqrtN, sqrtN, pam_d;
  double pam_d_hb[4];  // PAM half-spacing by bits per axis (1: QPSK, 2: 16-QAM, 3: 64-QAM), for descriptors
  const void* W;    // W[t] = exp(j2pi t/(MN)), t in [0, MN), complex R
  const void* Tab;  // Tab[(dl + N/2) M + k] = W[(dl k) mod MN], complex R
  // work distribution
  int n_frames, mode;
  int* work_counter;
  // inputs (complex vectors are complex R unless a dtype says otherwise)
  const void* y_pilot;
  const void* y_data;
  int y_is_dd;
  const float* noise_var;
  const float* theta;
  int iters;
  double eps2;  // CG stopping test: stop once ||c||^2 <= eps2 ||b||^2; 0 = off
  const void* v_in;
  int adjoint;
  const void* x_in;
  // path lists in global memory: read with kLoadPaths, written with kWritePaths.  With
  // path_ids (kLoadPaths), frame f reads list set path_ids[f] of n_path_sets (pilot reuse:
  // several data frames equalised with the lists of one pilot frame); else set f.
  const int32_t* path_ids;
  int n_path_sets;
  int32_t* pcount;
  int32_t* pstatus;
  int16_t* pdk;
  int16_t* pdl;
  void* ph;
  // outputs
  void* x_hat;
  float* llr;
  uint8_t* bits;
  int32_t* status;
  void* u_out;
  // uneven batches: per-frame buffers come from descriptors (frame f of this launch is
  // descriptor frame_ids[f]); single-shape calls: frame_ids, if set, is the order in which
  // the CTAs take the frames (a permutation of [0, n_frames))
  const zotfs_frame_desc* descs;
  const int* frame_ids;
  // status lives in host-mapped memory that the host polls: each frame's outputs are made
  // visible system-wide before its status is stored (serving: per-frame completion)
  int status_fence;
};

// Store a frame's final status (thread 0).  With A.status_fence every thread of the block has
// finished the frame's outputs (barrier) and they are fenced at system scope first, so a host
// that sees the status may read the outputs.
__device__ __forceinline__ void publish_status(const FrameArgs& A, int32_t* status, int st_bits) {
  if (A.status_fence) frame_sync();
  if (status && threadIdx.x == 0) {
    if (A.status_fence) {
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(status) = status_from_bits(st_bits);
    } else {
      *status = status_from_bits(st_bits);
    }
  }
}

// Global-memory path lists of one frame: list li (= r * n_tx + t) has count[li] entries at
// [li * p_max, li * p_max + count[li]) of dk, dl and h.
struct PathIO {
  int32_t* count;
  int32_t* status;  // may be NULL
  int16_t* dk;
  int16_t* dl;
  void* h;
  int tap_dtype;
  int invalid;      // the frame named a list set outside the call's: load nothing, flag it
};

// Everything one frame reads and writes, resolved at the start of the frame.
struct FrameIO {
  const char* y_pilot;  // pilot TD grids [t][r] of this frame (separate pilot mode)
  const char* y_data;   // data grids [r] (TD, or DD when y_is_dd)
  const char* v_in;     // operator input [b][MN] (apply mode)
  const char* x_in;     // x_hat input [t][MN] (demap-only mode)
  float lam, theta;
  int iters;
  double eps2;          // CG stopping test of this frame (0 = fixed iterations)
  int bps;              // bits per QAM symbol of this frame
  double pam_d;         // PAM half-spacing of this frame's QAM (unit mean energy)
  double a_pilot;       // pilot amplitude divided out of the read-off
  char* x_hat;          // [t][MN] or NULL
  float* llr;           // [t][MN][bps] or NULL
  uint8_t* bits;        // [t][MN bps / 8] or NULL
  char* u_out;          // [b][MN] (apply / DZT modes)
  PathIO paths;         // lists of this frame (in for kLoadPaths, out for kWritePaths)
  int32_t* status;      // this frame's status word or NULL
};

struct SharedHdr {       // fixed part of the dynamic shared memory
  uint64_t mbar;
  double dsc[4];
  double fsc[4];
  int isc[6];            // [4]: the CG stopping test has fired
  int scan[40];
  double red[32];
  int hist[128];         // radix-select histogram of the read-off (kept zero between uses)
};

// Shared-memory bytes needed by a frame kernel launch (host and device agree on this).
__host__ __device__ __forceinline__ int ext_rows(int N, int E) { return N + E + 3; }  // = column stride CS
__host__ __device__ __forceinline__ size_t ext_block_elems(int M, int N, int E) {
  return (size_t)ext_rows(N, E) * (size_t)(2 * M);
}
// Bytes of the per-(path, delay column) coefficient tables: forward and adjoint forms, one
// complex value per path and column k for every antenna pair.
__host__ __device__ __forceinline__ size_t coef_table_bytes(int M, int nrx, int ntx, int p_max, int real_bytes) {
  return ((size_t)2 * nrx * ntx * p_max * M * 2 * real_bytes + 127) & ~size_t(127);
}
__host__ __device__ __forceinline__ size_t frame_smem_bytes(int M, int N, int E, int nrx, int ntx, int p_max,
                                                            int real_bytes, bool coef = false) {
  size_t hdr = (sizeof(SharedHdr) + 127) & ~size_t(127);
  const size_t rec = (size_t)4 * real_bytes + 16;  // PathRecT<R>
  size_t paths = (size_t)nrx * ntx * p_max * rec + (size_t)nrx * ntx * sizeof(int) * 2;
  paths = (paths + 127) & ~size_t(127);
  paths += ((size_t)nrx * ntx * p_max * sizeof(RunRec) + 127) & ~size_t(127);  // run tables
  paths += ((size_t)p_max * rec + 127) & ~size_t(127);                        // sort scratch
  paths += ((size_t)((p_max + 3) & ~3) * sizeof(int) + 127) & ~size_t(127);     // sort keys
  if (coef) paths += coef_table_bytes(M, nrx, ntx, p_max, real_bytes);
  int nb = nrx > ntx ? nrx : ntx;
  size_t ext = (size_t)nb * ext_block_elems(M, N, E) * 2 * real_bytes;
  return hdr + paths + ext;
}

constexpr uint32_t kMaxPolls = 1u << 22;

// Most CTAs per SM the paper-scale grid receiver launches (its scratch holds their partials).
constexpr int kGridMaxCtasPerSm = 2;

// Algorithm 1's scalar ratios alpha = c_n / Re(p^H a) and beta = c_n' / c_n from their FP64
// inner products, with the readings alpha = 0 when Re(p^H a) = 0 and beta = 0 when c_n = 0.
// For FP32 arithmetic (R = float) the quotient is only used rounded to FP32, so it is formed
// in FP64 by one Newton-Raphson step on the FP32 reciprocal of the divisor (Markstein's
// correction): r0 = 1/float(b), e = 1 - b r0, r1 = r0 + r0 e, q = a r1.  r0 carries a relative
// error |d| of about 2^-23, r1 one of d^2 < 2^-44, so q rounds to the same float as a / b
// unless a / b lies within 2^-44 (relative) of a rounding boundary.  A full FP64 division costs
// several hundred cycles on this part and sits on the CTA's critical path twice per iteration;
// this costs three dependent FP64 operations.  Divisors whose FP32 image is not a normal
// number, and FP64 plans (R = double), take the full division.
template <typename R>
__device__ __forceinline__ double cg_ratio(double a, double b) {
  if (b == 0.0) return 0.0;
  if constexpr (std::is_same<R, float>::value) {
    const float bf = (float)b;
    const float abf = fabsf(bf);
    if (abf >= 1e-30f && abf <= 1e30f) {
      const double r0 = (double)__frcp_rn(bf);
      const double e = fma(-b, r0, 1.0);
      const double r1 = fma(r0, e, r0);
      return a * r1;
    }
  }
  return a / b;
}

// ------------------------------------------------------------------ staging + DZT

// Copy one TD grid (MN complex of `dtype`) into dst[0, MN) as complex R by a bulk async
// copy (narrower storage lands in the upper part of the buffer and is widened in place).
// All threads call; returns false (uniformly) if the bounded wait gave up.
template <typename R, int E>
__device__ __forceinline__ bool stage_grid(typename Cx<R>::C* dst, const void* src, int MN, int dtype,
                                           uint64_t* bar, uint32_t& phase) {
  using C = typename Cx<R>::C;
  const int tid = threadIdx.x, T = blockDim.x;
  const uint32_t bytes = (uint32_t)MN * (uint32_t)dtype_bytes(dtype);
  const bool native = dtype == Cx<R>::kIoDtype;
  char* d = reinterpret_cast<char*>(dst) + (native ? 0 : (size_t)MN * sizeof(C) - bytes);
  frame_sync();  // earlier generic accesses to dst are complete
  if (tid == 0) {
    fence_proxy_async_smem();
    bulk_g2s(d, src, bytes, bar);
  }
  bool ok = mbar_wait_bounded(bar, phase, kMaxPolls);
  if (!ok) ok = mbar_wait_bounded(bar, phase, kMaxPolls);  // let an in-flight copy land
  phase ^= 1u;
  if (frame_sync_or(!ok)) return false;
  if (!native) {
    C tmp[E];  // MN == T * E
#pragma unroll
    for (int i = 0; i < E; ++i) tmp[i] = load_complex<C>(d, (size_t)tid + (size_t)i * T, dtype);
    frame_sync();
#pragma unroll
    for (int i = 0; i < E; ++i) dst[tid + i * T] = tmp[i];
    frame_sync();
  }
  return true;
}

template <typename R>
__device__ __forceinline__ typename Cx<R>::C tw(const FrameArgs& A, size_t idx) {
  return __ldg(reinterpret_cast<const typename Cx<R>::C*>(A.W) + idx);
}
template <typename R>
__device__ __forceinline__ typename Cx<R>::C tab(const FrameArgs& A, size_t idx) {
  return __ldg(reinterpret_cast<const typename Cx<R>::C*>(A.Tab) + idx);
}

// In-place DIF FFT along the Doppler axis of X[n][k] (n < N rows of M): afterwards row
// bitrev(l) holds sqrt(N) Y[., l] of Eq. zak.  radix 4 fuses pairs of radix-2 stages.
template <typename R>
__device__ __forceinline__ void dzt_inplace(typename Cx<R>::C* X, const FrameArgs& A, int radix) {
  using C = typename Cx<R>::C;
  const int M = A.M, N = A.N, logM = A.logM, MN = M * N, T = blockDim.x;
  int h = N >> 1;
  if (radix == 4) {
    // radix-4 DIF stages handle spans (h, h/2) at once: 4 points n, n+q, n+2q, n+3q with q = h/2
    for (; h >= 2; h >>= 2) {
      const int q = h >> 1;         // quarter of the current block length 2h
      const int tws = N / (2 * h);  // twiddle stride of the first radix-2 stage
      for (int b = threadIdx.x; b < MN / 4; b += T) {
        const int k = b & (M - 1), g = b >> logM;  // g in [0, N/4)
        const int gi = g & (q - 1);
        const int n0 = (g - gi) * 4 + gi;
        C* p0 = X + (size_t)n0 * M + k;
        const C x0 = p0[0], x1 = p0[(size_t)q * M], x2 = p0[(size_t)2 * q * M], x3 = p0[(size_t)3 * q * M];
        // first radix-2 stage (span h = 2q): pairs (x0,x2), (x1,x3) with twiddles W_{2h}^{gi}, W_{2h}^{gi+q}
        const C w0 = conjf2(tw<R>(A, (size_t)(gi * tws) << logM));
        const C w1 = conjf2(tw<R>(A, (size_t)((gi + q) * tws) << logM));
        const C a0 = cadd(x0, x2), a2 = cmul(csub(x0, x2), w0);
        const C a1 = cadd(x1, x3), a3 = cmul(csub(x1, x3), w1);
        // second radix-2 stage (span q): pairs (a0,a1), (a2,a3) with twiddle W_{h}^{gi}
        const C w2 = conjf2(tw<R>(A, (size_t)(gi * tws * 2) << logM));
        p0[0] = cadd(a0, a1);
        p0[(size_t)q * M] = cmul(csub(a0, a1), w2);
        p0[(size_t)2 * q * M] = cadd(a2, a3);
        p0[(size_t)3 * q * M] = cmul(csub(a2, a3), w2);
      }
      frame_sync();
    }
  }
  for (; h >= 1; h >>= 1) {
    const int tws = N / (2 * h);
    for (int b = threadIdx.x; b < MN / 2; b += T) {
      const int k = b & (M - 1), g = b >> logM;
      const int gi = g & (h - 1);
      const int n = ((g - gi) << 1) + gi;
      C* p0 = X + (size_t)n * M + k;
      const C u = p0[0], v = p0[(size_t)h * M];
      const C w = conjf2(tw<R>(A, (size_t)(gi * tws) << logM));
      p0[0] = cadd(u, v);
      p0[(size_t)h * M] = cmul(csub(u, v), w);
    }
    frame_sync();
  }
}

__device__ __forceinline__ int bitrev(int l, int logN) { return (int)(__brev((unsigned)l) >> (32 - logN)); }

// --------------------------------------------------------------- ext writing

// Store the thread's E values of one block (column k, rows j0..j0+E-1) into ext, with the
// quasi-periodic halo column and the periodic halo rows.  kRowMajor selects the global-memory
// layout (element (A, r) at r * 2M + A + M/2) instead of the shared-memory column-major one.
template <typename R, int E, bool kRowMajor = false>
__device__ __forceinline__ void write_ext(typename Cx<R>::C* ext, const FrameArgs& A, int k, int j0,
                                          const typename Cx<R>::C (&v)[E]) {
  using C = typename Cx<R>::C;
  const int M = A.M, N = A.N, CS = N + E + 3, Hk = M >> 1, logM = A.logM, MN = M * N;
  const size_t rstep = kRowMajor ? (size_t)(2 * M) : 1;  // distance between consecutive rows
  // halo column: k < M/2 stores X_ext[k + M] = X[k] W_N[l]; k >= M/2 stores X_ext[k - M] = X[k] W_N[-l]
  const bool low = k < Hk;
  const int mc = k + Hk, hc = (low ? k + M : k - M) + Hk;
  C* mcol = ext + (kRowMajor ? (size_t)mc : (size_t)mc * CS);
  C* hcol = ext + (kRowMajor ? (size_t)hc : (size_t)hc * CS);
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int l = j0 + i;
    const int widx = low ? (l << logM) : ((MN - (l << logM)) & (MN - 1));
    const C hv = cmul(v[i], tw<R>(A, widx));
    mcol[l * rstep] = v[i];
    hcol[l * rstep] = hv;
    // periodic halo rows N .. N + E + 2 hold row (r mod N): one copy when N >= E + 3, two
    // for the short grids (N = 8 with E = 8, N = 16 with E = 16)
    for (int r = l + N; r < N + E + 3; r += N) {
      mcol[r * rstep] = v[i];
      hcol[r * rstep] = hv;
    }
  }
}

// ----------------------------------------------------------- operator gathers

// One run of L paths on E output rows.  kFwd: window rows start at (j0 - dl0 - (L-1)) mod N
// of column k - dk and path m reads window[L - 1 - m + i]; adjoint: rows start at
// (j0 + dl0) mod N of column k + dk and path m reads window[m + i].
//
// Coefficients: with kCoef == 1 they come from the frame's table `ct` (this list's column-k
// entry of path 0; path p at ct[p M]) -- hf W[dl k] for kFwd, h W[dl k] for the adjoint, whose
// conjugate the caller's final combine applies; with kCoef == 2 from a CTA's table (see
// GatherAt); else they are formed here from the path record and the twiddle table.
//
// A run is applied in two phases: load_run gathers its window and its L coefficients into
// registers, mac_run accumulates.  Kernels whose extensions live in global memory issue two
// runs' loads before either accumulates (two L2 round trips in flight per thread instead of
// one after the other).
// Where a gather's runs read: RS, the distance between rows of a row-major extension; the
// coefficients formed from the path records and the frame's twiddle table, or with ct from a
// table of the adjoint factors of a CTA's own delay columns, ct[p ct_rs + k - ct_c0] =
// h_p W[dl_p k] (path p in list order), whose forward factor is ct[..] phi[p] with
// phi[p] = W[-dl_p dk_p] (so that hf_p W[dl_p k] = h_p W[dl_p k] phi[p]).
template <typename R>
struct GatherAt {
  size_t RS;
  const typename Cx<R>::C* ct;
  const typename Cx<R>::C* phi;
  int ct_rs, ct_c0;
};

// Coefficient D of path p (list order, delay-Doppler (dk, dl0 + m) of run rr) at column k.
template <typename R, bool kFwd, bool kTab>
__device__ __forceinline__ typename Cx<R>::C path_coef(const FrameArgs& A, const GatherAt<R>& at,
                                                       const PathRecT<R>* pl, const RunRec& rr, int m, int k) {
  const int p = rr.start + m;
  if constexpr (kTab) {  // adjoint entries unconjugated: the caller's final combine conjugates them
    const typename Cx<R>::C c = at.ct[(size_t)p * at.ct_rs + (k - at.ct_c0)];
    return kFwd ? cmul(c, at.phi[p]) : c;
  } else {
    const PathRecT<R> rec = pl[p];
    const typename Cx<R>::C t = tab<R>(A, (rr.dl0 + m + (A.N >> 1)) * A.M + k);
    return kFwd ? cmul(rec.hf, t) : conjf2(cmul(rec.h, t));
  }
}

template <typename R, int E, int L, bool kFwd, bool kRowMajor, int kCoef>
__device__ __forceinline__ void load_run(const typename Cx<R>::C* src, const PathRecT<R>* pl,
                                         const typename Cx<R>::C* ct, const RunRec& rr, const FrameArgs& A, int k,
                                         int j0, const GatherAt<R>& at, typename Cx<R>::C (&W)[L + E - 1],
                                         typename Cx<R>::C (&D)[L]) {
  using C = typename Cx<R>::C;
  const int M = A.M, N = A.N;
  const int CS = kRowMajor ? 1 : N + E + 3;
  const size_t RS = at.RS;
  const int row0 = kFwd ? ((j0 - rr.dl0 - (L - 1)) & (N - 1)) : ((j0 + rr.dl0) & (N - 1));
  const C* a = src + (size_t)row0 * RS + (kFwd ? -rr.dk : rr.dk) * CS;
#pragma unroll
  for (int w = 0; w < L + E - 1; ++w) W[w] = a[w * RS];
  const C* cr = kCoef == 1 ? ct + (size_t)rr.start * M : nullptr;
#pragma unroll
  for (int m = 0; m < L; ++m) {
    if constexpr (kCoef == 1) {
      D[m] = cr[(size_t)m * M];
    } else {
      D[m] = path_coef<R, kFwd, kCoef == 2>(A, at, pl, rr, m, k);
    }
  }
}

template <typename R, int E, int L, bool kFwd>
__device__ __forceinline__ void mac_run(const typename Cx<R>::C (&W)[L + E - 1], const typename Cx<R>::C (&D)[L],
                                        typename Cx<R>::C (&accA)[E], typename Cx<R>::C (&accB)[E]) {
  using C = typename Cx<R>::C;
#pragma unroll
  for (int m = 0; m < L; ++m) {
    const C DX = Cx<R>::make(D[m].x, D[m].x), DY = Cx<R>::make(D[m].y, D[m].y);
#pragma unroll
    for (int i = 0; i < E; ++i) cmac_split(accA[i], accB[i], DX, DY, W[(kFwd ? L - 1 - m : m) + i]);
  }
}

template <typename R, int E, int L, bool kFwd, bool kRowMajor, int kCoef, bool kPair = kRowMajor>
__device__ __forceinline__ void apply_run(const typename Cx<R>::C* src, const PathRecT<R>* pl,
                                          const typename Cx<R>::C* ct, const RunRec& rr, const FrameArgs& A, int k,
                                          int j0, const GatherAt<R>& at, typename Cx<R>::C (&accA)[E],
                                          typename Cx<R>::C (&accB)[E]) {
  using C = typename Cx<R>::C;
  if constexpr (kRowMajor && kPair) {
    C W[L + E - 1], D[L];
    load_run<R, E, L, kFwd, kRowMajor, kCoef>(src, pl, ct, rr, A, k, j0, at, W, D);
    mac_run<R, E, L, kFwd>(W, D, accA, accB);
  } else {
    // shared-memory extension (column-major, or a row-major window): each coefficient is
    // loaded right before its MACs (fewer live registers)
    const int M = A.M, N = A.N, CS = kRowMajor ? 1 : N + E + 3;
    const size_t RS = kRowMajor ? at.RS : 1;
    const int row0 = kFwd ? ((j0 - rr.dl0 - (L - 1)) & (N - 1)) : ((j0 + rr.dl0) & (N - 1));
    const C* a = src + (size_t)row0 * RS + (kFwd ? -rr.dk : rr.dk) * CS;
    C W[L + E - 1];
#pragma unroll
    for (int w = 0; w < L + E - 1; ++w) W[w] = a[w * RS];
    const C* cr = kCoef == 1 ? ct + (size_t)rr.start * M : nullptr;
#pragma unroll
    for (int m = 0; m < L; ++m) {
      C D;
      if constexpr (kCoef == 1) {
        D = cr[(size_t)m * M];
      } else {
        D = path_coef<R, kFwd, kCoef == 2>(A, at, pl, rr, m, k);
      }
      const C DX = Cx<R>::make(D.x, D.x), DY = Cx<R>::make(D.y, D.y);
#pragma unroll
      for (int i = 0; i < E; ++i) cmac_split(accA[i], accB[i], DX, DY, W[(kFwd ? L - 1 - m : m) + i]);
    }
  }
}

// Runs [q, end) of one length class, two at a time when the extension is in global memory
// (kPair: two runs' loads in flight before either accumulates).
template <typename R, int E, int L, bool kFwd, bool kRowMajor, int kCoef, bool kPair = kRowMajor>
__device__ __forceinline__ int apply_runs(const typename Cx<R>::C* src, const PathRecT<R>* pl,
                                          const typename Cx<R>::C* ct, const RunRec* rl, int q, int end,
                                          const FrameArgs& A, int k, int j0, const GatherAt<R>& at,
                                          typename Cx<R>::C (&accA)[E], typename Cx<R>::C (&accB)[E]) {
  using C = typename Cx<R>::C;
  if constexpr (kRowMajor && kPair) {
    for (; q + 1 < end; q += 2) {
      C W0[L + E - 1], D0[L], W1[L + E - 1], D1[L];
      load_run<R, E, L, kFwd, kRowMajor, kCoef>(src, pl, ct, rl[q], A, k, j0, at, W0, D0);
      load_run<R, E, L, kFwd, kRowMajor, kCoef>(src, pl, ct, rl[q + 1], A, k, j0, at, W1, D1);
      mac_run<R, E, L, kFwd>(W0, D0, accA, accB);
      mac_run<R, E, L, kFwd>(W1, D1, accA, accB);
    }
  }
  for (; q < end; ++q) apply_run<R, E, L, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, rl[q], A, k, j0, at, accA, accB);
  return q;
}

constexpr int kColHalf = -0x40000000;  // gather column offset: the extension's own (M / 2)

// Forward rows (kFwd) of output block b: out[i] = (H p)_b[k, j0 + i], summed over the tx blocks
// and the runs of each (b, t) list; adjoint: out[i] = (H^H u)_b[k, j0 + i] over the rx blocks.
// Column k of the extension is column k + col0 of `ext` (col0 = M / 2 by default); a row-major
// extension's rows are `rs` elements apart (2 M by default) -- a shared-memory window of
// a row-major extension passes its own offset and stride; ct / phi / ct_rs / ct_c0: a CTA's
// coefficient table (see GatherAt), else the coefficients are formed per path.
template <typename R, int E, bool kFwd, bool kRowMajor, int kCoef, bool kPair = kRowMajor>
__device__ __forceinline__ void gather_runs(const typename Cx<R>::C* ext, size_t blk, const PathRecT<R>* paths,
                                            const RunRec* runs, const int* nruns, const typename Cx<R>::C* coef,
                                            const FrameArgs& A, int b, int k, int j0, typename Cx<R>::C (&out)[E],
                                            size_t rs = 0, int col0 = kColHalf,
                                            const typename Cx<R>::C* ct_tab = nullptr,
                                            const typename Cx<R>::C* phi = nullptr, int ct_rs = 0, int ct_c0 = 0) {
  using C = typename Cx<R>::C;
  // register budget: the window holds L + E - 1 complex values beside 2E accumulators
  constexpr int kLMax = E >= 32 ? 1 : (E >= 16 ? 2 : kMaxRun);
  const int c0 = col0 == kColHalf ? (A.M >> 1) : col0;
  const int CS = kRowMajor ? 1 : A.N + E + 3;
  const GatherAt<R> at{kRowMajor ? (rs ? rs : (size_t)(2 * A.M)) : 1, ct_tab, phi, ct_rs, ct_c0};
  C accA[E], accB[E];
#pragma unroll
  for (int i = 0; i < E; ++i) accA[i] = accB[i] = Cx<R>::make(0, 0);
  const C* colk = ext + (size_t)(k + c0) * CS;
  const int nother = kFwd ? A.ntx : A.nrx;
  for (int o = 0; o < nother; ++o) {
    const C* src = colk + (size_t)o * blk;
    const int li = kFwd ? b * A.ntx + o : o * A.ntx + b;
    const PathRecT<R>* pl = paths + (size_t)li * A.p_max;
    const RunRec* rl = runs + (size_t)li * A.p_max;
    const C* ct = kCoef == 1 ? coef + (size_t)li * A.p_max * A.M + k : nullptr;
    // runs are stored longest first: n4 of length 4, then n3, n2 and n1 (packed counts)
    const int packed = nruns[li];
    const int n4 = packed & 127, n3 = (packed >> 7) & 127, n2 = (packed >> 14) & 255, n1 = (packed >> 22) & 511;
    int q = 0;
    if constexpr (kLMax == 4) {
      q = apply_runs<R, E, 4, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, rl, q, n4, A, k, j0, at, accA, accB);
      q = apply_runs<R, E, 3, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, rl, q, n4 + n3, A, k, j0, at, accA, accB);
    } else {
      for (const int e3 = n4 + n3; q < e3; ++q) {  // split into runs of at most kLMax paths
        const RunRec rr = rl[q];
        for (int m = 0; m < rr.len; m += kLMax) {
          RunRec sub = rr;
          sub.start = (short)(rr.start + m);
          sub.dl0 = (short)(rr.dl0 + m);
          if (kLMax == 2 && rr.len - m >= 2) apply_run<R, E, (kLMax == 2 ? 2 : 1), kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, sub, A, k, j0, at, accA, accB);
          else apply_run<R, E, 1, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, sub, A, k, j0, at, accA, accB);
        }
      }
    }
    if constexpr (kLMax >= 2) {
      q = apply_runs<R, E, 2, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, rl, q, n4 + n3 + n2, A, k, j0, at, accA, accB);
    } else {
      for (const int e2 = n4 + n3 + n2; q < e2; ++q) {
        RunRec sub = rl[q];
        apply_run<R, E, 1, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, sub, A, k, j0, at, accA, accB);
        sub.start = (short)(sub.start + 1);
        sub.dl0 = (short)(sub.dl0 + 1);
        apply_run<R, E, 1, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, sub, A, k, j0, at, accA, accB);
      }
    }
    apply_runs<R, E, 1, kFwd, kRowMajor, kCoef, kPair>(src, pl, ct, rl, q, n4 + n3 + n2 + n1, A, k, j0, at, accA, accB);
  }
  // accA = sum D.x W, accB = sum D.y W: D W = (A.x - B.y, A.y + B.x); for the adjoint's table
  // entries c (D = conj(c)): (A.x + B.y, A.y - B.x)
  constexpr bool conj_tab = !kFwd && kCoef != 0;
#pragma unroll
  for (int i = 0; i < E; ++i)
    out[i] = conj_tab ? Cx<R>::make(accA[i].x + accB[i].y, accA[i].y - accB[i].x)
                      : Cx<R>::make(accA[i].x - accB[i].y, accA[i].y + accB[i].x);
}

// kCoef: 0 coefficients formed per path, 1 the frame's tables coefF / coefA, 2 a CTA's table
// ct_tab with the forward phases phi (see GatherAt).
template <typename R, int E, bool kRowMajor = false, int kCoef = 0, bool kPair = kRowMajor>
__device__ __forceinline__ void gather_fwd(const typename Cx<R>::C* ext, size_t blk, const PathRecT<R>* paths,
                                           const RunRec* runs, const int* nruns, const FrameArgs& A, int r, int k,
                                           int j0, typename Cx<R>::C (&out)[E],
                                           const typename Cx<R>::C* coefF = nullptr, size_t rs = 0,
                                           int col0 = kColHalf, const typename Cx<R>::C* ct_tab = nullptr,
                                           const typename Cx<R>::C* phi = nullptr, int ct_rs = 0, int ct_c0 = 0) {
  gather_runs<R, E, true, kRowMajor, kCoef, kPair>(ext, blk, paths, runs, nruns, coefF, A, r, k, j0, out, rs, col0,
                                                   ct_tab, phi, ct_rs, ct_c0);
}
template <typename R, int E, bool kRowMajor = false, int kCoef = 0, bool kPair = kRowMajor>
__device__ __forceinline__ void gather_adj(const typename Cx<R>::C* ext, size_t blk, const PathRecT<R>* paths,
                                           const RunRec* runs, const int* nruns, const FrameArgs& A, int t, int k,
                                           int j0, typename Cx<R>::C (&out)[E],
                                           const typename Cx<R>::C* coefA = nullptr, size_t rs = 0,
                                           int col0 = kColHalf, const typename Cx<R>::C* ct_tab = nullptr,
                                           const typename Cx<R>::C* phi = nullptr, int ct_rs = 0, int ct_c0 = 0) {
  gather_runs<R, E, false, kRowMajor, kCoef, kPair>(ext, blk, paths, runs, nruns, coefA, A, t, k, j0, out, rs, col0,
                                                    ct_tab, phi, ct_rs, ct_c0);
}

// The coefficient tables of one list (after build_runs: sorted order), all threads:
// cf[p M + k] = hf_p W[dl_p k] (forward), ca[p M + k] = h_p W[dl_p k] (adjoint, conjugated
// at use) -- the per-(path, column) factors of Eq. sparse_mvm / Eq. sparse_herm_mvm that do
// not change over the CG iterations.
template <typename R>
__device__ __forceinline__ void coef_tables(const PathRecT<R>* pl, int P, const FrameArgs& A, typename Cx<R>::C* cf,
                                            typename Cx<R>::C* ca, int first = -1, int stride = 0) {
  const int M = A.M, N = A.N;
  if (first < 0) {
    first = threadIdx.x;
    stride = blockDim.x;
  }
#pragma unroll 2
  for (int e = first; e < P * M; e += stride) {
    const int p = e >> A.logM, k = e & (M - 1);
    const PathRecT<R> rec = pl[p];
    const typename Cx<R>::C t = tab<R>(A, (rec.dl + (N >> 1)) * M + k);
    cf[e] = cmul(rec.hf, t);
    ca[e] = cmul(rec.h, t);
  }
}

// Sort one list's shared-memory copy by (dk, dl) (rank sort through `tmp`, which must hold P
// records and not alias the list; `keys` is scratch for max(P, 4) ints rounded up to a
// multiple of 4) and cut it into runs of at most kMaxRun paths with equal dk and consecutive
// dl, stored longest first; *nruns_out packs the counts of runs of length 4, 3, 2 and 1 into
// bits 0-6, 7-13, 14-21 and 22-30 (P <= 256).  All threads call.  Returns the number of runs.
template <typename R>
__device__ __forceinline__ int build_runs(PathRecT<R>* pl, int P, RunRec* runs, PathRecT<R>* tmp, int* keys,
                                          int* nruns_out) {
  return build_runs<R>(pl, P, runs, tmp, keys, nruns_out, [](int, int) {});
}

// build_runs that also runs side(i, n) on the sorted list, i = this thread's index among the
// n threads doing it: the warps other than warp 0, while warp 0 cuts the runs (for one-warp
// blocks, warp 0 after the cutting).
template <typename R, typename Side>
__device__ __forceinline__ int build_runs(PathRecT<R>* pl, int P, RunRec* runs, PathRecT<R>* tmp, int* keys,
                                          int* nruns_out, Side side) {
  const int P4 = (P + 3) & ~3;
  for (int p = threadIdx.x; p < P4; p += blockDim.x) keys[p] = p < P ? pl[p].dk * 256 + pl[p].dl : 0x7fffffff;
  frame_sync();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {  // keys are distinct: ranks are a permutation
    const int key = keys[p];
    int rank = 0;
    for (int u = 0; u < P4; u += 4) {
      const int4 kv = *reinterpret_cast<const int4*>(keys + u);
      rank += (kv.x < key) + (kv.y < key) + (kv.z < key) + (kv.w < key);
    }
    tmp[rank] = pl[p];
  }
  frame_sync();
  for (int p = threadIdx.x; p < P; p += blockDim.x) pl[p] = tmp[p];
  frame_sync();
  if (threadIdx.x < 32) {  // warp 0 cuts and places the runs from bit masks, 32 paths per word
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u, le = lt | (1u << lane);
    unsigned link[9];  // bit (p mod 32) of word p / 32: path p continues path p - 1's sequence
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int p = 32 * c + lane;
      const bool l = p > 0 && p < P && pl[p - 1].dk == pl[p].dk && pl[p - 1].dl + 1 == pl[p].dl;
      link[c] = __ballot_sync(0xffffffffu, l);
    }
    link[8] = 0u;
    int lens[8];  // run length starting at path 32 c + lane (0: not a run start)
    int n1 = 0, n2 = 0, n3 = 0, n4 = 0;
    int last_start = 0;  // start of the sequence that is open at the end of the previous word
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int p = 32 * c + lane;
      const unsigned heads = ~link[c];  // paths that begin a maximal sequence
      const unsigned below = heads & le;
      const int seq = below ? 32 * c + 31 - __clz(below) : last_start;
      const unsigned long long win = ((unsigned long long)link[c + 1] << 32 | link[c]) >> (lane + 1);
      const int follow = __ffsll(~win & 7ull) ? __ffsll(~win & 7ull) - 1 : 3;  // linked successors, <= 3
      const int len = (p < P && ((p - seq) & (kMaxRun - 1)) == 0) ? 1 + follow : 0;
      lens[c] = len;
      if (heads) last_start = 32 * c + 31 - __clz(heads);
      n1 += __popc(__ballot_sync(0xffffffffu, len == 1));
      n2 += __popc(__ballot_sync(0xffffffffu, len == 2));
      n3 += __popc(__ballot_sync(0xffffffffu, len == 3));
      n4 += __popc(__ballot_sync(0xffffffffu, len == 4));
    }
    int s4 = 0, s3 = n4, s2 = n4 + n3, s1 = n4 + n3 + n2;  // first slot of each length
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int p = 32 * c + lane;
      const int len = lens[c];
      const unsigned m1 = __ballot_sync(0xffffffffu, len == 1), m2 = __ballot_sync(0xffffffffu, len == 2);
      const unsigned m3 = __ballot_sync(0xffffffffu, len == 3), m4 = __ballot_sync(0xffffffffu, len == 4);
      if (len) {
        const int slot = len == 4 ? s4 + __popc(m4 & lt)
                       : len == 3 ? s3 + __popc(m3 & lt)
                       : len == 2 ? s2 + __popc(m2 & lt) : s1 + __popc(m1 & lt);
        RunRec rr;
        rr.start = (short)p;
        rr.len = (short)len;
        rr.dk = (short)pl[p].dk;
        rr.dl0 = (short)pl[p].dl;
        runs[slot] = rr;
      }
      s1 += __popc(m1);
      s2 += __popc(m2);
      s3 += __popc(m3);
      s4 += __popc(m4);
    }
    if (lane == 0) *nruns_out = n4 | (n3 << 7) | (n2 << 14) | (n1 << 22);
  } else {
    side((int)threadIdx.x - 32, (int)blockDim.x - 32);
  }
  frame_sync();
  if (blockDim.x == 32) {  // one warp: the side work follows the cutting
    side((int)threadIdx.x, 32);
    frame_sync();
  }
  const int packed = *nruns_out;
  return (packed & 127) + ((packed >> 7) & 127) + ((packed >> 14) & 255) + ((packed >> 22) & 511);
}

// ------------------------------------------------------------ read-off + compaction

// Read the effective channel off a Zak-transformed pilot grid X (DIF output, rows in
// bit-reversed order) and compact the taps with |h_eff| > theta (Eq. heff_hadamard,
// Eq. heff_thres) into out[0, P) in ascending q, keeping the p_max largest when more pass
// (ties to the lower q).  Returns P; sets `trunc`.  Every thread owns q in
// [tid*EQ, tid*EQ + EQ), EQ = MN/T.  When gout is set the list is also stored as list li.
template <typename R, int EQ>
__device__ __forceinline__ int readoff_compact(const typename Cx<R>::C* X, const FrameArgs& A, R theta, double a_pilot,
                                               PathRecT<R>* out, SharedHdr* S, const PathIO* gout, int li,
                                               int& trunc) {
  using C = typename Cx<R>::C;
  using Key = typename Cx<R>::Key;
  const int M = A.M, N = A.N, logM = A.logM, MN = M * N, tid = threadIdx.x;
  const R scale = (R)A.inv_sqrtN / (R)a_pilot;
  const R th2 = theta * theta;
  C hv[EQ];
  Key mb[EQ];
  short dks[EQ], dls[EQ];
  uint32_t pass = 0;
#pragma unroll
  for (int i = 0; i < EQ; ++i) {
    const int q = tid * EQ + i;
    const int k = q & (M - 1), l = q >> logM;
    const int dk = ((k - A.K0 + (M >> 1)) & (M - 1)) - (M >> 1);
    const int dl = ((l - A.L0 + (N >> 1)) & (N - 1)) - (N >> 1);
    const C Y = X[(size_t)bitrev(l, A.logN) * M + k];
    const C h = cscale(cmul(Y, tw<R>(A, (size_t)((-A.K0 * dl) & (MN - 1)))), scale);
    const R m2 = h.x * h.x + h.y * h.y;
    const bool region = (A.pilot_mode == ZOTFS_PILOT_SEPARATE) || (dk >= 0 && dk <= A.guard);
    hv[i] = h;
    mb[i] = Cx<R>::key(m2);
    dks[i] = (short)dk;
    dls[i] = (short)dl;
    if (region && m2 > th2) pass |= 1u << i;
  }
  int total;
  int base = block_exclusive_scan(__popc(pass), S->scan, total);
  uint32_t keep = pass;
  trunc = 0;
  if (total > A.p_max) {
    trunc = 1;
    // The K-th largest |h|^2 among the passing taps, exactly: radix select on the bit
    // patterns of the non-negative values (ordered like the values), 7 bits per pass from
    // the top.  Each pass histograms the taps that share the bits fixed so far; warp 0 finds
    // the bin holding the K-th largest from the top, fixes its bits and clears the bins.
    const int K = A.p_max;
    constexpr int kKeyBits = 8 * (int)sizeof(Key) - 1;  // the sign bit is 0
    Key prefix = 0, fixed = 0;
    int kleft = K;  // rank of the wanted value among the taps that match `prefix`
    const int lane = tid & 31;
    for (int b = tid; b < 128; b += blockDim.x) S->hist[b] = 0;
    frame_sync();
    for (int hb = kKeyBits; hb > 0; hb -= 7) {
      const int w = hb < 7 ? hb : 7, sh = hb - w;
#pragma unroll
      for (int i = 0; i < EQ; ++i)
        if (((pass >> i) & 1u) && ((mb[i] ^ prefix) & fixed) == 0)
          atomicAdd(&S->hist[(int)((mb[i] >> sh) & (Key)127)], 1);
      frame_sync();
      if (tid < 32) {
        int c[4], sum = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          c[j] = S->hist[4 * lane + j];
          S->hist[4 * lane + j] = 0;
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
      frame_sync();
      const int bin = S->isc[2];
      kleft = S->isc[3];
      prefix |= (Key)bin << sh;
      fixed |= (Key)((1u << w) - 1u) << sh;
    }
    const Key vK = prefix;  // the K-th largest |h|^2 among the passing taps
    const int need = kleft;  // taps equal to vK that are kept: the first `need` in ascending q
    uint32_t gt = 0, eq = 0;
#pragma unroll
    for (int i = 0; i < EQ; ++i)
      if ((pass >> i) & 1u) {
        if (mb[i] > vK) gt |= 1u << i;
        else if (mb[i] == vK) eq |= 1u << i;
      }
    // one scan of the packed counts (taps above vK in the high half, ties in the low half):
    // a kept tap's position = taps above vK before it + min(ties before it, need)
    int both_total;
    const int both = block_exclusive_scan((__popc(gt) << 16) | __popc(eq), S->scan, both_total);
    (void)both_total;
    int gt_before = both >> 16, eq_before = both & 0xffff;
    keep = 0;
    int pos0 = gt_before + min(eq_before, need);
#pragma unroll
    for (int i = 0; i < EQ; ++i) {
      if ((gt >> i) & 1u) {
        keep |= 1u << i;
      } else if ((eq >> i) & 1u) {
        if (eq_before < need) keep |= 1u << i;
        ++eq_before;
      }
    }
    base = pos0;
    total = K;
  }
  int pos = base;
#pragma unroll
  for (int i = 0; i < EQ; ++i) {
    if ((keep >> i) & 1u) {
      PathRecT<R> rec;
      rec.h = hv[i];
      rec.dk = dks[i];
      rec.dl = dls[i];
      rec.hf = cmul(hv[i], tw<R>(A, (size_t)((-dls[i] * dks[i]) & (MN - 1))));
      rec.pad0 = rec.pad1 = 0;
      out[pos] = rec;
      if (gout) {
        const size_t g = (size_t)li * A.p_max + pos;
        gout->dk[g] = (int16_t)dks[i];
        gout->dl[g] = (int16_t)dls[i];
        store_complex(gout->h, g, gout->tap_dtype, hv[i]);
      }
      ++pos;
    }
  }
  if (gout && threadIdx.x == 0) {
    gout->count[li] = total;
    if (gout->status) gout->status[li] = trunc ? ZOTFS_ETRUNCATED : ZOTFS_OK;
  }
  frame_sync();
  return total;
}

// Load a caller-provided path list; out-of-range entries are zeroed and flagged.
template <typename R>
__device__ __forceinline__ int load_paths(const FrameArgs& A, const PathIO& gin, int li, PathRecT<R>* out,
                                          int& bad) {
  using C = typename Cx<R>::C;
  const int M = A.M, N = A.N, MN = M * N;
  if (gin.invalid) {
    bad = 1;
    frame_sync();
    return 0;
  }
  int P = gin.count[li];
  bad = 0;
  if (P < 0 || P > A.p_max) {
    bad = 1;
    P = P < 0 ? 0 : A.p_max;
  }
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const size_t g = (size_t)li * A.p_max + p;
    int dk = gin.dk[g], dl = gin.dl[g];
    C h = load_complex<C>(gin.h, g, gin.tap_dtype);
    if (dk < -(M >> 1) || dk >= (M >> 1) || dl < -(N >> 1) || dl >= (N >> 1)) {
      bad = 1;
      dk = 0;
      dl = 0;
      h = Cx<R>::make(0, 0);
    }
    PathRecT<R> rec;
    rec.h = h;
    rec.dk = dk;
    rec.dl = dl;
    rec.hf = cmul(h, tw<R>(A, (size_t)((-dl * dk) & (MN - 1))));
    rec.pad0 = rec.pad1 = 0;
    out[p] = rec;
  }
  bad = frame_sync_or(bad);
  return P;
}

// ------------------------------------------------------------------------ demap

// Max-log LLRs of one sqrt(Q)-PAM axis with Gray labels (I or Q part of square QAM):
// bit j < hb of the axis label (MSB first).  Unused outputs are left at 0.
template <typename R>
__device__ __forceinline__ void pam_llr(R x, int hb, R d, R inv_lam, R& o0, R& o1, R& o2) {
  const int m = 1 << hb;
  const R inf = (R)INFINITY;
  R mn0a = inf, mn0b = inf, mn0c = inf, mn1a = inf, mn1b = inf, mn1c = inf;
  for (int i = 0; i < m; ++i) {
    const R a = (R)(2 * i - (m - 1)) * d;
    const R di = (x - a) * (x - a);
    const int g = i ^ (i >> 1);
    const int b0 = (g >> (hb - 1)) & 1;
    const int b1 = hb > 1 ? (g >> (hb - 2)) & 1 : 0;
    const int b2 = hb > 2 ? g & 1 : 0;
    if (b0) mn1a = fmin(mn1a, di); else mn0a = fmin(mn0a, di);
    if (b1) mn1b = fmin(mn1b, di); else mn0b = fmin(mn0b, di);
    if (b2) mn1c = fmin(mn1c, di); else mn0c = fmin(mn0c, di);
  }
  o0 = (mn1a - mn0a) * inv_lam;
  o1 = hb > 1 ? (mn1b - mn0b) * inv_lam : (R)0;
  o2 = hb > 2 ? (mn1c - mn0c) * inv_lam : (R)0;
}

// Max-log LLRs of one Gray square-QAM symbol: l[0..bps) = I-axis bits then Q-axis bits
// (output as float); returns the hard label, bit j set when LLR j < 0 in precision R.
template <typename R>
__device__ __forceinline__ int qam_llr(typename Cx<R>::C x, int bps, R d, R inv_lam, float (&l)[6]) {
  const int hb = bps >> 1;
  R i0, i1, i2, q0, q1, q2;
  pam_llr<R>(x.x, hb, d, inv_lam, i0, i1, i2);
  pam_llr<R>(x.y, hb, d, inv_lam, q0, q1, q2);
  R lr[6];
  if (hb == 1) {
    lr[0] = i0; lr[1] = q0; lr[2] = lr[3] = lr[4] = lr[5] = (R)0;
  } else if (hb == 2) {
    lr[0] = i0; lr[1] = i1; lr[2] = q0; lr[3] = q1; lr[4] = lr[5] = (R)0;
  } else {
    lr[0] = i0; lr[1] = i1; lr[2] = i2; lr[3] = q0; lr[4] = q1; lr[5] = q2;
  }
  int hard = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    l[j] = (float)lr[j];
    if (j < bps) hard |= (lr[j] < (R)0 ? 1 : 0) << (bps - 1 - j);
  }
  return hard;
}

// pam_llr with the constellation size a compile-time constant (levels and Gray labels fold
// into constants); bitwise the same results as pam_llr.
template <typename R, int HB>
__device__ __forceinline__ void pam_llr_c(R x, R d, R inv_lam, R& o0, R& o1, R& o2) {
  constexpr int m = 1 << HB;
  const R inf = (R)INFINITY;
  R mn0[3] = {inf, inf, inf}, mn1[3] = {inf, inf, inf};
#pragma unroll
  for (int i = 0; i < m; ++i) {
    const R a = (R)(2 * i - (m - 1)) * d;
    const R di = (x - a) * (x - a);
    const int g = i ^ (i >> 1);
#pragma unroll
    for (int b = 0; b < HB; ++b) {
      if ((g >> (HB - 1 - b)) & 1) mn1[b] = fmin(mn1[b], di);
      else mn0[b] = fmin(mn0[b], di);
    }
  }
  o0 = (mn1[0] - mn0[0]) * inv_lam;
  o1 = HB > 1 ? (mn1[1] - mn0[1]) * inv_lam : (R)0;
  o2 = HB > 2 ? (mn1[2] - mn0[2]) * inv_lam : (R)0;
}

// qam_llr_regs for a compile-time constellation (2 HB bits per symbol).
template <typename R, int HB>
__device__ __forceinline__ int qam_llr_c(typename Cx<R>::C x, R d, R inv_lam, float2& o01, float2& o23,
                                         float2& o45) {
  constexpr int bps = 2 * HB;
  R i0, i1, i2, q0, q1, q2;
  pam_llr_c<R, HB>(x.x, d, inv_lam, i0, i1, i2);
  pam_llr_c<R, HB>(x.y, d, inv_lam, q0, q1, q2);
  const R z = (R)0;
  const R l0 = i0;
  const R l1 = HB == 1 ? q0 : i1;
  const R l2 = HB == 1 ? z : (HB == 2 ? q0 : i2);
  const R l3 = HB == 1 ? z : (HB == 2 ? q1 : q0);
  const R l4 = HB == 3 ? q1 : z;
  const R l5 = HB == 3 ? q2 : z;
  o01 = make_float2((float)l0, (float)l1);
  o23 = make_float2((float)l2, (float)l3);
  o45 = make_float2((float)l4, (float)l5);
  int hard = ((l0 < z) << (bps - 1)) | ((l1 < z) << (bps - 2));
  if constexpr (bps > 2) hard |= ((l2 < z) << (bps - 3)) | ((l3 < z) << (bps - 4));
  if constexpr (bps > 4) hard |= ((l4 < z) << 1) | (l5 < z);
  return hard;
}

// The same LLRs and hard label as qam_llr, returned in registers: o01 = (l0, l1),
// o23 = (l2, l3), o45 = (l4, l5).
template <typename R>
__device__ __forceinline__ int qam_llr_regs(typename Cx<R>::C x, int bps, R d, R inv_lam, float2& o01, float2& o23,
                                            float2& o45) {
  const int hb = bps >> 1;
  R i0, i1, i2, q0, q1, q2;
  pam_llr<R>(x.x, hb, d, inv_lam, i0, i1, i2);
  pam_llr<R>(x.y, hb, d, inv_lam, q0, q1, q2);
  const R z = (R)0;
  const R l0 = i0;
  const R l1 = hb == 1 ? q0 : i1;
  const R l2 = hb == 1 ? z : (hb == 2 ? q0 : i2);
  const R l3 = hb == 1 ? z : (hb == 2 ? q1 : q0);
  const R l4 = hb == 3 ? q1 : z;
  const R l5 = hb == 3 ? q2 : z;
  o01 = make_float2((float)l0, (float)l1);
  o23 = make_float2((float)l2, (float)l3);
  o45 = make_float2((float)l4, (float)l5);
  int hard = ((l0 < z) << (bps - 1)) | ((l1 < z) << (bps - 2));
  if (bps > 2) hard |= ((l2 < z) << (bps - 3)) | ((l3 < z) << (bps - 4));
  if (bps > 4) hard |= ((l4 < z) << 1) | (l5 < z);
  return hard;
}

}  // namespace zotfs
