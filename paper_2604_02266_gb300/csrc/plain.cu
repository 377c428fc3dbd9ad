// The plain form of the receiver: one frame at a time, one kernel launch per stage and per
// CG step, vectors in global scratch, FP32 with FP64 scalar combines -- the structure of
// a host-driven GPU pipeline with fixed iteration count (Sec. IV-C "Profiling-based fixed
// termination": no host synchronisation inside the loop).  It is the comparison baseline
// for the fused kernels.  Its operator kernel evaluates the paper's index maps
// (Eq. map_chMatDD_col, Eq. herm_mapping) and phase literally, with explicit wraps.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace zotfs {

namespace {

constexpr int kBlock = 256;

struct PlainLayout {
  size_t grid, ydd, t, x, c, p, a, paths, counts, scal, flags, labels, llr, total;
};

PlainLayout plain_layout(int M, int N, int nrx, int ntx, int p_max) {
  const size_t MN = (size_t)M * N;
  const int nl = nrx * ntx;
  PlainLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  L.grid = take(MN * sizeof(float2));
  L.ydd = take(nrx * MN * sizeof(float2));
  L.t = take(nrx * MN * sizeof(float2));
  L.x = take(ntx * MN * sizeof(float2));
  L.c = take(ntx * MN * sizeof(float2));
  L.p = take(ntx * MN * sizeof(float2));
  L.a = take(ntx * MN * sizeof(float2));
  L.paths = take((size_t)nl * p_max * sizeof(PathRec));
  L.counts = take((size_t)nl * sizeof(int));
  L.scal = take(8 * sizeof(double));
  L.flags = take(4 * sizeof(int));
  L.labels = take(ntx * MN);
  L.llr = take(ntx * MN * 6 * sizeof(float));
  L.total = off;
  return L;
}

struct PlainGeo {
  int M, N, logM, logN, nrx, ntx, p_max;
  const float2* W;
};

// Direct DFT along Doppler of one TD grid (Eq. zak without the N^-1/2 unless `scale`):
// out[row(l) M + k] = scale * sum_n y[k + nM] exp(-j2pi n l / N), row(l) = bitrev(l) or l.
__global__ void plain_dzt_kernel(const void* y, int dtype, float2* out, PlainGeo G, int bitrev_rows, float scale) {
  const int MN = G.M * G.N;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= MN) return;
  const int k = q & (G.M - 1), l = q >> G.logM;
  float2 acc = make_float2(0.f, 0.f);
  for (int n = 0; n < G.N; ++n) {
    const float2 w = conjf2(__ldg(&G.W[(size_t)(((n * l) & (G.N - 1)) << G.logM)]));
    acc = cadd(acc, cmul(load_complex<float2>(y, (size_t)k + (size_t)n * G.M, dtype), w));
  }
  const int row = bitrev_rows ? bitrev(l, G.logN) : l;
  out[(size_t)row * G.M + k] = cscale(acc, scale);
}

// Read-off + threshold + compaction of one pilot grid, single CTA (the shared-memory copy of
// the grid feeds the same read-off routine as the fused kernel).
template <int EQ>
__global__ void plain_compact_kernel(const __grid_constant__ FrameArgs A, const float2* grid, int f, int list_local, int list_global,
                                     PathRec* paths_out, int* counts, int* flags, int write_global) {
  extern __shared__ __align__(128) unsigned char smem[];
  SharedHdr* S = reinterpret_cast<SharedHdr*>(smem);
  float2* X = reinterpret_cast<float2*>(smem + ((sizeof(SharedHdr) + 127) & ~size_t(127)));
  const int MN = A.M * A.N;
  for (int i = threadIdx.x; i < MN; i += blockDim.x) X[i] = grid[i];
  __syncthreads();
  PathIO gout;
  const int fo = list_global - list_local;  // first list of this frame
  gout.count = A.pcount ? A.pcount + fo : nullptr;
  gout.status = A.pstatus ? A.pstatus + fo : nullptr;
  gout.dk = A.pdk ? A.pdk + (size_t)fo * A.p_max : nullptr;
  gout.dl = A.pdl ? A.pdl + (size_t)fo * A.p_max : nullptr;
  gout.h = A.ph ? static_cast<char*>(A.ph) + (size_t)fo * A.p_max * dtype_bytes(A.tap_dtype) : nullptr;
  gout.tap_dtype = A.tap_dtype;
  int trunc;
  const int P = readoff_compact<float, EQ>(X, A, A.theta[f], A.a_pilot, paths_out + (size_t)list_local * A.p_max, S,
                                    write_global ? &gout : nullptr, list_local, trunc);
  if (threadIdx.x == 0) {
    counts[list_local] = P;
    if (trunc) flags[0] |= 1;
  }
}

// Forward coefficient of row (k, l) for one path, by the paper's formulas:
// column <l - dl>_N M + <k - dk>_M and phase 2pi/(MN) [dl A + n <l - dl>_N M], A = k - dk, n = floor(A/M).
__device__ __forceinline__ float2 fwd_coef(const PathRec& r, int k, int l, const PlainGeo& G, int& col) {
  const int MN = G.M * G.N;
  const int A = k - r.dk;
  const int n = A >> G.logM;
  const int ls = (l - r.dl) & (G.N - 1);
  col = ls * G.M + (A & (G.M - 1));
  return cmul(r.h, __ldg(&G.W[(size_t)((r.dl * A + n * ls * G.M) & (MN - 1))]));
}

// u = H v (adjoint == 0) or u = H^H v + lam * padd (adjoint != 0), one thread per output element.
__global__ void plain_apply_kernel(PlainGeo G, const PathRec* paths, const int* counts, const float2* v, float2* u,
                                   int adjoint, float lam, const float2* padd) {
  const int MN = G.M * G.N;
  const int nout = adjoint ? G.ntx : G.nrx, nin = adjoint ? G.nrx : G.ntx;
  const int gq = blockIdx.x * blockDim.x + threadIdx.x;
  if (gq >= nout * MN) return;
  const int b = gq / MN, q = gq - b * MN;
  const int k = q & (G.M - 1), l = q >> G.logM;
  float2 acc = make_float2(0.f, 0.f);
  for (int o = 0; o < nin; ++o) {
    const int li = adjoint ? (o * G.ntx + b) : (b * G.ntx + o);
    const PathRec* pl = paths + (size_t)li * G.p_max;
    const float2* src = v + (size_t)o * MN;
    for (int p = 0; p < counts[li]; ++p) {
      const PathRec r = pl[p];
      if (!adjoint) {
        int col;
        const float2 D = fwd_coef(r, k, l, G, col);
        acc = cadd(acc, cmul(D, src[col]));
      } else {
        // row s whose column for path p is q (Eq. herm_mapping), and that row's coefficient
        const int ks = (k + r.dk) & (G.M - 1), lsr = (l + r.dl) & (G.N - 1);
        int col;
        const float2 D = fwd_coef(r, ks, lsr, G, col);
        acc = cadd(acc, cmul(conjf2(D), src[(size_t)lsr * G.M + ks]));
      }
    }
  }
  if (adjoint && padd) {
    const float2 pv = padd[(size_t)b * MN + q];
    acc.x = fmaf(lam, pv.x, acc.x);
    acc.y = fmaf(lam, pv.y, acc.y);
  }
  u[(size_t)b * MN + q] = acc;
}

enum { kCn = 0, kAlpha = 1, kBeta = 2, kStopAt = 3, kStopped = 4 };
enum { kEpiCn0 = 0, kEpiAlpha = 1, kEpiBeta = 2 };

// Single CTA: sum of Re(conj(a) b); FP32 per thread, FP64 across warps; scalar epilogue.
// eps2 > 0: the CG stopping test (||c||^2 <= eps2 ||b||^2); once it fires, alpha = beta = 0
// leave x and c as they are for the remaining launches of the iteration loop.
__global__ void plain_dot_kernel(const float2* a, const float2* b, int n, double* scal, int epi, int* flags,
                                 double eps2) {
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmaf(a[i].x, b[i].x, fmaf(a[i].y, b[i].y, s));
  s = warp_sum(s);
  __shared__ float red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double d = lane < (int)(blockDim.x >> 5) ? (double)red[lane] : 0.0;
    d = warp_sum_f64(d);
    if (lane == 0) {
      if (epi == kEpiCn0) {
        scal[kCn] = d;
        scal[kStopAt] = eps2 > 0.0 ? eps2 * d : -1.0;
        scal[kStopped] = d <= scal[kStopAt] ? 1.0 : 0.0;
      } else if (epi == kEpiAlpha) {
        scal[kAlpha] = scal[kStopped] != 0.0 ? 0.0 : (d != 0.0 ? scal[kCn] / d : 0.0);
      } else if (scal[kStopped] != 0.0) {
        scal[kBeta] = 0.0;
      } else {
        scal[kBeta] = scal[kCn] != 0.0 ? d / scal[kCn] : 0.0;
        scal[kCn] = d;
        if (d <= scal[kStopAt]) scal[kStopped] = 1.0;
      }
      if (!isfinite(d)) flags[1] = 1;
    }
  }
}

__global__ void plain_init_kernel(const float2* b, float2* x, float2* c, float2* p, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = make_float2(0.f, 0.f);
  c[i] = b[i];
  p[i] = b[i];
}

__global__ void plain_xc_kernel(float2* x, float2* c, const float2* p, const float2* a, const double* scal, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float al = (float)scal[kAlpha];
  x[i].x = fmaf(al, p[i].x, x[i].x);
  x[i].y = fmaf(al, p[i].y, x[i].y);
  c[i].x = fmaf(-al, a[i].x, c[i].x);
  c[i].y = fmaf(-al, a[i].y, c[i].y);
}

__global__ void plain_p_kernel(float2* p, const float2* c, const double* scal, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float be = (float)scal[kBeta];
  p[i].x = fmaf(be, p[i].x, c[i].x);
  p[i].y = fmaf(be, p[i].y, c[i].y);
}

// Embedded pilot: y -= a_pilot H e_(K0,L0) on the normalised DD grid, one thread per path.
__global__ void plain_subtract_kernel(float2* ydd, PlainGeo G, const PathRec* paths, const int* counts, int K0, int L0,
                                      float a_pilot) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= counts[0]) return;
  const PathRec r = paths[p];
  const int kr = (K0 + r.dk) & (G.M - 1), lr = (L0 + r.dl) & (G.N - 1);
  int col;
  const float2 D = fwd_coef(r, kr, lr, G, col);  // col == L0 M + K0 by construction
  const float2 val = cscale(D, a_pilot);
  float2* y = ydd + (size_t)lr * G.M + kr;
  *y = csub(*y, val);
}

__global__ void plain_demap_kernel(const float2* x, int n, const float* lam, int bps, float pam_d, float* llr,
                                   uint8_t* labels) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  float l[6];
  const int hard = qam_llr<float>(x[q], bps, pam_d, 1.0f / *lam, l);
  for (int j = 0; j < bps; ++j) llr[(size_t)q * bps + j] = l[j];
  labels[q] = (uint8_t)hard;
}

// a += lambda p with lambda read from device memory
__global__ void plain_addlam_kernel(float2* a, const float2* p, const float* lam, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float l = *lam;
  a[i].x = fmaf(l, p[i].x, a[i].x);
  a[i].y = fmaf(l, p[i].y, a[i].y);
}

__global__ void plain_pack_kernel(const uint8_t* labels, int nbytes, int bps, uint8_t* bits) {
  const int B = blockIdx.x * blockDim.x + threadIdx.x;
  if (B >= nbytes) return;
  int byte = 0;
  for (int j = 0; j < 8; ++j) {
    const int bit = B * 8 + j;
    const int q = bit / bps, jj = bit - q * bps;
    byte |= ((labels[q] >> (bps - 1 - jj)) & 1) << j;
  }
  bits[B] = (uint8_t)byte;
}

__global__ void plain_status_kernel(const int* flags, int32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *status = flags[1] ? ZOTFS_ENONFINITE : (flags[0] ? ZOTFS_ETRUNCATED : ZOTFS_OK);
}

inline int nblk(int n) { return (n + kBlock - 1) / kBlock; }

}  // namespace

size_t plain_scratch_bytes(int M, int N, int nrx, int ntx, int p_max) {
  return plain_layout(M, N, nrx, ntx, p_max).total;
}

zotfs_status run_plain(zotfs_plan_s* plan, const void* y_pilot_td, const void* y_data_td, const float* noise_var,
                       const float* theta, int iters, const zotfs_paths* paths, float* x_hat, float* llr,
                       uint8_t* bits, int32_t* status, int n_frames, cudaStream_t stream) {
  const int M = plan->M, N = plan->N, MN = M * N, nrx = plan->nrx, ntx = plan->ntx, nl = nrx * ntx;
  const int p_max = plan->opt.p_max, bps = plan->bps;
  const PlainLayout L = plain_layout(M, N, nrx, ntx, p_max);
  char* base = static_cast<char*>(plan->d_plain);
  float2* grid = reinterpret_cast<float2*>(base + L.grid);
  float2* ydd = reinterpret_cast<float2*>(base + L.ydd);
  float2* tv = reinterpret_cast<float2*>(base + L.t);
  float2* xv = reinterpret_cast<float2*>(base + L.x);
  float2* cv = reinterpret_cast<float2*>(base + L.c);
  float2* pv = reinterpret_cast<float2*>(base + L.p);
  float2* av = reinterpret_cast<float2*>(base + L.a);
  PathRec* pl = reinterpret_cast<PathRec*>(base + L.paths);
  int* counts = reinterpret_cast<int*>(base + L.counts);
  double* scal = reinterpret_cast<double*>(base + L.scal);
  int* flags = reinterpret_cast<int*>(base + L.flags);
  uint8_t* labels = reinterpret_cast<uint8_t*>(base + L.labels);
  float* llr_s = reinterpret_cast<float*>(base + L.llr);

  FrameArgs A;
  fill_plan_args(plan, A);
  A.theta = theta;
  if (paths) {
    A.pcount = paths->count;
    A.pstatus = paths->status;
    A.pdk = paths->dk;
    A.pdl = paths->dl;
    A.ph = paths->h;
  }
  PlainGeo G{M, N, plan->logM, plan->logN, nrx, ntx, p_max, plan->d_W};
  const bool emb = plan->opt.pilot_mode == ZOTFS_PILOT_EMBEDDED;
  const size_t in_bytes = (size_t)MN * dtype_bytes(plan->opt.in_dtype);
  const int Tc = MN >= 1024 ? 1024 : MN;  // compaction CTA: MN / Tc <= 16
  const size_t csmem = ((sizeof(SharedHdr) + 127) & ~size_t(127)) + (size_t)MN * sizeof(float2);
  const int EQ = MN / Tc;
  void (*compact)(const FrameArgs, const float2*, int, int, int, PathRec*, int*, int*, int) =
      EQ == 1 ? plain_compact_kernel<1> : EQ == 2 ? plain_compact_kernel<2> : EQ == 4 ? plain_compact_kernel<4>
      : EQ == 8 ? plain_compact_kernel<8> : plain_compact_kernel<16>;
  // above the default 48 KB only when MN >= 8192, where Tc = 1024 fixes csmem per instance
  cudaError_t e = csmem > 48 * 1024
                      ? cudaFuncSetAttribute(compact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem)
                      : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "plain compact smem");
  const float inv_sqrtN = (float)(1.0 / std::sqrt((double)N));
  const int nx = ntx * MN;

  for (int f = 0; f < n_frames; ++f) {
    cudaMemsetAsync(flags, 0, 4 * sizeof(int), stream);
    // ---- channel estimation: pilot grids -> path lists
    if (!emb) {
      for (int t = 0; t < ntx; ++t)
        for (int r = 0; r < nrx; ++r) {
          const char* src = static_cast<const char*>(y_pilot_td) + (((size_t)f * ntx + t) * nrx + r) * in_bytes;
          plain_dzt_kernel<<<nblk(MN), kBlock, 0, stream>>>(src, plan->opt.in_dtype, grid, G, 1, 1.0f);
          compact<<<1, Tc, csmem, stream>>>(A, grid, f, r * ntx + t, f * nl + r * ntx + t, pl, counts,
                                                         flags, paths ? 1 : 0);
          g_launches += 2;
        }
    }
    // ---- data grids
    for (int r = 0; r < nrx; ++r) {
      const char* src = static_cast<const char*>(y_data_td) + ((size_t)f * nrx + r) * in_bytes;
      if (emb) {
        plain_dzt_kernel<<<nblk(MN), kBlock, 0, stream>>>(src, plan->opt.in_dtype, grid, G, 1, 1.0f);
        compact<<<1, Tc, csmem, stream>>>(A, grid, f, 0, f, pl, counts, flags, paths ? 1 : 0);
        g_launches += 2;
      }
      plain_dzt_kernel<<<nblk(MN), kBlock, 0, stream>>>(src, plan->opt.in_dtype, ydd + (size_t)r * MN, G, 0,
                                                        inv_sqrtN);
      ++g_launches;
    }
    if (emb) {
      plain_subtract_kernel<<<nblk(p_max), kBlock, 0, stream>>>(ydd, G, pl, counts, plan->opt.K0, plan->opt.L0,
                                                                (float)plan->opt.a_pilot);
      ++g_launches;
    }
    // ---- CGA (Algorithm 1)
    const float* lamp = noise_var + f;
    plain_apply_kernel<<<nblk(nx), kBlock, 0, stream>>>(G, pl, counts, ydd, cv, 1, 0.f, nullptr);  // b -> c
    plain_init_kernel<<<nblk(nx), kBlock, 0, stream>>>(cv, xv, cv, pv, nx);
    plain_dot_kernel<<<1, 1024, 0, stream>>>(cv, cv, nx, scal, kEpiCn0, flags, A.eps2);
    g_launches += 3;
    for (int it = 0; it < iters; ++it) {
      plain_apply_kernel<<<nblk(nrx * MN), kBlock, 0, stream>>>(G, pl, counts, pv, tv, 0, 0.f, nullptr);
      // a = H^H t, then a += lambda p (lambda stays on the device)
      plain_apply_kernel<<<nblk(nx), kBlock, 0, stream>>>(G, pl, counts, tv, av, 1, 0.f, nullptr);
      g_launches += 2;
      plain_addlam_kernel<<<nblk(nx), kBlock, 0, stream>>>(av, pv, lamp, nx);
      ++g_launches;
      plain_dot_kernel<<<1, 1024, 0, stream>>>(pv, av, nx, scal, kEpiAlpha, flags, A.eps2);
      plain_xc_kernel<<<nblk(nx), kBlock, 0, stream>>>(xv, cv, pv, av, scal, nx);
      plain_dot_kernel<<<1, 1024, 0, stream>>>(cv, cv, nx, scal, kEpiBeta, flags, A.eps2);
      plain_p_kernel<<<nblk(nx), kBlock, 0, stream>>>(pv, cv, scal, nx);
      g_launches += 4;
    }
    if (x_hat) {
      cudaMemcpyAsync(x_hat + (size_t)f * nx * 2, xv, (size_t)nx * sizeof(float2), cudaMemcpyDeviceToDevice, stream);
    }
    // ---- demapping
    if (llr || bits) {
      float* lo = llr ? llr + (size_t)f * nx * bps : llr_s;
      plain_demap_kernel<<<nblk(nx), kBlock, 0, stream>>>(xv, nx, lamp, bps, (float)A.pam_d, lo, labels);
      ++g_launches;
      if (bits) {
        const int nbytes = nx * bps / 8;
        plain_pack_kernel<<<nblk(nbytes), kBlock, 0, stream>>>(labels, nbytes, bps, bits + (size_t)f * nbytes);
        ++g_launches;
      }
    }
    plain_status_kernel<<<1, 32, 0, stream>>>(flags, status + f);
    ++g_launches;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "plain form launch");
  return ZOTFS_OK;
}

}  // namespace zotfs

// ------------------------------------------------------------------------------------
// Equalisation without any allocation: the plain-form CGA with its scratch in a fixed
// array that the library image carries, for callers that may not allocate device memory
// once they are running (see zotfs_equalize_static in include/zotfs.h).
// ------------------------------------------------------------------------------------

namespace zotfs {
namespace {

constexpr int kStaticMaxGrid = 4096;  // M * N
constexpr int kStaticMaxAnt = 4;      // n_rx, n_tx
constexpr int kStaticMaxPaths = 64;   // p_max
constexpr size_t kStaticBytes = 768 * 1024;

// The scratch every zotfs_equalize_static call uses, on every device that loads the library.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};  // device address of g_static_scratch per device

struct StaticLayout {
  size_t W, paths, counts, t, x, c, p, a, scal, flags, total;
};

StaticLayout static_layout(int MN, int nrx, int ntx, int p_max) {
  StaticLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  };
  L.W = take((size_t)MN * sizeof(float2));
  L.paths = take((size_t)nrx * ntx * p_max * sizeof(PathRec));
  L.counts = take((size_t)nrx * ntx * sizeof(int));
  L.t = take((size_t)nrx * MN * sizeof(float2));
  L.x = take((size_t)ntx * MN * sizeof(float2));
  L.c = take((size_t)ntx * MN * sizeof(float2));
  L.p = take((size_t)ntx * MN * sizeof(float2));
  L.a = take((size_t)ntx * MN * sizeof(float2));
  L.scal = take(8 * sizeof(double));
  L.flags = take(4 * sizeof(int));
  L.total = off;
  return L;
}

// W[t] = exp(j 2 pi t / MN) evaluated on the device (sincospi in FP64, rounded to FP32).
__global__ void static_twiddle_kernel(float2* W, int MN) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MN) return;
  double s, c;
  sincospi(2.0 * (double)t / (double)MN, &s, &c);
  W[t] = make_float2((float)c, (float)s);
}

// Caller path lists -> path records (h, dk, dl) the plain operator kernel reads; entries
// outside the centred offset range are zeroed.
__global__ void static_paths_kernel(const int32_t* count, const int16_t* dk, const int16_t* dl, const float2* h,
                                    int nl, int p_max, int M, int N, PathRec* out, int* counts, int* flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nl * p_max) return;
  const int li = i / p_max, p = i - li * p_max;
  int P = count[li];
  if (P < 0 || P > p_max) {
    if (p == 0) flags[2] = 1;
    P = P < 0 ? 0 : p_max;
  }
  if (p == 0) counts[li] = P;
  if (p >= P) return;
  PathRec r;
  r.dk = dk[i];
  r.dl = dl[i];
  r.h = h[i];
  if (r.dk < -(M / 2) || r.dk >= M / 2 || r.dl < -(N / 2) || r.dl >= N / 2) {
    r.dk = r.dl = 0;
    r.h = make_float2(0.f, 0.f);
    flags[2] = 1;
  }
  r.hf = r.h;
  r.pad0 = r.pad1 = 0;
  out[i] = r;
}

__global__ void static_status_kernel(const int* flags, int32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *status = flags[1] ? ZOTFS_ENONFINITE : (flags[2] ? ZOTFS_EINVAL : ZOTFS_OK);
}

}  // namespace
}  // namespace zotfs

extern "C" zotfs_status zotfs_equalize_static(int M, int N, int n_rx, int n_tx, const zotfs_paths* paths,
                                              const float* y_dd, const float* noise_var, int iters, float* x_hat,
                                              int32_t* status, int n_frames, zotfs_stream stream) {
  using namespace zotfs;
  g_launches = 0;
  if (!is_pow2(M) || M < 16 || M > 256 || !is_pow2(N) || N < 8 || N > 64) {
    set_error("zotfs_equalize_static: M, N must be powers of two, 16 <= M <= 256, 8 <= N <= 64");
    return ZOTFS_EINVAL;
  }
  if (M * N > kStaticMaxGrid || n_rx < 1 || n_tx < 1 || n_rx > kStaticMaxAnt || n_tx > kStaticMaxAnt) {
    set_error("zotfs_equalize_static: the fixed scratch holds M*N <= 4096 and at most 4 x 4 antennas");
    return ZOTFS_EUNSUPPORTED;
  }
  if (!paths || !paths->count || !paths->dk || !paths->dl || !paths->h) {
    set_error("zotfs_equalize_static: NULL path list");
    return ZOTFS_EINVAL;
  }
  if (paths->tap_dtype != ZOTFS_C64 || paths->p_max < 1 || paths->p_max > kStaticMaxPaths) {
    set_error("zotfs_equalize_static: path taps must be ZOTFS_C64 with 1 <= p_max <= 64");
    return paths->p_max > kStaticMaxPaths ? ZOTFS_EUNSUPPORTED : ZOTFS_EINVAL;
  }
  if (n_frames < 0 || iters < 0) {
    set_error("zotfs_equalize_static: n_frames and iters must be >= 0");
    return ZOTFS_EINVAL;
  }
  if (n_frames == 0) return ZOTFS_OK;
  if (!y_dd || !noise_var || !x_hat) {
    set_error("zotfs_equalize_static: NULL buffer");
    return ZOTFS_EINVAL;
  }
  const int MN = M * N, nl = n_rx * n_tx, p_max = paths->p_max;
  const StaticLayout L = static_layout(MN, n_rx, n_tx, p_max);
  if (L.total > kStaticBytes) {
    set_error("zotfs_equalize_static: problem larger than the fixed scratch");
    return ZOTFS_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("zotfs_equalize_static: device index out of range");
    return ZOTFS_EUNSUPPORTED;
  }
  char* base;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      g_static_ptr[dev] = ptr;
    }
    base = static_cast<char*>(g_static_ptr[dev]);
  }
  float2* W = reinterpret_cast<float2*>(base + L.W);
  PathRec* pl = reinterpret_cast<PathRec*>(base + L.paths);
  int* counts = reinterpret_cast<int*>(base + L.counts);
  float2* tv = reinterpret_cast<float2*>(base + L.t);
  float2* xv = reinterpret_cast<float2*>(base + L.x);
  float2* cv = reinterpret_cast<float2*>(base + L.c);
  float2* pv = reinterpret_cast<float2*>(base + L.p);
  float2* av = reinterpret_cast<float2*>(base + L.a);
  double* scal = reinterpret_cast<double*>(base + L.scal);
  int* flags = reinterpret_cast<int*>(base + L.flags);
  PlainGeo G{M, N, ilog2(M), ilog2(N), n_rx, n_tx, p_max, W};
  const int nx = n_tx * MN;
  static_twiddle_kernel<<<nblk(MN), kBlock, 0, stream>>>(W, MN);
  ++g_launches;
  for (int f = 0; f < n_frames; ++f) {
    e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(flags)");
    static_paths_kernel<<<nblk(nl * p_max), kBlock, 0, stream>>>(
        paths->count + (size_t)f * nl, paths->dk + (size_t)f * nl * p_max, paths->dl + (size_t)f * nl * p_max,
        reinterpret_cast<const float2*>(paths->h) + (size_t)f * nl * p_max, nl, p_max, M, N, pl, counts, flags);
    const float2* yf = reinterpret_cast<const float2*>(y_dd) + (size_t)f * n_rx * MN;
    const float* lamp = noise_var + f;
    plain_apply_kernel<<<nblk(nx), kBlock, 0, stream>>>(G, pl, counts, yf, cv, 1, 0.f, nullptr);  // b -> c
    plain_init_kernel<<<nblk(nx), kBlock, 0, stream>>>(cv, xv, cv, pv, nx);
    plain_dot_kernel<<<1, 1024, 0, stream>>>(cv, cv, nx, scal, kEpiCn0, flags, 0.0);  // fixed iterations
    g_launches += 4;
    for (int it = 0; it < iters; ++it) {
      plain_apply_kernel<<<nblk(n_rx * MN), kBlock, 0, stream>>>(G, pl, counts, pv, tv, 0, 0.f, nullptr);
      plain_apply_kernel<<<nblk(nx), kBlock, 0, stream>>>(G, pl, counts, tv, av, 1, 0.f, nullptr);
      plain_addlam_kernel<<<nblk(nx), kBlock, 0, stream>>>(av, pv, lamp, nx);
      plain_dot_kernel<<<1, 1024, 0, stream>>>(pv, av, nx, scal, kEpiAlpha, flags, 0.0);
      plain_xc_kernel<<<nblk(nx), kBlock, 0, stream>>>(xv, cv, pv, av, scal, nx);
      plain_dot_kernel<<<1, 1024, 0, stream>>>(cv, cv, nx, scal, kEpiBeta, flags, 0.0);
      plain_p_kernel<<<nblk(nx), kBlock, 0, stream>>>(pv, cv, scal, nx);
      g_launches += 7;
    }
    e = cudaMemcpyAsync(x_hat + (size_t)f * nx * 2, xv, (size_t)nx * sizeof(float2), cudaMemcpyDeviceToDevice,
                        stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(x_hat)");
    if (status) {
      static_status_kernel<<<1, 32, 0, stream>>>(flags, status + f);
      ++g_launches;
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "zotfs_equalize_static launch");
  return ZOTFS_OK;
}
