// SS-MRC: the maximal-ratio-combining decision-feedback equaliser of Sec. III-B
// ("Equalization", MRC paragraph) on the structured-sparse path list, one frame per warp.
//
// The equaliser walks the delay bins k = 0 .. M-1 in order, iteration after iteration (decision
// feedback is sequential over the symbol vectors), so one frame has only N-wide parallelism per
// step: a warp owns a frame, lane n the time index n (two for N = 64), and the CTA's warps work
// on different frames with no block barrier at all.
//
// Domain.  The combining runs on the delay-time (DT) grid, X_dt[k, n] = N^-1/2 sum_l
// X_dd[k, l] exp(j2pi n l/N); the received DT grid of a time-domain frame is the frame itself,
// y_dt[k, n] = y[k + n M].  There the operator of Sec. IV-B (Eq. sparse_mvm with the wrap count
// and twisted phase of Eq. map_chMatDD_col) splits into delay branches: the paths of delay offset
// d carry symbol vector k to received vector kt = <k + d>_M, element n landing at time
// <n + f>_N, f = floor((k + d)/M), through the diagonal gain
//     G_{k,d}[n] = sum_{p: dk_p = d} h_p W[dl_p (k + n M)],   W[t] = exp(j2pi t/(MN)).
// A branch is a diagonal gain and a cyclic shift, so the normal matrix of a symbol vector is
// diagonal, D_k[n] = sum_d |G_{k,d}[n]|^2, and each step is
//     c      = x_dt[k] + D^-1 sum_d conj(G_{k,d}) dy[kt_d, n + f_d]       (MRC, interference of
//                                                                          the current estimates
//                                                                          cancelled)
//     x_dd[k] = nearest QAM points of DFT(c)   (decision, Eq. demod)
//     dy[kt_d, n + f_d] -= G_{k,d} (x_dt_new[k] - x_dt_old[k])             (feedback)
// with dy = y - H x_hat the residual, kept in shared memory.  Decisions are kept as level
// indices (one byte per bin); the soft estimate DFT(c) of the last iteration is x_hat.
//
// The per-row DFT and its inverse are radix-2 butterflies across the warp's lanes
// (__shfl_xor_sync): decimation in frequency leaves the DD values in bit-reversed lane order,
// which the decisions are stored in, and the inverse (decimation in time) takes them back to
// natural time order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace zotfs {
namespace {

struct MrcArgs {
  int M, N, logM, logN, p_max, in_dtype, tap_dtype, y_is_dd, iters, n_frames, hb, warps;
  float pam_d, inv_sqrtN;
  const float2* W;  // W[t] = exp(j2pi t/(MN)), t < MN
  const void* y;
  const int32_t* pcount;
  const int16_t* pdk;
  const int16_t* pdl;
  const void* ph;
  float* x_hat;
  int32_t* status;
  int* work_counter;
};

// Shared memory of one warp (one frame), 16-byte aligned pieces.
struct MrcSmem {
  size_t dy, lab, hs, dls, dks, tmp, brd, brs, total;
};
__host__ __device__ inline MrcSmem mrc_smem_layout(int MN, int p_max) {
  MrcSmem L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 15) & ~size_t(15);
    return o;
  };
  L.dy = take((size_t)MN * sizeof(float2));
  L.lab = take((size_t)MN);
  L.hs = take((size_t)p_max * sizeof(float2));
  L.dls = take((size_t)p_max * sizeof(int));
  L.dks = take((size_t)p_max * sizeof(int));
  L.tmp = take((size_t)p_max * sizeof(int));
  L.brd = take((size_t)p_max * sizeof(int));
  L.brs = take((size_t)(p_max + 1) * sizeof(int));
  L.total = off;
  return L;
}

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGainRegs = 8;  // branch gains (times elements per lane) kept in registers per step
constexpr uint8_t kNoDecision = 0xff;  // x_hat = 0 before the first decision

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}

// Forward unitary DFT along the warp's N elements (element e of lane holds index lane + 32 e):
// decimation in frequency, natural order in, bit-reversed order out.
template <int EPL>
__device__ __forceinline__ void warp_dft(float2 (&a)[EPL], const MrcArgs& A, const float2* wN, int lane) {
  const int N = A.N;
  int h = N >> 1;
  if (EPL == 2) {  // N = 64: the span-32 stage pairs the lane's two elements
    const float2 w = conjf2(wN[lane]);  // exp(-j2pi lane/64)
    const float2 u = a[0], v = a[EPL - 1];
    a[0] = cadd(u, v);
    a[EPL - 1] = cmul(csub(u, v), w);
    h = 16;
  }
  for (; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const int j = lane & (h - 1);
    const float2 w = conjf2(wN[j * (N / (2 * h))]);  // exp(-j2pi j/(2h))
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const float2 p = shfl_xor2(a[e], h);
      a[e] = upper ? cmul(csub(p, a[e]), w) : cadd(a[e], p);
    }
  }
#pragma unroll
  for (int e = 0; e < EPL; ++e) a[e] = cscale(a[e], A.inv_sqrtN);
}

// Inverse unitary DFT: decimation in time, bit-reversed order in, natural order out.
template <int EPL>
__device__ __forceinline__ void warp_idft(float2 (&a)[EPL], const MrcArgs& A, const float2* wN, int lane) {
  const int N = A.N;
  const int hmax = N < 32 ? N : 32;
  for (int h = 1; h < hmax; h <<= 1) {
    const bool upper = (lane & h) != 0;
    const int j = lane & (h - 1);
    const float2 w = wN[j * (N / (2 * h))];  // exp(+j2pi j/(2h))
#pragma unroll
    for (int e = 0; e < EPL; ++e) {
      const float2 p = shfl_xor2(a[e], h);
      a[e] = upper ? csub(p, cmul(a[e], w)) : cadd(a[e], cmul(p, w));
    }
  }
  if (EPL == 2) {
    const float2 w = wN[lane];  // exp(+j2pi lane/64)
    const float2 u = a[0], t = cmul(a[EPL - 1], w);
    a[0] = cadd(u, t);
    a[EPL - 1] = csub(u, t);
  }
#pragma unroll
  for (int e = 0; e < EPL; ++e) a[e] = cscale(a[e], A.inv_sqrtN);
}

__device__ __forceinline__ float2 level_point(uint8_t lab, int m, float d) {
  if (lab == kNoDecision) return make_float2(0.f, 0.f);
  const int iI = lab >> 3, iQ = lab & 7;
  return make_float2((float)(2 * iI - (m - 1)) * d, (float)(2 * iQ - (m - 1)) * d);
}

__device__ __forceinline__ int nearest_level(float x, int m, float d) {
  const int i = __float2int_rn(0.5f * (x / d + (float)(m - 1)));
  return i < 0 ? 0 : (i > m - 1 ? m - 1 : i);
}

// Gain of branch b (paths [s, e) of the sorted list) for source delay k at time index n:
// sum_p h_p W[dl_p (k + n M)] = sum_p (h_p W[dl_p k]) exp(j2pi dl_p n / N).  The first factor,
// the same in every lane, is formed once per delay bin for all paths (hk, shared memory); the
// second comes from the N-entry shared table wN.  (Reading W[dl_p (k + n M)] directly puts the
// lanes dl_p M entries apart in the MN-entry table: 32 cache lines per load.)
__device__ __forceinline__ float2 branch_gain(const MrcArgs& A, const float2* wN, const float2* hk_all, const int* dls,
                                              int s, int e, int n) {
  const int N = A.N;
  float2 G = make_float2(0.f, 0.f);
  for (int p = s; p < e; ++p) {
    const int dl = dls[p];
    const float2 hk = hk_all[p];
    const float2 w = wN[(dl * n) & (N - 1)];
    G.x = fmaf(hk.x, w.x, fmaf(-hk.y, w.y, G.x));
    G.y = fmaf(hk.x, w.y, fmaf(hk.y, w.x, G.y));
  }
  return G;
}

template <int EPL>
__global__ void __launch_bounds__(384) mrc_kernel(const __grid_constant__ MrcArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = A.M, N = A.N, MN = M * N, logN = A.logN;
  const int m = 1 << A.hb;
  const float d = A.pam_d;
  const MrcSmem L = mrc_smem_layout(MN, A.p_max);
  // wN[j] = exp(j2pi j / N) = W[j M], shared by the CTA's warps, after their slices
  float2* wN = reinterpret_cast<float2*>(smem + (size_t)A.warps * L.total);
  for (int j = threadIdx.x; j < N; j += blockDim.x) wN[j] = __ldg(A.W + (size_t)j * M);
  __syncthreads();
  unsigned char* base = smem + (size_t)warp * L.total;
  float2* dy = reinterpret_cast<float2*>(base + L.dy);  // residual, DT layout [k][n]
  uint8_t* lab = base + L.lab;                           // decisions [k][bit-reversed l]
  float2* hs = reinterpret_cast<float2*>(base + L.hs);
  int* dls = reinterpret_cast<int*>(base + L.dls);
  int* dks = reinterpret_cast<int*>(base + L.dks);
  int* tmp = reinterpret_cast<int*>(base + L.tmp);
  int* brd = reinterpret_cast<int*>(base + L.brd);
  int* brs = reinterpret_cast<int*>(base + L.brs);

  for (;;) {
    int f = 0;
    if (lane == 0) f = atomicAdd(A.work_counter, 1);
    f = __shfl_sync(kFull, f, 0);
    if (f >= A.n_frames) break;

    // ---- path list: load, validate, sort by delay offset (stable), cut into branches
    int P = A.pcount[f];
    int bad = 0;
    if (P < 0 || P > A.p_max) {
      bad = 1;
      P = P < 0 ? 0 : A.p_max;
    }
    const size_t lb = (size_t)f * A.p_max;
    for (int p = lane; p < P; p += 32) {
      int dk = A.pdk[lb + p], dl = A.pdl[lb + p];
      float2 h = load_complex<float2>(A.ph, lb + p, A.tap_dtype);
      if (dk < -(M >> 1) || dk >= (M >> 1) || dl < -(N >> 1) || dl >= (N >> 1)) {
        bad = 1;
        dk = dl = 0;
        h = make_float2(0.f, 0.f);
      }
      tmp[p] = dk;
      hs[p] = h;       // unsorted for now
      dls[p] = dl;
    }
    bad = __any_sync(kFull, bad);
    __syncwarp();
    // rank of path p: paths with a smaller offset, or the same offset and a lower index
    float2 hv[8];
    int dlv[8], rk[8], dkv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int p = lane + 32 * i;
      rk[i] = -1;
      if (p < P) {
        const int key = tmp[p];
        int r = 0;
        for (int q = 0; q < P; ++q) {
          const int kq = tmp[q];
          r += (kq < key) || (kq == key && q < p);
        }
        rk[i] = r;
        hv[i] = hs[p];
        dlv[i] = dls[p];
        dkv[i] = key;
      }
    }
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (rk[i] >= 0) {
        hs[rk[i]] = hv[i];
        dls[rk[i]] = dlv[i];
        dks[rk[i]] = dkv[i];
      }
    __syncwarp();
    int nb = 0;
    for (int p0 = 0; p0 < P; p0 += 32) {
      const int p = p0 + lane;
      const bool head = p < P && (p == 0 || dks[p] != dks[p - 1]);
      const unsigned hm = __ballot_sync(kFull, head);
      if (head) {
        const int b = nb + __popc(hm & ((1u << lane) - 1u));
        brd[b] = dks[p];
        brs[b] = p;
      }
      nb += __popc(hm);
    }
    if (lane == 0) brs[nb] = P;
    // h_p W[dl_p k] of every path for the delay bin being processed, in the space of the sort's
    // keys and ranks (dks and tmp, free once the branches are cut: together >= 8 p_max bytes)
    float2* hk = reinterpret_cast<float2*>(dks);

    // ---- received DT grid into the residual (dy = y - H 0)
    if (!A.y_is_dd) {
      const size_t fb = (size_t)f * MN;
      for (int i = lane; i < MN; i += 32) {
        const int k = i & (M - 1), n = i >> A.logM;  // sample i = k + n M
        dy[k * N + n] = load_complex<float2>(A.y, fb + i, A.in_dtype);
      }
    } else {
      const float2* yd = static_cast<const float2*>(A.y) + (size_t)f * MN;
      for (int k = 0; k < M; ++k) {
        float2 a[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int pos = lane + 32 * e;  // position pos holds DD bin bitrev(pos)
          const int l = pos < N ? (int)(__brev((unsigned)pos) >> (32 - logN)) : 0;
          a[e] = pos < N ? yd[(size_t)l * M + k] : make_float2(0.f, 0.f);
        }
        warp_idft<EPL>(a, A, wN, lane);
#pragma unroll
        for (int e = 0; e < EPL; ++e)
          if (lane + 32 * e < N) dy[k * N + lane + 32 * e] = a[e];
      }
    }
    for (int i = lane; i < MN; i += 32) lab[i] = kNoDecision;
    __syncwarp();

    // ---- decision-feedback MRC sweeps
    bool finite = true;
    if (A.iters == 0 && A.x_hat)
      for (int i = lane; i < MN; i += 32) reinterpret_cast<float2*>(A.x_hat)[(size_t)f * MN + i] = make_float2(0.f, 0.f);
    for (int it = 0; it < A.iters; ++it) {
      const bool last = it + 1 == A.iters;
      for (int k = 0; k < M; ++k) {
        float2 old[EPL], g[EPL], c[EPL];
        float D[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int pos = lane + 32 * e;
          old[e] = level_point(pos < N ? lab[k * N + pos] : kNoDecision, m, d);
          g[e] = make_float2(0.f, 0.f);
          D[e] = 0.f;
        }
        if (it > 0) warp_idft<EPL>(old, A, wN, lane);  // current estimate of vector k, DT
        for (int p = lane; p < P; p += 32) hk[p] = cmul(hs[p], __ldg(A.W + ((dls[p] * k) & (MN - 1))));
        __syncwarp();
        // combining over the branches; the first kGainRegs / EPL branches' gains stay in
        // registers for the feedback below (the rest are formed again there)
        auto combine = [&](int b, float2 (&Gb)[EPL]) {
          const int dd = brd[b], kt = (k + dd) & (M - 1), fsh = (k + dd) >> A.logM;
#pragma unroll
          for (int e = 0; e < EPL; ++e) {
            const int n = lane + 32 * e;
            if (n < N) {
              const float2 G = branch_gain(A, wN, hk, dls, brs[b], brs[b + 1], n);
              Gb[e] = G;
              const float2 r = dy[kt * N + ((n + fsh) & (N - 1))];
              g[e].x = fmaf(G.x, r.x, fmaf(G.y, r.y, g[e].x));  // conj(G) r
              g[e].y = fmaf(G.x, r.y, fmaf(-G.y, r.x, g[e].y));
              D[e] = fmaf(G.x, G.x, fmaf(G.y, G.y, D[e]));
            }
          }
        };
        constexpr int kB = kGainRegs / EPL;
        float2 Gc[kB][EPL];
#pragma unroll
        for (int b = 0; b < kB; ++b)
          if (b < nb) combine(b, Gc[b]);
        for (int b = kB; b < nb; ++b) {
          float2 Gt[EPL];
          combine(b, Gt);
        }
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          c[e] = old[e];
          if (D[e] > 0.f) {
            const float inv = 1.f / D[e];
            c[e].x = fmaf(g[e].x, inv, c[e].x);
            c[e].y = fmaf(g[e].y, inv, c[e].y);
          }
        }
        warp_dft<EPL>(c, A, wN, lane);  // c: DD values at bit-reversed positions
        float2 s[EPL];
        uint8_t nl[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int iI = nearest_level(c[e].x, m, d), iQ = nearest_level(c[e].y, m, d);
          nl[e] = (uint8_t)((iI << 3) | iQ);
          s[e] = level_point(nl[e], m, d);
          const int pos = lane + 32 * e;
          if (pos < N) {
            finite = finite && isfinite(c[e].x) && isfinite(c[e].y);
            if (last && A.x_hat) {
              const int l = (int)(__brev((unsigned)pos) >> (32 - logN));
              reinterpret_cast<float2*>(A.x_hat)[(size_t)f * MN + (size_t)l * M + k] = c[e];
            }
          }
        }
        warp_idft<EPL>(s, A, wN, lane);  // new estimate of vector k, DT
        float2 delta[EPL];
#pragma unroll
        for (int e = 0; e < EPL; ++e) delta[e] = csub(s[e], old[e]);
        __syncwarp();  // every lane's reads of dy for this step are done
        auto feed_back = [&](int b, const float2* Gb) {
          const int dd = brd[b], kt = (k + dd) & (M - 1), fsh = (k + dd) >> A.logM;
#pragma unroll
          for (int e = 0; e < EPL; ++e) {
            const int n = lane + 32 * e;
            if (n < N) {
              const float2 G = Gb ? Gb[e] : branch_gain(A, wN, hk, dls, brs[b], brs[b + 1], n);
              float2* r = dy + kt * N + ((n + fsh) & (N - 1));
              *r = csub(*r, cmul(G, delta[e]));
            }
          }
        };
#pragma unroll
        for (int b = 0; b < kB; ++b)
          if (b < nb) feed_back(b, Gc[b]);
        for (int b = kB; b < nb; ++b) feed_back(b, nullptr);
#pragma unroll
        for (int e = 0; e < EPL; ++e)
          if (lane + 32 * e < N) lab[k * N + lane + 32 * e] = nl[e];
        __syncwarp();  // the residual and the decisions of vector k are final
      }
    }
    finite = __all_sync(kFull, finite);
    if (A.status && lane == 0)
      A.status[f] = !finite ? ZOTFS_ENONFINITE : (bad ? ZOTFS_EINVAL : ZOTFS_OK);
    __syncwarp();  // the next frame's list may overwrite the tables
  }
}

}  // namespace
}  // namespace zotfs

extern "C" zotfs_status zotfs_equalize_mrc(zotfs_plan plan, const void* y, int y_is_dd, const zotfs_paths* paths,
                                           int iters, float* x_hat, int32_t* status, int n_frames,
                                           zotfs_stream stream) {
  using namespace zotfs;
  g_launches = 0;
  if (!plan) {
    set_error("plan is NULL");
    return ZOTFS_EINVAL;
  }
  if (n_frames < 0 || iters < 0) {
    set_error("n_frames and iters must be >= 0");
    return ZOTFS_EINVAL;
  }
  if (!paths || !paths->count || !paths->dk || !paths->dl || !paths->h) {
    set_error("paths: NULL pointer");
    return ZOTFS_EINVAL;
  }
  if (paths->p_max != plan->opt.p_max || paths->tap_dtype != plan->opt.tap_dtype) {
    set_error("paths.p_max / tap_dtype differ from the plan's");
    return ZOTFS_EINVAL;
  }
  if (plan->nrx != 1 || plan->ntx != 1 || plan->opt.compute != ZOTFS_COMPUTE_FP32 ||
      plan->opt.pilot_mode != ZOTFS_PILOT_SEPARATE || plan->M > 256 || plan->M * plan->N > 16384 ||
      plan->opt.p_max > 256) {
    set_error("zotfs_equalize_mrc: SISO FP32 plans with separate pilot frames, M <= 256, M*N <= 16384, "
              "p_max <= 256");
    return ZOTFS_EUNSUPPORTED;
  }
  if (n_frames == 0) return ZOTFS_OK;
  if (!y) {
    set_error("y is NULL");
    return ZOTFS_EINVAL;
  }
  MrcArgs A;
  std::memset(&A, 0, sizeof(A));
  A.M = plan->M;
  A.N = plan->N;
  A.logM = plan->logM;
  A.logN = plan->logN;
  A.p_max = plan->opt.p_max;
  A.in_dtype = y_is_dd ? ZOTFS_C64 : plan->opt.in_dtype;
  A.tap_dtype = plan->opt.tap_dtype;
  A.y_is_dd = y_is_dd ? 1 : 0;
  A.iters = iters;
  A.n_frames = n_frames;
  A.hb = plan->bps / 2;
  A.pam_d = (float)std::sqrt(3.0 / (2.0 * (plan->qam - 1)));
  A.inv_sqrtN = (float)(1.0 / std::sqrt((double)plan->N));
  A.W = plan->d_W;
  A.y = y;
  A.pcount = paths->count;
  A.pdk = paths->dk;
  A.pdl = paths->dl;
  A.ph = paths->h;
  A.x_hat = x_hat;
  A.status = status;
  const size_t per_warp = mrc_smem_layout(plan->M * plan->N, A.p_max).total;
  const size_t kSmemCap = 227 * 1024;
  int warps = (int)std::min<size_t>(12, (kSmemCap - (size_t)plan->N * sizeof(float2)) / per_warp);
  if (warps < 1) {
    set_error("zotfs_equalize_mrc: frame does not fit one SM's shared memory");
    return ZOTFS_EUNSUPPORTED;
  }
  // no more warps (frames) per CTA than it takes to give every SM a CTA: a frame is one warp's
  // sequential work, so frames crowded onto fewer SMs only wait for each other
  const int spread = (int)std::max<long long>(1, ((long long)n_frames + plan->sm_count - 1) / plan->sm_count);
  warps = std::min(warps, spread);
  A.warps = warps;
  const size_t smem = per_warp * warps + (size_t)plan->N * sizeof(float2);
  int* counter = plan->d_counters + (plan->counter_next++ & 63);
  A.work_counter = counter;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work counter)");
  const bool two = plan->N > 32;
  auto kern = two ? mrc_kernel<2> : mrc_kernel<1>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mrc)");
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, 32 * warps, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query (mrc)");
  if (blocks < 1) {
    set_error("zotfs_equalize_mrc: kernel does not fit on an SM");
    return ZOTFS_EUNSUPPORTED;
  }
  long long grid = (long long)plan->sm_count * blocks;
  const long long need = (n_frames + warps - 1) / warps;
  if (grid > need) grid = need;
  kern<<<(int)grid, 32 * warps, smem, stream>>>(A);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "mrc kernel launch");
  ++g_launches;
  return ZOTFS_OK;
}
