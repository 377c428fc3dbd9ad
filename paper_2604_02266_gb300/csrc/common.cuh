// Device helpers shared by the zotfs kernels: complex arithmetic on float2, packed
// FP32x2 FMAs, warp/block reductions with an FP64 combine, and the mbarrier + bulk-copy
// (TMA, non-tensor) primitives used to stage frames in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/zotfs.h"

namespace zotfs {

// ------------------------------------------------------------------ complex float2

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// d = a * b + c on both lanes (sm_100+ packed FP32 FMA)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// complex double
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 conjf2(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// Real/complex type pair of the arithmetic precision R (float or double).
template <typename R> struct Cx;
template <> struct Cx<float> {
  using C = float2;
  using Key = uint32_t;  // order-preserving bit pattern of a non-negative value
  static constexpr int kIoDtype = ZOTFS_C64;
  __device__ static __forceinline__ C make(float a, float b) { return make_float2(a, b); }
  __device__ static __forceinline__ Key key(float v) { return __float_as_uint(v); }
  __device__ static __forceinline__ Key key_inf() { return 0x7f800000u; }
};
template <> struct Cx<double> {
  using C = double2;
  using Key = unsigned long long;
  static constexpr int kIoDtype = ZOTFS_C128;
  __device__ static __forceinline__ C make(double a, double b) { return make_double2(a, b); }
  __device__ static __forceinline__ Key key(double v) { return (Key)__double_as_longlong(v); }
  __device__ static __forceinline__ Key key_inf() { return 0x7ff0000000000000ull; }
};

// acc += D * v for a complex coefficient D split as (DX, DY) = ({Dr, Dr}, {Di, Di}) and two
// partial accumulators: A collects Dr*v, B collects Di*v; the product is
// (A.x - B.y, A.y + B.x).  FP32 uses packed FMAs.
__device__ __forceinline__ void cmac_split(float2& A, float2& B, float2 DX, float2 DY, float2 v) {
  A = ffma2(DX, v, A);
  B = ffma2(DY, v, B);
}
__device__ __forceinline__ void cmac_split(double2& A, double2& B, double2 DX, double2 DY, double2 v) {
  A.x = fma(DX.x, v.x, A.x);
  A.y = fma(DX.y, v.y, A.y);
  B.x = fma(DY.x, v.x, B.x);
  B.y = fma(DY.y, v.y, B.y);
}

// ---------------------------------------------------------------- element loads

// Read element e of a complex array stored as float64, float32, float16 or bfloat16 pairs.
template <typename C>
__device__ __forceinline__ C load_complex(const void* base, size_t e, int dtype);
template <>
__device__ __forceinline__ float2 load_complex<float2>(const void* base, size_t e, int dtype) {
  if (dtype == ZOTFS_C64) return reinterpret_cast<const float2*>(base)[e];
  if (dtype == ZOTFS_C32_F16) return __half22float2(reinterpret_cast<const __half2*>(base)[e]);
  if (dtype == ZOTFS_C32_BF16) return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(base)[e]);
  const double2 d = reinterpret_cast<const double2*>(base)[e];
  return make_float2((float)d.x, (float)d.y);
}
template <>
__device__ __forceinline__ double2 load_complex<double2>(const void* base, size_t e, int dtype) {
  if (dtype == ZOTFS_C128) return reinterpret_cast<const double2*>(base)[e];
  const float2 f = load_complex<float2>(base, e, dtype);
  return make_double2(f.x, f.y);
}
__device__ __forceinline__ void store_complex(void* base, size_t e, int dtype, float2 v) {
  if (dtype == ZOTFS_C64) reinterpret_cast<float2*>(base)[e] = v;
  else if (dtype == ZOTFS_C32_F16) reinterpret_cast<__half2*>(base)[e] = __float22half2_rn(v);
  else if (dtype == ZOTFS_C32_BF16) reinterpret_cast<__nv_bfloat162*>(base)[e] = __float22bfloat162_rn(v);
  else reinterpret_cast<double2*>(base)[e] = make_double2(v.x, v.y);
}
__device__ __forceinline__ void store_complex(void* base, size_t e, int dtype, double2 v) {
  if (dtype == ZOTFS_C128) reinterpret_cast<double2*>(base)[e] = v;
  else store_complex(base, e, dtype, make_float2((float)v.x, (float)v.y));
}
__host__ __device__ __forceinline__ int dtype_bytes(int dtype) {
  return dtype == ZOTFS_C128 ? 16 : dtype == ZOTFS_C64 ? 8 : 4;
}

// ------------------------------------------------------------ frame-scope barriers

// Barrier over the threads working on one frame.  A kernel launched with a one-dimensional
// block runs one frame per CTA at a time: the CTA barrier.  The frame kernel launched with a
// two-dimensional block packs blockDim.y frames into a CTA, blockDim.x threads (whole warps)
// each: row threadIdx.y synchronises on its own named barrier 1 + threadIdx.y, so the frames of
// one CTA never wait for each other.  Every helper below works on one frame: threadIdx.x and
// blockDim.x are the thread's index in, and the size of, its frame's row.
__device__ __forceinline__ void frame_sync() {
  if (blockDim.y == 1) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + threadIdx.y), "r"(blockDim.x) : "memory");
  }
}
// frame_sync() that also returns whether `pred` is nonzero in any thread of the frame.
__device__ __forceinline__ int frame_sync_or(int pred) {
  if (blockDim.y == 1) return __syncthreads_or(pred);
  int out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"(pred), "r"(1 + threadIdx.y), "r"(blockDim.x)
      : "memory");
  return out;
}

// ------------------------------------------------------------------- reductions

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive prefix sum of one int per thread; also returns the total.
// scratch: >= 33 ints of shared memory.  Two barriers; safe to call back to back.
__device__ __forceinline__ int block_exclusive_scan(int v, int* scratch, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) scratch[warp] = inc;
  frame_sync();
  if (warp == 0) {
    int w = lane < nwarps ? scratch[lane] : 0;
    int winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int n = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += n;
    }
    scratch[lane] = winc - w;  // exclusive offset of warp `lane`
    if (lane == 31) scratch[32] = winc;
  }
  frame_sync();
  total = scratch[32];
  const int off = scratch[warp];
  frame_sync();  // scratch may be reused by the next call
  return off + inc - v;
}

// Block-wide sum of one int per thread (two barriers).
__device__ __forceinline__ int block_sum_i(int v, int* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
  v = warp_sum_i(v);
  if (lane == 0) scratch[warp] = v;
  frame_sync();
  int t = 0;
  for (int w = 0; w < nwarps; ++w) t += scratch[w];
  frame_sync();
  return t;
}

// --------------------------------------------------- mbarrier + bulk async copy

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One elected thread: arm the barrier for `bytes` and start a global -> shared bulk copy.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of the barrier: gives up after `max_polls` polls
// (each try_wait itself suspends for a hardware-chosen interval) and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t max_polls) {
  for (uint32_t i = 0; i < max_polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace zotfs
