// Instantiations of the large-frame kernel (FP32; EW = rows per thread = MN / T).
#include <mutex>

#include "frame_big.cuh"
#include "internal.h"

namespace zotfs {

using BigKern = void (*)(const FrameArgs, int, char*, size_t);

static BigKern big_kern(int EW) {
  switch (EW) {
    case 8: return big_kernel<float, 8>;
    case 16: return big_kernel<float, 16>;
    case 32: return big_kernel<float, 32>;
    default: return nullptr;
  }
}

bool choose_big_cfg(int M, int N, int nrx, int ntx, int p_max, BigCfg& cfg) {
  const int MN = M * N;
  const int T = MN / 8 < kBigThreads ? MN / 8 : kBigThreads;
  const int EW = MN / T;
  if (T < 32 || (T % 32) != 0 || (T % M) != 0 || EW % kBigChunk != 0 || !big_kern(EW)) return false;
  if ((N % EW) != 0) return false;
  cfg.T = T;
  cfg.EW = EW;
  cfg.smem = big_smem_bytes(nrx, ntx, p_max, 4);
  cfg.slot_bytes = ((big_slot_elems(M, N, nrx, ntx) * sizeof(float2)) + 255) & ~size_t(255);
  return cfg.smem <= 227 * 1024;
}

// Raise a large-frame kernel's dynamic shared-memory limit to at least `smem` on the current
// device; the limit only grows (see grant_smem of the frame kernels).
static cudaError_t big_grant_smem(int EW, size_t smem) {
  static std::mutex mu;
  static int granted[3][64] = {{0}};
  const int slot = EW == 8 ? 0 : (EW == 16 ? 1 : 2);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && granted[slot][dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(big_kern(EW), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev < 64) granted[slot][dev] = (int)smem;
  return e;
}

cudaError_t big_launch(const BigCfg& cfg, const FrameArgs& A, int radix, int grid, char* scratch,
                       cudaStream_t stream) {
  BigKern k = big_kern(cfg.EW);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = big_grant_smem(cfg.EW, cfg.smem);
  if (e != cudaSuccess) return e;
  k<<<grid, cfg.T, cfg.smem, stream>>>(A, radix, scratch, cfg.slot_bytes);
  return cudaGetLastError();
}

cudaError_t big_occupancy(const BigCfg& cfg, int& blocks) {
  BigKern k = big_kern(cfg.EW);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = big_grant_smem(cfg.EW, cfg.smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k, cfg.T, cfg.smem);
}

}  // namespace zotfs
