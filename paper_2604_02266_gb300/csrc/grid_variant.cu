// Instantiations and cooperative launch of the paper-scale grid receiver (frame_grid.cuh).
#include <mutex>

#include "frame_grid.cuh"
#include "internal.h"

namespace zotfs {

namespace {

using GridKern = void (*)(const FrameArgs, GridScratch);

GridKern kern_of(int EQ) {
  switch (EQ) {
    case 8: return grid_kernel<8>;
    case 16: return grid_kernel<16>;
    case 32: return grid_kernel<32>;
    default: return nullptr;
  }
}

cudaError_t grant(int EQ, size_t smem) {
  static std::mutex mu;
  static int granted[3][64] = {{0}};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int slot = EQ == 8 ? 0 : (EQ == 16 ? 1 : 2);
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && granted[slot][dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern_of(EQ), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev < 64) granted[slot][dev] = (int)smem;
  return e;
}

// Self-checks of the bounded device waits (failure detection without a fault): each runs one
// wait against a condition nothing satisfies and stores the outcome.
__global__ void check_mbar_wait_kernel(uint32_t max_polls, int32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, max_polls);  // nothing arrives on the barrier
  if (threadIdx.x == 0) *status = ok ? ZOTFS_OK : ZOTFS_ETIMEOUT;
}

__device__ GridBarrier g_check_bar;

__global__ void check_grid_wait_kernel(uint32_t max_polls, int32_t* status) {
  if (blockIdx.x != 0) return;  // the other CTA leaves without arriving
  unsigned gen = 0;
  const bool ok = grid_sync(&g_check_bar, gen, max_polls);
  if (threadIdx.x == 0) *status = ok ? ZOTFS_OK : ZOTFS_ETIMEOUT;
}

}  // namespace

cudaError_t check_bounded_wait(int which, uint32_t max_polls, int32_t* status, cudaStream_t stream) {
  if (which == 0) {
    check_mbar_wait_kernel<<<1, 32, 0, stream>>>(max_polls, status);
    return cudaGetLastError();
  }
  void* bar = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&bar, g_check_bar);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), stream);
  if (e != cudaSuccess) return e;
  void* params[] = {&max_polls, &status};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(check_grid_wait_kernel), dim3(2), dim3(32), params,
                                     0, stream);
}

bool grid_shape(int M, int N, int nrx, int ntx) {
  return nrx == 1 && ntx == 1 && (M > 256 || M * N > 16384) && M >= kGridDftCols && M <= 16384 && N >= 8 &&
         N <= 64 && (size_t)M * N <= kGridMaxElems;
}

cudaError_t choose_grid_cfg(int M, int N, int p_max, int sm_count, GridCfg& cfg) {
  cfg.smem = grid_smem_bytes(N, p_max);
  cfg.T = kGridThreads;
  cfg.EQ = 0;
  for (int EQ : {8, 16, 32}) {
    cudaError_t e = grant(EQ, cfg.smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern_of(EQ), kGridThreads, cfg.smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) continue;
    if (occ > 2) occ = 2;  // the plan's scratch holds partials for two CTAs per SM
    const int grid = occ * sm_count;
    if (grid > kGridMaxCtas) return cudaErrorInvalidConfiguration;
    if ((long long)grid * kGridThreads * EQ >= (long long)M * N) {
      cfg.EQ = EQ;
      cfg.grid = grid;
      return cudaSuccess;
    }
  }
  return cudaErrorInvalidConfiguration;
}

size_t grid_scratch_size(int M, int N, int p_max, int grid) { return grid_scratch_bytes(M, N, p_max, grid); }

cudaError_t grid_launch(const GridCfg& cfg, const FrameArgs& A, char* scratch, cudaStream_t stream) {
  GridKern k = kern_of(cfg.EQ);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = grant(cfg.EQ, cfg.smem);
  if (e != cudaSuccess) return e;
  GridScratch G = grid_scratch_carve(scratch, A.M, A.N, A.p_max, cfg.grid);
  e = cudaMemsetAsync(G.bar, 0, sizeof(GridBarrier), stream);
  if (e != cudaSuccess) return e;
  FrameArgs args = A;
  void* params[] = {&args, &G};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3((unsigned)cfg.grid),
                                     dim3((unsigned)cfg.T), params, cfg.smem, stream);
}

}  // namespace zotfs
