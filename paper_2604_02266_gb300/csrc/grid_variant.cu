// Instantiations and cooperative launch of the paper-scale grid receiver (frame_grid.cuh).
#include <mutex>

#include "frame_grid.cuh"
#include "internal.h"

namespace zotfs {

namespace {

using GridKern = void (*)(const FrameArgs, GridScratch);

// Instantiations: (read-off entries per thread EQ, CG rows per item E, CTAs per SM MINB).
// Items of 4 rows at three CTAs per SM were measured slower than 8 rows at two (0.86 against
// 0.56 ms per 16384 x 32 packet: the per-path work of a gather is amortised over half the rows,
// and 80 registers spill), so every variant takes 8-row items.
struct GridVariant {
  int EQ, E, minb;
  GridKern k;
};
const GridVariant kGridVariants[] = {
    {8, 8, 2, grid_kernel<8, 8, 2>}, {16, 8, 2, grid_kernel<16, 8, 2>}, {32, 8, 2, grid_kernel<32, 8, 2>}};
constexpr int kNumGridVariants = sizeof(kGridVariants) / sizeof(kGridVariants[0]);

cudaError_t grant(int v, size_t smem) {
  static std::mutex mu;
  static int granted[kNumGridVariants][64] = {{0}};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && granted[v][dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kGridVariants[v].k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev < 64) granted[v][dev] = (int)smem;
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

cudaError_t choose_grid_cfg(int M, int N, int p_max, int sm_count, int ctas_per_sm, GridCfg& cfg) {
  cfg.smem = grid_smem_bytes(N, p_max);
  cfg.T = kGridThreads;
  cfg.EQ = 0;
  for (int v = 0; v < kNumGridVariants; ++v) {
    const GridVariant& gv = kGridVariants[v];
    cudaError_t e = grant(v, cfg.smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gv.k, kGridThreads, cfg.smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) continue;
    if (occ > gv.minb) occ = gv.minb;
    if (ctas_per_sm > 0 && occ > ctas_per_sm) occ = ctas_per_sm;
    if (occ > kGridMaxCtasPerSm) occ = kGridMaxCtasPerSm;  // the plan's scratch holds partials for that many
    const int grid = occ * sm_count;
    if (grid > kGridMaxCtas) return cudaErrorInvalidConfiguration;
    if ((long long)grid * kGridThreads * gv.EQ >= (long long)M * N) {
      cfg.EQ = gv.EQ;
      cfg.E = gv.E;
      cfg.variant = v;
      cfg.grid = grid;
      return cudaSuccess;
    }
  }
  return cudaErrorInvalidConfiguration;
}

size_t grid_scratch_size(int M, int N, int p_max, int grid) { return grid_scratch_bytes(M, N, p_max, grid); }

cudaError_t grid_launch(const GridCfg& cfg, const FrameArgs& A, char* scratch, cudaStream_t stream) {
  if (cfg.variant < 0 || cfg.variant >= kNumGridVariants) return cudaErrorInvalidValue;
  GridKern k = kGridVariants[cfg.variant].k;
  cudaError_t e = grant(cfg.variant, cfg.smem);
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
