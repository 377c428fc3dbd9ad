// Instantiations and cooperative launch of the paper-scale grid receiver (frame_grid.cuh).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "frame_grid.cuh"
#include "internal.h"

namespace zotfs {

namespace {

using GridKern = void (*)(const FrameArgs, GridScratch, const GridMaps);

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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver
// library); null when the driver does not provide it.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// The descriptor of one row-major CG extension (rows N + E + 3 of 2 M float2, 8-byte
// elements) with a box of win_cols columns by all rows.
bool encode_ext_map(CUtensorMap* map, float2* ext, int M, int N, int win_cols) {
  EncodeTiled fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * M), (cuuint64_t)(N + kGridE + 3)};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * M) * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)win_cols, (cuuint32_t)(N + kGridE + 3)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, ext, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
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

// The CG windows of one CTA at a given grid: its grid_cols_per_cta columns plus dcap on either
// side (and one for the even start), as much as the shared memory left at `occ` CTAs per SM
// holds, dcap at most M / 2 - 2 (the windows stay inside the extensions' halo) and 128, and the
// window at most 256 columns (the tensor copy's box).
void grid_window(int M, int N, int p_max, int grid, int occ, int smem_per_sm, int smem_reserved, int& cols,
                 int& dcap) {
  cols = 0;
  dcap = -1;
  const int cpc = grid_cols_per_cta(M, grid);
  const long long base = (long long)grid_smem_bytes(N, p_max, 0, cpc);
  const long long avail = (long long)smem_per_sm / occ - smem_reserved - base - 256;  // windows rounded to 128 B
  const long long row_bytes = 2LL * (N + kGridE + 3) * (long long)sizeof(float2);  // both windows, one column
  if (avail <= 0) return;
  const long long wmax = avail / row_bytes;
  int d = (int)std::min<long long>((wmax - cpc - 3) / 2, 128);  // cols below stays <= wmax
  d = std::min(d, M / 2 - 2);
  d = std::min(d, (256 - cpc - 3) / 2);  // a tensor copy's box spans at most 256 columns
  if (d < 1) return;
  dcap = d;
  cols = (cpc + 2 * d + 2 + 1) & ~1;
}

cudaError_t choose_grid_cfg(int M, int N, int p_max, int sm_count, int ctas_per_sm, GridCfg& cfg) {
  int dev = 0, smem_sm = 0, smem_res = 0, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cfg.T = kGridThreads;
  cfg.EQ = 0;
  for (int v = 0; v < kNumGridVariants; ++v) {
    const GridVariant& gv = kGridVariants[v];
    int want = gv.minb;
    if (ctas_per_sm > 0 && want > ctas_per_sm) want = ctas_per_sm;
    if (want > kGridMaxCtasPerSm) want = kGridMaxCtasPerSm;  // the plan's scratch holds partials for that many
    for (int occ_t = want; occ_t >= 1; --occ_t) {
      const int grid = occ_t * sm_count;
      if (grid > kGridMaxCtas) return cudaErrorInvalidConfiguration;
      if ((long long)grid * kGridThreads * gv.EQ < (long long)M * N) break;  // the read-off needs more threads
      // the coefficient table in shared memory (with windows when room is left), else in global
      // memory with no windows
      for (int tab_smem = 1; tab_smem >= 0; --tab_smem) {
        int cols = 0, dcap = -1;
        if (tab_smem) grid_window(M, N, p_max, grid, occ_t, smem_sm, smem_res, cols, dcap);
        const size_t smem = grid_smem_bytes(N, p_max, cols, tab_smem ? grid_cols_per_cta(M, grid) : 0);
        if (smem > (size_t)smem_optin) continue;
        e = grant(v, smem);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gv.k, kGridThreads, smem);
        if (e != cudaSuccess) return e;
        if (occ < occ_t) continue;
        cfg.EQ = gv.EQ;
        cfg.E = gv.E;
        cfg.variant = v;
        cfg.grid = grid;
        cfg.smem = smem;
        cfg.win_cols = cols;
        cfg.win_dcap = dcap;
        cfg.tab_smem = tab_smem;
        return cudaSuccess;
      }
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
  G.win_cols = cfg.win_cols;
  G.win_dcap = cfg.win_dcap;
  G.tab_smem = cfg.tab_smem;
  // the windows' tensor copies; without the descriptors the gathers read global memory
  GridMaps maps;
  memset(&maps, 0, sizeof(maps));
  if (G.win_cols > 0 && !(encode_ext_map(&maps.c, G.extC, A.M, A.N, G.win_cols) &&
                          encode_ext_map(&maps.t, G.extT, A.M, A.N, G.win_cols))) {
    G.win_cols = 0;
    G.win_dcap = -1;
  }
  e = cudaMemsetAsync(G.bar, 0, sizeof(GridBarrier), stream);
  if (e != cudaSuccess) return e;
  FrameArgs args = A;
  void* params[] = {&args, &G, &maps};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), dim3((unsigned)cfg.grid),
                                     dim3((unsigned)cfg.T), params, cfg.smem, stream);
}

}  // namespace zotfs
