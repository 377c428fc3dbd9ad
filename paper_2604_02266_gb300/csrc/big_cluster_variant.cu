// Instantiations and launch of the clustered large-frame receiver (frame_big_cluster.cuh):
// EQ = M N / T read-off elements per thread, CL CTAs per frame, EQ / CL in {8, 16} CG rows per
// thread.
#include <mutex>

#include "frame_big_cluster.cuh"
#include "internal.h"

namespace zotfs {

namespace {

using BigClusterKern = void (*)(const FrameArgs, int, char*, size_t);

// T <= 256 gets its own instantiation: its bound leaves the read-off twice the registers.
BigClusterKern kern_of(int EQ, int CL, int T) {
  if (CL == 2 && EQ == 16) return big_cluster_kernel<16, 2, 512>;
  if (CL == 2 && EQ == 32) return big_cluster_kernel<32, 2, 512>;
  if (CL == 4 && EQ == 32) return T <= 256 ? big_cluster_kernel<32, 4, 256> : big_cluster_kernel<32, 4, 512>;
  return nullptr;
}

int kern_slot(int EQ, int CL, int T) { return CL == 4 ? (T <= 256 ? 2 : 3) : (EQ == 32 ? 1 : 0); }

// Raise the kernel's dynamic shared-memory limit to at least `smem` (the limit only grows).
cudaError_t grant(const BigClusterCfg& c) {
  static std::mutex mu;
  static int granted[4][64] = {{0}};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  int& g = granted[kern_slot(c.EQ, c.CL, c.T)][dev < 64 ? dev : 0];
  if (dev < 64 && g >= (int)c.smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern_of(c.EQ, c.CL, c.T), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
  if (e == cudaSuccess && dev < 64) g = (int)c.smem;
  return e;
}

cudaLaunchConfig_t launch_cfg(const BigClusterCfg& c, int clusters, cudaStream_t stream, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * c.CL), 1, 1);
  cfg.blockDim = dim3((unsigned)c.T, 1, 1);
  cfg.dynamicSmemBytes = c.smem;
  cfg.stream = stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c.CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

}  // namespace

bool choose_big_cluster_cfg(int M, int N, int nrx, int ntx, int p_max, int CL, BigClusterCfg& cfg) {
  if (CL != 2 && CL != 4) return false;
  const int MN = M * N;
  for (int EQ : {16, 32}) {
    const int T = MN / EQ;
    if (T < 32 || T > 512 || (T % 32) != 0 || (T % M) != 0) continue;
    if ((EQ / CL) % kBigChunk != 0 || !kern_of(EQ, CL, T)) continue;
    if ((N % CL) != 0 || (T / M) * (EQ / CL) != N / CL) continue;
    const size_t smem = big_cluster_smem_bytes(nrx, ntx, p_max);
    if (smem > 227 * 1024) return false;
    cfg.CL = CL;
    cfg.T = T;
    cfg.EQ = EQ;
    cfg.smem = smem;
    cfg.slot_bytes = ((big_cluster_slot_elems(M, N, nrx, ntx, CL) * sizeof(float2)) + 255) & ~size_t(255);
    return true;
  }
  return false;
}

cudaError_t big_cluster_launch(const BigClusterCfg& c, const FrameArgs& A, int radix, int clusters, char* scratch,
                               cudaStream_t stream) {
  BigClusterKern k = kern_of(c.EQ, c.CL, c.T);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = grant(c);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = launch_cfg(c, clusters, stream, attr);
  return cudaLaunchKernelEx(&cfg, k, A, radix, scratch, c.slot_bytes);
}

cudaError_t big_cluster_max_active(const BigClusterCfg& c, int& clusters) {
  BigClusterKern k = kern_of(c.EQ, c.CL, c.T);
  if (!k) return cudaErrorInvalidValue;
  cudaError_t e = grant(c);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = launch_cfg(c, 1, nullptr, attr);
  return cudaOccupancyMaxActiveClusters(&clusters, k, &cfg);
}

int big_cluster_count(const BigClusterCfg& c, int max_active, int sm_count, int ctas_per_sm) {
  // Every resident cluster gets a slot: capping the live slots to what the L2 holds was
  // measured slower (4x4 128x64: 28.3 ms against 17.0 ms for 256 frames at CL = 2), the
  // gathers' L2 misses costing less than the idle SMs.
  int n = max_active;
  if (ctas_per_sm > 0) {
    const int want = sm_count * ctas_per_sm / c.CL;
    if (want < n) n = want;
  }
  return n < 1 ? 1 : n;
}

}  // namespace zotfs
