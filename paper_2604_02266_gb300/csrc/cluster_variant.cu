// Instantiations and launch of the cluster receiver (frame_cluster.cuh): C = 2 with up to 512
// threads per CTA, C = 4 with up to 256.
#include <mutex>

#include "frame_cluster.cuh"
#include "internal.h"

namespace zotfs {

namespace {

template <int C, int TMAX>
cudaError_t launch_c(const FrameArgs& A, int radix, int clusters, int T, size_t smem, cudaStream_t stream) {
  static std::mutex mu;
  static int granted[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (dev >= 64 || granted[dev] < (int)smem) {
      e = cudaFuncSetAttribute(cluster_kernel<C, TMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev < 64) granted[dev] = (int)smem;
    }
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * C), 1, 1);
  cfg.blockDim = dim3((unsigned)T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cluster_kernel<C, TMAX>, A, radix);
}

template <int C, int TMAX>
cudaError_t max_clusters_c(int T, size_t smem, int& n) {
  cudaError_t e = cudaFuncSetAttribute(cluster_kernel<C, TMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3((unsigned)T, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(&n, cluster_kernel<C, TMAX>, &cfg);
}

}  // namespace

bool choose_cluster_cfg(int M, int N, int nrx, int ntx, int p_max, int C, ClusterCfg& cfg) {
  if (nrx != 1 || ntx != 1 || (C != 2 && C != 4)) return false;
  if (N % C != 0 || N / C < kClusterE) return false;
  const int T = M * (N / C) / kClusterE;
  if (T < 32 || (T % 32) != 0 || T > (C == 2 ? 512 : 256)) return false;
  const size_t smem = cluster_smem_bytes(M, N, p_max);
  if (smem > 227 * 1024) return false;
  cfg.C = C;
  cfg.T = T;
  cfg.smem = smem;
  return true;
}

cudaError_t cluster_launch(const ClusterCfg& cfg, const FrameArgs& A, int radix, int clusters, cudaStream_t stream) {
  return cfg.C == 2 ? launch_c<2, 512>(A, radix, clusters, cfg.T, cfg.smem, stream)
                    : launch_c<4, 256>(A, radix, clusters, cfg.T, cfg.smem, stream);
}

cudaError_t cluster_max_active(const ClusterCfg& cfg, int& clusters) {
  return cfg.C == 2 ? max_clusters_c<2, 512>(cfg.T, cfg.smem, clusters)
                    : max_clusters_c<4, 256>(cfg.T, cfg.smem, clusters);
}

}  // namespace zotfs
