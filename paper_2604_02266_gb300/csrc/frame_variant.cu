// One instantiation of the frame kernel, selected by ZOTFS_VARIANT at compile time so the
// variants build in parallel.  The table in frame_table.cu lists them.
#include <mutex>

#include "frame_kernel.cuh"

#ifndef ZOTFS_VARIANT
#error "compile with -DZOTFS_VARIANT=<index>"
#endif

#if ZOTFS_VARIANT == 0
#define V_E 8
#define V_NB 1
#define V_TMAX 256
#define V_MINB 2
#elif ZOTFS_VARIANT == 1
#define V_E 8
#define V_NB 1
#define V_TMAX 512
#define V_MINB 1
#elif ZOTFS_VARIANT == 2
#define V_E 4
#define V_NB 1
#define V_TMAX 512
#define V_MINB 1
#elif ZOTFS_VARIANT == 3
#define V_E 16
#define V_NB 1
#define V_TMAX 256
#define V_MINB 1
#elif ZOTFS_VARIANT == 4
#define V_E 4
#define V_NB 2
#define V_TMAX 512
#define V_MINB 1
#elif ZOTFS_VARIANT == 5
#define V_E 2
#define V_NB 4
#define V_TMAX 512
#define V_MINB 1
#elif ZOTFS_VARIANT == 6
#define V_E 8
#define V_NB 1
#define V_TMAX 256
#define V_MINB 1
#define V_R double
#elif ZOTFS_VARIANT == 7
#define V_E 4
#define V_NB 2
#define V_TMAX 256
#define V_MINB 1
#define V_R double
#elif ZOTFS_VARIANT == 8
#define V_E 8
#define V_NB 1
#define V_TMAX 256
#define V_MINB 2
#define V_COEF 1
#elif ZOTFS_VARIANT == 9
#define V_E 8
#define V_NB 1
#define V_TMAX 512
#define V_MINB 1
#define V_COEF 1
#elif ZOTFS_VARIANT == 10
#define V_E 16
#define V_NB 1
#define V_TMAX 256
#define V_MINB 1
#define V_COEF 1
#else
#error "unknown ZOTFS_VARIANT"
#endif

#ifndef V_R
#define V_R float
#endif
// the variants small frames run on also get an instantiation that packs several frames per CTA
#if ZOTFS_VARIANT == 0 || ZOTFS_VARIANT == 2 || ZOTFS_VARIANT == 4 || ZOTFS_VARIANT == 5 || ZOTFS_VARIANT == 8
#define V_PACK 1
#else
#define V_PACK 0
#endif
#ifndef V_COEF
#define V_COEF 0
#endif

#define ZCAT2(a, b) a##b
#define ZCAT(a, b) ZCAT2(a, b)
#define VFUN(name) ZCAT(ZCAT(frame_v, ZOTFS_VARIANT), name)

namespace zotfs {

using KernT = void (*)(const FrameArgs, int);
static KernT kern(bool pack) {
#if V_PACK
  if (pack) return frame_kernel<V_R, V_E, V_NB, V_TMAX, V_MINB, (V_COEF != 0), true>;
#endif
  (void)pack;
  return frame_kernel<V_R, V_E, V_NB, V_TMAX, V_MINB, (V_COEF != 0), false>;
}

bool VFUN(_packs)() { return V_PACK != 0; }

void VFUN(_info)(int& E, int& NB, int& TMAX, int& real_bytes, int& minb, int& coef) {
  E = V_E;
  NB = V_NB;
  TMAX = V_TMAX;
  real_bytes = (int)sizeof(V_R);
  minb = V_MINB;
  coef = V_COEF;
}

// Raise the kernel's dynamic shared-memory limit to at least `smem` on the current device.
// The limit only ever grows (a lower value set later would break launches that rely on the
// higher one), and the server's scheduler thread launches concurrently with user threads.
static cudaError_t grant_smem(size_t smem, bool pack) {
  static std::mutex mu;
  static int granted[2][64] = {{0}};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 64 && granted[pack][dev] >= (int)smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern(pack), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev < 64) granted[pack][dev] = (int)smem;
  return e;
}

// fpc frames per CTA: a (T, fpc) block, fpc rows of `smem` bytes of shared memory each (rounded
// to 128 bytes, as the kernel places them).
static size_t cta_smem(size_t smem, int fpc) { return fpc <= 1 ? smem : ((smem + 127) & ~size_t(127)) * (size_t)fpc; }

cudaError_t VFUN(_launch)(const FrameArgs& A, int radix, int grid, int T, size_t smem, int fpc, cudaStream_t stream) {
  if (fpc < 1 || !V_PACK) fpc = 1;
  const bool pack = fpc > 1;
  cudaError_t e = grant_smem(cta_smem(smem, fpc), pack);
  if (e != cudaSuccess) return e;
  kern(pack)<<<grid, dim3((unsigned)T, (unsigned)fpc), cta_smem(smem, fpc), stream>>>(A, radix);
  return cudaGetLastError();
}

cudaError_t VFUN(_occupancy)(int T, size_t smem, int fpc, int& blocks) {
  if (fpc < 1 || !V_PACK) fpc = 1;
  const bool pack = fpc > 1;
  cudaError_t e = grant_smem(cta_smem(smem, fpc), pack);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern(pack), T * fpc, cta_smem(smem, fpc));
}

}  // namespace zotfs
