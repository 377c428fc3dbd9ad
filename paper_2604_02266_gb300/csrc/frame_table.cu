// Table of the frame-kernel instantiations built from frame_variant.cu.
#include "internal.h"

namespace zotfs {

#define DECL(i)                                                                                      \
  void frame_v##i##_info(int& E, int& NB, int& TMAX, int& real_bytes, int& minb, int& coef);                      \
  cudaError_t frame_v##i##_launch(const FrameArgs& A, int radix, int grid, int T, size_t smem, int fpc, \
                                  cudaStream_t stream);                                              \
  cudaError_t frame_v##i##_occupancy(int T, size_t smem, int fpc, int& blocks);                    \
  bool frame_v##i##_packs();
DECL(0)
DECL(1)
DECL(2)
DECL(3)
DECL(4)
DECL(5)
DECL(6)
DECL(7)
DECL(8)
DECL(9)
DECL(10)
#undef DECL

struct Entry {
  void (*info)(int&, int&, int&, int&, int&, int&);
  cudaError_t (*launch)(const FrameArgs&, int, int, int, size_t, int, cudaStream_t);
  cudaError_t (*occ)(int, size_t, int, int&);
  bool (*packs)();
};

static const Entry kTable[] = {
    {frame_v0_info, frame_v0_launch, frame_v0_occupancy, frame_v0_packs}, {frame_v1_info, frame_v1_launch, frame_v1_occupancy, frame_v1_packs},
    {frame_v2_info, frame_v2_launch, frame_v2_occupancy, frame_v2_packs}, {frame_v3_info, frame_v3_launch, frame_v3_occupancy, frame_v3_packs},
    {frame_v4_info, frame_v4_launch, frame_v4_occupancy, frame_v4_packs}, {frame_v5_info, frame_v5_launch, frame_v5_occupancy, frame_v5_packs},
    {frame_v6_info, frame_v6_launch, frame_v6_occupancy, frame_v6_packs}, {frame_v7_info, frame_v7_launch, frame_v7_occupancy, frame_v7_packs},
    {frame_v8_info, frame_v8_launch, frame_v8_occupancy, frame_v8_packs}, {frame_v9_info, frame_v9_launch, frame_v9_occupancy, frame_v9_packs},
    {frame_v10_info, frame_v10_launch, frame_v10_occupancy, frame_v10_packs},
};

int frame_variant_count() { return (int)(sizeof(kTable) / sizeof(kTable[0])); }

bool frame_variant_info(int v, int& E, int& NB, int& TMAX, int& real_bytes, int& minb, int& coef) {
  if (v < 0 || v >= frame_variant_count()) return false;
  kTable[v].info(E, NB, TMAX, real_bytes, minb, coef);
  return true;
}

cudaError_t frame_variant_launch(int v, const FrameArgs& A, int radix, int grid, int T, size_t smem,
                                 cudaStream_t stream, int fpc) {
  return kTable[v].launch(A, radix, grid, T, smem, fpc, stream);
}

cudaError_t frame_variant_occupancy(int v, int T, size_t smem, int& blocks, int fpc) {
  return kTable[v].occ(T, smem, fpc, blocks);
}

bool frame_variant_packs(int v) { return v >= 0 && v < frame_variant_count() && kTable[v].packs(); }

}  // namespace zotfs
