// kernels_vl.cu — instantiation of the two-cells-per-register score kernel (wavefront_vl.cuh):
// 8 rows x 2 x 8 columns per lane, i.e. column tasks of 32 x 128 cells.
#include "wavefront_vl.cuh"

namespace trioseq {

const void* wavefront_vl(int nj, int nk) {
  if (nj == 8 && nk == 16) return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8>);
  return nullptr;
}

size_t wavefront_vl_smem_bytes(int nj, int nk, int KP) {
  if (nj != 8 || nk != 16) return 0;
  using G = VlGeom<8, 8>;
  const size_t sigN = (size_t)((KP * KP + 3) & ~3);
  return (sigN + (size_t)kWarpsPerCta * (KP * (G::PJ + G::PK) + kRing * G::SLOT)) * sizeof(int);
}

}  // namespace trioseq
