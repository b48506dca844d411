// kernels_vl.cu — instantiations of the two-cells-per-register score kernel (wavefront_vl.cuh):
// 8 rows x 2 x 8 columns per lane (column tasks of 32 x 128 cells, 2 CTAs per SM) and 8 rows x
// 2 x 4 columns per lane (tasks of 32 x 64 cells, 3 CTAs per SM).
#include "wavefront_vl.cuh"

namespace trioseq {

const void* wavefront_vl(int nj, int nk) {
  if (nj == 8 && nk == 16) return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8>);
  if (nj == 8 && nk == 8) return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 4>);
  return nullptr;
}

namespace {
template <int NJ, int NH>
size_t vl_smem(int KP) {
  using G = VlGeom<NJ, NH>;
  const size_t sigN = (size_t)((KP * KP + 3) & ~3);
  return (sigN + (size_t)kWarpsPerCta * (KP * (G::PJ + G::PK) + kRing * G::SLOT)) * sizeof(int);
}
}  // namespace

size_t wavefront_vl_smem_bytes(int nj, int nk, int KP) {
  if (nj == 8 && nk == 16) return vl_smem<8, 8>(KP);
  if (nj == 8 && nk == 8) return vl_smem<8, 4>(KP);
  return 0;
}

}  // namespace trioseq
