// kernels_packed.cu — the packed int16x2 instantiations of the wavefront kernel (wavefront.cuh):
// two triplets per column task, one per 16-bit half, global alignment, score only. Compiled
// apart from the int32 instantiations.
#include "wavefront.cuh"

namespace trioseq {

namespace {

template <int NJ, int NK>
const void* pptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, false, kGlobal, true, false>);
}

}  // namespace

const void* wavefront_packed(int nj, int nk) {
  if (nj == 8 && nk == 8) return pptr<8, 8>();
  if (nj == 4 && nk == 8) return pptr<4, 8>();
  if (nj == 4 && nk == 4) return pptr<4, 4>();
  return nullptr;
}

}  // namespace trioseq
