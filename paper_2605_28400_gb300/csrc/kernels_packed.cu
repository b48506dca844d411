// kernels_packed.cu — the packed int16x2 instantiations of the wavefront kernel (wavefront.cuh):
// two triplets per column task, one per 16-bit half, global alignment, score only. Compiled
// apart from the int32 instantiations.
#include "wavefront.cuh"

namespace trioseq {

namespace {

template <int NJ, int NK, int PK>
const void* pptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, false, kGlobal, PK, false>);
}

template <int PK>
const void* pick_tile(int nj, int nk) {
  if (nj == 8 && nk == 8) return pptr<8, 8, PK>();
  if (nj == 4 && nk == 8) return pptr<4, 8, PK>();
  if (nj == 4 && nk == 4) return pptr<4, 4, PK>();
  return nullptr;
}

}  // namespace

const void* wavefront_packed(int nj, int nk, int mode) {
  if (mode == 1) return pick_tile<1>(nj, nk);
  if (mode == 2) return pick_tile<2>(nj, nk);
  return nullptr;
}

}  // namespace trioseq
