// kernels_slab.cu — slab-launch instantiations of the wavefront kernel (wavefront.cuh): one
// triplet's cube cut into slabs of slices, each seeded from the plane the slab below left. They
// serve the linear-space traceback and score runs whose boundary records would not fit at once.
#include "wavefront.cuh"

namespace trioseq {

namespace {

template <int NJ, int NK, bool TB>
const void* sptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, TB, kGlobal, 0, true>);
}

}  // namespace

const void* wavefront_slab(int nj, int nk, bool tb) {
  if (nj == 8 && nk == 8) return tb ? sptr<8, 8, true>() : sptr<8, 8, false>();
  if (nj == 4 && nk == 8) return tb ? sptr<4, 8, true>() : sptr<4, 8, false>();
  if (nj == 4 && nk == 4) return tb ? sptr<4, 4, true>() : sptr<4, 4, false>();
  if (nj == 8 && nk == 4) return tb ? sptr<8, 4, true>() : nullptr;  // traceback only
  return nullptr;
}

}  // namespace trioseq
