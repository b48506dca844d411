// kernels_variants.cu — the semi-global and local alignment types of Sec. II (score mode) of
// the wavefront kernel (wavefront.cuh), compiled apart from the global instantiations.
#include "wavefront.cuh"

namespace trioseq {

namespace {

template <int NJ, int NK, int AT>
const void* vptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, false, AT, false, false>);
}

}  // namespace

const void* wavefront_variant(int nj, int nk, int at) {
  if (at == kSemiGlobal) {
    if (nj == 8 && nk == 8) return vptr<8, 8, kSemiGlobal>();
    if (nj == 4 && nk == 8) return vptr<4, 8, kSemiGlobal>();
    if (nj == 4 && nk == 4) return vptr<4, 4, kSemiGlobal>();
  } else if (at == kLocal) {
    if (nj == 8 && nk == 8) return vptr<8, 8, kLocal>();
    if (nj == 4 && nk == 8) return vptr<4, 8, kLocal>();
    if (nj == 4 && nk == 4) return vptr<4, 4, kLocal>();
  }
  return nullptr;
}

}  // namespace trioseq
