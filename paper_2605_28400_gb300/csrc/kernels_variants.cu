// kernels_variants.cu — the semi-global and local alignment types of Sec. II (score and
// traceback modes) of the wavefront kernel (wavefront.cuh), compiled apart from the global
// instantiations.
#include "wavefront.cuh"

namespace trioseq {

namespace {

template <int NJ, int NK, bool TB, int AT>
const void* vptr() {
  return reinterpret_cast<const void*>(&wavefront_kernel<NJ, NK, TB, AT, 0, false>);
}

template <int AT>
const void* pick_type(int nj, int nk, bool tb) {
  if (nj == 8 && nk == 8) return tb ? vptr<8, 8, true, AT>() : vptr<8, 8, false, AT>();
  if (nj == 4 && nk == 8) return tb ? vptr<4, 8, true, AT>() : vptr<4, 8, false, AT>();
  if (nj == 4 && nk == 4) return tb ? vptr<4, 4, true, AT>() : vptr<4, 4, false, AT>();
  if (nj == 8 && nk == 4) return tb ? vptr<8, 4, true, AT>() : nullptr;  // traceback only
  return nullptr;
}

}  // namespace

const void* wavefront_variant(int nj, int nk, int at, bool tb) {
  if (at == kSemiGlobal) return pick_type<kSemiGlobal>(nj, nk, tb);
  if (at == kLocal) return pick_type<kLocal>(nj, nk, tb);
  return nullptr;
}

}  // namespace trioseq
