// kernels_vl.cu — instantiations of the two-cells-per-register score kernel (wavefront_vl.cuh):
// 8 rows x 2 x 8 columns per lane (column tasks of 32 x 128 cells, 2 CTAs per SM), 8 rows x
// 2 x 4 columns per lane (tasks of 32 x 64 cells, 3 CTAs per SM), and the 32 x 128 tasks with
// the lane's sigma''(y,z) tile and 16-bit profiles in shared memory (2-warp CTAs, 5 per SM, or
// 1-warp CTAs, 9 per SM); the first two also for the semi-global and local types.
#include "wavefront_vl.cuh"

namespace trioseq {

// cs: sigma''(y,z) tile in shared memory, 2-warp CTAs (1, tile label "8x16s") or 1-warp CTAs
// (2, "8x16t"); 0: in registers
// at: kGlobal, or kSemiGlobal / kLocal (cs = 0 only)
const void* wavefront_vl(int nj, int nk, int cs, int at) {
  if (at == kSemiGlobal || at == kLocal) {
    if (cs != 0) return nullptr;
    if (nj == 8 && nk == 16)
      return at == kLocal ? reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8, 0, kLocal>)
                          : reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8, 0, kSemiGlobal>);
    if (nj == 8 && nk == 8)
      return at == kLocal ? reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 4, 0, kLocal>)
                          : reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 4, 0, kSemiGlobal>);
    return nullptr;
  }
  if (at != kGlobal) return nullptr;
  if (nj == 8 && nk == 16) {
    if (cs == 1) return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8, 1, kGlobal>);
    if (cs == 2) return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8, 2, kGlobal>);
    return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 8, 0, kGlobal>);
  }
  if (nj == 8 && nk == 8 && cs == 0)
    return reinterpret_cast<const void*>(&wavefront_vl_kernel<8, 4, 0, kGlobal>);
  return nullptr;
}

int wavefront_vl_warps(int cs) {
  return cs == 1 ? VlLaunch<8, 1>::warps : (cs == 2 ? VlLaunch<8, 2>::warps : kWarpsPerCta);
}

namespace {
template <int NJ, int NH, int CS>
size_t vl_smem(int KP) {
  using G = VlGeom<NJ, NH>;
  const size_t sigN = (size_t)((KP * KP + 3) & ~3);
  // Without CS: the bank-conflict-free 16-bit layout (the local 8x8v kernel's 32-bit row-major
  // profiles take less); with CS: 16-bit row-major profiles.
  const size_t prof = !CS ? (size_t)KP * (kPR * kPC * NJ / 2 + kPC * NH)
                          : (size_t)KP * (G::PJ16 + G::PK16) / 2;
  const size_t cv = CS ? (size_t)32 * 4 * G::CVG : 0;
  return (sigN + (size_t)VlLaunch<NH, CS>::warps * (prof + kRing * G::SLOT + cv)) * sizeof(int);
}
}  // namespace

size_t wavefront_vl_smem_bytes(int nj, int nk, int KP, int cs) {
  if (nj == 8 && nk == 16)
    return cs == 1 ? vl_smem<8, 8, 1>(KP) : (cs == 2 ? vl_smem<8, 8, 2>(KP) : vl_smem<8, 8, 0>(KP));
  if (nj == 8 && nk == 8 && cs == 0) return vl_smem<8, 4, 0>(KP);
  return 0;
}

}  // namespace trioseq
