// Kernel instantiations for 4-word slots (one translation unit per slot
// width so the builds run in parallel).
#include "gx_kernels.cuh"

namespace gx {

const KernelSet* kernels_w4(int b, int g) {
  GX_CASE(4, 4, 1)
  GX_CASE(4, 8, 1)
  GX_CASE(4, 8, 2)
  GX_CASE(4, 16, 1)
  GX_CASE(4, 16, 2)
  GX_CASE(4, 16, 4)
  GX_CASE(4, 32, 1)
  GX_CASE(4, 32, 2)
  GX_CASE(4, 32, 4)
  GX_CASE(4, 32, 8)
  return nullptr;
}

}  // namespace gx
