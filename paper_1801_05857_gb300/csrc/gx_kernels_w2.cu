// Kernel instantiations for 2-word slots (one translation unit per slot
// width so the builds run in parallel).
#include "gx_kernels.cuh"

namespace gx {

const KernelSet* kernels_w2(int b, int g) {
  GX_CASE(2, 4, 1)
  GX_CASE(2, 4, 2)
  GX_CASE(2, 8, 1)
  GX_CASE(2, 8, 2)
  GX_CASE(2, 8, 4)
  GX_CASE(2, 16, 1)
  GX_CASE(2, 16, 2)
  GX_CASE(2, 16, 4)
  GX_CASE(2, 16, 8)
  GX_CASE(2, 32, 1)
  GX_CASE(2, 32, 2)
  GX_CASE(2, 32, 4)
  GX_CASE(2, 32, 8)
  GX_CASE(2, 32, 16)
  return nullptr;
}

}  // namespace gx
