// Kernel instantiations for 1-word slots (one translation unit per slot
// width so the builds run in parallel).
#include "gx_kernels.cuh"

namespace gx {

const KernelSet* kernels_w1(int b, int g) {
  GX_CASE(1, 4, 1)
  GX_CASE(1, 4, 2)
  GX_CASE(1, 4, 4)
  GX_CASE(1, 8, 1)
  GX_CASE(1, 8, 2)
  GX_CASE(1, 8, 4)
  GX_CASE(1, 8, 8)
  GX_CASE(1, 16, 1)
  GX_CASE(1, 16, 2)
  GX_CASE(1, 16, 4)
  GX_CASE(1, 16, 8)
  GX_CASE(1, 16, 16)
  GX_CASE(1, 32, 1)
  GX_CASE(1, 32, 2)
  GX_CASE(1, 32, 4)
  GX_CASE(1, 32, 8)
  GX_CASE(1, 32, 16)
  GX_CASE(1, 32, 32)
  return nullptr;
}

}  // namespace gx
