// Double-float register-resident Toeplitz passes for L = 256 and 512.
#include "toeplitz_reg.cuh"

namespace fde {
FDE_REG_INSTANTIATE(dd, double, 256)
FDE_REG_INSTANTIATE(dd, double, 512)
}  // namespace fde
