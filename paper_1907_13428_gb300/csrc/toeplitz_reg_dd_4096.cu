// Double-float register-resident Toeplitz passes for L = 4096.
#include "toeplitz_reg.cuh"

namespace fde {
FDE_REG_INSTANTIATE(dd, double, 4096)
}  // namespace fde
