// Double-float register-resident Toeplitz passes for L = 1024 and 2048.
#include "toeplitz_reg.cuh"

namespace fde {
FDE_REG_INSTANTIATE(dd, double, 1024)
FDE_REG_INSTANTIATE(dd, double, 2048)
}  // namespace fde
