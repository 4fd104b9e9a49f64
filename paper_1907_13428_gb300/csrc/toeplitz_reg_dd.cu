// Double-float register-resident Toeplitz passes on double vectors: the launchers,
// and the passes of L = 16 .. 128 (the longer lines compile in toeplitz_reg_dd_256.cu,
// toeplitz_reg_dd_1024.cu and toeplitz_reg_dd_4096.cu).
#include "toeplitz_reg.cuh"

namespace fde {

FDE_REG_INSTANTIATE(dd, double, 16)
FDE_REG_INSTANTIATE(dd, double, 32)
FDE_REG_INSTANTIATE(dd, double, 64)
FDE_REG_INSTANTIATE(dd, double, 128)
FDE_REG_EXTERN(dd, double, 256)
FDE_REG_EXTERN(dd, double, 512)
FDE_REG_EXTERN(dd, double, 1024)
FDE_REG_EXTERN(dd, double, 2048)
FDE_REG_EXTERN(dd, double, 4096)

template cudaError_t launch_rows_reg<dd, double>(fde_problem*, const double*, int, const dd2*, const AxisTables<dd>&,
                                                 const AxisEpi<double>&, cudaStream_t);
template cudaError_t launch_axis_reg<dd, double>(int, const double*, int, long long, long long, long long, long long,
                                                 const dd2*, const AxisTables<dd>&, int, const AxisEpi<double>&, int,
                                                 cudaStream_t);

cudaError_t toeplitz_reg_attrs_dd() { return reg_attrs_all<dd, double>(); }

}  // namespace fde
