// Double register-resident Toeplitz passes (256 threads per CTA).
#include "toeplitz_reg.cuh"

namespace fde {

#define FDE_INST(LL) FDE_REG_INSTANTIATE(double, double, LL)
FDE_FOR_EACH_L(FDE_INST)
#undef FDE_INST

template cudaError_t launch_rows_reg<double, double>(fde_problem*, const double*, int, const double2*,
                                                     const AxisTables<double>&, const AxisEpi<double>&, cudaStream_t);
template cudaError_t launch_axis_reg<double, double>(int, const double*, int, long long, long long, long long,
                                                     long long, const double2*, const AxisTables<double>&, int,
                                                     const AxisEpi<double>&, int, cudaStream_t);

cudaError_t toeplitz_reg_attrs_f64() { return reg_attrs_all<double, double>(); }

}  // namespace fde
