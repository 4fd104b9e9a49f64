// Float register-resident Toeplitz passes: the launchers and every tile the
// autotuner may pick (row passes of 256 or 128 threads, axis passes of 512 or 256).
#include "toeplitz_reg.cuh"

namespace fde {

#define FDE_INST(LL) FDE_REG_INSTANTIATE(float, float, LL)
FDE_FOR_EACH_L(FDE_INST)
#undef FDE_INST

template cudaError_t launch_rows_reg<float, float>(fde_problem*, const float*, int, const float2*,
                                                   const AxisTables<float>&, const AxisEpi<float>&, cudaStream_t);
template cudaError_t launch_axis_reg<float, float>(int, const float*, int, long long, long long, long long, long long,
                                                   const float2*, const AxisTables<float>&, int,
                                                   const AxisEpi<float>&, int, cudaStream_t);

cudaError_t toeplitz_reg_attrs_f32() { return reg_attrs_all<float, float>(); }

}  // namespace fde
