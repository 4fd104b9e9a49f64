// The operations the persistent executor can replay (persist.cu), and the launch
// helper every launcher of those operations goes through.
#pragma once
#include "op.cuh"

namespace fde {

template <typename RA, typename RB> struct DotOp;
struct FinishSumOp;
template <typename RV> struct PcgXrOp;
template <typename RV> struct PcgPOp;
struct ToF32Op;
struct ToF32UnlessOp;
struct AddF32UnlessOp;
struct ScalarStepOp;
template <typename R> struct FillOp;
template <typename R> struct CopyOp;
struct AdmmPreOp;
struct AdmmPostOp;
struct AdmmFinishOp;
struct FoldOp;
template <typename R> struct RowsOp;
template <typename R> struct AxisOp;
template <typename R> struct PrecRowsFwdOp;
template <typename R> struct PrecRowsInvOp;
template <typename R> struct PrecAxisOp;
template <typename R, int L, int NT, typename S, bool FULL> struct RowsRegOp;
template <typename R, int L, int NT, typename S, bool FULL> struct AxisRegOp;
template <typename R, int L, int NT, typename S, bool FULL> struct RowsSplitOp;
template <typename R, int L, int NT, typename S, bool FULL> struct AxisSplitOp;
template <typename R, int L, int NT, int MODE> struct PrecAxisRegOp;
template <typename R, int L, int NT> struct PrecRowsFwdRegOp;
template <typename R, int L, int NT> struct PrecRowsInvRegOp;

// register-resident float transforms of one power-of-two length (lines filling
// the transform, 256 threads): Toeplitz passes and preconditioner transforms
#define FDE_PERSIST_REG_OPS(LL)                                                                             \
  RowsRegOp<float, LL, 256, float, true>, AxisRegOp<float, LL, 256, float, true>,                          \
      PrecAxisRegOp<float, LL, 256, 0>, PrecAxisRegOp<float, LL, 256, 1>, PrecAxisRegOp<float, LL, 256, 2>, \
      PrecRowsFwdRegOp<float, LL, 256>, PrecRowsInvRegOp<float, LL, 256>

using PersistOps =
    OpList<DotOp<float, float>, DotOp<double, double>, FinishSumOp, PcgXrOp<float>, PcgXrOp<double>, PcgPOp<float>,
           PcgPOp<double>, ToF32Op, ToF32UnlessOp, AddF32UnlessOp, ScalarStepOp, FillOp<float>, FillOp<double>,
           CopyOp<float>, CopyOp<double>, AdmmPreOp, AdmmPostOp, AdmmFinishOp, FoldOp, RowsOp<float>, RowsOp<double>,
           AxisOp<float>, AxisOp<double>, PrecRowsFwdOp<float>, PrecRowsFwdOp<double>, PrecRowsInvOp<float>,
           PrecRowsInvOp<double>, PrecAxisOp<float>, PrecAxisOp<double>, FDE_PERSIST_REG_OPS(16),
           FDE_PERSIST_REG_OPS(32), FDE_PERSIST_REG_OPS(64), FDE_PERSIST_REG_OPS(128), FDE_PERSIST_REG_OPS(256),
           FDE_PERSIST_REG_OPS(512), FDE_PERSIST_REG_OPS(1024), FDE_PERSIST_REG_OPS(2048)>;

template <class Op>
cudaError_t launch_op(void (*kern)(typename Op::Args), unsigned grid, int threads, size_t smem, cudaStream_t st,
                      const typename Op::Args& a) {
  return launch_or_record<Op, PersistOps>(kern, grid, threads, smem, st, a);
}

}  // namespace fde
