// Streaming vector kernels and their launchers. The bodies of the kernels that
// the persistent executor can replay are operations in ops_vec.cuh; the
// kernels here run them once per hardware block.
#include <cmath>

#include "ops_vec.cuh"

namespace fde {

int red_grid(long long n) {
  long long g = (n + 4LL * kRedThreads - 1) / (4LL * kRedThreads);
  if (g < 1) g = 1;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)g;
}

// The reduction kernels run with kRedThreads threads; their bounds admit the
// executor's block size, with which recorded launches are replayed one by one.
template <typename RA, typename RB>
__global__ void __launch_bounds__(kPersistThreads) k_dot(DotArgs<RA, RB> a) {
  DotOp<RA, RB>::template run<false>(hw_ctx(), a);
}
__global__ void __launch_bounds__(1024) k_finish(FinishArgs a) { FinishSumOp::run<false>(hw_ctx(), a); }
template <typename RV>
__global__ void __launch_bounds__(kPersistThreads) k_pcg_xr(PcgXrArgs<RV> a) {
  PcgXrOp<RV>::template run<false>(hw_ctx(), a);
}
template <typename RV> __global__ void k_pcg_p(PcgPArgs<RV> a) { PcgPOp<RV>::template run<false>(hw_ctx(), a); }
__global__ void k_to_f32(ToF32Args a) { ToF32Op::run<false>(hw_ctx(), a); }
__global__ void k_to_f32_unless(ToF32UnlessArgs a) { ToF32UnlessOp::run<false>(hw_ctx(), a); }
__global__ void k_add_f32_unless(AddF32UnlessArgs a) { AddF32UnlessOp::run<false>(hw_ctx(), a); }
__global__ void k_scalar_step(ScalarStepArgs a) { ScalarStepOp::run<false>(hw_ctx(), a); }
template <typename R> __global__ void k_fill(FillArgs<R> a) { FillOp<R>::template run<false>(hw_ctx(), a); }
template <typename R> __global__ void k_copy(CopyArgs<R> a) { CopyOp<R>::template run<false>(hw_ctx(), a); }
__global__ void k_admm_pre(AdmmPreArgs a) { AdmmPreOp::run<false>(hw_ctx(), a); }
__global__ void __launch_bounds__(kPersistThreads) k_admm_post(AdmmPostArgs a) {
  AdmmPostOp::run<false>(hw_ctx(), a);
}
__global__ void __launch_bounds__(1024) k_admm_finish(AdmmFinishArgs a) { AdmmFinishOp::run<false>(hw_ctx(), a); }
__global__ void k_fold(FoldArgs a) { FoldOp::run<false>(hw_ctx(), a); }

// r = b - s (double); partials of r.r
__global__ void __launch_bounds__(kRedThreads) k_residual(const double* __restrict__ b, const double* __restrict__ s,
                                                           double* __restrict__ r, long long n,
                                                           double* __restrict__ partials) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = b[i] - s[i];
    r[i] = v;
    acc += v * v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// y64 += (double) d32
__global__ void k_add_f32(double* __restrict__ y, const float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += (double)d[i];
}

// dJ/dybar = -w (y - ybar); rhs of the adjoint: f = -w (y - ybar) - w_y
__global__ void k_grad_ybar(const double* __restrict__ y, const double* __restrict__ ybar, const double* __restrict__ wy,
                            double w0, double w1, long long last_start, long long n, double* __restrict__ dJ,
                            double* __restrict__ f) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = i >= last_start ? w1 : w0;
    const double v = -w * (y[i] - ybar[i]);
    if (dJ) dJ[i] = v;
    f[i] = v - (wy ? wy[i] : 0.0);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static unsigned sgrid(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Block size of a launch: while launches are recorded, the executor's (every
// body here takes any block size; the grids stay those of the plain launches).
static int vthreads(int t) { return recording() ? kPersistThreads : t; }
// one-block finishing kernels run with 1024 threads
static int fin_threads() { return vthreads(1024); }

template <typename RA, typename RB>
cudaError_t dot(fde_problem* P, const RA* a, const RB* b, long long n, int slot, int op, cudaStream_t st,
                double aux) {
  const int g = red_grid(n);
  cudaError_t e = launch_op<DotOp<RA, RB>>(k_dot<RA, RB>, g, vthreads(kRedThreads), 0, st, {a, b, n, P->partials});
  if (e != cudaSuccess) return e;
  return launch_op<FinishSumOp>(k_finish, 1, fin_threads(), 0, st, {P->partials, g, P->dscal, slot, op, aux});
}
template cudaError_t dot<double, double>(fde_problem*, const double*, const double*, long long, int, int, cudaStream_t,
                                         double);
template cudaError_t dot<float, float>(fde_problem*, const float*, const float*, long long, int, int, cudaStream_t,
                                       double);

template <typename RV>
cudaError_t pcg_xr(fde_problem* P, RV* x, RV* r, const RV* d, const RV* q, long long n, cudaStream_t st) {
  const int g = red_grid(n);
  cudaError_t e = launch_op<PcgXrOp<RV>>(k_pcg_xr<RV>, g, vthreads(kRedThreads), 0, st, {x, r, d, q, P->dscal, n, P->partials});
  if (e != cudaSuccess) return e;
  return launch_op<FinishSumOp>(k_finish, 1, fin_threads(), 0, st, {P->partials, g, P->dscal, S_RR, FIN_STORE, 0.0});
}
template cudaError_t pcg_xr<double>(fde_problem*, double*, double*, const double*, const double*, long long,
                                    cudaStream_t);
template cudaError_t pcg_xr<float>(fde_problem*, float*, float*, const float*, const float*, long long, cudaStream_t);

template <typename RV>
cudaError_t pcg_p(fde_problem* P, RV* d, const RV* z, long long n, cudaStream_t st) {
  return launch_op<PcgPOp<RV>>(k_pcg_p<RV>, sgrid(n), vthreads(256), 0, st, {d, z, P->dscal, n});
}
template cudaError_t pcg_p<double>(fde_problem*, double*, const double*, long long, cudaStream_t);
template cudaError_t pcg_p<float>(fde_problem*, float*, const float*, long long, cudaStream_t);

cudaError_t residual(fde_problem* P, const double* b, const double* s, double* r, long long n, int slot,
                     cudaStream_t st) {
  const int g = red_grid(n);
  k_residual<<<g, kRedThreads, 0, st>>>(b, s, r, n, P->partials);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_op<FinishSumOp>(k_finish, 1, fin_threads(), 0, st, {P->partials, g, P->dscal, slot, FIN_STORE, 0.0});
}

cudaError_t to_f32(const double* in, float* out, long long n, cudaStream_t st) {
  return launch_op<ToF32Op>(k_to_f32, sgrid(n), vthreads(256), 0, st, {in, out, n});
}
cudaError_t to_f32_unless_conv(fde_problem* P, const double* in, float* out, long long n, cudaStream_t st) {
  return launch_op<ToF32UnlessOp>(k_to_f32_unless, sgrid(n), vthreads(256), 0, st, {in, out, n, P->dscal});
}
cudaError_t add_f32_unless_conv(fde_problem* P, double* y, const float* d, long long n, cudaStream_t st) {
  cudaError_t e = launch_op<ScalarStepOp>(k_scalar_step, 1, vthreads(1), 0, st,
                                          {P->dscal, 0, 0, 1});
  if (e != cudaSuccess) return e;
  return launch_op<AddF32UnlessOp>(k_add_f32_unless, sgrid(n), vthreads(256), 0, st, {y, d, n, P->dscal});
}
cudaError_t scalar_max(fde_problem* P, int dst, int src, cudaStream_t st) {
  return launch_op<ScalarStepOp>(k_scalar_step, 1, vthreads(1), 0, st, {P->dscal, dst, src, 0});
}
cudaError_t add_f32(double* y, const float* d, long long n, cudaStream_t st) {
  k_add_f32<<<sgrid(n), 256, 0, st>>>(y, d, n);
  note_launches(1);
  return cudaGetLastError();
}
template <typename R>
cudaError_t fill(R* x, R v, long long n, cudaStream_t st) {
  return launch_op<FillOp<R>>(k_fill<R>, sgrid(n), vthreads(256), 0, st, {x, v, n});
}
template cudaError_t fill<double>(double*, double, long long, cudaStream_t);
template cudaError_t fill<float>(float*, float, long long, cudaStream_t);
template <typename R>
cudaError_t copy(R* dst, const R* src, long long n, cudaStream_t st) {
  return launch_op<CopyOp<R>>(k_copy<R>, sgrid(n), vthreads(256), 0, st, {dst, src, n});
}
template cudaError_t copy<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t copy<float>(float*, const float*, long long, cudaStream_t);

cudaError_t admm_pre(const AdmmArgs& A, double* c, double* bu, double* r0, double* q, cudaStream_t st) {
  return launch_op<AdmmPreOp>(k_admm_pre, sgrid(A.n), vthreads(256), 0, st, {A, c, bu, r0, q});
}

cudaError_t admm_post(fde_problem* P, const AdmmArgs& A, const double* y, const double* By, const double* bu,
                      const double* r0, double* u, cudaStream_t st) {
  int g = red_grid(A.n);
  if (g > kMaxPartials / 5) g = kMaxPartials / 5;
  cudaError_t e = launch_op<AdmmPostOp>(k_admm_post, g, vthreads(kRedThreads), 0, st, {A, y, By, bu, r0, u, P->partials, g});
  if (e != cudaSuccess) return e;
  return launch_op<AdmmFinishOp>(k_admm_finish, 1, fin_threads(), 0, st, {P->partials, g, P->dscal});
}

cudaError_t fold(const double* t, const double* q, const double* c, const double* y, const double m2inv[2],
                 const double m1[2], long long last_start, long long n, double* v, double* w, cudaStream_t st) {
  return launch_op<FoldOp>(k_fold, sgrid(n), vthreads(256), 0, st,
                           {t, q, c, y, m2inv[0], m2inv[1], m1[0], m1[1], last_start, n, v, w});
}

cudaError_t grad_ybar(const double* y, const double* ybar, const double* wy, double w0, double w1, long long last_start,
                      long long n, double* dJ, double* f, cudaStream_t st) {
  k_grad_ybar<<<sgrid(n), 256, 0, st>>>(y, ybar, wy, w0, w1, last_start, n, dJ, f);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fde
