// Multilevel circulant preconditioner (Section 5, Eq. multilevel circulant
// preconditioner, and Eq. first schur complement preconditioner with J ~ I):
//   z = F^-1 diag(1/sigma) F r,  sigma[k,i,j] = m1 + |Lambda[k,i,j]|^2 / m2,
//   Lambda = psi (lambda_t[k] - lambda_x[i] - lambda_y[j]),
// where lambda_* are the DFTs of the T. Chan circulants of C_t, X and Y and F
// is the three-level DFT (transform order is irrelevant: the levels commute).
// Mode 1 replaces sigma by |Lambda|^2, which is (C_3 C_3^T)^-1 for the adjoint
// solve of the gradient.
//
// Data path (r real, N = nt*nx*ny):
//   1. x2 rows: two real rows form one complex line; after the order-ny DFT the
//      half spectra of both rows (ny/2+1 bins) are separated and stored in
//      spec[t][x1][Hp] (Hp = padded row stride);
//   2. x1 columns of spec: forward DFT;
//   3. t columns of spec: forward DFT, divide by N*sigma, inverse DFT;
//   4. x1 columns: inverse DFT;
//   5. x2 rows: the two Hermitian half spectra are recombined into one complex
//      line, inverse DFT, real and imaginary parts are the two output rows.
#include "ops_prec_reg.cuh"

namespace fde {

template <typename R> static const AxisTables<R>& ptables(const Axis& A);
template <> const AxisTables<double>& ptables<double>(const Axis& A) { return A.d; }
template <> const AxisTables<float>& ptables<float>(const Axis& A) { return A.f; }

// Generic kernels (bodies in ops_prec.cuh): lengths with factors 3, 5, 7 or
// below 16, and every transform of a recorded (persistent) solve.
template <typename R> __global__ void __launch_bounds__(512) k_prec_rows_fwd(PrecRowsArgs<R> a) {
  PrecRowsFwdOp<R>::template run<false>(hw_ctx(), a);
}
template <typename R> __global__ void __launch_bounds__(512) k_prec_rows_inv(PrecRowsArgs<R> a) {
  PrecRowsInvOp<R>::template run<false>(hw_ctx(), a);
}
template <typename R> __global__ void __launch_bounds__(1024) k_prec_axis(PrecAxisArgs<R> a) {
  PrecAxisOp<R>::template run<false>(hw_ctx(), a);
}

template <typename R>
cudaError_t launch_prec_axis_reg(int L, cplx<R>* spec, long long axis_stride, long long n_inner,
                                 long long outer_stride, long long n_outer, const cplx<R>* twn, int mode,
                                 const DivArgs& dv, const cplx<R>* lt, const cplx<R>* lx, const cplx<R>* ly,
                                 cudaStream_t st);
cudaError_t precond_reg_set_smem_attrs();
template <typename R>
cudaError_t launch_prec_rows_reg(int L, int inverse, const R* r, R* z, cplx<R>* spec, long long nrows, int H, int Hp,
                                 const cplx<R>* twn, cudaStream_t st, Gate gate);
cudaError_t precond_rows_reg_set_smem_attrs();

template <typename R>
cudaError_t apply_precond(fde_problem* P, double m1, double m2, int mode, const R* r, R* z, cplx<R>* spec,
                          cudaStream_t st, Gate gate, double cre) {
  using C = cplx<R>;
  const Axis& At = P->ax[0];
  const Axis& Ax = P->ax[1];
  const Axis& Ay = P->ax[2];
  const long long nrows = (long long)P->nt * P->nx;
  const int ny = P->ny, H = P->H, Hp = P->Hp;
  cudaError_t err;
  // a recorded solve: float transforms register-resident (256 threads), double ones generic
  const bool gen = recording() && sizeof(R) != 4;
  const bool rec = recording();
  const bool rows_pow2 = ny >= 16 && (ny & (ny - 1)) == 0 && !gen;
  // 1. rows forward
  if (rows_pow2) {
    if ((err = launch_prec_rows_reg<R>(ny, 0, r, nullptr, spec, nrows, H, Hp, ptables<R>(Ay).twn, st, gate)) !=
        cudaSuccess)
      return err;
  } else {
    const int threads = rec ? kPersistThreads : (ny > kPEPT * 256) ? 512 : 256;
    int pairs = (kPEPT * threads) / ny;
    if (pairs < 1) pairs = 1;
    const long long np = (nrows + 1) / 2;
    if (pairs > np) pairs = (int)np;
    const long long grid = (np + pairs - 1) / pairs;
    err = launch_op<PrecRowsFwdOp<R>>(k_prec_rows_fwd<R>, (unsigned)grid, threads, (size_t)pairs * ny * sizeof(C), st,
                                      {r, nullptr, spec, nrows, ny, H, Hp, ptables<R>(Ay).twn, Ay.plann, pairs, gate});
    if (err != cudaSuccess) return err;
  }
  const int threads = rec ? kPersistThreads : (sizeof(R) == 4 ? 1024 : 512);
  const int cap = kPEPT * threads;
  DivArgs none{};
  none.gate = gate;
  // 2. x1 forward; 3. t forward/divide/inverse; 4. x1 inverse
  for (int step = 0; step < 3; ++step) {
    const bool tpass = (step == 1);
    const Axis& A = tpass ? At : Ax;
    const int n = A.n;
    long long axis_stride, n_inner, outer_stride, n_outer;
    if (!tpass) {
      axis_stride = Hp;
      n_inner = H;
      outer_stride = (long long)P->nx * Hp;
      n_outer = P->nt;
    } else {
      axis_stride = (long long)P->nx * Hp;
      n_inner = axis_stride;
      outer_stride = 0;
      n_outer = 1;
    }
    int lines = cap / n;
    if (lines < 1) lines = 1;
    const long long total = n_outer * n_inner;
    if (lines > total) lines = (int)total;
    const long long grid = (total + lines - 1) / lines;
    DivArgs dv = none;
    if (tpass) {
      dv.divide = 1;
      dv.adjoint = mode;
      dv.m1 = m1;
      dv.inv_m2 = 1.0 / m2;
      dv.cre = cre;
      dv.psi = P->psi;
      dv.inv_N = 1.0 / (double)P->N;
      dv.Hp = Hp;
      dv.H = H;
    }
    const bool pow2 = n >= 16 && (n & (n - 1)) == 0 && !gen;
    if (pow2) {
      err = launch_prec_axis_reg<R>(n, spec, axis_stride, n_inner, outer_stride, n_outer, ptables<R>(A).twn,
                                    tpass ? 2 : (step == 2 ? 1 : 0), dv, ptables<R>(At).lam, ptables<R>(Ax).lam,
                                    ptables<R>(Ay).lam, st);
      if (err != cudaSuccess) return err;
      continue;
    }
    err = launch_op<PrecAxisOp<R>>(k_prec_axis<R>, (unsigned)grid, threads, (size_t)lines * n * sizeof(C), st,
                                   {spec, n, axis_stride, n_inner, outer_stride, n_outer, ptables<R>(A).twn, A.plann,
                                    step == 2 ? 1 : 0, lines, dv, ptables<R>(At).lam, ptables<R>(Ax).lam,
                                    ptables<R>(Ay).lam});
    if (err != cudaSuccess) return err;
  }
  // 5. rows inverse
  if (rows_pow2) {
    if ((err = launch_prec_rows_reg<R>(ny, 1, nullptr, z, spec, nrows, H, Hp, ptables<R>(Ay).twn, st, gate)) !=
        cudaSuccess)
      return err;
  } else {
    const int threads2 = rec ? kPersistThreads : (ny > kPEPT * 256) ? 512 : 256;
    int pairs = (kPEPT * threads2) / ny;
    if (pairs < 1) pairs = 1;
    const long long np = (nrows + 1) / 2;
    if (pairs > np) pairs = (int)np;
    const long long grid = (np + pairs - 1) / pairs;
    err = launch_op<PrecRowsInvOp<R>>(k_prec_rows_inv<R>, (unsigned)grid, threads2, (size_t)pairs * ny * sizeof(C),
                                      st, {nullptr, z, spec, nrows, ny, H, Hp, ptables<R>(Ay).twn, Ay.plann, pairs,
                                           gate});
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template cudaError_t apply_precond<double>(fde_problem*, double, double, int, const double*, double*, double2*,
                                           cudaStream_t, Gate, double);
template cudaError_t apply_precond<float>(fde_problem*, double, double, int, const float*, float*, float2*,
                                          cudaStream_t, Gate, double);

// Dynamic shared memory above 48 KB must be opted into per kernel.
cudaError_t precond_set_smem_attrs() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_prec_rows_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  e = cudaFuncSetAttribute(k_prec_rows_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  e = cudaFuncSetAttribute(k_prec_rows_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  e = cudaFuncSetAttribute(k_prec_rows_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  e = cudaFuncSetAttribute(k_prec_axis<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  e = cudaFuncSetAttribute(k_prec_axis<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e) return e;
  if ((e = precond_reg_set_smem_attrs())) return e;
  return precond_rows_reg_set_smem_attrs();
}

}  // namespace fde

// ===========================================================================
// Register-resident column transforms and x2-row transforms for power-of-two
// lengths >= 16 (bodies in ops_prec_reg.cuh).
// ===========================================================================
namespace fde {

// Plain transforms (modes 0, 1) are compiled for two resident CTAs (at most 64
// registers a thread with 512 threads): they move the whole spectrum through HBM
// and need the warps to hide its latency; the divide pass keeps one CTA.
template <int MODE> constexpr int prec_min_blocks() { return MODE == 2 ? 1 : 2; }

template <typename R, int L, int NT, int MODE>
__global__ void __launch_bounds__(NT, prec_min_blocks<MODE>()) k_prec_axis_reg(PrecAxisRegArgs<R> a) {
  PrecAxisRegOp<R, L, NT, MODE>::template run<false>(hw_ctx(), a);
}
template <typename R, int L, int NT> __global__ void __launch_bounds__(NT) k_prec_rows_fwd_reg(PrecRowsRegArgs<R> a) {
  PrecRowsFwdRegOp<R, L, NT>::template run<false>(hw_ctx(), a);
}
template <typename R, int L, int NT> __global__ void __launch_bounds__(NT) k_prec_rows_inv_reg(PrecRowsRegArgs<R> a) {
  PrecRowsInvRegOp<R, L, NT>::template run<false>(hw_ctx(), a);
}

template <typename R> constexpr int prec_nt() { return sizeof(R) == 4 ? 512 : 256; }

template <typename R, int L, int NT>
static cudaError_t launch_prec_axis_reg_LN(cplx<R>* spec, long long axis_stride, long long n_inner,
                                           long long outer_stride, long long n_outer, const cplx<R>* twn, int mode,
                                           const DivArgs& dv, const cplx<R>* lt, const cplx<R>* lx,
                                           const cplx<R>* ly, cudaStream_t st) {
  constexpr int CP = NT / (L / 16);
  const long long total = n_outer * n_inner;
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * CP * sizeof(cplx<R>);
  const PrecAxisRegArgs<R> a{spec, axis_stride, n_inner, outer_stride, n_outer, twn, dv, lt, lx, ly};
  if (mode == 0)
    return launch_op<PrecAxisRegOp<R, L, NT, 0>>(k_prec_axis_reg<R, L, NT, 0>, (unsigned)grid, NT, smem, st, a);
  if (mode == 1)
    return launch_op<PrecAxisRegOp<R, L, NT, 1>>(k_prec_axis_reg<R, L, NT, 1>, (unsigned)grid, NT, smem, st, a);
  return launch_op<PrecAxisRegOp<R, L, NT, 2>>(k_prec_axis_reg<R, L, NT, 2>, (unsigned)grid, NT, smem, st, a);
}

template <typename R, int L>
static cudaError_t launch_prec_axis_reg_L(cplx<R>* spec, long long axis_stride, long long n_inner,
                                          long long outer_stride, long long n_outer, const cplx<R>* twn, int mode,
                                          const DivArgs& dv, const cplx<R>* lt, const cplx<R>* lx, const cplx<R>* ly,
                                          cudaStream_t st) {
  // a recorded (float) solve runs every launch with the executor's block size
  if constexpr (prec_nt<R>() != kPersistThreads) {
    if (recording())
      return launch_prec_axis_reg_LN<R, L, kPersistThreads>(spec, axis_stride, n_inner, outer_stride, n_outer, twn,
                                                            mode, dv, lt, lx, ly, st);
  }
  return launch_prec_axis_reg_LN<R, L, prec_nt<R>()>(spec, axis_stride, n_inner, outer_stride, n_outer, twn, mode, dv,
                                                     lt, lx, ly, st);
}

#define FDE_FOR_EACH_PL(M) M(16) M(32) M(64) M(128) M(256) M(512) M(1024) M(2048) M(4096)

template <typename R>
cudaError_t launch_prec_axis_reg(int L, cplx<R>* spec, long long axis_stride, long long n_inner,
                                 long long outer_stride, long long n_outer, const cplx<R>* twn, int mode,
                                 const DivArgs& dv, const cplx<R>* lt, const cplx<R>* lx, const cplx<R>* ly,
                                 cudaStream_t st) {
  switch (L) {
#define FDE_CASE(LL)                                                                                            \
  case LL:                                                                                                      \
    return launch_prec_axis_reg_L<R, LL>(spec, axis_stride, n_inner, outer_stride, n_outer, twn, mode, dv, lt, lx, \
                                         ly, st);
    FDE_FOR_EACH_PL(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_prec_axis_reg<float>(int, float2*, long long, long long, long long, long long,
                                                 const float2*, int, const DivArgs&, const float2*, const float2*,
                                                 const float2*, cudaStream_t);
template cudaError_t launch_prec_axis_reg<double>(int, double2*, long long, long long, long long, long long,
                                                  const double2*, int, const DivArgs&, const double2*,
                                                  const double2*, const double2*, cudaStream_t);

cudaError_t precond_reg_set_smem_attrs() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define FDE_ATTR1(LL, M)                                                                          \
  if (e == cudaSuccess)                                                                           \
    e = cudaFuncSetAttribute(k_prec_axis_reg<float, LL, prec_nt<float>(), M>,                     \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);                   \
  if (e == cudaSuccess)                                                                           \
    e = cudaFuncSetAttribute(k_prec_axis_reg<double, LL, prec_nt<double>(), M>,                   \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
#define FDE_ATTR(LL) FDE_ATTR1(LL, 0) FDE_ATTR1(LL, 1) FDE_ATTR1(LL, 2)
  FDE_FOR_EACH_PL(FDE_ATTR)
#undef FDE_ATTR
#undef FDE_ATTR1
  return e;
}

}  // namespace fde

// ===========================================================================
// Register-resident x2-row transforms of the preconditioner (power-of-two
// ny >= 16). Two real rows a, b form the complex line a + i b; the half
// spectra are A_k = (Z_k + conj Z_{n-k})/2 and B_k = (Z_k - conj Z_{n-k})/(2i).
// ===========================================================================
namespace fde {

template <typename R, int L, int NT>
static cudaError_t launch_prec_rows_reg_LN(int inverse, const R* r, R* z, cplx<R>* spec, long long nrows, int H,
                                           int Hp, const cplx<R>* twn, cudaStream_t st, Gate gate) {
  constexpr int PAIRS = NT / (L / 16);
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * (L + L / 16) * sizeof(cplx<R>);
  const PrecRowsRegArgs<R> a{r, z, spec, nrows, H, Hp, twn, gate};
  if (inverse)
    return launch_op<PrecRowsInvRegOp<R, L, NT>>(k_prec_rows_inv_reg<R, L, NT>, (unsigned)grid, NT, smem, st, a);
  return launch_op<PrecRowsFwdRegOp<R, L, NT>>(k_prec_rows_fwd_reg<R, L, NT>, (unsigned)grid, NT, smem, st, a);
}

template <typename R, int L>
static cudaError_t launch_prec_rows_reg_L(int inverse, const R* r, R* z, cplx<R>* spec, long long nrows, int H,
                                          int Hp, const cplx<R>* twn, cudaStream_t st, Gate gate) {
  static_assert(kPersistThreads == 256, "a recorded solve runs the rows transforms with the executor's block size");
  return launch_prec_rows_reg_LN<R, L, 256>(inverse, r, z, spec, nrows, H, Hp, twn, st, gate);
}

template <typename R>
cudaError_t launch_prec_rows_reg(int L, int inverse, const R* r, R* z, cplx<R>* spec, long long nrows, int H, int Hp,
                                 const cplx<R>* twn, cudaStream_t st, Gate gate) {
  switch (L) {
#define FDE_CASE(LL) \
  case LL: return launch_prec_rows_reg_L<R, LL>(inverse, r, z, spec, nrows, H, Hp, twn, st, gate);
    FDE_FOR_EACH_PL(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_prec_rows_reg<float>(int, int, const float*, float*, float2*, long long, int, int,
                                                 const float2*, cudaStream_t, Gate);
template cudaError_t launch_prec_rows_reg<double>(int, int, const double*, double*, double2*, long long, int, int,
                                                  const double2*, cudaStream_t, Gate);

cudaError_t precond_rows_reg_set_smem_attrs() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define FDE_ATTR(LL)                                                                                            \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(k_prec_rows_fwd_reg<float, LL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             big);                                                                              \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(k_prec_rows_inv_reg<float, LL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             big);                                                                              \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(k_prec_rows_fwd_reg<double, LL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);                                                                              \
  if (e == cudaSuccess)                                                                                         \
    e = cudaFuncSetAttribute(k_prec_rows_inv_reg<double, LL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);
  FDE_FOR_EACH_PL(FDE_ATTR)
#undef FDE_ATTR
#undef FDE_ATTR1
  return e;
}

}  // namespace fde
