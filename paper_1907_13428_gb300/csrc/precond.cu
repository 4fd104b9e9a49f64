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
#include "ops_prec.cuh"

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
  const bool rec = recording();
  const bool rows_pow2 = ny >= 16 && (ny & (ny - 1)) == 0 && !rec;
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
    const bool pow2 = n >= 16 && (n & (n - 1)) == 0 && !rec;
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
// Register-resident column transforms for power-of-two lengths >= 16
// (fftreg.cuh). Lanes run over columns (coalesced); shared memory is
// position-major, CP columns per position row, with the physical row
// pos ^ parity(pos bits 1..4) so that the two position groups of every
// half-warp (quarter-warp for double) land in different bank halves.
// mode 0: forward (natural order in, frequency layout out),
// mode 1: inverse, mode 2: forward, divide by N sigma, inverse.
// ===========================================================================
#include "fftreg.cuh"

namespace fde {

// Plain transforms (modes 0, 1) are compiled for two resident CTAs (at most 64
// registers a thread with 512 threads): they move the whole spectrum through HBM
// and need the warps to hide its latency; the divide pass keeps one CTA.
template <int MODE> constexpr int prec_min_blocks() { return MODE == 2 ? 1 : 2; }

// 1/sigma: the float pass uses the fast reciprocal (a preconditioner needs no
// correctly rounded quotient), the double pass the IEEE quotient.
__device__ __forceinline__ float prec_recip(float s) { return __frcp_rn(s); }
__device__ __forceinline__ double prec_recip(double s) { return 1.0 / s; }

template <typename R, int L, int NT, int MODE>
__global__ void __launch_bounds__(NT, prec_min_blocks<MODE>()) k_prec_axis_reg(
    cplx<R>* __restrict__ spec, long long axis_stride, long long n_inner, long long outer_stride, long long n_outer,
    const cplx<R>* __restrict__ twn, DivArgs dv, const cplx<R>* __restrict__ lt, const cplx<R>* __restrict__ lx,
    const cplx<R>* __restrict__ ly) {
  constexpr int mode = MODE;
  if (gate_closed(dv.gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, CP = NT / T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int cl = threadIdx.x % CP, t = threadIdx.x / CP;
  const long long total = n_outer * n_inner;
  const long long q = (long long)blockIdx.x * CP + cl;
  const bool valid = q < total;
  const long long o = valid ? q / n_inner : 0;
  const long long c = valid ? q - o * n_inner : 0;
  const long long base = o * outer_stride + c;
  const FlipLayout<C, CP> lay{sm, cl};
  C v[1][16];
  if constexpr (mode == 1) {
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      const int p = rf_freq<L>(t, idx);
      v[0][idx] = valid ? spec[base + p * axis_stride] : mk<C>(0, 0);
    }
    rf_inverse<R, L, 1>(v, t, twn, lay);
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      v[0][r] = valid ? spec[base + p * axis_stride] : mk<C>(0, 0);
    }
    rf_forward<R, L, 1>(v, t, twn, lay);
    if constexpr (mode == 2) {
      const int i = (int)(c / dv.Hp), j = (int)(c - (long long)i * dv.Hp);
      const bool pad = j >= dv.H;
      const C b = pad ? mk<C>(0, 0) : __ldg(&lx[i]);
      const C d = pad ? mk<C>(0, 0) : __ldg(&ly[j]);
#pragma unroll
      for (int idx = 0; idx < 16; ++idx) {
        const int k = rf_freq<L>(t, idx);
        // sigma in the arithmetic of the transform (float on the float path:
        // double divides would run at 1/58 of the float rate)
        const C a = __ldg(&lt[k]);
        const R lr = (R)dv.psi * (a.x - b.x - d.x);
        const R li = (R)dv.psi * (a.y - b.y - d.y);
        const R mag = lr * lr + li * li;
        const R sigma = dv.adjoint ? mag : (R)dv.m1 + mag * (R)dv.inv_m2 + (R)dv.cre * lr;
        const R sc = pad ? (R)0 : (R)dv.inv_N * prec_recip(sigma);
        v[0][idx] = cscale(v[0][idx], sc);
      }
      rf_inverse<R, L, 1>(v, t, twn, lay);
    }
  }
  if (!valid) return;
  if constexpr (mode == 0) {
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) spec[base + rf_freq<L>(t, idx) * axis_stride] = v[0][idx];
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) spec[base + (t + r * T) * axis_stride] = v[0][r];
  }
}

template <typename R> constexpr int prec_nt() { return sizeof(R) == 4 ? 512 : 256; }

template <typename R, int L>
static cudaError_t launch_prec_axis_reg_L(cplx<R>* spec, long long axis_stride, long long n_inner,
                                          long long outer_stride, long long n_outer, const cplx<R>* twn, int mode,
                                          const DivArgs& dv, const cplx<R>* lt, const cplx<R>* lx, const cplx<R>* ly,
                                          cudaStream_t st) {
  constexpr int NT = prec_nt<R>();
  constexpr int CP = NT / (L / 16);
  const long long total = n_outer * n_inner;
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * CP * sizeof(cplx<R>);
  if (mode == 0)
    k_prec_axis_reg<R, L, NT, 0><<<(unsigned)grid, NT, smem, st>>>(spec, axis_stride, n_inner, outer_stride, n_outer,
                                                                   twn, dv, lt, lx, ly);
  else if (mode == 1)
    k_prec_axis_reg<R, L, NT, 1><<<(unsigned)grid, NT, smem, st>>>(spec, axis_stride, n_inner, outer_stride, n_outer,
                                                                   twn, dv, lt, lx, ly);
  else
    k_prec_axis_reg<R, L, NT, 2><<<(unsigned)grid, NT, smem, st>>>(spec, axis_stride, n_inner, outer_stride, n_outer,
                                                                   twn, dv, lt, lx, ly);
  note_launches(1);
  return cudaGetLastError();
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
__global__ void __launch_bounds__(NT) k_prec_rows_fwd_reg(const R* __restrict__ r, cplx<R>* __restrict__ spec,
                                                           long long nrows, int H, int Hp,
                                                           const cplx<R>* __restrict__ twn, Gate gate) {
  if (gate_closed(gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
  const long long ra = ((long long)blockIdx.x * PAIRS + pr) * 2, rb = ra + 1;
  C* my = sm + pr * LS;
  auto at = [my](int, int pos) -> C& { return my[pos + (pos >> 4)]; };
  const PadLayout<C, LS> lay{my};
  C v[1][16];
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p = t + q * T;
    v[0][q] = mk<C>(ra < nrows ? r[ra * L + p] : (R)0, rb < nrows ? r[rb * L + p] : (R)0);
  }
  rf_forward<R, L, 1>(v, t, twn, lay);
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) at(0, rf_freq<L>(t, idx)) = v[0][idx];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int k = t + q * T;
    if (k < H) {
      const C zk = at(0, k);
      const C zm = cconj(at(0, k == 0 ? 0 : L - k));
      const C A = mk<C>((zk.x + zm.x) * (R)0.5, (zk.y + zm.y) * (R)0.5);
      const C B = mk<C>((zk.y - zm.y) * (R)0.5, -(zk.x - zm.x) * (R)0.5);
      if (ra < nrows) spec[ra * Hp + k] = A;
      if (rb < nrows) spec[rb * Hp + k] = B;
    }
  }
}

template <typename R, int L, int NT>
__global__ void __launch_bounds__(NT) k_prec_rows_inv_reg(const cplx<R>* __restrict__ spec, R* __restrict__ z,
                                                           long long nrows, int H, int Hp,
                                                           const cplx<R>* __restrict__ twn, Gate gate) {
  if (gate_closed(gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
  const long long ra = ((long long)blockIdx.x * PAIRS + pr) * 2, rb = ra + 1;
  C* my = sm + pr * LS;
  const PadLayout<C, LS> lay{my};
  C v[1][16];
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) {
    const int k = rf_freq<L>(t, idx);
    const bool lo = k < H;
    const int kk = lo ? k : L - k;
    C A = ra < nrows ? spec[ra * Hp + kk] : mk<C>(0, 0);
    C B = rb < nrows ? spec[rb * Hp + kk] : mk<C>(0, 0);
    if (!lo) {
      A = cconj(A);
      B = cconj(B);
    }
    v[0][idx] = mk<C>(A.x - B.y, A.y + B.x);  // A + i B
  }
  rf_inverse<R, L, 1>(v, t, twn, lay);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int p = t + q * T;
    if (ra < nrows) z[ra * L + p] = v[0][q].x;
    if (rb < nrows) z[rb * L + p] = v[0][q].y;
  }
}

template <typename R, int L>
static cudaError_t launch_prec_rows_reg_L(int inverse, const R* r, R* z, cplx<R>* spec, long long nrows, int H,
                                          int Hp, const cplx<R>* twn, cudaStream_t st, Gate gate) {
  constexpr int NT = 256;
  constexpr int PAIRS = NT / (L / 16);
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * (L + L / 16) * sizeof(cplx<R>);
  if (inverse)
    k_prec_rows_inv_reg<R, L, NT><<<(unsigned)grid, NT, smem, st>>>(spec, z, nrows, H, Hp, twn, gate);
  else
    k_prec_rows_fwd_reg<R, L, NT><<<(unsigned)grid, NT, smem, st>>>(r, spec, nrows, H, Hp, twn, gate);
  note_launches(1);
  return cudaGetLastError();
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
