// Epilogue shared by the Toeplitz passes and the launchers of the register-resident
// passes (toeplitz.cu: generic passes and operators; toeplitz_reg.cuh: register-
// resident kernels, instantiated per arithmetic in toeplitz_reg_{f32,f64,dd}.cu).
#pragma once
#include <type_traits>

#include "internal.h"

namespace fde {


constexpr int kEPT = 16;  // complex elements staged per thread in an FFT pass

// Epilogue of a pass, per output element idx on time slice t:
//   out = dsc(t) * (acc[idx] + res + ct * (xt[idx] - xt[idx -/+ plane])) + addc(t) * addv[idx]
// with dsc/addc taking v0 on slices 0..nt-2 and v1 on the last slice.
template <typename R> struct AxisEpi {
  R* out;
  const R* acc;   // nullable
  const R* xt;    // nullable: time-difference term source
  int tdir;       // +1: x_t - x_{t-1} (B), -1: x_t - x_{t+1} (B^T)
  R ct;           // psi / h_t
  long long plane;
  int nt;
  int t_is_axis;  // strided passes: 1: time index = position along the axis; 0: = outer index
  long long rows_per_slice;  // x2 pass: time index = row / rows_per_slice (= nx)
  int plain;      // 1: out = res only (no acc, time term, diagonal or addend)
  int nb_only;    // 1: time term is -ct xt[idx -/+ plane] only (+ct x_t is in the x1 symbol)
  int has_dsc;
  R dsc0, dsc1;
  const R* addv;  // nullable
  R addc0, addc1;
  Gate gate;      // device-side skip of the whole launch (host-sync-free solve)
};

template <bool PS = false, typename R>
__device__ __forceinline__ void axis_store(const AxisEpi<R>& E, long long idx, int t, R res) {
  if (E.plain) {
    E.out[idx] = res;
    return;
  }
  R v = res;
  if (E.acc) v += ldv<PS>(E.acc + idx);
  if (E.xt) {
    R nb = 0;
    if (E.tdir > 0) {
      if (t > 0) nb = ldv<PS>(E.xt + idx - E.plane);
    } else {
      if (t < E.nt - 1) nb = ldv<PS>(E.xt + idx + E.plane);
    }
    v += E.nb_only ? -E.ct * nb : E.ct * (ldv<PS>(E.xt + idx) - nb);
  }
  const bool last = (t == E.nt - 1);
  if (E.has_dsc) v *= last ? E.dsc1 : E.dsc0;
  if (E.addv) v += (last ? E.addc1 : E.addc0) * ldv<PS>(E.addv + idx);
  E.out[idx] = v;
}


// Two-phase form of axis_store for batching the epilogue's loads: epi_load
// fetches the operands of one element, epi_finish combines and stores.
template <typename R> struct EpiIn {
  R acc, x0, xn, add;
};

template <bool PS = false, typename R>
__device__ __forceinline__ EpiIn<R> epi_load(const AxisEpi<R>& E, long long idx, int t) {
  EpiIn<R> in{0, 0, 0, 0};
  if (E.plain) return in;
  if (E.acc) in.acc = ldv<PS>(E.acc + idx);
  if (E.xt) {
    if (!E.nb_only) in.x0 = ldv<PS>(E.xt + idx);
    if (E.tdir > 0) {
      if (t > 0) in.xn = ldv<PS>(E.xt + idx - E.plane);
    } else {
      if (t < E.nt - 1) in.xn = ldv<PS>(E.xt + idx + E.plane);
    }
  }
  if (E.addv) in.add = ldv<PS>(E.addv + idx);
  return in;
}

template <typename R>
__device__ __forceinline__ void epi_finish(const AxisEpi<R>& E, const EpiIn<R>& in, long long idx, int t, R res) {
  if (E.plain) {
    E.out[idx] = res;
    return;
  }
  R v = res + in.acc;
  if (E.xt) v += E.nb_only ? -E.ct * in.xn : E.ct * (in.x0 - in.xn);
  const bool last = (t == E.nt - 1);
  if (E.has_dsc) v *= last ? E.dsc1 : E.dsc0;
  if (E.addv) v += (last ? E.addc1 : E.addc0) * in.add;
  E.out[idx] = v;
}

// Register-resident variants used for power-of-two L >= 16.
// R: transform arithmetic, S: storage of the vectors (S = R, or S = double with
// double-float arithmetic R = dd).
template <typename R, typename S>
cudaError_t launch_rows_reg(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym, const AxisTables<R>& T,
                            const AxisEpi<S>& E, cudaStream_t st);
template <typename R, typename S>
cudaError_t launch_axis_reg(int L, const S* x, int n, long long axis_stride, long long n_inner,
                            long long outer_stride, long long n_outer, const cplx<R>* sym, const AxisTables<R>& T,
                            int conj_sym, const AxisEpi<S>& E, int nt_choice, cudaStream_t st);
// Raise the dynamic shared-memory limits of every register-resident kernel of one arithmetic.
cudaError_t toeplitz_reg_attrs_f32();
cudaError_t toeplitz_reg_attrs_f64();
cudaError_t toeplitz_reg_attrs_dd();

}  // namespace fde
