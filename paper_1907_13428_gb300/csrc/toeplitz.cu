// Matrix-free products with the three-level Toeplitz operator
//   B = psi (C_t (x) I - I (x) X (x) I - I (x) I (x) Y)
// (Eq. FDE constraint matrix scaled by psi, Section 5) and with B^T.
//
// Each one-dimensional Toeplitz factor T (n x n) is applied by circulant
// embedding (Table "Complexity table", Toeplitz row): with L the smallest power
// of two >= n, T sits in a circulant of order 2L whose symbol lambda is the
// DFT of the embedded first column. The order-2L transform is split into its
// even and odd frequencies, which are two order-L transforms of x and of
// x_j W_{2L}^j, so lines never need 2L storage:
//   (T x)_i = 1/2 sum_{s=0,1} W_{2L}^{-s i} IFFT_L(lambda_{2k+s} FFT_L(x_j W_{2L}^{s j}))_i.
// Real lines are processed two at a time as the real and imaginary parts of
// one complex line (the product of a real line with a real circulant stays
// real, so the two results separate exactly). The symbol halves are stored
// pre-multiplied by coef/(2L), so a pass writes -psi X x (space) or +psi C_t x
// (time) directly; B^T uses the conjugate symbol.
//
// Passes: the x2 axis (contiguous rows), then the x1 axis (columns of stride
// ny). For alpha_t = 1 the time term (psi/h_t)(x_t - x_{t-1}) (reversed for
// B^T) is folded into the x1 pass; for alpha_t < 1 a third pass applies the
// lower-triangular Toeplitz C_t along t (stride nx*ny) by the same embedding.

#include "ops_fft.cuh"

namespace fde {
// Generic passes (bodies in ops_fft.cuh): lengths below 16 or with factors 3, 5,
// 7, and every pass of a recorded (persistent) solve.
template <typename R> __global__ void __launch_bounds__(512) k_rows(RowsArgs<R> a) {
  RowsOp<R>::template run<false>(hw_ctx(), a);
}
template <typename R> __global__ void __launch_bounds__(1024) k_axis(AxisArgs<R> a) {
  AxisOp<R>::template run<false>(hw_ctx(), a);
}

template <typename R> static const AxisTables<R>& tables(const Axis& A);
template <> const AxisTables<double>& tables<double>(const Axis& A) { return A.d; }
template <> const AxisTables<float>& tables<float>(const Axis& A) { return A.f; }
template <> const AxisTables<dd>& tables<dd>(const Axis& A) { return A.q; }

// Geometry of the strided passes: x1 lines inside each time slice, or t lines.
static void axis_geometry(const fde_problem* P, int axis, long long* axis_stride, long long* n_inner,
                          long long* outer_stride, long long* n_outer) {
  if (axis == 1) {
    *axis_stride = P->ny;
    *n_inner = P->ny;
    *outer_stride = (long long)P->nx * P->ny;
    *n_outer = P->nt;
  } else {
    *axis_stride = (long long)P->nx * P->ny;
    *n_inner = *axis_stride;
    *outer_stride = 0;
    *n_outer = 1;
  }
}

template <typename R> static int rows_threads(int L) { return (2 * L > kEPT * 256) ? 512 : 256; }

template <typename R>
static cudaError_t launch_rows(fde_problem* P, const R* x, int conj_sym, const cplx<R>* sym, const AxisEpi<R>& E,
                               cudaStream_t st) {
  const Axis& A = P->ax[2];
  const AxisTables<R>& T = tables<R>(A);
  const int L = A.L;
  // a recorded solve: float passes register-resident (the executor's block
  // size), double ones generic (bound by the double pipe either way)
  const bool rec = recording(), gen = rec && sizeof(R) != 4;
  if (L >= 16 && !gen) return launch_rows_reg<R, R>(P, x, conj_sym, sym ? sym : T.sym, T, E, st);
  const int threads = rec ? kPersistThreads : rows_threads<R>(L);
  const int cap = kEPT * threads;  // complex elements per CTA
  int pairs = cap / (2 * L);
  if (pairs < 1) pairs = 1;
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  if (pairs > npairs) pairs = (int)npairs;
  const long long grid = (npairs + pairs - 1) / pairs;
  const size_t smem = (size_t)2 * pairs * L * sizeof(cplx<R>);
  return launch_op<RowsOp<R>>(k_rows<R>, (unsigned)grid, threads, smem, st,
                              {x, nrows, A.n, L, sym ? sym : T.sym, T.tw2, T.twL, A.planL, conj_sym, pairs, E});
}

template <typename R>
static cudaError_t launch_axis(fde_problem* P, int axis, const R* x, int conj_sym, const cplx<R>* sym,
                               const AxisEpi<R>& E, cudaStream_t st) {
  const Axis& A = P->ax[axis];
  const AxisTables<R>& T = tables<R>(A);
  const int L = A.L;
  const bool rec = recording(), gen = rec && sizeof(R) != 4;
  const int threads = rec ? kPersistThreads : (sizeof(R) == 4 ? 1024 : 512);
  const int cap = kEPT * threads;
  int pairs = cap / (2 * L);
  if (pairs < 1) pairs = 1;
  long long axis_stride, n_inner, outer_stride, n_outer;
  axis_geometry(P, axis, &axis_stride, &n_inner, &outer_stride, &n_outer);
  if (L >= 16 && !gen)
    return launch_axis_reg<R, R>(L, x, A.n, axis_stride, n_inner, outer_stride, n_outer, sym ? sym : T.sym, T,
                                 conj_sym, E, rec ? kPersistThreads : sizeof(R) == 4 ? P->axis_nt32 : P->axis_nt64,
                                 st);
  const long long total = n_outer * ((n_inner + 1) / 2);
  if (pairs > total) pairs = (int)total;
  const long long grid = (total + pairs - 1) / pairs;
  const size_t smem = (size_t)2 * pairs * L * sizeof(cplx<R>);
  return launch_op<AxisOp<R>>(k_axis<R>, (unsigned)grid, threads, smem, st,
                              {x, A.n, L, axis_stride, n_inner, outer_stride, n_outer, sym ? sym : T.sym, T.tw2,
                               T.twL, A.planL, conj_sym, pairs, E});
}

// One pass of B (S: storage type, R: transform arithmetic). `shifted`: the x1
// symbol that carries the implicit-Euler diagonal. Axes shorter than 16 take
// the generic kernels in the storage precision.
template <typename S, typename R>
static cudaError_t pass_axis(fde_problem* P, int axis, const S* x, int conj_sym, bool shifted, const AxisEpi<S>& E,
                             cudaStream_t st) {
  const Axis& A = P->ax[axis];
  if constexpr (std::is_same<R, S>::value) {
    return launch_axis<R>(P, axis, x, conj_sym, shifted ? tables<R>(A).symD : nullptr, E, st);
  } else {
    if (A.L < 16) return launch_axis<S>(P, axis, x, conj_sym, shifted ? tables<S>(A).symD : nullptr, E, st);
    if (Recorder* r = active_recorder()) {  // no generic double-float pass to record
      r->error = 1;
      return cudaSuccess;
    }
    const AxisTables<R>& T = tables<R>(A);
    long long axis_stride, n_inner, outer_stride, n_outer;
    axis_geometry(P, axis, &axis_stride, &n_inner, &outer_stride, &n_outer);
    return launch_axis_reg<R, S>(A.L, x, A.n, axis_stride, n_inner, outer_stride, n_outer, shifted ? T.symD : T.sym,
                                 T, conj_sym, E, P->axis_ntdd, st);
  }
}

template <typename S, typename R>
static cudaError_t pass_rows(fde_problem* P, const S* x, int conj_sym, const AxisEpi<S>& E, cudaStream_t st) {
  if constexpr (std::is_same<R, S>::value) {
    return launch_rows<R>(P, x, conj_sym, nullptr, E, st);
  } else {
    const Axis& A = P->ax[2];
    if (A.L < 16) return launch_rows<S>(P, x, conj_sym, nullptr, E, st);
    if (Recorder* r = active_recorder()) {
      r->error = 1;
      return cudaSuccess;
    }
    return launch_rows_reg<R, S>(P, x, conj_sym, tables<R>(A).sym, tables<R>(A), E, st);
  }
}

template <typename S, typename R>
static cudaError_t apply_B_t(fde_problem* P, int transpose, const S* x, S* y, const SliceDiag* dscale, const S* addv,
                             const SliceDiag* addc, S* tmp1, S* tmp2, cudaStream_t st, Gate gate) {
  // x1 pass first (plain store), then the optional time pass, then the x2 pass,
  // whose coalesced epilogue adds the partial results, the implicit-Euler time
  // term, the per-slice diagonal and the addend.
  AxisEpi<S> Ex{};
  Ex.out = tmp1;
  Ex.nt = P->nt;
  Ex.plain = 1;
  Ex.gate = gate;
  // implicit Euler: the x1 symbol shifted by psi/h_t also adds +psi/h_t x_t
  // (where the problem carries that symbol; otherwise the epilogue adds it)
  const bool shifted = P->euler && tables<S>(P->ax[1]).symD != nullptr;
  cudaError_t err = pass_axis<S, R>(P, 1, x, transpose, shifted, Ex, st);
  if (err != cudaSuccess) return err;
  const S* acc = tmp1;
  if (!P->euler) {
    AxisEpi<S> Et{};
    Et.out = tmp2;
    Et.acc = tmp1;
    Et.nt = P->nt;
    Et.t_is_axis = 1;
    Et.gate = gate;
    err = pass_axis<S, R>(P, 0, x, transpose, false, Et, st);
    if (err != cudaSuccess) return err;
    acc = tmp2;
  }
  AxisEpi<S> E{};
  E.out = y;
  E.acc = acc;
  E.nt = P->nt;
  E.plane = (long long)P->nx * P->ny;
  E.rows_per_slice = P->nx;
  E.gate = gate;
  if (P->euler) {
    E.xt = x;
    E.tdir = transpose ? -1 : 1;
    E.ct = (S)(P->psi / P->ht);
    E.nb_only = shifted;
  }
  if (dscale) {
    E.has_dsc = 1;
    E.dsc0 = (S)dscale->v[0];
    E.dsc1 = (S)dscale->v[1];
  }
  if (addv) {
    E.addv = addv;
    E.addc0 = (S)addc->v[0];
    E.addc1 = (S)addc->v[1];
  }
  return pass_rows<S, R>(P, x, transpose, E, st);
}

template <typename R>
cudaError_t apply_B(fde_problem* P, int transpose, const R* x, R* y, const SliceDiag* dscale, const R* addv,
                    const SliceDiag* addc, R* tmp1, R* tmp2, cudaStream_t st, Gate gate) {
  return apply_B_t<R, R>(P, transpose, x, y, dscale, addv, addc, tmp1, tmp2, st, gate);
}

cudaError_t apply_B_df(fde_problem* P, int transpose, const double* x, double* y, const SliceDiag* dscale,
                       const double* addv, const SliceDiag* addc, double* tmp1, double* tmp2, cudaStream_t st,
                       Gate gate) {
  return apply_B_t<double, dd>(P, transpose, x, y, dscale, addv, addc, tmp1, tmp2, st, gate);
}

template <typename R>
cudaError_t apply_S(fde_problem* P, const SliceDiag& M1, const SliceDiag& M2inv, const R* x, R* y, R* w, R* tmp1,
                    R* tmp2, cudaStream_t st, Gate gate) {
  cudaError_t err = apply_B<R>(P, 0, x, w, &M2inv, nullptr, nullptr, tmp1, tmp2, st, gate);
  if (err != cudaSuccess) return err;
  return apply_B<R>(P, 1, w, y, nullptr, x, &M1, tmp1, tmp2, st, gate);
}

template <typename R>
cudaError_t apply_axis_raw(fde_problem* P, int axis, const R* x, R* y, const cplx<R>* sym, int conj_sym,
                           cudaStream_t st) {
  // one spatial factor along one axis (no time term, no accumulation)
  AxisEpi<R> E{};
  E.out = y;
  E.nt = P->nt;
  E.plane = (long long)P->nx * P->ny;
  E.rows_per_slice = P->nx;
  E.plain = 1;
  if (axis == 2) return launch_rows<R>(P, x, conj_sym, sym, E, st);
  return launch_axis<R>(P, axis, x, conj_sym, sym, E, st);
}

cudaError_t apply_axis_raw_df(fde_problem* P, int axis, const double* x, double* y, int conj_sym, cudaStream_t st) {
  const Axis& A = P->ax[axis];
  if (A.L < 16) return apply_axis_raw<double>(P, axis, x, y, A.d.sym, conj_sym, st);
  AxisEpi<double> E{};
  E.out = y;
  E.nt = P->nt;
  E.plane = (long long)P->nx * P->ny;
  E.rows_per_slice = P->nx;
  E.plain = 1;
  if (axis == 2) return launch_rows_reg<dd, double>(P, x, conj_sym, A.q.sym, A.q, E, st);
  long long axis_stride, n_inner, outer_stride, n_outer;
  axis_geometry(P, axis, &axis_stride, &n_inner, &outer_stride, &n_outer);
  return launch_axis_reg<dd, double>(A.L, x, A.n, axis_stride, n_inner, outer_stride, n_outer, A.q.sym, A.q,
                                     conj_sym, E, P->axis_ntdd, st);
}

template cudaError_t apply_B<double>(fde_problem*, int, const double*, double*, const SliceDiag*, const double*,
                                     const SliceDiag*, double*, double*, cudaStream_t, Gate);
template cudaError_t apply_B<float>(fde_problem*, int, const float*, float*, const SliceDiag*, const float*,
                                    const SliceDiag*, float*, float*, cudaStream_t, Gate);
template cudaError_t apply_S<double>(fde_problem*, const SliceDiag&, const SliceDiag&, const double*, double*,
                                     double*, double*, double*, cudaStream_t, Gate);
template cudaError_t apply_S<float>(fde_problem*, const SliceDiag&, const SliceDiag&, const float*, float*, float*,
                                    float*, float*, cudaStream_t, Gate);
template cudaError_t apply_axis_raw<double>(fde_problem*, int, const double*, double*, const double2*, int,
                                            cudaStream_t);
template cudaError_t apply_axis_raw<float>(fde_problem*, int, const float*, float*, const float2*, int, cudaStream_t);

}  // namespace fde

namespace fde {
cudaError_t toeplitz_set_smem_attrs() {
  const int big = 200 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_axis<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = cudaFuncSetAttribute(k_axis<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big))) return e;
  if ((e = toeplitz_reg_attrs_f32())) return e;
  if ((e = toeplitz_reg_attrs_f64())) return e;
  return toeplitz_reg_attrs_dd();
}
}  // namespace fde

namespace fde {


// Tile autotuning of the float, double-float and double passes: each variant runs three
// times on the problem's own sizes (after one warm-up launch) and the fastest is
// kept. x, y / xd, yd: scratch vectors of length N.
cudaError_t autotune_tiles(fde_problem* P, const float* x, float* y, const double* xd, double* yd, cudaStream_t st) {
  cudaEvent_t a, b;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  // arithmetic of the timed pass: 0 float, 1 double-float, 2 double
  auto run = [&](int axis, int kind) -> cudaError_t {
    if (kind == 1) return apply_axis_raw_df(P, axis, xd, yd, 0, st);
    if (kind == 2) return apply_axis_raw<double>(P, axis, xd, yd, P->ax[axis].d.sym, 0, st);
    return apply_axis_raw<float>(P, axis, x, y, P->ax[axis].f.sym, 0, st);
  };
  auto time_it = [&](int axis, int kind, float* ms) -> cudaError_t {
    cudaError_t r = run(axis, kind);
    if (r != cudaSuccess) return r;
    cudaEventRecord(a, st);
    for (int k = 0; k < 3 && r == cudaSuccess; ++k) r = run(axis, kind);
    cudaEventRecord(b, st);
    if (r == cudaSuccess) r = cudaEventSynchronize(b);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, a, b);
    return r;
  };
  // candidates of one tile field; negative: the split-halves variant with that many threads
  auto tune = [&](int* field, const int* cand, int nc, int axis, int kind, bool short_only_mask) -> cudaError_t {
    float best = 0.f, ms = 0.f;
    int pick = cand[0];
    bool first = true;
    for (int i = 0; i < nc; ++i) {
      const int c = cand[i];
      // the 128-thread and 256-thread split x2 tiles need a line of at most 2048
      if (short_only_mask && (c == 128 || c == -256) && P->ax[axis].L > 2048) continue;
      if (c == 128 && P->ax[axis].L > 2048) continue;
      *field = c;
      const cudaError_t r = time_it(axis, kind, &ms);
      if (r != cudaSuccess) return r;
      if (first || ms < best) {
        best = ms;
        pick = c;
        first = false;
      }
    }
    *field = pick;
    return cudaSuccess;
  };
  const int rows32[3] = {256, 128, 512};
  const int axis32[2] = {512, 256};
  const int rows64[4] = {256, -512, -256, 128};
  const int axis64[3] = {256, -512, 128};
  if (e == cudaSuccess) e = tune(&P->rows_nt32, rows32, 3, 2, 0, true);
  if (e == cudaSuccess) e = tune(&P->axis_nt32, axis32, 2, 1, 0, false);
  if (e == cudaSuccess) e = tune(&P->rows_ntdd, rows64, 4, 2, 1, true);
  if (e == cudaSuccess) e = tune(&P->axis_ntdd, axis64, 3, 1, 1, false);
  if (e == cudaSuccess) e = tune(&P->rows_nt64, rows64, 4, 2, 2, true);
  if (e == cudaSuccess) e = tune(&P->axis_nt64, axis64, 3, 1, 2, false);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace fde
