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

template <typename R>
__device__ __forceinline__ void axis_store(const AxisEpi<R>& E, long long idx, int t, R res) {
  if (E.plain) {
    E.out[idx] = res;
    return;
  }
  R v = res;
  if (E.acc) v += E.acc[idx];
  if (E.xt) {
    R nb = 0;
    if (E.tdir > 0) {
      if (t > 0) nb = E.xt[idx - E.plane];
    } else {
      if (t < E.nt - 1) nb = E.xt[idx + E.plane];
    }
    v += E.nb_only ? -E.ct * nb : E.ct * (E.xt[idx] - nb);
  }
  const bool last = (t == E.nt - 1);
  if (E.has_dsc) v *= last ? E.dsc1 : E.dsc0;
  if (E.addv) v += (last ? E.addc1 : E.addc0) * E.addv[idx];
  E.out[idx] = v;
}


// Two-phase form of axis_store for batching the epilogue's loads: epi_load
// fetches the operands of one element, epi_finish combines and stores.
template <typename R> struct EpiIn {
  R acc, x0, xn, add;
};

template <typename R>
__device__ __forceinline__ EpiIn<R> epi_load(const AxisEpi<R>& E, long long idx, int t) {
  EpiIn<R> in{0, 0, 0, 0};
  if (E.plain) return in;
  if (E.acc) in.acc = E.acc[idx];
  if (E.xt) {
    if (!E.nb_only) in.x0 = E.xt[idx];
    if (E.tdir > 0) {
      if (t > 0) in.xn = E.xt[idx - E.plane];
    } else {
      if (t < E.nt - 1) in.xn = E.xt[idx + E.plane];
    }
  }
  if (E.addv) in.add = E.addv[idx];
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

// ---------------------------------------------------------------------------
// x2 axis: rows of n contiguous values; a CTA takes `pairs` row pairs and
// builds 2*pairs complex lines of length L (pair p, half s -> line 2p+s).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(512) k_rows(const R* __restrict__ x, long long nrows, int n, int L,
                                               const cplx<R>* __restrict__ sym, const cplx<R>* __restrict__ tw2,
                                               const cplx<R>* __restrict__ twL, FftPlan pl, int conj_sym, int pairs,
                                               AxisEpi<R> E) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const long long row0 = (long long)blockIdx.x * pairs * 2;
  const int nl = 2 * pairs;
  for (int e = threadIdx.x; e < pairs * L; e += blockDim.x) {
    const int p = e / L, j = e - p * L;
    const long long ra = row0 + 2 * p, rb = ra + 1;
    R a = 0, b = 0;
    if (j < n) {
      if (ra < nrows) a = x[ra * n + j];
      if (rb < nrows) b = x[rb * n + j];
    }
    const C v = mk<C>(a, b);
    buf[(2 * p) * L + j] = v;
    buf[(2 * p + 1) * L + j] = (j < n) ? cmul(v, __ldg(&tw2[j])) : mk<C>(0, 0);
  }
  __syncthreads();
  smem_fft<R, kEPT>(buf, nl, L, pl, twL, false);
  for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
    const int l = e / L, k = e - l * L;
    C w = __ldg(&sym[(l & 1) * L + k]);
    if (conj_sym) w.y = -w.y;
    buf[e] = cmul(buf[e], w);
  }
  __syncthreads();
  smem_fft<R, kEPT>(buf, nl, L, pl, twL, true);
  for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
    const int p = e / n, j = e - p * n;
    const long long ra = row0 + 2 * p, rb = ra + 1;
    const C v = cadd(buf[(2 * p) * L + j], cmul(buf[(2 * p + 1) * L + j], cconj(__ldg(&tw2[j]))));
    if (ra < nrows) axis_store(E, ra * n + j, (int)(ra / E.rows_per_slice), v.x);
    if (rb < nrows) axis_store(E, rb * n + j, (int)(rb / E.rows_per_slice), v.y);
  }
}

// ---------------------------------------------------------------------------
// Strided axis: line (o, c) reads x[o*outer_stride + c + a*axis_stride],
// a in [0, n); inner indices c are taken in pairs (c, c+1) packed as one
// complex line. A CTA takes `pairs` consecutive pairs (inner fastest).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(1024) k_axis(const R* __restrict__ x, int n, int L, long long axis_stride,
                                                long long n_inner, long long outer_stride, long long n_outer,
                                                const cplx<R>* __restrict__ sym, const cplx<R>* __restrict__ tw2,
                                                const cplx<R>* __restrict__ twL, FftPlan pl, int conj_sym,
                                                int pairs, AxisEpi<R> E) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const long long npi = (n_inner + 1) / 2;
  const long long total = n_outer * npi;
  const long long q0 = (long long)blockIdx.x * pairs;
  const int nl = 2 * pairs;
  for (int e = threadIdx.x; e < pairs * L; e += blockDim.x) {
    const int a = e / pairs, p = e - a * pairs;
    const long long q = q0 + p;
    R va = 0, vb = 0;
    if (q < total && a < n) {
      const long long o = q / npi, c = 2 * (q - o * npi);
      const long long idx = o * outer_stride + c + a * axis_stride;
      va = x[idx];
      if (c + 1 < n_inner) vb = x[idx + 1];
    }
    const C v = mk<C>(va, vb);
    buf[(2 * p) * L + a] = v;
    buf[(2 * p + 1) * L + a] = (a < n) ? cmul(v, __ldg(&tw2[a])) : mk<C>(0, 0);
  }
  __syncthreads();
  smem_fft<R, kEPT>(buf, nl, L, pl, twL, false);
  for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
    const int l = e / L, k = e - l * L;
    C w = __ldg(&sym[(l & 1) * L + k]);
    if (conj_sym) w.y = -w.y;
    buf[e] = cmul(buf[e], w);
  }
  __syncthreads();
  smem_fft<R, kEPT>(buf, nl, L, pl, twL, true);
  for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
    const int a = e / pairs, p = e - a * pairs;
    const long long q = q0 + p;
    if (q >= total) continue;
    const long long o = q / npi, c = 2 * (q - o * npi);
    const long long idx = o * outer_stride + c + a * axis_stride;
    const C v = cadd(buf[(2 * p) * L + a], cmul(buf[(2 * p + 1) * L + a], cconj(__ldg(&tw2[a]))));
    const int t = E.t_is_axis ? a : (int)o;
    axis_store(E, idx, t, v.x);
    if (c + 1 < n_inner) axis_store(E, idx + 1, t, v.y);
  }
}

// Register-resident variants (defined below) used for power-of-two L >= 16.
// R: transform arithmetic, S: storage of the vectors (S = R, or S = double with
// double-float arithmetic R = dd).
template <typename R, typename S>
cudaError_t launch_rows_reg(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym, const AxisTables<R>& T,
                            const AxisEpi<S>& E, cudaStream_t st);
template <typename R, typename S>
cudaError_t launch_axis_reg(int L, const S* x, int n, long long axis_stride, long long n_inner,
                            long long outer_stride, long long n_outer, const cplx<R>* sym, const AxisTables<R>& T,
                            int conj_sym, const AxisEpi<S>& E, int nt_choice, cudaStream_t st);
cudaError_t toeplitz_reg_set_smem_attrs();

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
  if (L >= 16) return launch_rows_reg<R, R>(P, x, conj_sym, sym ? sym : T.sym, T, E, st);
  const int threads = rows_threads<R>(L);
  const int cap = kEPT * threads;  // complex elements per CTA
  int pairs = cap / (2 * L);
  if (pairs < 1) pairs = 1;
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  if (pairs > npairs) pairs = (int)npairs;
  const long long grid = (npairs + pairs - 1) / pairs;
  const size_t smem = (size_t)2 * pairs * L * sizeof(cplx<R>);
  k_rows<R><<<(unsigned)grid, threads, smem, st>>>(x, nrows, A.n, L, sym ? sym : T.sym, T.tw2, T.twL, A.planL,
                                                   conj_sym, pairs, E);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_axis(fde_problem* P, int axis, const R* x, int conj_sym, const cplx<R>* sym,
                               const AxisEpi<R>& E, cudaStream_t st) {
  const Axis& A = P->ax[axis];
  const AxisTables<R>& T = tables<R>(A);
  const int L = A.L;
  const int threads = sizeof(R) == 4 ? 1024 : 512;
  const int cap = kEPT * threads;
  int pairs = cap / (2 * L);
  if (pairs < 1) pairs = 1;
  long long axis_stride, n_inner, outer_stride, n_outer;
  axis_geometry(P, axis, &axis_stride, &n_inner, &outer_stride, &n_outer);
  if (L >= 16)
    return launch_axis_reg<R, R>(L, x, A.n, axis_stride, n_inner, outer_stride, n_outer, sym ? sym : T.sym, T,
                                 conj_sym, E, P->axis_nt32, st);
  const long long total = n_outer * ((n_inner + 1) / 2);
  if (pairs > total) pairs = (int)total;
  const long long grid = (total + pairs - 1) / pairs;
  const size_t smem = (size_t)2 * pairs * L * sizeof(cplx<R>);
  k_axis<R><<<(unsigned)grid, threads, smem, st>>>(x, A.n, L, axis_stride, n_inner, outer_stride, n_outer,
                                                   sym ? sym : T.sym, T.tw2, T.twL, A.planL, conj_sym, pairs, E);
  note_launches(1);
  return cudaGetLastError();
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
  return toeplitz_reg_set_smem_attrs();
}
}  // namespace fde

// ===========================================================================
// Register-resident variants (power-of-two L >= 16): each thread holds 16
// values of both embedding halves of one complex line (fftreg.cuh).
// ===========================================================================
#include "fftreg.cuh"

namespace fde {

// x2 axis. NT threads = PAIRS row pairs x T threads per line; thread t of a
// pair holds positions t + r T of the pair's two half-lines. Shared memory is
// line-major with one pad element per 16 (conflict-free exchanges).
// R: arithmetic of the transforms; S: storage type of the vectors (R, or double
// for double-float arithmetic).
// FULL: the lines fill the transform (n == L), so no position is out of range.
template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 ? 2 : 1)) k_rows_reg(const S* __restrict__ x, long long nrows,
                                                  int n, const cplx<R>* __restrict__ sym,
                                                  const cplx<R>* __restrict__ tw2, const cplx<R>* __restrict__ twL,
                                                  int conj_sym, AxisEpi<S> E) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
  const long long ra = ((long long)blockIdx.x * PAIRS + pr) * 2, rb = ra + 1;
  C* my = sm + pr * 2 * LS;
  auto at = [my](int l, int pos) -> C& { return my[l * LS + pos + (pos >> 4)]; };
  C v[2][16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    R a = 0, b = 0;
    if (FULL || p < n) {
      if (ra < nrows) a = cvt_in<R, S>(x[ra * n + p]);
      if (rb < nrows) b = cvt_in<R, S>(x[rb * n + p]);
    }
    v[0][r] = mk<C>(a, b);
    v[1][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
  }
  rf_forward<R, L, 2>(v, t, twL, at);
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) {
    const int k = rf_freq<L>(t, idx);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      C w = ldg_(&sym[l * L + k]);
      if (conj_sym) w.y = -w.y;
      v[l][idx] = cmul(v[l][idx], w);
    }
  }
  rf_inverse<R, L, 2>(v, t, twL, at);
  const int ta = (int)(ra / E.rows_per_slice), tb = (int)(rb / E.rows_per_slice);
  // epilogue in chunks of 4 positions: all operand loads of a chunk are issued
  // before any arithmetic or store, so their latencies overlap
#pragma unroll
  for (int r0 = 0; r0 < 16; r0 += 4) {
    EpiIn<S> ia[4], ib[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p = t + (r0 + k) * T;
      const bool ok = FULL || p < n;
      ia[k] = (ok && ra < nrows) ? epi_load(E, ra * n + p, ta) : EpiIn<S>{0, 0, 0, 0};
      ib[k] = (ok && rb < nrows) ? epi_load(E, rb * n + p, tb) : EpiIn<S>{0, 0, 0, 0};
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p = t + (r0 + k) * T;
      if (FULL || p < n) {
        const C res = cadd(v[0][r0 + k], cmul(v[1][r0 + k], cconj(ldg_(&tw2[p]))));
        if (ra < nrows) epi_finish(E, ia[k], ra * n + p, ta, cvt_out<S, R>(res.x));
        if (rb < nrows) epi_finish(E, ib[k], rb * n + p, tb, cvt_out<S, R>(res.y));
      }
    }
  }
}

// Strided axis. NT threads = CP column pairs x T; lanes run over column pairs
// (coalesced global access). Shared memory is position-major with the two
// halves' lines side by side; the line index is XOR-swizzled by the parity of
// the low five position bits, which separates the two position groups of every
// half-warp into different banks.
template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT) k_axis_reg(const S* __restrict__ x, int n, long long axis_stride,
                                                  long long n_inner, long long outer_stride, long long n_outer,
                                                  const cplx<R>* __restrict__ sym, const cplx<R>* __restrict__ tw2,
                                                  const cplx<R>* __restrict__ twL, int conj_sym, AxisEpi<S> E,
                                                  int vec2) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, CP = NT / T, LW = 2 * CP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int cl = threadIdx.x % CP, t = threadIdx.x / CP;
  const long long npi = (n_inner + 1) / 2;
  const long long total = n_outer * npi;
  const long long q = (long long)blockIdx.x * CP + cl;
  const bool valid = q < total;
  const long long o = valid ? q / npi : 0;
  const long long c = valid ? 2 * (q - o * npi) : 0;
  const long long base = o * outer_stride + c;
  const bool has_b = valid && (c + 1 < n_inner);
  auto at = [sm, cl](int l, int pos) -> C& {
    const int sw = (__popc(pos & 31) & 1) ? CP : 0;
    return sm[pos * LW + ((l * CP + cl) ^ sw)];
  };
  C v[2][16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    R a = 0, b = 0;
    if (valid && (FULL || p < n)) {
      const long long idx = base + p * axis_stride;
      if (vec2 && has_b) {
        const cplx<S> ab = *reinterpret_cast<const cplx<S>*>(x + idx);  // (c, c+1) as one aligned vector load
        a = cvt_in<R, S>(ab.x);
        b = cvt_in<R, S>(ab.y);
      } else {
        a = cvt_in<R, S>(x[idx]);
        if (has_b) b = cvt_in<R, S>(x[idx + 1]);
      }
    }
    v[0][r] = mk<C>(a, b);
    v[1][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
  }
  rf_forward<R, L, 2>(v, t, twL, at);
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) {
    const int k = rf_freq<L>(t, idx);
#pragma unroll
    for (int l = 0; l < 2; ++l) {
      C w = ldg_(&sym[l * L + k]);
      if (conj_sym) w.y = -w.y;
      v[l][idx] = cmul(v[l][idx], w);
    }
  }
  rf_inverse<R, L, 2>(v, t, twL, at);
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    if (valid && (FULL || p < n)) {
      const C res = cadd(v[0][r], cmul(v[1][r], cconj(ldg_(&tw2[p]))));
      const long long idx = base + p * axis_stride;
      if (E.plain && vec2 && has_b) {
        *reinterpret_cast<cplx<S>*>(E.out + idx) = mk<cplx<S>>(cvt_out<S, R>(res.x), cvt_out<S, R>(res.y));
        continue;
      }
      const int ts = E.t_is_axis ? p : (int)o;
      axis_store(E, idx, ts, cvt_out<S, R>(res.x));
      if (has_b) axis_store(E, idx + 1, ts, cvt_out<S, R>(res.y));
    }
  }
}

// ---------------------------------------------------------------------------
// Split-halves variants (used for double-float on double vectors): the two
// embedding halves of a line pair are transformed by two thread groups, so a
// thread holds the 16 values of one line (half the registers of data) and twice
// as many warps fit on an SM (16 at 128 registers). For float the kernels that
// hold both halves per thread are faster (measured), so only the double-float
// instantiations are launched. After
// the inverse transforms each group finishes every other position r (r % 2 ==
// its half), taking the other half's term for those positions from shared
// memory (the exchange buffers are free once the inverse has passed its last
// barrier).
// ---------------------------------------------------------------------------
template <typename R> constexpr int split_min_blocks(int nt) { return (sizeof(R) == 4 ? 1024 : 512) / nt; }

template <typename R, int L, int NT, typename S = R>
__global__ void __launch_bounds__(NT, split_min_blocks<R>(NT)) k_rows_split(const S* __restrict__ x, long long nrows,
                                                                           int n, const cplx<R>* __restrict__ sym,
                                                                           const cplx<R>* __restrict__ tw2,
                                                                           const cplx<R>* __restrict__ twL,
                                                                           int conj_sym, AxisEpi<S> E) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, PAIRS = NT / (2 * T), LS = L + L / 16;
  static_assert(PAIRS >= 1, "at least one row pair per CTA");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int pr = threadIdx.x / (2 * T);
  const int h = (threadIdx.x / T) & 1;
  const int t = threadIdx.x % T;
  const long long ra = ((long long)blockIdx.x * PAIRS + pr) * 2, rb = ra + 1;
  C* my = sm + (pr * 2 + h) * LS;
  C* other = sm + (pr * 2 + (h ^ 1)) * LS;
  auto at = [my](int, int pos) -> C& { return my[pos + (pos >> 4)]; };
  C v[1][16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    R a = 0, b = 0;
    if (p < n) {
      if (ra < nrows) a = cvt_in<R, S>(x[ra * n + p]);
      if (rb < nrows) b = cvt_in<R, S>(x[rb * n + p]);
    }
    v[0][r] = mk<C>(a, b);
    if (h) v[0][r] = p < n ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
  }
  rf_forward<R, L, 1>(v, t, twL, at);
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) {
    C w = ldg_(&sym[h * L + rf_freq<L>(t, idx)]);
    if (conj_sym) w.y = -w.y;
    v[0][idx] = cmul(v[0][idx], w);
  }
  rf_inverse<R, L, 1>(v, t, twL, at);
  // the odd half's term is v conj(tw2[p]); hand over the positions the other group finishes
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    if (h) v[0][r] = p < n ? cmul(v[0][r], cconj(ldg_(&tw2[p]))) : mk<C>(0, 0);
    if ((r & 1) != h) my[p + (p >> 4)] = v[0][r];
  }
  __syncthreads();
  const int ta = (int)(ra / E.rows_per_slice), tb = (int)(rb / E.rows_per_slice);
#pragma unroll
  for (int c0 = 0; c0 < 8; c0 += 4) {
    EpiIn<S> ia[4], ib[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int p = t + (2 * (c0 + k) + h) * T;
      const bool ok = p < n;
      ia[k] = (ok && ra < nrows) ? epi_load(E, ra * n + p, ta) : EpiIn<S>{0, 0, 0, 0};
      ib[k] = (ok && rb < nrows) ? epi_load(E, rb * n + p, tb) : EpiIn<S>{0, 0, 0, 0};
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = 2 * (c0 + k) + h;
      const int p = t + r * T;
      if (p < n) {
        const C res = cadd(v[0][r], other[p + (p >> 4)]);
        if (ra < nrows) epi_finish(E, ia[k], ra * n + p, ta, cvt_out<S, R>(res.x));
        if (rb < nrows) epi_finish(E, ib[k], rb * n + p, tb, cvt_out<S, R>(res.y));
      }
    }
  }
}

template <typename R, int L, int NT, typename S = R>
__global__ void __launch_bounds__(NT, split_min_blocks<R>(NT)) k_axis_split(const S* __restrict__ x, int n,
                                                                           long long axis_stride, long long n_inner,
                                                                           long long outer_stride, long long n_outer,
                                                                           const cplx<R>* __restrict__ sym,
                                                                           const cplx<R>* __restrict__ tw2,
                                                                           const cplx<R>* __restrict__ twL,
                                                                           int conj_sym, AxisEpi<S> E, int vec2) {
  if (gate_closed(E.gate)) return;
  using C = cplx<R>;
  constexpr int T = L / 16, CP = NT / (2 * T), LW = 2 * CP;
  static_assert(CP >= 1, "at least one column pair per CTA");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  // lanes run over column pairs (coalesced), then over the two halves, then over t
  const int cl = threadIdx.x % CP;
  const int h = (threadIdx.x / CP) & 1;
  const int t = threadIdx.x / (2 * CP);
  const long long npi = (n_inner + 1) / 2;
  const long long total = n_outer * npi;
  const long long q = (long long)blockIdx.x * CP + cl;
  const bool valid = q < total;
  const long long o = valid ? q / npi : 0;
  const long long c = valid ? 2 * (q - o * npi) : 0;
  const long long base = o * outer_stride + c;
  const bool has_b = valid && (c + 1 < n_inner);
  auto slot = [cl](int l, int pos) -> int {
    const int sw = (__popc(pos & 31) & 1) ? CP : 0;
    return pos * LW + ((l * CP + cl) ^ sw);
  };
  auto at = [sm, h, slot](int, int pos) -> C& { return sm[slot(h, pos)]; };
  C v[1][16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    R a = 0, b = 0;
    if (valid && p < n) {
      const long long idx = base + p * axis_stride;
      if (vec2 && has_b) {
        const cplx<S> ab = *reinterpret_cast<const cplx<S>*>(x + idx);
        a = cvt_in<R, S>(ab.x);
        b = cvt_in<R, S>(ab.y);
      } else {
        a = cvt_in<R, S>(x[idx]);
        if (has_b) b = cvt_in<R, S>(x[idx + 1]);
      }
    }
    v[0][r] = mk<C>(a, b);
    if (h) v[0][r] = p < n ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
  }
  rf_forward<R, L, 1>(v, t, twL, at);
#pragma unroll
  for (int idx = 0; idx < 16; ++idx) {
    C w = ldg_(&sym[h * L + rf_freq<L>(t, idx)]);
    if (conj_sym) w.y = -w.y;
    v[0][idx] = cmul(v[0][idx], w);
  }
  rf_inverse<R, L, 1>(v, t, twL, at);
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int p = t + r * T;
    if (h) v[0][r] = p < n ? cmul(v[0][r], cconj(ldg_(&tw2[p]))) : mk<C>(0, 0);
    if ((r & 1) != h) sm[slot(h, p)] = v[0][r];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int r = 2 * k + h;
    const int p = t + r * T;
    if (valid && p < n) {
      const C res = cadd(v[0][r], sm[slot(h ^ 1, p)]);
      const long long idx = base + p * axis_stride;
      if (E.plain && vec2 && has_b) {
        *reinterpret_cast<cplx<S>*>(E.out + idx) = mk<cplx<S>>(cvt_out<S, R>(res.x), cvt_out<S, R>(res.y));
        continue;
      }
      const int ts = E.t_is_axis ? p : (int)o;
      axis_store(E, idx, ts, cvt_out<S, R>(res.x));
      if (has_b) axis_store(E, idx + 1, ts, cvt_out<S, R>(res.y));
    }
  }
}

template <typename R> constexpr int rows_nt() { return 256; }
template <typename R> constexpr int axis_nt() { return sizeof(R) == 4 ? 512 : 256; }

template <typename R, int L, int NT, typename S>
static cudaError_t launch_rows_reg_LN(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                      const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int PAIRS = NT / (L / 16);
  static_assert(PAIRS >= 1, "at least one row pair per CTA");
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * 2 * (L + L / 16) * sizeof(cplx<R>);
  if constexpr (std::is_same<R, float>::value) {
    if (P->ax[2].n == L) {
      k_rows_reg<R, L, NT, S, true><<<(unsigned)grid, NT, smem, st>>>(x, nrows, L, sym, T.tw2, T.twL, conj_sym, E);
      note_launches(1);
      return cudaGetLastError();
    }
  }
  k_rows_reg<R, L, NT, S><<<(unsigned)grid, NT, smem, st>>>(x, nrows, P->ax[2].n, sym, T.tw2, T.twL, conj_sym, E);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_rows_split_LN(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                        const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int PAIRS = NT / (2 * (L / 16));
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * 2 * (L + L / 16) * sizeof(cplx<R>);
  k_rows_split<R, L, NT, S><<<(unsigned)grid, NT, smem, st>>>(x, nrows, P->ax[2].n, sym, T.tw2, T.twL, conj_sym, E);
  note_launches(1);
  return cudaGetLastError();
}

// float: the tile chosen by fde_autotune (128 or 256 threads, or the split-halves
// variant with 256 or 512 threads, stored negated); double and double-float: 256
template <typename R, int L, typename S>
static cudaError_t launch_rows_reg_L(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                     const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value && std::is_same<S, float>::value) {
    if constexpr (L <= 2048) {
      if (P->rows_nt32 == 128) return launch_rows_reg_LN<R, L, 128, S>(P, x, conj_sym, sym, T, E, st);
    }
  }
  if constexpr (std::is_same<R, dd>::value) {
    if constexpr (2 * (L / 16) <= 256) {
      if (P->rows_ntdd == -256) return launch_rows_split_LN<R, L, 256, S>(P, x, conj_sym, sym, T, E, st);
    }
    if (P->rows_ntdd == -512) return launch_rows_split_LN<R, L, 512, S>(P, x, conj_sym, sym, T, E, st);
  }
  return launch_rows_reg_LN<R, L, rows_nt<R>(), S>(P, x, conj_sym, sym, T, E, st);
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_axis_reg_LN(const S* x, int n, long long axis_stride, long long n_inner,
                                      long long outer_stride, long long n_outer, const cplx<R>* sym,
                                      const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int CP = NT / (L / 16);
  static_assert(CP >= 1, "at least one column pair per CTA");
  const long long total = n_outer * ((n_inner + 1) / 2);
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * 2 * CP * sizeof(cplx<R>);
  const size_t al = 2 * sizeof(S);
  const int vec2 = ((n_inner | axis_stride | outer_stride) & 1) == 0 && ((uintptr_t)x % al) == 0 &&
                   ((uintptr_t)E.out % al) == 0;
  if constexpr (std::is_same<R, float>::value) {
    if (n == L) {
      k_axis_reg<R, L, NT, S, true><<<(unsigned)grid, NT, smem, st>>>(x, L, axis_stride, n_inner, outer_stride,
                                                                      n_outer, sym, T.tw2, T.twL, conj_sym, E, vec2);
      note_launches(1);
      return cudaGetLastError();
    }
  }
  k_axis_reg<R, L, NT, S><<<(unsigned)grid, NT, smem, st>>>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym,
                                                            T.tw2, T.twL, conj_sym, E, vec2);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_axis_split_LN(const S* x, int n, long long axis_stride, long long n_inner,
                                        long long outer_stride, long long n_outer, const cplx<R>* sym,
                                        const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E,
                                        cudaStream_t st) {
  constexpr int CP = NT / (2 * (L / 16));
  const long long total = n_outer * ((n_inner + 1) / 2);
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * 2 * CP * sizeof(cplx<R>);
  const size_t al = 2 * sizeof(S);
  const int vec2 = ((n_inner | axis_stride | outer_stride) & 1) == 0 && ((uintptr_t)x % al) == 0 &&
                   ((uintptr_t)E.out % al) == 0;
  k_axis_split<R, L, NT, S><<<(unsigned)grid, NT, smem, st>>>(x, n, axis_stride, n_inner, outer_stride, n_outer,
                                                              sym, T.tw2, T.twL, conj_sym, E, vec2);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R, int L, typename S>
static cudaError_t launch_axis_reg_L(const S* x, int n, long long axis_stride, long long n_inner,
                                     long long outer_stride, long long n_outer, const cplx<R>* sym,
                                     const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E, int nt_choice,
                                     cudaStream_t st) {
  if constexpr (std::is_same<R, dd>::value) {
    if (nt_choice == -512)
      return launch_axis_split_LN<R, L, 512, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym,
                                                E, st);
  }
  if constexpr (sizeof(R) == 4) {
    if (nt_choice == 256)
      return launch_axis_reg_LN<R, L, 256, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym,
                                              E, st);
  }
  return launch_axis_reg_LN<R, L, axis_nt<R>(), S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T,
                                                   conj_sym, E, st);
}

#define FDE_FOR_EACH_L(M) M(16) M(32) M(64) M(128) M(256) M(512) M(1024) M(2048) M(4096)

template <typename R, typename S>
cudaError_t launch_rows_reg(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym, const AxisTables<R>& T,
                            const AxisEpi<S>& E, cudaStream_t st) {
  switch (P->ax[2].L) {
#define FDE_CASE(LL) \
  case LL: return launch_rows_reg_L<R, LL, S>(P, x, conj_sym, sym, T, E, st);
    FDE_FOR_EACH_L(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, typename S>
cudaError_t launch_axis_reg(int L, const S* x, int n, long long axis_stride, long long n_inner,
                            long long outer_stride, long long n_outer, const cplx<R>* sym, const AxisTables<R>& T,
                            int conj_sym, const AxisEpi<S>& E, int nt_choice, cudaStream_t st) {
  switch (L) {
#define FDE_CASE(LL)                                                                                          \
  case LL:                                                                                                    \
    return launch_axis_reg_L<R, LL, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym, E, \
                                       nt_choice, st);
    FDE_FOR_EACH_L(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_rows_reg<double, double>(fde_problem*, const double*, int, const double2*,
                                                     const AxisTables<double>&, const AxisEpi<double>&, cudaStream_t);
template cudaError_t launch_rows_reg<float, float>(fde_problem*, const float*, int, const float2*,
                                                   const AxisTables<float>&, const AxisEpi<float>&, cudaStream_t);
template cudaError_t launch_rows_reg<dd, double>(fde_problem*, const double*, int, const dd2*, const AxisTables<dd>&,
                                                 const AxisEpi<double>&, cudaStream_t);
template cudaError_t launch_axis_reg<double, double>(int, const double*, int, long long, long long, long long,
                                                     long long, const double2*, const AxisTables<double>&, int,
                                                     const AxisEpi<double>&, int, cudaStream_t);
template cudaError_t launch_axis_reg<float, float>(int, const float*, int, long long, long long, long long, long long,
                                                   const float2*, const AxisTables<float>&, int,
                                                   const AxisEpi<float>&, int, cudaStream_t);
template cudaError_t launch_axis_reg<dd, double>(int, const double*, int, long long, long long, long long, long long,
                                                 const dd2*, const AxisTables<dd>&, int, const AxisEpi<double>&, int,
                                                 cudaStream_t);

template <typename R, typename S = R>
static cudaError_t set_attrs_reg() {
  const int big = 200 * 1024;
  cudaError_t e = cudaSuccess;
#define FDE_ATTR(LL)                                                                                           \
  if (e == cudaSuccess)                                                                                        \
    e = cudaFuncSetAttribute(k_rows_reg<R, LL, rows_nt<R>(), S>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                             big);                                                                             \
  if (e == cudaSuccess)                                                                                        \
    e = cudaFuncSetAttribute(k_axis_reg<R, LL, axis_nt<R>(), S>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  FDE_FOR_EACH_L(FDE_ATTR)
#undef FDE_ATTR
  return e;
}

cudaError_t toeplitz_reg_set_smem_attrs() {
  cudaError_t e = set_attrs_reg<float>();
  if (e != cudaSuccess) return e;
  if ((e = set_attrs_reg<double>()) != cudaSuccess) return e;
  if ((e = set_attrs_reg<dd, double>()) != cudaSuccess) return e;
  {
    const int big = 200 * 1024;
#define FDE_ATTR6(LL)                                                                                             \
    if (e == cudaSuccess)                                                                                         \
      e = cudaFuncSetAttribute(k_rows_split<dd, LL, 512, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                               big);                                                                              \
    if (e == cudaSuccess)                                                                                         \
      e = cudaFuncSetAttribute(k_axis_split<dd, LL, 512, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                               big);
    FDE_FOR_EACH_L(FDE_ATTR6)
#undef FDE_ATTR6
#define FDE_ATTR7(LL)                                                                                             \
    if (e == cudaSuccess)                                                                                         \
      e = cudaFuncSetAttribute(k_rows_split<dd, LL, 256, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                               big);
    FDE_ATTR7(16) FDE_ATTR7(32) FDE_ATTR7(64) FDE_ATTR7(128) FDE_ATTR7(256) FDE_ATTR7(512) FDE_ATTR7(1024)
    FDE_ATTR7(2048)
#undef FDE_ATTR7
    if (e != cudaSuccess) return e;
  }
  const int big = 200 * 1024;
#define FDE_ATTR2(LL)                                                                                        \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_axis_reg<float, LL, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  FDE_FOR_EACH_L(FDE_ATTR2)
#undef FDE_ATTR2
#define FDE_ATTR9(LL)                                                                                        \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_rows_reg<float, LL, 256, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);                                                                           \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_axis_reg<float, LL, 512, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);                                                                           \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_axis_reg<float, LL, 256, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);
  FDE_FOR_EACH_L(FDE_ATTR9)
#undef FDE_ATTR9
#define FDE_ATTR10(LL)                                                                                       \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_rows_reg<float, LL, 128, float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);
  FDE_ATTR10(16) FDE_ATTR10(32) FDE_ATTR10(64) FDE_ATTR10(128) FDE_ATTR10(256) FDE_ATTR10(512) FDE_ATTR10(1024)
  FDE_ATTR10(2048)
#undef FDE_ATTR10
#define FDE_ATTR3(LL)                                                                                        \
  if (e == cudaSuccess)                                                                                      \
    e = cudaFuncSetAttribute(k_rows_reg<float, LL, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  FDE_ATTR3(16) FDE_ATTR3(32) FDE_ATTR3(64) FDE_ATTR3(128) FDE_ATTR3(256) FDE_ATTR3(512) FDE_ATTR3(1024)
  FDE_ATTR3(2048)
#undef FDE_ATTR3
  return e;
}

// Tile autotuning of the float and double-float passes: each variant runs three
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
  auto run = [&](int axis, bool dfl) -> cudaError_t {
    return dfl ? apply_axis_raw_df(P, axis, xd, yd, 0, st)
               : apply_axis_raw<float>(P, axis, x, y, P->ax[axis].f.sym, 0, st);
  };
  auto time_it = [&](int axis, bool dfl, float* ms) -> cudaError_t {
    cudaError_t r = run(axis, dfl);
    if (r != cudaSuccess) return r;
    cudaEventRecord(a, st);
    for (int k = 0; k < 3 && r == cudaSuccess; ++k) r = run(axis, dfl);
    cudaEventRecord(b, st);
    if (r == cudaSuccess) r = cudaEventSynchronize(b);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, a, b);
    return r;
  };
  // candidates of one tile field; negative: the split-halves variant with that many threads
  auto tune = [&](int* field, const int* cand, int nc, int axis, bool dfl, bool short_only_mask) -> cudaError_t {
    float best = 0.f, ms = 0.f;
    int pick = cand[0];
    bool first = true;
    for (int i = 0; i < nc; ++i) {
      const int c = cand[i];
      // the 128-thread and 256-thread split x2 tiles need a line of at most 2048
      if (short_only_mask && (c == 128 || c == -256) && P->ax[axis].L > 2048) continue;
      *field = c;
      const cudaError_t r = time_it(axis, dfl, &ms);
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
  const int rows32[2] = {256, 128};
  const int axis32[2] = {512, 256};
  const int rowsdd[3] = {256, -512, -256};
  const int axisdd[2] = {256, -512};
  if (e == cudaSuccess) e = tune(&P->rows_nt32, rows32, 2, 2, false, true);
  if (e == cudaSuccess) e = tune(&P->axis_nt32, axis32, 2, 1, false, false);
  if (e == cudaSuccess) e = tune(&P->rows_ntdd, rowsdd, 3, 2, true, true);
  if (e == cudaSuccess) e = tune(&P->axis_ntdd, axisdd, 2, 1, true, false);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace fde
