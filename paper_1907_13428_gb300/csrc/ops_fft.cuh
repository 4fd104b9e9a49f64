// Bodies of the generic (any smooth length L) Toeplitz passes of toeplitz.cu:
// each block stages whole lines in shared memory and runs the radix-2/3/4/5/7
// Stockham transforms of common.cuh. The embedding and the two-lines-per-complex
// trick are those described at the top of toeplitz.cu.
#pragma once
#include "ops_list.cuh"
#include "toeplitz.cuh"

namespace fde {

// ---------------------------------------------------------------------------
// x2 axis: rows of n contiguous values; a block takes `pairs` row pairs and
// builds 2*pairs complex lines of length L (pair p, half s -> line 2p+s).
// ---------------------------------------------------------------------------
template <typename R> struct RowsArgs {
  const R* x;
  long long nrows;
  int n, L;
  const cplx<R>* sym;
  const cplx<R>* tw2;
  const cplx<R>* twL;
  FftPlan pl;
  int conj_sym, pairs;
  AxisEpi<R> E;
};
template <typename R> struct RowsOp {
  using Args = RowsArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& a) {
    if (gate_closed<PS>(a.E.gate)) return;
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n = a.n, L = a.L, pairs = a.pairs;
    const long long nrows = a.nrows;
    const long long row0 = c.bid * pairs * 2;
    const int nl = 2 * pairs;
    for (int e = threadIdx.x; e < pairs * L; e += blockDim.x) {
      const int p = e / L, j = e - p * L;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      R va = 0, vb = 0;
      if (j < n) {
        if (ra < nrows) va = ldv<PS>(a.x + ra * n + j);
        if (rb < nrows) vb = ldv<PS>(a.x + rb * n + j);
      }
      const C v = mk<C>(va, vb);
      buf[(2 * p) * L + j] = v;
      buf[(2 * p + 1) * L + j] = (j < n) ? cmul(v, __ldg(&a.tw2[j])) : mk<C>(0, 0);
    }
    __syncthreads();
    lines_fft<PS, R, kEPT>(buf, nl, L, a.pl, a.twL, false);
    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
      const int l = e / L, k = e - l * L;
      C w = __ldg(&a.sym[(l & 1) * L + k]);
      if (a.conj_sym) w.y = -w.y;
      buf[e] = cmul(buf[e], w);
    }
    __syncthreads();
    lines_fft<PS, R, kEPT>(buf, nl, L, a.pl, a.twL, true);
    for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
      const int p = e / n, j = e - p * n;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      const C v = cadd(buf[(2 * p) * L + j], cmul(buf[(2 * p + 1) * L + j], cconj(__ldg(&a.tw2[j]))));
      if (ra < nrows) axis_store<PS>(a.E, ra * n + j, (int)(ra / a.E.rows_per_slice), v.x);
      if (rb < nrows) axis_store<PS>(a.E, rb * n + j, (int)(rb / a.E.rows_per_slice), v.y);
    }
    __syncthreads();  // the shared lines are reused by the next block of a persistent CTA
  }
};

// ---------------------------------------------------------------------------
// Strided axis: line (o, c) reads x[o*outer_stride + c + a*axis_stride],
// a in [0, n); inner indices c are taken in pairs (c, c+1) packed as one
// complex line. A block takes `pairs` consecutive pairs (inner fastest).
// ---------------------------------------------------------------------------
template <typename R> struct AxisArgs {
  const R* x;
  int n, L;
  long long axis_stride, n_inner, outer_stride, n_outer;
  const cplx<R>* sym;
  const cplx<R>* tw2;
  const cplx<R>* twL;
  FftPlan pl;
  int conj_sym, pairs;
  AxisEpi<R> E;
};
template <typename R> struct AxisOp {
  using Args = AxisArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    if (gate_closed<PS>(g.E.gate)) return;
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n = g.n, L = g.L, pairs = g.pairs;
    const long long n_inner = g.n_inner, axis_stride = g.axis_stride, outer_stride = g.outer_stride;
    const long long npi = (n_inner + 1) / 2;
    const long long total = g.n_outer * npi;
    const long long q0 = cx.bid * pairs;
    const int nl = 2 * pairs;
    for (int e = threadIdx.x; e < pairs * L; e += blockDim.x) {
      const int a = e / pairs, p = e - a * pairs;
      const long long q = q0 + p;
      R va = 0, vb = 0;
      if (q < total && a < n) {
        const long long o = q / npi, c = 2 * (q - o * npi);
        const long long idx = o * outer_stride + c + a * axis_stride;
        va = ldv<PS>(g.x + idx);
        if (c + 1 < n_inner) vb = ldv<PS>(g.x + idx + 1);
      }
      const C v = mk<C>(va, vb);
      buf[(2 * p) * L + a] = v;
      buf[(2 * p + 1) * L + a] = (a < n) ? cmul(v, __ldg(&g.tw2[a])) : mk<C>(0, 0);
    }
    __syncthreads();
    lines_fft<PS, R, kEPT>(buf, nl, L, g.pl, g.twL, false);
    for (int e = threadIdx.x; e < nl * L; e += blockDim.x) {
      const int l = e / L, k = e - l * L;
      C w = __ldg(&g.sym[(l & 1) * L + k]);
      if (g.conj_sym) w.y = -w.y;
      buf[e] = cmul(buf[e], w);
    }
    __syncthreads();
    lines_fft<PS, R, kEPT>(buf, nl, L, g.pl, g.twL, true);
    for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
      const int a = e / pairs, p = e - a * pairs;
      const long long q = q0 + p;
      if (q >= total) continue;
      const long long o = q / npi, c = 2 * (q - o * npi);
      const long long idx = o * outer_stride + c + a * axis_stride;
      const C v = cadd(buf[(2 * p) * L + a], cmul(buf[(2 * p + 1) * L + a], cconj(__ldg(&g.tw2[a]))));
      const int t = g.E.t_is_axis ? a : (int)o;
      axis_store<PS>(g.E, idx, t, v.x);
      if (c + 1 < n_inner) axis_store<PS>(g.E, idx + 1, t, v.y);
    }
    __syncthreads();
  }
};

}  // namespace fde
