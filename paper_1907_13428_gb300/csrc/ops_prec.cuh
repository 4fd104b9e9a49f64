// Bodies of the generic (any smooth length) preconditioner kernels of
// precond.cu: x2 rows to half spectra, complex columns of the half spectra
// (forward, inverse, or forward-divide-inverse on the time axis), and half
// spectra back to rows. The data path is described at the top of precond.cu.
#pragma once
#include "internal.h"
#include "ops_list.cuh"

namespace fde {

constexpr int kPEPT = 16;

// Spectral divide of the time pass (mode 2 of the column transforms).
struct DivArgs {
  int divide;     // 1 on the time pass
  int adjoint;    // 1: sigma = |Lambda|^2
  double m1, inv_m2, psi, inv_N;
  double cre;     // matching approximation: sigma += cre Re(Lambda) (0: S-tilde)
  int Hp, H;
  Gate gate;  // device-side skip of the launch (host-sync-free solve)
};

// Step 1: rows of r -> half spectra.
template <typename R> struct PrecRowsArgs {
  const R* r;           // forward: input rows
  R* z;                 // inverse: output rows
  cplx<R>* spec;
  long long nrows;
  int n, H, Hp;
  const cplx<R>* twn;
  FftPlan pl;
  int pairs;
  Gate gate;
};
template <typename R> struct PrecRowsFwdOp {
  using Args = PrecRowsArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& a) {
    if (gate_closed<PS>(a.gate)) return;
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n = a.n, H = a.H, pairs = a.pairs;
    const long long nrows = a.nrows;
    const long long row0 = c.bid * pairs * 2;
    for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
      const int p = e / n, j = e - p * n;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      const R va = ra < nrows ? ldv<PS>(a.r + ra * n + j) : (R)0;
      const R vb = rb < nrows ? ldv<PS>(a.r + rb * n + j) : (R)0;
      buf[p * n + j] = mk<C>(va, vb);
    }
    __syncthreads();
    lines_fft<PS, R, kPEPT>(buf, pairs, n, a.pl, a.twn, false);
    for (int e = threadIdx.x; e < pairs * H; e += blockDim.x) {
      const int p = e / H, k = e - p * H;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      const C zk = buf[p * n + k];
      const C zm = cconj(buf[p * n + (k == 0 ? 0 : n - k)]);
      // A = (Z_k + conj Z_{-k}) / 2,  B = (Z_k - conj Z_{-k}) / (2i)
      const C A = mk<C>((zk.x + zm.x) * (R)0.5, (zk.y + zm.y) * (R)0.5);
      const C D = mk<C>((zk.x - zm.x) * (R)0.5, (zk.y - zm.y) * (R)0.5);
      const C B = mk<C>(D.y, -D.x);
      if (ra < nrows) a.spec[ra * a.Hp + k] = A;
      if (rb < nrows) a.spec[rb * a.Hp + k] = B;
    }
    __syncthreads();  // the shared lines are reused by the next block of a persistent CTA
  }
};

// Step 5: half spectra -> rows of z.
template <typename R> struct PrecRowsInvOp {
  using Args = PrecRowsArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& a) {
    if (gate_closed<PS>(a.gate)) return;
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n = a.n, H = a.H, pairs = a.pairs;
    const long long nrows = a.nrows;
    const long long row0 = c.bid * pairs * 2;
    for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
      const int p = e / n, k = e - p * n;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      const bool lo = k < H;
      const int kk = lo ? k : n - k;
      C A = ra < nrows ? ldv<PS>(a.spec + ra * a.Hp + kk) : mk<C>(0, 0);
      C B = rb < nrows ? ldv<PS>(a.spec + rb * a.Hp + kk) : mk<C>(0, 0);
      if (!lo) {
        A = cconj(A);
        B = cconj(B);
      }
      buf[p * n + k] = mk<C>(A.x - B.y, A.y + B.x);  // A + i B
    }
    __syncthreads();
    lines_fft<PS, R, kPEPT>(buf, pairs, n, a.pl, a.twn, true);
    for (int e = threadIdx.x; e < pairs * n; e += blockDim.x) {
      const int p = e / n, j = e - p * n;
      const long long ra = row0 + 2 * p, rb = ra + 1;
      const C v = buf[p * n + j];
      if (ra < nrows) a.z[ra * n + j] = v.x;
      if (rb < nrows) a.z[rb * n + j] = v.y;
    }
    __syncthreads();
  }
};

// Steps 2-4: complex columns of spec along an axis (x1: stride Hp inside each
// time slice; t: stride nx*Hp). dv.divide = 0: forward (inverse = 0) or inverse
// transform; dv.divide = 1: forward, divide by sigma*N (or |Lambda|^2 * N), inverse.
template <typename R> struct PrecAxisArgs {
  cplx<R>* spec;
  int n;
  long long axis_stride, n_inner, outer_stride, n_outer;
  const cplx<R>* twn;
  FftPlan pl;
  int inverse, lines;
  DivArgs dv;
  const cplx<R>* lt;
  const cplx<R>* lx;
  const cplx<R>* ly;
};
template <typename R> struct PrecAxisOp {
  using Args = PrecAxisArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    const DivArgs& dv = g.dv;
    if (gate_closed<PS>(dv.gate)) return;
    using C = cplx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    const int n = g.n, lines = g.lines;
    const long long n_inner = g.n_inner;
    const long long total = g.n_outer * n_inner;
    const long long l0 = cx.bid * lines;
    for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
      const int a = e / lines, l = e - a * lines;
      const long long q = l0 + l;
      C v = mk<C>(0, 0);
      if (q < total) {
        const long long o = q / n_inner, c = q - o * n_inner;
        v = ldv<PS>(g.spec + o * g.outer_stride + c + a * g.axis_stride);
      }
      buf[l * n + a] = v;
    }
    __syncthreads();
    lines_fft<PS, R, kPEPT>(buf, lines, n, g.pl, g.twn, dv.divide ? false : (g.inverse != 0));
    if (dv.divide) {
      for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
        const int l = e / n, k = e - l * n;
        const long long q = l0 + l;
        if (q >= total) continue;
        const long long c = q % n_inner;  // = i*Hp + j within a time slice
        const int i = (int)(c / dv.Hp), j = (int)(c - (long long)i * dv.Hp);
        if (j >= dv.H) continue;  // padding column: stays zero
        const C a = __ldg(&g.lt[k]), b = __ldg(&g.lx[i]), d = __ldg(&g.ly[j]);
        const R lr = (R)dv.psi * (a.x - b.x - d.x);
        const R li = (R)dv.psi * (a.y - b.y - d.y);
        const R mag = lr * lr + li * li;
        const R sigma = dv.adjoint ? mag : (R)dv.m1 + mag * (R)dv.inv_m2 + (R)dv.cre * lr;
        const R s = (R)dv.inv_N / sigma;
        buf[e] = cscale(buf[e], s);
      }
      __syncthreads();
      lines_fft<PS, R, kPEPT>(buf, lines, n, g.pl, g.twn, true);
    }
    for (int e = threadIdx.x; e < lines * n; e += blockDim.x) {
      const int a = e / lines, l = e - a * lines;
      const long long q = l0 + l;
      if (q >= total) continue;
      const long long o = q / n_inner, c = q - o * n_inner;
      g.spec[o * g.outer_stride + c + a * g.axis_stride] = buf[l * n + a];
    }
    __syncthreads();
  }
};

}  // namespace fde
