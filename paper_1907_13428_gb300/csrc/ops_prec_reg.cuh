// Bodies of the register-resident preconditioner kernels of precond.cu
// (power-of-two lengths >= 16, fftreg.cuh): the column transforms of the half
// spectra (mode 0 forward: natural order in, frequency layout out; mode 1
// inverse; mode 2 forward, divide by N sigma, inverse) and the x2-row
// transforms. Column kernels: lanes run over columns (coalesced); shared memory
// is position-major, CP columns per position row, with the physical row
// pos ^ parity(pos bits 1..4) so that the two position groups of every
// half-warp (quarter-warp for double) land in different bank halves. Row
// kernels: two real rows a, b form the complex line a + i b; the half spectra
// are A_k = (Z_k + conj Z_{n-k})/2 and B_k = (Z_k - conj Z_{n-k})/(2i).
#pragma once
#include "fftreg.cuh"
#include "ops_prec.cuh"

namespace fde {

// 1/sigma: the float pass uses the fast reciprocal (a preconditioner needs no
// correctly rounded quotient), the double pass the IEEE quotient.
__device__ __forceinline__ float prec_recip(float s) { return __frcp_rn(s); }
__device__ __forceinline__ double prec_recip(double s) { return 1.0 / s; }

template <typename R> struct PrecAxisRegArgs {
  cplx<R>* spec;
  long long axis_stride, n_inner, outer_stride, n_outer;
  const cplx<R>* twn;
  DivArgs dv;
  const cplx<R>* lt;
  const cplx<R>* lx;
  const cplx<R>* ly;
};

template <typename R, int L, int NT, int MODE> struct PrecAxisRegOp {
  using Args = PrecAxisRegArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    constexpr int mode = MODE;
    const DivArgs& dv = g.dv;
    if (gate_closed<PS>(dv.gate)) return;
    using C = cplx<R>;
    constexpr int T = L / 16, CP = NT / T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    cplx<R>* spec = g.spec;
    const long long axis_stride = g.axis_stride, n_inner = g.n_inner;
    const int cl = threadIdx.x % CP, t = threadIdx.x / CP;
    const long long total = g.n_outer * n_inner;
    const long long q = cx.bid * CP + cl;
    const bool valid = q < total;
    const long long o = valid ? q / n_inner : 0;
    const long long c = valid ? q - o * n_inner : 0;
    const long long base = o * g.outer_stride + c;
    const FlipLayout<C, CP> lay{sm, cl};
    C v[1][16];
    if constexpr (mode == 1) {
#pragma unroll
      for (int idx = 0; idx < 16; ++idx) {
        const int p = rf_freq<L>(t, idx);
        v[0][idx] = valid ? ldv<PS>(spec + base + p * axis_stride) : mk<C>(0, 0);
      }
      rf_inverse<R, L, 1>(v, t, g.twn, lay);
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = t + r * T;
        v[0][r] = valid ? ldv<PS>(spec + base + p * axis_stride) : mk<C>(0, 0);
      }
      rf_forward<R, L, 1>(v, t, g.twn, lay);
      if constexpr (mode == 2) {
        const int i = (int)(c / dv.Hp), j = (int)(c - (long long)i * dv.Hp);
        const bool pad = j >= dv.H;
        const C b = pad ? mk<C>(0, 0) : __ldg(&g.lx[i]);
        const C d = pad ? mk<C>(0, 0) : __ldg(&g.ly[j]);
#pragma unroll
        for (int idx = 0; idx < 16; ++idx) {
          const int k = rf_freq<L>(t, idx);
          // sigma in the arithmetic of the transform (float on the float path:
          // double divides would run at 1/58 of the float rate)
          const C a = __ldg(&g.lt[k]);
          const R lr = (R)dv.psi * (a.x - b.x - d.x);
          const R li = (R)dv.psi * (a.y - b.y - d.y);
          const R mag = lr * lr + li * li;
          const R sigma = dv.adjoint ? mag : (R)dv.m1 + mag * (R)dv.inv_m2 + (R)dv.cre * lr;
          const R sc = pad ? (R)0 : (R)dv.inv_N * prec_recip(sigma);
          v[0][idx] = cscale(v[0][idx], sc);
        }
        rf_inverse<R, L, 1>(v, t, g.twn, lay);
      }
    }
    if (valid) {
      if constexpr (mode == 0) {
#pragma unroll
        for (int idx = 0; idx < 16; ++idx) spec[base + rf_freq<L>(t, idx) * axis_stride] = v[0][idx];
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) spec[base + (t + r * T) * axis_stride] = v[0][r];
      }
    }
    if constexpr (PS) __syncthreads();  // the next block of a persistent CTA reuses the shared rows
  }
};

template <typename R> struct PrecRowsRegArgs {
  const R* r;  // forward: input rows
  R* z;        // inverse: output rows
  cplx<R>* spec;
  long long nrows;
  int H, Hp;
  const cplx<R>* twn;
  Gate gate;
};

template <typename R, int L, int NT> struct PrecRowsFwdRegOp {
  using Args = PrecRowsRegArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    if (gate_closed<PS>(g.gate)) return;
    using C = cplx<R>;
    constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const long long nrows = g.nrows;
    const int H = g.H, Hp = g.Hp;
    const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
    const long long ra = (cx.bid * PAIRS + pr) * 2, rb = ra + 1;
    C* my = sm + pr * LS;
    auto at = [my](int, int pos) -> C& { return my[pos + (pos >> 4)]; };
    const PadLayout<C, LS> lay{my};
    C v[1][16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = t + q * T;
      v[0][q] = mk<C>(ra < nrows ? ldv<PS>(g.r + ra * L + p) : (R)0, rb < nrows ? ldv<PS>(g.r + rb * L + p) : (R)0);
    }
    rf_forward<R, L, 1>(v, t, g.twn, lay);
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
        if (ra < nrows) g.spec[ra * Hp + k] = A;
        if (rb < nrows) g.spec[rb * Hp + k] = B;
      }
    }
    if constexpr (PS) __syncthreads();
  }
};

template <typename R, int L, int NT> struct PrecRowsInvRegOp {
  using Args = PrecRowsRegArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    if (gate_closed<PS>(g.gate)) return;
    using C = cplx<R>;
    constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const long long nrows = g.nrows;
    const int H = g.H, Hp = g.Hp;
    const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
    const long long ra = (cx.bid * PAIRS + pr) * 2, rb = ra + 1;
    C* my = sm + pr * LS;
    const PadLayout<C, LS> lay{my};
    C v[1][16];
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      const int k = rf_freq<L>(t, idx);
      const bool lo = k < H;
      const int kk = lo ? k : L - k;
      C A = ra < nrows ? ldv<PS>(g.spec + ra * Hp + kk) : mk<C>(0, 0);
      C B = rb < nrows ? ldv<PS>(g.spec + rb * Hp + kk) : mk<C>(0, 0);
      if (!lo) {
        A = cconj(A);
        B = cconj(B);
      }
      v[0][idx] = mk<C>(A.x - B.y, A.y + B.x);  // A + i B
    }
    rf_inverse<R, L, 1>(v, t, g.twn, lay);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int p = t + q * T;
      if (ra < nrows) g.z[ra * L + p] = v[0][q].x;
      if (rb < nrows) g.z[rb * L + p] = v[0][q].y;
    }
    if constexpr (PS) __syncthreads();
  }
};

}  // namespace fde
