// Bodies of the streaming vector kernels (vec.cu): deterministic reductions
// (per-block tree, then a one-block fixed-order tree), the fused PCG updates,
// the refinement conversions and the ADMM clip-and-update step (Algorithm 1
// steps for z, p and w with the psi scaling of Section 6.1).
#pragma once
#include <cmath>

#include "internal.h"
#include "ops_list.cuh"
#include "vec.h"

namespace fde {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  return v;
}

// Block maximum of non-negative values held as their bit patterns: for
// non-negative doubles the integer order is the numeric order, and infinities
// and NaNs (exponent all ones) compare above every finite value.
__device__ __forceinline__ long long block_max_bits(long long v, long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  return v;
}

__device__ __forceinline__ long long abs_bits(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// Per-thread accumulator: double for double data; for float data a
// compensated (Kahan) float sum, converted to double once per thread, so that
// no element pays a float->double conversion (the double pipe runs at 1/58 of
// the float rate on this GPU) while the sum keeps close to double accuracy.
template <typename R> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// first element and stride of the grid-stride loop of block c.bid
__device__ __forceinline__ long long gs_first(const Ctx& c) { return c.bid * (long long)blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gs_step(const Ctx& c) { return c.nblk * (long long)blockDim.x; }

// partials[b] = sum over the grid-stride share of block b of a[i]*b[i]
template <typename RA, typename RB> struct DotArgs {
  const RA* a;
  const RB* b;
  long long n;
  double* partials;
};
template <typename RA, typename RB> struct DotOp {
  using Args = DotArgs<RA, RB>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    __shared__ double sh[32];
    Acc<RA> acc;
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) acc.add(ldv<PS>(p.a + i) * ldv<PS>(p.b + i));
    const double s = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) p.partials[c.bid] = s;
  }
};

// Sum the partials in a fixed order and derive PCG scalars.
//   op FIN_STORE: dscal[slot] = sum
//   op FIN_ALPHA: dscal[S_PQ] = sum; alpha = rz / sum (flag breakdown if sum <= 0)
//   op FIN_BETA : beta = sum / rz; rz = sum
// (the masked forms of the host-sync-free solve are listed with enum FinishOp in vec.h)
struct FinishArgs {
  const double* partials;
  int np;
  double* dscal;
  int slot, op;
  double aux;
};
struct FinishSumOp {
  using Args = FinishArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx&, const Args& p) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < p.np; i += blockDim.x) s += ldv<PS>(p.partials + i);
    s = block_sum(s, sh);
    if (threadIdx.x != 0) return;
    double* dscal = p.dscal;
    auto rd = [&](int k) { return ldv<PS>(dscal + k); };
    if (!isfinite(s)) dscal[S_FLAG] = (double)FDE_ENONFINITE;
    if (p.op == FIN_STORE) {
      dscal[p.slot] = s;
    } else if (p.op == FIN_ALPHA) {
      dscal[S_PQ] = s;
      if (!(s > 0.0)) {
        dscal[S_FLAG] = (double)FDE_EBREAKDOWN;
        dscal[S_ALPHA] = 0.0;
      } else {
        dscal[S_ALPHA] = rd(S_RZ) / s;
      }
    } else if (p.op == FIN_BETA) {
      const double rz = rd(S_RZ);
      dscal[S_BETA] = rz != 0.0 ? s / rz : 0.0;
      dscal[S_RZ] = s;
    } else if (p.op == FIN_RZ0) {
      dscal[S_RZ] = s;
    } else if (p.op == FIN_BB_THR) {
      dscal[S_BB] = s;
      dscal[S_THR] = p.aux * p.aux * s;
    } else if (p.op == FIN_ALPHA_MASK) {
      dscal[S_PQ] = s;
      const bool active = rd(S_RR) > rd(S_THR) && s > 0.0 && isfinite(s);
      dscal[S_ALPHA] = active ? rd(S_RZ) / s : 0.0;
      if (active) dscal[S_PCGIT] = rd(S_PCGIT) + 1.0;
    } else if (p.op == FIN_BETA_MASK) {
      const double rz = rd(S_RZ);
      const bool active = rd(S_RR) > rd(S_THR) && rz != 0.0;
      dscal[S_BETA] = active ? s / rz : 0.0;
      dscal[S_RZ] = s;
    } else if (p.op == FIN_REFCHK) {
      dscal[S_RR] = s;
      const double bb = rd(S_TMP0);
      const double rel = bb > 0.0 ? sqrt(s / bb) : 0.0;
      dscal[S_RELRES] = rel;
      dscal[S_CONV] = (rel <= p.aux) ? 1.0 : 0.0;
    }
  }
};

// x += alpha d; r -= alpha q; partials of r.r (arithmetic in the vectors' type)
template <typename RV> struct PcgXrArgs {
  RV *x, *r;
  const RV *d, *q;
  const double* dscal;
  long long n;
  double* partials;
};
template <typename RV> struct PcgXrOp {
  using Args = PcgXrArgs<RV>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    __shared__ double sh[32];
    const RV alpha = (RV)ldv<PS>(p.dscal + S_ALPHA);
    Acc<RV> acc;
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) {
      p.x[i] = ldv<PS>(p.x + i) + alpha * ldv<PS>(p.d + i);
      const RV ri = ldv<PS>(p.r + i) - alpha * ldv<PS>(p.q + i);
      p.r[i] = ri;
      acc.add(ri * ri);
    }
    const double s = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) p.partials[c.bid] = s;
  }
};

// d = z + beta d
template <typename RV> struct PcgPArgs {
  RV* d;
  const RV* z;
  const double* dscal;
  long long n;
};
template <typename RV> struct PcgPOp {
  using Args = PcgPArgs<RV>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    const RV beta = (RV)ldv<PS>(p.dscal + S_BETA);
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.d[i] = ldv<PS>(p.z + i) + beta * ldv<PS>(p.d + i);
  }
};

// out32 = (float) in64
struct ToF32Args {
  const double* in;
  float* out;
  long long n;
};
struct ToF32Op {
  using Args = ToF32Args;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.out[i] = (float)ldv<PS>(p.in + i);
  }
};

// out32 = conv ? 0 : (float) in64 (conv read from the device)
struct ToF32UnlessArgs {
  const double* in;
  float* out;
  long long n;
  const double* dscal;
};
struct ToF32UnlessOp {
  using Args = ToF32UnlessArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    const bool conv = ldv<PS>(p.dscal + S_CONV) != 0.0;
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.out[i] = conv ? 0.f : (float)ldv<PS>(p.in + i);
  }
};

// y64 += (double) d32 unless conv
struct AddF32UnlessArgs {
  double* y;
  const float* d;
  long long n;
  const double* dscal;
};
struct AddF32UnlessOp {
  using Args = AddF32UnlessArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    if (ldv<PS>(p.dscal + S_CONV) != 0.0) return;
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.y[i] = ldv<PS>(p.y + i) + (double)ldv<PS>(p.d + i);
  }
};

// op 0: dscal[dst] = max(dscal[dst], dscal[src]); op 1: count an applied correction
// (thread 0 of block 0 only, whatever the launch shape)
struct ScalarStepArgs {
  double* dscal;
  int dst, src, op;
};
struct ScalarStepOp {
  using Args = ScalarStepArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    if (threadIdx.x != 0 || c.bid != 0) return;
    double* d = p.dscal;
    if (p.op == 0) d[p.dst] = fmax(ldv<PS>(d + p.dst), ldv<PS>(d + p.src));
    else if (p.op == 1 && ldv<PS>(d + S_CONV) == 0.0) d[S_REFINE] = ldv<PS>(d + S_REFINE) + 1.0;
  }
};

template <typename R> struct FillArgs {
  R* x;
  R v;
  long long n;
};
template <typename R> struct FillOp {
  using Args = FillArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.x[i] = p.v;
  }
};

template <typename R> struct CopyArgs {
  R* dst;
  const R* src;
  long long n;
};
template <typename R> struct CopyOp {
  using Args = CopyArgs<R>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& c, const Args& p) {
    for (long long i = gs_first(c); i < p.n; i += gs_step(c)) p.dst[i] = ldv<PS>(p.src + i);
  }
};

// ---------------------------------------------------------------------------
// ADMM (Algorithm 1, psi-scaled, sub-problem merged with the p update).
// Slice-constant diagonals (index 0: slices 0..nt-2, 1: last slice):
//   M1 = rho (w + 1/delta), Q = rho (gamma w + psi^2/delta), M2 = psi^2/Q + delta/rho.
// Pre-step, from (z_y, z_u, p, w_y, w_u):
//   c   = rho (w ybar - w_y + z_y/delta)
//   b_u = rho (-psi w_u + psi^2 z_u/delta) + (1-rho) psi p
//   r0  = psi b_u / Q - psi g + (delta/rho) p
//   q   = (1-rho) p - r0 / M2
// and then rhs = c + B^T q is the right-hand side of S y = rhs.
// ---------------------------------------------------------------------------
struct AdmmPreArgs {
  AdmmArgs A;
  double *c, *bu, *r0, *q;
};
struct AdmmPreOp {
  using Args = AdmmPreArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& a) {
    const AdmmArgs& A = a.A;
    // Coefficients folded once per thread: on this GPU the double pipe, not memory,
    // bounds these streaming steps, so each element costs fused multiply-adds only
    // (reciprocals instead of divides).
    const double cyb[2] = {A.rho * A.w[0], A.rho * A.w[1]};
    const double rod = A.rho * A.inv_delta;
    const double k1 = -A.rho * A.psi, k2 = A.rho * A.psi * A.psi * A.inv_delta, k3 = (1.0 - A.rho) * A.psi;
    const double k4[2] = {A.psi * A.inv_Q[0], A.psi * A.inv_Q[1]};
    const double omr = 1.0 - A.rho;
    for (long long i = gs_first(cx); i < A.n; i += gs_step(cx)) {
      const int last = (i >= A.last_start);
      const double p = ldv<PS>(A.p + i);
      // c = rho (w ybar - w_y + z_y / delta), b_u = rho (-psi w_u + psi^2 z_u / delta) + (1 - rho) psi p
      double cy = fma(cyb[last], ldv<PS>(A.ybar + i), fma(-A.rho, ldv<PS>(A.wy + i), rod * ldv<PS>(A.zy + i)));
      double b = fma(k1, ldv<PS>(A.wu + i), fma(k2, ldv<PS>(A.zu + i), k3 * p));
      if (A.gen) {  // proximal pulls towards the previous iterate (Algorithm 2)
        cy = fma(A.ry[last], ldv<PS>(A.yprev + i), cy);
        b = fma(A.ru[last], ldv<PS>(A.uprev + i), b);
      }
      a.c[i] = cy;
      a.bu[i] = b;
      // r0 = psi Q^-1 b_u - psi g + (delta/rho) p,  q = (1 - rho) p - M2^-1 r0
      double r = A.delta_over_rho * p;
      if (A.g) r = fma(-A.psi, ldv<PS>(A.g + i), r);
      r = fma(k4[last], b, r);
      a.r0[i] = r;
      a.q[i] = fma(-A.inv_M2[last], r, omr * p);
    }
  }
};

// Post-step, given y and By:
//   p   = (By + r0) / M2,  u = (b_u - psi p) / Q,
//   z_y = clip(y + delta w_y, ya, yb),  z_u = clip(u + delta w_u / psi, ua, ub),
//   w_y += (rho/delta)(y - z_y),  w_u += (rho/delta) psi (u - z_u),
// and block maxima of |By + psi (u - g)|, |y - z_y|, |u - z_u| plus block sums
// of the objective terms w (y - ybar)^2 and gamma w u^2.
struct AdmmPostArgs {
  AdmmArgs A;
  const double *y, *By, *bu, *r0;
  double* u;
  double* partials;
  int np;
};
struct AdmmPostOp {
  using Args = AdmmPostArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& a) {
    __shared__ double sh[32];
    __shared__ long long shl[32];
    const AdmmArgs& A = a.A;
    // residual maxima on bit patterns (integer pipe); non-finite values show up as
    // maxima with an all-ones exponent; the objective's two sums per weight class
    long long m_eq = 0, m_y = 0, m_u = 0;
    double oy = 0.0, ou = 0.0, oyl = 0.0, oul = 0.0;
    const double rpsi = A.rho_over_delta * A.psi;
    const double piq[2] = {A.psi * A.inv_Q[0], A.psi * A.inv_Q[1]};
    for (long long i = gs_first(cx); i < A.n; i += gs_step(cx)) {
      const int last = (i >= A.last_start);
      const double iM2 = A.inv_M2[last];
      const double yi = ldv<PS>(a.y + i), byi = ldv<PS>(a.By + i);
      const double p = A.given_up ? ldv<PS>(A.p + i) : iM2 * (byi + ldv<PS>(a.r0 + i));
      const double ui = A.given_up ? ldv<PS>(a.u + i) : fma(-piq[last], p, A.inv_Q[last] * ldv<PS>(a.bu + i));
      const double lo_y = A.ya ? ldv<PS>(A.ya + i) : A.ya_s, hi_y = A.yb ? ldv<PS>(A.yb + i) : A.yb_s;
      const double lo_u = A.ua ? ldv<PS>(A.ua + i) : A.ua_s, hi_u = A.ub ? ldv<PS>(A.ub + i) : A.ub_s;
      const double wy = ldv<PS>(A.wy + i), wu = ldv<PS>(A.wu + i);
      const double zy = fmin(fmax(fma(A.delta, wy, yi), lo_y), hi_y);
      const double zu = fmin(fmax(fma(A.delta_over_psi, wu, ui), lo_u), hi_u);
      const double dy = yi - zy, du = ui - zu;
      A.wy[i] = fma(A.rho_over_delta, dy, wy);
      A.wu[i] = fma(rpsi, du, wu);
      A.zy[i] = zy;
      A.zu[i] = zu;
      A.p[i] = p;
      a.u[i] = ui;
      const double e = A.g ? fma(A.psi, ui - ldv<PS>(A.g + i), byi) : fma(A.psi, ui, byi);
      m_eq = max(m_eq, abs_bits(e));
      m_y = max(m_y, abs_bits(dy));
      m_u = max(m_u, abs_bits(du));
      const double dd = yi - ldv<PS>(A.ybar + i);
      if (last) {
        oyl = fma(dd, dd, oyl);
        oul = fma(ui, ui, oul);
      } else {
        oy = fma(dd, dd, oy);
        ou = fma(ui, ui, ou);
      }
    }
    // objective 1/2 (y - ybar)^T J1 (y - ybar) + 1/2 u^T J2 u with J1 = diag(w), J2 = gamma J1
    double obj = 0.5 * (A.w[0] * fma(A.gamma, ou, oy) + A.w[1] * fma(A.gamma, oul, oyl));
    m_eq = block_max_bits(m_eq, shl);
    m_y = block_max_bits(m_y, shl);
    m_u = block_max_bits(m_u, shl);
    obj = block_sum(obj, sh);
    if (threadIdx.x == 0) {
      const long long inf_bits = 0x7ff0000000000000LL;
      const bool bad = m_eq >= inf_bits || m_y >= inf_bits || m_u >= inf_bits || !isfinite(obj);
      const int np = a.np;
      const long long b = cx.bid;
      a.partials[b] = bad ? 0.0 : __longlong_as_double(m_eq);
      a.partials[np + b] = bad ? 0.0 : __longlong_as_double(m_y);
      a.partials[2 * np + b] = bad ? 0.0 : __longlong_as_double(m_u);
      a.partials[3 * np + b] = obj;
      a.partials[4 * np + b] = bad ? 1.0 : 0.0;
    }
  }
};

struct AdmmFinishArgs {
  const double* partials;
  int np;
  double* dscal;
};
struct AdmmFinishOp {
  using Args = AdmmFinishArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx&, const Args& p) {
    __shared__ double sh[32];
    double a = 0.0, b = 0.0, c = 0.0, o = 0.0, f = 0.0;
    const int np = p.np;
    for (int i = threadIdx.x; i < np; i += blockDim.x) {
      a = fmax(a, ldv<PS>(p.partials + i));
      b = fmax(b, ldv<PS>(p.partials + np + i));
      c = fmax(c, ldv<PS>(p.partials + 2 * np + i));
      o += ldv<PS>(p.partials + 3 * np + i);
      f = fmax(f, ldv<PS>(p.partials + 4 * np + i));
    }
    a = block_max(a, sh);
    b = block_max(b, sh);
    c = block_max(c, sh);
    o = block_sum(o, sh);
    f = block_max(f, sh);
    if (threadIdx.x == 0) {
      p.dscal[S_RES_EQ] = a;
      p.dscal[S_RES_Y] = b;
      p.dscal[S_RES_U] = c;
      p.dscal[S_OBJ] = o;
      if (f > 0.0) p.dscal[S_FLAG] = (double)FDE_ENONFINITE;
    }
  }
};

// Folded sub-problem residual, first half: with t = B y,
//   v = q - M2^-1 t,  w = c - M1 y,
// so that rhs - S y = (c + B^T q) - (M1 y + B^T M2^-1 B y) = w + B^T v.
struct FoldArgs {
  const double *t, *q, *c, *y;
  double m2inv0, m2inv1, m10, m11;
  long long last_start, n;
  double *v, *w;
};
struct FoldOp {
  using Args = FoldArgs;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& a) {
    for (long long i = gs_first(cx); i < a.n; i += gs_step(cx)) {
      const bool last = i >= a.last_start;
      a.v[i] = ldv<PS>(a.q + i) - (last ? a.m2inv1 : a.m2inv0) * ldv<PS>(a.t + i);
      a.w[i] = ldv<PS>(a.c + i) - (last ? a.m11 : a.m10) * ldv<PS>(a.y + i);
    }
  }
};

}  // namespace fde
