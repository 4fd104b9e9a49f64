// Streaming vector kernels: deterministic reductions (fixed grid, per-block
// tree, then a one-block fixed-order tree), the fused PCG updates, the
// refinement conversions and the ADMM clip-and-update step (Algorithm 1 steps
// for z, p and w with the psi scaling of Section 6.1).
#include <cmath>

#include "internal.h"
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

int red_grid(long long n) {
  long long g = (n + 4LL * kRedThreads - 1) / (4LL * kRedThreads);
  if (g < 1) g = 1;
  if (g > kMaxPartials) g = kMaxPartials;
  return (int)g;
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

// partials[b] = sum over the grid-stride share of block b of a[i]*b[i]
template <typename RA, typename RB>
__global__ void __launch_bounds__(kRedThreads) k_dot(const RA* __restrict__ a, const RB* __restrict__ b, long long n,
                                                      double* __restrict__ partials) {
  __shared__ double sh[32];
  Acc<RA> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc.add(a[i] * b[i]);
  double s = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Sum the partials in a fixed order and derive PCG scalars.
//   op FIN_STORE: dscal[slot] = sum
//   op FIN_ALPHA: dscal[S_PQ] = sum; alpha = rz / sum (flag breakdown if sum <= 0)
//   op FIN_BETA : beta = sum / rz; rz = sum
__global__ void __launch_bounds__(1024) k_finish(const double* __restrict__ partials, int np, double* dscal, int slot,
                                                  int op, double aux) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += partials[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    if (!isfinite(s)) dscal[S_FLAG] = (double)FDE_ENONFINITE;
    if (op == FIN_STORE) {
      dscal[slot] = s;
    } else if (op == FIN_ALPHA) {
      dscal[S_PQ] = s;
      if (!(s > 0.0)) {
        dscal[S_FLAG] = (double)FDE_EBREAKDOWN;
        dscal[S_ALPHA] = 0.0;
      } else {
        dscal[S_ALPHA] = dscal[S_RZ] / s;
      }
    } else if (op == FIN_BETA) {
      const double rz = dscal[S_RZ];
      dscal[S_BETA] = rz != 0.0 ? s / rz : 0.0;
      dscal[S_RZ] = s;
    } else if (op == FIN_RZ0) {
      dscal[S_RZ] = s;
    } else if (op == FIN_BB_THR) {
      dscal[S_BB] = s;
      dscal[S_THR] = aux * aux * s;
    } else if (op == FIN_ALPHA_MASK) {
      dscal[S_PQ] = s;
      const bool active = dscal[S_RR] > dscal[S_THR] && s > 0.0 && isfinite(s);
      dscal[S_ALPHA] = active ? dscal[S_RZ] / s : 0.0;
      if (active) dscal[S_PCGIT] += 1.0;
    } else if (op == FIN_BETA_MASK) {
      const double rz = dscal[S_RZ];
      const bool active = dscal[S_RR] > dscal[S_THR] && rz != 0.0;
      dscal[S_BETA] = active ? s / rz : 0.0;
      dscal[S_RZ] = s;
    } else if (op == FIN_REFCHK) {
      dscal[S_RR] = s;
      const double bb = dscal[S_TMP0];
      const double rel = bb > 0.0 ? sqrt(s / bb) : 0.0;
      dscal[S_RELRES] = rel;
      dscal[S_CONV] = (rel <= aux) ? 1.0 : 0.0;
    }
  }
}

// x += alpha d; r -= alpha q; partials of r.r (arithmetic in the vectors' type)
template <typename RV>
__global__ void __launch_bounds__(kRedThreads) k_pcg_xr(RV* __restrict__ x, RV* __restrict__ r, const RV* __restrict__ d,
                                                         const RV* __restrict__ q, const double* __restrict__ dscal,
                                                         long long n, double* __restrict__ partials) {
  __shared__ double sh[32];
  const RV alpha = (RV)dscal[S_ALPHA];
  Acc<RV> acc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = x[i] + alpha * d[i];
    const RV ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc.add(ri * ri);
  }
  const double s = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// d = z + beta d
template <typename RV>
__global__ void k_pcg_p(RV* __restrict__ d, const RV* __restrict__ z, const double* __restrict__ dscal, long long n) {
  const RV beta = (RV)dscal[S_BETA];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d[i] = z[i] + beta * d[i];
}

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

// out32 = (float) in64
__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// out32 = conv ? 0 : (float) in64 (conv read from the device)
__global__ void k_to_f32_unless(const double* __restrict__ in, float* __restrict__ out, long long n,
                                const double* __restrict__ dscal) {
  const bool conv = dscal[S_CONV] != 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = conv ? 0.f : (float)in[i];
}

// y64 += (double) d32 unless conv; block 0 counts the applied correction
__global__ void k_add_f32_unless(double* __restrict__ y, const float* __restrict__ d, long long n,
                                 double* __restrict__ dscal) {
  const bool conv = dscal[S_CONV] != 0.0;
  if (conv) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += (double)d[i];
}

__global__ void k_scalar_step(double* dscal, int dst, int src, int op) {
  if (op == 0) dscal[dst] = fmax(dscal[dst], dscal[src]);
  else if (op == 1 && dscal[S_CONV] == 0.0) dscal[S_REFINE] += 1.0;
}

// y64 += (double) d32
__global__ void k_add_f32(double* __restrict__ y, const float* __restrict__ d, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += (double)d[i];
}

template <typename R>
__global__ void k_fill(R* __restrict__ x, R v, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = v;
}

template <typename R>
__global__ void k_copy(R* __restrict__ dst, const R* __restrict__ src, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

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
__global__ void k_admm_pre(const AdmmArgs A, double* __restrict__ c, double* __restrict__ bu, double* __restrict__ r0,
                           double* __restrict__ q) {
  // Coefficients folded once per thread: on this GPU the double pipe, not memory,
  // bounds these streaming steps, so each element costs fused multiply-adds only
  // (reciprocals instead of divides).
  const double cyb[2] = {A.rho * A.w[0], A.rho * A.w[1]};
  const double rod = A.rho * A.inv_delta;
  const double k1 = -A.rho * A.psi, k2 = A.rho * A.psi * A.psi * A.inv_delta, k3 = (1.0 - A.rho) * A.psi;
  const double k4[2] = {A.psi * A.inv_Q[0], A.psi * A.inv_Q[1]};
  const double omr = 1.0 - A.rho;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.n; i += (long long)gridDim.x * blockDim.x) {
    const int last = (i >= A.last_start);
    const double p = A.p[i];
    // c = rho (w ybar - w_y + z_y / delta), b_u = rho (-psi w_u + psi^2 z_u / delta) + (1 - rho) psi p
    double cy = fma(cyb[last], A.ybar[i], fma(-A.rho, A.wy[i], rod * A.zy[i]));
    double b = fma(k1, A.wu[i], fma(k2, A.zu[i], k3 * p));
    if (A.gen) {  // proximal pulls towards the previous iterate (Algorithm 2)
      cy = fma(A.ry[last], A.yprev[i], cy);
      b = fma(A.ru[last], A.uprev[i], b);
    }
    c[i] = cy;
    bu[i] = b;
    // r0 = psi Q^-1 b_u - psi g + (delta/rho) p,  q = (1 - rho) p - M2^-1 r0
    double r = A.delta_over_rho * p;
    if (A.g) r = fma(-A.psi, A.g[i], r);
    r = fma(k4[last], b, r);
    r0[i] = r;
    q[i] = fma(-A.inv_M2[last], r, omr * p);
  }
}

// Post-step, given y and By:
//   p   = (By + r0) / M2,  u = (b_u - psi p) / Q,
//   z_y = clip(y + delta w_y, ya, yb),  z_u = clip(u + delta w_u / psi, ua, ub),
//   w_y += (rho/delta)(y - z_y),  w_u += (rho/delta) psi (u - z_u),
// and block maxima of |By + psi (u - g)|, |y - z_y|, |u - z_u| plus block sums
// of the objective terms w (y - ybar)^2 and gamma w u^2.
__global__ void __launch_bounds__(kRedThreads) k_admm_post(const AdmmArgs A, const double* __restrict__ y,
                                                            const double* __restrict__ By,
                                                            const double* __restrict__ bu,
                                                            const double* __restrict__ r0, double* __restrict__ u,
                                                            double* __restrict__ partials, int np) {
  __shared__ double sh[32];
  __shared__ long long shl[32];
  // residual maxima on bit patterns (integer pipe); non-finite values show up as
  // maxima with an all-ones exponent; the objective's two sums per weight class
  long long m_eq = 0, m_y = 0, m_u = 0;
  double oy = 0.0, ou = 0.0, oyl = 0.0, oul = 0.0;
  const double rpsi = A.rho_over_delta * A.psi;
  const double piq[2] = {A.psi * A.inv_Q[0], A.psi * A.inv_Q[1]};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.n; i += (long long)gridDim.x * blockDim.x) {
    const int last = (i >= A.last_start);
    const double iM2 = A.inv_M2[last];
    const double yi = y[i], byi = By[i];
    const double p = A.given_up ? A.p[i] : iM2 * (byi + r0[i]);
    const double ui = A.given_up ? u[i] : fma(-piq[last], p, A.inv_Q[last] * bu[i]);
    const double lo_y = A.ya ? A.ya[i] : A.ya_s, hi_y = A.yb ? A.yb[i] : A.yb_s;
    const double lo_u = A.ua ? A.ua[i] : A.ua_s, hi_u = A.ub ? A.ub[i] : A.ub_s;
    const double zy = fmin(fmax(fma(A.delta, A.wy[i], yi), lo_y), hi_y);
    const double zu = fmin(fmax(fma(A.delta_over_psi, A.wu[i], ui), lo_u), hi_u);
    const double dy = yi - zy, du = ui - zu;
    A.wy[i] = fma(A.rho_over_delta, dy, A.wy[i]);
    A.wu[i] = fma(rpsi, du, A.wu[i]);
    A.zy[i] = zy;
    A.zu[i] = zu;
    A.p[i] = p;
    u[i] = ui;
    const double e = A.g ? fma(A.psi, ui - A.g[i], byi) : fma(A.psi, ui, byi);
    m_eq = max(m_eq, abs_bits(e));
    m_y = max(m_y, abs_bits(dy));
    m_u = max(m_u, abs_bits(du));
    const double dd = yi - A.ybar[i];
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
    partials[blockIdx.x] = bad ? 0.0 : __longlong_as_double(m_eq);
    partials[np + blockIdx.x] = bad ? 0.0 : __longlong_as_double(m_y);
    partials[2 * np + blockIdx.x] = bad ? 0.0 : __longlong_as_double(m_u);
    partials[3 * np + blockIdx.x] = obj;
    partials[4 * np + blockIdx.x] = bad ? 1.0 : 0.0;
  }
}

__global__ void __launch_bounds__(1024) k_admm_finish(const double* __restrict__ partials, int np, double* dscal) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0, c = 0.0, o = 0.0, f = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    a = fmax(a, partials[i]);
    b = fmax(b, partials[np + i]);
    c = fmax(c, partials[2 * np + i]);
    o += partials[3 * np + i];
    f = fmax(f, partials[4 * np + i]);
  }
  a = block_max(a, sh);
  b = block_max(b, sh);
  c = block_max(c, sh);
  o = block_sum(o, sh);
  f = block_max(f, sh);
  if (threadIdx.x == 0) {
    dscal[S_RES_EQ] = a;
    dscal[S_RES_Y] = b;
    dscal[S_RES_U] = c;
    dscal[S_OBJ] = o;
    if (f > 0.0) dscal[S_FLAG] = (double)FDE_ENONFINITE;
  }
}

// Folded sub-problem residual, first half: with t = B y,
//   v = q - M2^-1 t,  w = c - M1 y,
// so that rhs - S y = (c + B^T q) - (M1 y + B^T M2^-1 B y) = w + B^T v.
__global__ void k_fold(const double* __restrict__ t, const double* __restrict__ q, const double* __restrict__ c,
                       const double* __restrict__ y, double m2inv0, double m2inv1, double m10, double m11,
                       long long last_start, long long n, double* __restrict__ v, double* __restrict__ w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const bool last = i >= last_start;
    v[i] = q[i] - (last ? m2inv1 : m2inv0) * t[i];
    w[i] = c[i] - (last ? m11 : m10) * y[i];
  }
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

template <typename RA, typename RB>
cudaError_t dot(fde_problem* P, const RA* a, const RB* b, long long n, int slot, int op, cudaStream_t st,
                double aux) {
  const int g = red_grid(n);
  k_dot<RA, RB><<<g, kRedThreads, 0, st>>>(a, b, n, P->partials);
  note_launches(1);
  k_finish<<<1, 1024, 0, st>>>(P->partials, g, P->dscal, slot, op, aux);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t dot<double, double>(fde_problem*, const double*, const double*, long long, int, int, cudaStream_t,
                                         double);
template cudaError_t dot<float, float>(fde_problem*, const float*, const float*, long long, int, int, cudaStream_t,
                                       double);

template <typename RV>
cudaError_t pcg_xr(fde_problem* P, RV* x, RV* r, const RV* d, const RV* q, long long n, cudaStream_t st) {
  const int g = red_grid(n);
  k_pcg_xr<RV><<<g, kRedThreads, 0, st>>>(x, r, d, q, P->dscal, n, P->partials);
  note_launches(1);
  k_finish<<<1, 1024, 0, st>>>(P->partials, g, P->dscal, S_RR, FIN_STORE, 0.0);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t pcg_xr<double>(fde_problem*, double*, double*, const double*, const double*, long long,
                                    cudaStream_t);
template cudaError_t pcg_xr<float>(fde_problem*, float*, float*, const float*, const float*, long long, cudaStream_t);

template <typename RV>
cudaError_t pcg_p(fde_problem* P, RV* d, const RV* z, long long n, cudaStream_t st) {
  k_pcg_p<RV><<<sgrid(n), 256, 0, st>>>(d, z, P->dscal, n);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t pcg_p<double>(fde_problem*, double*, const double*, long long, cudaStream_t);
template cudaError_t pcg_p<float>(fde_problem*, float*, const float*, long long, cudaStream_t);

cudaError_t residual(fde_problem* P, const double* b, const double* s, double* r, long long n, int slot,
                     cudaStream_t st) {
  const int g = red_grid(n);
  k_residual<<<g, kRedThreads, 0, st>>>(b, s, r, n, P->partials);
  note_launches(1);
  k_finish<<<1, 1024, 0, st>>>(P->partials, g, P->dscal, slot, FIN_STORE, 0.0);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t to_f32(const double* in, float* out, long long n, cudaStream_t st) {
  k_to_f32<<<sgrid(n), 256, 0, st>>>(in, out, n);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t to_f32_unless_conv(fde_problem* P, const double* in, float* out, long long n, cudaStream_t st) {
  k_to_f32_unless<<<sgrid(n), 256, 0, st>>>(in, out, n, P->dscal);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t add_f32_unless_conv(fde_problem* P, double* y, const float* d, long long n, cudaStream_t st) {
  k_scalar_step<<<1, 1, 0, st>>>(P->dscal, 0, 0, 1);
  note_launches(1);
  k_add_f32_unless<<<sgrid(n), 256, 0, st>>>(y, d, n, P->dscal);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t scalar_max(fde_problem* P, int dst, int src, cudaStream_t st) {
  k_scalar_step<<<1, 1, 0, st>>>(P->dscal, dst, src, 0);
  note_launches(1);
  return cudaGetLastError();
}
cudaError_t add_f32(double* y, const float* d, long long n, cudaStream_t st) {
  k_add_f32<<<sgrid(n), 256, 0, st>>>(y, d, n);
  note_launches(1);
  return cudaGetLastError();
}
template <typename R>
cudaError_t fill(R* x, R v, long long n, cudaStream_t st) {
  k_fill<R><<<sgrid(n), 256, 0, st>>>(x, v, n);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t fill<double>(double*, double, long long, cudaStream_t);
template cudaError_t fill<float>(float*, float, long long, cudaStream_t);
template <typename R>
cudaError_t copy(R* dst, const R* src, long long n, cudaStream_t st) {
  k_copy<R><<<sgrid(n), 256, 0, st>>>(dst, src, n);
  note_launches(1);
  return cudaGetLastError();
}
template cudaError_t copy<double>(double*, const double*, long long, cudaStream_t);
template cudaError_t copy<float>(float*, const float*, long long, cudaStream_t);

cudaError_t admm_pre(const AdmmArgs& A, double* c, double* bu, double* r0, double* q, cudaStream_t st) {
  k_admm_pre<<<sgrid(A.n), 256, 0, st>>>(A, c, bu, r0, q);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t admm_post(fde_problem* P, const AdmmArgs& A, const double* y, const double* By, const double* bu,
                      const double* r0, double* u, cudaStream_t st) {
  int g = red_grid(A.n);
  if (g > kMaxPartials / 5) g = kMaxPartials / 5;
  k_admm_post<<<g, kRedThreads, 0, st>>>(A, y, By, bu, r0, u, P->partials, g);
  note_launches(1);
  k_admm_finish<<<1, 1024, 0, st>>>(P->partials, g, P->dscal);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t fold(const double* t, const double* q, const double* c, const double* y, const double m2inv[2],
                 const double m1[2], long long last_start, long long n, double* v, double* w, cudaStream_t st) {
  k_fold<<<sgrid(n), 256, 0, st>>>(t, q, c, y, m2inv[0], m2inv[1], m1[0], m1[1], last_start, n, v, w);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t grad_ybar(const double* y, const double* ybar, const double* wy, double w0, double w1, long long last_start,
                      long long n, double* dJ, double* f, cudaStream_t st) {
  k_grad_ybar<<<sgrid(n), 256, 0, st>>>(y, ybar, wy, w0, w1, last_start, n, dJ, f);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace fde
