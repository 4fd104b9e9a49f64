// Streaming kernels of the saddle-point sub-problem (Section 3.3.1): the
// diagonal and coupling parts of K, the block-diagonal preconditioner's
// diagonal blocks, and the MINRES vector recurrences. A vector of the 3N
// system is one contiguous array [y | u | p] (N each, layout [t][x1][x2]).
#include "saddle.h"

namespace fde {

namespace {

unsigned grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// K's u row and the rest of its p row, after q_p = B z_y:
//   q_u = Q z_u + psi z_p,   q_p += psi z_u - (delta/rho) z_p.
template <typename R>
__global__ void k_saddle_tail(long long n, long long last_start, double Q0, double Q1, double psi, double dr,
                              const R* __restrict__ zu, const R* __restrict__ zp, R* __restrict__ qu,
                              R* __restrict__ qp) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R Q = (R)(i >= last_start ? Q1 : Q0);
    const R u = zu[i], p = zp[i];
    qu[i] = Q * u + (R)psi * p;
    qp[i] = qp[i] + (R)psi * u - (R)dr * p;
  }
}

// Diagonal blocks of K-tilde^-1: z_y = M1^-1 r_y, z_u = Q^-1 r_u (2N entries).
template <typename R>
__global__ void k_block_diag(long long n, long long last_start, double iM10, double iM11, double iQ0, double iQ1,
                             const R* __restrict__ r, R* __restrict__ z) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 2 * n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool ublk = i >= n;
    const long long j = ublk ? i - n : i;
    const bool last = j >= last_start;
    const double s = ublk ? (last ? iQ1 : iQ0) : (last ? iM11 : iM10);
    z[i] = (R)s * r[i];
  }
}

// out = ca a + cb b + cc c, cb = cb_host * dscal[slot] when dscal != null (out may alias c).
template <typename R>
__global__ void k_lin3(long long n, double ca, const R* a, double cb_host, const double* dscal, int slot, const R* b,
                       double cc, const R* c, R* out) {
  const double cb = dscal ? cb_host * dscal[slot] : cb_host;
  const R fa = (R)ca, fb = (R)cb, fc = (R)cc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = fa * a[i] + fb * b[i] + fc * c[i];
}

// MINRES direction and iterate: w_prev <- s0 z + s1 w_prev + s2 w, x += cx w_prev.
template <typename R>
__global__ void k_minres_wx(long long n, double s0, const R* __restrict__ z, double s1, R* wp, double s2,
                            const R* __restrict__ w, double cx, R* x) {
  const R f0 = (R)s0, f1 = (R)s1, f2 = (R)s2, fx = (R)cx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R wn = f0 * z[i] + f1 * wp[i] + f2 * w[i];
    wp[i] = wn;
    x[i] += fx * wn;
  }
}

// Right-hand side blocks u and p of the merged system: f_u = b_u, f_p = psi g - (delta/rho) p^j.
__global__ void k_saddle_rhs(long long n, double psi, double dr, const double* __restrict__ bu,
                             const double* __restrict__ g, const double* __restrict__ p, double* __restrict__ fu,
                             double* __restrict__ fp) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    fu[i] = bu[i];
    fp[i] = (g ? psi * g[i] : 0.0) - dr * p[i];
  }
}

}  // namespace

template <typename R>
cudaError_t saddle_tail(long long n, long long last_start, const double Q[2], double psi, double dr, const R* zu,
                        const R* zp, R* qu, R* qp, cudaStream_t st) {
  k_saddle_tail<R><<<grid_for(n), 256, 0, st>>>(n, last_start, Q[0], Q[1], psi, dr, zu, zp, qu, qp);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t block_diag(long long n, long long last_start, const double M1[2], const double Q[2], const R* r, R* z,
                       cudaStream_t st) {
  k_block_diag<R><<<grid_for(2 * n), 256, 0, st>>>(n, last_start, 1.0 / M1[0], 1.0 / M1[1], 1.0 / Q[0], 1.0 / Q[1],
                                                   r, z);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t lin3(long long n, double ca, const R* a, double cb, const double* dscal, int slot, const R* b, double cc,
                 const R* c, R* out, cudaStream_t st) {
  k_lin3<R><<<grid_for(n), 256, 0, st>>>(n, ca, a, cb, dscal, slot, b, cc, c, out);
  note_launches(1);
  return cudaGetLastError();
}

template <typename R>
cudaError_t minres_wx(long long n, double s0, const R* z, double s1, R* wp, double s2, const R* w, double cx, R* x,
                      cudaStream_t st) {
  k_minres_wx<R><<<grid_for(n), 256, 0, st>>>(n, s0, z, s1, wp, s2, w, cx, x);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t saddle_rhs(long long n, double psi, double dr, const double* bu, const double* g, const double* p,
                       double* fu, double* fp, cudaStream_t st) {
  k_saddle_rhs<<<grid_for(n), 256, 0, st>>>(n, psi, dr, bu, g, p, fu, fp);
  note_launches(1);
  return cudaGetLastError();
}

#define FDE_SADDLE_INST(R)                                                                                        \
  template cudaError_t saddle_tail<R>(long long, long long, const double*, double, double, const R*, const R*, R*, \
                                      R*, cudaStream_t);                                                          \
  template cudaError_t block_diag<R>(long long, long long, const double*, const double*, const R*, R*,           \
                                     cudaStream_t);                                                               \
  template cudaError_t lin3<R>(long long, double, const R*, double, const double*, int, const R*, double,        \
                               const R*, R*, cudaStream_t);                                                       \
  template cudaError_t minres_wx<R>(long long, double, const R*, double, R*, double, const R*, double, R*,       \
                                    cudaStream_t);
FDE_SADDLE_INST(float)
FDE_SADDLE_INST(double)
#undef FDE_SADDLE_INST

}  // namespace fde
