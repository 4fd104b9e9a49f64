// Launchers of the saddle-point (MINRES) streaming kernels (saddle.cu).
#pragma once
#include "internal.h"

namespace fde {

// q_u = Q z_u + psi z_p and q_p += psi z_u - dr z_p (dr = delta/rho), N entries each.
template <typename R>
cudaError_t saddle_tail(long long n, long long last_start, const double Q[2], double psi, double dr, const R* zu,
                        const R* zp, R* qu, R* qp, cudaStream_t st);
// z[0:n] = r[0:n] / M1, z[n:2n] = r[n:2n] / Q (per-slice values).
template <typename R>
cudaError_t block_diag(long long n, long long last_start, const double M1[2], const double Q[2], const R* r, R* z,
                       cudaStream_t st);
// out = ca a + cb' b + cc c with cb' = cb * dscal[slot] if dscal, else cb (out may alias c).
template <typename R>
cudaError_t lin3(long long n, double ca, const R* a, double cb, const double* dscal, int slot, const R* b, double cc,
                 const R* c, R* out, cudaStream_t st);
// wp = s0 z + s1 wp + s2 w, then x += cx wp.
template <typename R>
cudaError_t minres_wx(long long n, double s0, const R* z, double s1, R* wp, double s2, const R* w, double cx, R* x,
                      cudaStream_t st);
// fu = bu, fp = psi g - dr p (g nullable = 0).
cudaError_t saddle_rhs(long long n, double psi, double dr, const double* bu, const double* g, const double* p,
                       double* fu, double* fp, cudaStream_t st);

}  // namespace fde
