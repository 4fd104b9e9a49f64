// Declarations of the streaming vector kernels' launchers (vec.cu).
#pragma once
#include "internal.h"

namespace fde {

constexpr int kMaxPartials = 4096;  // capacity of fde_problem::partials (doubles)

enum FinishOp {
  FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_RZ0 = 3,
  // masked forms for the host-sync-free solve (aux = tolerance where used)
  FIN_BB_THR = 4,      // S_BB = s, S_THR = aux^2 s
  FIN_ALPHA_MASK = 5,  // S_PQ = s; alpha = rz/s while S_RR > S_THR (counts S_PCGIT), else 0
  FIN_BETA_MASK = 6,   // beta = s/rz while S_RR > S_THR, else 0; rz = s
  FIN_REFCHK = 7       // S_RR = s; S_RELRES = sqrt(s/S_TMP0); S_CONV = (S_RELRES <= aux)
};

// Arguments of the ADMM pre/post kernels. Arrays are device pointers of length n;
// nullable bound arrays fall back to the matching scalar.
struct AdmmArgs {
  long long n, last_start;           // last_start = (nt-1)*nx*ny: first index of the last slice
  double rho, delta, inv_delta, rho_over_delta, delta_over_rho, psi, gamma;
  double w[2], Q[2], M2[2];          // slice-constant diagonals (0: slices < nt-1, 1: last slice)
  double inv_Q[2], inv_M2[2], delta_over_psi;
  const double* ybar;
  const double* g;                   // nullable
  const double *ya, *yb, *ua, *ub;   // nullable
  double ya_s, yb_s, ua_s, ub_s;
  double *zy, *zu, *p, *wy, *wu;     // state, updated in place
  // Algorithm 2: b_y += ry * y^j, b_u += ru * u^j (rho R_y, rho R_u per slice); gen = 0: Algorithm 1
  int gen;
  double ry[2], ru[2];
  const double *yprev, *uprev;
  // 1: the post-step reads p (in p) and u (in u) from a joint (y, u, p) solve
  // instead of pivoting them from B y
  int given_up;
};

int red_grid(long long n);

// out slot: dscal[slot] (op FIN_STORE) or the PCG scalars (FIN_ALPHA / FIN_BETA / FIN_RZ0)
template <typename RA, typename RB>
cudaError_t dot(fde_problem* P, const RA* a, const RB* b, long long n, int slot, int op, cudaStream_t st,
                double aux = 0.0);
template <typename RV>
cudaError_t pcg_xr(fde_problem* P, RV* x, RV* r, const RV* d, const RV* q, long long n, cudaStream_t st);
template <typename RV>
cudaError_t pcg_p(fde_problem* P, RV* d, const RV* z, long long n, cudaStream_t st);
cudaError_t residual(fde_problem* P, const double* b, const double* s, double* r, long long n, int slot,
                     cudaStream_t st);
cudaError_t to_f32(const double* in, float* out, long long n, cudaStream_t st);
// out32 = skip ? 0 : (float) in64, skip read from dscal[S_CONV] (device)
cudaError_t to_f32_unless_conv(fde_problem* P, const double* in, float* out, long long n, cudaStream_t st);
// y64 += (double) d32 unless dscal[S_CONV]; counts S_REFINE when applied
cudaError_t add_f32_unless_conv(fde_problem* P, double* y, const float* d, long long n, cudaStream_t st);
// dscal[dst] = max(dscal[dst], dscal[src])
cudaError_t scalar_max(fde_problem* P, int dst, int src, cudaStream_t st);
cudaError_t add_f32(double* y, const float* d, long long n, cudaStream_t st);
template <typename R> cudaError_t fill(R* x, R v, long long n, cudaStream_t st);
template <typename R> cudaError_t copy(R* dst, const R* src, long long n, cudaStream_t st);
cudaError_t admm_pre(const AdmmArgs& A, double* c, double* bu, double* r0, double* q, cudaStream_t st);
cudaError_t admm_post(fde_problem* P, const AdmmArgs& A, const double* y, const double* By, const double* bu,
                      const double* r0, double* u, cudaStream_t st);
cudaError_t fold(const double* t, const double* q, const double* c, const double* y, const double m2inv[2],
                 const double m1[2], long long last_start, long long n, double* v, double* w, cudaStream_t st);
cudaError_t grad_ybar(const double* y, const double* ybar, const double* wy, double w0, double w1, long long last_start,
                      long long n, double* dJ, double* f, cudaStream_t st);
cudaError_t precond_set_smem_attrs();
cudaError_t toeplitz_set_smem_attrs();

}  // namespace fde
