// C ABI entry points (include/fde.h): problem set-up, operator and
// preconditioner applications, the PCG / iterative-refinement sub-solves and
// the ADMM driver (Algorithm 1 with the sub-problem merged with the p update,
// Section 3.1; psi scaling and stopping rules of Section 6.1), and the
// gradient of the optimal value.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "persist.h"
#include "saddle.h"
#include "vec.h"

using namespace fde;

static thread_local char g_cuda_err[256] = "";
static std::atomic<long long> g_launches{0};

namespace fde {
void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace fde

cudaError_t fde_alloc(fde_problem* P, void** ptr, size_t bytes) {
  if (P->nallocs >= (int)(sizeof(P->allocs) / sizeof(P->allocs[0]))) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
  if (e == cudaSuccess) P->allocs[P->nallocs++] = *ptr;
  return e;
}

static int cuda_status(cudaError_t e) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FDE_ENOMEM : FDE_ECUDA;
}

#define CK(expr)                                 \
  do {                                           \
    cudaError_t _e = (expr);                     \
    if (_e != cudaSuccess) return cuda_status(_e); \
  } while (0)

#define RK(expr)                 \
  do {                           \
    int _s = (expr);             \
    if (_s != FDE_OK) return _s; \
  } while (0)

// FP64 workspace slots
enum {
  V_Y = 0, V_U, V_ZY, V_ZU, V_P, V_WY, V_WU, V_C, V_BU, V_R0, V_Q, V_RHS, V_BY, V_R, V_Z, V_D, V_SD, V_W, V_T1, V_T2,
  V_COUNT
};
// FP32 workspace slots
enum { F_B = 0, F_X, F_R, F_Z, F_D, F_Q, F_W, F_T1, F_T2, F_COUNT };

namespace {

struct Diags {
  SliceDiag w, M1, Q, M2, M2inv;
  double m1, m2;  // preconditioner scalars (J ~ I)
  double cre;     // matching approximation S^: 2 sqrt(m1/m2) (coefficient of Re Lambda), else 0
};

bool generalized(const fde_admm_opts* o) { return o->algorithm == 2; }

// Algorithm 1: M1 = rho (J1 + I/delta), Q = rho (J2 + psi^2/delta), M2 = psi^2/Q + delta/rho,
// preconditioner scalars with J ~ I. Algorithm 2: J1 + R_y = c_y I and J2 + R_u = c_u I, so
// all three are scalars and the preconditioner takes them as they are.
Diags make_diags(const fde_problem* P, const fde_admm_opts* o) {
  Diags d{};
  const double delta = o->delta, rho = o->rho;
  const double psi2 = P->psi * P->psi;
  d.w.v[0] = 1.0;
  d.w.v[1] = P->prm.weights == 0 ? 0.5 : 1.0;
  const bool gen = generalized(o);
  for (int s = 0; s < 2; ++s) {
    d.M1.v[s] = gen ? rho * (o->c_y + 1.0 / delta) : rho * (d.w.v[s] + 1.0 / delta);
    d.Q.v[s] = gen ? rho * (o->c_u + psi2 / delta) : rho * (P->prm.gamma * d.w.v[s] + psi2 / delta);
    d.M2.v[s] = psi2 / d.Q.v[s] + delta / rho;
    d.M2inv.v[s] = 1.0 / d.M2.v[s];
  }
  if (gen) {
    d.m1 = d.M1.v[0];
    d.m2 = d.M2.v[0];
  } else {
    d.m1 = rho * (1.0 + 1.0 / delta);
    d.m2 = psi2 / (rho * (P->prm.gamma + psi2 / delta)) + delta / rho;
  }
  // matching Schur approximation with D~ = C3(B): D^ = C3^T + sqrt(m1 m2) I is circulant and
  // S^ = D^ D^T / m2 has the eigenvalues m1 + |Lambda|^2/m2 + 2 sqrt(m1/m2) Re(Lambda)
  d.cre = o->precond == 1 ? 2.0 * std::sqrt(d.m1 / d.m2) : 0.0;
  return d;
}

AdmmArgs make_admm_args(fde_problem* P, const fde_admm_opts* o, const Diags& dg, const double* ybar, const double* g,
                        const double* ya, const double* yb, const double* ua, const double* ub, double ya_s,
                        double yb_s, double ua_s, double ub_s) {
  AdmmArgs A{};
  A.n = P->N;
  A.last_start = (long long)(P->nt - 1) * P->nx * P->ny;
  A.rho = o->rho;
  A.delta = o->delta;
  A.inv_delta = 1.0 / o->delta;
  A.rho_over_delta = o->rho / o->delta;
  A.delta_over_rho = o->delta / o->rho;
  A.psi = P->psi;
  A.gamma = P->prm.gamma;
  for (int s = 0; s < 2; ++s) {
    A.w[s] = dg.w.v[s];
    A.Q[s] = dg.Q.v[s];
    A.M2[s] = dg.M2.v[s];
    A.inv_Q[s] = 1.0 / dg.Q.v[s];
    A.inv_M2[s] = 1.0 / dg.M2.v[s];
  }
  A.delta_over_psi = o->delta / P->psi;
  A.ybar = ybar;
  A.g = g;
  A.ya = ya;
  A.yb = yb;
  A.ua = ua;
  A.ub = ub;
  A.ya_s = ya_s;
  A.yb_s = yb_s;
  A.ua_s = ua_s;
  A.ub_s = ub_s;
  A.zy = P->v64[V_ZY];
  A.zu = P->v64[V_ZU];
  A.p = P->v64[V_P];
  A.wy = P->v64[V_WY];
  A.wu = P->v64[V_WU];
  if (generalized(o)) {
    A.gen = 1;
    for (int s = 0; s < 2; ++s) {
      A.ry[s] = o->rho * (o->c_y - dg.w.v[s]);
      A.ru[s] = o->rho * (o->c_u - P->prm.gamma * dg.w.v[s]);
    }
    A.yprev = P->v64[V_Y];  // y^j and u^j: the iterates before this iteration's update
    A.uprev = P->v64[V_U];
  }
  return A;
}

bool valid_opts(const fde_admm_opts* o) {
  if (!o) return false;
  const double golden = (1.0 + std::sqrt(5.0)) / 2.0;
  if (!(std::isfinite(o->delta) && o->delta > 0 && std::isfinite(o->rho) && o->rho > 0 && o->rho < golden))
    return false;
  if (o->algorithm < 0 || o->algorithm > 2) return false;
  if (o->inner_solver < 0 || o->inner_solver > 1) return false;
  if (o->precond < 0 || o->precond > 1) return false;
  if (o->warm_start < 0 || o->warm_start > 1) return false;
  if (o->inner_x0 < 0 || o->inner_x0 > 1) return false;
  if (generalized(o)) return o->rho <= 1.0 && std::isfinite(o->c_y) && o->c_y >= 1.0 && std::isfinite(o->c_u);
  return true;
}

// Problem-dependent part of the option check: R_u = c_u I - J2 must be positive semi-definite.
bool valid_opts_for(const fde_problem* P, const fde_admm_opts* o) {
  return valid_opts(o) && (!generalized(o) || o->c_u >= P->prm.gamma);
}

// Double product of the mixed refinement: B or B^T on double vectors, with
// double (dd = false) or double-float (dd = true) transform arithmetic.
cudaError_t refine_B(fde_problem* P, bool dd, int transpose, const double* x, double* y, const double* addv,
                     const SliceDiag* addc, double* t1, double* t2, cudaStream_t st, Gate gate = {}) {
  if (dd) return apply_B_df(P, transpose, x, y, nullptr, addv, addc, t1, t2, st, gate);
  return apply_B<double>(P, transpose, x, y, nullptr, addv, addc, t1, t2, st, gate);
}

int read_scalars(fde_problem* P, cudaStream_t st) {
  CK(cudaMemcpyAsync(P->hscal, P->dscal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const int flag = (int)P->hscal[S_FLAG];
  return flag;  // 0 or a negative FDE status
}

int clear_flag(fde_problem* P, cudaStream_t st) {
  CK(cudaMemsetAsync(P->dscal + S_FLAG, 0, sizeof(double), st));
  return FDE_OK;
}

template <typename R> cplx<R>* spec(fde_problem* P);
template <> double2* spec<double>(fde_problem* P) { return P->spec64; }
template <> float2* spec<float>(fde_problem* P) { return P->spec32; }

// Scratch triple (w, tmp1, tmp2) of each precision for operator applications.
template <typename R> struct Scratch { R *w, *t1, *t2; };
Scratch<double> scratch64(fde_problem* P) { return {P->v64[V_W], P->v64[V_T1], P->v64[V_T2]}; }
Scratch<float> scratch32(fde_problem* P) { return {P->v32[F_W], P->v32[F_T1], P->v32[F_T2]}; }

// Preconditioned CG (the MATLAB pcg recurrence, Hestenes-Stiefel form) on an
// SPD operator `A` with preconditioner `M`; scalars and inner products in
// double on the device. Stops when ||r||_2 <= tol ||b||_2 (recursive residual).
// x holds the initial guess when x_zero == false (double vectors only).
template <typename R, class OpA, class OpM>
int pcg(fde_problem* P, OpA A, OpM M, const R* b, R* x, bool x_zero, double tol, int maxit, R* r, R* z, R* d, R* q,
        cudaStream_t st, int* iters, double* relres) {
  const long long N = P->N;
  *iters = 0;
  RK(clear_flag(P, st));
  CK((dot<R, R>(P, b, b, N, S_BB, FIN_STORE, st)));
  if (x_zero) {
    CK(fill<R>(x, (R)0, N, st));
    CK(copy<R>(r, b, N, st));
    CK((dot<R, R>(P, r, r, N, S_RR, FIN_STORE, st)));
  } else {
    RK(A(x, q));
    if constexpr (sizeof(R) == 8) {
      CK(residual(P, (const double*)b, (const double*)q, (double*)r, N, S_RR, st));
    } else {
      return FDE_EINVAL;
    }
  }
  int flag = read_scalars(P, st);
  if (flag < 0) return flag;
  const double bb = P->hscal[S_BB];
  double rr = P->hscal[S_RR];
  if (bb == 0.0) {
    CK(fill<R>(x, (R)0, N, st));
    *relres = 0.0;
    return FDE_OK;
  }
  const double thr = tol * tol * bb;
  if (rr <= thr) {
    *relres = std::sqrt(rr / bb);
    return FDE_OK;
  }
  RK(M(r, z));
  CK((dot<R, R>(P, r, z, N, 0, FIN_RZ0, st)));
  CK(copy<R>(d, z, N, st));
  for (int it = 1; it <= maxit; ++it) {
    RK(A(d, q));
    CK((dot<R, R>(P, d, q, N, 0, FIN_ALPHA, st)));
    CK(pcg_xr<R>(P, x, r, d, q, N, st));
    flag = read_scalars(P, st);
    if (flag < 0) return flag;
    rr = P->hscal[S_RR];
    *iters = it;
    if (rr <= thr) {
      *relres = std::sqrt(rr / bb);
      return FDE_OK;
    }
    RK(M(r, z));
    CK((dot<R, R>(P, r, z, N, 0, FIN_BETA, st)));
    CK(pcg_p<R>(P, d, z, N, st));
  }
  *relres = std::sqrt(rr / bb);
  return FDE_ENOCONV;
}

template <typename R>
int op_S(fde_problem* P, const Diags& dg, const R* x, R* y, Scratch<R> s, cudaStream_t st, Gate gate = {}) {
  CK(apply_S<R>(P, dg.M1, dg.M2inv, x, y, s.w, s.t1, s.t2, st, gate));
  return FDE_OK;
}
template <typename R>
int op_M(fde_problem* P, const Diags& dg, const R* r, R* z, cudaStream_t st, Gate gate = {}) {
  CK(apply_precond<R>(P, dg.m1, dg.m2, 0, r, z, spec<R>(P), st, gate, dg.cre));
  return FDE_OK;
}

struct SolveInfo {
  int pcg_iters = 0, refine = 0, fp64_matvecs = 0, recursive = 0, float_steers = 0;
  double relres = 0.0;
};

// Solve S y = rhs, y holding a warm start, with rhs = c + B^T q.
// FP64: PCG in double on rhs (formed by the caller). MIXED: double iterative
// refinement around float PCG on the correction; each residual is evaluated in
// the folded form rhs - S y = (c - M1 y) + B^T (q - M2^-1 B y), one double B and
// one double B^T, and leaves B y of the returned y in V_BY (by_valid = true).
// The norm of rhs, used only for the relative stopping test, is formed in float.
int subsolve(fde_problem* P, const Diags& dg, const fde_admm_opts* o, const double* rhs, const double* c,
             const double* q, double* y, double tol, cudaStream_t st, SolveInfo* info, bool by_on_entry,
             bool* by_valid) {
  const long long N = P->N;
  *by_valid = false;
  if (o->precision == FDE_FP64) {
    auto A = [&](const double* x, double* out) { return op_S<double>(P, dg, x, out, scratch64(P), st); };
    auto M = [&](const double* r, double* z) { return op_M<double>(P, dg, r, z, st); };
    int it = 0;
    double rel = 0;
    const int s = pcg<double>(P, A, M, rhs, y, false, tol, o->max_pcg, P->v64[V_R], P->v64[V_Z], P->v64[V_D],
                              P->v64[V_SD], st, &it, &rel);
    info->pcg_iters += it;
    info->fp64_matvecs += 2 * (it + 1);
    info->relres = rel;
    return s;
  }
  // mixed: ||rhs||^2 from a float evaluation of c + B^T q
  const long long last = (long long)(P->nt - 1) * P->nx * P->ny;
  const SliceDiag one{{1.0, 1.0}};
  auto s32 = scratch32(P);
  auto s64 = scratch64(P);
  CK(to_f32(q, P->v32[F_B], N, st));
  CK(to_f32(c, P->v32[F_R], N, st));
  CK(apply_B<float>(P, 1, P->v32[F_B], P->v32[F_Z], nullptr, P->v32[F_R], &one, s32.t1, s32.t2, st));
  CK((dot<float, float>(P, P->v32[F_Z], P->v32[F_Z], N, S_TMP0, FIN_STORE, st)));
  int flag = read_scalars(P, st);
  if (flag < 0) return flag;
  const double bb = P->hscal[S_TMP0];
  if (bb == 0.0) {
    CK(fill<double>(y, 0.0, N, st));
    info->relres = 0.0;
    return FDE_OK;
  }
  const double inner = o->inner_tol_mixed > 0 ? o->inner_tol_mixed : 1e-4;
  const int maxref = o->max_refine > 0 ? o->max_refine : 20;
  auto A32 = [&](const float* x, float* out) { return op_S<float>(P, dg, x, out, s32, st); };
  auto M32 = [&](const float* r, float* z) { return op_M<float>(P, dg, r, z, st); };
  // FDE_MIXED_DFV: an evaluation that cannot be the last one (the next correction cannot
  // reach tol: rel * inner > tol) runs its products in double-float; the others, and a
  // re-check of any double-float evaluation that meets tol, in double, so that the
  // accepted residual and B y are double products.
  const bool dfv = o->precision == FDE_MIXED_DFV;
  bool dd = o->precision == FDE_MIXED_DF || dfv;
  bool by_dd = o->precision == FDE_MIXED_DF;  // V_BY holds a double-float product
  // FDE_MIXED_DFV also lets the float PCG's recursive residual r - S d steer the next
  // correction when it is accurate enough: its error, rounding drift plus the float operator's
  // own error, is about kFloatDrift of the residual the correction started from, so a start
  // residual rel with rel * kFloatDrift <= tol / 10 skips one evaluation (two products).
  constexpr double kFloatDrift = 1e-6;
  // FDE_MIXED_DFV: the first evaluation of a warm-started sub-problem only steers the
  // first correction. When the previous sub-problem started far from its solution
  // (relative residual >= kFloatSteer) it runs in float: the folded halves are formed in
  // double and rounded, B^T runs in float, and the result, accurate to about 1e-7 of
  // ||rhs||, is the correction's right-hand side as it stands. It is used when its own
  // relative residual is >= kFloatSteer / 10 (a thousand times its rounding error);
  // otherwise the evaluation is repeated in double-float. It is never accepted.
  constexpr double kFloatSteer = 1e-3;
  const bool steer32 = dfv && by_on_entry && P->last_rel0 >= kFloatSteer && maxref > 0;
  bool implicit_next = false;
  double rel_implicit = 0.0;
  for (int k = 0; k <= maxref; ++k) {
    double rel = 0.0;
    const bool had_implicit = implicit_next;
    implicit_next = false;
    const bool implicit = had_implicit && rel_implicit > tol && k < maxref;
    bool used32 = false;
    if (k == 0 && steer32) {
      CK(fold(P->v64[V_BY], q, c, y, dg.M2inv.v, dg.M1.v, last, N, P->v64[V_SD], P->v64[V_Z], st));
      CK(to_f32(P->v64[V_SD], P->v32[F_D], N, st));
      CK(to_f32(P->v64[V_Z], P->v32[F_R], N, st));
      CK(apply_B<float>(P, 1, P->v32[F_D], P->v32[F_B], nullptr, P->v32[F_R], &one, s32.t1, s32.t2, st));
      CK((dot<float, float>(P, P->v32[F_B], P->v32[F_B], N, S_RR, FIN_STORE, st)));
      flag = read_scalars(P, st);
      if (flag < 0) return flag;
      rel = std::sqrt(P->hscal[S_RR] / bb);
      if (rel >= 0.1 * kFloatSteer) {
        used32 = true;
        P->last_rel0 = rel;
        info->float_steers += 1;
        info->relres = rel;
        dd = rel * inner > tol;
      }
    }
    if (used32) {
      // F_B holds the float residual: straight to the correction
    } else if (implicit) {
      rel = rel_implicit;
      CK(copy<float>(P->v32[F_B], P->v32[F_R], N, st));  // the recursive residual is the next right-hand side
      dd = rel * inner > tol;
      info->recursive += 1;
    } else {
      // the recursive residual already meets tol (or this is the last evaluation): verify in double
      if (had_implicit) dd = false;
      // on entry V_BY already holds B y for the warm start (kept by the ADMM loop)
      const bool y_changed = k > 0 || !by_on_entry;
      for (int pass = 0; pass < 2; ++pass) {
        if ((pass == 0 && y_changed) || (by_dd && !dd)) {
          CK(refine_B(P, dd, 0, y, P->v64[V_BY], nullptr, nullptr, s64.t1, s64.t2, st));
          info->fp64_matvecs += 1;
          by_dd = dd;
        }
        CK(fold(P->v64[V_BY], q, c, y, dg.M2inv.v, dg.M1.v, last, N, P->v64[V_SD], P->v64[V_Z], st));
        CK(refine_B(P, dd, 1, P->v64[V_SD], P->v64[V_R], P->v64[V_Z], &one, s64.t1, s64.t2, st));
        info->fp64_matvecs += 1;
        *by_valid = !by_dd || o->precision == FDE_MIXED_DF;
        CK((dot<double, double>(P, P->v64[V_R], P->v64[V_R], N, S_RR, FIN_STORE, st)));
        flag = read_scalars(P, st);
        if (flag < 0) return flag;
        rel = std::sqrt(P->hscal[S_RR] / bb);
        if (!(dfv && dd && rel <= tol)) break;
        dd = false;  // met tol in double-float: evaluate again in double
      }
      rel_implicit = 0.0;
      info->relres = rel;
      if (k == 0) P->last_rel0 = rel;
      if (rel <= tol) return FDE_OK;
      if (k == maxref) break;
      if (dfv) dd = rel * inner > tol;
      CK(to_f32(P->v64[V_R], P->v32[F_B], N, st));
    }
    int it = 0;
    double rr32 = 0;
    // the float correction only needs to reduce the residual by `inner`
    const int s = pcg<float>(P, A32, M32, P->v32[F_B], P->v32[F_X], true, std::fmax(inner, tol / rel * 0.5),
                             o->max_pcg, P->v32[F_R], P->v32[F_Z], P->v32[F_D], P->v32[F_Q], st, &it, &rr32);
    info->pcg_iters += it;
    info->refine += 1;
    if (s != FDE_OK && s != FDE_ENOCONV) return s;
    CK(add_f32(y, P->v32[F_X], N, st));
    *by_valid = false;
    if (dfv && !implicit && !used32 && rel * kFloatDrift <= 0.1 * tol) {
      implicit_next = true;
      rel_implicit = rr32 * rel;  // |r - S d| / |rhs| from the PCG's own residual
    }
  }
  return FDE_ENOCONV;
}

// ---------------------------------------------------------------------------
// Saddle-point sub-problem (Section 3.3.1): K [y; u; p] = [b_y; b_u; f_p] by
// preconditioned MINRES with K-tilde = blkdiag(M1, Q, Sigma-tilde), where
// Sigma-tilde = m2 I + C3 C3^T / m1 stands in for the p-block Schur complement
// M2 + B M1^-1 B^T (the FFT-diagonal form of S-tilde with m1 and m2 exchanged).
// A vector of this system is [y | u | p], 3N contiguous entries.
// ---------------------------------------------------------------------------

// Workspace of the saddle-point path, allocated on first use: 10 vectors of 3N
// doubles (x, f, and MINRES's or the refinement's vectors) and, for the mixed
// path, 10 of 3N floats.
int saddle_workspace(fde_problem* P, bool need32) {
  const size_t n3 = 3 * (size_t)P->N;
  void* ptr = nullptr;
  if (!P->mr64) {
    CK(fde_alloc(P, &ptr, sizeof(double) * n3 * 10));
    P->mr64 = (double*)ptr;
  }
  if (need32 && !P->mr32) {
    CK(fde_alloc(P, &ptr, sizeof(float) * n3 * 10));
    P->mr32 = (float*)ptr;
  }
  return FDE_OK;
}

// q = K z: q_y = M1 z_y + B^T z_p, q_u = Q z_u + psi z_p, q_p = B z_y + psi z_u - (delta/rho) z_p.
// df: the double products in double-float arithmetic.
template <typename R>
int op_K(fde_problem* P, const Diags& dg, const fde_admm_opts* o, const R* z, R* q, Scratch<R> s, cudaStream_t st,
         bool df = false) {
  const long long N = P->N, last = (long long)(P->nt - 1) * P->nx * P->ny;
  const R *zy = z, *zu = z + N, *zp = z + 2 * N;
  R *qy = q, *qu = q + N, *qp = q + 2 * N;
  if constexpr (sizeof(R) == 8) {
    if (df) {
      CK(apply_B_df(P, 1, zp, qy, nullptr, zy, &dg.M1, s.t1, s.t2, st));
      CK(apply_B_df(P, 0, zy, qp, nullptr, nullptr, nullptr, s.t1, s.t2, st));
    } else {
      CK(apply_B<R>(P, 1, zp, qy, nullptr, zy, &dg.M1, s.t1, s.t2, st));
      CK(apply_B<R>(P, 0, zy, qp, nullptr, nullptr, nullptr, s.t1, s.t2, st));
    }
  } else {
    CK(apply_B<R>(P, 1, zp, qy, nullptr, zy, &dg.M1, s.t1, s.t2, st));
    CK(apply_B<R>(P, 0, zy, qp, nullptr, nullptr, nullptr, s.t1, s.t2, st));
  }
  CK(saddle_tail<R>(N, last, dg.Q.v, P->psi, o->delta / o->rho, zu, zp, qu, qp, st));
  return FDE_OK;
}

// z = K-tilde^-1 r.
template <typename R>
int op_Kt(fde_problem* P, const Diags& dg, const R* r, R* z, cudaStream_t st) {
  const long long N = P->N, last = (long long)(P->nt - 1) * P->nx * P->ny;
  CK(block_diag<R>(N, last, dg.M1.v, dg.Q.v, r, z, st));
  CK(apply_precond<R>(P, dg.m2, dg.m1, 0, r + 2 * N, z + 2 * N, spec<R>(P), st));
  return FDE_OK;
}

// Preconditioned MINRES (Paige and Saunders) on a symmetric operator A with a
// symmetric positive definite preconditioner M: the Lanczos process in the
// M^-1 inner product; its tridiagonal is factored by Givens rotations on the
// host from the two inner products of each iteration (read back together). x
// minimises ||b - A x||_{M^-1} over the Krylov space; the rotations give that
// norm, |eta|, and the solve stops when |eta| <= tol ||b||_{M^-1}. x holds the
// initial guess unless x_zero. wk: 7 vectors of n.
template <typename R, class OpA, class OpM>
int minres(fde_problem* P, OpA A, OpM M, const R* b, R* x, bool x_zero, double tol, int maxit, R* const* wk,
           long long n, cudaStream_t st, int* iters, double* relres) {
  R *vp = wk[0], *v = wk[1], *z = wk[2], *zn = wk[3], *wp = wk[4], *w = wk[5], *q = wk[6];
  *iters = 0;
  RK(clear_flag(P, st));
  RK(M(b, z));
  CK((dot<R, R>(P, b, z, n, S_BB, FIN_STORE, st)));
  if (x_zero) {
    CK(fill<R>(x, (R)0, n, st));
    CK(copy<R>(v, b, n, st));
  } else {
    RK(A(x, q));
    CK(lin3<R>(n, 1.0, b, -1.0, nullptr, 0, q, 0.0, q, v, st));
  }
  RK(M(v, z));
  CK((dot<R, R>(P, v, z, n, S_RR, FIN_STORE, st)));
  int flag = read_scalars(P, st);
  if (flag < 0) return flag;
  const double bn = std::sqrt(std::fmax(P->hscal[S_BB], 0.0));
  double beta = std::sqrt(std::fmax(P->hscal[S_RR], 0.0));
  if (bn == 0.0) {
    CK(fill<R>(x, (R)0, n, st));
    *relres = 0.0;
    return FDE_OK;
  }
  double eta = beta;
  if (eta <= tol * bn) {
    *relres = eta / bn;
    return FDE_OK;
  }
  CK(fill<R>(vp, (R)0, n, st));
  CK(fill<R>(wp, (R)0, n, st));
  CK(fill<R>(w, (R)0, n, st));
  double beta_prev = 1.0, c_prev = 1.0, c = 1.0, s_prev = 0.0, s = 0.0;
  for (int it = 1; it <= maxit; ++it) {
    // z holds the unnormalised M^-1 v_k; the Lanczos vector is z / beta
    RK(A(z, q));
    CK((dot<R, R>(P, q, z, n, S_TMP0, FIN_STORE, st)));  // alpha beta^2
    // v_{k+1} = q / beta - (alpha / beta) v_k - (beta / beta_prev) v_{k-1}, into v_{k-1}'s storage
    CK(lin3<R>(n, 1.0 / beta, q, -1.0 / (beta * beta * beta), P->dscal, S_TMP0, v, -beta / beta_prev, vp, vp, st));
    RK(M(vp, zn));
    CK((dot<R, R>(P, vp, zn, n, S_TMP1, FIN_STORE, st)));
    flag = read_scalars(P, st);
    if (flag < 0) return flag;
    const double alpha = P->hscal[S_TMP0] / (beta * beta);
    const double beta_next = std::sqrt(std::fmax(P->hscal[S_TMP1], 0.0));
    // column k of the tridiagonal after the rotations k-2 and k-1, then the new rotation
    const double e3 = s_prev * beta;
    const double e2 = s * alpha + c_prev * c * beta;
    const double e0 = c * alpha - c_prev * s * beta;
    const double e1 = std::hypot(e0, beta_next);
    if (!(e1 > 0.0) || !std::isfinite(e1)) return FDE_EBREAKDOWN;
    const double c_new = e0 / e1, s_new = beta_next / e1;
    // w_{k+1} = (z / beta - e3 w_{k-1} - e2 w_k) / e1 into w_{k-1}'s storage; x += c_new eta w_{k+1}
    CK(minres_wx<R>(n, 1.0 / (beta * e1), z, -e3 / e1, wp, -e2 / e1, w, c_new * eta, x, st));
    eta = -s_new * eta;
    *iters = it;
    if (std::fabs(eta) <= tol * bn) {
      *relres = std::fabs(eta) / bn;
      return FDE_OK;
    }
    std::swap(vp, v);
    std::swap(wp, w);
    std::swap(z, zn);
    beta_prev = beta;
    beta = beta_next;
    c_prev = c;
    c = c_new;
    s_prev = s;
    s = s_new;
    if (beta == 0.0) {  // invariant Krylov space: x is exact
      *relres = std::fabs(eta) / bn;
      return FDE_OK;
    }
  }
  *relres = std::fabs(eta) / bn;
  return FDE_ENOCONV;
}

// Solve K x = f (3N, double), x holding a warm start. FP64: MINRES in double,
// stopping on ||r||_{K-tilde^-1} <= tol ||f||_{K-tilde^-1}. MIXED / MIXED_DF:
// double (or double-float) residuals r = f - K x, float MINRES on K d = r to
// max(inner, tol / (2 rel)), x += d, until ||r||_2 <= tol ||f||_2.
int saddle_solve(fde_problem* P, const Diags& dg, const fde_admm_opts* o, const double* f, double* x, double tol,
                 cudaStream_t st, SolveInfo* info) {
  const long long n3 = 3 * P->N;
  double* wk64[7];
  for (int i = 0; i < 7; ++i) wk64[i] = P->mr64 + (size_t)(3 + i) * n3;
  auto s64 = scratch64(P);
  if (o->precision == FDE_FP64) {
    auto A = [&](const double* z, double* q) { return op_K<double>(P, dg, o, z, q, s64, st); };
    auto M = [&](const double* r, double* z) { return op_Kt<double>(P, dg, r, z, st); };
    int it = 0;
    double rel = 0.0;
    const int s = minres<double>(P, A, M, f, x, false, tol, o->max_pcg, wk64, n3, st, &it, &rel);
    info->pcg_iters += it;
    info->fp64_matvecs += 2 * (it + 1);
    info->relres = rel;
    return s;
  }
  const bool dfv = o->precision == FDE_MIXED_DFV;
  bool dd = o->precision == FDE_MIXED_DF || dfv;
  double* r64 = P->mr64 + 2 * (size_t)n3;
  float* b32 = P->mr32;
  float* d32 = P->mr32 + n3;
  float* wk32[7];
  for (int i = 0; i < 7; ++i) wk32[i] = P->mr32 + (size_t)(2 + i) * n3;
  auto s32 = scratch32(P);
  auto A32 = [&](const float* z, float* q) { return op_K<float>(P, dg, o, z, q, s32, st); };
  auto M32 = [&](const float* r, float* z) { return op_Kt<float>(P, dg, r, z, st); };
  RK(clear_flag(P, st));
  CK((dot<double, double>(P, f, f, n3, S_BB, FIN_STORE, st)));
  int flag = read_scalars(P, st);
  if (flag < 0) return flag;
  const double ff = P->hscal[S_BB];  // read once: the float MINRES reuses the slot
  const double inner = o->inner_tol_mixed > 0 ? o->inner_tol_mixed : 1e-4;
  const int maxref = o->max_refine > 0 ? o->max_refine : 20;
  if (ff == 0.0) {
    CK(fill<double>(x, 0.0, n3, st));
    info->relres = 0.0;
    return FDE_OK;
  }
  for (int k = 0; k <= maxref; ++k) {
    double rel = 0.0;
    for (int pass = 0; pass < 2; ++pass) {  // as in subsolve: a double re-check of a double-float pass
      RK(op_K<double>(P, dg, o, x, r64, s64, st, dd));
      info->fp64_matvecs += 2;
      CK(lin3<double>(n3, 1.0, f, -1.0, nullptr, 0, r64, 0.0, r64, r64, st));
      CK((dot<double, double>(P, r64, r64, n3, S_RR, FIN_STORE, st)));
      flag = read_scalars(P, st);
      if (flag < 0) return flag;
      rel = std::sqrt(P->hscal[S_RR] / ff);
      if (!(dfv && dd && rel <= tol)) break;
      dd = false;
    }
    info->relres = rel;
    if (rel <= tol) return FDE_OK;
    if (k == maxref) break;
    if (dfv) dd = rel * inner > tol;
    CK(to_f32(r64, b32, n3, st));
    int it = 0;
    double rr = 0.0;
    const int s = minres<float>(P, A32, M32, b32, d32, true, std::fmax(inner, 0.5 * tol / rel), o->max_pcg, wk32, n3,
                                st, &it, &rr);
    info->pcg_iters += it;
    info->refine += 1;
    if (s != FDE_OK && s != FDE_ENOCONV) return s;
    CK(add_f32(x, d32, n3, st));
  }
  return FDE_ENOCONV;
}

}  // namespace

extern "C" {

const char* fde_strerror(int s) {
  switch (s) {
    case FDE_OK: return "ok";
    case FDE_EINVAL: return "invalid argument";
    case FDE_ENOMEM: return "device out of memory";
    case FDE_ECUDA: return "CUDA error";
    case FDE_ENOCONV: return "iteration cap reached before convergence";
    case FDE_EBREAKDOWN: return "PCG breakdown (non-positive curvature)";
    case FDE_ENONFINITE: return "non-finite value in a reduction";
    case FDE_EUNSUPPORTED: return "unsupported size or mode";
    case FDE_ETIMEOUT: return "a bounded device-side wait ran out";
    default: return "unknown status";
  }
}

const char* fde_last_cuda_error(void) { return g_cuda_err; }

long long fde_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

long long fde_size(const fde_problem* P) { return P ? P->N : 0; }
double fde_psi(const fde_problem* P) { return P ? P->psi : 0.0; }

void fde_destroy(fde_problem* P) {
  if (!P) return;
  for (int i = 0; i < P->nallocs; ++i) cudaFree(P->allocs[i]);
  if (P->hscal) cudaFreeHost(P->hscal);
  delete P;
}

int fde_setup(const fde_params* prm, fde_problem** out, void* stream) {
  if (!prm || !out) return FDE_EINVAL;
  *out = nullptr;
  const fde_params& q = *prm;
  auto fin = [](double v) { return std::isfinite(v); };
  if (q.nx < 1 || q.ny < 1 || q.nt < 1) return FDE_EINVAL;
  if (!(fin(q.beta_x) && q.beta_x > 1 && q.beta_x < 2 && fin(q.beta_y) && q.beta_y > 1 && q.beta_y < 2))
    return FDE_EINVAL;
  if (!(fin(q.alpha_t) && q.alpha_t > 0 && q.alpha_t <= 1)) return FDE_EINVAL;
  if (!(fin(q.dp) && fin(q.dm) && fin(q.ep) && fin(q.em) && q.dp >= 0 && q.dm >= 0 && q.ep >= 0 && q.em >= 0))
    return FDE_EINVAL;
  if (!(fin(q.gamma) && q.gamma > 0)) return FDE_EINVAL;
  if (!(fin(q.T) && q.T > 0)) return FDE_EINVAL;
  if ((q.weights != 0 && q.weights != 1) || (q.time_step_mode != 0 && q.time_step_mode != 1)) return FDE_EINVAL;
  if (q.nx > kMaxAxis || q.ny > kMaxAxis || q.nt > kMaxAxis) return FDE_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;

  static bool attrs_done = false;
  if (!attrs_done) {
    CK(toeplitz_set_smem_attrs());
    CK(precond_set_smem_attrs());
    attrs_done = true;
  }

  fde_problem* P = new fde_problem();
  P->prm = q;
  P->nx = q.nx;
  P->ny = q.ny;
  P->nt = q.nt;
  P->N = (long long)q.nx * q.ny * q.nt;
  P->hx = 1.0 / (q.nx + 1);
  P->hy = 1.0 / (q.ny + 1);
  P->ht = q.time_step_mode == 0 ? q.T / q.nt : P->hx;
  P->psi = std::fmin(std::pow(P->ht, q.alpha_t), std::fmin(std::pow(P->hx, q.beta_x), std::pow(P->hy, q.beta_y)));
  P->euler = (q.alpha_t == 1.0);
  P->H = q.ny / 2 + 1;
  P->Hp = (P->H + 1) & ~1;

  auto fail = [&](cudaError_t e) {
    const int s = cuda_status(e);
    fde_destroy(P);
    return s;
  };
  cudaError_t e;
  if ((e = cudaMallocHost((void**)&P->hscal, sizeof(double) * S_COUNT))) return fail(e);
  void* p;
  if ((e = fde_alloc(P, &p, sizeof(double) * kMaxPartials))) return fail(e);
  P->partials = (double*)p;
  if ((e = fde_alloc(P, &p, sizeof(double) * S_COUNT))) return fail(e);
  P->dscal = (double*)p;
  if ((e = cudaMemsetAsync(P->dscal, 0, sizeof(double) * S_COUNT, st))) return fail(e);
  if ((e = setup_axis_tables(P, st))) return fail(e);
  const size_t N = (size_t)P->N;
  for (int i = 0; i < V_COUNT; ++i) {
    if ((e = fde_alloc(P, &p, sizeof(double) * N))) return fail(e);
    P->v64[i] = (double*)p;
    if ((e = cudaMemsetAsync(p, 0, sizeof(double) * N, st))) return fail(e);
  }
  for (int i = 0; i < F_COUNT; ++i) {
    if ((e = fde_alloc(P, &p, sizeof(float) * N))) return fail(e);
    P->v32[i] = (float*)p;
    if ((e = cudaMemsetAsync(p, 0, sizeof(float) * N, st))) return fail(e);
  }
  const size_t ns = (size_t)P->nt * P->nx * P->Hp;
  if ((e = fde_alloc(P, &p, sizeof(double2) * ns))) return fail(e);
  P->spec64 = (double2*)p;
  if ((e = cudaMemsetAsync(p, 0, sizeof(double2) * ns, st))) return fail(e);
  if ((e = fde_alloc(P, &p, sizeof(float2) * ns))) return fail(e);
  P->spec32 = (float2*)p;
  if ((e = cudaMemsetAsync(p, 0, sizeof(float2) * ns, st))) return fail(e);
  if ((e = cudaStreamSynchronize(st))) return fail(e);
  *out = P;
  return FDE_OK;
}

int fde_matvec(fde_problem* P, int op, const fde_admm_opts* o, int precision, const void* x, void* y, void* stream) {
  if (!P || !x || !y || x == y) return FDE_EINVAL;
  if (op != FDE_OP_B && op != FDE_OP_BT && op != FDE_OP_S) return FDE_EINVAL;
  if (precision != FDE_FP64 && precision != FDE_FP32 && precision != FDE_MIXED_DF) return FDE_EINVAL;
  if (op == FDE_OP_S && !valid_opts_for(P, o)) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == FDE_MIXED_DF) {
    if (op == FDE_OP_S) return FDE_EINVAL;
    auto s = scratch64(P);
    CK(apply_B_df(P, op == FDE_OP_BT, (const double*)x, (double*)y, nullptr, nullptr, nullptr, s.t1, s.t2, st));
  } else if (precision == FDE_FP64) {
    auto s = scratch64(P);
    if (op == FDE_OP_S) {
      const Diags dg = make_diags(P, o);
      return op_S<double>(P, dg, (const double*)x, (double*)y, s, st);
    }
    CK(apply_B<double>(P, op == FDE_OP_BT, (const double*)x, (double*)y, nullptr, nullptr, nullptr, s.t1, s.t2, st));
  } else {
    auto s = scratch32(P);
    if (op == FDE_OP_S) {
      const Diags dg = make_diags(P, o);
      return op_S<float>(P, dg, (const float*)x, (float*)y, s, st);
    }
    CK(apply_B<float>(P, op == FDE_OP_BT, (const float*)x, (float*)y, nullptr, nullptr, nullptr, s.t1, s.t2, st));
  }
  return FDE_OK;
}

int fde_autotune(fde_problem* P, void* stream) {
  if (!P) return FDE_EINVAL;
  CK(autotune_tiles(P, P->v32[F_W], P->v32[F_T1], P->v64[V_W], P->v64[V_T1], (cudaStream_t)stream));
  return FDE_OK;
}

// Tile fields of one precision: float, double-float or double passes.
static void tile_fields(fde_problem* P, int precision, int** rows, int** axis) {
  *rows = precision == FDE_FP32 ? &P->rows_nt32 : precision == FDE_FP64 ? &P->rows_nt64 : &P->rows_ntdd;
  *axis = precision == FDE_FP32 ? &P->axis_nt32 : precision == FDE_FP64 ? &P->axis_nt64 : &P->axis_ntdd;
}

int fde_set_tiles(fde_problem* P, int precision, int rows_threads, int axis_threads) {
  if (!P || (precision != FDE_FP32 && precision != FDE_MIXED_DF && precision != FDE_FP64)) return FDE_EINVAL;
  const bool long_rows = P->ax[2].L > 2048;
  bool rows_ok, axis_ok;
  if (precision == FDE_FP32) {
    rows_ok = rows_threads == 0 || rows_threads == 256 || rows_threads == 512 || (!long_rows && rows_threads == 128);
    axis_ok = axis_threads == 0 || axis_threads == 512 || axis_threads == 256;
  } else {
    rows_ok = rows_threads == 0 || rows_threads == 256 || rows_threads == -512 ||
              (!long_rows && (rows_threads == -256 || rows_threads == 128));
    // 128 threads: lines of up to 2048 (longer lines keep the 256-thread tile)
    axis_ok = axis_threads == 0 || axis_threads == 256 || axis_threads == -512 || axis_threads == 128;
  }
  if (!rows_ok || !axis_ok) return FDE_EINVAL;
  int *rf, *af;
  tile_fields(P, precision, &rf, &af);
  if (rows_threads) *rf = rows_threads;
  if (axis_threads) *af = axis_threads;
  return FDE_OK;
}

int fde_tiles(const fde_problem* P, int precision, int* rows_threads, int* axis_threads) {
  if (!P || !rows_threads || !axis_threads ||
      (precision != FDE_FP32 && precision != FDE_MIXED_DF && precision != FDE_FP64))
    return FDE_EINVAL;
  int *rf, *af;
  tile_fields(const_cast<fde_problem*>(P), precision, &rf, &af);
  *rows_threads = *rf;
  *axis_threads = *af;
  return FDE_OK;
}

int fde_apply_factor(fde_problem* P, int axis, int op, int precision, const void* x, void* y, void* stream) {
  if (!P || !x || !y || x == y || (axis != 1 && axis != 2) || (op != FDE_OP_B && op != FDE_OP_BT)) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int conj = op == FDE_OP_BT;
  if (precision == FDE_FP64) {
    CK(apply_axis_raw<double>(P, axis, (const double*)x, (double*)y, P->ax[axis].d.sym, conj, st));
  } else if (precision == FDE_FP32) {
    CK(apply_axis_raw<float>(P, axis, (const float*)x, (float*)y, P->ax[axis].f.sym, conj, st));
  } else if (precision == FDE_MIXED_DF) {
    CK(apply_axis_raw_df(P, axis, (const double*)x, (double*)y, conj, st));
  } else {
    return FDE_EINVAL;
  }
  return FDE_OK;
}

int fde_precond(fde_problem* P, const fde_admm_opts* o, int precision, const void* r, void* z, void* stream) {
  if (!P || !r || !z || !valid_opts_for(P, o)) return FDE_EINVAL;
  if (precision != FDE_FP64 && precision != FDE_FP32) return FDE_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!P->ax[a].n_ok) return FDE_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const Diags dg = make_diags(P, o);
  if (precision == FDE_FP64) return op_M<double>(P, dg, (const double*)r, (double*)z, st);
  return op_M<float>(P, dg, (const float*)r, (float*)z, st);
}

// The ADMM solve; y, u, p, zu (device) may each be NULL (not copied out; the
// iterates stay in V_Y, V_U, V_P, V_ZU).
static int admm_solve_impl(fde_problem* P, const fde_admm_opts* o, const double* ybar, const double* g,
                           const double* ya, const double* yb, const double* ua, const double* ub, double ya_s,
                           double yb_s, double ua_s, double ub_s, double* y, double* u, double* p, double* zu,
                           fde_admm_stats* stats, cudaStream_t st) {
  if (!P || !valid_opts_for(P, o) || !ybar) return FDE_EINVAL;
  if (o->precision != FDE_FP64 && o->precision != FDE_MIXED && o->precision != FDE_MIXED_DF &&
      o->precision != FDE_MIXED_DFV)
    return FDE_EINVAL;
  if (o->max_admm < 1 || o->max_pcg < 1) return FDE_EINVAL;
  if (std::isnan(ya_s) || std::isnan(yb_s) || std::isnan(ua_s) || std::isnan(ub_s)) return FDE_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!P->ax[a].n_ok) return FDE_EUNSUPPORTED;
  const long long N = P->N;
  const Diags dg = make_diags(P, o);

  AdmmArgs A = make_admm_args(P, o, dg, ybar, g, ya, yb, ua, ub, ya_s, yb_s, ua_s, ub_s);
  double* Y = P->v64[V_Y];
  double* U = P->v64[V_U];
  // zero iterates, or (warm start) the iterates the previous solve ended with; V_BY = B Y
  // holds in both cases (B 0 = 0; a solve leaves B of its final y) and is kept across iterations
  if (o->warm_start) {
    if (!P->state_valid) return FDE_EINVAL;
  } else {
    for (int i : {V_Y, V_U, V_ZY, V_ZU, V_P, V_WY, V_WU, V_BY}) CK(fill<double>(P->v64[i], 0.0, N, st));
    P->last_rel0 = 1.0;
  }
  P->state_valid = false;  // set again once this solve has left a consistent state
  // a failed earlier call may have left its error flag set; the mixed sub-solve reads
  // the flag before its PCG clears it
  RK(clear_flag(P, st));

  fde_admm_stats S{};
  SolveInfo info;
  double res[3] = {1.0, 1.0, 1.0};
  int status = FDE_ENOCONV;
  auto s64 = scratch64(P);
  const SliceDiag one{{1.0, 1.0}};
  const bool saddle = o->inner_solver == 1;
  if (saddle) RK(saddle_workspace(P, o->precision != FDE_FP64));
  AdmmArgs Ag = A;  // post-step taking u and p from the saddle-point solve
  Ag.given_up = 1;
  for (int j = 0; j < o->max_admm; ++j) {
    CK(admm_pre(A, P->v64[V_C], P->v64[V_BU], P->v64[V_R0], P->v64[V_Q], st));
    double tol;
    if (o->inner_tol_mode == 1) {
      tol = o->inner_tol;
    } else {
      const double mn = std::fmin(res[0], std::fmin(res[1], res[2]));
      tol = 0.05 * std::fmax(mn, o->tol_admm);
    }
    if (saddle) {
      const size_t n3 = 3 * (size_t)N;
      double* X = P->mr64;
      double* F = P->mr64 + n3;
      // f_y = c + (1 - rho) B^T p^j, f_u = b_u, f_p = psi g - (delta/rho) p^j
      const SliceDiag omr{{1.0 - o->rho, 1.0 - o->rho}};
      if (o->precision == FDE_MIXED_DF)
        CK(apply_B_df(P, 1, A.p, F, &omr, P->v64[V_C], &one, s64.t1, s64.t2, st));
      else
        CK(apply_B<double>(P, 1, A.p, F, &omr, P->v64[V_C], &one, s64.t1, s64.t2, st));
      CK(saddle_rhs(N, P->psi, o->delta / o->rho, P->v64[V_BU], g, A.p, F + N, F + 2 * N, st));
      // initial guess (y^j, u^j, p^j), or zero
      if (o->inner_x0 == 1) {
        CK(fill<double>(X, 0.0, 3 * N, st));
      } else {
        CK(cudaMemcpyAsync(X, Y, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(X + N, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(X + 2 * N, A.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      }
      const int s = saddle_solve(P, dg, o, F, X, tol, st, &info);
      if (s != FDE_OK && s != FDE_ENOCONV) {
        status = s;
        break;
      }
      S.max_sub_relres = std::fmax(S.max_sub_relres, info.relres);
      CK(cudaMemcpyAsync(Y, X, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(U, X + N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      CK(cudaMemcpyAsync(A.p, X + 2 * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
      CK(refine_B(P, o->precision == FDE_MIXED_DF, 0, Y, P->v64[V_BY], nullptr, nullptr, s64.t1, s64.t2, st));
      info.fp64_matvecs += 1;
      RK(clear_flag(P, st));
      CK(admm_post(P, Ag, Y, P->v64[V_BY], P->v64[V_BU], P->v64[V_R0], U, st));
    } else {
    if (o->precision == FDE_FP64) {
      // rhs = c + B^T q
      CK(apply_B<double>(P, 1, P->v64[V_Q], P->v64[V_RHS], nullptr, P->v64[V_C], &one, s64.t1, s64.t2, st));
      info.fp64_matvecs += 1;
    }
    bool by_valid = false;
    if (o->inner_x0 == 1) {  // zero initial guess: y = 0 and B y = 0
      CK(fill<double>(Y, 0.0, N, st));
      CK(fill<double>(P->v64[V_BY], 0.0, N, st));
    }
    const int s = subsolve(P, dg, o, P->v64[V_RHS], P->v64[V_C], P->v64[V_Q], Y, tol, st, &info, true, &by_valid);
    if (s != FDE_OK && s != FDE_ENOCONV) {
      status = s;
      break;
    }
    S.max_sub_relres = std::fmax(S.max_sub_relres, info.relres);
    if (!by_valid) {
      CK(refine_B(P, o->precision == FDE_MIXED_DF, 0, Y, P->v64[V_BY], nullptr, nullptr, s64.t1, s64.t2, st));
      info.fp64_matvecs += 1;
    }
    RK(clear_flag(P, st));
    CK(admm_post(P, A, Y, P->v64[V_BY], P->v64[V_BU], P->v64[V_R0], U, st));
    }
    const int flag = read_scalars(P, st);
    S.admm_iters = j + 1;
    res[0] = P->hscal[S_RES_EQ];
    res[1] = P->hscal[S_RES_Y];
    res[2] = P->hscal[S_RES_U];
    S.objective = P->hscal[S_OBJ];
    if (flag < 0) {
      status = flag;
      break;
    }
    if (o->fixed_iters) {
      status = FDE_OK;
      continue;
    }
    if (res[0] <= o->tol_admm && res[1] <= o->tol_admm && res[2] <= o->tol_admm) {
      status = FDE_OK;
      break;
    }
  }
  S.pcg_iters = info.pcg_iters;
  S.refine_steps = info.refine;
  S.recursive_steers = info.recursive;
  S.float_steers = info.float_steers;
  S.fp64_matvecs = info.fp64_matvecs;
  S.res_eq = res[0];
  S.res_y = res[1];
  S.res_u = res[2];
  if (y) CK(cudaMemcpyAsync(y, Y, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  if (u) CK(cudaMemcpyAsync(u, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  if (p) CK(cudaMemcpyAsync(p, A.p, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  if (zu) CK(cudaMemcpyAsync(zu, A.zu, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  if (stats) *stats = S;
  P->state_valid = status == FDE_OK || status == FDE_ENOCONV;
  return status;
}

int fde_admm_solve(fde_problem* P, const fde_admm_opts* o, const double* ybar, const double* g, const double* ya,
                   const double* yb, const double* ua, const double* ub, double ya_s, double yb_s, double ua_s,
                   double ub_s, double* y, double* u, double* p, double* zu, fde_admm_stats* stats, void* stream) {
  if (!y || !u) return FDE_EINVAL;
  return admm_solve_impl(P, o, ybar, g, ya, yb, ua, ub, ya_s, yb_s, ua_s, ub_s, y, u, p, zu, stats,
                         (cudaStream_t)stream);
}

int fde_admm_solve_host(fde_problem* P, const fde_admm_opts* o, const double* ybar, const double* g,
                        const double* ya, const double* yb, const double* ua, const double* ub, double ya_s,
                        double yb_s, double ua_s, double ub_s, double* y, double* u, double* p, double* zu,
                        fde_admm_stats* stats, void* stream) {
  if (!P || !valid_opts_for(P, o) || !ybar || !y || !u) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = P->N;
  // inputs: ybar, g, ya, yb, ua, ub -> their device copies (NULL stays NULL)
  const double* in[6] = {ybar, g, ya, yb, ua, ub};
  const double* dev_in[6] = {};
  for (int k = 0; k < 6; ++k) {
    if (!in[k]) continue;
    if (!P->stage[k]) CK(fde_alloc(P, reinterpret_cast<void**>(&P->stage[k]), sizeof(double) * N));
    dev_in[k] = P->stage[k];
  }
  cudaEvent_t ev[4] = {};
  for (int k = 0; k < 4; ++k) {
    const cudaError_t e = cudaEventCreate(&ev[k]);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaEventDestroy(ev[j]);
      return cuda_status(e);
    }
  }
  struct Events {
    cudaEvent_t* e;
    ~Events() {
      for (int k = 0; k < 4; ++k) cudaEventDestroy(e[k]);
    }
  } guard{ev};
  // once a copy is queued, every return waits for the stream: no queued copy may still
  // read or write the caller's host arrays after the call returns
  auto drain = [st](int status) {
    cudaStreamSynchronize(st);
    return status;
  };
#define CKD(expr)                                          \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return drain(cuda_status(_e));  \
  } while (0)
  CKD(cudaEventRecord(ev[0], st));
  for (int k = 0; k < 6; ++k)
    if (in[k]) CKD(copy_from_host(P->stage[k], in[k], N, st));
  CKD(cudaEventRecord(ev[1], st));
  fde_admm_stats S{};
  const int status = admm_solve_impl(P, o, dev_in[0], dev_in[1], dev_in[2], dev_in[3], dev_in[4], dev_in[5], ya_s,
                                     yb_s, ua_s, ub_s, nullptr, nullptr, nullptr, nullptr, &S, st);
  if (status != FDE_OK && status != FDE_ENOCONV) return drain(status);
  CKD(cudaEventRecord(ev[2], st));
  CKD(copy_to_host(y, P->v64[V_Y], N, st));
  CKD(copy_to_host(u, P->v64[V_U], N, st));
  if (p) CKD(copy_to_host(p, P->v64[V_P], N, st));
  if (zu) CKD(copy_to_host(zu, P->v64[V_ZU], N, st));
  CKD(cudaEventRecord(ev[3], st));
  CKD(cudaStreamSynchronize(st));
#undef CKD
  float ms_in = 0.f, ms_out = 0.f;
  CK(cudaEventElapsedTime(&ms_in, ev[0], ev[1]));
  CK(cudaEventElapsedTime(&ms_out, ev[2], ev[3]));
  S.copy_in_ms = ms_in;
  S.copy_out_ms = ms_out;
  if (stats) *stats = S;
  return status;
}

int fde_admm_get_iterates(const fde_problem* P, double* y, double* u, double* zy, double* zu, double* p, double* wy,
                          double* wu, void* stream) {
  if (!P) return FDE_EINVAL;
  if (!P->state_valid) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)P->N;
  double* out[7] = {y, u, zy, zu, p, wy, wu};
  const int slot[7] = {V_Y, V_U, V_ZY, V_ZU, V_P, V_WY, V_WU};
  for (int k = 0; k < 7; ++k)
    if (out[k]) CK(cudaMemcpyAsync(out[k], P->v64[slot[k]], bytes, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return FDE_OK;
}

int fde_admm_set_iterates(fde_problem* P, const double* y, const double* u, const double* zy, const double* zu,
                          const double* p, const double* wy, const double* wu, void* stream) {
  if (!P) return FDE_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = P->N;
  const double* in[7] = {y, u, zy, zu, p, wy, wu};
  const int slot[7] = {V_Y, V_U, V_ZY, V_ZU, V_P, V_WY, V_WU};
  P->state_valid = false;
  for (int k = 0; k < 7; ++k) {
    if (in[k]) {
      CK(cudaMemcpyAsync(P->v64[slot[k]], in[k], sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      CK(fill<double>(P->v64[slot[k]], 0.0, N, st));
    }
  }
  // a warm-started solve expects V_BY = B y of the starting y (double product)
  auto s = scratch64(P);
  CK(apply_B<double>(P, 0, P->v64[V_Y], P->v64[V_BY], nullptr, nullptr, nullptr, s.t1, s.t2, st));
  CK(cudaStreamSynchronize(st));
  P->last_rel0 = 1.0;
  P->state_valid = true;
  return FDE_OK;
}

int fde_admm_grad(fde_problem* P, const double* y, const double* ybar, const double* wy, double tol, double* dJ_dybar,
                  double* dJ_dcoef, double* p_out, void* stream) {
  if (!P || !y || !ybar || !dJ_dcoef) return FDE_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!P->ax[a].n_ok) return FDE_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const long long N = P->N;
  if (!(tol > 0)) tol = 1e-12;
  const double w1 = P->prm.weights == 0 ? 0.5 : 1.0;
  double* f = P->v64[V_C];
  double* rhs = P->v64[V_RHS];
  double* pv = P->v64[V_BU];  // not V_P: the ADMM iterates stay intact (warm start)
  auto s = scratch64(P);
  // f = -J1 (y - ybar) - w_y
  CK(grad_ybar(y, ybar, wy, 1.0, w1, (long long)(P->nt - 1) * P->nx * P->ny, N, dJ_dybar, f, st));
  // B B^T p = B f
  CK(apply_B<double>(P, 0, f, rhs, nullptr, nullptr, nullptr, s.t1, s.t2, st));
  auto A = [&](const double* x, double* out) -> int {
    CK(apply_B<double>(P, 1, x, s.w, nullptr, nullptr, nullptr, s.t1, s.t2, st));
    CK(apply_B<double>(P, 0, s.w, out, nullptr, nullptr, nullptr, s.t1, s.t2, st));
    return FDE_OK;
  };
  auto M = [&](const double* r, double* z) -> int {
    CK(apply_precond<double>(P, 0.0, 1.0, 1, r, z, P->spec64, st));
    return FDE_OK;
  };
  int it = 0;
  double rel = 0;
  const int sres = pcg<double>(P, A, M, rhs, pv, true, tol, 5000, P->v64[V_R], P->v64[V_Z], P->v64[V_D],
                               P->v64[V_SD], st, &it, &rel);
  if (sres != FDE_OK) return sres;
  // dJ/d{d+, d-} along x1 with L_x, L_x^T; dJ/d{e+, e-} along x2 with L_y, L_y^T
  double* t = P->v64[V_Q];
  for (int c = 0; c < 4; ++c) {
    const int axis = c < 2 ? 1 : 2;
    // the conjugate symbol gives L^T
    CK(apply_axis_raw<double>(P, axis, y, t, P->ax[axis].d.symL, c % 2, st));
    CK((dot<double, double>(P, pv, t, N, S_TMP0 + 0, FIN_STORE, st)));
    const int flag = read_scalars(P, st);
    if (flag < 0) return flag;
    dJ_dcoef[c] = -P->psi * P->hscal[S_TMP0];
  }
  if (p_out) CK(cudaMemcpyAsync(p_out, pv, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return FDE_OK;
}

}  // extern "C"

// ===========================================================================
// Host-sync-free solve and batches of uneven instances.
//
// enqueue_admm_fixed queues a whole mixed-precision ADMM solve of one problem
// on one stream without reading anything back: a fixed number of ADMM
// iterations, of residual evaluations per sub-problem (max_refine + 1) and of
// float PCG iterations per correction (max_pcg). Convergence is decided on
// the device: a PCG iteration whose residual already met its threshold does
// nothing (alpha = beta = 0), and a correction whose double residual already
// met the sub-problem tolerance is skipped. Because nothing waits on the host,
// the queued work can be captured into a CUDA graph; a batch captures one such
// solve per instance on its own stream, forked from and joined to one capture
// stream, so the graph has one independent branch per instance and a single
// cudaGraphLaunch runs the whole batch.
// ===========================================================================
namespace {

template <typename R, class OpA, class OpM>
int pcg_fixed(fde_problem* P, OpA A, OpM M, const R* b, R* x, double tol, int iters, R* r, R* z, R* d, R* q,
              cudaStream_t st) {
  const long long N = P->N;
  CK(fill<R>(x, (R)0, N, st));
  CK(copy<R>(r, b, N, st));
  CK((dot<R, R>(P, b, b, N, 0, FIN_BB_THR, st, tol)));
  CK((dot<R, R>(P, r, r, N, S_RR, FIN_STORE, st)));
  RK(M(r, z));
  CK((dot<R, R>(P, r, z, N, 0, FIN_RZ0, st)));
  CK(copy<R>(d, z, N, st));
  for (int it = 0; it < iters; ++it) {
    RK(A(d, q));
    CK((dot<R, R>(P, d, q, N, 0, FIN_ALPHA_MASK, st)));
    CK(pcg_xr<R>(P, x, r, d, q, N, st));
    RK(M(r, z));
    CK((dot<R, R>(P, r, z, N, 0, FIN_BETA_MASK, st)));
    CK(pcg_p<R>(P, d, z, N, st));
  }
  return FDE_OK;
}

// Queue one mixed ADMM solve with scalar bounds; outputs y, u (device, N).
int enqueue_admm_fixed(fde_problem* P, const fde_admm_opts* o, const double* ybar, double ya_s, double yb_s,
                       double ua_s, double ub_s, double* y, double* u, cudaStream_t st) {
  const long long N = P->N;
  const Diags dg = make_diags(P, o);
  AdmmArgs A = make_admm_args(P, o, dg, ybar, nullptr, nullptr, nullptr, nullptr, nullptr, ya_s, yb_s, ua_s, ub_s);
  double* Y = P->v64[V_Y];
  double* U = P->v64[V_U];
  // kernels only (no memset or memcpy nodes), so that the launches can also be recorded
  CK(fill<double>(P->dscal, 0.0, S_COUNT, st));
  for (int i : {V_Y, V_U, V_ZY, V_ZU, V_P, V_WY, V_WU, V_BY}) CK(fill<double>(P->v64[i], 0.0, N, st));
  const long long last = (long long)(P->nt - 1) * P->nx * P->ny;
  const SliceDiag one{{1.0, 1.0}};
  auto s32 = scratch32(P);
  auto s64 = scratch64(P);
  // float PCG transforms do no work once the PCG has converged; double products
  // after the first residual evaluation do none once the refinement has
  const Gate pcg_gate{P->dscal, 1}, ref_gate{P->dscal, 2};
  auto A32 = [&](const float* xx, float* out) { return op_S<float>(P, dg, xx, out, s32, st, pcg_gate); };
  auto M32 = [&](const float* rr, float* zz) { return op_M<float>(P, dg, rr, zz, st, pcg_gate); };
  const double tol = o->inner_tol > 0 ? o->inner_tol : 1e-8;
  const double inner = o->inner_tol_mixed > 0 ? o->inner_tol_mixed : 1e-4;
  const int evals = (o->max_refine > 0 ? o->max_refine : 2) + 1;
  const bool dfv = o->precision == FDE_MIXED_DFV;
  for (int j = 0; j < o->max_admm; ++j) {
    CK(admm_pre(A, P->v64[V_C], P->v64[V_BU], P->v64[V_R0], P->v64[V_Q], st));
    // ||rhs||^2 of rhs = c + B^T q, in float (only the stopping test uses it)
    CK(to_f32(P->v64[V_Q], P->v32[F_B], N, st));
    CK(to_f32(P->v64[V_C], P->v32[F_R], N, st));
    CK(apply_B<float>(P, 1, P->v32[F_B], P->v32[F_Z], nullptr, P->v32[F_R], &one, s32.t1, s32.t2, st));
    CK((dot<float, float>(P, P->v32[F_Z], P->v32[F_Z], N, S_TMP0, FIN_STORE, st)));
    for (int k = 0; k < evals; ++k) {
      // once converged, y and hence B y and the residual are unchanged: skip the products.
      // FDE_MIXED_DFV: double-float products except in the last evaluation, which runs in
      // double whether or not an earlier one met tol (the accepted residual and B y are double)
      const bool final_dfv = dfv && k == evals - 1;
      const bool dd = o->precision == FDE_MIXED_DF || (dfv && !final_dfv);
      const Gate g = (k > 0 && !final_dfv) ? ref_gate : Gate{};
      if (k > 0) CK(refine_B(P, dd, 0, Y, P->v64[V_BY], nullptr, nullptr, s64.t1, s64.t2, st, g));
      CK(fold(P->v64[V_BY], P->v64[V_Q], P->v64[V_C], Y, dg.M2inv.v, dg.M1.v, last, N, P->v64[V_SD], P->v64[V_Z],
              st));
      CK(refine_B(P, dd, 1, P->v64[V_SD], P->v64[V_R], P->v64[V_Z], &one, s64.t1, s64.t2, st, g));
      CK((dot<double, double>(P, P->v64[V_R], P->v64[V_R], N, 0, FIN_REFCHK, st, tol)));
      if (k == evals - 1) break;
      CK(to_f32_unless_conv(P, P->v64[V_R], P->v32[F_B], N, st));
      RK(pcg_fixed<float>(P, A32, M32, P->v32[F_B], P->v32[F_X], inner, o->max_pcg, P->v32[F_R], P->v32[F_Z],
                          P->v32[F_D], P->v32[F_Q], st));
      CK(add_f32_unless_conv(P, Y, P->v32[F_X], N, st));
    }
    CK(scalar_max(P, S_MAXREL, S_RELRES, st));
    CK(admm_post(P, A, Y, P->v64[V_BY], P->v64[V_BU], P->v64[V_R0], U, st));
  }
  CK(copy<double>(y, Y, N, st));
  CK(copy<double>(u, U, N, st));
  return FDE_OK;
}

void stats_from_scalars(const double* h, int admm_iters, fde_admm_stats* S) {
  *S = fde_admm_stats{};
  S->admm_iters = admm_iters;
  S->pcg_iters = (int)h[S_PCGIT];
  S->refine_steps = (int)h[S_REFINE];
  S->res_eq = h[S_RES_EQ];
  S->res_y = h[S_RES_Y];
  S->res_u = h[S_RES_U];
  S->objective = h[S_OBJ];
  S->max_sub_relres = h[S_MAXREL];
}

}  // namespace

struct fde_batch {
  int count = 0;
  fde_problem** probs = nullptr;
  cudaStream_t* streams = nullptr;
  cudaEvent_t* joins = nullptr;
  cudaEvent_t fork = nullptr;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec = nullptr;
  // arguments the current graph was captured with
  fde_admm_opts opts{};
  const double** ybar = nullptr;
  double** y = nullptr;
  double** u = nullptr;
  double* bounds = nullptr;  // 4 per instance: ya, yb, ua, ub
  long long kernels = 0;     // kernel nodes of the captured graph
  // persistent solve: the recorded launches and the arguments they were recorded with
  bool rec_valid = false;
  fde_admm_opts rec_opts{};
  std::vector<const double*> rec_ybar;
  std::vector<double*> rec_y, rec_u;
  std::vector<double> rec_bounds;
  std::vector<unsigned char> rec_cmds;  // host copy (stream replay)
  std::vector<long long> rec_off;
  size_t rec_smem = 0;
  unsigned char* d_cmds = nullptr;  // device copy of the commands
  long long* d_off = nullptr;
  int rec_steps = 0;                // launches per instance when all are alike (lockstep), else 0
  int* d_vstart = nullptr;          // lockstep: [steps][count + 1] prefix sums of the grids
  int* d_order = nullptr;
  void* d_state = nullptr;  // barrier counters, queue, slots, status
  int state_groups = 0;
};

extern "C" {

void fde_batch_destroy(fde_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int i = 0; i < b->count; ++i) {
    if (b->probs && b->probs[i]) fde_destroy(b->probs[i]);
    if (b->streams && b->streams[i]) cudaStreamDestroy(b->streams[i]);
    if (b->joins && b->joins[i]) cudaEventDestroy(b->joins[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->capture) cudaStreamDestroy(b->capture);
  if (b->d_cmds) cudaFree(b->d_cmds);
  if (b->d_off) cudaFree(b->d_off);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_state) cudaFree(b->d_state);
  if (b->d_vstart) cudaFree(b->d_vstart);
  delete[] b->probs;
  delete[] b->streams;
  delete[] b->joins;
  delete[] b->ybar;
  delete[] b->y;
  delete[] b->u;
  delete[] b->bounds;
  delete b;
}

int fde_batch_setup(const fde_params* params, int count, fde_batch** out, void* stream) {
  if (!params || !out || count < 1) return FDE_EINVAL;
  *out = nullptr;
  fde_batch* b = new fde_batch();
  b->count = count;
  b->probs = new fde_problem*[count]();
  b->streams = new cudaStream_t[count]();
  b->joins = new cudaEvent_t[count]();
  b->ybar = new const double*[count]();
  b->y = new double*[count]();
  b->u = new double*[count]();
  b->bounds = new double[4 * count]();
  for (int i = 0; i < count; ++i) {
    const int s = fde_setup(&params[i], &b->probs[i], stream);
    if (s != FDE_OK) {
      fde_batch_destroy(b);
      return s;
    }
    for (int a = 0; a < 3; ++a)
      if (!b->probs[i]->ax[a].n_ok) {
        fde_batch_destroy(b);
        return FDE_EUNSUPPORTED;
      }
    // FFT tiles of every instance picked by timing on its own sizes
    const int t = fde_autotune(b->probs[i], stream);
    if (t != FDE_OK) {
      fde_batch_destroy(b);
      return t;
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      fde_batch_destroy(b);
      return cuda_status(e);
    }
  }
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    fde_batch_destroy(b);
    return cuda_status(e);
  }
  *out = b;
  return FDE_OK;
}

long long fde_batch_instance_size(const fde_batch* b, int i) {
  return (b && i >= 0 && i < b->count) ? b->probs[i]->N : 0;
}

int fde_batch_admm_solve(fde_batch* b, const fde_admm_opts* o, const double* const* ybar, const double* ya,
                         const double* yb, const double* ua, const double* ub, double* const* y, double* const* u,
                         fde_admm_stats* stats, void* stream) {
  if (!b || !valid_opts(o) || !ybar || !y || !u) return FDE_EINVAL;
  if ((o->precision != FDE_MIXED && o->precision != FDE_MIXED_DF && o->precision != FDE_MIXED_DFV) ||
      o->max_admm < 1 || o->max_pcg < 1)
    return FDE_EINVAL;
  const int n = b->count;
  for (int i = 0; i < n; ++i)
    if (!valid_opts_for(b->probs[i], o)) return FDE_EINVAL;
  if (o->inner_solver != 0) return FDE_EUNSUPPORTED;  // the graph solve runs PCG only
  if (o->warm_start) return FDE_EUNSUPPORTED;         // a replayed graph starts from zero
  if (o->inner_x0) return FDE_EUNSUPPORTED;           // its sub-solves start from the previous iterate
  bool same = b->exec && std::memcmp(&b->opts, o, sizeof(*o)) == 0;
  for (int i = 0; i < n; ++i) {
    if (!ybar[i] || !y[i] || !u[i]) return FDE_EINVAL;
    const double bd[4] = {ya ? ya[i] : -INFINITY, yb ? yb[i] : INFINITY, ua ? ua[i] : -INFINITY,
                          ub ? ub[i] : INFINITY};
    for (int k = 0; k < 4; ++k) {
      if (std::isnan(bd[k])) return FDE_EINVAL;
      same = same && b->bounds[4 * i + k] == bd[k];
    }
    same = same && b->ybar[i] == ybar[i] && b->y[i] == y[i] && b->u[i] == u[i];
  }
  if (!same) {
    // capture the batch: fork from the capture stream, one branch per instance, join
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    const long long before = g_launches.load();
    CK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    int status = FDE_OK;
    cudaError_t e = cudaEventRecord(b->fork, b->capture);
    for (int i = 0; i < n && status == FDE_OK && e == cudaSuccess; ++i) {
      e = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
      if (e != cudaSuccess) break;
      const double bd[4] = {ya ? ya[i] : -INFINITY, yb ? yb[i] : INFINITY, ua ? ua[i] : -INFINITY,
                            ub ? ub[i] : INFINITY};
      status = enqueue_admm_fixed(b->probs[i], o, ybar[i], bd[0], bd[1], bd[2], bd[3], y[i], u[i], b->streams[i]);
      if (status != FDE_OK) break;
      e = cudaEventRecord(b->joins[i], b->streams[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, b->joins[i], 0);
      for (int k = 0; k < 4; ++k) b->bounds[4 * i + k] = bd[k];
      b->ybar[i] = ybar[i];
      b->y[i] = y[i];
      b->u[i] = u[i];
    }
    const cudaError_t e2 = cudaStreamEndCapture(b->capture, &graph);
    if (status != FDE_OK) {
      if (graph) cudaGraphDestroy(graph);
      return status;
    }
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_status(e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e);
    b->opts = *o;
    // captured launches did not run; each graph launch runs them all
    b->kernels = g_launches.load() - before;
    g_launches.fetch_sub(b->kernels);
  }
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaGraphLaunch(b->exec, st));
  note_launches((int)b->kernels);
  CK(cudaStreamSynchronize(st));
  int status = FDE_OK;
  for (int i = 0; i < n; ++i) {
    fde_problem* P = b->probs[i];
    CK(cudaMemcpy(P->hscal, P->dscal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost));
    if (stats) stats_from_scalars(P->hscal, o->max_admm, &stats[i]);
    const int flag = (int)P->hscal[S_FLAG];
    if (flag < 0 && status == FDE_OK) status = flag;
  }
  return status;
}


int fde_batch_admm_solve_persistent(fde_batch* b, const fde_admm_opts* o, const double* const* ybar,
                                    const double* ya, const double* yb, const double* ua, const double* ub,
                                    double* const* y, double* const* u, const fde_persist_cfg* cfg,
                                    fde_admm_stats* stats, fde_persist_info* info, void* stream) {
  if (info) {
    *info = fde_persist_info{};
    info->timeout_group = -1;
    info->timeout_command = -1;
  }
  if (!b || !valid_opts(o) || !ybar || !y || !u) return FDE_EINVAL;
  if (o->precision != FDE_MIXED || o->max_admm < 1 || o->max_pcg < 1) return FDE_EINVAL;
  if (cfg && (cfg->group_ctas < 0 || !(cfg->timeout_s >= 0.0) || cfg->stall_group < 0 || cfg->schedule < 0 ||
              cfg->schedule > 1))
    return FDE_EINVAL;
  const int n = b->count;
  for (int i = 0; i < n; ++i) {
    if (!valid_opts_for(b->probs[i], o)) return FDE_EINVAL;
    if (!ybar[i] || !y[i] || !u[i]) return FDE_EINVAL;
  }
  if (o->inner_solver != 0 || o->warm_start || o->inner_x0) return FDE_EUNSUPPORTED;
  auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
  for (int i = 0; i < n; ++i) {
    // the executor holds the power-of-two transforms of lengths up to 2048 (the
    // preconditioner transforms the exact axis lengths)
    const fde_problem* P = b->probs[i];
    if (P->ax[1].L > 2048 || P->ax[2].L > 2048 || (!P->euler && P->ax[0].L > 2048)) return FDE_EUNSUPPORTED;
    if (!pow2(P->nx) || !pow2(P->ny) || !pow2(P->nt)) return FDE_EUNSUPPORTED;
  }
  std::vector<double> bd(4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const double v[4] = {ya ? ya[i] : -INFINITY, yb ? yb[i] : INFINITY, ua ? ua[i] : -INFINITY, ub ? ub[i] : INFINITY};
    for (int k = 0; k < 4; ++k) {
      if (std::isnan(v[k])) return FDE_EINVAL;
      bd[4 * i + k] = v[k];
    }
  }
  bool same = b->rec_valid && std::memcmp(&b->rec_opts, o, sizeof(*o)) == 0 && b->rec_bounds == bd;
  for (int i = 0; i < n && same; ++i) same = b->rec_ybar[i] == ybar[i] && b->rec_y[i] == y[i] && b->rec_u[i] == u[i];
  if (!same) {
    // record every instance's launches; a stream capture around the recording
    // catches any launch that did not go through the recorder
    b->rec_valid = false;
    Recorder rec;
    std::vector<long long> off(n + 1, 0);
    CK(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    active_recorder() = &rec;
    int status = FDE_OK;
    for (int i = 0; i < n && status == FDE_OK; ++i) {
      off[i] = rec.count();
      status = enqueue_admm_fixed(b->probs[i], o, ybar[i], bd[4 * i], bd[4 * i + 1], bd[4 * i + 2], bd[4 * i + 3],
                                  y[i], u[i], b->capture);
    }
    active_recorder() = nullptr;
    off[n] = rec.count();
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->capture, &graph);
    size_t stray = 0;
    if (graph) {
      cudaGraphGetNodes(graph, nullptr, &stray);
      cudaGraphDestroy(graph);
    }
    if (status != FDE_OK) return status;
    CK(ec);
    if (rec.error) return FDE_EUNSUPPORTED;
    if (stray != 0) {
      std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%zu launches escaped the recorder", stray);
      return FDE_ECUDA;
    }
    // queue order: largest instances first
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return b->probs[a]->N > b->probs[c]->N; });
    // lockstep table: equal launch counts, prefix sums of the grids of each step
    const long long steps = n > 0 ? off[1] - off[0] : 0;
    bool alike = steps > 0 && steps < (1LL << 30);
    for (int i = 0; i < n && alike; ++i) alike = off[i + 1] - off[i] == steps;
    std::vector<int> vstart;
    if (alike) {
      vstart.assign((size_t)steps * (n + 1), 0);
      for (long long k = 0; k < steps && alike; ++k) {
        long long acc = 0;
        for (int i = 0; i < n; ++i) {
          CmdHeader h;
          std::memcpy(&h, rec.cmds.data() + (off[i] + k) * kCmdBytes, sizeof(h));
          vstart[k * (n + 1) + i] = (int)acc;
          acc += h.grid;
        }
        vstart[k * (n + 1) + n] = (int)acc;
        alike = acc < (1LL << 31);
      }
    }
    if (b->d_cmds) cudaFree(b->d_cmds);
    if (b->d_off) cudaFree(b->d_off);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_vstart) cudaFree(b->d_vstart);
    b->d_cmds = nullptr;
    b->d_off = nullptr;
    b->d_order = nullptr;
    b->d_vstart = nullptr;
    b->rec_steps = 0;
    if (alike) {
      if (cudaMalloc(&b->d_vstart, sizeof(int) * vstart.size()) != cudaSuccess) return FDE_ENOMEM;
      CK(cudaMemcpy(b->d_vstart, vstart.data(), sizeof(int) * vstart.size(), cudaMemcpyHostToDevice));
      b->rec_steps = (int)steps;
    }
    if (cudaMalloc(&b->d_cmds, rec.cmds.size()) != cudaSuccess ||
        cudaMalloc(&b->d_off, sizeof(long long) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&b->d_order, sizeof(int) * n) != cudaSuccess)
      return FDE_ENOMEM;
    CK(cudaMemcpy(b->d_cmds, rec.cmds.data(), rec.cmds.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_off, off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_order, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    b->rec_cmds.swap(rec.cmds);
    b->rec_off.swap(off);
    b->rec_smem = rec.max_smem;
    b->rec_opts = *o;
    b->rec_bounds = bd;
    b->rec_ybar.assign(ybar, ybar + n);
    b->rec_y.assign(y, y + n);
    b->rec_u.assign(u, u + n);
    b->rec_valid = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long long ncmd = b->rec_off[n];
  int cps = 0, dev = 0, sms = 0;
  CK(fde::persist_prepare(b->rec_smem, &cps));
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (cps < 1) return FDE_EUNSUPPORTED;
  const int total = cps * sms;
  const bool lockstep = b->rec_steps > 0 && !(cfg && cfg->schedule == 1);
  int gc = lockstep ? total : (cfg && cfg->group_ctas > 0) ? cfg->group_ctas : total / std::min(16, n);
  gc = std::max(1, std::min(gc, total));
  const int groups = total / gc;
  if (info) {
    info->commands = ncmd;
    info->groups = groups;
    info->group_ctas = gc;
    info->ctas_per_sm = cps;
    info->smem_bytes = (int)b->rec_smem;
    info->schedule = lockstep ? 0 : 1;
  }
  if (cfg && cfg->replay) {
    CK(fde::persist_replay(b->rec_cmds.data(), ncmd, st));
    CK(cudaStreamSynchronize(st));
  } else {
    // executor state: [groups] counters, queue, [groups] slots, then 4 status words
    const size_t bytes = sizeof(long long) * 4 + sizeof(unsigned) * groups + sizeof(int) * (groups + 1);
    if (b->state_groups < groups) {
      if (b->d_state) cudaFree(b->d_state);
      b->d_state = nullptr;
      b->state_groups = 0;
      if (cudaMalloc(&b->d_state, bytes) != cudaSuccess) return FDE_ENOMEM;
      b->state_groups = groups;
    }
    CK(cudaMemsetAsync(b->d_state, 0, bytes, st));
    fde::PersistLaunch pl{};
    pl.status = reinterpret_cast<long long*>(b->d_state);
    pl.bar = reinterpret_cast<unsigned*>(pl.status + 4);
    pl.queue = reinterpret_cast<int*>(pl.bar + groups);
    pl.slot = pl.queue + 1;
    pl.cmds = b->d_cmds;
    pl.off = b->d_off;
    pl.order = b->d_order;
    pl.count = n;
    pl.groups = groups;
    pl.group_ctas = gc;
    const double lim = (cfg && cfg->timeout_s > 0.0) ? cfg->timeout_s : 1.0;
    pl.timeout_ns = (unsigned long long)(lim * 1e9);
    pl.stall_group = (cfg && cfg->stall_group > 0) ? cfg->stall_group - 1 : -1;
    pl.steps = lockstep ? b->rec_steps : 0;
    pl.vstart = b->d_vstart;
    CK(fde::persist_run(pl, b->rec_smem, st));
    CK(cudaStreamSynchronize(st));
    long long hs[4];
    CK(cudaMemcpy(hs, pl.status, sizeof(hs), cudaMemcpyDeviceToHost));
    if (hs[0] != 0) {
      if (info) {
        info->timeout_group = (int)hs[1];
        info->timeout_command = hs[2];
      }
      return (int)hs[0];
    }
  }
  int status = FDE_OK;
  for (int i = 0; i < n; ++i) {
    fde_problem* P = b->probs[i];
    CK(cudaMemcpy(P->hscal, P->dscal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost));
    if (stats) stats_from_scalars(P->hscal, o->max_admm, &stats[i]);
    const int flag = (int)P->hscal[S_FLAG];
    if (flag < 0 && status == FDE_OK) status = flag;
  }
  return status;
}

}  // extern "C"
