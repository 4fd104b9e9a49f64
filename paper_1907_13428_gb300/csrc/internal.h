// Internal host-side declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/fde.h"
#include "common.cuh"
#include "op.cuh"

namespace fde {

constexpr int kMaxAxis = 4096;

// Device tables of one axis in one precision.
template <typename R> struct AxisTables {
  cplx<R>* sym = nullptr;  // [2][L]: halves lambda_emb[2k+s] of the circulant embedding symbol,
                           //         pre-scaled by coef/(2L) (coef = -psi in space, +psi in time)
  cplx<R>* tw2 = nullptr;  // W_{2L}^m, m in [0, 2L): pre/post twists of the odd half
  cplx<R>* twL = nullptr;  // W_L^m, m in [0, L): FFT table of the embedding length
  cplx<R>* lam = nullptr;  // T. Chan circulant eigenvalues, length n (unscaled)
  cplx<R>* twn = nullptr;  // W_n^m, m in [0, n): FFT table of the exact length
  cplx<R>* symD = nullptr; // [2][L]: x1 axis, implicit Euler: sym + (psi/h_t)/(2L), i.e. the
                           //         symbol of X shifted by the diagonal that carries +psi/h_t x_t
  cplx<R>* symL = nullptr; // [2][L]: embedding symbol halves of the one-sided L alone,
                           //         scaled by 1/(2L) (space axes, double only; gradient)
};

struct Axis {
  int n = 0;        // points on this axis
  int L = 0;        // embedding half-length: smallest power of two >= n
  FftPlan planL{};  // radix plan of L
  FftPlan plann{};  // radix plan of n (preconditioner)
  bool n_ok = false;  // n factors into 2, 3, 5, 7
  AxisTables<double> d;
  AxisTables<float> f;
  AxisTables<dd> q;   // double-float copies of sym, tw2, twL, symD (L >= 16 only)
};

// Device-side gate of a transform launch in the host-sync-free solve: the
// kernel returns at once when its instance's PCG has converged (mode 1:
// dscal[S_RR] <= dscal[S_THR]) or its refinement has (mode 2: dscal[S_CONV]).
// mode 0: always run. The slot indices are those of fde::Scal.
struct Gate {
  const double* dscal = nullptr;
  int mode = 0;
};

// Per-time-slice diagonal: value on slices 0..nt-2 and on the last slice.
struct SliceDiag {
  double v[2];
};

}  // namespace fde

struct fde_problem {
  fde_params prm;
  long long N = 0;
  int nx = 0, ny = 0, nt = 0;
  double hx = 0, hy = 0, ht = 0, psi = 0;
  bool euler = true;   // alpha_t == 1: the time term is the two-point backward difference
  int H = 0, Hp = 0;   // half-spectrum length ny/2+1 and its padded row stride
  fde::Axis ax[3];     // 0: time, 1: x1, 2: x2
  // workspace (device)
  double* v64[24] = {};
  float* v32[12] = {};
  double2* spec64 = nullptr;
  float2* spec32 = nullptr;
  double* stage[6] = {};       // device copies of the host inputs of fde_admm_solve_host, allocated on first use
  double* mr64 = nullptr;      // saddle-point (MINRES) workspace, allocated on first use
  float* mr32 = nullptr;
  double* partials = nullptr;  // reduction partial sums
  double* dscal = nullptr;     // device scalars
  double* hscal = nullptr;     // pinned host mirror of a few scalars
  int npartials = 0;
  void* allocs[128] = {};
  int nallocs = 0;
  // FFT tile choice of the float register kernels (threads per CTA), set by fde_autotune
  int rows_nt32 = 256;  // x2 pass: 128, 256 or 512 (row pairs per CTA = threads / (L/16))
  int axis_nt32 = 512;  // x1 / t pass: 256 or 512 (column pairs per CTA = threads / (L/16))
  // negative values: the split-halves kernels with that many threads
  // tile choice of the double-float passes: 256 (both halves per thread) or split (-256/-512 x2, -512 x1)
  int rows_ntdd = 256;
  int axis_ntdd = 256;
  // tile choice of the double passes: the same values as the double-float ones
  int rows_nt64 = 256;
  int axis_nt64 = 256;
  bool state_valid = false;  // the ADMM iterates hold the end of a previous solve (warm start)
  double last_rel0 = 1.0;    // relative residual of the previous sub-problem's warm start (FDE_MIXED_DFV)
};

namespace fde {

// Process-wide count of kernel launches issued by this library (diagnostics).
void note_launches(int n);

// Device-scalar slots in fde_problem::dscal.
enum Scal {
  S_RZ = 0, S_RZ_NEW, S_PQ, S_ALPHA, S_BETA, S_RR, S_BB, S_TMP0, S_TMP1, S_TMP2,
  S_RES_EQ, S_RES_Y, S_RES_U, S_OBJ, S_FLAG,
  // device-side control of the host-sync-free (graph) solve
  S_THR,       // PCG stop threshold tol^2 ||b||^2
  S_CONV,      // 1 when the current sub-problem's double residual met its tolerance
  S_RELRES,    // last double relative residual of the sub-problem
  S_MAXREL,    // largest final relative residual over the sub-problems
  S_PCGIT,     // PCG iterations that did work (counted on the device)
  S_REFINE,    // refinement corrections that did work
  S_COUNT = 32
};

// PS: the scalars may have been written earlier in the same (persistent) kernel.
template <bool PS = false> __device__ __forceinline__ bool gate_closed(const Gate& g) {
  if (g.mode == 1) return ldv<PS>(g.dscal + S_RR) <= ldv<PS>(g.dscal + S_THR);
  if (g.mode == 2) return ldv<PS>(g.dscal + S_CONV) != 0.0;
  return false;
}

// ---- launchers (each returns cudaError_t of the launch) ----

// Set-up of the axis tables (setup.cu).
cudaError_t setup_axis_tables(fde_problem* P, cudaStream_t st);

// Toeplitz operator passes (toeplitz.cu).
//   op: 0 = B, 1 = B^T. If dscale != null the result is multiplied per slice
//   (M2^-1 for S). If addv != null, addc(t) * addv is added after that.
template <typename R>
cudaError_t apply_B(fde_problem* P, int transpose, const R* x, R* y, const SliceDiag* dscale,
                    const R* addv, const SliceDiag* addc, R* tmp1, R* tmp2, cudaStream_t st, Gate gate = {});
// apply_B<double> with the transforms in double-float arithmetic (about 48
// significand bits at float speed); vectors, epilogue and tables stay double.
cudaError_t apply_B_df(fde_problem* P, int transpose, const double* x, double* y, const SliceDiag* dscale,
                       const double* addv, const SliceDiag* addc, double* tmp1, double* tmp2, cudaStream_t st,
                       Gate gate = {});
// y = S x = M1 x + B^T (M2^-1 B x), using w (N) and tmp1, tmp2 (N) as scratch.
template <typename R>
cudaError_t apply_S(fde_problem* P, const SliceDiag& M1, const SliceDiag& M2inv, const R* x, R* y,
                    R* w, R* tmp1, R* tmp2, cudaStream_t st, Gate gate = {});
// One spatial factor along one axis (1: x1, 2: x2) with the given symbol
// halves (e.g. AxisTables::symL for the one-sided L), no time term, for the gradient.
template <typename R>
cudaError_t apply_axis_raw(fde_problem* P, int axis, const R* x, R* y, const cplx<R>* sym, int conj_sym,
                           cudaStream_t st);

// apply_axis_raw<double> with the axis' own symbol in double-float arithmetic.
cudaError_t apply_axis_raw_df(fde_problem* P, int axis, const double* x, double* y, int conj_sym, cudaStream_t st);

// n doubles between a host buffer and device memory (hostio.cu): a copy kernel
// through the mapped address of pinned memory, cudaMemcpyAsync for pageable memory.
cudaError_t copy_from_host(double* dev_dst, const double* host_src, long long n, cudaStream_t st);
cudaError_t copy_to_host(double* host_dst, const double* dev_src, long long n, cudaStream_t st);

// Times the float and double-float tile variants of the x2 and x1 passes on this
// problem (x, y and xd, yd: scratch vectors of length N) and keeps the fastest in
// P (toeplitz.cu).
cudaError_t autotune_tiles(fde_problem* P, const float* x, float* y, const double* xd, double* yd, cudaStream_t st);

// Preconditioner (precond.cu): z = S~^-1 r (r and z may alias). mode 0: S~
// (m1, m2), sigma = m1 + |Lambda|^2 / m2 + cre Re(Lambda) (cre != 0: the matching
// approximation S^); mode 1: (C3 C3^T)^-1 (the adjoint normal-equation preconditioner).
template <typename R>
cudaError_t apply_precond(fde_problem* P, double m1, double m2, int mode, const R* r, R* z,
                          cplx<R>* spec, cudaStream_t st, Gate gate = {}, double cre = 0.0);


}  // namespace fde
