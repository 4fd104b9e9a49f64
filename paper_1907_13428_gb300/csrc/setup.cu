// Set-up kernels: Gruenwald-Letnikov weights (Eq. C_GL), the Toeplitz entries
// of the time matrix (Eq. Caputo matrix) and of X = d+ L + d- L^T,
// Y = e+ L + e- L^T (Eq. RL_GL, Eq. Riesz matrix generalised to two sides),
// their circulant embeddings and T. Chan circulants (Eq. level 1 circulant
// optimization problem), and the DFTs of both (Section 5). All in double; the
// float tables are rounded copies.
#include <cmath>
#include <cstring>

#include "internal.h"

namespace fde {

// W_n^m = exp(-2 pi i m / n), m in [0, n).
__global__ void k_twiddle(double2* __restrict__ out, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    out[m] = make_double2(c, -s);
  }
}

struct AxisSpec {
  int n, L;
  int kind;       // 0: time (Caputo weights of order alpha), 1: space (two-sided shifted GL)
  double order;   // alpha_t or beta
  double cp, cm;  // coefficients of L and L^T (space only)
  double hpow;    // 1 / h^order
};

// One block. Weights by the recurrence g_0 = 1, g_k = (1 - (order+1)/k) g_{k-1}
// (thread 0), then the columns:
//   emb[0..2L): first column of the order-2L circulant embedding of T,
//   embL[0..2L): same for the one-sided L alone (space axes, for the gradient),
//   tchan[0..n): c_i = ((n - i) t_i + i t_{i-n}) / n.
__global__ void k_axis_columns(AxisSpec a, double* __restrict__ g, double* __restrict__ emb,
                               double* __restrict__ embL, double* __restrict__ tchan) {
  if (threadIdx.x == 0) {
    g[0] = 1.0;
    for (int k = 1; k <= a.n; ++k) g[k] = (1.0 - (a.order + 1.0) / (double)k) * g[k - 1];
  }
  __syncthreads();
  // Toeplitz entry t_k = T[i][i-k], k in [-(n-1), n-1]
  auto entry = [&](int k) -> double {
    if (a.kind == 0) return (k >= 0 && k < a.n) ? g[k] * a.hpow : 0.0;
    double v = 0.0;
    if (k + 1 >= 0 && k + 1 <= a.n) v += a.cp * g[k + 1];
    if (1 - k >= 0 && 1 - k <= a.n) v += a.cm * g[1 - k];
    return v * a.hpow;
  };
  auto entryL = [&](int k) -> double { return (k + 1 >= 0 && k + 1 <= a.n) ? g[k + 1] * a.hpow : 0.0; };
  const int m = 2 * a.L;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    int k = 0;
    bool used = false;
    if (j < a.n) {
      k = j;
      used = true;
    } else if (j > m - a.n) {
      k = j - m;
      used = true;
    }
    emb[j] = used ? entry(k) : 0.0;
    embL[j] = (used && a.kind == 1) ? entryL(k) : 0.0;
  }
  for (int i = threadIdx.x; i < a.n; i += blockDim.x) {
    const double ti = entry(i);
    const double tm = (i > 0) ? entry(i - a.n) : 0.0;
    tchan[i] = ((double)(a.n - i) * ti + (double)i * tm) / (double)a.n;
  }
}

// out[k] = scale * sum_j in[j] W_m^{j k}  (direct DFT with an exact twiddle index)
__global__ void k_dft(const double* __restrict__ in, int m, const double2* __restrict__ twm, double2* __restrict__ out,
                      double scale) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < m; ++j) {
      const double v = in[j];
      if (v == 0.0) continue;
      const double2 w = twm[(int)(((long long)j * k) % m)];
      re += v * w.x;
      im += v * w.y;
    }
    out[k] = make_double2(re * scale, im * scale);
  }
}

// sym[s*L + k] = lam[2k + s]
__global__ void k_halves(const double2* __restrict__ lam, int L, double2* __restrict__ sym) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * L; e += gridDim.x * blockDim.x) {
    const int s = e / L, k = e - s * L;
    sym[e] = lam[2 * k + s];
  }
}

// out[e] = in[e] + (d, 0): adds a real constant to every symbol entry (a
// diagonal shift of the Toeplitz factor).
__global__ void k_shift(const double2* __restrict__ in, double d, double2* __restrict__ out, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[e] = make_double2(in[e].x + d, in[e].y);
}

__global__ void k_to_float2(const double2* __restrict__ in, float2* __restrict__ out, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[e] = make_float2((float)in[e].x, (float)in[e].y);
}

__global__ void k_to_dd2(const double2* __restrict__ in, dd2* __restrict__ out, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[e] = dd2{to_dd(in[e].x), to_dd(in[e].y)};
}

static int next_pow2(int n) {
  int L = 1;
  while (L < n) L <<= 1;
  return L;
}

// Stockham radices for length n; returns false if n has a prime factor > 7.
static bool make_plan(int n, FftPlan* pl) {
  std::memset(pl, 0, sizeof(*pl));
  pl->L = n;
  int m = n, s = 0;
  while (m % 4 == 0) { pl->radix[s++] = 4; m /= 4; }
  while (m % 2 == 0) { pl->radix[s++] = 2; m /= 2; }
  const int odd[3] = {3, 5, 7};
  for (int q : odd)
    while (m % q == 0) { pl->radix[s++] = q; m /= q; }
  pl->nstages = s;
  return m == 1;
}

}  // namespace fde

// Allocation helper shared with api.cu.
extern cudaError_t fde_alloc(fde_problem* P, void** ptr, size_t bytes);

namespace fde {

cudaError_t setup_axis_tables(fde_problem* P, cudaStream_t st) {
  cudaError_t e;
  // scratch for one axis at a time (owned by the problem, freed with it)
  void* p;
  const int maxL = kMaxAxis;
  if ((e = fde_alloc(P, &p, sizeof(double) * (maxL + 2)))) return e;
  double* g = (double*)p;
  if ((e = fde_alloc(P, &p, sizeof(double) * 2 * maxL))) return e;
  double* emb = (double*)p;
  if ((e = fde_alloc(P, &p, sizeof(double) * 2 * maxL))) return e;
  double* embL = (double*)p;
  if ((e = fde_alloc(P, &p, sizeof(double) * maxL))) return e;
  double* tch = (double*)p;
  if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * maxL))) return e;
  double2* lam2 = (double2*)p;
  if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * maxL))) return e;
  double2* lamL = (double2*)p;

  for (int axis = 0; axis < 3; ++axis) {
    Axis& A = P->ax[axis];
    A.n = axis == 0 ? P->nt : (axis == 1 ? P->nx : P->ny);
    A.L = next_pow2(A.n);
    make_plan(A.L, &A.planL);
    A.n_ok = make_plan(A.n, &A.plann);
    const int L = A.L, n = A.n;
    AxisSpec s{};
    s.n = n;
    s.L = L;
    double coef;
    if (axis == 0) {
      s.kind = 0;
      s.order = P->prm.alpha_t;
      s.hpow = std::pow(P->ht, -P->prm.alpha_t);
      coef = P->psi;
    } else {
      s.kind = 1;
      s.order = axis == 1 ? P->prm.beta_x : P->prm.beta_y;
      s.cp = axis == 1 ? P->prm.dp : P->prm.ep;
      s.cm = axis == 1 ? P->prm.dm : P->prm.em;
      s.hpow = std::pow(axis == 1 ? P->hx : P->hy, -s.order);
      coef = -P->psi;
    }
    // tables (double)
    if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * L))) return e;
    A.d.sym = (double2*)p;
    if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * L))) return e;
    A.d.tw2 = (double2*)p;
    if ((e = fde_alloc(P, &p, sizeof(double2) * L))) return e;
    A.d.twL = (double2*)p;
    if ((e = fde_alloc(P, &p, sizeof(double2) * n))) return e;
    A.d.lam = (double2*)p;
    if ((e = fde_alloc(P, &p, sizeof(double2) * n))) return e;
    A.d.twn = (double2*)p;
    if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * L))) return e;
    A.d.symL = (double2*)p;
    // float copies
    if ((e = fde_alloc(P, &p, sizeof(float2) * 2 * L))) return e;
    A.f.sym = (float2*)p;
    if ((e = fde_alloc(P, &p, sizeof(float2) * 2 * L))) return e;
    A.f.tw2 = (float2*)p;
    if ((e = fde_alloc(P, &p, sizeof(float2) * L))) return e;
    A.f.twL = (float2*)p;
    if ((e = fde_alloc(P, &p, sizeof(float2) * n))) return e;
    A.f.lam = (float2*)p;
    if ((e = fde_alloc(P, &p, sizeof(float2) * n))) return e;
    A.f.twn = (float2*)p;

    k_twiddle<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.tw2, 2 * L);
  note_launches(1);
    k_twiddle<<<(L + 255) / 256, 256, 0, st>>>(A.d.twL, L);
  note_launches(1);
    k_twiddle<<<(n + 255) / 256, 256, 0, st>>>(A.d.twn, n);
  note_launches(1);
    k_axis_columns<<<1, 1024, 0, st>>>(s, g, emb, embL, tch);
  note_launches(1);
    // embedding symbol of order 2L, scaled by coef / (2L), split into halves
    k_dft<<<(2 * L + 127) / 128, 128, 0, st>>>(emb, 2 * L, A.d.tw2, lam2, coef / (2.0 * L));
  note_launches(1);
    k_halves<<<(2 * L + 255) / 256, 256, 0, st>>>(lam2, L, A.d.sym);
  note_launches(1);
    // one-sided L alone (unscaled apart from 1/(2L))
    k_dft<<<(2 * L + 127) / 128, 128, 0, st>>>(embL, 2 * L, A.d.tw2, lamL, 1.0 / (2.0 * L));
  note_launches(1);
    k_halves<<<(2 * L + 255) / 256, 256, 0, st>>>(lamL, L, A.d.symL);
  note_launches(1);
    if (axis == 1 && P->euler) {
      // +psi/h_t x_t of the implicit-Euler term as a diagonal shift of the x1 factor
      if ((e = fde_alloc(P, &p, sizeof(double2) * 2 * L))) return e;
      A.d.symD = (double2*)p;
      if ((e = fde_alloc(P, &p, sizeof(float2) * 2 * L))) return e;
      A.f.symD = (float2*)p;
      k_shift<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.sym, (P->psi / P->ht) / (2.0 * L), A.d.symD, 2 * L);
      note_launches(1);
      k_to_float2<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.symD, A.f.symD, 2 * L);
      note_launches(1);
    }
    // T. Chan eigenvalues of order n
    k_dft<<<(n + 127) / 128, 128, 0, st>>>(tch, n, A.d.twn, A.d.lam, 1.0);
  note_launches(1);
    k_to_float2<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.sym, A.f.sym, 2 * L);
  note_launches(1);
    k_to_float2<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.tw2, A.f.tw2, 2 * L);
  note_launches(1);
    k_to_float2<<<(L + 255) / 256, 256, 0, st>>>(A.d.twL, A.f.twL, L);
  note_launches(1);
    k_to_float2<<<(n + 255) / 256, 256, 0, st>>>(A.d.lam, A.f.lam, n);
  note_launches(1);
    k_to_float2<<<(n + 255) / 256, 256, 0, st>>>(A.d.twn, A.f.twn, n);
  note_launches(1);
    if (L >= 16) {
      // double-float copies for the register kernels of apply_B_df
      const double2* src[4] = {A.d.sym, A.d.tw2, A.d.twL, A.d.symD};
      dd2** dst[4] = {&A.q.sym, &A.q.tw2, &A.q.twL, &A.q.symD};
      const int len[4] = {2 * L, 2 * L, L, 2 * L};
      for (int i = 0; i < 4; ++i) {
        if (!src[i]) continue;
        if ((e = fde_alloc(P, &p, sizeof(dd2) * len[i]))) return e;
        *dst[i] = (dd2*)p;
        k_to_dd2<<<(len[i] + 255) / 256, 256, 0, st>>>(src[i], *dst[i], len[i]);
        note_launches(1);
      }
    }
    if ((e = cudaGetLastError())) return e;
    // scratch is reused by the next axis: wait for this one
    if ((e = cudaStreamSynchronize(st))) return e;
  }
  return cudaSuccess;
}

}  // namespace fde
