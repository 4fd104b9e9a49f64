// fde_matvec_noalloc: the Toeplitz product y = B x (or B^T x) in double
// precision for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available to it, e.g. a
// plug-in living inside a host framework whose caching allocator owns all of
// the device memory, or a latency-critical serving path that must not call
// cudaMalloc (the call can synchronise the device and can fail under memory
// pressure long after start-up). fde_setup cannot serve those callers because
// it allocates the problem's workspace.
//
// What it does instead: every buffer the product needs besides the caller's
// x and y - the intermediate of the x2 pass, the time pass's intermediate,
// the per-axis symbol and twiddle tables and the scratch of their set-up -
// lives in one file-scope device array of fixed size (about 18 MB), which
// every GPU that loads the library holds until the process exits. Problems
// with more than FDE_NOALLOC_MAX_N points are rejected with FDE_EUNSUPPORTED.
//
// Host code must not use the array's name as a device address (in host code it
// is only a host-side stand-in). The first call on each device looks up the
// array's device address with cudaGetSymbolAddress while that device is
// current, and also opts the transform kernels into their shared-memory size;
// make that first call before any stream capture. Every call rebuilds the tables
// in the array from `params` and overwrites the intermediates, so calls whose
// GPU work overlaps in time (two streams, two host threads) race on the array
// and give wrong results: serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "vec.h"

namespace fde {

// Kernels and their argument type defined in setup.cu (same definitions).
struct AxisSpec {
  int n, L;
  int kind;
  double order;
  double cp, cm;
  double hpow;
};
__global__ void k_twiddle(double2* __restrict__ out, int n);
__global__ void k_axis_columns(AxisSpec a, double* __restrict__ g, double* __restrict__ emb,
                               double* __restrict__ embL, double* __restrict__ tchan);
__global__ void k_dft(const double* __restrict__ in, int m, const double2* __restrict__ twm,
                      double2* __restrict__ out, double scale);
__global__ void k_halves(const double2* __restrict__ lam, int L, double2* __restrict__ sym);

namespace {

constexpr long long kMaxN = FDE_NOALLOC_MAX_N;
constexpr int kL = kMaxAxis;                        // largest embedding half-length
constexpr long long kTableDoubles = 3LL * 10 * kL;  // per axis: sym 2L + tw2 2L + twL L (complex)
constexpr long long kSetupDoubles = (kL + 2) + 2LL * kL + 2LL * kL + kL + 4LL * kL;
constexpr long long kScratchDoubles = 2 * kMaxN + kTableDoubles + kSetupDoubles;

}  // namespace

// The scratch array (device memory of every GPU that loads the library).
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

namespace {

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void* g_dev_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if ((e = toeplitz_set_smem_attrs()) != cudaSuccess) return e;
    g_dev_ptr[dev] = ptr;
  }
  *out = static_cast<double*>(g_dev_ptr[dev]);
  return cudaSuccess;
}

int next_pow2(int n) {
  int L = 1;
  while (L < n) L <<= 1;
  return L;
}

void pow2_plan(int L, FftPlan* pl) {
  std::memset(pl, 0, sizeof(*pl));
  pl->L = L;
  int m = L, s = 0;
  while (m % 4 == 0) { pl->radix[s++] = 4; m /= 4; }
  while (m % 2 == 0) { pl->radix[s++] = 2; m /= 2; }
  pl->nstages = s;
}

}  // namespace
}  // namespace fde

using namespace fde;

extern "C" int fde_matvec_noalloc(const fde_params* prm, int op, const double* x, double* y, void* stream) {
  if (!prm || !x || !y || x == y) return FDE_EINVAL;
  if (op != FDE_OP_B && op != FDE_OP_BT) return FDE_EINVAL;
  const fde_params& q = *prm;
  auto fin = [](double v) { return std::isfinite(v); };
  if (q.nx < 1 || q.ny < 1 || q.nt < 1) return FDE_EINVAL;
  if (!(fin(q.beta_x) && q.beta_x > 1 && q.beta_x < 2 && fin(q.beta_y) && q.beta_y > 1 && q.beta_y < 2))
    return FDE_EINVAL;
  if (!(fin(q.alpha_t) && q.alpha_t > 0 && q.alpha_t <= 1)) return FDE_EINVAL;
  if (!(fin(q.dp) && fin(q.dm) && fin(q.ep) && fin(q.em) && q.dp >= 0 && q.dm >= 0 && q.ep >= 0 && q.em >= 0))
    return FDE_EINVAL;
  if (!(fin(q.gamma) && q.gamma > 0) || !(fin(q.T) && q.T > 0)) return FDE_EINVAL;
  if ((q.weights != 0 && q.weights != 1) || (q.time_step_mode != 0 && q.time_step_mode != 1)) return FDE_EINVAL;
  if (q.nx > kMaxAxis || q.ny > kMaxAxis || q.nt > kMaxAxis) return FDE_EUNSUPPORTED;
  const long long N = (long long)q.nx * q.ny * q.nt;
  if (N > kMaxN) return FDE_EUNSUPPORTED;  // larger than the fixed scratch array holds

  double* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return FDE_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;

  // Problem description on the host stack; every device pointer points into the array.
  fde_problem P;
  P.prm = q;
  P.nx = q.nx;
  P.ny = q.ny;
  P.nt = q.nt;
  P.N = N;
  P.hx = 1.0 / (q.nx + 1);
  P.hy = 1.0 / (q.ny + 1);
  P.ht = q.time_step_mode == 0 ? q.T / q.nt : P.hx;
  P.psi = std::fmin(std::pow(P.ht, q.alpha_t), std::fmin(std::pow(P.hx, q.beta_x), std::pow(P.hy, q.beta_y)));
  P.euler = (q.alpha_t == 1.0);
  double* tmp1 = base;
  double* tmp2 = base + kMaxN;
  double* tables = base + 2 * kMaxN;
  double* setup = tables + kTableDoubles;
  double* g = setup;
  double* emb = g + (kL + 2);
  double* embL = emb + 2 * kL;
  double* tch = embL + 2 * kL;
  double2* lam2 = reinterpret_cast<double2*>(tch + kL);

  for (int axis = 0; axis < 3; ++axis) {
    Axis& A = P.ax[axis];
    A.n = axis == 0 ? q.nt : (axis == 1 ? q.nx : q.ny);
    A.L = next_pow2(A.n);
    pow2_plan(A.L, &A.planL);
    const int L = A.L;
    double2* t = reinterpret_cast<double2*>(tables + (long long)axis * 10 * kL);
    A.d.sym = t;
    A.d.tw2 = t + 2 * kL;
    A.d.twL = t + 4 * kL;
    AxisSpec s{};
    s.n = A.n;
    s.L = L;
    double coef;
    if (axis == 0) {
      s.kind = 0;
      s.order = q.alpha_t;
      s.hpow = std::pow(P.ht, -q.alpha_t);
      coef = P.psi;
    } else {
      s.kind = 1;
      s.order = axis == 1 ? q.beta_x : q.beta_y;
      s.cp = axis == 1 ? q.dp : q.ep;
      s.cm = axis == 1 ? q.dm : q.em;
      s.hpow = std::pow(axis == 1 ? P.hx : P.hy, -s.order);
      coef = -P.psi;
    }
    if (axis == 0 && P.euler) continue;  // the implicit-Euler time term needs no table
    // stream order keeps the shared set-up scratch consistent from one axis to the next
    k_twiddle<<<(2 * L + 255) / 256, 256, 0, st>>>(A.d.tw2, 2 * L);
    k_twiddle<<<(L + 255) / 256, 256, 0, st>>>(A.d.twL, L);
    k_axis_columns<<<1, 1024, 0, st>>>(s, g, emb, embL, tch);
    k_dft<<<(2 * L + 127) / 128, 128, 0, st>>>(emb, 2 * L, A.d.tw2, lam2, coef / (2.0 * L));
    k_halves<<<(2 * L + 255) / 256, 256, 0, st>>>(lam2, L, A.d.sym);
    note_launches(5);
    if ((e = cudaGetLastError()) != cudaSuccess) return FDE_ECUDA;
  }
  e = apply_B<double>(&P, op == FDE_OP_BT, x, y, nullptr, nullptr, nullptr, tmp1, tmp2, st);
  return e == cudaSuccess ? FDE_OK : FDE_ECUDA;
}
