// Common device helpers: complex arithmetic on float2/double2, type traits and
// the Stockham FFT passes used by every transform kernel of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace fde {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <> struct CplxOf<dd> { using type = dd2; };
template <typename R> using cplx = typename CplxOf<R>::type;

// population count on the device and on the host (index maps checked on the CPU)
__host__ __device__ __forceinline__ int fde_popc(unsigned x) {
#ifdef __CUDA_ARCH__
  return __popc(x);
#else
  return __builtin_popcount(x);
#endif
}

// read-only cached load
__device__ __forceinline__ float2 ldg_(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dd2 ldg_(const dd2* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dd2{dd(v.x, v.y), dd(v.z, v.w)};
}

// storage <-> compute conversions (identity unless double storage / double-float compute)
template <typename R, typename S> __device__ __forceinline__ R cvt_in(S v) { return (R)v; }
template <> __device__ __forceinline__ dd cvt_in<dd, double>(double v) { return to_dd(v); }
template <typename S, typename R> __device__ __forceinline__ S cvt_out(R v) { return (S)v; }
template <> __device__ __forceinline__ double cvt_out<double, dd>(dd v) { return to_double(v); }

template <typename C> __host__ __device__ __forceinline__ C mk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(C::x) s) { return mk<C>(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <typename C> __host__ __device__ __forceinline__ C mul_mi(C a) { return mk<C>(a.y, -a.x); }
template <typename C> __host__ __device__ __forceinline__ C mul_pi(C a) { return mk<C>(-a.y, a.x); }

// Factorisation of a transform length into Stockham radices (host-built, passed by value).
struct FftPlan {
  int L;          // transform length
  int nstages;    // number of radix passes
  int radix[16];  // radices in pass order, each in {2, 3, 4, 5, 7}
};

// One in-place Stockham pass (decimation in time, self-sorting) of radix RAD on
// `nlines` lines of length L stored at buf + line*lstride. The caller guarantees
// nlines * L <= EPT * blockDim.x, so every thread stages at most
// ceil(EPT / RAD) butterflies in registers; then the block synchronises, then the
// butterflies are computed and written back. Butterfly j reads entries
// j + r L/RAD, multiplies them by W_{Ns RAD}^{r (j mod Ns)}, applies the
// RAD-point DFT and writes entries (j div Ns) Ns RAD + (j mod Ns) + r Ns.
// tw holds W_L^m = exp(-2 pi i m / L), m in [0, L); inverse passes use conj.
template <typename R, int RAD, int EPT>
__device__ __forceinline__ void stockham_pass(cplx<R>* buf, int nlines, int lstride, int L, int Ns,
                                              const cplx<R>* __restrict__ tw, bool inv) {
  using C = cplx<R>;
  constexpr int MAXB = (EPT + RAD - 1) / RAD;
  const int nb = L / RAD;
  const int total = nlines * nb;
  C v[MAXB][RAD];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < total) {
      const int line = b / nb, j = b - line * nb;
      const C* src = buf + (size_t)line * lstride;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[q][r] = src[j + r * nb];
    }
  }
  __syncthreads();
  const int step = L / (Ns * RAD);
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = threadIdx.x + q * blockDim.x;
    if (b < total) {
      const int line = b / nb, j = b - line * nb;
      const int k = j % Ns;
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        C w = __ldg(&tw[r * k * step]);
        if (inv) w.y = -w.y;
        v[q][r] = cmul(v[q][r], w);
      }
      C o[RAD];
      if (RAD == 2) {
        o[0] = cadd(v[q][0], v[q][1]);
        o[1] = csub(v[q][0], v[q][1]);
      } else if (RAD == 4) {
        const C s02 = cadd(v[q][0], v[q][2]), d02 = csub(v[q][0], v[q][2]);
        const C s13 = cadd(v[q][1], v[q][3]), d13 = csub(v[q][1], v[q][3]);
        const C rot = inv ? mul_pi(d13) : mul_mi(d13);
        o[0] = cadd(s02, s13);
        o[2] = csub(s02, s13);
        o[1] = cadd(d02, rot);
        o[3] = csub(d02, rot);
      } else {
        // small odd radix: direct RAD-point DFT with W_RAD^m = W_L^{m L/RAD}
        const int rs = L / RAD;
#pragma unroll
        for (int kk = 0; kk < RAD; ++kk) {
          C acc = v[q][0];
#pragma unroll
          for (int r = 1; r < RAD; ++r) {
            C w = __ldg(&tw[((r * kk) % RAD) * rs]);
            if (inv) w.y = -w.y;
            acc = cadd(acc, cmul(v[q][r], w));
          }
          o[kk] = acc;
        }
      }
      C* dst = buf + (size_t)line * lstride + (j / Ns) * Ns * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) dst[r * Ns] = o[r];
    }
  }
  __syncthreads();
}

// Full transform of `nlines` lines in shared memory (unnormalised; inv selects
// the conjugate kernel). Must be called by every thread of the block, with
// nlines * L <= EPT * blockDim.x.
template <typename R, int EPT>
__device__ __forceinline__ void smem_fft(cplx<R>* buf, int nlines, int lstride, const FftPlan& pl,
                                         const cplx<R>* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < pl.nstages; ++s) {
    const int rad = pl.radix[s];
    switch (rad) {
      case 4: stockham_pass<R, 4, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv); break;
      case 2: stockham_pass<R, 2, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv); break;
      case 3: stockham_pass<R, 3, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv); break;
      case 5: stockham_pass<R, 5, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv); break;
      default: stockham_pass<R, 7, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv); break;
    }
    Ns *= rad;
  }
}

// smem_fft for power-of-two lengths (plans of radix-4 passes and at most one
// radix-2 pass): the same passes with only those two radices compiled in.
template <typename R, int EPT>
__device__ __forceinline__ void smem_fft_pow2(cplx<R>* buf, int nlines, int lstride, const FftPlan& pl,
                                              const cplx<R>* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < pl.nstages; ++s) {
    if (pl.radix[s] == 4) stockham_pass<R, 4, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv);
    else stockham_pass<R, 2, EPT>(buf, nlines, lstride, pl.L, Ns, tw, inv);
    Ns *= pl.radix[s];
  }
}

// The transform of the generic passes: inside the persistent executor (PS),
// whose problems have power-of-two axes, the power-of-two form.
template <bool PS, typename R, int EPT>
__device__ __forceinline__ void lines_fft(cplx<R>* buf, int nlines, int lstride, const FftPlan& pl,
                                          const cplx<R>* __restrict__ tw, bool inv) {
  if constexpr (PS) smem_fft_pow2<R, EPT>(buf, nlines, lstride, pl, tw, inv);
  else smem_fft<R, EPT>(buf, nlines, lstride, pl, tw, inv);
}

}  // namespace fde
