// Register-resident Stockham FFT for power-of-two lengths 16 <= L <= 4096.
//
// A line of length L is held by T = L/16 threads, 16 complex values each.
// The forward transform runs radix-16 passes and a last pass of radix
// RL = L / 16^(P-1) in {2, 4, 8, 16}; the inverse runs the radices in the
// opposite order. With the Stockham indexing (butterfly j reads j + r L/R,
// multiplies by W_{Ns R}^{r (j mod Ns)}, writes (j div Ns) Ns R + (j mod Ns) + r Ns)
// the registers of thread t hold
//   before the forward transform and after the inverse: positions t + r T;
//   after the forward transform and before the inverse:  positions
//     t + T q + r L/RL  (butterfly q < 16/RL, element r < RL),
// so the last forward pass and the first inverse pass touch the same values
// and a pointwise multiply in frequency needs no data exchange. Between the
// other passes the values go through shared memory (write, barrier, read,
// barrier). P = 1, 2, 3 passes for L = 16, 32..256, 512..4096.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace fde {

// Twiddle-table access through the read-only cache (overloadable for other
// table placements).
template <typename C> __device__ __forceinline__ C tw_get(const C* __restrict__ p, int i) { return ldg_(p + i); }

template <int L> struct RfShape {
  static constexpr int T = L / 16;
  static constexpr int P = (L <= 16) ? 1 : (L <= 256 ? 2 : 3);
  static constexpr int RL = (P == 1) ? 16 : (P == 2 ? L / 16 : L / 256);
  static_assert(L >= 16 && L <= 4096 && (L & (L - 1)) == 0, "power of two in [16, 4096]");
};

// a * W_16^M (forward) or a * conj(W_16^M) (inverse), W_16 = exp(-2 pi i / 16)
template <typename C, int M, bool INV>
__host__ __device__ __forceinline__ C w16(C a) {
  using R = decltype(C::x);
  constexpr int m = M & 15;
  constexpr R h = (R)0.70710678118654752440;
  constexpr R c1 = (R)0.92387953251128675613;  // cos(pi/8)
  constexpr R s1 = (R)0.38268343236508977173;  // sin(pi/8)
  if constexpr (m == 0) {
    return a;
  } else if constexpr (m == 8) {
    return mk<C>(-a.x, -a.y);
  } else if constexpr (m == 4) {
    return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
  } else if constexpr (m == 12) {
    return INV ? mk<C>(a.y, -a.x) : mk<C>(-a.y, a.x);
  } else {
    // cos(pi m / 8), sin(pi m / 8) for the remaining m
    constexpr R cs[16] = {1, c1, h, s1, 0, -s1, -h, -c1, -1, -c1, -h, -s1, 0, s1, h, c1};
    constexpr R sn[16] = {0, s1, h, c1, 1, c1, h, s1, 0, -s1, -h, -c1, -1, -c1, -h, -s1};
    constexpr R c = cs[m];
    constexpr R s = INV ? -sn[m] : sn[m];
    // (a.x + i a.y)(c - i s)
    return mk<C>(a.x * c + a.y * s, a.y * c - a.x * s);
  }
}

template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft2(C& a0, C& a1) {
  const C t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
  const C s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const C s13 = cadd(a1, a3), d13 = csub(a1, a3);
  const C rot = INV ? mul_pi(d13) : mul_mi(d13);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, rot);
  a3 = csub(d02, rot);
}

// in-place 8-point DFT of v[0..7] (natural order in and out)
template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft8(C* v) {
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<C, INV>(e0, e1, e2, e3);
  dft4<C, INV>(o0, o1, o2, o3);
  o1 = w16<C, 2, INV>(o1);
  o2 = w16<C, 4, INV>(o2);
  o3 = w16<C, 6, INV>(o3);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// in-place 16-point DFT of v[0..15]: 4-point DFTs over n1 (n = n2 + 4 n1),
// twiddles W16^{n2 k1}, 4-point DFTs over n2; output index k1 + 4 k2.
template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft16(C* v) {
  dft4<C, INV>(v[0], v[4], v[8], v[12]);
  dft4<C, INV>(v[1], v[5], v[9], v[13]);
  dft4<C, INV>(v[2], v[6], v[10], v[14]);
  dft4<C, INV>(v[3], v[7], v[11], v[15]);
  // b[n2][k1] sits at v[n2 + 4 k1]
  v[5] = w16<C, 1, INV>(v[5]);
  v[9] = w16<C, 2, INV>(v[9]);
  v[13] = w16<C, 3, INV>(v[13]);
  v[6] = w16<C, 2, INV>(v[6]);
  v[10] = w16<C, 4, INV>(v[10]);
  v[14] = w16<C, 6, INV>(v[14]);
  v[7] = w16<C, 3, INV>(v[7]);
  v[11] = w16<C, 6, INV>(v[11]);
  v[15] = w16<C, 9, INV>(v[15]);
  // outer DFTs over n2 for each k1: inputs v[4 k1 + n2]
  dft4<C, INV>(v[0], v[1], v[2], v[3]);
  dft4<C, INV>(v[4], v[5], v[6], v[7]);
  dft4<C, INV>(v[8], v[9], v[10], v[11]);
  dft4<C, INV>(v[12], v[13], v[14], v[15]);
  // now X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4x4 index
  C t;
  t = v[1]; v[1] = v[4]; v[4] = t;
  t = v[2]; v[2] = v[8]; v[8] = t;
  t = v[3]; v[3] = v[12]; v[12] = t;
  t = v[6]; v[6] = v[9]; v[9] = t;
  t = v[7]; v[7] = v[13]; v[13] = t;
  t = v[11]; v[11] = v[14]; v[14] = t;
}

__host__ __device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }

// The second-stage 4-point DFT of one row k1 of dft16 with its three twiddled
// inputs given as scale * (U-part, V-part): s02 = a0 + f2 a2, d02 = a0 - f2 a2
// (a2 = f2 * A2, f2 = 0 for an untwiddled a2 taken as is), s13 = f13 U,
// d13 = f13 V; the scalings f2, f13 fold into the additions as FMAs.
template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft4_scaled(C& o0, C& o1, C& o2, C& o3, C s02, C d02, C U, C V,
                                                     decltype(C::x) f13) {
  using R = decltype(C::x);
  constexpr R sg = INV ? (R)-1 : (R)1;
  // rot = (sg d13.y, -sg d13.x) = f13 (sg V.y, -sg V.x)
  o0 = mk<C>(fma_r(f13, U.x, s02.x), fma_r(f13, U.y, s02.y));
  o2 = mk<C>(fma_r(-f13, U.x, s02.x), fma_r(-f13, U.y, s02.y));
  o1 = mk<C>(fma_r(sg * f13, V.y, d02.x), fma_r(-sg * f13, V.x, d02.y));
  o3 = mk<C>(fma_r(-sg * f13, V.y, d02.x), fma_r(sg * f13, V.x, d02.y));
}

// 16-point DFT for types with a native FMA (float, double): the same 4 x 4
// factorisation as dft16, but the middle-stage twiddles W16^m are written as a
// common scale times a vector, c1 (1 + i t)-type factors with t = tan(pi/8) for
// odd m and h = sqrt(1/2) for m = 2, 6, and the scales are applied inside the
// second-stage additions as FMAs: 144 real operations instead of 160.
template <typename C, bool INV>
__host__ __device__ __forceinline__ void dft16_fma(C* v) {
  using R = decltype(C::x);
  constexpr R sg = INV ? (R)-1 : (R)1;
  constexpr R h = (R)0.70710678118654752440;   // cos(pi/4)
  constexpr R c1 = (R)0.92387953251128675613;  // cos(pi/8)
  constexpr R t = (R)0.41421356237309504880;   // tan(pi/8)
  dft4<C, INV>(v[0], v[4], v[8], v[12]);
  dft4<C, INV>(v[1], v[5], v[9], v[13]);
  dft4<C, INV>(v[2], v[6], v[10], v[14]);
  dft4<C, INV>(v[3], v[7], v[11], v[15]);
  // b[n2][k1] sits at v[n2 + 4 k1]; row k1 takes b[n2][k1] W16^(n2 k1), n2 = 0..3
  dft4<C, INV>(v[0], v[1], v[2], v[3]);
  {  // k1 = 1: W^1 = c1 (1 - i sg t), W^2 = h (1 - i sg), W^3 = c1 (t - i sg)
    const C a0 = v[4], x1 = v[5], x2 = v[6], x3 = v[7];
    const C A2 = mk<C>(x2.x + sg * x2.y, x2.y - sg * x2.x);
    const C s02 = mk<C>(fma_r(h, A2.x, a0.x), fma_r(h, A2.y, a0.y));
    const C d02 = mk<C>(fma_r(-h, A2.x, a0.x), fma_r(-h, A2.y, a0.y));
    const C P = mk<C>(fma_r(sg * t, x1.y, x1.x), fma_r(-sg * t, x1.x, x1.y));
    const C Q = mk<C>(fma_r(t, x3.x, sg * x3.y), fma_r(t, x3.y, -sg * x3.x));
    dft4_scaled<C, INV>(v[4], v[5], v[6], v[7], s02, d02, cadd(P, Q), csub(P, Q), c1);
  }
  {  // k1 = 2: W^2 = h (1 - i sg), W^4 = -i sg, W^6 = h (-1 - i sg)
    const C a0 = v[8], x1 = v[9], x2 = v[10], x3 = v[11];
    const C B4 = mk<C>(sg * x2.y, -sg * x2.x);
    const C s02 = cadd(a0, B4), d02 = csub(a0, B4);
    const C A = mk<C>(x1.x + sg * x1.y, x1.y - sg * x1.x);
    const C B = mk<C>(sg * x3.y - x3.x, -x3.y - sg * x3.x);
    dft4_scaled<C, INV>(v[8], v[9], v[10], v[11], s02, d02, cadd(A, B), csub(A, B), h);
  }
  {  // k1 = 3: W^3 = c1 (t - i sg), W^6 = h (-1 - i sg), W^9 = -c1 (1 - i sg t)
    const C a0 = v[12], x1 = v[13], x2 = v[14], x3 = v[15];
    const C B6 = mk<C>(sg * x2.y - x2.x, -x2.y - sg * x2.x);
    const C s02 = mk<C>(fma_r(h, B6.x, a0.x), fma_r(h, B6.y, a0.y));
    const C d02 = mk<C>(fma_r(-h, B6.x, a0.x), fma_r(-h, B6.y, a0.y));
    const C Q1 = mk<C>(fma_r(t, x1.x, sg * x1.y), fma_r(t, x1.y, -sg * x1.x));
    const C P3 = mk<C>(fma_r(sg * t, x3.y, x3.x), fma_r(-sg * t, x3.x, x3.y));
    // a1 = c1 Q1, a3 = -c1 P3: s13 = c1 (Q1 - P3), d13 = c1 (Q1 + P3)
    dft4_scaled<C, INV>(v[12], v[13], v[14], v[15], s02, d02, csub(Q1, P3), cadd(Q1, P3), c1);
  }
  // now X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4x4 index
  C tmp;
  tmp = v[1]; v[1] = v[4]; v[4] = tmp;
  tmp = v[2]; v[2] = v[8]; v[8] = tmp;
  tmp = v[3]; v[3] = v[12]; v[12] = tmp;
  tmp = v[6]; v[6] = v[9]; v[9] = tmp;
  tmp = v[7]; v[7] = v[13]; v[13] = tmp;
  tmp = v[11]; v[11] = v[14]; v[14] = tmp;
}

template <typename C> struct NativeFma : std::false_type {};
template <> struct NativeFma<float2> : std::true_type {};
template <> struct NativeFma<double2> : std::true_type {};

template <typename C, int RAD, bool INV>
__host__ __device__ __forceinline__ void dftR(C* v) {
  if constexpr (RAD == 2) dft2<C, INV>(v[0], v[1]);
  else if constexpr (RAD == 4) dft4<C, INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (RAD == 8) dft8<C, INV>(v);
  else if constexpr (NativeFma<C>::value) dft16_fma<C, INV>(v);
  else dft16<C, INV>(v);
}

// One pass' arithmetic on the 16 values of thread t: butterflies q < 16/RAD,
// j = t + T q, twiddles W_{NS RAD}^{r (j mod NS)} from tw = W_L^m, then DFT.
// The twiddle index r (j mod NS) L/(NS RAD) splits into a per-thread part and a
// compile-time part: for NS <= T (NS divides T) j mod NS = t mod NS for every q;
// for NS > T the butterflies of a thread hold j = t + T q < NS, so j mod NS = j.
template <int L, int RAD, int NS>
struct RfTwiddle {
  static constexpr int T = L / 16;
  static constexpr int B = 16 / RAD;
  static constexpr int step = L / (NS * RAD);
  static_assert(NS <= T ? T % NS == 0 : NS >= T * B, "butterflies of one thread share j mod NS");
  static constexpr int kq_unit = (NS <= T) ? 0 : T * step;  // compile-time part of k * step per q
  // per-thread part of k * step
  __host__ __device__ __forceinline__ static int thread_part(int t) {
    return (NS <= T) ? (t & (NS - 1)) * step : t * step;
  }
  // index of W_L^{r k step} for butterfly q of a thread whose thread_part is kt
  __host__ __device__ __forceinline__ static int index(int kt, int q, int r) { return r * kt + r * q * kq_unit; }
};

template <typename R, int L, int RAD, int NS, bool INV, int NL, class Tab>
__device__ __forceinline__ void rf_compute(cplx<R> (&v)[NL][16], int t, Tab tw) {
  using C = cplx<R>;
  using TW = RfTwiddle<L, RAD, NS>;
  constexpr int B = 16 / RAD;
  const int kt = TW::thread_part(t);
#pragma unroll
  for (int q = 0; q < B; ++q) {
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        C w = tw_get(tw, TW::index(kt, q, r));
        if (INV) w.y = -w.y;
#pragma unroll
        for (int l = 0; l < NL; ++l) v[l][q * RAD + r] = cmul(v[l][q * RAD + r], w);
      }
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) dftR<C, RAD, INV>(&v[l][q * RAD]);
  }
}

// Shared-memory exchange: write the outputs of a pass (radix RAD, NS), barrier,
// read the inputs of the next pass (radix RADN), barrier. Every position of the
// exchange is a thread part A and a compile-time part c occupying disjoint bits
// (write: A = (t div NS) NS RAD + t mod NS, c = T q RAD + r NS; read: A = t,
// c = T q + r L/RADN), so a layout `Lay` maps (line l, A + c) to shared memory as
// a per-thread base (lay.base(A), computed once) plus a constant (lay.at(b, l, c)).
template <typename R, int L, int RAD, int RADN, int NS, int NL, class Lay>
__device__ __forceinline__ void rf_exchange(cplx<R> (&v)[NL][16], int t, const Lay& lay) {
  constexpr int T = L / 16;
  static_assert(T % NS == 0, "exchanges run with NS dividing T");
  {
    const auto b = lay.base((t / NS) * NS * RAD + (t & (NS - 1)));
#pragma unroll
    for (int q = 0; q < 16 / RAD; ++q)
#pragma unroll
      for (int r = 0; r < RAD; ++r)
#pragma unroll
        for (int l = 0; l < NL; ++l) lay.at(b, l, T * q * RAD + r * NS) = v[l][q * RAD + r];
  }
  __syncthreads();
  {
    const auto b = lay.base(t);
#pragma unroll
    for (int q = 0; q < 16 / RADN; ++q)
#pragma unroll
      for (int r = 0; r < RADN; ++r)
#pragma unroll
        for (int l = 0; l < NL; ++l) v[l][q * RADN + r] = lay.at(b, l, T * q + r * (L / RADN));
  }
  __syncthreads();
}

// Forward transform: positions t + r T  ->  t + T q + r L/RL.
template <typename R, int L, int NL, class Lay, class Tab>
__device__ __forceinline__ void rf_forward(cplx<R> (&v)[NL][16], int t, Tab tw, const Lay& lay) {
  using S = RfShape<L>;
  if constexpr (S::P == 1) {
    rf_compute<R, L, 16, 1, false, NL>(v, t, tw);
  } else if constexpr (S::P == 2) {
    rf_compute<R, L, 16, 1, false, NL>(v, t, tw);
    rf_exchange<R, L, 16, S::RL, 1, NL>(v, t, lay);
    rf_compute<R, L, S::RL, 16, false, NL>(v, t, tw);
  } else {
    rf_compute<R, L, 16, 1, false, NL>(v, t, tw);
    rf_exchange<R, L, 16, 16, 1, NL>(v, t, lay);
    rf_compute<R, L, 16, 16, false, NL>(v, t, tw);
    rf_exchange<R, L, 16, S::RL, 16, NL>(v, t, lay);
    rf_compute<R, L, S::RL, 256, false, NL>(v, t, tw);
  }
}

// Inverse (unnormalised) transform: positions t + T q + r L/RL  ->  t + r T.
template <typename R, int L, int NL, class Lay, class Tab>
__device__ __forceinline__ void rf_inverse(cplx<R> (&v)[NL][16], int t, Tab tw, const Lay& lay) {
  using S = RfShape<L>;
  if constexpr (S::P == 1) {
    rf_compute<R, L, 16, 1, true, NL>(v, t, tw);
  } else if constexpr (S::P == 2) {
    rf_compute<R, L, S::RL, 1, true, NL>(v, t, tw);
    rf_exchange<R, L, S::RL, 16, 1, NL>(v, t, lay);
    rf_compute<R, L, 16, S::RL, true, NL>(v, t, tw);
  } else {
    rf_compute<R, L, S::RL, 1, true, NL>(v, t, tw);
    rf_exchange<R, L, S::RL, 16, 1, NL>(v, t, lay);
    rf_compute<R, L, 16, S::RL, true, NL>(v, t, tw);
    rf_exchange<R, L, 16, 16, S::RL, NL>(v, t, lay);
    rf_compute<R, L, 16, 16 * S::RL, true, NL>(v, t, tw);
  }
}

// ---------------------------------------------------------------------------
// Shared-memory layouts of the exchanges. base(A) returns two element pointers;
// at(b, l, c) picks one by a compile-time selector of (l, c) and adds a
// compile-time offset, which is valid because A and c have disjoint bits.
// ---------------------------------------------------------------------------

// Line-major with one pad element per 16 positions: element (l, pos) at
// line0 + l*LS + pos + pos/16 (conflict-free for the Stockham strides).
// Bases are 32-bit element offsets (one register each).
template <typename C, int LS>
struct PadLayout {
  C* line0;
  struct Base { int o; };
  __host__ __device__ __forceinline__ Base base(int A) const { return {A + (A >> 4)}; }
  __host__ __device__ __forceinline__ C& at(const Base& b, int l, int c) const {
    return line0[b.o + l * LS + c + (c >> 4)];
  }
};

// Position-major, 2 CP lines per position row (line l of column pair cl at
// l*CP + cl), the line index XOR-swizzled by CP when the low five position bits
// have odd parity: element (l, pos) at pos*LW + ((l*CP + cl) ^ (par(pos & 31) CP)).
// With par(A + c) = par(A) ^ par(c) the swizzle picks one of two per-thread bases.
template <typename C, int CP>
struct SwizzleLayout {
  C* sm;
  int cl;
  struct Base { int o[2]; };
  static constexpr int LW = 2 * CP;
  __host__ __device__ __forceinline__ Base base(int A) const {
    const int pa = fde_popc(A & 31) & 1;
    const int row = A * LW + cl;
    return {{row + CP * pa, row + CP * (pa ^ 1)}};
  }
  __host__ __device__ __forceinline__ C& at(const Base& b, int l, int c) const {
    const int k = (l ^ fde_popc(c & 31)) & 1;
    return sm[b.o[k] + c * LW];
  }
};

// SwizzleLayout with the line fixed at run time (the split-halves kernels: the
// thread group h owns line h): the selector becomes h ^ par(c).
template <typename C, int CP>
struct SwizzleLineLayout {
  C* sm;
  int cl, h;
  struct Base { int o[2]; };
  static constexpr int LW = 2 * CP;
  __host__ __device__ __forceinline__ Base base(int A) const {
    const int pa = fde_popc(A & 31) & 1;
    const int row = A * LW + cl;
    return {{row + CP * (pa ^ h), row + CP * (pa ^ h ^ 1)}};
  }
  __host__ __device__ __forceinline__ C& at(const Base& b, int, int c) const {
    return sm[b.o[fde_popc(c & 31) & 1] + c * LW];
  }
};

// Position-major, CP columns per position row, the physical row pos with bit 0
// flipped when position bits 1..4 have odd parity: element pos at
// (pos ^ par(pos & 30)) * CP + cl. Writing A + c = (A & ~1) + (c & ~1) + (A0 ^ c0)
// gives phys = (A & ~1) + (c & ~1) + (u ^ k), u = A0 ^ par(A & 30) per thread and
// k = c0 ^ par(c & 30) at compile time.
template <typename C, int CP>
struct FlipLayout {
  C* sm;
  int cl;
  struct Base { int o[2]; };
  __host__ __device__ __forceinline__ Base base(int A) const {
    const int u = (A & 1) ^ (fde_popc(A & 30) & 1);
    const int row = (A & ~1) * CP + cl;
    return {{row + CP * u, row + CP * (u ^ 1)}};
  }
  __host__ __device__ __forceinline__ C& at(const Base& b, int, int c) const {
    const int k = (c & 1) ^ (fde_popc(c & 30) & 1);
    return sm[b.o[k] + (c & ~1) * CP];
  }
};

// Frequency position held in v[.][q RL + r] after rf_forward.
template <int L>
__device__ __forceinline__ int rf_freq(int t, int idx) {
  using S = RfShape<L>;
  const int q = idx / S::RL, r = idx - q * S::RL;
  return t + S::T * q + r * (L / S::RL);
}

}  // namespace fde
