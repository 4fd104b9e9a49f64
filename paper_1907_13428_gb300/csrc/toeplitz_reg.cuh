// Register-resident Toeplitz passes (power-of-two L >= 16): each thread holds 16
// values of both embedding halves of one complex line (fftreg.cuh). Included by
// one translation unit per arithmetic, which instantiates its launchers.
#pragma once
#include "fftreg.cuh"
#include "ops_list.cuh"
#include "toeplitz.cuh"

namespace fde {

// x2 axis. NT threads = PAIRS row pairs x T threads per line; thread t of a
// pair holds positions t + r T of the pair's two half-lines. Shared memory is
// line-major with one pad element per 16 (conflict-free exchanges).
// R: arithmetic of the transforms; S: storage type of the vectors (R, or double
// for double-float arithmetic).
// FULL: the lines fill the transform (n == L), so no position is out of range.
// Resident CTAs per SM the x2 pass is compiled for: float tiles of up to 256
// threads run two CTAs (128 registers for 256 threads), the 512-thread tile one.
template <typename R> constexpr int rows_min_blocks(int nt) { return sizeof(R) == 4 && nt < 512 ? 2 : 1; }

// Arguments of the register-resident x2 pass.
template <typename R, typename S> struct RegRowsArgs {
  const S* x;
  long long nrows;
  int n;
  const cplx<R>* sym;
  const cplx<R>* tw2;
  const cplx<R>* twL;
  int conj_sym;
  AxisEpi<S> E;
};
template <typename R, int L, int NT, typename S, bool FULL> struct RowsRegOp {
  using Args = RegRowsArgs<R, S>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    if (gate_closed<PS>(g.E.gate)) return;
    using C = cplx<R>;
    constexpr int T = L / 16, PAIRS = NT / T, LS = L + L / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const S* x = g.x;
    const int n = g.n;
    const long long nrows = g.nrows;
    const AxisEpi<S>& E = g.E;
    const int pr = threadIdx.x / T, t = threadIdx.x - pr * T;
    const long long ra = (cx.bid * PAIRS + pr) * 2, rb = ra + 1;
    C* my = sm + pr * 2 * LS;
    const PadLayout<C, LS> lay{my};
    C v[2][16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      R a = 0, b = 0;
      if (FULL || p < n) {
        if (ra < nrows) a = cvt_in<R, S>(ldv<PS>(x + ra * n + p));
        if (rb < nrows) b = cvt_in<R, S>(ldv<PS>(x + rb * n + p));
      }
      v[0][r] = mk<C>(a, b);
      v[1][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&g.tw2[p])) : mk<C>(0, 0);
    }
    rf_forward<R, L, 2>(v, t, g.twL, lay);
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      const int k = rf_freq<L>(t, idx);
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        C w = ldg_(&g.sym[l * L + k]);
        if (g.conj_sym) w.y = -w.y;
        v[l][idx] = cmul(v[l][idx], w);
      }
    }
    rf_inverse<R, L, 2>(v, t, g.twL, lay);
    const int ta = (int)(ra / E.rows_per_slice), tb = (int)(rb / E.rows_per_slice);
    // epilogue in chunks of 4 positions: all operand loads of a chunk are issued
    // before any arithmetic or store, so their latencies overlap
#pragma unroll
    for (int r0 = 0; r0 < 16; r0 += 4) {
      EpiIn<S> ia[4], ib[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = t + (r0 + k) * T;
        const bool ok = FULL || p < n;
        ia[k] = (ok && ra < nrows) ? epi_load<PS>(E, ra * n + p, ta) : EpiIn<S>{0, 0, 0, 0};
        ib[k] = (ok && rb < nrows) ? epi_load<PS>(E, rb * n + p, tb) : EpiIn<S>{0, 0, 0, 0};
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = t + (r0 + k) * T;
        if (FULL || p < n) {
          const C res = cadd(v[0][r0 + k], cmul(v[1][r0 + k], cconj(ldg_(&g.tw2[p]))));
          if (ra < nrows) epi_finish(E, ia[k], ra * n + p, ta, cvt_out<S, R>(res.x));
          if (rb < nrows) epi_finish(E, ib[k], rb * n + p, tb, cvt_out<S, R>(res.y));
        }
      }
    }
    if constexpr (PS) __syncthreads();  // the next block of a persistent CTA reuses the shared lines
  }
};

template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT, rows_min_blocks<R>(NT)) k_rows_reg(RegRowsArgs<R, S> a) {
  RowsRegOp<R, L, NT, S, FULL>::template run<false>(hw_ctx(), a);
}

// Strided axis. NT threads = CP column pairs x T; lanes run over column pairs
// (coalesced global access). Shared memory is position-major with the two
// halves' lines side by side; the line index is XOR-swizzled by the parity of
// the low five position bits, which separates the two position groups of every
// half-warp into different banks.
template <typename R, typename S> struct RegAxisArgs {
  const S* x;
  int n;
  long long axis_stride, n_inner, outer_stride, n_outer;
  const cplx<R>* sym;
  const cplx<R>* tw2;
  const cplx<R>* twL;
  int conj_sym;
  AxisEpi<S> E;
  int vec2;
};
template <typename R, int L, int NT, typename S, bool FULL> struct AxisRegOp {
  using Args = RegAxisArgs<R, S>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    if (gate_closed<PS>(g.E.gate)) return;
    using C = cplx<R>;
    constexpr int T = L / 16, CP = NT / T, LW = 2 * CP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const S* x = g.x;
    const int n = g.n, vec2 = g.vec2;
    const long long axis_stride = g.axis_stride, n_inner = g.n_inner;
    const AxisEpi<S>& E = g.E;
    const int cl = threadIdx.x % CP, t = threadIdx.x / CP;
    const long long npi = (n_inner + 1) / 2;
    const long long total = g.n_outer * npi;
    const long long q = cx.bid * CP + cl;
    const bool valid = q < total;
    const long long o = valid ? q / npi : 0;
    const long long c = valid ? 2 * (q - o * npi) : 0;
    const long long base = o * g.outer_stride + c;
    const bool has_b = valid && (c + 1 < n_inner);
    const SwizzleLayout<C, CP> lay{sm, cl};
    static_assert(SwizzleLayout<C, CP>::LW == LW, "layout row width");
    C v[2][16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      R a = 0, b = 0;
      if (valid && (FULL || p < n)) {
        const long long idx = base + p * axis_stride;
        if (vec2 && has_b) {
          // (c, c+1) as one aligned vector load
          const cplx<S> ab = ldv<PS>(reinterpret_cast<const cplx<S>*>(x + idx));
          a = cvt_in<R, S>(ab.x);
          b = cvt_in<R, S>(ab.y);
        } else {
          a = cvt_in<R, S>(ldv<PS>(x + idx));
          if (has_b) b = cvt_in<R, S>(ldv<PS>(x + idx + 1));
        }
      }
      v[0][r] = mk<C>(a, b);
      v[1][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&g.tw2[p])) : mk<C>(0, 0);
    }
    rf_forward<R, L, 2>(v, t, g.twL, lay);
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      const int k = rf_freq<L>(t, idx);
#pragma unroll
      for (int l = 0; l < 2; ++l) {
        C w = ldg_(&g.sym[l * L + k]);
        if (g.conj_sym) w.y = -w.y;
        v[l][idx] = cmul(v[l][idx], w);
      }
    }
    rf_inverse<R, L, 2>(v, t, g.twL, lay);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      if (valid && (FULL || p < n)) {
        const C res = cadd(v[0][r], cmul(v[1][r], cconj(ldg_(&g.tw2[p]))));
        const long long idx = base + p * axis_stride;
        if (E.plain && vec2 && has_b) {
          *reinterpret_cast<cplx<S>*>(E.out + idx) = mk<cplx<S>>(cvt_out<S, R>(res.x), cvt_out<S, R>(res.y));
          continue;
        }
        const int ts = E.t_is_axis ? p : (int)o;
        axis_store<PS>(E, idx, ts, cvt_out<S, R>(res.x));
        if (has_b) axis_store<PS>(E, idx + 1, ts, cvt_out<S, R>(res.y));
      }
    }
    if constexpr (PS) __syncthreads();
  }
};

template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT) k_axis_reg(RegAxisArgs<R, S> a) {
  AxisRegOp<R, L, NT, S, FULL>::template run<false>(hw_ctx(), a);
}

// ---------------------------------------------------------------------------
// Split-halves variants (double-float and double on double vectors): the two
// embedding halves of a line pair are transformed by two thread groups, so a
// thread holds the 16 values of one line (half the registers of data) and twice
// as many warps fit on an SM (16 at 128 registers). For float the kernels that
// hold both halves per thread are faster (measured), so only the double-float
// and double instantiations are launched. After
// the inverse transforms each group finishes every other position r (r % 2 ==
// its half), taking the other half's term for those positions from shared
// memory (the exchange buffers are free once the inverse has passed its last
// barrier).
// ---------------------------------------------------------------------------
template <typename R> constexpr int split_min_blocks(int nt) { return (sizeof(R) == 4 ? 1024 : 512) / nt; }

template <typename R, int L, int NT, typename S, bool FULL> struct RowsSplitOp {
  using Args = RegRowsArgs<R, S>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    const AxisEpi<S>& E = g.E;
    if (gate_closed<PS>(E.gate)) return;
    const S* x = g.x;
    const long long nrows = g.nrows;
    const int n = g.n, conj_sym = g.conj_sym;
    const cplx<R>* sym = g.sym;
    const cplx<R>* tw2 = g.tw2;
    const cplx<R>* twL = g.twL;
    using C = cplx<R>;
    constexpr int T = L / 16, PAIRS = NT / (2 * T), LS = L + L / 16;
    static_assert(PAIRS >= 1, "at least one row pair per CTA");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int pr = threadIdx.x / (2 * T);
    const int h = (threadIdx.x / T) & 1;
    const int t = threadIdx.x % T;
    const long long ra = (cx.bid * PAIRS + pr) * 2, rb = ra + 1;
    C* my = sm + (pr * 2 + h) * LS;
    C* other = sm + (pr * 2 + (h ^ 1)) * LS;
    const PadLayout<C, LS> lay{my};
    C v[1][16];
    if constexpr (!std::is_same<R, S>::value) {
      // both groups need the whole line pair: each converts the positions of its own
      // parity (r & 1 == h) and takes the others from the other group's line buffer
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if ((r & 1) != h) continue;
        const int p = t + r * T;
        R a = 0, b = 0;
        if (FULL || p < n) {
          if (ra < nrows) a = cvt_in<R, S>(ldv<PS>(x + ra * n + p));
          if (rb < nrows) b = cvt_in<R, S>(ldv<PS>(x + rb * n + p));
        }
        v[0][r] = mk<C>(a, b);
        my[p + (p >> 4)] = v[0][r];
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = t + r * T;
        if ((r & 1) != h) v[0][r] = other[p + (p >> 4)];
      }
      __syncthreads();  // the transform's first exchange overwrites the line buffers
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = t + r * T;
        if (h) v[0][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
      }
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = t + r * T;
        R a = 0, b = 0;
        if (FULL || p < n) {
          if (ra < nrows) a = cvt_in<R, S>(ldv<PS>(x + ra * n + p));
          if (rb < nrows) b = cvt_in<R, S>(ldv<PS>(x + rb * n + p));
        }
        v[0][r] = mk<C>(a, b);
        if (h) v[0][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
      }
    }
    rf_forward<R, L, 1>(v, t, twL, lay);
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      C w = ldg_(&sym[h * L + rf_freq<L>(t, idx)]);
      if (conj_sym) w.y = -w.y;
      v[0][idx] = cmul(v[0][idx], w);
    }
    rf_inverse<R, L, 1>(v, t, twL, lay);
    // the odd half's term is v conj(tw2[p]); hand over the positions the other group finishes
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      if (h) v[0][r] = (FULL || p < n) ? cmul(v[0][r], cconj(ldg_(&tw2[p]))) : mk<C>(0, 0);
      if ((r & 1) != h) my[p + (p >> 4)] = v[0][r];
    }
    __syncthreads();
    const int ta = (int)(ra / E.rows_per_slice), tb = (int)(rb / E.rows_per_slice);
#pragma unroll
    for (int c0 = 0; c0 < 8; c0 += 4) {
      EpiIn<S> ia[4], ib[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = t + (2 * (c0 + k) + h) * T;
        const bool ok = FULL || p < n;
        ia[k] = (ok && ra < nrows) ? epi_load<PS>(E, ra * n + p, ta) : EpiIn<S>{0, 0, 0, 0};
        ib[k] = (ok && rb < nrows) ? epi_load<PS>(E, rb * n + p, tb) : EpiIn<S>{0, 0, 0, 0};
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = 2 * (c0 + k) + h;
        const int p = t + r * T;
        if (FULL || p < n) {
          // a select of two compile-time indices keeps v in registers (v[0][r] with
          // the run-time h would place the array in local memory)
          const C mine = h ? v[0][2 * (c0 + k) + 1] : v[0][2 * (c0 + k)];
          const C res = cadd(mine, other[p + (p >> 4)]);
          if (ra < nrows) epi_finish(E, ia[k], ra * n + p, ta, cvt_out<S, R>(res.x));
          if (rb < nrows) epi_finish(E, ib[k], rb * n + p, tb, cvt_out<S, R>(res.y));
        }
      }
    }
    if constexpr (PS) __syncthreads();  // the next block of a persistent CTA reuses the line buffers
  }
};

template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT, split_min_blocks<R>(NT)) k_rows_split(RegRowsArgs<R, S> a) {
  RowsSplitOp<R, L, NT, S, FULL>::template run<false>(hw_ctx(), a);
}


template <typename R, int L, int NT, typename S, bool FULL> struct AxisSplitOp {
  using Args = RegAxisArgs<R, S>;
  template <bool PS> static __device__ __forceinline__ void run(const Ctx& cx, const Args& g) {
    const AxisEpi<S>& E = g.E;
    if (gate_closed<PS>(E.gate)) return;
    const S* x = g.x;
    const int n = g.n, conj_sym = g.conj_sym, vec2 = g.vec2;
    const long long axis_stride = g.axis_stride, n_inner = g.n_inner, outer_stride = g.outer_stride;
    const long long n_outer = g.n_outer;
    const cplx<R>* sym = g.sym;
    const cplx<R>* tw2 = g.tw2;
    const cplx<R>* twL = g.twL;
    using C = cplx<R>;
    constexpr int T = L / 16, CP = NT / (2 * T), LW = 2 * CP;
    static_assert(CP >= 1, "at least one column pair per CTA");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    // lanes run over column pairs (coalesced), then over the two halves, then over t
    const int cl = threadIdx.x % CP;
    const int h = (threadIdx.x / CP) & 1;
    const int t = threadIdx.x / (2 * CP);
    const long long npi = (n_inner + 1) / 2;
    const long long total = n_outer * npi;
    const long long q = cx.bid * CP + cl;
    const bool valid = q < total;
    const long long o = valid ? q / npi : 0;
    const long long c = valid ? 2 * (q - o * npi) : 0;
    const long long base = o * outer_stride + c;
    const bool has_b = valid && (c + 1 < n_inner);
    auto slot = [cl](int l, int pos) -> int {
      const int sw = (__popc(pos & 31) & 1) ? CP : 0;
      return pos * LW + ((l * CP + cl) ^ sw);
    };
    const SwizzleLineLayout<C, CP> lay{sm, cl, h};
    C v[1][16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      R a = 0, b = 0;
      if (valid && (FULL || p < n)) {
        const long long idx = base + p * axis_stride;
        if (vec2 && has_b) {
          const cplx<S> ab = ldv<PS>(reinterpret_cast<const cplx<S>*>(x + idx));
          a = cvt_in<R, S>(ab.x);
          b = cvt_in<R, S>(ab.y);
        } else {
          a = cvt_in<R, S>(ldv<PS>(x + idx));
          if (has_b) b = cvt_in<R, S>(ldv<PS>(x + idx + 1));
        }
      }
      v[0][r] = mk<C>(a, b);
      if (h) v[0][r] = (FULL || p < n) ? cmul(v[0][r], ldg_(&tw2[p])) : mk<C>(0, 0);
    }
    rf_forward<R, L, 1>(v, t, twL, lay);
#pragma unroll
    for (int idx = 0; idx < 16; ++idx) {
      C w = ldg_(&sym[h * L + rf_freq<L>(t, idx)]);
      if (conj_sym) w.y = -w.y;
      v[0][idx] = cmul(v[0][idx], w);
    }
    rf_inverse<R, L, 1>(v, t, twL, lay);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int p = t + r * T;
      if (h) v[0][r] = (FULL || p < n) ? cmul(v[0][r], cconj(ldg_(&tw2[p]))) : mk<C>(0, 0);
      if ((r & 1) != h) sm[slot(h, p)] = v[0][r];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int r = 2 * k + h;
      const int p = t + r * T;
      if (valid && (FULL || p < n)) {
        const C mine = h ? v[0][2 * k + 1] : v[0][2 * k];
        const C res = cadd(mine, sm[slot(h ^ 1, p)]);
        const long long idx = base + p * axis_stride;
        if (E.plain && vec2 && has_b) {
          *reinterpret_cast<cplx<S>*>(E.out + idx) = mk<cplx<S>>(cvt_out<S, R>(res.x), cvt_out<S, R>(res.y));
          continue;
        }
        const int ts = E.t_is_axis ? p : (int)o;
        axis_store<PS>(E, idx, ts, cvt_out<S, R>(res.x));
        if (has_b) axis_store<PS>(E, idx + 1, ts, cvt_out<S, R>(res.y));
      }
    }
    if constexpr (PS) __syncthreads();
  }
};

template <typename R, int L, int NT, typename S = R, bool FULL = false>
__global__ void __launch_bounds__(NT, split_min_blocks<R>(NT)) k_axis_split(RegAxisArgs<R, S> a) {
  AxisSplitOp<R, L, NT, S, FULL>::template run<false>(hw_ctx(), a);
}


template <typename R> constexpr int rows_nt() { return 256; }
template <typename R> constexpr int axis_nt() { return sizeof(R) == 4 ? 512 : 256; }

template <typename R, int L, int NT, typename S>
static cudaError_t launch_rows_reg_LN(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                      const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int PAIRS = NT / (L / 16);
  static_assert(PAIRS >= 1, "at least one row pair per CTA");
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * 2 * (L + L / 16) * sizeof(cplx<R>);
  if (P->ax[2].n == L)
    return launch_op<RowsRegOp<R, L, NT, S, true>>(k_rows_reg<R, L, NT, S, true>, (unsigned)grid, NT, smem, st,
                                                   {x, nrows, L, sym, T.tw2, T.twL, conj_sym, E});
  return launch_op<RowsRegOp<R, L, NT, S, false>>(k_rows_reg<R, L, NT, S, false>, (unsigned)grid, NT, smem, st,
                                                  {x, nrows, P->ax[2].n, sym, T.tw2, T.twL, conj_sym, E});
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_rows_split_LN(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                        const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int PAIRS = NT / (2 * (L / 16));
  const long long nrows = (long long)P->nt * P->nx;
  const long long npairs = (nrows + 1) / 2;
  const long long grid = (npairs + PAIRS - 1) / PAIRS;
  const size_t smem = (size_t)PAIRS * 2 * (L + L / 16) * sizeof(cplx<R>);
  if (P->ax[2].n == L)
    return launch_op<RowsSplitOp<R, L, NT, S, true>>(k_rows_split<R, L, NT, S, true>, (unsigned)grid, NT, smem, st,
                                                     {x, nrows, L, sym, T.tw2, T.twL, conj_sym, E});
  return launch_op<RowsSplitOp<R, L, NT, S, false>>(k_rows_split<R, L, NT, S, false>, (unsigned)grid, NT, smem, st,
                                                    {x, nrows, P->ax[2].n, sym, T.tw2, T.twL, conj_sym, E});
}

// The tile chosen by fde_autotune: float 128, 256 or 512 threads; double and
// double-float 128 (lines up to 2048) or 256 threads, or the split-halves variant
// with 256 or 512 threads (stored negated).
template <typename R, int L, typename S>
cudaError_t launch_rows_reg_L(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym,
                                     const AxisTables<R>& T, const AxisEpi<S>& E, cudaStream_t st) {
  if constexpr (std::is_same<R, float>::value && std::is_same<S, float>::value) {
    // a recorded solve runs every launch with the executor's block size
    if (recording()) return launch_rows_reg_LN<R, L, kPersistThreads, S>(P, x, conj_sym, sym, T, E, st);
    if constexpr (L <= 2048) {
      if (P->rows_nt32 == 128) return launch_rows_reg_LN<R, L, 128, S>(P, x, conj_sym, sym, T, E, st);
    }
    if (P->rows_nt32 == 512) return launch_rows_reg_LN<R, L, 512, S>(P, x, conj_sym, sym, T, E, st);
  }
  if constexpr (!std::is_same<R, float>::value) {
    const int choice = std::is_same<R, dd>::value ? P->rows_ntdd : P->rows_nt64;
    if constexpr (2 * (L / 16) <= 256) {
      if (choice == -256) return launch_rows_split_LN<R, L, 256, S>(P, x, conj_sym, sym, T, E, st);
    }
    if constexpr (L / 16 <= 128) {
      // two CTAs of 128 threads per SM: one CTA's exchanges overlap the other's arithmetic
      if (choice == 128) return launch_rows_reg_LN<R, L, 128, S>(P, x, conj_sym, sym, T, E, st);
    }
    if (choice == -512) return launch_rows_split_LN<R, L, 512, S>(P, x, conj_sym, sym, T, E, st);
  }
  return launch_rows_reg_LN<R, L, rows_nt<R>(), S>(P, x, conj_sym, sym, T, E, st);
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_axis_reg_LN(const S* x, int n, long long axis_stride, long long n_inner,
                                      long long outer_stride, long long n_outer, const cplx<R>* sym,
                                      const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E, cudaStream_t st) {
  constexpr int CP = NT / (L / 16);
  static_assert(CP >= 1, "at least one column pair per CTA");
  const long long total = n_outer * ((n_inner + 1) / 2);
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * 2 * CP * sizeof(cplx<R>);
  const size_t al = 2 * sizeof(S);
  const int vec2 = ((n_inner | axis_stride | outer_stride) & 1) == 0 && ((uintptr_t)x % al) == 0 &&
                   ((uintptr_t)E.out % al) == 0;
  if (n == L)
    return launch_op<AxisRegOp<R, L, NT, S, true>>(
        k_axis_reg<R, L, NT, S, true>, (unsigned)grid, NT, smem, st,
        {x, L, axis_stride, n_inner, outer_stride, n_outer, sym, T.tw2, T.twL, conj_sym, E, vec2});
  return launch_op<AxisRegOp<R, L, NT, S, false>>(
      k_axis_reg<R, L, NT, S, false>, (unsigned)grid, NT, smem, st,
      {x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T.tw2, T.twL, conj_sym, E, vec2});
}

template <typename R, int L, int NT, typename S>
static cudaError_t launch_axis_split_LN(const S* x, int n, long long axis_stride, long long n_inner,
                                        long long outer_stride, long long n_outer, const cplx<R>* sym,
                                        const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E,
                                        cudaStream_t st) {
  constexpr int CP = NT / (2 * (L / 16));
  const long long total = n_outer * ((n_inner + 1) / 2);
  const long long grid = (total + CP - 1) / CP;
  const size_t smem = (size_t)L * 2 * CP * sizeof(cplx<R>);
  const size_t al = 2 * sizeof(S);
  const int vec2 = ((n_inner | axis_stride | outer_stride) & 1) == 0 && ((uintptr_t)x % al) == 0 &&
                   ((uintptr_t)E.out % al) == 0;
  if (n == L)
    return launch_op<AxisSplitOp<R, L, NT, S, true>>(
        k_axis_split<R, L, NT, S, true>, (unsigned)grid, NT, smem, st,
        {x, L, axis_stride, n_inner, outer_stride, n_outer, sym, T.tw2, T.twL, conj_sym, E, vec2});
  return launch_op<AxisSplitOp<R, L, NT, S, false>>(
      k_axis_split<R, L, NT, S, false>, (unsigned)grid, NT, smem, st,
      {x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T.tw2, T.twL, conj_sym, E, vec2});
}

template <typename R, int L, typename S>
cudaError_t launch_axis_reg_L(const S* x, int n, long long axis_stride, long long n_inner,
                                     long long outer_stride, long long n_outer, const cplx<R>* sym,
                                     const AxisTables<R>& T, int conj_sym, const AxisEpi<S>& E, int nt_choice,
                                     cudaStream_t st) {
  if constexpr (!std::is_same<R, float>::value) {
    if (nt_choice == -512)
      return launch_axis_split_LN<R, L, 512, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym,
                                                E, st);
    if constexpr (L / 16 <= 128) {
      if (nt_choice == 128)
        return launch_axis_reg_LN<R, L, 128, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym,
                                                E, st);
    }
  }
  if constexpr (sizeof(R) == 4) {
    if (nt_choice == 256)
      return launch_axis_reg_LN<R, L, 256, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym,
                                              E, st);
  }
  return launch_axis_reg_LN<R, L, axis_nt<R>(), S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T,
                                                   conj_sym, E, st);
}

#define FDE_FOR_EACH_L(M) M(16) M(32) M(64) M(128) M(256) M(512) M(1024) M(2048) M(4096)

template <typename R, typename S>
cudaError_t launch_rows_reg(fde_problem* P, const S* x, int conj_sym, const cplx<R>* sym, const AxisTables<R>& T,
                            const AxisEpi<S>& E, cudaStream_t st) {
  switch (P->ax[2].L) {
#define FDE_CASE(LL) \
  case LL: return launch_rows_reg_L<R, LL, S>(P, x, conj_sym, sym, T, E, st);
    FDE_FOR_EACH_L(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, typename S>
cudaError_t launch_axis_reg(int L, const S* x, int n, long long axis_stride, long long n_inner,
                            long long outer_stride, long long n_outer, const cplx<R>* sym, const AxisTables<R>& T,
                            int conj_sym, const AxisEpi<S>& E, int nt_choice, cudaStream_t st) {
  switch (L) {
#define FDE_CASE(LL)                                                                                          \
  case LL:                                                                                                    \
    return launch_axis_reg_L<R, LL, S>(x, n, axis_stride, n_inner, outer_stride, n_outer, sym, T, conj_sym, E, \
                                       nt_choice, st);
    FDE_FOR_EACH_L(FDE_CASE)
#undef FDE_CASE
    default: return cudaErrorInvalidValue;
  }
}

// Raises the dynamic shared-memory limit of a kernel and of its guard-free variant.
template <typename K>
static void smem_attr(cudaError_t& e, K plain, K full) {
  const int big = 200 * 1024;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(plain, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(full, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// Shared-memory limits of every tile launch_*_reg_L<R, L, S> may launch: the
// default tiles, the float 256-thread axis and 128-thread row tiles, the double
// and double-float split-halves tiles (512 threads; 256 threads for rows up to 2048).
template <typename R, int L, typename S>
cudaError_t reg_attrs_L() {
  cudaError_t e = cudaSuccess;
  smem_attr(e, k_rows_reg<R, L, rows_nt<R>(), S, false>, k_rows_reg<R, L, rows_nt<R>(), S, true>);
  smem_attr(e, k_axis_reg<R, L, axis_nt<R>(), S, false>, k_axis_reg<R, L, axis_nt<R>(), S, true>);
  if constexpr (std::is_same<R, float>::value) {
    smem_attr(e, k_axis_reg<R, L, 256, S, false>, k_axis_reg<R, L, 256, S, true>);
    if constexpr (L <= 2048) smem_attr(e, k_rows_reg<R, L, 128, S, false>, k_rows_reg<R, L, 128, S, true>);
    smem_attr(e, k_rows_reg<R, L, 512, S, false>, k_rows_reg<R, L, 512, S, true>);
  }
  if constexpr (!std::is_same<R, float>::value) {
    smem_attr(e, k_rows_split<R, L, 512, S, false>, k_rows_split<R, L, 512, S, true>);
    smem_attr(e, k_axis_split<R, L, 512, S, false>, k_axis_split<R, L, 512, S, true>);
    if constexpr (L <= 2048) smem_attr(e, k_rows_split<R, L, 256, S, false>, k_rows_split<R, L, 256, S, true>);
    if constexpr (L / 16 <= 128) {
      smem_attr(e, k_rows_reg<R, L, 128, S, false>, k_rows_reg<R, L, 128, S, true>);
      smem_attr(e, k_axis_reg<R, L, 128, S, false>, k_axis_reg<R, L, 128, S, true>);
    }
  }
  return e;
}

template <typename R, typename S>
cudaError_t reg_attrs_all() {
  cudaError_t e = cudaSuccess;
#define FDE_ATTR(LL) \
  if (e == cudaSuccess) e = reg_attrs_L<R, LL, S>();
  FDE_FOR_EACH_L(FDE_ATTR)
#undef FDE_ATTR
  return e;
}

// Explicit instantiation (FDE_REG_INSTANTIATE) or instantiation declaration
// (FDE_REG_EXTERN) of every pass of arithmetic R on vectors S for one L, so
// that the transform lengths of one arithmetic compile in separate units.
#define FDE_REG_DECLARE(PRE, R, S, LL)                                                                        \
  PRE template cudaError_t launch_rows_reg_L<R, LL, S>(fde_problem*, const S*, int, const cplx<R>*,           \
                                                       const AxisTables<R>&, const AxisEpi<S>&, cudaStream_t); \
  PRE template cudaError_t launch_axis_reg_L<R, LL, S>(const S*, int, long long, long long, long long,       \
                                                       long long, const cplx<R>*, const AxisTables<R>&, int,  \
                                                       const AxisEpi<S>&, int, cudaStream_t);                 \
  PRE template cudaError_t reg_attrs_L<R, LL, S>();
#define FDE_REG_INSTANTIATE(R, S, LL) FDE_REG_DECLARE(, R, S, LL)
#define FDE_REG_EXTERN(R, S, LL) FDE_REG_DECLARE(extern, R, S, LL)

}  // namespace fde
