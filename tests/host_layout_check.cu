// Host check of the register FFT's index maps (paper_1907_13428_gb300/csrc/fftreg.cuh):
// for every power-of-two length 16..4096 and every exchange the forward and
// inverse transforms perform, the shared-memory address that a layout forms as a
// per-thread base plus a compile-time offset equals the address of the layout's
// definition at the Stockham position, the write and read positions of the
// decomposition equal the Stockham ones, the addresses of one exchange are
// distinct, and the split twiddle index equals r (j mod NS) L/(NS RAD).
// Prints "<check> <mismatches>" lines; every count must be 0.
#include <cstdio>
#include <set>
#include <vector>

#include "../paper_1907_13428_gb300/csrc/fftreg.cuh"

using namespace fde;
using C = float2;

static long bad_pos = 0, bad_addr = 0, bad_unique = 0, bad_tw = 0, bad_disjoint = 0;

static int popc(unsigned x) { int n = 0; for (; x; x &= x - 1) ++n; return n; }

// definitions of the layouts at a Stockham position
static long ref_pad(int LS, int l, int pos) { return (long)l * LS + pos + (pos >> 4); }
static long ref_swz(int CP, int cl, int l, int pos) {
  const int sw = (popc(pos & 31) & 1) ? CP : 0;
  return (long)pos * 2 * CP + ((l * CP + cl) ^ sw);
}
static long ref_flip(int CP, int cl, int pos) { return (long)(pos ^ (popc(pos & 30) & 1)) * CP + cl; }

template <int L, int RAD, int RADN, int NS>
static void check_exchange() {
  constexpr int T = L / 16, LS = L + L / 16;
  std::vector<C> buf(64 * (LS + 64) + 64 * L * 16);
  C* b0 = buf.data();
  const PadLayout<C, LS> pad{b0};
  for (int phase = 0; phase < 2; ++phase) {
    const int nq = phase == 0 ? 16 / RAD : 16 / RADN;
    const int nr = phase == 0 ? RAD : RADN;
    for (int CP : {1, 2, 4, 8}) {
      std::set<long> seen_pad, seen_swz, seen_flip;
      for (int cl = 0; cl < CP; ++cl) {
        for (int t = 0; t < T; ++t) {
          const int A = phase == 0 ? (t / NS) * NS * RAD + (t & (NS - 1)) : t;
          for (int q = 0; q < nq; ++q)
            for (int r = 0; r < nr; ++r) {
              const int c = phase == 0 ? T * q * RAD + r * NS : T * q + r * (L / RADN);
              const int j = t + T * q;
              const int pos = phase == 0 ? (j / NS) * NS * RAD + (j & (NS - 1)) + r * NS : j + r * (L / RADN);
              if (A + c != pos) ++bad_pos;
              if (A & c) ++bad_disjoint;
              for (int l = 0; l < 2; ++l) {
                if (cl == 0 && CP == 1) {
                  const long a = &pad.at(pad.base(A), l, c) - b0;
                  if (a != ref_pad(LS, l, pos)) ++bad_addr;
                  if (!seen_pad.insert(a).second) ++bad_unique;
                }
                long a_swz = -1;
                switch (CP) {
                  case 1: { const SwizzleLayout<C, 1> s{b0, cl}; a_swz = &s.at(s.base(A), l, c) - b0; break; }
                  case 2: { const SwizzleLayout<C, 2> s{b0, cl}; a_swz = &s.at(s.base(A), l, c) - b0; break; }
                  case 4: { const SwizzleLayout<C, 4> s{b0, cl}; a_swz = &s.at(s.base(A), l, c) - b0; break; }
                  default: { const SwizzleLayout<C, 8> s{b0, cl}; a_swz = &s.at(s.base(A), l, c) - b0; break; }
                }
                if (a_swz != ref_swz(CP, cl, l, pos)) ++bad_addr;
                if (!seen_swz.insert(a_swz).second) ++bad_unique;
                long a_line = -1;
                switch (CP) {
                  case 1: { const SwizzleLineLayout<C, 1> s{b0, cl, l}; a_line = &s.at(s.base(A), 0, c) - b0; break; }
                  case 2: { const SwizzleLineLayout<C, 2> s{b0, cl, l}; a_line = &s.at(s.base(A), 0, c) - b0; break; }
                  case 4: { const SwizzleLineLayout<C, 4> s{b0, cl, l}; a_line = &s.at(s.base(A), 0, c) - b0; break; }
                  default: { const SwizzleLineLayout<C, 8> s{b0, cl, l}; a_line = &s.at(s.base(A), 0, c) - b0; break; }
                }
                if (a_line != ref_swz(CP, cl, l, pos)) ++bad_addr;
              }
              long a_flip = -1;
              switch (CP) {
                case 1: { const FlipLayout<C, 1> s{b0, cl}; a_flip = &s.at(s.base(A), 0, c) - b0; break; }
                case 2: { const FlipLayout<C, 2> s{b0, cl}; a_flip = &s.at(s.base(A), 0, c) - b0; break; }
                case 4: { const FlipLayout<C, 4> s{b0, cl}; a_flip = &s.at(s.base(A), 0, c) - b0; break; }
                default: { const FlipLayout<C, 8> s{b0, cl}; a_flip = &s.at(s.base(A), 0, c) - b0; break; }
              }
              if (a_flip != ref_flip(CP, cl, pos)) ++bad_addr;
              if (!seen_flip.insert(a_flip).second) ++bad_unique;
            }
        }
      }
    }
  }
}

template <int L, int RAD, int NS>
static void check_twiddle() {
  using TW = RfTwiddle<L, RAD, NS>;
  constexpr int T = L / 16;
  for (int t = 0; t < T; ++t) {
    const int kt = TW::thread_part(t);
    for (int q = 0; q < 16 / RAD; ++q)
      for (int r = 1; r < RAD; ++r) {
        const int j = t + T * q;
        const int expect = r * (j & (NS - 1)) * (L / (NS * RAD));
        if (TW::index(kt, q, r) != expect) ++bad_tw;
      }
  }
}

// the exchanges and passes of rf_forward / rf_inverse for one length
template <int L>
static void check_length() {
  using S = RfShape<L>;
  if constexpr (S::P == 2) {
    check_exchange<L, 16, S::RL, 1>();
    check_exchange<L, S::RL, 16, 1>();
    check_twiddle<L, S::RL, 16>();
    check_twiddle<L, 16, S::RL>();
  } else if constexpr (S::P == 3) {
    check_exchange<L, 16, 16, 1>();
    check_exchange<L, 16, S::RL, 16>();
    check_exchange<L, S::RL, 16, 1>();
    check_exchange<L, 16, 16, S::RL>();
    check_twiddle<L, 16, 16>();
    check_twiddle<L, S::RL, 256>();
    check_twiddle<L, 16, S::RL>();
    check_twiddle<L, 16, 16 * S::RL>();
  }
}

int main() {
  check_length<16>();
  check_length<32>();
  check_length<64>();
  check_length<128>();
  check_length<256>();
  check_length<512>();
  check_length<1024>();
  check_length<2048>();
  check_length<4096>();
  std::printf("positions %ld\naddresses %ld\nunique %ld\ntwiddles %ld\ndisjoint %ld\n", bad_pos, bad_addr,
              bad_unique, bad_tw, bad_disjoint);
  return 0;
}
