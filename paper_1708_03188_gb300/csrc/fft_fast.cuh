// fft_fast.cuh - compile-time FFT engine for lengths 2^a and 3 * 2^a (16 <= L <= 4096).
//
// Same self-sorting (Stockham) pass structure as fft_core.cuh, with the length, the radix
// sequence and the pass strides known at compile time, so every index is a shift or a
// mask.  A CTA holds LINES lines of L complex values in ONE shared-memory buffer: each pass
// loads every butterfly's R inputs into registers, synchronises, writes the R outputs to
// their Stockham positions in the same buffer and synchronises again.  Element e of a line
// sits at padded offset e + e/16, and lines are LDP = L + L/16 + 1 apart (LDP odd), which
// keeps the R-strided Stockham writes and the transposed tile loads free of bank conflicts.
// Twiddles of pass p (radix R, NS = product of the earlier radices) are read from a table
// laid out [k][r] = exp(-+2 pi i k r / (NS R)), k < NS, r < R (built by the host).
#pragma once
#include "fft_core.cuh"

namespace sgm {

template <int... Rs> struct Radices {};

template <int L> struct FastRadices;  // radix sequence per supported length
template <> struct FastRadices<16> { using type = Radices<16>; };
template <> struct FastRadices<32> { using type = Radices<8, 4>; };
template <> struct FastRadices<64> { using type = Radices<8, 8>; };
template <> struct FastRadices<128> { using type = Radices<16, 8>; };
template <> struct FastRadices<256> { using type = Radices<16, 16>; };
template <> struct FastRadices<512> { using type = Radices<8, 8, 8>; };
template <> struct FastRadices<1024> { using type = Radices<16, 16, 4>; };
template <> struct FastRadices<2048> { using type = Radices<16, 16, 8>; };
template <> struct FastRadices<4096> { using type = Radices<16, 16, 16>; };
template <> struct FastRadices<48> { using type = Radices<16, 3>; };
template <> struct FastRadices<96> { using type = Radices<8, 4, 3>; };
template <> struct FastRadices<192> { using type = Radices<16, 4, 3>; };
template <> struct FastRadices<384> { using type = Radices<16, 8, 3>; };
template <> struct FastRadices<768> { using type = Radices<16, 16, 3>; };
template <> struct FastRadices<1536> { using type = Radices<16, 8, 4, 3>; };
template <> struct FastRadices<3072> { using type = Radices<16, 16, 4, 3>; };

__host__ __device__ constexpr bool fast_length(int L) {
  return L == 16 || L == 32 || L == 64 || L == 128 || L == 256 || L == 512 || L == 1024 || L == 2048 ||
         L == 4096 || L == 48 || L == 96 || L == 192 || L == 384 || L == 768 || L == 1536 || L == 3072;
}

__host__ __device__ constexpr int pad_ld(int L) { return L + L / 16 + 1; }
// Line stride for buffers whose lines are only read along the line (row tiles): congruent to 8
// modulo 16 complex slots, so the two lines a half-warp touches in a pass of fewer than 16
// butterflies per line (the first pass at L = 32, 64, 128) land on disjoint halves of the banks.
__host__ __device__ constexpr int row_ld(int L) { return (L + L / 16 + 7) / 16 * 16 + 8; }
__device__ __forceinline__ constexpr int padi(int e) { return e + (e >> 4); }

// radix-16 butterfly as 4 x 4: inner DFT4 over n1 of x[s0 + 4 n1], twiddle W16^(s0 q),
// outer DFT4 over s0; output index q + 4 t.
template <bool INV, typename C> __device__ __forceinline__ void butterfly16(C* v) {
  using T = decltype(C::x);
  C a[4][4];
#pragma unroll
  for (int s0 = 0; s0 < 4; ++s0) {
    C w[4] = {v[s0], v[s0 + 4], v[s0 + 8], v[s0 + 12]};
    butterfly<4, INV>(w);
#pragma unroll
    for (int q = 0; q < 4; ++q) a[s0][q] = w[q];
  }
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
  const T h = (T)0.70710678118654752440;
  auto tw = [&](C x, T wr, T wi) -> C {  // x * (wr + i wi), wi negated for the inverse
    const T wii = INV ? -wi : wi;
    return mk<C>(x.x * wr - x.y * wii, x.x * wii + x.y * wr);
  };
  // W16^m = cos(2 pi m/16) - i sin(2 pi m/16) (forward)
  a[1][1] = tw(a[1][1], c1, -s1);
  a[1][2] = tw(a[1][2], h, -h);
  a[1][3] = tw(a[1][3], s1, -c1);
  a[2][1] = tw(a[2][1], h, -h);
  a[2][2] = rot90<INV>(a[2][2]);
  a[2][3] = tw(a[2][3], -h, -h);
  a[3][1] = tw(a[3][1], s1, -c1);
  a[3][2] = tw(a[3][2], -h, -h);
  a[3][3] = tw(a[3][3], -c1, s1);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    C w[4] = {a[0][q], a[1][q], a[2][q], a[3][q]};
    butterfly<4, INV>(w);
#pragma unroll
    for (int t = 0; t < 4; ++t) v[q + 4 * t] = w[t];
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void butterfly_any(C* v) {
  if constexpr (R == 16) butterfly16<INV>(v);
  else butterfly<R, INV>(v);
}

// One pass over LINES lines held in `buf`; NTHREADS threads; TWO = offset of this pass's
// twiddle table in `tw`.
template <int L, int R, int NS, int TWO, int LINES, int NTHREADS, bool INV, int LDP, typename C>
__device__ __forceinline__ void fast_pass(C* buf, int nlines, const C* __restrict__ tw) {
  constexpr int LR = L / R;
  constexpr int TOTAL = LINES * LR;
  constexpr int M = (TOTAL + NTHREADS - 1) / NTHREADS;
  C v[M][R];
  const int active = nlines * LR;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int b = threadIdx.x + m * NTHREADS;
    if (b < active) {
      const int line = b / LR, j = b - line * LR;   // LR is a compile-time constant
      const C* x = buf + line * LDP;
#pragma unroll
      for (int r = 0; r < R; ++r) v[m][r] = x[padi(j + r * LR)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int b = threadIdx.x + m * NTHREADS;
    if (b < active) {
      const int line = b / LR, j = b - line * LR;
      const int k = j % NS;
      if (NS > 1) {
        const C* t = tw + TWO + k * R;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(&t[r]);
          if (INV) w.y = -w.y;
          v[m][r] = cmul(v[m][r], w);
        }
      }
      butterfly_any<R, INV>(v[m]);
      C* y = buf + line * LDP;
      const int base = (j - k) * R + k;
#pragma unroll
      for (int s = 0; s < R; ++s) y[padi(base + s * NS)] = v[m][s];
    }
  }
  __syncthreads();
}

template <int L, int NS, int TWO, int LINES, int NTHREADS, bool INV, int LDP, typename C>
__device__ __forceinline__ void fast_passes(C*, int, const C*, Radices<>) {}

template <int L, int NS, int TWO, int LINES, int NTHREADS, bool INV, int LDP, typename C, int R, int... Rest>
__device__ __forceinline__ void fast_passes(C* buf, int nlines, const C* tw, Radices<R, Rest...>) {
  fast_pass<L, R, NS, TWO, LINES, NTHREADS, INV, LDP>(buf, nlines, tw);
  fast_passes<L, NS * R, TWO + NS * R, LINES, NTHREADS, INV, LDP>(buf, nlines, tw, Radices<Rest...>{});
}

// In-place transform of `nlines` (<= LINES) padded lines, LDP complex values apart (element e
// at e + e/16 within its line); ends with __syncthreads().
template <int L, int LINES, int NTHREADS, bool INV, int LDP = pad_ld(L), typename C>
__device__ __forceinline__ void fft_fast(C* buf, int nlines, const C* __restrict__ tw) {
  fast_passes<L, 1, 0, LINES, NTHREADS, INV, LDP>(buf, nlines, tw, typename FastRadices<L>::type{});
}

// ---- the same passes with other shared-memory layouts ------------------------------------------
// A pass reads its inputs through ld_at(line, e) from `src` and writes its outputs through
// st_at(line, e) to `dst` (src may equal dst: every input is read before the synchronisation
// that precedes the writes).  With COLS the butterflies of a warp run across lines first (line =
// b % LINES), which suits the column-tile layout e * LINES + line written by a TMA box of LINES
// neighbouring columns: a warp then touches consecutive words in every load and store, with no
// padding.  Without COLS the mapping is that of fast_pass (line = b / (L / R)).
template <int L, int R, int NS, int TWO, int LINES, int NTHREADS, bool INV, bool COLS, typename C, typename LA,
          typename SA>
__device__ __forceinline__ void gen_pass(const C* src, C* dst, const C* __restrict__ tw, LA ld_at, SA st_at) {
  constexpr int LR = L / R;
  constexpr int TOTAL = LINES * LR;
  constexpr int M = (TOTAL + NTHREADS - 1) / NTHREADS;
  C v[M][R];
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int b = threadIdx.x + m * NTHREADS;
    if (b < TOTAL) {
      const int line = COLS ? b % LINES : b / LR, j = COLS ? b / LINES : b % LR;
#pragma unroll
      for (int r = 0; r < R; ++r) v[m][r] = src[ld_at(line, j + r * LR)];
    }
  }
  __syncthreads();
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int b = threadIdx.x + m * NTHREADS;
    if (b < TOTAL) {
      const int line = COLS ? b % LINES : b / LR, j = COLS ? b / LINES : b % LR;
      const int k = j % NS;
      if (NS > 1) {
        const C* t = tw + TWO + k * R;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = __ldg(&t[r]);
          if (INV) w.y = -w.y;
          v[m][r] = cmul(v[m][r], w);
        }
      }
      butterfly_any<R, INV>(v[m]);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) dst[st_at(line, base + q * NS)] = v[m][q];
    }
  }
  __syncthreads();
}

template <int L, int NS, int TWO, int LINES, int NTHREADS, bool INV, bool COLS, bool FIRST, typename C, typename LA0,
          typename AT>
__device__ __forceinline__ void gen_passes(const C*, C*, const C*, LA0, AT, Radices<>) {}

template <int L, int NS, int TWO, int LINES, int NTHREADS, bool INV, bool COLS, bool FIRST, typename C, typename LA0,
          typename AT, int R, int... Rest>
__device__ __forceinline__ void gen_passes(const C* src, C* buf, const C* tw, LA0 ld0, AT at, Radices<R, Rest...>) {
  if constexpr (FIRST)
    gen_pass<L, R, NS, TWO, LINES, NTHREADS, INV, COLS>(src, buf, tw, ld0, at);
  else
    gen_pass<L, R, NS, TWO, LINES, NTHREADS, INV, COLS>(buf, buf, tw, at, at);
  gen_passes<L, NS * R, TWO + NS * R, LINES, NTHREADS, INV, COLS, false>(src, buf, tw, ld0, at, Radices<Rest...>{});
}

// Transform of LINES lines in the column-tile layout buf[e * LINES + line], in place.  The first
// pass reads input e of a line from position first(e) instead (for example a reordering), so the
// caller need not move the data beforehand.  Ends with __syncthreads().
template <int L, int LINES, int NTHREADS, bool INV, typename C, typename FM>
__device__ __forceinline__ void fft_cols(C* buf, const C* __restrict__ tw, FM first) {
  auto at = [](int line, int e) { return e * LINES + line; };
  auto ld0 = [first](int line, int e) { return first(e) * LINES + line; };
  gen_passes<L, 1, 0, LINES, NTHREADS, INV, true, true>(buf, buf, tw, ld0, at, typename FastRadices<L>::type{});
}

// Host: number of entries of the pass tables of length L (sum over passes of NS * R).
inline int fast_table_size(int L) {
  int rs[8], np = 0;
  if (L == 16) { rs[np++] = 16; }
  else if (L == 32) { rs[np++] = 8; rs[np++] = 4; }
  else if (L == 64) { rs[np++] = 8; rs[np++] = 8; }
  else if (L == 128) { rs[np++] = 16; rs[np++] = 8; }
  else if (L == 256) { rs[np++] = 16; rs[np++] = 16; }
  else if (L == 512) { rs[np++] = 8; rs[np++] = 8; rs[np++] = 8; }
  else if (L == 1024) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 4; }
  else if (L == 2048) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 8; }
  else if (L == 4096) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 16; }
  else if (L == 48) { rs[np++] = 16; rs[np++] = 3; }
  else if (L == 96) { rs[np++] = 8; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 192) { rs[np++] = 16; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 384) { rs[np++] = 16; rs[np++] = 8; rs[np++] = 3; }
  else if (L == 768) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 3; }
  else if (L == 1536) { rs[np++] = 16; rs[np++] = 8; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 3072) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 4; rs[np++] = 3; }
  else return 0;
  int ns = 1, total = 0;
  for (int p = 0; p < np; ++p) { total += ns * rs[p]; ns *= rs[p]; }
  return total;
}

// Host: fill the pass tables (the caller supplies cos/sin of 2 pi j / L evaluated in long
// double through `w(j)` = exp(-2 pi i j / L)); entry [k][r] of pass p = w(k r L / (NS R)).
template <typename C, typename W> inline void fill_fast_table(int L, C* out, W w) {
  int rs[8], np = 0;
  if (L == 16) { rs[np++] = 16; }
  else if (L == 32) { rs[np++] = 8; rs[np++] = 4; }
  else if (L == 64) { rs[np++] = 8; rs[np++] = 8; }
  else if (L == 128) { rs[np++] = 16; rs[np++] = 8; }
  else if (L == 256) { rs[np++] = 16; rs[np++] = 16; }
  else if (L == 512) { rs[np++] = 8; rs[np++] = 8; rs[np++] = 8; }
  else if (L == 1024) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 4; }
  else if (L == 2048) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 8; }
  else if (L == 4096) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 16; }
  else if (L == 48) { rs[np++] = 16; rs[np++] = 3; }
  else if (L == 96) { rs[np++] = 8; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 192) { rs[np++] = 16; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 384) { rs[np++] = 16; rs[np++] = 8; rs[np++] = 3; }
  else if (L == 768) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 3; }
  else if (L == 1536) { rs[np++] = 16; rs[np++] = 8; rs[np++] = 4; rs[np++] = 3; }
  else if (L == 3072) { rs[np++] = 16; rs[np++] = 16; rs[np++] = 4; rs[np++] = 3; }
  int ns = 1, off = 0;
  for (int p = 0; p < np; ++p) {
    const int R = rs[p];
    for (int k = 0; k < ns; ++k)
      for (int r = 0; r < R; ++r) out[off + k * R + r] = w((long)k * r * (L / (ns * R)) % L);
    off += ns * R;
    ns *= R;
  }
}

}  // namespace sgm
