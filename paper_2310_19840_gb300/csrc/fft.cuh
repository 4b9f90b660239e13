// fft.cuh - block-cooperative complex FFTs in registers and shared memory.
//
// The transforms F{.} and F^{-1}{.} of Sec. 2.2 are evaluated on the device by
// Stockham autosort passes: a transform of length N is split over N/R threads,
// each thread owning R elements in registers.  A pass with current sub-length
// Ls multiplies element r of butterfly b by w_{Ls*R}^{r*(b mod Ls)}, runs a
// radix-R DFT in registers and scatters the results to natural Stockham
// positions ((b - k) R + k + r Ls) in shared memory; the next pass gathers with
// stride N/R.  The first pass reads straight from registers (the caller loads
// element j + r N/R into slot r), the last pass leaves the transform in natural
// order in shared memory.  Forward transforms use w = exp(-2 pi i / L),
// inverse ones exp(+2 pi i / L); neither is normalised.
//
// Shared-memory indices are padded by one complex per 16 (pad()) to spread
// the power-of-two strides of the scatter over the banks: for the radix-8 and
// radix-16 passes used here this keeps every store and load of a warp at the
// minimum of two 128-byte wavefronts for lengths of 128 and up (one per 32
// left the radix-8 stores of lengths 128 and 256 at 3.3 and 2.7).  When a transform
// fits in one warp (N/R <= 32 threads) its passes synchronise with __syncwarp
// only; larger transforms use block barriers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sbi {

template <typename T> struct cplx;
template <> struct cplx<float>  { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cx = typename cplx<T>::type;

template <typename V> __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) { V v; v.x = a; v.y = b; return v; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { return mk<V>(a.x * s, a.y * s); }
// multiply by SIGN * i
template <int SIGN, typename V> __device__ __forceinline__ V rot(V a) {
  return SIGN > 0 ? mk<V>(-a.y, a.x) : mk<V>(a.y, -a.x);
}

__host__ __device__ constexpr int pad(int i) { return i + (i >> 4); }
// Every index of a Stockham pass splits as pad(a + c) = pad(a) + pad(c) with
// a run-time part a and a compile-time part c: c a multiple of a power of two
// P > a (the gathers j + r T, j < T; the last pass's b + m Ls, b < Ls), or
// a = (j - k) R + k with c = r Ls (a multiple of Ls R plus k < Ls).  pad(c)
// then folds into the address of the shared-memory access.
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + 1; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// exp(SIGN 2 pi i q / 16) for q = 0..7 (q a compile-time constant after
// unrolling)
template <int SIGN, typename V>
__device__ __forceinline__ V root16(int q) {
  using S = decltype(V::x);
  constexpr double c[8] = {1.0, 0.92387953251128675613, 0.70710678118654752440,
                           0.38268343236508977173, 0.0, -0.38268343236508977173,
                           -0.70710678118654752440, -0.92387953251128675613};
  constexpr double s[8] = {0.0, 0.38268343236508977173, 0.70710678118654752440,
                           0.92387953251128675613, 1.0, 0.92387953251128675613,
                           0.70710678118654752440, 0.38268343236508977173};
  return mk<V>(S(c[q]), SIGN > 0 ? S(s[q]) : S(-s[q]));
}

// ---------------------------------------------------------------------------
// Radix-R DFT in registers, R in {1, 2, 4, 8, 16}, y_q = sum_r x_r w_R^{r q}.
// ---------------------------------------------------------------------------
template <int R, int SIGN, typename V> struct Dft;

template <int SIGN, typename V> struct Dft<1, SIGN, V> {
  __device__ __forceinline__ static void run(V*) {}
};

template <int SIGN, typename V> struct Dft<2, SIGN, V> {
  __device__ __forceinline__ static void run(V* x) {
    V a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <int SIGN, typename V> struct Dft<4, SIGN, V> {
  __device__ __forceinline__ static void run(V* x) {
    V t0 = cadd(x[0], x[2]), t1 = csub(x[0], x[2]);
    V t2 = cadd(x[1], x[3]), t3 = rot<SIGN>(csub(x[1], x[3]));
    x[0] = cadd(t0, t2);
    x[2] = csub(t0, t2);
    x[1] = cadd(t1, t3);
    x[3] = csub(t1, t3);
  }
};

// Split radix-2 step: DFT of length R from two DFTs of length R/2 of the even
// and odd elements, y_q = E_q + w_R^q O_q, y_{q+R/2} = E_q - w_R^q O_q.
template <int SIGN, typename V> struct Dft<8, SIGN, V> {
  __device__ __forceinline__ static void run(V* x) {
    using S = decltype(V::x);
    V e[4] = {x[0], x[2], x[4], x[6]};
    V o[4] = {x[1], x[3], x[5], x[7]};
    Dft<4, SIGN, V>::run(e);
    Dft<4, SIGN, V>::run(o);
    const S h = S(0.70710678118654752440);
    // w8^1 = h (1 + SIGN i), w8^2 = SIGN i, w8^3 = h (-1 + SIGN i)
    V o1 = cscale(cadd(o[1], rot<SIGN>(o[1])), h);
    V o2 = rot<SIGN>(o[2]);
    V o3 = cscale(csub(rot<SIGN>(o[3]), o[3]), h);
    x[0] = cadd(e[0], o[0]); x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);   x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);   x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);   x[7] = csub(e[3], o3);
  }
};

template <int SIGN, typename V> struct Dft<16, SIGN, V> {
  __device__ __forceinline__ static void run(V* x) {
    using S = decltype(V::x);
    V e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { e[i] = x[2 * i]; o[i] = x[2 * i + 1]; }
    Dft<8, SIGN, V>::run(e);
    Dft<8, SIGN, V>::run(o);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      V t = q == 0 ? o[0] : cmul(o[q], root16<SIGN, V>(q));
      x[q] = cadd(e[q], t);
      x[q + 8] = csub(e[q], t);
    }
  }
};

// ---------------------------------------------------------------------------
// Twiddle tables: tw[off(N) + j] = exp(-2 pi i j / N), j < N, N = 2^q >= 2,
// off(N) = N - 2.  Built on the host in FP64.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tw_off(int n) { return n - 2; }

// FP32 transforms form most twiddle powers by complex products of a few
// table entries, which trades load/store-pipe work for FMA work; FP64
// transforms load every power, because FP64 arithmetic is the scarcer
// resource on this part.
template <typename V> inline constexpr bool kProductTwiddles = sizeof(V) == 8;

template <int SIGN, typename V>
__device__ __forceinline__ V twiddle(const V* __restrict__ tw, int N, int idx) {
  V w = __ldg(tw + tw_off(N) + idx);
  return SIGN > 0 ? cconj(w) : w;
}

// ---------------------------------------------------------------------------
// Stockham transform of length N by T = N/R threads (thread index j), data in
// registers on entry (x[r] = a[j + r T]) and in natural order in s[] (padded)
// on exit.  All threads of the block must call it (it contains barriers);
// threads without work still take part.  The caller must make sure nobody
// still reads s[] from earlier work (a barrier before the call).
// ---------------------------------------------------------------------------
template <bool WARP>
__device__ __forceinline__ void group_sync() {
  if constexpr (WARP) __syncwarp();
  else __syncthreads();
}

// Transforms of 128 and 256 points by 16 and 32 threads (radix 8, 8 and a
// last radix-2 / radix-4 pass) can hand the data from the second pass to the
// last one by warp shuffles instead of a shared-memory scatter and gather.
constexpr bool kShuffleLastExchange = true;

template <typename V>
__device__ __forceinline__ V shfl_xor_cx(V v, int mask) {
  V r;
  r.x = __shfl_xor_sync(0xffffffffu, v.x, mask);
  r.y = __shfl_xor_sync(0xffffffffu, v.y, mask);
  return r;
}
template <typename V>
__device__ __forceinline__ V pick(bool c, V a, V b) { return c ? a : b; }

// Last pass after the Ls = 8 pass, from registers: before it, thread j holds
// x[r] = element 64 a + (j & 7) + 8 r with a = j >> 3 (the Stockham order of
// the Ls = 8 pass); the last pass wants, for butterflies b = j + q T, the
// elements b + 64 m.  Those sit in the lanes j' = 8 m + (j & 7) of the same
// row, register (j >> 3) + (T / 8) q, so the exchange is a transpose between
// the lane bits above 7 and the low register bits: one shuffle stage per lane
// bit (xor 8, then xor 16), each lane keeping the half of its values that
// stays and receiving the other half.
// REGS: leave the result in registers instead of shared memory; thread j
// then holds element j + r T in x[r] (the last pass computes exactly those:
// b + 64 m = j + T (q + Q m)).
template <int N, int SIGN, bool REGS, typename V>
__device__ __forceinline__ void last_pass_by_shuffles(V (&x)[8], V* s, int j, const V* __restrict__ tw) {
  constexpr int T = N / 8;          // 16 or 32 threads per transform
  constexpr int Ls = 64, RP = N / Ls, Q = 8 / RP;
  const int b0 = (j >> 3) & 1;
  V v[Q][RP];
  if constexpr (RP == 2) {
    // N = 128: lanes j and j ^ 8 swap the registers of the other's parity
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const V keep = pick(b0, x[2 * q + 1], x[2 * q]);
      const V recv = shfl_xor_cx(pick(b0, x[2 * q], x[2 * q + 1]), 8);
      v[q][0] = pick(b0, recv, keep);
      v[q][1] = pick(b0, keep, recv);
    }
  } else {
    // N = 256: a 4 x 4 transpose per q between lane bits (3, 4) and register
    // bits (0, 1); register c + 4 q of lane a holds row a, column c
    const int b1 = (j >> 4) & 1;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      V t[2][2];   // [pair p: column 2 p + b0][row bit 0]
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const V keep = pick(b0, x[4 * q + 2 * p + 1], x[4 * q + 2 * p]);
        const V recv = shfl_xor_cx(pick(b0, x[4 * q + 2 * p], x[4 * q + 2 * p + 1]), 8);
        t[p][0] = pick(b0, recv, keep);
        t[p][1] = pick(b0, keep, recv);
      }
      // keep the pair of column a = 2 b1 + b0, send the other one
      V own[2], oth[2];
#pragma unroll
      for (int rb = 0; rb < 2; ++rb) {
        own[rb] = pick(b1, t[1][rb], t[0][rb]);
        oth[rb] = shfl_xor_cx(pick(b1, t[0][rb], t[1][rb]), 16);
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const bool mine = ((m >> 1) & 1) == b1;
        v[q][m] = pick(mine, own[m & 1], oth[m & 1]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int b = j + q * T;
    if constexpr (RP == 4 && kProductTwiddles<V>) {
      const V w1 = twiddle<SIGN>(tw, N, b), w2 = cmul(w1, w1);
      v[q][1] = cmul(v[q][1], w1);
      v[q][2] = cmul(v[q][2], w2);
      v[q][3] = cmul(v[q][3], cmul(w1, w2));
    } else {
#pragma unroll
      for (int m = 1; m < RP; ++m) v[q][m] = cmul(v[q][m], twiddle<SIGN>(tw, N, m * b));
    }
    Dft<RP, SIGN, V>::run(v[q]);
#pragma unroll
    for (int m = 0; m < RP; ++m) {
      if constexpr (REGS) x[q + Q * m] = v[q][m];
      else s[pad(j) + pad(q * T) + pad(m * Ls)] = v[q][m];
    }
  }
  if constexpr (!REGS) __syncwarp();
}

// transforms whose last pass is fed by shuffles (and can end in registers)
template <int N, int R>
inline constexpr bool kShuffleFft = kShuffleLastExchange && R == 8 && (N == 128 || N == 256);

template <int N, int R, int Ls, int SIGN, typename V, bool REGS = false>
struct StockhamPass {
  static constexpr bool WARP = (N / R) <= 32;
  __device__ __forceinline__ static void run(V (&x)[R], V* s, int j, const V* __restrict__ tw) {
    constexpr int T = N / R;
    if constexpr (kShuffleFft<N, R> && Ls == 8) {
      // the Ls = 8 pass, then the last pass fed by shuffles
      const int k = j & (Ls - 1);
      const int base = k * (N / (Ls * R));
      if constexpr (kProductTwiddles<V>) {
        const V w1 = twiddle<SIGN>(tw, N, base), w4 = twiddle<SIGN>(tw, N, 4 * base);
        const V w2 = cmul(w1, w1), w3 = cmul(w1, w2);
        x[1] = cmul(x[1], w1);
        x[2] = cmul(x[2], w2);
        x[3] = cmul(x[3], w3);
        x[4] = cmul(x[4], w4);
        x[5] = cmul(x[5], cmul(w4, w1));
        x[6] = cmul(x[6], cmul(w4, w2));
        x[7] = cmul(x[7], cmul(w4, w3));
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) x[r] = cmul(x[r], twiddle<SIGN>(tw, N, r * base));
      }
      Dft<R, SIGN, V>::run(x);
      last_pass_by_shuffles<N, SIGN, REGS, V>(x, s, j, tw);
      return;
    }
    if constexpr (N / Ls >= R) {
      // full pass of radix R
      const int k = j & (Ls - 1);
      if constexpr (Ls > 1) {
        const int base = k * (N / (Ls * R));
        if constexpr (R == 8 && kProductTwiddles<V>) {
          // w^1 and w^4 from the table, the other powers by products (at most
          // three roundings each): 2 loads instead of 7
          const V w1 = twiddle<SIGN>(tw, N, base), w4 = twiddle<SIGN>(tw, N, 4 * base);
          const V w2 = cmul(w1, w1), w3 = cmul(w1, w2);
          x[1] = cmul(x[1], w1);
          x[2] = cmul(x[2], w2);
          x[3] = cmul(x[3], w3);
          x[4] = cmul(x[4], w4);
          x[5] = cmul(x[5], cmul(w4, w1));
          x[6] = cmul(x[6], cmul(w4, w2));
          x[7] = cmul(x[7], cmul(w4, w3));
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) x[r] = cmul(x[r], twiddle<SIGN>(tw, N, r * base));
        }
      }
      Dft<R, SIGN, V>::run(x);
      const int sb = pad((j - k) * R) + pad(k);   // pad((j - k) R + k + r Ls) - pad(r Ls)
#pragma unroll
      for (int r = 0; r < R; ++r) s[sb + pad(r * Ls)] = x[r];
      group_sync<WARP>();
      if constexpr (Ls * R < N) {
        const int lb = pad(j);
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = s[lb + pad(r * T)];
        group_sync<WARP>();
        StockhamPass<N, R, Ls * R, SIGN, V, REGS>::run(x, s, j, tw);
      }
    } else {
      // last pass, radix RP = N / Ls < R: butterflies b_q = j + q T (q < R/RP),
      // b_q < Ls, with elements x[q + m R/RP] (m < RP); output b_q + m Ls.
      constexpr int RP = N / Ls;
      constexpr int Q = R / RP;
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        V v[RP];
        const int b = j + q * T;
#pragma unroll
        for (int m = 0; m < RP; ++m) v[m] = x[q + m * Q];
        if constexpr (RP == 4 && kProductTwiddles<V>) {
          // w^b from the table, w^2b and w^3b by products
          const V w1 = twiddle<SIGN>(tw, N, b), w2 = cmul(w1, w1);
          v[1] = cmul(v[1], w1);
          v[2] = cmul(v[2], w2);
          v[3] = cmul(v[3], cmul(w1, w2));
        } else {
#pragma unroll
          for (int m = 1; m < RP; ++m) v[m] = cmul(v[m], twiddle<SIGN>(tw, N, m * b));
        }
        Dft<RP, SIGN, V>::run(v);
#pragma unroll
        for (int m = 0; m < RP; ++m) s[pad(j) + pad(q * T) + pad(m * Ls)] = v[m];
      }
      group_sync<WARP>();
    }
  }
};

template <int N, int R, int SIGN, typename V>
__device__ __forceinline__ void fft_block(V (&x)[R], V* s, int j, const V* __restrict__ tw) {
  static_assert((N & (N - 1)) == 0 && N >= 1, "N must be a power of two");
  static_assert(R >= 1 && R <= N && (R & (R - 1)) == 0, "R must be a power of two <= N");
  if constexpr (N == 1) {
    s[0] = x[0];
    __syncwarp();
  } else {
    StockhamPass<N, R, 1, SIGN, V>::run(x, s, j, tw);
  }
}

// The same transform with the thread's own elements of the result in
// registers on exit: x[r] = X[j + r N/R].  Where the last pass is fed by
// shuffles it ends there (no final scatter and read-back); otherwise the
// result is read back from s.  s has no live data on exit either way.
template <int N, int R, int SIGN, typename V>
__device__ __forceinline__ void fft_block_regs(V (&x)[R], V* s, int j, const V* __restrict__ tw) {
  if constexpr (kShuffleFft<N, R>) {
    StockhamPass<N, R, 1, SIGN, V, true>::run(x, s, j, tw);
  } else {
    constexpr int T = N / R;
    fft_block<N, R, SIGN>(x, s, j, tw);
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = s[pad(j) + pad(r * T)];
  }
}

// ---------------------------------------------------------------------------
// Split transforms of N = S * 256 points (S = 2, 4, 8) by S warps: T = N / 8
// threads, thread j = 32 q + l (warp q, lane l).  In place of log_8 N
// block-synchronised Stockham passes: one radix-S step across the warps in
// registers, one exchange through shared memory (the only block barrier) and
// one 256-point transform inside each warp (shuffle-fed, warp-synchronous).
//   DIF (decimation in frequency), natural order in: thread j holds a[j + T r]
//   in x[r].  With e = m + 256 w (m < 256, w < S),
//     b_q[m] = w_N^{m q} sum_w a[m + 256 w] w_S^{w q},
//     X[S k + q] = sum_m b_q[m] w_256^{m k}:
//   thread j owns the radix-S columns m = j + T p (p < P = 8 / S, registers
//   x[p + P w]); warp q then transforms b_q.  On exit thread j holds
//   X[S (l + 32 r) + q] in x[r].
//   DIT (decimation in time), the same read backwards: thread j holds
//   c_q[l + 32 r] = a[S (l + 32 r) + q] in x[r]; warp q transforms c_q into
//   Y_q, and X[k + 256 w] = sum_q w_S^{q w} (w_N^{q k} Y_q[k]); on exit thread
//   j holds X[j + T r] in x[r].
// Scratch: S rows of padded_len(256) elements, row q holding warp q's part of
// the exchange and then its 256-point scratch.  Every thread of the block
// calls these (block barrier); the caller makes sure nobody still reads s.
// ---------------------------------------------------------------------------
constexpr bool kSplitTransforms = true;
template <int N, int R>
inline constexpr bool kSplitFft = kSplitTransforms && R == 8 && (N == 512 || N == 1024 || N == 2048);

// shared-memory elements a transform of N points by radix R needs
template <int N, int R>
__host__ __device__ constexpr int fft_scratch_len() {
  return kSplitFft<N, R> ? (N / 256) * padded_len(256) : padded_len(N);
}

// v[k] *= w_N^{k m} for k = 1 .. S - 1 (FP32: powers by products, at most
// three roundings each; FP64: every power from the table)
template <int S, int SIGN, typename V>
__device__ __forceinline__ void twiddle_run(V (&v)[S], const V* __restrict__ tw, int N, int m) {
  if constexpr (S == 1) {
    return;
  } else if constexpr (kProductTwiddles<V>) {
    const V w1 = twiddle<SIGN>(tw, N, m);
    const V w2 = cmul(w1, w1);
    v[1] = cmul(v[1], w1);
    if constexpr (S >= 4) {
      const V w3 = cmul(w1, w2);
      v[2] = cmul(v[2], w2);
      v[3] = cmul(v[3], w3);
      if constexpr (S == 8) {
        const V w4 = twiddle<SIGN>(tw, N, 4 * m);
        v[4] = cmul(v[4], w4);
        v[5] = cmul(v[5], cmul(w4, w1));
        v[6] = cmul(v[6], cmul(w4, w2));
        v[7] = cmul(v[7], cmul(w4, w3));
      }
    }
  } else {
#pragma unroll
    for (int k = 1; k < S; ++k) v[k] = cmul(v[k], twiddle<SIGN>(tw, N, k * m));
  }
}

template <int N, int SIGN, typename V>
__device__ __forceinline__ void fft_split_dif(V (&x)[8], V* s, int j, const V* __restrict__ tw) {
  constexpr int S = N / 256, P = 8 / S, T = N / 8, PP = padded_len(256);
  const int q = j >> 5, l = j & 31;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int m = j + T * p;
    V v[S];
#pragma unroll
    for (int w = 0; w < S; ++w) v[w] = x[p + P * w];
    Dft<S, SIGN, V>::run(v);
    twiddle_run<S, SIGN>(v, tw, N, m);
#pragma unroll
    for (int k = 0; k < S; ++k) s[k * PP + pad(m)] = v[k];
  }
  __syncthreads();
  V* row = s + q * PP;
#pragma unroll
  for (int r = 0; r < 8; ++r) x[r] = row[pad(l) + pad(32 * r)];
  __syncwarp();   // row q is read only by warp q: free for its transform
  fft_block_regs<256, 8, SIGN>(x, row, l, tw);
}

template <int N, int SIGN, typename V>
__device__ __forceinline__ void fft_split_dit(V (&x)[8], V* s, int j, const V* __restrict__ tw) {
  constexpr int S = N / 256, P = 8 / S, T = N / 8, PP = padded_len(256);
  const int q = j >> 5, l = j & 31;
  V* row = s + q * PP;
  fft_block_regs<256, 8, SIGN>(x, row, l, tw);   // x[r] = Y_q[l + 32 r]; row free again
  if (q > 0) {
    // w_N^{q (l + 32 r)} = w_N^{q l} w_N^{32 q r}
    if constexpr (kProductTwiddles<V>) {
      const V wl = twiddle<SIGN>(tw, N, q * l);
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = cmul(x[r], r == 0 ? wl : cmul(wl, twiddle<SIGN>(tw, N, 32 * q * r)));
    } else {
#pragma unroll
      for (int r = 0; r < 8; ++r) x[r] = cmul(x[r], twiddle<SIGN>(tw, N, q * (l + 32 * r)));
    }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) row[pad(l) + pad(32 * r)] = x[r];
  __syncthreads();
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const int m = j + T * p;
    V v[S];
#pragma unroll
    for (int k = 0; k < S; ++k) v[k] = s[k * PP + pad(m)];
    Dft<S, SIGN, V>::run(v);
#pragma unroll
    for (int w = 0; w < S; ++w) x[p + P * w] = v[w];
  }
}

// Thread j's inputs to fft_regs_in_order are the elements jin + T r with
// jin = fft_in_index(j): the decimated order of the split form, else j.
template <int N, int R>
__device__ __forceinline__ int fft_in_index(int j) {
  if constexpr (kSplitFft<N, R>) return (N / 256) * (j & 31) + (j >> 5);
  else return j;
}

// Transform with the inputs in fft_in_index order and the thread's own
// elements of the result in registers on exit, x[r] = X[j + r N/R].
// s has no live data on exit.
template <int N, int R, int SIGN, typename V>
__device__ __forceinline__ void fft_regs_in_order(V (&x)[R], V* s, int j, const V* __restrict__ tw) {
  if constexpr (kSplitFft<N, R>) fft_split_dit<N, SIGN>(x, s, j, tw);
  else fft_block_regs<N, R, SIGN>(x, s, j, tw);
}

// Transform of natural-order inputs (x[r] = a[j + r N/R]) that leaves the
// result in natural order in s[pad(k)]: readers in other threads need a
// block barrier (or a warp barrier where the transform fits one warp) first.
template <int N, int R, int SIGN, typename V>
__device__ __forceinline__ void fft_to_smem(V (&x)[R], V* s, int j, const V* __restrict__ tw) {
  if constexpr (kSplitFft<N, R>) {
    constexpr int T = N / R;
    fft_split_dif<N, SIGN>(x, s, j, tw);
    __syncthreads();   // every warp done with its rows of s
    const int jo = (N / 256) * (j & 31) + (j >> 5);
#pragma unroll
    for (int r = 0; r < R; ++r) s[pad(jo + r * T)] = x[r];
  } else {
    fft_block<N, R, SIGN>(x, s, j, tw);
  }
}

}  // namespace sbi
