// Shared-memory Stockham FFT building blocks for the demag convolution passes.
//
// The convolution-theorem evaluation of Eq. 1 (Sec. II: FFT -> pointwise product ->
// inverse FFT) needs length-L complex FFTs, L a power of two known at compile time, along
// x (half-length transform inside the real-to-complex step), y and z. A thread block holds
// LINES lines of length L; every thread owns 16 complex values per pass and runs 16/R
// radix-R butterflies on them, so a block has LINES * L / 16 threads.
//
// Forward Stockham pass P_s (radix R, Ns = product of the radices already applied):
//   for butterfly j in [0, L/R):   k = j mod Ns
//     v[r] = a[j + r L/R] * w^(r k),  w = exp(S 2 pi i / (Ns R))
//     v    = DFT_R(v)                (sign S)
//     a'[(j - k) R + k + q Ns] = v[q]
// P_p ... P_1 is the DFT in natural order. Its adjoint P_1^H ... P_p^H, where P_s^H
// reads at the positions P_s writes, applies the conjugate DFT_R and then the conjugate
// twiddles, and writes at the positions P_s reads, is the unnormalised inverse DFT.
// The convolution kernels run the forward chain, the kernel product and the adjoint
// chain, so the last forward pass and the first adjoint pass touch the same positions
// and fuse in registers with the product. In both chains the outer passes address the
// data in natural order (j + r L/R), so they can read or write global memory directly.
//
// Shared memory rows are padded: element i of a line sits at i + i/16, which makes the
// stride-16 accesses of the Ns = 1 pass and its adjoint conflict free.
//
// Twiddles come from one table of levels, written on the host in FP64 and rounded to FP32:
// level N holds E_N[m] = exp(-2 pi i m / N), m in [0, N), at index tw_base(N) + m, for the
// powers of two N <= GBD_TW_LEN and for N = 3 * 2^j and 5 * 2^j up to the largest padded
// length. A butterfly of a pass (Ns, R) at position k loads w^r = E_(Ns R / r)[k] for
// r = 1, 2, 4, 8, so the lanes of a warp, which hold consecutive k, read consecutive entries;
// it forms the other powers with at most three complex products.
//
// Lengths. L = r 2^k with r in {1, 3, 5}. For r > 1 the first forward pass (Ns = 1, no
// twiddles) is a radix-r pass and the power-of-two passes follow with Ns = r, 16 r, ...; a
// thread then runs ceil(16 / r) radix-r butterflies of that pass (the last ones of the block
// may be past the end and are skipped). This lets the zero padding of Sec. II stop at the
// smallest such length >= 2n - 1 instead of the next power of two.
#pragma once
#include <cuda_runtime.h>

#define GBD_TW_LEN 8192
#define GBD_E 16
// After the 2 GBD_TW_LEN twiddle entries the same buffer holds the tensor-core passes' split
// DFT-16 fragments (gbd_tc.cuh): 4 tables (sign x 16-bit type) of 32 registers x 32 lanes of
// 32 bits, i.e. 2048 float2 slots.
#define GBD_TC_FRAG_F2 2048
// Then the levels 3 * 2^j (up to 6144) and 5 * 2^j (up to 5120): level N of odd part r starts
// at its region's offset + N - r (the levels r, 2r, 4r, ... are stored back to back).
#define GBD_TW3_OFF (2 * GBD_TW_LEN + GBD_TC_FRAG_F2)
#define GBD_TW3_MAX 6144
#define GBD_TW5_OFF (GBD_TW3_OFF + 2 * GBD_TW3_MAX)
#define GBD_TW5_MAX 5120
#define GBD_TW_TOTAL (GBD_TW5_OFF + 2 * GBD_TW5_MAX)

namespace gbd {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
template <int S>
__device__ __forceinline__ float2 cmul_i(float2 a) {  // a * (S i)
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// L over its largest power-of-two factor (no recursion, so that it folds wherever L is known)
__host__ __device__ constexpr int odd_part(int L) { return L > 0 ? L / (L & -L) : L; }
// index of E_N[0] in the twiddle table (N = 2^j, 3 * 2^j or 5 * 2^j)
__host__ __device__ constexpr int tw_base(int N) {
  return odd_part(N) == 1 ? N : odd_part(N) == 3 ? GBD_TW3_OFF + N - 3 : GBD_TW5_OFF + N - 5;
}

// exp(S 2 pi i m / N) for a level N of the table and 0 <= m < N
template <int S>
__device__ __forceinline__ float2 twiddle_at(const float2* __restrict__ tw, int N, int m) {
  float2 w = __ldg(tw + tw_base(N) + m);
  return S < 0 ? w : cconj(w);
}
// exp(S 2 pi i m / GBD_TW_LEN) for any m
template <int S>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int m) {
  return twiddle_at<S>(tw, GBD_TW_LEN, m & (GBD_TW_LEN - 1));
}

// ---- radix decomposition (compile time) -------------------------------------------------
__host__ __device__ constexpr int ilog2(int L) { return L <= 1 ? 0 : 1 + ilog2(L / 2); }

// Power-of-two lengths: passes of radix 16 and one remainder. With CONV the last radix is at
// most 8 (the convolution kernels keep three components of that pass in registers).
__host__ __device__ constexpr int npasses2(int L, bool conv) {
  return ilog2(L) == 0 ? 0
         : ilog2(L) % 4 == 0 ? (conv ? ilog2(L) / 4 + 1 : ilog2(L) / 4)
         : ilog2(L) % 4 == 3 ? ilog2(L) / 4 + 1
         : (ilog2(L) <= 2 ? 1 : ilog2(L) / 4 + 1);
}
__host__ __device__ constexpr int radix_at2(int L, bool conv, int p) {
  // sequence: 16 ... 16, then the tail
  return ilog2(L) % 4 == 0
             ? (conv ? (p < ilog2(L) / 4 - 1 ? 16 : (p == ilog2(L) / 4 - 1 ? 2 : 8)) : 16)
         : ilog2(L) % 4 == 3 ? (p < ilog2(L) / 4 ? 16 : 8)
         : ilog2(L) == 1 ? 2
         : ilog2(L) == 2 ? 4
         : ilog2(L) % 4 == 1 ? (p < (ilog2(L) - 5) / 4 ? 16 : (p == (ilog2(L) - 5) / 4 ? 4 : 8))
                             : (p < (ilog2(L) - 6) / 4 ? 16 : 8);
}
// Any length r 2^k: a radix-r pass first when r > 1, then the power-of-two passes of 2^k.
__host__ __device__ constexpr int npasses(int L, bool conv) {
  return odd_part(L) > 1 ? 1 + npasses2(L / odd_part(L), conv) : npasses2(L, conv);
}
__host__ __device__ constexpr int radix_at(int L, bool conv, int p) {
  return odd_part(L) > 1 ? (p == 0 ? odd_part(L) : radix_at2(L / odd_part(L), conv, p - 1)) : radix_at2(L, conv, p);
}
__host__ __device__ constexpr int ns_at(int L, bool conv, int p) {
  return p == 0 ? 1 : ns_at(L, conv, p - 1) * radix_at(L, conv, p - 1);
}

// padded position of element i inside a shared-memory line
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
// float2 slots per line; LF (lines interleaved across threads) needs an odd stride
template <int L, bool LF>
__host__ __device__ constexpr int line_stride() {
  return (L + L / 16) + (LF ? ((L + L / 16) % 2 == 0 ? 1 : 0) : 0);
}

// ---- register DFTs of size 2, 4, 8, 16 (sign S) -----------------------------------------
template <int S>
__device__ __forceinline__ void dft4(float2* x) {
  float2 a0 = cadd(x[0], x[2]), a1 = csub(x[0], x[2]);
  float2 b0 = cadd(x[1], x[3]), b1 = cmul_i<S>(csub(x[1], x[3]));
  x[0] = cadd(a0, b0);
  x[2] = csub(a0, b0);
  x[1] = cadd(a1, b1);
  x[3] = csub(a1, b1);
}

// X[q] = E[q] + w8^q O[q], X[q+4] = E[q] - w8^q O[q]; E, O = DFT4 of even / odd samples.
template <int S>
__device__ __forceinline__ void dft8(float2* x) {
  const float h = 0.70710678118654752440f;
  float2 e[4] = {x[0], x[2], x[4], x[6]};
  float2 o[4] = {x[1], x[3], x[5], x[7]};
  dft4<S>(e);
  dft4<S>(o);
  float2 t1 = make_float2(h * (o[1].x - S * o[1].y), h * (o[1].y + S * o[1].x));   // w8^1 = h (1 + S i)
  float2 t2 = cmul_i<S>(o[2]);                                                     // w8^2 = S i
  float2 t3 = make_float2(h * (-o[3].x - S * o[3].y), h * (-o[3].y + S * o[3].x)); // w8^3 = h (-1 + S i)
  x[0] = cadd(e[0], o[0]);
  x[4] = csub(e[0], o[0]);
  x[1] = cadd(e[1], t1);
  x[5] = csub(e[1], t1);
  x[2] = cadd(e[2], t2);
  x[6] = csub(e[2], t2);
  x[3] = cadd(e[3], t3);
  x[7] = csub(e[3], t3);
}

template <int S>
__device__ __forceinline__ void dft16(float2* x) {
  // cos(q pi / 8), sin(q pi / 8), q = 0..7
  const float c[8] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                      0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f};
  const float s[8] = {0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f,
                      1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f};
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = x[2 * i];
    o[i] = x[2 * i + 1];
  }
  dft8<S>(e);
  dft8<S>(o);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    float2 t = (q == 0) ? o[0] : cmul(o[q], make_float2(c[q], S * s[q]));
    x[q] = cadd(e[q], t);
    x[q + 8] = csub(e[q], t);
  }
}

// DFT_3: X0 = x0 + x1 + x2, X1,2 = x0 - (x1 + x2)/2 +- S i (sqrt(3)/2)(x1 - x2)
template <int S>
__device__ __forceinline__ void dft3(float2* x) {
  const float h = 0.86602540378443864676f;   // sin(2 pi / 3)
  const float2 t1 = cadd(x[1], x[2]), t2 = csub(x[1], x[2]);
  const float2 m = make_float2(fmaf(-0.5f, t1.x, x[0].x), fmaf(-0.5f, t1.y, x[0].y));
  const float2 u = make_float2(-S * h * t2.y, S * h * t2.x);
  x[0] = cadd(x[0], t1);
  x[1] = cadd(m, u);
  x[2] = csub(m, u);
}

// DFT_5 by the symmetric pairs a_n = x_n + x_(5-n), b_n = x_n - x_(5-n) (n = 1, 2), with
// c_q = cos(2 pi q / 5), s_q = sin(2 pi q / 5):
//   X_1,4 = x0 + c1 a1 + c2 a2 +- S i (s1 b1 + s2 b2),  X_2,3 = x0 + c2 a1 + c1 a2 +- S i (s2 b1 - s1 b2)
template <int S>
__device__ __forceinline__ void dft5(float2* x) {
  const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
  const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
  const float2 a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]);
  const float2 a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
  const float2 p1 = make_float2(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
  const float2 p2 = make_float2(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
  const float2 q1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);   // times S i below
  const float2 q2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
  const float2 u1 = make_float2(-S * q1.y, S * q1.x), u2 = make_float2(-S * q2.y, S * q2.x);
  x[0] = cadd(x[0], cadd(a1, a2));
  x[1] = cadd(p1, u1);
  x[4] = csub(p1, u1);
  x[2] = cadd(p2, u2);
  x[3] = csub(p2, u2);
}

template <int R, int S>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 3) {
    dft3<S>(x);
  } else if constexpr (R == 5) {
    dft5<S>(x);
  } else if constexpr (R == 2) {
    float2 t = x[0];
    x[0] = cadd(t, x[1]);
    x[1] = csub(t, x[1]);
  } else if constexpr (R == 4) {
    dft4<S>(x);
  } else if constexpr (R == 8) {
    dft8<S>(x);
  } else {
    dft16<S>(x);
  }
}

// exp(S 2 pi i n / R) for R in {4, 8, 16} and 0 < n < R/2, from the literal constants of dft16
template <int S, int R>
__device__ __forceinline__ float2 wr(int n) {
  const float c[8] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                      0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f};
  const float s[8] = {0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f,
                      1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f};
  const int q = n * (16 / R);   // angle 2 pi n / R = q pi / 8
  return make_float2(c[q], S * s[q]);
}

// DFT_R (sign S) of x whose entries R/2 .. R-1 are zero; only x[0, R/2) are read. With H = R/2:
//   X[2m] = DFT_H(x)[m],  X[2m+1] = DFT_H(x[n] w_R^n)[m],  w_R = exp(S 2 pi i / R).
// The first pass of a transform whose upper half is zero padding (Ns = 1) needs no twiddles, so
// this is the whole butterfly there.
template <int R, int S>
__device__ __forceinline__ void dft_half_in(float2* x) {
  constexpr int H = R / 2;
  if constexpr (H == 1) {
    x[1] = x[0];
  } else {
    float2 e[H], o[H];
#pragma unroll
    for (int n = 0; n < H; ++n) {
      e[n] = x[n];
      o[n] = (n == 0) ? x[0] : (4 * n == R) ? cmul_i<S>(x[n]) : cmul(x[n], wr<S, R>(n));
    }
    dft<H, S>(e);
    dft<H, S>(o);
#pragma unroll
    for (int m = 0; m < H; ++m) {
      x[2 * m] = e[m];
      x[2 * m + 1] = o[m];
    }
  }
}

// The first R/2 outputs of DFT_R (sign S) of x: X[q] = E[q] + w_R^q O[q], q < R/2, with E, O the
// DFT_(R/2) of the even and odd entries (the first half of dft16's combination); x[R/2, R) are
// left undefined. The last adjoint pass of a cropped transform (Ns = 1) keeps only these.
template <int R, int S>
__device__ __forceinline__ void dft_half_out(float2* x) {
  constexpr int H = R / 2;
  if constexpr (H == 1) {
    x[0] = cadd(x[0], x[1]);
  } else {
    float2 e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      e[i] = x[2 * i];
      o[i] = x[2 * i + 1];
    }
    dft<H, S>(e);
    dft<H, S>(o);
#pragma unroll
    for (int q = 0; q < H; ++q) x[q] = cadd(e[q], (q == 0) ? o[0] : cmul(o[q], wr<S, R>(q)));
  }
}

// v[r] *= exp(S 2 pi i r k / (Ns R)) for r in [1, R): loads w, w^2, w^4, w^8 and forms each
// other power right before use (w^3 = w w^2, w^(8+r) = w^r w^8, ...), so at most the base
// powers and one product are live next to the data.
template <int S, int R, int Ns>
__device__ __forceinline__ void apply_twiddles(float2* v, int k, const float2* __restrict__ tw) {
  constexpr int NR = Ns * R;   // w = E_NR, and w^r = E_(NR / r) at the same k < Ns
  const float2 w1 = twiddle_at<S>(tw, NR, k);
  v[1] = cmul(v[1], w1);
  if constexpr (R >= 4) {
    const float2 w2 = twiddle_at<S>(tw, NR / 2, k);
    const float2 w3 = cmul(w1, w2);
    v[2] = cmul(v[2], w2);
    v[3] = cmul(v[3], w3);
    if constexpr (R >= 8) {
      const float2 w4 = twiddle_at<S>(tw, NR / 4, k);
      const float2 w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
      v[4] = cmul(v[4], w4);
      v[5] = cmul(v[5], w5);
      v[6] = cmul(v[6], w6);
      v[7] = cmul(v[7], w7);
      if constexpr (R >= 16) {
        const float2 w8 = twiddle_at<S>(tw, NR / 8, k);
        v[8] = cmul(v[8], w8);
        v[9] = cmul(v[9], cmul(w1, w8));
        v[10] = cmul(v[10], cmul(w2, w8));
        v[11] = cmul(v[11], cmul(w3, w8));
        v[12] = cmul(v[12], cmul(w4, w8));
        v[13] = cmul(v[13], cmul(w5, w8));
        v[14] = cmul(v[14], cmul(w6, w8));
        v[15] = cmul(v[15], cmul(w7, w8));
      }
    }
  }
}

// Forward butterfly: twiddle, then DFT. Adjoint butterfly: DFT, then twiddle.
template <int S, int R, int Ns, bool ADJ>
__device__ __forceinline__ void butterfly(float2* v, int k, const float2* __restrict__ tw) {
  if constexpr (!ADJ) {
    if constexpr (Ns > 1) apply_twiddles<S, R, Ns>(v, k, tw);
    dft<R, S>(v);
  } else {
    dft<R, S>(v);
    if constexpr (Ns > 1) apply_twiddles<S, R, Ns>(v, k, tw);
  }
}

// One pass over LINES lines, block of exactly LINES * L / 16 threads. Butterfly b maps to
// (line, j): LF puts consecutive b on consecutive lines, otherwise on consecutive j.
// Forward: loads at j + r L/R, stores at (j-k) R + k + q Ns. Adjoint: the reverse.
// LD(line, pos) -> float2, ST(line, pos, v). SYNC_MID separates loads from stores when the
// pass works in place. HALF (first pass, Ns = 1): forward, positions >= L/2 hold zeros and are
// not read (dft_half_in); adjoint, positions >= L/2 are not needed and not written
// (dft_half_out). LD and ST must still be valid there (the tensor-core pass ignores HALF).
template <int S, bool ADJ, int L, int R, int Ns, int LINES, bool LF, bool SYNC_MID, bool HALF = false, class LD,
          class ST>
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ tw, LD ld, ST st) {
  static_assert(!HALF || Ns == 1, "the half transforms are the Ns = 1 pass");
  static_assert(R % 2 == 0 || Ns == 1, "an odd radix is the Ns = 1 pass");
  constexpr int LR = L / R;
  constexpr int NB = (GBD_E + R - 1) / R;   // butterflies per thread (radix 3, 5: the last may be past the end)
  constexpr int T = LINES * L / GBD_E;
  constexpr int NBUT = LINES * LR;
  float2 v[NB][R];
  int bl[NB], bj[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * T;
    if (NB * T != NBUT && b >= NBUT) continue;
    int line, j;
    if (LF) {
      line = b % LINES;
      j = b / LINES;
    } else {
      line = b / LR;
      j = b % LR;
    }
    bl[i] = line;
    bj[i] = j;
    const int k = j % Ns;
#pragma unroll
    for (int r = 0; r < ((HALF && !ADJ) ? R / 2 : R); ++r) v[i][r] = ld(line, ADJ ? (j - k) * R + k + r * Ns : j + r * LR);
  }
  if (SYNC_MID) __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (NB * T != NBUT && threadIdx.x + i * T >= NBUT) continue;
    const int j = bj[i];
    const int k = j % Ns;
    if constexpr (HALF && ADJ)
      dft_half_out<R, S>(v[i]);
    else if constexpr (HALF)
      dft_half_in<R, S>(v[i]);
    else
      butterfly<S, R, Ns, ADJ>(v[i], k, tw);
#pragma unroll
    for (int q = 0; q < ((HALF && ADJ) ? R / 2 : R); ++q)
      st(bl[i], ADJ ? j + q * LR : (j - k) * R + k + q * Ns, v[i][q]);
  }
}

// The same pass in place in shared memory, with the padded addresses of a butterfly's R
// elements formed as one base plus compile-time strides where the padding allows it:
//   natural set  j + r L/R        : pad = pad(j) + r (L/R + L/R/16)     when L/R % 16 == 0
//   scattered set (j-k) R + k + q Ns: pad = pad(base) + q (Ns + Ns/16)   when Ns % 16 == 0,
//                                     pad = 17 j + q                      when Ns = 1, R = 16
// (other cases compute pad per element).
// HALF (the Ns = 1 pass, even R): forward, the upper half of each line is zero -- only the
// inputs r < R/2 are loaded and the butterfly is dft_half_in; adjoint, only the lower half of the
// output is kept -- dft_half_out and the stores q < R/2.
template <int S, bool ADJ, int L, int R, int Ns, int LINES, bool LF, int LS, bool HALF = false>
__device__ __forceinline__ void stockham_pass_sm(float2* sm, const float2* __restrict__ tw) {
  static_assert(R % 2 == 0 || Ns == 1, "an odd radix is the Ns = 1 pass");
  static_assert(!HALF || (Ns == 1 && R % 2 == 0), "the half transforms are the Ns = 1 pass of an even radix");
  constexpr int LR = L / R;
  constexpr int NB = (GBD_E + R - 1) / R;
  constexpr int T = LINES * L / GBD_E;
  constexpr int NBUT = LINES * LR;
  constexpr bool NAT_CONST = (LR % 16 == 0);
  constexpr bool SCA_CONST = (Ns % 16 == 0) || (Ns == 1 && R == 16);
  constexpr int NAT_STRIDE = LR + LR / 16;
  constexpr int SCA_STRIDE = (Ns == 1) ? 1 : Ns + Ns / 16;
  float2 v[NB][R];
  int nat0[NB], sca0[NB], bj[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * T;
    if (NB * T != NBUT && b >= NBUT) continue;
    int line, j;
    if (LF) {
      line = b % LINES;
      j = b / LINES;
    } else {
      line = b / LR;
      j = b % LR;
    }
    const int k = j % Ns;
    const int lb = line * LS;
    const int base = (j - k) * R + k;
    bj[i] = j;
    nat0[i] = lb + (NAT_CONST ? pad(j) : j);
    sca0[i] = lb + (SCA_CONST ? (Ns == 1 ? 17 * j : pad(base)) : base);
    auto nat = [&](int r) { return NAT_CONST ? nat0[i] + r * NAT_STRIDE : lb + pad(j + r * LR); };
    auto sca = [&](int q) { return SCA_CONST ? sca0[i] + q * SCA_STRIDE : lb + pad(base + q * Ns); };
#pragma unroll
    for (int r = 0; r < ((HALF && !ADJ) ? R / 2 : R); ++r) v[i][r] = sm[ADJ ? sca(r) : nat(r)];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (NB * T != NBUT && threadIdx.x + i * T >= NBUT) continue;
    const int j = bj[i];
    const int k = j % Ns;
    if constexpr (HALF && ADJ)
      dft_half_out<R, S>(v[i]);
    else if constexpr (HALF)
      dft_half_in<R, S>(v[i]);
    else
      butterfly<S, R, Ns, ADJ>(v[i], k, tw);
    const int lb_nat = nat0[i] - (NAT_CONST ? pad(j) : j);   // line base
    const int lb_sca = sca0[i] - (SCA_CONST ? (Ns == 1 ? 17 * j : pad((j - k) * R + k)) : (j - k) * R + k);
#pragma unroll
    for (int q = 0; q < ((HALF && ADJ) ? R / 2 : R); ++q) {
      int addr;
      if (ADJ)
        addr = NAT_CONST ? nat0[i] + q * NAT_STRIDE : lb_nat + pad(j + q * LR);
      else
        addr = SCA_CONST ? sca0[i] + q * SCA_STRIDE : lb_sca + pad((j - k) * R + k + q * Ns);
      sm[addr] = v[i][q];
    }
  }
}


}  // namespace gbd
