// Shared-memory Stockham FFT building blocks for the demag convolution passes.
//
// The convolution theorem step of Sec. II (Eq. 1 evaluated as FFT -> pointwise
// product -> inverse FFT) needs length-L complex FFTs, L a power of two, along
// x (half-length transform inside the real-to-complex step), y and z. Each
// thread block holds `lines` lines of length L in shared memory, laid out
// line-major with line stride LS (L plus optional padding). Every thread owns
// E = 16 complex values per pass and runs E/R radix-R butterflies on them, so
// a block has lines * L / 16 threads.
//
// Stockham autosort pass (radix R, Ns = product of the radices already done):
//   for butterfly j in [0, L/R):   k = j mod Ns
//     v[r] = a[j + r L/R] * w^(r k),  w = exp(s 2 pi i / (Ns R))
//     v    = DFT_R(v)
//     a'[(j / Ns) Ns R + k + q Ns] = v[q]
// After the last pass the line holds the DFT in natural order. s = -1 is the
// forward transform, s = +1 the unnormalised inverse.
//
// Twiddles come from one table tw[m] = exp(-2 pi i m / GBD_TW_LEN) written on
// the host in FP64 and rounded to FP32; a length-L transform reads it with
// stride GBD_TW_LEN / (Ns R).
#pragma once
#include <cuda_runtime.h>

#define GBD_TW_LEN 8192
#define GBD_E 16

namespace gbd {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by i (s = +1) or -i (s = -1)
template <int S>
__device__ __forceinline__ float2 cmul_i(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// exp(S * 2 pi i * m / GBD_TW_LEN) from the table (S = -1 table value, +1 its conjugate).
template <int S>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int m) {
  float2 w = __ldg(tw + (m & (GBD_TW_LEN - 1)));
  return S < 0 ? w : cconj(w);
}

// ---- register DFTs of size 2, 4, 8, 16 (sign S) -------------------------------------------
template <int S>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

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
  float2 t1 = make_float2(h * (o[1].x - S * o[1].y), h * (o[1].y + S * o[1].x));  // w8^1 = h (1 + S i)
  float2 t2 = cmul_i<S>(o[2]);                                                    // w8^2 = S i
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
  // cos(q pi / 8), sin(q pi / 8) for q = 0..7
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
    float2 w = make_float2(c[q], S * s[q]);
    float2 t = cmul(o[q], w);
    x[q] = cadd(e[q], t);
    x[q + 8] = csub(e[q], t);
  }
}

template <int R, int S>
__device__ __forceinline__ void dft(float2* x) {
  if constexpr (R == 2) {
    dft2<S>(x[0], x[1]);
  } else if constexpr (R == 4) {
    dft4<S>(x);
  } else if constexpr (R == 8) {
    dft8<S>(x);
  } else {
    dft16<S>(x);
  }
}

// ---- one Stockham pass over the lines of a block -------------------------------------------
// Butterfly b in [0, lines * L / R) maps to (line, j): LINE_FAST puts consecutive b on
// consecutive lines (for line-interleaved global data), otherwise on consecutive j.
// LD(line, idx) -> float2 and ST(line, idx, v) do the memory traffic; when both touch
// the same shared buffer the pass is in place, separated by the barrier between them.
template <int R, int S, bool LINE_FAST, class LD, class ST>
__device__ __forceinline__ void stockham_pass(int L, int Ns, int lines, const float2* __restrict__ tw,
                                              LD ld, ST st) {
  constexpr int NB = GBD_E / R;  // butterflies per thread
  const int LR = L / R;
  const int nthreads = blockDim.x;
  float2 v[NB][R];
  int bl[NB], bj[NB];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    int b = threadIdx.x + i * nthreads;
    int line, j;
    if (LINE_FAST) {
      line = b % lines;
      j = b / lines;
    } else {
      line = b / LR;
      j = b - line * LR;
    }
    bl[i] = line;
    bj[i] = j;
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = ld(line, j + r * LR);
  }
  __syncthreads();
  const int tstride = GBD_TW_LEN / (Ns * R);
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int j = bj[i];
    const int k = j & (Ns - 1);
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], twiddle<S>(tw, r * k * tstride));
    }
    dft<R, S>(v[i]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) st(bl[i], base + q * Ns, v[i][q]);
  }
  __syncthreads();
}

// Radix of pass p for a length-L transform: 16s first, then the remainder 8, 4 or 2.
__host__ __device__ inline int radix_count(int L) {
  int n = 0;
  while (L > 1) {
    L = (L >= 16) ? L / 16 : 1;
    ++n;
  }
  return n;
}

// Full length-L transform of every line in place in shared memory.
// buf: line-major, line stride LS (float2 units).
template <int S, bool LINE_FAST>
__device__ void fft_lines_smem(float2* buf, int L, int LS, int lines, const float2* __restrict__ tw) {
  auto ld = [=](int line, int idx) { return buf[line * LS + idx]; };
  auto st = [=](int line, int idx, float2 v) { buf[line * LS + idx] = v; };
  int Ns = 1;
  int rem = L;
  while (rem > 1) {
    if (rem >= 16) {
      stockham_pass<16, S, LINE_FAST>(L, Ns, lines, tw, ld, st);
      Ns *= 16;
      rem /= 16;
    } else if (rem == 8) {
      stockham_pass<8, S, LINE_FAST>(L, Ns, lines, tw, ld, st);
      Ns *= 8;
      rem = 1;
    } else if (rem == 4) {
      stockham_pass<4, S, LINE_FAST>(L, Ns, lines, tw, ld, st);
      Ns *= 4;
      rem = 1;
    } else {
      stockham_pass<2, S, LINE_FAST>(L, Ns, lines, tw, ld, st);
      Ns *= 2;
      rem = 1;
    }
  }
}

}  // namespace gbd
