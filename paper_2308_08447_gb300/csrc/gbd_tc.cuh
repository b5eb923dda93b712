// Radix-16 Stockham pass with the 16-point DFT on the tensor cores, split into two 16-bit
// halves (hi + lo) with FP32 accumulation -- the optional precision variants of the FFT stages:
// PREC = 1 splits into BF16, PREC = 2 into FP16.
//
// A butterfly's DFT is the real 32 x 32 product  [Yr; Yi] = [C, -sS; sS, C] [Xr; Xi]  with
// C_qr = cos(2 pi q r / 16), S_qr = sin(2 pi q r / 16) and s the transform sign. Both operands
// are split, A = Ah + Al and X = Xh + Xl with Ah = h(A), Al = h(A - Ah) (likewise X, h the
// rounding to the 16-bit type), and Y ~= Ah Xh + Ah Xl + Al Xh in FP32; the dropped Al Xl is
// below 2^-16 (BF16) or 2^-22 (FP16) of the terms.
// * BF16 keeps FP32's exponent range, so the data need no scaling; each operand is represented
//   to about 2^-16 relative.
// * FP16 has 11 significant bits but a range of about 6e-8 .. 65504, so each butterfly's 32 real
//   inputs are first scaled by a power of two that brings their largest magnitude into
//   [0.5, 1) (the Sec. II rule of halving the precision only after normalization) and its 32
//   outputs are scaled back; both scalings are exact. An operand is then represented to about
//   2^-22 of the butterfly's largest input.
//
// mma.sync.m16n8k16 (16-bit in, FP32 accumulate): a warp takes 8 butterflies (the n = 8 columns)
// per group and 4 groups per pass, the same 32 butterflies its threads take in the FP32 pass.
// With g = lane / 4 and t = lane % 4, lane holds for butterfly n = g the inputs r in
// {2t, 2t+1, 2t+8, 2t+9} (B fragment rows: k-tile 0 = real parts, k-tile 1 = imaginary parts)
// and receives the outputs q in {g, g+8} of butterflies {2t, 2t+1} (C fragment, m-tile 0 =
// real parts, m-tile 1 = imaginary parts). Twiddles stay in FP32: applied to the inputs in a
// forward pass and to the outputs in an adjoint pass, exactly as in the FP32 pass.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "gbd_fft.cuh"

namespace gbd {

// bits of a pair of 16-bit values (PREC 1: bfloat16, 2: half) with lo in the low half
template <int PREC>
__device__ __forceinline__ unsigned pack16(float lo, float hi) {
  if constexpr (PREC == 1) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
  } else {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
  }
}

// x = hi + lo in 16-bit pairs: (a, b) -> hi bits, lo bits
template <int PREC>
__device__ __forceinline__ void split2(float a, float b, unsigned& hi, unsigned& lo) {
  float ha, hb;
  if constexpr (PREC == 1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    ha = __low2float(h);
    hb = __high2float(h);
    hi = *reinterpret_cast<const unsigned*>(&h);
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    ha = __low2float(h);
    hb = __high2float(h);
    hi = *reinterpret_cast<const unsigned*>(&h);
  }
  lo = pack16<PREC>(a - ha, b - hb);
}

template <int PREC>
__device__ __forceinline__ void mma16(float* d, const unsigned* a, unsigned b0, unsigned b1) {
  if constexpr (PREC == 1)
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  else
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// cos / sin of pi m / 8, m in [0, 16)
__device__ __forceinline__ float cos16(int m) {
  const float c[16] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                       0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f,
                       -1.0f, -0.92387953251128675613f, -0.70710678118654752440f, -0.38268343236508977173f,
                       0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f};
  return c[m & 15];
}
__device__ __forceinline__ float sin16(int m) { return cos16(m - 4); }

// Element (row, col) of the real 32 x 32 DFT-16 matrix for sign S: rows 0..15 give Re Y_q,
// rows 16..31 Im Y_q; cols 0..15 take Re X_r, cols 16..31 Im X_r.
template <int S>
__device__ __forceinline__ float dft16_real(int row, int col) {
  const int q = row & 15, r = col & 15;
  const int m = (q * r) & 15;  // angle 2 pi q r / 16 = pi m / 8
  const float c = cos16(m), s = S * sin16(m);
  if (row < 16) return col < 16 ? c : -s;
  return col < 16 ? s : c;
}

// A fragments of the split matrix: frag[mt][kt][hi/lo][4 registers]
template <int S, int PREC>
struct Dft16Frags {
  unsigned f[2][2][2][4];
  __device__ __forceinline__ void build(int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        const int r0 = mt * 16 + g, c0 = kt * 16 + 2 * t;
        const float v[8] = {dft16_real<S>(r0, c0), dft16_real<S>(r0, c0 + 1),
                            dft16_real<S>(r0 + 8, c0), dft16_real<S>(r0 + 8, c0 + 1),
                            dft16_real<S>(r0, c0 + 8), dft16_real<S>(r0, c0 + 9),
                            dft16_real<S>(r0 + 8, c0 + 8), dft16_real<S>(r0 + 8, c0 + 9)};
#pragma unroll
        for (int i = 0; i < 4; ++i) split2<PREC>(v[2 * i], v[2 * i + 1], f[mt][kt][0][i], f[mt][kt][1][i]);
      }
  }
  // The same fragments from the table that dft16_frag_kernel wrote once per mesh after the
  // twiddle levels: register r of lane l at word r * 32 + l of table (PREC - 1) * 2 + (S > 0).
  __device__ __forceinline__ void load(const float2* __restrict__ tw, int lane) {
    const unsigned* F = reinterpret_cast<const unsigned*>(tw + 2 * GBD_TW_LEN) + ((PREC - 1) * 2 + (S > 0)) * 1024;
#pragma unroll
    for (int r = 0; r < 32; ++r) (&f[0][0][0][0])[r] = __ldg(F + r * 32 + lane);
  }
};

// Radix-16 pass (forward: loads j + r L/16, stores (j-k) 16 + k + q Ns; adjoint: reverse),
// block of exactly LINES * L / 16 threads, like stockham_pass.
template <int PREC, int S, bool ADJ, int L, int Ns, int LINES, bool LF, bool SYNC_MID, class LD, class ST>
__device__ __forceinline__ void stockham_pass_tc(const float2* __restrict__ tw, LD ld, ST st) {
  constexpr int R = 16;
  constexpr int LR = L / R;
  constexpr int NR = Ns * R;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int rin[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
  auto map = [&](int b, int& line, int& j) {
    if (LF) {
      line = b % LINES;
      j = b / LINES;
    } else {
      line = b / LR;
      j = b % LR;
    }
  };
  // loads: 4 groups of 8 butterflies, 4 inputs each
  float2 x[4][4];
#pragma unroll
  for (int grp = 0; grp < 4; ++grp) {
    int line, j;
    map(warp * 32 + grp * 8 + g, line, j);
    const int k = j % Ns;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rin[i];
      float2 v = ld(line, ADJ ? (j - k) * R + k + r * Ns : j + r * LR);
      if (!ADJ && Ns > 1 && r > 0) v = cmul(v, twiddle_at<S>(tw, NR, (r * k) & (NR - 1)));
      x[grp][i] = v;
    }
  }
  if (SYNC_MID) __syncthreads();
  Dft16Frags<S, PREC> A;
  A.load(tw, lane);
#pragma unroll
  for (int grp = 0; grp < 4; ++grp) {
    // FP16: butterfly g's inputs sit on lanes 4g .. 4g+3; scale them by 2^-e, e the binary
    // exponent of their largest magnitude (frexp: max = f 2^e, f in [0.5, 1); e = 0 for zero)
    int e = 0;
    if constexpr (PREC == 2) {
      float mx = 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) mx = fmaxf(mx, fmaxf(fabsf(x[grp][i].x), fabsf(x[grp][i].y)));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
      frexpf(mx, &e);
      e = max(e, -125);   // a subnormal maximum keeps the scale 2^125 finite
      const float sc = ldexpf(1.f, -e);
#pragma unroll
      for (int i = 0; i < 4; ++i) x[grp][i] = cscale(x[grp][i], sc);
    }
    // B fragments: k-tile 0 real parts, k-tile 1 imaginary parts; rows (r) 2t, 2t+1 | 2t+8, 2t+9
    unsigned bh[2][2], bl[2][2];
    split2<PREC>(x[grp][0].x, x[grp][1].x, bh[0][0], bl[0][0]);
    split2<PREC>(x[grp][2].x, x[grp][3].x, bh[0][1], bl[0][1]);
    split2<PREC>(x[grp][0].y, x[grp][1].y, bh[1][0], bl[1][0]);
    split2<PREC>(x[grp][2].y, x[grp][3].y, bh[1][1], bl[1][1]);
    float y[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
      for (int i = 0; i < 4; ++i) y[mt][i] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        mma16<PREC>(y[mt], A.f[mt][kt][1], bh[kt][0], bh[kt][1]);   // Al Xh
        mma16<PREC>(y[mt], A.f[mt][kt][0], bl[kt][0], bl[kt][1]);   // Ah Xl
        mma16<PREC>(y[mt], A.f[mt][kt][0], bh[kt][0], bh[kt][1]);   // Ah Xh
      }
    }
    // outputs: q in {g, g+8} of butterflies n in {2t, 2t+1}: (Re, Im) = (y[0][.], y[1][.])
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      int line, j;
      map(warp * 32 + grp * 8 + 2 * t + c, line, j);
      const int k = j % Ns;
      float usc = 1.f;
      if constexpr (PREC == 2) usc = ldexpf(1.f, __shfl_sync(0xffffffffu, e, 4 * (2 * t + c)));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = g + 8 * h;
        float2 v = make_float2(y[0][2 * h + c], y[1][2 * h + c]);
        if constexpr (PREC == 2) v = cscale(v, usc);
        if (ADJ && Ns > 1 && q > 0) v = cmul(v, twiddle_at<S>(tw, NR, (q * k) & (NR - 1)));
        st(line, ADJ ? j + q * LR : (j - k) * R + k + q * Ns, v);
      }
    }
  }
}

// ---- pass selection by precision -------------------------------------------------------------
// PREC = 0: FP32 everywhere. PREC = 1 / 2: every radix-16 pass on the tensor cores, split
// BF16 / split FP16.

// HALF: see stockham_pass (the tensor-core pass reads and writes every position through LD / ST).
template <int PREC, int S, bool ADJ, int L, int R, int Ns, int LINES, bool LF, bool SYNC_MID, bool HALF = false,
          class LD, class ST>
__device__ __forceinline__ void pass_any(const float2* __restrict__ tw, LD ld, ST st) {
  if constexpr (PREC != 0 && R == 16)
    stockham_pass_tc<PREC, S, ADJ, L, Ns, LINES, LF, SYNC_MID>(tw, ld, st);
  else
    stockham_pass<S, ADJ, L, R, Ns, LINES, LF, SYNC_MID, HALF>(tw, ld, st);
}

template <int PREC, int S, bool ADJ, int L, int R, int Ns, int LINES, bool LF, int LS>
__device__ __forceinline__ void pass_sm_any(float2* sm, const float2* __restrict__ tw) {
  if constexpr (PREC != 0 && R == 16) {
    auto ld = [&](int line, int i) { return sm[line * LS + pad(i)]; };
    auto st = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };
    stockham_pass_tc<PREC, S, ADJ, L, Ns, LINES, LF, true>(tw, ld, st);
  } else {
    stockham_pass_sm<S, ADJ, L, R, Ns, LINES, LF, LS>(sm, tw);
  }
}

// Passes [P, PEND) of the forward chain (sign S) in place in shared memory; LS is the
// caller's line stride in float2 units.
template <int S, int L, bool CONV, int LINES, bool LF, int LS, int P, int PEND, int PREC = 0>
__device__ __forceinline__ void fwd_passes_smem(float2* sm, const float2* __restrict__ tw) {
  if constexpr (P < PEND) {
    constexpr int R = radix_at(L, CONV, P);
    constexpr int Ns = ns_at(L, CONV, P);
    pass_sm_any<PREC, S, false, L, R, Ns, LINES, LF, LS>(sm, tw);
    __syncthreads();
    fwd_passes_smem<S, L, CONV, LINES, LF, LS, P + 1, PEND, PREC>(sm, tw);
  }
}

// Adjoint passes P-1 down to PEND (inclusive) in place in shared memory.
template <int S, int L, bool CONV, int LINES, bool LF, int LS, int P, int PEND, int PREC = 0>
__device__ __forceinline__ void adj_passes_smem(float2* sm, const float2* __restrict__ tw) {
  if constexpr (P > PEND) {
    constexpr int R = radix_at(L, CONV, P - 1);
    constexpr int Ns = ns_at(L, CONV, P - 1);
    pass_sm_any<PREC, S, true, L, R, Ns, LINES, LF, LS>(sm, tw);
    __syncthreads();
    adj_passes_smem<S, L, CONV, LINES, LF, LS, P - 1, PEND, PREC>(sm, tw);
  }
}

}  // namespace gbd
