// Device code of the convolution kernels (Sec. II, Eq. 1): the pointwise product with the
// transformed tensor (Appendix A, KernelMultiplication) fused with the transforms along the
// last axis -- y for a single-layer mesh (nz = 1), z for 3D meshes ("pipelined convolution ...
// in the same routine", Appendix A). Shared by the translation units of the FP32 kernels
// (gbd_conv.cu) and of the split 16-bit kernels (gbd_conv_bf16.cu, gbd_conv_fp16.cu).
#pragma once
#include <type_traits>

#include "gbd_launch.cuh"

namespace gbd {

// ---------------------------------------------------------------------------------------------
// Kernel product H~_a = sum_b K~_ab M~_b with the packed real spectrum. Stored indices are
// k' = k for k <= P/2 and P - k above; components odd along that axis change sign there
// (xy, yz odd in y; xz, yz odd in z). The 1/(Px Py Pz) and the minus sign of Eq. 1 are in K~.
// The last forward pass, the product and the first adjoint pass run in registers on one
// thread per butterfly position j, for the NC components that the product couples (lines
// line0 + c * lstride, c < NC): all three in 3D; for a film, where N_xz = N_yz = 0, the
// pair (x, y) and then z alone, which keeps fewer values live. mul(k, h0, h1, h2) gets the
// NC values as (v0, v1, v2) with the missing ones aliased to the last present one.
// ---------------------------------------------------------------------------------------------

template <int L, int RL, int NSL, class LD, class ST, class MUL, int NC = 3>
__device__ __forceinline__ void fused_item(int line0, int lstride, int j, const float2* __restrict__ tw, LD ld, ST st,
                                           MUL mul) {
  constexpr int LR = L / RL;
  float2 v[NC][RL];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int r = 0; r < RL; ++r) v[c][r] = ld(line0 + c * lstride, j + r * LR);
  if constexpr (RL > 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) butterfly<-1, RL, NSL, false>(v[c], j, tw);
#pragma unroll
    for (int q = 0; q < RL; ++q) mul(j + q * LR, v[0][q], v[NC > 1 ? 1 : 0][q], v[NC - 1][q]);
#pragma unroll
    for (int c = 0; c < NC; ++c) butterfly<1, RL, NSL, true>(v[c], j, tw);
  } else {
    mul(j, v[0][0], v[NC > 1 ? 1 : 0][0], v[NC - 1][0]);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int r = 0; r < RL; ++r) st(line0 + c * lstride, j + r * LR, v[c][r]);
}

// film: one block = C columns kx, three components each, lines = c * C + cc.
template <int L, int C_, int PREC>
__global__ void __launch_bounds__(3 * C_ * L / GBD_E,
                                  PREC == 0 ? min_blocks_film(3 * C_ * L / GBD_E) : min_blocks(3 * C_ * L / GBD_E))
    film_conv_kernel(ColArgs a, const float2* __restrict__ tw) {
  constexpr int C = C_;
  constexpr int LINES = 3 * C;
  constexpr int T = LINES * L / GBD_E;
  constexpr int LS = line_stride<L, false>();
  constexpr int NP = npasses(L, true);
  constexpr int RL = NP >= 1 ? radix_at(L, true, NP - 1) : 1;
  constexpr int NSL = NP >= 1 ? ns_at(L, true, NP - 1) : 1;
  constexpr int LR = L / RL;
  constexpr int KY = L / 2 + 1;
  extern __shared__ float2 sm[];
  pdl_wait_then_release();
  const int kx0 = blockIdx.x * C;
  const int ny = a.ny, Hx = a.Hx;
  float2* S = a.dst;

  auto gptr = [&](int line) { return S + (long long)((line / C) * Hx + kx0 + line % C) * ny; };
  auto gld = [&](int line, int y) {
    return (y < ny && kx0 + line % C < Hx) ? gptr(line)[y] : make_float2(0.f, 0.f);
  };
  auto gst = [&](int line, int y, float2 v) {
    if (y < ny && kx0 + line % C < Hx) gptr(line)[y] = v;
  };
  auto sld = [&](int line, int i) { return sm[line * LS + pad(i)]; };
  auto sst = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };

  // An item is a butterfly position j of column cc: the coupled (x, y) pair (two lines) and the
  // z line. When the C LR pair items leave threads over (C LR < T), the first C LR threads take
  // the pairs and the others the z lines, so that every thread does about two lines' work.
  auto run_fused = [&](auto ld, auto st) {
    constexpr bool SPLIT = (C * LR < T) && ((C * LR) % (T - C * LR) == 0);
    auto item = [&](int it, bool xy, bool zz) {
      const int cc = it / LR, j = it % LR;
      const int kx = kx0 + cc;
      auto kfetch = [&](int ky, float& sy) {
        int kyp = ky;
        sy = 1.f;
        if (L > 1 && ky > L / 2) {
          kyp = L - ky;
          sy = -1.f;
        }
        return __ldg(a.Kf + (long long)kx * KY + kyp);
      };
      auto mulxy = [&](int ky, float2& m0, float2& m1, float2&) {
        if (kx >= Hx) return;
        float sy;
        const float4 k4 = kfetch(ky, sy);
        const float kxy = sy * k4.w;
        const float2 h0 = make_float2(k4.x * m0.x + kxy * m1.x, k4.x * m0.y + kxy * m1.y);
        const float2 h1 = make_float2(kxy * m0.x + k4.y * m1.x, kxy * m0.y + k4.y * m1.y);
        m0 = h0;
        m1 = h1;
      };
      auto mulz = [&](int ky, float2&, float2&, float2& m2) {
        if (kx >= Hx) return;
        float sy;
        const float4 k4 = kfetch(ky, sy);
        m2 = make_float2(k4.z * m2.x, k4.z * m2.y);
      };
      if (xy) fused_item<L, RL, NSL, decltype(ld), decltype(st), decltype(mulxy), 2>(cc, C, j, tw, ld, st, mulxy);
      if (zz) fused_item<L, RL, NSL, decltype(ld), decltype(st), decltype(mulz), 1>(cc + 2 * C, C, j, tw, ld, st, mulz);
    };
    if constexpr (SPLIT) {
      if (threadIdx.x < C * LR) {
        item(threadIdx.x, true, false);
      } else {
        for (int it = threadIdx.x - C * LR; it < C * LR; it += T - C * LR) item(it, false, true);
      }
    } else {
      for (int it = threadIdx.x; it < C * LR; it += T) item(it, true, true);
    }
  };

  if constexpr (NP <= 1) {
    run_fused(gld, gst);
  } else {
    // Radix-16 outer passes (FP32, one butterfly per thread, lines not interleaved): the thread's
    // line and butterfly j are fixed, its global elements y = j + r L/16 of one column pointer and
    // its shared-memory elements 16 j + q at the padded 17 j + q; with the upper half of a y line
    // zero (2 ny <= L) the first pass is a half-input DFT and the last one computes and stores
    // only the kept half.
    constexpr int R0 = radix_at(L, true, 0);
    constexpr bool FAST = (PREC == 0 && R0 == 16);
    const int fline = threadIdx.x / (L / 16), fj = threadIdx.x % (L / 16);
    const bool fok = kx0 + fline % C < Hx;
    const bool half = 2 * ny <= L;
    if constexpr (FAST) {
      const float2* gp = gptr(fline);
      float2 v[16];
      if (half) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int y = fj + r * (L / 16);
          v[r] = (fok && y < ny) ? gp[y] : make_float2(0.f, 0.f);
        }
        dft_half_in<16, -1>(v);
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int y = fj + r * (L / 16);
          v[r] = (fok && y < ny) ? gp[y] : make_float2(0.f, 0.f);
        }
        dft<16, -1>(v);
      }
      float2* sp = sm + fline * LS + 17 * fj;
#pragma unroll
      for (int q = 0; q < 16; ++q) sp[q] = v[q];
    } else {
      pass_any<PREC, -1, false, L, R0, 1, LINES, false, false>(tw, gld, sst);
    }
    __syncthreads();
    fwd_passes_smem<-1, L, true, LINES, false, LS, 1, NP - 1, PREC>(sm, tw);
    run_fused(sld, sst);
    __syncthreads();
    adj_passes_smem<1, L, true, LINES, false, LS, NP - 1, 1, PREC>(sm, tw);
    if constexpr (FAST) {
      const float2* sp = sm + fline * LS + 17 * fj;
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = sp[r];
      float2* gp = gptr(fline);
      if (half) {
        dft_half_out<16, 1>(v);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int y = fj + q * (L / 16);
          if (fok && y < ny) gp[y] = v[q];
        }
      } else {
        dft<16, 1>(v);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int y = fj + q * (L / 16);
          if (fok && y < ny) gp[y] = v[q];
        }
      }
    } else {
      pass_any<PREC, 1, true, L, R0, 1, LINES, false, false>(tw, sld, gst);
    }
  }
}

// 3D z convolution: one block = W consecutive columns q = kx Py + ky of the y spectrum T,
// three components each (lines c W + w); the z FFT reads the nz planes (zero padding above),
// the product couples the three components, and the adjoint z FFT writes back the nz planes.
template <int L, int W_, int PREC>
__global__ void __launch_bounds__(3 * W_ * L / GBD_E,
                                  PREC == 0 ? min_blocks_film(3 * W_ * L / GBD_E) : min_blocks(3 * W_ * L / GBD_E))
    z_conv_kernel(ColArgs a, const float2* __restrict__ tw) {
  constexpr int W = W_;
  constexpr int LINES = 3 * W;
  constexpr int T = LINES * L / GBD_E;
  constexpr int LS = line_stride<L, true>();
  constexpr int NP = npasses(L, true);
  constexpr int RL = radix_at(L, true, NP - 1);
  constexpr int NSL = ns_at(L, true, NP - 1);
  constexpr int LR = L / RL;
  extern __shared__ float2 sm[];
  const long long q0 = (long long)blockIdx.x * W;
  const int nz = a.nz;
  const long long Q = a.Q;
  const int Qi = (int)Q;   // Hx Py <= 4097 * 4096: a plane offset z Q fits in 32-bit int arithmetic
  float2* D = a.dst;
  // element z of line (component c = line / W, column q0 + line % W): the line's base, computed
  // once per line by the compiler, plus z Q
  auto lbase = [&](int line) { return D + (long long)(line / W) * nz * Q + q0 + line % W; };
  auto gld = [&](int line, int z) {
    return (z < nz && q0 + line % W < Q) ? lbase(line)[(long long)z * Qi] : make_float2(0.f, 0.f);
  };
  auto gst = [&](int line, int z, float2 v) {
    if (z < nz && q0 + line % W < Q) lbase(line)[(long long)z * Qi] = v;
  };
  auto sld = [&](int line, int i) { return sm[line * LS + pad(i)]; };
  auto sst = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };
  const int Py = a.Py, KY = a.Py / 2 + 1, Pyq = a.Pyq;
  auto run_fused = [&](auto ld, auto st) {
    for (int it = threadIdx.x; it < W * LR; it += T) {
      const int w = it % W, j = it / W;
      const long long q = q0 + w;
      const int kx = (int)(q / Pyq);
      const int ky = (int)(q - (long long)kx * Pyq);
      int kyp = ky;
      float sy = 1.f;
      if (Py > 1 && ky > Py / 2) {
        kyp = Py - ky;
        sy = -1.f;
      }
      const float* kbase = a.K3 + ((long long)kx * KY + kyp) * 6;   // + kz' Hx KY 6
      auto mul = [&](int kz, float2& m0, float2& m1, float2& m2) {
        if (q >= Q) return;
        int kzp = kz;
        float sz = 1.f;
        if (kz > L / 2) {
          kzp = L - kz;
          sz = -1.f;
        }
        const float* kp = kbase + (long long)kzp * a.Hx * KY * 6;
        const float2 k01 = __ldg(reinterpret_cast<const float2*>(kp));
        const float2 k23 = __ldg(reinterpret_cast<const float2*>(kp + 2));
        const float2 k45 = __ldg(reinterpret_cast<const float2*>(kp + 4));
        const float kxx = k01.x, kyy = k01.y, kzz = k23.x;
        const float kxy = sy * k23.y, kxz = sz * k45.x, kyz = sy * sz * k45.y;
        const float2 h0 = make_float2(kxx * m0.x + kxy * m1.x + kxz * m2.x, kxx * m0.y + kxy * m1.y + kxz * m2.y);
        const float2 h1 = make_float2(kxy * m0.x + kyy * m1.x + kyz * m2.x, kxy * m0.y + kyy * m1.y + kyz * m2.y);
        const float2 h2 = make_float2(kxz * m0.x + kyz * m1.x + kzz * m2.x, kxz * m0.y + kyz * m1.y + kzz * m2.y);
        m0 = h0;
        m1 = h1;
        m2 = h2;
      };
      fused_item<L, RL, NSL>(w, W, j, tw, ld, st, mul);
    }
  };
  if constexpr (NP == 1) {
    run_fused(gld, gst);
  } else {
    // open z (Pz >= 2 nz): zero upper half in, cropped out; periodic z (Pz = nz): whole lines
    const bool half = 2 * nz <= L;
    // The outer passes of a radix-16 first pass (one butterfly per thread, FP32): the thread's
    // line and butterfly j are fixed, its global elements are z = j + r L/16 of one line base,
    // and its shared-memory elements 16 j + q sit at 17 j + q (padded), so addresses are one base
    // each plus constant offsets.
    constexpr int R0 = radix_at(L, true, 0);
    constexpr bool FAST = (PREC == 0 && R0 == 16 && T == LINES * (L / 16));
    const int fline = threadIdx.x % LINES, fj = threadIdx.x / LINES;
    const bool fq = q0 + fline % W < Q;
    if (FAST && half) {
      const float2* gp = lbase(fline);
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int z = fj + r * (L / 16);
        v[r] = (fq && z < nz) ? gp[(long long)z * Qi] : make_float2(0.f, 0.f);
      }
      dft_half_in<16, -1>(v);
      float2* sp = sm + fline * LS + 17 * fj;
#pragma unroll
      for (int q = 0; q < 16; ++q) sp[q] = v[q];
    } else if (half) {
      pass_any<PREC, -1, false, L, R0, 1, LINES, true, false, true>(tw, gld, sst);
    } else {
      pass_any<PREC, -1, false, L, R0, 1, LINES, true, false>(tw, gld, sst);
    }
    __syncthreads();
    fwd_passes_smem<-1, L, true, LINES, true, LS, 1, NP - 1, PREC>(sm, tw);
    // The last forward pass, the product and the first adjoint pass as three in-place phases
    // over all threads: the last pass (Ns R = L) leaves frequency j + q L/R at the position
    // it read, so each phase touches only its own items' positions.
    // T is a multiple of LINES, so a thread keeps one line through its 16 / RL items, and with
    // LR a multiple of 16 an item's RL elements sit at pad(j) + r (LR + LR/16): one base address
    // per item and compile-time offsets.
    static_assert(T % LINES == 0 && (LINES * LR) % T == 0, "z convolution: items per thread");
    auto last_pass = [&](auto adj) {
      constexpr bool ADJ = decltype(adj)::value;
      constexpr int NI = LINES * LR / T;
      constexpr bool NAT = (LR % 16 == 0);
      constexpr int STRIDE = LR + LR / 16;
      const int line = threadIdx.x % LINES;
      const int j0 = threadIdx.x / LINES;
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int j = j0 + i * (T / LINES);
        float2* lp = sm + line * LS + (NAT ? pad(j) : 0);
        float2 v[RL];
#pragma unroll
        for (int r = 0; r < RL; ++r) v[r] = NAT ? lp[r * STRIDE] : lp[pad(j + r * LR)];
        butterfly<ADJ ? 1 : -1, RL, NSL, ADJ>(v, j, tw);
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          if (NAT)
            lp[r * STRIDE] = v[r];
          else
            lp[pad(j + r * LR)] = v[r];
        }
      }
    };
    last_pass(std::false_type());
    __syncthreads();
    // product at (column w, frequencies kz and Pz - kz): consecutive lanes take consecutive
    // columns; T is a multiple of W, so each thread keeps one column and its (kx, ky) are worked
    // out once. The stored kernel at kz' = kz serves both kz and Pz - kz (the latter with the
    // z-odd components xz, yz negated), so an item loads it once for the pair.
    static_assert(T % W == 0, "a thread's product items share one column");
    const int w = threadIdx.x % W;
    const long long q = q0 + w;
    const int kx = (int)q / Pyq;   // q < Q = Hx Py fits in int: 32-bit division
    const int ky = (int)q - kx * Pyq;
    int kyp = ky;
    float sy = 1.f;
    if (Py > 1 && ky > Py / 2) {
      kyp = Py - ky;
      sy = -1.f;
    }
    const float* kcol = a.K3 + ((long long)kx * KY + kyp) * 6;
    const long long kzs = (long long)a.Hx * KY * 6;      // kernel stride between kz planes
    for (int kz = threadIdx.x / W; kz <= L / 2 && q < Q; kz += T / W) {
      const float* kp = kcol + kz * kzs;
      const float2 k01 = __ldg(reinterpret_cast<const float2*>(kp));
      const float2 k23 = __ldg(reinterpret_cast<const float2*>(kp + 2));
      const float2 k45 = __ldg(reinterpret_cast<const float2*>(kp + 4));
      const float kxx = k01.x, kyy = k01.y, kzz = k23.x;
      const float kxy = sy * k23.y, kxz0 = k45.x, kyz0 = sy * k45.y;
      auto apply = [&](int z, float sz) {
        const float kxz = sz * kxz0, kyz = sz * kyz0;
        const float2 m0 = sld(w, z), m1 = sld(W + w, z), m2 = sld(2 * W + w, z);
        sst(w, z, make_float2(kxx * m0.x + kxy * m1.x + kxz * m2.x, kxx * m0.y + kxy * m1.y + kxz * m2.y));
        sst(W + w, z, make_float2(kxy * m0.x + kyy * m1.x + kyz * m2.x, kxy * m0.y + kyy * m1.y + kyz * m2.y));
        sst(2 * W + w, z, make_float2(kxz * m0.x + kyz * m1.x + kzz * m2.x, kxz * m0.y + kyz * m1.y + kzz * m2.y));
      };
      apply(kz, 1.f);
      if (kz > 0 && kz < L / 2) apply(L - kz, -1.f);
    }
    __syncthreads();
    last_pass(std::true_type());
    __syncthreads();
    adj_passes_smem<1, L, true, LINES, true, LS, NP - 1, 1, PREC>(sm, tw);
    if (FAST && half) {
      const float2* sp = sm + fline * LS + 17 * fj;
      float2 v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = sp[r];
      dft_half_out<16, 1>(v);
      float2* gp = lbase(fline);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int z = fj + q * (L / 16);
        if (fq && z < nz) gp[(long long)z * Qi] = v[q];
      }
    } else if (half) {
      pass_any<PREC, 1, true, L, R0, 1, LINES, true, false, true>(tw, sld, gst);
    } else {
      pass_any<PREC, 1, true, L, R0, 1, LINES, true, false>(tw, sld, gst);
    }
  }
}


// ---- launchers -------------------------------------------------------------------------------

// a == nullptr only prepares the kernel (shared-memory attribute), without a launch.
template <int L, int C, int PREC>
static void film_launch_t(const ColArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * C * L / GBD_E;
  const size_t smem = (size_t)3 * C * line_stride<L, false>() * sizeof(float2);
  prep(film_conv_kernel<L, C, PREC>, smem);
  if (a) launch_pdl(film_conv_kernel<L, C, PREC>, (a->Hx + C - 1) / C, T, smem, st, *a, tw);
}

template <int L, int W, int PREC>
static void zconv_launch_t(const ColArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * W * L / GBD_E;
  const size_t smem = (size_t)3 * W * line_stride<L, true>() * sizeof(float2);
  prep(z_conv_kernel<L, W, PREC>, smem);
  if (a) z_conv_kernel<L, W, PREC><<<(unsigned)((a->Q + W - 1) / W), T, smem, st>>>(*a, tw);
}

// Calls f(std::integral_constant<int, L>) for a transform length L in {1, 4, 8, ..., 4096}
// (first = 1 or 4) ; false for a length without an instantiation.
template <class F>
static bool conv_switch(int L, F f) {
  switch (L) {
#define GBD_CONV_LEN(N)                       \
  case N:                                     \
    f(std::integral_constant<int, N>());      \
    return true;
    GBD_CONV_LEN(1)
    GBD_CONV_LEN(4)
    GBD_CONV_LEN(8)
    GBD_CONV_LEN(16)
    GBD_CONV_LEN(32)
    GBD_CONV_LEN(64)
    GBD_CONV_LEN(128)
    GBD_CONV_LEN(256)
    GBD_CONV_LEN(512)
    GBD_CONV_LEN(1024)
    GBD_CONV_LEN(2048)
    GBD_CONV_LEN(4096)
#undef GBD_CONV_LEN
    default: return false;
  }
}

// Launch (a == nullptr: prepare) the film / z convolution of precision PREC for transform
// length Py / Pz, tile variant var (both when var < 0). Explicitly instantiated once per
// precision, each in its own translation unit, so the units build in parallel.
template <int PREC>
bool film_dispatch_p(int Py, int var, const ColArgs* a, const float2* tw, cudaStream_t st) {
  return conv_switch(Py, [&](auto l) {
    constexpr int L = decltype(l)::value;
    if (var <= 0) film_launch_t<L, film_cols(L, 0), PREC>(a, tw, st);
    if (var != 0) film_launch_t<L, film_cols(L, 1), PREC>(a, tw, st);
  });
}
template <int PREC>
bool z_dispatch_p(int Pz, int var, const ColArgs* a, const float2* tw, cudaStream_t st) {
  if (Pz < 4) return false;
  return conv_switch(Pz, [&](auto l) {
    constexpr int L = decltype(l)::value;
    if constexpr (L >= 4) {
      if (var <= 0) zconv_launch_t<L, zconv_cols(L, 0), PREC>(a, tw, st);
      if (var != 0) zconv_launch_t<L, zconv_cols(L, 1), PREC>(a, tw, st);
    }
  });
}
extern template bool film_dispatch_p<1>(int, int, const ColArgs*, const float2*, cudaStream_t);
extern template bool film_dispatch_p<2>(int, int, const ColArgs*, const float2*, cudaStream_t);
extern template bool z_dispatch_p<1>(int, int, const ColArgs*, const float2*, cudaStream_t);
extern template bool z_dispatch_p<2>(int, int, const ColArgs*, const float2*, cudaStream_t);

}  // namespace gbd
