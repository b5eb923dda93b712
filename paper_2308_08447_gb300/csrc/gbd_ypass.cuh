// Device code of the 3D y passes of the demag convolution (Sec. II, Eq. 1; Appendix A yFFT
// forward and inverse): length-Py FFTs of contiguous y columns, the zero padding pruned on the
// way in and the crop applied on the way out. Shared by the power-of-two instances
// (gbd_ypass.cu) and the 3 * 2^k / 5 * 2^k ones (gbd_mixed_conv.cu).
#pragma once
#include "gbd_launch.cuh"

namespace gbd {

template <int L, int C_, bool INV, int PREC>
__global__ void __launch_bounds__(C_ * L / GBD_E, min_blocks(C_ * L / GBD_E))
    y_pass_kernel(ColArgs a, const float2* __restrict__ tw) {
  constexpr int LINES = C_;
  constexpr int LS = line_stride<L, false>();
  constexpr int NP = npasses(L, false);
  extern __shared__ float2 sm[];
  const long long l0 = (long long)blockIdx.x * LINES;
  const int ny = a.ny;
  const long long nl = a.lines_total;
  auto sld = [&](int line, int i) { return sm[line * LS + pad(i)]; };
  auto sst = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };
  if constexpr (!INV) {
    auto gld = [&](int line, int y) {
      return (y < ny && l0 + line < nl) ? a.src[(l0 + line) * ny + y] : make_float2(0.f, 0.f);
    };
    auto gst = [&](int line, int i, float2 v) {
      if (l0 + line < nl) a.dst[(l0 + line) * L + i] = v;
    };
    if constexpr (NP == 1) {
      pass_any<PREC, -1, false, L, radix_at(L, false, 0), 1, LINES, false, false>(tw, gld, gst);
    } else {
      pass_any<PREC, -1, false, L, radix_at(L, false, 0), 1, LINES, false, false>(tw, gld, sst);
      __syncthreads();
      fwd_passes_smem<-1, L, false, LINES, false, LS, 1, NP - 1, PREC>(sm, tw);
      pass_any<PREC, -1, false, L, radix_at(L, false, NP - 1), ns_at(L, false, NP - 1), LINES, false, false>(tw, sld,
                                                                                                           gst);
    }
  } else {
    auto gld = [&](int line, int i) {
      return (l0 + line < nl) ? a.src[(l0 + line) * L + i] : make_float2(0.f, 0.f);
    };
    auto gst = [&](int line, int y, float2 v) {
      if (y < ny && l0 + line < nl) a.dst[(l0 + line) * ny + y] = v;
    };
    if constexpr (NP == 1) {
      pass_any<PREC, 1, true, L, radix_at(L, false, 0), 1, LINES, false, false>(tw, gld, gst);
    } else {
      pass_any<PREC, 1, true, L, radix_at(L, false, NP - 1), ns_at(L, false, NP - 1), LINES, false, false>(tw, gld,
                                                                                                         sst);
      __syncthreads();
      adj_passes_smem<1, L, false, LINES, false, LS, NP - 1, 1, PREC>(sm, tw);
      pass_any<PREC, 1, true, L, radix_at(L, false, 0), 1, LINES, false, false>(tw, sld, gst);
    }
  }
}

// ---- launchers -------------------------------------------------------------------------------

// a == nullptr only prepares the kernel (shared-memory attribute), without a launch.
template <int L, int C, bool INV, int PREC>
static void ypass_launch_t(const ColArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = C * L / GBD_E;
  const size_t smem = (size_t)C * line_stride<L, false>() * sizeof(float2);
  prep(y_pass_kernel<L, C, INV, PREC>, smem);
  if (a) y_pass_kernel<L, C, INV, PREC><<<(unsigned)((a->lines_total + C - 1) / C), T, smem, st>>>(*a, tw);
}

}  // namespace gbd
