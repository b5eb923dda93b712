// x-row kernels for the transform lengths Lx = 3 * 2^k and 5 * 2^k (FP32; gbd_fft.cuh), so that
// the zero padding of Sec. II can stop at the smallest length 2 Lx >= 2 nx - 1 of the form
// 2^a 3^b 5^c with b + c <= 1 instead of the next power of two: row_kernel (one tile shape)
// and the persistent pipelined kernel (gbd_rowpipe.cuh) where it applies.
#include "gbd_rowpipe.cuh"

namespace gbd {

// Calls f(std::integral_constant<int, LX>) for an instantiated mixed length.
template <class F>
static bool mixed_switch(int L, F f) {
  switch (L) {
#define GBD_MIXED_LEN(N)                  \
  case N:                                 \
    f(std::integral_constant<int, N>());  \
    return true;
    GBD_MIXED_LEN(96)
    GBD_MIXED_LEN(160)
    GBD_MIXED_LEN(192)
    GBD_MIXED_LEN(320)
    GBD_MIXED_LEN(384)
    GBD_MIXED_LEN(640)
    GBD_MIXED_LEN(768)
    GBD_MIXED_LEN(1280)
    GBD_MIXED_LEN(1536)
    GBD_MIXED_LEN(2560)
    GBD_MIXED_LEN(3072)
#undef GBD_MIXED_LEN
    default: return false;
  }
}

bool row_dispatch_mixed(int Lx, int var, const RowArgs* a, const float2* tw, cudaStream_t st) {
  auto sw = [](int L, auto f) { return mixed_switch(L, f); };
  if (!a) {   // prepare every kernel of this length
    pipe_dispatch_with(sw, Lx, -1, nullptr, nullptr, nullptr);
    return mixed_switch(Lx, [&](auto lx) {
      constexpr int LX = decltype(lx)::value;
      row_launch_t<LX, row_rb(LX, 0), 0>(nullptr, nullptr, nullptr);
    });
  }
  if (var >= 2) {
    const int kind = pipe_kind(Lx, *a, var);
    if (kind >= 0 && pipe_dispatch_with(sw, Lx, kind, a, tw, st)) return true;
  }
  return mixed_switch(Lx, [&](auto lx) {
    constexpr int LX = decltype(lx)::value;
    row_launch_t<LX, row_rb(LX, 0), 0>(a, tw, st);
  });
}

}  // namespace gbd
