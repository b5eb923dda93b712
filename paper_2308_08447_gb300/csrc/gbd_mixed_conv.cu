// Film convolution and 3D y passes for the transform lengths Py = 3 * 2^k and 5 * 2^k (FP32;
// gbd_fft.cuh), one tile shape each: the y padding of Sec. II at the smallest length
// >= 2 ny - 1 of the form 2^a 3^b 5^c with b + c <= 1.
#include "gbd_conv.cuh"
#include "gbd_ypass.cuh"

namespace gbd {

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

bool film_dispatch_mixed(int Py, const ColArgs* a, const float2* tw, cudaStream_t st) {
  return mixed_switch(Py, [&](auto l) {
    constexpr int L = decltype(l)::value;
    film_launch_t<L, film_cols(L, 0), 0>(a, tw, st);
  });
}

bool ypass_dispatch_mixed(int Py, bool inv, const ColArgs* a, const float2* tw, cudaStream_t st) {
  return mixed_switch(Py, [&](auto l) {
    constexpr int L = decltype(l)::value;
    if (inv)
      ypass_launch_t<L, ypass_lines(L, 0), true, 0>(a, tw, st);
    else
      ypass_launch_t<L, ypass_lines(L, 0), false, 0>(a, tw, st);
  });
}

}  // namespace gbd
