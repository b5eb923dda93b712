// sm_103a y passes of the 3D demag convolution (Sec. II, Eq. 1; Appendix A yFFT forward and
// inverse; device code in gbd_ypass.cuh): the power-of-two instances and the launchers.
#include "gbd_ypass.cuh"

namespace gbd {

// prec < 0 (with a == nullptr) prepares every precision
template <int L, int C, bool INV>
static void ypass_launch_p(int prec, const ColArgs* a, const float2* tw, cudaStream_t st) {
  if (prec <= 0) ypass_launch_t<L, C, INV, 0>(a, tw, st);
  if (prec == 1 || prec < 0) ypass_launch_t<L, C, INV, 1>(a, tw, st);
  if (prec == 2 || prec < 0) ypass_launch_t<L, C, INV, 2>(a, tw, st);
}

#define GBD_Y_CASE(L)                                             \
  case L:                                                         \
    if (var <= 0)                                                 \
      ypass_launch_p<L, ypass_lines(L, 0), INV>(prec, a, tw, st);       \
    if (var != 0)                                                 \
      ypass_launch_p<L, ypass_lines(L, 1), INV>(prec, a, tw, st);       \
    return true;

template <bool INV>
static bool ypass_dispatch(int Py, int var, int prec, const ColArgs* a, const float2* tw, cudaStream_t st) {
  switch (Py) {
    GBD_Y_CASE(4)
    GBD_Y_CASE(8)
    GBD_Y_CASE(16)
    GBD_Y_CASE(32)
    GBD_Y_CASE(64)
    GBD_Y_CASE(128)
    GBD_Y_CASE(256)
    GBD_Y_CASE(512)
    GBD_Y_CASE(1024)
    GBD_Y_CASE(2048)
    GBD_Y_CASE(4096)
    default: return false;
  }
}

bool launch_y_fwd(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st) {
  if (mixed_len(a.Py)) return prec == 0 && ypass_dispatch_mixed(a.Py, false, &a, tw, st);
  return ypass_dispatch<false>(a.Py, var, prec, &a, tw, st);
}
bool launch_y_inv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st) {
  if (mixed_len(a.Py)) return prec == 0 && ypass_dispatch_mixed(a.Py, true, &a, tw, st);
  return ypass_dispatch<true>(a.Py, var, prec, &a, tw, st);
}
bool prepare_y_passes(int Py, int prec) {
  if (mixed_len(Py))
    return prec <= 0 && ypass_dispatch_mixed(Py, false, nullptr, nullptr, nullptr) &&
           ypass_dispatch_mixed(Py, true, nullptr, nullptr, nullptr);
  return ypass_dispatch<false>(Py, -1, prec, nullptr, nullptr, nullptr) &&
         ypass_dispatch<true>(Py, -1, prec, nullptr, nullptr, nullptr);
}

}  // namespace gbd
