// sm_103a convolution kernels of the demag field (gbd_conv.cuh): the FP32 instantiations and
// the launchers.
#include "gbd_conv.cuh"

namespace gbd {

// prec < 0 (with a == nullptr) prepares every precision
static bool film_dispatch(int Py, int var, int prec, const ColArgs* a, const float2* tw, cudaStream_t st) {
  bool ok = true;
  if (prec <= 0) ok = film_dispatch_p<0>(Py, var, a, tw, st);
  if (ok && (prec == 1 || prec < 0)) ok = film_dispatch_p<1>(Py, var, a, tw, st);
  if (ok && (prec == 2 || prec < 0)) ok = film_dispatch_p<2>(Py, var, a, tw, st);
  return ok;
}
static bool z_dispatch(int Pz, int var, int prec, const ColArgs* a, const float2* tw, cudaStream_t st) {
  bool ok = true;
  if (prec <= 0) ok = z_dispatch_p<0>(Pz, var, a, tw, st);
  if (ok && (prec == 1 || prec < 0)) ok = z_dispatch_p<1>(Pz, var, a, tw, st);
  if (ok && (prec == 2 || prec < 0)) ok = z_dispatch_p<2>(Pz, var, a, tw, st);
  return ok;
}

bool launch_film_conv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st) {
  if (mixed_len(a.Py)) return prec == 0 && film_dispatch_mixed(a.Py, &a, tw, st);
  return film_dispatch(a.Py, var, prec, &a, tw, st);
}
bool prepare_film_conv(int Py, int prec) {
  if (mixed_len(Py)) return prec <= 0 && film_dispatch_mixed(Py, nullptr, nullptr, nullptr);
  return film_dispatch(Py, -1, prec, nullptr, nullptr, nullptr);
}

bool launch_z_conv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st) {
  return z_dispatch(a.Pz, var, prec, &a, tw, st);
}
bool prepare_z_conv(int Pz, int prec) { return z_dispatch(Pz, -1, prec, nullptr, nullptr, nullptr); }

}  // namespace gbd
