// Transform-only x-row kernels (Sec. II, Eq. 1; the xFFT_R2C / xFFT_C2R steps of Appendix A with
// one GPU): the FP32 row kernel's KIND 1 instances for the power-of-two lengths, which serve the
// forward transform and the inverse transform to the demag field without the LLG epilogue and so
// run at three 384-thread blocks per SM. Their own translation unit, built in parallel with the
// others.
#include "gbd_row.cuh"

namespace gbd {

template <int LX, int RB>
static void row_io_launch_t(const RowArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * RB * LX / GBD_E;
  const size_t smem = (size_t)3 * RB * line_stride<LX, true>() * sizeof(float2);
  prep(row_kernel<LX, RB, 0, 1>, smem);
  if (a) launch_pdl(row_kernel<LX, RB, 0, 1>, (a->rows + RB - 1) / RB, T, smem, st, *a, tw);
}

bool row_io_dispatch(int Lx, int RB, const RowArgs* a, const float2* tw, cudaStream_t st) {
  bool done = false;
  row_switch(Lx, [&](auto lx) {
    constexpr int LX = decltype(lx)::value;
    if (RB == row_rb(LX, 0)) {
      row_io_launch_t<LX, row_rb(LX, 0)>(a, tw, st);
      done = true;
    } else if (RB == row_rb(LX, 1)) {
      row_io_launch_t<LX, row_rb(LX, 1)>(a, tw, st);
      done = true;
    }
  });
  return done;
}

}  // namespace gbd
