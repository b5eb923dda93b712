// Staged RK-stage x-row kernels (Sec. II, Eq. 1 and Sec. III: the inverse x transform, the
// exchange + LLG + RK4 stage epilogue and the next stage's forward x transform): the FP32 row
// kernel's KIND 2 instances for the power-of-two lengths whose tile takes the staged epilogue,
// compiled without the branches those launches never take. Their own translation unit, built in
// parallel with the others.
#include "gbd_row.cuh"

namespace gbd {

template <int LX, int RB>
static void row_rk_launch_t(const RowArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * RB * LX / GBD_E;
  const size_t smem = row_stage_smem<LX, RB>();
  prep(row_kernel<LX, RB, 0, 2>, smem);
  if (a) launch_pdl(row_kernel<LX, RB, 0, 2>, (a->rows + RB - 1) / RB, T, smem, st, *a, tw);
}

bool row_rk_dispatch(int Lx, int RB, const RowArgs* a, const float2* tw, cudaStream_t st) {
  bool done = false;
  row_switch(Lx, [&](auto lx) {
    constexpr int LX = decltype(lx)::value;
    constexpr int R0 = row_rb(LX, 0), R1 = row_rb(LX, 1);
    if constexpr (row_stage_ok<LX, R0, 0>()) {
      if (RB == R0) {
        row_rk_launch_t<LX, R0>(a, tw, st);
        done = true;
        return;
      }
    }
    if constexpr (R1 != R0 && row_stage_ok<LX, R1, 0>()) {
      if (RB == R1) {
        row_rk_launch_t<LX, R1>(a, tw, st);
        done = true;
      }
    }
  });
  return done;
}

}  // namespace gbd
