// Kernel argument blocks, block shapes and launch helpers for the demag / LLG passes.
#pragma once
#include <cuda_runtime.h>

namespace gbd {

// What the x-row kernel does after (or instead of) the inverse x transform.
enum RowMode : int {
  ROW_FWD = 0,      // forward only: R2C of the 3-component input field into the spectrum
  ROW_H = 1,        // inverse only: out = hscale * H_d
  ROW_HEFF = 2,     // inverse: out = H_eff = hscale * H_d + H_ex(ms) + H_ext
  ROW_RHS = 3,      // inverse: out = dm/dt of the LLG equation at ms
  ROW_RK1 = 4,      // inverse + RK4 stage 1..4 update (+ optional forward of the next stage)
  ROW_RK2 = 5,
  ROW_RK3 = 6,
  ROW_RK4 = 7,
};

// Block shapes, shared by host planning and the kernels (L = transform length).
__host__ __device__ constexpr int row_rb(int Lx) { return Lx >= 4096 ? 1 : 4096 / Lx; }  // rows per block
__host__ __device__ constexpr int film_cols(int Py) { return Py >= 1024 ? 1 : 1024 / Py; }
__host__ __device__ constexpr int ypass_lines(int Py) { return Py >= 4096 ? 1 : 4096 / Py; }
__host__ __device__ constexpr int zconv_cols(int Pz) { return Pz >= 2048 ? 1 : 2048 / Pz; }

struct RowArgs {
  int nx, ny, nz;           // mesh
  int rows;                 // ny * nz
  long long N;              // cells
  int mode, fwd_after;      // RowMode; run the forward transform of the next stage
  const float* in;          // ROW_FWD input, planar [3][nz][ny][nx]
  float2* S;                // x spectrum [3][nz][Hx][ny]
  float* out;               // ROW_H / ROW_HEFF / ROW_RHS output, planar
  const float* ms;          // stage input m (unit vectors), planar
  const float* m0;          // m at the start of the step
  float* m0_out;            // stage 4 writes the new m here (may alias m0)
  float* acc;               // RK4 k-sum
  float* mnext;             // next stage input (stages 1..3)
  float hscale;             // factor applied to the transformed field (Ms for unit m, 1 for M)
  float cx, cy, cz;         // 2 A / (mu0 Ms d^2) per axis (0 where n_d = 1)
  float hx, hy, hz;         // applied field, A/m
  float geff, alpha;        // gamma / (1 + alpha^2), alpha
  float dt;                 // time step, s
};

struct ColArgs {
  int Hx, ny, nz, Py, Pz;
  long long lines_total;    // y passes: 3 * nz * Hx independent lines
  const float2* src;
  float2* dst;
  const float4* Kf;         // film kernel [Hx][Py/2+1] (xx, yy, zz, xy)
  const float* K3;          // 3D kernel [Hx][Py/2+1][Pz/2+1][6]
  long long Q;              // z-conv columns per plane = Hx * Py (Hx when ny == 1)
  int Pyq;                  // y extent of the column index q (Py, or 1 when ny == 1)
};

// Launchers dispatch on the transform length (a power of two); they return false for a
// length without an instantiation.
bool launch_row(int Lx, const RowArgs& a, const float2* tw, cudaStream_t st);
bool launch_film_conv(const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_y_fwd(const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_y_inv(const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_z_conv(const ColArgs& a, const float2* tw, cudaStream_t st);

}  // namespace gbd
