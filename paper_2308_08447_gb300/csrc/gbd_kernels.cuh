// Kernel argument blocks, block shapes and launchers of the demag / LLG passes.
//
// Passes of one demag evaluation (Sec. II, Eq. 1; the single-GPU steps of Appendix A), with
// P the padded lengths, Lx = Px / 2, Hx = Lx + 1:
//   row kernel, forward:  x real-to-complex of the zero-padded rows -> S [3][nz][Hx][ny]
//   film (nz = 1):        film_conv: y FFT -> kernel product -> y IFFT, in place on S
//   3D:                   y_fwd S -> T [3][nz][Hx][Py]; z_conv on T (z FFT -> product ->
//                         z IFFT, only the nz stored planes); y_inv T -> S
//   row kernel, inverse:  x complex-to-real + crop, then the mode's epilogue (field, dm/dt,
//                         or exchange + LLG + RK4 stage followed by the next stage's forward
//                         x transform, Sec. III).
// The padding is never stored: loads past n_d read zeros and cropped outputs are not
// written, so S keeps ny rows and T keeps nz planes. Every transform length is a template
// parameter; the launchers dispatch on it and on a tile-shape variant (0 or 1) that the
// autotuner picks per mesh.
#pragma once
#include <cuda_runtime.h>

#include "gbd_fft.cuh"

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
  ROW_RKG = 8,      // inverse + a general explicit RK stage: k = dm/dt at ms into kout, and the
                    // next stage input m0 + sum_j kw[j] kin[j] + kw[nk] k (+ its forward)
};

// Block shapes per transform length L and tile variant v, shared by host planning and the
// kernels. Every kernel has 16 complex values per thread, so threads = lines * L / 16.
// Lengths 3 * 2^k and 5 * 2^k (FP32 only) have one tile shape, sized from the largest power
// of two below the length (576 or 480 threads per x-row block).
__host__ __device__ constexpr int pow2_floor(int L) { return L < 2 ? 1 : 2 * pow2_floor(L / 2); }
__host__ __device__ constexpr bool mixed_len(int L) { return L > 1 && odd_part(L) > 1; }
// rows per x-row block (3 lines each): 2048 or 4096 complex values per component
__host__ __device__ constexpr int row_rb(int Lx, int v) {
  return mixed_len(Lx) ? (Lx >= 4096 ? 1 : (2048 / pow2_floor(Lx) > 0 ? 2048 / pow2_floor(Lx) : 1))
         : v == 0      ? (Lx >= 2048 ? 1 : 2048 / Lx)
                       : (Lx >= 4096 ? 1 : 4096 / Lx);
}
// kx columns per film-convolution block (3 lines each)
__host__ __device__ constexpr int film_cols(int Py, int v) {
  return mixed_len(Py) ? (pow2_floor(Py) >= 1024 ? 1 : 1024 / pow2_floor(Py))
         : v == 0      ? (Py >= 1024 ? 1 : 1024 / Py)
                       : (Py >= 4096 ? 1 : 2 * (Py >= 1024 ? 1 : 1024 / Py));
}
// y lines per 3D y-pass block
__host__ __device__ constexpr int ypass_lines(int Py, int v) {
  return mixed_len(Py) ? (pow2_floor(Py) >= 4096 ? 1 : 4096 / pow2_floor(Py))
         : v == 0      ? (Py >= 4096 ? 1 : 4096 / Py)
                       : (Py >= 2048 ? 1 : 2048 / Py);
}
// (kx, ky) columns per z-convolution block (3 lines each)
__host__ __device__ constexpr int zconv_cols(int Pz, int v) {
  return v == 0 ? (Pz >= 2048 ? 1 : 2048 / Pz) : (Pz >= 1024 ? 1 : 1024 / Pz);
}

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
  int vec8;                 // the field pointers allow 8-byte accesses (set by launch_row)
  int stage;                // the RK-stage epilogue reads its field rows from shared memory,
                            // copied there while the inverse transform runs (set by the launcher)
  unsigned* status;         // the mesh's device status word: a wait that gives up ORs in
                            // GBD_DEV_WAIT_TIMEOUT (may be null)
  unsigned stage_extra;     // test hook: bytes the staged copy is expected to deliver beyond what
                            // it copies, so that its bounded wait runs out (0 in normal use)
  int per;                  // periodic axes (bit 0 x, 1 y, 2 z): the x transform has no zero
                            // half, and the exchange Laplacian wraps around
  // demag extrapolation at RK sub-steps (Sec. III): with extrap the stage's demag field is
  // sum_{k < nh} hw[k] hist[k] over the step-start history (newest first) and no inverse transform
  // runs; hrec, when set, receives the stage's demag field (hscale * H_d), [3][N]
  int extrap;
  int nh;                   // history terms used (5 for RK4, 6 for RKF5(6))
  float hw[6];
  const float* hist[6];
  float* hrec;
  // general explicit RK stage (ROW_RKG): kin[0..nk) are earlier stages' dm/dt, kw their
  // weights dt a_(i+1),j, kw[nk] the weight of this stage's k; mnext may be null (last stage).
  // With hdev set the step size lives on the device: kw holds a_(i+1),j and is scaled by *hdev.
  float* kout;
  const float* kin[7];
  float kw[8];
  int nk;
  const float* hdev;
};

// Final combination of an RKF5(6) step (Sec. III): m5 = normalize(m + sum_i b5dt[i] k_i) per
// cell into out, and the largest |sum_i db[i] k_i| over cells into *err_max (float bits, >= 0).
struct RkfArgs {
  long long N;
  const float* m;
  const float* k[8];
  float b5dt[8];            // dt b5 (or b5, scaled by *hdev when hdev is set)
  float db[8];
  float* out;
  unsigned* err_max;
  const float* hdev;
};

// Device-side step control of an adaptive RKF5(6) run (Sec. III), one CUDA-graph loop for the
// whole run: after each attempt the control kernel reads the attempt's error, accepts or rejects
// it, picks the next step size and sets the loop's condition.
struct RkfCtl {
  double t, t_end, tol;     // time reached, end time, tolerance
  double h;                 // step size of the next attempt (the last one is cut at t_end)
  double h_next;            // the controller's proposal after the last attempt
  unsigned err;             // largest error norm of the current attempt (float bits); reset after use
  float hf;                 // h in FP32, read by the stage kernels
  int acc, rej, max_steps;  // accepted and rejected attempts, attempt limit
  int accepted;             // the last attempt was accepted
};

struct ColArgs {
  int Hx, ny, nz, Py, Pz;
  long long lines_total;    // y passes: 3 * nz * Hx independent lines
  const float2* src;
  float2* dst;
  const float4* Kf;         // film kernel [Hx][Py/2+1] (xx, yy, zz, xy)
  const float* K3;          // 3D kernel [Pz/2+1][Hx][Py/2+1][6]
  long long Q;              // z-conv columns per plane = Hx * Py (Hx when ny == 1)
  int Pyq;                  // y extent of the column index q (Py, or 1 when ny == 1)
};

// Bits of a mesh's device status word (gbd_mesh_device_status).
#define GBD_DEV_WAIT_TIMEOUT 1u
// Longest wait of a block for its staged copies, in ns of the GPU's global timer.
#define GBD_WAIT_LIMIT_NS 100000000ull

// Launchers dispatch on the transform length (a power of two) and the tile variant; they
// return false for a length without an instantiation.
// prec: 0 FP32 stages; 1 / 2 radix-16 stages on the tensor cores in split BF16 / split FP16
// (gbd_tc.cuh).
bool launch_row(int Lx, int var, int prec, const RowArgs& a, const float2* tw, cudaStream_t st);
// An extrapolated RK4 stage with no forward transform after it (a.extrap = 1, a.fwd_after = 0):
// the row kernel's epilogue alone, at full occupancy.
void launch_extrap_stage(const RowArgs& a, cudaStream_t st);
void launch_rkf_final(const RkfArgs& a, cudaStream_t st);
// One thread: the step controller of RkfCtl (safety factor, smallest and largest step ratios),
// and cudaGraphSetConditional(cond, continue) for the enclosing graph loop.
void launch_rkf_control(RkfCtl* c, cudaGraphConditionalHandle cond, double safety, double fac_min, double fac_max,
                        cudaStream_t st);
// dst = src over n floats when the last attempt was accepted.
void launch_rkf_accept(const RkfCtl* c, const float* src, float* dst, long long n, cudaStream_t st);
// Writes the split DFT-16 fragment tables of the tensor-core passes (gbd_tc.cuh) into the
// GBD_TC_FRAG_F2 float2 slots at frag (the mesh's twiddle buffer after its levels).
void launch_dft16_frags(float2* frag, cudaStream_t st);
bool launch_film_conv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_y_fwd(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_y_inv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st);
bool launch_z_conv(int var, int prec, const ColArgs& a, const float2* tw, cudaStream_t st);

// The transform-only x-row instances (row kernel KIND 1, FP32, power-of-two Lx; gbd_row_io.cu):
// launches (a == nullptr: prepares) the instance with RB rows per block; false when there is none.
bool row_io_dispatch(int Lx, int RB, const RowArgs* a, const float2* tw, cudaStream_t st);
// The staged RK-stage instances (row kernel KIND 2, FP32, power-of-two Lx; gbd_row_rk.cu), likewise.
bool row_rk_dispatch(int Lx, int RB, const RowArgs* a, const float2* tw, cudaStream_t st);

// Transform lengths 3 * 2^k and 5 * 2^k (FP32 only; gbd_mixed_row.cu, gbd_mixed_conv.cu):
// the launchers above forward them here. a == nullptr prepares without launching. False for
// a length without an instantiation.
bool row_dispatch_mixed(int Lx, int var, const RowArgs* a, const float2* tw, cudaStream_t st);
bool film_dispatch_mixed(int Py, const ColArgs* a, const float2* tw, cudaStream_t st);
bool ypass_dispatch_mixed(int Py, bool inv, const ColArgs* a, const float2* tw, cudaStream_t st);

// Set the kernels' shared-memory attribute for both variants of a length without launching
// (done when a mesh is created, so later launches inside a stream capture need no driver
// configuration call). Return false for a length without an instantiation.
bool prepare_row(int Lx, int prec);
bool prepare_film_conv(int Py, int prec);
bool prepare_y_passes(int Py, int prec);
bool prepare_z_conv(int Pz, int prec);

}  // namespace gbd
