// Device code of the x-row kernel (Sec. II, Eq. 1; the xFFT_R2C / xFFT_C2R steps of Appendix A
// with one GPU) with the fused exchange (Eq. 4) + LLG (Eq. 5) + RK stage epilogue (Sec. III):
// the epilogue device functions and the row kernel template, shared by the translation units of
// the FP32 kernels (gbd_row.cu) and of the split 16-bit kernels (gbd_row_bf16.cu, gbd_row_fp16.cu).
#pragma once
#include <cstdint>
#include <type_traits>

#include "gbd_launch.cuh"

namespace gbd {

// One-dimensional bulk copies global -> shared (TMA, cp.async.bulk) completed through an mbarrier
// in shared memory: one thread initialises the barrier, announces the bytes to expect and issues
// the copies; every thread that needs the data waits for the barrier's phase, for at most
// limit_ns of the GPU's global timer (false when it gave up).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(b)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"((unsigned)__cvta_generic_to_shared(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   (unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes), "r"((unsigned)__cvta_generic_to_shared(b))
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, unsigned long long limit_ns) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(b);
  const unsigned long long t0 = global_ns();
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// Asynchronous global -> shared copies (cp.async, 16 or 8 bytes per thread), in commit groups.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------------------------
// x rows: real-to-complex through a half-length complex FFT (Lx = Px / 2).
// Forward: z[m] = x[2m] + i x[2m+1], Z = FFT_Lx(z), and for k in [0, Lx]
//   X[k] = (Z[k] + Z*[Lx-k]) / 2 - (i/2) W^k (Z[k] - Z*[Lx-k]),  W = exp(-2 pi i / Px).
// Inverse: Z[k] = (X[k] + X*[Lx-k]) + i W^-k (X[k] - X*[Lx-k]); the unnormalised inverse
// FFT of Z is x[2m] + i x[2m+1] (the 1/P factors are folded into the kernel spectrum).
// Only the first Lx/2 complex values (the first Lx >= nx real samples) are produced by the
// inverse, and the forward reads only those: the upper half is the zero padding.
// ---------------------------------------------------------------------------------------------

// ---------------------------------------------------------------------------------------------
// Epilogue of the inverse x transform (Sec. III): exchange field (Eq. 4, 7-point Laplacian with
// free boundaries), H_eff, the LLG right-hand side (Eq. 5 solved for dm/dt) and the RK4 stage
// update, per cell, from the demag field hd of the cell.
// ---------------------------------------------------------------------------------------------

// res = H_eff (ROW_HEFF) or dm/dt (ROW_RHS); in RK4 stages the k-sum in acc_out and the next
// stage's m in mn. m0v / accv: the cell's step-start m and k-sum (stages 2-4).
__device__ __forceinline__ void llg_update(const RowArgs& a, int mode, const float* hd, const float* m,
                                           const float* lap, const float* m0v, const float* accv, float* mn,
                                           float* acc_out, float* res) {
  float H[3] = {hd[0] + lap[0] + a.hx, hd[1] + lap[1] + a.hy, hd[2] + lap[2] + a.hz};
  if (mode == ROW_HEFF) {
#pragma unroll
    for (int c = 0; c < 3; ++c) res[c] = H[c];
    return;
  }
  // dm/dt = -gamma/(1+alpha^2) [m x H + alpha m x (m x H)]
  const float mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
  const float mmH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2], m[0] * mxH[1] - m[1] * mxH[0]};
  float f[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) f[c] = -a.geff * (mxH[c] + a.alpha * mmH[c]);
  if (mode == ROW_RHS) {
#pragma unroll
    for (int c = 0; c < 3; ++c) res[c] = f[c];
    return;
  }
  if (mode == ROW_RK1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc_out[c] = f[c];
      mn[c] = m[c] + 0.5f * a.dt * f[c];
    }
  } else if (mode == ROW_RK2 || mode == ROW_RK3) {
    const float h = (mode == ROW_RK2) ? 0.5f * a.dt : a.dt;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      acc_out[c] = accv[c] + 2.f * f[c];
      mn[c] = m0v[c] + h * f[c];
    }
  } else {  // ROW_RK4
    const float h = a.dt * (1.0f / 6.0f);
#pragma unroll
    for (int c = 0; c < 3; ++c) mn[c] = m0v[c] + h * (accv[c] + f[c]);
    const float inv = rsqrtf(mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) mn[c] *= inv;
  }
}

// Extrapolated demag field (sum_k hw[k] hist[k], k < NH) of cells idx, idx + 1. NH is a
// template argument so that all history loads of a thread issue back to back.
template <int NH>
__device__ __forceinline__ void extrap_pair_n(const RowArgs& a, long long idx, float (&hd)[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 h2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NH; ++k) {
      const float2 hk = *reinterpret_cast<const float2*>(a.hist[k] + c * a.N + idx);
      h2.x = fmaf(a.hw[k], hk.x, h2.x);
      h2.y = fmaf(a.hw[k], hk.y, h2.y);
    }
    hd[0][c] = h2.x;
    hd[1][c] = h2.y;
  }
}

template <int NH>
__device__ __forceinline__ void extrap_cell_n(const RowArgs& a, long long idx, float (&hd)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float h = 0.f;
#pragma unroll
    for (int k = 0; k < NH; ++k) h = fmaf(a.hw[k], a.hist[k][c * a.N + idx], h);
    hd[c] = h;
  }
}

// nh is 5 (quartic, RK4) or 6 (quintic, RKF5(6)); uniform over the grid.
__device__ __forceinline__ void extrap_pair(const RowArgs& a, long long idx, float (&hd)[2][3]) {
  if (a.nh == 6)
    extrap_pair_n<6>(a, idx, hd);
  else
    extrap_pair_n<5>(a, idx, hd);
}

__device__ __forceinline__ void extrap_cell(const RowArgs& a, long long idx, float (&hd)[3]) {
  if (a.nh == 6)
    extrap_cell_n<6>(a, idx, hd);
  else
    extrap_cell_n<5>(a, idx, hd);
}

// Epilogue of the pair of cells (x0, x0 + 1), x0 even, at linear index idx (row of plane z at
// y) for nx a multiple of 64 and 8-byte aligned fields: the 32 lanes of the warp hold 32
// consecutive pairs of the row, so the x neighbours outside a pair come from the adjacent
// lanes; loads and stores are 8-byte vectors. Records hd when hrec is set, writes the mode's
// outputs, and returns true with the next stage's m in mn for the RK4 stages.
__device__ __forceinline__ bool epilogue_pair(const RowArgs& a, int mode, int z, int y, long long idx, int x0,
                                              int lane, const float (&hd)[2][3], float (&mn)[2][3]) {
  const long long N = a.N;
  const int nx = a.nx, ny = a.ny;
  const long long sz = (long long)nx * ny;
  if (a.hrec) {
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(a.hrec + c * N + idx) = make_float2(hd[0][c], hd[1][c]);
  }
  if (mode == ROW_H) {
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(a.out + c * N + idx) = make_float2(hd[0][c], hd[1][c]);
    return false;
  }
  // neighbour offsets, once per pair: the adjacent cell, across a periodic axis the cell on the
  // opposite face, else (free boundary) the cell itself
  const long long wy = (long long)(ny - 1) * nx, wz = (long long)(a.nz - 1) * sz;
  const long long oym = y > 0 ? -(long long)nx : ((a.per & 2) ? wy : 0);
  const long long oyp = y < ny - 1 ? (long long)nx : ((a.per & 2) ? -wy : 0);
  const long long ozm = z > 0 ? -sz : ((a.per & 4) ? wz : 0);
  const long long ozp = z < a.nz - 1 ? sz : ((a.per & 4) ? -wz : 0);
  const int oxl = x0 > 0 ? -1 : ((a.per & 1) ? nx - 1 : 0);      // left of x0 (lane 0)
  const int oxr = x0 + 2 < nx ? 2 : ((a.per & 1) ? 2 - nx : 1);  // right of x0 + 1 (lane 31)
  float mv[2][3], lap[2][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* __restrict__ p = a.ms + c * N + idx;
    const float2 cc = *reinterpret_cast<const float2*>(p);
    const float2 ym = *reinterpret_cast<const float2*>(p + oym);
    const float2 yp = *reinterpret_cast<const float2*>(p + oyp);
    float2 zm = cc, zp = cc;
    if (a.nz > 1) {
      zm = *reinterpret_cast<const float2*>(p + ozm);
      zp = *reinterpret_cast<const float2*>(p + ozp);
    }
    float left = __shfl_up_sync(0xffffffffu, cc.y, 1);
    float right = __shfl_down_sync(0xffffffffu, cc.x, 1);
    if (lane == 0) left = p[oxl];
    if (lane == 31) right = p[oxr];
    mv[0][c] = cc.x;
    mv[1][c] = cc.y;
    lap[0][c] = a.cx * (left - 2.f * cc.x + cc.y) + a.cy * (ym.x - 2.f * cc.x + yp.x) + a.cz * (zm.x - 2.f * cc.x + zp.x);
    lap[1][c] = a.cx * (cc.x - 2.f * cc.y + right) + a.cy * (ym.y - 2.f * cc.y + yp.y) + a.cz * (zm.y - 2.f * cc.y + zp.y);
  }
  float m0v[2][3] = {}, accv[2][3] = {};
  if (mode == ROW_RKG) {
    float res[2][3], ao[2][3];
#pragma unroll
    for (int u = 0; u < 2; ++u) llg_update(a, ROW_RHS, hd[u], mv[u], lap[u], m0v[u], accv[u], mn[u], ao[u], res[u]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      *reinterpret_cast<float2*>(a.kout + c * N + idx) = make_float2(res[0][c], res[1][c]);
      if (!a.mnext) continue;
      float2 s = *reinterpret_cast<const float2*>(a.m0 + c * N + idx);
      const float hs = a.hdev ? *a.hdev : 1.f;   // step size on the device, or folded into kw
      for (int j = 0; j < a.nk; ++j) {
        const float2 kj = *reinterpret_cast<const float2*>(a.kin[j] + c * N + idx);
        s.x = fmaf(a.kw[j] * hs, kj.x, s.x);
        s.y = fmaf(a.kw[j] * hs, kj.y, s.y);
      }
      s.x = fmaf(a.kw[a.nk] * hs, res[0][c], s.x);
      s.y = fmaf(a.kw[a.nk] * hs, res[1][c], s.y);
      *reinterpret_cast<float2*>(a.mnext + c * N + idx) = s;
      mn[0][c] = s.x;
      mn[1][c] = s.y;
    }
    return a.mnext != nullptr;
  }
  if (mode == ROW_RK2 || mode == ROW_RK3 || mode == ROW_RK4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 q0 = *reinterpret_cast<const float2*>(a.m0 + c * N + idx);
      const float2 qa = *reinterpret_cast<const float2*>(a.acc + c * N + idx);
      m0v[0][c] = q0.x;
      m0v[1][c] = q0.y;
      accv[0][c] = qa.x;
      accv[1][c] = qa.y;
    }
  }
  float ao[2][3], res[2][3];
#pragma unroll
  for (int u = 0; u < 2; ++u) llg_update(a, mode, hd[u], mv[u], lap[u], m0v[u], accv[u], mn[u], ao[u], res[u]);
  if (mode == ROW_HEFF || mode == ROW_RHS) {
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<float2*>(a.out + c * N + idx) = make_float2(res[0][c], res[1][c]);
    return false;
  }
  // m0_out aliases m0 in stage 4: each cell is read, then written, by one thread
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 v = make_float2(mn[0][c], mn[1][c]);
    if (mode == ROW_RK4) {
      *reinterpret_cast<float2*>(a.m0_out + c * N + idx) = v;
    } else {
      *reinterpret_cast<float2*>(a.acc + c * N + idx) = make_float2(ao[0][c], ao[1][c]);
      *reinterpret_cast<float2*>(a.mnext + c * N + idx) = v;
    }
  }
  return true;
}

// The same for one cell at (x, y, z), linear index idx, any nx and 4-byte aligned fields.
__device__ __forceinline__ bool epilogue_cell(const RowArgs& a, int mode, int z, int y, int x, long long idx,
                                              const float (&hd)[3], float (&mn)[3]) {
  const long long N = a.N;
  const int nx = a.nx, ny = a.ny;
  const long long sz = (long long)nx * ny;
  if (a.hrec) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.hrec[c * N + idx] = hd[c];
  }
  if (mode == ROW_H) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out[c * N + idx] = hd[c];
    return false;
  }
  // exchange: 7-point Laplacian; a missing neighbour is the cell itself (free boundary) or,
  // across a periodic axis, the cell on the opposite face
  const bool px = a.per & 1, py = a.per & 2, pz = a.per & 4;
  const long long ixm = x > 0 ? idx - 1 : (px ? idx + (nx - 1) : idx);
  const long long ixp = x < nx - 1 ? idx + 1 : (px ? idx - (nx - 1) : idx);
  const long long iym = y > 0 ? idx - nx : (py ? idx + (long long)(ny - 1) * nx : idx);
  const long long iyp = y < ny - 1 ? idx + nx : (py ? idx - (long long)(ny - 1) * nx : idx);
  const long long izm = z > 0 ? idx - sz : (pz ? idx + (long long)(a.nz - 1) * sz : idx);
  const long long izp = z < a.nz - 1 ? idx + sz : (pz ? idx - (long long)(a.nz - 1) * sz : idx);
  float mv[3], lap[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* __restrict__ p = a.ms + c * N;
    const float mc = p[idx];
    mv[c] = mc;
    // (minus - 2 centre + plus) per axis, the operand order of epilogue_pair, so that every
    // epilogue path rounds alike
    lap[c] = a.cx * (p[ixm] - 2.f * mc + p[ixp]) + a.cy * (p[iym] - 2.f * mc + p[iyp]) +
             a.cz * (p[izm] - 2.f * mc + p[izp]);
  }
  float m0v[3] = {}, accv[3] = {};
  if (mode == ROW_RKG) {
    float res[3], ao[3];
    llg_update(a, ROW_RHS, hd, mv, lap, m0v, accv, mn, ao, res);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.kout[c * N + idx] = res[c];
      if (!a.mnext) continue;
      float s = a.m0[c * N + idx];
      const float hs = a.hdev ? *a.hdev : 1.f;
      for (int j = 0; j < a.nk; ++j) s = fmaf(a.kw[j] * hs, a.kin[j][c * N + idx], s);
      s = fmaf(a.kw[a.nk] * hs, res[c], s);
      a.mnext[c * N + idx] = s;
      mn[c] = s;
    }
    return a.mnext != nullptr;
  }
  if (mode == ROW_RK2 || mode == ROW_RK3 || mode == ROW_RK4) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      m0v[c] = a.m0[c * N + idx];
      accv[c] = a.acc[c * N + idx];
    }
  }
  float ao[3], res[3];
  llg_update(a, mode, hd, mv, lap, m0v, accv, mn, ao, res);
  if (mode == ROW_HEFF || mode == ROW_RHS) {
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out[c * N + idx] = res[c];
    return false;
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (mode == ROW_RK4) {
      a.m0_out[c * N + idx] = mn[c];
    } else {
      a.acc[c * N + idx] = ao[c];
      a.mnext[c * N + idx] = mn[c];
    }
  }
  return true;
}

// Staged RK-stage epilogue (FP32 row kernels that run one block per SM). The stage input m on
// the block's rows and the rows above and below ([RB + 2][3][LX] floats, after the lines on a
// 16-byte boundary) is copied into shared memory by one thread's bulk copies (one per row and
// component), requested when the block starts and waited for once after the inverse transform
// (a bounded wait: a block that gives up records GBD_DEV_WAIT_TIMEOUT in the mesh's status word
// and carries on), so the Laplacian reads shared memory; the step-start m and the k-sum (no
// reuse) stay in global memory and are requested one item ahead. Staging them too would cost more
// than it saves: the L1 cache shares the SM's 256 KB with shared memory, and the spectrum loads
// need the room.
template <int LX, int RB>
__host__ __device__ constexpr int row_stage_off() {   // float2 slots
  return (3 * RB * line_stride<LX, true>() + 1) / 2 * 2;
}
template <int LX, int RB>
__host__ __device__ constexpr size_t row_stage_smem() {
  return (size_t)row_stage_off<LX, RB>() * 8 + (size_t)(RB + 2) * 3 * LX * 4 + 16;   // + the mbarrier
}
template <int LX, int RB, int PREC>
__host__ __device__ constexpr bool row_stage_ok() {
  return PREC == 0 && npasses(LX, false) >= 1 && min_blocks(3 * RB * LX / GBD_E) == 1 &&
         row_stage_smem<LX, RB>() <= 232448;
}

// Blocks per SM of the transform-only instances (KIND 1: ROW_FWD and ROW_H without demag
// extrapolation): without the LLG epilogue a 384-thread block fits 56 registers, so three run per
// SM instead of two.
__host__ __device__ constexpr int io_blocks(int T) { return T >= 768 ? 1 : (T >= 384 ? 3 : 1152 / T); }

// KIND 0 serves every RowMode; KIND 1 only the transform-only launches (the forward transform,
// and the inverse transform to hscale * H_d), compiled without the epilogue's LLG code; KIND 2
// only the staged RK stages (a.stage set, every block's rows in one z plane, ny even), compiled
// with the branches those launches never take (extrapolation, periodic x, unvectorised spectrum
// and epilogue paths, the unstaged epilogue) left out.
template <int LX, int RB_, int PREC, int KIND = 0>
__global__ void __launch_bounds__(3 * RB_ * LX / GBD_E,
                                  KIND == 1 ? io_blocks(3 * RB_ * LX / GBD_E) : min_blocks(3 * RB_ * LX / GBD_E))
    row_kernel(RowArgs a, const float2* __restrict__ tw) {
  constexpr int RB = RB_;
  constexpr int LINES = 3 * RB;
  constexpr int T = LINES * LX / GBD_E;
  constexpr int LS = line_stride<LX, true>();  // odd: the rows' lines fall on different banks
  constexpr int NP = npasses(LX, false);
  constexpr int HX = LX + 1;
  constexpr int HALF = LX / 2;
  constexpr int FL = NP >= 1 ? LX : 2 * LX;    // real samples the forward transform reads
  // periodic x (Px = nx, no zero padding): the whole line holds data
  const bool xper = KIND == 2 ? false : (a.per & 1) != 0;
  const int flr = xper ? 2 * LX : FL;          // real samples of a line that hold data or zeros
  extern __shared__ float2 sm[];
  const int r0 = blockIdx.x * RB;
  const long long N = a.N;
  const int mode = a.mode;   // KIND 2: an RK stage
  const int nx = a.nx, ny = a.ny;
  // (z, y) of the block's first row; when the block's rows share a z plane (ny a multiple
  // of RB, always for the power-of-two meshes) the per-element division is skipped
  const int zb = r0 / ny, yb = r0 - zb * ny;
  const bool one_plane = (yb + RB <= ny);
  auto row_zy = [&](int rr, int& z, int& y) {
    if (one_plane) {
      z = zb;
      y = yb + rr;
    } else {
      z = (r0 + rr) / ny;
      y = r0 + rr - z * ny;
    }
  };
  const float* __restrict__ ms = a.ms;
  // rows per vector access of the [kx][y] spectrum: two adjacent rows are one 16-byte access
  constexpr int VR = (RB % 2 == 0) ? 2 : 1;
  constexpr int RG = RB / VR;
  static_assert(KIND != 2 || VR == 2, "the staged RK-stage instances read row pairs as 16-byte vectors");
  const bool vec = KIND == 2 ? true : (VR == 2) && one_plane && (ny % 2 == 0);
  // staged epilogue (a.stage: an RK stage with the next forward transform, free x boundary,
  // nx a multiple of 64, 16-byte aligned fields)
  constexpr bool SOK = KIND != 1 && row_stage_ok<LX, RB, PREC>();
  const bool stg = KIND == 2 ? true : SOK && a.stage && one_plane;
  float* sMs = reinterpret_cast<float*>(sm + row_stage_off<LX, RB>());   // [RB + 2][3][LX]
  unsigned long long* sbar = reinterpret_cast<unsigned long long*>(sMs + (RB + 2) * 3 * LX);  // after the rows
  // rows yb - 1 .. yb + RB of the stage input: a missing neighbour row is the row itself (free
  // boundary) or the row on the opposite face (periodic y)
  auto issue_stage_rows = [&]() {
    if (threadIdx.x == 0) {
      mbar_init(sbar, 1);
      mbar_expect_tx(sbar, (unsigned)((RB + 2) * 3 * nx * 4) + a.stage_extra);
      const long long plane = (long long)zb * ny;
      for (int s = 0; s < RB + 2; ++s) {
        int y = yb - 1 + s;
        if (y < 0) y = (a.per & 2) ? ny - 1 : 0;
        if (y >= ny) y = (a.per & 2) ? 0 : ny - 1;
        for (int c = 0; c < 3; ++c)
          bulk_g2s(sMs + (s * 3 + c) * LX, ms + c * N + (plane + y) * nx, (unsigned)(nx * 4), sbar);
      }
    }
  };
  // An RK stage that takes this path is launched right after a convolution launch (the film
  // convolution, or the 3D inverse y pass) -- or, in the autotuner's timing loop, after another
  // RK-stage launch that does not write this one's stage input -- and its stage input was written
  // by an x-row launch before that, so it is complete once this block runs (gbd_launch.cuh): it
  // is requested before the wait for the preceding launch.
  if constexpr (SOK) {
    if (stg) issue_stage_rows();
  }
  pdl_wait_then_release();

  if (KIND == 2 || mode != ROW_FWD) {
    if (KIND != 0 || !a.extrap) {  // uniform over the grid
    // 1. X (global, [kx][y] layout) -> Z pairwise into shared memory. An item is (row group,
    //    component, k) with VR adjacent rows per group, read as one 16-byte vector when the
    //    rows are adjacent in memory; every thread issues all its loads before using any.
    constexpr int ITEMS = RG * 3 * (HALF + 1);
    constexpr int IPT = (ITEMS + T - 1) / T;
    float2 A[IPT][VR], B[IPT][VR];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int e = threadIdx.x + i * T;
      const int g = e % RG;
      const int t2 = e / RG;
      const int c = t2 % 3;
      const int k = t2 / 3;
#pragma unroll
      for (int u = 0; u < VR; ++u) A[i][u] = B[i][u] = make_float2(0.f, 0.f);
      if (e < ITEMS) {
        if (vec) {
          const float2* base = a.S + (long long)(c * a.nz + zb) * HX * ny + yb + g * VR;
          const float4 va = *reinterpret_cast<const float4*>(base + (long long)k * ny);
          const float4 vb = *reinterpret_cast<const float4*>(base + (long long)(LX - k) * ny);
          A[i][0] = make_float2(va.x, va.y);
          A[i][VR - 1] = make_float2(va.z, va.w);
          B[i][0] = make_float2(vb.x, vb.y);
          B[i][VR - 1] = make_float2(vb.z, vb.w);
        } else {
#pragma unroll
          for (int u = 0; u < VR; ++u) {
            const int rr = g * VR + u;
            if (r0 + rr < a.rows) {
              int z, y;
              row_zy(rr, z, y);
              const float2* base = a.S + (long long)(c * a.nz + z) * HX * ny + y;
              A[i][u] = base[(long long)k * ny];
              B[i][u] = base[(long long)(LX - k) * ny];
            }
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int e = threadIdx.x + i * T;
      if (ITEMS % T != 0 && e >= ITEMS) break;
      const int g = e % RG;
      const int t2 = e / RG;
      const int c = t2 % 3;
      const int k = t2 / 3;
      const float2 wp = twiddle_at<-1>(tw, 2 * LX, k);  // W^k, W = exp(-2 pi i / Px)
      const float2 wm = cconj(wp);                  // W^-k
#pragma unroll
      for (int u = 0; u < VR; ++u) {
        const float2 Au = A[i][u], Bu = B[i][u];
        float2 zk, zl = make_float2(0.f, 0.f);
        if (k == 0) {
          zk = cadd(cadd(Au, cconj(Bu)), cmul_i<1>(csub(Au, cconj(Bu))));
        } else {
          zk = cadd(cadd(Au, cconj(Bu)), cmul_i<1>(cmul(wm, csub(Au, cconj(Bu)))));
          zl = csub(cadd(Bu, cconj(Au)), cmul_i<1>(cmul(wp, csub(Bu, cconj(Au)))));
        }
        float2* L = sm + (c * RB + g * VR + u) * LS;
        L[pad(k)] = zk;
        if (k != 0 && k != LX - k) L[pad(LX - k)] = zl;
      }
    }
    __syncthreads();
    // 2. unnormalised inverse FFT: adjoint passes, the last one keeping the lower half only.
    if constexpr (NP >= 1) {
      adj_passes_smem<1, LX, false, LINES, false, LS, NP, 1, PREC>(sm, tw);
      auto ld = [&](int line, int i) { return sm[line * LS + pad(i)]; };
      // the bound is a compile-time constant on the open-boundary path, so the pass is pruned
      auto st_half = [&](int line, int i, float2 v) {
        if (i < HALF) sm[line * LS + pad(i)] = v;
      };
      auto st_all = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };
      constexpr int R0 = radix_at(LX, false, 0);
      if (xper)
        pass_any<PREC, 1, true, LX, R0, 1, LINES, false, true>(tw, ld, st_all);
      else if constexpr (PREC == 0 && R0 % 2 == 0)
        stockham_pass_sm<1, true, LX, R0, 1, LINES, false, LS, true>(sm, tw);   // keeps the lower half
      else
        pass_any<PREC, 1, true, LX, R0, 1, LINES, false, true>(tw, ld, st_half);
      __syncthreads();
    }
    }
    if constexpr (SOK) {
      if (stg && !mbar_wait(sbar, 0, GBD_WAIT_LIMIT_NS) && a.status) atomicOr(a.status, GBD_DEV_WAIT_TIMEOUT);
    }
    // 3. epilogue on the real rows: float view of line position x is 2 pad(x/2) + (x & 1).
    if (KIND == 2 || ((nx % 64) == 0 && a.vec8)) {
      // Fast path (8-byte aligned fields): an item is a pair of cells (x0, x0 + 1); the 32
      // lanes of a warp take 32 consecutive pairs of one row (epilogue_pair).
      const int NP2 = nx / 2;
      bool staged = false;
      if constexpr (SOK) {
        if (stg) {
          // the field rows from shared memory (one_plane: all RB rows exist, in plane zb); the
          // arithmetic is epilogue_pair's, term for term
          const long long sz = (long long)nx * ny;
          const long long ozm = zb > 0 ? -sz : ((a.per & 4) ? (long long)(a.nz - 1) * sz : 0);
          const long long ozp = zb < a.nz - 1 ? sz : ((a.per & 4) ? -(long long)(a.nz - 1) * sz : 0);
          // the step-start m and k-sum of the next item are requested before this item's update
          const bool rk_acc = mode != ROW_RK1;   // stages 2-4 read them
          float2 q0n[3], qan[3];
          auto fetch = [&](int e, float2 (&q0)[3], float2 (&qa)[3]) {
            const int rr = e / NP2;
            const long long idx = (long long)(r0 + rr) * nx + 2 * (e - rr * NP2);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              q0[c] = *reinterpret_cast<const float2*>(a.m0 + c * N + idx);
              qa[c] = *reinterpret_cast<const float2*>(a.acc + c * N + idx);
            }
          };
          if (rk_acc && threadIdx.x < RB * NP2) fetch(threadIdx.x, q0n, qan);
          for (int e = threadIdx.x; e < RB * NP2; e += T) {
            const int rr = e / NP2;
            const int xp = e - rr * NP2;
            const int x0 = 2 * xp;
            const long long idx = (long long)(r0 + rr) * nx + x0;
            float hd[2][3], mv[2][3], lap[2][3], m0v[2][3] = {}, accv[2][3] = {}, mn[2][3], ao[2][3], res[2][3];
            if (rk_acc) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                m0v[0][c] = q0n[c].x;
                m0v[1][c] = q0n[c].y;
                accv[0][c] = qan[c].x;
                accv[1][c] = qan[c].y;
              }
              if (e + T < RB * NP2) fetch(e + T, q0n, qan);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 h2 = sm[(c * RB + rr) * LS + pad(xp)];
              hd[0][c] = h2.x * a.hscale;
              hd[1][c] = h2.y * a.hscale;
            }
            if (a.hrec) {
#pragma unroll
              for (int c = 0; c < 3; ++c)
                *reinterpret_cast<float2*>(a.hrec + c * N + idx) = make_float2(hd[0][c], hd[1][c]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float* rc = sMs + ((rr + 1) * 3 + c) * LX;
              const float2 cc = *reinterpret_cast<const float2*>(rc + x0);
              const float2 ym = *reinterpret_cast<const float2*>(sMs + (rr * 3 + c) * LX + x0);
              const float2 yp = *reinterpret_cast<const float2*>(sMs + ((rr + 2) * 3 + c) * LX + x0);
              const float left = x0 > 0 ? rc[x0 - 1] : cc.x;          // free x boundary
              const float right = x0 + 2 < nx ? rc[x0 + 2] : cc.y;
              float2 zm = cc, zp = cc;
              if (a.nz > 1) {
                const float* p = ms + c * N + idx;
                zm = *reinterpret_cast<const float2*>(p + ozm);
                zp = *reinterpret_cast<const float2*>(p + ozp);
              }
              mv[0][c] = cc.x;
              mv[1][c] = cc.y;
              lap[0][c] = a.cx * (left - 2.f * cc.x + cc.y) + a.cy * (ym.x - 2.f * cc.x + yp.x) +
                          a.cz * (zm.x - 2.f * cc.x + zp.x);
              lap[1][c] = a.cx * (cc.x - 2.f * cc.y + right) + a.cy * (ym.y - 2.f * cc.y + yp.y) +
                          a.cz * (zm.y - 2.f * cc.y + zp.y);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) llg_update(a, mode, hd[u], mv[u], lap[u], m0v[u], accv[u], mn[u], ao[u], res[u]);
            // m0_out aliases m0 in stage 4: each cell's m0 is read, then written, by one thread
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 v = make_float2(mn[0][c], mn[1][c]);
              if (mode == ROW_RK4) {
                *reinterpret_cast<float2*>(a.m0_out + c * N + idx) = v;
              } else {
                *reinterpret_cast<float2*>(a.acc + c * N + idx) = make_float2(ao[0][c], ao[1][c]);
                *reinterpret_cast<float2*>(a.mnext + c * N + idx) = v;
              }
              sm[(c * RB + rr) * LS + pad(xp)] = v;
            }
          }
          staged = true;
        }
      }
      if (!staged) {
        for (int e = threadIdx.x; e < RB * NP2; e += T) {
          const int rr = e / NP2;
          const int xp = e - rr * NP2;
          if (r0 + rr >= a.rows) continue;  // uniform per warp (NP2 is a multiple of 32)
          int z, y;
          row_zy(rr, z, y);
          const int x0 = 2 * xp;
          const long long idx = (long long)(r0 + rr) * nx + x0;
          float hd[2][3], mn[2][3];
          if constexpr (KIND == 1) {   // ROW_H: out = hscale * H_d (and the history record)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 h2 = sm[(c * RB + rr) * LS + pad(xp)];
              const float2 v = make_float2(h2.x * a.hscale, h2.y * a.hscale);
              if (a.hrec) *reinterpret_cast<float2*>(a.hrec + c * N + idx) = v;
              *reinterpret_cast<float2*>(a.out + c * N + idx) = v;
            }
            continue;
          }
          if (a.extrap) {
            extrap_pair(a, idx, hd);
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float2 h2 = sm[(c * RB + rr) * LS + pad(xp)];
              hd[0][c] = h2.x * a.hscale;
              hd[1][c] = h2.y * a.hscale;
            }
          }
          if (epilogue_pair(a, mode, z, y, idx, x0, threadIdx.x & 31, hd, mn) && a.fwd_after) {
#pragma unroll
            for (int c = 0; c < 3; ++c) sm[(c * RB + rr) * LS + pad(xp)] = make_float2(mn[0][c], mn[1][c]);
          }
        }
      }
    } else {
      // General path: one cell per item (epilogue_cell).
      for (int e = threadIdx.x; e < RB * nx; e += T) {
        const int rr = e / nx;
        const int x = e - rr * nx;
        if (r0 + rr >= a.rows) continue;
        int z, y;
        row_zy(rr, z, y);
        const long long idx = (long long)(r0 + rr) * nx + x;
        const int fpos = 2 * pad(x >> 1) + (x & 1);
        float hd[3], mn[3];
        if constexpr (KIND == 1) {   // ROW_H
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float v = reinterpret_cast<const float*>(sm + (c * RB + rr) * LS)[fpos] * a.hscale;
            if (a.hrec) a.hrec[c * N + idx] = v;
            a.out[c * N + idx] = v;
          }
          continue;
        }
        if (a.extrap) {
          extrap_cell(a, idx, hd);
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) hd[c] = reinterpret_cast<const float*>(sm + (c * RB + rr) * LS)[fpos] * a.hscale;
        }
        if (epilogue_cell(a, mode, z, y, x, idx, hd, mn) && a.fwd_after) {
#pragma unroll
          for (int c = 0; c < 3; ++c) reinterpret_cast<float*>(sm + (c * RB + rr) * LS)[fpos] = mn[c];
        }
      }
    }
    if (KIND != 2 && !a.fwd_after) return;  // uniform over the block
    // 4. zero what the forward transform reads beyond the data (positions the epilogue does not
    //    touch, so the barrier before the forward transform orders both)
    for (int line = 0; line < LINES; ++line) {
      const int rr = line % RB;
      const int x0 = (r0 + rr < a.rows) ? nx : 0;
      float* fl = reinterpret_cast<float*>(sm + line * LS);
      for (int x = x0 + threadIdx.x; x < flr; x += T) fl[2 * pad(x >> 1) + (x & 1)] = 0.f;
    }
  } else {
    // forward only: the input rows into the float view, zero beyond nx; pairs of samples
    // are one complex slot, read as 8-byte vectors when nx is even
    constexpr int PAIRS_MAX = LINES * LX;   // a whole line (periodic x)
    constexpr int IPT = (PAIRS_MAX + T - 1) / T;
    const int hl = flr / 2;                 // complex slots per line to fill
    const int pairs = LINES * hl;
    if (flr >= 2 && (nx % 2) == 0 && a.vec8) {
      float2 v[IPT];
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const int e = threadIdx.x + i * T;
        const int line = e / hl;
        const int xp = e % hl;
        const int c = line / RB, rr = line % RB;
        v[i] = make_float2(0.f, 0.f);
        if (e < pairs && 2 * xp < nx && r0 + rr < a.rows)
          v[i] = *reinterpret_cast<const float2*>(a.in + c * N + (long long)(r0 + rr) * nx + 2 * xp);
      }
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        const int e = threadIdx.x + i * T;
        if (e >= pairs) break;
        sm[(e / hl) * LS + pad(e % hl)] = v[i];
      }
    } else {
      for (int e = threadIdx.x; e < LINES * flr; e += T) {
        const int line = e / flr;
        const int x = e % flr;
        const int c = line / RB, rr = line % RB;
        const int row = r0 + rr;
        float v = 0.f;
        if (x < nx && row < a.rows) v = a.in[c * N + (long long)row * nx + x];
        reinterpret_cast<float*>(sm + line * LS)[2 * pad(x >> 1) + (x & 1)] = v;
      }
    }
  }
  __syncthreads();
  // 5. forward FFT; the first pass reads the lower half only (the upper half is zero).
  if constexpr (NP >= 1) {
    auto ld_half = [&](int line, int i) { return i < HALF ? sm[line * LS + pad(i)] : make_float2(0.f, 0.f); };
    auto ld_all = [&](int line, int i) { return sm[line * LS + pad(i)]; };
    auto st = [&](int line, int i, float2 v) { sm[line * LS + pad(i)] = v; };
    constexpr int R0 = radix_at(LX, false, 0);
    if (xper)
      pass_any<PREC, -1, false, LX, R0, 1, LINES, false, true>(tw, ld_all, st);
    else if constexpr (PREC == 0 && R0 % 2 == 0)
      stockham_pass_sm<-1, false, LX, R0, 1, LINES, false, LS, true>(sm, tw);   // reads the lower half
    else
      pass_any<PREC, -1, false, LX, R0, 1, LINES, false, true>(tw, ld_half, st);
    __syncthreads();
    fwd_passes_smem<-1, LX, false, LINES, false, LS, 1, NP, PREC>(sm, tw);
  }
  // 6. Z -> X pairwise and store the half spectrum, VR adjacent rows per item.
  for (int e = threadIdx.x; e < RG * 3 * (HALF + 1); e += T) {
    const int g = e % RG;
    const int t2 = e / RG;
    const int c = t2 % 3;
    const int k = t2 / 3;
    const float2 wp = twiddle_at<-1>(tw, 2 * LX, k);  // W^k, W = exp(-2 pi i / Px)
    const float2 wm = cconj(wp);
    float2 xk[VR], xl[VR];
#pragma unroll
    for (int u = 0; u < VR; ++u) {
      const float2* L = sm + (c * RB + g * VR + u) * LS;
      if (k == 0) {
        const float2 A = L[pad(0)];
        xk[u] = make_float2(A.x + A.y, 0.f);   // X[0]
        xl[u] = make_float2(A.x - A.y, 0.f);   // X[Lx]
      } else {
        const float2 A = L[pad(k)], B = L[pad(LX - k)];
        xk[u] = cscale(csub(cadd(A, cconj(B)), cmul_i<1>(cmul(wp, csub(A, cconj(B))))), 0.5f);
        xl[u] = cscale(cadd(cadd(B, cconj(A)), cmul_i<1>(cmul(wm, csub(B, cconj(A))))), 0.5f);
      }
    }
    const int kl = (k == 0) ? LX : LX - k;  // partner frequency written with xl
    const bool two = (k == 0) || (LX - k != k);
    if (vec) {
      float2* base = a.S + (long long)(c * a.nz + zb) * HX * ny + yb + g * VR;
      *reinterpret_cast<float4*>(base + (long long)k * ny) = make_float4(xk[0].x, xk[0].y, xk[VR - 1].x, xk[VR - 1].y);
      if (two)
        *reinterpret_cast<float4*>(base + (long long)kl * ny) = make_float4(xl[0].x, xl[0].y, xl[VR - 1].x, xl[VR - 1].y);
    } else {
#pragma unroll
      for (int u = 0; u < VR; ++u) {
        const int rr = g * VR + u;
        if (r0 + rr >= a.rows) continue;
        int z, y;
        row_zy(rr, z, y);
        float2* base = a.S + (long long)(c * a.nz + z) * HX * ny + y;
        base[(long long)k * ny] = xk[u];
        if (two) base[(long long)kl * ny] = xl[u];
      }
    }
  }
}


// ---- launcher --------------------------------------------------------------------------------

// Whether an RK-stage launch can take the staged epilogue (row_stage_ok instances): the next
// forward transform follows, x is not periodic (the staged Laplacian takes the free x boundary),
// the pair path applies, and the fields are 16-byte aligned (the bulk copies' sources).
static inline bool row_stage_applies(const RowArgs& a) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (a.mode < ROW_RK1 || a.mode > ROW_RK4 || a.extrap || !a.fwd_after || (a.per & 1)) return false;
  if (a.nx % 64 != 0 || !a.vec8 || !al16(a.ms)) return false;
  return a.mode == ROW_RK1 || (al16(a.m0) && al16(a.acc));
}

template <int LX, int RB, int PREC>
static void row_launch_t(const RowArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * RB * LX / GBD_E;
  constexpr bool SOK = row_stage_ok<LX, RB, PREC>();
  const size_t smem = (size_t)3 * RB * line_stride<LX, true>() * sizeof(float2);
  // transform-only launches of the FP32 power-of-two lengths take the KIND 1 instances
  // (gbd_row_io.cu)
  constexpr bool IO = PREC == 0 && !mixed_len(LX);
  prep(row_kernel<LX, RB, PREC>, SOK ? row_stage_smem<LX, RB>() : smem);
  if (!a) {
    if constexpr (IO) {
      row_io_dispatch(LX, RB, nullptr, nullptr, nullptr);
      row_rk_dispatch(LX, RB, nullptr, nullptr, nullptr);
    }
    return;
  }
  RowArgs b = *a;
  b.stage = SOK && row_stage_applies(b);
  if constexpr (IO) {
    if ((b.mode == ROW_FWD || (b.mode == ROW_H && !b.extrap)) && row_io_dispatch(LX, RB, &b, tw, st)) return;
    // staged RK stages whose blocks each lie in one z plane take the KIND 2 instances (gbd_row_rk.cu)
    if (b.stage && b.ny % RB == 0 && b.ny % 2 == 0 && row_rk_dispatch(LX, RB, &b, tw, st)) return;
  }
  launch_pdl(row_kernel<LX, RB, PREC>, (b.rows + RB - 1) / RB, T, b.stage ? row_stage_smem<LX, RB>() : smem, st, b, tw);
}

// prec < 0 (with a == nullptr) prepares both precisions
// Calls f(std::integral_constant<int, LX>) for the x transform length Lx; false for a length
// without an instantiation.
template <class F>
static bool row_switch(int Lx, F f) {
  switch (Lx) {
#define GBD_ROW_LEN(LX)                          \
  case LX:                                       \
    f(std::integral_constant<int, LX>());        \
    return true;
    GBD_ROW_LEN(1)
    GBD_ROW_LEN(2)
    GBD_ROW_LEN(4)
    GBD_ROW_LEN(8)
    GBD_ROW_LEN(16)
    GBD_ROW_LEN(32)
    GBD_ROW_LEN(64)
    GBD_ROW_LEN(128)
    GBD_ROW_LEN(256)
    GBD_ROW_LEN(512)
    GBD_ROW_LEN(1024)
    GBD_ROW_LEN(2048)
    GBD_ROW_LEN(4096)
#undef GBD_ROW_LEN
    default: return false;
  }
}

// Launches (a == nullptr: prepares) the row kernel of precision PREC for length Lx, tile
// variant var (both when var < 0). Explicitly instantiated once per precision, each in its own
// translation unit (gbd_row.cu, gbd_row_bf16.cu, gbd_row_fp16.cu) so the units build in
// parallel.
template <int PREC>
bool row_dispatch_p(int Lx, int var, const RowArgs* a, const float2* tw, cudaStream_t st) {
  return row_switch(Lx, [&](auto lx) {
    constexpr int LX = decltype(lx)::value;
    if (var <= 0) row_launch_t<LX, row_rb(LX, 0), PREC>(a, tw, st);
    if (var != 0) row_launch_t<LX, row_rb(LX, 1), PREC>(a, tw, st);
  });
}
extern template bool row_dispatch_p<1>(int, int, const RowArgs*, const float2*, cudaStream_t);
extern template bool row_dispatch_p<2>(int, int, const RowArgs*, const float2*, cudaStream_t);

}  // namespace gbd
