// Persistent x-row kernel (Sec. II, Eq. 1; the xFFT_R2C / xFFT_C2R steps of Appendix A with one
// GPU, with the exchange (Eq. 4) + LLG (Eq. 5) + RK4 stage epilogue of Sec. III) that keeps the
// next row group's inputs in flight while it transforms the current one.
//
// One block per SM (two for forward-only and inverse-only launches) walks the row groups
// g = blockIdx.x, blockIdx.x + gridDim.x, ... of RB rows
// (RB LX = 2048 complex values per component, as in row_kernel). The global inputs of a group
// -- its [kx][y] spectrum tile and the field rows its epilogue reads (stage input m with the
// rows above and below, step-start m, k-sum), or the input rows of a forward transform -- are
// copied into shared staging buffers with cp.async while the previous group is transformed:
// the spectrum of group g + G is requested as soon as group g's spectrum has been consumed,
// its field rows as soon as group g's epilogue is done. Each block thus waits for global
// memory once, at its first group, instead of at every phase of every group.
//
// cp.async groups per iteration (oldest first): spectrum(g), fields(g) are outstanding at the
// top; wait_group 1 completes the spectrum, the spectrum of g + G is committed; wait_group 1
// completes the fields, the fields of g + G are committed. Empty groups are committed past
// the last row group so that the counting stays uniform.
#pragma once
#include <cstdint>

#include "gbd_row.cuh"

namespace gbd {

// PIPE_RK stages the spectrum tile and the epilogue's field rows (one block per SM); PIPE_RKS
// stages only the spectrum tile and reads the field rows in the epilogue (epilogue_pair), which
// leaves room for two blocks per SM.
enum PipeKind : int { PIPE_FWD = 0, PIPE_INV = 1, PIPE_RK = 2, PIPE_RKS = 3 };

// rows per group: 2048 complex values per component (LX in [64, 2048]); for LX = 3 * 2^k or
// 5 * 2^k, 2048 over the next power of two above LX
__host__ __device__ constexpr int pipe_rb(int LX) {
  return mixed_len(LX) ? (2048 / (2 * pow2_floor(LX)) > 0 ? 2048 / (2 * pow2_floor(LX)) : 1) : (LX >= 2048 ? 1 : 2048 / LX);
}

// Shared-memory layout of the pipelined kernel, in float2 slots, each part starting on a
// 16-byte boundary: the lines, the staged spectrum tile [3][LX + 1][RB] (not for forward-only
// launches), the staged field rows (RK stages: stage input m on RB + 2 rows, step-start m and
// k-sum on RB rows; forward-only: the input rows), [row][3][LX] floats each.
template <int LX>
__host__ __device__ constexpr int pipe_off_s() {
  return (3 * pipe_rb(LX) * line_stride<LX, true>() + 1) / 2 * 2;
}
template <int LX, int K>
__host__ __device__ constexpr int pipe_off_f() {
  return pipe_off_s<LX>() + (K == PIPE_FWD ? 0 : (3 * (LX + 1) * pipe_rb(LX) + 1) / 2 * 2);
}
template <int LX, int K>
__host__ __device__ constexpr size_t pipe_smem() {
  return (size_t)pipe_off_f<LX, K>() * 8 +
         (K == PIPE_RK ? (size_t)(3 * pipe_rb(LX) + 2) * 3 * LX * 4 : K == PIPE_FWD ? (size_t)pipe_rb(LX) * 3 * LX * 4 : 0);
}

// blocks per SM: the RK stage stages its field rows and fills the SM alone; the forward-only and
// inverse-only launches stage half as much and run two blocks per SM
__host__ __device__ constexpr int pipe_blocks(int K) { return K == PIPE_RK ? 1 : 2; }
__host__ __device__ constexpr bool pipe_rk(int K) { return K == PIPE_RK || K == PIPE_RKS; }

template <int LX, int K>
__global__ void __launch_bounds__(3 * pipe_rb(LX) * LX / GBD_E, pipe_blocks(K))
    row_pipe_kernel(RowArgs a, const float2* __restrict__ tw, int ngroups) {
  pdl_wait_then_release();
  constexpr int RB = pipe_rb(LX);
  constexpr int LINES = 3 * RB;
  constexpr int T = LINES * LX / GBD_E;
  constexpr int LS = line_stride<LX, true>();
  constexpr int NP = npasses(LX, false);
  constexpr int HX = LX + 1;
  constexpr int HALF = LX / 2;
  constexpr int VR = RB >= 2 ? 2 : 1;   // rows per vector access of the spectrum tile
  constexpr int RG = RB / VR;
  static_assert(NP >= 1 && T <= 1024, "pipelined row kernel: LX in [64, 2048]");
  extern __shared__ float2 sm[];
  float2* lines = sm;
  float2* sS = sm + pipe_off_s<LX>();                                 // [3][HX][RB]
  float* sF = reinterpret_cast<float*>(sm + pipe_off_f<LX, K>());
  float* sMs = sF;                                                    // [RB + 2][3][LX]  (RK)
  float* sM0 = sF + (RB + 2) * 3 * LX;                                // [RB][3][LX]
  float* sAc = sM0 + RB * 3 * LX;                                     // [RB][3][LX]
  float* sIn = sF;                                                    // [RB][3][LX]      (FWD)
  const long long N = a.N;
  const int nx = a.nx, ny = a.ny, nz = a.nz, mode = a.mode;
  const int nq = nx / 4;                                              // 16-byte chunks per field row
  const bool rk_acc = (K == PIPE_RK) && mode != ROW_RK1;              // stages 2-4 read m0 and acc

  auto issue_spectrum = [&](int g) {
    if (g < ngroups) {
      const int row0 = g * RB;
      const int z = row0 / ny, y0 = row0 - z * ny;
      for (int e = threadIdx.x; e < 3 * HX * RG; e += T) {
        const int q = e % RG;
        const int t2 = e / RG;
        const int k = t2 % HX, c = t2 / HX;
        const float2* src = a.S + ((long long)(c * nz + z) * HX + k) * ny + y0 + q * VR;
        float2* dst = sS + (c * HX + k) * RB + q * VR;
        if constexpr (VR == 2)
          cp_async16(dst, src);
        else
          cp_async8(dst, src);
      }
    }
    cp_async_commit();
  };
  auto issue_fields = [&](int g) {
    if (g < ngroups) {
      const int row0 = g * RB;
      const int z = row0 / ny, y0 = row0 - z * ny;
      const long long plane = (long long)z * ny;
      if constexpr (K == PIPE_RK) {
        // stage input rows y0 - 1 .. y0 + RB: a missing neighbour row is the row itself (free
        // boundary) or the row on the opposite face (periodic y)
        for (int e = threadIdx.x; e < (RB + 2) * 3 * nq; e += T) {
          const int q = e % nq;
          const int t2 = e / nq;
          const int c = t2 % 3, s = t2 / 3;
          int y = y0 - 1 + s;
          if (y < 0) y = (a.per & 2) ? ny - 1 : 0;
          if (y >= ny) y = (a.per & 2) ? 0 : ny - 1;
          cp_async16(sMs + (s * 3 + c) * LX + 4 * q, a.ms + c * N + (plane + y) * nx + 4 * q);
        }
        if (rk_acc) {
          for (int e = threadIdx.x; e < RB * 3 * nq; e += T) {
            const int q = e % nq;
            const int t2 = e / nq;
            const int c = t2 % 3, r = t2 / 3;
            const long long off = c * N + (long long)(row0 + r) * nx + 4 * q;
            cp_async16(sM0 + (r * 3 + c) * LX + 4 * q, a.m0 + off);
            cp_async16(sAc + (r * 3 + c) * LX + 4 * q, a.acc + off);
          }
        }
      } else if constexpr (K == PIPE_FWD) {
        for (int e = threadIdx.x; e < RB * 3 * nq; e += T) {
          const int q = e % nq;
          const int t2 = e / nq;
          const int c = t2 % 3, r = t2 / 3;
          cp_async16(sIn + (r * 3 + c) * LX + 4 * q, a.in + c * N + (long long)(row0 + r) * nx + 4 * q);
        }
      }
    }
    cp_async_commit();
  };

  int g = blockIdx.x;
  if constexpr (K != PIPE_FWD) issue_spectrum(g);
  if constexpr (K == PIPE_RK || K == PIPE_FWD) issue_fields(g);
  for (; g < ngroups; g += gridDim.x) {
    const int gn = g + gridDim.x;
    const int row0 = g * RB;
    const int z = row0 / ny, y0 = row0 - z * ny;
    if constexpr (K != PIPE_FWD) {
      // 1. the staged half spectrum X ([kx][row]) -> Z in the lines (half-length inverse real FFT)
      if constexpr (K == PIPE_RK)
        cp_async_wait<1>();
      else
        cp_async_wait<0>();
      __syncthreads();
      for (int e = threadIdx.x; e < RG * 3 * (HALF + 1); e += T) {
        const int k = e % (HALF + 1);     // consecutive lanes: consecutive frequencies
        const int t2 = e / (HALF + 1);
        const int c = t2 % 3;
        const int gg = t2 / 3;
        const float2 wp = twiddle_at<-1>(tw, 2 * LX, k);  // W^k, W = exp(-2 pi i / Px)
        const float2 wm = cconj(wp);
        const float2* Ak = sS + (c * HX + k) * RB + gg * VR;
        const float2* Bk = sS + (c * HX + LX - k) * RB + gg * VR;
#pragma unroll
        for (int u = 0; u < VR; ++u) {
          const float2 Au = Ak[u], Bu = Bk[u];
          float2 zk, zl = make_float2(0.f, 0.f);
          if (k == 0) {
            zk = cadd(cadd(Au, cconj(Bu)), cmul_i<1>(csub(Au, cconj(Bu))));
          } else {
            zk = cadd(cadd(Au, cconj(Bu)), cmul_i<1>(cmul(wm, csub(Au, cconj(Bu)))));
            zl = csub(cadd(Bu, cconj(Au)), cmul_i<1>(cmul(wp, csub(Bu, cconj(Au)))));
          }
          float2* L = lines + (c * RB + gg * VR + u) * LS;
          L[pad(k)] = zk;
          if (k != 0 && k != LX - k) L[pad(LX - k)] = zl;
        }
      }
      __syncthreads();
      issue_spectrum(gn);   // the tile has been consumed
      // 2. unnormalised inverse FFT; the last pass keeps the lower half (the cropped rows)
      adj_passes_smem<1, LX, false, LINES, false, LS, NP, 1, 0>(lines, tw);
      {
        constexpr int R0 = radix_at(LX, false, 0);
        if constexpr (R0 % 2 == 0) {
          stockham_pass_sm<1, true, LX, R0, 1, LINES, false, LS, true>(lines, tw);   // keeps the lower half
        } else {
          auto ld = [&](int line, int i) { return lines[line * LS + pad(i)]; };
          auto st_half = [&](int line, int i, float2 v) {
            if (i < HALF) lines[line * LS + pad(i)] = v;
          };
          pass_any<0, 1, true, LX, R0, 1, LINES, false, true>(tw, ld, st_half);
        }
      }
      if constexpr (K == PIPE_RK)
        cp_async_wait<1>();   // this group's field rows (the next spectrum may stay in flight)
      __syncthreads();
    } else {
      cp_async_wait<0>();
      __syncthreads();
    }

    if constexpr (K == PIPE_INV) {
      // 3. H_d rows out: the float view of line position x is 2 pad(x/2) + (x & 1)
      const int NP2 = nx / 2;
      for (int e = threadIdx.x; e < RB * 3 * NP2; e += T) {
        const int xp = e % NP2;
        const int t2 = e / NP2;
        const int rr = t2 % RB, c = t2 / RB;
        const float2 h = lines[(c * RB + rr) * LS + pad(xp)];
        *reinterpret_cast<float2*>(a.out + c * N + (long long)(row0 + rr) * nx + 2 * xp) =
            make_float2(h.x * a.hscale, h.y * a.hscale);
      }
      continue;   // the next iteration's barrier orders these reads before the lines are rewritten
    }

    if constexpr (K == PIPE_RKS) {
      // 3. exchange + LLG + RK stage per pair of cells, the field rows read from global memory:
      //    the 32 lanes of a warp take 32 consecutive pairs of one row (nx a multiple of 64)
      const int NP2 = nx / 2;
      for (int e = threadIdx.x; e < RB * NP2; e += T) {
        const int rr = e / NP2;
        const int xp = e - rr * NP2;
        const long long idx = (long long)(row0 + rr) * nx + 2 * xp;
        float hd[2][3], mn[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 h2 = lines[(c * RB + rr) * LS + pad(xp)];
          hd[0][c] = h2.x * a.hscale;
          hd[1][c] = h2.y * a.hscale;
        }
        if (epilogue_pair(a, mode, z, y0 + rr, idx, 2 * xp, threadIdx.x & 31, hd, mn) && a.fwd_after) {
#pragma unroll
          for (int c = 0; c < 3; ++c) lines[(c * RB + rr) * LS + pad(xp)] = make_float2(mn[0][c], mn[1][c]);
        }
      }
    } else if constexpr (K == PIPE_RK) {
      // 3. exchange + LLG + RK stage per pair of cells, from the staged rows
      const int NP2 = nx / 2;
      const long long sz = (long long)nx * ny;
      for (int e = threadIdx.x; e < RB * NP2; e += T) {
        const int rr = e / NP2;
        const int xp = e - rr * NP2;
        const int x0 = 2 * xp;
        const int y = y0 + rr;
        const long long idx = (long long)(row0 + rr) * nx + x0;
        float hd[2][3], mv[2][3], lap[2][3], m0v[2][3] = {}, accv[2][3] = {}, mn[2][3], ao[2][3], res[2][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 h2 = lines[(c * RB + rr) * LS + pad(xp)];
          hd[0][c] = h2.x * a.hscale;
          hd[1][c] = h2.y * a.hscale;
        }
        if (a.hrec) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            *reinterpret_cast<float2*>(a.hrec + c * N + idx) = make_float2(hd[0][c], hd[1][c]);
        }
        const long long ozm = z > 0 ? -sz : ((a.per & 4) ? (long long)(nz - 1) * sz : 0);
        const long long ozp = z < nz - 1 ? sz : ((a.per & 4) ? -(long long)(nz - 1) * sz : 0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* r0 = sMs + ((rr + 1) * 3 + c) * LX;
          const float2 cc = *reinterpret_cast<const float2*>(r0 + x0);
          const float2 ym = *reinterpret_cast<const float2*>(sMs + (rr * 3 + c) * LX + x0);
          const float2 yp = *reinterpret_cast<const float2*>(sMs + ((rr + 2) * 3 + c) * LX + x0);
          const float left = x0 > 0 ? r0[x0 - 1] : cc.x;          // free x boundary
          const float right = x0 + 2 < nx ? r0[x0 + 2] : cc.y;
          float2 zm = cc, zp = cc;
          if (nz > 1) {
            const float* p = a.ms + c * N + idx;
            zm = *reinterpret_cast<const float2*>(p + ozm);
            zp = *reinterpret_cast<const float2*>(p + ozp);
          }
          mv[0][c] = cc.x;
          mv[1][c] = cc.y;
          lap[0][c] = a.cx * (left - 2.f * cc.x + cc.y) + a.cy * (ym.x - 2.f * cc.x + yp.x) +
                      a.cz * (zm.x - 2.f * cc.x + zp.x);
          lap[1][c] = a.cx * (cc.x - 2.f * cc.y + right) + a.cy * (ym.y - 2.f * cc.y + yp.y) +
                      a.cz * (zm.y - 2.f * cc.y + zp.y);
          if (rk_acc) {
            const float2 q0 = *reinterpret_cast<const float2*>(sM0 + (rr * 3 + c) * LX + x0);
            const float2 qa = *reinterpret_cast<const float2*>(sAc + (rr * 3 + c) * LX + x0);
            m0v[0][c] = q0.x;
            m0v[1][c] = q0.y;
            accv[0][c] = qa.x;
            accv[1][c] = qa.y;
          }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) llg_update(a, mode, hd[u], mv[u], lap[u], m0v[u], accv[u], mn[u], ao[u], res[u]);
        // m0_out aliases m0 in stage 4: each cell is read (staged) and written by one block
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float2 v = make_float2(mn[0][c], mn[1][c]);
          if (mode == ROW_RK4) {
            *reinterpret_cast<float2*>(a.m0_out + c * N + idx) = v;
          } else {
            *reinterpret_cast<float2*>(a.acc + c * N + idx) = make_float2(ao[0][c], ao[1][c]);
            *reinterpret_cast<float2*>(a.mnext + c * N + idx) = v;
          }
          if (a.fwd_after) lines[(c * RB + rr) * LS + pad(xp)] = v;
        }
      }
    } else {
      // 3. forward only: the staged input rows into the lines' float view
      for (int e = threadIdx.x; e < RB * 3 * (nx / 2); e += T) {
        const int xp = e % (nx / 2);
        const int t2 = e / (nx / 2);
        const int c = t2 % 3, r = t2 / 3;
        lines[(c * RB + r) * LS + pad(xp)] = *reinterpret_cast<const float2*>(sIn + (r * 3 + c) * LX + 2 * xp);
      }
    }
    // cells nx .. LX-1 of each line are zero padding for the forward transform
    if (nx < LX && (!pipe_rk(K) || a.fwd_after)) {
      for (int e = threadIdx.x; e < LINES * (LX - nx); e += T) {
        const int line = e / (LX - nx);
        const int x = nx + e % (LX - nx);
        reinterpret_cast<float*>(lines + line * LS)[2 * pad(x >> 1) + (x & 1)] = 0.f;
      }
    }
    __syncthreads();
    if constexpr (K == PIPE_RK || K == PIPE_FWD) issue_fields(gn);   // the staged rows have been consumed
    if (pipe_rk(K) && !a.fwd_after) continue;   // uniform over the grid
    // 4. forward FFT; the first pass reads the lower half only (the upper half is zero)
    {
      constexpr int R0 = radix_at(LX, false, 0);
      if constexpr (R0 % 2 == 0) {
        stockham_pass_sm<-1, false, LX, R0, 1, LINES, false, LS, true>(lines, tw);   // reads the lower half
      } else {
        auto ld_half = [&](int line, int i) { return i < HALF ? lines[line * LS + pad(i)] : make_float2(0.f, 0.f); };
        auto st = [&](int line, int i, float2 v) { lines[line * LS + pad(i)] = v; };
        pass_any<0, -1, false, LX, R0, 1, LINES, false, true>(tw, ld_half, st);
      }
      __syncthreads();
      fwd_passes_smem<-1, LX, false, LINES, false, LS, 1, NP, 0>(lines, tw);
    }
    // 5. Z -> X pairwise and store the half spectrum, VR adjacent rows per vector; adjacent lanes
    //    take the row groups of one frequency, so that a lane pair writes whole 32-byte sectors
    //    of the [kx][y] spectrum (RB = 4)
    for (int e = threadIdx.x; e < RG * 3 * (HALF + 1); e += T) {
      const int gg = e % RG;
      const int t2 = e / RG;
      const int k = t2 % (HALF + 1);
      const int c = t2 / (HALF + 1);
      const float2 wp = twiddle_at<-1>(tw, 2 * LX, k);
      const float2 wm = cconj(wp);
      float2 xk[VR], xl[VR];
#pragma unroll
      for (int u = 0; u < VR; ++u) {
        const float2* L = lines + (c * RB + gg * VR + u) * LS;
        if (k == 0) {
          const float2 A = L[pad(0)];
          xk[u] = make_float2(A.x + A.y, 0.f);
          xl[u] = make_float2(A.x - A.y, 0.f);
        } else {
          const float2 A = L[pad(k)], B = L[pad(LX - k)];
          xk[u] = cscale(csub(cadd(A, cconj(B)), cmul_i<1>(cmul(wp, csub(A, cconj(B))))), 0.5f);
          xl[u] = cscale(cadd(cadd(B, cconj(A)), cmul_i<1>(cmul(wm, csub(B, cconj(A))))), 0.5f);
        }
      }
      const int kl = (k == 0) ? LX : LX - k;
      const bool two = (k == 0) || (LX - k != k);
      float2* base = a.S + (long long)(c * nz + z) * HX * ny + y0 + gg * VR;
      if constexpr (VR == 2) {
        *reinterpret_cast<float4*>(base + (long long)k * ny) = make_float4(xk[0].x, xk[0].y, xk[1].x, xk[1].y);
        if (two) *reinterpret_cast<float4*>(base + (long long)kl * ny) = make_float4(xl[0].x, xl[0].y, xl[1].x, xl[1].y);
      } else {
        base[(long long)k * ny] = xk[0];
        if (two) base[(long long)kl * ny] = xl[0];
      }
    }
    // the next iteration's first barrier orders these reads before the lines are rewritten
  }
  cp_async_wait<0>();
}


// ---- launcher ------------------------------------------------------------------------------

int sm_count();   // multiprocessors of the current device (gbd_row.cu)

template <int LX, int K>
static void pipe_launch_t(const RowArgs* a, const float2* tw, cudaStream_t st) {
  constexpr int T = 3 * pipe_rb(LX) * LX / GBD_E;
  constexpr size_t smem = pipe_smem<LX, K>();
  prep(row_pipe_kernel<LX, K>, smem);
  const int nsm = sm_count();   // looked up when the mesh is created, not inside a capture
  if (!a) return;
  const int ngroups = a->rows / pipe_rb(LX);
  const int slots = pipe_blocks(K) * nsm;
  const int grid = ngroups < slots ? ngroups : slots;
  launch_pdl(row_pipe_kernel<LX, K>, grid, T, smem, st, *a, tw, ngroups);
}

// The kind of pipelined launch that serves a for tile variant var (2: RK stages stage their field
// rows, 3: they read them directly) (-1: none; the caller uses row_kernel). a.vec8 must be set.
// The staged rows are copied in 16-byte pieces, so the fields read through the staging buffers
// must be 16-byte aligned and nx a multiple of 4; a group's RB rows lie in one plane.
static int pipe_kind(int Lx, const RowArgs& a, int var) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (Lx < 64 || Lx > 2048 || (a.per & 1) || a.extrap || !a.vec8 || a.nx % 4 != 0 || a.ny % pipe_rb(Lx) != 0)
    return -1;
  if (a.mode == ROW_FWD) return al16(a.in) ? PIPE_FWD : -1;
  if (a.mode == ROW_H) return (a.hrec == nullptr) ? PIPE_INV : -1;
  if (a.mode >= ROW_RK1 && a.mode <= ROW_RK4) {
    if (var == 3) return (a.nx % 64 == 0) ? PIPE_RKS : -1;
    const bool reads_acc = a.mode != ROW_RK1;
    return (al16(a.ms) && (!reads_acc || (al16(a.m0) && al16(a.acc)))) ? PIPE_RK : -1;
  }
  return -1;
}

// Launches (a == nullptr: prepares every kind) the pipelined kernel for length Lx through the
// length switch SW (row_switch, or the mixed-length one); false when there is no
// instantiation for Lx.
template <class SW>
static bool pipe_dispatch_with(SW sw, int Lx, int kind, const RowArgs* a, const float2* tw, cudaStream_t st) {
  auto go = [&](auto lx) {
    constexpr int LX = decltype(lx)::value;
    if constexpr (LX >= 64 && LX <= 2048) {
      if (kind < 0 || kind == PIPE_FWD) pipe_launch_t<LX, PIPE_FWD>(a, tw, st);
      if (kind < 0 || kind == PIPE_INV) pipe_launch_t<LX, PIPE_INV>(a, tw, st);
      if (kind < 0 || kind == PIPE_RK) pipe_launch_t<LX, PIPE_RK>(a, tw, st);
      if (kind < 0 || kind == PIPE_RKS) pipe_launch_t<LX, PIPE_RKS>(a, tw, st);
    }
  };
  if (Lx < 64 || Lx > 2048) return false;
  return sw(Lx, go);
}
static bool pipe_dispatch(int Lx, int kind, const RowArgs* a, const float2* tw, cudaStream_t st) {
  return pipe_dispatch_with([](int L, auto f) { return row_switch(L, f); }, Lx, kind, a, tw, st);
}

}  // namespace gbd
