// sm_103a kernels of the demag convolution (Sec. II, Eq. 1; single-GPU steps of Appendix A)
// and of the fused exchange (Eq. 4) + LLG (Eq. 5) + RK4 update (Sec. III).
//
// Passes of one demag evaluation (P = padded lengths, Lx = Px / 2, Hx = Lx + 1):
//   row kernel, forward:  x real-to-complex of the zero-padded rows -> S [3][nz][Hx][ny]
//   film (nz = 1):        film_conv: y FFT -> kernel product -> y IFFT, in place on S
//   3D:                   y_fwd S -> T [3][nz][Hx][Py]; z_conv on T (z FFT -> product ->
//                         z IFFT, only the nz stored planes); y_inv T -> S
//   row kernel, inverse:  x complex-to-real + crop, then the mode's epilogue; the RK4
//                         modes also run the next stage's forward x transform.
// The padding is never stored: loads past n_d read zeros and cropped outputs are not
// written, so S keeps ny rows and T keeps nz planes.
#include "gbd_fft.cuh"
#include "gbd_kernels.cuh"

namespace gbd {

// ---------------------------------------------------------------------------------------------
// x rows: real-to-complex through a half-length complex FFT.
// For a real row x of length Px = 2 Lx: z[m] = x[2m] + i x[2m+1], Z = FFT_Lx(z), then for
// k in [0, Lx]:  X[k] = (Z[k] + Z*[Lx-k]) / 2 - (i/2) W^k (Z[k] - Z*[Lx-k]),  W = exp(-2 pi i / Px).
// The inverse builds Z[k] = (X[k] + X*[Lx-k]) + i W^-k (X[k] - X*[Lx-k]) and its unnormalised
// inverse FFT gives x[2m] + i x[2m+1] (times nothing: the 1/P factors live in the kernel).
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ long long s_index(int c, int z, int kx, int y, int nz, int Hx, int ny) {
  return ((long long)(c * nz + z) * Hx + kx) * ny + y;
}

template <int MODE, bool FWD_AFTER>
__global__ void __launch_bounds__(1024) row_kernel(RowArgs a, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int LS = a.Lx + 1;          // line stride (float2); slot Lx holds X[Lx] while staging
  const int RB = a.RB;
  const int lines = 3 * RB;
  const int r0 = blockIdx.x * RB;
  const int T = blockDim.x;
  const long long N = a.N;

  if (MODE != ROW_FWD) {
    // 1. stage the half spectrum X[kx], kx in [0, Hx), of the block's rows (rr fastest).
    for (int e = threadIdx.x; e < lines * a.Hx; e += T) {
      int rr = e % RB;
      int t2 = e / RB;
      int c = t2 % 3;
      int kx = t2 / 3;
      int row = r0 + rr;
      float2 v = make_float2(0.f, 0.f);
      if (row < a.rows) {
        int z = row / a.ny, y = row - (row / a.ny) * a.ny;
        v = a.S[s_index(c, z, kx, y, a.nz, a.Hx, a.ny)];
      }
      sm[(c * RB + rr) * LS + kx] = v;
    }
    __syncthreads();
    // 2. X -> Z pairwise, (k, Lx - k) for k in [0, Lx/2].
    const int half = a.Lx / 2;
    for (int e = threadIdx.x; e < lines * (half + 1); e += T) {
      int line = e / (half + 1);
      int k = e - line * (half + 1);
      float2* L = sm + line * LS;
      if (k == 0) {
        float2 A = L[0], B = L[a.Lx];
        float2 s = cadd(A, cconj(B)), d = csub(A, cconj(B));
        L[0] = cadd(s, cmul_i<1>(d));
      } else {
        float2 A = L[k], B = L[a.Lx - k];
        float2 wm = twiddle<1>(tw, k * a.tw_stride);   // W^-k = exp(+2 pi i k / Px)
        float2 wp = twiddle<-1>(tw, k * a.tw_stride);  // W^k
        float2 zk = cadd(cadd(A, cconj(B)), cmul_i<1>(cmul(wm, csub(A, cconj(B)))));
        float2 zl = csub(cadd(B, cconj(A)), cmul_i<1>(cmul(wp, csub(B, cconj(A)))));
        L[k] = zk;
        if (a.Lx - k != k) L[a.Lx - k] = zl;
      }
    }
    __syncthreads();
    // 3. unnormalised inverse FFT of length Lx on every line.
    fft_lines_smem<1, false>(sm, a.Lx, LS, lines, tw);
    // 4. epilogue on the real rows: float view xs[x] = x_un[x], x < nx.
    for (int e = threadIdx.x; e < RB * a.nx; e += T) {
      int rr = e / a.nx;
      int x = e - rr * a.nx;
      int row = r0 + rr;
      if (row >= a.rows) continue;
      const long long idx = (long long)row * a.nx + x;
      float hd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) hd[c] = reinterpret_cast<const float*>(sm + (c * RB + rr) * LS)[x] * a.hscale;
      if (MODE == ROW_H) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.out[c * N + idx] = hd[c];
        continue;
      }
      // exchange: 7-point Laplacian, free boundaries (missing neighbour = the cell itself)
      const int z = row / a.ny, y = row - z * a.ny;
      const long long sx = 1, sy = a.nx, sz = (long long)a.nx * a.ny;
      const long long ixm = x > 0 ? idx - sx : idx, ixp = x < a.nx - 1 ? idx + sx : idx;
      const long long iym = y > 0 ? idx - sy : idx, iyp = y < a.ny - 1 ? idx + sy : idx;
      const long long izm = z > 0 ? idx - sz : idx, izp = z < a.nz - 1 ? idx + sz : idx;
      float m[3], H[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* p = a.ms + c * N;
        float mc = p[idx];
        m[c] = mc;
        float lap = a.cx * (p[ixp] - 2.f * mc + p[ixm]) + a.cy * (p[iyp] - 2.f * mc + p[iym]) +
                    a.cz * (p[izp] - 2.f * mc + p[izm]);
        H[c] = hd[c] + lap;
      }
      H[0] += a.hx;
      H[1] += a.hy;
      H[2] += a.hz;
      if (MODE == ROW_HEFF) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.out[c * N + idx] = H[c];
        continue;
      }
      // dm/dt = -gamma/(1+alpha^2) [m x H + alpha m x (m x H)]
      float mxH[3] = {m[1] * H[2] - m[2] * H[1], m[2] * H[0] - m[0] * H[2], m[0] * H[1] - m[1] * H[0]};
      float mmH[3] = {m[1] * mxH[2] - m[2] * mxH[1], m[2] * mxH[0] - m[0] * mxH[2], m[0] * mxH[1] - m[1] * mxH[0]};
      float f[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) f[c] = -a.geff * (mxH[c] + a.alpha * mmH[c]);
      if (MODE == ROW_RHS) {
#pragma unroll
        for (int c = 0; c < 3; ++c) a.out[c * N + idx] = f[c];
        continue;
      }
      float mn[3];
      if (MODE == ROW_RK1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a.acc[c * N + idx] = f[c];
          mn[c] = m[c] + 0.5f * a.dt * f[c];
          a.mnext[c * N + idx] = mn[c];
        }
      } else if (MODE == ROW_RK2 || MODE == ROW_RK3) {
        const float h = (MODE == ROW_RK2) ? 0.5f * a.dt : a.dt;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          a.acc[c * N + idx] += 2.f * f[c];
          mn[c] = a.m0[c * N + idx] + h * f[c];
          a.mnext[c * N + idx] = mn[c];
        }
      } else {  // ROW_RK4
        const float h = a.dt * (1.0f / 6.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) mn[c] = a.m0[c * N + idx] + h * (a.acc[c * N + idx] + f[c]);
        float inv = rsqrtf(mn[0] * mn[0] + mn[1] * mn[1] + mn[2] * mn[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          mn[c] *= inv;
          a.m0_out[c * N + idx] = mn[c];
        }
      }
      if (FWD_AFTER) {
#pragma unroll
        for (int c = 0; c < 3; ++c) reinterpret_cast<float*>(sm + (c * RB + rr) * LS)[x] = mn[c];
      }
    }
    if (!FWD_AFTER) return;
    __syncthreads();
  }

  // 5. forward: rows in the float view, zero from nx up to Px (= 2 Lx floats).
  if (MODE == ROW_FWD) {
    for (int e = threadIdx.x; e < lines * 2 * a.Lx; e += T) {
      int line = e / (2 * a.Lx);
      int x = e - line * 2 * a.Lx;
      int c = line / RB, rr = line - c * RB;
      int row = r0 + rr;
      float v = 0.f;
      if (x < a.nx && row < a.rows) v = a.in[c * N + (long long)row * a.nx + x];
      reinterpret_cast<float*>(sm + line * LS)[x] = v;
    }
  } else {
    for (int e = threadIdx.x; e < lines * 2 * a.Lx; e += T) {
      int line = e / (2 * a.Lx);
      int x = e - line * 2 * a.Lx;
      int rr = line % RB;
      if (x >= a.nx || r0 + rr >= a.rows) reinterpret_cast<float*>(sm + line * LS)[x] = 0.f;
    }
  }
  __syncthreads();
  fft_lines_smem<-1, false>(sm, a.Lx, LS, lines, tw);
  // 6. Z -> X pairwise and store the half spectrum (rr fastest for the [kx][y] layout).
  const int half = a.Lx / 2;
  for (int e = threadIdx.x; e < lines * (half + 1); e += T) {
    int rr = e % RB;
    int t2 = e / RB;
    int c = t2 % 3;
    int k = t2 / 3;
    int row = r0 + rr;
    if (row >= a.rows) continue;
    int z = row / a.ny, y = row - z * a.ny;
    const float2* L = sm + (c * RB + rr) * LS;
    if (k == 0) {
      float2 A = L[0];
      a.S[s_index(c, z, 0, y, a.nz, a.Hx, a.ny)] = make_float2(A.x + A.y, 0.f);
      a.S[s_index(c, z, a.Lx, y, a.nz, a.Hx, a.ny)] = make_float2(A.x - A.y, 0.f);
    } else {
      float2 A = L[k], B = L[a.Lx - k];
      float2 wp = twiddle<-1>(tw, k * a.tw_stride);  // W^k
      float2 wm = twiddle<1>(tw, k * a.tw_stride);   // W^-k
      float2 xk = csub(cadd(A, cconj(B)), cmul_i<1>(cmul(wp, csub(A, cconj(B)))));
      float2 xl = cadd(cadd(B, cconj(A)), cmul_i<1>(cmul(wm, csub(B, cconj(A)))));
      a.S[s_index(c, z, k, y, a.nz, a.Hx, a.ny)] = cscale(xk, 0.5f);
      if (a.Lx - k != k) a.S[s_index(c, z, a.Lx - k, y, a.nz, a.Hx, a.ny)] = cscale(xl, 0.5f);
    }
  }
}

size_t row_smem_bytes(int RB, int Lx) { return (size_t)3 * RB * (Lx + 1) * sizeof(float2); }
int row_threads(int RB, int Lx) { return 3 * RB * Lx / GBD_E; }

template <int MODE, bool FWD>
static void row_launch_t(const RowArgs& a, const float2* tw, cudaStream_t st) {
  int blocks = (a.rows + a.RB - 1) / a.RB;
  size_t smem = row_smem_bytes(a.RB, a.Lx);
  auto k = row_kernel<MODE, FWD>;
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<blocks, row_threads(a.RB, a.Lx), smem, st>>>(a, tw);
}

void launch_row(int mode, bool fwd_after, const RowArgs& a, const float2* tw, cudaStream_t st) {
  switch (mode) {
    case ROW_FWD: row_launch_t<ROW_FWD, true>(a, tw, st); break;
    case ROW_H: row_launch_t<ROW_H, false>(a, tw, st); break;
    case ROW_HEFF: row_launch_t<ROW_HEFF, false>(a, tw, st); break;
    case ROW_RHS: row_launch_t<ROW_RHS, false>(a, tw, st); break;
    case ROW_RK1: fwd_after ? row_launch_t<ROW_RK1, true>(a, tw, st) : row_launch_t<ROW_RK1, false>(a, tw, st); break;
    case ROW_RK2: fwd_after ? row_launch_t<ROW_RK2, true>(a, tw, st) : row_launch_t<ROW_RK2, false>(a, tw, st); break;
    case ROW_RK3: fwd_after ? row_launch_t<ROW_RK3, true>(a, tw, st) : row_launch_t<ROW_RK3, false>(a, tw, st); break;
    default: fwd_after ? row_launch_t<ROW_RK4, true>(a, tw, st) : row_launch_t<ROW_RK4, false>(a, tw, st); break;
  }
}

// ---------------------------------------------------------------------------------------------
// Kernel product H~_a = sum_b K~_ab M~_b with the packed real spectrum. Stored indices are
// k' = k for k <= P/2 and P - k above; components odd along that axis change sign there
// (xy, yz odd in y; xz, yz odd in z). The 1/(Px Py Pz) and the minus sign of Eq. 1 are in K~.
// ---------------------------------------------------------------------------------------------

// film: one block = C columns kx, all three components, Py points each.
__global__ void __launch_bounds__(1024) film_conv_kernel(ColArgs a, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int C = a.C, Py = a.Py, LS = Py;
  const int lines = 3 * C;
  const int kx0 = blockIdx.x * C;
  const int T = blockDim.x;
  float2* S = a.dst;
  for (int e = threadIdx.x; e < lines * Py; e += T) {
    int line = e / Py;
    int y = e - line * Py;
    int c = line / C, cc = line - c * C;
    int kx = kx0 + cc;
    float2 v = make_float2(0.f, 0.f);
    if (y < a.ny && kx < a.Hx) v = S[s_index(c, 0, kx, y, 1, a.Hx, a.ny)];
    sm[line * LS + y] = v;
  }
  __syncthreads();
  fft_lines_smem<-1, false>(sm, Py, LS, lines, tw);
  const int Ky = Py / 2 + 1;
  for (int e = threadIdx.x; e < C * Py; e += T) {
    int cc = e / Py;
    int ky = e - cc * Py;
    int kx = kx0 + cc;
    if (kx >= a.Hx) continue;
    int kyp = ky;
    float sy = 1.f;
    if (Py > 1 && ky > Py / 2) {
      kyp = Py - ky;
      sy = -1.f;
    }
    float4 k4 = __ldg(a.Kf + (long long)kx * Ky + kyp);
    float kxy = sy * k4.w;
    float2 m0 = sm[(0 * C + cc) * LS + ky], m1 = sm[(1 * C + cc) * LS + ky], m2 = sm[(2 * C + cc) * LS + ky];
    sm[(0 * C + cc) * LS + ky] = make_float2(k4.x * m0.x + kxy * m1.x, k4.x * m0.y + kxy * m1.y);
    sm[(1 * C + cc) * LS + ky] = make_float2(kxy * m0.x + k4.y * m1.x, kxy * m0.y + k4.y * m1.y);
    sm[(2 * C + cc) * LS + ky] = make_float2(k4.z * m2.x, k4.z * m2.y);
  }
  __syncthreads();
  fft_lines_smem<1, false>(sm, Py, LS, lines, tw);
  for (int e = threadIdx.x; e < lines * a.ny; e += T) {
    int line = e / a.ny;
    int y = e - line * a.ny;
    int c = line / C, cc = line - c * C;
    int kx = kx0 + cc;
    if (kx < a.Hx) S[s_index(c, 0, kx, y, 1, a.Hx, a.ny)] = sm[line * LS + y];
  }
}

// 3D y passes: independent lines l = (c*nz + z)*Hx + kx; src line stride ny (fwd) or Py (inv).
template <bool INV>
__global__ void __launch_bounds__(1024) y_pass_kernel(ColArgs a, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int C = a.C, Py = a.Py, LS = Py;
  const long long l0 = (long long)blockIdx.x * C;
  const int T = blockDim.x;
  const int in_len = INV ? Py : a.ny;
  const int out_len = INV ? a.ny : Py;
  for (int e = threadIdx.x; e < C * Py; e += T) {
    int line = e / Py;
    int y = e - line * Py;
    long long l = l0 + line;
    float2 v = make_float2(0.f, 0.f);
    if (y < in_len && l < a.lines_total) v = a.src[l * in_len + y];
    sm[line * LS + y] = v;
  }
  __syncthreads();
  fft_lines_smem<INV ? 1 : -1, false>(sm, Py, LS, C, tw);
  for (int e = threadIdx.x; e < C * out_len; e += T) {
    int line = e / out_len;
    int y = e - line * out_len;
    long long l = l0 + line;
    if (l < a.lines_total) a.dst[l * out_len + y] = sm[line * LS + y];
  }
}

// 3D z convolution: block = C consecutive columns q of [3][nz][Q]; lines interleaved.
__global__ void __launch_bounds__(1024) z_conv_kernel(ColArgs a, const float2* __restrict__ tw) {
  extern __shared__ float2 sm[];
  const int W = a.C, Pz = a.Pz, LS = Pz + 1;
  const int lines = 3 * W;
  const long long q0 = (long long)blockIdx.x * W;
  const int T = blockDim.x;
  float2* D = a.dst;
  for (int e = threadIdx.x; e < lines * Pz; e += T) {
    int line = e % lines;
    int z = e / lines;
    int c = line / W, w = line - c * W;
    long long q = q0 + w;
    float2 v = make_float2(0.f, 0.f);
    if (z < a.nz && q < a.Q) v = D[(long long)(c * a.nz + z) * a.Q + q];
    sm[line * LS + z] = v;
  }
  __syncthreads();
  fft_lines_smem<-1, true>(sm, Pz, LS, lines, tw);
  const int Ky = a.Py / 2 + 1, Kz = Pz / 2 + 1;
  for (int e = threadIdx.x; e < W * Pz; e += T) {
    int w = e % W;
    int kz = e / W;
    long long q = q0 + w;
    if (q >= a.Q) continue;
    int kx = (int)(q / a.Pyq);
    int ky = (int)(q - (long long)kx * a.Pyq);
    int kyp = ky, kzp = kz;
    float sy = 1.f, sz = 1.f;
    if (a.Py > 1 && ky > a.Py / 2) {
      kyp = a.Py - ky;
      sy = -1.f;
    }
    if (Pz > 1 && kz > Pz / 2) {
      kzp = Pz - kz;
      sz = -1.f;
    }
    const float* kp = a.K3 + (((long long)kx * Ky + kyp) * Kz + kzp) * 6;
    float kxx = __ldg(kp), kyy = __ldg(kp + 1), kzz = __ldg(kp + 2);
    float kxy = sy * __ldg(kp + 3), kxz = sz * __ldg(kp + 4), kyz = sy * sz * __ldg(kp + 5);
    float2 m0 = sm[(0 * W + w) * LS + kz], m1 = sm[(1 * W + w) * LS + kz], m2 = sm[(2 * W + w) * LS + kz];
    sm[(0 * W + w) * LS + kz] = make_float2(kxx * m0.x + kxy * m1.x + kxz * m2.x, kxx * m0.y + kxy * m1.y + kxz * m2.y);
    sm[(1 * W + w) * LS + kz] = make_float2(kxy * m0.x + kyy * m1.x + kyz * m2.x, kxy * m0.y + kyy * m1.y + kyz * m2.y);
    sm[(2 * W + w) * LS + kz] = make_float2(kxz * m0.x + kyz * m1.x + kzz * m2.x, kxz * m0.y + kyz * m1.y + kzz * m2.y);
  }
  __syncthreads();
  fft_lines_smem<1, true>(sm, Pz, LS, lines, tw);
  for (int e = threadIdx.x; e < lines * a.nz; e += T) {
    int line = e % lines;
    int z = e / lines;
    int c = line / W, w = line - c * W;
    long long q = q0 + w;
    if (q < a.Q) D[(long long)(c * a.nz + z) * a.Q + q] = sm[line * LS + z];
  }
}

static void set_smem(const void* k, size_t smem) {
  if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

void launch_film_conv(const ColArgs& a, const float2* tw, cudaStream_t st) {
  size_t smem = (size_t)3 * a.C * a.Py * sizeof(float2);
  set_smem((const void*)film_conv_kernel, smem);
  int blocks = (a.Hx + a.C - 1) / a.C;
  film_conv_kernel<<<blocks, 3 * a.C * a.Py / GBD_E, smem, st>>>(a, tw);
}

void launch_y_fwd(const ColArgs& a, const float2* tw, cudaStream_t st) {
  size_t smem = (size_t)a.C * a.Py * sizeof(float2);
  set_smem((const void*)y_pass_kernel<false>, smem);
  int blocks = (a.lines_total + a.C - 1) / a.C;
  y_pass_kernel<false><<<blocks, a.C * a.Py / GBD_E, smem, st>>>(a, tw);
}

void launch_y_inv(const ColArgs& a, const float2* tw, cudaStream_t st) {
  size_t smem = (size_t)a.C * a.Py * sizeof(float2);
  set_smem((const void*)y_pass_kernel<true>, smem);
  int blocks = (a.lines_total + a.C - 1) / a.C;
  y_pass_kernel<true><<<blocks, a.C * a.Py / GBD_E, smem, st>>>(a, tw);
}

void launch_z_conv(const ColArgs& a, const float2* tw, cudaStream_t st) {
  size_t smem = (size_t)3 * a.C * (a.Pz + 1) * sizeof(float2);
  set_smem((const void*)z_conv_kernel, smem);
  long long blocks = (a.Q + a.C - 1) / a.C;
  z_conv_kernel<<<(unsigned)blocks, 3 * a.C * a.Pz / GBD_E, smem, st>>>(a, tw);
}

}  // namespace gbd
