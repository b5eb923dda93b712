// sm_103a x-row kernel of the demag convolution (Sec. II, Eq. 1; the xFFT_R2C / xFFT_C2R
// steps of Appendix A with one GPU) with the fused exchange (Eq. 4) + LLG (Eq. 5) + RK4
// epilogue (Sec. III). The inverse x transform, the epilogue and the next stage's forward
// x transform run in one launch on RB rows per block (gbd_row.cuh). This unit holds the FP32
// row kernels, the epilogue-only kernels and the launchers.
#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

#include "gbd_rowpipe.cuh"

namespace gbd {

int sm_count() {
  static int count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (count[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    count[dev] = n > 0 ? n : 1;
  }
  return count[dev];
}

bool prep_seen(const void* k, int dev) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> seen;
  std::lock_guard<std::mutex> lock(mu);
  return !seen.insert(std::make_pair(k, dev)).second;
}

// Final combination of an RKF5(6) step, one thread per cell, and the block's largest error
// norm folded into *err_max (non-negative floats order like their bit patterns).
__global__ void __launch_bounds__(256) rkf_final_kernel(const RkfArgs a) {
  __shared__ float red[8];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.f;
  if (i < a.N) {
    float v[3], d[3];
    const float hs = a.hdev ? *a.hdev : 1.f;   // step size on the device, or folded into b5dt
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c] = a.m[c * a.N + i];
      d[c] = 0.f;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float ks = a.k[s][c * a.N + i];
        v[c] = fmaf(a.b5dt[s] * hs, ks, v[c]);
        d[c] = fmaf(a.db[s], ks, d[c]);
      }
    }
    const float inv = rsqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) a.out[c * a.N + i] = v[c] * inv;
    e2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2 = fmaxf(e2, __shfl_xor_sync(0xffffffffu, e2, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
    atomicMax(a.err_max, __float_as_uint(sqrtf(mx)));
  }
}

// Extrapolated RK4 stage without a transform (stages 2 and 3, and a last stage 4): the
// epilogue alone over all cells, the demag field from the history. One thread per pair of
// cells (nx % 64 == 0, 8-byte aligned fields) or per cell.
__global__ void __launch_bounds__(256) extrap_stage_kernel(const RowArgs a) {
  pdl_wait_then_release();
  const int nx = a.nx, ny = a.ny;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((nx % 64) == 0 && a.vec8) {
    // items in a warp are 32 consecutive pairs of one row: nx / 2 and 256 are multiples of 32
    const int NP2 = nx / 2;
    if (i >= (long long)a.rows * NP2) return;
    const int row = (int)(i / NP2);
    const int xp = (int)(i - (long long)row * NP2);
    const int z = row / ny, y = row - z * ny;
    const long long idx = (long long)row * nx + 2 * xp;
    float hd[2][3], mn[2][3];
    extrap_pair(a, idx, hd);
    epilogue_pair(a, a.mode, z, y, idx, 2 * xp, threadIdx.x & 31, hd, mn);
  } else {
    if (i >= a.N) return;
    const int row = (int)(i / nx);
    const int x = (int)(i - (long long)row * nx);
    const int z = row / ny, y = row - z * ny;
    float hd[3], mn[3];
    extrap_cell(a, i, hd);
    epilogue_cell(a, a.mode, z, y, x, i, hd, mn);
  }
}


// ---- launchers -------------------------------------------------------------------------------

// FP32 kernels here, split 16-bit ones in gbd_row_bf16.cu / gbd_row_fp16.cu. a == nullptr only
// prepares the kernels (both tile variants when var < 0, every precision when prec < 0).
static bool row_dispatch(int Lx, int var, int prec, const RowArgs* a, const float2* tw, cudaStream_t st) {
  bool ok = true;
  if (prec <= 0) ok = row_dispatch_p<0>(Lx, var, a, tw, st);
  if (ok && (prec == 1 || prec < 0)) ok = row_dispatch_p<1>(Lx, var, a, tw, st);
  if (ok && (prec == 2 || prec < 0)) ok = row_dispatch_p<2>(Lx, var, a, tw, st);
  return ok;
}

// The caller's fields need only 4-byte alignment; the 8-byte vector paths are enabled per
// launch from the actual pointers.
static void set_vec8(RowArgs& a) {
  auto al8 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; };
  bool ok = al8(a.in) && al8(a.ms) && al8(a.m0) && al8(a.m0_out) && al8(a.acc) && al8(a.mnext) && al8(a.out) &&
            al8(a.hrec);
  for (int k = 0; k < 6; ++k) ok = ok && al8(a.hist[k]);
  ok = ok && al8(a.kout);
  for (int k = 0; k < 7; ++k) ok = ok && al8(a.kin[k]);
  a.vec8 = ok ? 1 : 0;
}

// Tile variants 2 and 3 are the persistent pipelined kernel (gbd_rowpipe.cuh, FP32 only) where it
// applies (3: the RK stages stage only the spectrum tile, two blocks per SM); other launches of
// variants 2 and 3 take row_kernel's variant 1.
bool launch_row(int Lx, int var, int prec, const RowArgs& a0, const float2* tw, cudaStream_t st) {
  RowArgs a = a0;
  set_vec8(a);
  if (mixed_len(Lx)) return prec == 0 && row_dispatch_mixed(Lx, var, &a, tw, st);
  if (var >= 2 && prec == 0) {
    const int kind = pipe_kind(Lx, a, var);
    if (kind >= 0) return pipe_dispatch(Lx, kind, &a, tw, st);
  }
  return row_dispatch(Lx, var >= 2 ? 1 : var, prec, &a, tw, st);
}

// One warp: lane l writes register r of each table at word r * 32 + l (Dft16Frags::load).
__global__ void __launch_bounds__(32) dft16_frag_kernel(unsigned* frag) {
  const int lane = threadIdx.x & 31;
  auto put = [&](const unsigned* f, int table) {
    for (int r = 0; r < 32; ++r) frag[table * 1024 + r * 32 + lane] = f[r];
  };
  Dft16Frags<-1, 1> a;
  a.build(lane);
  put(&a.f[0][0][0][0], 0);
  Dft16Frags<1, 1> b;
  b.build(lane);
  put(&b.f[0][0][0][0], 1);
  Dft16Frags<-1, 2> c;
  c.build(lane);
  put(&c.f[0][0][0][0], 2);
  Dft16Frags<1, 2> d;
  d.build(lane);
  put(&d.f[0][0][0][0], 3);
}

void launch_dft16_frags(float2* frag, cudaStream_t st) {
  dft16_frag_kernel<<<1, 32, 0, st>>>(reinterpret_cast<unsigned*>(frag));
}

void launch_rkf_final(const RkfArgs& a, cudaStream_t st) {
  rkf_final_kernel<<<(unsigned)((a.N + 255) / 256), 256, 0, st>>>(a);
}

// The host loop's rule on the device: err = h max|...| from the attempt's error word; accept when
// err <= tol; next size h min(fac_max, max(fac_min, safety (tol / err)^(1/6))), the last step cut
// at t_end; the loop goes on while t < t_end and fewer than max_steps attempts were made (so it
// always ends: every pass counts an attempt).
__global__ void rkf_control_kernel(RkfCtl* c, cudaGraphConditionalHandle cond, double safety, double fac_min,
                                   double fac_max) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double h = c->h;
  const double err = h * (double)__uint_as_float(c->err);
  const double fac = err == 0.0 ? fac_max : fmin(fac_max, fmax(fac_min, safety * pow(c->tol / err, 1.0 / 6.0)));
  const int ok = err <= c->tol;
  if (ok) {
    c->t += h;
    c->acc += 1;
  } else {
    c->rej += 1;
  }
  c->accepted = ok;
  c->err = 0u;
  c->h_next = h * fac;
  const double hn = fmin(c->h_next, c->t_end - c->t);
  c->h = hn;
  c->hf = (float)hn;
  const bool go = c->t < c->t_end && c->acc + c->rej < c->max_steps && hn > 0.0;
  cudaGraphSetConditional(cond, go ? 1u : 0u);
}

__global__ void __launch_bounds__(256) rkf_accept_kernel(const RkfCtl* c, const float* __restrict__ src,
                                                         float* __restrict__ dst, long long n) {
  if (!c->accepted) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

void launch_rkf_control(RkfCtl* c, cudaGraphConditionalHandle cond, double safety, double fac_min, double fac_max,
                        cudaStream_t st) {
  rkf_control_kernel<<<1, 32, 0, st>>>(c, cond, safety, fac_min, fac_max);
}

void launch_rkf_accept(const RkfCtl* c, const float* src, float* dst, long long n, cudaStream_t st) {
  rkf_accept_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(c, src, dst, n);
}

void launch_extrap_stage(const RowArgs& a0, cudaStream_t st) {
  RowArgs a = a0;
  set_vec8(a);
  const long long items = ((a.nx % 64) == 0 && a.vec8) ? (long long)a.rows * (a.nx / 2) : a.N;
  launch_pdl(extrap_stage_kernel, (unsigned)((items + 255) / 256), 256, 0, st, a);
}
bool prepare_row(int Lx, int prec) {
  if (mixed_len(Lx)) return prec <= 0 && row_dispatch_mixed(Lx, -1, nullptr, nullptr, nullptr);
  if (prec <= 0) pipe_dispatch(Lx, -1, nullptr, nullptr, nullptr);
  return row_dispatch(Lx, -1, prec, nullptr, nullptr, nullptr);
}

}  // namespace gbd
