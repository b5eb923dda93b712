// C ABI of the demag convolution + exchange/LLG/RK4 library (declarations and contracts in
// include/gbdemag.h). Host side: argument checks, planning, device buffers, the kernel
// spectrum upload and the launch sequences of Eq. 1 (Sec. II) and of the RK4 time step.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "gbdemag.h"
#include "gbd_fft.cuh"
#include "gbd_kernels.cuh"
#include "gbd_plan.h"

static thread_local std::string g_err;

static gbd_status fail(gbd_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

static gbd_status cuda_fail(cudaError_t e, const char* where) {
  return fail(GBD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

struct gbd_mesh {
  gbd_mesh_desc d;
  gbd::Plan p;
  int device = -1;
  float2* S = nullptr;      // x spectrum [3][nz][Hx][ny]
  float2* T = nullptr;      // 3D y spectrum [3][nz][Hx][Py] (ny > 1 and nz > 1)
  void* K = nullptr;        // packed kernel spectrum
  float* acc = nullptr;     // RK4 state: k-sum and two stage buffers, each [3][N]
  float* bufA = nullptr;
  float* bufB = nullptr;
  float2* tw = nullptr;     // twiddle table, GBD_TW_LEN entries
  bool kernel_set = false;
  // optional per-launch timing: events[2i], events[2i+1] bracket launch i of class cls[i]
  bool timing = false;
  std::vector<cudaEvent_t> events;
  std::vector<int> cls;
  size_t used = 0;
};

// Runs f() (which enqueues one kernel on st); with timing on, brackets it with events.
template <class F>
static void timed(gbd_mesh* m, int pass, cudaStream_t st, F f) {
  if (!m->timing) {
    f();
    return;
  }
  if (m->used + 2 > m->events.size()) {
    size_t grow = m->events.size() < 256 ? 256 : m->events.size();
    for (size_t i = 0; i < grow; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        f();
        return;
      }
      m->events.push_back(e);
    }
  }
  cudaEventRecord(m->events[m->used], st);
  f();
  cudaEventRecord(m->events[m->used + 1], st);
  m->cls.push_back(pass);
  m->used += 2;
}

namespace gbd {

static int pow2_at_least(long long v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

bool make_plan(int nx, int ny, int nz, Plan& p, const char** why) {
  if (nx < 1 || ny < 1 || nz < 1) {
    *why = "mesh sizes must be >= 1";
    return false;
  }
  p.nx = nx;
  p.ny = ny;
  p.nz = nz;
  p.N = (long long)nx * ny * nz;
  p.Px = nx == 1 ? 2 : pow2_at_least(2LL * nx - 1);
  p.Py = ny == 1 ? 1 : pow2_at_least(2LL * ny - 1);
  p.Pz = nz == 1 ? 1 : pow2_at_least(2LL * nz - 1);
  if (p.Px > kMaxPadX || p.Py > kMaxPad || p.Pz > kMaxPad) {
    *why = "mesh too large: supported nx <= 4096, ny <= 2048, nz <= 2048";
    return false;
  }
  p.Lx = p.Px / 2;
  p.Hx = p.Lx + 1;
  p.Ky = p.Py / 2 + 1;
  p.Kz = p.Pz / 2 + 1;
  p.film = (nz == 1);
  // block shapes (the kernels are compiled for these per transform length)
  p.RB = row_rb(p.Lx);
  p.Cf = film_cols(p.Py);
  p.Cy = ypass_lines(p.Py);
  p.Wz = zconv_cols(p.Pz);
  p.bytes_S = (size_t)3 * nz * p.Hx * ny * sizeof(float2);
  p.bytes_T = (!p.film && ny > 1) ? (size_t)3 * nz * p.Hx * p.Py * sizeof(float2) : 0;
  p.bytes_K = p.film ? (size_t)p.Hx * p.Ky * sizeof(float4) : (size_t)p.Hx * p.Ky * p.Kz * 6 * sizeof(float);
  p.bytes_state = (size_t)3 * 3 * p.N * sizeof(float);
  p.bytes_tw = (size_t)GBD_TW_LEN * sizeof(float2);
  return true;
}

}  // namespace gbd

static gbd_status check_desc(const gbd_mesh_desc* d, gbd::Plan& p) {
  if (!d) return fail(GBD_EINVAL, "desc is NULL");
  const char* why = nullptr;
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(GBD_EINVAL, "mesh sizes must be >= 1");
  if (!(d->dx > 0 && d->dy > 0 && d->dz > 0) || !std::isfinite(d->dx * d->dy * d->dz))
    return fail(GBD_EINVAL, "cell sizes must be finite and > 0");
  if (!(d->Ms > 0) || !std::isfinite(d->Ms)) return fail(GBD_EINVAL, "Ms must be finite and > 0");
  if (!(d->A_ex >= 0) || !std::isfinite(d->A_ex)) return fail(GBD_EINVAL, "A_ex must be finite and >= 0");
  if (!(d->alpha >= 0) || !std::isfinite(d->alpha)) return fail(GBD_EINVAL, "alpha must be finite and >= 0");
  if (!(d->gamma >= 0) || !std::isfinite(d->gamma)) return fail(GBD_EINVAL, "gamma must be finite and >= 0");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(d->Hext[i])) return fail(GBD_EINVAL, "Hext must be finite");
  if (d->precision != GBD_FP32) return fail(GBD_EUNSUPPORTED, "only GBD_FP32 meshes are built by gbd_mesh_create");
  if (!gbd::make_plan(d->nx, d->ny, d->nz, p, &why)) return fail(GBD_EUNSUPPORTED, why);
  return GBD_OK;
}

static bool ptr_ok(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) % 4 == 0); }

static gbd_status check_device(const gbd_mesh* m) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != m->device) return fail(GBD_ECUDA, "current device differs from the mesh's device");
  e = cudaPeekAtLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
  return GBD_OK;
}

static void free_mesh_buffers(gbd_mesh* m) {
  cudaFree(m->S);
  cudaFree(m->T);
  cudaFree(m->K);
  cudaFree(m->acc);
  cudaFree(m->bufA);
  cudaFree(m->bufB);
  cudaFree(m->tw);
  m->S = m->T = nullptr;
  m->K = nullptr;
  m->acc = m->bufA = m->bufB = nullptr;
  m->tw = nullptr;
}

// ---- launch sequences ------------------------------------------------------------------------

static gbd::RowArgs row_args(const gbd_mesh* m) {
  const gbd::Plan& p = m->p;
  const gbd_mesh_desc& d = m->d;
  gbd::RowArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nx = p.nx;
  a.ny = p.ny;
  a.nz = p.nz;
  a.rows = p.ny * p.nz;
  a.N = p.N;
  a.S = m->S;
  const double mu0 = 4.0e-7 * 3.14159265358979323846;
  const double lex = 2.0 * d.A_ex / (mu0 * d.Ms);
  a.cx = p.nx > 1 ? (float)(lex / (d.dx * d.dx)) : 0.f;
  a.cy = p.ny > 1 ? (float)(lex / (d.dy * d.dy)) : 0.f;
  a.cz = p.nz > 1 ? (float)(lex / (d.dz * d.dz)) : 0.f;
  a.hx = (float)d.Hext[0];
  a.hy = (float)d.Hext[1];
  a.hz = (float)d.Hext[2];
  const double gam = d.gamma > 0 ? d.gamma : 2.212761569e5;
  a.geff = (float)(gam / (1.0 + d.alpha * d.alpha));
  a.alpha = (float)d.alpha;
  a.hscale = (float)d.Ms;
  return a;
}

static gbd::ColArgs col_args(const gbd_mesh* m) {
  const gbd::Plan& p = m->p;
  gbd::ColArgs a;
  std::memset(&a, 0, sizeof(a));
  a.Hx = p.Hx;
  a.ny = p.ny;
  a.nz = p.nz;
  a.Py = p.Py;
  a.Pz = p.Pz;
  return a;
}

// Middle of Eq. 1: everything between the forward and the inverse x transforms.
static void enqueue_conv(gbd_mesh* m, cudaStream_t st) {
  const gbd::Plan& p = m->p;
  gbd::ColArgs a = col_args(m);
  if (p.film) {
    a.dst = m->S;
    a.Kf = static_cast<const float4*>(m->K);
    timed(m, GBD_PASS_FILM_CONV, st, [&] { gbd::launch_film_conv(a, m->tw, st); });
    return;
  }
  a.K3 = static_cast<const float*>(m->K);
  if (p.ny > 1) {
    a.lines_total = 3LL * p.nz * p.Hx;
    a.src = m->S;
    a.dst = m->T;
    timed(m, GBD_PASS_Y_FWD, st, [&] { gbd::launch_y_fwd(a, m->tw, st); });
    a.dst = m->T;
    a.Q = (long long)p.Hx * p.Py;
    a.Pyq = p.Py;
    timed(m, GBD_PASS_Z_CONV, st, [&] { gbd::launch_z_conv(a, m->tw, st); });
    a.src = m->T;
    a.dst = m->S;
    timed(m, GBD_PASS_Y_INV, st, [&] { gbd::launch_y_inv(a, m->tw, st); });
  } else {
    a.dst = m->S;
    a.Q = p.Hx;
    a.Pyq = 1;
    timed(m, GBD_PASS_Z_CONV, st, [&] { gbd::launch_z_conv(a, m->tw, st); });
  }
}

static gbd_status after_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, where);
  return GBD_OK;
}

// ---- C ABI -----------------------------------------------------------------------------------

extern "C" {

const char* gbd_last_error(void) { return g_err.c_str(); }

gbd_status gbd_plan_dims(const gbd_mesh_desc* desc, int out[6]) {
  gbd::Plan p;
  gbd_status s = check_desc(desc, p);
  if (s != GBD_OK) return s;
  if (!out) return fail(GBD_EINVAL, "out is NULL");
  out[0] = p.Px;
  out[1] = p.Py;
  out[2] = p.Pz;
  out[3] = p.Hx;
  out[4] = p.Ky;
  out[5] = p.Kz;
  return GBD_OK;
}

gbd_status gbd_mesh_bytes(const gbd_mesh_desc* desc, size_t* out) {
  gbd::Plan p;
  gbd_status s = check_desc(desc, p);
  if (s != GBD_OK) return s;
  if (!out) return fail(GBD_EINVAL, "out is NULL");
  *out = p.total_bytes();
  return GBD_OK;
}

gbd_status gbd_tensor_at(const gbd_mesh_desc* desc, int X, int Y, int Z, double out[6]) {
  if (!desc || !out) return fail(GBD_EINVAL, "NULL argument");
  if (!(desc->dx > 0 && desc->dy > 0 && desc->dz > 0)) return fail(GBD_EINVAL, "cell sizes must be > 0");
  gbdt::tensor_at(X, Y, Z, desc->dx, desc->dy, desc->dz, out);
  return GBD_OK;
}

gbd_status gbd_kernel_spectrum_host(const gbd_mesh_desc* desc, double* out, size_t count) {
  gbd::Plan p;
  gbd_status s = check_desc(desc, p);
  if (s != GBD_OK) return s;
  const size_t need = (size_t)6 * p.Kz * p.Ky * p.Hx;
  if (!out || count != need) return fail(GBD_EINVAL, "out is NULL or count != 6*Kz*Ky*Hx");
  std::vector<double> spec;
  if (!gbdt::kernel_spectrum(p, desc->dx, desc->dy, desc->dz, spec)) return fail(GBD_ENOMEM, "host allocation failed");
  std::memcpy(out, spec.data(), need * sizeof(double));
  return GBD_OK;
}

gbd_status gbd_mesh_create(const gbd_mesh_desc* desc, gbd_mesh** out) {
  if (!out) return fail(GBD_EINVAL, "out is NULL");
  *out = nullptr;
  gbd::Plan p;
  gbd_status s = check_desc(desc, p);
  if (s != GBD_OK) return s;
  gbd_mesh* m = new (std::nothrow) gbd_mesh();
  if (!m) return fail(GBD_ENOMEM, "host allocation failed");
  m->d = *desc;
  m->p = p;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  struct {
    void** ptr;
    size_t bytes;
  } allocs[] = {{(void**)&m->S, p.bytes_S},      {(void**)&m->T, p.bytes_T},
                {(void**)&m->K, p.bytes_K},      {(void**)&m->acc, p.bytes_state / 3},
                {(void**)&m->bufA, p.bytes_state / 3}, {(void**)&m->bufB, p.bytes_state / 3},
                {(void**)&m->tw, p.bytes_tw}};
  for (auto& al : allocs) {
    if (al.bytes == 0) continue;
    e = cudaMalloc(al.ptr, al.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      free_mesh_buffers(m);
      delete m;
      return fail(e == cudaErrorMemoryAllocation ? GBD_ENOMEM : GBD_ECUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  // twiddles exp(-2 pi i m / GBD_TW_LEN), FP64 on the host, rounded to FP32
  std::vector<float2> tw(GBD_TW_LEN);
  for (int k = 0; k < GBD_TW_LEN; ++k) {
    const double ang = -2.0 * 3.14159265358979323846264338327950288 * (double)k / GBD_TW_LEN;
    tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  e = cudaMemcpy(m->tw, tw.data(), p.bytes_tw, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    free_mesh_buffers(m);
    delete m;
    return cuda_fail(e, "cudaMemcpy twiddles");
  }
  *out = m;
  return GBD_OK;
}

gbd_status gbd_mesh_set_timing(gbd_mesh* m, int enable) {
  if (!m) return fail(GBD_EINVAL, "mesh is NULL");
  m->timing = enable != 0;
  return GBD_OK;
}

gbd_status gbd_mesh_read_timing(gbd_mesh* m, double* ms, long long* launches) {
  if (!m || !ms || !launches) return fail(GBD_EINVAL, "NULL argument");
  for (int i = 0; i < GBD_NPASS; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  for (size_t i = 0; i < m->cls.size(); ++i) {
    cudaError_t e = cudaEventSynchronize(m->events[2 * i + 1]);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, m->events[2 * i], m->events[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "gbd_mesh_read_timing");
    ms[m->cls[i]] += t;
    launches[m->cls[i]] += 1;
  }
  m->cls.clear();
  m->used = 0;
  return GBD_OK;
}

gbd_status gbd_mesh_destroy(gbd_mesh* m) {
  if (!m) return GBD_OK;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : m->events) cudaEventDestroy(e);
  free_mesh_buffers(m);
  delete m;
  return GBD_OK;
}

gbd_status gbd_set_kernel(gbd_mesh* m, void* stream) {
  if (!m) return fail(GBD_EINVAL, "mesh is NULL");
  gbd_status s = check_device(m);
  if (s != GBD_OK) return s;
  const gbd::Plan& p = m->p;
  std::vector<double> spec;
  if (!gbdt::kernel_spectrum(p, m->d.dx, m->d.dy, m->d.dz, spec)) return fail(GBD_ENOMEM, "host allocation failed");
  const size_t plane = (size_t)p.Ky * p.Hx;
  const size_t comp = (size_t)p.Kz * plane;
  std::vector<float> packed;
  try {
    packed.resize(p.bytes_K / sizeof(float));
  } catch (...) {
    return fail(GBD_ENOMEM, "host allocation failed");
  }
  if (p.film) {
    // [kx][ky] x (xx, yy, zz, xy)
    for (int kx = 0; kx < p.Hx; ++kx)
      for (int ky = 0; ky < p.Ky; ++ky)
        for (int c = 0; c < 4; ++c)
          packed[((size_t)kx * p.Ky + ky) * 4 + c] = (float)spec[c * comp + (size_t)ky * p.Hx + kx];
  } else {
    // [kx][ky][kz] x (xx, yy, zz, xy, xz, yz)
    for (int kx = 0; kx < p.Hx; ++kx)
      for (int ky = 0; ky < p.Ky; ++ky)
        for (int kz = 0; kz < p.Kz; ++kz)
          for (int c = 0; c < 6; ++c)
            packed[(((size_t)kx * p.Ky + ky) * p.Kz + kz) * 6 + c] =
                (float)spec[c * comp + (size_t)kz * plane + (size_t)ky * p.Hx + kx];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(m->K, packed.data(), p.bytes_K, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "kernel upload");
  m->kernel_set = true;
  return GBD_OK;
}

static gbd_status ready(gbd_mesh* m) {
  if (!m) return fail(GBD_EINVAL, "mesh is NULL");
  if (!m->kernel_set) return fail(GBD_ESTATE, "gbd_set_kernel has not been called on this mesh");
  return check_device(m);
}

gbd_status gbd_demag(gbd_mesh* m, const float* M, float* H, void* stream) {
  gbd_status s = ready(m);
  if (s != GBD_OK) return s;
  if (!ptr_ok(M) || !ptr_ok(H)) return fail(GBD_EINVAL, "M and H must be non-NULL, 4-byte aligned device pointers");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbd::RowArgs a = row_args(m);
  a.in = M;
  a.mode = gbd::ROW_FWD;
  a.fwd_after = 1;
  timed(m, GBD_PASS_ROW_FWD, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
  enqueue_conv(m, st);
  a.hscale = 1.f;
  a.out = H;
  a.mode = gbd::ROW_H;
  a.fwd_after = 0;
  timed(m, GBD_PASS_ROW_INV, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
  return after_launch("gbd_demag");
}

static gbd_status field_like(gbd_mesh* m, const float* mm, float* out, int mode, void* stream, const char* name) {
  gbd_status s = ready(m);
  if (s != GBD_OK) return s;
  if (!ptr_ok(mm) || !ptr_ok(out)) return fail(GBD_EINVAL, "m and out must be non-NULL, 4-byte aligned device pointers");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbd::RowArgs a = row_args(m);
  a.in = mm;
  a.mode = gbd::ROW_FWD;
  a.fwd_after = 1;
  timed(m, GBD_PASS_ROW_FWD, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
  enqueue_conv(m, st);
  a.ms = mm;
  a.out = out;
  a.mode = mode;
  a.fwd_after = 0;
  timed(m, GBD_PASS_ROW_INV, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
  return after_launch(name);
}

gbd_status gbd_effective_field(gbd_mesh* m, const float* mm, float* H, void* stream) {
  return field_like(m, mm, H, gbd::ROW_HEFF, stream, "gbd_effective_field");
}

gbd_status gbd_llg_rhs(gbd_mesh* m, const float* mm, float* dmdt, void* stream) {
  return field_like(m, mm, dmdt, gbd::ROW_RHS, stream, "gbd_llg_rhs");
}

gbd_status gbd_llg_step(gbd_mesh* m, float* mm, int nsteps, double dt, void* stream) {
  gbd_status s = ready(m);
  if (s != GBD_OK) return s;
  if (!ptr_ok(mm)) return fail(GBD_EINVAL, "m must be a non-NULL, 4-byte aligned device pointer");
  if (nsteps < 0) return fail(GBD_EINVAL, "nsteps must be >= 0");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(GBD_EINVAL, "dt must be finite and > 0");
  if (nsteps == 0) return GBD_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbd::RowArgs a = row_args(m);
  a.dt = (float)dt;
  a.in = mm;
  a.mode = gbd::ROW_FWD;
  a.fwd_after = 1;
  timed(m, GBD_PASS_ROW_FWD, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
  a.m0 = mm;
  a.m0_out = mm;
  a.acc = m->acc;
  for (int step = 0; step < nsteps; ++step) {
    const bool last = (step == nsteps - 1);
    // stage inputs: m -> A -> B -> A -> m
    const float* ms[4] = {mm, m->bufA, m->bufB, m->bufA};
    float* mn[4] = {m->bufA, m->bufB, m->bufA, nullptr};
    for (int stage = 0; stage < 4; ++stage) {
      enqueue_conv(m, st);
      a.ms = ms[stage];
      a.mnext = mn[stage];
      a.mode = gbd::ROW_RK1 + stage;
      a.fwd_after = (last && stage == 3) ? 0 : 1;
      timed(m, GBD_PASS_ROW_RK, st, [&] { gbd::launch_row(m->p.Lx, a, m->tw, st); });
    }
  }
  return after_launch("gbd_llg_step");
}

}  // extern "C"

// ---- allocation-free demag -------------------------------------------------------------------
//
// Scratch for gbd_demag_noalloc: the x spectrum and, for 3D meshes, the y spectrum of one
// demag evaluation live in this file-scope device array instead of the mesh's buffers.
// Every GPU that loads the library holds it (GBD_NOALLOC_MAX_BYTES) until the process exits.
// Host code cannot use the symbol as a device address: its device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GBD_NOALLOC_MAX_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoallocMaxDevices] = {nullptr};

// Same pass sequence as enqueue_conv, on caller-chosen spectrum buffers.
void enqueue_conv_on(const gbd_mesh* m, float2* S, float2* T, cudaStream_t st) {
  const gbd::Plan& p = m->p;
  gbd::ColArgs a = col_args(m);
  if (p.film) {
    a.dst = S;
    a.Kf = static_cast<const float4*>(m->K);
    gbd::launch_film_conv(a, m->tw, st);
    return;
  }
  a.K3 = static_cast<const float*>(m->K);
  if (p.ny > 1) {
    a.lines_total = 3LL * p.nz * p.Hx;
    a.src = S;
    a.dst = T;
    gbd::launch_y_fwd(a, m->tw, st);
    a.Q = (long long)p.Hx * p.Py;
    a.Pyq = p.Py;
    gbd::launch_z_conv(a, m->tw, st);
    a.src = T;
    a.dst = S;
    gbd::launch_y_inv(a, m->tw, st);
  } else {
    a.dst = S;
    a.Q = p.Hx;
    a.Pyq = 1;
    gbd::launch_z_conv(a, m->tw, st);
  }
}
}  // namespace

extern "C" gbd_status gbd_demag_noalloc(gbd_mesh* m, const float* M, float* H, void* stream) {
  gbd_status s = ready(m);
  if (s != GBD_OK) return s;
  if (!ptr_ok(M) || !ptr_ok(H)) return fail(GBD_EINVAL, "M and H must be non-NULL, 4-byte aligned device pointers");
  const gbd::Plan& p = m->p;
  const size_t s_bytes = (p.bytes_S + 255) / 256 * 256;
  const size_t need = s_bytes + p.bytes_T;
  if (need > (size_t)GBD_NOALLOC_MAX_BYTES)
    return fail(GBD_EBUDGET, "gbd_demag_noalloc: this mesh needs " + std::to_string(need) +
                                 " bytes of scratch, more than the static maximum of " +
                                 std::to_string((size_t)GBD_NOALLOC_MAX_BYTES));
  int dev = m->device;
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(GBD_EUNSUPPORTED, "gbd_demag_noalloc: device ordinal out of range");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) return cuda_fail(e, "gbd_demag_noalloc: cudaGetSymbolAddress");
      g_noalloc_addr[dev] = ptr;
    }
    base = g_noalloc_addr[dev];
  }
  float2* S = static_cast<float2*>(base);
  float2* T = p.bytes_T ? reinterpret_cast<float2*>(static_cast<unsigned char*>(base) + s_bytes) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  gbd::RowArgs a = row_args(m);
  a.S = S;
  a.in = M;
  a.mode = gbd::ROW_FWD;
  a.fwd_after = 1;
  gbd::launch_row(p.Lx, a, m->tw, st);
  enqueue_conv_on(m, S, T, st);
  a.hscale = 1.f;
  a.out = H;
  a.mode = gbd::ROW_H;
  a.fwd_after = 0;
  gbd::launch_row(p.Lx, a, m->tw, st);
  return after_launch("gbd_demag_noalloc");
}
