// Host FP64 demag tensor and its packed convolution-kernel spectrum.
//
// Eq. 1 (Sec. II) uses the cell-averaged demagnetizing tensor of two uniformly
// magnetized rectangular cells (the formulas the paper cites, Newell, Williams and
// Dunlop 1993). N(R) = (1/V) int_i int_j K(r - r') with the point-dipole kernel
// K(r) = (I - 3 r r^T / r^2) / (4 pi r^3).
//
// * |R| < 8 d_max: closed form, a 27-point second-difference stencil (weights 2, -1, -1 per
//   axis) of the antiderivatives f (diagonal) and g (off-diagonal), over 4 pi dx dy dz.
// * |R| >= 8 d_max: the FP64 stencil loses digits to cancellation there, so the same
//   integral is taken by quadrature over the overlap u of the two cells,
//   N(R) = int prod_d (1 - |u_d| / d_d) K(R + u) du, split at u_d = 0 with G Gauss-Legendre
//   nodes per half axis: G = 4 below 16 d_max, 3 below 64 d_max, 2 beyond (within 2e-8 of
//   the exact value relative to V / (4 pi |R|^3)).
//
// Kernel spectrum (Sec. II, the "convolution kernel" of Appendix A): the tensor is placed
// on the periodic P grid at X mod P_d for |X_d| <= n_d - 1 and transformed. Each component
// is even or odd along each axis (xx, yy, zz even; xy odd in x, y; xz odd in x, z; yz odd
// in y, z), so along each axis the transform reduces to
//   G[k] = sum_{X >= 0} w_X N(X) cos(2 pi k X / P)   (even),  w_0 = 1, w_{X>0} = 2,
//   G[k] = sum_{X >= 0} w_X N(X) sin(2 pi k X / P)   (odd; the full transform is -i G),
// every component's spectrum is real, and only k_d in [0, P_d / 2] is stored. With the
// Eq. 1 minus sign and the 1/(Px Py Pz) of the unnormalised inverse folded in:
//   K~ = -G_x G_y G_z / (Px Py Pz) for xx, yy, zz and +G_x G_y G_z / (Px Py Pz) for xy, xz, yz.
// Each G is computed with a complex FFT of the symmetric extension of the line.
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <utility>
#include <vector>

#include "gbd_plan.h"

namespace gbdt {

static const double PI = 3.14159265358979323846264338327950288;

static inline double asinh_ratio(double num, double den) { return den > 0.0 ? std::asinh(num / den) : 0.0; }
static inline double atan_ratio(double num, double den) { return den > 0.0 ? std::atan(num / den) : 0.0; }

// f for N_xx on |x|, |y|, |z|; terms whose prefactor vanishes at 0/0 are dropped.
static double newell_f(double x, double y, double z) {
  x = std::fabs(x);
  y = std::fabs(y);
  z = std::fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = std::sqrt(x2 + y2 + z2);
  double t = 0.0;
  if (y > 0.0) t += 0.5 * y * (z2 - x2) * asinh_ratio(y, std::sqrt(x2 + z2));
  if (z > 0.0) t += 0.5 * z * (y2 - x2) * asinh_ratio(z, std::sqrt(x2 + y2));
  if (x > 0.0) t -= x * y * z * atan_ratio(y * z, x * R);
  t += (2.0 * x2 - y2 - z2) * R / 6.0;
  return t;
}

// g for N_xy: g(|x|, |y|, |z|) * sign(x) * sign(y).
static double newell_g(double x, double y, double z) {
  const double s = (x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0)) * (y > 0 ? 1.0 : (y < 0 ? -1.0 : 0.0));
  if (s == 0.0) return 0.0;
  x = std::fabs(x);
  y = std::fabs(y);
  z = std::fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = std::sqrt(x2 + y2 + z2);
  double t = 0.0;
  t += x * y * z * asinh_ratio(z, std::sqrt(x2 + y2));
  t += y / 6.0 * (3.0 * z2 - y2) * asinh_ratio(x, std::sqrt(y2 + z2));
  t += x / 6.0 * (3.0 * z2 - x2) * asinh_ratio(y, std::sqrt(x2 + z2));
  if (z > 0.0) {
    t -= z2 * z / 6.0 * atan_ratio(x * y, z * R);
    t -= z * y2 / 2.0 * atan_ratio(x * z, y * R);
    t -= z * x2 / 2.0 * atan_ratio(y * z, x * R);
  }
  t -= x * y * R / 3.0;
  return s * t;
}

typedef double (*AntiDer)(double, double, double);

static double stencil27(AntiDer F, double X, double Y, double Z, double dx, double dy, double dz) {
  static const double w[3] = {-1.0, 2.0, -1.0};
  double acc = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        acc += w[i] * w[j] * w[k] * F(X + (i - 1) * dx, Y + (j - 1) * dy, Z + (k - 1) * dz);
  return acc / (4.0 * PI * dx * dy * dz);
}

void newell_closed_form(double X, double Y, double Z, double dx, double dy, double dz, double out[6]) {
  out[0] = stencil27(newell_f, X, Y, Z, dx, dy, dz);
  out[1] = stencil27(newell_f, Y, X, Z, dy, dx, dz);
  out[2] = stencil27(newell_f, Z, Y, X, dz, dy, dx);
  out[3] = stencil27(newell_g, X, Y, Z, dx, dy, dz);
  out[4] = stencil27(newell_g, X, Z, Y, dx, dz, dy);
  out[5] = stencil27(newell_g, Y, Z, X, dy, dz, dx);
}

// Gauss-Legendre nodes/weights on [-1, 1] for G = 2, 3, 4.
static void gauss_legendre(int G, double* x, double* w) {
  if (G == 2) {
    x[0] = -1.0 / std::sqrt(3.0);
    x[1] = -x[0];
    w[0] = w[1] = 1.0;
  } else if (G == 3) {
    x[0] = -std::sqrt(0.6);
    x[1] = 0.0;
    x[2] = -x[0];
    w[0] = w[2] = 5.0 / 9.0;
    w[1] = 8.0 / 9.0;
  } else {
    const double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2));
    const double b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    x[0] = -b; w[0] = wb;
    x[1] = -a; w[1] = wa;
    x[2] = a;  w[2] = wa;
    x[3] = b;  w[3] = wb;
  }
}

void dipole_quadrature(double X, double Y, double Z, double dx, double dy, double dz, int G, double out[6]) {
  double xg[4], wg[4];
  gauss_legendre(G, xg, wg);
  // Rule for int_{-1}^{1} (1 - |s|) h(s) ds: nodes s = +-(x+1)/2, weights w/2 (1 - |s|).
  double s[8], ws[8];
  for (int i = 0; i < G; ++i) {
    const double u = 0.5 * (xg[i] + 1.0);
    s[i] = -u;
    s[G + i] = u;
    ws[i] = ws[G + i] = 0.5 * wg[i] * (1.0 - u);
  }
  const double V = dx * dy * dz;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int a = 0; a < 2 * G; ++a) {
    const double rx = X + s[a] * dx;
    for (int b = 0; b < 2 * G; ++b) {
      const double ry = Y + s[b] * dy;
      for (int c = 0; c < 2 * G; ++c) {
        const double rz = Z + s[c] * dz;
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double r = std::sqrt(r2);
        const double pre = ws[a] * ws[b] * ws[c] / (r2 * r);
        const double q = 3.0 / r2;
        acc[0] += pre * (1.0 - q * rx * rx);
        acc[1] += pre * (1.0 - q * ry * ry);
        acc[2] += pre * (1.0 - q * rz * rz);
        acc[3] -= pre * q * rx * ry;
        acc[4] -= pre * q * rx * rz;
        acc[5] -= pre * q * ry * rz;
      }
    }
  }
  for (int i = 0; i < 6; ++i) out[i] = acc[i] * V / (4.0 * PI);
}

void tensor_at(int X, int Y, int Z, double dx, double dy, double dz, double out[6]) {
  const double px = X * dx, py = Y * dy, pz = Z * dz;
  const double dmax = std::fmax(dx, std::fmax(dy, dz));
  const double r = std::sqrt(px * px + py * py + pz * pz) / dmax;
  if (r < 8.0)
    newell_closed_form(px, py, pz, dx, dy, dz, out);
  else
    dipole_quadrature(px, py, pz, dx, dy, dz, r < 16.0 ? 4 : (r < 64.0 ? 3 : 2), out);
}

// ---- FP64 host FFT (mixed radix, any length) -------------------------------------------------
// Decimation in time: a length-n transform (n = p m, p the smallest prime factor of n) is p
// length-m transforms of the samples t, t + p, t + 2p, ... followed by
//   X[q + s m] = sum_t W_n^(t (q + s m)) Y_t[q],  W_n = exp(-2 pi i / n),
// recursively; W_n^j comes from the table of the whole length N at index j N / n. The padded
// lengths here are 2^a 3^b 5^c, so every stage is a short sum.
struct Fft1 {
  int n = 0;
  std::vector<std::complex<double>> w;      // exp(-2 pi i k / n), k < n
  explicit Fft1(int n_) : n(n_), w(n_ > 0 ? n_ : 1) {
    for (int k = 0; k < n; ++k) w[k] = std::polar(1.0, -2.0 * PI * k / n);
  }
  static int smallest_factor(int m) {
    for (int f = 2; f * f <= m; ++f)
      if (m % f == 0) return f;
    return m;
  }
  // out[0 .. len) = DFT of in[0], in[stride], ..., in[(len - 1) stride]; out and in do not overlap
  void rec(const std::complex<double>* in, std::complex<double>* out, int len, int stride) const {
    if (len == 1) {
      out[0] = in[0];
      return;
    }
    const int p = smallest_factor(len), m = len / p;
    for (int t = 0; t < p; ++t) rec(in + t * stride, out + t * m, m, stride * p);
    const int step = n / len;   // W_len^j = w[j step]
    std::complex<double> y[8];
    for (int q = 0; q < m; ++q) {
      for (int t = 0; t < p; ++t) y[t] = out[t * m + q];
      for (int s = 0; s < p; ++s) {
        std::complex<double> acc = 0.0;
        for (int t = 0; t < p; ++t) acc += y[t] * w[((long long)t * (q + s * m) % len) * step];
        out[s * m + q] = acc;
      }
    }
  }
  // in place; shared by the threads of a parallel loop (each has its own copy buffer)
  void forward(std::complex<double>* a) const {
    if (n <= 1) return;
    thread_local std::vector<std::complex<double>> tmp;
    tmp.assign(a, a + n);
    rec(tmp.data(), a, n, 1);
  }
};

// G[k], k in [0, H), of the line v[X], X in [0, n), with the given parity on a period P.
static void line_transform(const Fft1* fft, int P, int n, int H, int parity, const double* v, long long vstride,
                           double* out, long long ostride, std::vector<std::complex<double>>& buf) {
  if (P == 1) {
    out[0] = v[0];
    return;
  }
  std::fill(buf.begin(), buf.end(), std::complex<double>(0.0, 0.0));
  buf[0] = v[0];
  for (int X = 1; X < n; ++X) {
    const double val = v[X * vstride];
    buf[X] = val;
    buf[P - X] = parity > 0 ? val : -val;
  }
  fft->forward(buf.data());
  for (int k = 0; k < H; ++k) out[k * ostride] = parity > 0 ? buf[k].real() : -buf[k].imag();
}

static const int PARITY[6][3] = {{1, 1, 1}, {1, 1, 1}, {1, 1, 1}, {-1, -1, 1}, {-1, 1, -1}, {1, -1, -1}};

// Packed spectrum, FP64, layout [6][Kz][Ky][Hx] with Hx = Px/2+1, Ky = Py/2+1 (1 if Py = 1),
// Kz likewise. Returns false on allocation failure.
// Point-dipole tensor V/(4 pi) (I/r^3 - 3 R R^T / r^5) at offset (X, Y, Z) cells: the far-field
// limit of the cell-pair average, used for periodic images beyond kImageDipoleR cell sizes.
static void point_dipole(double X, double Y, double Z, double dx, double dy, double dz, double out[6]) {
  const double x = X * dx, y = Y * dy, z = Z * dz;
  const double r2 = x * x + y * y + z * z;
  const double r = std::sqrt(r2);
  const double c = dx * dy * dz / (4.0 * PI * r2 * r);
  const double q = 3.0 / r2;
  out[0] = c * (1.0 - q * x * x);
  out[1] = c * (1.0 - q * y * y);
  out[2] = c * (1.0 - q * z * z);
  out[3] = -c * q * x * y;
  out[4] = -c * q * x * z;
  out[5] = -c * q * y * z;
}

constexpr double kImageDipoleR = 256.0;   // in units of the largest cell side

// The tensor at a signed offset from its octant value and the component parities.
static void signed_term(int X, int Y, int Z, double dx, double dy, double dz, double dmax, double out[6]) {
  const double r = std::sqrt((double)X * X * dx * dx + (double)Y * Y * dy * dy + (double)Z * Z * dz * dz) / dmax;
  double v[6];
  if (r >= kImageDipoleR)
    point_dipole(std::abs(X), std::abs(Y), std::abs(Z), dx, dy, dz, v);
  else
    tensor_at(std::abs(X), std::abs(Y), std::abs(Z), dx, dy, dz, v);
  for (int c = 0; c < 6; ++c) {
    double s = 1.0;
    if (X < 0 && PARITY[c][0] < 0) s = -s;
    if (Y < 0 && PARITY[c][1] < 0) s = -s;
    if (Z < 0 && PARITY[c][2] < 0) s = -s;
    out[c] = s * v[c];
  }
}

// (offset, weight) terms summed at octant index b of one axis: the offset itself, or along a
// periodic axis of period n its images b + i n, |i| <= K, with the +n/2 and -n/2 image sets
// averaged at b = n/2 so that odd components cancel there exactly.
static void axis_terms(int b, int n, bool periodic, int K, std::vector<std::pair<int, double>>& t) {
  t.clear();
  if (!periodic) {
    t.emplace_back(b, 1.0);
    return;
  }
  for (int i = -K; i <= K; ++i) {
    if (2 * b == n) {
      t.emplace_back(b + i * n, 0.5);
      t.emplace_back(-b + i * n, 0.5);
    } else {
      t.emplace_back(b + i * n, 1.0);
    }
  }
}

bool kernel_spectrum(const gbd::Plan& p, double dx, double dy, double dz, std::vector<double>& out) {
  const int ox = p.ox, oy = p.oy, oz = p.oz;
  const long long Noct = (long long)ox * oy * oz;
  std::vector<double> oct;
  try {
    oct.resize((size_t)Noct * 6);
  } catch (...) {
    return false;
  }
  const double dmax = std::fmax(dx, std::fmax(dy, dz));
#pragma omp parallel
  {
    std::vector<std::pair<int, double>> tx, ty, tz;
#pragma omp for schedule(dynamic, 16)
    for (long long i = 0; i < Noct; ++i) {
      const int X = (int)(i % ox), Y = (int)((i / ox) % oy), Z = (int)(i / ((long long)ox * oy));
      double v[6] = {0, 0, 0, 0, 0, 0};
      if (p.per == 0) {
        tensor_at(X, Y, Z, dx, dy, dz, v);
      } else {
        axis_terms(X, p.nx, p.per & 1, p.images, tx);
        axis_terms(Y, p.ny, p.per & 2, p.images, ty);
        axis_terms(Z, p.nz, p.per & 4, p.images, tz);
        for (const auto& a : tz)
          for (const auto& b : ty)
            for (const auto& e : tx) {
              double t[6];
              signed_term(e.first, b.first, a.first, dx, dy, dz, dmax, t);
              const double w = e.second * b.second * a.second;
              for (int c = 0; c < 6; ++c) v[c] += w * t[c];
            }
      }
      for (int c = 0; c < 6; ++c) oct[(size_t)c * Noct + i] = v[c];
    }
  }
  return spectrum_from_octant(p, oct, out);
}

// Grid of a caller tensor along one axis: an open axis of n cells holds the offsets 1-n .. n-1
// at index X + n - 1 (2n - 1 entries); a periodic axis holds one period, offset X at index
// X mod n (n entries; the offsets taken as b for b <= n/2 and b - n above).
struct AxisGrid {
  int n = 1;
  bool per = false;
  int size() const { return per ? n : 2 * n - 1; }
  int index(int X) const { return per ? ((X % n) + n) % n : X + n - 1; }
  int offset(int g) const { return per ? (2 * g <= n ? g : g - n) : g - (n - 1); }
};

int octant_from_full(const gbd::Plan& p, const double* full, std::vector<double>& oct, double tol) {
  AxisGrid gx, gy, gz;
  gx.n = p.nx;
  gx.per = (p.per & 1) != 0;
  gy.n = p.ny;
  gy.per = (p.per & 2) != 0;
  gz.n = p.nz;
  gz.per = (p.per & 4) != 0;
  const size_t Gx = gx.size(), Gy = gy.size(), Gz = gz.size();
  auto at = [&](int c, int X, int Y, int Z) {
    return full[(((size_t)c * Gz + (size_t)gz.index(Z)) * Gy + (size_t)gy.index(Y)) * Gx + (size_t)gx.index(X)];
  };
  const int ox = p.ox, oy = p.oy, oz = p.oz;
  const long long Noct = (long long)ox * oy * oz;
  try {
    oct.resize((size_t)Noct * 6);
  } catch (...) {
    return -1;
  }
  const size_t total = (size_t)6 * Gz * Gy * Gx;
  double mx = 0.0;
  for (size_t i = 0; i < total; ++i) {
    if (!std::isfinite(full[i])) return 1;
    mx = std::fmax(mx, std::fabs(full[i]));
  }
  const double lim = tol * mx;
  for (int c = 0; c < 6; ++c) {
    for (size_t kz = 0; kz < Gz; ++kz)
      for (size_t ky = 0; ky < Gy; ++ky)
        for (size_t kx = 0; kx < Gx; ++kx) {
          const int X = gx.offset((int)kx), Y = gy.offset((int)ky), Z = gz.offset((int)kz);
          const double v = at(c, X, Y, Z);
          // the value at the mirrored offset, signed by the component's parities
          const double sgn = (X < 0 ? PARITY[c][0] : 1) * (Y < 0 ? PARITY[c][1] : 1) * (Z < 0 ? PARITY[c][2] : 1);
          if (std::fabs(v - sgn * at(c, std::abs(X), std::abs(Y), std::abs(Z))) > lim) return 1;
          // an odd component vanishes where its offset is its own mirror (0, or n/2 on a period)
          auto self_mirror = [](const AxisGrid& g, int O) { return O == 0 || (g.per && 2 * O == g.n); };
          if (((PARITY[c][0] < 0 && self_mirror(gx, X)) || (PARITY[c][1] < 0 && self_mirror(gy, Y)) ||
               (PARITY[c][2] < 0 && self_mirror(gz, Z))) &&
              std::fabs(v) > lim)
            return 1;
        }
    for (int Z = 0; Z < oz; ++Z)
      for (int Y = 0; Y < oy; ++Y)
        for (int X = 0; X < ox; ++X) oct[(size_t)c * Noct + ((size_t)Z * oy + Y) * ox + X] = at(c, X, Y, Z);
  }
  return 0;
}

bool spectrum_from_octant(const gbd::Plan& p, const std::vector<double>& oct, std::vector<double>& out) {
  // octant extents: n_d, or n_d / 2 + 1 along a periodic axis
  const int nx = p.ox, ny = p.oy, nz = p.oz;
  const long long Noct = (long long)nx * ny * nz;
  try {
    out.assign((size_t)6 * p.Kz * p.Ky * p.Hx, 0.0);
  } catch (...) {
    return false;
  }
  Fft1 fx(p.Px), fy(p.Py), fz(p.Pz);
  const double scale = 1.0 / ((double)p.Px * p.Py * p.Pz);
  const int ncomp = (p.nz == 1) ? 4 : 6;  // xz, yz vanish identically in a single-layer mesh
  for (int c = 0; c < ncomp; ++c) {
    const double* src = oct.data() + (size_t)c * Noct;
    // x: [Z][Y][X] -> A1 [Z][Y][kx]
    std::vector<double> A1((size_t)nz * ny * p.Hx);
#pragma omp parallel
    {
      std::vector<std::complex<double>> buf(p.Px);
#pragma omp for
      for (long long l = 0; l < (long long)nz * ny; ++l)
        line_transform(&fx, p.Px, nx, p.Hx, PARITY[c][0], src + l * nx, 1, A1.data() + l * p.Hx, 1, buf);
    }
    // y: A1 [Z][Y][kx] -> A2 [Z][ky][kx]
    std::vector<double> A2((size_t)nz * p.Ky * p.Hx);
#pragma omp parallel
    {
      std::vector<std::complex<double>> buf(p.Py);
#pragma omp for
      for (long long l = 0; l < (long long)nz * p.Hx; ++l) {
        const long long Z = l / p.Hx, kx = l % p.Hx;
        line_transform(&fy, p.Py, ny, p.Ky, PARITY[c][1], A1.data() + Z * ny * p.Hx + kx, p.Hx,
                       A2.data() + Z * p.Ky * p.Hx + kx, p.Hx, buf);
      }
    }
    A1.clear();
    A1.shrink_to_fit();
    // z: A2 [Z][ky][kx] -> out [kz][ky][kx], scaled and signed
    double* dst = out.data() + (size_t)c * p.Kz * p.Ky * p.Hx;
    const double sgn = (c < 3) ? -scale : scale;
    const long long plane = (long long)p.Ky * p.Hx;
#pragma omp parallel
    {
      std::vector<std::complex<double>> buf(p.Pz);
      std::vector<double> tmp(p.Kz);
#pragma omp for
      for (long long l = 0; l < plane; ++l) {
        line_transform(&fz, p.Pz, nz, p.Kz, PARITY[c][2], A2.data() + l, plane, tmp.data(), 1, buf);
        for (int kz = 0; kz < p.Kz; ++kz) dst[kz * plane + l] = sgn * tmp[kz];
      }
    }
  }
  return true;
}

}  // namespace gbdt
