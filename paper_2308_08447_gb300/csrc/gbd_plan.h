// Padded lengths and block shapes of one mesh's demag convolution.
#pragma once
#include <cstddef>
#include <vector>

namespace gbd {

// Largest supported padded length along any axis; it bounds the shared-memory lines
// (3 components x P complex values) and the twiddle table.
constexpr int kMaxPad = 4096;
constexpr int kMaxPadX = 8192;
// Transform lengths 3 * 2^k and 5 * 2^k with kernels (FP32): the half length Lx = Px / 2 of
// the x transform and the y length Py may take these values (gbd_mixed_row.cu,
// gbd_mixed_conv.cu); every other length is a power of two.
constexpr int kMixedLens[] = {96, 160, 192, 320, 384, 640, 768, 1280, 1536, 2560, 3072};

struct Plan {
  int nx = 0, ny = 0, nz = 0;
  long long N = 0;
  // Padded periods. Sec. II pads to 2n; any P_d >= 2 n_d - 1 gives the same cropped result.
  // The smallest power of two is taken, or, along open x and y axes of FP32 meshes, the
  // smallest of the lengths 3 * 2^k and 5 * 2^k in kMixedLens (2 Lx for x) when that is
  // smaller. Px >= 2 so that the half-length x transform exists; Py = 1 (Pz = 1) when
  // ny = 1 (nz = 1): no padding along a dimension of size 1.
  int Px = 0, Py = 0, Pz = 0;
  int Lx = 0, Hx = 0;   // Lx = Px / 2, Hx = Lx + 1 stored x frequencies
  int Ky = 0, Kz = 0;   // stored y / z kernel frequencies: P/2 + 1 (1 when P = 1)
  bool film = false;    // nz == 1: 3-pass path
  // periodic axes (bit 0 x, 1 y, 2 z): P_d = n_d, no padding, kernel summed over `images`
  // periodic images per side; the kernel octant then spans n_d/2 + 1 offsets along d
  int per = 0, images = 0;
  int ox = 0, oy = 0, oz = 0;   // kernel octant extents (n_d when not periodic)
  // tile variants (0 / 1) per kernel family, set by the autotuner, and the block shapes
  // they give; the x rows also have variant 2, the persistent pipelined kernel (FP32)
  int var_row = 1, var_film = 0, var_y = 0, var_z = 0;
  int var_row_io = 1;   // x-row variant of the transform-only launches (forward, inverse to H_d)
  // arithmetic of the radix-16 FFT stages: 0 FP32, 1 split BF16 on the tensor cores
  int prec = 0;
  int RB = 1;           // rows per x-row block
  int Cf = 1;           // columns per film-conv block
  int Cy = 1;           // lines per y-pass block
  int Wz = 1;           // columns per z-conv block
  // device bytes of each buffer
  size_t bytes_S = 0, bytes_T = 0, bytes_K = 0, bytes_state = 0, bytes_tw = 0;
  size_t total_bytes() const { return bytes_S + bytes_T + bytes_K + bytes_state + bytes_tw; }
};

// Fills p from the mesh size and periodic axes; returns false (with a message) when the mesh
// is out of range.
// mixed: the x and y lengths may be 3 * 2^k or 5 * 2^k (kMixedLens).
bool make_plan(int nx, int ny, int nz, int per, bool mixed, Plan& p, const char** why);

}  // namespace gbd

namespace gbdt {
void newell_closed_form(double X, double Y, double Z, double dx, double dy, double dz, double out[6]);
void dipole_quadrature(double X, double Y, double Z, double dx, double dy, double dz, int G, double out[6]);
void tensor_at(int X, int Y, int Z, double dx, double dy, double dz, double out[6]);
bool kernel_spectrum(const gbd::Plan& p, double dx, double dy, double dz, std::vector<double>& out);
// Packed spectrum from the octant X, Y, Z >= 0 of the six components, layout [6][nz][ny][nx].
bool spectrum_from_octant(const gbd::Plan& p, const std::vector<double>& oct, std::vector<double>& out);
// Octant of a caller tensor [6][Gz][Gy][Gx] (G_d = 2 n_d - 1 on an open axis, n_d on a periodic
// one) after checking that the values are finite and have the tensor's parities within tol times
// the largest magnitude of all components.
// Returns 0, 1 (not finite or not symmetric) or -1 (allocation failure).
int octant_from_full(const gbd::Plan& p, const double* full, std::vector<double>& oct, double tol);
}  // namespace gbdt
