/*
 * gbdemag -- demagnetizing-field FFT convolution and exchange + LLG/RK4 time stepping
 * for finite-difference micromagnetics on one GB300 (sm_103a).
 *
 * The operation (Lepadatu, "Accelerating micromagnetic and atomistic simulations using
 * multiple GPUs", Sec. II, Eq. 1):  H_d,i = - sum_j N(i - j) M_j  over all cells j of an
 * nx x ny x nz mesh of identical rectangular cells, with N the cell-averaged demagnetizing
 * tensor. It is evaluated as a zero-padded FFT convolution (Sec. II; the single-GPU steps
 * of Appendix A): pad M to (2nx, 2ny, 2nz) -- no padding along a dimension of size 1 --,
 * x real-to-complex FFT, y and z FFTs, pointwise product with the transformed tensor stored
 * as its 6 real symmetry-packed components, inverse FFTs, crop. The time integrator adds
 * the exchange field H_ex = 2A/(mu0 Ms) lap(m) (Sec. III, Eq. 4) and a uniform applied
 * field, and advances the LLG equation (Eq. 5) with classic RK4 (Sec. III), recomputing
 * the demag field at every stage.
 *
 * Conventions
 *   - Units are SI: metres, A/m, J/m, seconds; mu0 = 4 pi 1e-7.
 *   - Field arrays are float32, planar ("SoA"), shape [3][nz][ny][nx] (x fastest),
 *     components (x, y, z). M and H_d are in A/m; m is the unit magnetization M / Ms.
 *   - Device pointers are CUDA device (or managed) addresses on the current device, at
 *     least 4-byte aligned, owned by the caller. The library never frees them.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Compute calls only enqueue
 *     work on it and return; results are ready when the stream has reached them.
 *   - Every call returns a gbd_status. No call aborts, throws or prints. On failure
 *     gbd_last_error() gives a message (per calling thread). Argument errors are detected
 *     before any work is enqueued. A CUDA error raised by enqueued work surfaces as
 *     GBD_ECUDA from a later call on the same device (CUDA errors are sticky).
 *   - Boundaries are free unless an axis is made periodic (GBD_FLAG_PBC_*): the exchange
 *     Laplacian replaces a missing neighbour by the cell itself (Neumann).
 */
#ifndef GBDEMAG_H
#define GBDEMAG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GBD_OK = 0,
  GBD_EINVAL = 1,       /* bad argument: sizes, cell, material, NULL or misaligned pointer */
  GBD_ENOMEM = 2,       /* device or host allocation failed */
  GBD_ECUDA = 3,        /* a CUDA call failed (launch error, sticky fault, wrong device) */
  GBD_ESTATE = 4,       /* call order: e.g. gbd_demag before gbd_set_kernel */
  GBD_ETIMEOUT = 5,     /* a bounded device-side wait gave up (gbd_mesh_device_status) */
  GBD_EBUDGET = 6,      /* admission refused: the request does not fit the memory budget */
  GBD_EUNSUPPORTED = 7  /* mesh size or transform length without a kernel, or a call the mesh cannot take */
} gbd_status;

/* Arithmetic of the FFT stages (Sec. II on halving the transfer precision only after
 * normalization, applied here to the DFT stages). GBD_FP32 (default): every stage in FP32. GBD_SPLIT_BF16:
 * every radix-16 DFT stage runs on the tensor cores as dense products of two-term BF16
 * operands (hi + lo, three products, FP32 accumulation); twiddles, smaller radices, the
 * kernel product and the LLG update stay FP32; stated error bound e_inf <= 1e-4 on H_d.
 * GBD_SPLIT_FP16: the same with FP16 halves, each butterfly's inputs first scaled by a power
 * of two into [0.5, 1) (FP16's range) and its outputs scaled back; stated bound e_inf <= 1e-5.
 * Any other value: GBD_EINVAL. */
typedef enum { GBD_FP32 = 0, GBD_SPLIT_BF16 = 1, GBD_SPLIT_FP16 = 2 } gbd_precision;

/* Mesh and material. Sizes: 1 <= nx <= 4096, 1 <= ny <= 2048, 1 <= nz <= 2048. */
typedef struct {
  int nx, ny, nz;        /* cells along x, y, z */
  double dx, dy, dz;     /* cell size, m (> 0) */
  double Ms;             /* saturation magnetization, A/m (> 0) */
  double A_ex;           /* exchange stiffness, J/m (>= 0; Eq. 4) */
  double alpha;          /* Gilbert damping (>= 0; Eq. 5) */
  double gamma;          /* gyromagnetic ratio mu0*gamma_e, m/(A s); 0 selects 2.212761569e5 */
  double Hext[3];        /* uniform applied (Zeeman) field, A/m */
  int precision;         /* gbd_precision */
  unsigned flags;        /* GBD_FLAG_PBC_* and GBD_FLAG_POW2_PAD bits (0: open boundaries, shortest padding) */
  int pbc_images;        /* periodic images per side along each periodic axis (>= 1 with one) */
} gbd_mesh_desc;

/* Periodic boundary conditions (Sec. II: a modified kernel and no zero padding along the
 * periodic direction). Along a periodic axis d the magnetization repeats with period n_d, which
 * must be a power of two (n_x >= 2 for x): the convolution along d is circular of length n_d, the
 * kernel is the demag tensor summed over pbc_images images on each side (at the half-period
 * offset the +n_d/2 and -n_d/2 image sets are averaged, so every component keeps its parity),
 * and the exchange Laplacian wraps around. Images beyond 256 cell sizes enter as point dipoles.
 * The kernel set-up costs about octant * (2 pbc_images + 1)^(periodic axes) tensor terms on
 * the host. gbd_set_kernel_tensor takes a caller tensor on one period along periodic axes. */
#define GBD_FLAG_PBC_X 1u
#define GBD_FLAG_PBC_Y 2u
#define GBD_FLAG_PBC_Z 4u
/* Padded lengths (Sec. II pads each open axis to 2n; any length >= 2n - 1 gives the same
 * cropped result). By default an FP32 mesh pads x and y to the smallest length >= 2n - 1 among
 * the powers of two and the lengths 3 * 2^k, 5 * 2^k that have kernels (x: 2 Lx with
 * Lx in {96, 160, 192, 320, 384, 640, 768, 1280, 1536, 2560, 3072}; y: those values), which
 * is up to 37.5 % shorter per axis than the next power of two; z, periodic axes and the split
 * precisions use powers of two. GBD_FLAG_POW2_PAD forces powers of two on every axis. */
#define GBD_FLAG_POW2_PAD 8u

typedef struct gbd_mesh gbd_mesh; /* opaque: plan, kernel spectrum, scratch, RK4 state */

/* Validates desc, plans the padded lengths (>= 2n - 1, see GBD_FLAG_POW2_PAD; 1 where n = 1;
 * n along a periodic axis) and
 * allocates the mesh's device buffers on the current device: x spectrum, 3D y spectrum,
 * kernel spectrum, RK4 scratch, twiddle table. *out receives the mesh (NULL on failure).
 * Errors: GBD_EINVAL, GBD_EUNSUPPORTED, GBD_ENOMEM, GBD_ECUDA. On any error every buffer
 * allocated so far is freed. Test hook: with the environment variable GBD_TEST_FAIL_ALLOC=k
 * (read at each call) the k-th of these device allocations fails as out-of-memory. */
gbd_status gbd_mesh_create(const gbd_mesh_desc* desc, gbd_mesh** out);

/* Device bytes gbd_mesh_create would allocate for desc (for admission control). Host only. */
gbd_status gbd_mesh_bytes(const gbd_mesh_desc* desc, size_t* out);

/* Computes the demag tensor (Eq. 1) in FP64 on the host -- closed-form Newell stencil in
 * the near field, Gauss-Legendre cell-pair quadrature beyond 8 cell sizes --, transforms
 * it in FP64, folds in -1/(Px Py Pz), packs the stored quadrant (Appendix A's convolution
 * kernel, (nx+1)(ny+1)(nz+1)-sized up to padding) and copies it to the device in FP32.
 * Blocks until the copy is done. Must precede the compute calls. The packed FP32 spectrum is
 * kept in a process-wide host cache keyed by (nx, ny, nz, dx, dy, dz), so another mesh of
 * the same geometry only pays the copy; least recently used entries are dropped beyond
 * GBD_KERNEL_CACHE_BYTES (environment variable, default 4 GiB). */
gbd_status gbd_set_kernel(gbd_mesh* mesh, void* stream);

/* Like gbd_set_kernel, but with the caller's FP64 tensor instead of the built-in one (Eq. 1
 * holds for any interaction tensor with the demag tensor's symmetries, e.g. one summed over
 * periodic images or a dipole-dipole kernel). N6: host array [6][Gz][Gy][Gx] of
 * (xx, yy, zz, xy, xz, yz), element (X, Y, Z) at index ((c Gz + gz(Z)) Gy + gy(Y)) Gx + gx(X);
 * read only during the call. Along an open axis of n cells G = 2n - 1 and g(X) = X + n - 1 for
 * offsets |X| < n. Along a periodic axis (GBD_FLAG_PBC_*) G = n and g(X) = X mod n: one period
 * of the (image-summed) tensor, for offsets 0 .. n - 1 (equivalently -n/2 < X <= n/2).
 * Each component must be finite and have the parities of the demag tensor (xx, yy, zz even in
 * X, Y, Z; xy odd in X and Y; xz odd in X and Z; yz odd in Y and Z; on a period the mirror of
 * X is n - X, so an odd component vanishes at X = n/2), to within GBD_TENSOR_SYM_TOL times the
 * largest magnitude in N6; otherwise GBD_EINVAL and nothing changes.
 * Only the octant X, Y, Z >= 0 is then used. The result is not put into the host cache.
 * Blocks until the copy is done. */
#define GBD_TENSOR_SYM_TOL 1e-9
gbd_status gbd_set_kernel_tensor(gbd_mesh* mesh, const double* N6, void* stream);

/* H = H_d(M) of Eq. 1. M, H: device [3][nz][ny][nx] float32, A/m; M and H must not overlap. */
gbd_status gbd_demag(gbd_mesh* mesh, const float* M, float* H, void* stream);

/* H = Ms * H_d(m) + H_ex(m) + Hext (Sec. III: H_eff without anisotropy). m: unit vectors. */
gbd_status gbd_effective_field(gbd_mesh* mesh, const float* m, float* H, void* stream);

/* dmdt = -gamma/(1+alpha^2) [m x H_eff + alpha m x (m x H_eff)] (Eq. 5 solved for dm/dt). */
gbd_status gbd_llg_rhs(gbd_mesh* mesh, const float* m, float* dmdt, void* stream);

/* Advances m in place by nsteps classic RK4 steps of size dt (s > 0): four demag + exchange
 * + LLG evaluations per step, stage inputs not renormalized, m renormalized at the end of
 * each step. m: device [3][nz][ny][nx] float32 unit vectors. nsteps = 0 is a no-op. */
gbd_status gbd_llg_step(gbd_mesh* mesh, float* m, int nsteps, double dt, void* stream);

/* gbd_llg_step with options. flags = 0 is gbd_llg_step.
 * GBD_STEP_EXTRAP: demag extrapolation at RK4 sub-steps (Sec. III: one demag evaluation per
 *   step, the other stages from a quartic polynomial in time). The demag field is evaluated at
 *   the first stage of each step and kept in a five-entry history; once the history holds the
 *   four previous step starts, stages 2 and 3 (t + dt/2) and 4 (t + dt) take the Lagrange
 *   quartic through the last five step-start fields instead of an evaluation (exchange and
 *   Zeeman fields are still evaluated). The first four steps of a run evaluate every stage.
 *   The mesh allocates the history (60 bytes per cell, not counted by gbd_mesh_bytes) on the
 *   first such call; GBD_ENOMEM if it cannot.
 * GBD_STEP_CONTINUE (with GBD_STEP_EXTRAP): keep the history of the previous call, so no new
 *   start-up; valid only when m is that call's result, unchanged, and dt is the same (a
 *   different dt restarts the history). Without it every call starts a new history.
 * Other bits: GBD_EINVAL. */
/* Adaptive RKF5(6) stepping (Sec. III names the Runge-Kutta-Fehlberg 5th-order method with
 * 6th-order error estimation; its tableau is not in the paper): Fehlberg's eight-stage RK5(6)
 * pair. A step evaluates eight demag + exchange + LLG slopes k_i at the stage states
 * m + dt sum_j a_ij k_j, takes the fifth-order result m + dt sum_i b5_i k_i (renormalized per
 * cell) and the error estimate err = dt max_cells |sum_i (b6_i - b5_i) k_i|.
 * gbd_llg_rkf56_step: one step of size dt (> 0), always kept; *err receives the estimate.
 * gbd_llg_run_rkf56: integrates from 0 to t_end (>= 0) starting with step *dt (> 0), accepting a
 * step when err <= tol (> 0) and retrying otherwise, with the next size
 * h min(5, max(0.2, 0.9 (tol/err)^(1/6))); the last step ends exactly at t_end. Stops early
 * after max_steps (>= 1) attempts. On return *dt holds the next proposed size and
 * *accepted / *rejected (either may be NULL) the step counts. Both calls wait for the stream
 * after every step (the next size depends on the error); the first call allocates the stage
 * buffers (108 bytes per cell). m: device [3][nz][ny][nx] unit vectors, in/out. */
/* flags (both calls): GBD_STEP_EXTRAP extrapolates the demag field at stages 2-8 (Sec. III: a
 * quintic for RKF56, one demag evaluation per step): once five accepted step starts are
 * recorded, a stage at time t + c_i dt takes the Lagrange quintic through this step's stage-1
 * field and those five at their actual (unequal) times; exchange and Zeeman fields are still
 * evaluated. GBD_STEP_CONTINUE keeps the recorded history of the previous call (m must be its
 * result, unchanged). The history costs another 72 bytes per cell. */
gbd_status gbd_llg_rkf56_step(gbd_mesh* mesh, float* m, double dt, double* err, unsigned flags, void* stream);
gbd_status gbd_llg_run_rkf56(gbd_mesh* mesh, float* m, double t_end, double* dt, double tol, int max_steps,
                             int* accepted, int* rejected, unsigned flags, void* stream);

#define GBD_STEP_EXTRAP 1u
#define GBD_STEP_CONTINUE 2u
gbd_status gbd_llg_step_ex(gbd_mesh* mesh, float* m, int nsteps, double dt, unsigned flags, void* stream);

/* Changes the applied (Zeeman) field, A/m, and the damping of later calls on the mesh: a
 * time-dependent field, or relaxation with a larger alpha between dynamics runs. Hext NULL
 * keeps the field; alpha < 0 keeps the damping. Work already enqueued is unaffected; a batch
 * re-captures its graph on its next run. GBD_EINVAL for non-finite values. */
gbd_status gbd_mesh_set_params(gbd_mesh* mesh, const double Hext[3], double alpha);

/* Checkpoint / resume of the integrator state that lives in the mesh (no counterpart in the
 * paper): the demag-extrapolation histories of gbd_llg_step_ex (GBD_STEP_EXTRAP) and of the
 * RKF5(6) calls, with their ring positions and step times. m itself is the caller's array.
 * gbd_mesh_state_bytes gives the size of the host image (a header plus 5 resp. 6 slots of
 * [3][nz][ny][nx] float32 for each history the mesh has allocated). gbd_mesh_get_state waits
 * for stream, then copies the state into host (bytes >= that size, else GBD_EINVAL).
 * gbd_mesh_set_state waits for stream and replaces the mesh's state by an image from a mesh
 * of the same shape (nx, ny, nz) and periodic axes (GBD_EINVAL for a malformed or foreign
 * image, which changes nothing; a CUDA error while copying returns GBD_ECUDA and discards the
 * mesh's histories, so the next extrapolated call starts them afresh); a following call with GBD_STEP_CONTINUE resumes exactly where the saved mesh
 * stood, so a run split by get/set (even across processes) equals the unsplit run bit for
 * bit. Both block the host. */
gbd_status gbd_mesh_state_bytes(const gbd_mesh* mesh, size_t* out);
gbd_status gbd_mesh_get_state(gbd_mesh* mesh, void* host, size_t bytes, void* stream);
gbd_status gbd_mesh_set_state(gbd_mesh* mesh, const void* host, size_t bytes, void* stream);

/* ---- allocation-free demag --------------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot call
 * cudaMalloc at the moment they need the field -- for example code embedded in a host
 * application that owns every device allocation through its own pool, or code at a memory
 * cap where an allocation (and the device synchronisation it can imply) is not acceptable.
 *
 * gbd_demag_noalloc computes exactly what gbd_demag computes, H = H_d(M), with the same
 * kernels, but its scratch (the x spectrum and, for 3D meshes, the y spectrum) lives in a
 * fixed device array compiled into the library instead of the mesh's buffers, and the call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine). The mesh still
 * supplies its kernel spectrum and twiddle table (set up earlier by gbd_mesh_create and
 * gbd_set_kernel); M and H are the caller's, as for gbd_demag.
 *   - Limit: the scratch needed, x spectrum (3*nz*(Px/2+1)*ny complex64, rounded up to 256
 *     bytes) plus y spectrum (3*nz*(Px/2+1)*Py complex64 when nz > 1 and ny > 1), must not
 *     exceed GBD_NOALLOC_MAX_BYTES; a larger mesh is refused with GBD_EBUDGET before any
 *     work is enqueued. Every GPU that loads the library holds this array until exit.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 *     with that device current) and caches it; with lazy module loading that lookup may also
 *     load the library's device code, and with it the array, onto the device.
 *   - All calls on a device share the one array, which keeps the last call's contents. Each
 *     call writes every scratch element before reading it, so nothing needs clearing; but
 *     calls whose work overlaps on the GPU (different streams, other meshes) race on it and
 *     must be ordered by the caller.
 * Errors: as gbd_demag, plus GBD_EBUDGET (mesh too large for the static scratch). */
#define GBD_NOALLOC_MAX_BYTES (64u << 20)
gbd_status gbd_demag_noalloc(gbd_mesh* mesh, const float* M, float* H, void* stream);

/* Frees the mesh's device buffers without waiting: the frees are stream-ordered (the device's
 * memory pool, cudaFreeAsync) after the last work each stream was given for this mesh by the
 * calls above and by batch runs, so other work on the device is not stalled and the host
 * returns at once. Work that the caller captured into its own CUDA graphs must have finished
 * before this call. The mesh's buffers come from the same pool (cudaMallocAsync). NULL is
 * accepted. */
gbd_status gbd_mesh_destroy(gbd_mesh* mesh);

/* Status of the mesh's kernels on the device. The RK-stage x-row kernels wait for bulk copies
 * of their stage input (TMA, completed through an mbarrier); a block that has waited
 * 100 ms of the GPU's clock gives up, ORs a flag into the mesh's device status word and carries
 * on with what the copy has delivered, so no launch can hang and the context stays usable, but
 * the results of the steps since the last check are not to be trusted. This call reads the
 * word after the work queued on `stream` (NULL: the legacy default stream) so far, waits for
 * it on the host, clears it, and returns GBD_ETIMEOUT if a wait gave up, else GBD_OK. The
 * test hook GBD_TEST_WAIT_TIMEOUT=1 in the environment when a mesh is created makes its staged
 * copies announce 16 bytes more than they deliver, so every such wait runs out.
 * Errors: GBD_EINVAL (NULL mesh), GBD_ECUDA. */
gbd_status gbd_mesh_device_status(gbd_mesh* mesh, void* stream);

/* Message of the calling thread's last failure ("" if none). Valid until its next call. */
const char* gbd_last_error(void);

/* ---- tile-shape autotuning ---------------------------------------------------------------
 * Every kernel family has two tile shapes (lines of the transform per thread block); the x-row
 * pass has two more variants for FP32 meshes, 2 and 3: a persistent kernel that copies the next
 * row group's inputs into shared memory (cp.async) while it transforms the current group -- in
 * RK stages variant 2 stages the spectrum tile and the field rows (one block per SM), variant 3
 * the spectrum tile only (two blocks per SM; nx a multiple of 64); transform-only launches stage
 * their input (two blocks per SM). They are used where they apply (x transform length Px/2 in
 * [64, 2048], open x axis, nx a multiple of 4, ny a multiple of the group's rows, the staged
 * fields 16-byte aligned; otherwise variant 1 runs). A new mesh starts with variant 1. All variants give identical
 * results -- each line's FFT and each cell's update do not depend on how lines are grouped --
 * and differ only in speed, which depends on the mesh size. gbd_mesh_autotune times the
 * variants of each pass this mesh uses (on its own buffers, which it zeroes; the stream is
 * synchronized) and keeps the fastest; results are cached per (nx, ny, nz, device) in the
 * process and, when the environment variable GBD_AUTOTUNE_CACHE names a file, in that text
 * file. Requires gbd_set_kernel. Variants (row, film, y, z): row 0 to 3, the others 0 or 1.
 * The autotuner also chooses the padded lengths: a mesh planned with a 3 * 2^k or 5 * 2^k
 * length (see GBD_FLAG_POW2_PAD) is timed against the same mesh on power-of-two lengths (a
 * scratch twin with its own tuned tiles), and moves onto the power-of-two plan when that is
 * more than 2 % faster: new spectrum buffers, the kernel spectrum recomputed for the new
 * lengths (the cropped result is the same, Sec. II), GBD_FLAG_POW2_PAD then set in its
 * description. gbd_mesh_plan_dims gives the lengths a mesh uses. */
gbd_status gbd_mesh_autotune(gbd_mesh* mesh, void* stream);
gbd_status gbd_mesh_get_tuning(const gbd_mesh* mesh, int out[4]);
gbd_status gbd_mesh_set_tuning(gbd_mesh* mesh, const int in[4]);
/* The plan a mesh uses now: out = {Px, Py, Pz, Hx, Ky, Kz}, as gbd_plan_dims. */
gbd_status gbd_mesh_plan_dims(const gbd_mesh* mesh, int out[6]);

/* ---- batched meshes ------------------------------------------------------------------------
 * A batch advances many independent meshes (uneven sizes allowed) with one CUDA-graph launch
 * per run: each mesh's gbd_llg_step launch sequence is a chain on one of up to 32 branch
 * streams, captured into one graph behind a fork on `stream` and joined back into it, so
 * kernels of different meshes run concurrently. The instantiated graph is cached with the
 * run's arguments and relaunched while they repeat. Each mesh's result is bit-identical to
 * gbd_llg_step on that mesh alone. */
typedef struct gbd_batch gbd_batch;

/* meshes: count >= 1 distinct meshes on the current device, each after gbd_set_kernel; the
 * batch keeps the pointers (the meshes must outlive it). */
gbd_status gbd_batch_create(gbd_mesh* const* meshes, int count, gbd_batch** out);

/* Advances mesh i's state m[i] (device, [3][nz][ny][nx] unit vectors, in place) by nsteps[i]
 * RK4 steps of size dt[i] (nsteps[i] = 0 leaves it untouched). Enqueue-only on `stream`. Two
 * runs of one batch must not overlap on the GPU (they share the meshes' scratch).
 * Errors: GBD_EINVAL (NULL / misaligned pointer, nsteps < 0, dt <= 0), GBD_ECUDA. */
gbd_status gbd_batch_run(gbd_batch* batch, float* const* m, const int* nsteps, const double* dt, void* stream);

/* gbd_batch_run with per-mesh gbd_llg_step_ex flags (NULL: all 0). With GBD_STEP_EXTRAP a
 * mesh's history advances as in gbd_llg_step_ex; the cached graph is reused while every mesh's
 * arguments, flags and history state (ring position, fill, dt) repeat, which for a continued
 * run (GBD_STEP_CONTINUE) holds once the history is full and nsteps is a multiple of 5 (the
 * ring's length); otherwise the run is captured again. Each mesh's result is bit-identical to
 * gbd_llg_step_ex on that mesh alone with the same flags. */
gbd_status gbd_batch_run_ex(gbd_batch* batch, float* const* m, const int* nsteps, const double* dt,
                            const unsigned* flags, void* stream);

/* Waits for the batch's last graph launch (not the rest of the device) and frees the batch
 * (not the meshes). NULL is accepted. */
gbd_status gbd_batch_destroy(gbd_batch* batch);

/* ---- per-pass timing ------------------------------------------------------------------- */

/* Pass classes reported by gbd_mesh_read_timing. */
enum {
  GBD_PASS_ROW_FWD = 0,    /* x real-to-complex of an input field */
  GBD_PASS_ROW_INV = 1,    /* x complex-to-real + crop with a field / dm/dt epilogue */
  GBD_PASS_ROW_RK = 2,     /* x complex-to-real + exchange + LLG + RK4 stage (+ next forward) */
  GBD_PASS_FILM_CONV = 3,  /* y FFT -> kernel product -> y IFFT (nz = 1) */
  GBD_PASS_Y_FWD = 4,      /* 3D y FFT */
  GBD_PASS_Z_CONV = 5,     /* 3D z FFT -> kernel product -> z IFFT */
  GBD_PASS_Y_INV = 6,      /* 3D y IFFT + crop */
  GBD_PASS_EXTRAP = 7,     /* extrapolated RK4 stage without a transform (GBD_STEP_EXTRAP) */
  GBD_NPASS = 8
};

/* Tracing of this mesh's later launches (profiling only). enable = 0: off. GBD_TIMING_EVENTS
 * (also any other nonzero value without the NVTX bit): every launch is bracketed by two CUDA
 * events on its stream (it adds event records between launches), read by
 * gbd_mesh_read_timing. GBD_TIMING_NVTX: every launch's enqueue is wrapped in an NVTX range
 * named after its pass class ("row_fwd", "row_inv", "row_rk", "film_conv", "y_fwd", "z_conv",
 * "y_inv", "extrap_stage"), for profilers that filter kernels by NVTX range; the two combine.
 * Batched runs (gbd_batch_run*) are not traced. */
#define GBD_TIMING_EVENTS 1
#define GBD_TIMING_NVTX 2
gbd_status gbd_mesh_set_timing(gbd_mesh* mesh, int enable);

/* Waits for the recorded events, writes per pass class the summed device time in ms and
 * the launch count (arrays of GBD_NPASS), and clears the record. */
gbd_status gbd_mesh_read_timing(gbd_mesh* mesh, double* ms, long long* launches);

/* ---- host-only helpers (no GPU needed) ------------------------------------------------ */

/* The FP64 tensor components (xx, yy, zz, xy, xz, yz) at integer cell offset (X, Y, Z). */
gbd_status gbd_tensor_at(const gbd_mesh_desc* desc, int X, int Y, int Z, double out[6]);

/* Plan of desc: out = {Px, Py, Pz, Hx, Ky, Kz} with Hx = Px/2+1 and K_d = P_d/2+1 (1 if P_d = 1). */
gbd_status gbd_plan_dims(const gbd_mesh_desc* desc, int out[6]);

/* The FP64 packed kernel spectrum that gbd_set_kernel uploads (before rounding to FP32),
 * layout [6][Kz][Ky][Hx]; count must equal 6*Kz*Ky*Hx. Components xz, yz are zero when nz = 1. */
gbd_status gbd_kernel_spectrum_host(const gbd_mesh_desc* desc, double* out, size_t count);

/* The FP64 packed spectrum that gbd_set_kernel_tensor would upload for the caller tensor N6
 * (layout and checks as there), layout [6][Kz][Ky][Hx]; count must equal 6*Kz*Ky*Hx. */
gbd_status gbd_kernel_spectrum_from_tensor_host(const gbd_mesh_desc* desc, const double* N6, double* out,
                                                size_t count);

#ifdef __cplusplus
}
#endif

#endif /* GBDEMAG_H */
