"""Python binding of libgbdemag.so (the C ABI declared in include/gbdemag.h).

Argument marshalling only: every step of the demag convolution and of the LLG/RK4
update runs in the library's CUDA kernels. PyTorch supplies device memory and
streams: field arguments are contiguous float32 CUDA tensors of shape
(3, nz, ny, nx), and ``stream`` defaults to torch's current stream.

There is no fallback: if the shared library has not been built, ``load()`` raises.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgbdemag.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "gbdemag.h")

GBD_OK, GBD_EINVAL, GBD_ENOMEM, GBD_ECUDA, GBD_ESTATE, GBD_ETIMEOUT, GBD_EBUDGET, GBD_EUNSUPPORTED = range(8)
STATUS_NAMES = {0: "GBD_OK", 1: "GBD_EINVAL", 2: "GBD_ENOMEM", 3: "GBD_ECUDA", 4: "GBD_ESTATE",
                5: "GBD_ETIMEOUT", 6: "GBD_EBUDGET", 7: "GBD_EUNSUPPORTED"}
GBD_FP32, GBD_SPLIT_BF16, GBD_SPLIT_FP16 = 0, 1, 2


class GbdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class gbd_mesh_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("Ms", ctypes.c_double), ("A_ex", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gamma", ctypes.c_double), ("Hext", ctypes.c_double * 3),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint), ("pbc_images", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIG = {
    "gbd_mesh_create": [ctypes.POINTER(gbd_mesh_desc), ctypes.POINTER(_P)],
    "gbd_mesh_bytes": [ctypes.POINTER(gbd_mesh_desc), ctypes.POINTER(ctypes.c_size_t)],
    "gbd_set_kernel": [_P, _P],
    "gbd_set_kernel_tensor": [_P, ctypes.POINTER(_D), _P],
    "gbd_demag": [_P, _P, _P, _P],
    "gbd_effective_field": [_P, _P, _P, _P],
    "gbd_llg_rhs": [_P, _P, _P, _P],
    "gbd_llg_step": [_P, _P, _I, _D, _P],
    "gbd_llg_step_ex": [_P, _P, _I, _D, ctypes.c_uint, _P],
    "gbd_mesh_set_params": [_P, ctypes.POINTER(_D), _D],
    "gbd_mesh_state_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "gbd_mesh_get_state": [_P, _P, ctypes.c_size_t, _P],
    "gbd_mesh_set_state": [_P, _P, ctypes.c_size_t, _P],
    "gbd_llg_rkf56_step": [_P, _P, _D, ctypes.POINTER(_D), ctypes.c_uint, _P],
    "gbd_llg_run_rkf56": [_P, _P, _D, ctypes.POINTER(_D), _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.c_uint,
                          _P],
    "gbd_mesh_destroy": [_P],
    "gbd_mesh_device_status": [_P, _P],
    "gbd_tensor_at": [ctypes.POINTER(gbd_mesh_desc), _I, _I, _I, ctypes.POINTER(_D)],
    "gbd_plan_dims": [ctypes.POINTER(gbd_mesh_desc), ctypes.POINTER(_I)],
    "gbd_kernel_spectrum_host": [ctypes.POINTER(gbd_mesh_desc), ctypes.POINTER(_D), ctypes.c_size_t],
    "gbd_kernel_spectrum_from_tensor_host": [ctypes.POINTER(gbd_mesh_desc), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                             ctypes.c_size_t],
    "gbd_demag_noalloc": [_P, _P, _P, _P],
    "gbd_mesh_autotune": [_P, _P],
    "gbd_mesh_plan_dims": [_P, ctypes.POINTER(_I)],
    "gbd_mesh_get_tuning": [_P, ctypes.POINTER(_I)],
    "gbd_mesh_set_tuning": [_P, ctypes.POINTER(_I)],
    "gbd_batch_create": [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)],
    "gbd_batch_run": [_P, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_D), _P],
    "gbd_batch_run_ex": [_P, ctypes.POINTER(_P), ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_uint), _P],
    "gbd_batch_destroy": [_P],
    "gbd_mesh_set_timing": [_P, _I],
    "gbd_mesh_read_timing": [_P, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong)],
}
PASS_NAMES = ["row_fwd", "row_inv", "row_rk", "film_conv", "y_fwd", "z_conv", "y_inv", "extrap_stage"]
GBD_NPASS = 8


def load():
    """Loads the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgbdemag.so is not built: run `python -m paper_2308_08447_gb300.build` "
                          "(or __graft_entry__.build()); there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIG.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.gbd_last_error.argtypes = []
    lib.gbd_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def header_symbols():
    """Function names declared in include/gbdemag.h."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(gbd_[a-z_0-9]+)\s*\(", text)))


def _check(status):
    if status != GBD_OK:
        raise GbdError(status, load().gbd_last_error().decode())


GBD_FLAG_PBC_X, GBD_FLAG_PBC_Y, GBD_FLAG_PBC_Z, GBD_FLAG_POW2_PAD = 1, 2, 4, 8


def make_desc(n, cell, Ms, A_ex=0.0, alpha=0.0, gamma=0.0, Hext=(0.0, 0.0, 0.0), precision=GBD_FP32, pbc=(False,) * 3,
              pbc_images=0, pow2_pad=False):
    d = gbd_mesh_desc()
    d.nx, d.ny, d.nz = (int(v) for v in n)
    d.dx, d.dy, d.dz = (float(v) for v in cell)
    d.Ms, d.A_ex, d.alpha, d.gamma = float(Ms), float(A_ex), float(alpha), float(gamma)
    d.Hext[0], d.Hext[1], d.Hext[2] = (float(v) for v in Hext)
    d.precision = int(precision)
    d.flags = (GBD_FLAG_PBC_X if pbc[0] else 0) | (GBD_FLAG_PBC_Y if pbc[1] else 0) | (GBD_FLAG_PBC_Z if pbc[2] else 0)
    if pow2_pad:
        d.flags |= GBD_FLAG_POW2_PAD
    d.pbc_images = int(pbc_images)
    return d


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _field_ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


# ---- the C ABI, one Python function per entry point -----------------------------------------

def gbd_mesh_create(desc):
    h = ctypes.c_void_p()
    _check(load().gbd_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def gbd_mesh_bytes(desc):
    out = ctypes.c_size_t()
    _check(load().gbd_mesh_bytes(ctypes.byref(desc), ctypes.byref(out)))
    return out.value


def gbd_set_kernel(mesh, stream=None):
    _check(load().gbd_set_kernel(mesh, _stream_ptr(stream)))


def _tensor_arg(N6, n, pbc=(False,) * 3):
    """C-contiguous float64 copy of a caller tensor of shape (6, Gz, Gy, Gx): G = 2n - 1 along an
    open axis, n along a periodic one."""
    import numpy as np
    G = [n[d] if pbc[d] else 2 * n[d] - 1 for d in range(3)]
    want = (6, G[2], G[1], G[0])
    arr = np.ascontiguousarray(N6, dtype=np.float64)
    if arr.shape != want:
        raise ValueError("tensor shape %s != %s" % (arr.shape, want))
    return arr


def gbd_set_kernel_tensor(mesh, N6, n, stream=None, pbc=(False,) * 3):
    arr = _tensor_arg(N6, n, pbc)
    _check(load().gbd_set_kernel_tensor(mesh, arr.ctypes.data_as(ctypes.POINTER(_D)), _stream_ptr(stream)))


def gbd_demag(mesh, M, H, shape, stream=None):
    _check(load().gbd_demag(mesh, _field_ptr(M, shape, "M"), _field_ptr(H, shape, "H"), _stream_ptr(stream)))


def gbd_demag_noalloc(mesh, M, H, shape, stream=None):
    """H = H_d(M) like gbd_demag, with the scratch in the library's static device array
    (no allocation in the call; see include/gbdemag.h for the size limit and ordering)."""
    _check(load().gbd_demag_noalloc(mesh, _field_ptr(M, shape, "M"), _field_ptr(H, shape, "H"),
                                    _stream_ptr(stream)))


def gbd_effective_field(mesh, m, H, shape, stream=None):
    _check(load().gbd_effective_field(mesh, _field_ptr(m, shape, "m"), _field_ptr(H, shape, "H"),
                                      _stream_ptr(stream)))


def gbd_llg_rhs(mesh, m, dmdt, shape, stream=None):
    _check(load().gbd_llg_rhs(mesh, _field_ptr(m, shape, "m"), _field_ptr(dmdt, shape, "dmdt"),
                              _stream_ptr(stream)))


def gbd_llg_step(mesh, m, nsteps, dt, shape, stream=None):
    _check(load().gbd_llg_step(mesh, _field_ptr(m, shape, "m"), int(nsteps), float(dt), _stream_ptr(stream)))


GBD_STEP_EXTRAP = 1
GBD_STEP_CONTINUE = 2


def gbd_llg_step_ex(mesh, m, nsteps, dt, flags, shape, stream=None):
    _check(load().gbd_llg_step_ex(mesh, _field_ptr(m, shape, "m"), int(nsteps), float(dt), int(flags),
                                  _stream_ptr(stream)))


def gbd_mesh_set_params(mesh, Hext=None, alpha=None):
    h = None
    if Hext is not None:
        h = (_D * 3)(*(float(v) for v in Hext))
    _check(load().gbd_mesh_set_params(mesh, h, -1.0 if alpha is None else float(alpha)))


def gbd_mesh_get_state(mesh, stream=None):
    """The mesh's integrator state (extrapolation histories) as bytes (gbd_mesh_get_state)."""
    n = ctypes.c_size_t()
    _check(load().gbd_mesh_state_bytes(mesh, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(load().gbd_mesh_get_state(mesh, ctypes.cast(buf, _P), n.value, _stream_ptr(stream)))
    return buf.raw


def gbd_mesh_set_state(mesh, state, stream=None):
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(load().gbd_mesh_set_state(mesh, ctypes.cast(buf, _P), len(state), _stream_ptr(stream)))


def gbd_llg_rkf56_step(mesh, m, dt, shape, stream=None, flags=0):
    """One RKF5(6) step; returns the error estimate."""
    err = _D(0.0)
    _check(load().gbd_llg_rkf56_step(mesh, _field_ptr(m, shape, "m"), float(dt), ctypes.byref(err), int(flags),
                                     _stream_ptr(stream)))
    return err.value


def gbd_llg_run_rkf56(mesh, m, t_end, dt, tol, shape, max_steps=1000000, stream=None, flags=0):
    """Adaptive RKF5(6) from 0 to t_end; returns (next dt, accepted, rejected)."""
    d, acc, rej = _D(float(dt)), _I(0), _I(0)
    _check(load().gbd_llg_run_rkf56(mesh, _field_ptr(m, shape, "m"), float(t_end), ctypes.byref(d), float(tol),
                                    int(max_steps), ctypes.byref(acc), ctypes.byref(rej), int(flags),
                                    _stream_ptr(stream)))
    return d.value, acc.value, rej.value


def gbd_mesh_destroy(mesh):
    _check(load().gbd_mesh_destroy(mesh))


def gbd_mesh_device_status(mesh, stream=None):
    """GBD_OK, or GBD_ETIMEOUT when a kernel's bounded wait gave up since the last call (the
    word is cleared); other failures raise."""
    s = load().gbd_mesh_device_status(mesh, _stream_ptr(stream))
    if s not in (GBD_OK, GBD_ETIMEOUT):
        _check(s)
    return s


def gbd_mesh_autotune(mesh, stream=None):
    _check(load().gbd_mesh_autotune(mesh, _stream_ptr(stream)))


def gbd_mesh_get_tuning(mesh):
    out = (ctypes.c_int * 4)()
    _check(load().gbd_mesh_get_tuning(mesh, out))
    return tuple(out)


def gbd_mesh_set_tuning(mesh, variants):
    arr = (ctypes.c_int * 4)(*[int(v) for v in variants])
    _check(load().gbd_mesh_set_tuning(mesh, arr))


def gbd_batch_create(meshes):
    arr = (ctypes.c_void_p * len(meshes))(*[m.value if isinstance(m, ctypes.c_void_p) else m for m in meshes])
    out = ctypes.c_void_p()
    _check(load().gbd_batch_create(arr, len(meshes), ctypes.byref(out)))
    return out


def gbd_batch_run(batch, m_list, shapes, nsteps, dts, stream=None, flags=None):
    n = len(m_list)
    ptrs = (ctypes.c_void_p * n)(*[_field_ptr(t, s, "m[%d]" % i).value for i, (t, s) in enumerate(zip(m_list, shapes))])
    steps = (ctypes.c_int * n)(*[int(v) for v in nsteps])
    dt = (ctypes.c_double * n)(*[float(v) for v in dts])
    if flags is None:
        _check(load().gbd_batch_run(batch, ptrs, steps, dt, _stream_ptr(stream)))
    else:
        fl = (ctypes.c_uint * n)(*[int(v) for v in flags])
        _check(load().gbd_batch_run_ex(batch, ptrs, steps, dt, fl, _stream_ptr(stream)))


def gbd_batch_destroy(batch):
    _check(load().gbd_batch_destroy(batch))


GBD_TIMING_EVENTS, GBD_TIMING_NVTX = 1, 2


def gbd_mesh_set_timing(mesh, enable):
    """enable: False / True (CUDA events per launch) or GBD_TIMING_EVENTS | GBD_TIMING_NVTX bits."""
    flags = enable if isinstance(enable, int) and not isinstance(enable, bool) else (GBD_TIMING_EVENTS if enable else 0)
    _check(load().gbd_mesh_set_timing(mesh, int(flags)))


def gbd_mesh_read_timing(mesh):
    """{pass name: (total ms, launches)} since the last read."""
    ms = (ctypes.c_double * GBD_NPASS)()
    n = (ctypes.c_longlong * GBD_NPASS)()
    _check(load().gbd_mesh_read_timing(mesh, ms, n))
    return {PASS_NAMES[i]: (ms[i], n[i]) for i in range(GBD_NPASS) if n[i]}


def gbd_last_error():
    return load().gbd_last_error().decode()


def gbd_tensor_at(desc, X, Y, Z):
    out = (ctypes.c_double * 6)()
    _check(load().gbd_tensor_at(ctypes.byref(desc), int(X), int(Y), int(Z), out))
    return list(out)


def gbd_plan_dims(desc):
    out = (ctypes.c_int * 6)()
    _check(load().gbd_plan_dims(ctypes.byref(desc), out))
    return tuple(out)


def gbd_mesh_plan_dims(mesh):
    """(Px, Py, Pz, Hx, Ky, Kz) of the plan the mesh uses now (the autotuner may change it)."""
    out = (ctypes.c_int * 6)()
    _check(load().gbd_mesh_plan_dims(mesh, out))
    return tuple(out)


def gbd_kernel_spectrum_host(desc):
    import numpy as np
    Px, Py, Pz, Hx, Ky, Kz = gbd_plan_dims(desc)
    out = np.zeros((6, Kz, Ky, Hx), dtype=np.float64)
    _check(load().gbd_kernel_spectrum_host(ctypes.byref(desc), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           out.size))
    return out


def gbd_kernel_spectrum_from_tensor_host(desc, N6):
    import numpy as np
    Px, Py, Pz, Hx, Ky, Kz = gbd_plan_dims(desc)
    arr = _tensor_arg(N6, (desc.nx, desc.ny, desc.nz), tuple(bool(desc.flags >> d & 1) for d in range(3)))
    out = np.zeros((6, Kz, Ky, Hx), dtype=np.float64)
    _check(load().gbd_kernel_spectrum_from_tensor_host(ctypes.byref(desc), arr.ctypes.data_as(ctypes.POINTER(_D)),
                                                       out.ctypes.data_as(ctypes.POINTER(_D)), out.size))
    return out


# ---- convenience wrapper --------------------------------------------------------------------

class Mesh:
    """One mesh: owns the library handle; the kernel spectrum is computed on construction."""

    def __init__(self, n, cell, Ms, A_ex=0.0, alpha=0.0, gamma=0.0, Hext=(0.0, 0.0, 0.0),
                 precision=GBD_FP32, set_kernel=True, stream=None, pbc=(False,) * 3, pbc_images=0, pow2_pad=False):
        self.n = tuple(int(v) for v in n)
        self.pbc = tuple(bool(v) for v in pbc)
        self.shape = (3, self.n[2], self.n[1], self.n[0])
        self.desc = make_desc(n, cell, Ms, A_ex, alpha, gamma, Hext, precision, pbc, pbc_images, pow2_pad)
        self.handle = gbd_mesh_create(self.desc)
        if set_kernel:
            gbd_set_kernel(self.handle, stream)

    def set_kernel_tensor(self, N6, stream=None):
        """Replace the kernel by the caller's FP64 tensor, shape (6, Gz, Gy, Gx) with G = 2n - 1
        along open axes and n (one period, offset X at index X mod n) along periodic ones."""
        gbd_set_kernel_tensor(self.handle, N6, self.n, stream, self.pbc)

    def demag(self, M, H, stream=None):
        gbd_demag(self.handle, M, H, self.shape, stream)

    def effective_field(self, m, H, stream=None):
        gbd_effective_field(self.handle, m, H, self.shape, stream)

    def llg_rhs(self, m, dmdt, stream=None):
        gbd_llg_rhs(self.handle, m, dmdt, self.shape, stream)

    def llg_step(self, m, nsteps, dt, stream=None, extrap=False, cont=False):
        """nsteps RK4 steps; extrap: demag extrapolated at stages 2-4 (GBD_STEP_EXTRAP), cont:
        continue the previous call's demag history (GBD_STEP_CONTINUE)."""
        if not extrap and not cont:
            gbd_llg_step(self.handle, m, nsteps, dt, self.shape, stream)
        else:
            flags = (GBD_STEP_EXTRAP if extrap else 0) | (GBD_STEP_CONTINUE if cont else 0)
            gbd_llg_step_ex(self.handle, m, nsteps, dt, flags, self.shape, stream)

    def rkf56_step(self, m, dt, stream=None, extrap=False, cont=False):
        flags = (GBD_STEP_EXTRAP if extrap else 0) | (GBD_STEP_CONTINUE if cont else 0)
        return gbd_llg_rkf56_step(self.handle, m, dt, self.shape, stream, flags)

    def run_rkf56(self, m, t_end, dt, tol, max_steps=1000000, stream=None, extrap=False, cont=False):
        """Adaptive RKF5(6) over [0, t_end]; returns (next dt, accepted, rejected)."""
        flags = (GBD_STEP_EXTRAP if extrap else 0) | (GBD_STEP_CONTINUE if cont else 0)
        return gbd_llg_run_rkf56(self.handle, m, t_end, dt, tol, self.shape, max_steps, stream, flags)

    def get_state(self, stream=None):
        """Checkpoint of the integrator state kept in the mesh (bytes); m is the caller's."""
        return gbd_mesh_get_state(self.handle, stream)

    def set_state(self, state, stream=None):
        """Resume from get_state's bytes (a mesh with the same cell count); continue with cont=True."""
        gbd_mesh_set_state(self.handle, state, stream)

    def set_params(self, Hext=None, alpha=None):
        """Applied field (A/m) and/or damping of later calls (None keeps the current value)."""
        gbd_mesh_set_params(self.handle, Hext, alpha)

    def autotune(self, stream=None):
        gbd_mesh_autotune(self.handle, stream)
        return gbd_mesh_get_tuning(self.handle)

    def device_status(self, stream=None):
        return gbd_mesh_device_status(self.handle, stream)

    def close(self):
        if self.handle is not None:
            gbd_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many meshes advanced together with one CUDA-graph launch per run (gbd_batch_*)."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        self.handle = gbd_batch_create([m.handle for m in self.meshes])

    def run(self, m_list, nsteps, dts, stream=None, flags=None):
        """flags: per-mesh GBD_STEP_* bits (None: plain RK4 for every mesh)."""
        gbd_batch_run(self.handle, m_list, [m.shape for m in self.meshes], nsteps, dts, stream, flags)

    def close(self):
        if self.handle is not None:
            gbd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
