"""Guard-word bounds checks on the GPU (compute-sanitizer is not available) and the clean-up path
of a failed mesh creation.

Every caller field sits inside a larger allocation between two guard regions filled with a
sentinel bit pattern; after each public call the guards must be bit-identical. The cases cover
the scalar path (odd sizes, fields 4-byte aligned), the vector path (nx a multiple of 64, 8-byte
aligned), a 3D mesh, a periodic mesh, and every compute call that writes a caller field
(gbd_demag_noalloc included).
"""
import os

import numpy as np
import pytest

from gpu_util import lib
from paper_2308_08447_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GUARD = 96                      # float32 words before and after each field
SENTINEL = np.uint32(0x7F8A5A5A)  # a NaN payload no kernel produces


@pytest.fixture(scope="module")
def g():
    return lib()


class Guarded:
    """A (3, nz, ny, nx) float32 field at word offset GUARD + shift of a guarded buffer."""

    def __init__(self, shape, data, shift):
        import torch
        n = int(np.prod(shape))
        self.n, self.off = n, GUARD + shift
        host = np.full(n + 2 * GUARD + shift, SENTINEL, dtype=np.uint32).view(np.float32)
        host[self.off:self.off + n] = np.asarray(data, np.float32).ravel()
        self.buf = torch.from_numpy(host).cuda()
        self.t = self.buf[self.off:self.off + n].view(shape)

    def guards_intact(self):
        import torch
        torch.cuda.synchronize()
        h = self.buf.cpu().numpy().view(np.uint32)
        return bool((h[:self.off] == SENTINEL).all() and (h[self.off + self.n:] == SENTINEL).all())


CASES = [((7, 4, 3), (2e-9, 3e-9, 4e-9), (False,) * 3, 1),
         ((33, 17, 5), (4e-9, 4e-9, 4e-9), (False,) * 3, 0),
         ((128, 64, 1), (2e-9, 2e-9, 3e-9), (False,) * 3, 0),
         ((64, 32, 4), (3e-9, 3e-9, 3e-9), (False,) * 3, 1),
         ((32, 16, 4), (3e-9, 3e-9, 3e-9), (True, True, True), 0)]


@pytest.mark.parametrize("n,cell,pbc,shift", CASES)
def test_guard_words_untouched(g, n, cell, pbc, shift):
    shape = (3, n[2], n[1], n[0])
    m0 = W.random_unit(n, 31)
    mesh = g.Mesh(n, cell, 8e5, A_ex=1.3e-11, alpha=0.1, pbc=pbc, pbc_images=1 if any(pbc) else 0)
    M = Guarded(shape, 8e5 * m0, shift)
    H = Guarded(shape, np.zeros(shape), shift)
    mesh.demag(M.t, H.t)
    assert M.guards_intact() and H.guards_intact()
    g.gbd_demag_noalloc(mesh.handle, M.t, H.t, shape)   # the same field through the static scratch
    assert M.guards_intact() and H.guards_intact()
    m = Guarded(shape, m0, shift)
    mesh.effective_field(m.t, H.t)
    assert m.guards_intact() and H.guards_intact()
    mesh.llg_rhs(m.t, H.t)
    assert m.guards_intact() and H.guards_intact()
    mesh.llg_step(m.t, 3, 1e-13)
    assert m.guards_intact()
    mesh.llg_step(m.t, 6, 1e-13, extrap=True)
    assert m.guards_intact()
    mesh.rkf56_step(m.t, 1e-13)
    assert m.guards_intact()
    mesh.rkf56_step(m.t, 1e-13, extrap=True)
    assert m.guards_intact()
    assert np.isfinite(m.t.cpu().numpy()).all()
    mesh.close()


def test_failed_creation_frees_its_buffers(g):
    import torch
    n, cell = (96, 64, 8), (3e-9, 3e-9, 3e-9)      # 3D: seven device allocations
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in range(1, 8):
            os.environ["GBD_TEST_FAIL_ALLOC"] = str(k)
            with pytest.raises(g.GbdError) as ei:
                g.Mesh(n, cell, 8e5)
            assert ei.value.status == g.GBD_ENOMEM
    finally:
        del os.environ["GBD_TEST_FAIL_ALLOC"]
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (4 << 20)
    mesh = g.Mesh(n, cell, 8e5)                     # the hook is read at each call
    mesh.close()
