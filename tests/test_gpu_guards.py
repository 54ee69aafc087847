"""Guard bands around every device buffer an entry point writes: a kernel
that writes past its array's end (or before its start) changes the
sentinel bytes around it.  Tiny and odd shapes (axes of 3, 4, 5, 7 nodes)
are where index arithmetic breaks first.  Together with the determinism
test this stands in for a race / bounds checker, which this pool does not
offer."""
import ctypes

import numpy as np
import pytest

from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F

pytestmark = pytest.mark.gpu

GUARD = 4096          # bytes on each side; a multiple of 256 keeps alignment
SENTINEL = 0xA5


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2010_05872_gb300 import build as build_mod
    build_mod.build()
    B.lib()
    return torch


class Guarded:
    """A device byte buffer of `nbytes` with GUARD sentinel bytes on each side."""

    def __init__(self, torch, nbytes):
        self.torch = torch
        self.nbytes = int(nbytes)
        self.buf = torch.full((self.nbytes + 2 * GUARD,), SENTINEL, dtype=torch.uint8, device="cuda")

    @property
    def ptr(self):
        return self.buf.data_ptr() + GUARD

    def view(self, dtype, shape):
        n = int(np.prod(shape))
        return self.buf[GUARD:GUARD + self.nbytes].view(dtype)[:n].view(shape)

    def intact(self):
        self.torch.cuda.synchronize()
        lo = self.buf[:GUARD]
        hi = self.buf[GUARD + self.nbytes:]
        return bool((lo == SENTINEL).all().item()) and bool((hi == SENTINEL).all().item())


SHAPES_3D = [((3, 3, 3), None), ((4, 5, 7), None), ((7, 4, 3), "g"), ((33, 17, 9), "g"),
             ((5,), None), ((10, 7), "g"), ((65, 65, 65), None), ((70, 45, 133), None)]


def _coords(dims, kind):
    return None if kind is None else [F.geometric_coords(n, 1.04) for n in dims]


@pytest.mark.parametrize("dims,kind", SHAPES_3D)
@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_transform_and_quantizer_stay_in_bounds(cuda, dims, kind, dtype):
    torch = cuda
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    code = B.F32 if dtype == np.float32 else B.F64
    coords = _coords(dims, kind)
    es = np.dtype(dtype).itemsize
    n = int(np.prod(dims))
    data = Guarded(torch, n * es)
    ws = Guarded(torch, max(B.mgard_workspace_size(dims, code), 256))
    labels = Guarded(torch, 8 * n)
    x = data.view(tdt, dims)
    x.copy_(torch.from_numpy(F.sinusoid_field(dims, seed=3).astype(dtype)))
    L = B.mgard_num_levels(dims)
    for stop in sorted({0, min(1, L)}):
        assert B.mgard_decompose(dims, coords, code, stop, data.ptr, ws.ptr, ws.nbytes, 0) == 0
        rc, _ = B.mgard_quantize(dims, coords, code, stop, 1e-3, data.ptr, labels.ptr, 0)
        assert rc == 0
        assert B.mgard_dequantize(dims, coords, code, stop, 1e-3, labels.ptr, data.ptr, 0) == 0
        assert B.mgard_recompose(dims, coords, code, stop, data.ptr, ws.ptr, ws.nbytes, 0) == 0
        rc, _ = B.mgard_value_range(n, code, data.ptr, 0)
        assert rc == 0
    assert data.intact() and ws.intact() and labels.intact()


@pytest.mark.parametrize("dims", [(3, 4, 5, 7), (9, 9, 9, 9), (17, 9, 10, 6)])
@pytest.mark.parametrize("dtype", [np.float32, np.float64], ids=["f32", "f64"])
def test_4d_stays_in_bounds(cuda, dims, dtype):
    torch = cuda
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    code = B.F32 if dtype == np.float32 else B.F64
    n = int(np.prod(dims))
    es = np.dtype(dtype).itemsize
    data = Guarded(torch, n * es)
    ws = Guarded(torch, max(B.mgard_workspace_size_4d(dims, code), 256))
    labels = Guarded(torch, 8 * n)
    x = data.view(tdt, dims)
    x.copy_(torch.rand(dims, dtype=tdt, device="cuda"))
    L = B.mgard_num_levels_4d(dims)
    for stop in sorted({0, min(1, L)}):
        assert B.mgard_decompose_4d(dims, None, code, stop, data.ptr, ws.ptr, ws.nbytes, 0) == 0
        rc, _ = B.mgard_quantize_4d(dims, None, code, stop, 1e-3, data.ptr, labels.ptr, 0)
        assert rc == 0
        assert B.mgard_dequantize_4d(dims, None, code, stop, 1e-3, labels.ptr, data.ptr, 0) == 0
        assert B.mgard_recompose_4d(dims, None, code, stop, data.ptr, ws.ptr, ws.nbytes, 0) == 0
    assert data.intact() and ws.intact() and labels.intact()


@pytest.mark.parametrize("n", [1, 1023, 1025, 70001])
def test_label_coders_stay_in_bounds(cuda, n):
    """The packed and Huffman streams write nothing past their size, and
    their decoders nothing past the labels."""
    torch = cuda
    rng = np.random.default_rng(n)
    x = ((rng.geometric(0.05, n) - 1) * rng.choice([-1, 1], n)).astype(np.int64)
    x[0] = -2 ** 63
    lab = Guarded(torch, 8 * n)
    lab.view(torch.int64, (n,)).copy_(torch.from_numpy(x))
    for bound_fn, enc_fn, dec_fn in (
            (B.pack_bound, B.lib().mgard_pack_labels, B.lib().mgard_unpack_labels),
            (B.huffman_bound, B.lib().mgard_huffman_encode, B.lib().mgard_huffman_decode)):
        cap = bound_fn(n)
        out = Guarded(torch, cap)
        nb = ctypes.c_size_t()
        assert enc_fn(n, lab.ptr, out.ptr, cap, ctypes.byref(nb), 0) == 0
        torch.cuda.synchronize()
        tail = out.buf[GUARD + nb.value:]
        assert bool((tail == SENTINEL).all().item()), "stream written past its size"
        back = Guarded(torch, 8 * n)
        assert dec_fn(out.ptr, nb.value, n, back.ptr, 0) == 0
        assert back.intact() and out.intact()
        assert torch.equal(back.view(torch.int64, (n,)), lab.view(torch.int64, (n,)))
    assert lab.intact()
