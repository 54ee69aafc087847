"""GPU tests of the allocation-free decomposition entry point
(mgard_decompose_noalloc): the same result as mgard_decompose on two calls in
a row, the wait-and-report form, and the rejection of shapes that do not fit
its static scratch.  The file name keeps it last in collection, so it runs
both alone and after every other GPU test."""
import numpy as np
import pytest

from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def tol32(L):
    return 2e-5 * (L + 1)


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    return torch


@pytest.mark.parametrize("dims,kind,dtype,stop", [
    ((65, 65, 65), "u", np.float32, 0),
    ((40, 33, 50), "g", np.float64, 1),
    ((257, 129), "u", np.float32, 0),
    ((1000,), "g", np.float64, 0),
])
def test_noalloc_matches_decompose_twice(cuda, dims, kind, dtype, stop):
    torch = cuda
    coords = None
    if kind == "g":
        coords = [F.geometric_coords(n, 1.02 + 0.01 * d) for d, n in enumerate(dims)]
    u = F.sinusoid_field(dims, seed=sum(dims)).astype(dtype)
    ref = torch.from_numpy(u).cuda()
    B.decompose(ref, coords, stop)
    torch.cuda.synchronize()
    exp = ref.cpu().numpy().astype(np.float64)
    L = B.mgard_num_levels(dims)
    tol = (TOL64 if dtype == np.float64 else tol32(L)) * float(np.abs(u).max())
    for _ in range(2):
        x = torch.from_numpy(u).cuda()
        B.decompose_noalloc(x, coords, stop)
        torch.cuda.synchronize()
        got = x.cpu().numpy().astype(np.float64)
        assert np.abs(got - exp).max() <= tol


def test_noalloc_wait_reports_no_timeout(cuda):
    torch = cuda
    dims = (33, 33, 33)
    u = F.sinusoid_field(dims).astype(np.float32)
    x = torch.from_numpy(u).cuda()
    rc, timed_out = B.mgard_decompose_noalloc(dims, None, B.F32, 0, x.data_ptr(),
                                              torch.cuda.current_stream().cuda_stream, wait=True)
    assert rc == 0 and timed_out is False
    ref = torch.from_numpy(u).cuda()
    B.decompose(ref)
    torch.cuda.synchronize()
    assert (x - ref).abs().max().item() <= tol32(4) * float(np.abs(u).max())


def test_noalloc_rejects_shapes_beyond_its_scratch(cuda):
    torch = cuda
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, _ = B.mgard_decompose_noalloc((513, 513, 513), None, B.F32, 0, x.data_ptr(), stream)
    assert rc == -5  # MGARD_ERR_WORKSPACE, before any work is enqueued
    # A shape that fits still works after the rejection.
    dims = (17, 17, 17)
    u = F.sinusoid_field(dims).astype(np.float32)
    y = torch.from_numpy(u).cuda()
    B.decompose_noalloc(y)
    ref = torch.from_numpy(u).cuda()
    B.decompose(ref)
    torch.cuda.synchronize()
    assert (y - ref).abs().max().item() <= tol32(3) * float(np.abs(u).max())
