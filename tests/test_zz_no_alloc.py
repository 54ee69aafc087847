"""GPU tests of the allocation-free decomposition entry point
(mgard_decompose_noalloc), for callers such as an in-situ simulation that
holds nearly all device memory and cannot allocate while it compresses: the
same result as mgard_decompose on two calls in a row, agreement with the FP64
oracle, the wait-and-report form, the rejection of shapes that do not fit its
static scratch, and that calls after a warm-up call change neither the
device's free memory nor torch's allocated bytes.  The file name keeps it
last in collection, so it runs both alone and after every other GPU test."""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F
from tolerances import TOL64, tol32

pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_the_oracle(cuda):
    torch = cuda
    dims = (40, 33, 50)
    coords = [F.geometric_coords(n, 1.02 + 0.01 * d) for d, n in enumerate(dims)]
    u = F.sinusoid_field(dims, seed=7)
    H = O.Hierarchy(dims, coords)
    exp = O.decompose(u, H, 1)
    x = torch.from_numpy(u).cuda()
    B.decompose_noalloc(x, coords, 1, wait=True)
    assert np.abs(x.cpu().numpy() - exp).max() <= TOL64 * float(np.abs(u).max())


def test_noalloc_calls_reserve_no_device_memory(cuda):
    """After one warm-up call (which may load the library's device code and
    reserve the static scratch), further calls -- on the same shape and on a
    new shape served by the same kernels -- leave the device's free memory and
    torch's allocated bytes unchanged."""
    torch = cuda
    a_dims, b_dims = (65, 65, 65), (65, 33, 129)
    ua = F.sinusoid_field(a_dims, seed=1).astype(np.float32)
    ub = F.sinusoid_field(b_dims, seed=2).astype(np.float32)
    xs = [torch.from_numpy(ua).cuda() for _ in range(3)] + [torch.from_numpy(ub).cuda()]
    B.decompose_noalloc(xs[0], wait=True)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    B.decompose_noalloc(xs[3], wait=True)   # new shape: host tables, copy into the scratch
    B.decompose_noalloc(xs[1], wait=True)   # back to the first shape
    B.decompose_noalloc(xs[2])              # enqueue-only form
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.equal(xs[1], xs[2]) and torch.equal(xs[0], xs[1])
