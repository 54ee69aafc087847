"""GPU tests of the batched form (one persistent launch for many fields):
each field's result equals the per-field path within the FP32 tolerance and
the FP64 oracle, recomposition restores the fields, repeated launches of the
cached graph agree, and the autotuner keeps the fields' contents."""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F
from tolerances import tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.lib()
    return torch


def _fields(torch, shapes, seed):
    return [torch.from_numpy(F.grf_field(s, seed=seed + i)).cuda() for i, s in enumerate(shapes)]


SHAPES = [(33, 40, 57), (64, 33, 33), (50, 71, 38), (33, 33, 33), (97, 35, 66), (40, 129, 34),
          (35, 36, 37), (65, 65, 65), (34, 34, 100), (47, 52, 130)]


def test_batch_matches_per_field_and_oracle(cuda):
    torch = cuda
    xs = _fields(torch, SHAPES, 11)
    ref = [x.clone() for x in xs]
    for r in ref:
        B.decompose(r)
    ws = B.batch_workspace(xs)
    B.batch_decompose(xs, ws)
    torch.cuda.synchronize()
    for x, r, shp in zip(xs, ref, SHAPES):
        L = B.mgard_num_levels(shp)
        scale = r.abs().max().item()
        assert (x - r).abs().max().item() <= tol32(L) * scale, shp
    for i in (0, 4):  # two fields against the FP64 oracle
        u = F.grf_field(SHAPES[i], seed=11 + i).astype(np.float64)
        exp = O.decompose(u, O.Hierarchy(SHAPES[i]))
        L = B.mgard_num_levels(SHAPES[i])
        assert np.abs(xs[i].cpu().numpy() - exp).max() <= tol32(L) * np.abs(u).max()


def test_batch_recompose_identity_and_repeat(cuda):
    torch = cuda
    xs = _fields(torch, SHAPES, 31)
    orig = [x.clone() for x in xs]
    ws = B.batch_workspace(xs)
    for _ in range(3):  # the cached graph, launched again
        B.batch_decompose(xs, ws)
        B.batch_recompose(xs, ws)
    torch.cuda.synchronize()
    for x, o, shp in zip(xs, orig, SHAPES):
        L = B.mgard_num_levels(shp)
        assert (x - o).abs().max().item() <= 3 * tol32(L) * o.abs().max().item(), shp


def test_batch_autotune_keeps_fields(cuda):
    torch = cuda
    shapes = SHAPES[:4]
    xs = _fields(torch, shapes, 51)
    orig = [x.clone() for x in xs]
    ws = B.batch_workspace(xs)
    choice = B.batch_autotune(xs, ws)
    assert choice[0] in (8, 16, 32) and choice[1] in (4, 8, 16) and choice[2] in (64, 128)
    assert choice[3] in (1, 4, 8)
    for x, o in zip(xs, orig):
        assert torch.equal(x, o)
    ref = [x.clone() for x in xs]
    for r in ref:
        B.decompose(r)
    B.batch_decompose(xs, ws)
    torch.cuda.synchronize()
    for x, r, shp in zip(xs, ref, shapes):
        L = B.mgard_num_levels(shp)
        assert (x - r).abs().max().item() <= tol32(L) * r.abs().max().item()


def test_batch_rejects_bad_arguments(cuda):
    torch = cuda
    x = torch.zeros((33, 33, 33), device="cuda")
    ws = B.batch_workspace([x])
    shapes, ptrs = [(33, 33, 33)], [x.data_ptr()]
    assert B.mgard_batch_decompose(shapes, ptrs, ws.data_ptr(), ws.numel() - 512, 0) == -5
    assert B.mgard_batch_decompose([(33, 33, 2)], ptrs, ws.data_ptr(), ws.numel(), 0) == -2
    assert B.mgard_batch_decompose(shapes, [x.data_ptr() + 2], ws.data_ptr(), ws.numel(), 0) == -1


def test_bounded_wait_runs_out_and_is_reported(cuda):
    """A batched schedule whose dependency is never met, with a 5 ms wait
    limit: the kernel's wait gives up instead of spinning, the next value
    range call reports MGARD_ERR_TIMEOUT, and the call after it (and the
    transforms) work again."""
    import time
    torch = cuda
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.from_numpy(F.grf_field((33, 33, 33), seed=3)).cuda()
    torch.cuda.synchronize()
    assert B.mgard_batch_wait_selftest(0, stream) == -1
    t0 = time.perf_counter()
    assert B.mgard_batch_wait_selftest(5_000_000, stream) == 0
    assert time.perf_counter() - t0 < 1.0
    with pytest.raises(B.MgardError) as e:
        B.value_range(x)
    assert e.value.code == -9
    lo, hi = B.value_range(x)
    assert lo == x.min().item() and hi == x.max().item()
    r = x.clone()
    B.decompose(r)
    B.recompose(r)
    torch.cuda.synchronize()
    assert (r - x).abs().max().item() <= tol32(4) * x.abs().max().item()
