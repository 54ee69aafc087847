"""GPU parity of progressive recomposition (Q_k u on the level-k grid from a
decomposed field) and of the iso-surface area with the FP64 oracle.

Tolerances: partial recomposition as the transform (FP64 1e-12, FP32
tol32(L) = 24 u (L + 1) relative to max |u|, u = 2^-24); the iso area relative 1e-10 in FP64 and
1e-5 in FP32 (the vertex classification is exact in both; the crossing
points and areas carry the data's rounding)."""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F
from tolerances import tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2010_05872_gb300 import build as build_mod
    build_mod.build()
    B.lib()
    return torch


def _coords(dims, kind):
    if kind == "u":
        return None
    return [F.geometric_coords(n, 1.02 + 0.01 * d) for d, n in enumerate(dims)]


@pytest.mark.parametrize("dims,kind,stop", [((33, 33, 33), "u", 0), ((34, 40, 26), "g", 1),
                                            ((65, 33, 40), "u", 2), ((70, 45), "g", 0),
                                            ((1000,), "u", 1)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_recompose_partial_matches_oracle(cuda, dims, kind, stop, dtype):
    torch = cuda
    coords = _coords(dims, kind)
    H = O.Hierarchy(dims, coords)
    u = F.sinusoid_field(dims, seed=sum(dims))
    umc = O.decompose(u, H, stop).astype(dtype)
    x = torch.from_numpy(np.ascontiguousarray(umc)).cuda()
    scale = np.abs(u).max()
    tol = 1e-12 if dtype == np.float64 else tol32(H.L)
    for k in range(stop, H.L + 1):
        got = B.recompose_partial(x, k, coords, stop).cpu().numpy().astype(np.float64)
        exp = O.recompose_partial(umc.astype(np.float64), H, stop, k)
        assert got.shape == exp.shape
        assert np.abs(got - exp).max() / scale <= tol, k
    # The decomposed array is left unchanged.
    assert np.array_equal(x.cpu().numpy(), umc)


def _sphere(dims, coords):
    xs = [np.arange(n, dtype=np.float64) if coords is None else coords[d] for d, n in enumerate(dims)]
    X, Y, Z = np.meshgrid(*xs, indexing="ij")
    c = [0.5 * (a[0] + a[-1]) for a in xs]
    return (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2


@pytest.mark.parametrize("dims,kind,field", [((33, 33, 33), "u", "sin"), ((34, 40, 26), "g", "sin"),
                                             ((29, 31, 27), "u", "sphere"),
                                             ((20, 24, 22), "g", "sphere")])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_iso_area_matches_oracle(cuda, dims, kind, field, dtype):
    torch = cuda
    coords = _coords(dims, kind)
    u = F.sinusoid_field(dims, seed=5) if field == "sin" else _sphere(dims, coords)
    u = u.astype(dtype)
    for iso in (float(u.astype(np.float64).mean()), float(np.quantile(u, 0.3))):
        exp = O.iso_area(u.astype(np.float64), coords, iso)
        got = B.iso_area(torch.from_numpy(np.ascontiguousarray(u)).cuda(), iso, coords)
        assert exp > 0
        assert got == pytest.approx(exp, rel=1e-10 if dtype == np.float64 else 1e-5)


def test_iso_area_errors(cuda):
    torch = cuda
    x = torch.zeros((9, 9), device="cuda")
    with pytest.raises(B.MgardError) as e:
        B.iso_area(x, 0.5)
    assert e.value.code == -2
    x = torch.zeros((9, 9, 9), device="cuda")
    with pytest.raises(B.MgardError) as e:
        B.iso_area(x, float("nan"))
    assert e.value.code == -1
    with pytest.raises(B.MgardError) as e:
        B.recompose_partial(x, 9)
    assert e.value.code == -4


def test_full_size_513_cubed_progressive(cuda):
    """513^3 FP32: Q_k u from the full decomposition equals the nodal values
    of a decomposition stopped at k, for k = L-1 .. L-3; at k = L it equals
    the recomposition.  A planar field's iso area is the exact cross-section
    (512 x 512) at every level's own coordinates."""
    torch = cuda
    dims = (513, 513, 513)
    u = torch.from_numpy(F.grf_field(dims, seed=F.SEED_LARGE)).cuda()
    L = B.mgard_num_levels(dims)
    x = u.clone()
    B.decompose(x)
    scale = u.abs().max().item()
    tol = tol32(L)
    full = B.recompose_partial(x, L)
    assert (full - u).abs().max().item() / scale <= tol
    del full
    for k in (L - 1, L - 2, L - 3):
        qk = B.recompose_partial(x, k)
        y = u.clone()
        B.decompose(y, None, k)
        step = 2 ** (L - k)
        ref = y[::step, ::step, ::step]
        assert qk.shape == ref.shape
        assert (qk - ref).abs().max().item() / scale <= tol, k
        del y, ref
        shape, axes = B.level_grid(dims, None, k)
        plane = torch.from_numpy(np.broadcast_to(axes[0][:, None, None], shape).astype(np.float32)).cuda()
        area = B.iso_area(plane, 100.5, axes)
        assert area == pytest.approx(512.0 * 512.0, rel=1e-6)
