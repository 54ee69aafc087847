"""GPU parity of quantization with the other bin-width rules of Section 4.1:
labels bit-exact with the oracle given the same coefficients and level
tolerances, and the reconstruction within the L2 bound (L2 rule) or the
L-inf bound (L-inf-optimal rule)."""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2010_05872_gb300 import build as build_mod
    build_mod.build()
    B.lib()
    return torch


@pytest.mark.parametrize("dims,kind,stop", [((33, 33, 17), "u", 0), ((40, 26, 34), "g", 1)])
@pytest.mark.parametrize("mode", ["linf_optimal", "l2"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_modes_bit_exact_and_bound(cuda, dims, kind, stop, mode, dtype):
    torch = cuda
    coords = None if kind == "u" else [F.geometric_coords(n, 1.03 + 0.01 * d) for d, n in enumerate(dims)]
    H = O.Hierarchy(dims, coords)
    u = F.sinusoid_field(dims, seed=4).astype(dtype)
    rng = O.value_range(u)
    tau = 1e-3 * rng * (np.sqrt(np.prod(dims)) if mode == "l2" else 1.0)
    taus = B.mgard_level_tolerances_mode(dims, coords, stop, tau, mode)
    np.testing.assert_allclose(taus, O.level_tolerances_mode(H, stop, tau, mode), rtol=1e-12)
    x = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    B.decompose(x, coords, stop)
    labels = B.quantize_levels(x, taus, coords, stop)
    coeffs = x.cpu().numpy().astype(np.float64)
    exp = O.quantize(coeffs, H, stop, taus)
    assert np.array_equal(labels.cpu().numpy(), exp)
    deq = B.dequantize_levels(labels, taus, x.dtype, coords, stop)
    assert np.array_equal(deq.cpu().numpy(), O.dequantize(exp, H, stop, taus, dtype=dtype))
    B.recompose(deq, coords, stop)
    err = deq.cpu().numpy().astype(np.float64) - u.astype(np.float64)
    eps = 1e-9 if dtype == np.float64 else 4e-5 * (H.L + 1) * np.abs(u).max()
    if mode == "l2":
        assert O.l2_error(err, H) <= tau + eps * np.sqrt(np.prod(dims))
    else:
        assert np.abs(err).max() <= tau + eps


def test_mode_argument_errors(cuda):
    torch = cuda
    x = torch.zeros((17, 17, 17), device="cuda")
    taus = np.full(B.mgard_num_levels(x.shape) + 1, 0.1)
    taus[-1] = 0.0
    with pytest.raises(B.MgardError) as e:
        B.quantize_levels(x, taus)
    assert e.value.code == -1
