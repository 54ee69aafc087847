"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
* FP64: every output element within 1e-12 * max|u| of the oracle.  Each
  level applies operators of max norm < 2 per axis and a few dozen roundings
  of 1.1e-16 per value; over <= 12 levels the drift stays near 1e-14.
* FP32: within tol32(L) * max|u| = 24 u (L + 1) max|u| (u = 2^-24), about
  4-5x above the worst error measured on these cases (tests/tolerances.py
  gives the error model and the measurements).
* Quantization labels: bit-exact given the same coefficient array and the
  same tolerances (both sides divide in IEEE FP64).
"""
import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import fields as F
from tolerances import TOL64, tol32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
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
    if kind == "z":
        return [None] * (len(dims) - 1) + [F.geometric_coords(dims[-1], 1.03)]
    return [F.geometric_coords(n, 1.02 + 0.01 * d) for d, n in enumerate(dims)]


def gpu_decompose(torch, u, coords, stop, dtype):
    x = torch.from_numpy(np.ascontiguousarray(u.astype(dtype))).cuda()
    B.decompose(x, coords, stop)
    torch.cuda.synchronize()
    return x


def gpu_recompose(torch, x, coords, stop):
    y = x.clone()
    B.recompose(y, coords, stop)
    torch.cuda.synchronize()
    return y


CASES = [
    ((9,), "u", 0), ((10,), "g", 0), ((4,), "u", 0), ((3,), "u", 0), ((1000,), "g", 0),
    ((2049,), "u", 2), ((17, 17), "u", 0), ((12, 9), "g", 0), ((70, 45), "g", 1),
    ((1025, 33), "u", 0), ((9, 9, 9), "u", 0), ((5, 5, 5), "u", 0), ((10, 7, 12), "g", 0),
    ((17, 9, 6), "u", 1), ((33, 33, 33), "z", 0), ((70, 45, 133), "g", 0), ((65, 65, 65), "u", 0),
    ((40, 65, 100), "z", 2), ((100, 50, 4), "u", 0),
    # Levels of at least 2^17 nodes take the marching kernels: 2D with rows
    # in one chunk and in several, 3D with even axes, rows too wide to march.
    ((400, 1500), "g", 0), ((1030, 258), "u", 0), ((66, 64, 62), "g", 0), ((34, 40, 600), "u", 1),
    # 2^k + 1 rows (257 and 129 coarse columns): the left-over column of the
    # paired load-vector rows is taken one staged row per lane.
    ((129, 65, 257), "g", 0), ((300, 513), "z", 0),
    # Odd axes that are not 2^k + 1 (the all-odd-grid load vector at the top
    # level, general levels below it).
    ((75, 67, 139), "g", 0), ((301, 771), "u", 0),
    # Coarse planes of >= 19600 lines: the axis-0 (then axis-1) solves of the
    # top level take the persistent pipelined segmented form.
    ((40, 279, 279), "g", 0), ((279, 40, 279), "g", 0),
]


@pytest.mark.parametrize("dims,kind,stop", CASES, ids=lambda v: str(v))
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_decompose_recompose_parity(cuda, dims, kind, stop, dtype):
    torch = cuda
    coords = _coords(dims, kind)
    H = O.Hierarchy(dims, coords)
    stop = min(stop, H.L)
    u = F.sinusoid_field(dims, seed=sum(dims) + stop).astype(dtype)
    exp = O.decompose(u.astype(np.float64), H, stop)
    x = gpu_decompose(torch, u, coords, stop, dtype)
    got = x.cpu().numpy().astype(np.float64)
    scale = np.abs(u).max()
    tol = TOL64 if dtype == np.float64 else tol32(H.L)
    err = np.abs(got - exp).max() / scale
    assert err <= tol, f"decompose max rel err {err:.3e}"
    r = gpu_recompose(torch, x, coords, stop).cpu().numpy().astype(np.float64)
    err_r = np.abs(r - u.astype(np.float64)).max() / scale
    assert err_r <= tol, f"identity max rel err {err_r:.3e}"
    # The recomposition of the oracle's coefficients also matches.
    xr = torch.from_numpy(exp.astype(dtype)).cuda()
    r2 = gpu_recompose(torch, xr, coords, stop).cpu().numpy().astype(np.float64)
    exp_r = O.recompose(exp.astype(dtype).astype(np.float64), H, stop)
    assert np.abs(r2 - exp_r).max() / scale <= tol


@pytest.mark.parametrize("dims,kind", [((33, 33, 33), "g"), ((70, 45), "u"), ((1000,), "g")])
def test_multilinear_input_zero_coefficients(cuda, dims, kind):
    torch = cuda
    coords = _coords(dims, kind)
    u = F.multilinear_field(dims, coords)
    H = O.Hierarchy(dims, coords)
    x = gpu_decompose(torch, u, coords, 0, np.float64).cpu().numpy()
    lev = O.node_levels(H)
    assert np.abs(x[lev > 0]).max() < 1e-13
    np.testing.assert_allclose(x[np.ix_(*H.index[0])], u[np.ix_(*H.index[0])], atol=1e-13)


@pytest.mark.parametrize("dims,kind,stop", [((65, 65, 65), "u", 0), ((33, 20, 17), "g", 1),
                                            ((40, 65, 100), "z", 2), ((257, 129), "u", 0),
                                            ((3000,), "g", 0)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("rel", [1e-2, 1e-4])
def test_quantize_bit_exact_and_bound(cuda, dims, kind, stop, dtype, rel):
    torch = cuda
    coords = _coords(dims, kind)
    H = O.Hierarchy(dims, coords)
    u = F.grf_field(dims, seed=len(dims) * 1000 + stop, dtype=dtype)
    lo, hi = B.value_range(torch.from_numpy(u).cuda())
    assert lo == float(u.min()) and hi == float(u.max())
    tau = rel * (hi - lo)
    x = gpu_decompose(torch, u, coords, stop, dtype)
    labels, taus = B.quantize(x, tau, coords, stop)
    np.testing.assert_allclose(taus, O.level_tolerances(H, stop, tau), rtol=1e-12)
    coeffs = x.cpu().numpy()
    exp = O.quantize(coeffs.astype(np.float64), H, stop, taus)
    got = labels.cpu().numpy()
    assert np.array_equal(got, exp)
    deq = B.dequantize(labels, tau, x.dtype, coords, stop)
    exp_deq = O.dequantize(exp, H, stop, taus, dtype=dtype)
    assert np.array_equal(deq.cpu().numpy(), exp_deq)
    lev = O.node_levels(H, stop)
    assert np.all(np.abs(exp_deq.astype(np.float64) - coeffs) <= taus[lev] * (1 + 1e-9) +
                  np.abs(coeffs) * np.finfo(dtype).eps)
    rec = gpu_recompose(torch, deq, coords, stop).cpu().numpy().astype(np.float64)
    err = np.abs(rec - u.astype(np.float64)).max()
    assert err <= tau, f"L-inf error {err:.3e} > tau {tau:.3e}"


def test_stop_level_equal_L_is_identity(cuda):
    torch = cuda
    dims = (17, 17, 17)
    H = O.Hierarchy(dims)
    u = F.sinusoid_field(dims)
    x = gpu_decompose(cuda, u, None, H.L, np.float64).cpu().numpy()
    assert np.array_equal(x, u)


def test_deterministic(cuda):
    torch = cuda
    dims = (70, 45, 133)
    u = F.grf_field(dims, seed=5)
    a = gpu_decompose(torch, u, None, 0, np.float32).cpu().numpy()
    b = gpu_decompose(torch, u, None, 0, np.float32).cpu().numpy()
    assert np.array_equal(a, b)


def test_device_errors(cuda):
    torch = cuda
    dims = (33, 33, 33)
    x = torch.zeros(dims, device="cuda")
    ws = B.workspace(dims, torch.float32)
    small = B.mgard_workspace_size(dims, B.F32) - 256
    assert B.mgard_decompose(dims, None, B.F32, 0, x.data_ptr(), ws.data_ptr(), small, 0) == -5
    assert B.mgard_decompose(dims, None, B.F32, 0, x.data_ptr() + 2, ws.data_ptr(), ws.numel(), 0) == -1
    assert B.mgard_decompose(dims, None, B.F32, 0, x.data_ptr(), ws.data_ptr() + 16, ws.numel(), 0) == -5
    assert B.mgard_decompose(dims, None, B.F32, 9, x.data_ptr(), ws.data_ptr(), ws.numel(), 0) == -4
    x[3, 4, 5] = float("nan")
    with pytest.raises(B.MgardError) as e:
        B.quantize(x, 1e-3)
    assert e.value.code == -7
    with pytest.raises(B.MgardError) as e:
        B.value_range(x)
    assert e.value.code == -7
    y = torch.full(dims, 1e30, device="cuda")
    with pytest.raises(B.MgardError) as e:
        B.quantize(y, 1e-3)
    assert e.value.code == -6


def test_quantize_async_defers_its_checks(cuda):
    """mgard_quantize_async writes the labels of mgard_quantize and leaves
    its flags to mgard_quantize_status, which reports the first problem of
    every call since the last check and then clears it."""
    torch = cuda
    dims = (65, 33, 47)
    x = torch.from_numpy(F.grf_field(dims, seed=17)).cuda()
    B.quantize_status()  # start from a clear word
    want, taus = B.quantize(x, 1e-3)
    got, taus_a = B.quantize_async(x, 1e-3)
    B.quantize_status()
    assert torch.equal(got, want)
    assert np.array_equal(taus, taus_a)
    # A non-finite coefficient: the call returns, the check reports it once.
    y = x.clone()
    y[3, 4, 5] = float("nan")
    B.quantize_async(y, 1e-3)
    B.quantize_async(x, 1e-3)  # a later clean call does not hide it
    with pytest.raises(B.MgardError) as e:
        B.quantize_status()
    assert e.value.code == -7
    B.quantize_status()  # cleared
    big = torch.full(dims, 1e30, device="cuda")
    B.quantize_async(big, 1e-3)
    with pytest.raises(B.MgardError) as e:
        B.quantize_status()
    assert e.value.code == -6
    B.quantize_status()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_relative_bound_on_the_device_matches_the_host(cuda, dtype):
    """Range, labels and bin centres with tau formed on the device from the
    device range equal, bit for bit, those of the host calls given
    tau = rel x (max - min); a constant array (tau = 0) is reported."""
    torch = cuda
    tdt = torch.float32 if dtype == "f32" else torch.float64
    for dims, stop in (((65, 33, 47), 0), ((129, 100), 2), ((700,), 1)):
        x = torch.from_numpy(F.grf_field(dims, seed=23)).to(tdt).cuda()
        lo, hi = B.value_range(x)
        rng = B.value_range_async(x)
        B.quantize_status()
        assert rng.cpu().tolist() == [lo, hi]
        c = B.decompose(x.clone(), None, stop)
        for rel in (1e-2, 1e-3, 1e-4, 1e-5):
            tau = rel * (hi - lo)
            want, _ = B.quantize(c, tau, None, stop)
            got = B.quantize_rel_async(c, rel, rng, None, stop)
            B.quantize_status()
            assert torch.equal(got, want), (dims, rel)
            back = B.dequantize(want, tau, tdt, None, stop)
            back_rel = B.dequantize_rel(want, rel, rng, tdt, None, stop)
            assert torch.equal(back_rel, back), (dims, rel)
    flat = torch.ones((33, 33), dtype=tdt, device="cuda")
    rng = B.value_range_async(flat)
    B.quantize_rel_async(flat, 1e-3, rng)
    with pytest.raises(B.MgardError) as e:
        B.quantize_status()
    assert e.value.code == -1


def test_host_buffer_entry_points(cuda):
    torch = cuda
    dims = (65, 65, 65)
    u = F.sinusoid_field(dims).astype(np.float32)
    dev = torch.empty(dims, dtype=torch.float32, device="cuda")
    ws = B.workspace(dims, torch.float32)
    host_in = torch.from_numpy(u).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    rc = B.mgard_decompose_host(dims, None, B.F32, 0, host_in.data_ptr(), host_out.data_ptr(),
                                dev.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert rc == 0
    ref = gpu_decompose(torch, u, None, 0, np.float32).cpu().numpy()
    assert np.array_equal(host_out.numpy(), ref)
    back = torch.empty_like(host_in).pin_memory()
    rc = B.mgard_recompose_host(dims, None, B.F32, 0, host_out.data_ptr(), back.data_ptr(),
                                dev.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert rc == 0
    assert np.abs(back.numpy() - u).max() <= tol32(5) * np.abs(u).max()


# ---------------------------------------------------- full-size workloads ---

def test_full_size_65_cubed_fp64_pipeline(cuda):
    """65^3 FP64 sinusoids + noise, full depth, then quantization at 1e-3 x
    range: elementwise parity with the oracle and the L-inf bound."""
    torch = cuda
    dims = (65, 65, 65)
    u = F.sinusoid_field(dims, seed=F.SEED_TINY)
    H = O.Hierarchy(dims)
    exp = O.decompose(u, H)
    x = gpu_decompose(torch, u, None, 0, np.float64)
    assert np.abs(x.cpu().numpy() - exp).max() <= TOL64 * np.abs(u).max()
    tau = 1e-3 * O.value_range(u)
    labels, taus = B.quantize(x, tau)
    assert np.array_equal(labels.cpu().numpy(), O.quantize(x.cpu().numpy(), H, 0, taus))
    rec = gpu_recompose(torch, B.dequantize(labels, tau, torch.float64), None, 0).cpu().numpy()
    assert np.abs(rec - u).max() <= tau


def test_full_size_513_cubed_fp32(cuda):
    """513^3 FP32 k^-5/3 field: decomposition against the full FP64 oracle,
    identity, and at every relative bound {1e-2, 1e-3, 1e-4, 1e-5} the GPU
    recomposition of the bound's labels against the oracle's recomposition of
    the same labels and the L-inf bound against the input."""
    torch = cuda
    dims = (513, 513, 513)
    u = F.grf_field(dims, seed=F.SEED_LARGE)
    H = O.Hierarchy(dims)
    x = gpu_decompose(torch, u, None, 0, np.float32)
    exp = O.decompose(u.astype(np.float64), H)
    scale = float(np.abs(u).max())
    err = np.abs(x.cpu().numpy().astype(np.float64) - exp).max() / scale
    del exp
    assert err <= tol32(H.L), err
    r = gpu_recompose(torch, x, None, 0)
    assert (r - torch.from_numpy(u).cuda()).abs().max().item() / scale <= tol32(H.L)
    del r
    lo, hi = B.value_range(torch.from_numpy(u).cuda())
    ud = torch.from_numpy(u).cuda().double()
    for rel in (1e-2, 1e-3, 1e-4, 1e-5):
        tau = rel * (hi - lo)
        labels, taus = B.quantize(x, tau)
        deq = B.dequantize(labels, tau, torch.float32)
        rec_o = O.recompose(deq.cpu().numpy().astype(np.float64), H)
        rec = gpu_recompose(torch, deq, None, 0)
        d = np.abs(rec.cpu().numpy().astype(np.float64) - rec_o).max() / scale
        del rec_o
        assert d <= tol32(H.L), (rel, d)
        err = (rec.double() - ud).abs().max().item()
        assert err <= tau, (rel, err, tau)


@pytest.mark.parametrize("stop", [3, 0])
def test_full_size_nonuniform_500x500x100(cuda, stop):
    """500x500x100 FP32 with geometric z (ratio 1.03), sinusoids + tanh
    front, stopping level 3 and full depth: parity with the FP64 oracle and
    the L-inf bound at 1e-3 x range."""
    torch = cuda
    dims = (500, 500, 100)
    coords = [F.uniform_coords(500), F.uniform_coords(500), F.geometric_coords(100, 1.03)]
    u = F.front_field(dims, coords)
    H = O.Hierarchy(dims, coords)
    x = gpu_decompose(torch, u, coords, stop, np.float32)
    exp = O.decompose(u.astype(np.float64), H, stop)
    scale = float(np.abs(u).max())
    assert np.abs(x.cpu().numpy().astype(np.float64) - exp).max() / scale <= tol32(H.L)
    tau = 1e-3 * O.value_range(u)
    labels, taus = B.quantize(x, tau, coords, stop)
    rec = gpu_recompose(torch, B.dequantize(labels, tau, torch.float32, coords, stop), coords, stop)
    err = (rec.double() - torch.from_numpy(u).cuda().double()).abs().max().item()
    assert err <= tau


# --------------------------------------------- quantizer rounding edges ---

@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_quantize_rounding_boundaries(cuda, dtype):
    """Coefficients placed on, and a few ulps around, the half-integer bin
    boundaries of every level (where the FP32 fast path must defer to the
    FP64 division), plus huge and tiny magnitudes: labels equal the oracle's."""
    torch = cuda
    dims = (4097,)
    H = O.Hierarchy(dims)
    taus = B.mgard_level_tolerances(dims, None, 0, 0.37)
    lev = O.node_levels(H)
    q = 2.0 * taus[lev]
    rng = np.random.default_rng(3)
    k = rng.integers(-2 ** 21, 2 ** 21, size=dims).astype(np.float64)
    k[::7] = rng.integers(-40, 40, size=k[::7].shape)
    base = (k + np.where(k >= 0, 0.5, -0.5)) * q
    x = base.astype(dtype)
    steps = rng.integers(-3, 4, size=dims)
    for s in range(1, 4):
        sel = steps == s
        x[sel] = np.nextafter(x[sel], np.array(np.inf, dtype=dtype))
        sel = steps == -s
        x[sel] = np.nextafter(x[sel], np.array(-np.inf, dtype=dtype))
    x[::11] = (rng.standard_normal(x[::11].shape) * 1e-30).astype(dtype)
    x[::13] = (rng.standard_normal(x[::13].shape) * q[::13] * 3e5).astype(dtype)
    xt = torch.from_numpy(x).cuda()
    labels, t2 = B.quantize(xt, 0.37)
    exp = O.quantize(x.astype(np.float64), H, 0, t2)
    assert np.array_equal(labels.cpu().numpy(), exp)


@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_dequantize_exact_products(cuda, dtype):
    """label * q rounded to FP64 and then to the element type, for labels
    from 0 to 2^45 in magnitude and tolerances that put results from the
    subnormal to the overflow range of FP32: bit-exact with the oracle."""
    torch = cuda
    dims = (8193,)
    H = O.Hierarchy(dims)
    lev = O.node_levels(H)
    rng = np.random.default_rng(4)
    mags = rng.integers(0, 46, size=dims)
    labels = (rng.integers(0, 2 ** 62, size=dims) >> (62 - mags)) * rng.choice([-1, 1], size=dims)
    labels[::5] = rng.integers(-3, 4, size=labels[::5].shape)
    for tau in (0.37, 1e-30, 3e-45, 1e25):
        taus = B.mgard_level_tolerances(dims, None, 0, tau)
        lt = torch.from_numpy(labels.astype(np.int64)).cuda()
        got = B.dequantize(lt, tau, torch.float64 if dtype == np.float64 else torch.float32)
        with np.errstate(over="ignore"):
            exp = O.dequantize(labels, H, 0, taus, dtype=dtype)
        g = got.cpu().numpy()
        assert np.array_equal(g.view(np.uint8), exp.view(np.uint8)), tau
