"""GPU parity of the labels' lossless stage with the oracle's stream (bit for
bit), round trips, argument checks, and the packed host-buffer compression
path against the unpacked one."""
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


def _labels(n, seed, spread):
    rng = np.random.default_rng(seed)
    x = rng.integers(-spread, spread + 1, n).astype(np.int64)
    if n > 3000:
        x[100:1124] = 0                      # an all-zero chunk
        x[2000] = 2 ** 62
        x[2500] = -2 ** 63                   # a 64-bit chunk
        x[n - 1] = 2 ** 63 - 1
    return x


@pytest.mark.parametrize("n,spread", [(0, 1), (1, 5), (1023, 3), (1024, 0), (1025, 100),
                                      (5000, 7), (70001, 1000)])
def test_pack_matches_oracle_stream(cuda, n, spread):
    torch = cuda
    x = _labels(n, n, spread)
    got = B.pack_labels(torch.from_numpy(x).cuda()).cpu().numpy().tobytes()
    assert got == O.pack_labels(x)
    y = B.unpack_labels(torch.from_numpy(np.frombuffer(got, dtype=np.uint8).copy()).cuda(), n)
    assert np.array_equal(y.cpu().numpy(), x)


def test_unpack_rejects_bad_streams(cuda):
    torch = cuda
    x = _labels(5000, 1, 9)
    s = B.pack_labels(torch.from_numpy(x).cuda())
    with pytest.raises(B.MgardError):
        B.unpack_labels(s, 4999)                      # wrong count
    with pytest.raises(B.MgardError):
        B.unpack_labels(s[:-8].clone(), 5000)         # truncated payload
    bad = s.clone()
    bad[8] = 65                                       # width above 64
    with pytest.raises(B.MgardError):
        B.unpack_labels(bad, 5000)


def test_packed_host_path_matches_unpacked(cuda):
    """129 x 257 x 65 FP32: the packed host path returns the same field as
    the int64 host path, its stream unpacks to the same labels, and the
    stream is a fraction of the int64 labels."""
    torch = cuda
    dims = (129, 257, 65)
    u = F.grf_field(dims, seed=3)
    n = u.size
    ws = B.workspace(dims, torch.float32)
    dev = torch.empty(dims, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int64, device="cuda")
    cap = B.pack_bound(n)
    dstream = torch.empty(cap, dtype=torch.uint8, device="cuda")
    hf = torch.from_numpy(u).pin_memory()
    hs = torch.empty(cap, dtype=torch.uint8).pin_memory()
    rc, nbytes, tau = B.mgard_compress_host_packed(dims, None, B.F32, 0, 1e-3, hf.data_ptr(),
                                                   hs.data_ptr(), cap, dev.data_ptr(),
                                                   lab.data_ptr(), dstream.data_ptr(), cap,
                                                   ws.data_ptr(), ws.numel(), 0)
    assert rc == 0 and nbytes < 2 * n  # under 16 bits per label (64 unpacked) at this bound
    hl = torch.empty(n, dtype=torch.int64).pin_memory()
    rc, tau2 = B.mgard_compress_host(dims, None, B.F32, 0, 1e-3, hf.data_ptr(), hl.data_ptr(),
                                     dev.data_ptr(), lab.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert rc == 0 and tau2 == tau
    H = O.Hierarchy(dims)
    # The stream carries the labels with the coarse block's Lorenzo residuals.
    assert np.array_equal(O.unpack_labels(hs.numpy()[:nbytes].tobytes()),
                          O.lorenzo_encode(hl.numpy().reshape(dims), H, 0).ravel())
    out_p = torch.empty(dims, dtype=torch.float32).pin_memory()
    out_u = torch.empty(dims, dtype=torch.float32).pin_memory()
    assert B.mgard_decompress_host_packed(dims, None, B.F32, 0, tau, hs.data_ptr(), nbytes,
                                          out_p.data_ptr(), dev.data_ptr(), lab.data_ptr(),
                                          dstream.data_ptr(), cap, ws.data_ptr(), ws.numel(), 0) == 0
    assert B.mgard_decompress_host(dims, None, B.F32, 0, tau, hl.data_ptr(), out_u.data_ptr(),
                                   dev.data_ptr(), lab.data_ptr(), ws.data_ptr(), ws.numel(), 0) == 0
    assert np.array_equal(out_p.numpy(), out_u.numpy())
    assert np.abs(out_p.numpy().astype(np.float64) - u).max() <= tau


def _round_trips(torch, dims, u, bounds, stream, out):
    """Packed host round trips of field u at each bound on `stream` (0 = the
    legacy default stream); appends (stream bytes, tau, reconstruction)."""
    n = u.size
    ws = B.workspace(dims, torch.float32)
    dev = torch.empty(dims, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int64, device="cuda")
    cap = B.pack_bound(n)
    dstream = torch.empty(cap, dtype=torch.uint8, device="cuda")
    hf = torch.from_numpy(u).pin_memory()
    hs = torch.empty(cap, dtype=torch.uint8).pin_memory()
    ho = torch.empty(dims, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    sp = stream.cuda_stream if stream is not None else 0
    for rel in bounds:
        rc, nbytes, tau = B.mgard_compress_host_packed(
            dims, None, B.F32, 0, rel, hf.data_ptr(), hs.data_ptr(), cap, dev.data_ptr(),
            lab.data_ptr(), dstream.data_ptr(), cap, ws.data_ptr(), ws.numel(), sp)
        assert rc == 0, rc
        packed = hs.numpy()[:nbytes].copy()
        rc = B.mgard_decompress_host_packed(
            dims, None, B.F32, 0, tau, hs.data_ptr(), nbytes, ho.data_ptr(), dev.data_ptr(),
            lab.data_ptr(), dstream.data_ptr(), cap, ws.data_ptr(), ws.numel(), sp)
        assert rc == 0, rc
        out.append((packed, tau, ho.numpy().copy()))


def test_streams_from_several_threads_match_serial(cuda):
    """Four host threads each run packed round trips of their own field on
    their own stream at the same time (each stream's first calls make its
    scratch while the others have work in flight; the four shapes launch the
    same kernels with different shared-memory sizes): every packed stream
    and every reconstruction equals that of the same calls made one after
    another, and each reconstruction stays within tau of its field."""
    import threading
    torch = cuda
    shapes = [(129, 257, 65), (65, 129, 97), (257, 129, 33), (97, 65, 129)]
    cases = [(d, F.grf_field(d, seed=11 + i)) for i, d in enumerate(shapes)]
    bounds = (1e-2, 1e-3, 1e-4)
    serial = []
    for dims, u in cases:
        got = []
        _round_trips(torch, dims, u, bounds, None, got)
        serial.append(got)
    streams = [torch.cuda.Stream() for _ in cases]
    results = [[] for _ in cases]
    errors = []

    def run(q):
        try:
            dims, u = cases[q]
            _round_trips(torch, dims, u, bounds, streams[q], results[q])
        except BaseException as exc:  # re-raised in the test's thread
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(q,)) for q in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    for (dims, u), want, got in zip(cases, serial, results):
        assert len(got) == len(bounds)
        for (pw, tw, rw), (pg, tg, rg) in zip(want, got):
            assert tg == tw
            assert np.array_equal(pg, pw)
            assert np.array_equal(rg, rw)
            assert np.abs(rg.astype(np.float64) - u).max() <= tg


@pytest.mark.parametrize("dims,stop", [((17, 9, 12), 0), ((17, 9, 12), 2), ((33, 20), 1),
                                       ((100,), 3), ((65, 65, 65), 5)])
def test_lorenzo_matches_oracle(cuda, dims, stop):
    torch = cuda
    H = O.Hierarchy(dims)
    stop = min(stop, H.L)
    x = np.random.default_rng(7).integers(-2 ** 62, 2 ** 62, dims).astype(np.int64)
    x.flat[0] = 2 ** 62 - 1
    t = torch.from_numpy(x).cuda()
    B.lorenzo(t, torch.float32, True, None, stop)
    enc = t.cpu().numpy()
    assert np.array_equal(enc, O.lorenzo_encode(x, H, stop))
    B.lorenzo(t, torch.float32, False, None, stop)
    assert np.array_equal(t.cpu().numpy(), x)


def test_lorenzo_shrinks_a_smooth_coarse_part(cuda):
    """A smooth 65^3 field kept whole (stop level = L, the coarse block is the
    grid): the Lorenzo residuals of its labels pack to less than half the
    labels' stream."""
    torch = cuda
    dims = (65, 65, 65)
    H = O.Hierarchy(dims)
    u = torch.from_numpy(F.sinusoid_field(dims, seed=2, kmax=2.0, noise=0.0).astype(np.float32)).cuda()
    lo, hi = B.value_range(u)
    labels, _ = B.quantize(u, 1e-4 * (hi - lo), None, H.L)
    plain = B.pack_labels(labels.view(-1)).numel()
    B.lorenzo(labels, torch.float32, True, None, H.L)
    coded = B.pack_labels(labels.view(-1)).numel()
    assert coded * 2 < plain
