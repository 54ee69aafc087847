"""GPU tests of the serving loop (continuous batching): every request of a
mixed compress/decompress stream completes, each result equals the same
request run alone through the blocking host entry points, decompressed
fields meet their bound, served results agree with the FP64 oracle, and
admission keeps the device memory in use within the budget."""
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


SHAPES = [(257, 300), (65, 65, 65), (33, 40, 57), (1025, 129), (129, 129, 129), (100, 50, 4)]


def _alone_compress(torch, shape, field, rel):
    n = field.numel()
    dev = torch.empty(n, dtype=torch.float32, device="cuda")
    dl = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = B.workspace(shape, torch.float32)
    labels = torch.empty(n, dtype=torch.int64).pin_memory()
    rc, tau = B.mgard_compress_host(shape, None, B.F32, 0, rel, field.data_ptr(), labels.data_ptr(),
                                    dev.data_ptr(), dl.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert rc == 0
    return labels, tau


def _alone_decompress(torch, shape, labels, tau):
    n = labels.numel()
    dev = torch.empty(n, dtype=torch.float32, device="cuda")
    dl = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = B.workspace(shape, torch.float32)
    out = torch.empty(n, dtype=torch.float32).pin_memory()
    rc = B.mgard_decompress_host(shape, None, B.F32, 0, tau, labels.data_ptr(), out.data_ptr(),
                                 dev.data_ptr(), dl.data_ptr(), ws.data_ptr(), ws.numel(), 0)
    assert rc == 0
    return out


def test_mixed_stream_matches_alone(cuda):
    torch = cuda
    rng = np.random.default_rng(5)
    srv = B.Server(hbm_budget=2 << 30, slots=4)
    try:
        fields = [torch.from_numpy(F.grf_field(s, seed=40 + i).ravel()).pin_memory()
                  for i, s in enumerate(SHAPES)]
        # Compressed inputs for the decompress requests, made alone.
        packed = [_alone_compress(torch, s, f, 1e-3) for s, f in zip(SHAPES, fields)]
        reqs = []
        for k in range(24):
            i = int(rng.integers(len(SHAPES)))
            n = fields[i].numel()
            if k % 2 == 0:
                rel = [1e-2, 1e-3, 1e-4][int(rng.integers(3))]
                out = torch.empty(n, dtype=torch.int64).pin_memory()
                rid = srv.submit(B.OP_COMPRESS, SHAPES[i], fields[i], out, rel_bound=rel)
                reqs.append((rid, "c", i, rel, out))
            else:
                out = torch.empty(n, dtype=torch.float32).pin_memory()
                rid = srv.submit(B.OP_DECOMPRESS, SHAPES[i], packed[i][0], out, tau=packed[i][1])
                reqs.append((rid, "d", i, packed[i][1], out))
        srv.drain()
        done = {rid: (st, lat, tau) for rid, st, lat, tau in srv.poll()}
        assert len(done) == len(reqs)
        assert srv.counters()["peak_running"] >= 2  # requests overlapped
        for rid, kind, i, arg, out in reqs:
            st, lat, tau = done[rid]
            assert st == 0 and lat > 0
            if kind == "c":
                labels, tau_alone = _alone_compress(torch, SHAPES[i], fields[i], arg)
                assert tau == tau_alone
                assert torch.equal(out, labels)
            else:
                alone = _alone_decompress(torch, SHAPES[i], packed[i][0], arg)
                assert torch.equal(out, alone)
                err = (out.double() - fields[i].double()).abs().max().item()
                assert err <= arg
    finally:
        srv.close()


def test_served_results_match_the_oracle(cuda):
    """Eight served requests (2D and 3D; four compress, four decompress)
    checked against the FP64 oracle: compressed labels are the oracle's
    quantization (Section 4.1) of the device coefficients, which match the
    oracle's decomposition; the oracle's own dequantization and
    recomposition of the served labels meet the bound; decompressed fields
    match the oracle's recomposition of the same labels."""
    torch = cuda
    shapes = [(257, 300), (1025, 129), (65, 65, 65), (33, 40, 57)]
    rels = [1e-2, 1e-3, 1e-4, 1e-3]
    srv = B.Server(hbm_budget=2 << 30, slots=4)
    try:
        us = [F.grf_field(s, seed=70 + i) for i, s in enumerate(shapes)]
        fields = [torch.from_numpy(u.ravel()).pin_memory() for u in us]
        comp = []
        for i, s in enumerate(shapes):
            out = torch.empty(fields[i].numel(), dtype=torch.int64).pin_memory()
            comp.append((srv.submit(B.OP_COMPRESS, s, fields[i], out, rel_bound=rels[i]), out))
        srv.drain()
        taus = {rid: tau for rid, st, _, tau in srv.poll() if st == 0}
        assert len(taus) == len(shapes)
        dec = []
        for i, s in enumerate(shapes):
            rid, labels = comp[i]
            out = torch.empty(fields[i].numel(), dtype=torch.float32).pin_memory()
            dec.append((srv.submit(B.OP_DECOMPRESS, s, labels, out, tau=taus[rid]), out))
        srv.drain()
        assert all(st == 0 for _, st, _, _ in srv.poll())
        for i, s in enumerate(shapes):
            H = O.Hierarchy(s)
            u = us[i].astype(np.float64)
            rid, labels = comp[i]
            tau = taus[rid]
            assert tau == pytest.approx(rels[i] * O.value_range(u), rel=1e-15)
            t = B.mgard_level_tolerances(s, None, 0, tau)
            np.testing.assert_allclose(t, O.level_tolerances(H, 0, tau), rtol=1e-12)
            lab = labels.numpy().reshape(s)
            x = torch.from_numpy(us[i]).cuda()
            B.decompose(x)
            coeffs = x.cpu().numpy().astype(np.float64)
            assert np.array_equal(lab, O.quantize(coeffs, H, 0, t))
            exp = O.decompose(u, H)
            assert np.abs(coeffs - exp).max() <= tol32(H.L) * np.abs(u).max()
            deq = O.dequantize(lab, H, 0, t, dtype=np.float32).astype(np.float64)
            rec_o = O.recompose(deq, H)
            assert np.abs(rec_o - u).max() <= tau
            got = dec[i][1].numpy().reshape(s).astype(np.float64)
            assert np.abs(got - rec_o).max() <= tol32(H.L) * np.abs(u).max()
            assert np.abs(got - u).max() <= tau
    finally:
        srv.close()


def test_budget_admission(cuda):
    torch = cuda
    shape = (65, 65, 65)
    n = int(np.prod(shape))
    need = (n * 4 + n * 8) + B.mgard_workspace_size(shape, B.F32)
    srv = B.Server(hbm_budget=need + (1 << 20), slots=4)  # room for one request at a time
    try:
        field = torch.from_numpy(F.grf_field(shape, seed=9).ravel()).pin_memory()
        outs = [torch.empty(n, dtype=torch.int64).pin_memory() for _ in range(5)]
        ids = [srv.submit(B.OP_COMPRESS, shape, field, o, rel_bound=1e-3) for o in outs]
        srv.drain()
        res = srv.poll()
        assert sorted(r[0] for r in res) == sorted(ids) and all(r[1] == 0 for r in res)
        c = srv.counters()
        assert c["peak_running"] == 1 and c["peak_bytes"] <= need + (1 << 20)
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        big = torch.empty(1, dtype=torch.int64)
        with pytest.raises(B.MgardError):
            srv.submit(B.OP_COMPRESS, (257, 257, 257), big, big, rel_bound=1e-3)
    finally:
        srv.close()
