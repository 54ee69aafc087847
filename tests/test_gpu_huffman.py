"""GPU parity of the labels' Huffman stage and entropy with the oracle:
streams byte-identical to the oracle's, decoding of the oracle's streams,
the entropy within 1e-12 relative, round trips of real labels, and invalid
streams refused."""
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


def _labels(n, seed, p=0.08):
    rng = np.random.default_rng(seed)
    x = (rng.geometric(p, n) - 1) * rng.choice([-1, 1], n)
    if n > 20:
        x[1] = 2 ** 62
        x[n - 1] = -2 ** 63
        x[n // 2] = 2 ** 63 - 1
        x[7] = 16383      # zigzag 32766, a direct symbol
        x[9] = -16385     # zigzag 32769: bit length 16, 15 extra bits
        x[11] = 10 ** 6
    return x.astype(np.int64)


@pytest.mark.parametrize("n", [0, 1, 2, 1023, 1024, 1025, 5000])
def test_huffman_stream_matches_oracle(cuda, n):
    torch = cuda
    x = _labels(n, 10 + n)
    d = torch.from_numpy(x).cuda()
    s = B.huffman_encode(d)
    exp = O.huffman_encode(x)
    assert bytes(s.cpu().numpy().tobytes()) == exp
    # The oracle's stream decodes on the GPU.
    back = B.huffman_decode(torch.frombuffer(bytearray(exp), dtype=torch.uint8).cuda(), n)
    assert np.array_equal(back.cpu().numpy(), x)


def test_huffman_single_symbol_and_all_large(cuda):
    torch = cuda
    for x in (np.full(3000, -3, dtype=np.int64),
              np.arange(40000, 42000, dtype=np.int64) * 7):
        d = torch.from_numpy(x).cuda()
        s = B.huffman_encode(d)
        assert bytes(s.cpu().numpy().tobytes()) == O.huffman_encode(x)
        assert np.array_equal(B.huffman_decode(s, x.size).cpu().numpy(), x)


@pytest.mark.parametrize("n", [0, 1, 5000, 100000])
def test_label_entropy_matches_oracle(cuda, n):
    torch = cuda
    x = _labels(n, 99 + n, p=0.01)
    h = B.label_entropy(torch.from_numpy(x).cuda())
    assert h == pytest.approx(O.label_entropy(x), rel=1e-12, abs=1e-15)


def test_huffman_round_trip_of_field_labels(cuda):
    """Labels of a decomposed k^-5/3 field at four bounds: exact round trip,
    the stream within one bit per label of the entropy, and smaller than
    the bit-packed stream."""
    torch = cuda
    dims = (129, 129, 129)
    u = torch.from_numpy(F.grf_field(dims, seed=F.SEED_LARGE)).cuda()
    lo, hi = B.value_range(u)
    for rel in (1e-2, 1e-3, 1e-4, 1e-5):
        x = u.clone()
        B.decompose(x)
        labels, _ = B.quantize(x, rel * (hi - lo))
        flat = labels.reshape(-1)
        s = B.huffman_encode(flat)
        back = B.huffman_decode(s, flat.numel())
        assert torch.equal(back, flat)
        h = B.label_entropy(flat)
        # Within one bit per label of the entropy plus the extra bits of
        # the large codes (bounded by 64 per label past 2^15), the header
        # and one word per chunk.
        z = torch.where(flat >= 0, 2 * flat, -2 * flat - 1)
        big = z >= 32768
        nbig = int(big.sum().item())
        extra = 63 * nbig
        nchunks = (flat.numel() + 1023) // 1024
        assert 8 * s.numel() <= flat.numel() * (h + 1.0) + extra + 8 * (16 + 32817 + 7 + 4 * nchunks + 8) \
            + 64 * nchunks
        assert s.numel() < B.pack_labels(flat).numel()


def test_huffman_invalid_streams_refused(cuda):
    torch = cuda
    x = _labels(5000, 3)
    s = B.huffman_encode(torch.from_numpy(x).cuda())
    with pytest.raises(B.MgardError) as e:
        B.huffman_decode(s, 4999)                # count does not match
    assert e.value.code == -1
    with pytest.raises(B.MgardError) as e:
        B.huffman_decode(s[:-8], 5000)           # truncated
    assert e.value.code == -1
    bad = s.clone()
    bad[12] = 40                                 # longest code length > 31
    with pytest.raises(B.MgardError) as e:
        B.huffman_decode(bad, 5000)
    assert e.value.code == -1
    bad = s.clone()
    bad[16] = 1                                  # over-full code (Kraft sum > 1)
    bad[17] = 1
    bad[18] = 1
    with pytest.raises(B.MgardError) as e:
        B.huffman_decode(bad, 5000)
    assert e.value.code == -1


def test_huffman_capacity_checked_before_writing(cuda):
    """A destination smaller than the stream is refused (MGARD_ERR_WORKSPACE)
    and nothing is written past it."""
    import ctypes
    torch = cuda
    n = 5000
    x = torch.from_numpy(_labels(n, 21)).cuda()
    full = B.huffman_encode(x).numel()
    for cap in (100, full - 8):
        buf = torch.full((cap + 4096,), 0xA5, dtype=torch.uint8, device="cuda")
        nb = ctypes.c_size_t()
        rc = B.lib().mgard_huffman_encode(n, x.data_ptr(), buf.data_ptr(), cap, ctypes.byref(nb), 0)
        torch.cuda.synchronize()
        assert rc == -5
        assert bool((buf[cap:] == 0xA5).all().item())
