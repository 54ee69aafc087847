"""Host-side checks of the C ABI that need no GPU: the library builds and
exports every symbol its header declares, and the host-only entry points
(hierarchy depth, workspace size, level tolerances, argument errors) agree
with the oracle and the header."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import mgard_oracle as O
from paper_2010_05872_gb300 import binding as B
from paper_2010_05872_gb300 import build as build_mod
from paper_2010_05872_gb300 import fields as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return B.lib()


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mgard_\w+)\s*\(", text))
    return sorted(names)


def test_header_symbols_exported(lib):
    declared = _declared_symbols()
    assert "mgard_decompose" in declared and "mgard_quantize" in declared
    for name in declared:
        assert hasattr(lib, name), name
        ctypes.cast(getattr(lib, name), ctypes.c_void_p)
    assert sorted(B.exported_symbols()) == declared


@pytest.mark.parametrize("dims", [(3,), (4,), (9,), (10,), (65, 65, 65), (500, 500, 100),
                                  (513, 513, 513), (33, 257, 100), (1025, 4096)])
def test_num_levels_matches_oracle(lib, dims):
    assert B.mgard_num_levels(dims) == O.Hierarchy(dims).L


def test_workspace_size(lib):
    for dims in [(65, 65, 65), (500, 500, 100), (10,), (17, 12)]:
        H = O.Hierarchy(dims)
        for dtype, es in ((B.F32, 4), (B.F64, 8)):
            need = 2 * es * sum(int(np.prod(H.levels[l])) for l in range(H.L))
            got = B.mgard_workspace_size(dims, dtype)
            assert need <= got <= need + 2 * 256 * (H.L + 1)
            assert got % 256 == 0


@pytest.mark.parametrize("dims,kind,stop", [((65, 65, 65), "u", 0), ((500, 500, 100), "z", 3),
                                            ((500, 500, 100), "z", 0), ((33,), "g", 0),
                                            ((20, 17), "g", 1), ((9, 9, 9), "u", 2)])
def test_level_tolerances_match_oracle(lib, dims, kind, stop):
    if kind == "u":
        coords = None
    elif kind == "z":
        coords = [None] * (len(dims) - 1) + [F.geometric_coords(dims[-1], 1.03)]
    else:
        coords = [F.geometric_coords(n, 1.05) for n in dims]
    tau = 1e-3
    got = B.mgard_level_tolerances(dims, coords, stop, tau)
    exp = O.level_tolerances(O.Hierarchy(dims, coords), stop, tau)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=0)


def _rc(fn, *args):
    try:
        fn(*args)
    except B.MgardError as e:
        return e.code
    return 0


def test_argument_errors(lib):
    assert _rc(B.mgard_num_levels, (2, 5)) == -2
    assert _rc(B.mgard_num_levels, (5, 5, 5, 5)) == -2
    assert _rc(B.mgard_level_tolerances, (9, 9), None, 3, 1.0) == -4
    assert _rc(B.mgard_level_tolerances, (9, 9), None, 0, 0.0) == -1
    assert _rc(B.mgard_level_tolerances, (9, 9), None, 0, float("nan")) == -1
    bad = [np.array([0, 1, 2, 2, 3, 4, 5, 6, 7.0]), None]
    assert _rc(B.mgard_level_tolerances, (9, 9), bad, 0, 1.0) == -3
    assert _rc(B.mgard_workspace_size, (9, 9), 7) == -1
    # Shape and dtype errors of the device entry points are reported before
    # any CUDA call.
    assert B.mgard_decompose((2, 9), None, B.F32, 0, 0, 0, 0, 0) == -2
    assert B.mgard_recompose((9, 9), None, 5, 0, 0, 0, 0, 0) == -1
    assert lib.mgard_error_string(-5).decode().startswith("workspace")


def test_axis_length_limits(lib):
    """The last (contiguous) axis may have up to 2^30 nodes, every other
    axis up to 2^18 (they index CUDA grid dimensions); one more is a shape
    error, found on the host."""
    assert _rc(B.mgard_num_levels, (3, 2 ** 30)) == 0
    assert _rc(B.mgard_num_levels, (3, 2 ** 30 + 1)) == -2
    assert _rc(B.mgard_num_levels, (2 ** 18, 3)) == 0
    assert _rc(B.mgard_num_levels, (2 ** 18 + 1, 3)) == -2
    assert _rc(B.mgard_num_levels, (3, 2 ** 18 + 1, 3)) == -2
    assert _rc(B.mgard_num_levels, (2 ** 30,)) == 0
    assert _rc(B.mgard_num_levels, (2 ** 30 + 1,)) == -2


@pytest.mark.parametrize("dims,kind", [((33, 20, 17), "u"), ((10, 17, 9), "g"), ((1000,), "g"),
                                       ((70, 45), "u")])
def test_level_grid_matches_oracle(lib, dims, kind):
    coords = None if kind == "u" else [F.geometric_coords(n, 1.03) for n in dims]
    H = O.Hierarchy(dims, coords)
    for level in range(H.L + 1):
        shape, axes = B.level_grid(dims, coords, level)
        assert shape == H.levels[level]
        for d in range(len(dims)):
            np.testing.assert_array_equal(axes[d], H.coords[level][d])


@pytest.mark.parametrize("dims,kind,stop", [((33, 20, 17), "u", 0), ((10, 17, 9), "g", 1),
                                            ((1000,), "g", 2), ((70, 45), "u", 0)])
@pytest.mark.parametrize("mode", ["geometric", "linf_optimal", "l2"])
def test_level_tolerance_modes_match_oracle(lib, dims, kind, stop, mode):
    coords = None if kind == "u" else [F.geometric_coords(n, 1.03) for n in dims]
    H = O.Hierarchy(dims, coords)
    stop = min(stop, H.L)
    got = B.mgard_level_tolerances_mode(dims, coords, stop, 0.7, mode)
    exp = O.level_tolerances_mode(H, stop, 0.7, mode)
    np.testing.assert_allclose(got, exp, rtol=1e-12)


@pytest.mark.parametrize("dims", [(3, 3, 3, 3), (9, 5, 7, 6), (17, 17, 17, 17), (33, 9, 100, 12),
                                  (115, 69, 69, 288)])
def test_levels_4d_match_oracle(lib, dims):
    assert B.mgard_num_levels_4d(dims) == O.Hierarchy(dims).L


def test_workspace_size_4d(lib):
    for dims in [(9, 5, 7, 6), (17, 17, 17, 17), (33, 9, 10, 12)]:
        H = O.Hierarchy(dims)
        for dtype, es in ((B.F32, 4), (B.F64, 8)):
            need = es * (2 * int(np.prod(dims)) + int(np.prod(H.levels[max(H.L - 1, 0)]))
                         + sum(int(np.prod(H.levels[l])) for l in range(H.L)))
            got = B.mgard_workspace_size_4d(dims, dtype)
            assert need <= got <= need + 256 * (H.L + 4)
            assert got % 256 == 0


@pytest.mark.parametrize("dims,kind,stop", [((9, 9, 9, 9), "u", 0), ((17, 9, 10, 9), "g", 1),
                                            ((12, 17, 9, 33), "g", 0), ((9, 5, 7, 6), "u", 1)])
def test_level_tolerances_4d_match_oracle(lib, dims, kind, stop):
    coords = None if kind == "u" else [F.geometric_coords(n, 1.04 + 0.01 * d) for d, n in enumerate(dims)]
    got = B.mgard_level_tolerances_4d(dims, coords, stop, 1e-3)
    exp = O.level_tolerances(O.Hierarchy(dims, coords), stop, 1e-3)
    np.testing.assert_allclose(got, exp, rtol=1e-12, atol=0)


def test_argument_errors_4d(lib):
    assert _rc(B.mgard_num_levels_4d, (2, 5, 5, 5)) == -2
    assert _rc(B.mgard_level_tolerances_4d, (9, 9, 9, 9), None, 3, 1.0) == -4
    assert _rc(B.mgard_level_tolerances_4d, (9, 9, 9, 9), None, 0, -1.0) == -1
    bad = [None, np.array([0, 1, 2, 2, 3, 4, 5, 6, 7.0]), None, None]
    assert _rc(B.mgard_level_tolerances_4d, (9, 9, 9, 9), bad, 0, 1.0) == -3
    assert _rc(B.mgard_workspace_size_4d, (9, 9, 9, 9), 3) == -1
    with pytest.raises(ValueError):
        B.mgard_num_levels_4d((9, 9, 9))
    # Shape and dtype errors are reported before any CUDA call.
    assert B.mgard_decompose_4d((9, 2, 9, 9), None, B.F32, 0, 0, 0, 0, 0) == -2
    assert B.mgard_recompose_4d((9, 9, 9, 9), None, 5, 0, 0, 0, 0, 0) == -1


def test_node_limit_4d(lib):
    # 4D grids index in 32 bits: 2^31 nodes or more is a shape error.
    assert _rc(B.mgard_num_levels_4d, (2048, 1024, 1024, 3)) == -2
    assert B.mgard_num_levels_4d((1024, 1024, 682, 3)) == O.Hierarchy((1024, 1024, 682, 3)).L
    assert _rc(B.mgard_workspace_size_4d, (1024, 1024, 1024, 3), B.F32) == -2


@pytest.mark.parametrize("seed", range(5))
def test_huffman_lengths_match_oracle(lib, seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 3000))
    counts = rng.integers(0, 1000, n) * (rng.random(n) < 0.6)
    counts[rng.integers(0, n)] = 5   # at least one used symbol
    got = B.huffman_lengths(counts)
    assert list(got) == O.huffman_lengths(list(counts))


def test_huffman_lengths_special_cases(lib):
    assert list(B.huffman_lengths([45, 13, 12, 16, 9, 5])) == [1, 3, 3, 3, 4, 4]
    assert list(B.huffman_lengths([0, 0, 7, 0])) == [0, 0, 1, 0]
    assert list(B.huffman_lengths([0, 0])) == [0, 0]
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    got = B.huffman_lengths(fib)
    assert list(got) == O.huffman_lengths(fib) and max(got) <= 31
    assert _rc(B.huffman_lengths, np.zeros(65537)) == -1


@pytest.mark.parametrize("dims,stop", [((5,), 0), ((33, 20, 17), 1), ((65, 65, 65), 0)])
def test_cost_model_matches_oracle(lib, dims, stop):
    H = O.Hierarchy(dims)
    taus = O.level_tolerances(H, stop, 1e-3)
    got = B.cost_model(dims, stop, taus, 3.5)
    np.testing.assert_allclose(got, O.cost_model(H, stop, taus, 3.5), rtol=1e-12)
    assert _rc(B.cost_model, dims, stop, taus, 0.0) == -1


def test_huffman_bound(lib):
    assert B.huffman_bound(0) >= 16 + 32817
    for n in (1, 1024, 10 ** 6):
        nch = (n + 1023) // 1024
        # header, chunk table, and at most 31 code + 63 extra bits per label
        assert B.huffman_bound(n) >= 16 + 32817 + 4 * nch + (n * 94 + 7) // 8


def test_device_helpers_refuse_cpu_tensors(lib):
    # There is no CPU path: the tensor helpers raise before any call.
    import torch
    x = torch.zeros(1000, dtype=torch.int64)
    for fn in (B.huffman_encode, B.label_entropy, B.pack_labels):
        with pytest.raises(ValueError):
            fn(x)
    with pytest.raises(ValueError):
        B.decompose_4d(torch.zeros((3, 3, 3, 3)))


def _declared_prototypes():
    """name -> (return type, parameter count) from the header's prototypes."""
    out = {}
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"([A-Za-z_][\w \*]*?)\b(mgard_\w+)\s*\(([^;{]*?)\)\s*;", text, re.S):
            ret, name, params = m.group(1).strip(), m.group(2), " ".join(m.group(3).split())
            plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
            out[name] = (ret, len(plist), plist)
    return out


def _ctype_matches(param, ct):
    """Whether a ctypes argument type fits a C parameter declaration."""
    if "*" in param:
        return ct in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(ct, "_type_") and \
            issubclass(ct, ctypes._Pointer)
    base = param.replace("const ", "").split()[0]
    return {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "size_t": ctypes.c_size_t,
            "double": ctypes.c_double, "uint64_t": ctypes.c_uint64}.get(base) is ct


def test_binding_signatures_match_header(lib):
    # A ctypes argument list that disagrees with the C prototype would pass
    # garbage silently; every binding signature must have the header's arity
    # and return kind.
    protos = _declared_prototypes()
    assert set(protos) == set(B.exported_symbols())
    for name, (res, args) in B._SIGNATURES.items():
        ret, n, plist = protos[name]
        assert len(args) == n, (name, len(args), n)
        for param, ct in zip(plist, args):
            assert _ctype_matches(param, ct), (name, param, ct)
        if ret.startswith("const char"):
            assert res is ctypes.c_char_p, name
        elif ret == "int64_t":
            assert res is ctypes.c_int64, name
        else:
            assert ret == "int" and res is ctypes.c_int, (name, ret)


def test_product_never_reaches_the_oracle():
    # The oracle is test infrastructure: the package (binding, build, inputs)
    # and the CUDA sources neither import nor name it, and bench.py imports
    # it only in its oracle leg (the CPU baseline, the reference arm and the
    # comparison of the benchmarked results with the oracle).
    pkg = os.path.join(ROOT, "paper_2010_05872_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "mgard_oracle" not in text, f
    # Nor does the oracle import the product (it shares no code with it).
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2010_05872_gb300" not in text and "libmgardgb" not in text, f
    bench = open(os.path.join(ROOT, "bench.py")).read()
    imports = [m.start() for m in re.finditer(r"(from|import) oracle\b", bench)]
    assert len(imports) == 2
    start = bench.index("# ------------------------------------------------------------ oracle leg ---")
    end = bench.index("# ---------------------------------------------------------------- clocks ---")
    assert all(start < i < end for i in imports)


def test_host_plans_build_the_same_from_many_threads(lib):
    """The host-only calls build their operator tables per call: eight
    threads asking at once for the tolerances of mixed shapes and
    coordinates get what one thread gets."""
    import threading
    rng = np.random.default_rng(5)
    cases = []
    for i in range(24):
        dims = tuple(int(v) for v in rng.integers(3, 90, size=1 + i % 3))
        coords = None
        if i % 2:
            coords = [np.cumsum(rng.uniform(0.5, 1.5, n)) for n in dims]
        cases.append((dims, coords, i % 3, 10.0 ** -(1 + i % 4)))

    def run(case):
        dims, coords, stop, tau = case
        stop = min(stop, B.mgard_num_levels(dims))
        return B.mgard_level_tolerances(dims, coords, stop, tau)

    want = [run(c) for c in cases]
    got = [None] * len(cases)

    def worker(q):
        for k in range(q, len(cases), 8):
            got[k] = run(cases[k])

    threads = [threading.Thread(target=worker, args=(q,)) for q in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for w, g in zip(want, got):
        assert np.array_equal(np.asarray(w), np.asarray(g))
