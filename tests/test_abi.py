"""The C-ABI library builds, loads and exports every function include/rsrr.h
declares (no compute call: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rsrr.h")
LIB = os.path.join(ROOT, "paper_1605_07951_gb300", "librsrr.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(rsrr_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1605_07951_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("rsrr_create", "rsrr_sample", "rsrr_project", "rsrr_solve",
                     "rsrr_set_probe", "rsrr_get_samples", "rsrr_get_Q", "rsrr_get_projected",
                     "rsrr_get_stats", "rsrr_destroy", "rsrr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (rsrr_\w+)", out))
    assert set(declared_functions()) <= exported


def test_binding_uses_the_same_names(lib):
    from paper_1605_07951_gb300 import rsrr
    for name in declared_functions():
        assert callable(getattr(rsrr, name)), name


def test_struct_layouts_match_the_header(lib):
    from paper_1605_07951_gb300 import rsrr
    assert ctypes.sizeof(rsrr.rsrr_c128) == 16
    assert ctypes.sizeof(rsrr.rsrr_fn) == 48
    assert ctypes.sizeof(rsrr.rsrr_region) == 48
    # defaults come from the library itself
    o = rsrr.default_opts()
    assert o.precision == rsrr.RSRR_PREC_MIXED and o.eta_tol == 1e-10 and o.delta == 1e-14
    assert o.NQ == 500 and o.KQ == 2 and o.tol_gap == 1e3


def test_create_rejects_bad_descriptors_without_touching_the_gpu(lib):
    import numpy as np
    from paper_1605_07951_gb300 import rsrr
    import workloads as W
    p = W.random_banded(n=40, kl=2, ku=2, N=2, L=2)
    p.col_idx = p.col_idx.copy()
    p.col_idx[3] = 10_000  # column out of range
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.Solver(p)
    assert e.value.status == rsrr.RSRR_EINVAL
    p = W.random_banded(n=40, kl=2, ku=2, N=2, L=2)
    p.region.a = -1.0
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.Solver(p)
    assert e.value.status == rsrr.RSRR_EINVAL


def test_ctypes_structs_match_the_c_compiler(tmp_path):
    """sizeof and every field offset of the public structs, as gcc sees the
    header, against the binding's ctypes mirrors."""
    from paper_1605_07951_gb300 import rsrr
    structs = [rsrr.rsrr_opts, rsrr.rsrr_stats, rsrr.rsrr_nep, rsrr.rsrr_region,
               rsrr.rsrr_result, rsrr.rsrr_fn]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rsrr.h"', 'int main(void) {']
    for st in structs:
        name = st.__name__
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append('return 0; }')
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, val = line.split()
        st = getattr(rsrr, name)
        want = ctypes.sizeof(st) if field == "size" else getattr(st, field).offset
        assert int(val) == want, (name, field, int(val), want)
        seen += 1
    assert seen == sum(len(s._fields_) + 1 for s in structs)


def test_ctypes_structs_match_the_c_layouts(lib, tmp_path):
    """sizeof and field offsets of every struct the binding mirrors, as the C
    compiler lays them out from include/rsrr.h."""
    from paper_1605_07951_gb300 import rsrr
    structs = ["rsrr_c128", "rsrr_fn", "rsrr_nep", "rsrr_region", "rsrr_opts", "rsrr_stats",
               "rsrr_result", "rsrr_server_opts", "rsrr_reply", "rsrr_server_stats"]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rsrr.h"', "int main(void) {"]
    for s in structs:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f, _ in getattr(rsrr, s)._fields_:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        s, f, v = line.split()
        cls = getattr(rsrr, s)
        got = ctypes.sizeof(cls) if f == "size" else getattr(cls, f).offset
        assert got == int(v), (s, f, got, v)


def test_estimate_bytes_needs_no_gpu_and_counts_the_resident_buffers(lib):
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    p = W.config("c1")
    b = rsrr.estimate_bytes(p)
    kl = ku = 200
    band = (2 * kl + ku + 32) * p.n * p.N * 8        # complex64 factors of all points
    samples = 16 * p.n * p.N * p.L                   # S in complex128
    assert band + 3 * samples <= b <= 3 * (band + 3 * samples)
    assert rsrr.estimate_bytes(p, N=32) < b
    fp64 = rsrr.estimate_bytes(p, rsrr.default_opts(precision=rsrr.RSRR_PREC_FP64))
    assert fp64 > b  # complex128 factors
    bad = W.config("c1")
    bad.row_ptr = bad.row_ptr.copy()
    bad.row_ptr[0] = 1
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.estimate_bytes(bad)
    assert e.value.status == rsrr.RSRR_EINVAL


def test_create_refuses_a_handle_above_its_memory_budget(lib):
    """mem_budget_bytes is checked against rsrr_estimate_bytes before any
    device memory is touched."""
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    p = W.config("c1")
    need = rsrr.estimate_bytes(p)
    with pytest.raises(rsrr.RSRRError) as e:
        rsrr.Solver(p, rsrr.default_opts(mem_budget_bytes=need - 1))
    assert e.value.status == rsrr.RSRR_ENOMEM
    assert "mem_budget_bytes" in str(e.value)


def test_chunked_band_storage_is_smaller(lib):
    """opts.chunk_points holds the band factor storage of a chunk of points
    (rsrr_estimate_bytes counts it without a GPU)."""
    import workloads as W
    from paper_1605_07951_gb300 import rsrr
    p = W.rational_grid(g=40, N=16, L=4)
    full = rsrr.estimate_bytes(p)
    ch = [rsrr.estimate_bytes(p, rsrr.default_opts(chunk_points=c)) for c in (1, 4, 16, 64)]
    assert ch[0] < ch[1] < ch[2] == ch[3] == full
