"""The C-ABI library loads and exports every entry point the header declares;
host-only calls (geometry generation) agree with the oracle bit for bit. No
device work runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(fs_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding as B
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) > 20
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2002_11401_b300 import binding as B
    assert set(B.EXPORTS) == _declared()


def test_hash_init_is_fnv_offset_basis(lib):
    assert lib.fs_hash_init() == 0xcbf29ce484222325


@pytest.mark.parametrize("kind,n", [(I.SQUARE, 16), (I.PINWHEEL, 9), (I.KAGOME, 29),
                                    (I.KAGOME, 7), (3, 8), (4, 25), (5, 6), (6, 11)])
def test_geometry_matches_oracle_bitwise(lib, oracle, kind, n):
    from paper_2002_11401_b300 import binding as B
    sim = B.Sim.geometry(kind, n, n + 1)
    x, y, t = sim.geometry_arrays()
    ox, oy, ot = oracle.geometry(kind, n, n + 1)
    np.testing.assert_array_equal(x, ox)
    np.testing.assert_array_equal(y, oy)
    np.testing.assert_array_equal(t, ot)


def test_bad_arguments_are_rejected(lib):
    from paper_2002_11401_b300 import binding as B
    with pytest.raises(B.FsError):
        B.Sim.geometry(7, 4, 4)
    with pytest.raises(B.FsError):
        B.Sim.geometry(I.SQUARE, 0, 4)
    with pytest.raises(B.FsError):
        B.Sim.custom([0.0, np.nan], [0.0, 1.0], [0.0, 0.0])
    sim = B.Sim.geometry(I.SQUARE, 2, 2)
    # calls that need parameters fail with FS_ERR_STATE before any device work
    h = ctypes.c_uint64(0)
    nf = ctypes.c_int64(0)
    st = lib.fs_run_protocol(sim.handle, None, None, 0, 0, 1, None, None, 0, None,
                             ctypes.byref(h), ctypes.byref(nf))
    assert st == B.FS_ERR_STATE
    assert b"parameters" in lib.fs_last_error(sim.handle)


def test_workspace_calls_reject_bad_arguments_on_the_host(lib):
    """fs_workspace_bytes and fs_bind_workspace check their arguments before any
    device work: NULL handles and outputs, parameters out of range, a buffer that
    does not start on a 256-byte boundary."""
    from paper_2002_11401_b300 import binding as B
    sim = B.Sim.geometry(I.SQUARE, 2, 2)
    out = ctypes.c_size_t(7)
    p = B.make_params(alpha=1e-3)
    assert lib.fs_workspace_bytes(sim.handle, ctypes.byref(p), None) == B.FS_ERR_INVALID
    assert lib.fs_workspace_bytes(sim.handle, None, ctypes.byref(out)) == B.FS_ERR_INVALID
    bad = B.make_params(alpha=1e-3, cutoff=-1.0)
    assert lib.fs_workspace_bytes(sim.handle, ctypes.byref(bad), ctypes.byref(out)) == \
        B.FS_ERR_INVALID
    assert out.value == 0
    assert b"out of range" in lib.fs_last_error(sim.handle)
    assert lib.fs_bind_workspace(None, None, 0, None) == B.FS_ERR_INVALID
    assert lib.fs_bind_workspace(sim.handle, ctypes.c_void_p(0x1000 + 16), 1 << 20,
                                 None) == B.FS_ERR_INVALID
    assert b"256-byte" in lib.fs_last_error(sim.handle)
    # NULL returns to the pool: always allowed before the parameters are set
    assert lib.fs_bind_workspace(sim.handle, None, 0, None) == B.FS_OK


@pytest.mark.parametrize("kind,period,angle", [(0, 8, 0.0), (0, 13, 70.0), (1, 5, 30.0),
                                               (1, 40, 200.0), (2, 12, 15.0), (2, 7, -40.0)])
def test_encoders_match_oracle(lib, oracle, kind, period, angle):
    """fs_encode is host arithmetic: the same values as the oracle's encoder, to the
    last bit or one rounding apart."""
    from paper_2002_11401_b300 import binding as B
    u = np.array([0.0, 0.3, 1.0, 0.77])
    hx, hy = B.encode(kind, u, period, 0.05, 0.3, angle)
    ox, oy = oracle.encode(kind, u, period, 0.05, 0.3, angle)
    np.testing.assert_allclose(hx, ox, rtol=2e-16, atol=1e-17)
    np.testing.assert_allclose(hy, oy, rtol=2e-16, atol=1e-17)
    with pytest.raises(B.FsError):
        B.encode(1, u, 1, 0.0, 0.1, 0.0)  # a sawtooth needs two values per period
    with pytest.raises(B.FsError):
        B.encode(5, u, 4, 0.0, 0.1, 0.0)


def test_series_and_correlation_need_parameters(lib):
    from paper_2002_11401_b300 import binding as B
    sim = B.Sim.geometry(I.SQUARE, 3, 3)
    with pytest.raises(B.FsError) as e:
        sim.set_field_local(np.zeros((2, sim.n)), np.zeros((2, sim.n)))
    assert e.value.code == B.FS_ERR_STATE
    with pytest.raises(B.FsError) as e:
        sim.set_sigma_series([0.1, 0.2])
    assert e.value.code == B.FS_ERR_STATE
    with pytest.raises(B.FsError) as e:
        sim.correlation(3.0, 0.5, 8)
    assert e.value.code == B.FS_ERR_STATE
    p = B.make_params(alpha=1e-3, criterion=3)
    assert lib.fs_workspace_bytes(sim.handle, ctypes.byref(p), ctypes.byref(ctypes.c_size_t())) \
        == B.FS_ERR_INVALID


def _header_fields(src, name):
    """Field names of `typedef struct { ... } name;` in declaration order."""
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        # "type a" or "type a, b" (no arrays or function pointers in these structs)
        first, *others = [p.strip() for p in decl.split(",")]
        fields += [n.lstrip("*") for n in [first.rpartition(" ")[2]] + others]
    return fields


@pytest.mark.parametrize("name", ["fs_params", "fs_info", "fs_profile", "fs_request",
                                  "fs_result"])
def test_binding_structs_match_the_header_layout(name, tmp_path):
    """Each ctypes struct of the binding has the header's fields in its order, and
    gcc's sizeof and offsetof of the header's struct equal ctypes' own."""
    import shutil
    import subprocess

    from paper_2002_11401_b300 import binding as B

    hdr = os.path.join(ROOT, "include", "flatspin_b300.h")
    src = re.sub(r"/\*.*?\*/", "", open(hdr).read(), flags=re.S)
    want = _header_fields(src, name)
    cls = getattr(B, name)
    assert [f[0] for f in cls._fields_] == want
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    prog = tmp_path / "layout.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{hdr}"',
             "int main(void) {", f'  printf("%zu\\n", sizeof({name}));']
    lines += [f'  printf("%zu\\n", offsetof({name}, {f}));' for f in want]
    lines += ["  return 0;", "}"]
    prog.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", str(prog), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(cls)
    assert out[1:] == [getattr(cls, f).offset for f in want]
