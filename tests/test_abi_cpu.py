"""The C ABI library builds, loads and exports every declared symbol; host-side
argument checks return before any CUDA call (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_04865_gb300 import _abi, build_lib
    build_lib.build()
    return _abi.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "msf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msf_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    from paper_2110_04865_gb300 import _abi
    names = declared_functions()
    assert set(names) == set(_abi.EXPORTS)
    for name in names:
        assert hasattr(lib, name), name


def test_host_side_argument_checks(lib):
    from paper_2110_04865_gb300 import _abi
    out = ctypes.c_void_p()
    assert lib.msf_build_csr(-1, 0, None, None, None, None, 0, 0, None, ctypes.byref(out)) == 1
    assert lib.msf_build_csr(5, 0, None, None, None, None, 7, 0, None, ctypes.byref(out)) == 1
    assert lib.msf_build_csr(5, 0, None, None, None, None, 0, 3, None, ctypes.byref(out)) == 1
    assert lib.msf_build_csr(1 << 31, 0, None, None, None, None, 0, 0, None, ctypes.byref(out)) == 6
    assert lib.msf_build_csr(5, (1 << 32) - 1, None, None, None, None, 0, 0, None, ctypes.byref(out)) == 6
    assert lib.msf_build_csr(5, 3, None, None, None, None, 0, 0, None, ctypes.byref(out)) == 1
    assert b"NULL" in lib.msf_last_error()
    assert lib.msf_build_csr(5, 0, None, None, None, None, 0, 0, None, None) == 1
    assert lib.msf_compute(None, None, None, None, None) == 1
    assert lib.msf_compute_batched(-1, None, None, None, None, None, 0, None, None, None, None) == 1
    assert lib.msf_compute_batched(0, None, None, None, None, None, 0, None, None, None, None) == 0
    assert lib.msf_weight_backward(10, 0, None, None, None, None, None) == 1
    assert lib.msf_weight_backward(0, 1, None, None, None, None, None) == 0


def test_options_round_trip(lib):
    from paper_2110_04865_gb300 import _abi
    old = _abi.msf_get_option(_abi.OPT_COMPACT_TAU)
    _abi.msf_set_option(_abi.OPT_COMPACT_TAU, 0.25)
    assert _abi.msf_get_option(_abi.OPT_COMPACT_TAU) == 0.25
    _abi.msf_set_option(_abi.OPT_COMPACT_TAU, old)
    with pytest.raises(_abi.MsfError):
        _abi.msf_set_option(_abi.OPT_SLOTS_PER_LANE, 5)
    for opt, good, bad in ((_abi.OPT_PREFETCH, 0, 2), (_abi.OPT_EXEC_MODE, 1, 3), (_abi.OPT_BLOCKS_PER_SM, 2, 9),
                           (_abi.OPT_SWEEP, 1, 3), (_abi.OPT_BUILD, 3, 4),
                           (_abi.OPT_HOST_INPUT, 1, 2), (_abi.OPT_RELABEL, 0, 2)):
        prev = _abi.msf_get_option(opt)
        _abi.msf_set_option(opt, good)
        assert _abi.msf_get_option(opt) == good
        with pytest.raises(_abi.MsfError):
            _abi.msf_set_option(opt, bad)
        _abi.msf_set_option(opt, prev)
    with pytest.raises(_abi.MsfError):
        _abi.msf_set_option(99, 1)
    assert _abi.msf_get_option(99) == -1.0


def test_stats_struct_matches_the_header(tmp_path):
    """The ctypes mirror of msf_stats has the header's fields, in order, at
    the offsets a C compiler gives them, and the same size."""
    import shutil
    import subprocess
    from paper_2110_04865_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    text = open(os.path.join(ROOT, "include", "msf.h")).read()
    body = re.search(r"typedef struct msf_stats \{(.*?)\} msf_stats;", text, flags=re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [x.strip() for x in decl.split(None, 1)[1].split(",")]
    assert names == [f for f, _ in _abi.Stats._fields_]
    src = tmp_path / "stats.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "msf.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(msf_stats));']
    lines += [f'  printf("%zu\\n", offsetof(msf_stats, {n}));' for n in names]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "stats"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got[0] == ctypes.sizeof(_abi.Stats)
    assert got[1:] == [getattr(_abi.Stats, n).offset for n in names]
