"""The C-ABI library builds, loads and exports every entry point that
include/sss.h declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_1305_1157_gb300 as sss
from paper_1305_1157_gb300 import build as sbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    sbuild.build()
    return sss.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "sss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sss_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sss_sort", "sss_sort_batched", "sss_sort_learned", "sss_workspace_size",
                     "sss_get_last_stats", "sss_last_error", "sss_set_options"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_python_binding_covers_every_symbol():
    for n in declared_functions():
        assert callable(getattr(sss, n)), n


def test_options_roundtrip_and_validation(lib):
    o = sss.sss_get_options()
    assert o.k_max == 10 and o.base_threshold == 128 and o.medium_threshold == 8192 and o.chunk == 32768
    assert o.key_bytes == 16 and o.classifier == 0
    bad = sss.sss_options.from_buffer_copy(o)
    bad.k_max = 11
    with pytest.raises(sss.SSSError) as e:
        sss.sss_set_options(bad)
    assert e.value.code == -1
    bad = sss.sss_options.from_buffer_copy(o)
    bad.chunk = 1000
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    bad = sss.sss_options.from_buffer_copy(o)
    bad.base_threshold = 256  # above the warp-tile base case
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    bad = sss.sss_options.from_buffer_copy(o)
    bad.medium_threshold = 64  # below base_threshold
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    bad = sss.sss_options.from_buffer_copy(o)
    bad.key_bytes = 12  # keys are one or two 8-byte words
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    bad = sss.sss_options.from_buffer_copy(o)
    bad.classifier = 2  # pS5-Unroll (0) or pS5-Equal (1)
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    assert o.alphabet == 0  # alphabet compression is off by default
    bad = sss.sss_options.from_buffer_copy(o)
    bad.alphabet = 2  # off (0) or on (1)
    with pytest.raises(sss.SSSError):
        sss.sss_set_options(bad)
    sss.sss_set_options(o)
    assert sss.sss_get_options().k_max == 10
    with pytest.raises(TypeError):
        sss.sss_set_options(medium_threshhold=4096)  # misspelt field: rejected, not ignored
    assert sss.sss_get_options().medium_threshold == o.medium_threshold


def test_empty_input_is_a_noop(lib):
    assert lib.sss_sort(None, None, 0, None, None, None) == 0


def test_null_pointers_are_rejected(lib):
    assert lib.sss_sort(None, None, 5, None, None, None) == -1
    assert "null" in sss.sss_last_error()


def test_bad_splitter_arguments_are_rejected(lib):
    assert lib.sss_build_splitters(None, 3, 0, None, None, None) == -1
    assert lib.sss_build_splitters(None, 100, 2, None, None, None) == -1
    assert lib.sss_classify(None, 4, None, None, 11, None, None) == -1


def test_batched_set_boundaries_are_checked_on_the_host(lib):
    import numpy as np
    P = ctypes.c_void_p
    for sb, n in (([1, 5, 10], 10),    # does not start at 0
                  ([0, 5, 9], 10),     # does not end at n
                  ([0, 6, 5, 10], 10)):  # decreases
        a = np.array(sb, dtype=np.uint64)
        rc = lib.sss_sort_batched(P(1), P(1), n, a.ctypes.data, len(sb) - 1, P(1), P(1), None)
        assert rc == -1, (sb, rc)
        assert "set_begin" in sss.sss_last_error()
    assert lib.sss_sort_batched(P(1), P(1), 10, None, 2, P(1), P(1), None) == -1


def test_workspace_size_grows_with_n(lib):
    a, b = sss.sss_workspace_size(1000), sss.sss_workspace_size(1_000_000)
    assert 0 < a < b
    assert b >= 24 * 1_000_000  # two key and two index arrays at least


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a struct of include/sss.h, from a C program
    compiled with the host compiler."""
    src = tmp_path / "layout.c"
    body = "\n".join(f'    printf("{f} %zu\\n", offsetof({struct}, {f}));' for f in fields)
    src.write_text(f"""#include <stdio.h>
#include <stddef.h>
#include "sss.h"
int main(void) {{
    printf("sizeof %zu\\n", sizeof({struct}));
{body}
    return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("cls", [sss.sss_options, sss.sss_stats, sss.sss_learned_stats])
def test_binding_structs_match_the_header_layout(cls, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no host C compiler")
    fields = [f for f, _ in cls._fields_]
    c = _c_layout(cls.__name__, fields, tmp_path)
    assert c["sizeof"] == ctypes.sizeof(cls)
    for f in fields:
        assert c[f] == getattr(cls, f).offset, f
