"""The C-ABI library loads and exports every symbol include/hgp.h declares (no GPU needed).

Only host-side functions are called (no compute): hgp_strerror and hgp_default_options.
The struct layouts of the Python binding are checked against the header by compiling a tiny
C program with gcc that prints sizeof/offsetof.
"""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hgp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2010_10272_gb300 import build as b
    b.build()
    import paper_2010_10272_gb300 as p
    return p.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hgp_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_host_only_functions(lib):
    import paper_2010_10272_gb300 as p
    assert p.strerror(0) == "ok"
    assert p.strerror(1) == "invalid argument"
    assert p.strerror(3) == "unsupported size or parameter"
    assert p.strerror(99) == "unknown status"
    o = p.default_options()
    assert o.subrounds == 4 and o.phi_width == 0 and o.seed == 0 and not o.cuda_stream
    # argument checks that return before any CUDA call
    assert lib.hgp_set_pool_retention(-1) == 1
    assert lib.hgp_batch_get_stats(None, 1, None) == 1
    assert lib.hgp_batch_query(None, None) == 1
    assert lib.hgp_batch_get_partitions(None, None, 0, None) == 1


def test_struct_layout_matches_header(lib):
    from paper_2010_10272_gb300.native import Options, Profile, RoundStats
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "hgp.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(hgp_options), offsetof(hgp_options, phi_width),
         offsetof(hgp_options, seed), offsetof(hgp_options, debug), offsetof(hgp_options, graph),
         offsetof(hgp_options, cuda_stream), offsetof(hgp_options, balance_moves),
         offsetof(hgp_options, revert_negative), offsetof(hgp_options, gain_ctas_per_sm),
         offsetof(hgp_options, apply_ctas_per_sm), sizeof(hgp_round_stats), sizeof(hgp_profile),
         offsetof(hgp_profile, launches));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        vals = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [ctypes.sizeof(Options), Options.phi_width.offset, Options.seed.offset,
            Options.debug.offset, Options.graph.offset, Options.cuda_stream.offset,
            Options.balance_moves.offset, Options.revert_negative.offset, Options.gain_ctas_per_sm.offset,
            Options.apply_ctas_per_sm.offset, ctypes.sizeof(RoundStats), ctypes.sizeof(Profile),
            Profile.launches.offset]
    assert vals == want


def test_missing_library_fails_loudly(monkeypatch):
    import paper_2010_10272_gb300.native as nat
    monkeypatch.setattr(nat, "_lib", None)
    monkeypatch.setattr(nat, "_LIB_PATH", "/nonexistent/libhgp.so")
    with pytest.raises(ImportError):
        nat.load_library()
