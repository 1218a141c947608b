"""The C-ABI library loads and exports every entry point that include/pc.h declares.

No compute call is made, so this runs without a GPU.
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("pc_compress", "pc_decompress", "pc_train", "pc_quantize", "pc_compress_host",
                 "pc_decompress_host", "pc_header_info", "pc_decompress_noalloc", "pc_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    from paper_2309_09778_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    del __graft_entry__
