"""The C-ABI library builds, loads and exports every function include/ann.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ann.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(ann_[a-z_0-9]+)\s*\(", src, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("ann_index_create", "ann_index_destroy", "ann_search", "ann_search_ex",
                 "ann_search_host", "ann_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2201_13007_gb300 import _build
    path = _build.build()
    out = subprocess.check_output(["nm", "-D", "--defined-only", path], text=True)
    exported = set(l.split()[-1] for l in out.splitlines() if " T " in l)
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n)


def test_header_compiles_as_c():
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c",
                        os.path.join(ROOT, "include", "ann.h")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_argument_errors_without_gpu():
    """Calls rejected on the host before any CUDA work."""
    import paper_2201_13007_gb300 as ann
    with pytest.raises(ann.AnnError):
        ann.ann_index_create(None, 10, 4, 0, None, 2, 0, 0, 0)
    assert "NULL" in ann.ann_last_error()
    with pytest.raises(ann.AnnError):
        ann.ann_search(None, None, 1, 1, 1, 1, None, None, None)
    from paper_2201_13007_gb300 import _abi
    with pytest.raises(ann.AnnError):
        _abi.ann_serve_create(None, None)
    assert "NULL" in ann.ann_last_error()


def test_ctypes_mirrors_match_the_header_layout(tmp_path):
    """Every struct of the header and its ctypes mirror have the same size,
    field names, order and offsets (a C program compiled from the header
    prints them)."""
    from paper_2201_13007_gb300 import _abi
    pairs = {"ann_index_info": _abi.IndexInfo, "ann_query_stats": _abi.QueryStats,
             "ann_search_params": _abi.SearchParams, "ann_launch_info": _abi.LaunchInfo,
             "ann_bucket_config": _abi.BucketConfig, "ann_serve_config": _abi.ServeConfig,
             "ann_result": _abi.Result}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ann.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr  # a field missing from the header fails here
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
    # and no header field is missing from a mirror: the header's member count per struct
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ann.h")).read(), flags=re.S)
    for cname, cls in pairs.items():
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + cname + r"\s*;", hdr).group(1)
        members = [m for m in body.split(";") if m.strip()]
        assert len(members) == len(cls._fields_), (cname, len(members), len(cls._fields_))
