"""The C-ABI library builds, loads and exports every symbol include/mcev.h
declares, with the structure layouts the binding assumes (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_2408_07996_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "mcev.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcev_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_signatures():
    assert _declared() == sorted(L.SIGNATURES)


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(L.load().__getattribute__("_name"))
    for name in _declared():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(tmp_path):
    # ask the C compiler for sizeof/offsetof of every field the binding uses
    import subprocess
    structs = {"mcev_params": L.Params, "mcev_stats": L.Stats, "mcev_scene_desc": L.SceneDesc,
               "mcev_detect_args": L.DetectArgs, "mcev_quality": L.Quality}
    lines = []
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mcev.h"\nint main(void){' +
                   "".join(lines) + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2408_07996_gb300.api import Renderer
    with pytest.raises(RuntimeError):
        Renderer(8, 8)
