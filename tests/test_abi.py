"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "genga.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(genga_\w+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1404_2324_gb300 import build, genga
    path = build.build()
    lib = ctypes.CDLL(path)  # no CUDA call happens at load time
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(genga.EXPORTED) == names  # the binding covers exactly the declared ABI


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1404_2324_gb300 import build, genga
    monkeypatch.setattr(genga, "_lib", None)
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(genga.GengaError):
        genga.lib(build_if_missing=False)


def test_invalid_arguments_are_rejected_on_the_host():
    """Argument checks run before any CUDA call, so they work on a machine without a GPU."""
    import numpy as np
    from paper_1404_2324_gb300 import genga
    L = genga.lib()
    h = ctypes.c_void_p()
    m = np.array([1.0, 1e-6]); R = np.zeros(2); x = np.zeros(6); v = np.zeros(6)
    D = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    assert L.genga_init(ctypes.byref(h), 2, D(m), D(R), D(x), D(v), 1.0, 0.0, 2, 0) == genga.GENGA_EINVAL
    assert L.genga_init(ctypes.byref(h), 2, D(m), D(R), D(x), D(v), 1.0, 6.0, 3, 0) == genga.GENGA_EINVAL
    assert L.genga_init(ctypes.byref(h), 1, D(m), D(R), D(x), D(v), 1.0, 6.0, 2, 0) == genga.GENGA_EINVAL
    assert L.genga_init(ctypes.byref(h), 5000, D(m), D(R), D(x), D(v), 1.0, 6.0, 2, 0) == genga.GENGA_EINVAL
    bad = np.array([float("nan"), 1e-6])
    assert L.genga_init(ctypes.byref(h), 2, D(bad), D(R), D(x), D(v), 1.0, 6.0, 2, 0) == genga.GENGA_EINVAL
    assert not h.value
    p = genga.genga_default_params()
    assert (p.n1, p.n2, p.pc, p.bs_kmax) == (3.0, 0.4, 3.0, 8)
    assert (p.rcut, p.rcut_sun, p.nmin) == (0.0, 0.0, 0)  # ejections and the Nmin stop are off by default
    n = ctypes.c_int(-1)
    assert L.genga_ejections(None, None, 0, ctypes.byref(n)) == genga.GENGA_EINVAL
    assert L.genga_set_params(None, ctypes.byref(p)) == genga.GENGA_EINVAL


def _c_layout(tmp_path, header, struct, fields):
    """sizeof and field offsets of a C struct, from a small program compiled against the header."""
    import subprocess
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src.write_text(f'#include <stddef.h>\n#include <stdio.h>\n#include "{header}"\nint main(void) {{\n'
                   f'  printf("%zu\\n", sizeof({struct}));\n{body}  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("which", ["genga", "oracle"])
def test_params_struct_layout_matches_the_binding(tmp_path, which):
    """The ctypes mirrors of genga_params (include/genga.h) and orc_params (the oracle's header)
    have the C structs' size and field offsets: a field added on one side only shifts the rest."""
    if which == "genga":
        from paper_1404_2324_gb300 import genga as mod
        cls, header, struct = mod.genga_params, os.path.join(ROOT, "include", "genga.h"), "genga_params"
    else:
        import oracle as mod
        cls, header, struct = mod.Params, os.path.join(ROOT, "oracle", "genga_oracle.h"), "orc_params"
    names = [f[0] for f in cls._fields_]
    got = _c_layout(tmp_path, header, struct, names)
    assert got[0] == ctypes.sizeof(cls)
    assert got[1:] == [getattr(cls, n).offset for n in names]
