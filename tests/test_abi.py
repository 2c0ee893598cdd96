"""The C ABI library builds for sm_103a, loads, and exports every entry point
that include/polypic.h declares.  Host-side argument validation is exercised
without a GPU (every call below returns before any CUDA work)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(polypic_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2308_01060_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:  # libcudart not resolvable on this host
        pytest.skip(f"cannot load libpolypic: {e}")


def test_header_declares_the_documented_entry_points():
    names = _declared_functions()
    for required in ["polypic_p2g", "polypic_grid_update", "polypic_g2p", "polypic_step",
                     "polypic_p2g_adjoint", "polypic_grid_update_adjoint", "polypic_g2p_adjoint",
                     "polypic_sort", "polypic_create", "polypic_check_device_status"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2308_01060_gb300 import polypic
    assert sorted(polypic.EXPORTS) == _declared_functions()


def test_host_validation_without_gpu(lib):
    from paper_2308_01060_gb300 import polypic as pp
    L = pp.load_library()
    assert L.polypic_status_string(0) == b"ok"
    assert L.polypic_num_keys(None) == -1
    assert L.polypic_workspace_bytes(None, 10, 0) == 0
    cfg = pp.Config()
    cfg.n[0], cfg.n[1], cfg.n[2] = 16, 16, 3          # n < 4: rejected before any CUDA call
    cfg.dx, cfg.num_modes, cfg.coeff_format = 1 / 16, 27, 0
    h = ctypes.c_void_p()
    assert L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.n[2] = 16
    cfg.num_modes = 5                                   # not 1, 4, 8, 27
    assert L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.num_modes = 27
    cfg.map, cfg.coeff_format = 1, 1                    # Eq 12 map with 16-bit codes: not built
    assert L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)) == 2
    cfg.map, cfg.coeff_format = 2, 0                    # no such map
    assert L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.map, cfg.apic_variant = 0, 1                    # Eq 10's form needs the 4-mode set
    assert L.polypic_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    cfg.apic_variant = 0
    assert L.polypic_p2g(None, None, None, None, 0, None) == 1
    assert L.polypic_p2g_mapped(None, None, None, 1e-3, None, 0, None) == 1
    assert L.polypic_p2g_mapped(None, None, None, float("nan"), None, 0, None) == 1
    assert L.polypic_p2g_noalloc(None, None, None, None) == 1
    assert L.polypic_step(None, None, None, None, None, None, None, None, None, 0, None) == 1
    # the fused transfer, the stand-ins and the whole-update adjoint refuse a
    # missing context before touching anything
    assert L.polypic_g2p2g(None, None, None, None, None, None, 1e-3, None, 0, None) == 1
    fab = pp.FabricParams()
    assert L.polypic_fabric_forces(None, None, ctypes.byref(fab), 1e-3, None, 0, None) == 1
    assert L.polypic_absorb(None, None, None, ctypes.byref(fab), 1e-3, None) == 1
    assert L.polypic_step_coupled(None, None, None, None, None, None, None, None,
                                  ctypes.byref(fab), None, 0, None) == 1
    assert L.polypic_grid_update_adjoint(None, None, None, None, None, None, None, None, None,
                                         None, 0, None) == 1


def test_header_is_plain_c():
    """include/polypic.h compiles as C99 and as C++ (the ABI uses no C++ types)."""
    import shutil
    import subprocess
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                       "polypic.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++17")):
        if not shutil.which(cc):
            pytest.skip(f"{cc} not found")
        r = subprocess.run([cc, std, "-Wall", "-Werror", "-fsyntax-only", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size, field offsets and
    field sizes that the C compiler gives the header's structures (a
    mismatch would hand the library misread pointers)."""
    import json
    import subprocess
    from paper_2308_01060_gb300 import polypic as pp
    pairs = [("polypic_config", pp.Config), ("polypic_particles", pp.Particles),
             ("polypic_grid", pp.Grid), ("polypic_update_params", pp.UpdateParams),
             ("polypic_fabric_params", pp.FabricParams)]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "polypic.h"',
             'int main(void) {', '    printf("{");']
    for i, (cname, cls) in enumerate(pairs):
        sep = "," if i else ""
        lines.append(f'    printf("{sep}\\"{cname}\\": {{\\"size\\": %zu", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf(", \\"{fname}\\": [%zu, %zu]", offsetof({cname}, {fname}), '
                         f'sizeof((({cname} *)0)->{fname}));')
        lines.append('    printf("}");')
    lines += ['    printf("}\\n");', '    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), str(src)], check=True)
    got = json.loads(subprocess.run([str(exe)], check=True, capture_output=True,
                                    text=True).stdout)
    for cname, cls in pairs:
        c = got[cname]
        assert c["size"] == ctypes.sizeof(cls), cname
        for fname, ftype in cls._fields_:
            assert c[fname] == [getattr(cls, fname).offset, ctypes.sizeof(ftype)], (cname, fname)


def _c_kind(decl):
    """Coarse ABI class of a C parameter or return type."""
    d = decl.strip()
    if "*" in d or "[" in d:
        return "ptr"
    if d == "void":
        return "void"
    for key, kind in (("uint32_t", "u32"), ("int32_t", "i32"), ("int64_t", "i64"),
                      ("size_t", "size"), ("double", "f64"), ("float", "f32"),
                      ("polypic_status", "i32"), ("int", "i32")):
        if re.search(rf"\b{key}\b", d):
            return kind
    raise AssertionError(f"unclassified C type: {decl!r}")


def _ctypes_kind(t):
    if t is None:
        return "void"
    if t in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(t, ctypes._Pointer):
        return "ptr"
    for ct, kind in ((ctypes.c_uint32, "u32"), (ctypes.c_int32, "i32"), (ctypes.c_int64, "i64"),
                     (ctypes.c_size_t, "size"), (ctypes.c_double, "f64"),
                     (ctypes.c_float, "f32")):
        if t is ct:
            return kind
    raise AssertionError(f"unclassified ctypes type: {t!r}")


def test_binding_signatures_match_the_header(lib):
    """Each binding declaration has the header prototype's argument count and,
    argument by argument, its class (pointer, 32/64-bit integer, size_t,
    float, double), and the same return class."""
    from paper_2308_01060_gb300 import polypic as pp
    L = pp.load_library()
    text = open(os.path.join(ROOT, "include", "polypic.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    protos = re.findall(r"([A-Za-z_][\w \*]*?)\s*\b(polypic_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", text)
    seen = set()
    for ret, name, args in protos:
        seen.add(name)
        params = [a for a in (p.strip() for p in args.split(",")) if a and a != "void"]
        fn = getattr(L, name)
        # the parameter's type: a scalar loses its trailing name
        want = [_c_kind(p if ("*" in p or "[" in p) else p.rsplit(None, 1)[0]) for p in params]
        got = [_ctypes_kind(t) for t in fn.argtypes]
        assert got == want, (name, got, want)
        assert _ctypes_kind(fn.restype) == _c_kind(ret), (name, fn.restype, ret)
    assert seen == set(_declared_functions())


def test_readme_c_example_compiles_and_links(tmp_path, lib):
    """The plain-C usage example in README.md builds as C99 against the
    header and links against libpolypic.so and the CUDA runtime with no
    undefined symbol (running it needs a GPU)."""
    import subprocess
    readme = open(os.path.join(ROOT, "README.md")).read()
    section = readme[readme.index("## Calling the library from C"):]
    code = section[section.index("```c\n") + 5:]
    code = code[:code.index("```")]
    assert "polypic_step(" in code and "polypic_create(" in code
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("CUDA runtime headers not found")
    src = tmp_path / "example.c"
    src.write_text(code)
    pkg = os.path.join(ROOT, "paper_2308_01060_gb300")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-fPIC", "-shared",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                    "-o", str(tmp_path / "libexample.so"), str(src),
                    "-L", pkg, "-lpolypic", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                    "-Wl,--no-undefined"], check=True)
