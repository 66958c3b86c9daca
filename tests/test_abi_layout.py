"""The binding's view of the C ABI agrees with the headers (no GPU).

* The ctypes mirrors of the parameter structs (muster_params of include/muster.h, and the
  oracle's or_params) have the C compiler's field offsets and size: a small C program built
  with gcc against the headers prints offsetof and sizeof for every field.
* Every function declared in include/*.h has a ctypes signature with the same number of
  arguments, a compatible type for each (integers of the same width, float, pointers as
  pointers) and the same return type."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _c_layout(tmp_path, header_dir, header, ctype, fields):
    prog = ["#include <stddef.h>", "#include <stdio.h>", '#include "%s"' % header, "int main(void) {",
            '  printf("size %%zu\\n", sizeof(%s));' % ctype]
    for name in fields:
        prog.append('  printf("%s %%zu\\n", offsetof(%s, %s));' % (name, ctype, name))
    prog += ["  return 0;", "}"]
    src, exe = tmp_path / (ctype + ".c"), tmp_path / ctype
    src.write_text("\n".join(prog) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", header_dir, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("which", ["engine", "oracle"])
def test_parameter_structs_match_the_c_layout(tmp_path, which):
    if not shutil.which("gcc"):
        pytest.skip("gcc missing")
    if which == "engine":
        from paper_2412_14671_gb300 import _native

        cls, hdir, hdr, ctype = _native.MusterParams, os.path.join(ROOT, "include"), "muster.h", "muster_params"
    else:
        import oracle

        cls, hdir, hdr, ctype = oracle.OrParams, os.path.join(ROOT, "oracle"), "muster_oracle.h", "or_params"
    names = [f[0] for f in cls._fields_]
    c = _c_layout(tmp_path, hdir, hdr, ctype, names)
    assert c["size"] == ctypes.sizeof(cls)
    for name in names:
        assert c[name] == getattr(cls, name).offset, name


_SCALARS = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "size_t": ctypes.c_size_t, "float": ctypes.c_float,
            "double": ctypes.c_double}


def _declarations():
    """name -> (return type text, [parameter type texts]) for every function in include/*.h."""
    out = {}
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(inc, h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"typedef struct \{.*?\}\s*\w+;", "", text, flags=re.S)
        text = re.sub(r"^\s*#[^\n]*", "", text, flags=re.M)  # preprocessor lines
        text = re.sub(r'extern "C" \{|^\s*\}\s*$|\btypedef [^;]*;', "", text, flags=re.M)
        for m in re.finditer(r"([\w\s\*]+?)\b(muster_\w+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
            ret, name, params = " ".join(m.group(1).split()), m.group(2), " ".join(m.group(3).split())
            plist = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
            out[name] = (ret, plist)
    return out


def _param_type(decl):
    """Type of one parameter declaration with its name removed: (base, is_pointer)."""
    decl = decl.replace("const ", "")
    ptr = "*" in decl or "[" in decl
    base = decl.split("*")[0].split("[")[0].split()[0] if ptr else decl.split()[0]
    return base, ptr


def _is_pointer_type(t):
    return t in (ctypes.c_void_p, ctypes.c_char_p) or (isinstance(t, type) and issubclass(t, ctypes._Pointer))


def test_every_declaration_has_a_matching_ctypes_signature():
    from paper_2412_14671_gb300 import _native

    decls = _declarations()
    assert set(decls) == set(_native.SIGNATURES)
    for name, (ret, params) in decls.items():
        res, args = _native.SIGNATURES[name]
        assert len(args) == len(params), (name, params)
        for decl, t in zip(params, args):
            base, ptr = _param_type(decl)
            if ptr:
                assert _is_pointer_type(t), (name, decl, t)
                if base in _SCALARS and base != "float" and t is not ctypes.c_void_p:
                    assert t._type_ is _SCALARS[base], (name, decl, t)
            else:
                assert t is _SCALARS[base], (name, decl, t)
        if ret == "void":
            assert res is None, name
        elif ret == "int":
            assert res is ctypes.c_int, name
        else:
            assert ret == "const char*" and res is ctypes.c_char_p, (name, ret)
