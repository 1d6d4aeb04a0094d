"""CPU-side checks of the C ABI: libcc.so builds for sm_103a, loads, and exports every
function include/*.h declares; the Python binding binds each of them by name.
No compute call is made (no GPU is needed)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1612_01178_gb300 import build, cc
    build.build()
    return cc.load()


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("cc_create", "cc_labels_csr", "cc_labels_coo", "cc_labels_batched", "cc_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    so = os.path.join(ROOT, "paper_1612_01178_gb300", "lib", "libcc.so")
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert names <= exported, sorted(names - exported)


def test_binding_covers_every_declared_symbol(lib):
    from paper_1612_01178_gb300 import cc
    assert declared_functions() <= set(cc.SIGNATURES), sorted(declared_functions() - set(cc.SIGNATURES))


def test_status_strings_and_defaults(lib):
    from paper_1612_01178_gb300 import cc
    for code in range(7):
        assert lib.cc_status_string(code)
    o = cc.default_options()
    assert o.block == 0 and o.tile_vertices == 0 and o.chunk_arcs == 0
    assert o.timeout_ns == 2_000_000_000 and o.mode == cc.CC_MODE_AUTO


def test_library_is_built_for_sm_103a():
    from paper_1612_01178_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.NVCC_FLAGS)
    assert os.path.exists(build.build())


def test_null_context_is_rejected_without_a_gpu(lib):
    from paper_1612_01178_gb300 import cc
    assert lib.cc_sync(None) == cc.CC_ERR_INVALID_ARG
    assert lib.cc_labels_csr(None, 1, 0, None, 4, None, None) == cc.CC_ERR_INVALID_ARG
    lib.cc_destroy(None)


def test_no_cpu_fallback_in_the_product():
    """The package must not import the oracle or any CPU labelling path."""
    for path in glob.glob(os.path.join(ROOT, "paper_1612_01178_gb300", "**", "*.py"), recursive=True):
        text = open(path).read()
        assert "import oracle" not in text and "from oracle" not in text, path


def test_binding_constants_match_the_header():
    """Every enumerator of include/cc.h has the same value in the Python binding (status codes,
    index types, flags, modes), and the binding defines no CC_ constant the header lacks."""
    from paper_1612_01178_gb300 import cc
    text = open(os.path.join(ROOT, "include", "cc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    header = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(CC_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    assert {"CC_OK", "CC_FLAG_SYMMETRIC", "CC_MODE_AUTO", "CC_MODE_FILTERED", "CC_INDEX_I64"} <= set(header)
    binding = {k: v for k, v in vars(cc).items() if k.startswith("CC_") and isinstance(v, int)}
    assert binding == header, (sorted(set(binding.items()) ^ set(header.items())))


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of cc_options and cc_run_info have the C structs' size and field offsets."""
    import ctypes
    from paper_1612_01178_gb300 import cc
    src = tmp_path / "sizes.c"
    fields = {"cc_options": [f for f, _ in cc.cc_options._fields_], "cc_run_info": [f for f, _ in cc.cc_run_info._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cc.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("  return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for st, cls in (("cc_options", cc.cc_options), ("cc_run_info", cc.cc_run_info)):
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)
