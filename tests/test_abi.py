"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point ``include/gwn.h`` declares; the Python binding binds exactly
those.  No compute calls (no GPU needed)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gwn.h")).read()
    return sorted(set(re.findall(r"GWN_API\s+[\w\s\*]*?\b(gwn_\w+)\s*\(", src)))


def test_header_declares_api():
    names = _declared()
    for required in ("gwn_mesh_create", "gwn_build_accel", "gwn_query_batch", "gwn_query_direct",
                     "gwn_classify", "gwn_mesh_destroy", "gwn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2605_01536_gb300 as gwn
    path = gwn.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gwn_\w+)", out))
    assert set(_declared()) == exported
    lib = gwn.load()
    for name in _declared():
        assert hasattr(lib, name)
    assert set(gwn.SIGNATURES) == set(_declared())
    assert b"sm_103a" in lib.gwn_version()


def test_product_path_has_no_oracle_or_cpu_fallback():
    pkg = os.path.join(ROOT, "paper_2605_01536_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "gwn_oracle" not in text, f


def test_kernels_compile_for_sm103a():
    """Every translation unit is compiled for sm_103a only (the build's flags;
    gwn_version() above reports the target the library was built for)."""
    from paper_2605_01536_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
