"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/trioseq.h.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

from paper_2605_28400_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "trioseq.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(trioseq_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("trioseq_plan", "trioseq_align_batch", "trioseq_traceback", "trioseq_submit",
                 "trioseq_poll"):
        assert must in names


def test_library_builds_and_exports_all_symbols():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(binding.exported_symbols()) == declared_symbols()


def test_binding_loads_and_strerror():
    binding.load()
    assert binding.trioseq_strerror(binding.EOVERFLOW).startswith("score bound")
    assert binding.trioseq_strerror(binding.OK) == "ok"
