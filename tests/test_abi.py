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


def test_host_allocation_failure_returns_enomem_without_a_gpu():
    """A C++ exception never crosses the C boundary: with host allocation failure injected
    (TRIOSEQ_TEST_HOST_BAD_ALLOC, read at the first call), every call returns TRIOSEQ_ENOMEM
    instead of terminating the process, and trioseq_strerror still names it. Run in a child
    process, since the switch is read once per process."""
    import subprocess
    import sys

    code = (
        "from paper_2605_28400_gb300 import binding as B\n"
        "import numpy as np\n"
        "for call in (lambda: B.trioseq_partition([[3, 4, 5]], 2),\n"
        "             lambda: B.trioseq_plan('ACGT', np.eye(4, dtype=np.int8), -1)):\n"
        "    try:\n"
        "        call()\n"
        "        raise SystemExit('no error')\n"
        "    except B.TrioseqError as e:\n"
        "        assert e.status == B.ENOMEM, e.status\n"
        "print(B.trioseq_strerror(B.ENOMEM))\n")
    env = dict(os.environ, TRIOSEQ_TEST_HOST_BAD_ALLOC="1")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "out of memory"
