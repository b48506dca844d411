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


def test_triplet_marshalling_points_at_every_sequence():
    """The binding's triplet records (one joined buffer, no per-field Python calls) hold, for
    every sequence, a pointer and length that read back the exact input: str, bytes and code
    arrays, empty sequences and an empty batch."""
    import numpy as np

    trips = [("ACGT", "", "GGA"), (b"AC", b"T", b""), ("A" * 1000, "C", "G" * 7),
             (np.array([65, 67], dtype=np.uint8), "TT", b"G")]
    class Raw(ctypes.Structure):  # the record layout with the pointers as plain addresses
        _fields_ = [("s", ctypes.c_void_p * 3), ("len", ctypes.c_uint32 * 3)]

    assert ctypes.sizeof(Raw) == ctypes.sizeof(binding.Triplet)
    for batch in (trips[:1], trips, [trips[0]] * 3, []):
        ptr, keep = binding._triplet_array(batch)
        raw = ctypes.cast(ptr, ctypes.POINTER(Raw))
        for t, want in enumerate(batch):
            for q in range(3):
                assert raw[t].s[q]  # never null, even for an empty sequence
                got = ctypes.string_at(raw[t].s[q], raw[t].len[q])
                assert got == binding._as_bytes(want[q])
    try:
        binding._triplet_array([("A", "C")])
    except ValueError:
        pass
    else:
        raise AssertionError("a two-sequence triplet was accepted")


def test_noalloc_rejects_a_task_grid_beyond_int32_before_any_device_call():
    """The allocation-free entry point sizes its workspace in 64-bit arithmetic. A long, thin
    triplet whose task grid nJ * nK (65536 * 65537 with the 8x8 tile) exceeds 2^31 passes the
    length and score-range checks, and must be rejected with TRIOSEQ_ESCRATCH before any device
    access: the dummy non-null addresses below are never dereferenced, and no GPU is needed."""
    import numpy as np

    sub = np.array([[2 if i == j else -1 for j in range(4)] for i in range(4)], dtype=np.int8)
    dummy = 0x1000
    for a, b, c in ((0, 2097151, 4194367), (0, 4194367, 2097151), (1, 1 << 24, 1 << 24)):
        st = binding.trioseq_align_noalloc("ACGT", sub, -2, dummy if a else 0, a,
                                           dummy, b, dummy, c, dummy)
        assert st in (binding.ESCRATCH, binding.EOVERFLOW), (a, b, c, st)
    st = binding.trioseq_align_noalloc("ACGT", sub, -2, 0, 0, dummy, 2097151, dummy, 4194367, dummy)
    assert st == binding.ESCRATCH
