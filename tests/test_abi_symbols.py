"""The native library loads on a machine without a GPU and exports every
function include/sketch.h declares (no compute calls are made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                src = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(sk_\w+)\s*\(", src,
                                    flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sk_create", "sk_apply_left", "sk_apply_right", "sk_materialize",
                     "sk_destroy", "sk_stream_status"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2603_20966_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2603_20966_gb300 import _native
    assert _declared() <= set(_native.PROTOTYPES)


def test_host_side_validation_without_gpu():
    # calls that fail argument checks return before touching the device
    from paper_2603_20966_gb300 import _native as N
    L = N.lib()
    assert L.sk_create(1, 9, 4, ctypes.byref(ctypes.c_void_p())) == N.SK_EINVAL
    assert L.sk_create(1, 0, 0, ctypes.byref(ctypes.c_void_p())) == N.SK_EINVAL
    assert L.sk_apply_left(None, None, 1, 1, 1, None, 1, None) == N.SK_EINVAL
    assert N.status_string(N.SK_ETIMEOUT).startswith("SK_ETIMEOUT")
    assert N.sk_version() >= 100
