"""The C ABI library loads and exports every entry point the header declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ttn.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(ttn_[a-z_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_01331_gb300 import _abi
    if not os.path.exists(_abi.LIB_PATH):
        from paper_1905_01331_gb300 import build
        build.build()
    return _abi.load()


def test_header_declares_the_sweep_api():
    names = declared_functions()
    for required in ("ttn_create", "ttn_sweep", "ttn_energy", "ttn_rdm", "ttn_env",
                     "ttn_workspace_bytes", "ttn_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1905_01331_gb300 import _abi
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, name


def test_workspace_size_and_argument_checks_need_no_gpu(lib):
    """ttn_workspace_bytes is host-only arithmetic; bad shapes are rejected."""
    import numpy as np
    from paper_1905_01331_gb300 import _abi
    import ttn_inputs as ti
    m = ti.tfim_chain(1024, 1.0)
    o, A, B = (np.ascontiguousarray(x) for x in (m.o, m.A, m.B))
    p = _abi.Problem(1024, 1, 2, 128, 1, 0, o.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     B.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    opt = _abi.Options()
    lib.ttn_default_options(ctypes.byref(opt))
    n = lib.ttn_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(opt))
    # isometries alone: 6 full 128^3 layers + smaller ones, 8 bytes each
    assert n > 6 * 128 ** 3 * 8
    bad = _abi.Problem(1000, 1, 2, 128, 1, 0, p.onesite, p.A, p.B)   # L not a power of two
    assert lib.ttn_workspace_bytes(ctypes.byref(bad), 1, ctypes.byref(opt)) == 0


def test_no_forbidden_calls_in_sources():
    """The batched-memcpy family is closed on this machine; sources must not name it."""
    csrc = os.path.join(ROOT, "paper_1905_01331_gb300", "csrc")
    pat = re.compile("Memcpy" + "(3D)?" + "Batch" + "Async")
    for fn in os.listdir(csrc):
        with open(os.path.join(csrc, fn)) as f:
            assert not pat.search(f.read()), fn


def _problem(model, chi, per_node=False):
    import numpy as np
    from paper_1905_01331_gb300 import _abi
    o, A, B = (np.ascontiguousarray(x) for x in (model.o, model.A, model.B))
    dp = ctypes.POINTER(ctypes.c_double)
    p = _abi.Problem(model.Lx, model.Ly, 2, chi, A.shape[0], int(per_node),
                     o.ctypes.data_as(dp), A.ctypes.data_as(dp), B.ctypes.data_as(dp))
    return p, (o, A, B)


@pytest.mark.parametrize("prec", [0, 2])
def test_every_product_stays_inside_its_buffer(lib, prec):
    """The library's plan pass walks every product of a sweep (and of the
    energy / density-matrix / environment calls) over a fake address range and
    checks each operand's highest address against the buffer it points into;
    a violation makes ttn_workspace_bytes return 0.  Run on CPU for every
    workload shape before any GPU launch."""
    import ttn_inputs as ti
    from paper_1905_01331_gb300 import _abi
    cases = [(ti.tfim_chain(16, 1.0), 8, True), (ti.tfim_chain(1024, 1.0), 128, False),
             (ti.tfim_chain(1024, 1.0), 32, False), (ti.heisenberg_xxx(256), 256, False),
             (ti.tfim_torus(64, 4, 3.04), 128, False), (ti.tfim_torus(8, 4, 3.04), 32, True),
             (ti.heisenberg_xxx(8), 16, True), (ti.tfim_chain(4, 0.5), 4, False)]
    opt = _abi.Options()
    lib.ttn_default_options(ctypes.byref(opt))
    opt.prec = prec
    for m, chi, pn in cases:
        p, keep = _problem(m, chi, pn)
        assert lib.ttn_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(opt)) > 0, (m.name, chi, pn)
    # bond dimensions must be powers of two (index arithmetic uses shifts)
    p, keep = _problem(ti.tfim_chain(8, 0.5), 3)
    assert lib.ttn_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(opt)) == 0
    # several instances of different sizes in one context
    ps = [_problem(ti.tfim_chain(L, 1.0), chi) for L, chi in ((64, 32), (512, 128), (128, 64))]
    arr = (_abi.Problem * 3)(*[p for p, _ in ps])
    assert lib.ttn_workspace_bytes(arr, 3, ctypes.byref(opt)) > 0


def test_default_options_match_the_header(lib):
    """ttn_default_options fills the defaults include/ttn.h documents (host
    only): automatic top-solve tolerance (0: 1e-13 in FP64 mode, 1e-10 in the
    mixed modes), Krylov dimension 48 with 3 restarts, both persistent kernels,
    8 streams, automatic polar blocks, double-float polar factor."""
    from paper_1905_01331_gb300 import _abi
    opt = _abi.Options()
    lib.ttn_default_options(ctypes.byref(opt))
    assert opt.lanczos_tol == 0.0
    assert (opt.lanczos_max, opt.lanczos_restarts) == (48, 3)
    assert (opt.persistent, opt.streams, opt.polar_blocks, opt.double_float) == (3, 8, 0, 1)
    assert opt.polar_damping == 1e-7


def test_tiles_blob_is_validated_at_planning(lib):
    """ttn_options.tiles (the autotuner's table) is parsed before the plan
    pass: a foreign or damaged blob is rejected, an empty table accepted."""
    import struct
    import numpy as np
    from paper_1905_01331_gb300 import _abi
    import ttn_inputs as ti
    m = ti.tfim_chain(64, 1.0)
    o, A, B = (np.ascontiguousarray(x) for x in (m.o, m.A, m.B))
    dp = ctypes.POINTER(ctypes.c_double)
    p = _abi.Problem(64, 1, 2, 16, 1, 0, o.ctypes.data_as(dp), A.ctypes.data_as(dp),
                     B.ctypes.data_as(dp))

    def size_with(blob):
        opt = _abi.Options()
        lib.ttn_default_options(ctypes.byref(opt))
        buf = ctypes.create_string_buffer(blob, len(blob))
        opt.tiles = ctypes.cast(buf, ctypes.c_void_p)
        opt.tiles_bytes = len(blob)
        return lib.ttn_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(opt))

    empty = b"TTNT" + struct.pack("<III", 2, 0, 0)
    assert size_with(empty) > 0
    assert size_with(b"garbage-garbage-garbage") == 0
    assert size_with(b"TTNT" + struct.pack("<III", 1, 0, 0)) == 0           # another version
    entry = struct.pack("<Qiiiifi", 123, 0, 48, 4, 1, 1.0, 0)              # tile 48: not a width
    assert size_with(b"TTNT" + struct.pack("<III", 2, 1, 0) + entry) == 0
    entry = struct.pack("<Qiiiifi", 123, 1, 64, 2, 0, 1.0, 0)
    assert size_with(b"TTNT" + struct.pack("<III", 2, 1, 0) + entry) > 0
    assert size_with(b"TTNT" + struct.pack("<III", 2, 2, 0) + entry) == 0   # truncated


def test_polar_schedule_option_is_validated_at_planning(lib):
    """ttn_options.polar_blocks: 0 (adaptive with the first try), 1, 2, 3
    (fixed two-block schedule) and 4 (adaptive without the first try) are
    accepted; anything else is rejected before any device work."""
    import numpy as np
    from paper_1905_01331_gb300 import _abi
    import ttn_inputs as ti
    m = ti.tfim_chain(64, 1.0)
    o, A, B = (np.ascontiguousarray(x) for x in (m.o, m.A, m.B))
    dp = ctypes.POINTER(ctypes.c_double)
    p = _abi.Problem(64, 1, 2, 16, 1, 0, o.ctypes.data_as(dp), A.ctypes.data_as(dp),
                     B.ctypes.data_as(dp))

    def size_with(pb):
        opt = _abi.Options()
        lib.ttn_default_options(ctypes.byref(opt))
        opt.polar_blocks = pb
        return lib.ttn_workspace_bytes(ctypes.byref(p), 1, ctypes.byref(opt))

    assert all(size_with(pb) > 0 for pb in range(5))
    assert size_with(5) == 0 and size_with(-1) == 0
