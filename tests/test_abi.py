"""The C-ABI library loads and exports every symbol include/turret.h declares,
and the ctypes mirrors of its structs have the C layout.  No GPU needed."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2408_15115_gb300 import build as B
from paper_2408_15115_gb300 import turret as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "turret.h")


def _declared():
    src = open(HEADER).read()
    return re.findall(r"TURRET_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary_calls():
    names = set(_declared())
    for want in ("lbm_init", "ibm_load_surface", "step", "query_particle_state", "lbm_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(_declared()) == exported


def test_struct_layout_matches_c(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "turret.h"\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu\\n", sizeof(turret_window), sizeof(turret_flags),'
                    ' sizeof(turret_particle_state), offsetof(turret_window, anchor_frac),'
                    ' offsetof(turret_particle_state, volume)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    sizes = list(map(int, subprocess.check_output([str(exe)]).split()))
    assert sizes == [ctypes.sizeof(T.Window), ctypes.sizeof(T.Flags), ctypes.sizeof(T.ParticleState),
                     T.Window.anchor_frac.offset, T.ParticleState.volume.offset]


def test_host_side_validation_without_gpu(libpath):
    # size queries are pure host logic and reject invalid windows
    lib = T.lib()
    w = T.Window(16, 16, 16, 0, 0, 0, 0, 0, 0, 0, 0.25)
    assert lib.lbm_workspace_bytes(ctypes.byref(w), 0) > 27 * 4 * 16 ** 3 * 2
    assert lib.lbm_workspace_bytes(ctypes.byref(w), 1) < lib.lbm_workspace_bytes(ctypes.byref(w), 0)
    bad = T.Window(16, 16, 16, 0, 0, 1, 0, 0, 0, 0, 0.25)  # periodic top with closed bottom
    assert lib.lbm_workspace_bytes(ctypes.byref(bad), 0) == 0
    ctx = ctypes.c_void_p()
    g = (ctypes.c_double * 3)(0, 0, 0)
    rc = lib.lbm_init(ctypes.byref(ctx), ctypes.byref(w), 27, -0.1, 1.0, g, 0, None, 0, None)
    assert rc == 1 and b"tau" in lib.turret_last_error(None)
    rc = lib.lbm_init(ctypes.byref(ctx), ctypes.byref(w), 19, 0.1, 1.0, g, 0, None, 0, None)
    assert rc == 1


def test_window_limits_and_degenerate_windows(libpath):
    # 32-bit population offsets: 27 nx ny nz <= 2^31 cells is the largest window
    lib = T.lib()
    size = lambda *a: lib.lbm_workspace_bytes(ctypes.byref(T.Window(*a)), 0)
    n_max = (1 << 31) // 27  # 79,536,431 cells
    assert size(512, 512, n_max // (512 * 512), 0, 0, 1, 2, 0, 0, 0, 0.25) > 0   # 512 x 512 x 303
    assert size(512, 512, n_max // (512 * 512) + 1, 0, 0, 1, 2, 0, 0, 0, 0.25) == 0
    assert size(1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0.25) > 0          # a single periodic cell
    for bad in ((0, 16, 16, 0, 0, 1, 2, 0, 0, 0, 0.25),         # empty
                (16, 16, 70000, 0, 0, 1, 2, 0, 0, 0, 0.25),     # more planes than a launch allows
                (16, 16, 16, 0, 0, 2, 2, 0, 0, 0, 0.25),        # pressure at the bottom
                (16, 16, 16, 0, 0, 1, 2, 17, 0, 0, 0.25),       # sponge deeper than the window
                (16, 16, 16, 0, 0, 3, 3, 0, 1, 0, 0.25),        # moving walls in a sliding window
                (16, 16, 16, 0, 0, 1, 2, 0, 1, 0, 1.0),         # anchor outside (0, 1)
                (16, 16, 16, 2, 0, 1, 2, 0, 0, 0, 0.25)):       # unknown lateral code
        assert size(*bad) == 0, bad
    w = T.Window(16, 16, 16, 0, 0, 0, 0, 0, 0, 0, 0.25)
    assert lib.lbm_workspace_bytes(ctypes.byref(w), 3) == 0     # unknown storage
