"""Host-side checks of the C ABI (no GPU needed): the shared library loads,
exports every function include/lbib.h declares, the ctypes structures have
the C layout, and configuration checks reject bad input before any device
call."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

from paper_1606_01805_gb300 import build as B
from paper_1606_01805_gb300 import lbib

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "lbib.h"


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbib.load()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_binding_names():
    assert declared_functions() == sorted(lbib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", str(lbib.LIB_PATH)], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (lbm_\w+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, f"not exported: {missing}"
    for name in declared_functions():
        assert hasattr(lib, name)


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "lbib.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(lbm_config), "
        "sizeof(lbm_particle_desc), sizeof(lbm_particle_state), offsetof(lbm_config, cuda_stream), "
        "offsetof(lbm_config, workspace_bytes), offsetof(lbm_particle_desc, n_markers));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c11", "-I", str(ROOT / "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [C.sizeof(lbib.lbm_config), C.sizeof(lbib.lbm_particle_desc),
            C.sizeof(lbib.lbm_particle_state), lbib.lbm_config.cuda_stream.offset,
            lbib.lbm_config.workspace_bytes.offset, lbib.lbm_particle_desc.n_markers.offset]
    assert got == want


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(nx=2), dict(ny=2),
                                 dict(bc=(0, 1, 1, 1)), dict(bc=(0, 0, 0, 1)),
                                 dict(precision=7), dict(weight=9),
                                 dict(init=1, bc=(0, 0, 0, 0)), dict(check_every=3),
                                 dict(check_every=64), dict(check_every=-1)])
def test_invalid_configurations_rejected(lib, bad):
    kw = dict(nx=40, ny=30, tau=0.8)
    kw.update(bad)
    c = lbib.make_config(kw.pop("nx"), kw.pop("ny"), kw.pop("tau"), **kw)
    n = C.c_size_t()
    assert lib.lbm_workspace_bytes(C.byref(c), C.byref(n)) == lbib.LBM_EINVAL
    h = C.c_void_p()
    assert lib.lbm_init(C.byref(c), C.byref(h)) == lbib.LBM_EINVAL
    assert not h.value


def test_workspace_size_grows_with_lattice_and_precision(lib):
    sizes = {}
    for prec in (lbib.LBM_FP64, lbib.LBM_FP32, lbib.LBM_FP16_SHIFTED):
        c = lbib.make_config(1024, 256, 0.8, precision=prec)
        n = C.c_size_t()
        assert lib.lbm_workspace_bytes(C.byref(c), C.byref(n)) == lbib.LBM_OK
        sizes[prec] = n.value
    # two population buffers of 9 planes dominate: 8, 4, 2 bytes per value
    assert sizes[lbib.LBM_FP64] > sizes[lbib.LBM_FP32] > sizes[lbib.LBM_FP16_SHIFTED]
    assert sizes[lbib.LBM_FP32] >= 2 * 9 * 1024 * 256 * 4


def test_null_arguments(lib):
    assert lib.lbm_step(None, 1) == lbib.LBM_EINVAL
    assert lib.lbm_sync(None) == lbib.LBM_EINVAL
    assert lib.lbm_inject_status(None, lbib.LBM_ETIMEOUT) == lbib.LBM_EINVAL
    assert lib.lbm_steps_done(None) == 0
    assert lib.lbm_last_error(None) == b"null context"
    lib.lbm_destroy(None)


def test_tile_variants_per_precision(lib):
    """lbm_tile_info reports the ten tile shapes and which precisions have
    them: FP32 and FP16 storage all ten, FP64 the six direct kernels, the
    tangent mode the one-cell tile of 8 rows only."""
    shapes = [(4, 8, 0), (4, 4, 0), (1, 8, 0), (2, 8, 0), (2, 4, 0), (1, 4, 0),
              (4, 8, 2), (4, 8, 3), (2, 8, 3), (2, 8, 4)]
    assert len(shapes) == lbib.LBM_TILE_VARIANTS
    valid = {lbib.LBM_FP32: set(range(10)), lbib.LBM_FP16_SHIFTED: set(range(10)),
             lbib.LBM_FP64: set(range(6)), lbib.LBM_FP32_TANGENT: {2}}
    for prec, ok in valid.items():
        for v in range(-1, lbib.LBM_TILE_VARIANTS + 1):
            cpt, rows, st = C.c_int32(), C.c_int32(), C.c_int32()
            rc = lib.lbm_tile_info(v, prec, C.byref(cpt), C.byref(rows), C.byref(st))
            assert rc == (lbib.LBM_OK if v in ok else lbib.LBM_EINVAL), (prec, v)
            if 0 <= v < lbib.LBM_TILE_VARIANTS:
                assert (cpt.value, rows.value, st.value) == shapes[v]
    assert lbib.tile_info(4, lbib.LBM_FP32)[:3] == (2, 4, 0)
