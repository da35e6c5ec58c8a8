"""The C-ABI library loads, exports every entry point include/*.h declares,
and validates its descriptors on the host (no GPU calls)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(flash_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2604_17513_gb300 import build, flash
    build.build()
    return flash.lib()


def test_header_declares_entry_points():
    names = _declared()
    assert "flash_step" in names and "flash_scene_create" in names and len(names) >= 18


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_regular_build_has_no_poke_hook(lib):
    """flash_check_poke_element corrupts device tables only in the checked
    build; the regular library reports itself unchecked and refuses it
    before touching any scene."""
    import ctypes as C
    from paper_2604_17513_gb300 import flash
    assert lib.flash_checked_build() == 0
    old = C.c_int32(0)
    assert lib.flash_check_poke_element(None, 0, 0, 0, 0, C.byref(old)) == flash.ENOTIMPL


def test_header_compiles_as_c(tmp_path):
    """include/flash.h is a plain C header: a C99 translation unit that
    includes it and names its types and entry points compiles without
    warnings (gcc -std=c99 -Wall -Wextra -Werror, syntax only)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "uses_header.c"
    src.write_text('#include "flash.h"\n'
                   "int main(void) {\n"
                   "  flash_scene_desc d;\n  flash_scene *s = 0;\n  (void)d;\n"
                   "  return (int)flash_checked_build() + (int)flash_lane_count(s);\n}\n")
    res = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                          "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


def test_header_has_no_torch_types():
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        assert "torch" not in src.lower().replace("pytorch", "") and "at::" not in src


def test_scene_descriptor_validation(lib):
    from paper_2604_17513_gb300 import flash
    d = flash.SceneDesc()
    d.h = 0.0  # invalid
    h = C.c_void_p()
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    assert b"invalid" in lib.flash_last_error()
    d.h = 0.01
    d.k_max, d.k_cap, d.contact_cap = 10, 10, 16
    d.mode = 7
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    d.mode = 0
    # box-feature and self contacts are multi-vertex rows: the lite metric refuses them
    d.obstacle_features = 1
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    assert b"full metric" in lib.flash_last_error()
    d.obstacle_features = 2
    d.metric = flash.METRIC_FULL
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    d.obstacle_features, d.metric = 0, 0
    # the bf16 solve's refinement count and the grouped-solve switch are range checked
    d.solve, d.refine_steps = flash.SOLVE_BF16R, 5
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    assert b"refine_steps" in lib.flash_last_error()
    d.refine_steps, d.grouped_solve = 1, 3
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    d.solve, d.refine_steps, d.grouped_solve = 0, 0, 0
    # threads per environment: 0, tune (-1) or one of the instantiated counts
    for field, bad in (("local_threads", 128), ("local_threads", 768), ("ncp_threads", 1024), ("ncp_threads", -2)):
        setattr(d, field, bad)
        assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL, (field, bad)
        assert field.encode() in lib.flash_last_error()
        setattr(d, field, 0)
    d.local_threads, d.ncp_threads = flash.THREADS_TUNE, 512
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.OK
    lib.flash_scene_destroy(h)
    d.local_threads, d.ncp_threads = 0, 0
    d.split_k = 3
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.EINVAL
    assert b"split_k" in lib.flash_last_error()
    d.split_k = flash.SPLITK_ON
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.OK
    lib.flash_scene_destroy(h)
    d.split_k = 0
    assert lib.flash_scene_create(C.byref(d), C.byref(h)) == flash.OK
    # a mesh with an out-of-range element index is rejected on the host
    rest = np.zeros((3, 3))
    el = np.array([[0, 1, 5]], np.int32)
    mass = np.ones(3)
    m = flash.MeshDesc(0, 3, 1, rest.ctypes.data_as(C.POINTER(C.c_double)), el.ctypes.data_as(C.POINTER(C.c_int32)),
                       mass.ctypes.data_as(C.POINTER(C.c_double)), 1.0, 0.0, 1e-3)
    mid = C.c_int32()
    assert lib.flash_mesh_add(h, C.byref(m), C.byref(mid)) == flash.EINVAL
    el[0, 2] = 2
    assert lib.flash_mesh_add(h, C.byref(m), C.byref(mid)) == flash.OK
    # stepping before finalize is an ordering error, not a crash
    assert lib.flash_step(h, 1, None) == flash.ESTATE
    envs = (flash.EnvDesc * 1)()
    envs[0].n_obs = 9
    first = C.c_int32()
    assert lib.flash_envs_add(h, mid, 1, envs, C.byref(first)) == flash.EINVAL
    lib.flash_scene_destroy(h)
