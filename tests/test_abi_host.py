"""Host-side checks of the C ABI (no GPU needed): the library loads and
exports every entry point declared in include/tcurve.h, input validation
rejects malformed triangulations, and the Rohlin-Viro printer agrees with an
independent printer on the codes the oracle produces."""
import ctypes
import os
import re

import numpy as np
import pytest

import tcurve_inputs as ti
from schemes import rohlin_viro

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def eng():
    from paper_2604_09221_gb300 import build
    build.build()
    import paper_2604_09221_gb300 as e
    e.library()
    return e


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tcurve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ts_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(eng):
    names = declared_functions()
    assert len(names) >= 15
    lib = eng.library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def load_status(eng, d, edges):
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 4))
    h = ctypes.c_void_p()
    rc = eng.library().ts_load_triangulation(d, e.ctypes.data, len(e), ctypes.byref(h))
    if rc == 0:
        eng.library().ts_free_triangulation(h)
    return rc


def test_validation_rejects_bad_triangulations(eng):
    good = ti.standard_triangulation(5)
    assert load_status(eng, 5, good[:-1]) == 2                    # an edge missing
    assert load_status(eng, 5, np.vstack([good, good[:1]])) == 2  # repeated edge
    bad = good.copy()
    bad[0] = [0, 0, 5, 0]                                         # not primitive
    assert load_status(eng, 5, bad) == 2
    out = good.copy()
    out[3, 2] = 9                                                 # point outside A
    assert load_status(eng, 5, out) == 2
    assert load_status(eng, 4, good) == 2                         # wrong degree
    assert load_status(eng, 0, good) == 1
    assert load_status(eng, 17, ti.standard_triangulation(17)) == 8  # beyond 3 sign words


@pytest.mark.parametrize("d", [6, 10, 16])
def test_valid_triangulation_needs_a_device(eng, d):
    import torch
    rc = load_status(eng, d, ti.regular_triangulation(d, seed=d))
    assert rc == (0 if torch.cuda.is_available() else 4)


def test_degree_limits(eng):
    assert eng.library().ts_max_degree() == 16
    with pytest.raises(eng.TSError) as ex:   # specialised kernels: one sign word (d <= 9)
        eng.specialized_source(10, ti.standard_triangulation(10))
    assert ex.value.status == 8


def test_status_strings(eng):
    lib = eng.library()
    for s in range(9):
        assert lib.ts_status_str(s).decode().startswith("TS_")


@pytest.mark.parametrize("d", [4, 5, 6, 7, 8])
def test_scheme_string_matches_independent_printer(eng, orc, d):
    tri = orc.triangles(d, ti.standard_triangulation(d))
    codes = orc.real_schemes(d, tri, ti.random_masks(2000, d, 17))
    for c in sorted(set(orc.code_to_int(r) for r in codes)):
        assert eng.scheme_string(d, c).replace("+", "+") == rohlin_viro(d, c)
    assert eng.scheme_string(6, 458) == "<1<1> + 2>"
    assert eng.scheme_string(7, 1) == "<J>"
    assert eng.scheme_string(6, 1) == "<0>"


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_specialized_kernels_compile_for_sm103a(eng, d):
    """The generated source of every degree compiles with NVRTC for sm_103a
    with at most a few hundred bytes of spills (checked on the host: no device
    needed)."""
    import re
    e = ti.regular_triangulation(d, seed=d) if d > 2 else ti.standard_triangulation(d)
    src = eng.specialized_source(d, e)
    # every vertex appears once in the per-mask sweep; the block sweep has the
    # middle row in straight-line code twice (restore from registers only, or
    # also from the snapshot region); its half-diamonds run from tables
    V = 2 * d * d + 2 * d + 1
    assert "tc_classify" in src and src.count("// vertex ") == V + 2 * (2 * d + 1)
    assert "tc_sweep_table(" in src and "__constant__ u32 tc_ctab" in src
    log = eng.specialized_source(d, e, compile=True)
    # the three entry kernels
    spills = {k: int(v) for k, v in re.findall(
        r"Function properties for (tc_\w+)\n[^\n]*?\d+ bytes stack frame, (\d+) bytes spill stores", log)}
    assert set(spills) == {"tc_real_schemes", "tc_enumerate", "tc_enumerate_blocks"}, log[-2000:]
    assert max(spills.values()) <= 256, spills


@pytest.mark.parametrize("d", [1, 4, 7, 10, 11, 16])
def test_specialized_batch_code_compiles_and_links(eng, d):
    """The specialised batch code (one relocatable object per triangulation,
    the degree's persistent kernel, linked with nvJitLink) builds for
    sm_103a on the host: one to three sign words, one to four code words,
    narrow and wide back ends.  Every object of the log reports its
    resources; a broken edge list is refused before compiling."""
    e = [ti.regular_triangulation(d, seed=d)] if d > 2 else [ti.standard_triangulation(d)]
    if d in (7, 10):
        e.append(ti.regular_triangulation(d, seed=d + 100))
    size, log = eng.batch_specialized_link(d, e, with_log=True)
    assert size > 0
    assert log.count("object ") == len(e) + 1
    bad = np.asarray(e[0]).reshape(-1, 4)[1:]
    with pytest.raises(eng.TSError) as err:
        eng.batch_specialized_link(d, [bad])
    assert err.value.status == 2


@pytest.mark.parametrize("d", [2, 4, 6, 7, 8, 9])
def test_diamond_tables_match_the_table_1_sizes(eng, d):
    """The tables of T^diamond built on the host (read from the generated
    source, no device needed): |A^diamond| = 2d^2 + 2d + 1 vertices and
    |E(T^diamond)| = 6d^2 + 2d edges (Table 1), one fan entry per edge."""
    import re
    e = ti.regular_triangulation(d, seed=d) if d > 2 else ti.standard_triangulation(d)
    src = eng.specialized_source(d, e)
    V = int(re.search(r"static constexpr unsigned V = (\d+)u;", src).group(1))
    words = int(re.search(r"__constant__ u32 tc_ctab\[(\d+)\]", src).group(1))
    assert V == 2 * d * d + 2 * d + 1
    edges = 6 * d * d + 2 * d
    assert words == (2 * V + edges + 3) // 4 * 4   # vdesc[V], fan[|E|], vext[V], 16-byte padded


def test_selftest_wait_needs_a_device(eng):
    import torch
    if torch.cuda.is_available():
        pytest.skip("covered by the GPU test")
    assert eng.selftest_wait(16) == 4   # TS_ECUDA
    assert eng.library().ts_selftest_wait(0, None) == 1   # TS_EINVAL


def test_header_and_library_from_c(eng, tmp_path):
    """include/tcurve.h compiles as C11 and a plain C program links
    libtcurve.so and gets the documented answers from the entry points that
    need no device."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    lib = eng.lib_path()
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}",
                    "-o", str(exe), os.path.join(ROOT, "tests", "host", "abi_from_c.c"), lib,
                    f"-Wl,-rpath,{os.path.dirname(lib)}"], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr


def test_batch_launch_plan_calls_reject_bad_arguments(eng):
    """The fused-launch and group-order calls refuse a null batch and
    out-of-range values before they touch a device."""
    lib = eng.library()
    assert lib.ts_batch_set_fused(None, 1) == 1                        # TS_EINVAL
    assert lib.ts_batch_set_fused(None, 0) == 1
    assert lib.ts_batch_set_serial(None, 1) == 1
    assert lib.ts_batch_set_fused_tile(None, 8, eng.TS_KERNEL_TABLE, 1024) == 1
    assert lib.ts_batch_set_fused_tile(None, 8, eng.TS_KERNEL_WARP, 1024) == 1
