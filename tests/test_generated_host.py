"""The generated specialised sources, run on the CPU: the block sweep of a
triangulation's generated CUDA source is compiled as plain C++ with host
definitions of the CUDA intrinsics (tests/host/), run one lane at a time over
whole warps (each warp classifies all middle-row patterns of one value of
the high bits), and its histograms must equal the oracle's over the same
masks.  Catches mistakes of the code generator without a GPU; the GPU tests
check the same code compiled for sm_103a."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import tcurve_inputs as ti

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def eng():
    from paper_2604_09221_gb300 import build
    build.build()
    import paper_2604_09221_gb300 as e
    e.library()
    return e


SNAP_BRANCH = "  if (nl_o <= 32u) {\n"   # the generated choice of the lane loop


def build_block_sweep(eng, tmp_path, d, edges, count_snap=False):
    """Compile the generated block sweep of (d, edges) with the host driver;
    with count_snap, a copy of the source counts the lanes that take the
    snapshot path (more than 32 labels left by the half-diamonds)."""
    src = eng.specialized_source(d, edges)
    flags = []
    if count_snap:
        assert src.count(SNAP_BRANCH) == 1
        src = ("static long tc_test_snap_lanes = 0;\n" +
               src.replace(SNAP_BRANCH, "  if (nl_o > 32u) ++tc_test_snap_lanes;\n" + SNAP_BRANCH))
        flags = ["-DTC_TEST_COUNT_SNAP"]
    (tmp_path / "gen.cu").write_text(src)
    np.savetxt(tmp_path / "tri.txt", edges, fmt="%d")
    exe = tmp_path / "run"
    cmd = ["g++", "-std=c++17", "-O1", "-w", f'-DGEN="{tmp_path / "gen.cu"}"', *flags,
           f"-I{os.path.join(HERE, 'host')}", f"-I{os.path.join(ROOT, 'oracle')}",
           "-o", str(exe), os.path.join(HERE, "host", "run_block_sweep.cpp"),
           "-x", "c", os.path.join(ROOT, "oracle", "tcurve_oracle.c"), "-x", "none", "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


def run_block_sweep(exe, tmp_path, warps, mode):
    out = subprocess.run([str(exe), str(tmp_path / "tri.txt"), str(warps), mode],
                         capture_output=True, text=True)
    assert out.returncode == 0, (mode, out.stdout + out.stderr)
    return out.stdout


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
@pytest.mark.parametrize("d,seed", [(4, 4), (5, 5), (7, 7), (8, 8), (9, 9)])
def test_block_sweep_source_on_the_host(eng, tmp_path, d, seed):
    """Every mask map the block sweep serves: no flag (d + 1 middle-row bits),
    TS_ENUM_FLIP (d) and TS_ENUM_REDUCED (d - 1), where 32 lanes fit."""
    exe = build_block_sweep(eng, tmp_path, d, ti.regular_triangulation(d, seed=seed))
    for mode, ib in (("plain", d + 1), ("flip", d), ("reduced", d - 1)):
        if ib >= 5:
            run_block_sweep(exe, tmp_path, 6, mode)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
@pytest.mark.parametrize("name", ["bow_tie", "rank016", "rank015"])
def test_block_sweep_of_the_fig2_triangulations(eng, tmp_path, name):
    """The three printed d = 8 triangulations, swept as the exhaustive Fig. 2
    check sweeps them (TS_ENUM_REDUCED) and without flags.  On rank016 and
    rank015 most warps' half-diamonds leave more than 32 labels, so the lane
    loop that restores from the snapshot region runs too."""
    edges = np.loadtxt(os.path.join(HERE, "golden", f"fig2_{name}.edges"), dtype=np.int32,
                       comments="#")
    exe = build_block_sweep(eng, tmp_path, 8, edges, count_snap=True)
    for mode in ("reduced", "plain"):
        out = run_block_sweep(exe, tmp_path, 12, mode)
        lanes = int(out.split("snapshot_lanes=")[1].split()[0])
        if name != "bow_tie":
            assert lanes >= 32 * 4, out   # at least 4 of the 12 warps


CUDA_INCLUDE = "/usr/local/cuda/include"   # host.cpp's headers and the runtime it links
CUDA_LIB = "/usr/local/cuda/lib64"


@pytest.mark.skipif(shutil.which("g++") is None or not os.path.isdir(CUDA_INCLUDE)
                    or not os.path.isdir(CUDA_LIB),
                    reason="needs g++ and the CUDA headers")
@pytest.mark.parametrize("d", [5, 7, 8, 10, 11, 13, 16])
def test_table_sweep_on_the_host(tmp_path, d):
    """The table-driven sweep (both back ends, multi-word sign vectors and
    codes) compiled for the host, on the tables host.cpp builds, against the
    oracle: random and special sign vectors, standard and regular
    triangulations."""
    csrc = os.path.join(ROOT, "paper_2604_09221_gb300", "csrc")
    exe = tmp_path / "run"
    cmd = ["g++", "-std=c++17", "-O1", "-w", f"-I{csrc}", f"-I{os.path.join(HERE, 'host')}",
           f"-I{os.path.join(ROOT, 'oracle')}", f"-I{CUDA_INCLUDE}", "-o", str(exe),
           os.path.join(HERE, "host", "run_table_sweep.cpp"),
           "-x", "c", os.path.join(ROOT, "oracle", "tcurve_oracle.c"), "-x", "none",
           f"-L{CUDA_LIB}", f"-Wl,-rpath,{CUDA_LIB}", "-lcudart", "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    for name, edges in (("standard", ti.standard_triangulation(d)),
                        ("regular", ti.regular_triangulation(d, seed=100 + d))):
        np.savetxt(tmp_path / "tri.txt", edges, fmt="%d")
        out = subprocess.run([str(exe), str(d), str(tmp_path / "tri.txt"), "600"],
                             capture_output=True, text=True)
        assert out.returncode == 0, (name, out.stdout + out.stderr)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_histogram_inserts_on_the_host(tmp_path):
    """The device histogram inserts (one-word, block-private with spill,
    multi-word with the BUSY / READY flags) compiled for the host and run one
    call at a time against a std::map, including full tables."""
    csrc = os.path.join(ROOT, "paper_2604_09221_gb300", "csrc")
    exe = tmp_path / "run"
    subprocess.run(["g++", "-std=c++17", "-O1", "-w", f"-I{os.path.join(HERE, 'host')}", f"-I{csrc}",
                    "-o", str(exe), os.path.join(HERE, "host", "run_hash_insert.cpp")],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
