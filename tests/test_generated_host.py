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
from schemes import orbit_mask

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
ODD_SNAPSHOT = ("  for (u32 w = 1; w < nwo; ++w) S.word(TcK::OFF_SNAP + TcK::WLAB, w) = "
                "S.word(TcK::OFF_ODD, w);\n")     # the snapshot of the odd-cycle flags


def build_block_sweep(eng, tmp_path, d, edges, count_snap=False):
    """Compile the generated block sweep of (d, edges) with the host driver;
    with count_snap, a copy of the source counts the lanes that take the
    snapshot path (more than 32 labels left by the half-diamonds) and the
    lanes with an odd-cycle flag set when the snapshot is taken."""
    src = eng.specialized_source(d, edges)
    flags = []
    if count_snap:
        assert src.count(SNAP_BRANCH) == 1 and src.count(ODD_SNAPSHOT) == 1
        src = ("static long tc_test_snap_lanes = 0, tc_test_odd_lanes = 0;\n" +
               src.replace(SNAP_BRANCH, "  if (nl_o > 32u) ++tc_test_snap_lanes;\n" + SNAP_BRANCH)
                  .replace(ODD_SNAPSHOT, ODD_SNAPSHOT +
                           "  for (u32 w = 0; w < TcK::WODD; ++w)\n"
                           "    if (S.word(TcK::OFF_ODD, w)) { ++tc_test_odd_lanes; break; }\n"))
        flags = ["-DTC_TEST_COUNT_SNAP"]
    (tmp_path / "gen.cu").write_text(src)
    np.savetxt(tmp_path / "tri.txt", edges, fmt="%d")
    exe = tmp_path / "run"
    cmd = ["g++", "-std=c++17", "-O1", "-w", f'-DGEN="{tmp_path / "gen.cu"}"', *flags,
           f"-I{os.path.join(HERE, 'host')}", f"-I{os.path.join(ROOT, 'oracle')}",
           f"-I{os.path.join(ROOT, 'paper_2604_09221_gb300', 'csrc')}",
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
    TS_ENUM_FLIP (d), TS_ENUM_REDUCED (d - 1) and TS_ENUM_ORBITS (d + 1,
    blocks of orbit high parts), where 32 lanes fit; and the per-mask
    classifier of the same source on random masks."""
    exe = build_block_sweep(eng, tmp_path, d, ti.regular_triangulation(d, seed=seed))
    for mode, ib in (("plain", d + 1), ("flip", d), ("reduced", d - 1), ("orbits", d + 1)):
        if ib >= 5:
            run_block_sweep(exe, tmp_path, 6, mode)
    run_block_sweep(exe, tmp_path, 16, "classify")


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
@pytest.mark.parametrize("name", ["bow_tie", "rank016", "rank015"])
def test_block_sweep_of_the_fig2_triangulations(eng, tmp_path, name):
    """The three printed d = 8 triangulations, swept as the exhaustive Fig. 2
    check sweeps them (TS_ENUM_REDUCED) and without flags.  On rank016 and
    rank015 most warps' half-diamonds leave more than 32 labels, so the lane
    loop that restores from the snapshot region runs too.  No odd-cycle flag
    is ever set when the snapshot is taken: before the middle row the two
    halves are linked only by antipodal pairs, so every cycle closed by then
    crosses between them an even number of times and has even parity."""
    edges = np.loadtxt(os.path.join(HERE, "golden", f"fig2_{name}.edges"), dtype=np.int32,
                       comments="#")
    exe = build_block_sweep(eng, tmp_path, 8, edges, count_snap=True)
    for mode in ("reduced", "plain"):
        out = run_block_sweep(exe, tmp_path, 12, mode)
        lanes = int(out.split("snapshot_lanes=")[1].split()[0])
        if name != "bow_tie":
            assert lanes >= 32 * 4, out   # at least 4 of the 12 warps
        assert int(out.split("odd_lanes=")[1].split()[0]) == 0, out
    run_block_sweep(exe, tmp_path, 16, "classify")


CUDA_INCLUDE = "/usr/local/cuda/include"   # host.cpp's headers and the runtime it links
CUDA_LIB = "/usr/local/cuda/lib64"


@pytest.fixture(scope="module")
def table_sweep_exe(tmp_path_factory):
    """The host build of the table-driven sweep driver (every degree)."""
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INCLUDE) or not os.path.isdir(CUDA_LIB):
        pytest.skip("needs g++ and the CUDA headers")
    csrc = os.path.join(ROOT, "paper_2604_09221_gb300", "csrc")
    exe = tmp_path_factory.mktemp("table_sweep") / "run"
    cmd = ["g++", "-std=c++17", "-O1", "-w", f"-I{csrc}", f"-I{os.path.join(HERE, 'host')}",
           f"-I{os.path.join(ROOT, 'oracle')}", f"-I{CUDA_INCLUDE}", "-o", str(exe),
           os.path.join(HERE, "host", "run_table_sweep.cpp"),
           "-x", "c", os.path.join(ROOT, "oracle", "tcurve_oracle.c"), "-x", "none",
           f"-L{CUDA_LIB}", f"-Wl,-rpath,{CUDA_LIB}", "-lcudart", "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("d", list(range(1, 17)))
def test_table_sweep_on_the_host(table_sweep_exe, tmp_path, d):
    """The table-driven sweep (both back ends, multi-word sign vectors and
    codes) compiled for the host, on the tables host.cpp builds, against the
    oracle: random and special sign vectors, the standard triangulation,
    (d >= 3) a regular one and (d >= 2) the fan triangulation, whose origin
    has 4d - 1 earlier neighbours in T^diamond (the longest fans the join
    list's flush schedule has to fit).  Every other instance keeps its label
    slots in a buffer of their own, sized to the table's slot count, as the
    kernels with global scratch keep them in shared memory, and every fourth
    one also reads fan entries rewritten to their slots' byte offsets, as
    those kernels stage them."""
    cases = [("standard", ti.standard_triangulation(d))]
    if d >= 3:
        cases.append(("regular", ti.regular_triangulation(d, seed=100 + d)))
    if d >= 2:
        cases.append(("fan", ti.fan_triangulation(d)))
    for name, edges in cases:
        np.savetxt(tmp_path / "tri.txt", edges, fmt="%d")
        out = subprocess.run([str(table_sweep_exe), str(d), str(tmp_path / "tri.txt"), "600"],
                             capture_output=True, text=True)
        assert out.returncode == 0, (name, out.stdout + out.stderr)


@pytest.mark.parametrize("d", list(range(1, 17)))
def test_warp_sweep_on_the_host(table_sweep_exe, tmp_path, d):
    """The warp-per-instance sweep (tc_warp_sweep.cuh) compiled for the host,
    its 32 lanes run one after another (forward for even instances, in
    reverse for odd ones: no phase may depend on the order of the lanes), on
    the tables host.cpp builds, against the oracle: standard, regular and fan
    triangulations, random and special sign vectors."""
    cases = [("standard", ti.standard_triangulation(d))]
    if d >= 3:
        cases.append(("regular", ti.regular_triangulation(d, seed=200 + d)))
    if d >= 2:
        cases.append(("fan", ti.fan_triangulation(d)))
    for name, edges in cases:
        np.savetxt(tmp_path / "tri.txt", edges, fmt="%d")
        out = subprocess.run([str(table_sweep_exe), str(d), str(tmp_path / "tri.txt"), "400", "warp"],
                             capture_output=True, text=True)
        assert out.returncode == 0, (name, out.stdout + out.stderr)
        assert "warp" in out.stdout


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


def expected_mask_words(d, flags, k):
    """The masks of include/tcurve.h written out with Python integers: k;
    k << 1 (TS_ENUM_FLIP); k with zero bits inserted at positions 0, 1 and
    d + 1 (TS_ENUM_REDUCED); word w = splitmix64(k * W + w), bits >= |A|
    cleared (TS_ENUM_SPLITMIX); schemes.orbit_mask (TS_ENUM_ORBITS, one
    word).  Words beyond the W sign words are dropped."""
    W, npts, m64 = ti.sign_words(d), ti.num_points(d), (1 << 64) - 1
    if flags == 8:
        return [orbit_mask(d, k)] + [0] * (W - 1)
    if flags == 4:
        words = [ti.splitmix64_int((k * W + w) & m64) for w in range(W)]
        top = npts - 64 * (W - 1)
        if top < 64:
            words[-1] &= (1 << top) - 1
        return words
    if flags == 1:
        m = k << 1
    elif flags == 2:
        low, high = k & ((1 << (d - 1)) - 1), k >> (d - 1)
        m = (low << 2) | (high << (d + 2))
    else:
        m = k
    return [(m >> (64 * w)) & m64 for w in range(W)]


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_orbit_masks_are_one_per_class(d):
    """TS_ENUM_ORBITS's masks over its whole range [0, 2^(|A|-3)) hold
    exactly one sign distribution of every (Z/2)^3 class (Sec. 3: sigma ->
    sigma + a + b i + c j mod 2), found by brute force over the group."""
    npts = ti.num_points(d)
    pts = [(i, j) for j in range(d + 1) for i in range(d + 1 - j)]   # bit k = index in this order
    pats = []
    for a in (0, 1):
        for b in (0, 1):
            for c in (0, 1):
                pats.append(sum(((a + b * i + c * j) % 2) << k for k, (i, j) in enumerate(pts)))
    assert len(set(pats)) == 8
    seen = set()
    for k in range(1 << (npts - 3)):
        m = orbit_mask(d, k)
        assert m < 1 << npts and not (m >> (d + 1)) & 1   # sigma(0, 1) = 0
        cls = min(m ^ p for p in pats)
        assert cls not in seen, (d, k)
        seen.add(cls)
    assert len(seen) == 1 << (npts - 3)


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_sweep_mask_maps_on_the_host(tmp_path):
    """tc_enum_sig against the mask maps' definitions, at the edges of the
    64-bit counter (carries from word 0 into word 1) for one to three sign
    words."""
    csrc = os.path.join(ROOT, "paper_2604_09221_gb300", "csrc")
    exe = tmp_path / "run"
    subprocess.run(["g++", "-std=c++17", "-O1", "-w", f"-I{os.path.join(HERE, 'host')}", f"-I{csrc}",
                    "-o", str(exe), os.path.join(HERE, "host", "run_enum_sig.cpp")],
                   check=True, capture_output=True)
    rng = np.random.default_rng(12)
    cases = []
    for d in (4, 5, 9, 10, 11, 12, 15, 16):
        ks = {0, 1, 2, (1 << (d - 1)) - 1, 1 << (d - 1), (1 << 62) + 5, (1 << 63) - 1, 1 << 63,
              (1 << 64) - 1, *[int(x) for x in rng.integers(0, 1 << 63, 6, dtype=np.int64)]}
        for flags in (0, 1, 2, 4, 8):
            if flags == 8 and ti.sign_words(d) > 1:
                continue   # the orbit sweep: one sign word (d <= 9)
            for k in sorted(ks):
                if ti.sign_words(d) == 1 and flags != 4 and k >= 1 << (ti.num_points(d) - 3):
                    continue   # one sign word: the ABI bounds the range so that masks fit
                cases.append((d, flags, k))
    inp = "".join(f"{d} {f} {k}\n" for d, f, k in cases)
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True)
    lines = out.stdout.split("\n")
    for (d, f, k), line in zip(cases, lines):
        assert [int(x, 16) for x in line.split()] == expected_mask_words(d, f, k), (d, f, k)
    assert len(lines) == len(cases) + 1
