"""Host-side logic without a GPU.

* The ctypes structures of the binding have the size and field offsets of the
  C structures in include/rix.h (compiled here with the host C compiler), so
  no option or statistic is read from the wrong place.
* The bench's FLOP bookkeeping: the screened counts replace the setup-time
  ones, and each stage's rate is quoted on the pipe that runs it.
"""
import ctypes
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2403_10343_gb300 import rix  # noqa: E402
import bench  # noqa: E402


def _c_layout(struct, fields):
    """sizeof and offsetof of a C struct of include/rix.h, from the host compiler."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields]
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"rix.h\"\nint main(void) {\n"
           + "\n".join(lines) + "\nreturn 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run([cc, "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(x) for x in out[1:]]


@pytest.mark.parametrize("py, c", [(rix._System, "rix_system"), (rix._Options, "rix_options"),
                                   (rix._Stats, "rix_stats_t")])
def test_binding_structs_match_header(py, c):
    names = [f for f, _ in py._fields_]
    size, offs = _c_layout(c, names)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, f).offset for f in names] == offs


STATS = {
    "flops_stage": [10.0, 1.0, 40.0, 20.0, 8.0, 2.0], "flops_fp64": 81.0, "flops_term2": 6.0,
    "flops_term1_tc": 30.0, "flops_z_tc": 20.0, "flops_t_tc": 10.0, "tensor_flops": 1e4,
    "tensor_flops_stage": [1e3, 2e3, 3e3, 2.5e3, 1.5e3],
}


def test_screened_counts_replace_setup_counts():
    cnt = {"T": 5.0, "U2": 1.0, "X12": 30.0, "Z": 12.0, "X34": 8.0, "sym": 2.0, "term2": 4.0,
           "term1_tc": 20.0, "z_tc": 12.0, "t_tc": 5.0}
    s = bench.screened(STATS, cnt)
    assert s["flops_stage"] == [5.0, 1.0, 30.0, 12.0, 8.0, 2.0]
    assert s["flops_fp64"] == 58.0 and s["flops_fp64_unscreened"] == 81.0
    assert (s["flops_term2"], s["flops_term1_tc"], s["flops_z_tc"], s["flops_t_tc"]) == (4.0, 20.0, 12.0, 5.0)
    assert s["tensor_flops"] == STATS["tensor_flops"]  # issued tensor FLOPs do not depend on screening


def test_stage_split_between_pipes():
    # FP64 build: every stage on the FP64 pipe with its whole count
    for st, i in (("T", 0), ("U2", 1), ("X12", 2), ("Z", 3), ("X34", 4)):
        assert bench.stage_flops(STATS, st, "fp64") == STATS["flops_stage"][i]
        assert bench.stage_fp64_share(STATS, st, "fp64") == 1.0
    # mixed build: terms 1 (moved part) and 2 form TC12, the FP64 kernel keeps the rest of X12
    assert bench.stage_flops(STATS, "TC12", "mixed") == 36.0
    assert bench.stage_flops(STATS, "X12", "mixed") == 4.0
    assert bench.stage_fp64_share(STATS, "X34", "mixed") == 0.0
    assert bench.stage_fp64_share(STATS, "Z", "mixed") == 0.0
    assert bench.stage_fp64_share(STATS, "T", "mixed") == 0.0


def test_term1_flops_follow_the_stage_that_runs_them():
    # several row blocks: term 1 on the tensor cores runs per block inside the X12 stage, so
    # TC12 holds term 2 only and X12 holds the FP64 remainder plus the tensor-core term 1
    st = dict(STATS, n_row_blocks=3)
    assert bench.stage_flops(st, "TC12", "mixed") == 6.0
    assert bench.stage_flops(st, "X12", "mixed") == 34.0
    assert bench.stage_flops(dict(STATS, n_row_blocks=1), "TC12", "mixed") == 36.0
    # the FP64 build is unaffected by the block count
    assert bench.stage_flops(st, "X12", "fp64") == 40.0


def test_traffic_scales_with_the_mmas_of_a_launch():
    gemm = {"ms_per_build": 2.0, "launches_per_build": 4.0, "stage_pairs_per_build": 1000.0}
    roof = bench.roofline("mixed", {"stats": STATS, "stage_ms": {}, "gemm": gemm})
    if bench.GEMM_DRAM_BYTES_PER_STAGE_PAIR is None:
        assert roof["traffic"] is None
    else:
        assert roof["traffic"] == bench.GEMM_DRAM_BYTES_PER_STAGE_PAIR * 250.0


def test_roofline_picks_the_longest_stage():
    r = {"stats": STATS, "stage_ms": {"T": 1.0, "U2": 0.5, "X12": 10.0, "Z": 4.0, "X34": 2.0}}
    roof = bench.roofline("fp64", r)
    assert roof["kernel"] == "k_X12" and roof["bound"] == "alu"
    assert abs(roof["achieved"] - 40.0 / 1e-2 / 1e12) < 1e-18
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-18


def test_tensor_roofline_uses_algorithmic_flops_over_kernel_time():
    # mixed: k_gemm_sliced, algorithmic FLOPs of the tensor-core work over its launch time
    gemm = {"ms_per_build": 2.0, "launches_per_build": 4.0, "stage_pairs_per_build": 1000.0}
    r = {"stats": STATS, "stage_ms": {"TC12": 5.0}, "gemm": gemm}
    roof = bench.roofline("mixed", r)
    alg = 10.0 + 30.0 + 6.0 + 20.0 + 8.0          # T, term 1, term 2, Z on the tensor cores + terms 3+4
    assert bench.tensor_alg_flops(STATS) == alg
    assert roof["kernel"] == "k_gemm_sliced" and roof["bound"] == "tensor"
    assert abs(roof["achieved"] - alg / 2e-3 / 1e12) < 1e-24
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-24
    issued = 1000.0 * 2 * 128 * 80 * 16
    assert roof["issued_bf16_flops_per_build"] == issued
    assert abs(roof["issued_tflops"] - issued / 2e-3 / 1e12) < 1e-9
