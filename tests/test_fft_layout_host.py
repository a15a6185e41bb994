"""CPU check of the z passes' shared-memory line layout (no GPU call).

A host program compiled with nvcc prints, for every row length the library supports, the
values a thread and the line stride that the z kernels use (`z_values`, `z_line` in
fft_engine.cuh).  The checks: a line holds the padded Stockham layout and the unpadded
layout of the real-transform split (index M included), and rows that share a 16-lane phase
of a warp's 8-byte shared-memory accesses fall into disjoint banks, so those accesses are
free of bank conflicts.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_13394_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "fft_engine.cuh"
template <int LOGN> void row() {
  std::printf("%d %d %d\n", LOGN, pmnu::fft::z_values<LOGN>(), pmnu::fft::z_line<LOGN>());
}
int main() {
  row<5>(); row<6>(); row<7>(); row<8>(); row<9>(); row<10>(); row<11>();
  return 0;
}
"""


@pytest.fixture(scope="module")
def layouts(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("zline")
    src, exe = d / "zline.cu", d / "zline"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [tuple(int(x) for x in line.split()) for line in out.split("\n") if line.strip()]


def test_every_row_length_is_listed(layouts):
    assert [r[0] for r in layouts] == list(range(5, 12))


def test_line_holds_both_layouts(layouts):
    for logn, v, ls in layouts:
        m = 1 << (logn - 1)
        pad = 32 if v >= 32 else 16
        assert m % v == 0
        assert ls >= m + (m - 1) // pad + 1       # padded Stockham layout: index pad(M - 1)
        assert ls >= m + 1                       # unpadded split: index M (c2r)


def test_rows_in_one_phase_use_disjoint_banks(layouts):
    # 8-byte accesses: a warp's request splits into two phases of 16 lanes; a row is held by
    # tpl = M / V consecutive lanes, so 16 / tpl rows share a phase.  Lane j of row q reads
    # float2 q * ls + base + j (base: the same offset for every row), i.e. 32-bit banks
    # 2 (q ls + base + j) and the next one, mod 32.
    for logn, v, ls in layouts:
        m = 1 << (logn - 1)
        tpl = m // v
        rows = max(1, 16 // tpl)
        for base in range(0, 64, 3):
            banks = []
            for q in range(rows):
                for j in range(min(tpl, 16)):
                    w = 2 * (q * ls + base + j)
                    banks += [w % 32, (w + 1) % 32]
            assert len(banks) == len(set(banks)), (logn, v, ls, base)
