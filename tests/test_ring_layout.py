"""CPU check of the FE_BF16R forward GEMM's window-row ring (no GPU).

The tensor-core kernel's FE_BF16R form reads the forward A operand in place
from a ring of u^{n+1} rows: entry (row r, column c) holds the 8 window
values u(r, c .. c + 7) of the hi and of the lo plane, row r sits in slot
r % XSLOTS (the first XMIRROR slots also after the last one), and window row
dy of block b is one MMA whose A operand starts at the slot of row 4 b + dy.
This test takes the layout constants from the kernel's own header (a small
host program compiled with nvcc), replays the kernel's ring writes in their
order (10 rows before block 0, then rows 4 b + 10 .. 4 b + 13 before block
b + 1) and checks that every byte each MMA reads lies in the ring and holds
the row and column of its pixel's window.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r'''
#include "fe_tc_kernel.cuh"
#include <cstdio>
int main() {
    using C = fe::Cfg<3>;
    printf("%zu %zu %zu %zu %zu %d %d %d %d %d %d %d %d\n", C::OFF_R, C::R_BYTES, C::OFF_AF, C::AF_BYTES, C::OFF_H,
           C::XSLOTS, C::XMIRROR, C::XROW_BYTES, C::XPLANE, C::PL_WORDS, fe::PP, fe::R3X, fe::R6Y);
    return 0;
}
'''


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("ring")
    src, exe = d / "ring.cu", d / "ring"
    src.write_text(PROBE)
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1404_5344_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    keys = ("OFF_R R_BYTES OFF_AF AF_BYTES OFF_H XSLOTS XMIRROR XROW XPLANE PL_WORDS PP R3X R6Y").split()
    return dict(zip(keys, vals))


def test_ring_rows_and_bounds(layout):
    L = layout
    R3X, R6Y, KS, NBLK = L["R3X"], L["R6Y"], 7, L["R6Y"] // 4 - 1
    row_words = L["PP"] * 2 // 4
    ring = {}

    def write(r, c, pl):
        w0 = r * row_words + (c >> 1)                     # the five source words of the entry
        assert 0 <= r < R6Y and (c >> 1) + 4 < row_words and w0 + 4 < L["PL_WORDS"]
        slot = r % L["XSLOTS"]
        for s in [slot] + ([slot + L["XSLOTS"]] if slot < L["XMIRROR"] else []):
            off = pl * L["XPLANE"] + s * L["XROW"] + c * 16
            assert 0 <= off and off + 16 <= L["AF_BYTES"]
            ring[(pl, off)] = (r, c)

    def mma(b):
        for dy in range(KS):
            start = ((4 * b + dy) % L["XSLOTS"]) * L["XROW"]
            for m in range(128):
                for kc in range(2):                       # K chunk 0: hi plane, 1: lo plane
                    off = start + (m // 8) * 128 + (m % 8) * 16 + kc * L["XPLANE"]
                    assert off + 16 <= L["AF_BYTES"]
                    assert ring.get((kc, off)) == (4 * b + dy + m // 32, m % 32), (b, dy, m, kc)

    assert NBLK == 16 and R3X == 32
    for e in range(2 * L["XSLOTS"] * R3X):                 # rows 0..9 before block 0
        pl, rem = divmod(e, L["XSLOTS"] * R3X)
        write(rem // R3X, rem % R3X, pl)
    mma(0)
    for b in range(NBLK - 1):                              # rows 4b+10 .. 4b+13 before block b+1
        for tid in range(256):
            write(4 * b + 10 + ((tid >> 5) & 3), tid & 31, tid >> 7)
        mma(b + 1)
    assert max(r for r, _ in ring.values()) == R6Y - 1
    assert L["OFF_R"] + L["R_BYTES"] <= L["OFF_AF"] and L["OFF_AF"] + L["AF_BYTES"] <= L["OFF_H"]
