"""CPU check of the BF16 forms' forward GEMM window-row ring (no GPU).

The tensor-core kernel's BF16 forms read the forward A operand in place
from a ring of u^{n+1} rows: entry (row r, column c) holds the 8 window
values u(r, c .. c + 7) of the hi and of the lo plane, row r sits in slot
r % XSLOTS (the first XMIRROR slots also after the last one), and window
rows 2j, 2j + 1 of block b are one MMA whose A operand starts at the slot of
row 4 b + 2j with its second K chunk one slot further (row 7 is the
bank's zero-weight padding row: its chunk must only read finite ring data).
This test takes the layout constants from the kernel's own header (a small
host program compiled with nvcc), replays the kernel's ring writes in their
order (10 rows before block 0, then rows 4 b + 10 .. 4 b + 13 before block
b + 1) and checks, for both BF16 forms, that every byte each MMA reads lies
in the ring and holds the row and column of its pixel's window (the padding
row: some written ring row).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r'''
#include "fe_tc_kernel.cuh"
#include <cstdio>
template <int F> void show() {
    using C = fe::Cfg<F>;
    printf("%zu %zu %zu %zu %zu %d %d %d %d %d %d %d %d\n", C::OFF_R, C::R_BYTES, C::OFF_AF, C::AF_BYTES, C::OFF_H,
           C::XSLOTS, C::XMIRROR, C::XROW_BYTES, C::XPLANE, C::PL_WORDS, fe::PP, fe::R3X, fe::R6Y);
}
int main() {
    show<1>();
    show<3>();
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
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines()
    keys = ("OFF_R R_BYTES OFF_AF AF_BYTES OFF_H XSLOTS XMIRROR XROW XPLANE PL_WORDS PP R3X R6Y").split()
    return {fmt: dict(zip(keys, (int(v) for v in line.split()))) for fmt, line in zip((1, 3), lines)}


@pytest.mark.parametrize("fmt", [1, 3])
def test_ring_rows_and_bounds(layout, fmt):
    L = layout[fmt]
    R3X, R6Y, KS, NBLK = L["R3X"], L["R6Y"], 7, L["R6Y"] // 4 - 1
    row_words = L["PP"] * 2 // 4
    ring = {}

    def write(r, c, pl):
        w0 = r * row_words + (c >> 1)                     # the five source words of the entry
        assert 0 <= r < R6Y and (c >> 1) + 4 < row_words and w0 + 4 < L["PL_WORDS"]
        slot = r % L["XSLOTS"]
        for s in [slot] + ([slot + L["XSLOTS"]] if slot < L["XMIRROR"] else []):
            off = s * L["XROW"] + c * 16
            assert 0 <= off and off + 16 <= L["XPLANE"] and 2 * L["XPLANE"] <= L["AF_BYTES"]
            ring[(pl, off)] = (r, c)

    def mma(b):
        for pl in range(2):                               # hi plane, lo plane
            for j in range(4):                            # window rows 2j, 2j + 1
                start = pl * L["XPLANE"] + ((4 * b + 2 * j) % L["XSLOTS"]) * L["XROW"]
                for m in range(128):
                    for kc in range(2):                   # K chunk: window row 2j + kc
                        off = start + (m // 8) * 128 + (m % 8) * 16 + kc * L["XROW"]
                        assert pl * L["XPLANE"] <= off and off + 16 <= (pl + 1) * L["XPLANE"]
                        dy = 2 * j + kc
                        got = ring.get((pl, off - pl * L["XPLANE"]))
                        if dy < KS:
                            assert got == (4 * b + dy + m // 32, m % 32), (b, pl, j, m, kc, got)
                        else:                             # the padding row (weight 0): any written entry
                            assert got is not None, (b, pl, j, m)

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
