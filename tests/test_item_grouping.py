"""Host logic of the work-item grouping (paper_2209_11337_gb300/csrc/qmccpw_internal.h,
set_item_grouping), compiled with the host compiler and run on the CPU.

A replicate's tiles are grouped into work items of tpi consecutive tiles:
tpi a power of two from 1 to 16, the largest that keeps at least 256 items
per replicate; the items cover every tile once and the last one is never
empty.  The grouping is a function of the tiles per replicate alone, which
is what makes a replicate's estimate the same in every call, batch,
replicate range and the server.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_11337_gb300", "csrc")

TILES = [1, 2, 3, 255, 256, 511, 512, 513, 1023, 1024, 1025, 2047, 2048, 4095, 4096, 4097, 8191, 8192, 8193,
         65536, 65537, 1 << 20, (1 << 24) + 5]

PROGRAM = r"""
#include <cstdio>
#include "qmccpw_internal.h"
int main() {
    const long long tiles[] = {%s};
    for (long long t : tiles) {
        qmccpw::ContractDev c{};
        c.tiles = static_cast<int32_t>(t);
        c.R = 7;
        qmccpw::set_item_grouping(c);
        std::printf("%%lld %%d %%d\n", t, c.tpi, c.items);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def grouping(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("grouping")
    src, exe = d / "grouping.cpp", d / "grouping"
    src.write_text(PROGRAM % ", ".join(str(t) for t in TILES))
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {int(t): (int(g), int(n)) for t, g, n in (line.split() for line in out.strip().splitlines())}


@pytest.mark.parametrize("tiles", TILES)
def test_grouping_covers_every_tile_with_enough_items(grouping, tiles):
    tpi, items = grouping[tiles]
    assert tpi in (1, 2, 4, 8, 16)
    assert (items - 1) * tpi < tiles <= items * tpi        # every tile once, the last item not empty
    if tpi > 1:
        assert items >= 256                                 # enough items per replicate to balance
    assert tpi == 16 or 2 * tpi * 256 > tiles               # the largest grouping that keeps 256


def test_large_contracts_take_sixteen_tiles_per_item(grouping):
    assert grouping[1 << 20][0] == 16 and grouping[8192][0] == 16
    assert grouping[511][0] == 1 and grouping[512][0] == 2
