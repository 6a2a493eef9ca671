"""CPU: the class mapping's launch grid (class_grid in the library's launch code), compiled for the
host with nvcc and checked on frame and row-band shapes up to the largest the ABI accepts.

The grid is (4 row classes x band height, patch columns, bands); the kernel takes patch row
blockIdx.z * band height + blockIdx.x / 4.  So every patch row of the launch must fall in exactly
one (band, row) slot, no band may be empty, the raster order (bands of one patch row) must be kept
when no band height is asked for, and the grid must stay within CUDA's limits."""
import os
import shutil
import subprocess

import pytest

import paper_2301_11376_gb300 as ssilvb

HELPER = r'''
#include <cstdio>
#include "launch_impl.cuh"
int main() {
    int W, y0, y1, band;
    while (std::scanf("%d %d %d %d", &W, &y0, &y1, &band) == 4) {
        ssilvb::GatherParams P{};
        P.W = W;
        P.y0 = y0;
        P.y1 = y1;
        P.band_rows = band;
        const dim3 g = ssilvb::class_grid(P);
        std::printf("%u %u %u\n", g.x, g.y, g.z);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def grid_tool(tmp_path_factory):
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("grid")
    src = d / "grid.cu"
    src.write_text(HELPER)
    exe = d / "grid"
    csrc = os.path.join(os.path.dirname(ssilvb.__file__), "csrc")
    subprocess.run(["nvcc", "-std=c++17", "-I" + ssilvb.INCLUDE, "-I" + csrc, "-o", str(exe), str(src)], check=True,
                   capture_output=True)
    return exe


def _cases():
    out = []
    for W in (1, 31, 32, 33, 333, 1920, 2560, 3840, 16384):
        for H in (1, 15, 16, 17, 77, 1080, 1100, 1440, 1601, 2160, 16384):
            for band in (1, 32):
                out.append((W, 0, H, band))
    # row bands of the host-buffer path: uneven cuts of a 4K frame, offsets not multiples of 16
    cuts = [0, 393, 747, 1062, 1338, 1574, 1771, 1928, 2160]
    for a, b in zip(cuts, cuts[1:]):
        out.append((3840, a, b, 32))
        out.append((3840, a, b, 1))
    out.append((6, 0, 16384, 32))
    out.append((16384, 0, 5, 32))
    return out


def test_class_grid_covers_every_patch_row_once(grid_tool):
    cases = _cases()
    inp = "".join(f"{W} {y0} {y1} {band}\n" for W, y0, y1, band in cases)
    r = subprocess.run([str(grid_tool)], input=inp, capture_output=True, text=True, check=True)
    rows = [tuple(int(v) for v in line.split()) for line in r.stdout.strip().splitlines()]
    assert len(rows) == len(cases)
    for (W, y0, y1, band), (gx, gy, gz) in zip(cases, rows):
        px, py = (W + 31) // 32, (y1 - y0 + 15) // 16
        assert gx % 4 == 0 and gx >= 4, (W, y0, y1, band)
        th = gx // 4
        assert gy == px
        if band <= 1:
            assert th == 1 and gz == py  # raster order
        else:
            assert th <= band
        assert gz * th >= py and (gz - 1) * th < py  # every row in a slot, no empty band
        assert gy <= 65535 and gz <= 65535
        # each patch row in exactly one (band z, row r < th) slot of prow = z * th + r
        slots = {}
        for z in range(gz):
            for rr in range(th):
                slots.setdefault(z * th + rr, []).append((z, rr))
        assert all(len(slots[p]) == 1 for p in range(py))
