"""The Poisson sweep ordering of the CUDA path, checked on the host (no GPU):
the colour functions of csrc/elbm_device.cuh are __host__ __device__, so a
small host program compiled by nvcc runs them here. Red-black, (x + y + z)
mod 2, where every periodic extent is even; three colours where one is odd.
Every face neighbour (the periodic wrap included) must have another colour,
otherwise a parallel sweep would update two neighbours at once."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

SRC = r'''
#include <cstdio>
#include "elbm_device.cuh"
using namespace elbm;
int main()
{
    int bad = 0, cases = 0, three = 0;
    for (int nx = 2; nx <= 13; nx++)
        for (int ny = 2; ny <= 7; ny++)
            for (int nz = 1; nz <= 5; nz++)
                for (int pm = 0; pm < 8; pm++) {
                    const int per[3] = {pm & 1, (pm >> 1) & 1, (pm >> 2) & 1};
                    const int n[3] = {nx, ny, nz};
                    const int nc = ncolors_of(per, nx, ny, nz);
                    cases++;
                    if (nc == 3) three++;
                    for (int z = 0; z < nz; z++)
                        for (int y = 0; y < ny; y++)
                            for (int x = 0; x < nx; x++) {
                                const int c = nc == 3 ? color3(per, x, y, z, nx, ny, nz) : ((x + y + z) & 1);
                                if (c < 0 || c >= nc) bad++;
                                const int p[3] = {x, y, z};
                                for (int a = 0; a < 3; a++) {
                                    int q[3] = {p[0], p[1], p[2]};
                                    q[a] = p[a] + 1;
                                    if (q[a] >= n[a]) {
                                        if (!per[a] || n[a] == 1) continue;
                                        q[a] = 0;
                                    }
                                    const int d = nc == 3 ? color3(per, q[0], q[1], q[2], nx, ny, nz)
                                                          : ((q[0] + q[1] + q[2]) & 1);
                                    if (d == c) bad++;
                                }
                            }
                }
    printf("%d %d %d\n", cases, three, bad);
    return 0;
}
'''


def test_sweep_colouring_is_proper_for_every_extent(tmp_path):
    from paper_1612_05404_gb300 import build
    nvcc = build.nvcc()
    if not shutil.which(nvcc) and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "colouring.cu"
    src.write_text(SRC)
    exe = tmp_path / "colouring"
    csrc = os.path.join(ROOT, "paper_1612_05404_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", csrc, "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    cases, three, bad = (int(v) for v in out)
    assert cases == 12 * 6 * 5 * 8 and three > 0 and bad == 0, out
