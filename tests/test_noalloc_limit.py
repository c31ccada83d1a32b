"""Host-side check of the size limit of the allocation-free conservation sums:
the check in csrc/noalloc_limits.h, compiled on its own with the host C++
compiler (no GPU), accepts up to 65,536 reduction blocks of 256 cells and at
most 4 variables, and rejects anything larger."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2106_06280_gb300", "csrc", "noalloc_limits.h")

PROG = r'''
#include <stdio.h>
#include "%s"
int main(void)
{
    const long long cases[][2] = {{1, 1}, {256, 4}, {257, 4}, {16777216LL, 4}, {16777217LL, 4}, {16777216LL, 5},
                                  {0, 1}, {100, 0}, {65536LL * 256 - 1, 1}, {65537LL * 256, 1}};
    for (unsigned i = 0; i < sizeof(cases) / sizeof(cases[0]); ++i)
        printf("%%d", (int)csw_noalloc_fits(cases[i][0], (int)cases[i][1]));
    printf("\n");
    return 0;
}
'''


def test_noalloc_size_check():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        with open(src, "w") as f:
            f.write(PROG % HDR)
        subprocess.check_call(["g++", "-O1", "-o", exe, src])
        out = subprocess.check_output([exe], text=True).strip()
    # 1 cell; 256 cells x 4 vars; 257 (two blocks); the maximum; one cell over; 5 vars;
    # no cells; no variables; last cell of the last block; one block over
    assert out == "1111000010", out
