"""Host check of the storages of a level's BF16 factor (``fac_index`` in
``csrc/lsw_internal.cuh``): the two operand-tile layouts of the tensor-core
level products are permutations of a block's nb x rp entries, a stage of the
partials (64 rows, every column) and a row tile of the apply (128 rows, every
column) each occupy one contiguous range (one bulk copy each), and the
column-major storage is the plain column-major index.  Compiled with nvcc as a
host program; no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "lsw_internal.cuh"
using namespace lsw;
int main() {
    int bad = 0;
    const int shapes[][3] = {{128, 40, 3}, {256, 12, 2}, {1024, 64, 2}, {384, 8, 4}, {512, 20, 2}};
    for (auto& sh : shapes) {
        const int nb = sh[0], r = sh[1], nblk = sh[2], rp = (r + 7) & ~7;
        for (int lay : {FAC_TILE_P, FAC_TILE_A}) {
            std::vector<int> hit((size_t)nblk * nb * rp, 0);
            for (int j = 0; j < nblk; ++j)
                for (int o = 0; o < nb; ++o)
                    for (int i = 0; i < rp; ++i) {
                        const long long e = fac_index(lay, nb, r, rp, j, o, i);
                        if (e < 0 || e >= (long long)hit.size()) { ++bad; continue; }
                        ++hit[e];
                    }
            for (int h : hit) if (h != 1) ++bad;
            const int rows = lay == FAC_TILE_P ? 64 : 128;
            for (int j = 0; j < nblk; ++j)
                for (int o0 = 0; o0 + rows <= nb; o0 += rows) {
                    const long long b0 = fac_index(lay, nb, r, rp, j, o0, 0);
                    for (int o = o0; o < o0 + rows; ++o)
                        for (int i = 0; i < rp; ++i) {
                            const long long e = fac_index(lay, nb, r, rp, j, o, i);
                            if (e < b0 || e >= b0 + (long long)rows * rp) ++bad;
                        }
                }
        }
        for (int j = 0; j < nblk; ++j)
            for (int o = 0; o < nb; ++o)
                for (int i = 0; i < r; ++i)
                    if (fac_index(FAC_PLAIN, nb, r, rp, j, o, i) != ((long long)j * r + i) * nb + o) ++bad;
    }
    printf("%d\n", bad);
    return bad != 0;
}
"""


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_factor_tile_layouts_are_contiguous_permutations(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not available")
    src = tmp_path / "fac_layout.cu"
    exe = tmp_path / "fac_layout"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                        "-I", os.path.join(ROOT, "paper_2005_01372_gb300", "csrc"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "0", out.stdout + out.stderr
