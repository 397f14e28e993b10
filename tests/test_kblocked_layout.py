"""The value network's K-blocked activation layout (host logic, no GPU): the
library's own index function, compiled for the host, is a bijection onto the
matrix's elements, a 64-wide K slice of a 128-row tile is one contiguous
16 KB piece (one bulk copy), and the 8-column half of a 16-column block for 32
consecutive rows is 512 contiguous bytes (one coalesced warp store)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include "dvc_gemm.cuh"
int main() {
    const int R = 384, W = 640;
    for (int r = 0; r < R; ++r)
        for (int c = 0; c < W; ++c) std::printf("%zu\n", dvc::kblocked_index(r, c, W));
    return 0;
}
'''


@pytest.fixture(scope="module")
def index_table(tmp_path_factory):
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("kblocked")
    src, exe = d / "k.cu", d / "k"
    src.write_text(SRC)
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17",
                    "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_2403_10720_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return np.array(out.split(), dtype=np.int64).reshape(384, 640)


def test_bijection(index_table):
    flat = np.sort(index_table.ravel())
    assert (flat == np.arange(384 * 640)).all()


def test_k_slice_of_a_row_tile_is_one_piece(index_table):
    for m in range(3):
        for kc in range(640 // 64):
            idx = index_table[128 * m:128 * (m + 1), 64 * kc:64 * (kc + 1)]
            lo = idx.min()
            assert idx.max() - lo + 1 == 128 * 64                  # 16 KB of BF16, no gaps
            assert lo * 2 % 16 == 0                                 # 16-byte aligned start


def test_warp_store_is_contiguous(index_table):
    for r0 in (0, 32, 96, 160, 352):
        for c in (0, 8, 16, 632):
            idx = index_table[r0:r0 + 32, c:c + 8]
            assert (np.diff(idx.ravel()) == 1).all()                # 32 rows x 8 columns, one run of 256 elements
