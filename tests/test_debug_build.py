"""The debug build's bounds checks (-DTILD_DEBUG=1) compile: a translation
unit that instantiates the bead kernels in every mode (where the checks
live) and the binning kernels is compiled for sm_103a with the flag on, and
with it off (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2302_02474_gb300 import _build

TU = r'''
#include "bead_kernels.cuh"
namespace tild {
template __global__ void bead_kernel<2, kModeStep, float>(BeadParams<float>, BeadBuffers<float>);
template __global__ void bead_kernel<2, kModeForce, float>(BeadParams<float>, BeadBuffers<float>);
template __global__ void bead_kernel<3, kModeSpread, double>(BeadParams<double>, BeadBuffers<double>);
template __global__ void bin_count_fine<float>(int, const float*, const float*, const float*, float, int, int, int, int,
                                              int, Topology, const unsigned char*, const int*, int*, int*, int*);
}
'''


@pytest.mark.parametrize("debug", [True, False])
def test_bead_kernels_compile_with_and_without_the_debug_checks(tmp_path, debug):
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("no nvcc")
    src = tmp_path / "debug_tu.cu"
    src.write_text(TU)
    cmd = [_build._nvcc(), *_build.ARCH, *_build.FLAGS, "-I", _build.CSRC, "-c", str(src), "-o",
           str(tmp_path / "debug_tu.o")]
    if debug:
        cmd.insert(-4, "-DTILD_DEBUG=1")
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
