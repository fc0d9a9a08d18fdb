"""CPU checks of host-side scheduling logic shared by the library: the z-segment length
the fused D3Q27 kernels march over (choose_tz in csrc/elbm_internal.h), compiled here
into a small host program against the library's own header (nvcc, no GPU needed)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_09512_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "elbm_internal.h"
int main() {
    int cases[][6] = {  // nx, ny, nz, tile height, SMs, CTAs per SM
        {256, 256, 256, 8, 152, 1}, {256, 256, 256, 8, 152, 2}, {128, 128, 128, 8, 152, 1},
        {128, 128, 128, 8, 152, 2}, {512, 512, 512, 8, 152, 1}, {19, 13, 11, 8, 152, 1},
        {256, 256, 256, 8, 0, 0}, {64, 64, 5, 8, 152, 2}};
    for (auto& c : cases) {
        elbm::KParams k{};
        k.nx = c[0]; k.ny = c[1]; k.nz = c[2];
        std::printf("%d\n", elbm::choose_tz(k, c[3], c[4], c[5], 64));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def tz_values():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "tz.cu")
        exe = os.path.join(d, "tz")
        with open(src, "w") as fh:
            fh.write(PROGRAM)
        subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [int(v) for v in out.split()]


def test_z_segments_of_the_bench_workload(tz_values):
    # 256^3 on 152 SMs: FP32 (one CTA per SM) keeps 64 planes (6.74 waves); FP16 (two
    # per SM) takes 37 (5.89 waves, a fuller last wave than 32 planes' 6.74)
    assert tz_values[0] == 64
    assert tz_values[1] == 37


def test_z_segments_stay_within_bounds(tz_values):
    for tz, nz in zip(tz_values, (256, 256, 128, 128, 512, 11, 256, 5)):
        assert 1 <= tz <= min(nz, 128)
    assert tz_values[5] == 11          # a grid shorter than 16 planes keeps one segment
    assert tz_values[6] == 64          # without device information the fallback stands
    assert tz_values[7] == 5


def test_z_segment_choice_fills_the_last_wave(tz_values):
    """Every choice scores at least as well as the fallback by the rule the header
    states: last-wave fill times tz / (tz + 2)."""
    import math

    def score(nx, ny, nz, ty, sms, per_sm, tz):
        tiles = math.ceil(nx / 32) * math.ceil(ny / ty)
        waves = tiles * math.ceil(nz / tz) / (sms * per_sm)
        return waves / math.ceil(waves) * tz / (tz + 2.0)

    for (nx, ny, nz, ty, sms, per), tz in zip(((256, 256, 256, 8, 152, 1), (256, 256, 256, 8, 152, 2),
                                               (128, 128, 128, 8, 152, 1), (128, 128, 128, 8, 152, 2),
                                               (512, 512, 512, 8, 152, 1)), tz_values[:5]):
        assert score(nx, ny, nz, ty, sms, per, tz) >= score(nx, ny, nz, ty, sms, per, min(64, nz)) - 1e-12
