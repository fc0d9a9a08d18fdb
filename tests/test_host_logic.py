"""CPU checks of host-side logic shared by the library, compiled here into small host
programs against the library's own header (nvcc, no GPU needed): the z-segment length the
fused D3Q27 kernels march over (choose_tz in csrc/elbm_internal.h), and the scratch layout
of the allocation-free step (noalloc_layout), whose size decides which grids that entry
point rejects before launching anything."""
import os
import shutil
import subprocess
import sys
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


NOALLOC_PROGRAM = r"""
#include <cstdio>
#include "elbm_internal.h"
// largest node count whose layout fits the static scratch, for D values of `real` bytes
static long long max_nodes(int D, size_t real) {
    long long lo = 1, hi = 1LL << 31;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (elbm::noalloc_layout(mid, D, real).bytes <= elbm::kNoallocScratchBytes) lo = mid; else hi = mid - 1;
    }
    return lo;
}
int main() {
    std::printf("%zu\n", elbm::kNoallocScratchBytes);
    std::printf("%lld %lld %lld %lld\n", max_nodes(3, 4), max_nodes(3, 8), max_nodes(2, 4), max_nodes(2, 8));
    const elbm::NoallocLayout a = elbm::noalloc_layout(128LL * 128 * 128, 3, 4);
    const elbm::NoallocLayout b = elbm::noalloc_layout(29LL * 17 * 11, 3, 8);
    std::printf("%zu %zu\n", a.bytes, b.bytes);
    std::printf("%zu %zu %zu %lld\n", b.status, b.partials, b.qfield, elbm::blocks_1d_of(29LL * 17 * 11));
    return 0;
}
"""


@pytest.fixture(scope="module")
def noalloc_values():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "na.cu")
        exe = os.path.join(d, "na")
        with open(src, "w") as fh:
            fh.write(NOALLOC_PROGRAM)
        subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return [[int(v) for v in line.split()] for line in out.strip().splitlines()]


def test_noalloc_scratch_limits(noalloc_values):
    """The grid limits stated in include/elbm.h for elbm_step_noalloc: about 1.37 M nodes
    for D3Q27 with an FP32 arithmetic type (FP32, FP16 and BF16 stores), 0.69 M for FP64,
    2.05 M for D2Q9 FP32 in 16 MiB of scratch."""
    cap = noalloc_values[0][0]
    assert cap == 16 << 20
    d3_f32, d3_f64, d2_f32, d2_f64 = noalloc_values[1]
    assert 1.37e6 <= d3_f32 < 1.39e6
    assert 0.68e6 <= d3_f64 < 0.70e6
    assert 2.05e6 <= d2_f32 < 2.07e6
    assert 1.03e6 <= d2_f64 < 1.05e6


def test_noalloc_rejects_grids_beyond_its_scratch(noalloc_values):
    """128^3 D3Q27 FP32 needs 25 MB of scratch (rejected); the GPU test's 29 x 17 x 11
    FP64 grid fits, with the partials sized by the two-pass grid (256 threads per CTA)."""
    big, small = noalloc_values[2]
    assert big > 16 << 20
    assert small <= 16 << 20
    status, partials, qfield, nblocks = noalloc_values[3]
    assert status == 0 and partials == 256 and nblocks == (29 * 17 * 11 + 255) // 256
    assert qfield >= partials + 5 * 8 * nblocks and qfield % 256 == 0


NOALLOC_CALL = r"""
import sys
sys.path.insert(0, sys.argv[1])
from paper_2102_09512_gb300 import elbm as E
big = E.make_params(3, 128, 128, 128, store="f32")
small = E.make_params(3, 29, 17, 11, store="f64")
# dummy 256-byte-aligned pointers: no kernel may ever see them (no device is visible)
print(E.elbm_step_noalloc(big, 4096, 8192, 0), E.elbm_step_noalloc(small, 4096, 8192, 0))
"""


def test_noalloc_entry_point_rejects_before_any_cuda_call():
    """The entry point itself, called in a process that sees no GPU: the oversized grid is
    rejected (ELBM_ERR_UNSUPPORTED) before any CUDA call, while a grid that fits gets as
    far as the device lookup and fails there (ELBM_ERR_CUDA).  No kernel can run."""
    lib = os.path.join(ROOT, "paper_2102_09512_gb300", "_build", "libelbm.so")
    if not os.path.exists(lib):
        pytest.skip("libelbm.so is not built")
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", NOALLOC_CALL, ROOT], env=env, check=True,
                         capture_output=True, text=True).stdout.split()
    assert [int(v) for v in out] == [-2, -3]
