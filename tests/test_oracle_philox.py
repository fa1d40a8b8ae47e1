"""Pins for the oracle's Philox4x32-10 (the noise source of Eq. 2).

The generator is the published Philox4x32-10 (Salmon, Moraes, Dror & Shaw,
SC'11).  The oracle's C implementation is pinned against an independent
implementation: PyTorch's open-source ``at::philox_engine`` header, compiled
here with g++ (mapping: key = seed, counter = (offset lo, offset hi,
subsequence lo, subsequence hi)).  A statistical check guards the 24-bit
uniform that the alignment step draws from word 0.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

CASES = [
    (0, 0, 0),
    (1, 0, 0),
    (1, 7, 3),
    (0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF, 0xFFFFFFFFFFFFFFFF),
    (0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0),
    (12345, (5 << 32) | 2047, (3 << 32) | 49),
]

ATEN_SRC = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdlib>
int main(int argc, char** argv) {
  for (int a = 1; a + 2 < argc; a += 3) {
    unsigned long long seed = strtoull(argv[a], 0, 0);
    unsigned long long sub = strtoull(argv[a + 1], 0, 0);
    unsigned long long off = strtoull(argv[a + 2], 0, 0);
    at::philox_engine eng(seed, sub, off);
    unsigned w0 = eng(), w1 = eng(), w2 = eng(), w3 = eng();
    printf("%u %u %u %u\n", w0, w1, w2, w3);
  }
  return 0;
}
"""


def _aten_outputs(cases):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    try:
        from torch.utils.cpp_extension import include_paths
        incs = include_paths()
    except Exception:
        pytest.skip("torch headers not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cpp")
        exe = os.path.join(d, "p")
        with open(src, "w") as f:
            f.write(ATEN_SRC)
        cmd = [gxx, "-std=c++17", "-O1", src, "-o", exe] + [f"-I{p}" for p in incs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("could not compile the ATen Philox header: " + r.stderr[-300:])
        args = []
        for s, sub, off in cases:
            args += [str(s), str(sub), str(off)]
        out = subprocess.check_output([exe] + args, text=True)
    return [list(map(int, line.split())) for line in out.strip().splitlines()]


def test_philox_matches_aten_engine(orc):
    ref = _aten_outputs(CASES)
    for (seed, sub, off), want in zip(CASES, ref):
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = orc.philox4x32_10(ctr, key)
        assert list(map(int, got)) == want, (seed, sub, off)


def test_philox_counter_layout_used_by_the_noise(orc):
    """The noise counter is (particle id, step, replica, 0) with key = seed;
    in the ATen mapping that is offset = id | step<<32, subsequence = replica."""
    ids = [0, 1, 2047, 4194303]
    steps = [0, 1, 49, 199]
    reps = [0, 511]
    cases = [(1, r, i | (t << 32)) for i in ids for t in steps for r in reps]
    ref = _aten_outputs(cases)
    for (seed, sub, off), want in zip(cases, ref):
        got = orc.philox4x32_10([off & 0xFFFFFFFF, off >> 32, sub, 0], [seed, 0])
        assert list(map(int, got)) == want


def test_unit24_uniformity(orc):
    """u = (w0 >> 8) * 2^-24 over 2^14 consecutive ids: chi-square on 64 bins."""
    n = 1 << 14
    u = np.array([orc.philox4x32_10([i, 3, 0, 0], [1, 0])[0] >> 8 for i in range(n)],
                 dtype=np.float64) / 2.0 ** 24
    assert u.min() >= 0.0 and u.max() < 1.0
    h, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    e = n / 64.0
    chi2 = float(((h - e) ** 2 / e).sum())
    # 63 dof: mean 63, sd ~11.2; 120 is > 5 sd
    assert chi2 < 120.0, chi2
    assert abs(u.mean() - 0.5) < 5 * (1 / np.sqrt(12 * n))
