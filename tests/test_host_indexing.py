"""Host checks of device index arithmetic (no GPU): the bank swizzle of the cluster kernel's
shared-memory twiddle table, compiled from the device header as sequential host code."""
import shutil
import subprocess

import pytest

from paper_2007_06427_gb300 import build as B

NMAX = 1024

PROG = r"""
#include <cstdio>
#define KS_HOST_EMULATION 1
#include "ks_items.cuh"
int main() {
    for (int t = 0; t < ks::NMAX; ++t) std::printf("%d %d\n", ks::tw_swz<double>(t), ks::tw_swz<float>(t));
    return 0;
}
"""


@pytest.fixture(scope="module")
def positions(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("swz")
    src = d / "swz.cpp"
    src.write_text(PROG)
    exe = d / "swz"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", B.CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    vals = list(map(int, out))
    return {16: vals[0::2], 8: vals[1::2]}   # element size (bytes) -> position of entry t


@pytest.mark.parametrize("esize", [16, 8])
def test_swizzle_is_a_permutation(positions, esize):
    assert sorted(positions[esize]) == list(range(NMAX))


def _conflict_degree(addrs, esize):
    """Wavefront count of one 128-byte wavefront's lanes: the largest number of distinct
    addresses that share a 4-byte bank (equal addresses are broadcast)."""
    banks = {}
    for a in set(addrs):
        for w in range(esize // 4):
            banks.setdefault((a // 4 + w) % 32, set()).add(a)
    return max(len(v) for v in banks.values())


@pytest.mark.parametrize("esize", [16, 8])
def test_swizzle_spreads_the_radix4_twiddle_loads(positions, esize):
    """Every twiddle load of every radix-4 pass (t, 2t and 3t with t = jm NMAX / 4 span) of
    every length 8 .. 1024, lanes grouped into 128-byte wavefronts as the transforms issue them:
    the plain table puts up to 16 lanes in one bank group, the swizzled one at most 3."""
    pos = positions[esize]
    lanes = 128 // esize
    stats = {}
    for name, where in (("plain", list(range(NMAX))), ("swizzled", pos)):
        worst, total, count = 0, 0, 0
        for lg in range(3, 11):
            n = 1 << lg
            span = 2 if lg & 1 else 1
            while span * 4 <= n:
                if span > 1:
                    tu = NMAX // (span * 4)
                    for mult in (1, 2, 3):
                        for base in range(0, 32, lanes):
                            addrs = [where[mult * ((l % (n // 4)) & (span - 1)) * tu] * esize
                                     for l in range(base, base + lanes)]
                            w = _conflict_degree(addrs, esize)
                            worst, total, count = max(worst, w), total + w, count + 1
                span *= 4
        stats[name] = (worst, total / count)
    assert stats["plain"][0] >= 8
    assert stats["swizzled"][0] <= 3 and stats["swizzled"][1] < 1.5, stats


@pytest.mark.parametrize("esize", [16, 8])
@pytest.mark.parametrize("nm", [16, 64, 128, 256, 1024])
def test_compact_swizzled_table(positions, esize, nm):
    """The per-phase launches' compact table: entry t = i NMAX / nm at slot tw_swz(i), read with
    t >> log2(NMAX / nm).  The slots are a permutation of 0 .. nm-1, and the radix-4 passes of
    every length up to nm stay spread over the banks."""
    pos = positions[esize]
    sh = (NMAX // nm).bit_length() - 1
    slots = [pos[i] for i in range(nm)]
    assert sorted(slots) == list(range(nm))
    lanes = 128 // esize
    worst, total, count = 0, 0, 0
    for lg in range(3, nm.bit_length()):
        n = 1 << lg
        span = 2 if lg & 1 else 1
        while span * 4 <= n:
            if span > 1:
                tu = NMAX // (span * 4)
                for mult in (1, 2, 3):
                    for base in range(0, 32, lanes):
                        addrs = [pos[(mult * ((l % (n // 4)) & (span - 1)) * tu) >> sh] * esize
                                 for l in range(base, base + lanes)]
                        w = _conflict_degree(addrs, esize)
                        worst, total, count = max(worst, w), total + w, count + 1
            span *= 4
    if count:
        assert worst <= 3 and total / count < 1.6, (worst, total / count)
