"""The kernel's schedule walk divides by launch-invariant divisors with one
widening multiply (FastDiv in csrc/sk_args.h).  Check the host-side constants
and the device formula, compiled here as plain C++, against integer division
on edge and random dividends below 2^31."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_2301_03598_gb300", "csrc", "sk_args.h")

PROGRAM = r"""
#include <cstdint>
#include <cstdio>
#include <random>
#include "sk_args.h"
static uint32_t q_of(uint32_t n, sk::FastDiv f) { return uint32_t((uint64_t(n) * f.m) >> f.shift); }
int main() {
  std::mt19937_64 rng(2301);
  long bad = 0, checked = 0;
  const uint32_t ds[] = {1, 2, 3, 7, 16, 17, 36, 63, 64, 65, 76, 127, 128, 129, 151, 152, 255, 256,
                         4095, 4097, 65535, 65536, 1u << 20, (1u << 30) + 1, (1u << 31) - 1, 1u << 31};
  for (uint32_t d : ds) {
    const sk::FastDiv f = sk::make_fastdiv(d);
    for (uint32_t i = 0; i < 200000; ++i) {
      const uint32_t n = i < 2000 ? i : i < 4000 ? (1u << 31) - 1 - (i - 2000)
                                               : uint32_t(rng() & 0x7fffffffu);
      bad += q_of(n, f) != n / d;
      ++checked;
    }
  }
  for (int t = 0; t < 50000; ++t) {
    const uint32_t d = 1 + uint32_t(rng() % 0x7fffffffu);
    const sk::FastDiv f = sk::make_fastdiv(d);
    for (int i = 0; i < 8; ++i) {
      const uint32_t n = uint32_t(rng() & 0x7fffffffu);
      bad += q_of(n, f) != n / d;
      ++checked;
    }
  }
  std::printf("%ld %ld\n", checked, bad);
  return bad != 0;
}
"""


def test_fast_division_matches_integer_division(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "fastdiv.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv"
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), "-I", cuda_inc,
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split())
    assert out.returncode == 0 and bad == 0 and checked > 5_000_000
