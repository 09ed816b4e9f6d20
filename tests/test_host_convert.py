"""The library's exact binary32 -> binary64 conversion (``ml_convert.cuh``),
which the folds and products run on the integer pipe, checked on the host
against the C++ conversion for every one of the 2^32 binary32 inputs (the
header compiles for host and device from the same source)."""

import os
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1309_3859_b300", "csrc")

DRIVER = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include "ml_convert.cuh"
#include <cstdio>
#include <cstring>
int main() {
  unsigned long long bad = 0, seen = 0;
  uint32_t u = 0;
  do {
    float f;
    memcpy(&f, &u, 4);
    const double a = ml::exact_double(f), b = static_cast<double>(f);
    uint64_t x, y;
    memcpy(&x, &a, 8);
    memcpy(&y, &b, 8);
    const bool both_nan = a != a && b != b;
    if (x != y && !both_nan) {
      if (bad < 4) printf("mismatch %08x\n", u);
      ++bad;
    }
    ++seen;
  } while (++u != 0);
  printf("checked %llu mismatches %llu\n", seen, bad);
  return bad != 0;
}
"""


def test_exact_double_matches_cpp_conversion_for_every_float(tmp_path):
    src = tmp_path / "conv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "conv"
    subprocess.run(["g++", "-O2", "-I", CSRC, "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "checked 4294967296 mismatches 0" in out.stdout
