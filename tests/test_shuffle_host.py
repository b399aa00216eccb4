"""Host build of the surrogate's training shuffle (no GPU): the per-epoch map of
gl_shuffle.cuh is a bijection of [0, n) for sizes around powers of four and
ragged ones, it differs between epochs and seeds, and SplitMix64 reproduces the
published reference outputs of that generator (seed 1234567, five outputs)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r'''
#include <cstdio>
#include <vector>
#include "gl_shuffle.cuh"
int main() {
  long bad = 0;
  const long sizes[] = {1, 2, 3, 4, 5, 15, 16, 17, 63, 64, 65, 1000, 1023, 1024, 1025, 4095, 4096,
                        4097, 65535, 65536, 65537, 300000};
  for (long n : sizes) {
    for (int seed = 0; seed < 3; ++seed) {
      for (int epoch = 0; epoch < 3; ++epoch) {
        gl::Shuffle s = gl::make_shuffle(seed * 7919ull + 1, epoch, n);
        std::vector<char> seen(n, 0);
        long moved = 0;
        for (long j = 0; j < n; ++j) {
          long i = gl::shuffle_index(s, j, n);
          if (i < 0 || i >= n || seen[i]) { ++bad; continue; }
          seen[i] = 1;
          moved += i != j;
        }
        if (n >= 64 && moved < n / 2) ++bad;   // a real shuffle moves most indices
      }
    }
    if (n >= 64) {   // different epochs give different orders
      gl::Shuffle a = gl::make_shuffle(1, 0, n), b = gl::make_shuffle(1, 1, n);
      long same = 0;
      for (long j = 0; j < n; ++j) same += gl::shuffle_index(a, j, n) == gl::shuffle_index(b, j, n);
      if (same > n / 8) ++bad;
    }
  }
  // SplitMix64 from state 1234567: each output is splitmix64(state + k * golden),
  // golden = 0x9e3779b97f4a7c15 (the published reference sequence)
  const unsigned long long ref[5] = {6457827717110365317ull, 3203168211198807973ull,
                                     9817491932198370423ull, 4593380528125082431ull,
                                     16408922859458223821ull};
  unsigned long long st = 1234567ull;
  for (int k = 0; k < 5; ++k) {
    if (gl::splitmix64(st) != ref[k]) ++bad;
    st += 0x9e3779b97f4a7c15ull;
  }
  printf("%ld\n", bad);
}
'''


def test_epoch_permutation_is_a_bijection():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "s.cpp"), os.path.join(d, "s")
        with open(src, "w") as fh:
            fh.write(SRC)
        inc = os.path.join(ROOT, "paper_2410_05408_b300", "csrc")
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", inc, src, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    assert int(out) == 0
