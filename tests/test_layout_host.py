"""Host checks of the stored-linearisation layout of the CUDA library (no GPU):
a small C++ program compiled against the library's internal header.

For every quadrature order Q of the element kernels (2..5), over one block of
EB = 256 / Q^2 elements:

* the FP32 quad layout `lin32_word(w, k, t)` maps the (word, slice, thread)
  triples one-to-one onto the block's kLinWords Q^3 EB words;
* the four words of a quad are consecutive and every quad starts on a 16-byte
  boundary, in every block (so 128-bit loads are aligned);
* the tail words (64..69) keep the FP64 layout's offsets;
* the block size in words is a multiple of 4, so the lo plane of the
  double-float action (offset = total word count) is 16-byte aligned too.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2607_21150_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "pff_internal.h"
using namespace pff;
int main() {
  int bad = 0;
  for (int Q = 2; Q <= 5; ++Q) {
    const long long EB = elems_per_block(Q), q2eb = (long long)Q * Q * EB, q3eb = q2eb * Q;
    const long long words = (long long)kLinWords * q3eb;
    if (words % 4) { std::printf("Q=%d block words %lld not a multiple of 4\n", Q, words); ++bad; }
    std::vector<int> seen(words, 0);
    for (int w = 0; w < kLinWords; ++w)
      for (int k = 0; k < Q; ++k)
        for (long long t = 0; t < q2eb; ++t) {
          const long long o = lin32_word(w, k, (int)t, q3eb, q2eb);
          if (o < 0 || o >= words) { std::printf("Q=%d w=%d k=%d t=%lld out of range\n", Q, w, k, t); return 1; }
          ++seen[o];
          if (w < kLinQuadWords) {
            const long long q0 = lin32_word(w & ~3, k, (int)t, q3eb, q2eb);
            if (o != q0 + (w & 3)) { std::printf("Q=%d quad not consecutive\n", Q); ++bad; }
            // 16-byte start of the quad in block b: (b * words + q0) * 4 bytes
            for (long long b = 0; b < 3; ++b)
              if (((b * words + q0) * 4) % 16) { std::printf("Q=%d quad start unaligned\n", Q); ++bad; }
          } else if (o != (long long)w * q3eb + (long long)k * q2eb + t) {
            std::printf("Q=%d tail word %d moved\n", Q, w); ++bad;
          }
        }
    for (long long i = 0; i < words; ++i)
      if (seen[i] != 1) { std::printf("Q=%d word %lld hit %d times\n", Q, i, seen[i]); ++bad; break; }
  }
  std::printf(bad ? "FAIL\n" : "OK\n");
  return bad ? 1 : 0;
}
"""


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


def test_fp32_quad_layout(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "layout.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "layout"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]
