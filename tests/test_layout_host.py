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


# The bulk copies of the persistent FP32-arithmetic level kernel (the issue
# logic of pff_elem_pipe.cuh restated on the byte offsets it computes, with
# the layout functions and the stage geometry of the library's own header):
# every copy starts and ends on 16-byte boundaries in global and shared
# memory, stays inside its slot and inside the allocation (FP32 planes plus
# their padding), a stage's byte count fits the mbarrier's transaction count,
# the consumer reads of the tail runs stay inside their widened copies, and
# two blocks fit on an SM where the dispatch uses the kernel.
PIPE_PROGRAM = r"""
#include <cstdarg>
#include <cstdio>
#include "pff_internal.h"
using namespace pff;
static int bad = 0;
static void CHECK(bool c, const char* fmt, ...) {
  if (c) return;
  va_list ap;
  va_start(ap, fmt);
  std::vprintf(fmt, ap);
  va_end(ap);
  std::printf("\n");
  ++bad;
}

template <int P, int Q, bool BF, bool KX> void check_smem(bool used) {
  CHECK(pipe_slot_bytes<Q, BF, KX>() % 16 == 0, "Q=%d slot bytes not a multiple of 16", Q);
  CHECK(pipe_smem_bytes<P, Q, BF, KX>() <= 227 * 1024, "P=%d Q=%d smem above the per-block limit", P, Q);
  if (used) CHECK(pipe_fits<P, Q, BF, KX>(), "P=%d Q=%d BF=%d KX=%d: two blocks do not fit", P, Q, BF, KX);
  CHECK(pipe_elem_stride<Q>() >= pipe_elem_words<Q>() && pipe_elem_stride<Q>() % 32 == (Q * Q) % 32,
        "Q=%d element stride", Q);
}

template <int Q> void check_copies() {
  const long long q2eb = pipe_q2eb<Q>(), q3eb = q2eb * Q;
  const long long nblk = 7;
  // FP32 words (byte addresses relative to a 256-byte aligned allocation)
  const long long lin_len = nblk * kLinWords * q3eb;
  const long long alloc = 4 * (lin_len + kLin32Pad);
  for (int kx = 0; kx < 2; ++kx) {
    const int NT = kx ? pipe_tails<false, true>() : pipe_tails<false, false>();
    const long long slot = kx ? pipe_slot_bytes<Q, false, true>() : pipe_slot_bytes<Q, false, false>();
    for (long long b = 0; b < nblk; ++b)
      for (int k = 0; k < Q; ++k) {
        const long long g = 4 * b * kLinWords * q3eb;
        long long tot0 = 0, tot1 = 0;
        for (int o = 0; o < 8; ++o) {
          const long long s0 = g + 4 * lin32_word(4 * o, k, 0, q3eb, q2eb);
          const long long s1 = g + 4 * lin32_word(32 + 4 * o, k, 0, q3eb, q2eb);
          CHECK(s0 % 16 == 0 && s1 % 16 == 0 && (16 * q2eb) % 16 == 0, "Q=%d FP32 quad run unaligned", Q);
          CHECK(s0 + 16 * q2eb <= 4 * lin_len && s1 + 16 * q2eb <= 4 * lin_len, "Q=%d FP32 quad run out of range", Q);
          CHECK((o + 1) * 16 * q2eb <= slot, "Q=%d FP32 quad run beyond its slot", Q);
          tot0 += 16 * q2eb;
          tot1 += 16 * q2eb;
        }
        for (int jt = 0; jt < NT; ++jt) {
          const long long ad = g + 4 * lin32_word(kLinQuadWords + jt, k, 0, q3eb, q2eb);
          const long long lo = ad & ~15LL;
          const long long nb = (ad - lo + 4 * q2eb + 15) & ~15LL;
          CHECK(nb <= pipe_tail_bytes<Q>(), "Q=%d tail copy larger than its region", Q);
          CHECK(lo >= 0 && lo + nb <= alloc, "Q=%d tail copy beyond the allocation", Q);
          CHECK(128 * q2eb + (jt + 1) * pipe_tail_bytes<Q>() <= slot, "Q=%d tail region beyond the slot", Q);
          // thread t reads 4 bytes at (ad - lo) + 4 t of the region
          CHECK((ad - lo) + 4 * (q2eb - 1) + 4 <= nb, "Q=%d tail read beyond the copy", Q);
          tot1 += nb;
        }
        CHECK(tot0 < (1 << 20) && tot1 < (1 << 20), "Q=%d stage above the transaction count", Q);
      }
  }
  // BF16 words
  const long long len16 = nblk * kLin16Words * q3eb;
  for (int kx = 0; kx < 2; ++kx) {
    const long long slot = kx ? pipe_slot_bytes<Q, true, true>() : pipe_slot_bytes<Q, true, false>();
    for (long long b = 0; b < nblk; ++b)
      for (int k = 0; k < Q; ++k) {
        const long long g = 2 * b * kLin16Words * q3eb;
        long long tot = 0;
        for (int o = 0; o < 8; ++o) {
          const long long s0 = g + o * 16 * q3eb + k * 16 * q2eb;
          CHECK(s0 == g + 2 * lin16_word(8 * o, k, 0, q3eb, q2eb), "Q=%d BF16 octet run differs from the layout", Q);
          CHECK(s0 % 16 == 0 && s0 + 16 * q2eb <= 2 * len16, "Q=%d BF16 octet run unaligned or out of range", Q);
          tot += 16 * q2eb;
        }
        for (int tp = 0; tp < 1 + kx; ++tp) {
          const long long s0 = g + (128 + 8 * tp) * q3eb + k * 8 * q2eb;
          CHECK(s0 == g + 2 * lin16_word(64 + 4 * tp, k, 0, q3eb, q2eb), "Q=%d BF16 tail run differs from the layout", Q);
          CHECK(s0 % 16 == 0 && (8 * q2eb) % 16 == 0 && s0 + 8 * q2eb <= 2 * len16, "Q=%d BF16 tail run", Q);
          CHECK((128 + 8 * (tp + 1)) * q2eb <= slot, "Q=%d BF16 tail beyond the slot", Q);
          tot += 8 * q2eb;
        }
        CHECK(tot == (kx ? 144 : 136) * q2eb && tot < (1 << 20), "Q=%d BF16 stage bytes", Q);
      }
  }
}

int main() {
  check_copies<2>(); check_copies<3>(); check_copies<4>(); check_copies<5>();
  // the dispatch: BF16 words always, FP32 words on the box always, FP32 on
  // mapped meshes where two slots fit
  check_smem<2, 2, true, false>(true); check_smem<2, 2, true, true>(true); check_smem<2, 2, false, false>(true);
  check_smem<3, 3, true, false>(true); check_smem<3, 3, true, true>(true); check_smem<3, 3, false, false>(true);
  check_smem<2, 3, true, false>(true); check_smem<2, 3, false, false>(true);
  check_smem<4, 4, true, false>(true); check_smem<4, 4, true, true>(true); check_smem<4, 4, false, false>(true);
  check_smem<2, 4, true, false>(true); check_smem<3, 4, false, false>(true);
  check_smem<5, 5, true, false>(true); check_smem<5, 5, true, true>(true); check_smem<5, 5, false, false>(true);
  check_smem<4, 5, true, true>(true); check_smem<3, 5, false, false>(true); check_smem<2, 5, true, false>(true);
  check_smem<5, 5, false, true>(false);
  std::printf(bad ? "FAIL\n" : "OK\n");
  return bad ? 1 : 0;
}
"""


def test_level_pipe_bulk_copies(tmp_path):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "pipe.cpp"
    src.write_text(PIPE_PROGRAM)
    exe = tmp_path / "pipe"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]
