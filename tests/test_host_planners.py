"""Host-side logic of the tensor-core passes, compiled for the CPU (-m "not gpu").

The work decomposition of the Gram pass (which tile pairs each work item covers) and the
sub-stage pass's shared-memory plan are plain integer functions in the CUDA sources. These tests
lift them out of the sources as they are, compile them with the host compiler and check them
exhaustively: every pair of sample tiles (i, j >= i) is covered exactly once and no item is
empty; every plan fits the shared memory, TMEM and the ring each mode needs.
"""

import os
import shutil
import subprocess
import tempfile

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1911_03813_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs a host C++ compiler")


def _between(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


def _run(program):
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "t.cpp")
        exe = os.path.join(tmp, "t")
        with open(src, "w") as f:
            f.write(program)
        subprocess.run(["g++", "-std=c++17", "-O1", "-o", exe, src], check=True,
                       capture_output=True)
        return subprocess.run([exe], check=True, capture_output=True, text=True).stdout


def test_gram_items_cover_each_tile_pair_once():
    text = open(os.path.join(CSRC, "gram_tc.cu")).read()
    jb = _between(text, "constexpr int JB", ";")
    funcs = _between(text, "__host__ __device__ __forceinline__ long long row_start",
                     "__device__ __forceinline__ void kahan_add")
    program = """#include <cstdio>
#include <vector>
#define __host__
#define __device__
#define __forceinline__ inline
""" + jb + ";\n" + funcs + """
int main() {
  long long bad = 0;
  for (long long T = 1; T <= 400; ++T) {
    std::vector<int> cov(T * T, 0);
    const long long TB = (T + 1) / 2, items = total_items(T);
    for (long long k = 0; k < items; ++k) {
      long long c, m, b0, b1;
      item_of(k, T, c, m);
      brange(c, m, T, b0, b1);
      if (!(b0 < b1) || m < 0 || m >= TB || b0 < m || b1 > TB) { ++bad; continue; }
      // I tiles 2m and 2m + 1 (when it exists) against the tiles 2b, 2b + 1 of each J block
      const int nI = 2 * m + 1 < T ? 2 : 1;
      if (nI == 1 && k != items - 1) ++bad;  // the odd last I tile comes last
      for (long long b = b0; b < b1; ++b)
        for (int u = 0; u < nI; ++u)
          for (int h = 0; h < 2; ++h) {
            const long long i = 2 * m + u, j = 2 * b + h;
            if (j < T && j >= i) cov[i * T + j] += 1;
          }
    }
    for (long long i = 0; i < T; ++i)
      for (long long j = 0; j < T; ++j)
        if (cov[i * T + j] != (j >= i ? 1 : 0)) ++bad;
  }
  printf("%lld\\n", bad);
}
"""
    assert _run(program).strip() == "0"


def test_sub_stage_plans_fit_every_shape():
    text = open(os.path.join(CSRC, "fg_tc_sub.cu")).read()
    internal = open(os.path.join(CSRC, "stmf_internal.h")).read()
    smem = _between(internal, "constexpr size_t kMaxSmem", ";")
    consts = "\n".join(_between(text, "constexpr int " + name, ";") + ";"
                       for name in ("TM", "REG_BYTES", "SUB_BYTES", "MAX_SUB"))
    mode = _between(text, "enum SubMode", ";") + ";"
    fps = _between(text, "__host__ __device__ constexpr int feats_per_sub", "\n") + "\n"
    struct = _between(text, "struct SubExtra {", "};") + "};"
    tmem = _between(text, "__host__ __device__ constexpr int tmem_need", "\n}") + "\n}"
    rp = _between(text, "int rp_of(int r)", "\n") + "\n"
    plan = _between(text, "SubExtra plan_sub(int mode, int n, int r) {", "\ntemplate <int RP")
    program = """#include <cstdio>
#include <cstddef>
#define __host__
#define __device__
""" + smem + ";\n" + consts + "\n" + mode + "\n" + fps + struct + "\n" + tmem + "\n" + rp + \
        plan + """
int main() {
  int bad = 0;
  for (int m = 0; m < 3; ++m)
    for (int r = 1; r <= 16; ++r)
      for (int n = 1; n <= (m == kF32 ? 256 : 512); ++n) {
        const SubExtra ex = plan_sub(m, n, r);
        const int RP = rp_of(r), N1 = (3 * RP + 15) / 16 * 16, fs = feats_per_sub(m);
        const int RR = m == kE4M3 ? ex.raw : 0, NF = m == kE4M3 ? RR : ex.ring;
        const int layout = ex.ring * SUB_BYTES + RR * REG_BYTES + ex.wbufs * 2 * (2 * RP * 128) +
                           ex.nsub * (fs / 64) * N1 * 128;
        const int bars = (NF + 2 * ex.ring + RR + 12) * 8 + 8 + 4 * RP * 8;
        const bool ok = ex.nsub == (n + fs - 1) / fs && ex.ring >= ex.nsub &&
                        ex.smem_bytes <= (int)kMaxSmem && layout + 1023 + bars <= ex.smem_bytes &&
                        bars <= 1024 && ex.tmem_cols <= 512 && ex.wbufs >= 1 &&
                        (m != kE4M3 || ex.raw >= 2) &&
                        (m != kF32 || ex.ring >= ex.nsub + 1);  // the FP32 gathered-rows path
        if (!ok) ++bad;
      }
  printf("%d\\n", bad);
}
"""
    assert _run(program).strip() == "0"
