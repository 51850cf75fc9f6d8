"""CPU pin of the host-side planning of the batched Algorithm 1's segmented
products (seg_tn_plan / seg_tn_bind in csrc/batch.cu, called through the built
library with no GPU): for every problem's C_p = A_p^T B_p the split-K chunks
partition [0, K) in order, each at most the chunk length, each reading its own
rows of A_p and B_p with the right strides; every chunk's partial tile has its
own disjoint slot of the partial buffer; the reduction of each problem sums
exactly its chunks into C_p.  Also the tensor-core operand layout rules."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_2111_11728_gb300 as fg

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2111_11728_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include <cstdint>
#include <cstdio>
#include <vector>
#include "kernels.h"
using namespace feti;
static const double* at(int64_t base, int64_t off) {
  return reinterpret_cast<const double*>(static_cast<uintptr_t>(base + 8 * off));
}
int main() {
  int n;
  long long kchunk;
  if (scanf("%d %lld", &n, &kchunk) != 2) return 1;
  const int64_t A0 = 1ll << 32, B0 = 1ll << 36, C0 = 1ll << 40, P0 = 1ll << 44;
  std::vector<SegTN> ops(n);
  for (int i = 0; i < n; ++i) {
    long long M, N, K, lda, ldb, ldc, tri, ao, bo, co;
    scanf("%lld %lld %lld %lld %lld %lld %lld %lld %lld %lld", &M, &N, &K, &lda, &ldb, &ldc, &tri, &ao, &bo, &co);
    ops[i] = SegTN{at(A0, ao), lda, at(B0, bo), ldb, const_cast<double*>(at(C0, co)), ldc, (int)M, (int)N, K, (int)tri};
  }
  std::vector<GemmDesc> descs;
  std::vector<int64_t> coff;
  std::vector<SegRed> reds;
  int64_t plen = 0;
  int mm = 0, mn = 0;
  seg_tn_plan(ops, kchunk, descs, coff, reds, &plen, &mm, &mn);
  seg_tn_bind(descs, coff, const_cast<double*>(at(P0, 0)));
  auto off = [](const void* p, int64_t base) { return (long long)((reinterpret_cast<uintptr_t>(p) - base) / 8); };
  printf("{\"plen\": %lld, \"max_m\": %d, \"max_n\": %d, \"descs\": [", (long long)plen, mm, mn);
  for (size_t i = 0; i < descs.size(); ++i) {
    const GemmDesc& d = descs[i];
    printf("%s[%lld, %lld, %lld, %d, %d, %d, %d, %lld, %lld, %lld, %lld, %lld, %lld]", i ? ", " : "",
           off(d.A, A0), off(d.B, B0), off(d.C, P0), d.M, d.N, d.K, d.tri, (long long)d.ars, (long long)d.acs,
           (long long)d.brs, (long long)d.bcs, (long long)d.crs, (long long)d.ccs);
  }
  printf("], \"reds\": [");
  for (size_t i = 0; i < reds.size(); ++i) {
    const SegRed& r = reds[i];
    printf("%s[%lld, %lld, %lld, %d, %d, %d, %d, %lld]", i ? ", " : "", off(r.C, C0), (long long)r.crs,
           (long long)r.ccs, r.M, r.N, r.nz, r.tri, (long long)r.poff);
  }
  printf("]}\n");
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers not available")
    if not os.path.exists(fg.LIB_PATH):
        from paper_2111_11728_gb300 import build
        build.build()
    d = tmp_path_factory.mktemp("plan")
    src = d / "main.cpp"
    src.write_text(HARNESS)
    exe = d / "plan"
    libdir = os.path.dirname(fg.LIB_PATH)
    libname = os.path.basename(fg.LIB_PATH)[3:-3]
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-L", libdir, "-l" + libname,
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True, capture_output=True)
    return exe


def test_segmented_plan(harness):
    rng = np.random.default_rng(11)
    kchunk = 1000
    ops = []
    ao = bo = co = 0
    for _ in range(12):
        M, N = int(rng.integers(1, 300)), int(rng.integers(1, 300))
        K = int(rng.integers(1, 5000))
        lda, ldb, ldc = K + int(rng.integers(0, 50)), K + int(rng.integers(0, 50)), M + int(rng.integers(0, 5))
        ops.append((M, N, K, lda, ldb, ldc, int(rng.integers(0, 2)), ao, bo, co))
        ao += lda * M
        bo += ldb * N
        co += ldc * N
    ops.append((0, 5, 100, 100, 100, 1, 0, ao, bo, co))          # an empty product is skipped
    text = f"{len(ops)} {kchunk}\n" + "\n".join(" ".join(map(str, o)) for o in ops)
    out = json.loads(subprocess.run([str(harness)], input=text, capture_output=True, text=True, check=True).stdout)
    descs, reds = out["descs"], out["reds"]
    live = [o for o in ops if o[0] > 0 and o[1] > 0]
    assert len(reds) == len(live)
    assert out["max_m"] == max(o[0] for o in live) and out["max_n"] == max(o[1] for o in live)
    slots, di, poff = [], 0, 0
    for o, r in zip(live, reds):
        M, N, K, lda, ldb, ldc, tri, a0, b0, c0 = o
        cr, crs, ccs, rM, rN, nz, rtri, rpoff = r
        assert (cr, crs, ccs, rM, rN, rtri, rpoff) == (c0, 1, ldc, M, N, tri, poff)
        assert nz == max(1, -(-K // kchunk))
        k = 0
        for z in range(nz):
            dA, dB, dC, dM, dN, dK, dtri, ars, acs, brs, bcs, crs2, ccs2 = descs[di]
            assert (dM, dN, dtri, ars, acs, brs, bcs, crs2, ccs2) == (M, N, tri, lda, 1, 1, ldb, 1, M)
            assert dA == a0 + k and dB == b0 + k and 0 < dK <= kchunk
            assert dC == rpoff + z * M * N                          # chunk z's slot
            slots.append((dC, dC + M * N))
            k += dK
            di += 1
        assert k == K                                               # the chunks partition [0, K)
        poff += nz * M * N
    assert di == len(descs) and out["plen"] == poff
    slots.sort()
    assert all(a1 <= b0 for (_, a1), (b0, _) in zip(slots, slots[1:]))   # disjoint partial slots


LAYOUT = r'''
#include <cstdio>
#include "kernels.h"
int main() {
  for (int p = 1; p <= 4; ++p) printf("%d %d %zu\n", p, feti::tc_chunk(p), feti::tc_elem_bytes(p));
  for (int nb = 0; nb <= 300; nb += 7)
    for (int nc = 0; nc <= 64; nc += 3)
      for (int aug = 0; aug <= 1; ++aug)
        for (int kc : {32, 64}) printf("k %d %d %d %d %d\n", nb, nc, aug, kc, feti::tc_k_extent(nb, nc, aug, kc));
  return 0;
}
'''


def test_tensor_operand_layout_rules(harness, tmp_path):
    """The tensor-core operand layout (csrc/tc_apply.cu): K chunk of 32 TF32 or 64
    BF16 values (one 128-byte swizzle row), and a subdomain's K extent = n_b
    rounded up to the chunk plus, with the primal coupling, n_c rounded up to
    the chunk -- so every TMA x coordinate is a whole number of 128-byte rows."""
    gxx = shutil.which("g++")
    src = tmp_path / "layout.cpp"
    src.write_text(LAYOUT)
    exe = tmp_path / "layout"
    libdir = os.path.dirname(fg.LIB_PATH)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-L", libdir,
                    "-l" + os.path.basename(fg.LIB_PATH)[3:-3], "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True, capture_output=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    fmt = {int(a): (int(b), int(c)) for a, b, c in (ln.split() for ln in lines if not ln.startswith("k"))}
    assert fmt == {fg.FETI_TF32: (32, 4), fg.FETI_TF32X3: (32, 4), fg.FETI_BF16: (64, 2), fg.FETI_BF16X3: (64, 2)}
    for ln in lines:
        if not ln.startswith("k"):
            continue
        nb, nc, aug, kc, ext = map(int, ln.split()[1:])
        up = lambda x: -(-x // kc) * kc
        assert ext == up(nb) + (up(nc) if aug and nc > 0 else 0)
        assert ext % kc == 0
