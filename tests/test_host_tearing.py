"""CPU pin of the library's host-side tearing (csrc/setup.cpp, compiled here as
plain C++ with no GPU): for TFETI and FETI-DP (corners, and corners plus edge
averages) in 2D and 3D, the multiplier rows it emits -- as (subdomain, local
DOF, sign) pairs -- are exactly the oracle's pair-wise rows of Eqs. (4) / (10),
its primal count is the oracle's, and its b space is the set of local DOFs the
oracle's B touches."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads
from oracle.fetidp import FETIDP
from oracle.tfeti import TFETI

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2111_11728_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "feti_internal.h"
using namespace feti;
int main(int argc, char** argv) {
  FILE* fi = fopen(argv[1], "rb");
  int n_prob = 0;
  fread(&n_prob, sizeof(int), 1, fi);
  std::vector<HostProblem> parts(n_prob);
  for (int q = 0; q < n_prob; ++q) {
    int hdr[10];
    fread(hdr, sizeof(int), 10, fi);          // dim, tiles[3], elems[3], method, edges, n_el
    double par[4];
    fread(par, sizeof(double), 4, fi);
    const int dim = hdr[0], n_el = hdr[9];
    long n_nodes = 1;
    for (int a = 0; a < dim; ++a) n_nodes *= (long)hdr[1 + a] * hdr[4 + a] + 1;
    std::vector<double> rho(n_el), f(n_nodes * dim);
    std::vector<unsigned char> dir(n_nodes * dim);
    fread(rho.data(), sizeof(double), n_el, fi);
    fread(dir.data(), 1, dir.size(), fi);
    fread(f.data(), sizeof(double), f.size(), fi);
    feti_problem p{};
    p.dim = dim;
    for (int a = 0; a < 3; ++a) { p.tiles[a] = hdr[1 + a]; p.elems[a] = hdr[4 + a]; }
    p.E0 = par[0]; p.Emin = par[1]; p.nu = par[2]; p.p = par[3];
    p.rho = rho.data(); p.dirichlet = dir.data(); p.f = f.data(); p.on_device = 0;
    std::string msg = build_host_problem(p, hdr[7], 1, rho.data(), parts[q], hdr[8]);
    if (!msg.empty()) { printf("{\"error\": \"%s\"}\n", msg.c_str()); return 1; }
  }
  fclose(fi);
  HostProblem hp;
  if (n_prob == 1) {
    hp = parts[0];
  } else {
    std::string msg = merge_host_problems(parts, hp);
    if (!msg.empty()) { printf("{\"error\": \"%s\"}\n", msg.c_str()); return 1; }
  }
  FILE* fo = fopen(argv[2], "w");
  fprintf(fo, "{\"n_lam\": %lld, \"n_primal\": %d, \"rows\": [", (long long)hp.n_lam, hp.n_primal);
  auto loc = [&](int b, int& s, int& ld) {
    s = hp.b_sub[b];
    const StructType& T = hp.types[hp.sub_type[s]];
    ld = T.blist[b - hp.b_off[s]];
  };
  for (long long l = 0; l < hp.n_lam; ++l) {
    int s0, d0;
    loc(hp.lam_b0[l], s0, d0);
    fprintf(fo, "%s[[%d, %d, %d]", l ? ", " : "", s0, d0, (int)hp.lam_s0[l]);
    if (hp.lam_b1[l] >= 0) {
      int s1, d1;
      loc(hp.lam_b1[l], s1, d1);
      fprintf(fo, ", [%d, %d, %d]", s1, d1, (int)hp.lam_s1[l]);
    }
    fprintf(fo, "]");
  }
  fprintf(fo, "], \"bsets\": [");
  for (int s = 0; s < hp.n_sub; ++s) {
    const StructType& T = hp.types[hp.sub_type[s]];
    fprintf(fo, "%s[", s ? ", " : "");
    for (int k = 0; k < T.n_b; ++k) fprintf(fo, "%s%d", k ? ", " : "", T.blist[k]);
    fprintf(fo, "]");
  }
  fprintf(fo, "], \"avgs\": [");
  for (int s = 0; s < hp.n_sub; ++s) {
    const StructType& T = hp.types[hp.sub_type[s]];
    fprintf(fo, "%s[", s ? ", " : "");
    for (size_t a = 0; a < T.avg_c.size(); ++a) {
      fprintf(fo, "%s[%d", a ? ", " : "", T.clist[T.avg_c[a]]);
      for (int k = T.avg_off[a]; k < T.avg_off[a + 1]; ++k) fprintf(fo, ", %d", T.blist[T.avg_b[k]]);
      fprintf(fo, "]");
    }
    fprintf(fo, "]");
  }
  fprintf(fo, "], \"lam_b\": [");
  for (long long l = 0; l < hp.n_lam; ++l)
    fprintf(fo, "%s[%d, %d, %d, %d]", l ? ", " : "", hp.lam_b0[l], (int)hp.lam_s0[l], hp.lam_b1[l], (int)hp.lam_s1[l]);
  // the precision form's spread tables, positions = the DOF index
  std::vector<int64_t> pos(hp.n_b_total);
  for (long long b = 0; b < hp.n_b_total; ++b) pos[b] = b;
  SpreadTables sp;
  const int max_rows = argc > 3 ? atoi(argv[3]) : 128;
  const std::string smsg = build_spread_tables(hp, pos, max_rows, sp);
  fprintf(fo, "], \"n_b_total\": %lld, \"spread_error\": \"%s\", \"spread\": {", (long long)hp.n_b_total, smsg.c_str());
  auto dump = [&](const char* name, const auto& v, bool last) {
    fprintf(fo, "\"%s\": [", name);
    for (size_t i = 0; i < v.size(); ++i) fprintf(fo, "%s%d", i ? ", " : "", (int)v[i]);
    fprintf(fo, "]%s", last ? "" : ", ");
  };
  dump("row0", sp.row0, false);
  dump("slot_off", sp.slot_off, false);
  dump("slot_pos", sp.slot_pos, false);
  dump("slot_b", sp.slot_b, false);
  dump("ent_off", sp.ent_off, false);
  dump("ent", sp.ent, true);
  fprintf(fo, "}}\n");
  fclose(fo);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers not available")
    d = tmp_path_factory.mktemp("tearing")
    src = d / "main.cpp"
    src.write_text(HARNESS)
    exe = d / "tear"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src),
                    os.path.join(CSRC, "setup.cpp"), "-o", str(exe)], check=True, capture_output=True)
    return exe, d


def _run(harness, probs, method, edges, max_rows=128):
    exe, d = harness
    inp, out = d / "in.bin", d / "out.json"
    with open(inp, "wb") as f:
        f.write(np.array([len(probs)], np.int32).tobytes())
        for p in probs:
            tiles = list(p.tiles) + [1] * (3 - p.dim)
            elems = list(p.elems) + [1] * (3 - p.dim)
            mode = 2 if edges == "adaptive" else int(bool(edges))
            hdr = np.array([p.dim, *tiles, *elems, 1 if method == "fetidp" else 0, mode, p.n_elements],
                           np.int32)
            f.write(hdr.tobytes())
            f.write(np.array([p.E0, p.Emin, p.nu, p.p], np.float64).tobytes())
            f.write(np.ascontiguousarray(p.rho, np.float64).tobytes())
            f.write(np.ascontiguousarray(p.dirichlet, np.uint8).tobytes())
            f.write(np.ascontiguousarray(p.f, np.float64).tobytes())
    subprocess.run([str(exe), str(inp), str(out), str(max_rows)], check=True, capture_output=True)
    return json.loads(out.read_text())


def _oracle_rows(p, method, edges, s0=0):
    """Pair-wise rows as (subdomain + s0, local DOF, sign), the interface sets and the primal count."""
    if method == "tfeti":
        op = TFETI(p, "k")
        rows = [[(s + s0, k, g) for (s, k, g) in ent] for ent in op.cons.entries]
        bsets = [sorted({k for ent in op.cons.entries for (s2, k, _) in ent if s2 == s}) for s in range(op.n_sub)]
        return rows, bsets, None, op.n_lam
    op = FETIDP(p, "k", primal="adaptive" if edges == "adaptive" else ("edges" if edges else "corners"))
    rows = [[(s + s0, int(op.r_loc[s][k]), g) for (s, k, g) in ent] for ent in op.cons.entries]
    bsets = [sorted(int(op.r_loc[s][k]) for k in op.bset[s]) for s in range(op.n_sub)]
    return rows, bsets, op.n_c, op.n_lam


def _canon(rows):
    out = []
    for r in rows:
        ents = sorted((int(s), int(k), int(np.sign(g))) for s, k, g in r)
        if ents[0][2] < 0:                       # fix the overall sign of a row
            ents = sorted((s, k, -g) for s, k, g in ents)
        out.append(tuple(ents))
    return sorted(out)


CASES = [
    ("tfeti", False, lambda: workloads.config1()),
    ("fetidp", False, lambda: workloads.config2(tiles=3, elems=4)),
    ("fetidp", True, lambda: workloads.layered_grid(elems=4, layers=4)),
    ("fetidp", False, lambda: workloads.config4(tiles=2, elems=2)),
    ("fetidp", True, lambda: workloads.config4(tiles=2, elems=3)),
    ("tfeti", False, lambda: workloads.config4(tiles=2, elems=2)),
    ("fetidp", "adaptive", lambda: workloads.layered_grid(elems=4, layers=4)),
    ("fetidp", "adaptive", lambda: workloads.config4(tiles=2, elems=3)),
]


@pytest.mark.parametrize("method,edges,make", CASES)
def test_library_tearing_matches_oracle(harness, method, edges, make):
    p = make()
    got = _run(harness, [p], method, edges)
    rows, bsets, n_c, n_lam = _oracle_rows(p, method, edges)
    if n_c is not None:
        assert got["n_primal"] == n_c
    assert got["n_lam"] == n_lam
    assert _canon(got["rows"]) == _canon(rows)
    assert [sorted(b) for b in got["bsets"]] == bsets


@pytest.mark.parametrize("mode", [True, "adaptive"])
@pytest.mark.parametrize("make", [lambda: workloads.config4(tiles=2, elems=3), lambda: workloads.config4(tiles=3, elems=2),
                                  lambda: workloads.layered_grid(elems=4, layers=4)])
def test_edge_average_tables_match_oracle(harness, make, mode):
    """The change-of-basis tables of every subdomain (the average's slot, then
    the slots of the edge's other nodes, as local DOFs) are the oracle's edges,
    for every shared edge and for the adaptive selection."""
    p = make()
    got = _run(harness, [p], "fetidp", mode)
    op = FETIDP(p, "k", primal="adaptive" if mode == "adaptive" else "edges")
    mesh = op.mesh
    for s in range(op.n_sub):
        g2 = list(mesh.local_to_global_nodes(s))
        want = sorted([g2.index(gn) * p.dim + d for gn in nodes] for nodes, d in op.edges if nodes[0] in g2)
        assert sorted(got["avgs"][s]) == want, s


@pytest.mark.parametrize("edges", [False, True])
def test_batch_merge_keeps_each_problems_tearing(harness, edges):
    """A batch of uneven problems merged into one description: the rows are
    each problem's own rows, its subdomains shifted by the preceding problems'."""
    probs = workloads.config3(n_problems=3, tile_range=(2, 3), elem_range=(3, 5), seed=7)
    got = _run(harness, probs, "fetidp", edges)
    rows, bsets, n_c, n_lam, s0 = [], [], 0, 0, 0
    for p in probs:
        r, b, c, n = _oracle_rows(p, "fetidp", edges, s0)
        rows += r
        bsets += b
        n_c += c
        n_lam += n
        s0 += p.n_subdomains
    assert got["n_primal"] == n_c and got["n_lam"] == n_lam
    assert _canon(got["rows"]) == _canon(rows)
    assert [sorted(b) for b in got["bsets"]] == bsets


@pytest.mark.parametrize("max_rows", [128, 30])
@pytest.mark.parametrize("method,edges,make", [CASES[1], CASES[3], CASES[4], CASES[5],
                                               ("fetidp", False, lambda: workloads.config4(tiles=3, elems=2))])
def test_spread_tables_reproduce_the_signed_rows(harness, method, edges, make, max_rows):
    """The precision form's multiplier-side operand tables: ranges of at most
    max_rows consecutive rows covering every row once; every interface DOF with
    rows is one slot, inside the range that holds all of its rows; the slots'
    signed entries are exactly the rows' entries (B, entry by entry); within a
    range the single-row slots come first, each class in position order."""
    p = make()
    got = _run(harness, [p], method, edges, max_rows)
    assert got["spread_error"] == ""
    sp = got["spread"]
    row0, soff, spos, sb, eoff, ent = (np.array(sp[k]) for k in ("row0", "slot_off", "slot_pos", "slot_b",
                                                                   "ent_off", "ent"))
    n_lam = got["n_lam"]
    assert row0[0] == 0 and row0[-1] == n_lam
    assert np.all(np.diff(row0) >= 1) and np.all(np.diff(row0) <= max_rows)
    # B from the rows: (row, DOF) -> sign
    want = {}
    for l, (b0, s0, b1, s1) in enumerate(got["lam_b"]):
        want[(l, b0)] = s0
        if b1 >= 0:
            want[(l, b1)] = s1
    have = {}
    for r in range(len(row0) - 1):
        slots = range(soff[r], soff[r + 1])
        multi = [eoff[q + 1] - eoff[q] > 1 for q in slots]
        assert multi == sorted(multi)                        # single-row slots first
        for cls in (False, True):
            ps = [spos[q] for q, m in zip(slots, multi) if m == cls]
            assert ps == sorted(ps)
        for q in slots:
            assert spos[q] == sb[q]                          # positions given as the DOF index
            for t in range(eoff[q], eoff[q + 1]):
                e = int(ent[t])
                rel, sign = (e, 1) if e >= 0 else (~e, -1)
                assert 0 <= rel < row0[r + 1] - row0[r]
                key = (int(row0[r] + rel), int(sb[q]))
                assert key not in have
                have[key] = sign
    assert have == want
    assert len(set(sb.tolist())) == len(sb)                  # one slot per DOF


def test_spread_tables_refuse_a_dof_wider_than_a_range(harness):
    """A DOF shared by eight subdomains (TFETI, 3D) has its copies' rows spread
    over its 28 pair-wise rows: ranges shorter than that cannot hold them."""
    got = _run(harness, [workloads.config4(tiles=2, elems=2)], "tfeti", False, 9)
    assert "rows apart" in got["spread_error"]
