// Host-side tearing of a regular tile mesh into subdomains and construction of
// every index map the device kernels use.
//
// * TFETI (Section 2.1, Eqs. 4-5): every subdomain keeps all of its DOFs; a
//   fixed DOF gets one single-entry row per subdomain copy (the Dirichlet part
//   of B u = c); a free DOF shared by several subdomains gets one row
//   u^a - u^b = 0 per pair of copies (pair-wise, redundant at cross points,
//   Section 3.1).
// * FETI-DP (Section 2.2, Eqs. 8-10): fixed DOFs are eliminated, the DOFs at
//   the vertices of the tile grid are primal (corner nodes of a regular
//   partition), and the remaining shared DOFs get pair-wise rows of B_r.
//
// Subdomains whose local DOF classification is identical share a "type";
// subdomains of one type whose element densities are also identical share a
// "module" (one factorization, Section 1: repeated modules are reused).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>

#include "feti_internal.h"

namespace feti {

namespace {

struct NodeOwners {
  int n = 0;
  int sub[8];
  int lnode[8];
  int mask[8];   // per owner: bitmask of the relative offsets of the *other* owners
};

inline int sub_index(const HostProblem& hp, const int t[3]) {
  return t[0] + hp.tiles[0] * (t[1] + hp.tiles[1] * t[2]);
}

inline int64_t gnode_index(const HostProblem& hp, const int g[3]) {
  return g[0] + (int64_t)hp.nnod[0] * (g[1] + (int64_t)hp.nnod[1] * g[2]);
}

inline int lnode_index(const HostProblem& hp, const int c[3]) {
  return c[0] + hp.lnod[0] * (c[1] + hp.lnod[1] * c[2]);
}

// All subdomains whose closed tile contains global node g, sorted by index.
void owners_of(const HostProblem& hp, const int g[3], NodeOwners& o) {
  int cand[3][2], nc[3];
  for (int a = 0; a < 3; ++a) {
    nc[a] = 0;
    if (a >= hp.dim) { cand[a][0] = 0; nc[a] = 1; continue; }
    int e = hp.elems[a];
    int t = g[a] / e;
    int r = g[a] % e;
    if (r == 0) {
      if (t > 0) cand[a][nc[a]++] = t - 1;
      if (t < hp.tiles[a]) cand[a][nc[a]++] = t;
    } else {
      cand[a][nc[a]++] = t;
    }
  }
  o.n = 0;
  int tt[3];
  for (int i = 0; i < nc[0]; ++i)
    for (int j = 0; j < nc[1]; ++j)
      for (int k = 0; k < nc[2]; ++k) {
        tt[0] = cand[0][i]; tt[1] = cand[1][j]; tt[2] = cand[2][k];
        int c[3] = {0, 0, 0};
        for (int a = 0; a < hp.dim; ++a) c[a] = g[a] - tt[a] * hp.elems[a];
        o.sub[o.n] = sub_index(hp, tt);
        o.lnode[o.n] = lnode_index(hp, c);
        o.n++;
      }
  // sort by subdomain (insertion sort, n <= 8)
  for (int a = 1; a < o.n; ++a)
    for (int b = a; b > 0 && o.sub[b] < o.sub[b - 1]; --b) {
      std::swap(o.sub[b], o.sub[b - 1]);
      std::swap(o.lnode[b], o.lnode[b - 1]);
    }
  // relative-offset masks
  for (int a = 0; a < o.n; ++a) {
    int ta[3] = {o.sub[a] % hp.tiles[0], (o.sub[a] / hp.tiles[0]) % hp.tiles[1],
                 o.sub[a] / (hp.tiles[0] * hp.tiles[1])};
    int m = 0;
    for (int b = 0; b < o.n; ++b) {
      if (b == a) continue;
      int tb[3] = {o.sub[b] % hp.tiles[0], (o.sub[b] / hp.tiles[0]) % hp.tiles[1],
                   o.sub[b] / (hp.tiles[0] * hp.tiles[1])};
      int code = (tb[0] - ta[0] + 1) + 3 * (tb[1] - ta[1] + 1) + 9 * (tb[2] - ta[2] + 1);
      m |= 1 << code;
    }
    o.mask[a] = m;
  }
}

}  // namespace

std::string build_host_problem(const feti_problem& prob, int method, int dedup,
                               const double* rho_host, HostProblem& hp, int edge_mode, double jump_ratio) {
  hp = HostProblem();
  if (prob.dim != 2 && prob.dim != 3) return "dim must be 2 or 3";
  hp.dim = prob.dim;
  hp.method = method;
  for (int a = 0; a < 3; ++a) {
    int t = a < hp.dim ? prob.tiles[a] : 1;
    int e = a < hp.dim ? prob.elems[a] : 1;
    if (t < 1 || e < 1) return "tiles and elems must be >= 1";
    hp.tiles[a] = t;
    hp.elems[a] = a < hp.dim ? e : 0;
    hp.nel[a] = a < hp.dim ? t * e : 1;
    hp.nnod[a] = a < hp.dim ? t * e + 1 : 1;
    hp.lnod[a] = a < hp.dim ? e + 1 : 1;
  }
  if (hp.dim == 2) { hp.elems[2] = 0; }
  hp.n_nodes = (int64_t)hp.nnod[0] * hp.nnod[1] * hp.nnod[2];
  hp.n_elements = (int64_t)hp.nel[0] * hp.nel[1] * hp.nel[2];
  hp.n_dofs = hp.n_nodes * hp.dim;
  hp.n_sub = hp.tiles[0] * hp.tiles[1] * hp.tiles[2];
  hp.n_loc_nodes = hp.lnod[0] * hp.lnod[1] * hp.lnod[2];
  hp.n_loc_dofs = hp.n_loc_nodes * hp.dim;
  hp.n_loc_elems = 1;
  for (int a = 0; a < hp.dim; ++a) hp.n_loc_elems *= hp.elems[a];
  hp.E0 = prob.E0; hp.Emin = prob.Emin; hp.nu = prob.nu; hp.p = prob.p;
  if (!(hp.nu > -1.0 && hp.nu < 0.5)) return "nu must lie in (-1, 0.5)";
  if (hp.n_sub < 2) return "at least two subdomains are required";
  hp.dirichlet.assign(prob.dirichlet, prob.dirichlet + hp.n_dofs);
  hp.n_rbm = method == FETI_TFETI ? (hp.dim == 2 ? 3 : 6) : 0;

  const int dim = hp.dim;
  const int nld = hp.n_loc_dofs;
  const bool edges = edge_mode != 0 && method == FETI_FETIDP;
  const bool adaptive = edges && edge_mode == 2;

  // Edge averages: a node with exactly dim - 1 coordinates on tile-grid planes
  // lies inside a tile-grid edge along the remaining axis `run`; the edge gets
  // an average in component d when it is shared (>= 2 owners) and all its
  // interior nodes are free in d.  The average takes the slot of the edge's
  // first interior node (global coordinate t * e + 1 along run).
  auto edge_axis = [&](const int g[3]) -> int {
    int run = -1, on = 0;
    for (int a = 0; a < dim; ++a) {
      if (g[a] % hp.elems[a] == 0) ++on;
      else run = a;
    }
    return on == dim - 1 ? run : -1;
  };
  // Adaptive selection: the stiffness jump across the edge through node g --
  // over its interior nodes, the largest ratio between the sharers' diagonal
  // stiffness entries of the node.  On these square / cubic elements the
  // element stiffness has one diagonal value, so a sharer's entry is that value
  // times the sum of the SIMP moduli of its elements around the node.
  auto modulus = [&](int64_t e) {
    return hp.Emin + std::pow(rho_host[e], hp.p) * (hp.E0 - hp.Emin);
  };
  auto edge_jump = [&](const int g[3], int run) -> double {
    int h[3] = {g[0], g[1], g[2]};
    const int base = g[run] - g[run] % hp.elems[run];
    double jump = 1.0;
    NodeOwners on;
    for (int k = 1; k < hp.elems[run]; ++k) {
      h[run] = base + k;
      owners_of(hp, h, on);
      double lo = 0.0, hi = 0.0;
      for (int q = 0; q < on.n; ++q) {
        const int s = on.sub[q];
        const int ts[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
        double sum = 0.0;
        for (int dz = (dim == 3 ? -1 : 0); dz <= 0; ++dz)
          for (int dy = -1; dy <= 0; ++dy)
            for (int dx = -1; dx <= 0; ++dx) {
              const int e3[3] = {h[0] + dx, h[1] + dy, dim == 3 ? h[2] + dz : 0};
              bool inside = true;
              for (int a = 0; a < dim; ++a)
                if (e3[a] < ts[a] * hp.elems[a] || e3[a] >= (ts[a] + 1) * hp.elems[a]) inside = false;
              if (inside) sum += modulus(e3[0] + (int64_t)hp.nel[0] * (e3[1] + (int64_t)hp.nel[1] * e3[2]));
            }
        if (q == 0 || sum < lo) lo = sum;
        if (q == 0 || sum > hi) hi = sum;
      }
      if (lo > 0.0) jump = std::max(jump, hi / lo);
      else if (hi > 0.0) jump = HUGE_VAL;
    }
    return jump;
  };
  auto edge_free = [&](const int g[3], int run, int d) -> bool {
    int h[3] = {g[0], g[1], g[2]};
    const int base = g[run] - g[run] % hp.elems[run];
    for (int k = 1; k < hp.elems[run]; ++k) {
      h[run] = base + k;
      if (hp.dirichlet[gnode_index(hp, h) * dim + d]) return false;
    }
    return true;
  };

  // ---- classify local DOFs of every subdomain, group into types ----------------
  std::map<std::vector<int>, int> type_of_key;
  hp.sub_type.assign(hp.n_sub, -1);
  std::vector<std::vector<int>> type_masks;   // per type: neighbour mask per local DOF
  NodeOwners own;
  for (int s = 0; s < hp.n_sub; ++s) {
    int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
    std::vector<int> key(2 * nld);
    for (int ln = 0; ln < hp.n_loc_nodes; ++ln) {
      int c[3];
      local_node_coords(hp, ln, c);
      int g[3] = {0, 0, 0};
      bool vertex = true;
      for (int a = 0; a < dim; ++a) {
        g[a] = t[a] * hp.elems[a] + c[a];
        if (c[a] != 0 && c[a] != hp.elems[a]) vertex = false;
      }
      owners_of(hp, g, own);
      int me = 0;
      for (int q = 0; q < own.n; ++q) if (own.sub[q] == s) me = q;
      int64_t gn = gnode_index(hp, g);
      for (int d = 0; d < dim; ++d) {
        int ld = ln * dim + d;
        bool fixed = hp.dirichlet[gn * dim + d] != 0;
        int cls;
        if (method == FETI_FETIDP) {
          int run = edges && !vertex && own.n > 1 ? edge_axis(g) : -1;
          bool avg = run >= 0 && g[run] % hp.elems[run] == 1 && edge_free(g, run, d) &&
                     (!adaptive || edge_jump(g, run) >= jump_ratio);
          if (fixed) cls = CLS_X;
          else if (vertex || avg) cls = CLS_C;
          else if (own.n > 1) cls = CLS_B;
          else cls = CLS_I;
        } else {
          cls = (fixed || own.n > 1) ? CLS_B : CLS_I;
        }
        key[2 * ld] = cls;
        key[2 * ld + 1] = own.mask[me];
      }
    }
    auto it = type_of_key.find(key);
    if (it == type_of_key.end()) {
      int id = (int)hp.types.size();
      type_of_key.emplace(key, id);
      StructType T;
      T.n_loc = nld;
      for (int a = 0; a < 3; ++a) {
        T.e[a] = a < dim ? hp.elems[a] : 1;
        T.ln[a] = hp.lnod[a];
      }
      T.cls.resize(nld);
      T.idx.assign(nld, -1);
      std::vector<int> masks(nld);
      for (int ld = 0; ld < nld; ++ld) { T.cls[ld] = key[2 * ld]; masks[ld] = key[2 * ld + 1]; }
      // i and c lists: lexicographic; b list: grouped by neighbour set, then lexicographic
      std::vector<std::pair<int64_t, int>> bkeys;
      for (int ld = 0; ld < nld; ++ld) {
        if (T.cls[ld] == CLS_I) T.ilist.push_back(ld);
        else if (T.cls[ld] == CLS_C) T.clist.push_back(ld);
        else if (T.cls[ld] == CLS_B) bkeys.push_back({((int64_t)masks[ld] << 32) | ld, ld});
      }
      std::sort(bkeys.begin(), bkeys.end());
      for (auto& kv : bkeys) T.blist.push_back(kv.second);
      T.n_i = (int)T.ilist.size();
      T.n_b = (int)T.blist.size();
      T.n_c = (int)T.clist.size();
      for (int k = 0; k < T.n_i; ++k) T.idx[T.ilist[k]] = k;
      for (int k = 0; k < T.n_b; ++k) T.idx[T.blist[k]] = k;
      for (int k = 0; k < T.n_c; ++k) T.idx[T.clist[k]] = k;
      // edge averages: c slots that are not at a tile vertex
      T.avg_off.push_back(0);
      for (int k = 0; k < T.n_c; ++k) {
        const int ld = T.clist[k], ln = ld / dim, d = ld % dim;
        int c[3];
        local_node_coords(hp, ln, c);
        int run = -1, on = 0;
        for (int a = 0; a < dim; ++a) {
          if (c[a] == 0 || c[a] == hp.elems[a]) ++on;
          else run = a;
        }
        if (on == dim) continue;                          // a corner
        if (on != dim - 1 || c[run] != 1) return "internal error: primal DOF off the tile edges";
        T.avg_c.push_back(k);
        for (int j = 2; j < hp.elems[run]; ++j) {
          int cc[3] = {c[0], c[1], c[2]};
          cc[run] = j;
          const int l2 = lnode_index(hp, cc) * dim + d;
          if (T.cls[l2] != CLS_B) return "internal error: edge node is not an interface DOF";
          T.avg_b.push_back(T.idx[l2]);
        }
        T.avg_off.push_back((int)T.avg_b.size());
      }
      // half-bandwidth of K_ii in i-order (element-neighbour coupling)
      int bw = 0;
      for (int k = 0; k < T.n_i; ++k) {
        int ld = T.ilist[k];
        int ln = ld / dim;
        int c[3];
        local_node_coords(hp, ln, c);
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int cc[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
              bool ok = true;
              for (int a = 0; a < dim; ++a) if (cc[a] < 0 || cc[a] > hp.elems[a]) ok = false;
              if (!ok) continue;
              int m = lnode_index(hp, cc);
              for (int d2 = 0; d2 < dim; ++d2) {
                int l2 = m * dim + d2;
                if (T.cls[l2] != CLS_I) continue;
                bw = std::max(bw, std::abs(T.idx[l2] - k));
              }
            }
      }
      T.bw = bw;
      hp.types.push_back(std::move(T));
      type_masks.push_back(std::move(masks));
      hp.sub_type[s] = id;
    } else {
      hp.sub_type[s] = it->second;
    }
  }

  // ---- modules (identical type + identical densities share one factorization) --
  hp.sub_module.assign(hp.n_sub, -1);
  std::unordered_map<std::string, int> mod_of_key;
  std::vector<double> tile_rho(hp.n_loc_elems);
  for (int s = 0; s < hp.n_sub; ++s) {
    int id;
    if (dedup && rho_host) {
      int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
      int k = 0;
      int ez = dim == 3 ? hp.elems[2] : 1;
      for (int z = 0; z < ez; ++z)
        for (int y = 0; y < hp.elems[1]; ++y)
          for (int x = 0; x < hp.elems[0]; ++x) {
            int64_t gx = t[0] * hp.elems[0] + x, gy = t[1] * hp.elems[1] + y,
                    gz = dim == 3 ? t[2] * hp.elems[2] + z : 0;
            tile_rho[k++] = rho_host[gx + hp.nel[0] * (gy + (int64_t)hp.nel[1] * gz)];
          }
      std::string key((const char*)tile_rho.data(), tile_rho.size() * sizeof(double));
      key.append((const char*)&hp.sub_type[s], sizeof(int));
      auto it = mod_of_key.find(key);
      if (it == mod_of_key.end()) {
        id = (int)hp.module_rep.size();
        mod_of_key.emplace(std::move(key), id);
        hp.module_rep.push_back(s);
        hp.module_type.push_back(hp.sub_type[s]);
      } else {
        id = it->second;
      }
    } else {
      id = (int)hp.module_rep.size();
      hp.module_rep.push_back(s);
      hp.module_type.push_back(hp.sub_type[s]);
    }
    hp.sub_module[s] = id;
  }

  // ---- b space --------------------------------------------------------------
  hp.b_off.assign(hp.n_sub + 1, 0);
  for (int s = 0; s < hp.n_sub; ++s) hp.b_off[s + 1] = hp.b_off[s] + hp.types[hp.sub_type[s]].n_b;
  hp.n_b_total = hp.b_off[hp.n_sub];
  hp.b_sub.resize(hp.n_b_total);
  for (int s = 0; s < hp.n_sub; ++s)
    for (int64_t b = hp.b_off[s]; b < hp.b_off[s + 1]; ++b) hp.b_sub[b] = s;

  auto global_b = [&](int q, int lnode, int d) -> int64_t {
    const StructType& T = hp.types[hp.sub_type[q]];
    int ld = lnode * dim + d;
    if (T.cls[ld] != CLS_B) return -1;
    return hp.b_off[q] + T.idx[ld];
  };

  // ---- multipliers ------------------------------------------------------------
  hp.group_off.push_back(0);
  for (int s = 0; s < hp.n_sub; ++s) {
    const StructType& T = hp.types[hp.sub_type[s]];
    int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
    for (int k = 0; k < T.n_b; ++k) {
      int ld = T.blist[k];
      int ln = ld / dim, d = ld % dim;
      int c[3];
      local_node_coords(hp, ln, c);
      int g[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) g[a] = t[a] * hp.elems[a] + c[a];
      owners_of(hp, g, own);
      int64_t gn = gnode_index(hp, g);
      bool fixed = hp.dirichlet[gn * dim + d] != 0;
      int64_t my_b = hp.b_off[s] + k;
      if (method == FETI_TFETI && fixed) {
        int grp = (int)hp.group_off.size() - 1;
        hp.group_b.push_back((int)my_b);
        hp.group_off.push_back((int)hp.group_b.size());
        hp.lam_b0.push_back((int)my_b); hp.lam_s0.push_back(1);
        hp.lam_b1.push_back(-1); hp.lam_s1.push_back(0);
        hp.lam_group.push_back(grp);
        continue;
      }
      if (own.sub[0] != s || own.n < 2) continue;   // rows are emitted by the lowest owner
      int grp = (int)hp.group_off.size() - 1;
      int64_t gb[8];
      for (int q = 0; q < own.n; ++q) {
        gb[q] = global_b(own.sub[q], own.lnode[q], d);
        if (gb[q] < 0) return "internal error: shared DOF is not an interface DOF in every copy";
        hp.group_b.push_back((int)gb[q]);
      }
      hp.group_off.push_back((int)hp.group_b.size());
      for (int a = 0; a < own.n; ++a)
        for (int b = a + 1; b < own.n; ++b) {
          hp.lam_b0.push_back((int)gb[a]); hp.lam_s0.push_back(1);
          hp.lam_b1.push_back((int)gb[b]); hp.lam_s1.push_back(-1);
          hp.lam_group.push_back(grp);
        }
    }
  }
  hp.n_lam = (int64_t)hp.lam_b0.size();
  if (hp.n_lam == 0) return "the problem has no interface multipliers";
  // b -> lambda CSR
  std::vector<int> cnt(hp.n_b_total + 1, 0);
  for (int64_t l = 0; l < hp.n_lam; ++l) {
    cnt[hp.lam_b0[l] + 1]++;
    if (hp.lam_b1[l] >= 0) cnt[hp.lam_b1[l] + 1]++;
  }
  hp.b2l_off.assign(hp.n_b_total + 1, 0);
  for (int64_t b = 0; b < hp.n_b_total; ++b) hp.b2l_off[b + 1] = hp.b2l_off[b] + cnt[b + 1];
  hp.b2l_lam.resize(hp.b2l_off[hp.n_b_total]);
  hp.b2l_sign.resize(hp.b2l_off[hp.n_b_total]);
  std::vector<int> fill(hp.b2l_off.begin(), hp.b2l_off.end() - 1);
  for (int64_t l = 0; l < hp.n_lam; ++l) {
    int b0 = hp.lam_b0[l];
    hp.b2l_lam[fill[b0]] = (int)l; hp.b2l_sign[fill[b0]] = hp.lam_s0[l]; fill[b0]++;
    int b1 = hp.lam_b1[l];
    if (b1 >= 0) { hp.b2l_lam[fill[b1]] = (int)l; hp.b2l_sign[fill[b1]] = hp.lam_s1[l]; fill[b1]++; }
  }

  // ---- primal corners (FETI-DP) ------------------------------------------------
  hp.c_off.assign(hp.n_sub + 1, 0);
  if (method == FETI_FETIDP) {
    std::unordered_map<int64_t, int> prim;
    // enumerate tile-grid vertices lexicographically
    int nv[3] = {hp.tiles[0] + 1, hp.tiles[1] + 1, dim == 3 ? hp.tiles[2] + 1 : 1};
    for (int vz = 0; vz < nv[2]; ++vz)
      for (int vy = 0; vy < nv[1]; ++vy)
        for (int vx = 0; vx < nv[0]; ++vx) {
          int g[3] = {vx * hp.elems[0], vy * hp.elems[1], dim == 3 ? vz * hp.elems[2] : 0};
          int64_t gn = gnode_index(hp, g);
          for (int d = 0; d < dim; ++d)
            if (!hp.dirichlet[gn * dim + d]) prim.emplace(gn * dim + d, hp.n_primal++);
        }
    for (int s = 0; s < hp.n_sub; ++s) hp.c_off[s + 1] = hp.c_off[s] + hp.types[hp.sub_type[s]].n_c;
    hp.c_glob.resize(hp.c_off[hp.n_sub]);
    std::vector<std::vector<int>> src;
    for (int s = 0; s < hp.n_sub; ++s) {
      const StructType& T = hp.types[hp.sub_type[s]];
      int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
      for (int k = 0; k < T.n_c; ++k) {
        int ld = T.clist[k];
        int c[3];
        local_node_coords(hp, ld / dim, c);
        int g[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) g[a] = t[a] * hp.elems[a] + c[a];
        int64_t gd = gnode_index(hp, g) * dim + ld % dim;
        auto pit = prim.find(gd);
        if (pit == prim.end()) pit = prim.emplace(gd, hp.n_primal++).first;   // an edge average
        int pidx = pit->second;
        hp.c_glob[hp.c_off[s] + k] = pidx;
        if ((int)src.size() < hp.n_primal) src.resize(hp.n_primal);
        src[pidx].push_back((int)(hp.c_off[s] + k));
      }
    }
    src.resize(hp.n_primal);
    hp.prim_off.assign(hp.n_primal + 1, 0);
    for (int q = 0; q < hp.n_primal; ++q) {
      hp.prim_off[q + 1] = hp.prim_off[q] + (int)src[q].size();
      for (int v : src[q]) hp.prim_src.push_back(v);
    }
  }

  // ---- loads (lowest owner takes a shared node's load) and output gather ---------
  hp.load_src.assign((int64_t)hp.n_sub * nld, -1);
  std::vector<int64_t> copies_cnt(hp.n_dofs + 1, 0);
  for (int s = 0; s < hp.n_sub; ++s) {
    const StructType& T = hp.types[hp.sub_type[s]];
    int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
    for (int ln = 0; ln < hp.n_loc_nodes; ++ln) {
      int c[3];
      local_node_coords(hp, ln, c);
      int g[3] = {0, 0, 0};
      bool lowest = true;
      for (int a = 0; a < dim; ++a) {
        g[a] = t[a] * hp.elems[a] + c[a];
        if (c[a] == 0 && t[a] > 0) lowest = false;     // a lower-index tile also owns it
      }
      int64_t gn = gnode_index(hp, g);
      for (int d = 0; d < dim; ++d) {
        int ld = ln * dim + d;
        copies_cnt[gn * dim + d + 1]++;
        if (lowest && T.cls[ld] != CLS_X) hp.load_src[(int64_t)s * nld + ld] = gn * dim + d;
      }
    }
  }
  hp.dof_copy_off.assign(hp.n_dofs + 1, 0);
  for (int64_t q = 0; q < hp.n_dofs; ++q) hp.dof_copy_off[q + 1] = hp.dof_copy_off[q] + copies_cnt[q + 1];
  hp.dof_copy.resize(hp.dof_copy_off[hp.n_dofs]);
  std::vector<int64_t> pos(hp.dof_copy_off.begin(), hp.dof_copy_off.end() - 1);
  for (int s = 0; s < hp.n_sub; ++s) {
    int t[3] = {s % hp.tiles[0], (s / hp.tiles[0]) % hp.tiles[1], s / (hp.tiles[0] * hp.tiles[1])};
    for (int ln = 0; ln < hp.n_loc_nodes; ++ln) {
      int c[3];
      local_node_coords(hp, ln, c);
      int g[3] = {0, 0, 0};
      for (int a = 0; a < dim; ++a) g[a] = t[a] * hp.elems[a] + c[a];
      int64_t gn = gnode_index(hp, g);
      for (int d = 0; d < dim; ++d) hp.dof_copy[pos[gn * dim + d]++] = (int64_t)s * nld + ln * dim + d;
    }
  }
  // ---- single-problem placement tables ----------------------------------------
  hp.loc_off.resize(hp.n_sub + 1);
  for (int s2 = 0; s2 <= hp.n_sub; ++s2) hp.loc_off[s2] = (int64_t)s2 * nld;
  hp.n_loc_total = (int64_t)hp.n_sub * nld;
  hp.sub_prob.assign(hp.n_sub, 0);
  hp.n_prob = 1;
  hp.prob_dof_off = {0, hp.n_dofs};
  hp.prob_el_off = {0, hp.n_elements};
  hp.prob_lam_off = {0, hp.n_lam};
  hp.prob_sub_off = {0, hp.n_sub};
  hp.prob_primal_off = {0, hp.n_primal};
  hp.prob_nel = {hp.nel[0], hp.nel[1], hp.nel[2]};
  return "";
}

std::string merge_host_problems(std::vector<HostProblem>& parts, HostProblem& out) {
  out = HostProblem();
  if (parts.empty()) return "empty batch";
  const HostProblem& f = parts[0];
  out.dim = f.dim;
  out.method = f.method;
  out.E0 = f.E0; out.Emin = f.Emin; out.nu = f.nu; out.p = f.p;
  out.n_rbm = f.n_rbm;
  out.n_prob = (int)parts.size();
  out.prob_dof_off.push_back(0);
  out.prob_el_off.push_back(0);
  out.prob_lam_off.push_back(0);
  out.prob_sub_off.push_back(0);
  out.prob_primal_off.push_back(0);
  out.loc_off.push_back(0);
  out.b_off.push_back(0);
  out.c_off.push_back(0);
  out.group_off.push_back(0);
  out.prim_off.push_back(0);
  out.dof_copy_off.push_back(0);
  for (int q = 0; q < out.n_prob; ++q) {
    HostProblem& P = parts[q];
    if (P.dim != out.dim || P.method != out.method) return "batch problems differ in dim or method";
    if (P.E0 != out.E0 || P.Emin != out.Emin || P.nu != out.nu || P.p != out.p)
      return "batch problems must share E0, Emin, nu and p";
    const int t0 = (int)out.types.size(), m0 = (int)out.module_rep.size(), s0 = out.n_sub;
    const int64_t dof0 = out.n_dofs, el0 = out.n_elements, lam0 = out.n_lam, b0 = out.n_b_total;
    const int pr0 = out.n_primal;
    const int64_t c0 = out.c_off.back(), l0 = out.n_loc_total;
    const int grp0 = (int)out.group_off.size() - 1;
    const int64_t src0 = (int64_t)out.prim_src.size();
    for (auto& T : P.types) out.types.push_back(T);
    for (int s = 0; s < P.n_sub; ++s) {
      out.sub_type.push_back(P.sub_type[s] + t0);
      out.sub_module.push_back(P.sub_module[s] + m0);
      out.sub_prob.push_back(q);
      out.b_off.push_back(b0 + P.b_off[s + 1]);
      out.c_off.push_back(c0 + P.c_off[s + 1]);
      out.loc_off.push_back(l0 + P.loc_off[s + 1]);
    }
    for (size_t m = 0; m < P.module_rep.size(); ++m) {
      out.module_rep.push_back(P.module_rep[m] + s0);
      out.module_type.push_back(P.module_type[m] + t0);
    }
    for (int64_t b = 0; b < P.n_b_total; ++b) out.b_sub.push_back(P.b_sub[b] + s0);
    for (int64_t l = 0; l < P.n_lam; ++l) {
      out.lam_b0.push_back(P.lam_b0[l] + (int)b0);
      out.lam_b1.push_back(P.lam_b1[l] >= 0 ? P.lam_b1[l] + (int)b0 : -1);
      out.lam_s0.push_back(P.lam_s0[l]);
      out.lam_s1.push_back(P.lam_s1[l]);
      out.lam_group.push_back(P.lam_group[l] + grp0);
    }
    {
      const int gb0 = (int)out.group_b.size();
      for (size_t g = 1; g < P.group_off.size(); ++g) out.group_off.push_back(P.group_off[g] + gb0);
      for (int v : P.group_b) out.group_b.push_back(v + (int)b0);
    }
    for (int v : P.c_glob) out.c_glob.push_back(v + pr0);
    for (size_t g = 1; g < P.prim_off.size(); ++g) out.prim_off.push_back(P.prim_off[g] + (int)src0);
    for (int v : P.prim_src) out.prim_src.push_back(v + (int)c0);
    for (int64_t v : P.load_src) out.load_src.push_back(v >= 0 ? v + dof0 : -1);
    const int64_t dc0 = (int64_t)out.dof_copy.size();
    for (size_t g = 1; g < P.dof_copy_off.size(); ++g) out.dof_copy_off.push_back(P.dof_copy_off[g] + dc0);
    for (int64_t v : P.dof_copy) out.dof_copy.push_back(v + l0);
    for (unsigned char v : P.dirichlet) out.dirichlet.push_back(v);
    out.n_sub += P.n_sub;
    out.n_dofs += P.n_dofs;
    out.n_nodes += P.n_nodes;
    out.n_elements += P.n_elements;
    out.n_lam += P.n_lam;
    out.n_b_total += P.n_b_total;
    out.n_primal += P.n_primal;
    out.n_loc_total += P.n_loc_total;
    out.prob_dof_off.push_back(out.n_dofs);
    out.prob_el_off.push_back(out.n_elements);
    out.prob_lam_off.push_back(out.n_lam);
    out.prob_sub_off.push_back(out.n_sub);
    out.prob_primal_off.push_back(out.n_primal);
    for (int a = 0; a < 3; ++a) out.prob_nel.push_back(P.nel[a]);
  }
  // b -> lambda CSR of the merged multipliers
  std::vector<int> cnt(out.n_b_total + 1, 0);
  for (int64_t l = 0; l < out.n_lam; ++l) {
    cnt[out.lam_b0[l] + 1]++;
    if (out.lam_b1[l] >= 0) cnt[out.lam_b1[l] + 1]++;
  }
  out.b2l_off.assign(out.n_b_total + 1, 0);
  for (int64_t b = 0; b < out.n_b_total; ++b) out.b2l_off[b + 1] = out.b2l_off[b] + cnt[b + 1];
  out.b2l_lam.resize(out.b2l_off[out.n_b_total]);
  out.b2l_sign.resize(out.b2l_off[out.n_b_total]);
  std::vector<int> fill(out.b2l_off.begin(), out.b2l_off.end() - 1);
  for (int64_t l = 0; l < out.n_lam; ++l) {
    const int a = out.lam_b0[l];
    out.b2l_lam[fill[a]] = (int)l; out.b2l_sign[fill[a]] = out.lam_s0[l]; fill[a]++;
    const int b = out.lam_b1[l];
    if (b >= 0) { out.b2l_lam[fill[b]] = (int)l; out.b2l_sign[fill[b]] = out.lam_s1[l]; fill[b]++; }
  }
  // the single-mesh fields describe the first problem (used only where a batch is not accepted)
  for (int a = 0; a < 3; ++a) {
    out.tiles[a] = f.tiles[a]; out.elems[a] = f.elems[a]; out.nel[a] = f.nel[a];
    out.nnod[a] = f.nnod[a]; out.lnod[a] = f.lnod[a];
  }
  out.n_loc_nodes = f.n_loc_nodes;
  out.n_loc_dofs = f.n_loc_dofs;
  out.n_loc_elems = f.n_loc_elems;
  return "";
}

}  // namespace feti

namespace feti {

std::string build_spread_tables(const HostProblem& hp, const std::vector<int64_t>& pos_of_b, int max_rows,
                                SpreadTables& out) {
  const int64_t nl = hp.n_lam, nbt = hp.n_b_total;
  if (max_rows < 1 || max_rows > 32767) return "range length out of range";
  out = SpreadTables{};
  // cut_bad[l] > 0: some DOF has rows on both sides of the cut before row l
  std::vector<int> cut_bad(nl + 2, 0);
  std::vector<int> first(std::max<int64_t>(nbt, 1), -1);
  for (int64_t b = 0; b < nbt; ++b) {
    const int q0 = hp.b2l_off[b], q1 = hp.b2l_off[b + 1];
    if (q1 == q0) continue;
    int lo = hp.b2l_lam[q0], hi = lo;
    for (int q = q0; q < q1; ++q) { lo = std::min(lo, hp.b2l_lam[q]); hi = std::max(hi, hp.b2l_lam[q]); }
    first[b] = lo;
    if (hi > lo) {
      cut_bad[lo + 1]++;
      cut_bad[hi + 1]--;
    }
  }
  for (int64_t l = 1; l <= nl; ++l) cut_bad[l] += cut_bad[l - 1];
  out.row0.push_back(0);
  for (int64_t l0 = 0; l0 < nl;) {
    int64_t l1 = std::min<int64_t>(l0 + max_rows, nl);
    while (l1 > l0 && l1 < nl && cut_bad[l1] > 0) --l1;
    if (l1 == l0) return "an interface DOF has multiplier rows more than " + std::to_string(max_rows) + " rows apart";
    out.row0.push_back((int)l1);
    l0 = l1;
  }
  const int nr = (int)out.row0.size() - 1;
  std::vector<int> range_of(std::max<int64_t>(nl, 1), 0);
  for (int r = 0; r < nr; ++r)
    for (int l = out.row0[r]; l < out.row0[r + 1]; ++l) range_of[l] = r;
  // key: (several rows?, position)
  std::vector<std::vector<std::pair<std::pair<int, int64_t>, int>>> by_range(nr);
  for (int64_t b = 0; b < nbt; ++b) {
    if (first[b] < 0) continue;
    const int multi = hp.b2l_off[b + 1] - hp.b2l_off[b] > 1 ? 1 : 0;
    by_range[range_of[first[b]]].push_back({{multi, pos_of_b[b]}, (int)b});
  }
  out.slot_off.push_back(0);
  out.ent_off.push_back(0);
  for (int r = 0; r < nr; ++r) {
    std::sort(by_range[r].begin(), by_range[r].end());
    for (const auto& kb : by_range[r]) {
      const int b = kb.second;
      if (kb.first.second > (int64_t)0x7fffffff) return "operand position beyond 32 bits";
      out.slot_pos.push_back((int)kb.first.second);
      out.slot_b.push_back(b);
      for (int q = hp.b2l_off[b]; q < hp.b2l_off[b + 1]; ++q) {
        const int rel = hp.b2l_lam[q] - out.row0[r];
        out.ent.push_back((short)(hp.b2l_sign[q] > 0 ? rel : ~rel));
      }
      out.ent_off.push_back((int)out.ent.size());
    }
    out.slot_off.push_back((int)out.slot_pos.size());
  }
  return "";
}

}  // namespace feti
