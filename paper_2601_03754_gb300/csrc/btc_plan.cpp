// Host planner: the level schedule of the multi-stage permutation P_inf
// (Sec. 4.3) for Alg. 5 (factorization) and Alg. 7 (solve). Integer work only.
//
// Levels l = 1 .. floor(log2 N) + 1 with stride s = 2^(l-1); at level l the
// eliminated nodes are the odd multiples of s that are <= N (1-based labels,
// as in the paper), and the surviving nodes are the multiples of s.
#include <algorithm>
#include <cmath>

#include "btc_internal.h"

namespace btc {

static const int kSizes[] = {8, 16, 32, 48, 64, 96, 128, 256};

// Smallest compiled block size >= n. FP64 stops at 96: three 128 x 128 FP64
// blocks do not fit in one SM's shared memory. 256 (the blocked node of tile
// tasks) exists for the tensor-core dtypes (3: TF32, 4: BF16) only.
int padded_size(int n, int dtype) {
  for (int s : kSizes) {
    if (dtype == 0 && s > 96) break;
    if (s > 128 && dtype != 3 && dtype != 4) break;
    if (n <= s) return s;
  }
  return 0;
}

int64_t count_offdiag(int N) {
  int64_t t = 0;
  for (int64_t s = 1; s <= N; s *= 2) t += N / s - 1;
  return t;
}

void build_host_plan(int N, int n, int np, int64_t d_base, int64_t e_base, int64_t y_base, int inst,
                     HostPlan *P) {
  P->N = N;
  P->n = n;
  P->np = np;
  const int64_t bs = (int64_t)np * np;
  int levels = 0;
  for (int64_t s = 1; s <= N; s *= 2) ++levels;
  P->levels = levels;
  // U slots: level-major, K_l = floor(N/s) - 1 per level; one more (empty) level
  // index is reserved so that fill targets of the last level are addressable.
  P->level_slot_off.assign(levels + 2, 0);
  for (int l = 1; l <= levels + 1; ++l) {
    int64_t s = int64_t(1) << (l - 1);
    int64_t K = s <= N ? N / s - 1 : 0;
    P->level_slot_off[l] = P->level_slot_off[l - 1] + (K > 0 ? K : 0);
  }
  P->offdiag = P->level_slot_off[levels];
  P->fill = P->offdiag - (N - 1);
  P->slot_e.assign(P->offdiag, -1);
  P->slot_o.assign(P->offdiag, -1);

  // 1-based node v -> pool offsets
  auto dOff = [&](int64_t v) { return (d_base + v - 1) * bs; };
  auto eSlot = [&](int l, int64_t k) { return P->level_slot_off[l - 1] + (k - 1); };  // k 1-based
  auto eOff = [&](int l, int64_t k) { return (e_base + eSlot(l, k)) * bs; };
  auto yNode = [&](int64_t v) { return y_base + v - 1; };

  P->lv.assign(levels, LevelSchedule());
  const double n3 = (double)n * n * n, n2 = (double)n * n;
  double fl = 0, crit = 0, sol = 0;
  for (int l = 1; l <= levels; ++l) {
    const int64_t s = int64_t(1) << (l - 1);
    const int64_t h = s / 2;
    LevelSchedule &L = P->lv[l - 1];
    L.s = (int)s;
    double level_max = 0;
    for (int64_t e = s; e <= N; e += 2 * s) {
      FactorItem it;
      it.d_self = dOff(e);
      it.d_next = (e + s <= N) ? dOff(e + s) : -1;
      it.r_down = (e + s <= N) ? eOff(l, e / s) : -1;
      it.r_up = (e > s) ? eOff(l, e / s - 1) : -1;
      it.p_a = (l > 1 && e + h <= N) ? eOff(l - 1, 2 * e / s) : -1;
      it.p_b = (l > 1 && e + s + h <= N) ? eOff(l - 1, 2 * e / s + 2) : -1;
      it.fill = (e > s && e + s <= N) ? eOff(l + 1, (e - s) / (2 * s)) : -1;
      it.d_prev = (e > s) ? dOff(e - s) : -1;
      it.flags = 0;
      if (it.fill >= 0 && (((e - s) / (2 * s)) & 1)) it.flags |= FI_FILL_UPFIRST;
      if (l == levels) it.flags |= FI_ROOT;
      it.node = (int32_t)(e - 1);
      it.inst = inst;
      it.pad = 0;
      L.fac.push_back(it);
      if (it.r_down >= 0) {
        P->slot_e[eSlot(l, e / s)] = (int)(e - 1);
        P->slot_o[eSlot(l, e / s)] = (int)(e + s - 1);
      }
      if (it.r_up >= 0) {
        P->slot_e[eSlot(l, e / s - 1)] = (int)(e - 1);
        P->slot_o[eSlot(l, e / s - 1)] = (int)(e - s - 1);
      }
      // Table 1 costs: potrf n^3/3, trsm n^3, syrk n^3, gemm 2 n^3 (square blocks)
      double c = n3 / 3.0;
      if (it.p_a >= 0) c += n3;
      if (it.p_b >= 0) c += n3;
      if (it.r_down >= 0) c += 2 * n3;  // trsm + immediate syrk onto Dhat_{e+s}
      if (it.r_up >= 0) c += n3;        // trsm
      if (it.fill >= 0) c += 2 * n3;    // gemm
      fl += c;
      if (c > level_max) level_max = c;
      BwdItem b;
      b.x_self = yNode(e);
      b.d_self = dOff(e);
      b.x_dn = (e + s <= N) ? yNode(e + s) : -1;
      b.e_dn = it.r_down;
      b.x_up = (e > s) ? yNode(e - s) : -1;
      b.e_up = it.r_up;
      L.bwd.push_back(b);
    }
    crit += level_max;
    for (int64_t j = s; j <= N; j += s) {
      FwdItem f;
      f.y_self = yNode(j);
      f.y_l = f.e_l = f.y_r = f.e_r = -1;
      if (l > 1) {
        f.y_l = yNode(j - h);
        f.e_l = eOff(l - 1, (j - h) / h);
        if (j + h <= N) {
          f.y_r = yNode(j + h);
          f.e_r = eOff(l - 1, j / h);
        }
      }
      f.d_self = ((j / s) & 1) ? dOff(j) : -1;
      if (f.y_l < 0 && f.y_r < 0 && f.d_self < 0) continue;  // a level-1 survivor: nothing to do
      L.fwd.push_back(f);
    }
  }
  // ---- dataflow dependencies (indices into the flat level-ordered lists)
  // Factor item (e, l), h = s/2, reads Dhat_e and the fill S(e-s, e) written at level
  // l-1 by node e-h; P_a, S(e, e+s) and Dhat_{e+s} written by node e+h; P_b written by
  // node e+3h. Every one of these nodes is eliminated at level l-1.
  {
    std::vector<int32_t> fac_index(N + 1, -1);  // node (1-based) -> flat factor index
    int32_t idx = 0;
    for (int l = 1; l <= levels; ++l)
      for (const FactorItem &it : P->lv[l - 1].fac) fac_index[it.node + 1] = idx++;
    P->fac_deps.assign(3 * (size_t)idx, -1);
    P->fac_deps_rl.assign(3 * (size_t)idx, -1);
    idx = 0;
    for (int l = 1; l <= levels; ++l) {
      const int64_t s = int64_t(1) << (l - 1), h = s / 2;
      for (const FactorItem &it : P->lv[l - 1].fac) {
        const int64_t e = it.node + 1;
        if (l > 1) {
          const int64_t cand[3] = {e - h, e + h, e + 3 * h};
          for (int k = 0; k < 3; ++k)
            if (cand[k] >= 1 && cand[k] <= N) P->fac_deps[3 * (size_t)idx + k] = fac_index[cand[k]];
          // of e+3h only the deferred block P_b is read, which it stores with its factor blocks (its
          // next-diagonal update and fill go to nodes other than e)
          if (P->fac_deps[3 * (size_t)idx + 2] >= 0)
            P->fac_deps[3 * (size_t)idx + 2] = core_dep(P->fac_deps[3 * (size_t)idx + 2]);
          // Alg. 6: Dhat_e receives its last (atomic) updates at level l-1 from e-h and e+h,
          // which also write the two fill blocks e reads; nothing is deferred.
          for (int k = 0; k < 2; ++k)
            if (cand[k] >= 1 && cand[k] <= N) P->fac_deps_rl[3 * (size_t)idx + k] = fac_index[cand[k]];
        }
        ++idx;
      }
    }
    // Solve: forward items (j, l) for every survivor j at every level, then backward
    // items (e, l) from the top level down. Forward (j, l) waits for (j-h, l-1),
    // (j, l-1), (j+h, l-1); backward (e, l) waits for the backward items of e-s and
    // e+s (finished at higher levels) and for the forward item that finished y_e.
    std::vector<std::vector<int32_t>> fwd_index(levels + 1);
    std::vector<int32_t> fwd_final(N + 1, -1), bwd_index(N + 1, -1);
    P->solve_flow.clear();
    P->fwd_node.clear();
    P->fwd_level.clear();
    for (int l = 1; l <= levels; ++l) {
      const int64_t s = int64_t(1) << (l - 1), h = s / 2;
      fwd_index[l].assign(N + 1, -1);
      for (const FwdItem &f : P->lv[l - 1].fwd) {
        const int64_t j = f.y_self - y_base + 1;
        SolveFlowItem q;
        q.y_self = f.y_self;
        q.y_a = f.y_l;
        q.e_a = f.e_l;
        q.y_b = f.y_r;
        q.e_b = f.e_r;
        q.d_self = f.d_self;
        q.kind = 0;
        q.dep[0] = q.dep[1] = q.dep[2] = -1;
        if (l > 1) {
          const int64_t cand[3] = {j - h, j, j + h};
          for (int k = 0; k < 3; ++k)
            if (cand[k] >= 1 && cand[k] <= N) q.dep[k] = fwd_index[l - 1][cand[k]];
        }
        fwd_index[l][j] = (int32_t)P->solve_flow.size();
        if (f.d_self >= 0) fwd_final[j] = (int32_t)P->solve_flow.size();
        P->solve_flow.push_back(q);
        P->fwd_node.push_back((int32_t)j);
        P->fwd_level.push_back(l);
      }
    }
    P->n_fwd = (int32_t)P->solve_flow.size();
    for (int l = levels; l >= 1; --l) {
      for (const BwdItem &b : P->lv[l - 1].bwd) {
        const int64_t e = b.x_self - y_base + 1;
        SolveFlowItem q;
        q.y_self = b.x_self;
        q.y_a = b.x_dn;
        q.e_a = b.e_dn;
        q.y_b = b.x_up;
        q.e_b = b.e_up;
        q.d_self = b.d_self;
        q.kind = 1;
        const int64_t s = int64_t(1) << (l - 1);
        q.dep[0] = (e + s <= N) ? bwd_index[e + s] : -1;
        q.dep[1] = (e - s >= 1) ? bwd_index[e - s] : -1;
        q.dep[2] = fwd_final[e];
        bwd_index[e] = (int32_t)P->solve_flow.size();
        P->solve_flow.push_back(q);
      }
    }
  }
  // Solve flops (Alg. 7 costs): trsm n^2 m per node and direction, gemm 2 n^2 m per
  // off-diagonal block and direction.
  sol = 2.0 * N * n2 + 4.0 * (double)P->offdiag * n2;
  P->factor_flops = fl;
  P->seq_factor_flops = (7.0 / 3.0 * N - 2.0) * n3;
  P->crit_flops = crit;
  // Sec. 4.3 closed form with p = infinity (N >= 2): 16/3 + 22/3 (floor(log2 N) - 1) + 4/3, times n^3
  int lg = levels - 1;
  P->crit_formula = N >= 2 ? (16.0 / 3.0 + 22.0 / 3.0 * (lg - 1) + 4.0 / 3.0) * n3 : n3 / 3.0;
  P->solve_flops_per_rhs = sol;
}

void build_interlaced(const HostPlan &P, bool root_separate, std::vector<int32_t> *code, std::vector<int32_t> *deps,
                      std::vector<SolveFlowItem> *tail) {
  const int N = P.N, levels = P.levels;
  code->clear();
  deps->clear();
  tail->clear();
  // flat factor index of the node eliminated at each level
  std::vector<int32_t> fac_start(levels + 1, 0), fac_of_node(N + 1, -1);
  for (int l = 1; l <= levels; ++l) {
    fac_start[l] = fac_start[l - 1] + (int32_t)P.lv[l - 1].fac.size();
    for (size_t q = 0; q < P.lv[l - 1].fac.size(); ++q) fac_of_node[P.lv[l - 1].fac[q].node + 1] = fac_start[l - 1] + (int32_t)q;
  }
  std::vector<int32_t> fac_ticket(fac_start[levels], -1), fwd_ticket(P.n_fwd, -1);
  auto push = [&](int32_t c, const int32_t (&d)[kInterDeps]) {
    code->push_back(c);
    deps->insert(deps->end(), d, d + kInterDeps);
    return (int32_t)code->size() - 1;
  };
  int32_t w = 0;  // next forward item
  for (int l = 1; l <= levels; ++l) {
    if (root_separate && l == levels) break;  // the top separator: factored by its own kernel
    const int64_t h = (int64_t(1) << (l - 1)) / 2;
    for (int32_t f = fac_start[l - 1]; f < fac_start[l]; ++f) {
      int32_t d[kInterDeps] = {-1, -1, -1, -1, -1, -1};
      for (int k = 0; k < 3; ++k) {
        const int32_t src = P.fac_deps[3 * (size_t)f + k];
        d[k] = src == -1 ? -1 : src >= 0 ? fac_ticket[src] : core_dep(fac_ticket[dep_item(src)]);
      }
      fac_ticket[f] = push(f, d);
    }
    for (; w < P.n_fwd && P.fwd_level[w] == l; ++w) {
      const SolveFlowItem &it = P.solve_flow[w];
      const int64_t j = P.fwd_node[w];
      int32_t d[kInterDeps] = {-1, -1, -1, -1, -1, -1};
      for (int k = 0; k < 3; ++k) d[k] = it.dep[k] >= 0 ? fwd_ticket[it.dep[k]] : -1;
      // the factor items that write U_j (level l), U(j-h, j) and U(j+h, j) (level l-1): their factor
      // blocks suffice
      if (it.d_self >= 0) d[3] = core_dep(fac_ticket[fac_of_node[j]]);
      if (it.y_a >= 0) d[4] = core_dep(fac_ticket[fac_of_node[j - h]]);
      if (it.y_b >= 0) d[5] = core_dep(fac_ticket[fac_of_node[j + h]]);
      fwd_ticket[w] = push(-1 - w, d);
    }
  }
  // the tail: [top-separator forward item] + backward items
  int32_t root_fwd = -1;
  if (root_separate) {
    root_fwd = P.n_fwd - 1;  // the single forward item of the top level
    SolveFlowItem r = P.solve_flow[root_fwd];
    r.dep[0] = r.dep[1] = r.dep[2] = -1;  // its inputs are complete before the tail starts
    tail->push_back(r);
  }
  const int32_t off = root_separate ? 1 : 0;
  for (size_t b = (size_t)P.n_fwd; b < P.solve_flow.size(); ++b) {
    SolveFlowItem q = P.solve_flow[b];
    for (int k = 0; k < 2; ++k) q.dep[k] = q.dep[k] >= 0 ? q.dep[k] - P.n_fwd + off : -1;
    q.dep[2] = (root_fwd >= 0 && q.dep[2] == root_fwd) ? 0 : -1;
    tail->push_back(q);
  }
}

}  // namespace btc

namespace btc {

int build_solve_waves(const std::vector<SolveFlowItem> &items, std::vector<int32_t> *order,
                      std::vector<int32_t> *wave_off) {
  const int n = (int)items.size();
  std::vector<int32_t> depth(n, 0);
  int nw = 0;
  for (int i = 0; i < n; ++i) {
    for (int32_t d : items[i].dep) {
      if (d == -1) continue;
      if (d < 0 || d >= i) return -1;
      depth[i] = std::max(depth[i], depth[d] + 1);
    }
    nw = std::max(nw, depth[i] + 1);
  }
  wave_off->assign(nw + 1, 0);
  for (int i = 0; i < n; ++i) ++(*wave_off)[depth[i] + 1];
  int widest = 0;
  for (int w = 0; w < nw; ++w) {
    widest = std::max(widest, (*wave_off)[w + 1]);
    (*wave_off)[w + 1] += (*wave_off)[w];
  }
  order->assign(n, 0);
  std::vector<int32_t> pos(wave_off->begin(), wave_off->end() - 1);
  for (int i = 0; i < n; ++i) (*order)[pos[depth[i]]++] = i;
  return widest;
}

void build_tile_tasks(const HostPlan &P, std::vector<TileTask> *tasks, std::vector<int32_t> *node_total) {
  constexpr int64_t T = kTileT, LDG = kTileNP;
  tasks->clear();
  int32_t nitems = 0;
  for (const LevelSchedule &L : P.lv) nitems += (int32_t)L.fac.size();
  node_total->assign(nitems, 0);
  // per-node task counts by phase
  auto count_phases = [](const FactorItem &it, int32_t c[4]) {
    c[0] = it.p_a >= 0 ? 3 : 0;
    c[1] = 1;
    c[2] = (it.r_up >= 0 ? 2 : 0) + (it.r_down >= 0 ? 2 : 0);
    c[3] = (it.d_next >= 0 ? 3 : 0) + (it.fill >= 0 ? 4 : 0);
  };
  int32_t base = 0;  // flat index of the level's first item
  for (const LevelSchedule &L : P.lv) {
    const int32_t nl = (int32_t)L.fac.size();
    for (int32_t q = 0; q < nl; ++q) {
      int32_t c[4];
      count_phases(L.fac[q], c);
      (*node_total)[base + q] = c[0] + c[1] + c[2] + c[3];
    }
    for (int phase = 0; phase < 4; ++phase)
      for (int32_t q = 0; q < nl; ++q) {
        const FactorItem &it = L.fac[q];
        const int32_t f = base + q;
        int32_t c[4];
        count_phases(it, c);
        int32_t before = 0;
        for (int k = 0; k < phase; ++k) before += c[k];
        TileTask t;
        t.c = t.x0 = t.y0 = t.x1 = t.y1 = -1;
        t.kind = TK_GEMM;
        t.flags = 0;
        t.ti = t.tj = 0;
        t.counter = f;
        t.wait_self = before;
        for (int k = 0; k < 3; ++k) {
          // the tile tasks count a node's completed tasks only: a dependency on another node's
          // factor blocks waits for the whole node
          const int32_t raw = P.fac_deps.empty() ? -1 : P.fac_deps[3 * (size_t)f + k];
          const int32_t d = raw == -1 ? -1 : dep_item(raw);
          t.dep[k] = d;
          t.dep_n[k] = d >= 0 ? (*node_total)[d] : 0;
        }
        t.node = it.node;
        t.inst = it.inst;
        auto gemm = [&](int64_t c_blk, int flags, int64_t x0, int64_t y0, int64_t x1, int64_t y1, int i, int j) {
          TileTask g = t;
          g.kind = TK_GEMM;
          g.flags = flags;
          g.c = c_blk;
          g.x0 = x0;
          g.y0 = y0;
          g.x1 = x1;
          g.y1 = y1;
          g.ti = i;
          g.tj = j;
          tasks->push_back(g);
        };
        static const int up3[3][2] = {{0, 0}, {0, 1}, {1, 1}};
        if (phase == 0 && it.p_a >= 0)
          for (auto &ij : up3) gemm(it.d_self, 0, it.p_a, it.p_a, -1, -1, ij[0], ij[1]);
        if (phase == 1) {
          TileTask pt = t;
          pt.kind = TK_POTRF;
          pt.c = it.d_self;
          tasks->push_back(pt);
        }
        if (phase == 2)
          for (int64_t r : {it.r_up, it.r_down}) {
            if (r < 0) continue;
            for (int j = 0; j < 2; ++j) {
              TileTask tt = t;
              tt.kind = TK_TRSM;
              tt.c = it.d_self;
              tt.x0 = r;
              tt.tj = j;
              tasks->push_back(tt);
            }
          }
        if (phase == 3) {
          if (it.d_next >= 0) {
            const int64_t pb = it.p_b >= 0 ? it.p_b : -1;
            for (auto &ij : up3)
              if (pb >= 0) gemm(it.d_next, 0, pb, pb, it.r_down, it.r_down, ij[0], ij[1]);
              else gemm(it.d_next, 0, it.r_down, it.r_down, -1, -1, ij[0], ij[1]);
          }
          if (it.fill >= 0) {
            const bool upfirst = (it.flags & FI_FILL_UPFIRST) != 0;
            const int64_t X = upfirst ? it.r_up : it.r_down, Y = upfirst ? it.r_down : it.r_up;
            for (int i = 0; i < 2; ++i)
              for (int j = 0; j < 2; ++j) gemm(it.fill, TG_NEG_STORE | TG_C_EPOOL, X, Y, -1, -1, i, j);
          }
        }
      }
    base += nl;
  }
  (void)T;
  (void)LDG;
}

}  // namespace btc

namespace btc {

// Chunk sizes of the partition permutation (Proposition 1): N_k* = (7N - 7p + 7) / (7p + 12) rounded down
// and up, N_1 = N - (p - 1)(N_k + 1), keeping the split whose larger parallel-phase cost
// max(7/3 N_1 - 1, 19/3 N_k - 1) is smaller; chunks k > 1 hold at least one node. nk = 0 when p = 1.
void partition_sizes(int N, int chunks, int *n1, int *nk) {
  *n1 = N;
  *nk = 0;
  if (chunks <= 1) return;
  const double star = (7.0 * N - 7.0 * chunks + 7.0) / (7.0 * chunks + 12.0);
  double best = 1e300;
  for (int c : {(int)std::floor(star), (int)std::ceil(star)}) {
    c = std::max(c, 1);
    const int a = N - (chunks - 1) * (c + 1);
    if (a < 1) continue;
    const double cost = std::max(7.0 / 3.0 * a - 1.0, 19.0 / 3.0 * c - 1.0);
    if (cost < best) {
      best = cost;
      *n1 = a;
      *nk = c;
    }
  }
  if (best == 1e300) *n1 = *nk = -1;
}

bool build_partition_plan(int N, int n, int np, int chunks, int64_t d_base, int64_t e_base, int64_t y_base, int inst,
                          HostPlan *P) {
  int n1, nk;
  partition_sizes(N, std::max(chunks, 1), &n1, &nk);
  if (n1 < 1) return false;
  const int p = std::max(chunks, 1);
  *P = HostPlan();
  P->N = N;
  P->n = n;
  P->np = np;
  P->chunks = p;
  P->packed = true;
  const int64_t bs = (int64_t)np * np;
  auto dOff = [&](int v) { return (d_base + v) * bs; };
  // chunk of every node (0 = chunk 1; k - 1 for chunk k) and pivots (-1)
  std::vector<int> chunk_of(N, 0), pivot(p + 1, -1);  // pivot[k] = node of A_k, k = 2..p
  std::vector<std::vector<int>> members(p);
  for (int v = 0; v < n1; ++v) members[0].push_back(v);
  int v = n1;
  for (int k = 2; k <= p; ++k) {
    pivot[k] = v;
    chunk_of[v] = -1;
    ++v;
    for (int i = 0; i < nk; ++i, ++v) {
      chunk_of[v] = k - 1;
      members[k - 1].push_back(v);
    }
  }
  // elimination order: chain positions across chunks, then the pivots
  std::vector<std::vector<int>> lev;
  const int maxlen = std::max(n1, nk);
  for (int pos = 0; pos < maxlen; ++pos) {
    std::vector<int> L;
    for (int k = 0; k < p; ++k)
      if (pos < (int)members[k].size()) L.push_back(members[k][pos]);
    lev.push_back(L);
  }
  for (int k = 2; k <= p; ++k) lev.push_back({pivot[k]});
  std::vector<int> order, posn(N, -1), level_of(N, 0);
  for (size_t l = 0; l < lev.size(); ++l)
    for (int e : lev[l]) {
      posn[e] = (int)order.size();
      level_of[e] = (int)l + 1;
      order.push_back(e);
    }
  // slots: original couplings (v, v+1) at slot v, fills appended
  int64_t nslots = std::max(N - 1, 0);
  P->slot_transposed.assign(std::max(N - 1, 0), 0);
  P->slot_e.assign(std::max(N - 1, 0), -1);
  P->slot_o.assign(std::max(N - 1, 0), -1);
  for (int s = 0; s + 1 < N; ++s) P->slot_transposed[s] = posn[s] < posn[s + 1] ? 1 : 0;
  // path elimination: current neighbours and coupling slots
  std::vector<int> lft(N), rgt(N);
  std::vector<int64_t> sl(N, -1), sr(N, -1);
  for (int u = 0; u < N; ++u) {
    lft[u] = u - 1;
    rgt[u] = u + 1 < N ? u + 1 : -1;
    sl[u] = u > 0 ? u - 1 : -1;
    sr[u] = u + 1 < N ? u : -1;
  }
  auto eOff = [&](int64_t slot) { return (e_base + slot) * bs; };
  std::vector<int32_t> item_of(N, -1);      // flat factor index of each node
  std::vector<int64_t> deferred_from(N, -1);  // slot of the block deferred onto a node (its p_a)
  std::vector<int32_t> deferred_item(N, -1);  // ... and the item that wrote it
  std::vector<int32_t> last_imm(N, -1);       // last item that updated a node immediately
  std::vector<int32_t> slot_writer;           // item that created a fill slot (index - (N - 1))
  std::vector<std::pair<int, int>> nbr_at(N, {-1, -1});
  std::vector<std::pair<int64_t, int64_t>> nbr_slot(N, {-1, -1});
  auto last_of_chunk = [&](int k) { return members[k - 1].empty() ? -1 : members[k - 1].back(); };
  P->lv.assign(lev.size(), LevelSchedule());
  P->fac_deps.clear();
  const double n3 = (double)n * n * n, n2 = (double)n * n;
  double fl = 0, crit = 0;
  int32_t idx = 0;
  for (size_t l = 0; l < lev.size(); ++l) {
    LevelSchedule &LS = P->lv[l];
    LS.s = 0;
    double level_max = 0;
    for (int e : lev[l]) {
      const int a = lft[e], b = rgt[e];
      const int64_t sa = sl[e], sb = sr[e];
      nbr_at[e] = {a, b};
      nbr_slot[e] = {sa, sb};
      // roles: chains of chunks k > 1 update their pivot (left) at once and defer the right neighbour;
      // chunk 1 updates its right neighbour at once unless that is a pivot (deferred); pivots update
      // the next pivot at once
      int down = -1, up = -1;
      int64_t s_down = -1, s_up = -1;
      if (chunk_of[e] >= 1) {
        down = a, s_down = sa, up = b, s_up = sb;
      } else if (chunk_of[e] == 0) {
        if (b >= 0 && chunk_of[b] == -1) up = b, s_up = sb;
        else down = b, s_down = sb;
      } else {
        down = b, s_down = sb;
        if (a >= 0) up = a, s_up = sa;  // (never: the previous pivot is eliminated first)
      }
      FactorItem it;
      it.d_self = dOff(e);
      it.d_next = down >= 0 ? dOff(down) : -1;
      it.r_down = down >= 0 ? eOff(s_down) : -1;
      it.r_up = up >= 0 ? eOff(s_up) : -1;
      it.p_a = deferred_from[e] >= 0 ? eOff(deferred_from[e]) : -1;
      it.p_b = -1;
      it.d_prev = -1;
      it.fill = -1;
      it.flags = 0;
      it.node = e;
      it.inst = inst;
      it.pad = 0;
      int64_t fslot = -1;
      if (up >= 0 && down >= 0) {
        fslot = nslots++;
        it.fill = eOff(fslot);
        if (posn[up] < posn[down]) it.flags |= FI_FILL_UPFIRST;
        slot_writer.push_back(idx);
        P->slot_e.push_back(posn[up] < posn[down] ? up : down);
        P->slot_o.push_back(posn[up] < posn[down] ? down : up);
      }
      if (l + 1 == lev.size()) it.flags |= FI_ROOT;
      // factor-pool slot bookkeeping for btc_get_factor: the blocks this node stores
      if (s_up >= 0 && s_up < N - 1) {
        P->slot_e[s_up] = e;
        P->slot_o[s_up] = up;
      }
      if (s_down >= 0 && s_down < N - 1) {
        P->slot_e[s_down] = e;
        P->slot_o[s_down] = down;
      }
      // dependencies (at most three): the producer of the deferred block, the last immediate writer of
      // D_e, the creators of the fill slots it reads; and, for a pivot, the chain that still updates the
      // pivot it writes (chunk k + 1)
      std::vector<int32_t> dep;
      auto add = [&](int32_t d) {
        if (d >= 0 && std::find(dep.begin(), dep.end(), d) == dep.end()) dep.push_back(d);
      };
      if (chunk_of[e] == -1) {
        int k = 0;
        for (int q = 2; q <= p; ++q)
          if (pivot[q] == e) k = q;
        if (k == 2) {
          add(item_of[last_of_chunk(1)]);
          add(item_of[last_of_chunk(2)]);
        } else {
          add(item_of[pivot[k - 1]]);  // transitively: chunks up to k
        }
        if (k + 1 <= p) add(item_of[last_of_chunk(k + 1)]);  // chunk k + 1 still updates A_(k+1)
      } else {
        add(deferred_item[e]);
        add(last_imm[e]);
        for (int64_t s2 : {sa, sb})
          if (s2 >= N - 1) add(slot_writer[s2 - (N - 1)]);
      }
      if (dep.size() > 3) return false;  // (cannot happen for this order)
      while (dep.size() < 3) dep.push_back(-1);
      P->fac_deps.insert(P->fac_deps.end(), dep.begin(), dep.end());
      // state after eliminating e
      if (up >= 0) {
        deferred_from[up] = s_up;
        deferred_item[up] = idx;
      }
      if (down >= 0) last_imm[down] = idx;
      if (a >= 0) rgt[a] = b, sr[a] = fslot;
      if (b >= 0) lft[b] = a, sl[b] = fslot;
      item_of[e] = idx++;
      double c = n3 / 3.0;
      if (it.p_a >= 0) c += n3;
      if (it.r_down >= 0) c += 2 * n3;  // trsm + immediate syrk
      if (it.r_up >= 0) c += n3;
      if (it.fill >= 0) c += 2 * n3;
      fl += c;
      level_max = std::max(level_max, c);
      LS.fac.push_back(it);
    }
    crit += level_max;
  }
  P->levels = (int)lev.size();
  P->offdiag = nslots;
  P->fill = nslots - std::max(N - 1, 0);
  P->fac_deps_rl.assign(P->fac_deps.size(), -1);
  P->level_slot_off.assign(P->levels + 2, 0);
  // ---- solve (pull form forward in elimination order, backward in reverse)
  auto yNode = [&](int u) { return y_base + u; };
  P->solve_flow.clear();
  P->solve_key.clear();
  std::vector<int32_t> fwd_final(N, -1), bwd_item(N, -1);
  auto push = [&](int64_t self, int qa, int64_t ea, int qb, int64_t eb, int64_t dself, int kind, int32_t d0, int32_t d1,
                  int32_t d2) {
    SolveFlowItem q;
    q.y_self = yNode(self);
    q.y_a = qa >= 0 ? yNode(qa) : -1;
    q.e_a = qa >= 0 ? ea : -1;
    q.y_b = qb >= 0 ? yNode(qb) : -1;
    q.e_b = qb >= 0 ? eb : -1;
    q.d_self = dself;
    q.kind = kind;
    q.dep[0] = d0;
    q.dep[1] = d1;
    q.dep[2] = d2;
    P->solve_flow.push_back(q);
    const int lvl = level_of[self];
    P->solve_key.push_back(kind == 0 ? lvl : -lvl);
    return (int32_t)P->solve_flow.size() - 1;
  };
  // the block stored by eliminated node q for its coupling with e (rows: q's variables)
  auto stored = [&](int q, int e) -> int64_t {
    return nbr_at[q].first == e ? eOff(nbr_slot[q].first) : eOff(nbr_slot[q].second);
  };
  // chain nodes (elimination order): the only earlier-eliminated node coupled with a chain node is its
  // predecessor in the chunk (whose right neighbour it was); pull its contribution, then solve
  for (int e : order) {
    if (chunk_of[e] == -1) continue;
    const auto &mem = members[chunk_of[e]];
    const size_t i = std::find(mem.begin(), mem.end(), e) - mem.begin();
    const int contrib = i > 0 ? mem[i - 1] : -1;
    fwd_final[e] = push(e, contrib, contrib >= 0 ? stored(contrib, e) : -1, -1, -1, dOff(e), 0,
                        contrib >= 0 ? fwd_final[contrib] : -1, -1, -1);
  }
  // pivots: accumulate the contributions of their chunk in pairs, then the previous chunk's last node and
  // the previous pivot, and solve
  for (int k = 2; k <= p; ++k) {
    const int A = pivot[k];
    const auto &mem = members[k - 1];
    int32_t prev_item = -1;
    for (size_t i = 0; i < mem.size(); i += 2) {
      const int qa = mem[i], qb = i + 1 < mem.size() ? mem[i + 1] : -1;
      prev_item = push(A, qa, stored(qa, A), qb, qb >= 0 ? stored(qb, A) : -1, -1, 0, prev_item, fwd_final[qa],
                       qb >= 0 ? fwd_final[qb] : -1);
    }
    const int lastp = last_of_chunk(k - 1);
    const int prevA = k > 2 ? pivot[k - 1] : -1;
    // the previous pivot's final item (listed before this one) orders the writes to y_A as well
    fwd_final[A] = push(A, lastp, stored(lastp, A), prevA, prevA >= 0 ? stored(prevA, A) : -1, dOff(A), 0, prev_item,
                        fwd_final[lastp], prevA >= 0 ? fwd_final[prevA] : -1);
  }
  P->n_fwd = (int32_t)P->solve_flow.size();
  P->fwd_node.assign(P->n_fwd, 0);
  P->fwd_level.assign(P->n_fwd, 0);
  for (auto it = order.rbegin(); it != order.rend(); ++it) {
    const int e = *it;
    const int a = nbr_at[e].first, b = nbr_at[e].second;
    bwd_item[e] = push(e, a, a >= 0 ? eOff(nbr_slot[e].first) : -1, b, b >= 0 ? eOff(nbr_slot[e].second) : -1, dOff(e),
                       1, a >= 0 ? bwd_item[a] : -1, b >= 0 ? bwd_item[b] : -1, fwd_final[e]);
  }
  P->factor_flops = fl;
  P->seq_factor_flops = (7.0 / 3.0 * N - 2.0) * n3;
  P->crit_flops = crit;
  P->crit_formula = crit;
  P->solve_flops_per_rhs = 2.0 * N * n2 + 4.0 * (double)P->offdiag * n2;
  return true;
}

}  // namespace btc
