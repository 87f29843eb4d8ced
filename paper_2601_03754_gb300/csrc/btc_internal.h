// Internal types shared by the host planner (btc_plan.cpp), the kernels and
// the runtime. Not part of the public ABI.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

namespace btc {

// Storage convention of the factor pools.
//  * Dhat pool: one padded np x np block per node (row-major); after the
//    factorization it holds L(e, e) (lower triangle, zeros above).
//  * U pool: one np x np block per slot, level-major. Level l (stride
//    s = 2^(l-1)) has K_l = floor(N/s) - 1 slots; slot k (1-based) couples the
//    surviving nodes k*s and (k+1)*s. Exactly one of the two is eliminated at
//    level l (the odd multiple of s), call it e, the other o. Before level l
//    the slot holds the Schur-complement block S(e, o) (rows: e's variables);
//    level l overwrites it with U(e, o) = Dhat_e^{-1} S(e, o) = L(o, e)^T.
//  With this orientation every block product of Alg. 5 is C -= X^T Y and
//  every triangular solve is Z = L^{-1} R (left, lower).

enum : int32_t {
  FI_FILL_UPFIRST = 1,  // fill block stores S'(e-s, e+s) = -Zu^T Zd (e-s is eliminated next); else S'(e+s, e-s)
  FI_ROOT = 2,          // last level (the top separator)
};

// One eliminated node e at level l (Alg. 5, one iteration of the parallel loop).
// Offsets are in ELEMENTS into the Dhat / U pools, -1 when the step is absent.
// Dependency encoding of the persistent launches: d >= 0 waits for item d to be
// complete; core_dep(d) (<= -2) waits only until item d has stored its factor
// blocks (U_e and its two off-diagonal blocks), before its trailing products;
// -1 is none.
constexpr int32_t core_dep(int32_t item) { return -item - 2; }
constexpr int32_t dep_item(int32_t d) { return d >= 0 ? d : -d - 2; }

struct FactorItem {
  int64_t d_self;  // Dhat_e
  int64_t d_next;  // Dhat_{e+s}                      (syrk target)
  int64_t r_up;    // slot of S(e, e-s) -> U(e, e-s)  (trsm)
  int64_t r_down;  // slot of S(e, e+s) -> U(e, e+s)  (trsm)
  int64_t p_a;     // deferred block onto Dhat_e:     U(e+s/2, e)        (level > 1)
  int64_t p_b;     // deferred block onto Dhat_{e+s}: U(e+3s/2, e+s)     (level > 1)
  int64_t fill;    // new slot at level l+1 for the pair (e-s, e+s)
  int64_t d_prev;  // Dhat_{e-s} (Alg. 6 updates it immediately; Alg. 5 defers the update)
  int32_t node;    // e, 0-based, within its instance
  int32_t flags;
  int32_t inst;    // instance index (batched plans)
  int32_t pad;
};

// Forward substitution at level l for a surviving node j (pull form):
// y_j -= U(j-h, j)^T y_{j-h} + U(j+h, j)^T y_{j+h}  (contributions of level l-1,
// h = s/2), then y_j <- Dhat_j^{-1} y_j if j is eliminated at level l.
struct FwdItem {
  int64_t y_self;      // node index (global across instances) of y_j
  int64_t y_l, e_l;    // y_{j-h} node and U(j-h, j) offset, or -1
  int64_t y_r, e_r;    // y_{j+h} node and U(j+h, j) offset, or -1
  int64_t d_self;      // Dhat_j offset, or -1 if j survives this level
};

// Backward substitution at level l for an eliminated node e:
// x_e <- Dhat_e^{-T} (y_e - U(e, e+s) x_{e+s} - U(e, e-s) x_{e-s}).
struct BwdItem {
  int64_t x_self, d_self;
  int64_t x_dn, e_dn;  // x_{e+s} node and U(e, e+s) offset, or -1
  int64_t x_up, e_up;  // x_{e-s} node and U(e, e-s) offset, or -1
};

// One item of the fused forward+backward solve of the persistent kernel
// (forward items of all levels, then backward items from the top level down).
// kind 0 (forward, survivor j):  y_j -= U(a)^T y_a + U(b)^T y_b; if d_self: y_j <- U_j^{-T} y_j
// kind 1 (backward, eliminated e): y_e <- U_e^{-1} (y_e - U(a) y_a - U(b) y_b)
struct SolveFlowItem {
  int64_t y_self;
  int64_t y_a, e_a;  // fwd: left contribution; bwd: down neighbour
  int64_t y_b, e_b;  // fwd: right contribution; bwd: up neighbour
  int64_t d_self;
  int32_t kind;
  int32_t dep[3];    // indices of the items this one waits for (-1: none), all smaller
};

// Blocked node elimination for blocks larger than one CTA's shared memory
// (padded n = 256): every node of Alg. 5 becomes a few tasks on 128 x 128
// tiles (kTileT) of its 256 x 256 blocks (row stride kTileNP), run by one
// persistent launch. Per node, in phase order:
//   A  deferred syrk: S_e(i,j) -= sum_k P_a(k,i)^T P_a(k,j), upper tiles   (TK_GEMM x3)
//   P  blocked potrf of S_e: U00, U01 = U00^-T S01, S11 -= U01^T U01, U11 (TK_POTRF)
//   T  trsm of S(e,e-s) and S(e,e+s), one task per column tile j:
//      Z0j = U00^-T R0j, R1j -= U01^T Z0j, Z1j = U11^-T R1j            (TK_TRSM x2 per block)
//   G  S_{e+s}(i,j) -= P_b^T P_b + U_dn^T U_dn, upper tiles              (TK_GEMM x3)
//      fill(i,j) = -U_up^T U_dn or -U_dn^T U_up, all four tiles          (TK_GEMM x4)
// A node's tasks wait for its earlier phases (node counter >= wait_self) and
// for the nodes of the previous level that produce its blocks (the producers
// of Alg. 5's dataflow, each counter >= its task total).
constexpr int kTileT = 128, kTileNP = 256;
enum : int32_t { TK_GEMM = 0, TK_POTRF = 1, TK_TRSM = 2 };
enum : int32_t {
  TG_NEG_STORE = 1,  // gemm: C = -(sum) (a fill block); else C -= sum
  TG_C_EPOOL = 2,    // gemm: C lives in the off-diagonal pool; else in the diagonal pool
};
struct TileTask {
  int64_t c;       // GEMM: C block; POTRF: S_e block; TRSM: U_e block (element offsets)
  int64_t x0, y0;  // GEMM: first operand pair (blocks of the off-diagonal pool); TRSM: x0 = R block
  int64_t x1, y1;  // GEMM: second operand pair, or -1
  int32_t kind, flags;
  int32_t ti, tj;       // GEMM: output tile; TRSM: tj = column tile
  int32_t counter;      // this node's completion counter
  int32_t wait_self;    // tasks of this node in earlier phases
  int32_t dep[3];       // producer counters (-1: none)
  int32_t dep_n[3];     // ... and their task totals
  int32_t node, inst;   // node (0-based, for pivot reports) and instance
};

constexpr int kTileThreads = 256;  // threads of a tile-task CTA (a 16 x 16 grid of 8 x 8 register tiles)

// Arguments of the persistent tile-task launch.
struct TileArgs {
  const TileTask *tasks;
  int count;
  float *dpool, *epool;
  int *counters;             // one per node (flat factor index): its tasks finished
  unsigned long long *info;  // pivot report per instance
};

struct LevelSchedule {
  int s;  // stride 2^(l-1)
  std::vector<FactorItem> fac;
  std::vector<FwdItem> fwd;
  std::vector<BwdItem> bwd;
};

struct HostPlan {
  int N = 0, n = 0, np = 0, levels = 0;
  // elimination order: 0 = nested dissection (P_inf, Sec. 4.3); c >= 1 = the partition permutation
  // of Sec. 4.1 with c chunks (c = 1: the natural order of Alg. 1). Partition plans read packed pools
  // at every level (packed), whose original coupling slot v (nodes v, v + 1) holds B_v^T when v is
  // eliminated first (slot_transposed[v] = 1), else B_v.
  int chunks = 0;
  bool packed = false;
  std::vector<int8_t> slot_transposed;
  // dataflow form: factor items in level order with the (<= 3) items of the
  // previous level that produce their inputs, and the fused solve list
  std::vector<int32_t> fac_deps;           // 3 per factor item (flat level order), -1: none
  std::vector<int32_t> fac_deps_rl;        // the same for the right-looking variant (Alg. 6)
  std::vector<SolveFlowItem> solve_flow;
  int64_t offdiag = 0, fill = 0;
  std::vector<int64_t> level_slot_off;  // first U slot of each level (in blocks)
  std::vector<LevelSchedule> lv;
  std::vector<int> slot_e, slot_o;      // per U slot: eliminated node and partner (0-based)
  double factor_flops = 0, seq_factor_flops = 0, crit_flops = 0, crit_formula = 0;
  double solve_flops_per_rhs = 0;
  // forward items of solve_flow (the first n_fwd entries): node (1-based) and level
  int32_t n_fwd = 0;
  std::vector<int32_t> fwd_node, fwd_level;
  // partition plans: per solve_flow item, its merge key among instances (forward: the launch level of
  // its node; backward: minus that level), so that every dependency sorts before its consumer
  std::vector<int32_t> solve_key;
};

// Interlaced factorization and forward substitution in one persistent launch
// (the forward sweep of level l runs as soon as the blocks it reads are
// factored). Entry t of `code` is a factor item (code >= 0, flat level-order
// index) or a forward item (code < 0: solve_flow index -code-1); its
// dependencies are kInterDeps earlier entries (-1: none). Order: factor items
// of level 1, forward items of level 1, factor items of level 2, ...
// root_separate (mixed path): the top separator's factor and forward items
// are left out; its FP64 factor runs between the two launches. `tail` is the
// rest of the solve for a second persistent launch: the top separator's
// forward item (root_separate only, first), then every backward item, with
// dependencies renumbered within the tail.
constexpr int kInterDeps = 6;
void build_interlaced(const HostPlan &P, bool root_separate, std::vector<int32_t> *code, std::vector<int32_t> *deps,
                      std::vector<SolveFlowItem> *tail);

// Build the schedule. Offsets are relative to the given bases (in blocks for
// the pools, in nodes for the work vector) so that batched plans can
// concatenate instances.
void build_host_plan(int N, int n, int np, int64_t d_base, int64_t e_base, int64_t y_base, int inst,
                     HostPlan *out);

// Tile tasks of a plan in launch order (level by level, phase by phase within
// a level) and the task total of every node (indexed like the flat factor list).
// Dependency waves of a solve item list (for the one-CTA small solve): `order` lists the items wave
// by wave (an item's dependencies all lie in earlier waves), `wave_off` holds the waves' start
// offsets and the total. Returns the widest wave, or -1 when a dependency is not an earlier item.
int build_solve_waves(const std::vector<SolveFlowItem> &items, std::vector<int32_t> *order,
                      std::vector<int32_t> *wave_off);

void build_tile_tasks(const HostPlan &P, std::vector<TileTask> *tasks, std::vector<int32_t> *node_total);

// The partition permutation (Sec. 4.1, Alg. 4, chunk sizes by Proposition 1) as a plan: chunk interiors
// eliminated left to right (chains, interleaved across chunks by position), then the pivots in order.
// Returns false when `chunks` chunks do not fit in N nodes.
bool build_partition_plan(int N, int n, int np, int chunks, int64_t d_base, int64_t e_base, int64_t y_base, int inst,
                          HostPlan *out);
void partition_sizes(int N, int chunks, int *n1, int *nk);

int padded_size(int n, int dtype);       // np for a block size (0 if unsupported)
int64_t count_offdiag(int N);            // sum over levels of floor(N/s) - 1

}  // namespace btc
