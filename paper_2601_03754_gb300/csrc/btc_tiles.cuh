// Blocked node elimination for 256 x 256 blocks (Alg. 5 with every node split
// into tasks on 128 x 128 tiles; see TileTask in btc_internal.h). One block
// of 256 x 256 FP32 values (256 KB) is larger than an SM's shared memory, so a
// node cannot be one CTA; instead its deferred products, its blocked
// Cholesky, the column strips of its two triangular solves and its
// next-diagonal and fill products are separate tasks of one persistent
// launch, exchanging tiles through global memory (L2-resident at these sizes)
// and ordered by per-node completion counters. Independent tasks of one node
// (four trsm strips, seven products) run on different SMs at the same time.
//
// Arithmetic: the n^3 products (tile GEMMs, K = 128 per MMA group) on tcgen05
// with TF32 or BF16 operands and FP32 accumulation in TMEM; the 128 x 128
// Cholesky and triangular-solve chains on the FP32 pipes (btc_tile.cuh), as
// in the single-CTA node kernels of btc_tc.cuh.
#pragma once
#include "btc_internal.h"
#include "btc_make.cuh"
#include "btc_tc.cuh"
#include "btc_tile.cuh"

namespace btc {

using TileC = TileCfg<float, kTileT, 8>;  // 128 x 128 tiles, 256 threads, 8 x 8 register tiles
static_assert(TileC::NT == kTileThreads, "tile tasks run 256-thread CTAs");

constexpr size_t tile_smem_bytes() { return sizeof(float) * (3 * (size_t)TileC::BLK + kTileT); }

// Wait until this task's own node has finished its earlier phases and every
// producer node has finished all its tasks. Thread 0 polls (acquire); bounded
// like flow_wait (a wait that gives up records kFlowTimeout in *fs.status, and
// a nonzero status makes every later wait give up at once). false: gave up.
__device__ __forceinline__ bool tile_wait(const FlowSync &fs, const int *counters, const TileTask &tk, int *s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int k = 0; k < 4 && ok; ++k) {
      const int idx = k < 3 ? tk.dep[k] : tk.counter;
      const int target = k < 3 ? tk.dep_n[k] : tk.wait_self;
      if (idx < 0 || target <= 0) continue;
      long long polls = 0;
      while (ld_acquire_gpu(counters + idx) < target) {
        if ((++polls & 63) == 0 && (polls > fs.max_polls || *((volatile int *)fs.status) != 0)) {
          atomicOr(fs.status, kFlowTimeout);
          ok = 0;
          break;
        }
        if (polls > 32) __nanosleep(64);
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// One more task of the node is done (after all of this CTA's global writes for it).
__device__ __forceinline__ void tile_publish(int *counter) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
  }
}

// C tile (-)= sum over the operand pairs and both k-tiles of X(k, ti)^T Y(k, tj).
template <int OPB>
__device__ __forceinline__ void tile_gemm(const TileTask &tk, const TileArgs &a, unsigned char *smem, TcState &st) {
  constexpr int64_t T = kTileT, LDG = kTileNP;
  unsigned char *opA = smem, *opB = smem + TcOp<OPB>::BYTES;
  int q = 0;
#pragma unroll 1
  for (int pair = 0; pair < 2; ++pair) {
    const int64_t xo = pair ? tk.x1 : tk.x0, yo = pair ? tk.y1 : tk.y0;
    if (xo < 0) continue;
#pragma unroll 1
    for (int kt = 0; kt < 2; ++kt) {
      if (q > 0) tc_sync(st);  // the previous MMAs have read the operand buffers
      stage_operand_from_pool<kTileThreads, OPB>(opA, a.epool + xo + kt * T * LDG + tk.ti * T, (int)LDG);
      stage_operand_from_pool<kTileThreads, OPB>(opB, a.epool + yo + kt * T * LDG + tk.tj * T, (int)LDG);
      tc_publish_smem();
      if (threadIdx.x == 0) {
        tc_product<OPB>(st.tmem, opA, opB, q > 0);
        tc_commit(st.mbar);
      }
      ++q;
    }
  }
  tc_sync(st);
  float *C = ((tk.flags & TG_C_EPOOL) ? a.epool : a.dpool) + tk.c + tk.ti * T * LDG + tk.tj * T;
  const bool neg_store = (tk.flags & TG_NEG_STORE) != 0;
  tc_read_rows(st.tmem, [&](int i, int j0, const float (&v)[32]) {
#pragma unroll
    for (int t = 0; t < 32; t += 4) {
      float4 *dst = reinterpret_cast<float4 *>(C + i * LDG + j0 + t);
      float4 c;
      if (neg_store) {
        c = make_float4(-v[t], -v[t + 1], -v[t + 2], -v[t + 3]);
      } else {
        c = __ldcg(dst);
        c.x -= v[t];
        c.y -= v[t + 1];
        c.z -= v[t + 2];
        c.w -= v[t + 3];
      }
      *dst = c;
    }
  });
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// sS[i][j] -= acc[i][j] (TMEM accumulator, padded shared tile).
__device__ __forceinline__ void tile_sub_acc(float *sS, uint32_t tmem) {
  tc_read_rows(tmem, [&](int i, int j0, const float (&v)[32]) {
#pragma unroll
    for (int t = 0; t < 32; t += 4) {
      float4 s = *reinterpret_cast<float4 *>(sS + i * TileC::LD + j0 + t);
      s.x -= v[t];
      s.y -= v[t + 1];
      s.z -= v[t + 2];
      s.w -= v[t + 3];
      *reinterpret_cast<float4 *>(sS + i * TileC::LD + j0 + t) = s;
    }
  });
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Blocked Cholesky of one 256 x 256 Schur complement S (upper triangle valid):
// U00 and U01 = U00^-T S01 (one pipelined panel sweep), S11 -= U01^T U01 on
// the tensor cores, U11; the lower-left tile is zeroed.
template <int OPB>
__device__ __forceinline__ void tile_potrf(const TileTask &tk, const TileArgs &a, unsigned char *smem, TcState &st) {
  using C = TileC;
  constexpr int64_t T = kTileT, LDG = kTileNP;
  float *sA = reinterpret_cast<float *>(smem);  // S00 -> U00
  float *sB = sA + C::BLK;                      // S01 -> U01 -> operand
  float *sC = sB + C::BLK;                      // S11 -> U11
  float *dinv = sC + C::BLK;
  float *S = a.dpool + tk.c;
  unsigned long long *info = a.info + tk.inst;
  block_to_smem_async<C>(sA, S, (int)LDG);
  block_to_smem_async<C>(sB, S + T, (int)LDG);
  block_to_smem_async<C>(sC, S + T * LDG + T, (int)LDG);
  cp_async_commit_wait_all();
  __syncthreads();
  block_potrf_trsm<C>(sA, dinv, sB, (float *)nullptr, info, tk.node, [] {}, 0);
  smem_to_block<C>(S, sA, true, (int)LDG);
  smem_to_block<C>(S + T, sB, false, (int)LDG);
  __syncthreads();
  convert_operand_in_place<kTileThreads, C::LD, OPB>(sB);
  tc_publish_smem();
  if (threadIdx.x == 0) {
    tc_product<OPB>(st.tmem, sB, sB, false);  // U01^T U01
    tc_commit(st.mbar);
  }
  tc_sync(st);
  tile_sub_acc(sC, st.tmem);
  __syncthreads();
  block_potrf_trsm<C>(sC, dinv, (float *)nullptr, (float *)nullptr, info, tk.node, [] {}, (int)T);
  smem_to_block<C>(S + T * LDG + T, sC, true, (int)LDG);
  for (int q = threadIdx.x; q < (int)(T * T / 4); q += kTileThreads) {  // lower-left tile of U_e
    const int r = q / (int)(T / 4), c = (q % (int)(T / 4)) * 4;
    *reinterpret_cast<float4 *>(S + (T + r) * LDG + c) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// 1 / U_kk of a factored diagonal tile in shared memory.
__device__ __forceinline__ void tile_dinv(float *dinv, const float *U) {
  for (int k = threadIdx.x; k < kTileT; k += kTileThreads) dinv[k] = 1.0f / U[k * TileC::LD + k];
}

// Column strip j of Z = U_e^-T R (R: S(e,e-s) or S(e,e+s), overwritten):
// Z0 = U00^-T R0j; R1j -= U01^T Z0 (tensor cores); Z1 = U11^-T R1j.
template <int OPB>
__device__ __forceinline__ void tile_trsm(const TileTask &tk, const TileArgs &a, unsigned char *smem, TcState &st) {
  using C = TileC;
  constexpr int64_t T = kTileT, LDG = kTileNP;
  float *sU = reinterpret_cast<float *>(smem);  // U00 -> U01 (operand) -> U11
  float *sZ = sU + C::BLK;                      // R0j -> Z0 (-> operand)
  float *sR = sZ + C::BLK;                      // R1j -> Z1
  float *dinv = sR + C::BLK;
  const float *U = a.dpool + tk.c;
  float *R = a.epool + tk.x0 + tk.tj * T;
  block_to_smem_async<C>(sU, U, (int)LDG);
  block_to_smem_async<C>(sZ, R, (int)LDG);
  block_to_smem_async<C>(sR, R + T * LDG, (int)LDG);
  cp_async_commit_wait_all();
  __syncthreads();
  tile_dinv(dinv, sU);
  __syncthreads();
  block_trsm_ut<C>(sZ, sU, dinv);
  smem_to_block<C>(R, sZ, false, (int)LDG);
  __syncthreads();
  block_to_smem_async<C>(sU, U + T, (int)LDG);  // U01
  cp_async_commit_wait_all();
  __syncthreads();
  convert_operand_in_place<kTileThreads, C::LD, OPB>(sU);
  convert_operand_in_place<kTileThreads, C::LD, OPB>(sZ);
  tc_publish_smem();
  if (threadIdx.x == 0) {
    tc_product<OPB>(st.tmem, sU, sZ, false);  // U01^T Z0
    tc_commit(st.mbar);
  }
  tc_sync(st);
  tile_sub_acc(sR, st.tmem);
  __syncthreads();
  block_to_smem_async<C>(sU, U + T * LDG + T, (int)LDG);  // U11 (the MMAs that read sU are complete)
  cp_async_commit_wait_all();
  __syncthreads();
  tile_dinv(dinv, sU);
  __syncthreads();
  block_trsm_ut<C>(sR, sU, dinv);
  smem_to_block<C>(R + T * LDG, sR, false, (int)LDG);
}

// The persistent launch: CTAs claim tasks in launch order (which is a
// topological order) and run each once its counters allow. One CTA per SM
// (about 200 KB of shared memory), holding its TMEM for its lifetime.
template <int OPB>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile_flow(TileArgs a, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  TcState st;
  tc_begin(st, &s_tmem, s_mbar, fs.status);
  for (;;) {
    const int t = flow_claim(fs, a.count, &s_slot);
    if (t < 0) break;
    const TileTask tk = a.tasks[t];
    flow_trace(fs, t, 0);
    if (tile_wait(fs, a.counters, tk, &s_ok)) {
      flow_trace(fs, t, 1);
      if (tk.kind == TK_GEMM) tile_gemm<OPB>(tk, a, smem_raw, st);
      else if (tk.kind == TK_POTRF) tile_potrf<OPB>(tk, a, smem_raw, st);
      else tile_trsm<OPB>(tk, a, smem_raw, st);
    }
    flow_trace(fs, t, 2);
    tile_publish(a.counters + tk.counter);
  }
  tc_end(st);
}

// Kernel set of the blocked 256 x 256 nodes (tile tasks, btc_tiles.cuh; OPB:
// operand bytes of the tensor-core products): the persistent tile-task launch
// after a packing pass, the solves with the diagonal factor read from global
// memory, and the FP64 residual. No per-level, interlaced or right-looking
// forms and no separate top-separator kernel.
template <int OPB>
KernelSet make_set_tiled() {
  constexpr int NP = kTileNP;
  KernelSet k;
  k.valid = true;
  k.np = NP;
  k.elem = sizeof(float);
  k.src_elem = sizeof(double);
  k.fac_threads = kTileThreads;
  k.fac_smem = tile_smem_bytes();
  k.tiled = true;
  k.tensor_cores = true;
  k.tile_flow = (const void *)&k_tile_flow<OPB>;
  k.tile_smem = tile_smem_bytes();
  k.n_flow_v = 0;
  k.flow_default = 0;
  k.fused_smem = &zero_smem_fn;
  k.pack_pools = &launch_pack<float, double, NP>;
  k.solve_flow = (const void *)&k_solve_flow<float, NP>;
  k.fwd = (const void *)&k_fwd_level<float, NP>;
  k.bwd = (const void *)&k_bwd_level<float, NP>;
  k.fwd_smem = &fwd_smem_fn<float, NP>;
  k.bwd_smem = &bwd_smem_fn<float, NP>;
  k.max_cols = 8;  // the FP64 residual's shared memory grows with n * columns
  k.pack = (const void *)&k_pack_rhs<float, double>;
  k.unpack = (const void *)&k_unpack<float, double>;
  k.resid = (const void *)&k_residual<float>;
  k.residual = &launch_residual<float>;
  return k;
}

}  // namespace btc
