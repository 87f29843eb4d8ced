// Tensor-core (tcgen05) form of the level elimination for 128 x 128 blocks:
// the four n^3 products of a node (Alg. 5: the two deferred syrk, the
// immediate syrk onto the next diagonal block and the fill gemm) run as
// tcgen05.mma with operands in shared memory and FP32 accumulators in TMEM;
// the Cholesky and the two triangular solves stay on the FP32 FMA pipes
// (btc_tile.cuh). Operands are TF32 (kind::tf32, 4-byte elements) or BF16
// (kind::f16 with BF16 A and B, 2-byte elements), both accumulated in FP32.
// The accuracy lost to the short operands is won back by the FP64 refinement
// of the mixed-precision solve.
//
// Operand layout (tcgen05 shared-memory descriptor, no swizzle, K-major): an
// M x K operand is stored as core matrices of 8 rows x 16 bytes (4 TF32 or 8
// BF16 elements along K); element (m, k) sits at byte
// (m/8)*SBO + (k/CK)*LBO + (m%8)*16 + (k%CK)*OPB, with CK = 16/OPB elements
// per core-matrix row, LBO = 128 (core matrices adjacent along K) and
// SBO = 128 * OPB * 8 (adjacent 8-row groups; the whole K extent of 128 lies
// between them). One MMA consumes 32 bytes of K (two core matrices): K = 8
// for TF32, 16 for BF16. A product C[i][j] = sum_k X[k][i] Y[k][j] takes
// A(m=i, k) = X[k][i] and B(n=j, k) = Y[k][j], i.e. both pool blocks in the
// same "transposed" operand layout.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "btc_factor.cuh"
#include "btc_solve.cuh"
#include "btc_tile.cuh"

namespace btc {

constexpr int kTcNP = 128;               // block size of the tensor-core path
constexpr int kTcCols = 256;             // TMEM columns per CTA: two 128-column FP32 accumulators
constexpr long long kTcMaxPolls = 1ll << 24;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Operand element format: OPB = bytes per element (4: TF32, 2: BF16).
template <int OPB>
struct TcOp {
  static_assert(OPB == 4 || OPB == 2, "TF32 or BF16 operands");
  static constexpr int CK = 16 / OPB;                  // K elements per core-matrix row
  static constexpr uint32_t LBO = 128;                 // bytes between core matrices along K
  static constexpr uint32_t SBO = kTcNP * OPB * 8;     // bytes between 8-row groups (K = 128)
  static constexpr int KMMA = 32 / OPB;                // K per MMA instruction
  static constexpr int NMMA = kTcNP / KMMA;            // MMAs per 128-deep product
  static constexpr uint32_t BYTES = kTcNP * kTcNP * OPB;  // one 128 x 128 operand
  // instruction descriptor: FP32 accumulator, A and B of the operand format (TF32 = 2 under
  // kind::tf32, BF16 = 1 under kind::f16), both K-major, N = M = 128
  static constexpr uint32_t FMT = OPB == 4 ? 2u : 1u;
  static constexpr uint32_t IDESC = (1u << 4) | (FMT << 7) | (FMT << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
};

// byte offset of element (m, k) of a K-major operand with K = 128
template <int OPB>
__device__ __forceinline__ uint32_t op_off(int m, int k) {
  using O = TcOp<OPB>;
  return (uint32_t)((m >> 3) * O::SBO + (k / O::CK) * O::LBO + (m & 7) * 16 + (k % O::CK) * OPB);
}

template <int OPB>
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr) {
  using O = TcOp<OPB>;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((O::LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((O::SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Two consecutive-K operand elements packed into the 32-bit word written at op_off(m, k) (k even for
// BF16): TF32 takes one element (x0), BF16 two (x0 at k, x1 at k + 1), each rounded to nearest even.
template <int OPB>
__device__ __forceinline__ uint32_t pack_operand(float x0, float x1) {
  if constexpr (OPB == 4) {
    (void)x1;
    return to_tf32(x0);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);  // .x = x0 (low half), .y = x1
    return *reinterpret_cast<const uint32_t *>(&h);
  }
}

// D (TMEM, 128 lanes x 128 columns at tmem) (+)= A^T-form product over K = 128,
// issued by one thread: NMMA instructions of 32 bytes of K each.
template <int OPB>
__device__ __forceinline__ void tc_product(uint32_t tmem, const void *opA, const void *opB, bool accumulate) {
  using O = TcOp<OPB>;
  const uint32_t a0 = smem_addr(opA), b0 = smem_addr(opB);
#pragma unroll
  for (int kk = 0; kk < O::NMMA; ++kk) {
    const uint64_t ad = op_desc<OPB>(a0 + kk * 2 * O::LBO), bd = op_desc<OPB>(b0 + kk * 2 * O::LBO);
    const uint32_t acc = (accumulate || kk > 0) ? 1u : 0u;
    if constexpr (OPB == 4)
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(O::IDESC), "r"(acc));
    else
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(O::IDESC), "r"(acc));
  }
}

__device__ __forceinline__ void tc_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar)));
}

// Bounded wait for the MMAs of the given phase parity; false after kTcMaxPolls.
__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long polls = 0; !done && polls < kTcMaxPolls; ++polls) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return done != 0;
}

// Make the CTA's shared-memory stores visible to the tensor core, then barrier.
__device__ __forceinline__ void tc_publish_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

#define BTC_TMEM_LD32(r, taddr)                                                                                 \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"  \
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                       \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), \
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),       \
                 "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),      \
                 "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),      \
                 "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                          \
               : "r"(taddr))

// Accumulator rows of this thread: warp w reads TMEM lanes 32 (w % 4) .. + 31
// (row i = 32 (w % 4) + lane) and the column half 64 (w / 4) .. + 63 (8 warps).
// f(i, j0, v[32]) receives 32 consecutive columns j0 .. j0+31 of row i.
template <class F>
__device__ __forceinline__ void tc_read_rows(uint32_t tmem_acc, F &&f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2;
  const int i = 32 * q + lane;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int j0 = 64 * h + 32 * c;
    uint32_t r[32];
    BTC_TMEM_LD32(r, tmem_acc + ((uint32_t)(32 * q) << 16) + (uint32_t)j0);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float v[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
    f(i, j0, v);
  }
}

// Pool block (row-major 128 x 128 FP32 with row stride ldg, X[k][m]) -> K-major
// operand (A(m, k) = X[k][m]). Each warp writes whole 128-byte core matrices:
// lane -> (m = m0 + lane/4, k = k0 + (lane%4) * EPL), EPL = 4 / OPB elements
// packed in one 32-bit word.
template <int NT, int OPB>
__device__ __forceinline__ void stage_operand_from_pool(unsigned char *op, const float *g, int ldg = kTcNP) {
  using O = TcOp<OPB>;
  constexpr int EPL = 4 / OPB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32, KCM = kTcNP / O::CK, NCM = (kTcNP / 8) * KCM;  // core matrices
  const int dm = lane >> 2, dk = (lane & 3) * EPL;
#pragma unroll 4
  for (int cm = warp; cm < NCM; cm += NW) {
    const int m0 = (cm / KCM) * 8, k0 = (cm % KCM) * O::CK;
    const float x0 = __ldcg(g + (size_t)(k0 + dk) * ldg + m0 + dm);
    const float x1 = EPL == 2 ? __ldcg(g + (size_t)(k0 + dk + 1) * ldg + m0 + dm) : 0.0f;
    *reinterpret_cast<uint32_t *>(op + op_off<OPB>(m0 + dm, k0 + dk)) = pack_operand<OPB>(x0, x1);
  }
}

// Padded row-major shared block (X[k][m], leading dimension LD) -> K-major
// operand in the same buffer: every thread first reads its elements, then all
// write after a barrier.
template <int NT, int LD, int OPB>
__device__ __forceinline__ void convert_operand_in_place(float *buf) {
  using O = TcOp<OPB>;
  constexpr int EPL = 4 / OPB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = NT / 32, KCM = kTcNP / O::CK, NCM = (kTcNP / 8) * KCM;
  constexpr int PER = NCM / NW;  // core matrices per warp
  const int dm = lane >> 2, dk = (lane & 3) * EPL;
  uint32_t v[PER];
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int cm = warp + t * NW;
    const int m0 = (cm / KCM) * 8, k0 = (cm % KCM) * O::CK;
    v[t] = pack_operand<OPB>(buf[(k0 + dk) * LD + m0 + dm], EPL == 2 ? buf[(k0 + dk + 1) * LD + m0 + dm] : 0.0f);
  }
  __syncthreads();
  unsigned char *op = reinterpret_cast<unsigned char *>(buf);
#pragma unroll
  for (int t = 0; t < PER; ++t) {
    const int cm = warp + t * NW;
    const int m0 = (cm / KCM) * 8, k0 = (cm % KCM) * O::CK;
    *reinterpret_cast<uint32_t *>(op + op_off<OPB>(m0 + dm, k0 + dk)) = v[t];
  }
}

// Per-CTA tensor-core state of the node kernel: TMEM base (two accumulators at
// columns 0 and 128), the MMA completion barrier and its phase, and the
// barrier that counts the bytes of the bulk (TMA) block copies.
struct TcState {
  uint32_t tmem;
  uint64_t *mbar;
  uint32_t phase;
  uint64_t *tma_mbar;
  uint32_t tma_phase;
  int *status;  // set to kFlowTimeout when a wait gives up
};

// Allocation by warp 0 (all lanes), barrier init by thread 0; call with all threads.
__device__ __forceinline__ void tc_begin(TcState &st, uint32_t *tmem_slot, uint64_t *mbar, int *status) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar + 1)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  st.tmem = *tmem_slot;
  st.mbar = mbar;
  st.phase = 0;
  st.tma_mbar = mbar + 1;
  st.tma_phase = 0;
  st.status = status;
}

// Bulk-async (TMA engine) copies of up to three 128 x 128 FP32 pool blocks
// into padded shared rows (one 512-byte copy per row, issued by the CTA's last
// warp, so that warp 0 can start the Cholesky panel at once); the
// bytes complete on st.tma_mbar. Call with all threads; complete with
// tc_bulk_wait. The proxy fences order the copies after this CTA's earlier
// shared-memory accesses and after the acquire of the blocks' producers.
__device__ __forceinline__ void tc_bulk_load(TcState &st, float *d0, const float *g0, float *d1, const float *g1,
                                             float *d2, const float *g2) {
  constexpr int LD = TileCfg<float, kTcNP, 8>::LD;
  constexpr uint32_t row_bytes = kTcNP * sizeof(float);
  if ((threadIdx.x >> 5) != (blockDim.x >> 5) - 1) return;
  const int lane = threadIdx.x & 31;
  const uint32_t nblk = (d0 ? 1u : 0u) + (d1 ? 1u : 0u) + (d2 ? 1u : 0u);
  if (lane == 0) {
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(st.tma_mbar)),
                 "r"(nblk * row_bytes * kTcNP)
                 : "memory");
  }
  __syncwarp();
  float *dst[3] = {d0, d1, d2};
  const float *src[3] = {g0, g1, g2};
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    if (!dst[b]) continue;
    for (int r = lane; r < kTcNP; r += 32)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(dst[b] + r * LD)),
          "l"(src[b] + (size_t)r * kTcNP), "r"(row_bytes), "r"(smem_addr(st.tma_mbar))
          : "memory");
  }
}

// Bounded wait (all threads) for the bulk copies of the current phase.
__device__ __forceinline__ void tc_bulk_wait(TcState &st) {
  uint32_t done = 0;
  for (long long polls = 0; !done && polls < kTcMaxPolls; ++polls) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(st.tma_mbar)), "r"(st.tma_phase)
        : "memory");
  }
  st.tma_phase ^= 1u;
  if (!done && threadIdx.x == 0 && st.status) atomicExch(st.status, kFlowTimeout);
}

__device__ __forceinline__ void tc_end(TcState &st) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(st.tmem), "r"(kTcCols));
}

// Wait for the MMAs committed in the current phase; records a timeout.
__device__ __forceinline__ void tc_sync(TcState &st) {
  const bool ok = tc_wait(st.mbar, st.phase);
  st.phase ^= 1u;
  if (!ok && threadIdx.x == 0 && st.status) atomicExch(st.status, kFlowTimeout);
}

// One node of Alg. 5 with block size 128 (T = P = float, S = caller's type).
// Same inputs, outputs and pool conventions as factor_node (btc_factor.cuh).
template <typename S, bool FIRST, int OPB>
__device__ __forceinline__ void factor_node_tc(const FactorItem &it, const FactorArgs &args, const InstDesc &single,
                                               unsigned char *smem_raw, TcState &st) {
  using C = TileCfg<float, kTcNP, 8>;
  constexpr int NT = C::NT, LD = C::LD;
  float *sS = reinterpret_cast<float *>(smem_raw);  // S_e -> U_e (row-major, padded)
  float *sA = sS + C::BLK;                          // P_a operand, then S(e,e-s) -> U(e,e-s) -> operand
  float *sB = sA + C::BLK;                          // P_b operand, then S(e,e+s) -> U(e,e+s) -> operand
  float *dinv = sB + C::BLK;
  float *dpool = reinterpret_cast<float *>(args.dpool);
  float *epool = reinterpret_cast<float *>(args.epool);
  const int tid = threadIdx.x;
  unsigned long long *info = args.info + it.inst;
  const InstDesc ins = args.inst ? args.inst[it.inst] : single;
  const int e = it.node;
  const S *uD = reinterpret_cast<const S *>(ins.D);
  const S *uB = reinterpret_cast<const S *>(ins.B);
  const size_t ubs = (size_t)ins.n * ins.n;
  const bool has_up = it.r_up >= 0, has_dn = it.r_down >= 0, has_next = it.d_next >= 0;
  const uint32_t acc_fill = st.tmem, acc_next = st.tmem + 128;
  bool next_started = false;  // acc_next holds P_b^T P_b

  if constexpr (FIRST) {
    user_to_smem<C>(sS, uD + e * ubs, ins.n, true, 1.0f);                      // S[i][j] = D_e[j][i]
    if (has_up) user_to_smem<C>(sA, uB + (e - 1) * ubs, ins.n, false, 0.0f);  // S(e, e-1) = B_{e-1}
    if (has_dn) user_to_smem<C>(sB, uB + e * ubs, ins.n, true, 0.0f);         // S(e, e+1) = B_e^T
    __syncthreads();
  } else {
    const bool pa = it.p_a >= 0, pb = it.p_b >= 0 && has_next;
    tc_bulk_load(st, sS, dpool + it.d_self, nullptr, nullptr, nullptr, nullptr);
    if (pa) stage_operand_from_pool<NT, OPB>(reinterpret_cast<unsigned char *>(sA), epool + it.p_a);
    if (pb) stage_operand_from_pool<NT, OPB>(reinterpret_cast<unsigned char *>(sB), epool + it.p_b);
    tc_bulk_wait(st);
    tc_publish_smem();
    if (pa || pb) {
      if (tid == 0) {
        if (pa) tc_product<OPB>(acc_fill, sA, sA, false);  // P_a^T P_a
        if (pb) tc_product<OPB>(acc_next, sB, sB, false);  // P_b^T P_b, kept for S_{e+s}
        tc_commit(st.mbar);
      }
      tc_sync(st);
      next_started = pb;
      if (pa)  // S_e -= P_a^T P_a (rows of this thread, 64 columns)
        tc_read_rows(acc_fill, [&](int i, int j0, const float (&v)[32]) {
#pragma unroll
          for (int t = 0; t < 32; t += 4) {
            float4 s = *reinterpret_cast<float4 *>(sS + i * LD + j0 + t);
            s.x -= v[t];
            s.y -= v[t + 1];
            s.z -= v[t + 2];
            s.w -= v[t + 3];
            *reinterpret_cast<float4 *>(sS + i * LD + j0 + t) = s;
          }
        });
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
    }
    // the off-diagonal operands arrive (bulk copies) while the Cholesky runs
    if (has_up || has_dn)
      tc_bulk_load(st, has_up ? sA : nullptr, has_up ? epool + it.r_up : nullptr, has_dn ? sB : nullptr,
                   has_dn ? epool + it.r_down : nullptr, nullptr, nullptr);
  }

  // ---- potrf with the two trsm, pipelined by panels (FP32 FMA)
  const bool bulk = !FIRST && (has_up || has_dn);
  block_potrf_trsm<C>(sS, dinv, has_up ? sA : nullptr, has_dn ? sB : nullptr, info, e, [&] {
    if (bulk) tc_bulk_wait(st);
  });
  smem_to_block<C>(dpool + it.d_self, sS, true);
  if (has_up) smem_to_block<C>(epool + it.r_up, sA, false);
  if (has_dn) smem_to_block<C>(epool + it.r_down, sB, false);

  // ---- S_{e+s} -= U_dn^T U_dn and the fill, on the tensor cores
  const bool fill = it.fill >= 0;
  if (!(has_next || fill)) return;
  __syncthreads();
  if (has_dn) convert_operand_in_place<NT, LD, OPB>(sB);
  if (fill) convert_operand_in_place<NT, LD, OPB>(sA);
  tc_publish_smem();
  if (tid == 0) {
    if (has_next) tc_product<OPB>(acc_next, sB, sB, next_started);
    if (fill) {
      if (it.flags & FI_FILL_UPFIRST) tc_product<OPB>(acc_fill, sA, sB, false);  // S'(e-s, e+s) = -U_up^T U_dn
      else tc_product<OPB>(acc_fill, sB, sA, false);                             // S'(e+s, e-s) = -U_dn^T U_up
    }
    tc_commit(st.mbar);
  }
  tc_sync(st);
  if (has_next) {
    float *g = dpool + it.d_next;
    tc_read_rows(acc_next, [&](int i, int j0, const float (&v)[32]) {
#pragma unroll
      for (int t = 0; t < 32; t += 4) {
        const int j = j0 + t;
        float4 s;
        if constexpr (FIRST) {  // S_{e+1} = D_{e+1} (upper form of the caller's lower triangle), padded
          const S *Dn = uD + (e + 1) * ubs;
          float w[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int jj = j + u;
            w[u] = (i < ins.n && jj < ins.n) ? convert_in<float, S>(i <= jj ? Dn[(size_t)jj * ins.n + i]
                                                                           : Dn[(size_t)i * ins.n + jj])
                                             : (i == jj ? 1.0f : 0.0f);
          }
          s = make_float4(w[0], w[1], w[2], w[3]);
        } else {
          s = __ldcg(reinterpret_cast<const float4 *>(g + (size_t)i * kTcNP + j));
        }
        s.x -= v[t];
        s.y -= v[t + 1];
        s.z -= v[t + 2];
        s.w -= v[t + 3];
        *reinterpret_cast<float4 *>(g + (size_t)i * kTcNP + j) = s;
      }
    });
  }
  if (fill) {
    float *g = epool + it.fill;
    tc_read_rows(acc_fill, [&](int i, int j0, const float (&v)[32]) {
#pragma unroll
      for (int t = 0; t < 32; t += 4)
        *reinterpret_cast<float4 *>(g + (size_t)i * kTcNP + j0 + t) =
            make_float4(-v[t], -v[t + 1], -v[t + 2], -v[t + 3]);
    });
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// ---------------------------------------------------------------- kernels
// The tensor-core counterparts of k_factor_level, k_factor_flow and
// k_factor_fwd_flow (same arguments and schedules); each CTA holds its TMEM
// accumulators for its whole lifetime (one CTA per SM: the three 128 x 128
// FP32 shared blocks take 198 KB).
constexpr int kTcThreads = TileCfg<float, kTcNP, 8>::NT;

template <typename S, bool FIRST, int OPB>
__global__ void __launch_bounds__(kTcThreads, 1) k_factor_level_tc(FactorArgs args, InstDesc single) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  TcState st;
  tc_begin(st, &s_tmem, s_mbar, args.status);
  const FactorItem it = args.items[blockIdx.x];
  factor_node_tc<S, FIRST, OPB>(it, args, single, smem_raw, st);
  tc_end(st);
}

template <typename S, int OPB>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_factor_flow_tc(FactorArgs args, InstDesc single, const int32_t *deps, int nfirst, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  TcState st;
  tc_begin(st, &s_tmem, s_mbar, fs.status);
  for (;;) {
    const int t = flow_claim(fs, args.count, &s_slot);
    if (t < 0) break;
    const FactorItem it = args.items[t];
    flow_trace(fs, t, 0);
    if (flow_wait(fs, deps + 3 * t, 3, &s_ok)) {
      flow_trace(fs, t, 1);
      if (t < nfirst) factor_node_tc<S, true, OPB>(it, args, single, smem_raw, st);
      else factor_node_tc<S, false, OPB>(it, args, single, smem_raw, st);
    }
    __syncthreads();
    flow_trace(fs, t, 2);
    flow_publish(fs, t);
  }
  tc_end(st);
}

template <typename S, int OPB>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_factor_fwd_flow_tc(FactorArgs fa, InstDesc single, SolveArgs sa, const int32_t *code, const int32_t *deps,
                         int nfirst, int count, FlowSync fs) {
  grid_dep_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_slot, s_ok;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar[2];
  TcState st;
  tc_begin(st, &s_tmem, s_mbar, fs.status);
  const SolveFlowItem *fwd = reinterpret_cast<const SolveFlowItem *>(sa.items);
  for (;;) {
    const int t = flow_claim(fs, count, &s_slot);
    if (t < 0) break;
    const int c = code[t];
    flow_trace(fs, t, 0);
    if (flow_wait(fs, deps + (size_t)kInterDeps * t, kInterDeps, &s_ok)) {
      flow_trace(fs, t, 1);
      if (c >= 0) {
        const FactorItem it = fa.items[c];
        if (c < nfirst) factor_node_tc<S, true, OPB>(it, fa, single, smem_raw, st);
        else factor_node_tc<S, false, OPB>(it, fa, single, smem_raw, st);
      } else {
        const SolveFlowItem it = fwd[-1 - c];
        fwd_node<float, kTcNP>(it.y_self, it.y_a, it.e_a, it.y_b, it.e_b, it.d_self, sa, smem_raw);
      }
    }
    __syncthreads();
    flow_trace(fs, t, 2);
    flow_publish(fs, t);
  }
  tc_end(st);
}

}  // namespace btc
