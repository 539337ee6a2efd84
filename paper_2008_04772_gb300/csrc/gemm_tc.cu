// A10: multi-right-hand-side product on the 5th-generation tensor cores.
//
// Z[M][NB] += A[M][K] * Bt[NB][K]^T in float32 by the 3xTF32 split
// (A = Ah + Al, B = Bh + Bl with Ah, Bh the TF32 parts, Z ~ AhBh + AhBl + AlBh),
// which keeps float32 accuracy. A complex64 operator block read as a real
// [rows][2 cols] matrix and the real embedding of the right-hand sides
//   Bt[2j][2c] = Re X(c,j), Bt[2j][2c+1] = -Im X(c,j),
//   Bt[2j+1][2c] = Im X(c,j), Bt[2j+1][2c+1] = Re X(c,j)
// give Z[r][2j] = Re (A X)(r,j), Z[r][2j+1] = Im (A X)(r,j).
//
// One CTA of 128 threads owns a 128-row tile, all NB (<= 256) columns and a
// slice of K (split-K, atomic epilogue). Per 32-wide K tile: TMA brings the
// float32 A and Bt tiles into 128-byte-swizzled shared memory, the threads
// round them to TF32 in place and write the low parts next to them, one thread issues 3 x 4
// tcgen05.mma.kind::tf32 (M = 128, N = NB, K = 8) into a TMEM accumulator and
// commits to an mbarrier that releases the stage. Two stages in flight.
// Every mbarrier wait is bounded; on timeout the CTA records an error flag,
// waits (bounded) for its own copies and returns its TMEM.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace cal {

namespace {

constexpr int BM = 128;          // rows per CTA (TMEM lanes)
constexpr int BK = 32;           // float32 per K tile = 128 bytes = one swizzle row
constexpr int STAGES = 2;
constexpr int THREADS = 128;
constexpr unsigned long long WAIT_LIMIT = 1ull << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// bounded wait on the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const uint32_t a = smem_u32(bar);
  for (unsigned long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;                  // start address
  d |= (uint64_t)(16 >> 4) << 16;                // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// instruction descriptor: D float32, A and B TF32, both K-major, N x M
__device__ __forceinline__ uint32_t instr_desc(int n) {
  uint32_t d = 0;
  d |= 1u << 4;                    // D format: float32
  d |= 2u << 7;                    // A format: TF32
  d |= 2u << 10;                   // B format: TF32
  d |= (uint32_t)(n >> 3) << 17;   // N / 8
  d |= (uint32_t)(BM >> 4) << 24;  // M / 16
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// split x = hi + lo with hi the nearest TF32 value (the tensor core reads the
// top 19 bits of each 32-bit operand, so hi is taken exactly) and lo = x - hi,
// exact in float32 and itself read to TF32 precision: |error| <= 2^-21 |x|
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct __align__(8) Bars {
  uint64_t full[STAGES];
  uint64_t done[STAGES];
  uint32_t tmem_base;
  uint32_t fail;
};

__global__ void __launch_bounds__(THREADS, 1) gemm_tf32x3_kernel(
    const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, float* __restrict__ Z,
    int64_t M, int NB, int BN, int64_t K, int ktiles_per_cta, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned tiles: per stage Ah [BM][BK], Bh [BN][BK], Al, Bl
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = BM * BK * 4, b_bytes = BN * BK * 4;
  const int stage_bytes = 2 * (a_bytes + b_bytes);
  Bars* bars = reinterpret_cast<Bars*>(base + STAGES * stage_bytes);
  auto Ah = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes); };
  auto Bh = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + a_bytes); };
  auto Al = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + a_bytes + b_bytes); };
  auto Bl = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + 2 * a_bytes + b_bytes); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t ktotal = (K + BK - 1) / BK;
  const int64_t kt0 = (int64_t)blockIdx.y * ktiles_per_cta;
  const int64_t nk_full = ktotal - kt0 < (int64_t)ktiles_per_cta ? ktotal - kt0 : (int64_t)ktiles_per_cta;
  const int nk = nk_full > 0 ? (int)nk_full : 0;
  if (nk == 0) return;
  int acc_cols = 32;
  while (acc_cols < BN) acc_cols <<= 1;
  // up to 4 accumulators taking the K tiles in turn (at most 256 TMEM columns,
  // so that two CTAs share an SM): the tensor core adds each MMA step into its
  // float32 accumulator without a round-to-nearest, so the error grows with the
  // chain length; the epilogue adds the partial sums
  const int nacc_max = min(4, 256 / acc_cols) > 1 ? min(4, 256 / acc_cols) : 1;
  const int nacc = nacc_max < nk ? nacc_max : nk;
  const int tmem_cols = acc_cols * (nacc <= 1 ? 1 : (nacc <= 2 ? 2 : 4));

  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->done[s], 1);
    }
    bars->fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bars->tmem_base;
  const uint32_t idesc = instr_desc(BN);
  const unsigned tx_bytes = (unsigned)(a_bytes + b_bytes);

  bool ok = true;
  if (tid == 0) {
    mbar_expect_tx(&bars->full[0], tx_bytes);
    tma_load_2d(Ah(0), &mapA, &bars->full[0], (int)(kt0 * BK), (int)row0);
    tma_load_2d(Bh(0), &mapB, &bars->full[0], (int)(kt0 * BK), 0);
  }
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (tid == 0 && kt + 1 < nk) {
      // stage s^1 is free once the MMAs of tile kt-1 have completed
      if (kt >= 1 && !mbar_wait(&bars->done[s ^ 1], ((kt - 1) >> 1) & 1)) atomicOr(&bars->fail, 1u);
      mbar_expect_tx(&bars->full[s ^ 1], tx_bytes);
      tma_load_2d(Ah(s ^ 1), &mapA, &bars->full[s ^ 1], (int)((kt0 + kt + 1) * BK), (int)row0);
      tma_load_2d(Bh(s ^ 1), &mapB, &bars->full[s ^ 1], (int)((kt0 + kt + 1) * BK), 0);
    }
    if (!mbar_wait(&bars->full[s], (kt >> 1) & 1)) atomicOr(&bars->fail, 1u);
    __syncthreads();
    if (bars->fail) { ok = false; break; }
    // hi (rounded to TF32 in place) and lo parts, same swizzled positions
    float* ah = Ah(s);
    float* bh = Bh(s);
    float* al = Al(s);
    float* bl = Bl(s);
    for (int i = tid; i < BM * BK; i += THREADS) {
      const float x = ah[i], h = tf32_round(x);
      ah[i] = h;
      al[i] = x - h;
    }
    for (int i = tid; i < BN * BK; i += THREADS) {
      const float x = bh[i], h = tf32_round(x);
      bh[i] = h;
      bl[i] = x - h;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      const uint32_t tacc = tmem + (uint32_t)((kt % nacc) * acc_cols);
      for (int k8 = 0; k8 < BK / 8; ++k8) {
        const uint64_t a_h = smem_desc(Ah(s) + 8 * k8), b_h = smem_desc(Bh(s) + 8 * k8);
        const uint64_t a_l = smem_desc(Al(s) + 8 * k8), b_l = smem_desc(Bl(s) + 8 * k8);
        const uint32_t first = (kt < nacc && k8 == 0) ? 0u : 1u;
        mma_tf32(tacc, a_h, b_h, idesc, first);
        mma_tf32(tacc, a_h, b_l, idesc, 1u);
        mma_tf32(tacc, a_l, b_h, idesc, 1u);
      }
      mma_commit(&bars->done[s]);
    }
  }
  // wait for the last MMAs (their commit also covers all earlier ones)
  if (tid == 0 && ok) {
    if (!mbar_wait(&bars->done[(nk - 1) & 1], ((nk - 1) >> 1) & 1)) atomicOr(&bars->fail, 1u);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!bars->fail) {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 (rows), 32 columns per load
    const int64_t row = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float sum[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) sum[q] = 0.f;
      for (int a = 0; a < nacc; ++a) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * acc_cols + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 32; ++q) sum[q] += __uint_as_float(v[q]);
      }
      if (row < M) {
        float* zr = Z + row * NB + c0;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (c0 + q < NB) atomicAdd(zr + q, sum[q]);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
    // bounded drain of copies that may still be in flight
    for (int s = 0; s < STAGES; ++s) mbar_wait(&bars->full[s], 0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------------------
// The same product with both operands split beforehand (A = Ah + Al stored
// once per operator, B = Bh + Bl per call), so no thread touches a tile: one
// thread issues the TMA loads of a ring of stages, one thread issues the MMAs
// (3 per K step into up to 4 round-robin accumulators) and commits each stage
// back to the producer, and all warps run the epilogue. STAGES_S stages of
// (Ah, Al, Bh, Bl) tiles are in flight.
// ---------------------------------------------------------------------------
constexpr int STAGES_S = 3;

struct __align__(8) BarsS {
  uint64_t full[STAGES_S];
  uint64_t empty[STAGES_S];
  uint32_t tmem_base;
  uint32_t fail;
  int32_t issued;  // K tiles whose loads were issued
};

__global__ void __launch_bounds__(THREADS, 1) gemm_tf32x3_split_kernel(
    const __grid_constant__ CUtensorMap mapAh, const __grid_constant__ CUtensorMap mapAl,
    const __grid_constant__ CUtensorMap mapBh, const __grid_constant__ CUtensorMap mapBl, float* __restrict__ Z,
    int64_t M, int NB, int BN, int64_t K, int ktiles_per_cta, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = BM * BK * 4, b_bytes = BN * BK * 4;
  const int stage_bytes = 2 * (a_bytes + b_bytes);
  BarsS* bars = reinterpret_cast<BarsS*>(base + STAGES_S * stage_bytes);
  auto Ah = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes); };
  auto Al = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + a_bytes); };
  auto Bh = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + 2 * a_bytes); };
  auto Bl = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + 2 * a_bytes + b_bytes); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int64_t ktotal = (K + BK - 1) / BK;
  const int64_t kt0 = (int64_t)blockIdx.y * ktiles_per_cta;
  const int64_t nk_full = ktotal - kt0 < (int64_t)ktiles_per_cta ? ktotal - kt0 : (int64_t)ktiles_per_cta;
  const int nk = nk_full > 0 ? (int)nk_full : 0;
  if (nk == 0) return;
  int acc_cols = 32;
  while (acc_cols < BN) acc_cols <<= 1;
  const int nacc_max = min(4, 512 / acc_cols) > 1 ? min(4, 512 / acc_cols) : 1;
  const int nacc = nacc_max < nk ? nacc_max : nk;
  const int tmem_cols = acc_cols * (nacc <= 1 ? 1 : (nacc <= 2 ? 2 : 4));

  if (tid == 0) {
    for (int s = 0; s < STAGES_S; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->empty[s], 1);
    }
    bars->fail = 0;
    bars->issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bars->tmem_base;
  const uint32_t idesc = instr_desc(BN);
  const unsigned tx_bytes = (unsigned)(2 * (a_bytes + b_bytes));

  if (tid == 0) {
    // producer: stage s is free again once the MMAs of the tile that last used it completed
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES_S;
      if (kt >= STAGES_S && !mbar_wait(&bars->empty[s], ((kt / STAGES_S) - 1) & 1)) {
        atomicOr(&bars->fail, 1u);
        break;
      }
      if (*(volatile uint32_t*)&bars->fail) break;
      const int x = (int)((kt0 + kt) * BK);
      mbar_expect_tx(&bars->full[s], tx_bytes);
      tma_load_2d(Ah(s), &mapAh, &bars->full[s], x, (int)row0);
      tma_load_2d(Al(s), &mapAl, &bars->full[s], x, (int)row0);
      tma_load_2d(Bh(s), &mapBh, &bars->full[s], x, 0);
      tma_load_2d(Bl(s), &mapBl, &bars->full[s], x, 0);
      *(volatile int32_t*)&bars->issued = kt + 1;
    }
  } else if (tid == 32) {
    // MMA issuer
    int last = -1;  // last tile whose MMAs were committed
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % STAGES_S;
      if (!mbar_wait(&bars->full[s], (kt / STAGES_S) & 1)) {
        atomicOr(&bars->fail, 1u);
        break;
      }
      if (*(volatile uint32_t*)&bars->fail) break;
      last = kt;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tacc = tmem + (uint32_t)((kt % nacc) * acc_cols);
#pragma unroll
      for (int k8 = 0; k8 < BK / 8; ++k8) {
        const uint64_t a_h = smem_desc(Ah(s) + 8 * k8), b_h = smem_desc(Bh(s) + 8 * k8);
        const uint64_t a_l = smem_desc(Al(s) + 8 * k8), b_l = smem_desc(Bl(s) + 8 * k8);
        const uint32_t first = (kt < nacc && k8 == 0) ? 0u : 1u;
        mma_tf32(tacc, a_h, b_h, idesc, first);
        mma_tf32(tacc, a_h, b_l, idesc, 1u);
        mma_tf32(tacc, a_l, b_h, idesc, 1u);
      }
      mma_commit(&bars->empty[s]);
    }
    // the commit of the last issued tile covers every earlier MMA; wait for it
    // (bounded) also after a failure, before the TMEM is returned
    if (last >= 0 && !mbar_wait(&bars->empty[last % STAGES_S], (last / STAGES_S) & 1)) atomicOr(&bars->fail, 1u);
    if (last != nk - 1) atomicOr(&bars->fail, 1u);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!bars->fail) {
    const int64_t row = row0 + warp * 32 + lane;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float sum[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) sum[q] = 0.f;
      for (int a = 0; a < nacc; ++a) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * acc_cols + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 32; ++q) sum[q] += __uint_as_float(v[q]);
      }
      if (row < M) {
        float* zr = Z + row * NB + c0;
#pragma unroll
        for (int q = 0; q < 32; ++q)
          if (c0 + q < NB) atomicAdd(zr + q, sum[q]);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
    // bounded drain of the loads that were issued, so no copy lands after exit
    const int issued = bars->issued;
    for (int kt = (issued > STAGES_S ? issued - STAGES_S : 0); kt < issued; ++kt)
      mbar_wait(&bars->full[kt % STAGES_S], (kt / STAGES_S) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

__global__ void split_tf32_kernel(const float* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo,
                                  int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = x[i], h = tf32_round(v);
    hi[i] = h;
    lo[i] = v - h;
  }
}

// real embedding of the right-hand sides of one block (see the file header):
// X is complex [nrhs][n2] (component-major halves of length n_total), the block
// reads columns [col_off, col_off + ncols) of both halves. Output Bt is
// [NB][K] float32 with K = 2 ncols and NB = 8 nrhs (x1 and x2 halves).
template <typename VT>
__global__ void embed_rhs_kernel(const VT* __restrict__ X, int nrhs, int64_t n_total, int64_t col_off,
                                 int64_t ncols, float* __restrict__ Bt, int NB) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;  // complex column: (rhs q, half h) -> j = 2 q + h
  if (c >= ncols) return;
  const int K = (int)(2 * ncols);
  if (j >= 2 * nrhs) {  // padding columns
    Bt[(int64_t)(2 * j) * K + 2 * c] = 0.f;
    Bt[(int64_t)(2 * j) * K + 2 * c + 1] = 0.f;
    Bt[(int64_t)(2 * j + 1) * K + 2 * c] = 0.f;
    Bt[(int64_t)(2 * j + 1) * K + 2 * c + 1] = 0.f;
    return;
  }
  const int q = j >> 1, h = j & 1;
  const VT x = X[(int64_t)q * 2 * n_total + h * n_total + col_off + c];
  const float re = (float)x.x, im = (float)x.y;
  Bt[(int64_t)(2 * j) * K + 2 * c] = re;
  Bt[(int64_t)(2 * j) * K + 2 * c + 1] = -im;
  Bt[(int64_t)(2 * j + 1) * K + 2 * c] = im;
  Bt[(int64_t)(2 * j + 1) * K + 2 * c + 1] = re;
}

// y1 += ZC(x1) + alpha ZS(x2), y2 += ZC(x2) + beta ZS(x1) for every right-hand side
template <typename VT>
__global__ void combine_rhs_kernel(const float* __restrict__ ZS, const float* __restrict__ ZC, int64_t rows,
                                   int NB, int nrhs, int64_t n_total, int64_t row_off, VT* __restrict__ Y,
                                   double ar, double ai, double br, double bi) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (r >= rows) return;
  auto cz = [&](const float* Zp, int h) {
    if (!Zp) return double2{0.0, 0.0};
    const int j = 2 * q + h;
    return double2{Zp[r * NB + 2 * j], Zp[r * NB + 2 * j + 1]};
  };
  const double2 c1 = cz(ZC, 0), c2 = cz(ZC, 1), s1 = cz(ZS, 0), s2 = cz(ZS, 1);
  VT* y1 = Y + (int64_t)q * 2 * n_total + row_off + r;
  VT* y2 = y1 + n_total;
  VT a = *y1, b = *y2;
  a.x += c1.x + ar * s2.x - ai * s2.y;
  a.y += c1.y + ar * s2.y + ai * s2.x;
  b.x += c2.x + br * s1.x - bi * s1.y;
  b.y += c2.y + br * s1.y + bi * s1.x;
  *y1 = a;
  *y2 = b;
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  });
  return fn;
}

int make_map(CUtensorMap* map, const float* ptr, int64_t inner, int64_t outer, int box_outer) {
  EncodeFn enc = encode_fn();
  if (!enc) return fail(CAL_ECUDA, "tensor map encoder unavailable");
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_outer};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(ptr), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CAL_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return CAL_OK;
}

}  // namespace

bool gemm_tc_supported(int64_t cols, int nrhs) {
  // rows of the real [rows][2 cols] view must start on 16-byte boundaries, and
  // 4 real columns per right-hand side (two halves, re/im) must fit one tile
  return (cols % 2 == 0) && nrhs >= 1 && 4 * nrhs <= 256;
}

// Z[M][NB] = A[M][K] Bt[NB][K]^T (Z is zeroed here), float32 via 3xTF32
int gemm_tf32x3(const float* A, int64_t M, int64_t K, const float* Bt, int NB, float* Z, int* d_err,
                int n_sm, cudaStream_t st) {
  if (NB < 16 || NB > 256 || NB % 16) return fail(CAL_EINVAL, "gemm: NB must be a multiple of 16 in [16, 256]");
  if ((uintptr_t)A % 16 || (uintptr_t)Bt % 16 || (K * 4) % 16) return fail(CAL_EINVAL, "gemm: operands not 16-byte aligned");
  CUtensorMap mA, mB;
  int rc;
  if ((rc = make_map(&mA, A, K, M, BM))) return rc;
  if ((rc = make_map(&mB, Bt, K, NB, NB))) return rc;
  CAL_TRY_CUDA(cudaMemsetAsync(Z, 0, (size_t)M * NB * sizeof(float), st));
  const int64_t mt = (M + BM - 1) / BM;
  const int64_t ktotal = (K + BK - 1) / BK;
  int64_t split = std::max<int64_t>(1, std::min<int64_t>(ktotal, (2 * (int64_t)n_sm + mt - 1) / mt));
  const int per = (int)((ktotal + split - 1) / split);
  split = (ktotal + per - 1) / per;
  const int smem = STAGES * 2 * (BM * BK * 4 + NB * BK * 4) + (int)sizeof(Bars) + 1024;
  if (int rc = ensure_dyn_smem((const void*)gemm_tf32x3_kernel, smem)) return rc;
  const int tok = prof_begin(st, "gemm_tc", 2.0 * 3.0 * (double)M * K * NB);
  gemm_tf32x3_kernel<<<dim3((unsigned)mt, (unsigned)split), THREADS, smem, st>>>(mA, mB, Z, M, NB, NB, K, per, d_err);
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

int split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n <= 0) return CAL_OK;
  split_tf32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, hi, lo, n);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// Z[M][NB] = (Ah + Al)[M][K] (Bh + Bl)[NB][K]^T (Z is zeroed here), 3xTF32
int gemm_tf32x3_split(const float* Ah, const float* Al, int64_t M, int64_t K, const float* Bh, const float* Bl, int NB,
                      float* Z, int* d_err, int n_sm, cudaStream_t st) {
  if (NB < 16 || NB > 256 || NB % 16) return fail(CAL_EINVAL, "gemm: NB must be a multiple of 16 in [16, 256]");
  for (const float* p : {Ah, Al, Bh, Bl})
    if ((uintptr_t)p % 16) return fail(CAL_EINVAL, "gemm: operands not 16-byte aligned");
  if ((K * 4) % 16) return fail(CAL_EINVAL, "gemm: rows not 16-byte aligned");
  CUtensorMap mAh, mAl, mBh, mBl;
  int rc;
  if ((rc = make_map(&mAh, Ah, K, M, BM)) || (rc = make_map(&mAl, Al, K, M, BM)) ||
      (rc = make_map(&mBh, Bh, K, NB, NB)) || (rc = make_map(&mBl, Bl, K, NB, NB)))
    return rc;
  CAL_TRY_CUDA(cudaMemsetAsync(Z, 0, (size_t)M * NB * sizeof(float), st));
  const int64_t mt = (M + BM - 1) / BM;
  const int64_t ktotal = (K + BK - 1) / BK;
  const int smem = STAGES_S * 2 * (BM * BK * 4 + NB * BK * 4) + (int)sizeof(BarsS) + 1024;
  if (smem > 227 * 1024) return fail(CAL_EINVAL, "gemm: %d columns do not fit the split-operand pipeline", NB);
  if (int rc2 = ensure_dyn_smem((const void*)gemm_tf32x3_split_kernel, smem)) return rc2;
  // one CTA per SM; about two waves of (row tile, K slice) units
  int64_t split = std::max<int64_t>(1, std::min<int64_t>(ktotal, (2 * (int64_t)n_sm + mt - 1) / mt));
  const int per = (int)((ktotal + split - 1) / split);
  split = (ktotal + per - 1) / per;
  const int tok = prof_begin(st, "gemm_tc", 2.0 * 3.0 * (double)M * K * NB);
  gemm_tf32x3_split_kernel<<<dim3((unsigned)mt, (unsigned)split), THREADS, smem, st>>>(mAh, mAl, mBh, mBl, Z, M, NB,
                                                                                      NB, K, per, d_err);
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

template <typename VT>
int embed_rhs(const VT* X, int nrhs, int64_t n_total, int64_t col_off, int64_t ncols, float* Bt, int NB,
              cudaStream_t st) {
  dim3 grid((unsigned)((ncols + 255) / 256), NB / 2);
  embed_rhs_kernel<VT><<<grid, 256, 0, st>>>(X, nrhs, n_total, col_off, ncols, Bt, NB);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

template <typename VT>
int combine_rhs(const float* ZS, const float* ZC, int64_t rows, int NB, int nrhs, int64_t n_total, int64_t row_off,
                VT* Y, double ar, double ai, double br, double bi, cudaStream_t st) {
  dim3 grid((unsigned)((rows + 255) / 256), nrhs);
  combine_rhs_kernel<VT><<<grid, 256, 0, st>>>(ZS, ZC, rows, NB, nrhs, n_total, row_off, Y, ar, ai, br, bi);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// y[j][r] = Z[r][2j] + i Z[r][2j+1] for j < ncol (plain multi-vector product)
__global__ void unembed_kernel(const float* __restrict__ Z, int64_t rows, int NB, int ncol, float2* __restrict__ y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r < rows && j < ncol) y[(int64_t)j * rows + r] = make_float2(Z[r * NB + 2 * j], Z[r * NB + 2 * j + 1]);
}

// Y[nrhs][rows] = X^T applied: plain complex product of a float32 dense operator
// with nrhs vectors x [nrhs][cols] through the tensor-core path
int multi_matvec_tc(const float2* Xop, int64_t rows, int64_t cols, const float2* x, float2* y, int nrhs, int n_sm,
                    cudaStream_t st, const float* Xh, const float* Xl) {
  const int npair = (nrhs + 1) / 2;  // the embedding works on (x1, x2) column pairs
  const int NB = ((4 * npair + 15) / 16) * 16;
  if (NB > 256 || cols % 2) return fail(CAL_EINVAL, "multi-vector product: unsupported size");
  float *Bt, *Z;
  int* err;
  float2* xp = nullptr;
  CAL_TRY_CUDA(cudaMallocAsync((void**)&Bt, (size_t)NB * 2 * cols * sizeof(float), st));
  CAL_TRY_CUDA(cudaMallocAsync((void**)&Z, (size_t)rows * NB * sizeof(float), st));
  CAL_TRY_CUDA(cudaMallocAsync((void**)&err, sizeof(int), st));
  CAL_TRY_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const float2* xin = x;
  if (nrhs % 2) {  // pad to an even number of vectors
    CAL_TRY_CUDA(cudaMallocAsync((void**)&xp, (size_t)(nrhs + 1) * cols * sizeof(float2), st));
    CAL_TRY_CUDA(cudaMemsetAsync(xp, 0, (size_t)(nrhs + 1) * cols * sizeof(float2), st));
    CAL_TRY_CUDA(cudaMemcpyAsync(xp, x, (size_t)nrhs * cols * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    xin = xp;
  }
  int rc = embed_rhs<float2>(xin, npair, cols, 0, cols, Bt, NB, st);
  float* Bs = nullptr;  // split operand: [2][NB][2 cols]
  const bool split = Xh && Xl && NB <= 128;
  if (!rc && split) {
    if (cudaMallocAsync((void**)&Bs, (size_t)2 * NB * 2 * cols * sizeof(float), st) != cudaSuccess)
      rc = fail(CAL_ENOMEM, "multi-vector product: cannot allocate the split operand");
    else
      rc = split_tf32(Bt, Bs, Bs + (size_t)NB * 2 * cols, (int64_t)NB * 2 * cols, st);
  }
  if (!rc)
    rc = split ? gemm_tf32x3_split(Xh, Xl, rows, 2 * cols, Bs, Bs + (size_t)NB * 2 * cols, NB, Z, err, n_sm, st)
               : gemm_tf32x3(reinterpret_cast<const float*>(Xop), rows, 2 * cols, Bt, NB, Z, err, n_sm, st);
  if (!rc) {
    unembed_kernel<<<dim3((unsigned)((rows + 255) / 256), nrhs), 256, 0, st>>>(Z, rows, NB, nrhs, y);
    note_launch();
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  cudaFreeAsync(Bt, st);
  if (Bs) cudaFreeAsync(Bs, st);
  cudaFreeAsync(Z, st);
  cudaFreeAsync(err, st);
  if (xp) cudaFreeAsync(xp, st);
  if (!rc && herr) rc = fail(CAL_ETIMEOUT, "tensor-core product: a bounded wait gave up");
  CAL_TRY_CUDA(cudaGetLastError());
  return rc;
}

template int embed_rhs<float2>(const float2*, int, int64_t, int64_t, int64_t, float*, int, cudaStream_t);
template int embed_rhs<double2>(const double2*, int, int64_t, int64_t, int64_t, float*, int, cudaStream_t);
template int combine_rhs<float2>(const float*, const float*, int64_t, int, int, int64_t, int64_t, float2*, double,
                                 double, double, double, cudaStream_t);
template int combine_rhs<double2>(const float*, const float*, int64_t, int, int, int64_t, int64_t, double2*, double,
                                  double, double, double, cudaStream_t);

}  // namespace cal
