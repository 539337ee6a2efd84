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
// One CTA owns a 128-row tile, a block of at most 128 of the NB columns and a
// slice of K (split-K, atomic epilogue). Per 32-wide K tile TMA brings the
// operand tiles into 128-byte-swizzled shared memory and one thread issues
// 3 x 4 tcgen05.mma.kind::tf32 (M = 128, N = block width, K = 8) into a TMEM
// accumulator; the partial product of each K tile is read back and summed in
// registers with round-to-nearest float32 additions (see the kernel). Every
// mbarrier wait is bounded; on timeout the CTA records an error flag, waits
// (bounded) for its own copies and MMAs, and returns its TMEM.
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

// Roles (256 threads): warps 0-3 own TMEM lanes 32w..32w+31 (one output row per
// thread) and keep the running float32 sums of their row in registers; warp 4
// lane 0 issues the TMA loads of a ring of stages; warp 5 lane 0 issues the MMAs.
//
// The tensor core adds the products of an MMA into its float32 accumulator
// without rounding to nearest, so a long chain of MMAs into one accumulator
// drifts (a 7680-column block with 96 K tiles per accumulator chain measured
// 1.0e-5 relative, 25 times the float32 floor). Here every K tile (3 products
// x 4 steps of K = 8) starts a fresh accumulator; the four row warps read it
// with tcgen05.ld and add it to their register sums with ordinary
// round-to-nearest additions, while the MMAs of the next tiles go into the
// other accumulators of a ring of up to four. The chain in TMEM is thus 12 MMAs
// long whatever K is.
//
// A is loaded as float32 into the "h" slot of a stage, and two more warps
// (6, 7) round it to TF32 in place and write the low parts beside it before
// the MMA warp may use the stage, so the operator crosses HBM once, as
// float32, and needs no split copy. MODE 0: B is loaded and split the same
// way. MODE 1: B = Bh + Bl is split beforehand (the vectors are small and
// reused by every row block) and the producer loads both parts.
constexpr int MAX_STAGES = 3;  // stages of the ring (a deeper ring measured no faster)
constexpr int ROW_THREADS = 128;
constexpr int SPLIT_THREADS = 64;  // two warps: eight in all, two per SM sub-partition (register file)
constexpr int GEMM_THREADS = ROW_THREADS + 64 + SPLIT_THREADS;
constexpr int MAX_BN = 128;   // columns per CTA: 128 float32 sums per row thread
constexpr int MAX_ACC = 4;

struct __align__(8) Bars {
  uint64_t full[MAX_STAGES];    // TMA bytes of the stage landed
  uint64_t ready[MAX_STAGES];   // in-kernel split of the stage done (split warps)
  uint64_t empty[MAX_STAGES];   // MMAs reading the stage completed
  uint64_t accf[MAX_ACC];   // accumulator holds a finished K tile
  uint64_t acce[MAX_ACC];   // accumulator read out by the four row warps
  uint32_t tmem_base;
  uint32_t fail;
  int32_t issued;           // K tiles whose loads were issued
  int32_t committed;        // K tiles whose MMAs were committed
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool failed(Bars* b) { return *(volatile uint32_t*)&b->fail != 0; }

template <int MODE>
__global__ void __launch_bounds__(GEMM_THREADS, 1) gemm_tf32x3_kernel(
    const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapBh,
    const __grid_constant__ CUtensorMap mapBl, float* __restrict__ Z,
    int64_t M, int NB, int BN, int64_t K, int ktiles_per_cta, int stages, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int a_bytes = BM * BK * 4, b_bytes = BN * BK * 4;
  const int stage_bytes = 2 * (a_bytes + b_bytes);
  Bars* bars = reinterpret_cast<Bars*>(base + stages * stage_bytes);
  auto Ah = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes); };
  auto Al = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + a_bytes); };
  auto Bh = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + 2 * a_bytes); };
  auto Bl = [&](int s) { return reinterpret_cast<float*>(base + s * stage_bytes + 2 * a_bytes + b_bytes); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const int col0 = blockIdx.z * BN;  // first column of this CTA's column block
  const int64_t ktotal = (K + BK - 1) / BK;
  const int64_t kt0 = (int64_t)blockIdx.y * ktiles_per_cta;
  const int64_t nk_full = ktotal - kt0 < (int64_t)ktiles_per_cta ? ktotal - kt0 : (int64_t)ktiles_per_cta;
  const int nk = nk_full > 0 ? (int)nk_full : 0;
  if (nk == 0) return;
  int acc_cols = 32;
  while (acc_cols < BN) acc_cols <<= 1;
  const int nacc = min(MAX_ACC, 512 / acc_cols);  // 4 for BN <= 128
  const int tmem_cols = acc_cols * nacc;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->ready[s], SPLIT_THREADS);
      mbar_init(&bars->empty[s], 1);
    }
    for (int a = 0; a < MAX_ACC; ++a) {
      mbar_init(&bars->accf[a], 1);
      mbar_init(&bars->acce[a], ROW_THREADS);
    }
    bars->fail = 0;
    bars->issued = 0;
    bars->committed = 0;
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

  float acc[MAX_BN];
#pragma unroll
  for (int q = 0; q < MAX_BN; ++q) acc[q] = 0.f;

  if (warp == 4) {
    if (lane == 0) {
      // producer: stage s is free again once the MMAs of the tile that last used it completed
      const unsigned tx = (unsigned)(a_bytes + (MODE == 0 ? 1 : 2) * b_bytes);
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % stages;
        if (kt >= stages && !mbar_wait(&bars->empty[s], ((kt / stages) - 1) & 1)) {
          atomicOr(&bars->fail, 1u);
          break;
        }
        if (failed(bars)) break;
        const int x = (int)((kt0 + kt) * BK);
        mbar_expect_tx(&bars->full[s], tx);
        tma_load_2d(Ah(s), &mapA, &bars->full[s], x, (int)row0);
        tma_load_2d(Bh(s), &mapBh, &bars->full[s], x, col0);
        if (MODE == 1) tma_load_2d(Bl(s), &mapBl, &bars->full[s], x, col0);
        *(volatile int32_t*)&bars->issued = kt + 1;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(BN);
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % stages, a = kt % nacc, use = kt / nacc;
        if (!mbar_wait(&bars->ready[s], (kt / stages) & 1) || (use >= 1 && !mbar_wait(&bars->acce[a], (use - 1) & 1))) {
          atomicOr(&bars->fail, 1u);
          break;
        }
        if (failed(bars)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t tacc = tmem + (uint32_t)(a * acc_cols);
#pragma unroll
        for (int k8 = 0; k8 < BK / 8; ++k8) {
          const uint64_t a_h = smem_desc(Ah(s) + 8 * k8), b_h = smem_desc(Bh(s) + 8 * k8);
          const uint64_t a_l = smem_desc(Al(s) + 8 * k8), b_l = smem_desc(Bl(s) + 8 * k8);
          mma_tf32(tacc, a_h, b_h, idesc, k8 == 0 ? 0u : 1u);  // a fresh accumulator per K tile
          mma_tf32(tacc, a_h, b_l, idesc, 1u);
          mma_tf32(tacc, a_l, b_h, idesc, 1u);
        }
        mma_commit(&bars->empty[s]);
        mma_commit(&bars->accf[a]);
        *(volatile int32_t*)&bars->committed = kt + 1;
      }
    }
  } else if (warp >= 6) {
    // split warps: round the stage's float32 tiles to TF32 in place (the low
    // parts beside them), vector by vector
    const int st_id = tid - (ROW_THREADS + 64);
    for (int kt = 0; kt < nk; ++kt) {
      const int s = kt % stages;
      if (!mbar_wait(&bars->full[s], (kt / stages) & 1) || failed(bars)) {
        atomicOr(&bars->fail, 1u);
        break;
      }
      float4* ah = reinterpret_cast<float4*>(Ah(s));
      float4* al = reinterpret_cast<float4*>(Al(s));
#pragma unroll 4
      for (int i = st_id; i < BM * BK / 4; i += SPLIT_THREADS) {
        const float4 x = ah[i];
        const float4 h = {tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w)};
        ah[i] = h;
        al[i] = {x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w};
      }
      if (MODE == 0) {
        float4* bh = reinterpret_cast<float4*>(Bh(s));
        float4* bl = reinterpret_cast<float4*>(Bl(s));
        for (int i = st_id; i < BN * BK / 4; i += SPLIT_THREADS) {
          const float4 x = bh[i];
          const float4 h = {tf32_round(x.x), tf32_round(x.y), tf32_round(x.z), tf32_round(x.w)};
          bh[i] = h;
          bl[i] = {x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w};
        }
      }
      // the generic-proxy writes must be visible to the tensor core's reads
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&bars->ready[s]);
    }
  } else {
    // row warps: read out the accumulator of each tile and add it to the
    // register sums
    auto drain = [&](int kt) -> bool {
      const int a = kt % nacc;
      // warp-uniform outcome: tcgen05.ld below is a warp-collective instruction
      if (!__all_sync(0xffffffffu, mbar_wait(&bars->accf[a], (kt / nacc) & 1))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c0 = 0; c0 < MAX_BN; c0 += 32) {
        if (c0 < BN) {
          uint32_t v[32];
          const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * acc_cols + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[c0 + q] += __uint_as_float(v[q]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&bars->acce[a]);
      return true;
    };
    bool ok = true;
    for (int kt = 0; kt < nk && ok; ++kt) {
      if (kt >= 1 && !drain(kt - 1)) ok = false;
      if (__any_sync(0xffffffffu, failed(bars))) ok = false;
    }
    if (ok && !drain(nk - 1)) ok = false;
    if (!ok) atomicOr(&bars->fail, 1u);
  }
  __syncthreads();
  if (!failed(bars)) {
    if (warp < 4) {
      const int64_t row = row0 + warp * 32 + lane;
      if (row < M) {
        float* zr = Z + row * NB + col0;
#pragma unroll
        for (int q = 0; q < MAX_BN; ++q)
          if (q < BN && col0 + q < NB) atomicAdd(zr + q, acc[q]);
      }
    }
  } else if (tid == 0) {
    atomicOr(err, 1);
    // bounded drains, so that neither a copy nor an MMA lands after the exit:
    // the loads that were issued, and the last committed MMA group (its commit
    // covers every earlier MMA of this thread)
    const int issued = bars->issued;
    for (int kt = (issued > stages ? issued - stages : 0); kt < issued; ++kt)
      mbar_wait(&bars->full[kt % stages], (kt / stages) & 1);
    const int committed = bars->committed;
    if (committed > 0) mbar_wait(&bars->empty[(committed - 1) % stages], ((committed - 1) / stages) & 1);
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

// Launch shape of one product: column blocks of at most MAX_BN columns, and
// the number of K slices (split-K) that minimises the makespan
// waves x (K tiles per slice + a fixed per-CTA cost) at one CTA per SM.
struct GemmPlan {
  int BN, nz, per;
  int64_t mt, split;
};

GemmPlan plan_gemm(int64_t M, int64_t K, int NB, int n_sm) {
  GemmPlan p;
  p.BN = NB <= MAX_BN ? NB : 16 * ((NB + 31) / 32);
  p.nz = (NB + p.BN - 1) / p.BN;
  p.mt = (M + BM - 1) / BM;
  const int64_t ktotal = (K + BK - 1) / BK;
  const int64_t base = p.mt * p.nz;
  const int64_t sm = std::max(1, n_sm);
  int64_t best_split = 1, best_cost = INT64_MAX;
  const int64_t max_split = std::min<int64_t>(ktotal, std::max<int64_t>(1, 8 * sm / base + 1));
  for (int64_t sp = 1; sp <= max_split; ++sp) {
    const int64_t per = (ktotal + sp - 1) / sp, used = (ktotal + per - 1) / per;
    const int64_t waves = (base * used + sm - 1) / sm;
    const int64_t cost = waves * (per + 8);
    if (cost < best_cost) { best_cost = cost; best_split = used; }
  }
  p.per = (int)((ktotal + best_split - 1) / best_split);
  p.split = (ktotal + p.per - 1) / p.per;
  return p;
}

template <int MODE>
int launch_gemm(const CUtensorMap& mA, const CUtensorMap& mBh, const CUtensorMap& mBl, const GemmPlan& p, int64_t M, int64_t K, int NB, float* Z, int* d_err, cudaStream_t st) {
  const int stage_bytes = 2 * (BM * BK * 4 + p.BN * BK * 4);
  const int stages = std::min(MAX_STAGES, (227 * 1024 - (int)sizeof(Bars) - 1024) / stage_bytes);
  if (stages < 2) return fail(CAL_EINVAL, "gemm: %d columns do not fit the pipeline", p.BN);
  const int smem = stages * stage_bytes + (int)sizeof(Bars) + 1024;
  if (int rc = ensure_dyn_smem((const void*)gemm_tf32x3_kernel<MODE>, smem)) return rc;
  CAL_TRY_CUDA(cudaMemsetAsync(Z, 0, (size_t)M * NB * sizeof(float), st));
  const int tok = prof_begin(st, "gemm_tc", 2.0 * 3.0 * (double)M * K * NB);
  gemm_tf32x3_kernel<MODE><<<dim3((unsigned)p.mt, (unsigned)p.split, (unsigned)p.nz), GEMM_THREADS, smem, st>>>(
      mA, mBh, mBl, Z, M, NB, p.BN, K, p.per, stages, d_err);
  prof_end(st, tok);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

}  // namespace

bool gemm_tc_supported(int64_t cols, int nrhs) {
  // rows of the real [rows][2 cols] view must start on 16-byte boundaries, and
  // 4 real columns per right-hand side (two halves, re/im) must fit one tile
  return (cols % 2 == 0) && nrhs >= 1 && 4 * nrhs <= 256;
}

// Z[M][NB] = A[M][K] Bt[NB][K]^T (Z is zeroed here), float32 via 3xTF32 with
// the split into TF32 parts done in the kernel
int gemm_tf32x3(const float* A, int64_t M, int64_t K, const float* Bt, int NB, float* Z, int* d_err,
                int n_sm, cudaStream_t st) {
  if (NB < 16 || NB > 256 || NB % 16) return fail(CAL_EINVAL, "gemm: NB must be a multiple of 16 in [16, 256]");
  if ((uintptr_t)A % 16 || (uintptr_t)Bt % 16 || (K * 4) % 16) return fail(CAL_EINVAL, "gemm: operands not 16-byte aligned");
  const GemmPlan p = plan_gemm(M, K, NB, n_sm);
  CUtensorMap mA, mB;
  int rc;
  if ((rc = make_map(&mA, A, K, M, BM)) || (rc = make_map(&mB, Bt, K, NB, p.BN))) return rc;
  return launch_gemm<0>(mA, mB, mB, p, M, K, NB, Z, d_err, st);
}

int split_tf32(const float* x, float* hi, float* lo, int64_t n, cudaStream_t st) {
  if (n <= 0) return CAL_OK;
  split_tf32_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, hi, lo, n);
  note_launch();
  CAL_TRY_CUDA(cudaGetLastError());
  return CAL_OK;
}

// Z[M][NB] = A[M][K] (Bh + Bl)[NB][K]^T (Z is zeroed here), 3xTF32 with A split
// in the kernel and B split beforehand: A crosses HBM once, as float32
int gemm_tf32x3_bsplit(const float* A, int64_t M, int64_t K, const float* Bh, const float* Bl, int NB, float* Z,
                       int* d_err, int n_sm, cudaStream_t st) {
  if (NB < 16 || NB > 256 || NB % 16) return fail(CAL_EINVAL, "gemm: NB must be a multiple of 16 in [16, 256]");
  for (const float* p : {A, Bh, Bl})
    if ((uintptr_t)p % 16) return fail(CAL_EINVAL, "gemm: operands not 16-byte aligned");
  if ((K * 4) % 16) return fail(CAL_EINVAL, "gemm: rows not 16-byte aligned");
  const GemmPlan p = plan_gemm(M, K, NB, n_sm);
  CUtensorMap mA, mBh, mBl;
  int rc;
  if ((rc = make_map(&mA, A, K, M, BM)) || (rc = make_map(&mBh, Bh, K, NB, p.BN)) || (rc = make_map(&mBl, Bl, K, NB, p.BN)))
    return rc;
  return launch_gemm<1>(mA, mBh, mBl, p, M, K, NB, Z, d_err, st);
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
                    cudaStream_t st) {
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
  float* Bs = nullptr;  // the vectors' TF32 parts: [2][NB][2 cols]
  if (!rc) {
    if (cudaMallocAsync((void**)&Bs, (size_t)2 * NB * 2 * cols * sizeof(float), st) != cudaSuccess)
      rc = fail(CAL_ENOMEM, "multi-vector product: cannot allocate the split vectors");
    else
      rc = split_tf32(Bt, Bs, Bs + (size_t)NB * 2 * cols, (int64_t)NB * 2 * cols, st);
  }
  if (!rc)
    rc = gemm_tf32x3_bsplit(reinterpret_cast<const float*>(Xop), rows, 2 * cols, Bs, Bs + (size_t)NB * 2 * cols, NB,
                            Z, err, n_sm, st);
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
