// Tensor-core (tcgen05, sm_103a) bfloat16 GEMMs of the inverse chain
// (Alg. 2, ChainProduct, "2d matrix multiplications" of Sec. 3.1):
//
//  * square: S~_{i+1} = S~_i S~_i for the symmetric bf16 level S~_i. Only the
//    256 x 256 blocks (I, J) with I <= J are computed (two 128 x 256 MMA
//    tiles each); every block is also written transposed, so the stored
//    level is exactly symmetric. Output bf16 (float32 accumulation).
//  * apply: partial[s] = M [x_hi | x_lo] over the k-range of split s for a
//    bf16 matrix M (a chain level, or a bf16 half of the graph for the
//    residual update), where x_hi + x_lo is a float32 block of right-hand
//    sides split into two bfloat16 halves (about 16 significant bits). Output
//    float32 partials.
//
// Structure: persistent CTAs (one per SM), warp-specialised. Warp 0 issues TMA
// loads of 128-byte-swizzled K-major tiles into a 4-stage shared-memory ring;
// warp 1 (one thread) issues tcgen05.mma (M = 128, N <= 256, K = 16) into one
// of two TMEM accumulators; warps 2-5 drain the other accumulator with
// tcgen05.ld and store to global memory. Every mbarrier wait is bounded: on
// expiry the CTA records DEV_WAIT_TIMEOUT in the status word and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ff.cuh"
#include "internal.h"

namespace cdl {
namespace {

constexpr int BM = 128;           // MMA M = TMEM lanes
constexpr int BK = 64;            // bf16 per 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int MAX_BN = 256;
constexpr int A_TILE = BM * BK * 2;          // 16 KiB
constexpr int B_TILE = MAX_BN * BK * 2;      // 32 KiB
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int BAR_BYTES = 256;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + BAR_BYTES + 1024;
constexpr int THREADS = 192;
constexpr int PACE_KB = 32;                          // k-blocks per pacing step (2048 of K)
constexpr int PACE_SLACK = 2;                        // steps a CTA may run ahead of the slowest
constexpr int PACE_MIN_KBLOCKS = 1024;               // paced from K = 65536 on
constexpr unsigned long long PACE_WAIT_NS = 200000;  // a wait longer than this ends the CTA's pacing
constexpr int TMEM_COLS = 512;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;   // 2 s per wait

enum { MODE_SQUARE = 0, MODE_APPLY = 1, MODE_SQUARE_FP8 = 2 };



struct TcParams {
  const uint32_t* tiles;   // packed tile descriptors
  int num_tiles;
  int kblocks;             // 64-wide k-blocks per tile
  int bn;                  // MMA N (multiple of 16, <= 256)
  uint32_t idesc;          // tcgen05 instruction descriptor
  int mode;
  int npad;                // matrix order
  void* out;               // square: bf16 level (npad x npad); apply: float partials
  int ldo;                 // apply: partial row stride (= bn)
  unsigned* status;
  // fp8 squaring: level value = amax/448 * stored value; amax[level] of the
  // input, amax[level + 1] of the output (float bits); out16 = bf16 copy
  const unsigned* amax;
  int level;
  void* out16;
  int debug_withhold_load;   // test hook: never issue the first A load (its wait must expire)
  const TcGroup* groups;     // grouped launch: per-graph maps/outputs (nullptr otherwise)
  int gate_mask;             // grouped: a graph's tiles run iff *gate & gate_mask (or gate is null)
  // K pacing (long k loops): the producer of every CTA counts its arrival at
  // each step of PACE_KB k-blocks in pace[step] and does not start step s
  // before all CTAs have reached step s - PACE_SLACK (bounded wait; null: off)
  unsigned* pace;
  int pace_steps;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok;
}
// Bounded wait. Returns false (after flagging) if the phase did not complete
// within WAIT_LIMIT_NS or another role of this CTA already gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          unsigned* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > WAIT_LIMIT_NS) {
      *abort_flag = 1;
      atomicOr(status, DEV_WAIT_TIMEOUT);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// The same load with an L2 eviction policy (createpolicy), for operands that
// many CTAs read again later and should outlive streamed data in L2.
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset
  d |= (uint64_t)1 << 46;                          // version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_fp8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-level scale of an fp8 level from its bound amax (float bits): the level
// holds value / scale with scale = amax / 448 (448 = largest finite e4m3).
__device__ __forceinline__ float fp8_scale(unsigned amax_bits) {
  const float a = __uint_as_float(amax_bits);
  return a > 0.f ? a * (1.0f / 448.0f) : 1.0f;
}

// Tile descriptors. square: I (bits 0-14), J (bits 15-29), half (bit 30).
// apply: row block m (bits 0-15), split s (bits 16-31). bke = elements per
// 128-byte k-block (64 bf16 or 128 fp8). Grouped launches carry the graph g in
// bits 0-15; grouped squaring then I (16-22), J (23-29), half (30); grouped
// apply the row block m (16-30), without split-K.
__device__ __forceinline__ void decode(const TcParams& p, uint32_t t, int bke, int& a_row, int& b_row,
                                       int& k0, int& I, int& J, int& split, int& g) {
  if (p.groups) {
    g = t & 0xFFFF;
    split = 0;
    k0 = 0;
    if (p.mode == MODE_APPLY) {
      I = (t >> 16) & 0x7FFF;
      J = 0;
      a_row = I * 128;
      b_row = 0;
    } else if (p.groups[g].bn == 128) {   // 128-blocks: I (16-23), J (24-31)
      I = (t >> 16) & 0xFF;
      J = (t >> 24) & 0xFF;
      a_row = I * 128;
      b_row = J * 128;
    } else {
      I = (t >> 16) & 0x7F;
      J = (t >> 23) & 0x7F;
      a_row = I * 256 + ((t >> 30) & 1) * 128;
      b_row = J * 256;
    }
    return;
  }
  g = -1;
  if (p.mode != MODE_APPLY) {
    I = t & 0x7FFF;
    J = (t >> 15) & 0x7FFF;
    const int half = (t >> 30) & 1;
    a_row = I * 256 + half * 128;
    b_row = J * 256;
    k0 = 0;
    split = 0;
  } else {
    const int m = t & 0xFFFF;
    split = (t >> 16) & 0xFFFF;
    a_row = m * 128;
    b_row = 0;
    k0 = split * p.kblocks * bke;
    I = m;
    J = 0;
  }
}

// Grouped launches: a tile runs unless its graph's gate word masks it out.
// Every role of the CTA evaluates this for the same tile and sees the same
// value (the gate is written by an earlier launch).
__device__ __forceinline__ bool tile_runs(const TcParams& p, uint32_t t) {
  if (!p.groups) return true;
  const int* gate = p.groups[t & 0xFFFF].gate;
  return gate == nullptr || (*gate & p.gate_mask) != 0;
}

template <bool FP8>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const TcParams p) {
  constexpr int BKE = FP8 ? 128 : 64;   // elements per 128-byte k-block
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  // bars[0..3] full, [4..7] empty, [8..9] tmem full, [10..11] tmem empty, [12] drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 16);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 17);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 128);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t b_bytes = (uint32_t)p.bn * BK * 2;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    // K pacing: the CTAs sweeping K over tiles that share row panels stay
    // within a few steps of each other, so a panel's k-blocks are read from
    // DRAM once and served from L2 to the other CTAs (without it, CTAs drift
    // apart over long k loops and each streams its panels from DRAM)
    bool pacing = p.pace != nullptr;
    const int steps_per_tile = (p.kblocks + PACE_KB - 1) / PACE_KB;
    int lt = 0;   // tiles this CTA has started
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x) {
      const uint32_t td = p.tiles[t];
      if (!tile_runs(p, td)) continue;
      int a_row, b_row, k0, I, J, split, g;
      decode(p, td, BKE, a_row, b_row, k0, I, J, split, g);
      const CUtensorMap* ma = &tmA;
      const CUtensorMap* mb = &tmB;
      int kblocks = p.kblocks;
      uint32_t tile_b_bytes = b_bytes;
      if (p.groups) {
        const TcGroup& gd = p.groups[g];
        ma = &gd.mapA;
        mb = &gd.mapB;
        kblocks = gd.kblocks;
        tile_b_bytes = (uint32_t)gd.bn * BK * 2;
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ma))
                     : "memory");
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mb))
                     : "memory");
      }
      for (int kb = 0; kb < kblocks; ++kb, ++it) {
        if (p.pace && kb % PACE_KB == 0) {
          const int step = lt * steps_per_tile + kb / PACE_KB;
          if (step < p.pace_steps) atomicAdd(p.pace + step, 1u);
          if (pacing && step >= PACE_SLACK && step - PACE_SLACK < p.pace_steps) {
            const unsigned* c = p.pace + step - PACE_SLACK;
            const unsigned long long t0 = globaltimer();
            unsigned v;
            for (;;) {
              asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
              if (v >= gridDim.x) break;
              if (globaltimer() - t0 > PACE_WAIT_NS) {   // a CTA not resident or stalled: stop pacing
                pacing = false;
                break;
              }
            }
          }
        }
        const int s = it % STAGES;
        const uint32_t r = (uint32_t)(it / STAGES);
        if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t a_dst = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b_dst = a_dst + A_TILE;
        mbar_expect_tx(full_bar(s), A_TILE + tile_b_bytes);
        if (!(p.debug_withhold_load && it == 0)) tma_load_2d(a_dst, ma, k0 + kb * BKE, a_row, full_bar(s));
        tma_load_2d(b_dst, mb, k0 + kb * BKE, b_row, full_bar(s));
      }
      ++lt;
    }
    if (p.pace)   // arrive at the steps this CTA has no tile for, so no CTA waits on it
      for (int step = lt * steps_per_tile; step < p.pace_steps; ++step) atomicAdd(p.pace + step, 1u);
    if (!ok) {
      // let copies already issued land before the CTA exits (bounded)
      for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full_bar(j % STAGES), (uint32_t)(j / STAGES) & 1) &&
               globaltimer() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer
    int it = 0, tc = 0;
    bool ok = true, issued = false;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x) {
      const uint32_t td = p.tiles[t];
      if (!tile_runs(p, td)) continue;
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(tempty_bar(acc), (ar & 1) ^ 1, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * MAX_BN);
      int kblocks = p.kblocks;
      uint32_t idesc = p.idesc;
      if (p.groups) {
        kblocks = p.groups[td & 0xFFFF].kblocks;
        idesc = p.groups[td & 0xFFFF].idesc;
      }
      for (int kb = 0; kb < kblocks; ++kb, ++it) {
        const int s = it % STAGES;
        const uint32_t r = (uint32_t)(it / STAGES);
        if (!mbar_wait(full_bar(s), r & 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(smem + s * STAGE_BYTES);
        const uint64_t adesc = smem_desc(a_addr);
        const uint64_t bdesc = smem_desc(a_addr + A_TILE);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          // advance 32 bytes (16 bf16 or 32 fp8) along K inside the swizzle atom
          if constexpr (FP8)
            mma_fp8(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (kb | kk) != 0);
          else
            mma_bf16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), idesc, (kb | kk) != 0);
        }
        issued = true;
        mma_commit(empty_bar(s));
      }
      if (!ok) break;
      mma_commit(tfull_bar(acc));
    }
    if (!ok && issued) {
      mma_commit(drain_bar);   // wait (bounded) for MMAs in flight
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue
    const int q = warp & 3;                 // TMEM lane quarter of this warp
    const int row_in_tile = q * 32 + lane;
    int tc = 0;
    for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x) {
      const uint32_t td = p.tiles[t];
      if (!tile_runs(p, td)) continue;
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(tfull_bar(acc), ar & 1, abort_flag, p.status)) break;
      tc_fence_after();
      int a_row, b_row, k0, I, J, split, g;
      decode(p, td, BKE, a_row, b_row, k0, I, J, split, g);
      const int r = a_row + row_in_tile;
      void* out = p.out;
      int npad = p.npad;
      int bn = p.bn;
      if (p.groups) {
        out = p.groups[g].out;
        npad = p.groups[g].npad;
        bn = p.groups[g].bn;
      }
      const uint32_t taddr = tmem_base + (uint32_t)(acc * MAX_BN) + ((uint32_t)(q * 32) << 16);
      for (int c = 0; c < bn / 32; ++c) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(c * 32), v);
        if (p.mode == MODE_SQUARE) {
          __nv_bfloat16* C = static_cast<__nv_bfloat16*>(out);
          const int col0 = b_row + c * 32;
          if (I != J) {
            uint32_t packed[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
              packed[e] = *reinterpret_cast<uint32_t*>(&h);
            }
            uint4* dst = reinterpret_cast<uint4*>(C + (size_t)r * npad + col0);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              dst[e] = make_uint4(packed[4 * e], packed[4 * e + 1], packed[4 * e + 2], packed[4 * e + 3]);
#pragma unroll
            for (int e = 0; e < 32; ++e) C[(size_t)(col0 + e) * npad + r] = __float2bfloat16_rn(v[e]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int col = col0 + e;
              const __nv_bfloat16 h = __float2bfloat16_rn(v[e]);
              if (col >= r) C[(size_t)r * npad + col] = h;
              if (col > r) C[(size_t)col * npad + r] = h;
            }
          }
        } else if (p.mode == MODE_SQUARE_FP8) {
          // value = acc * s_in^2; fp8 level stores value / s_out, bf16 copy the value
          const float s_in = fp8_scale(p.amax[p.level]);
          const float sc = s_in * s_in;
          const float inv_out = 1.0f / fp8_scale(p.amax[p.level + 1]);
          uint8_t* C8 = static_cast<uint8_t*>(out);
          __nv_bfloat16* C16 = static_cast<__nv_bfloat16*>(p.out16);
          const int col0 = b_row + c * 32;
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] *= sc;
          uint8_t q8[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) q8[e] = (uint8_t)__nv_cvt_float_to_fp8(v[e] * inv_out, __NV_SATFINITE, __NV_E4M3);
          if (I != J) {
            uint32_t w8[8], packed[16];
#pragma unroll
            for (int e = 0; e < 8; ++e)
              w8[e] = (uint32_t)q8[4 * e] | ((uint32_t)q8[4 * e + 1] << 8) | ((uint32_t)q8[4 * e + 2] << 16) |
                      ((uint32_t)q8[4 * e + 3] << 24);
            uint4* d8 = reinterpret_cast<uint4*>(C8 + (size_t)r * npad + col0);
            d8[0] = make_uint4(w8[0], w8[1], w8[2], w8[3]);
            d8[1] = make_uint4(w8[4], w8[5], w8[6], w8[7]);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
              packed[e] = *reinterpret_cast<uint32_t*>(&h);
            }
            uint4* d16 = reinterpret_cast<uint4*>(C16 + (size_t)r * npad + col0);
#pragma unroll
            for (int e = 0; e < 4; ++e)
              d16[e] = make_uint4(packed[4 * e], packed[4 * e + 1], packed[4 * e + 2], packed[4 * e + 3]);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              C8[(size_t)(col0 + e) * npad + r] = q8[e];
              C16[(size_t)(col0 + e) * npad + r] = __float2bfloat16_rn(v[e]);
            }
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
              const int col = col0 + e;
              const __nv_bfloat16 h = __float2bfloat16_rn(v[e]);
              if (col >= r) {
                C8[(size_t)r * npad + col] = q8[e];
                C16[(size_t)r * npad + col] = h;
              }
              if (col > r) {
                C8[(size_t)col * npad + r] = q8[e];
                C16[(size_t)col * npad + r] = h;
              }
            }
          }
        } else {
          float* P = static_cast<float*>(out) + ((size_t)split * npad + r) * p.ldo + c * 32;
          float4* dst = reinterpret_cast<float4*>(P);
#pragma unroll
          for (int e = 0; e < 8; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
        }
      }
      tc_fence_before();
      mbar_arrive(tempty_bar(acc));
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}


// ---------------------------------------------------------------- 576-thread tensor-core kernels
// Shared by the e4m3 tile squaring (k_tc_mx8), the exact-slice residual, the
// distance and the score kernels: warp 0 TMA, warp 1 MMA, warps 2-17
// epilogue. The e4m3 squaring's stage: an A K tile of 128 rows and a B K
// tile of 256 rows, 128 e4m3 (128 bytes) each.
constexpr int T8_STAGES = 4;
constexpr int T8_A = 128 * 128;                       // A k-tile bytes
constexpr int T8_B = 256 * 128;                       // B k-tile bytes
constexpr int T8_STAGE_BYTES = T8_A + T8_B;
constexpr int T8_SMEM_BYTES = T8_STAGES * T8_STAGE_BYTES + 512 + 1024;
constexpr int T8_TMEM_COLS = 512;
constexpr int T8_THREADS = 576;   // warp 0 TMA, warp 1 MMA, warps 2-17 epilogue (four per TMEM lane quarter)
constexpr int T8_EPI = 512;       // epilogue threads
constexpr int T8_COLS = 64;       // output columns per epilogue thread


__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- exact-slice residual product
// A Z for the float64-class residual, on the bf16 tensor cores. A / 2^q (2^q
// the least power of two, q >= 0, not below max A: entries in [0, 1]) and
// Z / c (c a power of two per column with |Z / c| < 1) are written as sums of
// six bf16 slices on the fixed grids 2^-8s (signed base-256 digits of the
// values rounded to 2^-48: the leading digit at most 256 in magnitude, the
// others 128), so every slice product a_s z_t is exact in float32 (at most
// 2^16 grid steps) and lies on the grid 2^-8(s+t), and a float32 sum of 256
// of them (one K-chunk of one slice pair) is exact too (at most 2^24 grid
// steps). The MMA sums one K-chunk of one slice pair into a TMEM buffer; the
// epilogue converts it to an integer count of grid steps, adds it to int32
// accumulators, and every 64 chunks (at most 2^30 steps) adds them, scaled
// by 2^-8(s+t), to the float64 plane of its slice pair. The 21 slice pairs
// with s + t <= 7 leave about 2^-50 of |A| |Z / c|: A Z = 2^q c G with G
// the sum of the 21 planes in pair order, to float64 accuracy, as the
// ordering of the float64 additions allows. A CTA's unit of work is one
// 128-row tile with one slice pair over the whole K range, units numbered
// tile-major, so the pairs sharing an A slice tile run on neighbouring CTAs
// at the same time and read it from L2 (pair-major per CTA, each A slice
// would come from HBM once for every pair it is in: 21 / 6 times the bytes).
// Warp roles as in k_tc_mx8 (576 threads, 16 epilogue warps).
constexpr int RS_SLICES = 6;
constexpr int RS_MAX_PAIRS = 21;
constexpr int RS_STAGES = 6;
constexpr int RS_A = 128 * 128;                 // A k-block: 128 rows x 64 bf16
constexpr int RS_STAGE_BYTES = RS_A + 128 * 128; // + B k-block: up to 128 rows x 64 bf16
constexpr int RS_SMEM_BYTES = RS_STAGES * RS_STAGE_BYTES + 512 + 1024;
constexpr int RS_NBUF = 4;                       // ring of TMEM accumulators of up to 128 columns
constexpr int RS_TMEM_COLS = RS_NBUF * 128;
constexpr int RS_CHUNK_KB = 4;                   // k-blocks (of 64) per exact chunk: K = 256
constexpr int RS_FLUSH = 64;                     // chunks per int32 flush

struct ResidMaps {
  CUtensorMap a[RS_SLICES];   // slice planes of A, box 64 x 128 rows
  CUtensorMap b[RS_SLICES];   // slice planes of Z / c, transposed (kp x npad), box 64 x kp rows
};

struct ResidParams {
  int num_tiles;   // npad / 128 (grouped: entries of units)
  int kblocks;     // npad / 64
  int kp;          // MMA N (multiple of 32, <= 128)
  int npairs;
  int pair_s[RS_MAX_PAIRS];
  int pair_t[RS_MAX_PAIRS];
  double* G;       // npairs planes npad x kp (one per slice pair, gstride apart), zeroed before
  size_t gstride;
  uint32_t idesc;
  unsigned* status;
  const ResidGroup* groups;   // grouped launch: per-graph maps, planes, k loop, gate (null otherwise)
  const uint32_t* units;      // grouped: graph | row tile << 16
  int gate_mask;
  int assign;                 // the first flush of a unit stores instead of adding
};

// Unit u of a launch: its row tile, slice pair, operand maps, k loop and
// output planes, and whether it runs (grouped: its graph's gate).
struct ResidUnit {
  bool run;
  int t, pr, kblocks;
  const CUtensorMap* ma;
  const CUtensorMap* mb;
  double* G;
  size_t gstride;
};
__device__ __forceinline__ ResidUnit resid_unit(const ResidMaps& maps, const ResidParams& p, int u) {
  ResidUnit r;
  const int e = u / p.npairs;
  r.pr = u % p.npairs;
  const int sa = p.pair_s[r.pr] - 1, sz = p.pair_t[r.pr] - 1;
  if (p.groups) {
    const uint32_t ud = p.units[e];
    const ResidGroup& gr = p.groups[ud & 0xFFFF];
    r.run = gr.gate == nullptr || (*gr.gate & p.gate_mask) != 0;
    r.t = (int)(ud >> 16);
    r.kblocks = gr.kblocks;
    r.ma = &gr.a[sa];
    r.mb = &gr.b[sz];
    r.G = gr.G;
    r.gstride = gr.gstride;
  } else {
    r.run = true;
    r.t = e;
    r.kblocks = p.kblocks;
    r.ma = &maps.a[sa];
    r.mb = &maps.b[sz];
    r.G = p.G;
    r.gstride = p.gstride;
  }
  return r;
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 18 warps: an SM sub-partition holds five of them, so at most 96 registers
// per thread fit.
__global__ void __launch_bounds__(T8_THREADS, 1)
    k_tc_resid(const __grid_constant__ ResidMaps maps, const ResidParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + RS_STAGES * RS_STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * RS_STAGES + 2 * RS_NBUF + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * RS_STAGES + 2 * RS_NBUF + 3);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (RS_STAGES + s); };
  auto pfull_bar = [&](int b) { return bar0 + 8u * (2 * RS_STAGES + b); };
  auto pempty_bar = [&](int b) { return bar0 + 8u * (2 * RS_STAGES + RS_NBUF + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * RS_STAGES + 2 * RS_NBUF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t b_bytes = (uint32_t)p.kp * 128;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RS_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < RS_NBUF; ++b) {
      mbar_init(pfull_bar(b), 1);
      mbar_init(pempty_bar(b), T8_EPI);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(RS_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    const uint64_t zpol = l2_policy_evict_last();
    for (int u = blockIdx.x; u < p.num_tiles * p.npairs && ok; u += gridDim.x) {
      const ResidUnit ru = resid_unit(maps, p, u);
      if (!ru.run) continue;
      const int t = ru.t;
      {
        const CUtensorMap* ma = ru.ma;
        const CUtensorMap* mb = ru.mb;
        if (p.groups) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(ma))
                       : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mb))
                       : "memory");
        }
        for (int kb = 0; kb < ru.kblocks; ++kb, ++it) {
          const int s = it % RS_STAGES;
          const uint32_t r = (uint32_t)(it / RS_STAGES);
          if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
            ok = false;
            break;
          }
          const uint32_t a_dst = smem_u32(smem + s * RS_STAGE_BYTES);
          mbar_expect_tx(full_bar(s), RS_A + b_bytes);
          tma_load_2d(a_dst, ma, kb * 64, t * 128, full_bar(s));
          // every unit reads a whole Z slice: keep the Z slices in L2 while the A slices stream
          tma_load_2d_hint(a_dst + RS_A, mb, kb * 64, 0, full_bar(s), zpol);
        }
      }
    }
    if (!ok) {
      for (int j = (it > RS_STAGES ? it - RS_STAGES : 0); j < it; ++j) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full_bar(j % RS_STAGES), (uint32_t)(j / RS_STAGES) & 1) &&
               globaltimer() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer: one exact K-chunk per TMEM buffer
    int it = 0, pc = 0;
    bool ok = true, issued = false;
    for (int u = blockIdx.x; u < p.num_tiles * p.npairs && ok; u += gridDim.x) {
        const ResidUnit ru = resid_unit(maps, p, u);
        if (!ru.run) continue;
        const int nchunks = ru.kblocks / RS_CHUNK_KB;
        for (int c = 0; c < nchunks && ok; ++c, ++pc) {
          const int b = pc % RS_NBUF;
          const uint32_t ph = (uint32_t)(pc / RS_NBUF);
          if (!mbar_wait(pempty_bar(b), (ph & 1) ^ 1, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(b * 128);
          for (int kb = 0; kb < RS_CHUNK_KB; ++kb, ++it) {
            const int s = it % RS_STAGES;
            if (!mbar_wait(full_bar(s), (uint32_t)(it / RS_STAGES) & 1, abort_flag, p.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a_addr = smem_u32(smem + s * RS_STAGE_BYTES);
            const uint64_t adesc = smem_desc(a_addr);
            const uint64_t bdesc = smem_desc(a_addr + RS_A);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              mma_bf16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc, (kb | kk) != 0);
            issued = true;
            mma_commit(empty_bar(s));
          }
          if (!ok) break;
          mma_commit(pfull_bar(b));
        }
    }
    if (!ok && issued) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: exact chunk counts, int32 sums, float64 flushes
    const int q = warp & 3;
    const int part = (warp - 2) >> 2;                 // column quarter
    const int ncol = p.kp / 4;                        // columns of this warp (8, 16 or 32)
    const int col0 = part * ncol;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int pc = 0;
    bool failed = false;
    for (int u = blockIdx.x; u < p.num_tiles * p.npairs; u += gridDim.x) {
      const ResidUnit ru = resid_unit(maps, p, u);
      if (!ru.run) continue;
      const int t = ru.t, pr = ru.pr;
      const int nchunks = ru.kblocks / RS_CHUNK_KB;
      const int row = t * 128 + q * 32 + lane;
      double* Grow = ru.G + (size_t)pr * ru.gstride + (size_t)row * p.kp + col0;
      bool first_flush = p.assign != 0;
      {
        const int m = p.pair_s[pr] + p.pair_t[pr];
        const float up = __int_as_float((127 + 8 * m) << 23);   // 2^(8m)
        int acc[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = 0;
        for (int ch = 0; ch < nchunks; ++ch, ++pc) {
          if (!failed) {
            const int b = pc % RS_NBUF;
            const uint32_t ph = (uint32_t)(pc / RS_NBUF);
            if (!mbar_wait(pfull_bar(b), ph & 1, abort_flag, p.status)) {
              failed = true;
            } else {
              tc_fence_after();
              if (ncol == 32) {   // one load and one wait per drain
                float v[32];
                tmem_ld32(tmem_base + lane_off + (uint32_t)(b * 128 + col0), v);
#pragma unroll
                for (int e = 0; e < 32; ++e) acc[e] += __float2int_rn(v[e] * up);
              } else {
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                  if (g * 8 < ncol) {
                    float v[8];
                    tmem_ld8(tmem_base + lane_off + (uint32_t)(b * 128 + col0 + g * 8), v);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[g * 8 + e] += __float2int_rn(v[e] * up);
                  }
                }
              }
              tc_fence_before();
              mbar_arrive(pempty_bar(b));
            }
          }
          if (!failed && ((ch + 1) % RS_FLUSH == 0 || ch + 1 == nchunks)) {
            const double down = ldexp(1.0, -8 * m);
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              if (c < ncol) Grow[c] = (first_flush ? 0.0 : Grow[c]) + (double)acc[c] * down;
              acc[c] = 0;
            }
            first_flush = false;
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(RS_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- exact squared distances
// d2_ij = |a_i|^2 + |a_j|^2 - 2 a_i . a_j for node series on the 2^-16 grid
// (a = x 2^16, integers below 2^23 in magnitude). Each a is written as three
// signed base-256 digits (|digit| <= 128, exact in bf16), so the Gram matrix is
// a_i . a_j = sum_{s,t} 2^(8(s+t)) (D_s D_t^T)_ij over nine bf16 products.
// Every digit product is exact in float32 (<= 2^14) and the slice pairs of
// one weight w = s + t (at most three) summed over a 256-sample chunk stay
// below 2^24, so the MMA's float32 accumulator holds an exact integer; the
// epilogue adds it, shifted by 8w, to int64 accumulators. The result equals
// the int64 sum of squared differences exactly; it is written as float64
// multiples of 2^-32 to (i, j) and, off the diagonal blocks, to (j, i).
// Tiles are 128 rows x 64 columns of the upper block triangle; warp roles as
// in k_tc_resid. Each pipeline stage holds the three digit planes of both
// sides for one K block (72 KB, loaded once), and the MMA issuer feeds all
// nine slice products into the five weight accumulators of the K chunk, slots
// of a ring of eight 64-column TMEM accumulators, so that the MMAs of a tile
// run ahead of its epilogue.
constexpr int DS_SLICES = 3;
constexpr int DS_N = 64;
constexpr int DS_STAGES = 2;
constexpr int DS_A = 128 * 128;                  // one digit plane: 128 rows x 64 bf16
constexpr int DS_B = DS_N * 128;                 // one digit plane: 64 rows x 64 bf16
constexpr int DS_STAGE_BYTES = DS_SLICES * (DS_A + DS_B);   // all three planes of both sides
constexpr int EPI_STAGE_DOUBLES = 16 * 32 * 17;          // per epilogue warp: 32 rows x 16 columns, padded
constexpr int DS_SMEM_BYTES = DS_STAGES * DS_STAGE_BYTES + 512 + EPI_STAGE_DOUBLES * 8 + 1024;
constexpr int DS_NBUF = 8;                     // ring of TMEM accumulators
constexpr int DS_TMEM_COLS = DS_NBUF * DS_N;
constexpr int DS_CHUNK_KB = 4;                   // 256 samples per exact chunk

struct DistMaps {
  CUtensorMap a[DS_SLICES];   // digit planes, box 64 x 128 rows
  CUtensorMap b[DS_SLICES];   // digit planes, box 64 x 64 rows
};

struct DistParams {
  int nb128;                  // row blocks of 128
  int nb64;                   // column blocks of 64 (2 nb128)
  int num_tiles;              // tiles (I, J) with J >= 2 I
  int kblocks;                // padded samples / 64
  int n;
  const long long* norms;     // |a_i|^2, rows padded with 0
  double* A;                  // n x n output
  const int* offgrid;         // bit 0 set: input off the grid (the float64 kernel runs instead)
  uint32_t idesc;
  unsigned* status;
  // Row panels (graphs regenerated panel by panel): A holds rows row0 ..
  // (A[(i - row0) n + j]), nothing is mirrored, and the tiles are either the
  // upper-triangle tiles tile0 .. tile0 + num_tiles - 1 (rect = 0; the rows of
  // the panel when the range is the panel's row blocks) or every tile
  // (I0 + t / nb64, t % nb64) of the panel's rect row blocks (rect > 0: whole rows).
  int panel;
  int row0;
  long long tile0;
  int rect;
  int I0;
};

// tile t -> (I, J): row block I holds nb64 - 2 I tiles J = 2 I .. nb64 - 1
__device__ __forceinline__ void dist_tile(int t, int nb128, int nb64, int& I, int& J) {
  int lo = 0, hi = nb128 - 1;
  while (lo < hi) {                                      // last I with off(I) <= t
    const int mid = (lo + hi + 1) >> 1;
    const long long off = (long long)mid * nb64 - (long long)mid * (mid - 1);
    if (off <= t) lo = mid; else hi = mid - 1;
  }
  I = lo;
  J = 2 * lo + (int)(t - ((long long)lo * nb64 - (long long)lo * (lo - 1)));
}

__device__ __forceinline__ void dist_decode(const DistParams& p, int t, int& I, int& J) {
  if (p.rect > 0) {
    I = p.I0 + t / p.nb64;
    J = t % p.nb64;
  } else {
    dist_tile((int)(t + p.tile0), p.nb128, p.nb64, I, J);
  }
}

__global__ void __launch_bounds__(T8_THREADS, 1)
    k_tc_dist(const __grid_constant__ DistMaps maps, const DistParams p) {
  if (*p.offgrid & 1) return;                            // uniform: before any barrier or allocation
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + DS_STAGES * DS_STAGE_BYTES);
  double* stage = reinterpret_cast<double*>(smem + DS_STAGES * DS_STAGE_BYTES + 512);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * DS_STAGES + 2 * DS_NBUF + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * DS_STAGES + 2 * DS_NBUF + 3);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (DS_STAGES + s); };
  auto pfull_bar = [&](int b) { return bar0 + 8u * (2 * DS_STAGES + b); };
  auto pempty_bar = [&](int b) { return bar0 + 8u * (2 * DS_STAGES + DS_NBUF + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * DS_STAGES + 2 * DS_NBUF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (p.kblocks + DS_CHUNK_KB - 1) / DS_CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < DS_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < DS_NBUF; ++b) {
      mbar_init(pfull_bar(b), 1);
      mbar_init(pempty_bar(b), T8_EPI);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(DS_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x) {
      int I, J;
      dist_decode(p, t, I, J);
      // one stage per K block: the three digit planes of the row block and of the column block
      for (int kb = 0; kb < p.kblocks && ok; ++kb, ++it) {
        const int s = it % DS_STAGES;
        const uint32_t r = (uint32_t)(it / DS_STAGES);
        if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t dst = smem_u32(smem + s * DS_STAGE_BYTES);
        mbar_expect_tx(full_bar(s), DS_STAGE_BYTES);
        for (int pl = 0; pl < DS_SLICES; ++pl) {
          tma_load_2d(dst + pl * DS_A, &maps.a[pl], kb * 64, I * 128, full_bar(s));
          tma_load_2d(dst + DS_SLICES * DS_A + pl * DS_B, &maps.b[pl], kb * 64, J * DS_N, full_bar(s));
        }
      }
    }
    if (!ok) {
      for (int j = (it > DS_STAGES ? it - DS_STAGES : 0); j < it; ++j) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full_bar(j % DS_STAGES), (uint32_t)(j / DS_STAGES) & 1) &&
               globaltimer() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer: per K chunk, the five weight
    // accumulators (ring slots pc .. pc + 4) take all nine slice products of each K block
    constexpr int NW = 2 * DS_SLICES - 1;
    int it = 0, pc = 0;
    bool ok = true, issued = false;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x)
      for (int c = 0; c < nchunks && ok; ++c, pc += NW) {
        for (int w = 0; w < NW && ok; ++w) {
          const int b = (pc + w) % DS_NBUF;
          const uint32_t ph = (uint32_t)((pc + w) / DS_NBUF);
          if (!mbar_wait(pempty_bar(b), (ph & 1) ^ 1, abort_flag, p.status)) ok = false;
        }
        if (!ok) break;
        tc_fence_after();
        for (int kb = c * DS_CHUNK_KB; kb < min(p.kblocks, (c + 1) * DS_CHUNK_KB) && ok; ++kb, ++it) {
          const int s = it % DS_STAGES;
          if (!mbar_wait(full_bar(s), (uint32_t)(it / DS_STAGES) & 1, abort_flag, p.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(smem + s * DS_STAGE_BYTES);
          const bool first_kb = kb == c * DS_CHUNK_KB;
          for (int sa = 0; sa < DS_SLICES; ++sa)
            for (int sb = 0; sb < DS_SLICES; ++sb) {
              const int w = sa + sb;
              const uint32_t d_tmem = tmem_base + (uint32_t)(((pc + w) % DS_NBUF) * DS_N);
              // the first product of a weight in the chunk starts its accumulator
              const bool first = first_kb && sa == (w < DS_SLICES ? 0 : w - (DS_SLICES - 1));
              const uint64_t adesc = smem_desc(base + sa * DS_A);
              const uint64_t bdesc = smem_desc(base + DS_SLICES * DS_A + sb * DS_B);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                mma_bf16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc,
                         (first && kk == 0) ? 0u : 1u);
            }
          issued = true;
          mma_commit(empty_bar(s));
        }
        if (!ok) break;
        for (int w = 0; w < NW; ++w) mma_commit(pfull_bar((pc + w) % DS_NBUF));
      }
    if (!ok && issued) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: exact integer Gram, d2, both triangles
    const int q = warp & 3;                              // TMEM lane quarter
    const int part = (warp - 2) >> 2;                    // 16-column part of the tile
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    int pc = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x) {
      int I, J;
      dist_decode(p, t, I, J);
      long long g[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) g[e] = 0;
      for (int c = 0; c < nchunks; ++c)
        for (int w = 0; w <= 2 * (DS_SLICES - 1); ++w, ++pc) {
          if (failed) continue;
          const int b = pc % DS_NBUF;
          const uint32_t ph = (uint32_t)(pc / DS_NBUF);
          if (!mbar_wait(pfull_bar(b), ph & 1, abort_flag, p.status)) {
            failed = true;
            continue;
          }
          tc_fence_after();
          {
            float v[16];   // one load and one wait per drain
            tmem_ld16(tmem_base + lane_off + (uint32_t)(b * DS_N + part * 16), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) g[e] += (long long)__float2int_rn(v[e]) * (1LL << (8 * w));
          }
          tc_fence_before();
          mbar_arrive(pempty_bar(b));
        }
      if (__any_sync(0xffffffffu, failed)) continue;
      const int row = I * 128 + q * 32 + lane;
      const bool rowok = row < p.n;
      const long long ni = rowok ? p.norms[row] : 0;
      const int col0 = J * DS_N + part * 16;
      const bool mirror = !p.panel && J >= 2 * I + 2;    // off the diagonal 128-block
      double* stg = stage + (warp - 2) * (32 * 17);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int col = col0 + e;
        double d2 = 0.0;
        if (rowok && col < p.n) {
          // d2 >= 0 exactly; integer-only conversion (float64 is the scarce pipe)
          d2 = u64_to_double_rn((unsigned long long)(ni + p.norms[col] - 2 * g[e]), -32);
          if (mirror) p.A[(size_t)col * p.n + row] = d2;   // lanes write 32 consecutive entries
        }
        stg[lane * 17 + e] = d2;
      }
      __syncwarp();
      // the warp's 32 x 16 block row-wise, two 128-byte row segments per store
#pragma unroll 4
      for (int it = 0; it < 16; ++it) {
        const int rr = 2 * it + (lane >> 4), c = lane & 15;
        const int grow = I * 128 + q * 32 + rr, gcol = col0 + c;
        if (grow < p.n && gcol < p.n) p.A[(size_t)(grow - p.row0) * p.n + gcol] = stg[rr * 17 + c];
      }
      __syncwarp();
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(DS_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- CAD scores, Gram on the tensor cores
// Delta c_ij = c2(i,j) - c1(i,j) = (a_i - a_j).(b_i - b_j) = d_i + d_j - M_ij with
// a = sqrt(vol2) Z2 - sqrt(vol1) Z1, b = sqrt(vol2) Z2 + sqrt(vol1) Z1,
// d_i = a_i.b_i and M_ij = a_i.b_j + b_i.a_j = u_i.v_j for the rows
// u = [a / g | b g] and v = [b g | a / g] (g a power of two per column that
// balances the two halves; it cancels in every product). u / c and v / c
// (c twice a power of two above every entry) are six bf16 slices on the
// grids 2^-8s (signed base-256 digits of the values rounded to 2^-48, each at
// most 128 in magnitude, so every digit product is at most 2^14). The slice
// pairs s + t = w of the weights w = 2, 3, 4 and 5 (1, 2, 3 and 4 pairs)
// summed over a K-chunk of 256 stay within 2^24 grid steps of 2^-8w, so those
// four TMEM accumulators hold exact integers; the pairs of weights 6 and 7
// (11 pairs, 21 in all) share a fifth accumulator in plain float32 (the
// slices carry their 2^-8s scales), whose value is below 2^-23 of the top
// weight's bound and is rounded to the unit. The epilogue adds each chunk,
// shifted to the common unit c^2 2^-48, in int64. Per K block two pipeline
// stages (u slices 1-3 with all six v slices, then u slices 4-6 with v slices
// 1-3) feed the five live accumulators of the chunk. With d_i in the same unit, Delta c_ij is
// formed in int64 (no cancellation error beyond the slicing's, about 2^-45
// of max |u . v|),
// and E_ij = |A1_ij - A2_ij| |Delta c_ij| and its row and column sums are
// float64. Tiles are 128 x 64 of the upper block triangle (pairs i < j only);
// each 64 x 64 sub-block writes its row sums to contrib[partner block][i]
// and column sums to contrib[row block][j] (row plus column sums on the
// diagonal), the slots of the 64-node block layout of k_score_reduce, in
// units of c^2 2^-48 times oscale. Warp roles as in k_tc_resid, with a ring
// of eight 64-column TMEM accumulators.
constexpr int SC_SLICES = 6;
constexpr int SC_N = 64;
constexpr int SC_STAGES = 2;
constexpr int SC_A = 128 * 128;                  // one slice plane: 128 rows x 64 bf16
constexpr int SC_B = SC_N * 128;                 // one slice plane: 64 rows x 64 bf16
constexpr int SC_HALF = SC_SLICES / 2;           // u slices per stage (two stages per K block)
constexpr int SC_STAGE_BYTES = SC_HALF * SC_A + SC_SLICES * SC_B;   // 3 u planes + all 6 v planes
constexpr int SC_XPOSE = 32 * 4;                 // per epilogue warp: |A1 - A2| of 32 rows x 4 columns
constexpr int SC_PARTS = 128 * 4 + 4 * SC_N;        // row and column partials of one tile
constexpr int SC_EPI_DOUBLES = SC_PARTS + 16 * SC_XPOSE + SC_PARTS;   // partials double-buffered
constexpr int SC_SMEM_BYTES = SC_STAGES * SC_STAGE_BYTES + 512 + SC_EPI_DOUBLES * 8 + 1024;
constexpr int SC_NBUF = 8;                     // ring of TMEM accumulators
constexpr int SC_TMEM_COLS = SC_NBUF * SC_N;
constexpr int SC_CHUNK_KB = 4;                   // 256 K per exact chunk
constexpr int SC_NW = 5;                         // accumulators per chunk: weights 2, 3, 4, 5 and 6-7

// accumulator of a slice pair's weight w = s + t within a chunk
__device__ __forceinline__ int sc_slot(int w) { return w < 6 ? w - 2 : 4; }

struct ScoreMaps {
  CUtensorMap u[SC_SLICES];   // slices of u, box 64 x 128 rows
  CUtensorMap v[SC_SLICES];   // slices of v, box 64 x 64 rows
};

struct ScoreParams {
  int nb128, nb64, num_tiles, kblocks, n;
  long long tile0;            // first tile of the upper-triangle numbering
  int row0;                   // A1, A2 hold rows row0 .. (A[(i - row0) n + j])
  const double* A1;
  const double* A2;
  const long long* dint;      // d_i in units of c^2 2^-48 (padded rows 0)
  const double* oscale;       // c^2 2^-48
  double* contrib;            // (n / 64 rounded up) x n partial sums
  uint32_t idesc;
  unsigned* status;
};


__global__ void __launch_bounds__(T8_THREADS, 1)
    k_tc_score(const __grid_constant__ ScoreMaps maps, const ScoreParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SC_STAGES * SC_STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * SC_STAGES + 2 * SC_NBUF + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * SC_STAGES + 2 * SC_NBUF + 3);
  double* epi = reinterpret_cast<double*>(smem + SC_STAGES * SC_STAGE_BYTES + 512);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (SC_STAGES + s); };
  auto pfull_bar = [&](int b) { return bar0 + 8u * (2 * SC_STAGES + b); };
  auto pempty_bar = [&](int b) { return bar0 + 8u * (2 * SC_STAGES + SC_NBUF + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * SC_STAGES + 2 * SC_NBUF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunks = (p.kblocks + SC_CHUNK_KB - 1) / SC_CHUNK_KB;

  if (threadIdx.x == 0) {
    for (int s = 0; s < SC_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < SC_NBUF; ++b) {
      mbar_init(pfull_bar(b), 1);
      mbar_init(pempty_bar(b), T8_EPI);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(SC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer: per K block two stages, u slices
    // 1-3 with v slices 1-6, then u slices 4-6 with v slices 1-3
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x) {
      int I, J;
      dist_tile((int)(t + p.tile0), p.nb128, p.nb64, I, J);
      for (int kb = 0; kb < p.kblocks && ok; ++kb)
        for (int h = 0; h < 2 && ok; ++h, ++it) {
          const int s = it % SC_STAGES;
          const uint32_t r = (uint32_t)(it / SC_STAGES);
          if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
            ok = false;
            break;
          }
          const uint32_t dst = smem_u32(smem + s * SC_STAGE_BYTES);
          // u slices 4-6 pair with v slices 1-3 only (s + t <= 7)
          const int nv = h == 0 ? SC_SLICES : SC_SLICES + 1 - (SC_HALF + 1);
          mbar_expect_tx(full_bar(s), SC_HALF * SC_A + nv * SC_B);
          for (int pl = 0; pl < SC_HALF; ++pl)
            tma_load_2d(dst + pl * SC_A, &maps.u[h * SC_HALF + pl], kb * 64, I * 128, full_bar(s));
          for (int pl = 0; pl < nv; ++pl)
            tma_load_2d(dst + SC_HALF * SC_A + pl * SC_B, &maps.v[pl], kb * 64, J * SC_N, full_bar(s));
        }
    }
    if (!ok) {
      for (int j = (it > SC_STAGES ? it - SC_STAGES : 0); j < it; ++j) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full_bar(j % SC_STAGES), (uint32_t)(j / SC_STAGES) & 1) &&
               globaltimer() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer: per K chunk, the five
    // accumulators (ring slots pc .. pc + 4) take the 21 slice products of each K block
    constexpr int NW = SC_NW;
    int it = 0, pc = 0;
    bool ok = true, issued = false;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x)
      for (int c = 0; c < nchunks && ok; ++c, pc += NW) {
        for (int w = 0; w < NW && ok; ++w) {
          const int b = (pc + w) % SC_NBUF;
          const uint32_t ph = (uint32_t)((pc + w) / SC_NBUF);
          if (!mbar_wait(pempty_bar(b), (ph & 1) ^ 1, abort_flag, p.status)) ok = false;
        }
        if (!ok) break;
        tc_fence_after();
        for (int kb = c * SC_CHUNK_KB; kb < min(p.kblocks, (c + 1) * SC_CHUNK_KB) && ok; ++kb)
          for (int h = 0; h < 2 && ok; ++h, ++it) {
            const int s = it % SC_STAGES;
            if (!mbar_wait(full_bar(s), (uint32_t)(it / SC_STAGES) & 1, abort_flag, p.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * SC_STAGE_BYTES);
            const bool first_kb = kb == c * SC_CHUNK_KB;
            for (int pl = 0; pl < SC_HALF; ++pl) {
              const int sa = h * SC_HALF + pl + 1;         // u slice, 1-based
              for (int sb = 1; sa + sb <= SC_SLICES + 1; ++sb) {
                const int w = sa + sb;                     // 2 .. 7
                const uint32_t d_tmem = tmem_base + (uint32_t)(((pc + sc_slot(w)) % SC_NBUF) * SC_N);
                // the first product of an accumulator in the chunk (u slice 1; for weights
                // 6 and 7 the pair (1, 5)) starts it
                const bool first = first_kb && sa == 1 && sb <= 5;
                const uint64_t adesc = smem_desc(base + pl * SC_A);
                const uint64_t bdesc = smem_desc(base + SC_HALF * SC_A + (sb - 1) * SC_B);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                  mma_bf16(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc,
                           (first && kk == 0) ? 0u : 1u);
              }
            }
            issued = true;
            mma_commit(empty_bar(s));
          }
        if (!ok) break;
        for (int w = 0; w < NW; ++w) mma_commit(pfull_bar((pc + w) % SC_NBUF));
      }
    if (!ok && issued) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue
    const int q = warp & 3;                              // TMEM lane quarter (32 rows)
    const int part = (warp - 2) >> 2;                    // 16-column part of the tile
    const int et = threadIdx.x - 64;                     // epilogue thread 0 .. 511
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    // partials of even tiles at epi, of odd tiles past the transposition buffers, so
    // one barrier per tile separates their writes from their reads
    int tpar = 0;
    const double osc = *p.oscale;
    int pc = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x) {
      int I, J;
      dist_tile((int)(t + p.tile0), p.nb128, p.nb64, I, J);
      {
        // bring this thread's A1 and A2 row segments into L2 while the MMAs run
        const int prow = I * 128 + q * 32 + lane, pc0 = J * SC_N + part * 16;
        if (prow < p.n && pc0 < p.n) {
          const size_t o0 = (size_t)(prow - p.row0) * p.n + pc0, o1 = o0 + min(15, p.n - 1 - pc0);
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.A1 + o0));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.A2 + o0));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.A1 + o1));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(p.A2 + o1));
        }
      }
      // d_j of the warp's 16 columns, one per lane (lanes 16-31 repeat them)
      const long long dcol = p.dint[J * SC_N + part * 16 + (lane & 15)];
      long long m[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) m[e] = 0;
      // drains in the ring order of the MMA issuer: K chunk outer, accumulator inner;
      // each chunk sum goes to the unit c^2 2^-48 (the exact weights 2-5 shifted
      // there, the float32 sum of weights 6 and 7 rounded there)
      for (int c = 0; c < nchunks; ++c)
        for (int a = 0; a < SC_NW; ++a, ++pc) {
          if (failed) continue;
          const int b = pc % SC_NBUF;
          const uint32_t ph = (uint32_t)(pc / SC_NBUF);
          if (!mbar_wait(pfull_bar(b), ph & 1, abort_flag, p.status)) {
            failed = true;
            continue;
          }
          tc_fence_after();
          // weight w = a + 2 for the exact accumulators: 2^(8w) makes the sum an integer
          // (|x| <= 2^24), shifted by 48 - 8w; the last one times 2^48 is below 2^31
          const float up = __int_as_float((127 + (a < 4 ? 8 * (a + 2) : 48)) << 23);
          const int sh = a < 4 ? 48 - 8 * (a + 2) : 0;
          {
            float v[16];   // one load and one wait per drain
            tmem_ld16(tmem_base + lane_off + (uint32_t)(b * SC_N + part * 16), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) m[e] += (long long)__float2int_rn(v[e] * up) * (1LL << sh);
          }
          tc_fence_before();
          mbar_arrive(pempty_bar(b));
        }
      // edge scores of the thread's 16 pairs (row i, columns col0 ..): one
      // float64 subtraction for Delta A, the rest in float-float on the float32
      // pipes (float64 is the scarce pipe)
      const int rl = q * 32 + lane;                      // row within the tile
      const int row = I * 128 + rl;
      const int col0 = J * SC_N + part * 16;
      const int br = 2 * I + (q >> 1);                   // 64-row block of the row
      const bool rowok = !failed && row < p.n && br <= J;
      const long long di = rowok ? p.dint[row] : 0;
      ff ev[16];
      ff rs = {0.f, 0.f};
      // |A1 - A2| of the warp's 32 rows x 16 columns, four columns at a time:
      // loaded with lanes along the columns (each load instruction reads eight
      // 32-byte row segments instead of 32 single elements of 32 rows), passed
      // through shared memory to the row-per-lane layout of the drained sums
      double* xp = epi + SC_PARTS + (warp - 2) * SC_XPOSE;
      const int rbase = I * 128 + q * 32;
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {
        __syncwarp();
#pragma unroll
        for (int st = 0; st < 4; ++st) {
          const int rr = st * 8 + (lane >> 2), cc = jq * 4 + (lane & 3);
          const int grow = rbase + rr, gcol = col0 + cc;
          double da = 0.0;
          if (!failed && grow < p.n && gcol < p.n) {
            const size_t o = (size_t)(grow - p.row0) * p.n + gcol;
            da = fabs(p.A1[o] - p.A2[o]);
          }
          xp[rr * 4 + (lane & 3)] = da;
        }
        __syncwarp();
#pragma unroll
        for (int e4 = 0; e4 < 4; ++e4) {
          const int e = jq * 4 + e4;
          const int col = col0 + e;
          ff x = {0.f, 0.f};
          const long long dj = __shfl_sync(0xffffffffu, dcol, e);   // converged: the whole warp
          if (rowok && col < p.n && (br < J || row < col)) {
            const long long dc = di + dj - m[e];
            const unsigned long long adc = dc < 0 ? (unsigned long long)(-dc) : (unsigned long long)dc;
            x = ff_mul(split_nonneg(xp[lane * 4 + e4]), ff_from_u64(adc));
          }
          ev[e] = x;
          rs = ff_add(rs, x);
        }
      }
      double* rowpart = epi + tpar * (SC_PARTS + 16 * SC_XPOSE);   // [128][4]
      double* colpart = rowpart + 128 * 4;                          // [4][64]
      tpar ^= 1;
      rowpart[rl * 4 + part] = (double)rs.hi + (double)rs.lo;
      // column sums over the warp's 32 rows: reduce-scatter, lane pairs end with one column each
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const bool hi = lane & 16;
        const ff keep = hi ? ev[e + 8] : ev[e], send = hi ? ev[e] : ev[e + 8];
        ev[e] = ff_add(keep, {__shfl_xor_sync(0xffffffffu, send.hi, 16), __shfl_xor_sync(0xffffffffu, send.lo, 16)});
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool hi = lane & 8;
        const ff keep = hi ? ev[e + 4] : ev[e], send = hi ? ev[e] : ev[e + 4];
        ev[e] = ff_add(keep, {__shfl_xor_sync(0xffffffffu, send.hi, 8), __shfl_xor_sync(0xffffffffu, send.lo, 8)});
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const bool hi = lane & 4;
        const ff keep = hi ? ev[e + 2] : ev[e], send = hi ? ev[e] : ev[e + 2];
        ev[e] = ff_add(keep, {__shfl_xor_sync(0xffffffffu, send.hi, 4), __shfl_xor_sync(0xffffffffu, send.lo, 4)});
      }
      {
        const bool hi = lane & 2;
        const ff keep = hi ? ev[1] : ev[0], send = hi ? ev[0] : ev[1];
        ev[0] = ff_add(keep, {__shfl_xor_sync(0xffffffffu, send.hi, 2), __shfl_xor_sync(0xffffffffu, send.lo, 2)});
      }
      ev[0] = ff_add(ev[0], {__shfl_xor_sync(0xffffffffu, ev[0].hi, 1), __shfl_xor_sync(0xffffffffu, ev[0].lo, 1)});
      const int cidx = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
      if ((lane & 1) == 0) colpart[q * SC_N + part * 16 + cidx] = (double)ev[0].hi + (double)ev[0].lo;
      asm volatile("bar.sync 1, 512;" ::: "memory");
      if (et < 128 && !failed) {
        // row partial of tile row et over the 64 columns
        const int r2 = I * 128 + et;
        const int b2 = 2 * I + (et >> 6);
        if (r2 < p.n && b2 <= J && J * SC_N < p.n) {
          double v = ((rowpart[et * 4] + rowpart[et * 4 + 1]) + rowpart[et * 4 + 2]) + rowpart[et * 4 + 3];
          if (b2 == J) {                                 // diagonal 64-block: add the column sum of the same node
            const int hh = et >> 6, c = et - 64 * hh;
            v += colpart[(2 * hh) * SC_N + c] + colpart[(2 * hh + 1) * SC_N + c];
          }
          p.contrib[(size_t)J * p.n + r2] = v * osc;
        }
      } else if (et < 256 && !failed) {
        // column partial of column c over the 64 rows of half hh (off the diagonal 64-block)
        const int x = et - 128, hh = x >> 6, c = x & 63;
        const int col = J * SC_N + c, b2 = 2 * I + hh;
        if (col < p.n && b2 < J)
          p.contrib[(size_t)b2 * p.n + col] = (colpart[(2 * hh) * SC_N + c] + colpart[(2 * hh + 1) * SC_N + c]) * osc;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(SC_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- bf16 squaring on CTA pairs
// S~^2 with tcgen05.mma.cta_group::2: the two CTAs of a cluster compute one
// 256 x 256 block (I, J) of the upper block triangle. CTA rank r loads, per
// 64-wide k-block, rows I*256 + 128 r of the level (its A half) and rows
// J*256 + 128 r (its half of B) into its own shared memory; each copy
// completes on the rank-0 CTA's stage barrier. The rank-0 CTA issues one
// M = 256, N = 256 MMA per 16 of K that reads both CTAs' halves; each CTA's
// TMEM holds its 128 rows of the block (two 256-column accumulators, so one
// block drains while the next accumulates), and both CTAs' epilogues store
// their rows (mirrored below the diagonal) as in the one-CTA kernel. Per SM
// a k-block stages 32 KB (16 KB of A, 16 KB of B) for a 128 x 256 x 64
// product instead of 48 KB, so six stages fit and the L2-to-shared traffic
// per flop drops by a third. Stage release and accumulator-full signals are
// multicast by the MMA commits to both CTAs; the epilogue warps of both
// CTAs arrive on the rank-0 accumulator-empty barrier. K pacing as in the
// one-CTA kernel. Every wait is bounded; the teardown waits for the last
// stage releases (no signal lands after a CTA has left) and passes a
// cluster barrier before the pair frees its TMEM.
constexpr int S2_STAGES = 6;
constexpr int S2_HALF = 128 * BK * 2;                  // 16 KiB: 128 rows x 64 bf16
constexpr int S2_STAGE = 2 * S2_HALF;                  // A half + B half
constexpr int S2_NBARS = 2 * S2_STAGES + 5;            // full, empty, tfull x2, tempty x2, drain
constexpr int S2_XT_WORDS = 32 * 17;                   // per epilogue warp: a 32 x 32 bf16 chunk, padded rows
constexpr int S2_SMEM_BYTES = S2_STAGES * S2_STAGE + 256 + 8 * S2_XT_WORDS * 4 + 1024;
constexpr int S2_TMEM_COLS = 512;
constexpr int S2_THREADS = 320;                        // producer, MMA issuer, 8 epilogue warps
constexpr int S2_PACE_MIN_KBLOCKS = 512;               // K pacing from n = 32768 on

struct Sq2Params {
  const uint32_t* tiles;   // upper-triangle 256-blocks: I (bits 0-14), J (bits 15-29); grouped: graph
                           // (bits 0-15), I (16-22), J (23-29)
  int num_tiles;
  int kblocks;
  int npad;
  const TcGroup* groups;   // grouped launch: each graph's level map (mapA), output, order, k loop
  uint32_t idesc;          // kind::f16, bf16 x bf16 -> f32, M = 256, N = 256
  __nv_bfloat16* out;
  unsigned* status;
  unsigned* pace;          // K pacing counters (null: off)
  int pace_steps;
  int debug_withhold_load;   // test hook: the rank-0 CTA never issues its first A load
};

// One pair tile: its blocks, the level's map, k loop, output and order.
struct Sq2Tile {
  int I, J, kblocks, npad;
  const CUtensorMap* map;
  __nv_bfloat16* out;
};
__device__ __forceinline__ Sq2Tile sq2_tile(const Sq2Params& p, const CUtensorMap* tm, uint32_t td) {
  Sq2Tile q;
  if (p.groups) {
    const TcGroup& g = p.groups[td & 0xFFFF];
    q.I = (td >> 16) & 0x7F;
    q.J = (td >> 23) & 0x7F;
    q.kblocks = g.kblocks;
    q.npad = g.npad;
    q.map = &g.mapA;
    q.out = static_cast<__nv_bfloat16*>(g.out);
  } else {
    q.I = td & 0x7FFF;
    q.J = (td >> 15) & 0x7FFF;
    q.kblocks = p.kblocks;
    q.npad = p.npad;
    q.map = tm;
    q.out = p.out;
  }
  return q;
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// TMA load into this CTA's shared memory, completing on a barrier of either
// CTA of the pair (cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the barrier at this offset in both CTAs once the MMAs issued so
// far have completed
__device__ __forceinline__ void mma_commit_pair(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(bar),
      "h"((unsigned short)3)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// A 32 x 32 chunk (rows r0 .., columns col0 ..) of a block on the diagonal:
// above the diagonal as any other chunk (rows and mirrored rows, staged);
// below it nothing (the mirror of the chunk above writes it); the chunk the
// diagonal crosses (col0 == r0) through shared memory too, its upper
// triangle row by row and its strict upper triangle mirrored, each store
// instruction covering 32 consecutive columns of one row.
__device__ __forceinline__ void square_store32_diag(__nv_bfloat16* C, int npad, int r0, int col0, int lane,
                                                    const float (&v)[32], uint32_t* T);

// An off-diagonal 32 x 32 chunk through the warp's staging tile T: rows
// r0 + lane (one per lane, as drained from TMEM), columns col0 .. col0 + 31.
// The rows are stored two per instruction (16 lanes x 4 bytes: one 64-byte
// segment each) and so are the mirrored rows, where stores straight from
// the row-per-lane layout touch 32 rows per instruction.
__device__ __forceinline__ void square_store32_staged(__nv_bfloat16* C, int npad, int r0, int col0, int lane,
                                                      const float (&v)[32], uint32_t* T) {
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    T[lane * 17 + e] = *reinterpret_cast<uint32_t*>(&h);
  }
  __syncwarp();
  const int w = lane & 15, hl = lane >> 4;
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int row = 2 * it + hl;
    reinterpret_cast<uint32_t*>(C + (size_t)(r0 + row) * npad + col0)[w] = T[row * 17 + w];
  }
#pragma unroll
  for (int it = 0; it < 16; ++it) {
    const int e = 2 * it + hl;   // mirrored row col0 + e, columns r0 + 2w, r0 + 2w + 1
    const uint32_t a = T[(2 * w) * 17 + it], b = T[(2 * w + 1) * 17 + it];
    const uint32_t lo = hl ? (a >> 16) : (a & 0xFFFFu), hi = hl ? (b >> 16) : (b & 0xFFFFu);
    reinterpret_cast<uint32_t*>(C + (size_t)(col0 + e) * npad + r0)[w] = lo | (hi << 16);
  }
  __syncwarp();
}
__device__ __forceinline__ void square_store32_diag(__nv_bfloat16* C, int npad, int r0, int col0, int lane,
                                                    const float (&v)[32], uint32_t* T) {
  if (col0 >= r0 + 32) {
    square_store32_staged(C, npad, r0, col0, lane, v, T);
    return;
  }
  if (col0 + 32 <= r0) return;
  // col0 == r0: this lane holds row r0 + lane; T[row * 17 + c / 2] holds columns c, c + 1
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
    T[lane * 17 + e] = *reinterpret_cast<uint32_t*>(&h);
  }
  __syncwarp();
  auto elem = [&](int row, int col) {
    const uint32_t w = T[row * 17 + (col >> 1)];
    return __ushort_as_bfloat16((unsigned short)((col & 1) ? (w >> 16) : (w & 0xFFFFu)));
  };
  for (int row = 0; row < 32; ++row)   // row r0 + row, columns col0 + lane >= that row
    if (lane >= row) C[(size_t)(r0 + row) * npad + col0 + lane] = elem(row, lane);
  for (int m = 1; m < 32; ++m)         // mirrored row col0 + m, columns r0 + lane < that row
    if (lane < m) C[(size_t)(col0 + m) * npad + r0 + lane] = elem(lane, m);
  __syncwarp();
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(S2_THREADS, 1)
    k_tc_sq2(const __grid_constant__ CUtensorMap tmL, const Sq2Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S2_STAGES * S2_STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S2_NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + S2_NBARS + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S2_STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S2_STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * S2_STAGES + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S2_STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const uint32_t lead_bar0 = mapa_rank(bar0, 0);   // the rank-0 CTA's barriers, cluster addresses

  if (threadIdx.x == 0) {
    for (int s = 0; s < S2_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 16);   // the eight epilogue warps of each CTA
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmL)) : "memory");
  }
  if (warp == 0) {   // one warp of each CTA allocates the pair's TMEM
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S2_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();   // both CTAs' barriers initialised before any remote signal
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer (both CTAs)
    int it = 0;
    bool ok = true;
    bool pacing = p.pace != nullptr;
    const int steps_per_tile = (p.kblocks + PACE_KB - 1) / PACE_KB;
    int lt = 0;
    for (int t = cid; t < p.num_tiles && ok; t += ncl) {
      const Sq2Tile q = sq2_tile(p, &tmL, p.tiles[t]);
      if (p.groups)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(q.map))
                     : "memory");
      // grouped: a 256-block may end past the padded order (a multiple of
      // 128); those rows come back as the map's zero fill
      const int a_row = q.I * 256 + (int)rank * 128, b_row = q.J * 256 + (int)rank * 128;
      for (int kb = 0; kb < q.kblocks; ++kb, ++it) {
        if (p.pace && kb % PACE_KB == 0) {
          const int step = lt * steps_per_tile + kb / PACE_KB;
          if (step < p.pace_steps) atomicAdd(p.pace + step, 1u);
          if (pacing && step >= PACE_SLACK && step - PACE_SLACK < p.pace_steps) {
            const unsigned* c = p.pace + step - PACE_SLACK;
            const unsigned long long t0 = globaltimer();
            unsigned v;
            for (;;) {
              asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
              if (v >= gridDim.x) break;
              if (globaltimer() - t0 > PACE_WAIT_NS) {
                pacing = false;
                break;
              }
            }
          }
        }
        const int s = it % S2_STAGES;
        const uint32_t r = (uint32_t)(it / S2_STAGES);
        if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        if (rank == 0) mbar_expect_tx(full_bar(s), 2 * S2_STAGE);   // both CTAs' copies
        const uint32_t dst = smem_u32(smem + s * S2_STAGE);
        const uint32_t fb = lead_bar0 + 8u * s;
        if (!(p.debug_withhold_load && it == 0 && rank == 0)) tma_load_2d_pair(dst, q.map, kb * BK, a_row, fb);
        tma_load_2d_pair(dst + S2_HALF, q.map, kb * BK, b_row, fb);
      }
      ++lt;
    }
    if (p.pace)
      for (int step = lt * steps_per_tile; step < p.pace_steps; ++step) atomicAdd(p.pace + step, 1u);
    if (ok) {
      // the last releases of every stage (MMA commits multicast to this CTA)
      for (int j = it; j < it + S2_STAGES && ok; ++j)
        if (!mbar_wait(empty_bar(j % S2_STAGES), ((uint32_t)(j / S2_STAGES) & 1) ^ 1, abort_flag, p.status)) ok = false;
    }
    if (!ok) {   // copies already issued land within microseconds: give them time (bounded)
      const unsigned long long t0 = globaltimer();
      while (globaltimer() - t0 < 50000ull) {
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------ MMA issuer (rank 0 for the pair)
    int it = 0, tc = 0;
    bool ok = true, issued = false;
    for (int t = cid; t < p.num_tiles && ok; t += ncl) {
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(tempty_bar(acc), (ar & 1) ^ 1, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
      const int kblocks = p.groups ? p.groups[p.tiles[t] & 0xFFFF].kblocks : p.kblocks;
      for (int kb = 0; kb < kblocks; ++kb, ++it) {
        const int s = it % S2_STAGES;
        const uint32_t r = (uint32_t)(it / S2_STAGES);
        if (!mbar_wait(full_bar(s), r & 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(smem + s * S2_STAGE);
        const uint64_t adesc = smem_desc(a_addr);
        const uint64_t bdesc = smem_desc(a_addr + S2_HALF);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16_pair(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc, (kb | kk) != 0);
        issued = true;
        mma_commit_pair(empty_bar(s));
      }
      if (!ok) break;
      mma_commit_pair(tfull_bar(acc));
    }
    if (!ok && issued) {
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain_bar)
                   : "memory");
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue (both CTAs: 128 rows each; two
    // warps per TMEM lane quarter, 128 columns each)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row_in_tile = q * 32 + lane;
    uint32_t* xt = reinterpret_cast<uint32_t*>(reinterpret_cast<uint8_t*>(bars) + 256) + (warp - 2) * S2_XT_WORDS;
    int tc = 0;
    for (int t = cid; t < p.num_tiles; t += ncl) {
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(tfull_bar(acc), ar & 1, abort_flag, p.status)) break;
      tc_fence_after();
      const Sq2Tile tq = sq2_tile(p, &tmL, p.tiles[t]);
      const int r = tq.I * 256 + (int)rank * 128 + row_in_tile;
      const uint32_t taddr = tmem_base + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
      for (int c = half * 4; c < half * 4 + 4; ++c) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(c * 32), v);   // every warp loads (.sync.aligned), in range or not
        const int col0 = tq.J * 256 + c * 32;
        if (r - lane < tq.npad && col0 < tq.npad) {   // the warp's 32 rows and 32 columns are all in or all out
          if (tq.I != tq.J)
            square_store32_staged(tq.out, tq.npad, r - lane, col0, lane, v, xt);
          else
            square_store32_diag(tq.out, tq.npad, r - lane, col0, lane, v, xt);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_bar0 + 8u * (2 * S2_STAGES + 2 + acc));
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // neither CTA leaves (or frees TMEM) while the pair still works
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(S2_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- chain application on CTA pairs
// x <- level x for one level, as k_tc_gemm's apply mode computes it (float
// partial products per split of K, summed by the update kernel), with
// tcgen05.mma.cta_group::2: the two CTAs of a cluster compute a 256-row block
// of one split, each CTA's 128 rows in its TMEM. Per 64-wide k-block CTA rank
// r stages its 128 rows of the level (16 KB) and rows r bn / 2 .. (r + 1)
// bn / 2 of the right-hand-side operand (the pair's B operand is split
// between the two CTAs, at most 16 KB), so a stage is at most 32 KB and six
// stages fit: twice the level bytes in flight of the one-CTA kernel's four
// 48 KB stages (the level streams from HBM). Barriers as in k_tc_sq2.
struct Apply2Params {
  int num_units;   // 256-row blocks x splits (block-major)
  int splits;
  int kblocks;     // k-blocks per split
  int npad;
  int bn;          // N = 2 kp (hi and lo halves of the right-hand sides)
  uint32_t idesc;  // kind::f16, M = 256, N = bn
  float* out;      // splits x npad x bn partial products
  unsigned* status;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(S2_THREADS, 1)
    k_tc_apply2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const Apply2Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S2_STAGES * S2_STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + S2_NBARS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + S2_NBARS + 1);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (S2_STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * S2_STAGES + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * S2_STAGES + 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const int cid = blockIdx.x >> 1, ncl = gridDim.x >> 1;
  const uint32_t lead_bar0 = mapa_rank(bar0, 0);   // the rank-0 CTA's barriers, cluster addresses
  const int bhalf = p.bn / 2;
  const uint32_t b_bytes = (uint32_t)bhalf * 128;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S2_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(bar0 + 8u * (2 * S2_STAGES + 2 + a), 16);   // tempty: the eight epilogue warps of each CTA
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {   // one warp of each CTA allocates the pair's TMEM
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S2_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  cluster_sync_all();   // both CTAs' barriers initialised before any remote signal
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer (both CTAs)
    int it = 0;
    bool ok = true;
    for (int u = cid; u < p.num_units && ok; u += ncl) {
      const int m = u / p.splits, split = u % p.splits;
      const int a_row = m * 256 + (int)rank * 128, b_row = (int)rank * bhalf;
      for (int kb = 0; kb < p.kblocks; ++kb, ++it) {
        const int s = it % S2_STAGES;
        if (!mbar_wait(empty_bar(s), ((uint32_t)(it / S2_STAGES) & 1) ^ 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        if (rank == 0) mbar_expect_tx(full_bar(s), 2 * (S2_HALF + b_bytes));   // both CTAs' copies
        const uint32_t dst = smem_u32(smem + s * S2_STAGE);
        const uint32_t fb = lead_bar0 + 8u * s;
        const int kx = (split * p.kblocks + kb) * BK;
        tma_load_2d_pair(dst, &tmA, kx, a_row, fb);
        tma_load_2d_pair(dst + S2_HALF, &tmB, kx, b_row, fb);
      }
    }
    if (ok) {
      // the last releases of every stage (MMA commits multicast to this CTA)
      for (int j = it; j < it + S2_STAGES && ok; ++j)
        if (!mbar_wait(empty_bar(j % S2_STAGES), ((uint32_t)(j / S2_STAGES) & 1) ^ 1, abort_flag, p.status)) ok = false;
    }
    if (!ok) {   // copies already issued land within microseconds: give them time (bounded)
      const unsigned long long t0 = globaltimer();
      while (globaltimer() - t0 < 50000ull) {
      }
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ------------------------------------------------ MMA issuer (rank 0 for the pair)
    int it = 0, tc = 0;
    bool ok = true, issued = false;
    for (int u = cid; u < p.num_units && ok; u += ncl) {
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(bar0 + 8u * (2 * S2_STAGES + 2 + acc), (ar & 1) ^ 1, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
      for (int kb = 0; kb < p.kblocks; ++kb, ++it) {
        const int s = it % S2_STAGES;
        if (!mbar_wait(full_bar(s), (uint32_t)(it / S2_STAGES) & 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(smem + s * S2_STAGE);
        const uint64_t adesc = smem_desc(a_addr);
        const uint64_t bdesc = smem_desc(a_addr + S2_HALF);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          mma_bf16_pair(d_tmem, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc, (kb | kk) != 0);
        issued = true;
        mma_commit_pair(empty_bar(s));
      }
      if (!ok) break;
      mma_commit_pair(tfull_bar(acc));
    }
    if (!ok && issued) {
      asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(drain_bar)
                   : "memory");
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue (both CTAs: 128 rows each; two
    // warps per TMEM lane quarter, half of the columns each)
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    const int row_in_tile = q * 32 + lane;
    const int nchunk = p.bn / 64;   // 32-column chunks per warp
    int tc = 0;
    for (int u = cid; u < p.num_units; u += ncl) {
      const int acc = tc & 1;
      const uint32_t ar = (uint32_t)(tc >> 1);
      ++tc;
      if (!mbar_wait(tfull_bar(acc), ar & 1, abort_flag, p.status)) break;
      tc_fence_after();
      const int m = u / p.splits, split = u % p.splits;
      const int r = m * 256 + (int)rank * 128 + row_in_tile;
      const uint32_t taddr = tmem_base + (uint32_t)(acc * 256) + ((uint32_t)(q * 32) << 16);
      float* P = p.out + ((size_t)split * p.npad + r) * p.bn;
      const bool in = r - lane < p.npad;   // the warp's 32 rows are all in or all past the padded order
      for (int c = half * nchunk; c < half * nchunk + nchunk; ++c) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(c * 32), v);   // every warp loads (.sync.aligned)
        if (in) {
          float4* dst = reinterpret_cast<float4*>(P + c * 32);
#pragma unroll
          for (int e = 0; e < 8; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(lead_bar0 + 8u * (2 * S2_STAGES + 2 + acc));
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync_all();   // neither CTA leaves (or frees TMEM) while the pair still works
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(S2_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------- e4m3 squaring, hardware block scaling
// S~^2 for an e4m3 level with one power-of-two scale 2^e per 128 x 128 tile,
// on tcgen05.mma kind::mxf8f6f4 with block scaling: the tensor core applies
// the e8m0 scale of each operand's 32-element K block itself, so the whole
// K range accumulates in one float32 TMEM accumulator (no per-K-tile
// promotion in the epilogue). A tile's 128 rows share one scale per 128-wide
// K tile, so every scale byte of an A operand K tile is e(I, K); the 256
// columns of a B operand take e(J0, K) for the first 128 and e(J1, K) for the
// second (the level is symmetric: e(K, J) = e(J, K)). The scales sit in
// global memory as 512-byte atoms, one per tile, every byte the tile's e8m0
// exponent; each pipeline stage brings the A atom and the two B atoms with
// its operand tiles (bulk copies on the same barrier), and the MMA issuer
// moves them into a TMEM ring (tcgen05.cp 32x128b, replicated to the four
// lane quarters) right before the stage's MMAs. An atom's bytes are all
// equal, so where the MMA reads inside an atom does not matter; which atom
// covers which 128 columns of B does, and the exact-product test checks it.
// The epilogue drains the accumulator into registers at once (one buffer:
// TMEM holds it plus the scale ring), then forms each output tile's
// power-of-two scale from its maximum, stores e4m3 and the bf16 copy (both
// mirrored), the float scales and the output level's atoms.
constexpr int M8_STAGES = 4;
constexpr int M8_SF = 512;                            // one scale atom: 32 rows x 16 bytes
constexpr int M8_OPS = M8_STAGES * T8_STAGE_BYTES;    // operand tiles (1024-aligned stages)
constexpr int M8_SFB = 3 * M8_SF;                     // atoms per stage: A, B0, B1
constexpr int M8_SMEM_BYTES = M8_OPS + M8_STAGES * M8_SFB + 512 + 1024;
constexpr int M8_TMEM_COLS = 512;                     // accumulator [0, 256) + scale ring [256, 320)
constexpr int M8_SF_COL = 256;
constexpr int M8_SF_SLOT = 16;                        // TMEM columns per stage: A at +0, B at +4 .. +11

struct Mx8Params {
  const uint32_t* tiles;   // square tile descriptors (as for the bf16 squaring)
  int num_tiles;
  int nt;                  // npad / 128
  int npad;
  uint8_t* out8;
  __nv_bfloat16* out16;
  const uint8_t* atoms_in;  // nt x nt atoms of the input level
  uint8_t* atoms_out;       // nt x nt atoms of the output level
  float* sout;              // nt x nt float scales (2^e) of the output level
  uint32_t idesc[4];        // per K step of a K tile (scale byte id = step)
  unsigned* status;
};

// Least e with amax <= 448 * 2^e (448 = largest finite e4m3), in [-126, 126];
// 0 for amax = 0. From the bits of amax = m 2^x (1 <= m < 2): 448 = 1.75 * 2^8,
// so e = x - 8 when m <= 1.75, else x - 7.
__device__ __forceinline__ int fp8_tile_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  const unsigned b = __float_as_uint(amax);
  const unsigned ef = (b >> 23) & 255u;
  if (ef == 0) return -126;   // subnormal amax: 448 * 2^-126 covers it
  const int x = (int)ef - 127;
  const int e = (b & 0x7FFFFFu) <= 0x600000u ? x - 8 : x - 7;
  return max(-126, min(126, e));
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory descriptor of a scale atom for tcgen05.cp: no swizzle, 8-row
// core matrices of 16-byte rows, 128 bytes apart.
__device__ __forceinline__ uint64_t atom_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(128 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void sf_copy(uint32_t taddr, uint64_t sdesc) {
  asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}

__device__ __forceinline__ void mma_mx8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t sfa, uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(T8_THREADS, 1)
    k_tc_mx8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Mx8Params p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sf_smem = smem + M8_OPS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sf_smem + M8_STAGES * M8_SFB);
  // bars[0..S) full, [S..2S) empty, [2S] accumulator full, [2S+1] accumulator empty, [2S+2] drain
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * M8_STAGES + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * M8_STAGES + 5);
  float* red = reinterpret_cast<float*>(bars + 2 * M8_STAGES + 6);   // [2 output tiles][8 warps]
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (M8_STAGES + s); };
  const uint32_t afull_bar = bar0 + 8u * (2 * M8_STAGES);
  const uint32_t aempty_bar = bar0 + 8u * (2 * M8_STAGES + 1);
  const uint32_t drain_bar = bar0 + 8u * (2 * M8_STAGES + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nt = p.nt;

  if (threadIdx.x == 0) {
    for (int s = 0; s < M8_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    mbar_init(afull_bar, 1);
    mbar_init(aempty_bar, T8_EPI);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(M8_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ------------------------------------------------ TMA producer: operand tiles and scale atoms
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x) {
      const uint32_t td = p.tiles[t];
      const int I = td & 0x7FFF, J = (td >> 15) & 0x7FFF, half = (td >> 30) & 1;
      const int R = 2 * I + half;
      for (int kb = 0; kb < nt; ++kb, ++it) {
        const int s = it % M8_STAGES;
        const uint32_t r = (uint32_t)(it / M8_STAGES);
        if (!mbar_wait(empty_bar(s), (r & 1) ^ 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t a_dst = smem_u32(smem + s * T8_STAGE_BYTES);
        const uint32_t f_dst = smem_u32(sf_smem + s * M8_SFB);
        mbar_expect_tx(full_bar(s), T8_STAGE_BYTES + M8_SFB);
        tma_load_2d(a_dst, &tmA, kb * 128, R * 128, full_bar(s));
        tma_load_2d(a_dst + T8_A, &tmB, kb * 128, J * 256, full_bar(s));
        bulk_load(f_dst, p.atoms_in + ((size_t)R * nt + kb) * M8_SF, M8_SF, full_bar(s));
        bulk_load(f_dst + M8_SF, p.atoms_in + ((size_t)(2 * J) * nt + kb) * M8_SF, M8_SF, full_bar(s));
        bulk_load(f_dst + 2 * M8_SF, p.atoms_in + ((size_t)(2 * J + 1) * nt + kb) * M8_SF, M8_SF, full_bar(s));
      }
    }
    if (!ok) {
      for (int j = (it > M8_STAGES ? it - M8_STAGES : 0); j < it; ++j) {
        const unsigned long long t0 = globaltimer();
        while (!mbar_try_wait(full_bar(j % M8_STAGES), (uint32_t)(j / M8_STAGES) & 1) &&
               globaltimer() - t0 < WAIT_LIMIT_NS) {
        }
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------------------------ MMA issuer: the whole K range into one accumulator
    int it = 0, tc = 0;
    bool ok = true, issued = false;
    for (int t = blockIdx.x; t < p.num_tiles && ok; t += gridDim.x, ++tc) {
      if (!mbar_wait(aempty_bar, ((uint32_t)tc & 1) ^ 1, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int kb = 0; kb < nt; ++kb, ++it) {
        const int s = it % M8_STAGES;
        if (!mbar_wait(full_bar(s), (uint32_t)(it / M8_STAGES) & 1, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a_addr = smem_u32(smem + s * T8_STAGE_BYTES);
        const uint32_t f_addr = smem_u32(sf_smem + s * M8_SFB);
        const uint32_t sf_t = tmem_base + (uint32_t)(M8_SF_COL + s * M8_SF_SLOT);
        sf_copy(sf_t, atom_desc(f_addr));                  // A: columns +0 .. +3
        sf_copy(sf_t + 4, atom_desc(f_addr + M8_SF));      // B columns 0-127: +4 .. +7
        sf_copy(sf_t + 8, atom_desc(f_addr + 2 * M8_SF));  // B columns 128-255: +8 .. +11
        const uint64_t adesc = smem_desc(a_addr);
        const uint64_t bdesc = smem_desc(a_addr + T8_A);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)   // 32 e4m3 (32 bytes, one scale block) per MMA
          mma_mx8(tmem_base, adesc + (uint64_t)(kk * 2), bdesc + (uint64_t)(kk * 2), p.idesc[kk], sf_t, sf_t + 4,
                  (kb | kk) != 0);
        issued = true;
        mma_commit(empty_bar(s));
      }
      if (!ok) break;
      mma_commit(afull_bar);
    }
    if (!ok && issued) {
      mma_commit(drain_bar);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(drain_bar, 0) && globaltimer() - t0 < WAIT_LIMIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ------------------------------------------------ epilogue: drain, scale, store
    const int q = warp & 3;                  // TMEM lane quarter
    const int cq = (warp - 2) >> 2;          // 64-column quarter of the 256 columns
    const int ob = cq >> 1;                  // output tile (0: first 128 columns, 1: second)
    const int row_in_tile = q * 32 + lane;
    const uint32_t lane_off = (uint32_t)(q * 32) << 16;
    const int np = p.npad;
    int tc = 0;
    // The epilogue warps of an output tile meet at a named barrier per tile,
    // so they walk the same tiles whatever happens: after a failed (expired
    // or aborted) wait a warp stops loading and storing but keeps the barrier
    // count, and every later wait returns at once because the abort flag is set.
    bool failed = false;
    for (int t = blockIdx.x; t < p.num_tiles; t += gridDim.x, ++tc) {
      const uint32_t td = p.tiles[t];
      const int I = td & 0x7FFF, J = (td >> 15) & 0x7FFF, half = (td >> 30) & 1;
      const int R = 2 * I + half, C = 2 * J + ob;   // output 128-block
      float acc[T8_COLS];
#pragma unroll
      for (int c = 0; c < T8_COLS; ++c) acc[c] = 0.f;
      if (!failed) {
        if (!mbar_wait(afull_bar, (uint32_t)tc & 1, abort_flag, p.status)) {
          failed = true;
        } else {
          tc_fence_after();
#pragma unroll
          for (int c = 0; c < T8_COLS / 16; ++c) {
            float v[16];
            tmem_ld16(tmem_base + lane_off + (uint32_t)(cq * T8_COLS + c * 16), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[c * 16 + e] = v[e];
          }
          tc_fence_before();
          mbar_arrive(aempty_bar);
        }
      }
      float m = 0.f;
#pragma unroll
      for (int c = 0; c < T8_COLS; ++c) m = fmaxf(m, fabsf(acc[c]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const int slot = ob * 8 + (q + 4 * (cq & 1));
      if (lane == 0) red[slot] = m;
      if (ob == 0)
        asm volatile("bar.sync 1, 256;" ::: "memory");
      else
        asm volatile("bar.sync 2, 256;" ::: "memory");
      float amax = 0.f;
#pragma unroll
      for (int w = 0; w < 8; ++w) amax = fmaxf(amax, red[ob * 8 + w]);
      if (ob == 0)
        asm volatile("bar.sync 1, 256;" ::: "memory");
      else
        asm volatile("bar.sync 2, 256;" ::: "memory");
      if (failed || R > C) continue;   // R > C: the mirror of (C, R), written by the other half
      const int e = fp8_tile_exp(amax);
      const float scale = __int_as_float((e + 127) << 23);
      const float inv = __int_as_float((127 - e) << 23);
      const int r = R * 128 + row_in_tile;
      const int col0 = C * 128 + (cq & 1) * T8_COLS;
      uint8_t* C8 = p.out8;
      __nv_bfloat16* C16 = p.out16;
      if (R != C) {
#pragma unroll
        for (int c = 0; c < T8_COLS / 16; ++c) {   // 16 columns per 16-byte store
          uint32_t w8[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            uint32_t wv = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f)
              wv |= (uint32_t)__nv_cvt_float_to_fp8(acc[c * 16 + g * 4 + f] * inv, __NV_SATFINITE, __NV_E4M3)
                    << (8 * f);
            w8[g] = wv;
          }
          *reinterpret_cast<uint4*>(C8 + (size_t)r * np + col0 + c * 16) = make_uint4(w8[0], w8[1], w8[2], w8[3]);
        }
#pragma unroll
        for (int c = 0; c < T8_COLS / 8; ++c) {   // 8 columns per 16-byte store
          uint32_t w[4];
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            __nv_bfloat162 hh = __floats2bfloat162_rn(acc[c * 8 + 2 * g], acc[c * 8 + 2 * g + 1]);
            w[g] = *reinterpret_cast<uint32_t*>(&hh);
          }
          *reinterpret_cast<uint4*>(C16 + (size_t)r * np + col0 + c * 8) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        {   // mirrored tile: lanes write consecutive rows of a column
          uint8_t* m8 = C8 + (size_t)col0 * np + r;
          __nv_bfloat16* m16 = C16 + (size_t)col0 * np + r;
#pragma unroll
          for (int c = 0; c < T8_COLS; ++c) {
            m8[(size_t)c * np] = (uint8_t)__nv_cvt_float_to_fp8(acc[c] * inv, __NV_SATFINITE, __NV_E4M3);
            m16[(size_t)c * np] = __float2bfloat16_rn(acc[c]);
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < T8_COLS; ++c) {
          const int col = col0 + c;
          const uint8_t q8 = (uint8_t)__nv_cvt_float_to_fp8(acc[c] * inv, __NV_SATFINITE, __NV_E4M3);
          const __nv_bfloat16 hv = __float2bfloat16_rn(acc[c]);
          if (col >= r) {
            C8[(size_t)r * np + col] = q8;
            C16[(size_t)r * np + col] = hv;
          }
          if (col > r) {
            C8[(size_t)col * np + r] = q8;
            C16[(size_t)col * np + r] = hv;
          }
        }
      }
      if (q == 0 && (cq & 1) == 0) {   // one warp per output tile: scales and atoms
        const uint32_t wb = (uint32_t)(e + 127) * 0x01010101u;
        const uint4 atom = make_uint4(wb, wb, wb, wb);
        *reinterpret_cast<uint4*>(p.atoms_out + ((size_t)R * nt + C) * M8_SF + lane * 16) = atom;
        *reinterpret_cast<uint4*>(p.atoms_out + ((size_t)C * nt + R) * M8_SF + lane * 16) = atom;
        if (lane == 0) {
          p.sout[R * nt + C] = scale;
          p.sout[C * nt + R] = scale;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(M8_TMEM_COLS)
                 : "memory");
  }
}

// Level 0 of a per-tile e4m3 chain from its bf16 copy: one block per 128 x
// 128 tile; scale = the least power of two 2^e with tile max <= 448 * 2^e,
// stored as a float and as the tile's 512-byte atom of e8m0 bytes.
__global__ void __launch_bounds__(256) k_quant_fp8_tiles(const __nv_bfloat16* __restrict__ L16, int np,
                                                          uint8_t* __restrict__ L8, float* __restrict__ scales,
                                                          uint8_t* __restrict__ atoms) {
  __shared__ float red[8];
  const int nt = np / 128;
  const int I = blockIdx.x / nt, J = blockIdx.x % nt;
  float m = 0.f;
  for (int e = threadIdx.x; e < 128 * 128; e += 256) {
    const int r = I * 128 + e / 128, c = J * 128 + e % 128;
    m = fmaxf(m, fabsf(__bfloat162float(L16[(size_t)r * np + c])));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  float amax = 0.f;
  for (int w = 0; w < 8; ++w) amax = fmaxf(amax, red[w]);
  const int ex = fp8_tile_exp(amax);
  const float scale = __int_as_float((ex + 127) << 23);
  const float inv = __int_as_float((127 - ex) << 23);
  for (int e = threadIdx.x; e < 128 * 128; e += 256) {
    const size_t o = (size_t)(I * 128 + e / 128) * np + J * 128 + e % 128;
    L8[o] = (uint8_t)__nv_cvt_float_to_fp8(__bfloat162float(L16[o]) * inv, __NV_SATFINITE, __NV_E4M3);
  }
  if (threadIdx.x == 0) scales[I * nt + J] = scale;
  if (threadIdx.x < 32) {
    const uint32_t wb = (uint32_t)(ex + 127) * 0x01010101u;
    *reinterpret_cast<uint4*>(atoms + ((size_t)I * nt + J) * M8_SF + threadIdx.x * 16) = make_uint4(wb, wb, wb, wb);
  }
}

// ---------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D tensor map over a rows x cols row-major matrix of bf16 (elem = 2) or
// fp8 bytes (elem = 1); box = one 128-byte row segment x box_rows.
// 2-D tensor map of a row-major matrix (rows x cols, `stride` elements
// between rows, 0 = cols), 128-byte boxes of box_rows rows, 128-byte swizzle.
int make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int box_rows, int elem = 2,
             int64_t stride = 0) {
  auto fn = encode_fn();
  if (!fn) return CDL_ERR_UNSUPPORTED;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)(stride ? stride : cols) * elem};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, elem == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                  const_cast<void*>(base), gdim, gstride, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_last_error("cuTensorMapEncodeTiled failed", __FILE__, __LINE__);
    return CDL_ERR_CUDA;
  }
  return CDL_OK;
}

uint32_t make_idesc(int n, bool fp8 = false) {
  const uint32_t fmt = fp8 ? 0u : 1u;   // kind::f8f6f4: e4m3 = 0; kind::f16: bf16 = 1
  return (1u << 4)                      // D: float32
         | (fmt << 7)                   // A format
         | (fmt << 10)                  // B format
         | ((uint32_t)(n >> 3) << 17)   // N / 8
         | ((uint32_t)(BM >> 4) << 24); // M / 16
}

// Upper-triangle 256-blocks in 8 x 8 super-block groups (L2 reuse), both
// 128-row halves of a block adjacent.
std::vector<uint32_t> square_tiles(int nb) {
  std::vector<uint32_t> v;
  const int G = 8;
  for (int P = 0; P < nb; P += G)
    for (int Q = P; Q < nb; Q += G)
      for (int I = P; I < std::min(P + G, nb); ++I)
        for (int J = std::max(Q, I); J < std::min(Q + G, nb); ++J)
          for (int h = 0; h < 2; ++h) v.push_back((uint32_t)I | ((uint32_t)J << 15) | ((uint32_t)h << 30));
  return v;
}

// Upper-triangle 256-blocks for the CTA-pair kernel, in the same 8 x 8
// super-block order (one entry per block).
std::vector<uint32_t> square_pair_tiles(int nb) {
  std::vector<uint32_t> v;
  const int G = 8;
  for (int P = 0; P < nb; P += G)
    for (int Q = P; Q < nb; Q += G)
      for (int I = P; I < std::min(P + G, nb); ++I)
        for (int J = std::max(Q, I); J < std::min(Q + G, nb); ++J) v.push_back((uint32_t)I | ((uint32_t)J << 15));
  return v;
}

std::vector<uint32_t> apply_tiles(int mb, int splits) {
  std::vector<uint32_t> v;
  for (int s = 0; s < splits; ++s)
    for (int m = 0; m < mb; ++m) v.push_back((uint32_t)m | ((uint32_t)s << 16));
  return v;
}

// Device copy of a tile schedule, built once per (kind, sizes) and kept in
// the context's workspace under a name that encodes those sizes.
template <typename Builder>
int get_tiles(cdl_ctx* ctx, const std::string& name, Builder build, const uint32_t** out, int* count) {
  auto it = ctx->tile_lists.find(name);
  if (it != ctx->tile_lists.end() && ctx->ws.count(name)) {
    *out = static_cast<const uint32_t*>(ctx->ws[name].first);
    *count = it->second;
    return CDL_OK;
  }
  std::vector<uint32_t> tiles = build();
  void* buf;
  CDL_TRY(ws_get(ctx, name.c_str(), tiles.size() * sizeof(uint32_t), &buf));
  CDL_CUDA_TRY(cudaMemcpyAsync(buf, tiles.data(), tiles.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  CDL_CUDA_TRY(cudaStreamSynchronize(ctx->stream));   // the host vector goes out of scope
  ctx->tile_lists[name] = (int)tiles.size();
  *out = static_cast<const uint32_t*>(buf);
  *count = (int)tiles.size();
  return CDL_OK;
}

int launch(cdl_ctx* ctx, const CUtensorMap& a, const CUtensorMap& b, const TcParams& p, int kc,
           double work, bool fp8 = false) {
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr = true;
  }
  const int grid = std::min(p.num_tiles, ctx->sm_count);
  Launch L(ctx, kc, work);
  if (fp8)
    k_tc_gemm<true><<<grid, THREADS, SMEM_BYTES, ctx->stream>>>(a, b, p);
  else
    k_tc_gemm<false><<<grid, THREADS, SMEM_BYTES, ctx->stream>>>(a, b, p);
  return L.done();
}

}  // namespace

bool tc_supported(cdl_ctx* ctx) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

// Grouped CTA-pair squaring: the 256-blocks holding rows of each graph
// (largest graphs first), as graph | I << 16 | J << 23.
std::vector<uint32_t> pair_tiles_grouped(const std::vector<int>& npad, const std::vector<int>& n) {
  std::vector<int> order(npad.size());
  for (size_t g = 0; g < order.size(); ++g) order[g] = (int)g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return npad[a] > npad[b]; });
  std::vector<uint32_t> v;
  for (int g : order) {
    const int nb = (n[g] + 255) / 256;
    for (int I = 0; I < nb; ++I)
      for (int J = I; J < nb; ++J) v.push_back((uint32_t)g | ((uint32_t)I << 16) | ((uint32_t)J << 23));
  }
  return v;
}

// kind::f16 instruction descriptor for the CTA-pair MMA (M = 256)
uint32_t make_idesc_m256(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(256 >> 4) << 24);
}

// Clusters of two that can be resident at once (0: cluster launch unavailable).
int pair_clusters(cdl_ctx* ctx) {
  static int max_clusters = -1;
  if (max_clusters < 0) {
    if (cudaFuncSetAttribute(k_tc_sq2, cudaFuncAttributeMaxDynamicSharedMemorySize, S2_SMEM_BYTES) != cudaSuccess) {
      cudaGetLastError();
      max_clusters = 0;
      return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * (ctx->sm_count / 2), 1, 1);
    cfg.blockDim = dim3(S2_THREADS, 1, 1);
    cfg.dynamicSmemBytes = S2_SMEM_BYTES;
    int mc = 0;
    if (cudaOccupancyMaxActiveClusters(&mc, k_tc_sq2, &cfg) != cudaSuccess) {
      cudaGetLastError();
      mc = 0;
    }
    max_clusters = std::max(mc, 0);
  }
  return max_clusters;
}

// bf16 squaring of a level on CTA pairs (k_tc_sq2)
int square_pairs(cdl_ctx* ctx, const void* in, void* out, int np, double flops, int clusters_max) {
  const int nb = np / 256;
  const uint32_t* tiles;
  int count;
  CDL_TRY(get_tiles(ctx, "tc.sq2." + std::to_string(nb), [&] { return square_pair_tiles(nb); }, &tiles, &count));
  CUtensorMap ml;
  CDL_TRY(make_map(&ml, in, np, np, 128));
  Sq2Params p{};
  p.tiles = tiles;
  p.num_tiles = count;
  p.kblocks = np / BK;
  p.npad = np;
  p.idesc = make_idesc_m256(256);
  p.out = static_cast<__nv_bfloat16*>(out);
  p.status = ctx->dev_status;
  p.debug_withhold_load = ctx->debug_flags & 1;
  const int clusters = std::min(count, clusters_max);
  if (p.kblocks >= S2_PACE_MIN_KBLOCKS) {
    const int steps_per_tile = (p.kblocks + PACE_KB - 1) / PACE_KB;
    p.pace_steps = ((count + clusters - 1) / clusters) * steps_per_tile;
    void* pb;
    CDL_TRY(ws_get(ctx, "tc.pace", (size_t)p.pace_steps * sizeof(unsigned), &pb));
    CDL_CUDA_TRY(cudaMemsetAsync(pb, 0, (size_t)p.pace_steps * sizeof(unsigned), ctx->stream));
    p.pace = static_cast<unsigned*>(pb);
  }
  Launch L(ctx, CDL_KC_SQUARE, flops);
  k_tc_sq2<<<2 * clusters, S2_THREADS, S2_SMEM_BYTES, ctx->stream>>>(ml, p);
  return L.done();
}

int tc_square_grouped_pairs(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups,
                            const uint32_t* dtiles, int ntiles, double flops) {
  const int mc = pair_clusters(ctx);
  if (mc < 1) return CDL_ERR_UNSUPPORTED;
  Sq2Params p{};
  p.tiles = dtiles;
  p.num_tiles = ntiles;
  p.groups = dgroups;
  p.idesc = make_idesc_m256(256);
  p.status = ctx->dev_status;
  const int clusters = std::min(ntiles, mc);
  Launch L(ctx, CDL_KC_SQUARE, flops);
  // the kernel-parameter map is unused in grouped mode: pass the first graph's
  k_tc_sq2<<<2 * clusters, S2_THREADS, S2_SMEM_BYTES, ctx->stream>>>(host_first->mapA, p);
  return L.done();
}

int chain_square_tc(cdl_ctx* ctx, cdl_chain* ch, int level) {
  const int np = (int)ch->npad;
  const int nb = np / 256;
  const uint32_t* tiles;
  int count;
  CDL_TRY(get_tiles(ctx, "tc.square." + std::to_string(nb), [&] { return square_tiles(nb); }, &tiles, &count));
  const bool fp8 = ch->dtype == CDL_FP8E4M3;
  const int elem = fp8 ? 1 : 2;
  const void* in = ch->level(level);
  void* out = ch->level(level + 1);
  if (ch->host_levels) {   // level `level` is in a slot (just written); level + 1 goes to the other
    in = ooc_read(ctx, ch, level);
    out = ooc_write_begin(ctx, ch, level + 1);
    if (!in) return CDL_ERR_CUDA;
  }
  const int clusters = fp8 ? 0 : pair_clusters(ctx);
  if (clusters > 0) {   // bf16: CTA pairs
    CDL_TRY(square_pairs(ctx, in, out, np, (double)ch->n * ch->n * (ch->n + 1.0), clusters));
    return ch->host_levels ? ooc_write_end(ctx, ch, level + 1) : CDL_OK;
  }
  CUtensorMap ma, mb;
  CDL_TRY(make_map(&ma, in, np, np, 128, elem));
  CDL_TRY(make_map(&mb, in, np, np, 256, elem));
  TcParams p{};
  p.tiles = tiles;
  p.num_tiles = count;
  p.kblocks = np / (128 / elem);
  p.bn = 256;
  p.idesc = make_idesc(256, fp8);
  p.mode = fp8 ? MODE_SQUARE_FP8 : MODE_SQUARE;
  p.npad = np;
  p.out = out;
  p.ldo = np;
  p.status = ctx->dev_status;
  p.amax = ch->amax;
  p.level = level;
  p.out16 = fp8 ? ch->level16(level + 1) : nullptr;
  p.debug_withhold_load = ctx->debug_flags & 1;
  p.groups = nullptr;
  p.pace = nullptr;
  p.pace_steps = 0;
  if (p.kblocks >= PACE_MIN_KBLOCKS) {
    const int grid = std::min(p.num_tiles, ctx->sm_count);
    p.pace_steps = ((p.num_tiles + grid - 1) / grid) * ((p.kblocks + PACE_KB - 1) / PACE_KB);
    void* pb;
    CDL_TRY(ws_get(ctx, "tc.pace", (size_t)p.pace_steps * sizeof(unsigned), &pb));
    CDL_CUDA_TRY(cudaMemsetAsync(pb, 0, (size_t)p.pace_steps * sizeof(unsigned), ctx->stream));
    p.pace = static_cast<unsigned*>(pb);
  }
  const double flops = (double)ch->n * ch->n * (ch->n + 1.0);
  CDL_TRY(launch(ctx, ma, mb, p, CDL_KC_SQUARE, flops, fp8));
  return ch->host_levels ? ooc_write_end(ctx, ch, level + 1) : CDL_OK;
}

int tc_group_square(TcGroup* g, const void* level, void* out, int np, int bn, int n) {
  std::memset(g, 0, sizeof(TcGroup));
  if ((bn != 128 && bn != 256) || np % bn || np > 32768 || n < 1 || n > np) return CDL_ERR_INVALID_ARG;
  CDL_TRY(make_map(&g->mapA, level, np, np, 128));
  CDL_TRY(make_map(&g->mapB, level, np, np, bn));
  g->out = out;
  g->npad = np;
  g->kblocks = (n + BK - 1) / BK;   // k-blocks past n hold only zero padding
  g->bn = bn;
  g->idesc = make_idesc(bn);
  return CDL_OK;
}

int tc_group_apply(TcGroup* g, const void* amat, const void* xop, float* out, int np, int kp, const int* gate) {
  std::memset(g, 0, sizeof(TcGroup));
  const int bn = 2 * kp;
  if (np % 128 || np / 128 > 0x7FFF || bn % 32 || bn > MAX_BN) return CDL_ERR_INVALID_ARG;
  CDL_TRY(make_map(&g->mapA, amat, np, np, 128));
  CDL_TRY(make_map(&g->mapB, xop, bn, np, bn));
  g->out = out;
  g->gate = gate;
  g->npad = np;
  g->kblocks = np / BK;
  g->bn = bn;
  g->idesc = make_idesc(bn);
  return CDL_OK;
}

// Upper-triangle blocks of every graph (256-blocks as two 128 x 256 tiles,
// or 128 x 128 tiles), graphs ordered largest first.
std::vector<uint32_t> tc_grouped_square_tiles(const std::vector<int>& npad, const std::vector<int>& n,
                                              const std::vector<int>& bn) {
  std::vector<int> order(npad.size());
  for (size_t g = 0; g < order.size(); ++g) order[g] = (int)g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return npad[a] > npad[b]; });
  std::vector<uint32_t> v;
  // only tiles with a row of the graph (rows and columns past n are zero
  // padding in every level: the plan's memory starts zeroed and no tile
  // writes there)
  for (int g : order) {
    if (bn[g] == 128) {
      const int nb = (n[g] + 127) / 128;
      for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J) v.push_back((uint32_t)g | ((uint32_t)I << 16) | ((uint32_t)J << 24));
    } else {
      const int nb = (n[g] + 255) / 256;
      for (int I = 0; I < nb; ++I)
        for (int J = I; J < nb; ++J)
          for (int h = 0; h < 2; ++h)
            if (I * 256 + h * 128 < n[g])
              v.push_back((uint32_t)g | ((uint32_t)I << 16) | ((uint32_t)J << 23) | ((uint32_t)h << 30));
    }
  }
  return v;
}

// 128-row blocks of every graph, largest graphs (longest k loops) first.
std::vector<uint32_t> tc_grouped_apply_tiles(const std::vector<int>& npad) {
  std::vector<int> order(npad.size());
  for (size_t g = 0; g < order.size(); ++g) order[g] = (int)g;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return npad[a] > npad[b]; });
  std::vector<uint32_t> v;
  for (int g : order)
    for (int m = 0; m < npad[g] / 128; ++m) v.push_back((uint32_t)g | ((uint32_t)m << 16));
  return v;
}

int tc_square_grouped(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups, const uint32_t* dtiles,
                      int ntiles, double flops) {
  TcParams p{};
  std::memset(&p, 0, sizeof(p));
  p.tiles = dtiles;
  p.num_tiles = ntiles;
  p.bn = 256;
  p.idesc = make_idesc(256);
  p.mode = MODE_SQUARE;
  p.status = ctx->dev_status;
  p.groups = dgroups;
  // the kernel-parameter maps are unused in grouped mode: pass the first graph's
  return launch(ctx, host_first->mapA, host_first->mapB, p, CDL_KC_SQUARE, flops);
}

int tc_apply_grouped(cdl_ctx* ctx, const TcGroup* host_first, const TcGroup* dgroups, const uint32_t* dtiles,
                     int ntiles, int kp, int gate_mask, int kc, double work) {
  TcParams p{};
  std::memset(&p, 0, sizeof(p));
  p.tiles = dtiles;
  p.num_tiles = ntiles;
  p.bn = 2 * kp;
  p.idesc = make_idesc(2 * kp);
  p.mode = MODE_APPLY;
  p.ldo = 2 * kp;
  p.status = ctx->dev_status;
  p.groups = dgroups;
  p.gate_mask = gate_mask;
  return launch(ctx, host_first->mapA, host_first->mapB, p, kc, work);
}

// Instruction descriptor of kind::mxf8f6f4 with block scaling: e4m3 A and B,
// K-major, float32 accumulator, e8m0 scales, scale byte `id` of A and B.
uint32_t make_idesc_mx8(int n, int id) {
  return ((uint32_t)id << 4)              // B scale byte
         | (0u << 7) | (0u << 10)         // A, B: e4m3
         | ((uint32_t)(n >> 3) << 17)     // N / 8
         | (1u << 23)                     // scales: ue8m0
         | ((uint32_t)(BM >> 4) << 24)    // M / 16
         | ((uint32_t)id << 29);          // A scale byte
}

int chain_square_fp8t(cdl_ctx* ctx, cdl_chain* ch, int level) {
  const int np = (int)ch->npad;   // multiple of 256
  const int nt = np / 128;
  const int nb = np / 256;
  const uint32_t* tiles;
  int count;
  CDL_TRY(get_tiles(ctx, "tc.square." + std::to_string(nb), [&] { return square_tiles(nb); }, &tiles, &count));
  CUtensorMap ma, mb;
  CDL_TRY(make_map(&ma, ch->level(level), np, np, 128, 1));
  CDL_TRY(make_map(&mb, ch->level(level), np, np, 256, 1));
  if (!ch->tatoms) return CDL_ERR_INVALID_ARG;
  {
    static bool mattr = false;
    if (!mattr) {
      CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_mx8, cudaFuncAttributeMaxDynamicSharedMemorySize, M8_SMEM_BYTES));
      mattr = true;
    }
    const size_t atoms = (size_t)nt * nt * M8_SF;
    Mx8Params p;
    std::memset(&p, 0, sizeof(p));
    p.tiles = tiles;
    p.num_tiles = count;
    p.nt = nt;
    p.npad = np;
    p.out8 = static_cast<uint8_t*>(ch->level(level + 1));
    p.out16 = static_cast<__nv_bfloat16*>(ch->level16(level + 1));
    p.atoms_in = ch->tatoms + (size_t)(level & 1) * atoms;
    p.atoms_out = ch->tatoms + (size_t)((level + 1) & 1) * atoms;
    p.sout = ch->tscale + (size_t)(level + 1) * nt * nt;
    for (int kk = 0; kk < 4; ++kk) p.idesc[kk] = make_idesc_mx8(256, kk);
    p.status = ctx->dev_status;
    const double flops = (double)ch->n * ch->n * (ch->n + 1.0);
    const int grid = std::min(count, ctx->sm_count);
    Launch L(ctx, CDL_KC_SQUARE, flops);
    k_tc_mx8<<<grid, T8_THREADS, M8_SMEM_BYTES, ctx->stream>>>(ma, mb, p);
    return L.done();
  }
}

int fp8t_quantize_level0(cdl_ctx* ctx, cdl_chain* ch) {
  const int np = (int)ch->npad;
  const int nt = np / 128;
  Launch L(ctx, CDL_KC_CHAIN_INIT, 3.0 * np * (double)np);
  k_quant_fp8_tiles<<<nt * nt, 256, 0, ctx->stream>>>(static_cast<const __nv_bfloat16*>(ch->level16(0)), np,
                                                      static_cast<uint8_t*>(ch->level(0)), ch->tscale, ch->tatoms);
  return L.done();
}

// A Z (A from its six slices in the chain, Z / c from `zslices`: six bf16
// planes kp x npad) into G (npad x kp float64, overwritten).
int resid_tc(cdl_ctx* ctx, const cdl_chain* ch, const void* zslices, int kp, double* G) {
  const int np = (int)ch->npad;
  if (kp % 32 || kp > 128 || np % 256) return CDL_ERR_INVALID_ARG;
  ResidMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int s = 0; s < RS_SLICES; ++s) {
    CDL_TRY(make_map(&maps.a[s], static_cast<const char*>(ch->aslices) + (size_t)s * np * np * 2, np, np, 128));
    CDL_TRY(make_map(&maps.b[s], static_cast<const char*>(zslices) + (size_t)s * kp * np * 2, kp, np, kp));
  }
  ResidParams p;
  std::memset(&p, 0, sizeof(p));
  p.num_tiles = np / 128;
  p.kblocks = np / 64;
  p.kp = kp;
  for (int m = 2; m <= RS_SLICES + 1; ++m)
    for (int sa = 1; sa < m; ++sa) {
      const int sz = m - sa;
      if (sa > RS_SLICES || sz > RS_SLICES) continue;
      p.pair_s[p.npairs] = sa;
      p.pair_t[p.npairs] = sz;
      ++p.npairs;
    }
  p.G = G;
  p.gstride = (size_t)np * kp;
  p.idesc = make_idesc(kp);
  p.status = ctx->dev_status;
  p.assign = 1;   // every element of every plane belongs to one unit: its first flush stores it
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_BYTES));
    attr = true;
  }
  const int grid = std::min(p.num_tiles * p.npairs, ctx->sm_count);
  Launch L(ctx, CDL_KC_RESIDUAL, 2.0 * p.npairs * (double)np * np * kp);
  k_tc_resid<<<grid, T8_THREADS, RS_SMEM_BYTES, ctx->stream>>>(maps, p);
  return L.done();
}

int resid_group_init(ResidGroup* g, const void* aslices, const void* zslices, double* G, int npad, int kg,
                     const int* gate) {
  std::memset(g, 0, sizeof(ResidGroup));
  if (kg % 32 || kg > 128 || npad % 128) return CDL_ERR_INVALID_ARG;
  for (int s = 0; s < RS_SLICES; ++s) {
    CDL_TRY(make_map(&g->a[s], static_cast<const char*>(aslices) + (size_t)s * npad * npad * 2, npad, npad, 128));
    CDL_TRY(make_map(&g->b[s], static_cast<const char*>(zslices) + (size_t)s * kg * npad * 2, kg, npad, kg));
  }
  g->G = G;
  g->gstride = (size_t)npad * kg;
  g->gate = gate;
  g->kblocks = (npad + 255) / 256 * 4;
  return CDL_OK;
}

int resid_tc_grouped(cdl_ctx* ctx, const ResidGroup* dgroups, const uint32_t* units, int nunits, int kg,
                     int gate_mask, double work) {
  if (kg % 32 || kg > 128) return CDL_ERR_INVALID_ARG;
  if (nunits == 0) return CDL_OK;
  ResidMaps maps;   // unused in grouped mode
  std::memset(&maps, 0, sizeof(maps));
  ResidParams p;
  std::memset(&p, 0, sizeof(p));
  p.num_tiles = nunits;
  p.kp = kg;
  for (int m = 2; m <= RS_SLICES + 1; ++m)
    for (int sa = 1; sa < m; ++sa) {
      const int sz = m - sa;
      if (sa > RS_SLICES || sz > RS_SLICES) continue;
      p.pair_s[p.npairs] = sa;
      p.pair_t[p.npairs] = sz;
      ++p.npairs;
    }
  p.idesc = make_idesc(kg);
  p.status = ctx->dev_status;
  p.groups = dgroups;
  p.units = units;
  p.gate_mask = gate_mask;
  p.assign = 1;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_BYTES));
    attr = true;
  }
  const int grid = std::min(nunits * p.npairs, ctx->sm_count);
  Launch L(ctx, CDL_KC_RESIDUAL, work);
  k_tc_resid<<<grid, T8_THREADS, RS_SMEM_BYTES, ctx->stream>>>(maps, p);
  return L.done();
}

namespace {
int dist_launch(cdl_ctx* ctx, const void* planes, int rows, int tp, DistParams& p, double terms) {
  DistMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int s = 0; s < DS_SLICES; ++s) {
    const char* base = static_cast<const char*>(planes) + (size_t)s * rows * tp * 2;
    CDL_TRY(make_map(&maps.a[s], base, rows, tp, 128));
    CDL_TRY(make_map(&maps.b[s], base, rows, tp, DS_N));
  }
  p.kblocks = tp / 64;
  p.idesc = make_idesc(DS_N);
  p.status = ctx->dev_status;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, DS_SMEM_BYTES));
    attr = true;
  }
  if (p.num_tiles <= 0) return CDL_OK;
  const int grid = std::min(p.num_tiles, ctx->sm_count);
  Launch L(ctx, CDL_KC_DISTANCE, terms);
  k_tc_dist<<<grid, T8_THREADS, DS_SMEM_BYTES, ctx->stream>>>(maps, p);
  return L.done();
}
}  // namespace

int dist_tc(cdl_ctx* ctx, const void* planes, const long long* norms, int n, int rows, int tp, double* A,
            const int* offgrid, double terms) {
  if (rows % 128 || tp % 64 || rows < n || tp < 64) return CDL_ERR_INVALID_ARG;
  DistParams p;
  std::memset(&p, 0, sizeof(p));
  p.nb128 = rows / 128;
  p.nb64 = 2 * p.nb128;
  const long long tiles = (long long)p.nb128 * p.nb64 - (long long)p.nb128 * (p.nb128 - 1);
  if (tiles > 0x7fffffffLL) return CDL_ERR_INVALID_ARG;
  p.num_tiles = (int)tiles;
  p.n = n;
  p.norms = norms;
  p.A = A;
  p.offgrid = offgrid;
  // algorithmic work: n (n - 1) T / 2 squared differences
  return dist_launch(ctx, planes, rows, tp, p, terms);
}

int dist_tc_panel(cdl_ctx* ctx, const void* planes, const long long* norms, int n, int rows, int tp, double* panel,
                  int row0, int prows, bool upper, const int* offgrid) {
  if (rows % 128 || tp % 64 || rows < n || tp < 64 || row0 % 128 || prows % 128 || prows <= 0 ||
      row0 + prows > rows)
    return CDL_ERR_INVALID_ARG;
  DistParams p;
  std::memset(&p, 0, sizeof(p));
  p.nb128 = rows / 128;
  p.nb64 = 2 * p.nb128;
  p.n = n;
  p.norms = norms;
  p.A = panel;
  p.offgrid = offgrid;
  p.panel = 1;
  p.row0 = row0;
  const int I0 = row0 / 128, PI = prows / 128;
  auto off = [&](long long I) { return I * p.nb64 - I * (I - 1); };   // first upper tile of row block I
  long long tiles;
  if (upper) {
    p.tile0 = off(I0);
    tiles = off(I0 + PI) - off(I0);
  } else {
    p.rect = PI;
    p.I0 = I0;
    tiles = (long long)PI * p.nb64;
  }
  if (tiles > 0x7fffffffLL) return CDL_ERR_INVALID_ARG;
  p.num_tiles = (int)tiles;
  const double terms = (double)tiles * 128.0 * DS_N * tp;
  return dist_launch(ctx, planes, rows, tp, p, terms);
}

int resid_tc_panel(cdl_ctx* ctx, const void* slicesT, int np, int Pw, int Pk, int c0, const void* zslices, int kp,
                   double* G) {
  if (kp % 32 || kp > 128 || np % 256 || Pw % 256 || Pk % 256 || Pk <= 0 || Pk > Pw || c0 % 64 || c0 + Pk > np)
    return CDL_ERR_INVALID_ARG;
  ResidMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int s = 0; s < RS_SLICES; ++s) {
    // A operand: the panel's Pk columns of rows 0 .. np - 1 (the transposed panel slices, np x Pw planes)
    CDL_TRY(make_map(&maps.a[s], static_cast<const char*>(slicesT) + (size_t)s * np * Pw * 2, np, Pk, 128, 2, Pw));
    // B operand: columns c0 .. c0 + Pk - 1 of the kp x np slice plane of Z / c
    CDL_TRY(make_map(&maps.b[s], static_cast<const char*>(zslices) + (size_t)s * kp * np * 2 + (size_t)c0 * 2, kp,
                     Pk, kp, 2, np));
  }
  ResidParams p;
  std::memset(&p, 0, sizeof(p));
  p.num_tiles = np / 128;
  p.kblocks = Pk / 64;
  p.kp = kp;
  for (int m = 2; m <= RS_SLICES + 1; ++m)
    for (int sa = 1; sa < m; ++sa) {
      const int sz = m - sa;
      if (sa > RS_SLICES || sz > RS_SLICES) continue;
      p.pair_s[p.npairs] = sa;
      p.pair_t[p.npairs] = sz;
      ++p.npairs;
    }
  p.G = G;
  p.gstride = (size_t)np * kp;
  p.idesc = make_idesc(kp);
  p.status = ctx->dev_status;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_resid, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_BYTES));
    attr = true;
  }
  const int grid = std::min(p.num_tiles * p.npairs, ctx->sm_count);
  Launch L(ctx, CDL_KC_RESIDUAL, 2.0 * p.npairs * (double)np * Pk * kp);
  k_tc_resid<<<grid, T8_THREADS, RS_SMEM_BYTES, ctx->stream>>>(maps, p);
  return L.done();
}

int score_tc_tiles(cdl_ctx* ctx, const void* uplanes, const void* vplanes, const long long* dint,
                   const double* oscale, int n, int rows, int k2p, const double* A1, const double* A2, int row0,
                   long long tile0, long long tile1, double* contrib) {
  if (rows % 128 || k2p % 64 || rows < n || k2p < 64) return CDL_ERR_INVALID_ARG;
  ScoreMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  for (int s = 0; s < SC_SLICES; ++s) {
    const size_t off = (size_t)s * rows * k2p * 2;
    CDL_TRY(make_map(&maps.u[s], static_cast<const char*>(uplanes) + off, rows, k2p, 128));
    CDL_TRY(make_map(&maps.v[s], static_cast<const char*>(vplanes) + off, rows, k2p, SC_N));
  }
  ScoreParams p;
  std::memset(&p, 0, sizeof(p));
  p.nb128 = rows / 128;
  p.nb64 = 2 * p.nb128;
  const long long all = (long long)p.nb128 * p.nb64 - (long long)p.nb128 * (p.nb128 - 1);
  if (tile1 < 0) tile1 = all;
  if (tile0 < 0 || tile1 > all || tile0 > tile1 || tile1 - tile0 > 0x7fffffffLL) return CDL_ERR_INVALID_ARG;
  const long long tiles = tile1 - tile0;
  if (tiles == 0) return CDL_OK;
  p.num_tiles = (int)tiles;
  p.tile0 = tile0;
  p.row0 = row0;
  p.kblocks = k2p / 64;
  p.n = n;
  p.A1 = A1;
  p.A2 = A2;
  p.dint = dint;
  p.oscale = oscale;
  p.contrib = contrib;
  p.idesc = make_idesc(SC_N);
  p.status = ctx->dev_status;
  static bool attr = false;
  if (!attr) {
    CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_score, cudaFuncAttributeMaxDynamicSharedMemorySize, SC_SMEM_BYTES));
    attr = true;
  }
  const int grid = (int)std::min<long long>(tiles, ctx->sm_count);
  // 21 slice products over the computed tiles
  Launch L(ctx, CDL_KC_SCORE, 2.0 * 21 * (double)tiles * 128 * SC_N * k2p);
  k_tc_score<<<grid, T8_THREADS, SC_SMEM_BYTES, ctx->stream>>>(maps, p);
  return L.done();
}

int score_tc(cdl_ctx* ctx, const void* uplanes, const void* vplanes, const long long* dint, const double* oscale,
             int n, int rows, int k2p, const double* A1, const double* A2, double* contrib) {
  return score_tc_tiles(ctx, uplanes, vplanes, dint, oscale, n, rows, k2p, A1, A2, 0, 0, -1, contrib);
}

int apply_tc(cdl_ctx* ctx, const cdl_chain* ch, int level, const void* xop, float* partial, int kp,
             int splits) {
  if (!ch->host_levels) return apply_tc_mat(ctx, ch->level16(level), (int)ch->npad, xop, partial, kp, splits);
  cdl_chain* mch = const_cast<cdl_chain*>(ch);   // slot bookkeeping only
  const void* lv = ooc_read(ctx, mch, level);
  if (!lv) return CDL_ERR_CUDA;
  CDL_TRY(apply_tc_mat(ctx, lv, (int)ch->npad, xop, partial, kp, splits));
  CDL_TRY(ooc_read_done(ctx, mch, level));
  return ooc_prefetch(ctx, mch, (level + 1) % ch->d_eff);   // overlaps the next level's load with this update
}

int apply_tc_mat(cdl_ctx* ctx, const void* amat, int np, const void* xop, float* partial, int kp, int splits) {
  const int bn = 2 * kp;
  if (bn % 32 || bn < 32 || bn > MAX_BN) return CDL_ERR_UNSUPPORTED;
  const int mb = np / BM;
  if ((np / BK) % splits) return CDL_ERR_INVALID_ARG;
  const int ncl = pair_clusters(ctx);
  if (ncl > 0 && bn % 64 == 0) {
    // CTA pairs: 256-row blocks, each CTA staging half of the right-hand-side operand
    static bool attr = false;
    if (!attr) {
      CDL_CUDA_TRY(cudaFuncSetAttribute(k_tc_apply2, cudaFuncAttributeMaxDynamicSharedMemorySize, S2_SMEM_BYTES));
      attr = true;
    }
    CUtensorMap ma, mbm;
    CDL_TRY(make_map(&ma, amat, np, np, 128));
    CDL_TRY(make_map(&mbm, xop, bn, np, bn / 2));
    Apply2Params p{};
    p.num_units = ((np + 255) / 256) * splits;
    p.splits = splits;
    p.kblocks = np / BK / splits;
    p.npad = np;
    p.bn = bn;
    p.idesc = make_idesc_m256(bn);
    p.out = partial;
    p.status = ctx->dev_status;
    const int clusters = std::min(p.num_units, ncl);
    Launch L(ctx, CDL_KC_APPLY, 2.0 * np * (double)np);
    k_tc_apply2<<<2 * clusters, S2_THREADS, S2_SMEM_BYTES, ctx->stream>>>(ma, mbm, p);
    return L.done();
  }
  const uint32_t* tiles;
  int count;
  CDL_TRY(get_tiles(ctx, "tc.apply." + std::to_string(mb) + "." + std::to_string(splits),
                    [&] { return apply_tiles(mb, splits); }, &tiles, &count));
  CUtensorMap ma, mbm;
  CDL_TRY(make_map(&ma, amat, np, np, 128));
  CDL_TRY(make_map(&mbm, xop, bn, np, bn));
  TcParams p{};
  p.tiles = tiles;
  p.num_tiles = count;
  p.kblocks = np / BK / splits;
  p.bn = bn;
  p.idesc = make_idesc(bn);
  p.mode = MODE_APPLY;
  p.npad = np;
  p.out = partial;
  p.ldo = bn;
  p.status = ctx->dev_status;
  p.amax = nullptr;
  p.level = 0;
  p.out16 = nullptr;
  p.debug_withhold_load = 0;
  p.groups = nullptr;
  const double bytes = 2.0 * np * (double)np;
  return launch(ctx, ma, mbm, p, CDL_KC_APPLY, bytes);
}

}  // namespace cdl
