// Split-bf16 theta projection on the 5th-generation tensor cores (tcgen05 + TMA + TMEM).
//
// For every azimuthal wavenumber m (Sect. 3.2) the projection is the product
//   D[m][n][r] = sum_k A[m][r][k] B[m][n][k]      (r < M = Ntheta rows, k < K = Ntheta)
// with A the (H^T W)_m or H_m table and B the K-contiguous float32 spectral panel of
// 2 Nr columns n = (i, re/im).  Both operands enter the products as NP bf16 planes
// x = x0 + x1 (+ x2) (x0 = RN_bf16(x), x1 = RN_bf16(x - x0), x2 = RN_bf16(x - x0 - x1),
// for a float32 x the exact remainder); the table's planes are precomputed, the panel's
// are formed in shared memory.  The
// product keeps every plane pair whose index sum is below NP, smallest terms first:
//   NP = 2: A1 B0 + A0 B1 + A0 B0                              (3 products, ~2^-16)
//   NP = 3: A2 B0 + A0 B2 + A1 B1 + A1 B0 + A0 B1 + A0 B0      (6 products, ~2^-24)
// accumulated in float32 in tensor memory.
//
// Persistent, warp-specialised pipeline (448 threads, one CTA per SM).  The column tiles
// of all m form one list g = m x tiles + t; CTA c takes the contiguous range
// [G c / grid, G (c+1) / grid), so every SM gets the same number of tiles give or take one,
// and the range covers a few consecutive m (a segment per m):
//  - warp 0 (one lane) loads the A planes of each segment's m (TMA, 128B-swizzled K-major
//    boxes of 64 K-elements), the next segment's only after the products of the previous
//    one have completed;
//  - warps 6..13 stream the panel rows of the CTA's column tiles one K block at a time
//    (float4 loads, the next two blocks in flight while the current one is converted),
//    split them into bf16 planes and store those in the 128B-swizzled K-major layout of
//    a ring of stages (full/empty mbarriers per stage, fence.proxy.async before the
//    arrival);
//  - warp 1 (one lane) issues, per K block, the K-steps x products of tcgen05.mma
//    (M=128, N=BN=128, K=16, kind::f16, bf16 inputs, f32 accumulator) into one of two
//    TMEM accumulators and commits to the stage's empty barrier (and, after a tile's
//    last K block, to the accumulator's full barrier);
//  - warps 2..5 drain the other accumulator meanwhile (tcgen05.ld; warp w owns TMEM
//    lanes 32 (w mod 4) .. +31 = output rows) and store float32 rows coalesced along r.
// Every wait is bounded and also watches a shared abort flag: on expiry the CTA records
// kErrTimeout, the other roles leave their loops, and TMEM is still freed.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace sp {
namespace tc {

constexpr int kM = 128;          // UMMA M (rows = l or j)
constexpr int kKBlk = 64;        // K elements per 128-byte swizzle row
constexpr int kMaxKBlocks = 2;   // K <= 128
constexpr uint32_t kABlockBytes = kM * 128;   // 16 KB per K block and plane

template <int NP> struct Cfg;
// N = 128 per MMA (N = 64 runs at about half the per-column rate); the panel streams
// through shared memory one K block (64 K-elements) of a tile at a time
template <> struct Cfg<2> { static constexpr int BN = 128; static constexpr int kStages = 4; };
template <> struct Cfg<3> { static constexpr int BN = 128; static constexpr int kStages = 2; };
constexpr int kConvWarps = 8;
constexpr int kConvThreads = 32 * kConvWarps;
constexpr int kThreads = 192 + kConvThreads;
constexpr int kConvPer = 8;   // float4 chunks per converter thread and K block (BN = 128 rows x 16)

// one stage: the NP planes of one K block of a BN-column tile
template <int NP>
__host__ __device__ constexpr uint32_t stage_bytes() { return NP * (uint32_t)Cfg<NP>::BN * 128u; }

template <int NP>
constexpr uint32_t smem_bytes() {
  return NP * kMaxKBlocks * kABlockBytes + Cfg<NP>::kStages * stage_bytes<NP>() + 1024u;
}
constexpr int kErrTimeout = 4;
constexpr long long kSpinLimit = 1ll << 26;

struct Params {
  float* D;          // [mh][ncol][M]
  const float* B;    // panel [mh][ncol][kstride] float32
  int M;             // valid rows (Ntheta)
  int K;             // valid K (Ntheta)
  int kstride;       // panel row stride (multiple of 8)
  int ncol;          // columns per m
  int kblocks;       // ceil(K / 64)
  int mh;            // number of m (batch of the products)
  int* err;
};

struct Maps {
  CUtensorMap a[3];   // A planes
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// Round-to-nearest-even of a finite float to bf16 with integer operations (faster than
// the conversion unit here), returned as float bits with the low half zero.
// Two float32 values rounded to nearest-even bf16 and packed, `lo` in bits 0-15: one
// conversion instruction, for finite values the same words as the integer form
// (u + 0x7FFF + ((u >> 16) & 1)) >> 16.
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned address and size).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout or when *abort is set.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  return false;
}

// Bounded wait for phase `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms of 1024 B.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);          // start address
  d |= (uint64_t)1 << 16;                            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                            // swizzle: 128B
  return d;
}

// Instruction descriptor: kind::f16, bf16 A and B (K-major), f32 accumulator, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 32; ++q) v[q] = __uint_as_float(r[q]);
}

// One instance's CTA bx of gx (the persistent range split below).
template <int NP>
__device__ __forceinline__ void tc_gemm_split_body(const Maps& maps, const Params& prm, int bx, int gx) {
  constexpr int BN = Cfg<NP>::BN;
  constexpr int S = Cfg<NP>::kStages;
  constexpr uint32_t kPlaneBytes = BN * 128u;   // one plane of one K block
  constexpr uint32_t kStage = stage_bytes<NP>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the swizzle atoms
  const uint32_t base_u32 = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t sA = base_u32;                                  // [NP][kMaxKBlocks] x 16 KB
  const uint32_t sB = sA + NP * kMaxKBlocks * kABlockBytes;      // [S][NP] x BN*128 B
  __shared__ __align__(8) uint64_t bar_a, bar_afree;
  __shared__ __align__(8) uint64_t bar_full[S], bar_empty[S];
  __shared__ __align__(8) uint64_t bar_tfull[2], bar_tempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int kb = prm.kblocks;
  const int tiles = (prm.ncol + BN - 1) / BN;
  const long long gtot = (long long)tiles * prm.mh;
  const int g0 = (int)((gtot * bx) / gx);
  const int g1 = (int)((gtot * (bx + 1)) / gx);
  const int nt = g1 - g0;
  const int nq = nt * kb;   // work chunks q = (tile g0 + q / kb, K block q % kb)
  const int m0 = g0 / tiles;
  const int nseg = nt > 0 ? (g1 - 1) / tiles - m0 + 1 : 0;   // consecutive m values covered

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"((uint32_t)(2 * BN)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 32) {
    s_abort = 0;
    mbar_init(smem_u32(&bar_a), 1);
    mbar_init(smem_u32(&bar_afree), 1);
    for (int q = 0; q < S; ++q) {
      mbar_init(smem_u32(&bar_full[q]), kConvThreads);
      mbar_init(smem_u32(&bar_empty[q]), 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&bar_tfull[q]), 1);
      mbar_init(smem_u32(&bar_tempty[q]), 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int* abort = &s_abort;
  auto fail = [&]() {
    *abort = 1;
    atomicOr(prm.err, kErrTimeout);
  };
  auto load_a = [&](int m) {
    const uint32_t ba = smem_u32(&bar_a);
    mbar_expect_tx(ba, (uint32_t)kb * NP * kABlockBytes);
    for (int pl = 0; pl < NP; ++pl)
      for (int b = 0; b < kb; ++b) tma_load_3d(sA + (pl * kMaxKBlocks + b) * kABlockBytes, &maps.a[pl], b * kKBlk, 0, m, ba);
  };
  // the table planes are plan constants: loaded while the previous kernel may still run
  pdl_trigger();
  if (warp == 0 && lane == 0 && nseg > 0) load_a(m0);
  pdl_wait();

  if (warp == 0) {
    if (lane == 0 && nseg > 0) {
      // segment sg's table replaces sg-1's once the products reading it have completed
      int issued = 1;
      for (; issued < nseg; ++issued) {
        if (!mbar_wait_or_abort(smem_u32(&bar_afree), (uint32_t)(issued - 1) & 1u, abort)) {
          fail();
          break;
        }
        load_a(m0 + issued);
      }
      // the last table copy issued lands before the CTA frees its shared memory
      mbar_wait(smem_u32(&bar_a), (uint32_t)(issued - 1) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0 && nt > 0) {
      // ---- MMA issuer
      const uint32_t idesc = idesc_bf16_f32(kM, BN);
      constexpr int npairs = NP == 2 ? 3 : 6;
      constexpr int pa[6] = {NP == 2 ? 1 : 2, 0, NP == 2 ? 0 : 1, 1, 0, 0};
      constexpr int pb[6] = {0, NP == 2 ? 1 : 2, NP == 2 ? 0 : 1, 0, 1, 0};
      // descriptors differ only in the start-address field (address >> 4, below 2^14 for
      // any shared-memory address), so each is a base plus a compile-time offset
      const uint64_t dA0 = smem_desc_sw128(sA);
      bool ok = true;
      for (int q = 0; ok && q < nq; ++q) {
        const int t = q / kb, b = q - t * kb;
        const int g = g0 + t, sg = g / tiles - m0;
        // first chunk of a segment: its table has landed
        if (b == 0 && (t == 0 || g % tiles == 0) && !mbar_wait_or_abort(smem_u32(&bar_a), (uint32_t)sg & 1u, abort)) {
          ok = false;
          break;
        }
        const int st = q % S;
        const uint32_t ph = (uint32_t)(q / S) & 1u;
        const int acc_buf = t & 1;
        const uint32_t aph = (uint32_t)(t >> 1) & 1u;
        if (!mbar_wait_or_abort(smem_u32(&bar_full[st]), ph, abort) ||
            (b == 0 && t >= 2 && !mbar_wait_or_abort(smem_u32(&bar_tempty[acc_buf]), aph ^ 1u, abort))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dt = tmem + (uint32_t)(acc_buf * BN);
        const uint64_t dB0 = smem_desc_sw128(sB + st * kStage);
        const uint64_t dAb = dA0 + (uint64_t)(((uint32_t)b * kABlockBytes) >> 4);
#pragma unroll
        for (int k4 = 0; k4 < kKBlk / 16; ++k4) {   // 16 bf16 = 32 B along the swizzled row
#pragma unroll
          for (int i = 0; i < npairs; ++i) {
            const uint64_t da = dAb + (((uint32_t)pa[i] * kMaxKBlocks * kABlockBytes + k4 * 32u) >> 4);
            const uint64_t db = dB0 + (((uint32_t)pb[i] * kPlaneBytes + k4 * 32u) >> 4);
            umma_bf16(dt, da, db, idesc, (b | k4 | i) ? 1u : 0u);
          }
        }
        umma_commit(smem_u32(&bar_empty[st]));
        if (b == kb - 1) umma_commit(smem_u32(&bar_tfull[acc_buf]));
        // last chunk of a segment with another one after it: the table may be replaced
        // once these products complete
        if (b == kb - 1 && (g + 1) % tiles == 0 && sg + 1 < nseg) umma_commit(smem_u32(&bar_afree));
      }
      if (!ok) fail();
    }
  } else if (warp < 6) {
    // ---- epilogue: warps 2..5
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    for (int t = 0; t < nt; ++t) {
      const int acc_buf = t & 1;
      const uint32_t aph = (uint32_t)(t >> 1) & 1u;
      // every lane polls; the warp proceeds only together (tcgen05.ld is warp-collective)
      const bool ok_lane = mbar_wait_or_abort(smem_u32(&bar_tfull[acc_buf]), aph, abort);
      if (!__all_sync(0xffffffffu, ok_lane)) {
        if (lane == 0) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int g = g0 + t, m = g / tiles;
      const int n0 = (g - m * tiles) * BN;
      float* dst = prm.D + ((size_t)m * prm.ncol + n0) * prm.M + row;
      const bool full = n0 + BN <= prm.ncol;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tmem_ld_32x32b_x32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc_buf * BN + c0), v);
        if (row < prm.M) {
          if (full) {
#pragma unroll
            for (int i = 0; i < 32; ++i) dst[(size_t)(c0 + i) * prm.M] = v[i];
          } else {
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (n0 + c0 + i < prm.ncol) dst[(size_t)(c0 + i) * prm.M] = v[i];
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_tempty[acc_buf]));
    }
  } else {
    // ---- panel converter: warps 6..13.  Chunk c = ct + kConvThreads u of a K block is
    // the float4 (row r = c / 16, k = 64 b + 4 (c mod 16) .. + 3), so a half-warp reads
    // one 256-byte row segment.
    const int ct = tid - 192;
    // first panel row of tile t of the CTA's range (tiles of one m are consecutive rows)
    auto tile_rows = [&](int t, int& n0) -> const float* {
      const int g = g0 + t, m = g / tiles;
      n0 = (g - m * tiles) * BN;
      return prm.B + ((size_t)m * prm.ncol + n0) * prm.kstride;
    };
    // the thread's chunks u = 0..kConvPer-1 of a K block: rows r0 + 16 u, K-elements
    // 4 kc4 .. +3 of the block; rows 16 apart share r mod 8, so their swizzled positions
    // are 16 x 128 bytes apart
    const int r0 = ct >> 4, kc4 = ct & 15;
    const uint32_t off0 = (uint32_t)r0 * 128u + ((uint32_t)((kc4 >> 1) ^ (r0 & 7)) << 4) + (uint32_t)(kc4 & 1) * 8u;
    auto fetch = [&](int q, float4 (&v)[kConvPer]) {
      const int t = q / kb, b = q - t * kb;
      int n0;
      const float* Bt = tile_rows(t, n0);
      const int k = b * kKBlk + 4 * kc4;
      const float* src = Bt + (size_t)r0 * prm.kstride + k;
      const int rows = prm.ncol - n0 - r0;   // rows r0 + 16 u exist while 16 u < rows
      const bool kin = k < prm.kstride;
#pragma unroll
      for (int u = 0; u < kConvPer; ++u)
        v[u] = (kin && 16 * u < rows) ? __ldg(reinterpret_cast<const float4*>(src + (size_t)(16 * u) * prm.kstride))
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // one thread keeps the rows of the tiles two ahead on their way into L2 (a tile's
    // rows are contiguous), so the register loads of the next K block hit L2
    auto prefetch_tile = [&](int t) {
      if (ct != 0 || t >= nt) return;
      int n0;
      const float* Bt = tile_rows(t, n0);
      const int rows = min(BN, prm.ncol - n0);
      prefetch_l2_bulk(Bt, (uint32_t)rows * (uint32_t)prm.kstride * 4u);
    };
    prefetch_tile(0);
    prefetch_tile(1);
    // two K blocks in flight beyond the one being converted
    float4 cur[kConvPer], nxt[kConvPer], nx2[kConvPer];
    if (nq > 0) fetch(0, cur);
    if (nq > 1) fetch(1, nxt);
    for (int q = 0; q < nq; ++q) {
      if (q % kb == 0) prefetch_tile(q / kb + 2);
      if (q + 2 < nq) fetch(q + 2, nx2);
      const int st = q % S;
      const uint32_t ph = (uint32_t)(q / S) & 1u;
      if (q >= S && !mbar_wait_or_abort(smem_u32(&bar_empty[st]), ph ^ 1u, abort)) {
        fail();
        break;
      }
      const int b = q % kb;
      const uint32_t bst = sB + st * kStage + off0;
      const int k = b * kKBlk + 4 * kc4;
      const bool kfull = k + 4 <= prm.K;   // else the elements at and beyond K enter as zeros
#pragma unroll
      for (int u = 0; u < kConvPer; ++u) {
        // 16-byte chunk kc4/2 of row r sits at chunk (kc4/2) ^ (r mod 8) of the 128-byte row
        const uint32_t off = 2048u * (uint32_t)u;
        const float x[4] = {cur[u].x, cur[u].y, cur[u].z, cur[u].w};
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (kfull || k + e < prm.K) ? x[e] : 0.f;
        // planes in pairs of elements: bf16 words of (e, e+1) packed by one conversion,
        // unpacked to float to form the exact remainder (<= 16 significant bits), whose
        // rounding is the second plane; the second remainder (<= 8 bits) is already bf16
        uint32_t w[3][2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float a = v[2 * q], b = v[2 * q + 1];
          w[0][q] = bf16x2_rn(a, b);
          const float ra = __fsub_rn(a, __uint_as_float(w[0][q] << 16));
          const float rb = __fsub_rn(b, __uint_as_float(w[0][q] & 0xFFFF0000u));
          w[1][q] = bf16x2_rn(ra, rb);
          if (NP == 3) {
            const float sa = __fsub_rn(ra, __uint_as_float(w[1][q] << 16));
            const float sb = __fsub_rn(rb, __uint_as_float(w[1][q] & 0xFFFF0000u));
            w[2][q] = __byte_perm(__float_as_uint(sa), __float_as_uint(sb), 0x7632);
          }
        }
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) st_shared_v2(bst + (uint32_t)pl * kPlaneBytes + off, w[pl][0], w[pl][1]);
      }
      fence_proxy_async_smem();
      mbar_arrive(smem_u32(&bar_full[st]));
#pragma unroll
      for (int u = 0; u < kConvPer; ++u) {
        cur[u] = nxt[u];
        nxt[u] = nx2[u];
      }
    }
  }
  // the last products complete before TMEM is freed
  if (tid == 32 && nt > 0 && !*abort) mbar_wait(smem_u32(&bar_tfull[(nt - 1) & 1]), (uint32_t)((nt - 1) >> 1) & 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)));
  }
}

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm_split(const __grid_constant__ Maps maps, Params prm) {
  tc_gemm_split_body<NP>(maps, prm, blockIdx.x, gridDim.x);
}

// Ragged batches: instance q owns CTAs start[q] .. start[q+1]-1 and splits its (m, tile)
// list over them; its table maps are read from the argument table in global memory.
struct alignas(64) TcArgs {
  Maps maps;
  Params prm;
};

template <int NP>
__global__ void __launch_bounds__(kThreads, 1) k_tc_gemm_split_rag(const TcArgs* __restrict__ tab,
                                                                  const int* __restrict__ start, int n) {
  const int q = rag_instance(start, n, blockIdx.x);
  tc_gemm_split_body<NP>(tab[q].maps, tab[q].prm, (int)blockIdx.x - start[q], start[q + 1] - start[q]);
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  // resolved once, thread-safely (function-local static initialisation)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

// Tensor map of a bf16 array [batch][rows][K] with row stride `kstride` elements
// (kstride*2 bytes must be a multiple of 16); boxes of 64 K-elements x box_rows rows.
inline bool make_map(CUtensorMap* map, const void* base, int K, int kstride, int rows, int batch, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)kstride * 2, (cuuint64_t)kstride * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)kKBlk, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc
}  // namespace sp
