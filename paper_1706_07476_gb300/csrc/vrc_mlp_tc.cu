// Per-ray forward pass of the learned cross-section surrogate on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// One persistent block per SM holds the bfloat16 weights once and runs two
// independent groups of 512 threads (16 warps each), each on its own tiles
// of 128 rays with its own operand buffer, mbarrier, named barrier and 128
// tensor-memory columns.  Threads t, t + 128, t + 256 and t + 384 of a group
// own ray t of the tile, which is row t of every matrix and lane t of the
// tensor memory (warps j, j + 4, j + 8 and j + 12 of the group read lane
// quarter j); each takes a quarter of the row's columns (features,
// activations, outputs).  Eight warps per scheduler hide the latency of the
// per-element work (sines, SiLU, the hi/lo splits); with one thread per row
// (two warps per scheduler) it was exposed: 5.8 ms per 2^24 rays, against
// 4.6 ms with two threads per row and 4.4 ms with four.
// Every activation enters the tensor cores as
// a pair of bfloat16 matrices, hi = bf16(v) and lo = bf16(v - hi), whose two
// products go into one accumulator (about 16 significant bits per value).
// Per tile:
//   1. each thread writes its ray's 64 embedding features to A0hi, A0lo;
//   2. one thread issues D = A0hi W1^T + A0lo W1^T (M = N = 128, K = 64, four
//      K = 16 steps each) into the group's columns and commits to the
//      group's mbarrier;
//   3. each thread loads its row of D, adds b1, applies SiLU and writes the
//      row's hi and lo parts to A1hi, A1lo;
//   4. D = A1hi W2^T + A1lo W2^T (K = 128, eight steps each) into the same
//      columns;
//   5. each thread loads its row, h2 = SiLU(D + b2), and writes its hi and lo
//      parts to A2hi, A2lo (A1's bytes: the layer-2 MMAs have completed);
//   6. D3 = A2 W3^T (M = 128, K = 128) with W3 held as three bfloat16 parts
//      (hi, mid, lo: about 24 significant bits) stacked as one [48][128]
//      matrix: A2hi [W3hi; W3mid; W3lo] (N = 48) and A2lo [W3hi; W3mid]
//      (N = 32) into two column ranges of the group;
//   7. each thread loads its outputs' five products (hi hi, hi mid, hi lo,
//      lo hi, lo mid), sums them, adds b3 and the 1/v prior and writes log
//      sigma or sigma.
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, consecutive along K 128 bytes
// apart (leading byte offset) and along rows K*16 bytes apart (stride byte
// offset).
#include <cuda_bf16.h>
#include <math.h>

#include "vrc_internal.h"
#include "vrc_mlp.h"
#include "vrc_mlp_dev.cuh"

namespace vrc {
namespace mlp {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTile = 128;            // rays per tile: the MMA's M and the tensor-memory lanes
constexpr int kGroups = 2;            // independent groups of kGroupThreads threads per block
constexpr int kRowParts = 4;          // threads per ray row: each takes a quarter of the row's columns
constexpr int kGroupThreads = 128 * kRowParts;
constexpr int kTcThreads = kGroupThreads * kGroups;
constexpr uint32_t kTmemCols = 256;   // allocated once per block; group g uses columns 128 g ..
constexpr int kWaitLimit = 1 << 22;   // mbarrier polls before a wait gives up

// shared memory (bytes from the block's base)
constexpr uint32_t kSW1 = 0;          // W1 [128][64] bfloat16, 16 KiB
constexpr uint32_t kSW2 = 16384;      // W2 [128][128], 32 KiB
constexpr uint32_t kSW3 = 49152;      // W3 [16][128] as bfloat16 hi, mid, lo: 3 x 4 KiB
constexpr uint32_t kW3Part = 4096;
constexpr uint32_t kSB = 61440;       // b1, b2, b3, then the prior C [16][2] (float32, 304 values)
constexpr uint32_t kSBar = 62720;     // per group an mbarrier (8 B); then the tensor-memory address
// Per group one 64 KiB operand buffer: A1hi [128][128] at 0 and A1lo at
// 32 KiB; A0hi [128][64] at 0 and A0lo at 16 KiB share A1hi's bytes (A0 is
// read only by the layer-1 MMAs, which have completed before A1 is written;
// A1 is read only by the layer-2 MMAs, which have completed before the next
// tile's A0 is written).
constexpr uint32_t kSGroup = 63488;
constexpr uint32_t kGroupBytes = 65536;
constexpr uint32_t kA0Lo = 16384, kA1Lo = 32768;
constexpr uint32_t kSmemTc = kSGroup + kGroups * kGroupBytes;  // 194,560

// Byte offset of element (r, k) of a K-column matrix in the core-matrix layout.
__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Two floats as bfloat16 pairs hi = bf16(v), lo = bf16(v - hi) (first value
// in the low half of each word).
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = pack2(a - hf.x, b - hf.y);
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all in 16-byte units), the fixed version bits 46-48 = 0b001, base
// offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= 1ull << 46;
  return d;
}

// Instruction descriptor of kind::f16: float32 D (bits 4-5 = 1), bfloat16 A
// and B (bits 7-9 and 10-12 = 1), both K-major, N / 8 at bits 17-22, M / 16
// at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc48 = (1u << 4) | (1u << 7) | (1u << 10) | ((48u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdesc32 = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
// Output-layer accumulators within the group's columns: A2hi [W3hi; W3mid;
// W3lo] (N = 48) at 0, A2lo [W3hi; W3mid] (N = 32) at kD3Lo.
constexpr uint32_t kD3Lo = 64;

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate,
                                            uint32_t idesc = kIdesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :: "r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Polls the mbarrier for completion of the phase with the given parity, at
// most kWaitLimit times.  Returns false if it gave up.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (int it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  }
  return done != 0;
}

// 32 consecutive float32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t (&r)[32], uint32_t taddr) {
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
}

// N = 4 or 8 consecutive float32 columns of this thread's lane, without
// waiting: several loads are issued before one tmem_wait_ld.
template <int N>
__device__ __forceinline__ void tmem_ld_cols_async(uint32_t (&r)[N], uint32_t taddr);
template <>
__device__ __forceinline__ void tmem_ld_cols_async<8>(uint32_t (&r)[8], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld_cols_async<4>(uint32_t (&r)[4], uint32_t taddr) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Stages W3 [16][128] (float32) as three bfloat16 parts w = hi + mid + lo
// (hi = bf16(w), mid = bf16(w - hi), lo = bf16(w - hi - mid)), each in core
// matrices of K = 128 columns.
__device__ __forceinline__ void stage_w3(unsigned char *smem, const float *W) {
  for (int i = threadIdx.x; i < kOut * kHid / 8; i += blockDim.x) {
    const int r = i / (kHid / 8), k = (i % (kHid / 8)) * 8;
    uint32_t h[4], m[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float w0 = W[r * kHid + k + 2 * e], w1 = W[r * kHid + k + 2 * e + 1];
      const __nv_bfloat162 hb = __floats2bfloat162_rn(w0, w1);
      const float2 hf = __bfloat1622float2(hb);
      const float r0 = w0 - hf.x, r1 = w1 - hf.y;  // exact
      const __nv_bfloat162 mb = __floats2bfloat162_rn(r0, r1);
      const float2 mf = __bfloat1622float2(mb);
      h[e] = *reinterpret_cast<const uint32_t *>(&hb);
      m[e] = *reinterpret_cast<const uint32_t *>(&mb);
      l[e] = pack2(r0 - mf.x, r1 - mf.y);
    }
    const uint32_t o = kSW3 + cm_off(r, k, kHid);
    *reinterpret_cast<uint4 *>(smem + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(smem + o + kW3Part) = make_uint4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<uint4 *>(smem + o + 2 * kW3Part) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// Stages a [128][K] float32 weight block as bfloat16 core matrices.
__device__ __forceinline__ void stage_weights(unsigned char *smem, uint32_t off, const float *W, int K) {
  const int chunks = kTile * K / 8;
  for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
    const int r = i / (K / 8), k = (i % (K / 8)) * 8;
    const float *w = W + r * K + k;
    const uint4 v = make_uint4(pack2(w[0], w[1]), pack2(w[2], w[3]), pack2(w[4], w[5]), pack2(w[6], w[7]));
    *reinterpret_cast<uint4 *>(smem + off + cm_off(r, k, K)) = v;
  }
}

// Barrier of the threads of one group (named barrier 1 + g); returns
// nonzero in every thread of the group if any thread passed nonzero.
__device__ __forceinline__ uint32_t group_sync_or(int g, uint32_t v) {
  uint32_t any;
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t"
      "bar.red.popc.u32 %0, %1, %3, p;\n\t}"
      : "=r"(any) : "r"(1 + g), "r"(v), "r"(kGroupThreads) : "memory");
  return any;
}

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "r"(kGroupThreads) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_apply_tc(ApplyArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int g = tid / kGroupThreads, gt = tid % kGroupThreads;  // group, thread within the group
  const int rt = gt & 127, part = gt >> 7;  // the thread's row in the tile; its part of the columns
  static_assert(kRowParts == 2 || kRowParts == 4, "a row is split into 2 or 4 parts");
  // rows to evaluate: all n, or the device count (e.g. the accepted rays of a cast)
  const int64_t n = a.n_limit ? min(a.n, (int64_t)*a.n_limit) : a.n;
  const int64_t tiles = (n + kTile - 1) / kTile;
  if ((int64_t)blockIdx.x * kGroups >= tiles) return;  // the whole block has no tile

  float *bs = reinterpret_cast<float *>(smem + kSB);
  const uint32_t bar = smem_u32(smem + kSBar + 8 * g);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + kSBar + 8 * kGroups);
  unsigned char *A0 = smem + kSGroup + g * kGroupBytes;
  unsigned char *A1 = A0;
  const float *P = a.params;

  stage_weights(smem, kSW1, P + kOffW1, kEmb);
  stage_weights(smem, kSW2, P + kOffW2, kHid);
  stage_w3(smem, P + kOffW3);
  for (int i = tid; i < kHid; i += kTcThreads) { bs[i] = P[kOffB1 + i]; bs[kHid + i] = P[kOffB2 + i]; }
  if (tid < kOut) bs[2 * kHid + tid] = P[kOffB3 + tid];
  if (tid < 2 * kOut) bs[2 * kHid + kOut + tid] = P[kOffC + tid];
  if (gt == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar) : "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tslot)), "r"(kTmemCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot + 128u * (uint32_t)g;                     // the group's columns
  const uint32_t tmem_row = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lane quarter
  const uint32_t sA0 = smem_u32(A0), sA1 = smem_u32(A1);
  const uint32_t sW1 = smem_u32(smem + kSW1), sW2 = smem_u32(smem + kSW2), sW3 = smem_u32(smem + kSW3);
  const float *C = bs + 2 * kHid + kOut;  // prior (a_m, b_m)
  uint32_t phase = 0;  // parity of the group's next mbarrier phase (three commits per tile)

  // Each tile's energies are loaded one tile ahead, so that no tile starts
  // by waiting on global memory (4 % less time per 2^24 rays).
  const int64_t tile_step = (int64_t)gridDim.x * kGroups;
  auto load_E = [&](int64_t t) -> float {
    const int64_t r = t * kTile + rt;
    return (t < tiles && r < n) ? (a.aos ? __ldg(a.aos + 2 * r + 1).z : a.E[r]) : 1.0f;
  };
  float E_next = load_E((int64_t)blockIdx.x * kGroups + g);

  for (int64_t tile = (int64_t)blockIdx.x * kGroups + g; tile < tiles; tile += tile_step) {
    const int64_t row = tile * kTile + rt;
    const float E = E_next;
    E_next = load_E(tile + tile_step);

    // mode 1: whether the ray's hash bin is flagged, looked up now and used
    // after the output layer
    bool flagged = false;
    if (a.mode == 1 && a.flags && part == 0 && row < n) {
      const double e = (double)E;
      if (!(e >= a.e_first && e <= a.e_last)) {
        flagged = true;
      } else {
        int b = (int)((__log2f(E) - a.l2min) * a.inv_bw);
        b = min(max(b, 0), a.n_hash - 1);
        flagged = __ldg(a.flags + b) != 0;
      }
    }

    // 1. embedding row: features 2f, 2f + 1 = sin, cos of pi f_f x, as hi and lo
    const float x = embed_x(a.emb, E);
#pragma unroll
    for (int kc = part * (kEmb / 8 / kRowParts); kc < (part + 1) * (kEmb / 8 / kRowParts); ++kc) {
      uint32_t wh[4], wl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float sn, cs;
        embed_pair_x(a.emb, x, kc * 4 + q, &sn, &cs);
        split2(sn, cs, wh[q], wl[q]);
      }
      const uint32_t o = cm_off(rt, kc * 8, kEmb);
      *reinterpret_cast<uint4 *>(A0 + o) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
      *reinterpret_cast<uint4 *>(A0 + kA0Lo + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
    }
    fence_async_smem();
    fence_before();
    group_sync(g);

    // 2. D = A0hi W1^T + A0lo W1^T
    if (gt == 0) {
      fence_after();
#pragma unroll
      for (int kk = 0; kk < kEmb / 16; ++kk)
        mma_bf16_tc(tmem, smem_desc(sA0 + kk * 256, 128, kEmb * 16), smem_desc(sW1 + kk * 256, 128, kEmb * 16),
                    kk > 0);
#pragma unroll
      for (int kk = 0; kk < kEmb / 16; ++kk)
        mma_bf16_tc(tmem, smem_desc(sA0 + kA0Lo + kk * 256, 128, kEmb * 16),
                    smem_desc(sW1 + kk * 256, 128, kEmb * 16), 1);
      mma_commit(bar);
    }
    if (group_sync_or(g, !wait_phase(bar, phase))) {
      if (gt == 0 && a.status) atomicOr(a.status, kStatusTimeout);
      break;
    }
    phase ^= 1u;
    fence_after();

    // 3. h1 = SiLU(D + b1) as hi and lo bfloat16 into A1hi, A1lo
#pragma unroll
    for (int c = part * (kHid / 32 / kRowParts); c < (part + 1) * (kHid / 32 / kRowParts); ++c) {
      uint32_t r[32];
      tmem_ld32(r, tmem_row + c * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = q * 8 + 2 * e, k = c * 32 + j;
          split2(silu(__uint_as_float(r[j]) + bs[k]), silu(__uint_as_float(r[j + 1]) + bs[k + 1]), wh[e], wl[e]);
        }
        const uint32_t o = cm_off(rt, c * 32 + q * 8, kHid);
        *reinterpret_cast<uint4 *>(A1 + o) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4 *>(A1 + kA1Lo + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      }
    }
    fence_async_smem();
    fence_before();
    group_sync(g);

    // 4. D = A1hi W2^T + A1lo W2^T
    if (gt == 0) {
      fence_after();
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        mma_bf16_tc(tmem, smem_desc(sA1 + kk * 256, 128, kHid * 16), smem_desc(sW2 + kk * 256, 128, kHid * 16),
                    kk > 0);
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        mma_bf16_tc(tmem, smem_desc(sA1 + kA1Lo + kk * 256, 128, kHid * 16),
                    smem_desc(sW2 + kk * 256, 128, kHid * 16), 1);
      mma_commit(bar);
    }
    if (group_sync_or(g, !wait_phase(bar, phase))) {
      if (gt == 0 && a.status) atomicOr(a.status, kStatusTimeout);
      break;
    }
    phase ^= 1u;
    fence_after();

    // 5. h2 = SiLU(D + b2) as hi and lo bfloat16 into A2hi, A2lo (A1's bytes)
#pragma unroll
    for (int c = part * (kHid / 32 / kRowParts); c < (part + 1) * (kHid / 32 / kRowParts); ++c) {
      uint32_t r[32];
      tmem_ld32(r, tmem_row + c * 32);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t wh[4], wl[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j = q * 8 + 2 * e, k = c * 32 + j;
          split2(silu(__uint_as_float(r[j]) + bs[kHid + k]), silu(__uint_as_float(r[j + 1]) + bs[kHid + k + 1]),
                 wh[e], wl[e]);
        }
        const uint32_t o = cm_off(rt, c * 32 + q * 8, kHid);
        *reinterpret_cast<uint4 *>(A1 + o) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
        *reinterpret_cast<uint4 *>(A1 + kA1Lo + o) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
      }
    }
    fence_async_smem();
    fence_before();
    group_sync(g);

    // 6. D3 = A2 W3^T with W3 as three bfloat16 parts, whose [16][128]
    // blocks lie back to back as one [48][128] matrix: A2hi [W3hi; W3mid;
    // W3lo] (N = 48) and A2lo [W3hi; W3mid] (N = 32), 16 MMAs in place of
    // 40 with N = 16; the five 16-column products are summed in step 7
    if (gt == 0) {
      fence_after();
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        mma_bf16_tc(tmem, smem_desc(sA1 + kk * 256, 128, kHid * 16), smem_desc(sW3 + kk * 256, 128, kHid * 16),
                    kk > 0, kIdesc48);
#pragma unroll
      for (int kk = 0; kk < kHid / 16; ++kk)
        mma_bf16_tc(tmem + kD3Lo, smem_desc(sA1 + kA1Lo + kk * 256, 128, kHid * 16),
                    smem_desc(sW3 + kk * 256, 128, kHid * 16), kk > 0, kIdesc32);
      mma_commit(bar);
    }
    if (group_sync_or(g, !wait_phase(bar, phase))) {
      if (gt == 0 && a.status) atomicOr(a.status, kStatusTimeout);
      break;
    }
    phase ^= 1u;
    fence_after();

    // 7. this thread's kPer of the 16 outputs (part h: outputs kPer h ..):
    // the five products (hi hi, hi mid, hi lo, lo hi, lo mid) plus b3
    constexpr int kPer = kOut / kRowParts;
    float p[kPer];
    {
      uint32_t hh[kPer], hm[kPer], hl[kPer], lh[kPer], lm[kPer];
      const uint32_t c0 = tmem_row + (uint32_t)(part * kPer);
      tmem_ld_cols_async<kPer>(hh, c0);
      tmem_ld_cols_async<kPer>(hm, c0 + 16);
      tmem_ld_cols_async<kPer>(hl, c0 + 32);
      tmem_ld_cols_async<kPer>(lh, c0 + kD3Lo);
      tmem_ld_cols_async<kPer>(lm, c0 + kD3Lo + 16);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const float small = (__uint_as_float(hl[j]) + __uint_as_float(lm[j])) +
                            (__uint_as_float(hm[j]) + __uint_as_float(lh[j]));
        p[j] = (__uint_as_float(hh[j]) + small) + bs[2 * kHid + part * kPer + j];
      }
    }
    fence_before();

    if (row < n) {
      const float rs = rsqrtf(E);
      if (a.mode == 1) {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int m = part * kPer + j;
          p[j] = ((a.mat_mask >> m) & 1u) ? fmaf(C[2 * m + 1], rs, C[2 * m]) * expf(p[j]) : 0.f;
        }
        if (flagged) p[0] = __int_as_float(0x7fc00000);  // output 0 (part 0) marks a flagged bin
      } else {
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
          const int m = part * kPer + j;
          p[j] += logf(fmaf(C[2 * m + 1], rs, C[2 * m]));
        }
      }
      float4 *o = reinterpret_cast<float4 *>(a.out + row * kOut + part * kPer);
#pragma unroll
      for (int q = 0; q < kPer / 4; ++q) o[q] = make_float4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
    }
  }
  // every tensor-memory read has completed (tcgen05.wait::ld) before the barrier
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(*tslot), "r"(kTmemCols) : "memory");
}

}  // namespace

cudaError_t launch_apply(const ApplyArgs &a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc);
  if (e != cudaSuccess) return e;
  // one resident block per SM (its shared memory allows no second one), so
  // its 512 tensor-memory columns are free when it allocates them
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_mlp_apply_tc, kTcThreads, kSmemTc);
  if (e != cudaSuccess) return e;
  if (bps != 1) return cudaErrorInvalidConfiguration;
  // a device row limit is read by the kernel: size the grid for all n rows
  // (blocks without a tile return at once)
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  const int64_t want = (tiles + kGroups - 1) / kGroups;
  const int grid = (int)(want < (int64_t)num_sms ? want : (int64_t)num_sms);
  k_mlp_apply_tc<<<grid, kTcThreads, kSmemTc, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace vrc
