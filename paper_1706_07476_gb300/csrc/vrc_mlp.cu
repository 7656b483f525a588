// Learned cross-section surrogate: training step (forward, loss, backward in
// one kernel) and Adam.  The training step's matrix products are warp-level
// mma.sync.m16n8k16 with bfloat16 operands and float32 accumulation; operand
// tiles come from shared memory through ldmatrix (.trans where the stored
// layout is the transpose of the operand).  The forward products take each
// activation as a bfloat16 pair hi + lo (two products into one
// accumulator), as the per-ray forward pass on tcgen05 does (vrc_mlp_tc.cu);
// the backward products use the hi parts (gradient noise of 2^-9 relative).
#include <cuda_bf16.h>
#include <math.h>

#include "vrc_internal.h"
#include "vrc_mlp.h"
#include "vrc_mlp_dev.cuh"

namespace vrc {
namespace mlp {

Embed make_embed(double e_lo, double e_hi) {
  Embed e;
  const double a = log10(e_lo), b = log10(e_hi);
  e.l0 = (float)a;
  e.inv_range = (float)(1.0 / (b - a));
  for (int k = 0; k < kFreq; ++k) e.freq[k] = (float)exp2(kFreqMaxLog2 * k / (kFreq - 1));
  return e;
}

namespace {

typedef __nv_bfloat16 bf16;
constexpr int LD64 = kEmb + 8;   // padded row strides (elements): 16-byte aligned
constexpr int LD128 = kHid + 8;  // rows, conflict-free ldmatrix
constexpr int BM = 64;           // rows per training block (16 per warp)
constexpr int kTrainThreads = 128;

__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldm_x4(uint32_t (&r)[4], const bf16 *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sm_addr(p)));
}

__device__ __forceinline__ void ldm_x4_t(uint32_t (&r)[4], const bf16 *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(sm_addr(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + expf(-z));
  return s * (1.f + z * (1.f - s));
}

// Fragment address helpers (lane = thread index in the warp; j = lane/8
// selects one of the four 8x8 matrices, r = lane%8 its row).
// A (m16 x k16) from S stored [m][k]:
__device__ __forceinline__ const bf16 *a_rows(const bf16 *S, int ld, int m0, int k0, int lane) {
  return S + (m0 + (lane & 15)) * ld + k0 + ((lane >> 4) << 3);
}
// A (m16 x k16) from S stored [k][m]  (use with .trans):
__device__ __forceinline__ const bf16 *a_cols(const bf16 *S, int ld, int m0, int k0, int lane) {
  const int j = lane >> 3, r = lane & 7;
  return S + (k0 + r + ((j >> 1) << 3)) * ld + m0 + ((j & 1) << 3);
}
// Two B tiles (k16 x n8 at n0 and n0+8) from S stored [n][k]:
__device__ __forceinline__ const bf16 *b_rows(const bf16 *S, int ld, int n0, int k0, int lane) {
  const int j = lane >> 3, r = lane & 7;
  return S + (n0 + r + ((j >> 1) << 3)) * ld + k0 + ((j & 1) << 3);
}
// Two B tiles from S stored [k][n]  (use with .trans):
__device__ __forceinline__ const bf16 *b_cols(const bf16 *S, int ld, int n0, int k0, int lane) {
  const int j = lane >> 3, r = lane & 7;
  return S + (k0 + r + ((j & 1) << 3)) * ld + n0 + ((j >> 1) << 3);
}

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Column sums over a warp's 16 rows of an accumulator tile, added to dst[col].
__device__ __forceinline__ void add_col_sums(const float (&d)[4], float *dst, int col, int lane) {
  float s0 = d[0] + d[2], s1 = d[1] + d[3];
  for (int o = 4; o < 32; o <<= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (lane < 4) {
    atomicAdd(dst + col, s0);
    atomicAdd(dst + col + 1, s1);
  }
}

// ---------------------------------------------------------------------------
// Training step: one block = 64 rows, 4 warps of 16 rows.
// ---------------------------------------------------------------------------
constexpr int LDH = kHid + 1;  // float32 h2 rows, padded so row-wise reads spread over banks
constexpr size_t kTrainSmem =
    sizeof(bf16) * (size_t)(kHid * LD64 + kHid * LD128 + 2 * BM * LD64 + 3 * BM * LD128 + 2 * BM * kHid) +
    sizeof(float) * (size_t)(BM * LDH + kOut * kHid + 2 * BM * kOut + 2 * kHid + 3 * kOut + BM);

// Two floats as bfloat16 pairs hi = bf16(v), lo = bf16(v - hi).
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  hi = *reinterpret_cast<const uint32_t *>(&h);
  lo = pack2(a - hf.x, b - hf.y);
}

__global__ void __launch_bounds__(kTrainThreads) k_mlp_train(TrainArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  bf16 *W1s = reinterpret_cast<bf16 *>(smem);  // [128][72]
  bf16 *W2s = W1s + kHid * LD64;               // [128][136]
  bf16 *X0 = W2s + kHid * LD128;               // [64][72] features, hi
  bf16 *X0l = X0 + BM * LD64;                  // [64][72] features, lo
  bf16 *H1 = X0l + BM * LD64;                  // [64][136] h1, hi
  bf16 *H1l = H1 + BM * LD128;                 // [64][136] h1, lo
  bf16 *DZ2 = H1l + BM * LD128;                // [64][136]
  bf16 *D1 = DZ2 + BM * LD128;                 // [64][128] silu'(z1)
  bf16 *D2 = D1 + BM * kHid;                   // [64][128] silu'(z2)
  float *H2 = reinterpret_cast<float *>(D2 + BM * kHid);  // [64][129] float32 h2; later dz1 (bf16)
  float *W3f = H2 + BM * LDH;                  // [16][128] W3, float32
  float *DY = W3f + kOut * kHid;               // [64][16]
  float *Q = DY + BM * kOut;                   // [64][16] prior a + b E^(-1/2)
  float *bs = Q + BM * kOut;                   // b1, b2, b3, C [16][2]
  float *Es = bs + 2 * kHid + 3 * kOut;        // [64]
  __shared__ int64_t src[BM];
  __shared__ float red[kTrainThreads / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const float *P = a.params;

  for (int i = tid; i < kHid * kEmb; i += kTrainThreads) W1s[(i / kEmb) * LD64 + i % kEmb] = __float2bfloat16_rn(P[kOffW1 + i]);
  for (int i = tid; i < kHid * kHid; i += kTrainThreads) W2s[(i / kHid) * LD128 + i % kHid] = __float2bfloat16_rn(P[kOffW2 + i]);
  for (int i = tid; i < kOut * kHid; i += kTrainThreads) W3f[i] = P[kOffW3 + i];
  for (int i = tid; i < kHid; i += kTrainThreads) { bs[i] = P[kOffB1 + i]; bs[kHid + i] = P[kOffB2 + i]; }
  if (tid < kOut) bs[2 * kHid + tid] = P[kOffB3 + tid];
  if (tid < 2 * kOut) bs[2 * kHid + kOut + tid] = P[kOffC + tid];
  if (tid < BM) {
    const int64_t R = (int64_t)blockIdx.x * BM + tid;
    int64_t s = -1;
    if (R < a.m) s = a.set_n > 0 ? (int64_t)(mix64(a.seed + (uint64_t)R) % (uint64_t)a.set_n) : R;
    src[tid] = s;
    Es[tid] = s >= 0 ? a.E[s] : 1.0f;
  }
  __syncthreads();
  for (int i = tid; i < BM * kFreq; i += kTrainThreads) {
    const int r = i / kFreq, f = i % kFreq;
    float sn, cs;
    embed_pair(a.emb, Es[r], f, &sn, &cs);
    uint32_t hi, lo;
    split2(sn, cs, hi, lo);
    *reinterpret_cast<uint32_t *>(X0 + r * LD64 + 2 * f) = hi;
    *reinterpret_cast<uint32_t *>(X0l + r * LD64 + 2 * f) = lo;
  }
  __syncthreads();

  const int rw = warp * 16;
  // ---- layer 1: z1 = x0 W1^T + b1 -> h1 = silu(z1), d1 = silu'(z1)
  {
    float acc[16][4] = {};
    for (int k0 = 0; k0 < kEmb; k0 += 16) {
      uint32_t af[4], al[4];
      ldm_x4(af, a_rows(X0, LD64, rw, k0, lane));
      ldm_x4(al, a_rows(X0l, LD64, rw, k0, lane));
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        uint32_t bf[4];
        ldm_x4(bf, b_rows(W1s, LD64, np * 16, k0, lane));
        mma_bf16(acc[2 * np], af, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], af, bf[2], bf[3]);
        mma_bf16(acc[2 * np], al, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], al, bf[2], bf[3]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int c = nt * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = rw + g + 8 * h;
        const float z0 = acc[nt][2 * h] + bs[c], z1 = acc[nt][2 * h + 1] + bs[c + 1];
        uint32_t hi, lo;
        split2(silu(z0), silu(z1), hi, lo);
        *reinterpret_cast<uint32_t *>(H1 + row * LD128 + c) = hi;
        *reinterpret_cast<uint32_t *>(H1l + row * LD128 + c) = lo;
        *reinterpret_cast<uint32_t *>(D1 + row * kHid + c) = pack2(silu_grad(z0), silu_grad(z1));
      }
    }
  }
  __syncwarp();
  // ---- layer 2: z2 = h1 W2^T + b2 -> h2 (float32), d2
  {
    float acc[16][4] = {};
    for (int k0 = 0; k0 < kHid; k0 += 16) {
      uint32_t af[4], al[4];
      ldm_x4(af, a_rows(H1, LD128, rw, k0, lane));
      ldm_x4(al, a_rows(H1l, LD128, rw, k0, lane));
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        uint32_t bf[4];
        ldm_x4(bf, b_rows(W2s, LD128, np * 16, k0, lane));
        mma_bf16(acc[2 * np], af, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], af, bf[2], bf[3]);
        mma_bf16(acc[2 * np], al, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], al, bf[2], bf[3]);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int c = nt * 8 + 2 * t;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = rw + g + 8 * h;
        const float z0 = acc[nt][2 * h] + bs[kHid + c], z1 = acc[nt][2 * h + 1] + bs[kHid + c + 1];
        H2[row * LDH + c] = silu(z0);
        H2[row * LDH + c + 1] = silu(z1);
        *reinterpret_cast<uint32_t *>(D2 + row * kHid + c) = pack2(silu_grad(z0), silu_grad(z1));
      }
    }
  }
  __syncthreads();
  // ---- layer 3 in float32 (CUDA cores): y = W3 h2 + b3; residual, loss, dy.
  // Thread tid: row tid/2, outputs 8 (tid & 1) .. +7.
  float lsum = 0.f;
  {
    const int r = tid >> 1, m0 = (tid & 1) * 8;
    const int64_t s = src[r];
    const float rs = rsqrtf(Es[r]);
    const float *C = bs + 2 * kHid + kOut;
    float y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // b3 and the prior log(a + b E^(-1/2))
      const float q = fmaf(C[2 * (m0 + j) + 1], rs, C[2 * (m0 + j)]);
      Q[r * kOut + m0 + j] = q;
      y[j] = bs[2 * kHid + m0 + j] + logf(q);
    }
    const float *h = H2 + r * LDH;
    for (int k = 0; k < kHid; ++k) {
      const float hk = h[k];
#pragma unroll
      for (int j = 0; j < 8; ++j) y[j] = fmaf(W3f[(m0 + j) * kHid + k], hk, y[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = m0 + j;
      bool on = s >= 0 && ((a.mat_mask >> col) & 1u);
      if (on && a.mask) on = a.mask[s * kOut + col] != 0;
      const float res = on ? y[j] - a.target[s * kOut + col] : 0.f;
      lsum += res * res;
      DY[r * kOut + col] = 2.f * res * a.inv_count;
    }
  }
  __syncthreads();
  // ---- dW3 = dy^T h2, dz2 = (dy W3) * silu'(z2)  (float32; thread tid = hidden unit k)
  {
    const int k = tid;
    float gw[kOut];
#pragma unroll
    for (int m = 0; m < kOut; ++m) gw[m] = 0.f;
    float db = 0.f;
    for (int r = 0; r < BM; ++r) {
      const float hk = H2[r * LDH + k];
      float dot = 0.f;
#pragma unroll
      for (int m = 0; m < kOut; ++m) {
        const float dy = DY[r * kOut + m];
        gw[m] = fmaf(dy, hk, gw[m]);
        dot = fmaf(dy, W3f[m * kHid + k], dot);
      }
      const float dz = dot * __bfloat162float(D2[r * kHid + k]);
      DZ2[r * LD128 + k] = __float2bfloat16_rn(dz);
      db += dz;
    }
#pragma unroll
    for (int m = 0; m < kOut; ++m) atomicAdd(a.grad + kOffW3 + m * kHid + k, gw[m]);
    atomicAdd(a.grad + kOffB2 + k, db);
    if (tid < kOut) {
      // b3, and the prior: dy/da = 1/q, dy/db = E^(-1/2)/q
      float sb = 0.f, sa = 0.f, sc = 0.f;
      for (int r = 0; r < BM; ++r) {
        const float dy = DY[r * kOut + tid], iq = 1.f / Q[r * kOut + tid];
        sb += dy;
        sa = fmaf(dy, iq, sa);
        sc = fmaf(dy * iq, rsqrtf(Es[r]), sc);
      }
      atomicAdd(a.grad + kOffB3 + tid, sb);
      atomicAdd(a.grad + kOffC + 2 * tid, sa);
      atomicAdd(a.grad + kOffC + 2 * tid + 1, sc);
    }
  }
  __syncthreads();
  // ---- dW2 = dz2^T h1  ([128][128]); warp w owns rows 32w..32w+31, two passes
  for (int mt = 0; mt < 2; ++mt) {
    const int m0 = warp * 32 + mt * 16;
    float acc[16][4] = {};
    for (int k0 = 0; k0 < BM; k0 += 16) {
      uint32_t af[4];
      ldm_x4_t(af, a_cols(DZ2, LD128, m0, k0, lane));
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        uint32_t bf[4];
        ldm_x4_t(bf, b_cols(H1, LD128, np * 16, k0, lane));
        mma_bf16(acc[2 * np], af, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], af, bf[2], bf[3]);
      }
    }
    float *G = a.grad + kOffW2;
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int n = nt * 8 + 2 * t;
      atomicAdd(G + (m0 + g) * kHid + n, acc[nt][0]);
      atomicAdd(G + (m0 + g) * kHid + n + 1, acc[nt][1]);
      atomicAdd(G + (m0 + g + 8) * kHid + n, acc[nt][2]);
      atomicAdd(G + (m0 + g + 8) * kHid + n + 1, acc[nt][3]);
    }
  }
  // ---- dz1 = (dz2 W2) * silu'(z1), stored over h2
  bf16 *DZ1 = reinterpret_cast<bf16 *>(H2);
  {
    float acc[16][4] = {};
    for (int k0 = 0; k0 < kHid; k0 += 16) {
      uint32_t af[4];
      ldm_x4(af, a_rows(DZ2, LD128, rw, k0, lane));
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        uint32_t bf[4];
        ldm_x4_t(bf, b_cols(W2s, LD128, np * 16, k0, lane));
        mma_bf16(acc[2 * np], af, bf[0], bf[1]);
        mma_bf16(acc[2 * np + 1], af, bf[2], bf[3]);
      }
    }
    __syncthreads();  // every warp has finished reading h2 (dW3) before dz1 overwrites it
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int c = nt * 8 + 2 * t;
      float dz[4];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int row = rw + g + 8 * h;
        dz[2 * h] = acc[nt][2 * h] * __bfloat162float(D1[row * kHid + c]);
        dz[2 * h + 1] = acc[nt][2 * h + 1] * __bfloat162float(D1[row * kHid + c + 1]);
        *reinterpret_cast<uint32_t *>(DZ1 + row * LD128 + c) = pack2(dz[2 * h], dz[2 * h + 1]);
      }
      add_col_sums(dz, a.grad + kOffB1, c, lane);
    }
  }
  __syncthreads();
  // ---- dW1 = dz1^T x0  ([128][64]); warp w owns rows 32w..32w+31
  {
    float acc[2][8][4] = {};
    for (int k0 = 0; k0 < BM; k0 += 16) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t af[4];
        ldm_x4_t(af, a_cols(DZ1, LD128, warp * 32 + mt * 16, k0, lane));
#pragma unroll
        for (int np = 0; np < 4; ++np) {
          uint32_t bf[4];
          ldm_x4_t(bf, b_cols(X0, LD64, np * 16, k0, lane));
          mma_bf16(acc[mt][2 * np], af, bf[0], bf[1]);
          mma_bf16(acc[mt][2 * np + 1], af, bf[2], bf[3]);
        }
      }
    }
    float *G = a.grad + kOffW1;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int m0 = warp * 32 + mt * 16;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int n = nt * 8 + 2 * t;
        atomicAdd(G + (m0 + g) * kEmb + n, acc[mt][nt][0]);
        atomicAdd(G + (m0 + g) * kEmb + n + 1, acc[mt][nt][1]);
        atomicAdd(G + (m0 + g + 8) * kEmb + n, acc[mt][nt][2]);
        atomicAdd(G + (m0 + g + 8) * kEmb + n + 1, acc[mt][nt][3]);
      }
    }
  }
  // ---- loss
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) red[warp] = lsum;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kTrainThreads / 32; ++w) s += red[w];
    atomicAdd(a.loss, s * a.inv_count);
  }
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    p[i] -= lr * (a * c1) / (sqrtf(v * c2) + eps);
  }
}

// ---------------------------------------------------------------------------
// Forward pass per ray: activations stay in registers (the m16n8 accumulator
// pair of one layer is the m16k16 A operand of the next).  Block = 4 warps,
// each warp 16 rays per pass; weights staged once per block.
// ---------------------------------------------------------------------------
}  // namespace

cudaError_t launch_train(const TrainArgs &a, cudaStream_t s) {
  if (a.m <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
  if (e != cudaSuccess) return e;
  const int blocks = (int)((a.m + BM - 1) / BM);
  k_mlp_train<<<blocks, kTrainThreads, kTrainSmem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_adam(float *params, const float *grad, float *m1, float *m2, int n, float lr,
                        float beta1, float beta2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.f / (1.f - powf(beta1, (float)step));
  const float c2 = 1.f / (1.f - powf(beta2, (float)step));
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(params, grad, m1, m2, n, lr, beta1, beta2, eps, c1, c2);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace vrc
