// Learned refinement flags: per-element features, a 3-layer MLP (136-128-128-3)
// with bfloat16 tensor-core forward products and float32 accumulation, its
// backward pass and Adam.
//
// The paper's velocity criterion (Sec. 3.1) fires only once intensification
// has started (Sec. 5); the network predicts the criterion's flags some steps
// ahead from the current state, so that adaptation can run less often while
// the criterion stays the fallback.
//
// Precision contract (shared with the CPU oracle): inputs, weights and the two
// hidden activations enter their products rounded to bfloat16 (nearest even);
// products accumulate in float32; the backward pass is float32 on the same
// rounded values (the gradient of the loss with respect to the rounded
// weights); master weights and Adam moments are float32.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>
#include <cuda_bf16.h>

#include "sem_internal.h"
#include "tcgen05.cuh"

namespace sem {
namespace {

constexpr int IN = 136, HID = 128, OUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + IN * HID, OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID, OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + HID * OUT;
constexpr int NPARAM = OFF_B3 + OUT;
// transposed bfloat16 weights for the tensor-core B operands, padded strides
// (in bfloat16 elements) that keep the fragment loads free of bank conflicts
constexpr int K1P = 152, K2P = 136;
constexpr int W1T_SZ = HID * K1P, W2T_SZ = HID * K2P, W3T_SZ = 8 * K2P;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<unsigned*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// refresh the transposed bfloat16 weights and the rounded float32 copies
__global__ void mlp_refresh(const float* __restrict__ P, __nv_bfloat16* __restrict__ w1t,
                            __nv_bfloat16* __restrict__ w2t, __nv_bfloat16* __restrict__ w3t,
                            float* __restrict__ R) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < W1T_SZ + W2T_SZ + W3T_SZ;
       i += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (i < W1T_SZ) {
      const int n = i / K1P, k = i % K1P;
      if (k < IN) v = P[OFF_W1 + k * HID + n];
      w1t[i] = __float2bfloat16_rn(v);
    } else if (i < W1T_SZ + W2T_SZ) {
      const int r = i - W1T_SZ, n = r / K2P, k = r % K2P;
      if (k < HID) v = P[OFF_W2 + k * HID + n];
      w2t[r] = __float2bfloat16_rn(v);
    } else {
      const int r = i - W1T_SZ - W2T_SZ, n = r / K2P, k = r % K2P;
      if (k < HID && n < OUT) v = P[OFF_W3 + k * OUT + n];
      w3t[r] = __float2bfloat16_rn(v);
    }
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += gridDim.x * blockDim.x)
    R[i] = bf16r(P[i]);
}

// Forward pass.  One warp per 16 rows, 4 warps per CTA.  Writes the class
// probabilities, and in training mode the rounded inputs and activations.
constexpr int FWD_ROWS = 64;
constexpr size_t FWD_SMEM = (size_t)(W1T_SZ + W2T_SZ + W3T_SZ) * 2 + (2 * HID + 8) * 4;

__global__ void __launch_bounds__(128)
mlp_forward(const float* __restrict__ X, int n, const __nv_bfloat16* __restrict__ w1t,
            const __nv_bfloat16* __restrict__ w2t, const __nv_bfloat16* __restrict__ w3t,
            const float* __restrict__ P, float* __restrict__ prob, float* __restrict__ Xr,
            float* __restrict__ H1r, float* __restrict__ H2r, int8_t* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char sm[];
  __nv_bfloat16* s1 = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* s2 = s1 + W1T_SZ;
  __nv_bfloat16* s3 = s2 + W2T_SZ;
  float* sb = reinterpret_cast<float*>(s3 + W3T_SZ);   // b1 | b2 | b3
  {
    const uint4* src = reinterpret_cast<const uint4*>(w1t);
    uint4* dst = reinterpret_cast<uint4*>(s1);
    for (int i = threadIdx.x; i < (W1T_SZ + W2T_SZ + W3T_SZ) / 8; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < HID; i += blockDim.x) {
      sb[i] = P[OFF_B1 + i];
      sb[HID + i] = P[OFF_B2 + i];
    }
    if (threadIdx.x < 8) sb[2 * HID + threadIdx.x] = threadIdx.x < OUT ? P[OFF_B3 + threadIdx.x] : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const int row0 = blockIdx.x * FWD_ROWS + warp * 16;
  const int ra = row0 + gid, rb = row0 + gid + 8;
  // A fragments of the input rows, 9 k-steps of 16 (136 padded to 144)
  unsigned a[9][4];
#pragma unroll
  for (int s = 0; s < 9; ++s) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 16 * s + 8 * h + 2 * tig;
      float x0 = 0.f, x1 = 0.f, y0 = 0.f, y1 = 0.f;
      if (ra < n && c < IN) { x0 = X[(long long)ra * IN + c]; x1 = X[(long long)ra * IN + c + 1]; }
      if (rb < n && c < IN) { y0 = X[(long long)rb * IN + c]; y1 = X[(long long)rb * IN + c + 1]; }
      a[s][2 * h + 0] = pack_bf16(x0, x1);
      a[s][2 * h + 1] = pack_bf16(y0, y1);
      if (Xr && c < IN) {
        if (ra < n) { Xr[(long long)ra * IN + c] = bf16r(x0); Xr[(long long)ra * IN + c + 1] = bf16r(x1); }
        if (rb < n) { Xr[(long long)rb * IN + c] = bf16r(y0); Xr[(long long)rb * IN + c + 1] = bf16r(y1); }
      }
    }
  }
  // layer 1: 16 column tiles of 8; results become layer 2's A fragments
  unsigned h1[8][4];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* wb = s1 + (8 * t + gid) * K1P + 2 * tig;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const unsigned b0 = *reinterpret_cast<const unsigned*>(wb + 16 * s);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(wb + 16 * s + 8);
      mma_bf16(d, a[s], b0, b1);
    }
    const int c = 8 * t + 2 * tig;
    const float v0 = fmaxf(d[0] + sb[c], 0.f), v1 = fmaxf(d[1] + sb[c + 1], 0.f);
    const float v2 = fmaxf(d[2] + sb[c], 0.f), v3 = fmaxf(d[3] + sb[c + 1], 0.f);
    h1[t >> 1][(t & 1) * 2 + 0] = pack_bf16(v0, v1);
    h1[t >> 1][(t & 1) * 2 + 1] = pack_bf16(v2, v3);
    if (H1r) {
      if (ra < n) { H1r[(long long)ra * HID + c] = bf16r(v0); H1r[(long long)ra * HID + c + 1] = bf16r(v1); }
      if (rb < n) { H1r[(long long)rb * HID + c] = bf16r(v2); H1r[(long long)rb * HID + c + 1] = bf16r(v3); }
    }
  }
  // layer 2
  unsigned h2[8][4];
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16* wb = s2 + (8 * t + gid) * K2P + 2 * tig;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const unsigned b0 = *reinterpret_cast<const unsigned*>(wb + 16 * s);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(wb + 16 * s + 8);
      mma_bf16(d, h1[s], b0, b1);
    }
    const int c = 8 * t + 2 * tig;
    const float v0 = fmaxf(d[0] + sb[HID + c], 0.f), v1 = fmaxf(d[1] + sb[HID + c + 1], 0.f);
    const float v2 = fmaxf(d[2] + sb[HID + c], 0.f), v3 = fmaxf(d[3] + sb[HID + c + 1], 0.f);
    h2[t >> 1][(t & 1) * 2 + 0] = pack_bf16(v0, v1);
    h2[t >> 1][(t & 1) * 2 + 1] = pack_bf16(v2, v3);
    if (H2r) {
      if (ra < n) { H2r[(long long)ra * HID + c] = bf16r(v0); H2r[(long long)ra * HID + c + 1] = bf16r(v1); }
      if (rb < n) { H2r[(long long)rb * HID + c] = bf16r(v2); H2r[(long long)rb * HID + c + 1] = bf16r(v3); }
    }
  }
  // layer 3: one column tile (3 of 8 used)
  float d[4] = {0.f, 0.f, 0.f, 0.f};
  {
    const __nv_bfloat16* wb = s3 + gid * K2P + 2 * tig;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const unsigned b0 = *reinterpret_cast<const unsigned*>(wb + 16 * s);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(wb + 16 * s + 8);
      mma_bf16(d, h2[s], b0, b1);
    }
  }
  // logits of rows ra (d0, d1 at columns 2 tig, 2 tig + 1) and rb (d2, d3);
  // columns 0..2 live in lanes tig = 0, 1 of each quad
  const float za0 = d[0] + sb[2 * HID + 2 * tig], za1 = d[1] + sb[2 * HID + 2 * tig + 1];
  const float zb0 = d[2] + sb[2 * HID + 2 * tig], zb1 = d[3] + sb[2 * HID + 2 * tig + 1];
  const int q0 = lane & ~3;
  const float a00 = __shfl_sync(0xffffffffu, za0, q0), a01 = __shfl_sync(0xffffffffu, za1, q0);
  const float a02 = __shfl_sync(0xffffffffu, za0, q0 + 1);
  const float b00 = __shfl_sync(0xffffffffu, zb0, q0), b01 = __shfl_sync(0xffffffffu, zb1, q0);
  const float b02 = __shfl_sync(0xffffffffu, zb0, q0 + 1);
  if (tig == 0) {
    const float zs[2][3] = {{a00, a01, a02}, {b00, b01, b02}};
    const int rows[2] = {ra, rb};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (rows[h] >= n) continue;
      const float m = fmaxf(zs[h][0], fmaxf(zs[h][1], zs[h][2]));
      const float e0 = expf(zs[h][0] - m), e1 = expf(zs[h][1] - m), e2 = expf(zs[h][2] - m);
      const float inv = 1.f / (e0 + e1 + e2);
      if (prob) {
        prob[(long long)rows[h] * OUT + 0] = e0 * inv;
        prob[(long long)rows[h] * OUT + 1] = e1 * inv;
        prob[(long long)rows[h] * OUT + 2] = e2 * inv;
      }
      if (flags) {
        int cls = 0;
        if (zs[h][1] > zs[h][cls]) cls = 1;
        if (zs[h][2] > zs[h][cls]) cls = 2;
        flags[rows[h]] = (int8_t)(cls - 1);
      }
    }
  }
}

// Forward pass on the fifth-generation tensor cores (tcgen05), the
// default: persistent CTAs of 128 threads (two per SM) keep the weights in
// shared memory and walk over tiles of 128 rows, thread t owning row t of a
// tile (tensor memory lane t).  The three layers are GEMMs of M = 128 rows by N = 128 (16
// for the 3 logits) by K = 144 (the 136 inputs padded) or 128, as
// tcgen05.mma.cta_group::1.kind::f16 with bfloat16 operands from shared memory
// (K-major, no swizzle: core matrices of 8 rows x 8 bfloat16) and float32
// accumulators in tensor memory (256 columns: layer 1 at 0, layer 2 at 128,
// layer 3 at 0 again).  Each thread reads its row's accumulators back
// (tcgen05.ld), adds the bias, applies ReLU, rounds to bfloat16 and writes the
// next layer's A operand over the previous one (the MMAs that read it have
// completed).  Same precision contract as mlp_forward; waits on the MMA
// completion barrier are bounded, a wait that runs out leaves the outputs of
// the CTA unwritten and sets *err.
constexpr int TC_ROWS = 128;
constexpr int TC_X_BYTES = TC_ROWS * 144 * 2;                  // A operand (X, then H1, H2)
constexpr int TC_W1_BYTES = HID * 144 * 2, TC_W2_BYTES = HID * HID * 2, TC_W3_BYTES = 16 * HID * 2;
constexpr size_t TC_SMEM = (size_t)TC_X_BYTES + TC_W1_BYTES + TC_W2_BYTES + TC_W3_BYTES +
                           (2 * HID + 16) * sizeof(float) + 16;

// byte offset of element (row r, k) of a K-major bfloat16 operand with kc
// core matrices (8 bfloat16 each) along K
__device__ __forceinline__ int boff(int r, int k, int kc) {
  return (r & 7) * 16 + (k & 7) * 2 + (k >> 3) * 128 + (r >> 3) * (kc * 128);
}

__global__ void __launch_bounds__(TC_ROWS, 2)
mlp_forward_tc(const float* __restrict__ X, int n, const __nv_bfloat16* __restrict__ w1t,
               const __nv_bfloat16* __restrict__ w2t, const __nv_bfloat16* __restrict__ w3t,
               const float* __restrict__ P, float* __restrict__ prob, float* __restrict__ Xr,
               float* __restrict__ H1r, float* __restrict__ H2r, int8_t* __restrict__ flags, int* err) {
  extern __shared__ __align__(1024) unsigned char sm_tc[];
  unsigned char* sA = sm_tc;
  unsigned char* sW1 = sA + TC_X_BYTES;
  unsigned char* sW2 = sW1 + TC_W1_BYTES;
  unsigned char* sW3 = sW2 + TC_W2_BYTES;
  float* sb = reinterpret_cast<float*>(sW3 + TC_W3_BYTES);   // b1 | b2 | b3 (16)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sb + 2 * HID + 16);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 1);
  const int t = threadIdx.x, warp = t >> 5;
  // weights: 8 bfloat16 (16 bytes) per core-matrix row; the transposed
  // arrays hold row n of W^T with k contiguous (zero beyond the inputs)
  for (int i = t; i < HID * 18; i += TC_ROWS) {
    const int nn = i / 18, c = i % 18;
    *reinterpret_cast<uint4*>(sW1 + boff(nn, 8 * c, 18)) = *reinterpret_cast<const uint4*>(w1t + nn * K1P + 8 * c);
  }
  for (int i = t; i < HID * 16; i += TC_ROWS) {
    const int nn = i / 16, c = i % 16;
    *reinterpret_cast<uint4*>(sW2 + boff(nn, 8 * c, 16)) = *reinterpret_cast<const uint4*>(w2t + nn * K2P + 8 * c);
  }
  for (int i = t; i < 16 * 16; i += TC_ROWS) {
    const int nn = i / 16, c = i % 16;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(sW3 + boff(nn, 8 * c, 16)) =
        nn < 8 ? *reinterpret_cast<const uint4*>(w3t + nn * K2P + 8 * c) : z;
  }
  for (int i = t; i < HID; i += TC_ROWS) {
    sb[i] = P[OFF_B1 + i];
    sb[HID + i] = P[OFF_B2 + i];
  }
  if (t < 16) sb[2 * HID + t] = t < OUT ? P[OFF_B3 + t] : 0.f;
  if (warp == 0) tcg::alloc(taddr_s, 256);
  if (t == 0) tcg::mbar_init(tcg::smem_u32(mbar), 1);
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  const uint32_t taddr = *taddr_s, bar = tcg::smem_u32(mbar);
  const uint32_t aA = tcg::smem_u32(sA), a1 = tcg::smem_u32(sW1), a2 = tcg::smem_u32(sW2), a3 = tcg::smem_u32(sW3);
  const uint32_t lane_addr = taddr + ((uint32_t)(32 * warp) << 16);
  bool ok = true;
  uint32_t phase = 0;   // completions of the barrier so far (three per tile)
  const int ntiles = (n + TC_ROWS - 1) / TC_ROWS;
  // persistent: the CTA keeps the weights and walks over tiles of 128 rows
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
  const long long row0 = (long long)tile * TC_ROWS;
  // inputs: the 128 x 136 tile is contiguous; coalesced float4 loads, each
  // inside one row (136 is a multiple of 4), rounded to bfloat16
  for (int i = t; i < TC_ROWS * (IN / 4); i += TC_ROWS) {
    const int r = i / (IN / 4), k = 4 * (i % (IN / 4));
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (row0 + r < n) v = *reinterpret_cast<const float4*>(X + (row0 + r) * IN + k);
    const unsigned lo = pack_bf16(v.x, v.y), hi = pack_bf16(v.z, v.w);
    *reinterpret_cast<uint2*>(sA + boff(r, k, 18)) = make_uint2(lo, hi);
    if (Xr && row0 + r < n)
      *reinterpret_cast<float4*>(Xr + (row0 + r) * IN + k) = make_float4(bf16r(v.x), bf16r(v.y), bf16r(v.z), bf16r(v.w));
  }
  *reinterpret_cast<uint4*>(sA + boff(t, IN, 18)) = make_uint4(0u, 0u, 0u, 0u);   // k = 136..143
  tcg::fence_async_smem();
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  const long long row = row0 + t;
  // layer 1: 9 steps of K = 16 (two core matrices each)
  if (t == 0) {
    for (int ks = 0; ks < 9; ++ks)
      tcg::mma_f16(taddr, tcg::sdesc(aA + 256 * ks, 128, 18 * 128), tcg::sdesc(a1 + 256 * ks, 128, 18 * 128),
                   tcg::idesc_bf16(128, 128), ks > 0);
    tcg::commit(bar);
  }
  ok = __syncthreads_and(tcg::mbar_wait(bar, phase & 1));   // the same answer in every thread
  ++phase;
  tcg::fence_after();
  // hidden layers: bias, ReLU, bfloat16, written as the next A operand
  auto hidden = [&](uint32_t col0, const float* bias, float* Hr) {
#pragma unroll 1
    for (int c0 = 0; c0 < HID; c0 += 16) {
      float v[16];
      tcg::ld16(lane_addr + col0 + c0, v);
      tcg::wait_ld();
#pragma unroll
      for (int q = 0; q < 16; ++q) v[q] = bf16r(fmaxf(v[q] + bias[c0 + q], 0.f));
#pragma unroll
      for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4*>(sA + boff(t, c0 + 8 * h, 16)) =
            make_uint4(pack_bf16(v[8 * h + 0], v[8 * h + 1]), pack_bf16(v[8 * h + 2], v[8 * h + 3]),
                       pack_bf16(v[8 * h + 4], v[8 * h + 5]), pack_bf16(v[8 * h + 6], v[8 * h + 7]));
      if (Hr && row < n) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(Hr + row * HID + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      }
    }
  };
  if (ok) hidden(0, sb, H1r);
  tcg::fence_async_smem();
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  if (ok && t == 0) {
    for (int ks = 0; ks < 8; ++ks)
      tcg::mma_f16(taddr + 128, tcg::sdesc(aA + 256 * ks, 128, 16 * 128), tcg::sdesc(a2 + 256 * ks, 128, 16 * 128),
                   tcg::idesc_bf16(128, 128), ks > 0);
    tcg::commit(bar);
  }
  ok = __syncthreads_and(ok && tcg::mbar_wait(bar, phase & 1));
  ++phase;
  tcg::fence_after();
  if (ok) hidden(128, sb + HID, H2r);
  tcg::fence_async_smem();
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  if (ok && t == 0) {
    for (int ks = 0; ks < 8; ++ks)
      tcg::mma_f16(taddr, tcg::sdesc(aA + 256 * ks, 128, 16 * 128), tcg::sdesc(a3 + 256 * ks, 128, 16 * 128),
                   tcg::idesc_bf16(128, 16), ks > 0);
    tcg::commit(bar);
  }
  ok = __syncthreads_and(ok && tcg::mbar_wait(bar, phase & 1));
  ++phase;
  tcg::fence_after();
  if (ok) {
    float z[16];
    tcg::ld16(lane_addr, z);
    tcg::wait_ld();
    if (row < n) {
      const float z0 = z[0] + sb[2 * HID], z1 = z[1] + sb[2 * HID + 1], z2 = z[2] + sb[2 * HID + 2];
      const float m = fmaxf(z0, fmaxf(z1, z2));
      const float e0 = expf(z0 - m), e1 = expf(z1 - m), e2 = expf(z2 - m);
      const float inv = 1.f / (e0 + e1 + e2);
      if (prob) {
        prob[row * OUT + 0] = e0 * inv;
        prob[row * OUT + 1] = e1 * inv;
        prob[row * OUT + 2] = e2 * inv;
      }
      if (flags) {
        int cls = 0;
        if (z1 > z0) cls = 1;
        if (z2 > (cls == 1 ? z1 : z0)) cls = 2;
        flags[row] = (int8_t)(cls - 1);
      }
    }
  } else if ((t & 31) == 0) {
    atomicOr(err, 4);
  }
  // the next tile overwrites the A operand and the accumulators: every
  // thread has read its rows
  tcg::fence_before();
  __syncthreads();
  tcg::fence_after();
  }
  tcg::fence_before();
  __syncthreads();
  if (warp == 0) tcg::dealloc(taddr, 256);
}

// dZ3 = w_y (p - onehot) / sum(w_y); loss partial sums into acc[0] (sum w_y
// (-log p_y)) -- acc[1] holds sum w_y from mlp_wsum.
__global__ void mlp_wsum(const int8_t* __restrict__ y, int n, float w0, float w1, float w2,
                         double* __restrict__ acc) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = y[i];
    s += c == 0 ? w0 : (c == 1 ? w1 : w2);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc + 1, red[0]);
}

__global__ void mlp_dz3(const float* __restrict__ prob, const int8_t* __restrict__ y, int n, float w0,
                        float w1, float w2, const double* __restrict__ acc_in, float* __restrict__ dz,
                        double* __restrict__ acc) {
  __shared__ double red[256];
  const float inv = (float)(1.0 / acc_in[1]);
  double l = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = y[i];
    const float w = c == 0 ? w0 : (c == 1 ? w1 : w2);
    for (int k = 0; k < OUT; ++k) dz[(long long)i * OUT + k] = w * inv * (prob[(long long)i * OUT + k] - (k == c ? 1.f : 0.f));
    l += (double)w * -log((double)prob[(long long)i * OUT + c]);
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(acc, red[0]);
}

// C (M x N, row-major, ldc) = op(A) op(B) over the k range of this split;
// op(A)[m][k] = transA ? A[k * lda + m] : A[m * lda + k], same for B with
// op(B)[k][n].  Partial results of split s go to C + s * M * ldc; a second
// kernel sums the splits in order (deterministic).
constexpr int GT = 32;
__global__ void __launch_bounds__(256)
gemm_f32(const float* __restrict__ A, int lda, int transA, const float* __restrict__ B, int ldb,
         int transB, float* __restrict__ C, int ldc, int M, int N, int K, int kchunk) {
  __shared__ float sA[GT][GT + 1], sB[GT][GT + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 2 x 2 outputs each
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k0 = kb; k0 < ke; k0 += GT) {
    for (int i = threadIdx.x; i < GT * GT; i += 256) {
      const int r = i / GT, c = i % GT;
      const int m = m0 + r, k = k0 + c;
      sA[r][c] = (m < M && k < ke) ? (transA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.f;
      const int kk = k0 + r, nn = n0 + c;
      sB[r][c] = (kk < ke && nn < N) ? (transB ? B[(long long)nn * ldb + kk] : B[(long long)kk * ldb + nn]) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GT; ++k) {
      const float a0 = sA[ty * 2][k], a1 = sA[ty * 2 + 1][k];
      const float b0 = sB[k][tx * 2], b1 = sB[k][tx * 2 + 1];
      acc[0][0] = fmaf(a0, b0, acc[0][0]);
      acc[0][1] = fmaf(a0, b1, acc[0][1]);
      acc[1][0] = fmaf(a1, b0, acc[1][0]);
      acc[1][1] = fmaf(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  float* Cs = C + (long long)blockIdx.z * M * ldc;
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty * 2 + i, nn = n0 + tx * 2 + j;
      if (m < M && nn < N) Cs[(long long)m * ldc + nn] = acc[i][j];
    }
}

__global__ void sum_splits(const float* __restrict__ part, int splits, int count, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(long long)k * count + i];
    out[i] = s;
  }
}

// column sums of an n x c matrix (bias gradients), two passes
__global__ void colsum_partial(const float* __restrict__ Z, int n, int c, int rows_per, float* __restrict__ part) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c) return;
  const int r0 = blockIdx.y * rows_per, r1 = min(n, r0 + rows_per);
  float s = 0.f;
  for (int r = r0; r < r1; ++r) s += Z[(long long)r * c + col];
  part[(long long)blockIdx.y * c + col] = s;
}

__global__ void relu_mask(float* __restrict__ dZ, const float* __restrict__ H, long long count) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    if (!(H[i] > 0.f)) dZ[i] = 0.f;
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                            float* __restrict__ v, int count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const float g = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// features: the state at the 27 points {-1, 0, 1}^3 of every element
__constant__ double c_fw[kMaxN + 1][3][kMaxN + 1];   // h_m at -1, 0, 1

__global__ void mlp_features_kernel(const double* __restrict__ q, const int* __restrict__ hmap,
                                    const int* __restrict__ hang_h, const double* __restrict__ hang_w,
                                    const int* __restrict__ col_level, int N, int nz, int NZ,
                                    long long NG, int ncol, float s0, float s1, float s2, float s3,
                                    float s4, float* __restrict__ F) {
  const int n1 = N + 1, Nq = n1 * n1;
  const long long total = (long long)ncol * nz * 27;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int pnt = (int)(idx % 27);
    const long long e = idx / 27;
    const int col = (int)(e / nz), k = (int)(e % nz);
    const int pa = pnt % 3, pb = (pnt / 3) % 3, pc = pnt / 9;
    double acc[kFields] = {0, 0, 0, 0, 0};
    for (int c = 0; c < n1; ++c) {
      const double wc = c_fw[N][pc][c];
      if (wc == 0.0) continue;
      for (int j = 0; j < n1; ++j) {
        const double wj = c_fw[N][pb][j];
        if (wj == 0.0) continue;
        for (int i = 0; i < n1; ++i) {
          const double wi = c_fw[N][pa][i];
          if (wi == 0.0) continue;
          const double w = wi * wj * wc;
          const int hm = hmap[(long long)col * Nq + i + n1 * j];
          const int kz = k * N + c;
          if (hm >= 0) {
            for (int f = 0; f < kFields; ++f) acc[f] += w * q[(long long)f * NG + (long long)hm * NZ + kz];
          } else {
            const int hk = -1 - hm;
            for (int mm = 0; mm < n1; ++mm) {
              const double ww = w * hang_w[hk * n1 + mm];
              const long long o = (long long)hang_h[hk * n1 + mm] * NZ + kz;
              for (int f = 0; f < kFields; ++f) acc[f] += ww * q[(long long)f * NG + o];
            }
          }
        }
      }
    }
    const float sc[kFields] = {s0, s1, s2, s3, s4};
    float* row = F + e * IN;
    for (int f = 0; f < kFields; ++f) row[f * 27 + pnt] = (float)(acc[f] / sc[f]);
    if (pnt == 0) row[135] = (float)col_level[col];
  }
}

}  // namespace

struct MlpImpl {
  float* P = nullptr;      // master parameters
  float* R = nullptr;      // bfloat16-rounded parameters (float32 storage)
  float* G = nullptr;      // gradients
  float* M1 = nullptr;     // Adam moments
  float* M2 = nullptr;
  __nv_bfloat16* wt = nullptr;  // transposed bfloat16 weights (W1T | W2T | W3T)
  int max_rows = 0;
  float *Xr = nullptr, *H1 = nullptr, *H2 = nullptr, *prob = nullptr, *dz3 = nullptr, *dz2 = nullptr,
        *dz1 = nullptr, *part = nullptr;
  double* acc = nullptr;   // loss, weight sum
  int* err = nullptr;      // bit 4: a bounded wait of the tensor-core forward ran out
  int step = 0;
  int dev = -1;
  int forward_tc = 1;      // 1: tcgen05 forward (mlp_forward_tc), 0: mma.sync forward
};

static int gemm(const float* A, int lda, int tA, const float* B, int ldb, int tB, float* C, int M, int N,
                int K, float* part, size_t part_floats, cudaStream_t st) {
  int splits = std::max(1, std::min(64, K / 512));
  while ((size_t)splits * M * N > part_floats && splits > 1) splits /= 2;
  const int kchunk = ((K + splits - 1) / splits + GT - 1) / GT * GT;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, splits);
  gemm_f32<<<grid, 256, 0, st>>>(A, lda, tA, B, ldb, tB, splits > 1 ? part : C, N, M, N, K, kchunk);
  if (splits > 1) sum_splits<<<std::min(1024, (M * N + 255) / 256), 256, 0, st>>>(part, splits, M * N, C);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

static int colsum(const float* Z, int n, int c, float* out, float* part, cudaStream_t st) {
  const int rows_per = 1024;
  const int chunks = (n + rows_per - 1) / rows_per;
  dim3 grid((c + 127) / 128, chunks);
  colsum_partial<<<grid, 128, 0, st>>>(Z, n, c, rows_per, part);
  sum_splits<<<std::max(1, (c + 255) / 256), 256, 0, st>>>(part, chunks, c, out);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

int mlp_create(unsigned long long seed, int max_rows, void** out) {
  MlpImpl* m = new MlpImpl();
  m->max_rows = max_rows;
  cudaGetDevice(&m->dev);
  const size_t rows = (size_t)std::max(max_rows, 1);
  const size_t part_floats = std::max<size_t>(64 * HID * IN, (rows / 1024 + 1) * IN);
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(p, bytes); };
  A((void**)&m->P, NPARAM * 4);
  A((void**)&m->R, NPARAM * 4);
  A((void**)&m->G, NPARAM * 4);
  A((void**)&m->M1, NPARAM * 4);
  A((void**)&m->M2, NPARAM * 4);
  A((void**)&m->wt, (size_t)(W1T_SZ + W2T_SZ + W3T_SZ) * 2);
  A((void**)&m->Xr, rows * IN * 4);
  A((void**)&m->H1, rows * HID * 4);
  A((void**)&m->H2, rows * HID * 4);
  A((void**)&m->prob, rows * OUT * 4);
  A((void**)&m->dz3, rows * OUT * 4);
  A((void**)&m->dz2, rows * HID * 4);
  A((void**)&m->dz1, rows * HID * 4);
  A((void**)&m->part, part_floats * 4);
  A((void**)&m->acc, 2 * sizeof(double));
  A((void**)&m->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(m->M1, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(m->M2, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(m->G, 0, NPARAM * 4);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FWD_SMEM);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
  if (e == cudaSuccess) {
    // Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from splitmix64 of
    // (seed, index), zero biases
    std::vector<float> h(NPARAM, 0.f);
    auto u01 = [&](unsigned long long i) {
      unsigned long long z = seed * 0x9E3779B97F4A7C15ull + i + 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    const int offs[3] = {OFF_W1, OFF_W2, OFF_W3}, sz[3] = {IN * HID, HID * HID, HID * OUT}, fan[3] = {IN, HID, HID};
    for (int l = 0; l < 3; ++l)
      for (int i = 0; i < sz[l]; ++i) h[offs[l] + i] = (float)((2.0 * u01(offs[l] + i) - 1.0) / std::sqrt((double)fan[l]));
    e = cudaMemcpy(m->P, h.data(), NPARAM * 4, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    std::string msg = cudaGetErrorString(e);
    void* ps[] = {m->P, m->R, m->G, m->M1, m->M2, m->wt, m->Xr, m->H1, m->H2, m->prob, m->dz3, m->dz2, m->dz1, m->part, m->acc,
                m->err};
    for (void* p : ps)
      if (p) cudaFree(p);
    delete m;
    return fail(SEM_ERR_CUDA, "mlp allocation: " + msg);
  }
  mlp_refresh<<<64, 256>>>(m->P, m->wt, m->wt + W1T_SZ, m->wt + W1T_SZ + W2T_SZ, m->R);
  SEM_CUDA_TRY(cudaDeviceSynchronize());
  *out = m;
  return SEM_OK;
}

void mlp_destroy(void* h) {
  MlpImpl* m = (MlpImpl*)h;
  if (!m) return;
  void* ps[] = {m->P, m->R, m->G, m->M1, m->M2, m->wt, m->Xr, m->H1, m->H2, m->prob, m->dz3, m->dz2, m->dz1, m->part, m->acc};
  for (void* p : ps)
    if (p) cudaFree(p);
  delete m;
}

int mlp_params(void* h, float* host, int set, int which) {
  MlpImpl* m = (MlpImpl*)h;
  float* d = which == 0 ? m->P : (which == 1 ? m->G : m->R);
  if (set) {
    SEM_CUDA_TRY(cudaMemcpy(d, host, NPARAM * 4, cudaMemcpyHostToDevice));
    if (which == 0) {
      mlp_refresh<<<64, 256>>>(m->P, m->wt, m->wt + W1T_SZ, m->wt + W1T_SZ + W2T_SZ, m->R);
      SEM_CUDA_TRY(cudaDeviceSynchronize());
    }
  } else {
    SEM_CUDA_TRY(cudaMemcpy(host, d, NPARAM * 4, cudaMemcpyDeviceToHost));
  }
  return SEM_OK;
}

int mlp_param_count() { return NPARAM; }

static void launch_forward(MlpImpl* m, const float* X, int n, float* prob, float* Xr, float* H1, float* H2,
                           int8_t* flags, cudaStream_t st) {
  if (m->forward_tc) {
    ProfScope ps("mlp_forward_tc", st);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (n + TC_ROWS - 1) / TC_ROWS;
    mlp_forward_tc<<<std::min(tiles, 2 * nsm), TC_ROWS, TC_SMEM, st>>>(
        X, n, m->wt, m->wt + W1T_SZ, m->wt + W1T_SZ + W2T_SZ, m->P, prob, Xr, H1, H2, flags, m->err);
    return;
  }
  const int grid = (n + FWD_ROWS - 1) / FWD_ROWS;
  ProfScope ps("mlp_forward", st);
  mlp_forward<<<grid, 128, FWD_SMEM, st>>>(X, n, m->wt, m->wt + W1T_SZ, m->wt + W1T_SZ + W2T_SZ, m->P, prob, Xr,
                                            H1, H2, flags);
}

int mlp_select_forward(void* h, int tc) {
  MlpImpl* m = (MlpImpl*)h;
  if (tc != 0 && tc != 1) return fail(SEM_ERR_ARG, "forward: 0 (mma.sync) or 1 (tcgen05)");
  m->forward_tc = tc;
  return SEM_OK;
}

int mlp_status(void* h, int* status, cudaStream_t st) {
  MlpImpl* m = (MlpImpl*)h;
  int v = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&v, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaMemsetAsync(m->err, 0, sizeof(int), st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  *status = v ? SEM_ERR_TIMEOUT : SEM_OK;
  return SEM_OK;
}

int mlp_forward_api(void* h, const float* X, int n, float* prob, int8_t* flags, cudaStream_t st) {
  MlpImpl* m = (MlpImpl*)h;
  if (n <= 0) return SEM_OK;
  launch_forward(m, X, n, prob, nullptr, nullptr, nullptr, flags, st);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

int mlp_backward_api(void* h, const float* X, const int8_t* y, const float* cw, int n, double* loss_host,
                     cudaStream_t st) {
  MlpImpl* m = (MlpImpl*)h;
  if (n <= 0 || n > m->max_rows) return fail(SEM_ERR_ARG, "row count outside 1..max_rows");
  const size_t part_floats = std::max<size_t>(64 * HID * IN, ((size_t)m->max_rows / 1024 + 1) * IN);
  launch_forward(m, X, n, m->prob, m->Xr, m->H1, m->H2, nullptr, st);
  SEM_CUDA_TRY(cudaMemsetAsync(m->acc, 0, 2 * sizeof(double), st));
  const int rb = std::min(1024, (n + 255) / 256);
  mlp_wsum<<<rb, 256, 0, st>>>(y, n, cw[0], cw[1], cw[2], m->acc);
  mlp_dz3<<<rb, 256, 0, st>>>(m->prob, y, n, cw[0], cw[1], cw[2], m->acc, m->dz3, m->acc);
  int rc;
  ProfScope ps("mlp_backward", st);
  // gW3 = H2r^T dZ3, gb3 = colsum dZ3
  if ((rc = gemm(m->H2, HID, 1, m->dz3, OUT, 0, m->G + OFF_W3, HID, OUT, n, m->part, part_floats, st))) return rc;
  if ((rc = colsum(m->dz3, n, OUT, m->G + OFF_B3, m->part, st))) return rc;
  // dZ2 = (dZ3 W3r^T) * [H2 > 0]
  if ((rc = gemm(m->dz3, OUT, 0, m->R + OFF_W3, OUT, 1, m->dz2, n, HID, OUT, m->part, part_floats, st))) return rc;
  relu_mask<<<1024, 256, 0, st>>>(m->dz2, m->H2, (long long)n * HID);
  if ((rc = gemm(m->H1, HID, 1, m->dz2, HID, 0, m->G + OFF_W2, HID, HID, n, m->part, part_floats, st))) return rc;
  if ((rc = colsum(m->dz2, n, HID, m->G + OFF_B2, m->part, st))) return rc;
  // dZ1 = (dZ2 W2r^T) * [H1 > 0]
  if ((rc = gemm(m->dz2, HID, 0, m->R + OFF_W2, HID, 1, m->dz1, n, HID, HID, m->part, part_floats, st))) return rc;
  relu_mask<<<1024, 256, 0, st>>>(m->dz1, m->H1, (long long)n * HID);
  if ((rc = gemm(m->Xr, IN, 1, m->dz1, HID, 0, m->G + OFF_W1, IN, HID, n, m->part, part_floats, st))) return rc;
  if ((rc = colsum(m->dz1, n, HID, m->G + OFF_B1, m->part, st))) return rc;
  SEM_CUDA_TRY(cudaGetLastError());
  if (loss_host) {
    double a[2];
    SEM_CUDA_TRY(cudaMemcpyAsync(a, m->acc, sizeof(a), cudaMemcpyDeviceToHost, st));
    SEM_CUDA_TRY(cudaStreamSynchronize(st));
    *loss_host = a[0] / a[1];
  }
  return SEM_OK;
}

int mlp_adam_api(void* h, float lr, cudaStream_t st) {
  MlpImpl* m = (MlpImpl*)h;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - std::pow(0.9, m->step)), c2 = (float)(1.0 - std::pow(0.999, m->step));
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(m->P, m->G, m->M1, m->M2, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
  mlp_refresh<<<64, 256, 0, st>>>(m->P, m->wt, m->wt + W1T_SZ, m->wt + W1T_SZ + W2T_SZ, m->R);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

int mlp_features_api(Mesh& mesh, const double* q, const float* scales, float* F, cudaStream_t st) {
  // the interpolation rows of the current device (uploaded on its first use)
  static DeviceOnce once;
  int rc = device_once(once, [] {
    double fw[kMaxN + 1][3][kMaxN + 1] = {};
    for (int N = 2; N <= kMaxN; ++N) {
      const Basis1D& B = basis(N);
      const double pts[3] = {-1.0, 0.0, 1.0};
      for (int p = 0; p < 3; ++p)
        for (int mm = 0; mm <= N; ++mm) {
          double v = lagrange(B.xi, mm, pts[p]);
          for (int r = 0; r <= N; ++r)
            if (pts[p] == B.xi[r]) v = (r == mm) ? 1.0 : 0.0;
          fw[N][p][mm] = v;
        }
    }
    SEM_CUDA_TRY(cudaMemcpyToSymbol(c_fw, fw, sizeof(fw)));
    return SEM_OK;
  });
  if (rc) return rc;
  DeviceTables& D = *mesh.dev;
  const long long total = mesh.Ne() * 27;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  ProfScope ps("mlp_features", st);
  mlp_features_kernel<<<blocks, 256, 0, st>>>(q, D.hmap, D.hang_h, D.hang_w, D.col_level, mesh.N, mesh.nz,
                                              mesh.NZ, mesh.NG, (int)mesh.Ncol(), scales[0], scales[1],
                                              scales[2], scales[3], scales[4], F);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
