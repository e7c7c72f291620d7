// Learned row proposal: per-row features, the 12-128-128-1 GELU network
// (forward, backward, per-node softmax cross-entropy, Adam) and the weighted
// draw without replacement from a candidate pool.
//
// The network replaces the leverage-score row distribution of §3 (Def.
// "Statistical Leverage"; §4.1.3 "Leverage sampling"), which needs a basis of
// the full far-field block, by a prediction from 12 cheap features. Weights
// are kept as an FP32 master copy and used rounded to FP16 (round to nearest
// even); every product accumulates in FP32.
//
// Layout of the parameter vector (FFC_MLP_PARAMS floats, matrices row-major,
// W[j][k] = weight from input k to unit j):
//   W1 128x12 @0 | b1 128 @1536 | W2 128x128 @1664 | b2 128 @18048 | w3 128 @18176 | b3 @18304
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ffc_internal.cuh"

namespace ffc {

constexpr int NF = FFC_N_FEATURES;   // 12
constexpr int NH = 128;
constexpr int OFF_W1 = 0, OFF_B1 = 1536, OFF_W2 = 1664, OFF_B2 = 18048, OFF_W3 = 18176, OFF_B3 = 18304;
static_assert(OFF_B3 + 1 == FFC_MLP_PARAMS, "parameter layout");
static_assert(NF == 12, "feature count");

constexpr int FT = 64;          // rows per network tile
constexpr int NET_THREADS = 256;

__device__ __forceinline__ float half_round(float w) { return __half2float(__float2half_rn(w)); }

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// Inference GELU, z Phi(z) = z erfc(-z / sqrt 2) / 2, with erfc from the rational
// approximation of Abramowitz & Stegun 7.1.26 (Hastings): for x >= 0,
// erfc(x) ~ (a1 t + a2 t^2 + ... + a5 t^5) e^{-x^2}, t = 1 / (1 + p x), |error| <= 1.5e-7.
// Negative z take erfc directly (no cancellation in 1 + erf). The GELU's error is then
// at most 0.75e-7 |z|, about one FP32 rounding of h for |z| near 1.
__device__ __forceinline__ float gelu_inf(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  float p = fmaf(1.061405429f, t, -1.453152027f);
  p = fmaf(p, t, 1.421413741f);
  p = fmaf(p, t, -0.284496736f);
  p = fmaf(p, t, 0.254829592f);
  const float q = p * t * __expf(-x * x);   // erfc(|z| / sqrt 2)
  return 0.5f * z * (z >= 0.0f ? 2.0f - q : q);
}

// d/dz z Phi(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_prime_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ----------------------------------------------------------------------------
// features
//
// Grid: blockIdx.y = item, blockIdx.x strides over the item's rows. The
// node's centroid and the 8 projection directions are staged in shared
// memory as FP32. Small d: one thread per row; large d: one warp per row.
// All sums and transforms are FP32 (coordinates rounded to FP32 first).

constexpr int FEAT_THREADS = 256;
constexpr int FEAT_SMALL_D = 64;

template <typename TP, bool WARP_PER_ROW>
__global__ void __launch_bounds__(FEAT_THREADS) features_kernel(const TP* __restrict__ Y, int d, const FeatItem* items,
                                                                ffc_kernel k, const double* __restrict__ proj,
                                                                float* __restrict__ out) {
  extern __shared__ __align__(16) float fsm[];   // xc[d], proj[8][d]
  const FeatItem& it = items[blockIdx.y];
  const int64_t cnt = it.count ? *it.count : it.cap;
  const int64_t per_cta = WARP_PER_ROW ? FEAT_THREADS / 32 : FEAT_THREADS;
  if ((int64_t)blockIdx.x * per_cta >= it.cap) return;
  float* xc = fsm;
  float* pj = fsm + d;
  for (int c = threadIdx.x; c < d; c += blockDim.x) xc[c] = (float)it.x_c[c];
  for (int c = threadIdx.x; c < 8 * d; c += blockDim.x) pj[c] = (float)proj[c];
  __syncthreads();
  float rho = (float)(it.radius ? *it.radius : it.radius_host);
  if (!(rho > 0.0f)) rho = 1.0f;
  const int64_t stride = (int64_t)gridDim.x * per_cta;
  if (!WARP_PER_ROW) {
    for (int64_t i = (int64_t)blockIdx.x * per_cta + threadIdx.x; i < it.cap; i += stride) {
      float* o = out + (it.out_begin + i) * NF;
      if (i >= cnt) {
#pragma unroll
        for (int f = 0; f < NF; ++f) o[f] = 0.0f;
        continue;
      }
      const TP* y = Y + it.rows[i] * (int64_t)d;
      FeatSums S{0.f, 0.f, 0.f, 0.f, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
      for (int c = 0; c < d; ++c) {
        const float yv = (float)y[c], xv = xc[c];
        const float dl = yv - xv;
        S.dd = fmaf(dl, dl, S.dd); S.yy = fmaf(yv, yv, S.yy); S.yx = fmaf(yv, xv, S.yx); S.xx = fmaf(xv, xv, S.xx);
#pragma unroll
        for (int q = 0; q < 8; ++q) S.p[q] = fmaf(pj[q * d + c], dl, S.p[q]);
      }
      float v[NF];
      feature_values(S, rho, k, d, v);
#pragma unroll
      for (int f = 0; f < NF; ++f) o[f] = v[f];
    }
  } else {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t i = (int64_t)blockIdx.x * per_cta + warp; i < it.cap; i += stride) {
      float* o = out + (it.out_begin + i) * NF;
      if (i >= cnt) {
        if (lane < NF) o[lane] = 0.0f;
        continue;
      }
      const TP* y = Y + it.rows[i] * (int64_t)d;
      FeatSums S{0.f, 0.f, 0.f, 0.f, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
      for (int c = lane; c < d; c += 32) {
        const float yv = (float)__ldg(y + c), xv = xc[c];
        const float dl = yv - xv;
        S.dd = fmaf(dl, dl, S.dd); S.yy = fmaf(yv, yv, S.yy); S.yx = fmaf(yv, xv, S.yx); S.xx = fmaf(xv, xv, S.xx);
#pragma unroll
        for (int q = 0; q < 8; ++q) S.p[q] = fmaf(pj[q * d + c], dl, S.p[q]);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        S.dd += __shfl_xor_sync(0xffffffffu, S.dd, off);
        S.yy += __shfl_xor_sync(0xffffffffu, S.yy, off);
        S.yx += __shfl_xor_sync(0xffffffffu, S.yx, off);
        S.xx += __shfl_xor_sync(0xffffffffu, S.xx, off);
#pragma unroll
        for (int q = 0; q < 8; ++q) S.p[q] += __shfl_xor_sync(0xffffffffu, S.p[q], off);
      }
      if (lane == 0) {
        float v[NF];
        feature_values(S, rho, k, d, v);
#pragma unroll
        for (int f = 0; f < NF; ++f) o[f] = v[f];
      }
    }
  }
}

// ----------------------------------------------------------------------------
// network: shared tiles and the two dense layers of one 64-row tile
//
// Thread (ty = warp, tx = lane) computes rows 8 ty .. 8 ty + 7 and units
// 4 tx .. 4 tx + 3 of a 64 x 128 layer output.

struct NetWeights {
  alignas(16) __half W2T[NH * NH];     // W2T[k * NH + j] = W2[j][k]
  alignas(16) float W1T[NF * NH];      // W1T[k * NH + j] = W1[j][k]
  alignas(16) float b1[NH];
  alignas(16) float b2[NH];
  alignas(16) float w3[NH];
  float b3;
};

__device__ void load_weights(const float* __restrict__ P, NetWeights& w) {
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) {
    const int j = e / NH, kk = e % NH;
    w.W2T[kk * NH + j] = __float2half_rn(P[OFF_W2 + e]);
  }
  for (int e = threadIdx.x; e < NH * NF; e += blockDim.x) {
    const int j = e / NF, kk = e % NF;
    w.W1T[kk * NH + j] = half_round(P[OFF_W1 + e]);
  }
  for (int j = threadIdx.x; j < NH; j += blockDim.x) {
    w.b1[j] = half_round(P[OFF_B1 + j]);
    w.b2[j] = half_round(P[OFF_B2 + j]);
    w.w3[j] = half_round(P[OFF_W3 + j]);
  }
  if (threadIdx.x == 0) w.b3 = half_round(P[OFF_B3]);
}

// z1 = W1 x + b1 for the thread's 8 x 4 block; X is FT x NF row-major.
__device__ __forceinline__ void layer1(const NetWeights& w, const float* X, int ty, int tx, float z[8][4]) {
  const float4 b = *reinterpret_cast<const float4*>(&w.b1[4 * tx]);
#pragma unroll
  for (int i = 0; i < 8; ++i) { z[i][0] = b.x; z[i][1] = b.y; z[i][2] = b.z; z[i][3] = b.w; }
#pragma unroll
  for (int kk = 0; kk < NF; ++kk) {
    const float4 wv = *reinterpret_cast<const float4*>(&w.W1T[kk * NH + 4 * tx]);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float x = X[(8 * ty + i) * NF + kk];
      z[i][0] = fmaf(wv.x, x, z[i][0]); z[i][1] = fmaf(wv.y, x, z[i][1]);
      z[i][2] = fmaf(wv.z, x, z[i][2]); z[i][3] = fmaf(wv.w, x, z[i][3]);
    }
  }
}

// z2 = W2 h1 + b2; H1 is FT x NH row-major (k contiguous).
__device__ __forceinline__ void layer2(const NetWeights& w, const float* H1, int ty, int tx, float z[8][4]) {
  const float4 b = *reinterpret_cast<const float4*>(&w.b2[4 * tx]);
#pragma unroll
  for (int i = 0; i < 8; ++i) { z[i][0] = b.x; z[i][1] = b.y; z[i][2] = b.z; z[i][3] = b.w; }
#pragma unroll 2
  for (int k0 = 0; k0 < NH; k0 += 4) {
    float4 hv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) hv[i] = *reinterpret_cast<const float4*>(&H1[(8 * ty + i) * NH + k0]);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const __half2* wp = reinterpret_cast<const __half2*>(&w.W2T[(k0 + kk) * NH + 4 * tx]);
      const float2 w01 = __half22float2(wp[0]), w23 = __half22float2(wp[1]);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float h = kk == 0 ? hv[i].x : (kk == 1 ? hv[i].y : (kk == 2 ? hv[i].z : hv[i].w));
        z[i][0] = fmaf(w01.x, h, z[i][0]); z[i][1] = fmaf(w01.y, h, z[i][1]);
        z[i][2] = fmaf(w23.x, h, z[i][2]); z[i][3] = fmaf(w23.y, h, z[i][3]);
      }
    }
  }
}

__device__ __forceinline__ void load_x_tile(const float* __restrict__ F, int64_t row0, int64_t R, float* X) {
  for (int e = threadIdx.x; e < FT * NF; e += blockDim.x) {
    const int64_t r = row0 + e / NF;
    X[e] = r < R ? F[row0 * NF + e] : 0.0f;
  }
}

struct FwdSmem {
  NetWeights w;
  alignas(16) float X[FT * NF];
  alignas(16) float H1[FT * NH];
};

// logits o[r] for R feature rows
__global__ void __launch_bounds__(NET_THREADS) mlp_forward_kernel(const float* __restrict__ P,
                                                                  const float* __restrict__ F, int64_t R,
                                                                  float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FwdSmem& S = *reinterpret_cast<FwdSmem*>(smem_raw);
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
  load_weights(P, S.w);
  const int64_t tiles = (R + FT - 1) / FT;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t row0 = t * FT;
    __syncthreads();
    load_x_tile(F, row0, R, S.X);
    __syncthreads();
    float z[8][4];
    layer1(S.w, S.X, ty, tx, z);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4 h = make_float4(gelu_f(z[i][0]), gelu_f(z[i][1]), gelu_f(z[i][2]), gelu_f(z[i][3]));
      *reinterpret_cast<float4*>(&S.H1[(8 * ty + i) * NH + 4 * tx]) = h;
    }
    __syncthreads();
    layer2(S.w, S.H1, ty, tx, z);
    float po[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      po[i] = 0.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) po[i] = fmaf(S.w.w3[4 * tx + u], gelu_f(z[i][u]), po[i]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i) po[i] += __shfl_xor_sync(0xffffffffu, po[i], off);
    if (tx < 8) {
      float v = po[0];
#pragma unroll
      for (int i = 1; i < 8; ++i) if (tx == i) v = po[i];
      const int64_t r = row0 + 8 * ty + tx;
      if (r < R) logits[r] = v + S.w.b3;
    }
  }
}

// ----------------------------------------------------------------------------
// inference forward on the tensor cores: the 128 x 128 layer as FP16 x FP16
// products with FP32 accumulation (mma.sync m16n8k16); the first layer (K = 12)
// on the FP32 pipes. The FP32 activations h1 enter the product as two FP16
// planes, hi = fp16(h1) and lo = fp16(h1 - hi), so W2 h1 = W2 hi + W2 lo keeps
// h1 to about 2^-22 relative (the FP16 weights are exact in both products):
// the logits are those of FP32 activations, not of FP16-rounded ones.

// Layout: one warp per tile of 16 rows, with no block barrier after the weights are staged.
// The first layer is computed straight into the A fragments of m16n8k16: lane (g, q) =
// (lane / 4, lane % 4) owns rows g and g + 8 and, in k-slice ks, units 16 ks + 2q + {0, 1, 8, 9}.
// Each h1 value is computed once, by the lane whose fragment holds it, so h1 never goes through
// shared memory. The warp's 16 n-tiles of 8 units (64 FP32 accumulators per lane) cover all 128
// units of layer 2. Every value is formed with the same operations in the same order as a
// row-at-a-time evaluation of the network:
// * z1 = b1 + w1[0] x[0] + ... + w1[11] x[11] (one FMA chain);
// * per output unit, k-slices in increasing order, the lo plane's product before the hi plane's;
// * the logit = (sum over units 0..63 + sum over units 64..127) + b3, each half summed over the
//   n-tiles in order and then across the 4 lanes of a row.
constexpr int TC_WARPS = 8;
constexpr int TC_THREADS = 32 * TC_WARPS;
constexpr int TC_WROWS = 16;       // rows per warp tile
constexpr int HS = NH + 8;         // FP16 row stride of W2 in shared memory (272 B: ldmatrix rows hit distinct banks)

struct TcSmem {
  alignas(16) __half W2[NH * HS];   // W2[j][k]: the B operand (k x n, "col")
  alignas(16) float W1[NH * NF];    // W1[j][k], FP16-rounded, row-major (48 B per unit)
  alignas(16) float b1[NH];
  alignas(16) float b2[NH];
  alignas(16) float w3[NH];
  float b3;
};

__device__ __forceinline__ void ldsm_x4(const void* p, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ void mma_16816(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                          unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// h1 of unit j for two rows (x0, x1): GELU(b1 + w1 . x) in FP32, returned as hi = fp16(h),
// lo = fp16(h - hi)
__device__ __forceinline__ void h1_pair(const float* __restrict__ w1row, float b1j, const float (&x0)[NF],
                                        const float (&x1)[NF], __half& h0, __half& l0, __half& h1, __half& l1) {
  const float4* w4 = reinterpret_cast<const float4*>(w1row);
  float za = b1j, zb = b1j;
#pragma unroll
  for (int q = 0; q < NF / 4; ++q) {
    const float4 w = w4[q];
    za = fmaf(w.x, x0[4 * q], za); zb = fmaf(w.x, x1[4 * q], zb);
    za = fmaf(w.y, x0[4 * q + 1], za); zb = fmaf(w.y, x1[4 * q + 1], zb);
    za = fmaf(w.z, x0[4 * q + 2], za); zb = fmaf(w.z, x1[4 * q + 2], zb);
    za = fmaf(w.w, x0[4 * q + 3], za); zb = fmaf(w.w, x1[4 * q + 3], zb);
  }
  const float ga = gelu_inf(za), gb = gelu_inf(zb);
  h0 = __float2half_rn(ga);
  l0 = __float2half_rn(ga - __half2float(h0));
  h1 = __float2half_rn(gb);
  l1 = __float2half_rn(gb - __half2float(h1));
}

__device__ __forceinline__ unsigned pack_h2(__half lo_col, __half hi_col) {
  const __half2 v = __halves2half2(lo_col, hi_col);   // .x (low 16 bits): the lower column
  return *reinterpret_cast<const unsigned*>(&v);
}

__global__ void __launch_bounds__(TC_THREADS, 2) mlp_forward_tc_kernel(const float* __restrict__ P,
                                                                        const float* __restrict__ F, int64_t R,
                                                                        float* __restrict__ logits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < NH * NH; e += blockDim.x) S.W2[(e / NH) * HS + (e % NH)] = __float2half_rn(P[OFF_W2 + e]);
  for (int e = tid; e < NH * NF; e += blockDim.x) S.W1[e] = half_round(P[OFF_W1 + e]);
  for (int j = tid; j < NH; j += blockDim.x) {
    S.b1[j] = half_round(P[OFF_B1 + j]);
    S.b2[j] = half_round(P[OFF_B2 + j]);
    S.w3[j] = half_round(P[OFF_W3 + j]);
  }
  if (tid == 0) S.b3 = half_round(P[OFF_B3]);
  __syncthreads();
  const int g = lane >> 2, q = lane & 3;
  const int64_t tiles = (R + TC_WROWS - 1) / TC_WROWS;
  const int64_t wstride = (int64_t)gridDim.x * TC_WARPS;
  for (int64_t t = (int64_t)blockIdx.x * TC_WARPS + warp; t < tiles; t += wstride) {
    const int64_t ra = t * TC_WROWS + g, rb = ra + 8;
    float xa[NF], xb[NF];
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      xa[k] = ra < R ? __ldg(F + ra * NF + k) : 0.0f;
      xb[k] = rb < R ? __ldg(F + rb * NF + k) : 0.0f;
    }
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) { acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f; }
#pragma unroll 1
    for (int ks = 0; ks < NH / 16; ++ks) {
      // this lane's A fragments of k-slice ks: units u0, u0 + 1 (a0: row g, a1: row g + 8) and
      // u0 + 8, u0 + 9 (a2, a3)
      const int u0 = 16 * ks + 2 * q;
      __half h[4][2], l[4][2];   // [unit][row]
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int u = u0 + (c & 1) + 8 * (c >> 1);
        h1_pair(&S.W1[u * NF], S.b1[u], xa, xb, h[c][0], l[c][0], h[c][1], l[c][1]);
      }
      const unsigned a0 = pack_h2(h[0][0], h[1][0]), a1 = pack_h2(h[0][1], h[1][1]);
      const unsigned a2 = pack_h2(h[2][0], h[3][0]), a3 = pack_h2(h[2][1], h[3][1]);
      const unsigned l0 = pack_h2(l[0][0], l[1][0]), l1 = pack_h2(l[0][1], l[1][1]);
      const unsigned l2 = pack_h2(l[2][0], l[3][0]), l3 = pack_h2(l[2][1], l[3][1]);
      const int qm = lane >> 3;   // ldmatrix: the matrix this lane addresses a row of
#pragma unroll
      for (int np = 0; np < 8; ++np) {
        unsigned b0, b1, b2, b3;
        ldsm_x4(&S.W2[(np * 16 + (qm >> 1) * 8 + (lane & 7)) * HS + ks * 16 + (qm & 1) * 8], b0, b1, b2, b3);
        mma_16816(acc[2 * np], l0, l1, l2, l3, b0, b1);
        mma_16816(acc[2 * np + 1], l0, l1, l2, l3, b2, b3);
        mma_16816(acc[2 * np], a0, a1, a2, a3, b0, b1);
        mma_16816(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
      }
    }
    // epilogue: h2 = GELU(z2 + b2) and w3 . h2, per half of the units; lane holds rows g and g + 8,
    // columns 8 nt + 2q + {0, 1}
    float pa[2], pb[2];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      float sa = 0.0f, sb = 0.0f;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int c = 64 * hf + nt * 8 + 2 * q;
        const float* ac = acc[8 * hf + nt];
        sa = fmaf(S.w3[c], gelu_inf(ac[0] + S.b2[c]), sa);
        sa = fmaf(S.w3[c + 1], gelu_inf(ac[1] + S.b2[c + 1]), sa);
        sb = fmaf(S.w3[c], gelu_inf(ac[2] + S.b2[c]), sb);
        sb = fmaf(S.w3[c + 1], gelu_inf(ac[3] + S.b2[c + 1]), sb);
      }
      sa += __shfl_xor_sync(0xffffffffu, sa, 1);
      sa += __shfl_xor_sync(0xffffffffu, sa, 2);
      sb += __shfl_xor_sync(0xffffffffu, sb, 1);
      sb += __shfl_xor_sync(0xffffffffu, sb, 2);
      pa[hf] = sa;
      pb[hf] = sb;
    }
    if (q == 0) {
      if (ra < R) logits[ra] = (pa[0] + pa[1]) + S.b3;
      if (rb < R) logits[rb] = (pb[0] + pb[1]) + S.b3;
    }
  }
}

// ----------------------------------------------------------------------------
// training: per-node softmax cross-entropy and the backward pass

template <typename T>
__device__ T block_sum(T v, T* red) {   // blockDim.x == 256, deterministic order
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

__device__ float block_max(float v, float* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = red[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) s = fmaxf(s, red[i]);
  return s;
}

// One CTA per node b, targets normalised to q_i = t_i / sum_b t: lse_b,
// loss_b = -sum q (o - lse) = lse - (sum t o) / (sum t), g_o = (softmax - q) / B.
__global__ void __launch_bounds__(256) node_ce_kernel(const float* __restrict__ logits,
                                                      const double* __restrict__ targets,
                                                      const int64_t* __restrict__ node_off, int n_nodes,
                                                      float* __restrict__ g_o, double* __restrict__ loss_part) {
  __shared__ double redd[8];
  __shared__ float redf[8];
  const int b = blockIdx.x;
  const int64_t a = node_off[b], e = node_off[b + 1];
  float mx = -INFINITY;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) mx = fmaxf(mx, logits[i]);
  mx = block_max(mx, redf);
  double se = 0.0, st = 0.0, sto = 0.0;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x) {
    const double o = logits[i], t = targets[i];
    se += exp(o - (double)mx); st += t; sto += t * o;
  }
  se = block_sum(se, redd);
  st = block_sum(st, redd);
  sto = block_sum(sto, redd);
  const double lse = (double)mx + log(se);
  const double inv_t = st > 0.0 ? 1.0 / st : 0.0;
  for (int64_t i = a + threadIdx.x; i < e; i += blockDim.x)
    g_o[i] = (float)((exp((double)logits[i] - lse) - targets[i] * inv_t) / (double)n_nodes);
  if (threadIdx.x == 0) loss_part[b] = (e > a && st > 0.0) ? (lse - sto * inv_t) : 0.0;
}

struct BwdSmem {
  NetWeights w;
  alignas(16) __half W2[NH * NH];      // row-major W2[j][k]
  alignas(16) float X[FT * NF];
  alignas(16) float go[FT];
  alignas(16) float Z1[FT * NH];
  alignas(16) float H1[FT * NH];       // h1, later g_z1
  alignas(16) float GZ2[FT * NH];
  alignas(16) float red[8 * NH];
};

// Gradient partials of one CTA over its row tiles; part: gridDim.x x FFC_MLP_PARAMS.
__global__ void __launch_bounds__(NET_THREADS, 1) mlp_backward_kernel(const float* __restrict__ P,
                                                                      const float* __restrict__ F,
                                                                      const float* __restrict__ g_o, int64_t R,
                                                                      float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BwdSmem& S = *reinterpret_cast<BwdSmem*>(smem_raw);
  const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
  load_weights(P, S.w);
  for (int e = threadIdx.x; e < NH * NH; e += blockDim.x) S.W2[e] = __float2half_rn(P[OFF_W2 + e]);

  float dW2[4][16];            // units 4 tx + u, inputs 16 ty + c
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < 16; ++c) dW2[u][c] = 0.0f;
  float dW1[6];                // unit threadIdx.x / 2, inputs 6 (threadIdx.x & 1) + c
#pragma unroll
  for (int c = 0; c < 6; ++c) dW1[c] = 0.0f;
  float dw3[4] = {0, 0, 0, 0}, db2[4] = {0, 0, 0, 0}, db1[4] = {0, 0, 0, 0};
  float db3 = 0.0f;
  const int j1 = threadIdx.x >> 1, c1 = 6 * (threadIdx.x & 1);

  const int64_t tiles = (R + FT - 1) / FT;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int64_t row0 = t * FT;
    __syncthreads();
    load_x_tile(F, row0, R, S.X);
    for (int e = threadIdx.x; e < FT; e += blockDim.x) S.go[e] = row0 + e < R ? g_o[row0 + e] : 0.0f;
    __syncthreads();
    float z[8][4];
    layer1(S.w, S.X, ty, tx, z);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      *reinterpret_cast<float4*>(&S.Z1[(8 * ty + i) * NH + 4 * tx]) = make_float4(z[i][0], z[i][1], z[i][2], z[i][3]);
      *reinterpret_cast<float4*>(&S.H1[(8 * ty + i) * NH + 4 * tx]) =
          make_float4(gelu_f(z[i][0]), gelu_f(z[i][1]), gelu_f(z[i][2]), gelu_f(z[i][3]));
    }
    if (threadIdx.x == 0) {
      float s = 0.0f;
      for (int r = 0; r < FT; ++r) s += S.go[r];
      db3 += s;
    }
    __syncthreads();
    layer2(S.w, S.H1, ty, tx, z);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float go = S.go[8 * ty + i];
      float g4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        dw3[u] = fmaf(go, gelu_f(z[i][u]), dw3[u]);
        g4[u] = go * S.w.w3[4 * tx + u] * gelu_prime_f(z[i][u]);
        db2[u] += g4[u];
      }
      *reinterpret_cast<float4*>(&S.GZ2[(8 * ty + i) * NH + 4 * tx]) = make_float4(g4[0], g4[1], g4[2], g4[3]);
    }
    __syncthreads();
    // dW2[j][k] += sum_r gz2[r][j] h1[r][k]
    for (int r = 0; r < FT; ++r) {
      const float4 g = *reinterpret_cast<const float4*>(&S.GZ2[r * NH + 4 * tx]);
      const float gg[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const float4 h = *reinterpret_cast<const float4*>(&S.H1[r * NH + 16 * ty + 4 * c4]);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dW2[u][4 * c4 + 0] = fmaf(gg[u], h.x, dW2[u][4 * c4 + 0]);
          dW2[u][4 * c4 + 1] = fmaf(gg[u], h.y, dW2[u][4 * c4 + 1]);
          dW2[u][4 * c4 + 2] = fmaf(gg[u], h.z, dW2[u][4 * c4 + 2]);
          dW2[u][4 * c4 + 3] = fmaf(gg[u], h.w, dW2[u][4 * c4 + 3]);
        }
      }
    }
    // g_h1[r][k] = sum_j W2[j][k] gz2[r][j] for rows 8 ty + i, inputs 4 tx + u
    float gh[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int u = 0; u < 4; ++u) gh[i][u] = 0.0f;
#pragma unroll 2
    for (int j0 = 0; j0 < NH; j0 += 4) {
      float4 gv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) gv[i] = *reinterpret_cast<const float4*>(&S.GZ2[(8 * ty + i) * NH + j0]);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const __half2* wp = reinterpret_cast<const __half2*>(&S.W2[(j0 + jj) * NH + 4 * tx]);
        const float2 w01 = __half22float2(wp[0]), w23 = __half22float2(wp[1]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float g = jj == 0 ? gv[i].x : (jj == 1 ? gv[i].y : (jj == 2 ? gv[i].z : gv[i].w));
          gh[i][0] = fmaf(w01.x, g, gh[i][0]); gh[i][1] = fmaf(w01.y, g, gh[i][1]);
          gh[i][2] = fmaf(w23.x, g, gh[i][2]); gh[i][3] = fmaf(w23.y, g, gh[i][3]);
        }
      }
    }
    __syncthreads();   // every thread is done reading H1 (dW2) before it becomes g_z1
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 z1 = *reinterpret_cast<const float4*>(&S.Z1[(8 * ty + i) * NH + 4 * tx]);
      const float g0 = gh[i][0] * gelu_prime_f(z1.x), g1 = gh[i][1] * gelu_prime_f(z1.y);
      const float g2 = gh[i][2] * gelu_prime_f(z1.z), g3 = gh[i][3] * gelu_prime_f(z1.w);
      db1[0] += g0; db1[1] += g1; db1[2] += g2; db1[3] += g3;
      *reinterpret_cast<float4*>(&S.H1[(8 * ty + i) * NH + 4 * tx]) = make_float4(g0, g1, g2, g3);
    }
    __syncthreads();
    // dW1[j][k] += sum_r gz1[r][j] x[r][k]
    for (int r = 0; r < FT; ++r) {
      const float g = S.H1[r * NH + j1];
#pragma unroll
      for (int c = 0; c < 6; ++c) dW1[c] = fmaf(g, S.X[r * NF + c1 + c], dW1[c]);
    }
  }

  // write this CTA's partial gradient
  float* out = part + (int64_t)blockIdx.x * FFC_MLP_PARAMS;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int c = 0; c < 16; ++c) out[OFF_W2 + (4 * tx + u) * NH + 16 * ty + c] = dW2[u][c];
#pragma unroll
  for (int c = 0; c < 6; ++c) out[OFF_W1 + j1 * NF + c1 + c] = dW1[c];
  // per-unit sums over the 8 row groups (warps), in warp order
  auto emit = [&](const float (&src)[4], int off) {
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) S.red[ty * NH + 4 * tx + u] = src[u];
    __syncthreads();
    if (threadIdx.x < NH) {
      float s = 0.0f;
      for (int w = 0; w < 8; ++w) s += S.red[w * NH + threadIdx.x];
      out[off + threadIdx.x] = s;
    }
  };
  emit(dw3, OFF_W3);
  emit(db2, OFF_B2);
  emit(db1, OFF_B1);
  if (threadIdx.x == 0) out[OFF_B3] = db3;
}

__global__ void grad_reduce_kernel(const float* __restrict__ part, int n_part, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= FFC_MLP_PARAMS) return;
  float s = 0.0f;
  for (int c = 0; c < n_part; ++c) s += part[(int64_t)c * FFC_MLP_PARAMS + p];
  grad[p] = s;
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, double lr, double b1, double b2, double eps,
                            double bc1, double bc2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double gg = g[p];
  const double mm = b1 * (double)m[p] + (1.0 - b1) * gg;
  const double vv = b2 * (double)v[p] + (1.0 - b2) * gg * gg;
  const double mh = mm / bc1, vh = vv / bc2;
  theta[p] = (float)((double)theta[p] - lr * mh / (sqrt(vh) + eps));
  m[p] = (float)mm;
  v[p] = (float)vv;
}

// ----------------------------------------------------------------------------
// weighted draw without replacement (Efraimidis-Spirakis keys), one CTA per pool

constexpr int SEL_THREADS = 1024;
constexpr int SEL_CAP = 16384;      // entries sorted at once in shared memory
constexpr int SEL_MAX_KEEP = 8192;  // largest min(s, P) of one draw

__device__ __forceinline__ bool sel_less(uint64_t ka, uint32_t pa, uint64_t kb, uint32_t pb) {
  return ka < kb || (ka == kb && pa < pb);
}

// Ascending bitonic sort of (key, pos) pairs [0, n) in shared memory, n a power of two.
__device__ void bitonic_sort(uint64_t* key, uint32_t* pos, int n) {
  for (int kk = 2; kk <= n; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & kk) == 0;
          const bool gt = sel_less(key[l], pos[l], key[i], pos[i]);
          if (gt == up) {
            const uint64_t tk = key[i]; key[i] = key[l]; key[l] = tk;
            const uint32_t tp = pos[i]; pos[i] = pos[l]; pos[l] = tp;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Sort key of pool position i: -ln(u_i) / w'_i > 0, whose bit pattern sorts
// ascending exactly as the key ln(u_i) / w'_i sorts descending.
__device__ __forceinline__ uint64_t es_sort_key_w(double w, double mean, uint64_t seed, uint64_t stream_id,
                                                  int64_t i) {
  const double wp = 0.9 * w / mean + 0.1;
  const uint64_t draw = philox_draw(seed, stream_id, DOMAIN_WEIGHTED_KEYS, (uint64_t)i);
  const double u = ((double)(draw >> 11) + 0.5) * 0x1.0p-53;
  return (uint64_t)__double_as_longlong(-log(u) / wp);
}

// the same key from the logit (w = exp(logit - max))
__device__ __forceinline__ uint64_t es_sort_key(float logit, double mx, double mean, uint64_t seed,
                                                uint64_t stream_id, int64_t i) {
  return es_sort_key_w(exp((double)logit - mx), mean, seed, stream_id, i);
}

// One CTA per pool: the min(s, P) pool rows with the largest keys, in key
// order, ties to the lower pool position. Pools of at most SEL_CAP rows are
// sorted whole in shared memory. Larger pools with a key buffer (it.keys)
// take the FP32 pre-selection below: exact keys only for its candidates.
// Otherwise (no buffer, or more than SEL_CAP candidates) the exact sort keys
// are recomputed per pass; a radix select on their bit patterns (SEL_BITS per
// level, a histogram in shared memory) narrows a key prefix until the keys at
// or below it hold the n_keep best and number at most SEL_CAP; those are
// gathered and sorted. Only exact ties of more than SEL_CAP keys (not met
// with distinct draws) take the ordered tie path.
constexpr int SEL_BITS = 12, SEL_BINS = 1 << SEL_BITS;

size_t select_smem_bytes() { return (size_t)SEL_CAP * (sizeof(uint64_t) + sizeof(uint32_t)) + SEL_BINS * sizeof(int); }

// ---- FP32 pre-selection of large pools with stored weights
//
// The n_keep smallest FP64 sort keys k_i are found without computing k_i for every row: an FP32
// approximation k~_i with |k~_i - k_i| <= DELTA k_i (DELTA = 2^-18) ranks the rows, and the exact
// keys are computed only for the rows with k~_i <= T, where T bounds t~ (1 + DELTA) / (1 - DELTA)
// from above and t~ is the n_keep-th smallest k~. That set holds every row of the exact selection:
// the n_keep rows with k~ <= t~ have exact keys <= t~ / (1 - DELTA), so the exact n_keep-th key t
// is at most that, and a selected row's k~ <= (1 + DELTA) k <= (1 + DELTA) t <= T. Sorting the
// set by (exact key, position) then gives the exact selection.
//
// Error of k~ = L~ / w~', first order in u = 2^-24 (IEEE FP32 division and conversions; logf and
// log1pf within 1 ulp, the CUDA maximum-error bound without fast-math):
// * u_d (the FP64 uniform of the exact key) is rebuilt from the integer draw as a correctly rounded
//   FP32 value (relative error u). For u_d < 1/2, L~ = -logf(u~): the conversion moves ln u_d by at
//   most u, and |ln u_d| >= ln 2, so 1.443u, plus 2u for logf. For u_d >= 1/2, L~ = -log1pf(-v~)
//   with v~ the FP32 value of 1 - u_d (exact as an integer): d(-ln(1-v))/dv * v / (-ln(1-v)) <= 1.443
//   on [0, 1/2], so again 1.443u + 2u.
// * w~' = fmaf(0.9f, w~ / m~, 0.1f) with w~, m~ the FP32 values of w and the mean: the ratio 3u,
//   0.9f 1u, 0.1f 1u, the final rounding 1u: at most 5u relative (both terms are positive; a w
//   below the FP32 range only drops a term below 1e-37 of w' >= 0.1).
// * the division: 1u. In all 9.5u ~ 5.7e-7 relative, below DELTA = 64u ~ 3.8e-6.
constexpr float SEL_DELTA4 = 0x1.0p-16f;   // 4 DELTA: T = U (1 + 4 DELTA) > U (1 + DELTA) / (1 - DELTA)

__device__ __forceinline__ float es_key_f32(double w, float mean_f, uint64_t seed, uint64_t stream_id, int64_t i) {
  const uint64_t draw = philox_draw(seed, stream_id, DOMAIN_WEIGHTED_KEYS, (uint64_t)i);
  const uint64_t m = draw >> 11;   // the exact key takes u_d = fl(m + 1/2) 2^-53
  float L;
  if (m < (1ull << 52)) {          // m + 1/2 is exact: u_d = (2m + 1) 2^-54 < 1/2
    L = -logf(__ull2float_rn(2 * m + 1) * 0x1.0p-54f);
  } else {                         // m + 1/2 rounds to the even neighbour; 1 - u_d = (2^53 - that) 2^-53
    const uint64_t me = m + (m & 1ull);
    L = -log1pf(-(__ull2float_rn((1ull << 53) - me) * 0x1.0p-53f));
  }
  const float wp = fmaf(0.9f, (float)w / mean_f, 0.1f);
  return L / wp;
}

// The exact selection's candidates, gathered into pos[0, m) with their exact keys in key[0, m);
// false (and nothing usable in it.keys) when more than SEL_CAP rows pass the threshold.
__device__ bool select_prefiltered(const SelectItem& it, int64_t P, int64_t n_keep, double dmx, double mean,
                                   uint64_t seed, uint64_t* key, uint32_t* pos, int* hist, int& m_out) {
  __shared__ int f_bin, f_fill;
  __shared__ long long f_lt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float mean_f = (float)mean;
  uint64_t* kb = it.keys;   // holds w_i (FP64 bits); overwritten with the bits of k~_i
  unsigned pv = 0;
  long long c_lt = 0;
  for (int level = 0; level < 2; ++level) {   // key bits [31, 20), then [20, 8)
    const int sh = 20 - 12 * level;
    for (int b = tid; b < SEL_BINS; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (int64_t i = tid; i < P; i += blockDim.x) {
      unsigned k;
      if (level == 0) {
        k = __float_as_uint(es_key_f32(__longlong_as_double((long long)kb[i]), mean_f, seed, it.stream_id, i));
        kb[i] = k;
      } else {
        k = (unsigned)kb[i];
      }
      if (level == 0 || (k >> 20) == pv) atomicAdd(&hist[(k >> sh) & (SEL_BINS - 1)], 1);
    }
    __syncthreads();
    if (warp == 0) {   // the bin where the count of smaller keys first reaches n_keep
      constexpr int per = SEL_BINS / 32;
      const int b0 = lane * per;
      long long own = 0;
      for (int b = b0; b < b0 + per; ++b) own += hist[b];
      long long inc = own;
      for (int off = 1; off < 32; off <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += v;
      }
      const long long excl = inc - own;
      if (c_lt + excl < n_keep && c_lt + inc >= n_keep) {
        long long run = c_lt + excl;
        for (int b = b0; b < b0 + per; ++b) {
          if (run + hist[b] >= n_keep) {
            f_bin = b;
            f_lt = run;
            break;
          }
          run += hist[b];
        }
      }
    }
    __syncthreads();
    pv = (pv << 12) | (unsigned)f_bin;
    c_lt = f_lt;
    __syncthreads();
  }
  // t~ lies in the bin of the 24-bit prefix pv, below U; keys are below 400, so pv + 1 does not carry out
  const float U = __uint_as_float((pv + 1u) << 8);
  const unsigned Tb = __float_as_uint(U * (1.0f + SEL_DELTA4));
  if (tid == 0) f_fill = 0;
  __syncthreads();
  for (int64_t i = tid; i < P; i += blockDim.x) {
    if ((unsigned)kb[i] <= Tb) {
      const int slot = atomicAdd(&f_fill, 1);
      if (slot < SEL_CAP) pos[slot] = (uint32_t)i;
    }
  }
  __syncthreads();
  const int m = f_fill;
  if (m > SEL_CAP) return false;
  for (int e = tid; e < m; e += blockDim.x)
    key[e] = es_sort_key(it.logits[pos[e]], dmx, mean, seed, it.stream_id, (int64_t)pos[e]);
  __syncthreads();
  m_out = m;
  return true;
}


// The selection with the ascending sort keys given (it.given): the n_keep smallest keys, in key order,
// ties to the lower pool position (radix narrowing and a shared-memory sort as in select_kernel).
__device__ void select_given(const SelectItem& it, int64_t P, int64_t n_keep, uint64_t* key, uint32_t* pos,
                             int* hist) {
  __shared__ int s_bin, s_fill;
  __shared__ long long s_lt, s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t* gk = it.given;
  int m = 0;
  if (P <= SEL_CAP) {
    m = (int)P;
    for (int e = tid; e < m; e += blockDim.x) {
      key[e] = gk[e];
      pos[e] = (uint32_t)e;
    }
    __syncthreads();
  } else {
    uint64_t pv = 0;
    int pl = 0;
    long long c_lt = 0, c_in = P;
    while (pl < 64 && c_lt + c_in > SEL_CAP) {
      const int nb = min(SEL_BITS, 64 - pl);
      const int sh = 64 - pl - nb;
      const int bins = 1 << nb;
      for (int b = tid; b < bins; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      for (int64_t i = tid; i < P; i += blockDim.x) {
        const uint64_t k = gk[i];
        if (pl == 0 || (k >> (64 - pl)) == pv) atomicAdd(&hist[(int)((k >> sh) & (uint64_t)(bins - 1))], 1);
      }
      __syncthreads();
      if (warp == 0) {
        const int per = (bins + 31) / 32;
        const int b0 = lane * per;
        long long own = 0;
        for (int b = b0; b < b0 + per && b < bins; ++b) own += hist[b];
        long long inc = own;
        for (int off = 1; off < 32; off <<= 1) {
          const long long v = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += v;
        }
        const long long excl = inc - own;
        if (c_lt + excl < n_keep && c_lt + inc >= n_keep) {
          long long run = c_lt + excl;
          for (int b = b0; b < b0 + per && b < bins; ++b) {
            if (run + hist[b] >= n_keep) {
              s_bin = b;
              s_lt = run;
              s_cnt = hist[b];
              break;
            }
            run += hist[b];
          }
        }
      }
      __syncthreads();
      pv = (pv << nb) | (uint64_t)s_bin;
      pl += nb;
      c_lt = s_lt;
      c_in = s_cnt;
      __syncthreads();
    }
    if (tid == 0) s_fill = 0;
    __syncthreads();
    const bool ties = c_lt + c_in > SEL_CAP;
    for (int64_t i = tid; i < P; i += blockDim.x) {
      const uint64_t k = gk[i];
      if (ties ? k < pv : (k >> (64 - pl)) <= pv) {
        const int slot = atomicAdd(&s_fill, 1);
        key[slot] = k;
        pos[slot] = (uint32_t)i;
      }
    }
    __syncthreads();
    if (ties && warp == 0) {
      int fill = s_fill;
      for (int64_t base = 0; base < P && fill < n_keep; base += 32) {
        const int64_t i = base + lane;
        const bool eq = i < P && gk[i] == pv;
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        const int rank = __popc(bal & ((1u << lane) - 1u));
        if (eq && fill + rank < n_keep) {
          key[fill + rank] = pv;
          pos[fill + rank] = (uint32_t)i;
        }
        fill = min((int)n_keep, fill + __popc(bal));
      }
      if (lane == 0) s_fill = fill;
    }
    __syncthreads();
    m = s_fill;
  }
  int Pp = 1;
  while (Pp < m) Pp <<= 1;
  for (int e = m + tid; e < Pp; e += blockDim.x) {
    key[e] = ~0ull;
    pos[e] = 0xFFFFFFFFu;
  }
  __syncthreads();
  bitonic_sort(key, pos, Pp);
  for (int64_t i = tid; i < n_keep; i += blockDim.x) it.rows_out[i] = it.pool[pos[i]];
}

__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const SelectItem* items, uint64_t seed) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SelectItem& it = items[blockIdx.x];
  const int64_t P = it.count ? *it.count : it.P;
  const int64_t n_keep = P < it.s ? P : it.s;
  if (threadIdx.x == 0 && it.s_out) *it.s_out = n_keep;
  if (n_keep <= 0) return;
  if (P > SEL_CAP && n_keep > SEL_MAX_KEEP) return;   // rejected on the host
  uint64_t* key = reinterpret_cast<uint64_t*>(smem_raw);
  uint32_t* pos = reinterpret_cast<uint32_t*>(key + SEL_CAP);
  int* hist = reinterpret_cast<int*>(pos + SEL_CAP);
  __shared__ double redd[32];
  __shared__ float redf[32];
  __shared__ int s_bin, s_fill;
  __shared__ long long s_lt, s_cnt;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (it.given) {
    select_given(it, P, n_keep, key, pos, hist);
    return;
  }
  float mx = -INFINITY;
  for (int64_t i = tid; i < P; i += blockDim.x) mx = fmaxf(mx, it.logits[i]);
  for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (lane == 0) redf[warp] = mx;
  __syncthreads();
  mx = redf[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmaxf(mx, redf[i]);
  // with a key buffer (large pools), w_i = exp(o_i - max) is kept there for the key pass
  const bool keep_w = it.keys != nullptr && P > SEL_CAP;
  double sw = 0.0;
  for (int64_t i = tid; i < P; i += blockDim.x) {
    const double w = exp((double)it.logits[i] - (double)mx);
    if (keep_w) it.keys[i] = (uint64_t)__double_as_longlong(w);
    sw += w;
  }
  for (int off = 16; off > 0; off >>= 1) sw += __shfl_xor_sync(0xffffffffu, sw, off);
  if (lane == 0) redd[warp] = sw;
  __syncthreads();
  sw = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) sw += redd[i];
  const double mean = sw / (double)P;
  const double dmx = (double)mx;
  auto key_of = [&](int64_t i) -> uint64_t { return es_sort_key(it.logits[i], dmx, mean, seed, it.stream_id, i); };
  int m = 0;
  // large pools with a key buffer: FP32 pre-selection, exact keys for the candidates only; when it
  // overflows, the exact radix selection below recomputes every key (the buffer no longer holds w)
  const bool pre = keep_w && select_prefiltered(it, P, n_keep, dmx, mean, seed, key, pos, hist, m);
  if (pre) {
  } else if (P <= SEL_CAP) {
    m = (int)P;
    for (int e = tid; e < m; e += blockDim.x) {
      key[e] = key_of(e);
      pos[e] = (uint32_t)e;
    }
  } else {
    uint64_t pv = 0;        // the top pl bits of the selected prefix
    int pl = 0;
    long long c_lt = 0;     // keys below the prefix range
    long long c_in = P;     // keys inside it
    while (pl < 64 && c_lt + c_in > SEL_CAP) {
      const int nb = min(SEL_BITS, 64 - pl);
      const int sh = 64 - pl - nb;
      const int bins = 1 << nb;
      for (int b = tid; b < bins; b += blockDim.x) hist[b] = 0;
      __syncthreads();
      for (int64_t i = tid; i < P; i += blockDim.x) {
        const uint64_t k = key_of(i);
        if (pl == 0 || (k >> (64 - pl)) == pv) atomicAdd(&hist[(int)((k >> sh) & (uint64_t)(bins - 1))], 1);
      }
      __syncthreads();
      if (warp == 0) {
        // the bin where c_lt + (keys in lower bins) + (its own keys) first reaches n_keep
        const int per = (bins + 31) / 32;
        const int b0 = lane * per;
        long long own = 0;
        for (int b = b0; b < b0 + per && b < bins; ++b) own += hist[b];
        long long inc = own;
        for (int off = 1; off < 32; off <<= 1) {
          const long long v = __shfl_up_sync(0xffffffffu, inc, off);
          if (lane >= off) inc += v;
        }
        const long long excl = inc - own;
        const bool cross = c_lt + excl < n_keep && c_lt + inc >= n_keep;
        if (cross) {
          long long run = c_lt + excl;
          for (int b = b0; b < b0 + per && b < bins; ++b) {
            if (run + hist[b] >= n_keep) {
              s_bin = b;
              s_lt = run;
              s_cnt = hist[b];
              break;
            }
            run += hist[b];
          }
        }
      }
      __syncthreads();
      pv = (pv << nb) | (uint64_t)s_bin;
      pl += nb;
      c_lt = s_lt;
      c_in = s_cnt;
      __syncthreads();
    }
    if (tid == 0) s_fill = 0;
    __syncthreads();
    const bool ties = c_lt + c_in > SEL_CAP;   // pl == 64: more than SEL_CAP keys equal pv
    for (int64_t i = tid; i < P; i += blockDim.x) {
      const uint64_t k = key_of(i);
      const bool take = ties ? k < pv : (k >> (64 - pl)) <= pv;
      if (take) {
        const int slot = atomicAdd(&s_fill, 1);
        key[slot] = k;
        pos[slot] = (uint32_t)i;
      }
    }
    __syncthreads();
    if (ties && warp == 0) {
      // the lowest positions among the keys equal to pv, in position order
      int fill = s_fill;
      for (int64_t base = 0; base < P && fill < n_keep; base += 32) {
        const int64_t i = base + lane;
        const bool eq = i < P && key_of(i) == pv;
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        const int rank = __popc(bal & ((1u << lane) - 1u));
        if (eq && fill + rank < n_keep) {
          key[fill + rank] = pv;
          pos[fill + rank] = (uint32_t)i;
        }
        fill = min((int)n_keep, fill + __popc(bal));
      }
      if (lane == 0) s_fill = fill;
    }
    __syncthreads();
    m = s_fill;
  }
  int Pp = 1;
  while (Pp < m) Pp <<= 1;
  for (int e = m + tid; e < Pp; e += blockDim.x) {
    key[e] = ~0ull;
    pos[e] = 0xFFFFFFFFu;
  }
  __syncthreads();
  bitonic_sort(key, pos, Pp);
  for (int64_t i = tid; i < n_keep; i += blockDim.x) it.rows_out[i] = it.pool[pos[i]];
}

// ----------------------------------------------------------------------------
// launchers

static int net_grid(int64_t R, int per_sm) {
  const int64_t tiles = (R + FT - 1) / FT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sm_count() * per_sm));
}

ffc_status launch_features(ffc_kernel k, const void* Y, int dtype, int d, const FeatItem* items_dev, int n_items,
                           int64_t cap_max, const double* proj, float* out, cudaStream_t st) {
  if (cap_max <= 0 || n_items <= 0) return FFC_OK;
  FFC_REQUIRE(n_items <= 65535, "features: at most 65535 items per launch");
  const size_t smem = (size_t)9 * d * sizeof(float);
  FFC_REQUIRE(smem <= 200 * 1024, "features: d = %d too large", d);
  const bool warp_rows = d > FEAT_SMALL_D;
  const int64_t per_cta = warp_rows ? FEAT_THREADS / 32 : FEAT_THREADS;
  // enough CTAs for about 8 per SM over all items, each striding over its item
  int64_t gx = std::max<int64_t>(1, std::min<int64_t>((cap_max + per_cta - 1) / per_cta,
                                                      std::max<int64_t>(1, (int64_t)sm_count() * 8 / n_items)));
  gx = std::min<int64_t>(gx, 65535);
  const dim3 grid((unsigned)gx, (unsigned)n_items);
#define FFC_FEAT_LAUNCH(TP, WR)                                                                              \
  do {                                                                                                       \
    auto kfn = features_kernel<TP, WR>;                                                                      \
    FFC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));             \
    kfn<<<grid, FEAT_THREADS, smem, st>>>((const TP*)Y, d, items_dev, k, proj, out);                         \
  } while (0)
  if (dtype == FFC_F64) {
    if (warp_rows) FFC_FEAT_LAUNCH(double, true); else FFC_FEAT_LAUNCH(double, false);
  } else {
    if (warp_rows) FFC_FEAT_LAUNCH(float, true); else FFC_FEAT_LAUNCH(float, false);
  }
#undef FFC_FEAT_LAUNCH
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

// training forward: FP32 activations throughout (the backward recomputes them the same way)
static ffc_status launch_mlp_forward_f32(const float* params, const float* feats, int64_t R, float* logits,
                                         cudaStream_t st) {
  if (R <= 0) return FFC_OK;
  const size_t smem = sizeof(FwdSmem);
  FFC_CUDA(cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  mlp_forward_kernel<<<net_grid(R, 2), NET_THREADS, smem, st>>>(params, feats, R, logits);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

// inference forward: the 128 x 128 layer on the tensor cores (FP16 weights, two FP16 planes of h1)
ffc_status launch_mlp_forward(const float* params, const float* feats, int64_t R, float* logits, cudaStream_t st) {
  if (R <= 0) return FFC_OK;
  const size_t smem = sizeof(TcSmem);
  FFC_CUDA(cudaFuncSetAttribute(mlp_forward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ctas = (R + TC_WROWS * TC_WARPS - 1) / (TC_WROWS * TC_WARPS);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)sm_count() * 2));
  mlp_forward_tc_kernel<<<grid, TC_THREADS, smem, st>>>(params, feats, R, logits);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

ffc_status launch_select(const SelectItem* items_dev, int n_items, int64_t keep_max, uint64_t seed, cudaStream_t st) {
  if (n_items <= 0) return FFC_OK;
  if (keep_max > SEL_MAX_KEEP) {
    set_error("weighted draw of %lld rows exceeds %d", (long long)keep_max, SEL_MAX_KEEP);
    return FFC_E_INVALID;
  }
  const size_t smem = select_smem_bytes();
  FFC_CUDA(cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  select_kernel<<<n_items, SEL_THREADS, smem, st>>>(items_dev, seed);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

ffc_status launch_mlp_loss_grad(const float* params, const float* feats, const double* targets,
                                const int64_t* node_off_dev, int n_nodes, int64_t R, float* logits, float* g_o,
                                double* loss_part, float* part, int n_part, float* grad, cudaStream_t st) {
  FFC_REQUIRE(n_part >= 1, "gradient partial count must be >= 1");
  ffc_status rc = launch_mlp_forward_f32(params, feats, R, logits, st);
  if (rc != FFC_OK) return rc;
  node_ce_kernel<<<n_nodes, 256, 0, st>>>(logits, targets, node_off_dev, n_nodes, g_o, loss_part);
  FFC_CUDA(cudaGetLastError());
  const size_t smem = sizeof(BwdSmem);
  FFC_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  mlp_backward_kernel<<<n_part, NET_THREADS, smem, st>>>(params, feats, g_o, R, part);
  FFC_CUDA(cudaGetLastError());
  grad_reduce_kernel<<<(FFC_MLP_PARAMS + 255) / 256, 256, 0, st>>>(part, n_part, grad);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

int mlp_backward_grid(int64_t R) { return net_grid(R, 1); }

ffc_status launch_adam(float* theta, const float* g, float* m, float* v, int64_t n, int64_t step, double lr,
                       double b1, double b2, double eps, cudaStream_t st) {
  if (n <= 0) return FFC_OK;
  const double bc1 = 1.0 - std::pow(b1, (double)step), bc2 = 1.0 - std::pow(b2, (double)step);
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace ffc
