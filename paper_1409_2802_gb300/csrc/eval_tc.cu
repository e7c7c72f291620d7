// Kernel-block evaluation on the tensor cores (mixed precision, Gaussian and
// polynomial kernels): K'_ij = K(Y[rows_i], X_j) from the inner products
// y_i . x_j (§2.2 block; kernels of §4.2 and §4.4).
//
// The block is a GEMM: D2_ij = ||y_i||^2 + ||x_j||^2 - 2 y_i . x_j (Gaussian,
// coordinates centred at the node centroid) or the plain inner product
// (polynomial). Each FP32 coordinate a is split into three BF16 parts
// a = a_hi + a_mid + a_lo (each the BF16 rounding of the remainder), and the
// product keeps the six partial products whose order is at least 2^-16:
//   hi.hi + hi.mid + mid.hi + hi.lo + lo.hi + mid.mid,
// accumulated in FP32 by mma.sync m16n8k16 (BF16 x BF16 -> FP32). The
// dropped terms are below 2^-24 of |a||b|, so the products carry FP32
// accuracy. Where the Gaussian's D2 cancels (D2 < (||y||^2 + ||x||^2) / 16),
// D2 is recomputed from direct FP32 differences.
//
// Tiles: 128 targets x 128 sources per CTA (8 warps of 64 x 32), 32
// coordinates per stage. Eight threads stage a target or source row, four
// coordinates each, with coalesced 16-byte loads: centred (FP32 points
// against the FP32-rounded centre, FP64 points in FP64), rounded to FP32 and
// split; their partial squared norms are summed in a fixed order at the end
// of the tile.
#include <cuda_bf16.h>

#include <algorithm>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int TC_M = 128, TC_N = 128, TC_K = 32, TC_LD = TC_K + 8, TC_THREADS = 256;

constexpr int TC_MAX_D = 4096;   // the FP32 centre of a block is staged whole

struct EvalTcSmem {
  alignas(16) __nv_bfloat16 A[3][TC_M * TC_LD];   // targets [i][k], planes hi / mid / lo
  alignas(16) __nv_bfloat16 B[3][TC_N * TC_LD];   // sources [j][k]
  float yn[TC_M];
  float xn[TC_N];
  int64_t yrow[TC_M];
  alignas(16) float c32[TC_MAX_D];   // the centre rounded to FP32 (FP32 points)
  float nsum[2 * TC_M][8];             // per row, the partial squared norms of its 8 staging threads
};

__device__ __forceinline__ void ldsm4(const void* p, unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};\n"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ int find_item_tc(const EvalItem* items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Split of one FP32 coordinate into three BF16 parts (each the rounding of the remainder).
__device__ __forceinline__ void split3(float a, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// Four coordinates [k, k + 4) of one row, centred: FP32 points against the FP32 centre (its
// rounding is common to targets and sources and cancels in their differences), FP64 points in
// FP64 before rounding; zero beyond d.
template <typename TP>
__device__ __forceinline__ void load4(const TP* __restrict__ row, int k, int d, bool vec, const double* ctr,
                                     const float* c32, float (&a)[4]);

template <>
__device__ __forceinline__ void load4<float>(const float* __restrict__ row, int k, int d, bool vec, const double* ctr,
                                            const float* c32, float (&a)[4]) {
  if (vec && k + 3 < d) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(row + k));
    a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = k + e < d ? __ldg(row + k + e) : 0.0f;
  }
  if (ctr) {
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = k + e < d ? a[e] - c32[k + e] : 0.0f;
  }
}

template <>
__device__ __forceinline__ void load4<double>(const double* __restrict__ row, int k, int d, bool vec,
                                             const double* ctr, const float* c32, float (&a)[4]) {
  double v[4];
  if (vec && k + 3 < d) {
    const double2 v01 = __ldg(reinterpret_cast<const double2*>(row + k));
    const double2 v23 = __ldg(reinterpret_cast<const double2*>(row + k + 2));
    v[0] = v01.x; v[1] = v01.y; v[2] = v23.x; v[3] = v23.y;
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[e] = k + e < d ? __ldg(row + k + e) : 0.0;
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) a[e] = k + e < d ? (float)(ctr ? v[e] - ctr[k + e] : v[e]) : 0.0f;
}

// MODE 0: Gaussian (centred distances), 2: polynomial (inner products)
template <typename TP, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 2)
eval_tc_kernel(const TP* __restrict__ Y, const TP* __restrict__ X, int d, ffc_kernel kp,
               const EvalItem* __restrict__ items, int n_items, int64_t total_tiles, bool vec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EvalTcSmem& S = *reinterpret_cast<EvalTcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wm = warp & 1, wn = warp >> 1;   // warp tile: rows 64 wm .., columns 32 wn ..
  const int q = lane >> 3;
  const float inv2h2 = (float)(0.5 / (kp.h * kp.h));
  for (int64_t g = blockIdx.x; g < total_tiles; g += gridDim.x) {
    const int qi = find_item_tc(items, n_items, g);
    const EvalItem it = items[qi];
    const int64_t s = it.s, n = it.n;
    const int64_t rt = it.row_tiles > 0 ? it.row_tiles : 1;
    const int64_t local = g - it.tile_begin;
    const int64_t i0 = (local % rt) * TC_M, j0 = (local / rt) * TC_N;
    if (i0 >= s || j0 >= n) continue;   // uniform across the CTA
    const double* ctr = MODE == 0 ? it.center : nullptr;
    __syncthreads();   // the previous tile's epilogue reads S.yn / S.xn / S.yrow / S.c32
    for (int r = tid; r < TC_M; r += TC_THREADS) S.yrow[r] = i0 + r < s ? it.rows[i0 + r] : 0;
    if (ctr && sizeof(TP) == 4)
      for (int k = tid; k < d; k += TC_THREADS) S.c32[k] = (float)ctr[k];
    __syncthreads();
    // staging: rows 0..127 targets, 128..255 sources (rb + 32 it); 8 threads per row, 4 coordinates each
    const int kq = tid & 7, rb = tid >> 3;
#pragma unroll
    for (int it2 = 0; it2 < 8; ++it2) S.nsum[rb + 32 * it2][kq] = 0.0f;
    float acc[4][4][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) acc[mt][nt][0] = acc[mt][nt][1] = acc[mt][nt][2] = acc[mt][nt][3] = 0.0f;
    for (int c0 = 0; c0 < d; c0 += TC_K) {
#pragma unroll
      for (int it2 = 0; it2 < 8; ++it2) {
        const int r = rb + 32 * it2;
        const bool is_a = r < TC_M;
        const int rr = r & (TC_M - 1);
        const bool valid = is_a ? (i0 + rr < s) : (j0 + rr < n);
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (valid) {
          const TP* row = is_a ? Y + S.yrow[rr] * (int64_t)d : X + (it.x_begin + j0 + rr) * (int64_t)d;
          load4<TP>(row, c0 + 4 * kq, d, vec, ctr, S.c32, a);
        }
        __align__(8) __nv_bfloat16 ph[4], pm[4], pl[4];
        float nr = S.nsum[r][kq];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          nr = fmaf(a[e], a[e], nr);
          split3(a[e], ph[e], pm[e], pl[e]);
        }
        S.nsum[r][kq] = nr;
        __nv_bfloat16* base = is_a ? &S.A[0][rr * TC_LD + 4 * kq] : &S.B[0][rr * TC_LD + 4 * kq];
        constexpr int plane = TC_M * TC_LD;
        *reinterpret_cast<uint2*>(base) = *reinterpret_cast<const uint2*>(ph);
        *reinterpret_cast<uint2*>(base + plane) = *reinterpret_cast<const uint2*>(pm);
        *reinterpret_cast<uint2*>(base + 2 * plane) = *reinterpret_cast<const uint2*>(pl);
      }
      __syncthreads();
#pragma unroll
      for (int ks = 0; ks < TC_K / 16; ++ks) {
        unsigned b[3][8];   // plane, (n-tile pair, 4 regs): tiles 0-1 then 2-3
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int np = 0; np < 2; ++np)
            ldsm4(&S.B[p][(32 * wn + np * 16 + (q >> 1) * 8 + (lane & 7)) * TC_LD + ks * 16 + (q & 1) * 8],
                  b[p][4 * np], b[p][4 * np + 1], b[p][4 * np + 2], b[p][4 * np + 3]);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          unsigned a[3][4];
#pragma unroll
          for (int p = 0; p < 3; ++p)
            ldsm4(&S.A[p][(64 * wm + 16 * mt + (lane & 15)) * TC_LD + ks * 16 + (lane >> 4) * 8], a[p][0], a[p][1],
                  a[p][2], a[p][3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const int bo = 4 * (nt >> 1) + 2 * (nt & 1);
            // smallest partial products first
            mma_bf16(acc[mt][nt], a[2], b[0][bo], b[0][bo + 1]);   // lo . hi
            mma_bf16(acc[mt][nt], a[0], b[2][bo], b[2][bo + 1]);   // hi . lo
            mma_bf16(acc[mt][nt], a[1], b[1][bo], b[1][bo + 1]);   // mid . mid
            mma_bf16(acc[mt][nt], a[1], b[0][bo], b[0][bo + 1]);   // mid . hi
            mma_bf16(acc[mt][nt], a[0], b[1][bo], b[1][bo + 1]);   // hi . mid
            mma_bf16(acc[mt][nt], a[0], b[0][bo], b[0][bo + 1]);   // hi . hi
          }
        }
      }
      __syncthreads();
    }
    // row norms: the partial sums of a row's 8 staging threads, in a fixed order
    for (int r = tid; r < 2 * TC_M; r += TC_THREADS) {
      float v = 0.0f;
#pragma unroll
      for (int e = 0; e < 8; ++e) v += S.nsum[r][e];
      if (r < TC_M) S.yn[r] = v; else S.xn[r - TC_M] = v;
    }
    __syncthreads();
    float* K = reinterpret_cast<float*>(it.K);
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int li = 64 * wm + 16 * mt + (lane >> 2) + 8 * (e >> 1);
          const int lj = 32 * wn + 8 * nt + 2 * (lane & 3) + (e & 1);
          const int64_t i = i0 + li, j = j0 + lj;
          if (i >= s || j >= n) continue;
          const float dot = acc[mt][nt][e];
          float v;
          if (MODE == 0) {
            const float ny = S.yn[li], nx = S.xn[lj];
            float d2 = ny + nx - 2.0f * dot;
            if (d2 < 0.0625f * (ny + nx)) {
              // cancellation: direct FP32 differences of the same centred, rounded coordinates
              const TP* yr = Y + S.yrow[li] * (int64_t)d;
              const TP* xr = X + (it.x_begin + j) * (int64_t)d;
              float a2 = 0.0f;
              for (int k = 0; k < d; ++k) {
                float yv, xv;
                if (sizeof(TP) == 4) {
                  yv = (float)__ldg(yr + k);
                  xv = (float)__ldg(xr + k);
                  if (ctr) { yv -= S.c32[k]; xv -= S.c32[k]; }
                } else {
                  double y64 = (double)__ldg(yr + k), x64 = (double)__ldg(xr + k);
                  if (ctr) { y64 -= ctr[k]; x64 -= ctr[k]; }
                  yv = (float)y64;
                  xv = (float)x64;
                }
                const float df = yv - xv;
                a2 = fmaf(df, df, a2);
              }
              d2 = a2;
            }
            v = expf(-fmaxf(d2, 0.0f) * inv2h2);
          } else {
            const float base = dot * (float)(1.0 / kp.h) + (float)kp.c;
            float pw = base;
            for (int t = 1; t < kp.p; ++t) pw *= base;
            v = pw;
          }
          K[i + j * it.ldk] = v;
        }
      }
    }
  }
}

}  // namespace

int64_t eval_tc_tiles(int64_t s, int64_t n) { return ((s + TC_M - 1) / TC_M) * ((n + TC_N - 1) / TC_N); }
int64_t eval_tc_row_tiles(int64_t s) { return (s + TC_M - 1) / TC_M; }

ffc_status launch_eval_tc(ffc_kernel k, const void* Y, int dtype, const void* X, int d, const EvalItem* items_dev,
                          int n_items, int64_t total_tiles, double* log_scale, cudaStream_t st) {
  if (total_tiles <= 0) return FFC_OK;
  FFC_REQUIRE(k.kind == FFC_GAUSSIAN || k.kind == FFC_POLYNOMIAL, "tensor-core evaluation: Gaussian or polynomial");
  FFC_REQUIRE(d <= TC_MAX_D, "tensor-core evaluation: d = %d above %d", d, TC_MAX_D);
  const int grid = (int)std::min<int64_t>(total_tiles, (int64_t)sm_count() * 2);
  const size_t smem = sizeof(EvalTcSmem);
  const size_t esz = dtype == FFC_F64 ? 8 : 4;
  const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(Y) | reinterpret_cast<uintptr_t>(X)) % 16 == 0) &&
                   ((size_t)d * esz) % 16 == 0;
#define FFC_TC_LAUNCH(TP, MODE)                                                                               \
  do {                                                                                                        \
    FFC_CUDA(cudaFuncSetAttribute(eval_tc_kernel<TP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                  (int)smem));                                                                \
    eval_tc_kernel<TP, MODE><<<grid, TC_THREADS, smem, st>>>((const TP*)Y, (const TP*)X, d, k, items_dev,     \
                                                             n_items, total_tiles, vec);                      \
  } while (0)
  if (dtype == FFC_F64) {
    if (k.kind == FFC_GAUSSIAN) FFC_TC_LAUNCH(double, 0); else FFC_TC_LAUNCH(double, 2);
  } else {
    if (k.kind == FFC_GAUSSIAN) FFC_TC_LAUNCH(float, 0); else FFC_TC_LAUNCH(float, 2);
  }
#undef FFC_TC_LAUNCH
  if (log_scale) FFC_CUDA(cudaMemsetAsync(log_scale, 0, sizeof(double) * n_items, st));
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace ffc
