// Kernel-block evaluation K'_ij = K(Y[rows_i], X_j), SIMT path (FP64 and mixed).
//
// Kernels: Gaussian (§4.2, eq. gaussian_kernel), Laplace ||x-y||^(2-d)
// (§4.3), polynomial (x.y/h + c)^p (§4.4). The block is the s x n matrix of
// sampled targets against the node's sources (§2.2).
//
// Batched over work items (one item = one sampled block); each CTA walks a
// 64-row x 32-column output tile, staging coordinates through shared memory
// in 32-coordinate chunks. Distances are formed from direct differences in
// FP64. A Laplace block is scaled by its largest entry, which needs the
// block's smallest distance first (a min-reduction pass over the same tiles).
#include <atomic>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int TI = 64, TJ = 32, DC = 32, EVAL_THREADS = 256;

__device__ __forceinline__ int find_item(const EvalItem* items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void atomic_min_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMin(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// MODE 0: Gaussian, 1: Laplace (map), 2: polynomial, 3: Laplace min-distance pass.
// CT: type of the staged coordinates and the distance / inner-product sums;
// OT: type of the stored block. With CT = float and a centre given, the
// coordinates are centred at it in FP64 before rounding to FP32, so the
// differences keep the precision of the node's scale rather than of |x|.
// Squared distance in FP64 from the stored coordinates (the FP64 path's formula).
template <typename TP>
__device__ __forceinline__ double dist2_fp64(const TP* __restrict__ y, const TP* __restrict__ x, int d) {
  double a = 0.0;
  for (int k = 0; k < d; ++k) {
    const double df = ld_point(y + k) - ld_point(x + k);
    a = fma(df, df, a);
  }
  return a;
}

// Mixed-precision Laplace (CT = float, MODE 3 and 1): FP32 centred distances, with
//  * an FP64 recompute where the FP32 distance cancels, D2 < (|y~|^2 + |x~|^2) / 16
//    (the centred norms come with the tile);
//  * in the map, an FP64 recompute of every entry the FP32 distance puts at or above
//    LAP_RECOMPUTE of the block's largest: the map multiplies the distance's relative
//    error by (d - 2) / 2, so only entries that small keep the FP32 distance.
// The block is scaled by the minimum of these distances (the FP32 pass's), a constant
// factor within FP32 rounding of the FP64 path's; J, T and every relative error are
// invariant to it, and the scale is returned with the block.
constexpr float LAP_RECOMPUTE = 1e-6f;

template <typename TP, int MODE, typename CT, typename OT>
__global__ void __launch_bounds__(EVAL_THREADS)
eval_kernel(const TP* __restrict__ Y, const TP* __restrict__ X, int d, ffc_kernel kp,
            const EvalItem* __restrict__ items, int n_items, int64_t total_tiles, double* min_d2) {
  __shared__ CT ys[TI][DC + 1];
  __shared__ CT xs[TJ][DC + 1];
  constexpr bool lap32 = (MODE == 1 || MODE == 3) && sizeof(CT) == 4;
  __shared__ float yns[lap32 ? TI : 1], xns[lap32 ? TJ : 1];
  const int tid = threadIdx.x;
  const int r = tid % TI, cg = tid / TI;   // row in tile, column group (0..3)
  constexpr bool centre = (sizeof(CT) == 4) && (MODE != 2);
  for (int64_t g = blockIdx.x; g < total_tiles; g += gridDim.x) {
    const int q = find_item(items, n_items, g);
    const EvalItem it = items[q];
    const int64_t s = it.s, n = it.n;
    const int64_t rt = it.row_tiles > 0 ? it.row_tiles : 1;
    const int64_t local = g - it.tile_begin;
    const int64_t i0 = (local % rt) * TI, j0 = (local / rt) * TJ;
    if (i0 >= s || j0 >= n) continue;   // tile beyond the rows actually sampled
    const double* ctr = (centre && it.center) ? it.center : nullptr;
    CT acc[TJ / 4];
#pragma unroll
    for (int u = 0; u < TJ / 4; ++u) acc[u] = (CT)0;
    float ynr = 0.0f, xnc = 0.0f;   // lap32: row r's and (tid < TJ) column tid's centred squared norms
    for (int k0 = 0; k0 < d; k0 += DC) {
      const int kc = min(DC, d - k0);
      for (int e = tid; e < TI * DC; e += EVAL_THREADS) {
        int rr = e / DC, kk = e % DC;
        double v = 0.0;
        if (i0 + rr < s && kk < kc) {
          v = ld_point(Y + it.rows[i0 + rr] * (int64_t)d + k0 + kk);
          if (ctr) v -= ctr[k0 + kk];
        }
        ys[rr][kk] = (CT)v;
      }
      for (int e = tid; e < TJ * DC; e += EVAL_THREADS) {
        int cc = e / DC, kk = e % DC;
        double v = 0.0;
        if (j0 + cc < n && kk < kc) {
          v = ld_point(X + (it.x_begin + j0 + cc) * (int64_t)d + k0 + kk);
          if (ctr) v -= ctr[k0 + kk];
        }
        xs[cc][kk] = (CT)v;
      }
      __syncthreads();
      if (lap32) {
        for (int kk = 0; kk < kc; ++kk) {
          const float yv = (float)ys[r][kk];
          ynr = fmaf(yv, yv, ynr);
          if (tid < TJ) {
            const float xv = (float)xs[tid][kk];
            xnc = fmaf(xv, xv, xnc);
          }
        }
      }
      for (int kk = 0; kk < kc; ++kk) {
        const CT y = ys[r][kk];
#pragma unroll
        for (int u = 0; u < TJ / 4; ++u) {
          const CT x = xs[cg + 4 * u][kk];
          if (MODE == 2) {
            acc[u] = fma(y, x, acc[u]);
          } else {
            const CT df = y - x;
            acc[u] = fma(df, df, acc[u]);
          }
        }
      }
      __syncthreads();
    }
    const int64_t i = i0 + r;
    if (lap32) {
      if (cg == 0) yns[r] = ynr;
      if (tid < TJ) xns[tid] = xnc;
      __syncthreads();
      if (i < s) {
#pragma unroll
        for (int u = 0; u < TJ / 4; ++u) {
          const int c = cg + 4 * u;
          const int64_t j = j0 + c;
          if (j < n && (float)acc[u] < 0.0625f * (yns[r] + xns[c]))
            acc[u] = (CT)dist2_fp64(Y + it.rows[i] * (int64_t)d, X + (it.x_begin + j) * (int64_t)d, d);
        }
      }
      __syncthreads();   // the next tile restages the norms
    }
    if (MODE == 3) {
      double mn = INFINITY;
#pragma unroll
      for (int u = 0; u < TJ / 4; ++u)
        if (i < s && j0 + cg + 4 * u < n) mn = fmin(mn, (double)acc[u]);
      for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      if ((tid & 31) == 0 && mn < INFINITY) atomic_min_pos(&min_d2[q], mn);
      continue;
    }
    if (i >= s) continue;
    OT* K = reinterpret_cast<OT*>(it.K);
    const double ln_rmin = (MODE == 1) ? 0.5 * log(min_d2[q]) : 0.0;
#pragma unroll
    for (int u = 0; u < TJ / 4; ++u) {
      const int64_t j = j0 + cg + 4 * u;
      if (j >= n) continue;
      OT v;
      if (sizeof(CT) == 8) {
        const double a = (double)acc[u];
        if (MODE == 0) v = (OT)exp(-a / (2.0 * kp.h * kp.h));
        else if (MODE == 1) v = (OT)exp(-(double)(d - 2) * (0.5 * log(a) - ln_rmin));
        else v = (OT)pow(a / kp.h + kp.c, (double)kp.p);
      } else if (MODE == 1) {
        const float lr = 0.5f * logf((float)acc[u]) - (float)ln_rmin;
        const float v32 = expf(-(float)(d - 2) * lr);
        if (v32 >= LAP_RECOMPUTE) {
          const double a = dist2_fp64(Y + it.rows[i] * (int64_t)d, X + (it.x_begin + j) * (int64_t)d, d);
          v = (OT)exp(-(double)(d - 2) * (0.5 * log(a) - ln_rmin));
        } else {
          v = (OT)v32;
        }
      } else {
        const float a = (float)acc[u];
        if (MODE == 0) {
          v = (OT)expf(-a * (float)(0.5 / (kp.h * kp.h)));
        } else {
          const float base = a * (float)(1.0 / kp.h) + (float)kp.c;
          float pw = base;
          for (int e = 1; e < kp.p; ++e) pw *= base;
          v = (OT)pw;
        }
      }
      K[i + j * it.ldk] = v;
    }
  }
}

__global__ void laplace_scale_kernel(const double* min_d2, int n_items, int d, double* log_scale,
                                     int32_t* status) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_items) return;
  double m = min_d2[q];
  if (!(m > 0.0)) {
    status[q] = FFC_E_SINGULAR;
    log_scale[q] = 0.0;
  } else {
    log_scale[q] = -(double)(d - 2) * 0.5 * log(m);
  }
}

__global__ void fill_kernel(double* p, int n, double v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <typename TP, typename CT, typename OT>
ffc_status launch_eval_t(ffc_kernel k, const TP* Y, const TP* X, int d, const EvalItem* items, int n_items,
                         int64_t total_tiles, double* min_d2, double* log_scale, int32_t* status, cudaStream_t st) {
  int grid = (int)std::min<int64_t>(total_tiles, (int64_t)sm_count() * 16);
  if (grid <= 0) return FFC_OK;
  if (k.kind == FFC_GAUSSIAN) {
    eval_kernel<TP, 0, CT, OT><<<grid, EVAL_THREADS, 0, st>>>(Y, X, d, k, items, n_items, total_tiles, min_d2);
    if (log_scale) FFC_CUDA(cudaMemsetAsync(log_scale, 0, sizeof(double) * n_items, st));
  } else if (k.kind == FFC_POLYNOMIAL) {
    eval_kernel<TP, 2, CT, OT><<<grid, EVAL_THREADS, 0, st>>>(Y, X, d, k, items, n_items, total_tiles, min_d2);
    if (log_scale) FFC_CUDA(cudaMemsetAsync(log_scale, 0, sizeof(double) * n_items, st));
  } else {
    // Laplace: the map amplifies the distances' relative error (d-2)/2 times. FP64: FP64 distances.
    // Mixed: FP32 centred distances with FP64 recomputes (cancellation; entries near the largest).
    fill_kernel<<<(n_items + 255) / 256, 256, 0, st>>>(min_d2, n_items, INFINITY);
    eval_kernel<TP, 3, CT, OT><<<grid, EVAL_THREADS, 0, st>>>(Y, X, d, k, items, n_items, total_tiles, min_d2);
    laplace_scale_kernel<<<(n_items + 255) / 256, 256, 0, st>>>(min_d2, n_items, d, log_scale, status);
    eval_kernel<TP, 1, CT, OT><<<grid, EVAL_THREADS, 0, st>>>(Y, X, d, k, items, n_items, total_tiles, min_d2);
  }
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace

// Mixed precision, Gaussian or polynomial, d >= 64: the tensor cores, by default the tcgen05 path
// (128 x 256 tiles); otherwise the SIMT path (64 x 32 tiles). At small d the block is bound by its
// stores and the SIMT path's direct FP32 differences are the more accurate form. An explicit path
// request takes a tensor-core path for any d, where the kernel and precision allow it.
constexpr int TC_MIN_D = 64;

namespace {
std::atomic<int> g_eval_path{FFC_EVAL_DEFAULT};
}

int eval_default_path() { return g_eval_path.load(std::memory_order_relaxed); }
void set_eval_default_path(int path) { g_eval_path.store(path, std::memory_order_relaxed); }

int eval_shape(ffc_kernel k, int d, int precision, int path) {
  if (path == FFC_EVAL_DEFAULT) path = eval_default_path();
  const bool tc_ok = precision == FFC_MIXED && (k.kind == FFC_GAUSSIAN || k.kind == FFC_POLYNOMIAL);
  if (!tc_ok || path == FFC_EVAL_SIMT) return 0;
  if (path == FFC_EVAL_MMA_SYNC) return 1;
  if (path == FFC_EVAL_TCGEN05) return 2 + FFC_EVAL_TCGEN05_DEFAULT_TILE;
  if (path >= FFC_EVAL_TCGEN05_TILE0 && path < FFC_EVAL_TCGEN05_TILE0 + FFC_EVAL_TCGEN05_TILES)
    return 2 + (path - FFC_EVAL_TCGEN05_TILE0);
  return d >= TC_MIN_D ? 2 + FFC_EVAL_TCGEN05_DEFAULT_TILE : 0;
}

int64_t eval_tiles(int64_t s, int64_t n, int shape) {
  return shape >= 2 ? eval_tc5_tiles(s, n, shape - 2)
         : shape == 1 ? eval_tc_tiles(s, n) : ((s + TI - 1) / TI) * ((n + TJ - 1) / TJ);
}
int64_t eval_row_tiles(int64_t s, int shape) {
  return shape >= 2 ? eval_tc5_row_tiles(s) : shape == 1 ? eval_tc_row_tiles(s) : (s + TI - 1) / TI;
}

ffc_status launch_eval(ffc_kernel k, const void* Y, int dtype, const void* X, int d, int precision, int shape,
                       const EvalItem* items_dev, int n_items, int64_t total_tiles, double* min_d2,
                       double* log_scale, int32_t* status, void* tc5_scratch, int64_t tc5_rows, cudaStream_t st) {
  if (shape >= 2)
    return launch_eval_tc5(k, Y, dtype, X, d, shape - 2, items_dev, n_items, total_tiles, tc5_rows, tc5_scratch,
                           log_scale, status, st);
  if (shape == 1)
    return launch_eval_tc(k, Y, dtype, X, d, items_dev, n_items, total_tiles, log_scale, st);
  if (precision == FFC_MIXED) {
    if (dtype == FFC_F64)
      return launch_eval_t<double, float, float>(k, (const double*)Y, (const double*)X, d, items_dev, n_items,
                                                 total_tiles, min_d2, log_scale, status, st);
    return launch_eval_t<float, float, float>(k, (const float*)Y, (const float*)X, d, items_dev, n_items,
                                              total_tiles, min_d2, log_scale, status, st);
  }
  if (dtype == FFC_F64)
    return launch_eval_t<double, double, double>(k, (const double*)Y, (const double*)X, d, items_dev, n_items,
                                                 total_tiles, min_d2, log_scale, status, st);
  return launch_eval_t<float, double, double>(k, (const float*)Y, (const float*)X, d, items_dev, n_items,
                                              total_tiles, min_d2, log_scale, status, st);
}

}  // namespace ffc
