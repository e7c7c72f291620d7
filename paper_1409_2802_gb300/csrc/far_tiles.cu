// Far-field lists and proposal features of many tree nodes at once.
//
// For the learned proposal every node scores its whole far field
// T = {y outside the node : ||y - x_c|| >= xi rho} (§4.1 steps 2-3), so a
// level of a tree touches (points x nodes) pairs. Instead of one thread per
// pair with a serial FP64 distance, a CTA takes a tile of 128 points (one
// per thread), stages their coordinates in shared memory as FP32 and runs
// them against 16 nodes, reading each point tile once per 16 nodes.
//
// Membership stays the FP64 test of the uniform sampler: the FP32 distance
// decides only where it is further from the threshold than its rounding
// error bound, and the few pairs inside that band are retested in FP64.
// Bound, for y and x_c rounded to FP32 (u = 2^-24) and the sum of squares
// of the d rounded differences accumulated in FP32:
//   |r2_32 - r2| <= 8 u (||y||^2 + ||x_c||^2) + (d + 1) u r2_32 (+ O(u^2)),
// used with a factor of two on the first term and 1.1 on the second.
//
// Pass 1 (far_mark) writes one bit per pair and the far count of every
// (node, point tile); an exclusive scan gives each tile's first list
// position; pass 2 (far_features) recomputes the FP32 distance and writes
// the ascending far-field list and the 12 features of every far pair. The
// projections are <g_q, y> - <g_q, x_c>, with <g_q, y> computed once per
// point (point_stats) and <g_q, x_c> once per node (node_stats).
#include <algorithm>

#include "ffc_internal.cuh"

namespace ffc {

constexpr int FT_PTS = 128;   // points per tile, one thread each
constexpr int FT_NB = 16;     // nodes per CTA
constexpr int FT_DC = 32;     // coordinates staged per pass

struct TileNode {
  float xx;      // sum of squares of the FP32 centroid
  float rho;     // radius as FP32 (1 when not positive)
  float xg[8];   // <g_q, x_c> of the FP32 centroid and directions
  double thr2;   // (xi radius)^2 in FP64
};

int64_t far_tiles_count(int64_t N) { return (N + FT_PTS - 1) / FT_PTS; }

size_t far_tiles_node_bytes(int n_items, int d) {
  return (size_t)n_items * (sizeof(TileNode) + (size_t)d * sizeof(float));
}

// one warp per point: yy = sum of squares, yg[q] = <g_q, y>, all FP32 on FP32-rounded values
template <typename TP>
__global__ void point_stats_kernel(const TP* __restrict__ Y, int64_t N, int d, const double* __restrict__ proj,
                                   float* __restrict__ yy, float* __restrict__ yg) {
  extern __shared__ __align__(16) float pj[];   // 8 x d
  for (int c = threadIdx.x; c < 8 * d; c += blockDim.x) pj[c] = (float)proj[c];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < N; j += warps) {
    const TP* y = Y + j * (int64_t)d;
    float s = 0.0f, g[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c = lane; c < d; c += 32) {
      const float v = (float)__ldg(y + c);
      s = fmaf(v, v, s);
#pragma unroll
      for (int q = 0; q < 8; ++q) g[q] = fmaf(pj[q * d + c], v, g[q]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, off);
#pragma unroll
      for (int q = 0; q < 8; ++q) g[q] += __shfl_xor_sync(0xffffffffu, g[q], off);
    }
    if (lane == 0) {
      yy[j] = s;
#pragma unroll
      for (int q = 0; q < 8; ++q) yg[j * 8 + q] = g[q];
    }
  }
}

// one CTA per node: FP32 centroid, its squared norm and projections, the FP64 threshold
__global__ void node_stats_kernel(const FarItem* __restrict__ items, int d, const double* __restrict__ proj,
                                  float* __restrict__ xc32, TileNode* __restrict__ nodes) {
  __shared__ float red[9][32];
  const FarItem& it = items[blockIdx.x];
  float* xc = xc32 + (int64_t)blockIdx.x * d;
  float v9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    const float v = (float)it.x_c[c];
    xc[c] = v;
    v9[0] = fmaf(v, v, v9[0]);
#pragma unroll
    for (int q = 0; q < 8; ++q) v9[1 + q] = fmaf((float)proj[q * d + c], v, v9[1 + q]);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q)
    for (int off = 16; off > 0; off >>= 1) v9[q] += __shfl_xor_sync(0xffffffffu, v9[q], off);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < 9; ++q) red[q][w] = v9[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    TileNode nd;
    float t9[9];
    for (int q = 0; q < 9; ++q) {
      float s = 0.0f;
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += red[q][ww];
      t9[q] = s;
    }
    nd.xx = t9[0];
    for (int q = 0; q < 8; ++q) nd.xg[q] = t9[1 + q];
    float rho = (float)(it.radius ? *it.radius : it.radius_host);
    nd.rho = rho > 0.0f ? rho : 1.0f;
    nd.thr2 = far_thr2(it);
    nodes[blockIdx.x] = nd;
  }
}

// Stage coordinates [c0, c0 + FT_DC) of the tile's points (transposed, FP32) and of the CTA's node
// centroids; zero beyond d, beyond N and beyond the last node, so padded terms add exactly zero.
template <typename TP>
__device__ __forceinline__ void stage_chunk(const TP* __restrict__ Y, int64_t N, int d, int c0, int64_t j0,
                                            const float* __restrict__ xc32, int nb0, int nbn,
                                            float (*ys)[FT_PTS + 1], float (*xs)[FT_DC]) {
  const int dc = min(FT_DC, d - c0);
  for (int e = threadIdx.x; e < FT_PTS * FT_DC; e += FT_PTS) {
    const int r = e / FT_DC, k = e % FT_DC;
    const int64_t j = j0 + r;
    ys[k][r] = (k < dc && j < N) ? (float)__ldg(Y + j * (int64_t)d + c0 + k) : 0.0f;
  }
  for (int e = threadIdx.x; e < FT_NB * FT_DC; e += FT_PTS) {
    const int nb = e / FT_DC, k = e % FT_DC;
    xs[nb][k] = (nb < nbn && k < dc) ? xc32[(int64_t)(nb0 + nb) * d + c0 + k] : 0.0f;
  }
}

// acc[nb] += sum_k (y_k - x_k)^2 over one staged chunk (and yx[nb] += sum_k y_k x_k when DOT)
template <bool DOT>
__device__ __forceinline__ void chunk_sums(int dc, const float (*ys)[FT_PTS + 1], const float (*xs)[FT_DC],
                                           float (&acc)[FT_NB], float (&yx)[FT_NB]) {
  const int t = threadIdx.x;
  const int dc4 = (dc + 3) & ~3;
  for (int k = 0; k < dc4; k += 4) {
    const float y0 = ys[k][t], y1 = ys[k + 1][t], y2 = ys[k + 2][t], y3 = ys[k + 3][t];
#pragma unroll
    for (int nb = 0; nb < FT_NB; ++nb) {
      const float4 x = *reinterpret_cast<const float4*>(&xs[nb][k]);
      float dl = y0 - x.x;
      acc[nb] = fmaf(dl, dl, acc[nb]);
      dl = y1 - x.y;
      acc[nb] = fmaf(dl, dl, acc[nb]);
      dl = y2 - x.z;
      acc[nb] = fmaf(dl, dl, acc[nb]);
      dl = y3 - x.w;
      acc[nb] = fmaf(dl, dl, acc[nb]);
      if (DOT) {
        yx[nb] = fmaf(y0, x.x, yx[nb]);
        yx[nb] = fmaf(y1, x.y, yx[nb]);
        yx[nb] = fmaf(y2, x.z, yx[nb]);
        yx[nb] = fmaf(y3, x.w, yx[nb]);
      }
    }
  }
}

template <typename TP, bool DOT>
__device__ __forceinline__ void tile_distances(const TP* __restrict__ Y, int64_t N, int d, int64_t j0,
                                               const float* __restrict__ xc32, int nb0, int nbn,
                                               float (*ys)[FT_PTS + 1], float (*xs)[FT_DC], float (&acc)[FT_NB],
                                               float (&yx)[FT_NB]) {
#pragma unroll
  for (int nb = 0; nb < FT_NB; ++nb) acc[nb] = yx[nb] = 0.0f;
  for (int c0 = 0; c0 < d; c0 += FT_DC) {
    stage_chunk(Y, N, d, c0, j0, xc32, nb0, nbn, ys, xs);
    __syncthreads();
    chunk_sums<DOT>(min(FT_DC, d - c0), ys, xs, acc, yx);
    __syncthreads();
  }
}

// grid: x = point tile, y = node batch of FT_NB; block FT_PTS threads
template <typename TP>
__global__ void __launch_bounds__(FT_PTS) far_mark_kernel(const TP* __restrict__ Y, int64_t N, int d,
                                                          const FarItem* __restrict__ items, int n_items,
                                                          const float* __restrict__ xc32,
                                                          const TileNode* __restrict__ nodes,
                                                          const float* __restrict__ yy, int64_t tiles,
                                                          int64_t* __restrict__ tile_cnt, uint32_t* __restrict__ mask) {
  __shared__ float ys[FT_DC][FT_PTS + 1];
  __shared__ __align__(16) float xs[FT_NB][FT_DC];
  __shared__ int wc[FT_NB][FT_PTS / 32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * FT_PTS, j = j0 + t;
  const int nb0 = blockIdx.y * FT_NB, nbn = min(FT_NB, n_items - nb0);
  const int64_t words = tiles * (FT_PTS / 32);
  float acc[FT_NB], yx[FT_NB];
  tile_distances<TP, false>(Y, N, d, j0, xc32, nb0, nbn, ys, xs, acc, yx);
  const float yyj = j < N ? yy[j] : 0.0f;
  // state per node: 0 near / excluded, 1 far, 2 inside the rounding band (FP64 retest)
  unsigned band = 0u, far = 0u;
#pragma unroll
  for (int nb = 0; nb < FT_NB; ++nb) {
    if (nb < nbn && j < N) {
      const FarItem& it = items[nb0 + nb];
      if (j < it.M && !(j >= it.ex_begin && j < it.ex_end)) {
        const TileNode& nd = nodes[nb0 + nb];
        const double a = (double)acc[nb];
        const double m = 0x1.0p-24 * (16.0 * ((double)yyj + (double)nd.xx) + 1.1 * (double)(d + 1) * a) + 1e-300;
        if (a - m >= nd.thr2) far |= 1u << nb;
        else if (!(a + m < nd.thr2)) band |= 1u << nb;
      }
    }
  }
  while (band) {
    const int nb = __ffs(band) - 1;
    band &= band - 1;
    if (far_member(Y, d, j, items[nb0 + nb], nodes[nb0 + nb].thr2)) far |= 1u << nb;
  }
#pragma unroll
  for (int nb = 0; nb < FT_NB; ++nb) {
    const unsigned b = __ballot_sync(0xffffffffu, (far >> nb) & 1u);
    if (lane == 0) {
      wc[nb][w] = __popc(b);
      if (nb < nbn) mask[(int64_t)(nb0 + nb) * words + (j0 >> 5) + w] = b;
    }
  }
  __syncthreads();
  if (t < nbn) {
    int c = 0;
#pragma unroll
    for (int q = 0; q < FT_PTS / 32; ++q) c += wc[t][q];
    tile_cnt[(int64_t)(nb0 + t) * tiles + blockIdx.x] = c;
  }
}

// pass 2: list entries and features of the far pairs, at the scanned positions
template <typename TP, bool DOT>
__global__ void __launch_bounds__(FT_PTS) far_features_kernel(const TP* __restrict__ Y, int64_t N, int d,
                                                              const FarItem* __restrict__ items,
                                                              const FeatItem* __restrict__ fitems, int n_items,
                                                              const float* __restrict__ xc32,
                                                              const TileNode* __restrict__ nodes,
                                                              const float* __restrict__ yy,
                                                              const float* __restrict__ yg, int64_t tiles,
                                                              const int64_t* __restrict__ tile_off,
                                                              const uint32_t* __restrict__ mask, ffc_kernel k,
                                                              float* __restrict__ out) {
  __shared__ float ys[FT_DC][FT_PTS + 1];
  __shared__ __align__(16) float xs[FT_NB][FT_DC];
  __shared__ uint32_t mw[FT_NB][FT_PTS / 32];
  __shared__ int any;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t j0 = (int64_t)blockIdx.x * FT_PTS, j = j0 + t;
  const int nb0 = blockIdx.y * FT_NB, nbn = min(FT_NB, n_items - nb0);
  const int64_t words = tiles * (FT_PTS / 32);
  if (t == 0) any = 0;
  __syncthreads();
  if (t < FT_NB * (FT_PTS / 32)) {
    const int nb = t / (FT_PTS / 32), q = t % (FT_PTS / 32);
    const uint32_t v = nb < nbn ? mask[(int64_t)(nb0 + nb) * words + (j0 >> 5) + q] : 0u;
    mw[nb][q] = v;
    if (v) atomicOr(&any, 1);
  }
  __syncthreads();
  if (!any) return;   // uniform across the CTA
  float acc[FT_NB], yx[FT_NB];
  tile_distances<TP, DOT>(Y, N, d, j0, xc32, nb0, nbn, ys, xs, acc, yx);
  if (j >= N) return;
  const float yyj = yy[j];
#pragma unroll
  for (int nb = 0; nb < FT_NB; ++nb) {
    const uint32_t bits = mw[nb][w];
    if (!((bits >> lane) & 1u)) continue;
    int before = __popc(bits & ((1u << lane) - 1u));
    for (int q = 0; q < w; ++q) before += __popc(mw[nb][q]);
    const int64_t pos = tile_off[(int64_t)(nb0 + nb) * tiles + blockIdx.x] + before;
    const TileNode& nd = nodes[nb0 + nb];
    FeatSums S;
    S.dd = acc[nb];
    S.yy = yyj;
    S.yx = yx[nb];
    S.xx = nd.xx;
#pragma unroll
    for (int q = 0; q < 8; ++q) S.p[q] = yg[j * 8 + q] - nd.xg[q];
    float v[FEAT_NF];
    feature_values(S, nd.rho, k, d, v);
    const FarItem& it = items[nb0 + nb];
    it.list[pos] = j;
    float* o = out + (fitems[nb0 + nb].out_begin + pos) * FEAT_NF;
#pragma unroll
    for (int f = 0; f < FEAT_NF; ++f) o[f] = v[f];
  }
}

// zero the feature rows [count, cap) of every item (rows the network scores but the draw never reads)
__global__ void feature_tail_kernel(const FeatItem* __restrict__ fitems, float* __restrict__ out) {
  const FeatItem& it = fitems[blockIdx.y];
  const int64_t cnt = *it.count;
  for (int64_t e = cnt * FEAT_NF + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < it.cap * FEAT_NF;
       e += (int64_t)gridDim.x * blockDim.x)
    out[it.out_begin * FEAT_NF + e] = 0.0f;
}

__global__ void far_scan_tiles_kernel(const FarItem* items, int64_t tiles, int64_t* tile_cnt) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry;
  int64_t* tc = tile_cnt + (int64_t)blockIdx.x * tiles;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < tiles; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < tiles ? tc[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int64_t add = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < tiles) tc[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *items[blockIdx.x].count = carry;
}

ffc_status launch_point_stats(const void* Y, int dtype, int64_t N, int d, const double* proj, float* yy, float* yg,
                              cudaStream_t st) {
  if (N <= 0) return FFC_OK;
  const size_t smem = (size_t)8 * d * sizeof(float);
  FFC_REQUIRE(smem <= 200 * 1024, "point stats: d = %d too large", d);
  const int grid = (int)std::min<int64_t>((N + 7) / 8, (int64_t)sm_count() * 8);
  if (dtype == FFC_F64) {
    FFC_CUDA(cudaFuncSetAttribute(point_stats_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    point_stats_kernel<double><<<grid, 256, smem, st>>>((const double*)Y, N, d, proj, yy, yg);
  } else {
    FFC_CUDA(cudaFuncSetAttribute(point_stats_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    point_stats_kernel<float><<<grid, 256, smem, st>>>((const float*)Y, N, d, proj, yy, yg);
  }
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

ffc_status launch_far_features_tiled(ffc_kernel k, const void* Y, int dtype, int64_t N, int d,
                                     const FarItem* items_dev, const FeatItem* fitems_dev, int n_items,
                                     const double* proj, const float* yy, const float* yg, void* node_ws,
                                     int64_t* tile_cnt, uint32_t* mask, float* feats, cudaStream_t st) {
  if (n_items <= 0 || N <= 0) return FFC_OK;
  const int64_t tiles = far_tiles_count(N);
  const int batches = (n_items + FT_NB - 1) / FT_NB;
  FFC_REQUIRE(batches <= 65535, "tiled far field: too many nodes in one launch (%d)", n_items);
  FFC_REQUIRE(tiles <= 0x7FFFFFFF, "tiled far field: too many points");
  TileNode* nodes = (TileNode*)node_ws;
  float* xc32 = (float*)(nodes + n_items);
  node_stats_kernel<<<n_items, 128, 0, st>>>(items_dev, d, proj, xc32, nodes);
  const dim3 grid((unsigned)tiles, (unsigned)batches);
  const bool dot = k.kind == FFC_POLYNOMIAL;
  if (dtype == FFC_F64) {
    far_mark_kernel<double><<<grid, FT_PTS, 0, st>>>((const double*)Y, N, d, items_dev, n_items, xc32, nodes, yy,
                                                    tiles, tile_cnt, mask);
    far_scan_tiles_kernel<<<n_items, 1024, 0, st>>>(items_dev, tiles, tile_cnt);
    if (dot)
      far_features_kernel<double, true><<<grid, FT_PTS, 0, st>>>((const double*)Y, N, d, items_dev, fitems_dev,
                                                                 n_items, xc32, nodes, yy, yg, tiles, tile_cnt,
                                                                 mask, k, feats);
    else
      far_features_kernel<double, false><<<grid, FT_PTS, 0, st>>>((const double*)Y, N, d, items_dev, fitems_dev,
                                                                  n_items, xc32, nodes, yy, yg, tiles, tile_cnt,
                                                                  mask, k, feats);
  } else {
    far_mark_kernel<float><<<grid, FT_PTS, 0, st>>>((const float*)Y, N, d, items_dev, n_items, xc32, nodes, yy,
                                                   tiles, tile_cnt, mask);
    far_scan_tiles_kernel<<<n_items, 1024, 0, st>>>(items_dev, tiles, tile_cnt);
    if (dot)
      far_features_kernel<float, true><<<grid, FT_PTS, 0, st>>>((const float*)Y, N, d, items_dev, fitems_dev,
                                                                n_items, xc32, nodes, yy, yg, tiles, tile_cnt,
                                                                mask, k, feats);
    else
      far_features_kernel<float, false><<<grid, FT_PTS, 0, st>>>((const float*)Y, N, d, items_dev, fitems_dev,
                                                                 n_items, xc32, nodes, yy, yg, tiles, tile_cnt,
                                                                 mask, k, feats);
  }
  feature_tail_kernel<<<dim3(8, (unsigned)n_items), 256, 0, st>>>(fitems_dev, feats);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace ffc
