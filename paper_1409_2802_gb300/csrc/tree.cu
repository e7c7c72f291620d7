// PCA median-split binary tree (the space-partitioning tree that defines the
// nodes' far fields, §2; node centre and radius as in the §4.1 setup).
//
// Level by level: per node, the centroid (mean), the radius (max distance to
// the centroid), the principal direction of the centred points from 32 power
// iterations v <- C^T (C v) / ||.|| starting at (1,...,1)/sqrt(d) (sign: the
// largest-magnitude component positive), then a segmented bitonic sort of the
// node's points by (projection, original index); the first floor(count/2)
// go to the left child. Reductions go through per-chunk partials summed in a
// fixed order, so the tree is deterministic.
#include <algorithm>
#include <vector>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int CHUNK = 2048;      // points per CTA for the reductions
constexpr int TREE_THREADS = 256;
constexpr int POWER_ITERS = 32;

struct LevelInfo {
  const int64_t* begin;   // device, indexed by node - first
  const int64_t* count;
  int64_t first;          // heap id of the level's first node
  int n_nodes;
  int chunks;             // chunks per node
};

__global__ void iota_kernel(int64_t* perm, int64_t N) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < N) perm[i] = i;
}

// partial sums of the node's points (mode 0), or of (c.v) c for centred points (mode 1)
template <typename TP, int MODE>
__global__ void __launch_bounds__(TREE_THREADS)
partial_kernel(const TP* __restrict__ X, int d, const int64_t* __restrict__ perm, LevelInfo L,
               const double* __restrict__ centroid, const double* __restrict__ v, double* partial) {
  extern __shared__ double sm[];      // [8 warps][d] partial + [d] centroid + [d] v
  const int node = blockIdx.x / L.chunks, chunk = blockIdx.x % L.chunks;
  const int64_t b = L.begin[node], c = L.count[node];
  const int64_t p0 = (int64_t)chunk * CHUNK, p1 = (c < p0 + CHUNK) ? c : p0 + CHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* wpart = sm + warp * d;
  double* xc = sm + 8 * d;
  double* vv = xc + d;
  const int64_t gnode = L.first + node;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    if (MODE == 1) { xc[k] = centroid[gnode * d + k]; vv[k] = v[node * (int64_t)d + k]; }
  }
  for (int e = threadIdx.x; e < 8 * d; e += blockDim.x) sm[e] = 0.0;
  __syncthreads();
  for (int64_t p = p0 + warp; p < p1; p += 8) {
    const TP* x = X + perm[b + p] * (int64_t)d;
    if (MODE == 0) {
      for (int k = lane; k < d; k += 32) wpart[k] += ld_point(x + k);
    } else {
      double dot = 0.0;
      for (int k = lane; k < d; k += 32) dot = fma(ld_point(x + k) - xc[k], vv[k], dot);
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
      for (int k = lane; k < d; k += 32) wpart[k] = fma(dot, ld_point(x + k) - xc[k], wpart[k]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += sm[w * d + k];
    partial[(int64_t)blockIdx.x * d + k] = t;
  }
}

// mode 0: centroid = sum / count ; mode 1: v = w / ||w|| (keep v if w = 0);
// mode 2: like 1, then fix the sign
__global__ void reduce_kernel(const double* partial, int d, LevelInfo L, double* centroid, double* v, int mode) {
  extern __shared__ double w[];
  __shared__ double nrm2;
  const int node = blockIdx.x;
  const int64_t gnode = L.first + node;
  for (int k = threadIdx.x; k < d; k += blockDim.x) {
    double t = 0.0;
    for (int ch = 0; ch < L.chunks; ++ch) t += partial[((int64_t)node * L.chunks + ch) * d + k];
    w[k] = t;
  }
  __syncthreads();
  if (mode == 0) {
    const double c = (double)L.count[node];
    for (int k = threadIdx.x; k < d; k += blockDim.x) centroid[gnode * d + k] = c > 0 ? w[k] / c : 0.0;
    return;
  }
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < d; ++k) t = fma(w[k], w[k], t);
    nrm2 = t;
  }
  __syncthreads();
  double* vn = v + (int64_t)node * d;
  if (nrm2 > 0.0) {
    const double nr = sqrt(nrm2);
    for (int k = threadIdx.x; k < d; k += blockDim.x) vn[k] = w[k] / nr;
  }
  if (mode == 2) {
    __syncthreads();
    __shared__ int sgn;
    if (threadIdx.x == 0) {
      int bi = 0;
      double bv = -1.0;
      for (int k = 0; k < d; ++k)
        if (fabs(vn[k]) > bv) { bv = fabs(vn[k]); bi = k; }
      sgn = vn[bi] < 0.0 ? -1 : 1;
    }
    __syncthreads();
    if (sgn < 0)
      for (int k = threadIdx.x; k < d; k += blockDim.x) vn[k] = -vn[k];
  }
}

__global__ void init_v_kernel(double* v, int n_nodes, int d) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < (int64_t)n_nodes * d) v[e] = 1.0 / sqrt((double)d);
}

template <typename TP>
__global__ void radius_kernel(const TP* __restrict__ X, int d, const int64_t* perm, LevelInfo L,
                              const double* centroid, double* partial_max) {
  const int node = blockIdx.x / L.chunks, chunk = blockIdx.x % L.chunks;
  const int64_t b = L.begin[node], c = L.count[node];
  const int64_t p0 = (int64_t)chunk * CHUNK, p1 = (c < p0 + CHUNK) ? c : p0 + CHUNK;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* xc = centroid + (L.first + node) * d;
  __shared__ double wm[8];
  double mx = 0.0;
  for (int64_t p = p0 + warp; p < p1; p += 8) {
    const TP* x = X + perm[b + p] * (int64_t)d;
    double acc = 0.0;
    for (int k = lane; k < d; k += 32) {
      double df = ld_point(x + k) - xc[k];
      acc = fma(df, df, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    mx = fmax(mx, acc);
  }
  if (lane == 0) wm[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t = fmax(t, wm[w]);
    partial_max[blockIdx.x] = t;
  }
}

__global__ void radius_reduce_kernel(const double* partial_max, LevelInfo L, double* radius) {
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= L.n_nodes) return;
  double t = 0.0;
  for (int ch = 0; ch < L.chunks; ++ch) t = fmax(t, partial_max[node * L.chunks + ch]);
  radius[L.first + node] = sqrt(t);
}

// keys of the segmented sort: (projection, original index), padded with +inf
template <typename TP>
__global__ void proj_kernel(const TP* __restrict__ X, int d, const int64_t* perm, LevelInfo L,
                            const double* centroid, const double* v, int64_t P, double* key, int64_t* idx) {
  const int64_t e = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= (int64_t)L.n_nodes * P) return;
  const int node = (int)(e / P);
  const int64_t t = e % P;
  const int64_t c = L.count[node];
  if (t >= c) {
    if (lane == 0) { key[e] = INFINITY; idx[e] = INT64_MAX; }
    return;
  }
  const int64_t pt = perm[L.begin[node] + t];
  const TP* x = X + pt * (int64_t)d;
  const double* xc = centroid + (L.first + node) * d;
  const double* vn = v + (int64_t)node * d;
  double acc = 0.0;
  for (int k = lane; k < d; k += 32) acc = fma(ld_point(x + k) - xc[k], vn[k], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) { key[e] = acc; idx[e] = pt; }
}

__global__ void bitonic_step_kernel(double* key, int64_t* idx, int64_t total, int64_t P, int64_t j, int64_t k) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int64_t i = e % P, base = e - i;
  const int64_t l = i ^ j;
  if (l <= i) return;
  const bool asc = (i & k) == 0;
  const double ka = key[base + i], kb = key[base + l];
  const int64_t ia = idx[base + i], ib = idx[base + l];
  const bool gt = (ka > kb) || (ka == kb && ia > ib);
  if (gt == asc) {
    key[base + i] = kb; key[base + l] = ka;
    idx[base + i] = ib; idx[base + l] = ia;
  }
}

__global__ void scatter_perm_kernel(const int64_t* idx, LevelInfo L, int64_t P, int64_t* perm) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)L.n_nodes * P) return;
  const int node = (int)(e / P);
  const int64_t t = e % P;
  if (t < L.count[node]) perm[L.begin[node] + t] = idx[e];
}

template <typename TP>
ffc_status build_t(const TP* X, int64_t N, int d, int depth, int64_t* perm, const int64_t* begin_host,
                   const int64_t* count_host, const int64_t* begin_dev, const int64_t* count_dev,
                   double* centroid, double* radius, cudaStream_t st) {
  iota_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(perm, N);
  const int64_t n_nodes_max = (int64_t)1 << depth;
  int64_t max_chunks_total = 0, max_sort = 0;
  for (int l = 0; l <= depth; ++l) {
    const int64_t first = ((int64_t)1 << l) - 1, nn = (int64_t)1 << l;
    int64_t cmax = 0;
    for (int64_t i = 0; i < nn; ++i) cmax = std::max(cmax, count_host[first + i]);
    const int64_t chunks = std::max<int64_t>(1, (cmax + CHUNK - 1) / CHUNK);
    max_chunks_total = std::max(max_chunks_total, nn * chunks);
    int64_t P = 1;
    while (P < cmax) P <<= 1;
    max_sort = std::max(max_sort, nn * P);
  }
  double *partial = nullptr, *v = nullptr, *key = nullptr;
  int64_t* idx = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&partial, sizeof(double) * max_chunks_total * std::max(d, 1), st));
  FFC_CUDA(cudaMallocAsync((void**)&v, sizeof(double) * n_nodes_max * d, st));
  FFC_CUDA(cudaMallocAsync((void**)&key, sizeof(double) * max_sort, st));
  FFC_CUDA(cudaMallocAsync((void**)&idx, sizeof(int64_t) * max_sort, st));
  const size_t psmem = sizeof(double) * 10 * d;
  FFC_CUDA(cudaFuncSetAttribute(partial_kernel<TP, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  FFC_CUDA(cudaFuncSetAttribute(partial_kernel<TP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem));
  FFC_CUDA(cudaFuncSetAttribute(reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(double) * d)));
  for (int l = 0; l <= depth; ++l) {
    const int64_t first = ((int64_t)1 << l) - 1;
    const int nn = 1 << l;
    int64_t cmax = 0;
    for (int i = 0; i < nn; ++i) cmax = std::max(cmax, count_host[first + i]);
    LevelInfo L;
    L.begin = begin_dev + first;
    L.count = count_dev + first;
    L.first = first;
    L.n_nodes = nn;
    L.chunks = (int)std::max<int64_t>(1, (cmax + CHUNK - 1) / CHUNK);
    const unsigned grid = (unsigned)(nn * L.chunks);
    partial_kernel<TP, 0><<<grid, TREE_THREADS, psmem, st>>>(X, d, perm, L, centroid, v, partial);
    reduce_kernel<<<nn, 128, sizeof(double) * d, st>>>(partial, d, L, centroid, v, 0);
    radius_kernel<TP><<<grid, TREE_THREADS, 0, st>>>(X, d, perm, L, centroid, partial);
    radius_reduce_kernel<<<(nn + 127) / 128, 128, 0, st>>>(partial, L, radius);
    if (l == depth) break;
    init_v_kernel<<<(unsigned)((nn * (int64_t)d + 255) / 256), 256, 0, st>>>(v, nn, d);
    for (int itn = 0; itn < POWER_ITERS; ++itn) {
      partial_kernel<TP, 1><<<grid, TREE_THREADS, psmem, st>>>(X, d, perm, L, centroid, v, partial);
      reduce_kernel<<<nn, 128, sizeof(double) * d, st>>>(partial, d, L, centroid, v,
                                                          itn == POWER_ITERS - 1 ? 2 : 1);
    }
    int64_t P = 1;
    while (P < cmax) P <<= 1;
    const int64_t total = (int64_t)nn * P;
    proj_kernel<TP><<<(unsigned)((total + 7) / 8), 256, 0, st>>>(X, d, perm, L, centroid, v, P, key, idx);
    const unsigned sg = (unsigned)((total + 255) / 256);
    for (int64_t k = 2; k <= P; k <<= 1)
      for (int64_t j = k >> 1; j > 0; j >>= 1) bitonic_step_kernel<<<sg, 256, 0, st>>>(key, idx, total, P, j, k);
    scatter_perm_kernel<<<sg, 256, 0, st>>>(idx, L, P, perm);
  }
  FFC_CUDA(cudaGetLastError());
  FFC_CUDA(cudaFreeAsync(partial, st));
  FFC_CUDA(cudaFreeAsync(v, st));
  FFC_CUDA(cudaFreeAsync(key, st));
  FFC_CUDA(cudaFreeAsync(idx, st));
  return FFC_OK;
}

}  // namespace

void node_layout(int64_t N, int depth, int64_t* begin, int64_t* count, int32_t* level) {
  const int64_t n_nodes = ((int64_t)1 << (depth + 1)) - 1;
  for (int64_t i = 0; i < n_nodes; ++i) { begin[i] = 0; count[i] = 0; if (level) level[i] = 0; }
  count[0] = N;
  for (int64_t i = 0; i < n_nodes; ++i) {
    if (2 * i + 2 < n_nodes) {
      const int64_t left = count[i] / 2;
      begin[2 * i + 1] = begin[i];
      count[2 * i + 1] = left;
      begin[2 * i + 2] = begin[i] + left;
      count[2 * i + 2] = count[i] - left;
      if (level) level[2 * i + 1] = level[2 * i + 2] = level[i] + 1;
    }
  }
}

ffc_status launch_build_tree(const void* points, int dtype, int64_t N, int d, int depth, int64_t* perm,
                             const int64_t* begin_host, const int64_t* count_host, const int64_t* begin_dev,
                             const int64_t* count_dev, double* centroid, double* radius, cudaStream_t st) {
  if (dtype == FFC_F64)
    return build_t<double>((const double*)points, N, d, depth, perm, begin_host, count_host, begin_dev, count_dev,
                           centroid, radius, st);
  return build_t<float>((const float*)points, N, d, depth, perm, begin_host, count_host, begin_dev, count_dev,
                        centroid, radius, st);
}

}  // namespace ffc
