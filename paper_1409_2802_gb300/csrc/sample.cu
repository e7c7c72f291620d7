// Far-field listing and uniform far-field row sampling without replacement.
//
// Method: §2.2 (sample s of the far-field targets), §4.1 step 3 (far field
// T = {y : ||y - x_c|| >= xi rho}), §4.1.3 "Uniform sampling" (s rows chosen
// uniformly without replacement). The exact draw order (Philox4x64-10 stream,
// phase A rejection, phase B Fisher-Yates) is stated in include/ffc.h.
//
// GPU layout: one CTA per sampling problem; the "already taken" set is a
// bitmap of M bits in shared memory; candidates are tested 256 at a time in
// parallel (the distance test is the expensive part) and accepted in draw
// order by one warp at a time with ballot/match, so the result equals the
// sequential definition.
#include <cstdio>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int SAMPLE_THREADS = 256;

template <typename TP>
__device__ __forceinline__ bool far_test(const TP* __restrict__ Y, int d, int64_t j, const double* xc,
                                         double thr2, bool has_c) {
  if (!has_c) return true;
  const TP* y = Y + j * (int64_t)d;
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double df = ld_point(y + k) - xc[k];
    acc = fma(df, df, acc);
  }
  return acc >= thr2;
}

// Ordered compaction over candidates in [0, M): flags -> ascending list.
// Three steps: per-tile far flags and counts, exclusive scan, scatter.
constexpr int FF_TILE = 256;

template <typename TP>
__global__ void ff_count_kernel(const TP* __restrict__ Y, int64_t M, int d, const double* __restrict__ x_c,
                                double thr2, int64_t ex_b, int64_t ex_e, uint8_t* flags, int64_t* tile_cnt) {
  __shared__ int wc[FF_TILE / 32];
  int64_t j = (int64_t)blockIdx.x * FF_TILE + threadIdx.x;
  bool f = false;
  if (j < M && !(j >= ex_b && j < ex_e)) {
    if (x_c == nullptr) {
      f = true;
    } else {
      const TP* y = Y + j * (int64_t)d;
      double acc = 0.0;
      for (int k = 0; k < d; ++k) {
        double df = ld_point(y + k) - __ldg(x_c + k);
        acc = fma(df, df, acc);
      }
      f = acc >= thr2;
    }
  }
  if (j < M) flags[j] = f ? 1 : 0;
  unsigned b = __ballot_sync(0xffffffffu, f);
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = __popc(b);
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < FF_TILE / 32; ++w) t += wc[w];
    tile_cnt[blockIdx.x] = t;
  }
}

__global__ void ff_scan_kernel(int64_t* tile_cnt, int64_t n_tiles, int64_t* total) {
  // single CTA; tiles are few (M / 256)
  __shared__ int64_t carry;
  __shared__ int64_t part[1024];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n_tiles; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n_tiles ? tile_cnt[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      int64_t add = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n_tiles) tile_cnt[i] = carry + part[threadIdx.x] - v;   // exclusive
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void ff_scatter_kernel(const uint8_t* flags, int64_t M, const int64_t* tile_off, int64_t* idx) {
  __shared__ int wc[FF_TILE / 32];
  int64_t j = (int64_t)blockIdx.x * FF_TILE + threadIdx.x;
  bool f = j < M && flags[j];
  unsigned b = __ballot_sync(0xffffffffu, f);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) wc[w] = __popc(b);
  __syncthreads();
  int off = 0;
  for (int q = 0; q < w; ++q) off += wc[q];
  if (f) idx[tile_off[blockIdx.x] + off + __popc(b & ((1u << lane) - 1u))] = j;
}

template <typename TP>
__global__ void __launch_bounds__(SAMPLE_THREADS)
sample_kernel(const TP* __restrict__ Y, int d, const SampleItem* __restrict__ items, int n_items,
              uint64_t seed, int64_t* s_out, int64_t* far_count, int32_t* status, int32_t* scratch,
              int64_t M_max) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* xc = reinterpret_cast<double*>(smem);
  uint32_t* bitmap = reinterpret_cast<uint32_t*>(xc + d);
  __shared__ int k_acc;
  __shared__ int wc[SAMPLE_THREADS / 32];
  __shared__ long long list_cnt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (int q = blockIdx.x; q < n_items; q += gridDim.x) {
    SampleItem it = items[q];
    const int64_t M = it.M, s = it.s;
    const int64_t words = (M + 31) >> 5;
    for (int64_t w = threadIdx.x; w < words; w += blockDim.x) bitmap[w] = 0u;
    const bool has_c = it.x_c != nullptr;
    if (has_c)
      for (int k = threadIdx.x; k < d; k += blockDim.x) xc[k] = it.x_c[k];
    if (it.radius != nullptr) {
      const double thr = it.xi * *it.radius;
      it.thr2 = thr * thr;
    }
    if (threadIdx.x == 0) k_acc = 0;
    __syncthreads();

    // Phase A: rejection over the candidate stream, accepted in draw order.
    const int64_t A = (int64_t)ATTEMPT_FACTOR * s;
    for (int64_t base = 0; base < A && M > 0; base += blockDim.x) {
      if (k_acc >= s) break;
      const int64_t t = base + threadIdx.x;
      bool far = false;
      int64_t j = -1;
      if (t < A) {
        uint64_t w = philox_draw(seed, it.stream_id, DOMAIN_UNIFORM_ROWS, (uint64_t)t);
        j = (int64_t)__umul64hi(w, (uint64_t)M);
        far = !(j >= it.ex_begin && j < it.ex_end) && far_test(Y, d, j, xc, it.thr2, has_c);
      }
      for (int wv = 0; wv < SAMPLE_THREADS / 32; ++wv) {
        if (warp == wv) {
          const int k0 = k_acc;
          // first occurrence of each candidate within the warp
          long long key = far ? (long long)j : -1ll - lane;
          unsigned same = __match_any_sync(0xffffffffu, key);
          bool keep = far && (lane == __ffs(same) - 1);
          bool taken = keep && ((bitmap[j >> 5] >> (j & 31)) & 1u);
          bool acc = keep && !taken;
          unsigned am = __ballot_sync(0xffffffffu, acc);
          int rk = __popc(am & lt_mask);
          int room = (int)(s - k0);
          if (acc && rk < room) {
            it.rows[k0 + rk] = j;
            atomicOr(&bitmap[j >> 5], 1u << (j & 31));
          }
          __syncwarp();
          if (lane == 0) k_acc = k0 + min(__popc(am), room);
        }
        __syncthreads();
      }
    }
    __syncthreads();

    // Phase B: enumerate the remaining far field in ascending order.
    int64_t k = k_acc;
    int64_t fc = -1;
    if (k < s) {
      int32_t* list = scratch + (int64_t)blockIdx.x * M_max;
      if (threadIdx.x == 0) list_cnt = 0;
      __syncthreads();
      for (int64_t base = 0; base < M; base += blockDim.x) {
        const int64_t j = base + threadIdx.x;
        bool f = j < M && !(j >= it.ex_begin && j < it.ex_end) &&
                 !((bitmap[j >> 5] >> (j & 31)) & 1u) && far_test(Y, d, j, xc, it.thr2, has_c);
        unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wc[warp] = __popc(b);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < SAMPLE_THREADS / 32; ++w) {
          if (w < warp) off += wc[w];
          tot += wc[w];
        }
        if (f) list[list_cnt + off + __popc(b & lt_mask)] = (int32_t)j;
        __syncthreads();
        if (threadIdx.x == 0) list_cnt += tot;
        __syncthreads();
      }
      const int64_t L = list_cnt;
      fc = k + L;
      const int64_t need = s - k;
      if (L <= need) {
        for (int64_t i = threadIdx.x; i < L; i += blockDim.x) it.rows[k + i] = list[i];
        k += L;
      } else {
        if (threadIdx.x == 0) {
          for (int64_t i = 0; i < need; ++i) {
            uint64_t w = philox_draw(seed, it.stream_id, DOMAIN_UNIFORM_ROWS, (uint64_t)(A + i));
            int64_t u = i + (int64_t)__umul64hi(w, (uint64_t)(L - i));
            int32_t tmp = list[i];
            list[i] = list[u];
            list[u] = tmp;
            it.rows[k + i] = list[i];
          }
        }
        k += need;
      }
    }
    if (threadIdx.x == 0) {
      s_out[q] = k;
      if (far_count) far_count[q] = fc;
      status[q] = (k < s) ? FFC_E_FARFIELD_TOO_SMALL : FFC_OK;
    }
    __syncthreads();
  }
}

}  // namespace

ffc_status launch_far_field(const void* Y, int dtype, int64_t M, int d, const double* x_c, double thr2,
                            int64_t ex_begin, int64_t ex_end, int64_t* idx, int64_t* count_dev,
                            cudaStream_t st) {
  int64_t n_tiles = (M + FF_TILE - 1) / FF_TILE;
  if (n_tiles == 0) {
    FFC_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int64_t), st));
    return FFC_OK;
  }
  uint8_t* flags = nullptr;
  int64_t* tiles = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&flags, (size_t)M, st));
  FFC_CUDA(cudaMallocAsync((void**)&tiles, (size_t)n_tiles * sizeof(int64_t), st));
  if (dtype == FFC_F64)
    ff_count_kernel<double><<<(unsigned)n_tiles, FF_TILE, 0, st>>>((const double*)Y, M, d, x_c, thr2, ex_begin,
                                                                 ex_end, flags, tiles);
  else
    ff_count_kernel<float><<<(unsigned)n_tiles, FF_TILE, 0, st>>>((const float*)Y, M, d, x_c, thr2, ex_begin,
                                                                ex_end, flags, tiles);
  ff_scan_kernel<<<1, 1024, 0, st>>>(tiles, n_tiles, count_dev);
  ff_scatter_kernel<<<(unsigned)n_tiles, FF_TILE, 0, st>>>(flags, M, tiles, idx);
  FFC_CUDA(cudaGetLastError());
  FFC_CUDA(cudaFreeAsync(flags, st));
  FFC_CUDA(cudaFreeAsync(tiles, st));
  return FFC_OK;
}

size_t sample_smem_bytes(int64_t M_max, int d) {
  return (size_t)d * sizeof(double) + (size_t)((M_max + 31) / 32) * sizeof(uint32_t);
}

ffc_status launch_sample(const void* Y, int dtype, int d, const SampleItem* items_dev, int n_items,
                         int64_t M_max, int64_t s_max, uint64_t seed, int64_t* s_out, int64_t* far_count,
                         int32_t* status, int32_t* scratch, cudaStream_t st) {
  (void)s_max;
  if (n_items <= 0) return FFC_OK;
  size_t smem = sample_smem_bytes(M_max, d);
  // the caller's scratch holds min(n_items, SAMPLE_MAX_GRID) slices of M_max
  int grid = n_items < SAMPLE_MAX_GRID ? n_items : SAMPLE_MAX_GRID;
  if (dtype == FFC_F64) {
    auto kfn = sample_kernel<double>;
    FFC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, SAMPLE_THREADS, smem, st>>>((const double*)Y, d, items_dev, n_items, seed, s_out, far_count,
                                            status, scratch, M_max);
  } else {
    auto kfn = sample_kernel<float>;
    FFC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kfn<<<grid, SAMPLE_THREADS, smem, st>>>((const float*)Y, d, items_dev, n_items, seed, s_out, far_count,
                                            status, scratch, M_max);
  }
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace ffc
