// The paper's other row samplers for the sampled block (§4.1.3; the heuristics
// of §3): distance sampling in both readings, deterministic nearest neighbours
// and leverage sampling, as sort keys for the weighted draw's selection.
//
// * Distance: probability proportional to w = ||y - x_c|| (§4.1.3's list) or
//   to 1 / ||y - x_c|| (§3: rows near the sources carry the block), drawn
//   without replacement by Efraimidis & Spirakis' keys ln(u_i) / w_i, u_i the
//   unit double of draw i (i = candidate position) of stream (seed, stream_id,
//   domain 3). The sort key -ln(u_i) / w_i > 0 orders ascending exactly as the
//   key orders descending.
// * Nearest neighbours: the candidates closest to the node's sources, sort key
//   the squared distance to the nearest source (FP64; non-negative doubles
//   order like their bit patterns).
// * Leverage: probability proportional to the row's leverage score of the
//   full far-field block at its eps-rank (§3, Def. "Statistical Leverage"),
//   over the rows with a positive score, Efraimidis-Spirakis keys as above.
// The selection (the s smallest sort keys, ties to the lower position, in key
// order) is the weighted draw's (select_kernel with given keys).
#include <algorithm>

#include "ffc_internal.cuh"

namespace ffc {

constexpr uint64_t DOMAIN_PAPER_SAMPLERS = 3;

namespace {

constexpr int KEY_THREADS = 128;

__device__ __forceinline__ uint64_t es_key(double w, uint64_t seed, uint64_t stream_id, int64_t i) {
  const uint64_t draw = philox_draw(seed, stream_id, DOMAIN_PAPER_SAMPLERS, (uint64_t)i);
  const double u = ((double)(draw >> 11) + 0.5) * 0x1.0p-53;
  return (uint64_t)__double_as_longlong(-log(u) / w);
}

// Grid: blockIdx.y = item, blockIdx.x strides over the item's candidates (KEY_THREADS each).
// NEAREST stages the item's sources through shared memory in chunks of kp points.
template <typename TP, int MODE>
__global__ void __launch_bounds__(KEY_THREADS)
paper_keys_kernel(const TP* __restrict__ Y, const TP* __restrict__ X, int d, const KeyItem* __restrict__ items,
                  uint64_t seed, int kp_max) {
  extern __shared__ double ksm[];
  const KeyItem& it = items[blockIdx.y];
  const int64_t P = it.count ? *it.count : it.cap;
  const int64_t stride = (int64_t)gridDim.x * KEY_THREADS;
  if (MODE != FFC_DRAW_NEAREST) {
    for (int64_t i = (int64_t)blockIdx.x * KEY_THREADS + threadIdx.x; i < P; i += stride) {
      const TP* y = Y + it.pool[i] * (int64_t)d;
      double dd = 0.0;
      for (int j = 0; j < d; ++j) {
        const double df = ld_point(y + j) - __ldg(it.x_c + j);
        dd = fma(df, df, dd);
      }
      const double r = sqrt(dd);
      it.keys[i] = es_key(MODE == FFC_DRAW_INV_DISTANCE ? 1.0 / r : r, seed, it.stream_id, i);
    }
    return;
  }
  // nearest neighbours: the CTA's candidates against every source of the item
  for (int64_t i0 = (int64_t)blockIdx.x * KEY_THREADS; i0 < P; i0 += stride) {
    const int64_t i = i0 + threadIdx.x;
    const bool live = i < P;
    const TP* y = Y + (live ? it.pool[i] : 0) * (int64_t)d;
    double best = INFINITY;
    for (int64_t c0 = 0; c0 < it.src_n; c0 += kp_max) {
      const int kp = (int)min((int64_t)kp_max, it.src_n - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < kp * d; e += KEY_THREADS) {
        const int c = e / d, j = e % d;
        ksm[e] = ld_point(X + (it.src_begin + c0 + c) * d + j);
      }
      __syncthreads();
      if (live) {
        for (int c = 0; c < kp; ++c) {
          const double* x = ksm + (int64_t)c * d;
          double dd = 0.0;
          for (int j = 0; j < d; ++j) {
            const double df = ld_point(y + j) - x[j];
            dd = fma(df, df, dd);
          }
          best = fmin(best, dd);
        }
      }
    }
    if (live) it.keys[i] = (uint64_t)__double_as_longlong(best);
  }
}

// Leverage sampling: one CTA compacts the rows with a positive score (candidate order kept) and
// writes their keys; *count = how many.
__global__ void __launch_bounds__(1024) leverage_keys_kernel(const double* __restrict__ lev, const int64_t* cand,
                                                             int64_t m, uint64_t seed, uint64_t stream_id,
                                                             int64_t* __restrict__ pool, uint64_t* __restrict__ keys,
                                                             int64_t* __restrict__ count) {
  __shared__ int wsum[32];
  __shared__ int64_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t i0 = 0; i0 < m; i0 += blockDim.x) {
    const int64_t i = i0 + threadIdx.x;
    const bool pos = i < m && lev[i] > 0.0;
    const unsigned bal = __ballot_sync(0xffffffffu, pos);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) off += wsum[w];
      tot += wsum[w];
    }
    if (pos) {
      const int64_t k = base + off + __popc(bal & ((1u << lane) - 1u));
      pool[k] = cand ? cand[i] : i;
      keys[k] = es_key(lev[i], seed, stream_id, k);
    }
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base;
}

int key_chunk(int d) { return std::max(1, std::min(64, 8192 / std::max(d, 1))); }

}  // namespace

ffc_status launch_paper_keys(int sampler, const void* Y, const void* X, int dtype, int d, const KeyItem* items_dev,
                             int n_items, int64_t cap_max, uint64_t seed, cudaStream_t st) {
  if (n_items <= 0 || cap_max <= 0) return FFC_OK;
  FFC_REQUIRE(n_items <= 65535, "paper sampler keys: at most 65535 items per launch");
  const int kp = key_chunk(d);
  const size_t smem = sampler == FFC_DRAW_NEAREST ? (size_t)kp * d * sizeof(double) : 0;
  const int64_t blocks = std::min<int64_t>((cap_max + KEY_THREADS - 1) / KEY_THREADS,
                                           std::max<int64_t>(1, (int64_t)sm_count() * 16 / n_items));
  const dim3 grid((unsigned)std::max<int64_t>(blocks, 1), (unsigned)n_items);
#define FFC_KEYS(TP, MODE)                                                                                   \
  do {                                                                                                       \
    FFC_CUDA(cudaFuncSetAttribute(paper_keys_kernel<TP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)std::max<size_t>(smem, 1)));                                           \
    paper_keys_kernel<TP, MODE><<<grid, KEY_THREADS, smem, st>>>((const TP*)Y, (const TP*)X, d, items_dev,  \
                                                                 seed, kp);                                  \
  } while (0)
  if (dtype == FFC_F64) {
    if (sampler == FFC_DRAW_DISTANCE) FFC_KEYS(double, FFC_DRAW_DISTANCE);
    else if (sampler == FFC_DRAW_INV_DISTANCE) FFC_KEYS(double, FFC_DRAW_INV_DISTANCE);
    else FFC_KEYS(double, FFC_DRAW_NEAREST);
  } else {
    if (sampler == FFC_DRAW_DISTANCE) FFC_KEYS(float, FFC_DRAW_DISTANCE);
    else if (sampler == FFC_DRAW_INV_DISTANCE) FFC_KEYS(float, FFC_DRAW_INV_DISTANCE);
    else FFC_KEYS(float, FFC_DRAW_NEAREST);
  }
#undef FFC_KEYS
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace ffc

using namespace ffc;

namespace {

// Workspace of one single-node draw: items and keys, freed on the stream after the selection.
struct DrawScratch {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    const size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return reinterpret_cast<T*>(base + o);
  }
};

}  // namespace

extern "C" {

ffc_status ffc_sample_paper(int32_t sampler, const void* Y_dev, int32_t dtype, int32_t d, const int64_t* cand_dev,
                            int64_t P, const double* x_c_dev, const void* X_dev, int64_t n, int64_t s, uint64_t seed,
                            uint64_t stream_id, int64_t* rows_dev, void* stream) {
  FFC_REQUIRE(sampler == FFC_DRAW_DISTANCE || sampler == FFC_DRAW_INV_DISTANCE || sampler == FFC_DRAW_NEAREST,
              "ffc_sample_paper: unknown sampler %d", sampler);
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_sample_paper: bad dtype");
  FFC_REQUIRE(d >= 1 && P >= 0 && s >= 0 && n >= 0, "ffc_sample_paper: need d >= 1 and P, s, n >= 0");
  FFC_REQUIRE(P <= ((int64_t)1 << 31), "ffc_sample_paper: at most 2^31 candidates");
  const int64_t keep = std::min(P, s);
  FFC_REQUIRE(P <= 16384 || keep <= FFC_MAX_DRAW, "ffc_sample_paper: min(s, P) = %lld exceeds %d",
              (long long)keep, FFC_MAX_DRAW);
  if (keep == 0) return FFC_OK;
  FFC_REQUIRE(Y_dev && cand_dev && rows_dev, "ffc_sample_paper: null pointer");
  FFC_REQUIRE(sampler == FFC_DRAW_NEAREST ? (X_dev && n >= 1) : (x_c_dev != nullptr),
              "ffc_sample_paper: distance samplers need x_c_dev, nearest neighbours the sources X_dev (n >= 1)");
  cudaStream_t st = as_stream(stream);
  DrawScratch sc;
  const size_t bytes = 3 * 256 + sizeof(KeyItem) + sizeof(SelectItem) + (size_t)P * sizeof(uint64_t);
  FFC_CUDA(cudaMallocAsync((void**)&sc.base, bytes, st));
  KeyItem* kitem = sc.take<KeyItem>(1);
  SelectItem* sitem = sc.take<SelectItem>(1);
  uint64_t* keys = sc.take<uint64_t>((size_t)P);
  KeyItem hk{};
  hk.pool = cand_dev; hk.count = nullptr; hk.cap = P; hk.x_c = x_c_dev; hk.src_begin = 0; hk.src_n = n;
  hk.stream_id = stream_id; hk.keys = keys;
  SelectItem hs{};
  hs.pool = cand_dev; hs.count = nullptr; hs.P = P; hs.s = s; hs.stream_id = stream_id; hs.rows_out = rows_dev;
  hs.given = keys;
  ffc_status rc = FFC_OK;
  cudaError_t e = cudaMemcpyAsync(kitem, &hk, sizeof(hk), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sitem, &hs, sizeof(hs), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(draw items)");
  if (rc == FFC_OK) rc = launch_paper_keys(sampler, Y_dev, X_dev, dtype, d, kitem, 1, P, seed, st);
  if (rc == FFC_OK) rc = launch_select(sitem, 1, keep, seed, st);
  e = cudaFreeAsync(sc.base, st);
  if (rc == FFC_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  return rc;
}

ffc_status ffc_sample_leverage(const double* K_dev, int64_t m, int64_t n, int64_t ldk, const int64_t* cand_dev,
                               double eps, int64_t s, uint64_t seed, uint64_t stream_id, int64_t* rows_dev,
                               int64_t* s_out_host, int64_t* rank_host, void* stream) {
  FFC_REQUIRE(m >= 1 && n >= 1 && ldk >= m && s >= 0, "ffc_sample_leverage: need m, n >= 1, ldk >= m, s >= 0");
  FFC_REQUIRE(n <= 1024, "ffc_sample_leverage: n = %lld exceeds 1024 columns", (long long)n);
  FFC_REQUIRE(m <= ((int64_t)1 << 31), "ffc_sample_leverage: at most 2^31 rows");
  FFC_REQUIRE(m <= 16384 || std::min(m, s) <= FFC_MAX_DRAW, "ffc_sample_leverage: min(s, m) exceeds %d",
              FFC_MAX_DRAW);
  FFC_REQUIRE(K_dev && rows_dev && s_out_host && rank_host, "ffc_sample_leverage: null pointer");
  FFC_REQUIRE(eps >= 0.0, "ffc_sample_leverage: eps must be >= 0");
  cudaStream_t st = as_stream(stream);
  DrawScratch sc;
  const size_t bytes = 6 * 256 + sizeof(SelectItem) + (size_t)m * (2 * sizeof(double) + sizeof(int64_t)) +
                       (size_t)n * sizeof(double) + 2 * sizeof(int64_t);
  FFC_CUDA(cudaMallocAsync((void**)&sc.base, bytes, st));
  SelectItem* sitem = sc.take<SelectItem>(1);
  double* lev = sc.take<double>((size_t)m);
  double* sigma = sc.take<double>((size_t)n);
  int64_t* pool = sc.take<int64_t>((size_t)m);
  uint64_t* keys = sc.take<uint64_t>((size_t)m);
  int64_t* cnt = sc.take<int64_t>(2);
  int64_t rank = 0;
  int32_t sweeps = 0;
  const double* Kp[1] = {K_dev};
  const int64_t mm[1] = {m}, nn[1] = {n}, ll[1] = {ldk};
  double* levp[1] = {lev};
  double* sigp[1] = {sigma};
  ffc_status rc = launch_leverage_batched(1, Kp, mm, nn, ll, eps, 0, levp, sigp, &rank, &sweeps, st);
  ffc_status soft = rc == FFC_E_TOL_NOT_REACHED ? rc : FFC_OK;
  if (rc == FFC_E_TOL_NOT_REACHED) rc = FFC_OK;
  int64_t count = 0;
  if (rc == FFC_OK) {
    leverage_keys_kernel<<<1, 1024, 0, st>>>(lev, cand_dev, m, seed, stream_id, pool, keys, cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "leverage keys");
  }
  if (rc == FFC_OK && std::min(count, s) > 0) {
    SelectItem hs{};
    hs.pool = pool; hs.count = nullptr; hs.P = count; hs.s = s; hs.stream_id = stream_id; hs.rows_out = rows_dev;
    hs.given = keys;
    cudaError_t e = cudaMemcpyAsync(sitem, &hs, sizeof(hs), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpyAsync(select item)");
    if (rc == FFC_OK) rc = launch_select(sitem, 1, std::min(count, s), seed, st);
  }
  cudaError_t e = cudaFreeAsync(sc.base, st);
  if (rc == FFC_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  if (rc == FFC_OK) {
    FFC_CUDA(cudaStreamSynchronize(st));
    *s_out_host = std::min(count, s);
    *rank_host = rank;
  }
  return rc == FFC_OK ? soft : rc;
}

}  // extern "C"
