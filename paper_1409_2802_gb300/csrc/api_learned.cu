// C ABI of the learned row proposal and its training (contracts in include/ffc.h).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ffc_internal.cuh"

using namespace ffc;

namespace {

// Scratch carved from one stream-ordered allocation.
struct Scratch {
  char* base = nullptr;
  size_t used = 0;
  template <typename T>
  T* take(size_t count) {
    const size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

constexpr int64_t MAX_CANDIDATES = 1500000;

}  // namespace

extern "C" {

ffc_status ffc_features(ffc_kernel k, const void* Y_dev, int32_t dtype, int64_t M, int32_t d, const int64_t* rows_dev,
                        int64_t R, const double* x_c_dev, double radius, const double* proj_dev, float* feats_dev,
                        void* stream) {
  FFC_REQUIRE(M >= 0 && d >= 1 && R >= 0, "ffc_features: need M >= 0, d >= 1, R >= 0");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_features: bad dtype");
  if (!kernel_ok(k, d)) return FFC_E_INVALID;
  if (R == 0) return FFC_OK;
  FFC_REQUIRE(Y_dev && rows_dev && x_c_dev && proj_dev && feats_dev, "ffc_features: null pointer");
  cudaStream_t st = as_stream(stream);
  FeatItem* item = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&item, sizeof(FeatItem), st));
  FeatItem h;
  h.rows = rows_dev; h.count = nullptr; h.cap = R; h.out_begin = 0; h.x_c = x_c_dev;
  h.radius = nullptr; h.radius_host = radius;
  FFC_CUDA(cudaMemcpyAsync(item, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  ffc_status rc = launch_features(k, Y_dev, dtype, d, item, 1, R, proj_dev, feats_dev, st);
  cudaFreeAsync(item, st);
  return rc;
}

ffc_status ffc_mlp_forward(const float* params_dev, const float* feats_dev, int64_t R, float* logits_dev,
                           void* stream) {
  FFC_REQUIRE(R >= 0, "ffc_mlp_forward: R must be >= 0");
  if (R == 0) return FFC_OK;
  FFC_REQUIRE(params_dev && feats_dev && logits_dev, "ffc_mlp_forward: null pointer");
  return launch_mlp_forward(params_dev, feats_dev, R, logits_dev, as_stream(stream));
}

ffc_status ffc_sample_weighted(const int64_t* pool_dev, const float* logits_dev, int64_t P, int64_t s, uint64_t seed,
                               uint64_t stream_id, int64_t* rows_dev, void* stream) {
  FFC_REQUIRE(P >= 0 && s >= 0, "ffc_sample_weighted: need P, s >= 0");
  FFC_REQUIRE(std::min(P, s) <= FFC_MAX_DRAW, "ffc_sample_weighted: min(s, P) exceeds FFC_MAX_DRAW");
  FFC_REQUIRE(P < ((int64_t)1 << 32), "ffc_sample_weighted: P must be < 2^32");
  if (P == 0 || s == 0) return FFC_OK;
  FFC_REQUIRE(pool_dev && logits_dev && rows_dev, "ffc_sample_weighted: null pointer");
  cudaStream_t st = as_stream(stream);
  // one allocation: the item, then a key buffer of P words (used by pools above the shared-memory sort)
  const size_t kbeg = (sizeof(SelectItem) + 255) & ~(size_t)255;
  unsigned char* buf = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&buf, kbeg + (size_t)P * sizeof(uint64_t), st));
  SelectItem* item = reinterpret_cast<SelectItem*>(buf);
  SelectItem h{};
  h.pool = pool_dev; h.count = nullptr; h.P = P; h.logits = logits_dev; h.s = s; h.stream_id = stream_id;
  h.rows_out = rows_dev; h.s_out = nullptr; h.keys = reinterpret_cast<uint64_t*>(buf + kbeg);
  FFC_CUDA(cudaMemcpyAsync(item, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  ffc_status rc = launch_select(item, 1, std::min(P, s), seed, st);
  cudaFreeAsync(buf, st);
  return rc;
}

ffc_status ffc_propose_rows(ffc_kernel k, const void* Y_dev, int32_t dtype, int64_t M, int32_t d,
                            const double* x_c_dev, double radius, double xi, int64_t ex_begin, int64_t ex_end,
                            const double* proj_dev, const float* params_dev, int64_t pool_rows, int64_t s,
                            uint64_t seed, uint64_t stream_id, int64_t* rows_dev, int64_t* s_out_host,
                            int64_t* far_count_host, void* stream) {
  FFC_REQUIRE(M >= 0 && M <= MAX_CANDIDATES, "ffc_propose_rows: need 0 <= M <= %lld", (long long)MAX_CANDIDATES);
  FFC_REQUIRE(d >= 1 && s >= 0 && pool_rows >= 0, "ffc_propose_rows: need d >= 1, s >= 0, pool_rows >= 0");
  FFC_REQUIRE(s <= FFC_MAX_DRAW, "ffc_propose_rows: s exceeds FFC_MAX_DRAW");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_propose_rows: bad dtype");
  FFC_REQUIRE(s_out_host, "ffc_propose_rows: s_out_host is null");
  if (!kernel_ok(k, d)) return FFC_E_INVALID;
  FFC_REQUIRE(s == 0 || M == 0 || (Y_dev && rows_dev && x_c_dev && proj_dev && params_dev),
              "ffc_propose_rows: null pointer");
  cudaStream_t st = as_stream(stream);
  if (s == 0 || M == 0) {
    *s_out_host = 0;
    if (far_count_host) *far_count_host = 0;
    return s == 0 ? FFC_OK : FFC_E_FARFIELD_TOO_SMALL;
  }
  const bool whole = pool_rows == 0;
  const int64_t cap = whole ? M : std::min(pool_rows, M);
  Scratch sc;
  const size_t bytes = 12 * 256 + sizeof(SampleItem) + sizeof(FeatItem) + sizeof(SelectItem) +
                       (size_t)cap * (2 * sizeof(int64_t) + FFC_N_FEATURES * sizeof(float) + sizeof(float)) +
                       (size_t)M * sizeof(int32_t) + 64;
  FFC_CUDA(cudaMallocAsync((void**)&sc.base, bytes, st));
  SampleItem* sitem = sc.take<SampleItem>(1);
  FeatItem* fitem = sc.take<FeatItem>(1);
  SelectItem* pitem = sc.take<SelectItem>(1);
  int64_t* pool = sc.take<int64_t>((size_t)cap);
  float* feats = sc.take<float>((size_t)cap * FFC_N_FEATURES);
  float* logits = sc.take<float>((size_t)cap);
  int64_t* p_count = sc.take<int64_t>(1);
  int64_t* fc = sc.take<int64_t>(1);
  int64_t* s_sel = sc.take<int64_t>(1);
  int32_t* status = sc.take<int32_t>(1);
  int32_t* scratch = sc.take<int32_t>((size_t)M);
  uint64_t* skeys = sc.take<uint64_t>((size_t)cap);

  const double thr = xi * radius;
  FeatItem hf;
  hf.rows = pool; hf.count = p_count; hf.cap = cap; hf.out_begin = 0; hf.x_c = x_c_dev;
  hf.radius = nullptr; hf.radius_host = radius;
  SelectItem hp{};
  hp.pool = pool; hp.count = p_count; hp.P = cap; hp.logits = logits; hp.s = s; hp.stream_id = stream_id;
  hp.rows_out = rows_dev; hp.s_out = s_sel; hp.keys = skeys;
  FFC_CUDA(cudaMemcpyAsync(fitem, &hf, sizeof(hf), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(pitem, &hp, sizeof(hp), cudaMemcpyHostToDevice, st));
  ffc_status rc;
  if (whole) {
    rc = launch_far_field(Y_dev, dtype, M, d, x_c_dev, thr * thr, ex_begin, ex_end, pool, p_count, st);
    if (rc == FFC_OK)
      FFC_CUDA(cudaMemcpyAsync(fc, p_count, sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
  } else {
    SampleItem hs;
    hs.M = M; hs.ex_begin = ex_begin; hs.ex_end = ex_end; hs.x_c = x_c_dev;
    hs.thr2 = thr * thr; hs.radius = nullptr; hs.xi = xi;
    hs.s = cap; hs.stream_id = stream_id; hs.rows = pool;
    FFC_CUDA(cudaMemcpyAsync(sitem, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    rc = launch_sample(Y_dev, dtype, d, sitem, 1, M, cap, seed, p_count, fc, status, scratch, st);
  }
  if (rc == FFC_OK) rc = launch_features(k, Y_dev, dtype, d, fitem, 1, cap, proj_dev, feats, st);
  if (rc == FFC_OK) rc = launch_mlp_forward(params_dev, feats, cap, logits, st);
  if (rc == FFC_OK) rc = launch_select(pitem, 1, std::min(s, cap), seed, st);
  if (rc != FFC_OK) {
    cudaFreeAsync(sc.base, st);
    return rc;
  }
  int64_t h_sel = 0, h_fc = 0;
  FFC_CUDA(cudaMemcpyAsync(&h_sel, s_sel, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&h_fc, fc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  *s_out_host = h_sel;
  if (far_count_host) {
    if (h_fc >= 0) {
      *far_count_host = h_fc;
    } else {
      int64_t* idx = nullptr;
      FFC_CUDA(cudaMallocAsync((void**)&idx, (size_t)M * sizeof(int64_t), st));
      rc = ffc_far_field(Y_dev, dtype, M, d, x_c_dev, radius, xi, ex_begin, ex_end, idx, far_count_host, stream);
      cudaFreeAsync(idx, st);
      if (rc != FFC_OK) {
        cudaFreeAsync(sc.base, st);
        return rc;
      }
    }
  }
  FFC_CUDA(cudaFreeAsync(sc.base, st));
  return h_sel < s ? FFC_E_FARFIELD_TOO_SMALL : FFC_OK;
}

ffc_status ffc_mlp_loss_grad(const float* params_dev, const float* feats_dev, const double* targets_dev,
                             const int64_t* node_off_dev, int32_t n_nodes, int64_t R, double* loss_host,
                             float* grad_dev, void* stream) {
  FFC_REQUIRE(n_nodes >= 1 && R >= 1, "ffc_mlp_loss_grad: need n_nodes >= 1 and R >= 1");
  FFC_REQUIRE(params_dev && feats_dev && targets_dev && node_off_dev && grad_dev && loss_host,
              "ffc_mlp_loss_grad: null pointer");
  cudaStream_t st = as_stream(stream);
  const int n_part = mlp_backward_grid(R);
  Scratch sc;
  const size_t bytes = 6 * 256 + (size_t)R * 2 * sizeof(float) + (size_t)n_nodes * sizeof(double) +
                       (size_t)n_part * FFC_MLP_PARAMS * sizeof(float);
  FFC_CUDA(cudaMallocAsync((void**)&sc.base, bytes, st));
  float* logits = sc.take<float>((size_t)R);
  float* g_o = sc.take<float>((size_t)R);
  double* loss_part = sc.take<double>((size_t)n_nodes);
  float* part = sc.take<float>((size_t)n_part * FFC_MLP_PARAMS);
  ffc_status rc = launch_mlp_loss_grad(params_dev, feats_dev, targets_dev, node_off_dev, n_nodes, R, logits, g_o,
                                       loss_part, part, n_part, grad_dev, st);
  if (rc != FFC_OK) {
    cudaFreeAsync(sc.base, st);
    return rc;
  }
  std::vector<double> lp((size_t)n_nodes);
  FFC_CUDA(cudaMemcpyAsync(lp.data(), loss_part, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(sc.base, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  double L = 0.0;
  for (double v : lp) L += v;
  *loss_host = L / (double)n_nodes;
  return FFC_OK;
}

ffc_status ffc_adam_step(float* params_dev, const float* grad_dev, float* m_dev, float* v_dev, int64_t n,
                         int64_t step, double lr, double beta1, double beta2, double eps, void* stream) {
  FFC_REQUIRE(n >= 0 && step >= 1, "ffc_adam_step: need n >= 0 and step >= 1");
  FFC_REQUIRE(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps >= 0.0,
              "ffc_adam_step: need 0 <= beta < 1 and eps >= 0");
  if (n == 0) return FFC_OK;
  FFC_REQUIRE(params_dev && grad_dev && m_dev && v_dev, "ffc_adam_step: null pointer");
  return launch_adam(params_dev, grad_dev, m_dev, v_dev, n, step, lr, beta1, beta2, eps, as_stream(stream));
}

ffc_status ffc_leverage(const double* K_dev, int64_t m, int64_t n, int64_t ldk, double eps, int64_t r_fixed,
                        double* lev_dev, double* sigma_dev, int64_t* rank_host, void* stream) {
  FFC_REQUIRE(K_dev && lev_dev && sigma_dev, "ffc_leverage: null pointer");
  int64_t r = 0;
  ffc_status rc = launch_leverage_batched(1, &K_dev, &m, &n, &ldk, eps, r_fixed, &lev_dev, &sigma_dev, &r, nullptr,
                                          as_stream(stream));
  if (rank_host) *rank_host = r;
  return rc;
}

ffc_status ffc_leverage_batched(int32_t B, const double* const* K_dev, const int64_t* m, const int64_t* n,
                                const int64_t* ldk, double eps, int64_t r_fixed, double* const* lev_dev,
                                double* const* sigma_dev, int64_t* rank_host, void* stream) {
  FFC_REQUIRE(B >= 1 && K_dev && m && n && ldk && lev_dev && sigma_dev && rank_host,
              "ffc_leverage_batched: null argument");
  return launch_leverage_batched(B, K_dev, m, n, ldk, eps, r_fixed, lev_dev, sigma_dev, rank_host, nullptr,
                                 as_stream(stream));
}

}  // extern "C"
