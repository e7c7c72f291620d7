// ffc_compress_tree: sampled-row ID of every tree node at level >= min_level.
//
// For each node (far field of the node's centroid and radius, §4.1 steps
// 2-3): uniform sample of s far-field rows (§2.2) or the learned proposal
// (features and network logits of the candidate pool, weighted draw without
// replacement; drawn once per call for s_max rows), K' = K(rows, node sources),
// pivoted QR in tolerance mode for at most s/2 steps, T = R11^-1 R12
// (§2.1.3, App. A.1). Nodes whose tolerance is not met within s/2 steps are
// re-run with s doubled (the sample is prefix consistent) while s <= s_max.
//
// All nodes of all compressed levels run together: one "round" per sample
// size. A round is a fixed sequence of batched launches over the round's work
// items (sampling, size patch, block evaluation, cooperative QR, finalize and
// triangular solve, epilogue); only the epilogue's per-node "needs a larger
// sample" flags come back to the host, once per round.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ffc_internal.cuh"

namespace ffc {
int cpqr_rows_per_lane(int s_max);
size_t sample_smem_bytes(int64_t M_max, int d);
}  // namespace ffc

using namespace ffc;

struct ffc_tree_result {
  int64_t N = 0;
  int d = 0, dtype = 0;
  int64_t n_tree_nodes = 0;
  ffc_params p{};
  int64_t n_out = 0;
  std::vector<int32_t> node_h;
  std::vector<int64_t> begin_h, count_h, rows_off_h, skel_off_h, T_off_h;
  // outputs
  char* out_mem = nullptr;
  int32_t *node = nullptr, *rank = nullptr, *s = nullptr, *status = nullptr, *skel = nullptr;
  double *r22 = nullptr, *log_scale = nullptr, *T = nullptr;
  int64_t *far_count = nullptr, *rows_off = nullptr, *rows = nullptr, *skel_off = nullptr, *T_off = nullptr;
  // T is solved into per-node slots of capacity min(n, s_max/2) x n (T, T_off: capacity offsets) and
  // packed at the end of each call into Tp (node i at Tp_off[i], r_i x (n_i - r_i), ld r_i)
  double* Tp = nullptr;
  int64_t *Tp_off = nullptr, *count_dev = nullptr;
  // ID columns per node (node-local point indices at skel_off): identity unless nested
  int32_t *cols = nullptr, *ncols = nullptr;
  int64_t* ncols64 = nullptr;          // the same counts as int64, for the packing of T
  std::vector<int64_t> ncols_h;
  std::vector<int32_t> cols_h;         // host copy of cols
  bool cols_custom = false;            // cols differ from the identity (a nested call ran)
  // round workspace (grow-only)
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int rounds = 0;
  // learned sampler: per output node, rows drawn (<= s_max, best first) and far-field size;
  // proposal workspace (grow-only)
  int64_t *lcount = nullptr, *lfar = nullptr;
  char* pws = nullptr;
  size_t pws_bytes = 0;
  // per-point sums of the tiled far-field kernels (N x 9 floats, grow-only)
  char* pst = nullptr;
  size_t pst_bytes = 0;
  // tracing
  ffc_tree_profile prof{};
  cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  // CUDA graphs of the rounds already run: a round's memsets and launches, keyed by every byte that shapes
  // them (its item tables, launch sizes, pointers, parameters); replayed when the same round recurs
  struct RoundGraph {
    std::string key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
  };
  std::vector<RoundGraph> graphs;
  uint64_t graph_clock = 0;
  cudaStream_t cap_stream = nullptr;   // private stream the rounds are captured on
};

namespace {

struct Layout {
  size_t off = 0;
  template <typename T>
  size_t add(size_t count) {
    size_t o = (off + 255) & ~size_t(255);
    off = o + count * sizeof(T);
    return o;
  }
};

// Nested form: the column points of item q (cols of its node, node-local) copied to rows xoff.. of the
// arena, so that the block evaluation reads them as a contiguous source range.
struct GatherItem {
  int64_t xoff, begin;
  const int32_t* cols;
  int64_t n;
};

__global__ void gather_cols_kernel(const GatherItem* __restrict__ items, const void* __restrict__ X,
                                   void* __restrict__ Xc, int d, size_t esz) {
  const GatherItem it = items[blockIdx.y];
  const int64_t tot = it.n * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / d, j = e % d;
    const int64_t src = (it.begin + it.cols[c]) * d + j, dst = (it.xoff + c) * d + j;
    if (esz == sizeof(double)) reinterpret_cast<double*>(Xc)[dst] = reinterpret_cast<const double*>(X)[src];
    else reinterpret_cast<float*>(Xc)[dst] = reinterpret_cast<const float*>(X)[src];
  }
}

__global__ void patch_kernel(int W, const int64_t* s_out, int64_t s_nom, int r_cap, EvalItem* ev, CpqrItem* qr) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W) return;
  const int64_t s_eff = s_out[q];
  const bool all_rows = s_eff < s_nom;
  const int n = qr[q].n;
  int cap = all_rows ? (int)s_eff : (int)(s_eff / 2);
  cap = min(cap, min(n, r_cap));
  ev[q].s = s_eff;
  qr[q].s = (int32_t)s_eff;
  qr[q].r_max = cap;
}

// Rank handed to the finalize / triangular solve: -1 (skip) for an attempt
// that will be redone with a doubled sample, whose T would be discarded.
__global__ void gate_kernel(int W, int64_t s_nom, int s_max, const int64_t* s_out, const int32_t* st_qr,
                            const int32_t* qr_rank, int32_t* trsm_rank) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W) return;
  const int64_t s_eff = s_out[q];
  const bool again = st_qr[q] == FFC_E_TOL_NOT_REACHED && s_eff > 0 && !(s_eff < s_nom) && 2 * s_nom <= s_max;
  trsm_rank[q] = again ? -1 : qr_rank[q];
}

__global__ void epilogue_kernel(int W, const int32_t* out_idx, int64_t s_nom, int s_max, const int64_t* s_out,
                                const int64_t* fc, const double* lsc, const int32_t* st_eval,
                                const int32_t* qr_rank, const double* qr_r22, const int32_t* st_qr,
                                int32_t* res_rank, int32_t* res_s, int32_t* res_status, double* res_r22,
                                double* res_lsc, int64_t* res_fc, int32_t* flags) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W) return;
  const int o = out_idx[q];
  const int64_t s_eff = s_out[q];
  const bool all_rows = s_eff < s_nom;
  const int qs = st_qr[q], es = st_eval[q];
  int status = FFC_OK;
  if (s_eff == 0) status = FFC_E_FARFIELD_TOO_SMALL;
  else if (es == FFC_E_SINGULAR) status = FFC_E_SINGULAR;
  else if (qs == FFC_E_TIMEOUT) status = FFC_E_TIMEOUT;
  else if (qs == FFC_E_TOL_NOT_REACHED) status = FFC_E_TOL_NOT_REACHED;
  const bool again = status == FFC_E_TOL_NOT_REACHED && !all_rows && 2 * s_nom <= s_max;
  flags[q] = again ? 1 : 0;
  res_rank[o] = qr_rank[q];
  res_s[o] = (int32_t)s_eff;
  res_status[o] = status;
  res_r22[o] = qr_r22[q];
  res_lsc[o] = lsc[q];
  res_fc[o] = fc[q];
}

// Packed offsets of T: node i holds rank_i x (n_i - rank_i) doubles.
__global__ void pack_offsets_kernel(int64_t n_out, const int32_t* rank, const int64_t* count, int64_t* off) {
  __shared__ int64_t part[1024];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n_out; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < n_out ? (int64_t)rank[i] * (count[i] - rank[i]) : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const int64_t add = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n_out) off[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) off[n_out] = carry;
}

__global__ void pack_copy_kernel(int64_t n_out, const int64_t* cap_off, const int64_t* off, const double* src,
                                 double* dst) {
  const int64_t i = blockIdx.y;
  if (i >= n_out) return;
  const int64_t len = off[i + 1] - off[i];
  const double* s = src + cap_off[i];
  double* d = dst + off[i];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = s[e];
}

ffc_status alloc_outputs(ffc_tree_result* R) {
  const int64_t n = R->n_out;
  const int64_t rows_cap = R->rows_off_h[n], skel_cap = R->skel_off_h[n], T_cap = R->T_off_h[n];
  Layout L;
  size_t o_node = L.add<int32_t>(n), o_rank = L.add<int32_t>(n), o_s = L.add<int32_t>(n),
         o_status = L.add<int32_t>(n), o_r22 = L.add<double>(n), o_lsc = L.add<double>(n),
         o_fc = L.add<int64_t>(n), o_rows_off = L.add<int64_t>(n + 1), o_rows = L.add<int64_t>(rows_cap),
         o_skel_off = L.add<int64_t>(n + 1), o_skel = L.add<int32_t>(skel_cap), o_T_off = L.add<int64_t>(n + 1),
         o_T = L.add<double>(T_cap), o_Tp = L.add<double>(T_cap), o_Tp_off = L.add<int64_t>(n + 1),
         o_cnt = L.add<int64_t>(n), o_cols = L.add<int32_t>(skel_cap), o_nc = L.add<int32_t>(n),
         o_nc64 = L.add<int64_t>(n);
  FFC_CUDA(cudaMalloc((void**)&R->out_mem, L.off));
  char* b = R->out_mem;
  R->node = (int32_t*)(b + o_node); R->rank = (int32_t*)(b + o_rank); R->s = (int32_t*)(b + o_s);
  R->status = (int32_t*)(b + o_status); R->r22 = (double*)(b + o_r22); R->log_scale = (double*)(b + o_lsc);
  R->far_count = (int64_t*)(b + o_fc); R->rows_off = (int64_t*)(b + o_rows_off); R->rows = (int64_t*)(b + o_rows);
  R->skel_off = (int64_t*)(b + o_skel_off); R->skel = (int32_t*)(b + o_skel); R->T_off = (int64_t*)(b + o_T_off);
  R->T = (double*)(b + o_T);
  R->Tp = (double*)(b + o_Tp); R->Tp_off = (int64_t*)(b + o_Tp_off); R->count_dev = (int64_t*)(b + o_cnt);
  R->cols = (int32_t*)(b + o_cols); R->ncols = (int32_t*)(b + o_nc); R->ncols64 = (int64_t*)(b + o_nc64);
  FFC_CUDA(cudaMemcpy(R->count_dev, R->count_h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  // every node starts with all of its points as its columns
  R->ncols_h = R->count_h;
  {
    std::vector<int32_t> c(skel_cap), nc(n);
    for (int64_t i = 0; i < n; ++i) {
      nc[i] = (int32_t)R->count_h[i];
      for (int64_t j = 0; j < R->count_h[i]; ++j) c[R->skel_off_h[i] + j] = (int32_t)j;
    }
    FFC_CUDA(cudaMemcpy(R->cols, c.data(), sizeof(int32_t) * skel_cap, cudaMemcpyHostToDevice));
    R->cols_h = c;
    FFC_CUDA(cudaMemcpy(R->ncols, nc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    FFC_CUDA(cudaMemcpy(R->ncols64, R->count_h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  }
  FFC_CUDA(cudaMemcpy(R->node, R->node_h.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
  FFC_CUDA(cudaMemcpy(R->rows_off, R->rows_off_h.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
  FFC_CUDA(cudaMemcpy(R->skel_off, R->skel_off_h.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
  FFC_CUDA(cudaMemcpy(R->T_off, R->T_off_h.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
  return FFC_OK;
}

__global__ void learned_round_kernel(int W, const int32_t* out_idx, int64_t s_nom, const int64_t* lcount,
                                     const int64_t* lfar, int64_t* s_out, int64_t* fc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= W) return;
  const int o = out_idx[q];
  const int64_t c = lcount[o];
  s_out[q] = c < s_nom ? c : s_nom;
  fc[q] = lfar[o];
}

__global__ void copy_counts_kernel(int n, const int64_t* src, int64_t* dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

ffc_status grow(char** buf, size_t* have, size_t want, cudaStream_t st) {
  if (want <= *have) return FFC_OK;
  if (*buf) {
    FFC_CUDA(cudaStreamSynchronize(st));
    FFC_CUDA(cudaFree(*buf));
    *buf = nullptr;
  }
  const size_t bytes = want + want / 4;
  FFC_CUDA(cudaMalloc((void**)buf, bytes));
  *have = bytes;
  return FFC_OK;
}

// Every node's columns back to all of its points.
ffc_status reset_columns(ffc_tree_result* R, cudaStream_t st) {
  const int64_t n = R->n_out;
  for (int64_t i = 0; i < n; ++i) {
    R->ncols_h[i] = R->count_h[i];
    for (int64_t j = 0; j < R->count_h[i]; ++j) R->cols_h[R->skel_off_h[i] + j] = (int32_t)j;
  }
  std::vector<int32_t> nc(R->ncols_h.begin(), R->ncols_h.end());
  FFC_CUDA(cudaMemcpyAsync(R->cols, R->cols_h.data(), sizeof(int32_t) * R->cols_h.size(), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(R->ncols, nc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(R->ncols64, R->ncols_h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaStreamSynchronize(st));   // the host vectors may change before the copies would run
  R->cols_custom = false;
  return FFC_OK;
}

// Nested form: the columns of the output nodes `lv` (one level) from their children's results: the
// left child's skeleton points, then the right child's, each in pivot order (node-local indices of
// the parent); a child whose ID is not usable (status other than OK / TOL_NOT_REACHED, or no rows)
// contributes all of its points.
ffc_status nested_columns(ffc_tree_result* R, const std::vector<int>& lv, int64_t first, cudaStream_t st) {
  const int64_t n = R->n_out;
  std::vector<int32_t> rank(n), status(n), sv(n), skel(R->cols_h.size());
  FFC_CUDA(cudaMemcpyAsync(rank.data(), R->rank, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(status.data(), R->status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(sv.data(), R->s, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(skel.data(), R->skel, sizeof(int32_t) * skel.size(), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  int64_t lo = INT64_MAX, hi = 0;
  for (int o : lv) {
    const int64_t b = R->node_h[o];
    int64_t c = 0;
    for (int64_t ch = 2 * b + 1; ch <= 2 * b + 2; ++ch) {
      const int64_t oc = ch - first;
      const int64_t shift = R->begin_h[oc] - R->begin_h[o];
      const bool usable = (status[oc] == FFC_OK || status[oc] == FFC_E_TOL_NOT_REACHED) && sv[oc] > 0;
      const int64_t base = R->skel_off_h[oc];
      if (usable) {
        for (int k = 0; k < rank[oc]; ++k)
          R->cols_h[R->skel_off_h[o] + c++] = (int32_t)(shift + R->cols_h[base + skel[base + k]]);
      } else {
        for (int64_t j = 0; j < R->count_h[oc]; ++j) R->cols_h[R->skel_off_h[o] + c++] = (int32_t)(shift + j);
      }
    }
    R->ncols_h[o] = c;
    lo = std::min(lo, R->skel_off_h[o]);
    hi = std::max(hi, R->skel_off_h[o] + c);
  }
  std::vector<int32_t> nc(R->ncols_h.begin(), R->ncols_h.end());
  FFC_CUDA(cudaMemcpyAsync(R->cols + lo, R->cols_h.data() + lo, sizeof(int32_t) * (hi - lo), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(R->ncols, nc.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(R->ncols64, R->ncols_h.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  return FFC_OK;
}

// Bytes of sampled blocks one QR launch may hold: below the 129 MB L2 (ffc_params.qr_l2_budget_mb,
// default QR_L2_BUDGET_MB_DEFAULT).

// Learned sampler: for every output node, the candidate pool (whole far field
// or a uniform pool), features, network logits and the weighted draw of its
// min(s_max, P) best rows, in key order. The keys do not depend on s, so
// every sample-size round takes a prefix of these rows. Nodes are processed
// in groups of at most PROPOSE_ROWS candidate rows.
constexpr int64_t PROPOSE_ROWS = 48ll << 20;

ffc_status propose_tree(ffc_tree_result* R, const void* X, const ffc_tree* tree, cudaStream_t st) {
  const ffc_params& P = R->p;
  const int d = R->d;
  const int64_t n_out = R->n_out;
  // the paper's samplers (distance, nearest neighbours) draw from the whole far field by their own keys
  const bool paper = P.sampler >= FFC_SAMPLE_DISTANCE;
  const bool whole = paper || P.pool_rows == 0;
  if (!R->lcount) {
    FFC_CUDA(cudaMalloc((void**)&R->lcount, sizeof(int64_t) * 2 * n_out));
    R->lfar = R->lcount + n_out;
  }
  float *pyy = nullptr, *pyg = nullptr;
  const double* proj = P.proj_dev;
  if (whole) {
    // per-point sums (N x 9 floats), then room for 8 x d zero directions (the far-field kernels form the
    // learned features as they go; the paper's samplers ignore them)
    const size_t pts = ((size_t)R->N * 9 * sizeof(float) + 255) & ~size_t(255);
    ffc_status rc = grow(&R->pst, &R->pst_bytes, pts + (size_t)8 * d * sizeof(double), st);
    if (rc != FFC_OK) return rc;
    pyy = (float*)R->pst;
    pyg = pyy + R->N;
    if (!proj) {
      double* z = (double*)(R->pst + pts);
      FFC_CUDA(cudaMemsetAsync(z, 0, (size_t)8 * d * sizeof(double), st));
      proj = z;
    }
    rc = launch_point_stats(X, R->dtype, R->N, d, proj, pyy, pyg, st);
    if (rc != FFC_OK) return rc;
  }
  int64_t o0 = 0;
  while (o0 < n_out) {
    // group [o0, o1)
    int64_t o1 = o0, rows = 0;
    while (o1 < n_out && (o1 == o0 || rows + (whole ? R->N - R->count_h[o1] : P.pool_rows) <= PROPOSE_ROWS) &&
           o1 - o0 < 2048) {
      rows += whole ? R->N - R->count_h[o1] : P.pool_rows;
      ++o1;
    }
    const int g = (int)(o1 - o0);
    std::vector<int64_t> cap(g), base(g);
    int64_t tot = 0;
    for (int i = 0; i < g; ++i) {
      cap[i] = whole ? std::max<int64_t>(R->N - R->count_h[o0 + i], 1) : P.pool_rows;
      base[i] = tot;
      tot += cap[i];
    }
    const int64_t tiles = far_tiles_count(R->N);
    Layout L;
    const size_t o_far = L.add<FarItem>(g), o_smp = L.add<SampleItem>(g), o_fi = L.add<FeatItem>(g),
                 o_si = L.add<SelectItem>(g), o_ki = L.add<KeyItem>(paper ? g : 0), o_pool = L.add<int64_t>(tot),
                 o_feat = L.add<float>((size_t)tot * FFC_N_FEATURES), o_lg = L.add<float>(tot),
                 o_key = L.add<uint64_t>(tot),
                 o_cnt = L.add<int64_t>(g), o_fc = L.add<int64_t>(g), o_st = L.add<int32_t>(g),
                 o_tc = L.add<int64_t>(whole ? (size_t)g * tiles : 0),
                 o_mask = L.add<uint32_t>(whole ? (size_t)g * tiles * 4 : 0),
                 o_nst = L.add<char>(whole ? far_tiles_node_bytes(g, d) : 0),
                 o_scr = L.add<int32_t>(whole ? 0 : (size_t)std::min(g, 2048) * R->N);
    ffc_status rc = grow(&R->pws, &R->pws_bytes, L.off, st);
    if (rc != FFC_OK) return rc;
    char* b = R->pws;
    FarItem* d_far = (FarItem*)(b + o_far);
    SampleItem* d_smp = (SampleItem*)(b + o_smp);
    FeatItem* d_fi = (FeatItem*)(b + o_fi);
    SelectItem* d_si = (SelectItem*)(b + o_si);
    KeyItem* d_ki = (KeyItem*)(b + o_ki);
    int64_t* pool = (int64_t*)(b + o_pool);
    float* feats = (float*)(b + o_feat);
    float* logits = (float*)(b + o_lg);
    uint64_t* skeys = (uint64_t*)(b + o_key);
    int64_t* cnt = (int64_t*)(b + o_cnt);
    int64_t* fc = (int64_t*)(b + o_fc);
    int32_t* sst = (int32_t*)(b + o_st);
    int64_t* tcnt = (int64_t*)(b + o_tc);
    uint32_t* fmask = (uint32_t*)(b + o_mask);
    void* nst = (void*)(b + o_nst);
    int32_t* scratch = (int32_t*)(b + o_scr);
    std::vector<FarItem> hfar(whole ? g : 0);
    std::vector<SampleItem> hsmp(whole ? 0 : g);
    std::vector<FeatItem> hfi(g);
    std::vector<SelectItem> hsi(g);
    std::vector<KeyItem> hki(paper ? g : 0);
    for (int i = 0; i < g; ++i) {
      const int64_t o = o0 + i, node = R->node_h[o], bgn = R->begin_h[o], n = R->count_h[o];
      const double* xc = tree->centroid_dev + node * d;
      const double* rad = tree->radius_dev + node;
      if (whole) {
        FarItem& f = hfar[i];
        f.M = R->N; f.ex_begin = bgn; f.ex_end = bgn + n; f.x_c = xc; f.radius = rad; f.radius_host = 0.0;
        f.xi = P.xi; f.list = pool + base[i]; f.count = cnt + i;
      } else {
        SampleItem& si = hsmp[i];
        si.M = R->N; si.ex_begin = bgn; si.ex_end = bgn + n; si.x_c = xc; si.thr2 = 0.0; si.radius = rad;
        si.xi = P.xi; si.s = cap[i]; si.stream_id = (uint64_t)node; si.rows = pool + base[i];
      }
      FeatItem& fi = hfi[i];
      fi.rows = pool + base[i]; fi.count = cnt + i; fi.cap = cap[i]; fi.out_begin = base[i];
      fi.x_c = xc; fi.radius = rad; fi.radius_host = 0.0;
      SelectItem& se = hsi[i];
      se.pool = pool + base[i]; se.count = cnt + i; se.P = cap[i]; se.logits = logits + base[i]; se.s = P.s_max;
      se.stream_id = (uint64_t)node; se.rows_out = R->rows + R->rows_off_h[o]; se.s_out = R->lcount + o;
      se.keys = skeys + base[i];
      if (paper) {
        KeyItem& ki = hki[i];
        ki.pool = pool + base[i]; ki.count = cnt + i; ki.cap = cap[i]; ki.x_c = xc; ki.src_begin = bgn; ki.src_n = n;
        ki.stream_id = (uint64_t)node; ki.keys = skeys + base[i];
        se.given = skeys + base[i];
        se.keys = nullptr;
      }
    }
    if (whole) FFC_CUDA(cudaMemcpyAsync(d_far, hfar.data(), sizeof(FarItem) * g, cudaMemcpyHostToDevice, st));
    else FFC_CUDA(cudaMemcpyAsync(d_smp, hsmp.data(), sizeof(SampleItem) * g, cudaMemcpyHostToDevice, st));
    FFC_CUDA(cudaMemcpyAsync(d_fi, hfi.data(), sizeof(FeatItem) * g, cudaMemcpyHostToDevice, st));
    FFC_CUDA(cudaMemcpyAsync(d_si, hsi.data(), sizeof(SelectItem) * g, cudaMemcpyHostToDevice, st));
    if (paper) FFC_CUDA(cudaMemcpyAsync(d_ki, hki.data(), sizeof(KeyItem) * g, cudaMemcpyHostToDevice, st));
    if (whole) {
      // far-field lists and features together, tiled over (points x nodes)
      rc = launch_far_features_tiled(P.kernel, X, R->dtype, R->N, d, d_far, d_fi, g, proj, pyy, pyg, nst,
                                     tcnt, fmask, feats, st);
      if (rc == FFC_OK) {
        copy_counts_kernel<<<(g + 127) / 128, 128, 0, st>>>(g, cnt, fc);
        FFC_CUDA(cudaGetLastError());
      }
    } else {
      rc = launch_sample(X, R->dtype, d, d_smp, g, R->N, P.pool_rows, P.seed, cnt, fc, sst, scratch, st);
      const int64_t cap_max = *std::max_element(cap.begin(), cap.end());
      if (rc == FFC_OK) rc = launch_features(P.kernel, X, R->dtype, d, d_fi, g, cap_max, P.proj_dev, feats, st);
    }
    if (paper) {
      const int draw = P.sampler == FFC_SAMPLE_DISTANCE ? FFC_DRAW_DISTANCE
                     : P.sampler == FFC_SAMPLE_INV_DISTANCE ? FFC_DRAW_INV_DISTANCE : FFC_DRAW_NEAREST;
      const int64_t cap_max = *std::max_element(cap.begin(), cap.end());
      if (rc == FFC_OK) rc = launch_paper_keys(draw, X, X, R->dtype, d, d_ki, g, cap_max, P.seed, st);
    } else if (rc == FFC_OK) {
      rc = launch_mlp_forward(P.mlp_dev, feats, tot, logits, st);
    }
    if (rc == FFC_OK) rc = launch_select(d_si, g, P.s_max, P.seed, st);
    if (rc != FFC_OK) return rc;
    copy_counts_kernel<<<(g + 127) / 128, 128, 0, st>>>(g, fc, R->lfar + o0);
    FFC_CUDA(cudaGetLastError());
    if (R->prof.enabled) R->prof.launches += (whole ? 6 : 2) + 3;
    o0 = o1;
  }
  return FFC_OK;
}

int group_size_tree(int64_t s, int64_t n, int64_t elems) {
  int64_t g = (s * n + elems - 1) / std::max<int64_t>(elems, 1);
  g = std::min<int64_t>(g, std::max<int64_t>(1, n / 4));
  return (int)std::max<int64_t>(1, g);
}

// One sample-size round over the work items `items` (indices into outputs).
ffc_status run_round(ffc_tree_result* R, const void* X, const ffc_tree* tree, const std::vector<int>& items,
                     int64_t s_nom, std::vector<int>& again, cudaStream_t st) {
  const int W = (int)items.size();
  const ffc_params& P = R->p;
  const int d = R->d;
  const int r_cap_glob = P.s_max / 2;
  const int rcap_round = (int)std::min<int64_t>(s_nom, r_cap_glob);
  const size_t esz = P.precision == FFC_MIXED ? sizeof(float) : sizeof(double);   // K' element size
  const bool nested = P.nested != 0;
  const size_t pts_esz = R->dtype == FFC_F64 ? sizeof(double) : sizeof(float);
  // per-item sizes
  std::vector<int64_t> koff(W), noff(W), goff(W), r11off(W), r11foff(W), tiles(W), t5base(W);
  std::vector<int> g(W);
  int64_t SN = 0, elems = 0, RC = 0, RCF = 0, tiles_tot = 0, n_max = 0, t5rows = 0;
  const int eshape = eval_shape(P.kernel, d, P.precision, P.eval_path);
  for (int q = 0; q < W; ++q) {
    const int64_t n = R->ncols_h[items[q]];
    noff[q] = SN;
    koff[q] = SN * s_nom;
    SN += n;
    elems += n * s_nom;
    r11off[q] = RC;
    const int64_t rc = std::min<int64_t>(n, rcap_round);
    RC += rc * rc;
    r11foff[q] = RCF;
    RCF += ((rc + 3) & ~3) * ((rc + 3) & ~3);   // the FP32 copy's padded leading dimension
    tiles[q] = tiles_tot;
    tiles_tot += eval_tiles(s_nom, n, eshape);
    n_max = std::max(n_max, n);
    t5base[q] = t5rows;
    if (eshape >= 2) t5rows += eval_tc5_pad_s(s_nom) + eval_tc5_pad_n(n);
  }
  const int big_min = P.qr_big_min_s > 0 ? P.qr_big_min_s : QR_BIG_MIN_S_DEFAULT;
  const int big = (P.precision == FFC_MIXED && s_nom >= big_min) ? 1 : 0;
  // the blocked QR needs 16-byte aligned columns (ld = s_nom elements)
  int nb = P.qr_panel > 0 ? P.qr_panel : qr_panel(P.precision, (int)s_nom, big);
  if (((size_t)s_nom * esz) % 16 != 0) nb = 1;
  // the lazy form's write-back depth (unblocked rounds only; cpqr_lazy() says where it runs)
  const int defer = nb > 1 ? 0 : (P.qr_defer > 0 ? P.qr_defer : QR_DEFER_DEFAULT);
  const int cap = cpqr_max_ctas(P.precision, (int)s_nom, big, nb, defer);
  if (cap <= 0) { set_error("compress_tree: QR kernel cannot be resident"); return FFC_E_CUDA; }
  // The round's QR runs as one cooperative launch per sub-batch of
  // consecutive items whose blocks together fit in QR_L2_BUDGET bytes: the
  // unblocked QR streams each block once per step, so a sub-batch that stays
  // L2-resident runs its steps from L2 instead of HBM.
  // Group sizes within a sub-batch: about 16K elements per CTA when it fits
  // in one co-resident launch; otherwise the groups shrink in proportion and
  // CTAs are shared round-robin between items (each CTA walks its items in
  // increasing order).
  std::vector<int> sb;   // sub-batch starts, then W
  {
    const size_t QR_L2_BUDGET = (size_t)(P.qr_l2_budget_mb > 0 ? P.qr_l2_budget_mb : QR_L2_BUDGET_MB_DEFAULT) << 20;
    size_t acc = 0;
    for (int q = 0; q < W; ++q) {
      const size_t bq = esz * (size_t)s_nom * (size_t)R->ncols_h[items[q]];
      if (q == 0 || acc + bq > QR_L2_BUDGET) {
        sb.push_back(q);
        acc = 0;
      }
      acc += bq;
    }
    sb.push_back(W);
  }
  const int n_sb = (int)sb.size() - 1;
  std::vector<int> sb_grid(n_sb), sb_as(n_sb), sb_coff(n_sb), sb_nb;
  std::vector<int32_t> hoff;
  std::vector<CtaAssign> ha;
  int64_t G = 0;
  for (int b = 0; b < n_sb; ++b) {
    const int q0 = sb[b], q1 = sb[b + 1];
    int64_t Gb = 0, elems_b = 0;
    for (int q = q0; q < q1; ++q) {
      const int64_t n = R->ncols_h[items[q]];
      Gb += std::max<int64_t>(cpqr_min_group(n), group_size_tree(s_nom, n, 4096));
      elems_b += s_nom * n;
    }
    const bool shared_ctas = Gb > cap;
    const int64_t per_cta = shared_ctas ? std::max<int64_t>(1, elems_b / cap) : 16384;
    int64_t Gsum = 0;
    for (int q = q0; q < q1; ++q) {
      const int64_t n = R->ncols_h[items[q]];
      int64_t gq = shared_ctas ? (s_nom * n) / per_cta : group_size_tree(s_nom, n, 4096);
      gq = std::max<int64_t>(1, std::min<int64_t>({gq, (int64_t)cap, std::max<int64_t>(1, n / 4)}));
      gq = std::max<int64_t>(gq, cpqr_min_group(n));   // per-CTA column cap (<= cap for N <= 1.5M)
      g[q] = (int)gq;
      goff[q] = G;
      G += g[q];
      Gsum += g[q];
    }
    const int grid = shared_ctas ? cap : (int)Gsum;
    int ncmax = 0;
    for (int q = q0; q < q1; ++q)
      ncmax = std::max<int>(ncmax, (int)((R->ncols_h[items[q]] + g[q] - 1) / g[q]));
    sb_nb.push_back(ncmax <= QR_FS_COLS ? nb : 1);
    std::vector<std::vector<CtaAssign>> lists(grid);
    int64_t ptr = 0;
    for (int q = q0; q < q1; ++q) {
      for (int c = 0; c < g[q]; ++c) lists[(ptr + c) % grid].push_back(CtaAssign{q, c, g[q], 0});
      ptr = (ptr + g[q]) % grid;
    }
    sb_grid[b] = grid;
    sb_as[b] = (int)ha.size();
    sb_coff[b] = (int)hoff.size();
    const int32_t base = (int32_t)ha.size();
    for (int c = 0; c < grid; ++c) {
      hoff.push_back((int32_t)ha.size() - base);
      ha.insert(ha.end(), lists[c].begin(), lists[c].end());
    }
    hoff.push_back((int32_t)ha.size() - base);
  }
  // triangular-solve tiles
  std::vector<int64_t> ttiles(W);
  int64_t ttot = 0;
  for (int q = 0; q < W; ++q) { ttiles[q] = ttot; ttot += trsm_tiles(R->ncols_h[items[q]]); }

  const int64_t scratch_ctas = std::min<int64_t>(W, 2048);
  const bool learned = P.sampler != FFC_SAMPLE_UNIFORM;   // learned or paper sampler: rows drawn once per call
  Layout L;
  const size_t o_si = L.add<SampleItem>(W), o_ei = L.add<EvalItem>(W), o_qi = L.add<CpqrItem>(W),
               o_ti = L.add<TrsmItem>(W), o_as = L.add<CtaAssign>(ha.size()), o_coff = L.add<int32_t>(hoff.size()),
               o_sout = L.add<int64_t>(W),
               o_fc = L.add<int64_t>(W), o_sst = L.add<int32_t>(W), o_md = L.add<double>(W), o_ls = L.add<double>(W),
               o_est = L.add<int32_t>(W), o_K = L.add<double>((size_t)s_nom * SN),
               o_piv = L.add<int32_t>((size_t)W * rcap_round), o_beta = L.add<double>((size_t)W * rcap_round),
               o_vn1 = L.add<double>(SN), o_vn2 = L.add<double>(SN), o_sel = L.add<uint8_t>(SN),
               o_slots = L.add<Slot>(2 * G), o_red = L.add<unsigned long long>(12 * (size_t)W),
               o_bar = L.add<unsigned>(W), o_rank = L.add<int32_t>(W),
               o_r22 = L.add<double>(W), o_qst = L.add<int32_t>(W), o_R11 = L.add<double>(std::max<int64_t>(RC, 1)),
               o_R11f = L.add<float>(P.precision == FFC_MIXED ? std::max<int64_t>(RCF, 1) : 0),
               o_scr = L.add<int32_t>((size_t)scratch_ctas * R->N), o_flag = L.add<int32_t>(W),
               o_oidx = L.add<int32_t>(W), o_trank = L.add<int32_t>(W),
               o_F = L.add<char>(nb > 1 ? (size_t)SN * QR_F_STRIDE * esz : 0),
               o_xa = L.add<char>(nested ? (size_t)SN * d * pts_esz : 0), o_gi = L.add<GatherItem>(nested ? W : 0),
               o_t5 = L.add<char>(eshape >= 2 ? eval_tc5_scratch_bytes(t5rows, d) : 0);
  if (L.off > R->ws_bytes) {
    if (R->ws) {
      FFC_CUDA(cudaStreamSynchronize(st));
      FFC_CUDA(cudaFree(R->ws));
      R->ws = nullptr;
    }
    size_t want = L.off + L.off / 4;
    FFC_CUDA(cudaMalloc((void**)&R->ws, want));
    R->ws_bytes = want;
  }
  char* b = R->ws;
  SampleItem* d_si = (SampleItem*)(b + o_si);
  EvalItem* d_ei = (EvalItem*)(b + o_ei);
  CpqrItem* d_qi = (CpqrItem*)(b + o_qi);
  TrsmItem* d_ti = (TrsmItem*)(b + o_ti);
  CtaAssign* d_as = (CtaAssign*)(b + o_as);
  int32_t* d_coff = (int32_t*)(b + o_coff);
  int64_t* s_out = (int64_t*)(b + o_sout);
  int64_t* fc = (int64_t*)(b + o_fc);
  int32_t* sst = (int32_t*)(b + o_sst);
  double* mind2 = (double*)(b + o_md);
  double* lsc = (double*)(b + o_ls);
  int32_t* est = (int32_t*)(b + o_est);
  double* K = (double*)(b + o_K);
  int32_t* piv = (int32_t*)(b + o_piv);
  double* beta = (double*)(b + o_beta);
  double* vn1 = (double*)(b + o_vn1);
  double* vn2 = (double*)(b + o_vn2);
  uint8_t* sel = (uint8_t*)(b + o_sel);
  Slot* slots = (Slot*)(b + o_slots);
  unsigned long long* red = (unsigned long long*)(b + o_red);
  unsigned* bar = (unsigned*)(b + o_bar);
  int32_t* qrank = (int32_t*)(b + o_rank);
  double* qr22 = (double*)(b + o_r22);
  int32_t* qst = (int32_t*)(b + o_qst);
  double* R11 = (double*)(b + o_R11);
  float* R11f = P.precision == FFC_MIXED ? (float*)(b + o_R11f) : nullptr;
  int32_t* scratch = (int32_t*)(b + o_scr);
  int32_t* flags = (int32_t*)(b + o_flag);
  int32_t* oidx = (int32_t*)(b + o_oidx);
  int32_t* trank = (int32_t*)(b + o_trank);
  char* Fbuf = nb > 1 ? (char*)(b + o_F) : nullptr;
  void* Xcols = nested ? (void*)(b + o_xa) : nullptr;
  GatherItem* d_gi = (GatherItem*)(b + o_gi);
  void* t5scr = eshape >= 2 ? (void*)(b + o_t5) : nullptr;

  std::vector<SampleItem> hs(W);
  std::vector<EvalItem> he(W);
  std::vector<CpqrItem> hq(W);
  std::vector<TrsmItem> ht(W);
  std::vector<int32_t> ho(W);
  for (int q = 0; q < W; ++q) {
    const int o = items[q];
    // n: the ID's columns (the node's points unless nested); the far field excludes all of its points
    const int64_t node = R->node_h[o], bgn = R->begin_h[o], npts = R->count_h[o], n = R->ncols_h[o];
    ho[q] = o;
    SampleItem& si = hs[q];
    si.M = R->N; si.ex_begin = bgn; si.ex_end = bgn + npts;
    si.x_c = tree->centroid_dev + node * d; si.thr2 = 0.0; si.radius = tree->radius_dev + node; si.xi = P.xi;
    si.s = s_nom; si.stream_id = (uint64_t)node; si.rows = R->rows + R->rows_off_h[o];
    EvalItem& ei = he[q];
    ei.rows = R->rows + R->rows_off_h[o]; ei.s = s_nom; ei.x_begin = nested ? noff[q] : bgn; ei.n = n; ei.K = (void*)((char*)K + esz * koff[q]); ei.ldk = s_nom;
    ei.center = P.precision == FFC_MIXED ? tree->centroid_dev + node * d : nullptr;
    ei.tile_begin = tiles[q]; ei.row_tiles = eval_row_tiles(s_nom, eshape);
    ei.tc_base = t5base[q]; ei.tc_spad = eval_tc5_pad_s(s_nom); ei.tc_npad = eval_tc5_pad_n(n);
    CpqrItem& qi = hq[q];
    qi = CpqrItem{};
    qi.A = (void*)((char*)K + esz * koff[q]); qi.lda = s_nom; qi.s = (int32_t)s_nom; qi.n = (int32_t)n; qi.r_max = 0; qi.tol = P.tol;
    qi.piv = piv + (size_t)q * rcap_round; qi.beta = beta + (size_t)q * rcap_round;
    qi.vn1 = vn1 + noff[q]; qi.vn2 = vn2 + noff[q]; qi.selected = sel + noff[q];
    qi.slots = slots + 2 * goff[q]; qi.red = red + 12 * (size_t)q; qi.barrier = bar + q; qi.rank_out = qrank + q;
    qi.r22_out = qr22 + q;
    qi.status_out = qst + q;
    qi.F = Fbuf ? (void*)(Fbuf + (size_t)noff[q] * QR_F_STRIDE * esz) : nullptr;
    TrsmItem& ti = ht[q];
    ti = TrsmItem{};
    ti.A = (void*)((char*)K + esz * koff[q]); ti.lda = s_nom; ti.n = (int32_t)n; ti.rank = trank + q; ti.piv = qi.piv; ti.beta = qi.beta;
    ti.selected = qi.selected; ti.skel_perm = R->skel + R->skel_off_h[o]; ti.R11 = R11 + r11off[q]; ti.R11f = R11f ? R11f + r11foff[q] : nullptr;
    ti.T = R->T + R->T_off_h[o]; ti.ldt = 0; ti.r_cap = (int32_t)std::min<int64_t>(n, rcap_round);
    ti.tile_begin = ttiles[q];
  }
  FFC_CUDA(cudaMemcpyAsync(d_si, hs.data(), sizeof(SampleItem) * W, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_ei, he.data(), sizeof(EvalItem) * W, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_qi, hq.data(), sizeof(CpqrItem) * W, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_ti, ht.data(), sizeof(TrsmItem) * W, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_as, ha.data(), sizeof(CtaAssign) * ha.size(), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_coff, hoff.data(), sizeof(int32_t) * hoff.size(), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(oidx, ho.data(), sizeof(int32_t) * W, cudaMemcpyHostToDevice, st));
  std::vector<GatherItem> hg(nested ? W : 0);
  for (int q = 0; q < (int)hg.size(); ++q) {
    const int o = items[q];
    hg[q] = GatherItem{noff[q], R->begin_h[o], R->cols + R->skel_off_h[o], R->ncols_h[o]};
  }
  if (nested) FFC_CUDA(cudaMemcpyAsync(d_gi, hg.data(), sizeof(GatherItem) * W, cudaMemcpyHostToDevice, st));

  const bool prof = R->prof.enabled != 0;
  // The round's memsets and launches on stream cs; while cs is capturing, the profile's events become
  // event-record nodes of the graph.
  auto record = [&](int i, cudaStream_t cs, bool capturing) -> ffc_status {
    if (prof)
      FFC_CUDA(capturing ? cudaEventRecordWithFlags(R->ev[i], cs, cudaEventRecordExternal) : cudaEventRecord(R->ev[i], cs));
    return FFC_OK;
  };
  auto enqueue = [&](cudaStream_t cs, bool capturing) -> ffc_status {
    FFC_CUDA(cudaMemsetAsync(est, 0, sizeof(int32_t) * W, cs));
    FFC_CUDA(cudaMemsetAsync(bar, 0, sizeof(unsigned) * W, cs));
    FFC_CUDA(cudaMemsetAsync(slots, 0, sizeof(Slot) * 2 * G, cs));   // the QR's group accumulators start at zero
    FFC_CUDA(cudaMemsetAsync(red, 0, sizeof(unsigned long long) * 12 * (size_t)W, cs));
    FFC_CUDA(cudaMemsetAsync(qst, 0, sizeof(int32_t) * W, cs));
    FFC_CUDA(cudaMemsetAsync(qrank, 0, sizeof(int32_t) * W, cs));
    FFC_CUDA(cudaMemsetAsync(qr22, 0, sizeof(double) * W, cs));
    ffc_status rc = record(0, cs, capturing);
    if (rc != FFC_OK) return rc;
    if (learned) {   // the node's best s_max rows were drawn once per call: take the first s_nom
      learned_round_kernel<<<(W + 127) / 128, 128, 0, cs>>>(W, oidx, s_nom, R->lcount, R->lfar, s_out, fc);
      FFC_CUDA(cudaGetLastError());
    } else {
      rc = launch_sample(X, R->dtype, d, d_si, W, R->N, s_nom, P.seed, s_out, fc, sst, scratch, cs);
      if (rc != FFC_OK) return rc;
    }
    if ((rc = record(1, cs, capturing)) != FFC_OK) return rc;
    patch_kernel<<<(W + 127) / 128, 128, 0, cs>>>(W, s_out, s_nom, r_cap_glob, d_ei, d_qi);
    if (nested) {   // the ID's column points of every item, packed (item q at rows noff[q] of the arena)
      gather_cols_kernel<<<dim3(8, (unsigned)W), 256, 0, cs>>>(d_gi, X, Xcols, d, pts_esz);
      FFC_CUDA(cudaGetLastError());
    }
    rc = launch_eval(P.kernel, X, R->dtype, nested ? Xcols : X, d, P.precision, eshape, d_ei, W, tiles_tot, mind2,
                     lsc, est, t5scr, t5rows, cs);
    if (rc != FFC_OK) return rc;
    if ((rc = record(2, cs, capturing)) != FFC_OK) return rc;
    // one cooperative QR launch per L2-sized sub-batch of the round
    for (int bb = 0; bb < n_sb; ++bb) {
      rc = launch_cpqr(P.precision, d_qi, d_as + sb_as[bb], sb_grid[bb], (int)s_nom, cs, d_coff + sb_coff[bb], big,
                       sb_nb[bb], sb_nb[bb] > 1 ? 0 : defer);
      if (rc != FFC_OK) return rc;
    }
    if ((rc = record(3, cs, capturing)) != FFC_OK) return rc;
    gate_kernel<<<(W + 127) / 128, 128, 0, cs>>>(W, s_nom, P.s_max, s_out, qst, qrank, trank);
    rc = launch_trsm_batched(P.precision, d_ti, W, ttot, rcap_round, cs, P.solve);
    if (rc != FFC_OK) return rc;
    if ((rc = record(4, cs, capturing)) != FFC_OK) return rc;
    epilogue_kernel<<<(W + 127) / 128, 128, 0, cs>>>(W, oidx, s_nom, P.s_max, s_out, fc, lsc, est, qrank, qr22, qst,
                                                     R->rank, R->s, R->status, R->r22, R->log_scale, R->far_count,
                                                     flags);
    FFC_CUDA(cudaGetLastError());
    return record(5, cs, capturing);
  };
  bool launched = false;
  if (P.graphs == 0) {
    // the key: every byte the launches depend on (the tables hold the items' device pointers)
    std::string key;
    auto put = [&key](const void* p, size_t n) { key.append(static_cast<const char*>(p), n); };
    const long long wl = wait_limit();
    const void* ptrs[] = {X, Xcols, R->ws, R->lcount, R->lfar, R->rank, R->s, R->status, R->r22, R->log_scale,
                          R->far_count};
    const int64_t sc[] = {W, s_nom, learned, nested, prof, eshape, tiles_tot, t5rows, n_sb, big, ttot, rcap_round,
                          r_cap_glob, G, d, R->dtype, R->N, (int64_t)R->ws_bytes, (int64_t)pts_esz, wl};
    put(ptrs, sizeof(ptrs));
    put(sc, sizeof(sc));
    put(&P, sizeof(P));
    put(sb_grid.data(), sizeof(int) * sb_grid.size());
    put(sb_as.data(), sizeof(int) * sb_as.size());
    put(sb_coff.data(), sizeof(int) * sb_coff.size());
    put(sb_nb.data(), sizeof(int) * sb_nb.size());
    put(hs.data(), sizeof(SampleItem) * W);
    put(he.data(), sizeof(EvalItem) * W);
    put(hq.data(), sizeof(CpqrItem) * W);
    put(ht.data(), sizeof(TrsmItem) * W);
    put(ha.data(), sizeof(CtaAssign) * ha.size());
    put(hoff.data(), sizeof(int32_t) * hoff.size());
    put(ho.data(), sizeof(int32_t) * W);
    put(hg.data(), sizeof(GatherItem) * hg.size());
    ffc_tree_result::RoundGraph* hit = nullptr;
    for (auto& g : R->graphs)
      if (g.key == key) { hit = &g; break; }
    if (!hit) {
      // capture on the result's private stream; any refusal leaves the round to the direct launches below
      if (!R->cap_stream) FFC_CUDA(cudaStreamCreateWithFlags(&R->cap_stream, cudaStreamNonBlocking));
      cudaGraphExec_t ex = nullptr;
      if (cudaStreamBeginCapture(R->cap_stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
        const ffc_status crc = enqueue(R->cap_stream, true);
        cudaGraph_t gr = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(R->cap_stream, &gr);
        if (crc == FFC_OK && ce == cudaSuccess && gr && cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) ex = nullptr;
        if (gr) cudaGraphDestroy(gr);
      }
      (void)cudaGetLastError();
      if (ex) {
        if (R->graphs.size() >= 16) {   // least recently used out
          auto lru = std::min_element(R->graphs.begin(), R->graphs.end(),
                                      [](const auto& x, const auto& y) { return x.used < y.used; });
          cudaGraphExecDestroy(lru->exec);
          R->graphs.erase(lru);
        }
        R->graphs.push_back({std::move(key), ex, 0});
        hit = &R->graphs.back();
        R->prof.graph_captures += 1;
      }
    }
    if (hit) {
      hit->used = ++R->graph_clock;
      FFC_CUDA(cudaGraphLaunch(hit->exec, st));
      R->prof.graph_launches += 1;
      launched = true;
    }
  }
  if (!launched) {
    const ffc_status rc = enqueue(st, false);
    if (rc != FFC_OK) return rc;
  }
  const int qr_launches = n_sb;
  std::vector<int32_t> hf(W), hr(prof ? W : 0);
  std::vector<int64_t> hsz(prof ? W : 0);
  FFC_CUDA(cudaMemcpyAsync(hf.data(), flags, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, st));
  if (prof) {
    FFC_CUDA(cudaMemcpyAsync(hr.data(), qrank, sizeof(int32_t) * W, cudaMemcpyDeviceToHost, st));
    FFC_CUDA(cudaMemcpyAsync(hsz.data(), s_out, sizeof(int64_t) * W, cudaMemcpyDeviceToHost, st));
  }
  FFC_CUDA(cudaStreamSynchronize(st));
  again.clear();
  for (int q = 0; q < W; ++q)
    if (hf[q]) again.push_back(items[q]);
  if (prof) {
    ffc_tree_profile& pf = R->prof;
    for (int ph = 0; ph < 5; ++ph) {
      float ms = 0.f;
      FFC_CUDA(cudaEventElapsedTime(&ms, R->ev[ph], R->ev[ph + 1]));
      pf.ms[ph] += ms;
      if (ph == 2) {
        const int rd = std::min(R->rounds, 7);
        pf.qr_ms_round[rd] += ms;
        pf.items_round[rd] += W;
      }
    }
    // Laplace: distances, scale and block; tcgen05: plane prep and block; else one block kernel
    const int eval_launches = P.kernel.kind == FFC_LAPLACE ? 4 : eshape >= 2 ? 2 : 1;
    pf.launches += 1 + 1 + (nested ? 1 : 0) + eval_launches + qr_launches + 1 + 2 + 1;
    pf.qr_launches += qr_launches;
    pf.rounds += 1;
    const double per_coord = P.kernel.kind == FFC_POLYNOMIAL ? 2.0 : 3.0;
    for (int q = 0; q < W; ++q) {
      const double s = (double)hsz[q], n = (double)R->ncols_h[items[q]];
      double fl = 0.0;
      for (int k = 0; k < hr[q]; ++k) fl += 4.0 * (s - k) * (n - k);
      pf.qr_flops += fl;
      pf.eval_flops += per_coord * s * n * d;
      pf.qr_bytes += 2.0 * s * n * (double)esz;
    }
  }
  return FFC_OK;
}

}  // namespace

namespace ffc {
// The parameters the result was computed with, and the heap id of its first compressed node.
const ffc_params* tree_result_params(const ffc_tree_result* r) { return &r->p; }
int64_t tree_result_first_node(const ffc_tree_result* r) { return r->node_h.empty() ? 0 : r->node_h[0]; }
}  // namespace ffc

extern "C" {

ffc_status ffc_compress_tree(const void* points_perm_dev, int32_t dtype, int64_t N, int32_t d, const ffc_tree* tree,
                             const ffc_params* params, ffc_tree_result** result, void* stream) {
  FFC_REQUIRE(tree && params && result, "ffc_compress_tree: null argument");
  FFC_REQUIRE(N >= 1 && d >= 1 && N <= 1500000, "ffc_compress_tree: need 1 <= N <= 1,500,000 and d >= 1");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_compress_tree: bad dtype");
  FFC_REQUIRE(points_perm_dev && tree->begin_dev && tree->count_dev && tree->centroid_dev && tree->radius_dev,
              "ffc_compress_tree: null pointer");
  const ffc_params& P = *params;
  FFC_REQUIRE(P.precision == FFC_FP64 || P.precision == FFC_MIXED, "ffc_compress_tree: bad precision");
  FFC_REQUIRE(P.s0 >= 2 && P.s_max >= P.s0 && P.s_max <= 2048, "ffc_compress_tree: need 2 <= s0 <= s_max <= 2048");
  FFC_REQUIRE(P.qr_panel >= 0 && P.qr_panel <= QR_PANEL_MAX, "ffc_compress_tree: qr_panel must be in [0, %d]",
              QR_PANEL_MAX);
  FFC_REQUIRE(P.eval_path >= FFC_EVAL_DEFAULT && P.eval_path <= FFC_EVAL_LAST, "ffc_compress_tree: bad eval_path");
  FFC_REQUIRE(P.graphs == 0 || P.graphs == 1, "ffc_compress_tree: graphs must be 0 or 1");
  FFC_REQUIRE(P.qr_defer >= 0 && P.qr_defer <= 4, "ffc_compress_tree: qr_defer must be in [0, 4]");
  FFC_REQUIRE(P.solve == FFC_SOLVE_DEFAULT || P.solve == FFC_SOLVE_FP64, "ffc_compress_tree: bad solve");
  FFC_REQUIRE(P.tol > 0.0 && P.xi > 0.0, "ffc_compress_tree: need tol > 0 and xi > 0");
  FFC_REQUIRE(tree->depth >= 0 && tree->n_nodes == ((int64_t)1 << (tree->depth + 1)) - 1,
              "ffc_compress_tree: n_nodes must be 2^(depth+1) - 1");
  FFC_REQUIRE(P.min_level >= 0 && P.min_level <= tree->depth, "ffc_compress_tree: min_level out of range");
  if (!kernel_ok(P.kernel, d)) return FFC_E_INVALID;
  FFC_REQUIRE(P.sampler >= FFC_SAMPLE_UNIFORM && P.sampler <= FFC_SAMPLE_NEAREST, "ffc_compress_tree: bad sampler");
  if (P.sampler == FFC_SAMPLE_LEARNED) {
    FFC_REQUIRE(P.pool_rows == 0 || P.pool_rows >= P.s_max,
                "ffc_compress_tree: pool_rows must be 0 (whole far field) or >= s_max");
    FFC_REQUIRE(P.proj_dev && P.mlp_dev, "ffc_compress_tree: the learned sampler needs proj_dev and mlp_dev");
  }
  cudaStream_t st = as_stream(stream);

  ffc_tree_result* R = *result;
  const bool fresh = (R == nullptr);
  if (!fresh) {
    FFC_REQUIRE(R->N == N && R->d == d && R->dtype == dtype && R->n_tree_nodes == tree->n_nodes &&
                    R->p.min_level == P.min_level && R->p.s_max == P.s_max,
                "ffc_compress_tree: result was created for a different tree shape or params");
    R->p = P;
  } else {
    R = new ffc_tree_result();
    R->N = N; R->d = d; R->dtype = dtype; R->n_tree_nodes = tree->n_nodes; R->p = P;
    std::vector<int64_t> b(tree->n_nodes), c(tree->n_nodes);
    node_layout(N, tree->depth, b.data(), c.data(), nullptr);
    const int64_t first = ((int64_t)1 << P.min_level) - 1;
    const int64_t rcap = P.s_max / 2;
    R->rows_off_h.push_back(0);
    R->skel_off_h.push_back(0);
    R->T_off_h.push_back(0);
    for (int64_t i = first; i < tree->n_nodes; ++i) {
      R->node_h.push_back((int32_t)i);
      R->begin_h.push_back(b[i]);
      R->count_h.push_back(c[i]);
      R->rows_off_h.push_back(R->rows_off_h.back() + P.s_max);
      R->skel_off_h.push_back(R->skel_off_h.back() + c[i]);
      R->T_off_h.push_back(R->T_off_h.back() + std::min<int64_t>(c[i], rcap) * c[i]);
    }
    R->n_out = (int64_t)R->node_h.size();
    ffc_status rc = alloc_outputs(R);
    if (rc != FFC_OK) { ffc_tree_result_free(R); return rc; }
    *result = R;
  }
  std::vector<int> active(R->n_out), again;
  for (int64_t i = 0; i < R->n_out; ++i) active[i] = (int)i;
  int64_t s_nom = P.s0;
  R->rounds = 0;
  if (R->prof.enabled) R->prof.calls += 1;
  if (P.sampler != FFC_SAMPLE_UNIFORM) {
    const bool prof = R->prof.enabled != 0;
    if (prof) FFC_CUDA(cudaEventRecord(R->ev[0], st));
    ffc_status rc = propose_tree(R, points_perm_dev, tree, st);
    if (rc != FFC_OK) return rc;
    if (prof) {
      FFC_CUDA(cudaEventRecord(R->ev[1], st));
      FFC_CUDA(cudaEventSynchronize(R->ev[1]));
      float ms = 0.f;
      FFC_CUDA(cudaEventElapsedTime(&ms, R->ev[0], R->ev[1]));
      R->prof.ms[0] += ms;
    }
  }
  auto rounds_of = [&](std::vector<int> act) -> ffc_status {
    int64_t sn = P.s0;
    while (!act.empty()) {
      ffc_status rc = run_round(R, points_perm_dev, tree, act, sn, again, st);
      if (rc != FFC_OK) return rc;
      ++R->rounds;
      act.swap(again);
      sn *= 2;
    }
    return FFC_OK;
  };
  if (!P.nested) {
    if (R->cols_custom) {
      ffc_status rc = reset_columns(R, st);
      if (rc != FFC_OK) return rc;
    }
    ffc_status rc = rounds_of(active);
    if (rc != FFC_OK) return rc;
  } else {
    // the upward pass: each level after the one below it, with its children's skeletons as columns
    const int64_t first = R->node_h.empty() ? 0 : R->node_h[0];
    for (int L = tree->depth; L >= P.min_level; --L) {
      std::vector<int> lv;
      for (int64_t o = ((int64_t)1 << L) - 1 - first; o < ((int64_t)1 << (L + 1)) - 1 - first; ++o) lv.push_back((int)o);
      ffc_status rc = L == tree->depth ? reset_columns(R, st) : nested_columns(R, lv, first, st);
      if (rc != FFC_OK) return rc;
      R->cols_custom = true;
      rc = rounds_of(lv);
      if (rc != FFC_OK) return rc;
    }
  }
  (void)s_nom;
  pack_offsets_kernel<<<1, 1024, 0, st>>>(R->n_out, R->rank, R->ncols64, R->Tp_off);
  pack_copy_kernel<<<dim3(8, (unsigned)R->n_out), 256, 0, st>>>(R->n_out, R->T_off, R->Tp_off, R->T, R->Tp);
  FFC_CUDA(cudaGetLastError());
  if (R->prof.enabled) R->prof.launches += 2;
  return FFC_OK;
}

ffc_status ffc_tree_result_view(const ffc_tree_result* R, ffc_tree_view* v) {
  FFC_REQUIRE(R && v, "ffc_tree_result_view: null argument");
  v->n_out = R->n_out; v->rounds = R->rounds;
  v->node_dev = R->node; v->rank_dev = R->rank; v->s_dev = R->s; v->status_dev = R->status;
  v->r22_rel_dev = R->r22; v->log_scale_dev = R->log_scale; v->far_count_dev = R->far_count;
  v->rows_off_dev = R->rows_off; v->rows_dev = R->rows; v->skel_off_dev = R->skel_off; v->skel_dev = R->skel;
  v->T_off_dev = R->Tp_off; v->T_dev = R->Tp;
  v->ncols_dev = R->ncols; v->cols_dev = R->cols;
  return FFC_OK;
}

void ffc_tree_result_free(ffc_tree_result* R) {
  if (!R) return;
  for (auto& g : R->graphs) cudaGraphExecDestroy(g.exec);
  if (R->cap_stream) cudaStreamDestroy(R->cap_stream);
  if (R->out_mem) cudaFree(R->out_mem);
  if (R->ws) cudaFree(R->ws);
  if (R->pws) cudaFree(R->pws);
  if (R->pst) cudaFree(R->pst);
  if (R->lcount) cudaFree(R->lcount);
  for (auto& e : R->ev)
    if (e) cudaEventDestroy(e);
  delete R;
}

ffc_status ffc_tree_profile_enable(ffc_tree_result* R, int32_t enabled) {
  FFC_REQUIRE(R, "ffc_tree_profile_enable: null result");
  if (enabled && !R->ev[0])
    for (auto& e : R->ev) FFC_CUDA(cudaEventCreate(&e));
  R->prof.enabled = enabled ? 1 : 0;
  return FFC_OK;
}

ffc_status ffc_tree_profile_reset(ffc_tree_result* R) {
  FFC_REQUIRE(R, "ffc_tree_profile_reset: null result");
  const int32_t en = R->prof.enabled;
  R->prof = ffc_tree_profile{};
  R->prof.enabled = en;
  return FFC_OK;
}

ffc_status ffc_tree_profile_get(const ffc_tree_result* R, ffc_tree_profile* out) {
  FFC_REQUIRE(R && out, "ffc_tree_profile_get: null argument");
  *out = R->prof;
  return FFC_OK;
}

}  // extern "C"
