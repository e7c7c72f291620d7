// Internal declarations shared by libffc's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ffc.h"

namespace ffc {

// ----------------------------------------------------------------------------
// error state (thread-local message, see ffc_last_error)
void set_error(const char* fmt, ...);
ffc_status cuda_fail(cudaError_t e, const char* what);

#define FFC_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return ::ffc::cuda_fail(e_, #call);           \
  } while (0)

#define FFC_REQUIRE(cond, ...)                                           \
  do {                                                                   \
    if (!(cond)) {                                                       \
      ::ffc::set_error(__VA_ARGS__);                                     \
      return FFC_E_INVALID;                                              \
    }                                                                    \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ----------------------------------------------------------------------------
// device helpers

// Philox4x64-10 (Salmon et al., SC'11): counter (c0..c3), key (k0, k1).
struct u64x4 { uint64_t x[4]; };

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += W0; k1 += W1;
  }
  u64x4 o; o.x[0] = c0; o.x[1] = c1; o.x[2] = c2; o.x[3] = c3;
  return o;
}

// Draw t of stream (seed, stream_id, domain): word t%4 of block t/4.
__device__ __forceinline__ uint64_t philox_draw(uint64_t seed, uint64_t stream_id, uint64_t domain,
                                                uint64_t t) {
  u64x4 b = philox4x64_10(t >> 2, stream_id, domain, 0, seed, 0);
  uint32_t w = (uint32_t)(t & 3);
  return w == 0 ? b.x[0] : (w == 1 ? b.x[1] : (w == 2 ? b.x[2] : b.x[3]));
}

constexpr uint64_t DOMAIN_UNIFORM_ROWS = 0;
constexpr uint64_t DOMAIN_WEIGHTED_POOL = 1;
constexpr uint64_t DOMAIN_WEIGHTED_KEYS = 2;
constexpr int ATTEMPT_FACTOR = 64;
constexpr int SAMPLE_MAX_GRID = 2048;   // sampler CTAs; one scratch slice of M_max each

template <typename TP>
__device__ __forceinline__ double ld_point(const TP* p) { return (double)__ldg(p); }

// Bounded spin limit for waits on other CTAs (about a second or more); ffc_set_wait_limit
// changes it for later launches, wait_limit() reads the current value on the host.
constexpr long long SPIN_LIMIT_DEFAULT = 20000000ll;
long long wait_limit();

// ----------------------------------------------------------------------------
// work items (host-built tables, copied to the device)

struct SampleItem {
  int64_t M;            // candidates (rows of Y)
  int64_t ex_begin, ex_end;
  const double* x_c;    // NULL: no distance test
  double thr2;          // (xi * radius)^2, used when radius == NULL
  const double* radius; // device radius (tree nodes) or NULL
  double xi;
  int64_t s;            // requested rows
  uint64_t stream_id;
  int64_t* rows;        // capacity s
};

struct EvalItem {
  const int64_t* rows;  // s indices into Y
  int64_t s;
  int64_t x_begin;      // first source row in X
  int64_t n;
  void* K;              // column-major s x n
  int64_t ldk;
  const double* center; // d doubles or NULL
  int64_t tile_begin;   // prefix of tiles over items
  int64_t row_tiles;    // row tiles of the nominal s (tiles past the actual s are skipped)
  // tcgen05 path only: the item's first row of the plane arena's norm index (a prefix over items of
  // tc_spad + tc_npad; its planes start at row 3 tc_base) and its padded target / source counts
  int64_t tc_base;
  int64_t tc_spad, tc_npad;
};

struct CpqrItem {
  void* A;              // s x n column-major, ld lda (double or float)
  int64_t lda;
  int32_t s, n;
  int32_t r_max;        // step cap
  int32_t pad0;
  double tol;           // <= 0: fixed rank
  int32_t* piv;         // r_max
  double* beta;         // r_max
  double* vn1;          // n  current residual norms
  double* vn2;          // n  reference norms (downdating safeguard)
  uint8_t* selected;    // n
  void* slots;          // g step-0 slots (16 B each)
  unsigned long long* red;  // 12 words: the group reduction of steps >= 1, zeroed before the launch
  unsigned int* barrier;
  int32_t* rank_out;
  double* r22_out;      // ||R22||_F / ||K'||_F
  int32_t* status_out;
  void* F;              // blocked form: n x 32 (T) panel coefficients, or NULL for the unblocked form
};

struct CtaAssign { int32_t item, rank, g, pad; };

struct Slot { double best; double sum; int32_t col; int32_t pad; };

struct TrsmItem {
  const void* A; int64_t lda;
  int32_t n, pad0;
  const int32_t* rank;  // device scalar
  const int32_t* piv;
  const double* beta;
  const uint8_t* selected;
  int32_t* skel_perm;   // n
  double* R11;          // r_cap x r_cap workspace (row-major, ld r)
  float* R11f;          // FP32 copy, column-major, ld = r rounded up to 4, (r_cap rounded up to 4)^2 floats,
                        // 16-byte aligned (mixed precision's refined solve; NULL otherwise)
  double* T;            // output
  int64_t ldt;          // <= 0: ld = rank (packed)
  int32_t r_cap, pad1;
  int64_t tile_begin;   // prefix of 8-column tiles over items
};

struct FeatItem {
  const int64_t* rows;   // candidate indices into Y
  const int64_t* count;  // device count of valid rows, or NULL: all cap rows are valid
  int64_t cap;           // output rows reserved for the item
  int64_t out_begin;     // first output row (flat over items)
  const double* x_c;     // node centroid (d)
  const double* radius;  // device radius or NULL
  double radius_host;    // used when radius == NULL
};

struct FarItem {
  int64_t M;             // candidates [0, M)
  int64_t ex_begin, ex_end;
  const double* x_c;     // d doubles
  const double* radius;  // device radius or NULL
  double radius_host;
  double xi;
  int64_t* list;         // capacity M: far candidates, ascending
  int64_t* count;        // device: |list|
};

struct SelectItem {
  const int64_t* pool;   // candidate rows
  const int64_t* count;  // device pool size, or NULL: P
  int64_t P;
  const float* logits;   // network output per pool row
  int64_t s;             // rows wanted
  uint64_t stream_id;
  int64_t* rows_out;     // capacity s
  int64_t* s_out;        // device: rows written (may be NULL)
  uint64_t* keys;        // capacity P: w_i, then the FP32 pre-selection keys (pools above 16,384 rows), or NULL
  const uint64_t* given; // or: ascending sort keys per pool position, computed elsewhere (logits unused)
};

// A candidate pool whose sort keys the paper's samplers compute (csrc/samplers.cu).
struct KeyItem {
  const int64_t* pool;   // candidate rows
  const int64_t* count;  // device pool size, or NULL: cap
  int64_t cap;
  const double* x_c;     // distance samplers: the node centre (d doubles)
  int64_t src_begin;     // nearest neighbours: the node's sources are rows [src_begin, src_begin + src_n) of X
  int64_t src_n;
  uint64_t stream_id;
  uint64_t* keys;        // capacity cap: ascending sort keys
};

// ----------------------------------------------------------------------------
// far-field membership (FP64, the uniform sampler's test) and the proposal's
// feature transform, shared by the per-node and the tiled tree kernels

template <typename TP>
__device__ __forceinline__ bool far_member(const TP* __restrict__ Y, int d, int64_t j, const FarItem& it,
                                           double thr2) {
  if (j >= it.M || (j >= it.ex_begin && j < it.ex_end)) return false;
  const TP* y = Y + j * (int64_t)d;
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    const double df = ld_point(y + k) - __ldg(it.x_c + k);
    acc = fma(df, df, acc);
  }
  return acc >= thr2;
}

__device__ __forceinline__ double far_thr2(const FarItem& it) {
  const double thr = it.xi * (it.radius ? *it.radius : it.radius_host);
  return thr * thr;
}

// FP32 sums of one (target row, node) pair and the 12 features made from them
constexpr int FEAT_NF = 12;
struct FeatSums { float dd, yy, yx, xx, p[8]; };

__device__ __forceinline__ void feature_values(const FeatSums& S, float rho, ffc_kernel k, int d, float out[FEAT_NF]) {
  const float r = sqrtf(S.dd);
  const float inv_rho = 1.0f / rho;
  out[0] = r * inv_rho;
  float kc;
  if (k.kind == FFC_GAUSSIAN) {
    kc = expf(-S.dd / (2.0f * (float)(k.h * k.h)));
  } else if (k.kind == FFC_LAPLACE) {
    kc = exp2f((float)(d - 2) * log2f(rho / r));
  } else {
    const float num = S.yx / (float)k.h + (float)k.c;
    const float den = sqrtf(S.yy) * sqrtf(S.xx) / (float)k.h + (float)k.c;
    kc = powf(num / den, (float)k.p);
  }
  out[1] = kc;
  out[2] = sqrtf(S.yy) * inv_rho;
  out[3] = rho / (k.kind == FFC_LAPLACE ? 1.0f : (float)k.h);
#pragma unroll
  for (int q = 0; q < 8; ++q) out[4 + q] = S.p[q] * inv_rho;
}

// ----------------------------------------------------------------------------
// launchers (implemented in the .cu files; all enqueue on `st`)

ffc_status launch_far_field(const void* Y, int dtype, int64_t M, int d, const double* x_c, double thr2,
                            int64_t ex_begin, int64_t ex_end, int64_t* idx, int64_t* count_dev,
                            cudaStream_t st);
ffc_status launch_sample(const void* Y, int dtype, int d, const SampleItem* items_dev, int n_items,
                         int64_t M_max, int64_t s_max, uint64_t seed, int64_t* s_out, int64_t* far_count,
                         int32_t* status, int32_t* scratch, cudaStream_t st);
// Tile decomposition of the evaluation: shape = eval_shape(k, d, precision, path) (0 SIMT, 1 mma.sync
// tensor cores, 2 + v tcgen05 with tile variant v); items' tile_begin and row_tiles must come from
// eval_tiles / eval_row_tiles of that shape. path: an FFC_EVAL_* request (FFC_EVAL_DEFAULT: the library default, which
// eval_default_path() may override).
int eval_shape(ffc_kernel k, int d, int precision, int path);
constexpr int FFC_EVAL_TCGEN05_DEFAULT_TILE = 0;   // the tcgen05 tile variant FFC_EVAL_TCGEN05 stands for
constexpr int FFC_EVAL_LAST = FFC_EVAL_TCGEN05_TILE0 + FFC_EVAL_TCGEN05_TILES - 1;
int eval_default_path();
void set_eval_default_path(int path);
int64_t eval_tiles(int64_t s, int64_t n, int shape);
int64_t eval_row_tiles(int64_t s, int shape);
int64_t eval_tc_tiles(int64_t s, int64_t n);
int64_t eval_tc_row_tiles(int64_t s);
ffc_status launch_eval_tc(ffc_kernel k, const void* Y, int dtype, const void* X, int d, const EvalItem* items_dev,
                          int n_items, int64_t total_tiles, double* log_scale, cudaStream_t st);
// tcgen05 shape: items carry tc_base / tc_spad / tc_npad (tc_spad = eval_tc5_pad_s(nominal s),
// tc_npad = eval_tc5_pad_n(n)); the scratch holds eval_tc5_scratch_bytes(sum of tc_spad + tc_npad, d)
// bytes, 256-byte aligned.
int64_t eval_tc5_pad_s(int64_t s);
int64_t eval_tc5_pad_n(int64_t n);
int eval_tc5_dpad(int d);
int64_t eval_tc5_tiles(int64_t s, int64_t n, int v);
int64_t eval_tc5_row_tiles(int64_t s);
size_t eval_tc5_scratch_bytes(int64_t total_rows, int d);
ffc_status launch_eval_tc5(ffc_kernel k, const void* Y, int dtype, const void* X, int d, int v,
                           const EvalItem* items_dev, int n_items, int64_t total_tiles, int64_t total_rows,
                           void* scratch, double* log_scale, int32_t* status, cudaStream_t st);
ffc_status launch_eval(ffc_kernel k, const void* Y, int dtype, const void* X, int d, int precision, int shape,
                       const EvalItem* items_dev, int n_items, int64_t total_tiles,
                       double* min_d2 /* n_items, Laplace */, double* log_scale /* n_items */,
                       int32_t* status /* n_items */, void* tc5_scratch, int64_t tc5_rows, cudaStream_t st);
// entries: per-CTA work lists (CTA b runs entries[cta_off[b] .. cta_off[b+1]) in order), or with
// cta_off == NULL one entry per CTA.
// big: the register-resident variant (mixed precision only; -1 = the default rule s_max >= 1024)
// nb: panel width of the blocked form (items with F set; 1 = every item unblocked); qr_panel() gives the
// library's default for a round of s_max rows
// defer: >= 2 runs the lazy form (write-back every `defer` steps, at most 4) where cpqr_lazy() allows it;
// the same results as 0 or 1 up to FP32 summation order (and the same for every depth >= 2)
ffc_status launch_cpqr(int precision, const CpqrItem* items_dev, const CtaAssign* assign_dev, int grid,
                       int s_max, cudaStream_t st, const int32_t* cta_off = nullptr, int big = -1, int nb = 1,
                       int defer = 0);
int cpqr_max_ctas(int precision, int s_max, int big = -1, int nb = 1, int defer = 0);
bool cpqr_lazy(int precision, int s_max, int big, int nb, int defer);
constexpr int QR_DEFER_DEFAULT = 1;   // deferral depth of the lazy form when ffc_params.qr_defer is 0
int qr_panel(int precision, int s_max, int big, bool blocked = false);
constexpr int QR_F_STRIDE = 32;   // elements per column of the blocked form's F
constexpr int QR_PANEL_MAX = 8;   // widest panel of the blocked form
constexpr int QR_FS_COLS = 128;   // most columns one CTA of the blocked form may own (their F rows are on chip)
constexpr int QR_BIG_MIN_S_DEFAULT = 1024;
constexpr int QR_L2_BUDGET_MB_DEFAULT = 96;
int cpqr_min_group(int64_t n);   // fewest CTAs a group of n columns may have (per-CTA column cap)
int64_t trsm_tiles(int64_t n);   // CTAs of the triangular solve for n columns
// solve: FFC_SOLVE_DEFAULT (mixed precision: FP32 solves refined once) or FFC_SOLVE_FP64
ffc_status launch_trsm_batched(int precision, const TrsmItem* items_dev, int n_items, int64_t total_tiles,
                               int r_cap_max, cudaStream_t st, int solve = FFC_SOLVE_DEFAULT);
ffc_status launch_id_error(ffc_kernel k, const void* Y, int dtype, const int64_t* rows, int64_t m,
                           const void* X, int64_t n, int d, const int32_t* skel, const double* T,
                           int64_t ldt, int64_t r, double* partial /* workspace */, int64_t n_partial,
                           double* min_d2_dev, double* out_host_num, double* out_host_den, cudaStream_t st);
ffc_status launch_build_tree(const void* points, int dtype, int64_t N, int d, int depth, int64_t* perm,
                             const int64_t* begin_host, const int64_t* count_host, const int64_t* begin_dev,
                             const int64_t* count_dev, double* centroid, double* radius, cudaStream_t st);

// cap_max: largest item cap (rows reserved per item)
ffc_status launch_features(ffc_kernel k, const void* Y, int dtype, int d, const FeatItem* items_dev, int n_items,
                           int64_t cap_max, const double* proj, float* out, cudaStream_t st);
ffc_status launch_mlp_forward(const float* params, const float* feats, int64_t R, float* logits, cudaStream_t st);
// keep_max: largest min(s, P) over the items (<= 8192); any pool size P
ffc_status launch_select(const SelectItem* items_dev, int n_items, int64_t keep_max, uint64_t seed, cudaStream_t st);
// Tiled far-field lists and features of n_items nodes over all N points (candidates [0, N)):
// yy, yg from launch_point_stats (N and N x 8 floats); node_ws: far_tiles_node_bytes(n_items, d);
// tile_cnt: n_items x far_tiles_count(N) int64; mask: n_items x 4 far_tiles_count(N) words.
// Writes each item's ascending list, *count and the features of its rows [0, count); rows
// [count, cap) of the features are zeroed.
int64_t far_tiles_count(int64_t N);
size_t far_tiles_node_bytes(int n_items, int d);
ffc_status launch_point_stats(const void* Y, int dtype, int64_t N, int d, const double* proj, float* yy, float* yg,
                              cudaStream_t st);
ffc_status launch_far_features_tiled(ffc_kernel k, const void* Y, int dtype, int64_t N, int d,
                                     const FarItem* items_dev, const FeatItem* fitems_dev, int n_items,
                                     const double* proj, const float* yy, const float* yg, void* node_ws,
                                     int64_t* tile_cnt, uint32_t* mask, float* feats, cudaStream_t st);
// Sort keys of the paper's samplers (FFC_DRAW_*) for n_items pools; cap_max: largest pool.
ffc_status launch_paper_keys(int sampler, const void* Y, const void* X, int dtype, int d, const KeyItem* items_dev,
                             int n_items, int64_t cap_max, uint64_t seed, cudaStream_t st);
ffc_status launch_mlp_loss_grad(const float* params, const float* feats, const double* targets,
                                const int64_t* node_off_dev, int n_nodes, int64_t R, float* logits, float* g_o,
                                double* loss_part, float* part, int n_part, float* grad, cudaStream_t st);
int mlp_backward_grid(int64_t R);
ffc_status launch_adam(float* theta, const float* g, float* m, float* v, int64_t n, int64_t step, double lr,
                       double b1, double b2, double eps, cudaStream_t st);
ffc_status launch_leverage_batched(int B, const double* const* K, const int64_t* m, const int64_t* n,
                                   const int64_t* ldk, double eps, int64_t r_fixed, double* const* lev,
                                   double* const* sigma, int64_t* rank_host, int32_t* sweeps_host, cudaStream_t st);

// host helpers
int sm_count();
bool kernel_ok(const ffc_kernel& k, int d);   // sets the error message when false
void node_layout(int64_t N, int depth, int64_t* begin, int64_t* count, int32_t* level);

}  // namespace ffc
