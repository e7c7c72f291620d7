// C ABI of libffc (declarations and contracts in include/ffc.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "ffc_internal.cuh"

namespace ffc {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

ffc_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FFC_E_NOMEM : FFC_E_CUDA;
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
  return cache[dev];
}

// defined in the kernel translation units
int64_t id_error_blocks(int64_t m, int64_t n, int64_t r);
int cpqr_rows_per_lane(int s_max);
size_t sample_smem_bytes(int64_t M_max, int d);

constexpr int64_t MAX_CANDIDATES = 1500000;
constexpr int MAX_ROWS = 2048;     // rows of a block held by the QR (32 lanes x 64 registers)
constexpr int MAX_RANK = 1024;     // triangular-solve register tile

// Stream-ordered scratch arena: one cudaMallocAsync per call, carved up.
struct Arena {
  char* base = nullptr;
  size_t used = 0, cap = 0;
  cudaStream_t st = nullptr;
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
};

static size_t round_up(size_t x) { return (x + 255) & ~size_t(255); }

bool kernel_ok(const ffc_kernel& k, int d) {
  if (k.kind == FFC_GAUSSIAN) {
    if (!(k.h > 0.0)) { set_error("Gaussian bandwidth h must be > 0"); return false; }
  } else if (k.kind == FFC_LAPLACE) {
    if (d == 2) { set_error("the d = 2 (logarithmic) Laplace kernel is not supported"); return false; }
  } else if (k.kind == FFC_POLYNOMIAL) {
    if (k.h == 0.0 || k.p < 1) { set_error("polynomial kernel needs h != 0 and p >= 1"); return false; }
  } else {
    set_error("unknown kernel kind %d", k.kind);
    return false;
  }
  return true;
}

// Group size per item for the cooperative QR launch.
static int group_size(int64_t s, int64_t n, int64_t elems_per_cta) {
  int64_t g = (s * n + elems_per_cta - 1) / std::max<int64_t>(elems_per_cta, 1);
  g = std::min<int64_t>(g, std::max<int64_t>(1, n / 4));
  return (int)std::max<int64_t>(1, g);
}

static std::atomic<long long> g_wait_limit{SPIN_LIMIT_DEFAULT};

long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

}  // namespace ffc

using namespace ffc;

extern "C" {

const char* ffc_last_error(void) { return g_err; }

ffc_status ffc_set_wait_limit(int64_t polls) {
  g_wait_limit.store(polls < 0 ? SPIN_LIMIT_DEFAULT : (long long)polls, std::memory_order_relaxed);
  return FFC_OK;
}

namespace {
// The current device's default memory pool keeps what stream-ordered frees return instead of handing it
// back to the system at each synchronisation, so large per-call scratch (the tcgen05 evaluation's
// plane arena) is reused rather than mapped again on every call. Process-local; set once per device.
void retain_pool_memory() {
  static std::once_flag once[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { (void)cudaGetLastError(); return; }
  std::call_once(once[dev], [dev] {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) (void)cudaGetLastError();
    } else {
      (void)cudaGetLastError();
    }
  });
}
}  // namespace

ffc_status ffc_set_eval_path(int32_t path) {
  FFC_REQUIRE(path >= FFC_EVAL_DEFAULT && path <= FFC_EVAL_LAST, "ffc_set_eval_path: unknown path %d", (int)path);
  set_eval_default_path(path);
  return FFC_OK;
}

const char* ffc_version(void) { return "ffc 0.1 (sm_103a)"; }

ffc_status ffc_far_field(const void* Y_dev, int32_t dtype, int64_t M, int32_t d, const double* x_c_dev,
                         double radius, double xi, int64_t ex_begin, int64_t ex_end, int64_t* idx_dev,
                         int64_t* count_host, void* stream) {
  FFC_REQUIRE(M >= 0 && d >= 1, "ffc_far_field: need M >= 0, d >= 1");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_far_field: dtype must be FFC_F64 or FFC_F32");
  FFC_REQUIRE(M == 0 || (Y_dev && idx_dev), "ffc_far_field: null pointer");
  FFC_REQUIRE(count_host, "ffc_far_field: count_host is null");
  cudaStream_t st = as_stream(stream);
  int64_t* cnt = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int64_t), st));
  const double thr = xi * radius;
  ffc_status rc = launch_far_field(Y_dev, dtype, M, d, x_c_dev, thr * thr, ex_begin, ex_end, idx_dev, cnt, st);
  if (rc != FFC_OK) return rc;
  FFC_CUDA(cudaMemcpyAsync(count_host, cnt, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(cnt, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  return FFC_OK;
}

ffc_status ffc_sample_rows(const void* Y_dev, int32_t dtype, int64_t M, int32_t d, const double* x_c_dev,
                           double radius, double xi, int64_t ex_begin, int64_t ex_end, int64_t s, uint64_t seed,
                           uint64_t stream_id, int64_t* rows_dev, int64_t* s_out_host, int64_t* far_count_host,
                           void* stream) {
  FFC_REQUIRE(M >= 0 && M <= MAX_CANDIDATES, "ffc_sample_rows: need 0 <= M <= %lld", (long long)MAX_CANDIDATES);
  FFC_REQUIRE(d >= 1 && s >= 0, "ffc_sample_rows: need d >= 1, s >= 0");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_sample_rows: bad dtype");
  FFC_REQUIRE(s_out_host, "ffc_sample_rows: s_out_host is null");
  FFC_REQUIRE(s == 0 || M == 0 || (Y_dev && rows_dev), "ffc_sample_rows: null pointer");
  cudaStream_t st = as_stream(stream);
  if (s == 0 || M == 0) {
    *s_out_host = 0;
    if (far_count_host) *far_count_host = 0;
    return s == 0 ? FFC_OK : FFC_E_FARFIELD_TOO_SMALL;
  }
  Arena ar;
  size_t bytes = round_up(sizeof(SampleItem)) + 3 * 256 + round_up((size_t)M * sizeof(int32_t)) + 256;
  FFC_CUDA(cudaMallocAsync((void**)&ar.base, bytes, st));
  SampleItem* item = ar.take<SampleItem>(1);
  int64_t* s_out = ar.take<int64_t>(1);
  int64_t* fc = ar.take<int64_t>(1);
  int32_t* status = ar.take<int32_t>(1);
  int32_t* scratch = ar.take<int32_t>((size_t)M);
  SampleItem h;
  h.M = M; h.ex_begin = ex_begin; h.ex_end = ex_end; h.x_c = x_c_dev;
  const double thr = xi * radius;
  h.thr2 = thr * thr; h.radius = nullptr; h.xi = xi;
  h.s = s; h.stream_id = stream_id; h.rows = rows_dev;
  FFC_CUDA(cudaMemcpyAsync(item, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  ffc_status rc = launch_sample(Y_dev, dtype, d, item, 1, M, s, seed, s_out, fc, status, scratch, st);
  if (rc != FFC_OK) return rc;
  int64_t hs[2];
  int32_t hst = 0;
  FFC_CUDA(cudaMemcpyAsync(&hs[0], s_out, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&hs[1], fc, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&hst, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  *s_out_host = hs[0];
  if (far_count_host) {
    if (hs[1] >= 0) {
      *far_count_host = hs[1];
    } else {
      int64_t* idx = nullptr;
      FFC_CUDA(cudaMallocAsync((void**)&idx, (size_t)M * sizeof(int64_t), st));
      rc = ffc_far_field(Y_dev, dtype, M, d, x_c_dev, radius, xi, ex_begin, ex_end, idx, far_count_host, stream);
      cudaFreeAsync(idx, st);
      if (rc != FFC_OK) return rc;
    }
  }
  FFC_CUDA(cudaFreeAsync(ar.base, st));
  return (ffc_status)hst;
}

ffc_status ffc_eval_block(ffc_kernel kernel, const void* Y_dev, int32_t dtype, const int64_t* rows_dev, int64_t s,
                          const void* X_dev, int64_t n, int32_t d, const double* center_dev, int32_t precision,
                          void* K_dev, int64_t ldk, double* log_scale_host, void* stream) {
  FFC_REQUIRE(s >= 0 && n >= 0 && d >= 1, "ffc_eval_block: need s, n >= 0 and d >= 1");
  FFC_REQUIRE(ldk >= std::max<int64_t>(s, 1), "ffc_eval_block: ldk must be >= s");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_eval_block: bad dtype");
  FFC_REQUIRE(precision == FFC_FP64 || precision == FFC_MIXED, "ffc_eval_block: bad precision");
  if (!kernel_ok(kernel, d)) return FFC_E_INVALID;
  FFC_REQUIRE(s == 0 || n == 0 || (Y_dev && rows_dev && X_dev && K_dev), "ffc_eval_block: null pointer");
  (void)center_dev;
  if (log_scale_host) *log_scale_host = 0.0;
  if (s == 0 || n == 0) return FFC_OK;
  cudaStream_t st = as_stream(stream);
  Arena ar;
  FFC_CUDA(cudaMallocAsync((void**)&ar.base, 4096, st));
  EvalItem* item = ar.take<EvalItem>(1);
  double* mind2 = ar.take<double>(1);
  double* lsc = ar.take<double>(1);
  int32_t* status = ar.take<int32_t>(1);
  EvalItem h;
  h.rows = rows_dev; h.s = s; h.x_begin = 0; h.n = n; h.K = K_dev; h.ldk = ldk; h.center = center_dev;
  h.tile_begin = 0;
  const int shape = eval_shape(kernel, d, precision, FFC_EVAL_DEFAULT);
  h.row_tiles = eval_row_tiles(s, shape);
  h.tc_base = 0;
  h.tc_spad = eval_tc5_pad_s(s);
  h.tc_npad = eval_tc5_pad_n(n);
  char* tc_raw = nullptr;
  void* tc_scr = nullptr;
  const int64_t tc_rows = h.tc_spad + h.tc_npad;
  if (shape >= 2) {   // the tcgen05 path's plane arena, 256-byte aligned
    retain_pool_memory();
    FFC_CUDA(cudaMallocAsync((void**)&tc_raw, eval_tc5_scratch_bytes(tc_rows, d) + 256, st));
    tc_scr = (void*)(((uintptr_t)tc_raw + 255) & ~(uintptr_t)255);
  }
  FFC_CUDA(cudaMemcpyAsync(item, &h, sizeof(h), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  ffc_status rc = launch_eval(kernel, Y_dev, dtype, X_dev, d, precision, shape, item, 1, eval_tiles(s, n, shape), mind2,
                              lsc, status, tc_scr, tc_rows, st);
  if (tc_raw) FFC_CUDA(cudaFreeAsync(tc_raw, st));
  if (rc != FFC_OK) return rc;
  double hl = 0.0;
  int32_t hst = 0;
  FFC_CUDA(cudaMemcpyAsync(&hl, lsc, sizeof(double), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&hst, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(ar.base, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  if (log_scale_host) *log_scale_host = hl;
  if (hst == FFC_E_SINGULAR) set_error("ffc_eval_block: Laplace kernel at a zero distance");
  if (hst == FFC_E_TIMEOUT) set_error("ffc_eval_block: a bounded wait of the tcgen05 pipeline ran out");
  return (ffc_status)hst;
}

ffc_status ffc_id(void* K_dev, int64_t s, int64_t n, int64_t ldk, int32_t precision, int64_t r_max, double tol,
                  int32_t* skel_perm_dev, double* T_dev, int64_t ldt, int64_t* rank_host, double* r22_rel_host,
                  void* stream) {
  FFC_REQUIRE(s >= 0 && n >= 0 && ldk >= std::max<int64_t>(s, 1), "ffc_id: need s, n >= 0 and ldk >= s");
  FFC_REQUIRE(s <= MAX_ROWS, "ffc_id: s = %lld exceeds %d rows", (long long)s, MAX_ROWS);
  FFC_REQUIRE(r_max >= 0, "ffc_id: r_max must be >= 0");
  FFC_REQUIRE(std::min<int64_t>(r_max, std::min(s, n)) <= MAX_RANK, "ffc_id: rank cap above %d", MAX_RANK);
  FFC_REQUIRE(ldt >= std::max<int64_t>(r_max, 1), "ffc_id: ldt must be >= max(r_max, 1)");
  FFC_REQUIRE(precision == FFC_FP64 || precision == FFC_MIXED, "ffc_id: bad precision");
  FFC_REQUIRE(rank_host && r22_rel_host, "ffc_id: null output pointer");
  FFC_REQUIRE(n == 0 || (K_dev && skel_perm_dev && T_dev), "ffc_id: null pointer");
  cudaStream_t st = as_stream(stream);
  const int kcap = (int)std::min<int64_t>(r_max, std::min(s, n));
  if (n == 0) { *rank_host = 0; *r22_rel_host = 0.0; return FFC_OK; }
  const int sm = std::max<int64_t>(s, 1) > 0 ? (int)std::max<int64_t>(s, 1) : 1;
  // the blocked QR (panel width nb) when the columns are 16-byte aligned
  const size_t esz = precision == FFC_MIXED ? sizeof(float) : sizeof(double);
  const bool aligned = (reinterpret_cast<uintptr_t>(K_dev) % 16 == 0) && ((size_t)ldk * esz) % 16 == 0;
  const int nb = aligned ? qr_panel(precision, sm, -1) : 1;
  const int cap = cpqr_max_ctas(precision, sm, -1, nb);
  FFC_REQUIRE(cap > 0, "ffc_id: the QR kernel cannot be resident on this device");
  FFC_REQUIRE(cpqr_min_group(n) <= cap, "ffc_id: n = %lld columns exceed what the QR can hold", (long long)n);
  const int g = std::min(cap, std::max(cpqr_min_group(n), group_size(s, n, 4096)));
  const int nbl = (n + g - 1) / g <= QR_FS_COLS ? nb : 1;   // the blocked form keeps each CTA's F rows on chip
  const int rc_cap = std::max(kcap, 1);
  Arena ar;
  size_t bytes = 16 * 256 + round_up(sizeof(CpqrItem)) + round_up(sizeof(TrsmItem)) +
                 round_up(sizeof(CtaAssign) * g) + round_up(sizeof(int32_t) * rc_cap) +
                 round_up(sizeof(double) * rc_cap) + 2 * round_up(sizeof(double) * n) + round_up((size_t)n) +
                 round_up(sizeof(Slot) * 2 * g) + round_up((size_t)rc_cap * rc_cap * sizeof(double)) +
                 (precision == FFC_MIXED ? round_up((size_t)((rc_cap + 3) & ~3) * ((rc_cap + 3) & ~3) * sizeof(float)) : 0) +
                 round_up(12 * sizeof(unsigned long long)) +
                 (nbl > 1 ? round_up((size_t)n * QR_F_STRIDE * esz) : 0);
  FFC_CUDA(cudaMallocAsync((void**)&ar.base, bytes, st));
  CpqrItem* d_item = ar.take<CpqrItem>(1);
  TrsmItem* d_titem = ar.take<TrsmItem>(1);
  CtaAssign* d_assign = ar.take<CtaAssign>(g);
  int32_t* piv = ar.take<int32_t>(rc_cap);
  double* beta = ar.take<double>(rc_cap);
  double* vn1 = ar.take<double>(n);
  double* vn2 = ar.take<double>(n);
  uint8_t* sel = ar.take<uint8_t>(n);
  Slot* slots = ar.take<Slot>(2 * g);
  double* R11 = ar.take<double>((size_t)rc_cap * rc_cap);
  float* R11f = precision == FFC_MIXED ? ar.take<float>((size_t)((rc_cap + 3) & ~3) * ((rc_cap + 3) & ~3)) : nullptr;
  unsigned* barrier = ar.take<unsigned>(1);
  unsigned long long* red = ar.take<unsigned long long>(12);
  int32_t* rank = ar.take<int32_t>(1);
  double* r22 = ar.take<double>(1);
  int32_t* status = ar.take<int32_t>(1);
  char* Fbuf = nbl > 1 ? ar.take<char>((size_t)n * QR_F_STRIDE * esz) : nullptr;
  CpqrItem hi = {};
  hi.A = K_dev; hi.lda = ldk; hi.s = (int32_t)s; hi.n = (int32_t)n; hi.r_max = kcap; hi.tol = tol;
  hi.piv = piv; hi.beta = beta; hi.vn1 = vn1; hi.vn2 = vn2; hi.selected = sel; hi.slots = slots;
  hi.barrier = barrier; hi.red = red; hi.rank_out = rank; hi.r22_out = r22; hi.status_out = status;
  hi.F = Fbuf;
  std::vector<CtaAssign> asg(g);
  for (int c = 0; c < g; ++c) asg[c] = CtaAssign{0, c, g, 0};
  TrsmItem ti = {};
  ti.A = K_dev; ti.lda = ldk; ti.n = (int32_t)n; ti.rank = rank; ti.piv = piv; ti.beta = beta; ti.selected = sel;
  ti.skel_perm = skel_perm_dev; ti.R11 = R11; ti.R11f = R11f; ti.T = T_dev; ti.ldt = ldt; ti.r_cap = rc_cap;
  ti.tile_begin = 0;
  FFC_CUDA(cudaMemcpyAsync(d_item, &hi, sizeof(hi), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_titem, &ti, sizeof(ti), cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(d_assign, asg.data(), sizeof(CtaAssign) * g, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemsetAsync(barrier, 0, sizeof(unsigned), st));
  FFC_CUDA(cudaMemsetAsync(slots, 0, sizeof(Slot) * 2 * g, st));   // the QR's group accumulators start at zero
  FFC_CUDA(cudaMemsetAsync(red, 0, sizeof(unsigned long long) * 12, st));
  FFC_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  FFC_CUDA(cudaMemsetAsync(rank, 0, sizeof(int32_t), st));
  ffc_status rc = launch_cpqr(precision, d_item, d_assign, g, (int)std::max<int64_t>(s, 1), st, nullptr, -1, nbl);
  if (rc != FFC_OK) return rc;
  rc = launch_trsm_batched(precision, d_titem, 1, trsm_tiles(n), rc_cap, st);
  if (rc != FFC_OK) return rc;
  int32_t hr = 0, hs = 0;
  double hr22 = 0.0;
  FFC_CUDA(cudaMemcpyAsync(&hr, rank, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&hr22, r22, sizeof(double), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(&hs, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(ar.base, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  *rank_host = hr;
  *r22_rel_host = hr22;
  if (hs == FFC_E_TIMEOUT) set_error("ffc_id: a QR group barrier timed out");
  return (ffc_status)hs;
}

ffc_status ffc_id_error(ffc_kernel kernel, const void* Y_dev, int32_t dtype, const int64_t* rows_dev, int64_t m,
                        const void* X_dev, int64_t n, int32_t d, const int32_t* skel_perm_dev, const double* T_dev,
                        int64_t ldt, int64_t r, double* err_host, void* stream) {
  FFC_REQUIRE(m >= 0 && n >= 0 && d >= 1 && r >= 0 && r <= n, "ffc_id_error: need m, n >= 0, d >= 1, 0 <= r <= n");
  FFC_REQUIRE(ldt >= std::max<int64_t>(r, 1), "ffc_id_error: ldt must be >= r");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_id_error: bad dtype");
  FFC_REQUIRE(err_host, "ffc_id_error: err_host is null");
  if (!kernel_ok(kernel, d)) return FFC_E_INVALID;
  if (m == 0 || n == 0) { *err_host = 0.0; return FFC_OK; }
  FFC_REQUIRE(Y_dev && X_dev && skel_perm_dev && (r == 0 || T_dev), "ffc_id_error: null pointer");
  cudaStream_t st = as_stream(stream);
  const int64_t blocks = id_error_blocks(m, n, r);
  Arena ar;
  FFC_CUDA(cudaMallocAsync((void**)&ar.base, round_up(sizeof(double) * 2 * blocks) + 512, st));
  double* partial = ar.take<double>(2 * blocks);
  double* mind2 = ar.take<double>(1);
  ffc_status rc = launch_id_error(kernel, Y_dev, dtype, rows_dev, m, X_dev, n, d, skel_perm_dev, T_dev, ldt, r,
                                  partial, blocks, mind2, nullptr, nullptr, st);
  if (rc != FFC_OK) return rc;
  std::vector<double> hp(2 * blocks);
  double hm = 1.0;
  FFC_CUDA(cudaMemcpyAsync(hp.data(), partial, sizeof(double) * 2 * blocks, cudaMemcpyDeviceToHost, st));
  if (kernel.kind == FFC_LAPLACE) FFC_CUDA(cudaMemcpyAsync(&hm, mind2, sizeof(double), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(ar.base, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  if (kernel.kind == FFC_LAPLACE && !(hm > 0.0)) {
    set_error("ffc_id_error: Laplace kernel at a zero distance");
    return FFC_E_SINGULAR;
  }
  double num = 0.0, den = 0.0;
  for (int64_t b = 0; b < blocks; ++b) { num += hp[2 * b]; den += hp[2 * b + 1]; }
  *err_host = den > 0.0 ? std::sqrt(num / den) : 0.0;
  return FFC_OK;
}

int32_t ffc_tree_depth(int64_t N, int64_t leaf_size) {
  if (N <= 0 || leaf_size <= 0) return 0;
  int32_t D = 0;
  while (((N + ((int64_t)1 << D) - 1) >> D) > leaf_size) ++D;
  return D;
}

ffc_status ffc_build_tree(const void* points_dev, int32_t dtype, int64_t N, int32_t d, int64_t leaf_size,
                          int64_t* perm_dev, int64_t* begin_dev, int64_t* count_dev, double* centroid_dev,
                          double* radius_dev, void* stream) {
  FFC_REQUIRE(N >= 1 && d >= 1 && leaf_size >= 1, "ffc_build_tree: need N, d, leaf_size >= 1");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_build_tree: bad dtype");
  FFC_REQUIRE(points_dev && perm_dev && begin_dev && count_dev && centroid_dev && radius_dev,
              "ffc_build_tree: null pointer");
  const int depth = ffc_tree_depth(N, leaf_size);
  FFC_REQUIRE(depth <= 24, "ffc_build_tree: depth %d too large", depth);
  const int64_t n_nodes = ((int64_t)1 << (depth + 1)) - 1;
  std::vector<int64_t> b(n_nodes), c(n_nodes);
  node_layout(N, depth, b.data(), c.data(), nullptr);
  cudaStream_t st = as_stream(stream);
  FFC_CUDA(cudaMemcpyAsync(begin_dev, b.data(), sizeof(int64_t) * n_nodes, cudaMemcpyHostToDevice, st));
  FFC_CUDA(cudaMemcpyAsync(count_dev, c.data(), sizeof(int64_t) * n_nodes, cudaMemcpyHostToDevice, st));
  ffc_status rc = launch_build_tree(points_dev, dtype, N, d, depth, perm_dev, b.data(), c.data(), begin_dev,
                                    count_dev, centroid_dev, radius_dev, st);
  if (rc != FFC_OK) return rc;
  FFC_CUDA(cudaStreamSynchronize(st));
  return FFC_OK;
}

}  // extern "C"
