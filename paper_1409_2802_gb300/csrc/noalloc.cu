// ffc_id_noalloc: the interpolative decomposition of ffc_id without any
// device allocation. The QR and triangular-solve kernels are the ones ffc_id
// launches; their scratch lives in one file-scope device array instead of
// memory obtained from cudaMallocAsync.
#include <algorithm>
#include <atomic>

#include "ffc_internal.cuh"

namespace ffc {
int cpqr_rows_per_lane(int s_max);
}  // namespace ffc

using namespace ffc;

namespace {

// Largest problem the fixed scratch holds (see include/ffc.h).
constexpr int64_t NA_MAX_COLS = FFC_NOALLOC_MAX_COLS;
constexpr int64_t NA_MAX_RANK = FFC_NOALLOC_MAX_RANK;
constexpr int64_t NA_MAX_GROUP = 256;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// fixed layout of the scratch array
constexpr size_t OFF_ITEM = 0;
constexpr size_t OFF_TITEM = OFF_ITEM + align256(sizeof(CpqrItem));
constexpr size_t OFF_ASSIGN = OFF_TITEM + align256(sizeof(TrsmItem));
constexpr size_t OFF_PIV = OFF_ASSIGN + align256(sizeof(CtaAssign) * NA_MAX_GROUP);
constexpr size_t OFF_BETA = OFF_PIV + align256(sizeof(int32_t) * NA_MAX_RANK);
constexpr size_t OFF_VN1 = OFF_BETA + align256(sizeof(double) * NA_MAX_RANK);
constexpr size_t OFF_VN2 = OFF_VN1 + align256(sizeof(double) * NA_MAX_COLS);
constexpr size_t OFF_SEL = OFF_VN2 + align256(sizeof(double) * NA_MAX_COLS);
constexpr size_t OFF_SLOTS = OFF_SEL + align256(NA_MAX_COLS);
constexpr size_t OFF_R11 = OFF_SLOTS + align256(sizeof(Slot) * 2 * NA_MAX_GROUP);
constexpr size_t OFF_SCAL = OFF_R11 + align256(sizeof(double) * NA_MAX_RANK * NA_MAX_RANK);
constexpr size_t SCRATCH_BYTES = OFF_SCAL + 256;
static_assert(SCRATCH_BYTES <= (size_t)1 << 20, "no-allocation scratch must stay under 1 MiB");

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, taken once per device. Host threads making
// their first call on a device at the same time may both look it up; they store the same value.
static std::atomic<char*> g_scratch_addr[64];

struct Scalars {
  unsigned barrier;
  int32_t rank;
  int32_t status;
  int32_t pad;
  double r22;
  unsigned long long red[12];   // the QR's group reduction words (steps >= 1)
};
static_assert(sizeof(Scalars) <= 256, "scalars fit their scratch slot");

// Writes the work tables into the scratch array and clears what must start
// at zero (the array keeps the previous call's contents).
__global__ void noalloc_setup_kernel(CpqrItem item, TrsmItem titem, int g, Scalars* sc, CpqrItem* d_item,
                                     TrsmItem* d_titem, CtaAssign* d_assign) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // the QR's group accumulators (start of the slot area) start at zero
  if (t < 16) reinterpret_cast<unsigned long long*>(item.slots)[t] = 0ull;
  if (t == 0) {
    *d_item = item;
    *d_titem = titem;
    sc->barrier = 0u;
    sc->rank = 0;
    sc->status = FFC_OK;
    sc->r22 = 0.0;
  }
  if (t < 12) sc->red[t] = 0ull;
  for (int c = t; c < g; c += gridDim.x * blockDim.x) d_assign[c] = CtaAssign{0, c, g, 0};
}

ffc_status scratch_base(char** out) {
  int dev = 0;
  FFC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("ffc_id_noalloc: device ordinal %d out of range", dev);
    return FFC_E_INVALID;
  }
  char* addr = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!addr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    addr = static_cast<char*>(p);
    g_scratch_addr[dev].store(addr, std::memory_order_release);
  }
  *out = addr;
  return FFC_OK;
}

int group_size_noalloc(int64_t s, int64_t n) {
  int64_t g = (s * n + 16383) / 16384;
  g = std::min<int64_t>(g, std::max<int64_t>(1, n / 4));
  return (int)std::max<int64_t>(1, g);
}

}  // namespace

extern "C" ffc_status ffc_id_noalloc(void* K_dev, int64_t s, int64_t n, int64_t ldk, int32_t precision,
                                     int64_t r_max, double tol, int32_t* skel_perm_dev, double* T_dev, int64_t ldt,
                                     int64_t* rank_host, double* r22_rel_host, void* stream) {
  FFC_REQUIRE(s >= 0 && n >= 0 && ldk >= std::max<int64_t>(s, 1), "ffc_id_noalloc: need s, n >= 0 and ldk >= s");
  FFC_REQUIRE(s <= 2048, "ffc_id_noalloc: s = %lld exceeds 2048 rows", (long long)s);
  FFC_REQUIRE(n <= NA_MAX_COLS, "ffc_id_noalloc: n = %lld exceeds the fixed scratch limit of %lld columns",
              (long long)n, (long long)NA_MAX_COLS);
  FFC_REQUIRE(r_max >= 0, "ffc_id_noalloc: r_max must be >= 0");
  const int64_t kcap = std::min<int64_t>(r_max, std::min(s, n));
  FFC_REQUIRE(kcap <= NA_MAX_RANK, "ffc_id_noalloc: min(r_max, s, n) = %lld exceeds the fixed scratch limit of %lld",
              (long long)kcap, (long long)NA_MAX_RANK);
  FFC_REQUIRE(ldt >= std::max<int64_t>(r_max, 1), "ffc_id_noalloc: ldt must be >= max(r_max, 1)");
  FFC_REQUIRE(precision == FFC_FP64, "ffc_id_noalloc: only FFC_FP64 is supported");
  FFC_REQUIRE(rank_host && r22_rel_host, "ffc_id_noalloc: null output pointer");
  FFC_REQUIRE(n == 0 || (K_dev && skel_perm_dev && T_dev), "ffc_id_noalloc: null pointer");
  if (n == 0) { *rank_host = 0; *r22_rel_host = 0.0; return FFC_OK; }
  char* base = nullptr;
  ffc_status rc = scratch_base(&base);
  if (rc != FFC_OK) return rc;
  cudaStream_t st = as_stream(stream);
  const int s_launch = (int)std::max<int64_t>(s, 1);
  const int cap = cpqr_max_ctas(precision, s_launch);
  FFC_REQUIRE(cap > 0, "ffc_id_noalloc: the QR kernel cannot be resident on this device");
  // each CTA of the group owns at most a fixed number of columns (their norms live in its shared memory)
  FFC_REQUIRE(cpqr_min_group(n) <= std::min<int>(cap, (int)NA_MAX_GROUP),
              "ffc_id_noalloc: n = %lld needs %d resident QR blocks, this device holds %d", (long long)n,
              cpqr_min_group(n), std::min<int>(cap, (int)NA_MAX_GROUP));
  const int g = std::min<int>({cap, (int)NA_MAX_GROUP, std::max(cpqr_min_group(n), group_size_noalloc(s, n))});
  const int rc_cap = (int)std::max<int64_t>(kcap, 1);

  CpqrItem* d_item = reinterpret_cast<CpqrItem*>(base + OFF_ITEM);
  TrsmItem* d_titem = reinterpret_cast<TrsmItem*>(base + OFF_TITEM);
  CtaAssign* d_assign = reinterpret_cast<CtaAssign*>(base + OFF_ASSIGN);
  Scalars* sc = reinterpret_cast<Scalars*>(base + OFF_SCAL);
  CpqrItem hi = {};
  hi.A = K_dev; hi.lda = ldk; hi.s = (int32_t)s; hi.n = (int32_t)n; hi.r_max = (int32_t)kcap; hi.tol = tol;
  hi.piv = reinterpret_cast<int32_t*>(base + OFF_PIV);
  hi.beta = reinterpret_cast<double*>(base + OFF_BETA);
  hi.vn1 = reinterpret_cast<double*>(base + OFF_VN1);
  hi.vn2 = reinterpret_cast<double*>(base + OFF_VN2);
  hi.selected = reinterpret_cast<uint8_t*>(base + OFF_SEL);
  hi.slots = base + OFF_SLOTS;
  hi.barrier = &sc->barrier; hi.red = sc->red; hi.rank_out = &sc->rank; hi.r22_out = &sc->r22;
  hi.status_out = &sc->status;
  TrsmItem ti = {};
  ti.A = K_dev; ti.lda = ldk; ti.n = (int32_t)n; ti.rank = &sc->rank; ti.piv = hi.piv; ti.beta = hi.beta;
  ti.selected = hi.selected; ti.skel_perm = skel_perm_dev; ti.R11 = reinterpret_cast<double*>(base + OFF_R11);
  ti.T = T_dev; ti.ldt = ldt; ti.r_cap = rc_cap; ti.tile_begin = 0;

  noalloc_setup_kernel<<<1, 256, 0, st>>>(hi, ti, g, sc, d_item, d_titem, d_assign);
  FFC_CUDA(cudaGetLastError());
  rc = launch_cpqr(precision, d_item, d_assign, g, s_launch, st);
  if (rc != FFC_OK) return rc;
  rc = launch_trsm_batched(precision, d_titem, 1, trsm_tiles(n), rc_cap, st);
  if (rc != FFC_OK) return rc;
  Scalars hs = {};
  FFC_CUDA(cudaMemcpyAsync(&hs, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  *rank_host = hs.rank;
  *r22_rel_host = hs.r22;
  if (hs.status == FFC_E_TIMEOUT) set_error("ffc_id_noalloc: a QR group barrier timed out");
  return (ffc_status)hs.status;
}
