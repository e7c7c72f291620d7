// Column-pivoted Householder QR and T = R11^-1 R12 (FP64 path).
//
// Method: the ID of the sampled block comes from a rank-revealing QR
// K' Pi = Q [R11 R12; 0 R22] (§2.1.3, ID theorem; Appendix A.1): the
// skeleton is the first r pivots and P solves R11 P = R12.
//
// GPU design. A launch holds many independent blocks (work items). Each item
// gets a group of g CTAs; CTA c of the group owns the contiguous column range
// [n c / g, n (c+1) / g) for the whole factorisation. Columns never move: a
// pivot is marked selected and its rows >= k are never read again, so R is
// formed in place in the original column positions. One step k:
//   1. every CTA reduces the g published (best norm, column, sum of squared
//      norms) slots of the previous step -> the same pivot p and ||R22||_F on
//      every CTA (deterministic reduction order);
//   2. every CTA loads column p (rows k..s-1) from L2 and forms the LAPACK
//      dlarfg reflector redundantly in shared memory;
//   3. each warp applies the reflector to one owned column at a time, held
//      in registers (R values per lane, s <= 32 R): one read and one write
//      of the column per step; the residual norm is downdated as in LAPACK
//      xLAQP2 and recomputed from the registers when cancellation makes the
//      downdate unsafe;
//   4. the CTA publishes its new local (best, column, sum) slot and joins a
//      group barrier (global atomic counter, bounded spin).
// Groups are co-resident (cooperative launch), so the barriers cannot
// deadlock; a wait that runs out sets FFC_E_TIMEOUT and ends the item.
#include <algorithm>
#include <cfloat>
#include <climits>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// better (value, column): larger value, then lower column
__device__ __forceinline__ bool better(double v, int c, double bv, int bc) {
  return v > bv || (v == bv && c < bc);
}

// Block-wide deterministic reduction of per-thread (best, col, sum).
__device__ void block_reduce_slot(double& best, int& col, double& sum, double* sb, int* sc, double* ss) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oc = __shfl_xor_sync(0xffffffffu, col, o);
    double os = __shfl_xor_sync(0xffffffffu, sum, o);
    if (better(ob, oc, best, col)) { best = ob; col = oc; }
    sum += os;
  }
  if (lane == 0) { sb[warp] = best; sc[warp] = col; ss[warp] = sum; }
  __syncthreads();
  best = sb[0]; col = sc[0]; sum = ss[0];
  for (int w = 1; w < QR_WARPS; ++w) {
    if (better(sb[w], sc[w], best, col)) { best = sb[w]; col = sc[w]; }
    sum += ss[w];
  }
  __syncthreads();
}

// Thread 0 only: arrive and wait until `target` arrivals. false on timeout.
__device__ bool group_barrier(unsigned* ctr, unsigned target) {
  __threadfence();
  atomicAdd(ctr, 1u);
  long long spins = 0;
  while (ld_acquire_u32(ctr) < target) {
    if (++spins > SPIN_LIMIT) return false;
    __nanosleep(40);
  }
  __threadfence();
  return true;
}

template <int R>
__global__ void __launch_bounds__(QR_THREADS)
cpqr_fp64_kernel(const CpqrItem* __restrict__ items, const CtaAssign* __restrict__ assign) {
  extern __shared__ double vsh[];   // Householder vector, s entries
  __shared__ double sb[QR_WARPS], ss[QR_WARPS];
  __shared__ int sc[QR_WARPS];
  __shared__ double sh_tau, sh_beta;
  __shared__ int sh_fail;

  const CtaAssign a = assign[blockIdx.x];
  const CpqrItem it = items[a.item];
  const int s = it.s, n = it.n;
  double* __restrict__ A = reinterpret_cast<double*>(it.A);
  const int64_t lda = it.lda;
  const int c0 = (int)((int64_t)n * a.rank / a.g), c1 = (int)((int64_t)n * (a.rank + 1) / a.g);
  Slot* slots = reinterpret_cast<Slot*>(it.slots);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kmax = min(it.r_max, min(s, n));
  const double TOL3Z = 1.0536712127723509e-08;   // sqrt(2^-53)
  if (threadIdx.x == 0) sh_fail = 0;

  // initial residual norms of the owned columns
  double best = -1.0, sum = 0.0;
  int col = INT_MAX;
  for (int j = c0 + warp; j < c1; j += QR_WARPS) {
    const double* cj = A + (int64_t)j * lda;
    double acc = 0.0;
    for (int i = lane; i < s; i += 32) { double x = cj[i]; acc = fma(x, x, acc); }
    acc = warp_sum(acc);
    const double nr = sqrt(acc);
    if (lane == 0) { it.vn1[j] = nr; it.vn2[j] = nr; it.selected[j] = 0; }
    if (better(nr, j, best, col)) { best = nr; col = j; }
    sum += acc;
  }
  if (lane != 0) sum = 0.0;   // one copy per warp
  block_reduce_slot(best, col, sum, sb, sc, ss);

  double fro2 = 0.0;
  int k = 0;
  int status = FFC_OK;
  for (;; ++k) {
    // publish this CTA's slot for step k and synchronise the group
    if (a.g > 1) {
      if (threadIdx.x == 0) {
        Slot* sl = slots + (k & 1) * a.g + a.rank;
        sl->best = best; sl->sum = sum; sl->col = col;
        if (!group_barrier(it.barrier, (unsigned)a.g * (unsigned)(k + 1))) sh_fail = 1;
      }
      __syncthreads();
      if (sh_fail) { status = FFC_E_TIMEOUT; break; }
      // reduce the group's slots (same order on every CTA)
      best = -1.0; col = INT_MAX; sum = 0.0;
      for (int t = threadIdx.x; t < a.g; t += QR_THREADS) {
        const Slot* sl = slots + (k & 1) * a.g + t;
        double b = __ldcg(&sl->best), su = __ldcg(&sl->sum);
        int c = __ldcg(&sl->col);
        if (better(b, c, best, col)) { best = b; col = c; }
        sum += su;
      }
      block_reduce_slot(best, col, sum, sb, sc, ss);
    }
    if (k == 0) fro2 = sum;
    const double r22sq = sum;
    if (it.tol > 0.0 && sqrt(r22sq) <= it.tol * sqrt(fro2)) break;
    if (k >= kmax || col == INT_MAX || !(best > 0.0)) {
      if (it.tol > 0.0) status = FFC_E_TOL_NOT_REACHED;
      break;
    }
    const int p = col;

    // reflector from column p, rows k..s-1 (written by its owner before the barrier)
    const double* cp = A + (int64_t)p * lda;
    double part = 0.0;
    for (int i = k + threadIdx.x; i < s; i += QR_THREADS) {
      double x = __ldcg(cp + i);
      vsh[i] = x;
      if (i > k) part = fma(x, x, part);
    }
    part = warp_sum(part);
    if (lane == 0) sb[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double xn2 = 0.0;
      for (int w = 0; w < QR_WARPS; ++w) xn2 += sb[w];
      const double alpha = vsh[k];
      if (xn2 == 0.0) {
        sh_tau = 0.0; sh_beta = alpha;
      } else {
        const double nrm = hypot(alpha, sqrt(xn2));
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        sh_tau = (beta - alpha) / beta;
        sh_beta = beta;
      }
    }
    __syncthreads();
    const double tau = sh_tau, beta = sh_beta;
    if (tau != 0.0) {
      const double den = vsh[k] - beta;
      for (int i = k + 1 + threadIdx.x; i < s; i += QR_THREADS) vsh[i] = vsh[i] / den;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      vsh[k] = 1.0;
      if (a.rank == 0) { it.piv[k] = p; it.beta[k] = beta; }
      if (p >= c0 && p < c1) it.selected[p] = 1;
    }
    __syncthreads();

    // apply H_k to the owned free columns and downdate their norms
    best = -1.0; col = INT_MAX; sum = 0.0;
    for (int j = c0 + warp; j < c1; j += QR_WARPS) {
      if (j == p || it.selected[j]) continue;
      double* cj = A + (int64_t)j * lda;
      double x[R];
      double dot = 0.0;
#pragma unroll
      for (int c = 0; c < R; ++c) {
        const int i = k + lane + 32 * c;
        x[c] = (i < s) ? cj[i] : 0.0;
        if (i < s) dot = fma(vsh[i], x[c], dot);
      }
      if (tau != 0.0) {
        dot = warp_sum(dot);
        const double tw = tau * dot;
#pragma unroll
        for (int c = 0; c < R; ++c) {
          const int i = k + lane + 32 * c;
          if (i < s) { x[c] = fma(-tw, vsh[i], x[c]); cj[i] = x[c]; }
        }
      }
      const double akj = __shfl_sync(0xffffffffu, x[0], 0);
      double nr1 = it.vn1[j], nr2 = it.vn2[j];
      if (nr1 != 0.0) {
        double t = fabs(akj) / nr1;
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        const double q = nr1 / nr2;
        const double t2 = t * q * q;
        if (t2 <= TOL3Z) {
          double acc = 0.0;
#pragma unroll
          for (int c = 0; c < R; ++c) {
            const int i = k + lane + 32 * c;
            if (i > k && i < s) acc = fma(x[c], x[c], acc);
          }
          acc = warp_sum(acc);
          nr1 = sqrt(acc);
          nr2 = nr1;
        } else {
          nr1 = nr1 * sqrt(t);
        }
      }
      if (lane == 0) { it.vn1[j] = nr1; it.vn2[j] = nr2; }
      if (better(nr1, j, best, col)) { best = nr1; col = j; }
      if (lane == 0) sum += nr1 * nr1;
    }
    block_reduce_slot(best, col, sum, sb, sc, ss);
  }

  // status_out starts at FFC_OK; a timeout anywhere in the group wins
  if (threadIdx.x == 0) {
    if (status == FFC_E_TIMEOUT) atomicExch(it.status_out, (int)FFC_E_TIMEOUT);
    if (a.rank == 0) {
      *it.rank_out = k;
      *it.r22_out = fro2 > 0.0 ? sqrt(sum) / sqrt(fro2) : 0.0;
      if (status != FFC_E_TIMEOUT) atomicCAS(it.status_out, (int)FFC_OK, status);
    }
  }
}

// -------- finalize: skeleton order and dense R11 -----------------------------

__global__ void __launch_bounds__(256)
finalize_kernel(const TrsmItem* __restrict__ items) {
  __shared__ int wc[8];
  __shared__ int base;
  const TrsmItem it = items[blockIdx.x];
  const int r = *it.rank, n = it.n;
  const double* A = reinterpret_cast<const double*>(it.A);
  for (int i = threadIdx.x; i < r; i += blockDim.x) it.skel_perm[i] = it.piv[i];
  if (threadIdx.x == 0) base = r;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const bool f = j < n && !it.selected[j];
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wc[warp] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < 8; ++w) { if (w < warp) off += wc[w]; tot += wc[w]; }
    if (f) it.skel_perm[base + off + __popc(b & ((1u << lane) - 1u))] = j;
    __syncthreads();
    if (threadIdx.x == 0) base += tot;
    __syncthreads();
  }
  // R11 (r x r, row-major, ld r): R11[i][k] = A[i, piv[k]] above the diagonal, beta[k] on it
  for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x) {
    const int i = (int)(e / r), kk = (int)(e % r);
    double v = 0.0;
    if (i < kk) v = A[i + (int64_t)it.piv[kk] * it.lda];
    else if (i == kk) v = it.beta[kk];
    it.R11[e] = v;
  }
}

// -------- T = R11^-1 R12: one warp per non-skeleton column --------------------

__device__ __forceinline__ int find_trsm_item(const TrsmItem* items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int RT>
__global__ void __launch_bounds__(256)
trsm_kernel(const TrsmItem* __restrict__ items, int n_items) {
  const int q = find_trsm_item(items, n_items, blockIdx.x);
  const TrsmItem it = items[q];
  const int r = *it.rank, n = it.n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = (int)(blockIdx.x - it.tile_begin) * 8 + warp;   // index among the n - r free columns
  if (c >= n - r || r == 0) return;
  const int j = it.skel_perm[r + c];
  const double* A = reinterpret_cast<const double*>(it.A);
  const double* b = A + (int64_t)j * it.lda;
  const double* R11 = it.R11;
  double t[RT];
#pragma unroll
  for (int u = 0; u < RT; ++u) {
    const int i = lane + 32 * u;
    t[u] = (i < r) ? b[i] : 0.0;
  }
  for (int i = r - 1; i >= 0; --i) {
    const double* row = R11 + (int64_t)i * r;
    double part = 0.0;
#pragma unroll
    for (int u = 0; u < RT; ++u) {
      const int kk = lane + 32 * u;
      if (kk > i && kk < r) part = fma(row[kk], t[u], part);
    }
    part = warp_sum(part);
    const int owner_u = i >> 5;
#pragma unroll
    for (int u = 0; u < RT; ++u)
      if (u == owner_u && lane == (i & 31)) t[u] = (t[u] - part) / row[i];
  }
  const int64_t ldt = it.ldt > 0 ? it.ldt : r;
  double* T = it.T + (int64_t)c * ldt;
#pragma unroll
  for (int u = 0; u < RT; ++u) {
    const int i = lane + 32 * u;
    if (i < r) T[i] = t[u];
  }
}

template <int R>
ffc_status launch_cpqr_r(const CpqrItem* items, const CtaAssign* assign, int grid, int s_max, cudaStream_t st) {
  const size_t smem = (size_t)s_max * sizeof(double);
  auto kfn = cpqr_fp64_kernel<R>;
  FFC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(QR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FFC_CUDA(cudaLaunchKernelEx(&cfg, kfn, items, assign));
  return FFC_OK;
}

template <int R>
int max_ctas_r(int s_max) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cpqr_fp64_kernel<R>, QR_THREADS,
                                                (size_t)s_max * sizeof(double));
  return per_sm * sm_count();
}

template <int RT>
ffc_status launch_trsm_rt(const TrsmItem* items, int n_items, int64_t total_tiles, cudaStream_t st) {
  if (total_tiles <= 0) return FFC_OK;
  trsm_kernel<RT><<<(unsigned)total_tiles, 256, 0, st>>>(items, n_items);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace

int cpqr_rows_per_lane(int s_max) {
  int R = 1;
  while (32 * R < s_max) R *= 2;
  return R;
}

int cpqr_max_ctas(int precision, int s_max) {
  (void)precision;
  switch (cpqr_rows_per_lane(s_max)) {
    case 1: return max_ctas_r<1>(s_max);
    case 2: return max_ctas_r<2>(s_max);
    case 4: return max_ctas_r<4>(s_max);
    case 8: return max_ctas_r<8>(s_max);
    case 16: return max_ctas_r<16>(s_max);
    case 32: return max_ctas_r<32>(s_max);
    default: return max_ctas_r<64>(s_max);
  }
}

ffc_status launch_cpqr(int precision, const CpqrItem* items_dev, const CtaAssign* assign_dev, int grid,
                       int s_max, cudaStream_t st) {
  (void)precision;
  if (grid <= 0) return FFC_OK;
  switch (cpqr_rows_per_lane(s_max)) {
    case 1: return launch_cpqr_r<1>(items_dev, assign_dev, grid, s_max, st);
    case 2: return launch_cpqr_r<2>(items_dev, assign_dev, grid, s_max, st);
    case 4: return launch_cpqr_r<4>(items_dev, assign_dev, grid, s_max, st);
    case 8: return launch_cpqr_r<8>(items_dev, assign_dev, grid, s_max, st);
    case 16: return launch_cpqr_r<16>(items_dev, assign_dev, grid, s_max, st);
    case 32: return launch_cpqr_r<32>(items_dev, assign_dev, grid, s_max, st);
    case 64: return launch_cpqr_r<64>(items_dev, assign_dev, grid, s_max, st);
    default:
      set_error("cpqr: s = %d exceeds the supported 2048 rows", s_max);
      return FFC_E_INVALID;
  }
}

ffc_status launch_trsm_batched(int precision, const TrsmItem* items_dev, int n_items, int64_t total_tiles,
                               int r_cap_max, cudaStream_t st) {
  (void)precision;
  if (n_items <= 0) return FFC_OK;
  finalize_kernel<<<n_items, 256, 0, st>>>(items_dev);
  FFC_CUDA(cudaGetLastError());
  if (r_cap_max <= 32) return launch_trsm_rt<1>(items_dev, n_items, total_tiles, st);
  if (r_cap_max <= 64) return launch_trsm_rt<2>(items_dev, n_items, total_tiles, st);
  if (r_cap_max <= 128) return launch_trsm_rt<4>(items_dev, n_items, total_tiles, st);
  if (r_cap_max <= 256) return launch_trsm_rt<8>(items_dev, n_items, total_tiles, st);
  if (r_cap_max <= 512) return launch_trsm_rt<16>(items_dev, n_items, total_tiles, st);
  if (r_cap_max <= 1024) return launch_trsm_rt<32>(items_dev, n_items, total_tiles, st);
  set_error("trsm: rank cap %d exceeds 1024", r_cap_max);
  return FFC_E_INVALID;
}

}  // namespace ffc
