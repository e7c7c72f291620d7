// T = R11^-1 R12 after the pivoted QR (§2.1.3, the ID theorem: P = [I T] Pi^T; Appendix A.1: R11 is
// square and nonsingular while the pivots are nonzero, so T comes from back-substitution).
//
// finalize_kernel puts the skeleton in pivot order (the other columns ascending after it) and forms the
// dense R11 from the QR's in-place R (FP64, row-major; for mixed precision also its FP32 copy).
// trsm_kernel solves in FP64; trsm_refine_kernel (mixed precision, the default there) solves in FP32 and
// refines once with an exact double-float residual. A CTA owns TS_COLS columns of T in both.
#include <algorithm>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

// -------- finalize: skeleton order and dense R11 -----------------------------

template <typename T>
__global__ void __launch_bounds__(256)
finalize_kernel(const TrsmItem* __restrict__ items) {
  __shared__ int wc[8];
  __shared__ int base;
  const TrsmItem it = items[blockIdx.x];
  const int r = *it.rank, n = it.n;
  if (r < 0) return;   // attempt that will be redone with a larger sample
  const T* A = reinterpret_cast<const T*>(it.A);
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
  // R11 (r x r, row-major, ld r): R11[i][k] = A[i, piv[k]] above the diagonal, beta[k] on it;
  // walked column by column so that the reads of A are contiguous
  for (int64_t e = threadIdx.x; e < (int64_t)r * r; e += blockDim.x) {
    const int kk = (int)(e / r), i = (int)(e % r);
    double v = 0.0;
    if (i < kk) v = (double)A[i + (int64_t)it.piv[kk] * it.lda];
    else if (i == kk) v = it.beta[kk];
    it.R11[(int64_t)i * r + kk] = v;
    // FP32 copy, column-major with the leading dimension r rounded up to 4 (exact off the diagonal)
    if (it.R11f) it.R11f[(int64_t)kk * ((r + 3) & ~3) + i] = (float)v;
  }
  // zeros in the copy's padding rows r .. ld - 1 (read by the residual's 16-byte loads)
  if (it.R11f) {
    const int ldf = (r + 3) & ~3, pad = ldf - r;
    for (int e = threadIdx.x; e < r * pad; e += blockDim.x) it.R11f[(int64_t)(e / pad) * ldf + r + e % pad] = 0.0f;
  }
}

// -------- T = R11^-1 R12 (FP64) -----------------------------------------------

__device__ __forceinline__ int find_trsm_item(const TrsmItem* items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// T = R11^-1 R12 for a tile of TS_COLS non-skeleton columns per CTA, FP64.
// The tile (r x TS_COLS) lives in shared memory. Going up in diagonal blocks
// of TS_NB rows: each warp solves the block for its columns by substitution
// (lane = row, the solved entry broadcast by shuffle), then the CTA subtracts
// R11[0:i0, block] * T[block, :] from the rows above (an FP64 GEMM slab with
// R11 rows read contiguously).
constexpr int TS_COLS = 16, TS_NB = 32;

template <typename T>
__global__ void __launch_bounds__(256)
trsm_kernel(const TrsmItem* __restrict__ items, int n_items) {
  extern __shared__ double Ts[];   // [r][TS_COLS]
  __shared__ double Rd[TS_NB][TS_NB + 1];
  __shared__ double dinv[TS_NB];
  const int q = find_trsm_item(items, n_items, blockIdx.x);
  const TrsmItem it = items[q];
  const int r = *it.rank, n = it.n;
  const int c0 = (int)(blockIdx.x - it.tile_begin) * TS_COLS;
  const int nc = min(TS_COLS, n - r - c0);
  if (nc <= 0 || r <= 0) return;
  const T* A = reinterpret_cast<const T*>(it.A);
  const double* R11 = it.R11;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < r * nc; e += blockDim.x) {
    const int c = e / r, i = e % r;
    Ts[i * TS_COLS + c] = (double)A[i + (int64_t)it.skel_perm[r + c0 + c] * it.lda];
  }
  __syncthreads();
  for (int i1 = r; i1 > 0;) {
    const int i0 = max(0, i1 - TS_NB), nb = i1 - i0;
    // the diagonal block in shared memory (padded rows) and its reciprocal
    // diagonal: the substitution chain then multiplies instead of dividing
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, kk = e % nb;
      Rd[i][kk] = R11[(int64_t)(i0 + i) * r + i0 + kk];
    }
    __syncthreads();
    if (tid < nb) dinv[tid] = 1.0 / Rd[tid][tid];
    __syncthreads();
    for (int c = warp; c < nc; c += 8) {
      double t = lane < nb ? Ts[(i0 + lane) * TS_COLS + c] : 0.0;
      const double dl = lane < nb ? dinv[lane] : 0.0;
      for (int ii = nb - 1; ii >= 0; --ii) {
        if (lane == ii) t *= dl;
        const double ti = __shfl_sync(0xffffffffu, t, ii);
        if (lane < ii) t = fma(-Rd[lane][ii], ti, t);
      }
      if (lane < nb) Ts[(i0 + lane) * TS_COLS + c] = t;
    }
    __syncthreads();
    // T[0:i0, :] -= R11[0:i0, block] T[block, :]: each thread a 4 x 4 register
    // tile (rows j0..j0+3, columns cg..cg+3), 8 loads per 16 FMAs
    {
      const int cg = 4 * (tid & 3);
      for (int j0 = 4 * (tid >> 2); j0 < i0; j0 += 4 * (int)(blockDim.x >> 2)) {
        double acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = j0 + u < i0 ? Ts[(j0 + u) * TS_COLS + cg + v] : 0.0;
        for (int ii = 0; ii < nb; ++ii) {
          const double2 t01 = *reinterpret_cast<const double2*>(&Ts[(i0 + ii) * TS_COLS + cg]);
          const double2 t23 = *reinterpret_cast<const double2*>(&Ts[(i0 + ii) * TS_COLS + cg + 2]);
          const double t[4] = {t01.x, t01.y, t23.x, t23.y};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const double rr = j0 + u < i0 ? R11[(int64_t)(j0 + u) * r + i0 + ii] : 0.0;
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(-rr, t[v], acc[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < i0)
#pragma unroll
            for (int v = 0; v < 4; ++v) Ts[(j0 + u) * TS_COLS + cg + v] = acc[u][v];
      }
    }
    __syncthreads();
    i1 = i0;
  }
  const int64_t ldt = it.ldt > 0 ? it.ldt : r;
  for (int e = tid; e < r * nc; e += blockDim.x) {
    const int c = e / r, i = e % r;
    it.T[(int64_t)(c0 + c) * ldt + i] = Ts[i * TS_COLS + c];
  }
}

// -------- T = R11^-1 R12 for mixed precision: FP32 solves refined once ---------------------------
// The FP32 blocks' R has FP32 entries off the diagonal (beta, on it, is FP64). One step of iterative
// refinement (Wilkinson; Higham, "Accuracy and Stability of Numerical Algorithms", §12.1) keeps the FP64
// solve's accuracy at the FP32 rate: T1 = solve with R11 rounded to FP32; E = R12 - R11 T1 with every
// product exact (FP32 times FP32 is exactly hi + lo, fmaf) summed in double-float, the diagonal term in
// FP64; dT = the FP32 solve of E; T = T1 + dT in FP64. A CTA owns TS_COLS columns, as trsm_kernel.

constexpr int TR_THREADS = 1024;   // 32 warps: the diagonal substitution takes one per column of the tile

// (hi, lo) += p: Knuth's two-sum into the high part, its error into the low part
__device__ __forceinline__ void df_add(float& hi, float& lo, float p) {
  const float t = hi + p;
  const float bb = t - hi;
  lo += (hi - (t - bb)) + (p - bb);
  hi = t;
}

// (hi, lo) -= a t, with a t = p + pe exactly (fmaf)
__device__ __forceinline__ void residual_term(float& hi, float& lo, float a, float t) {
  const float p = a * t;
  const float pe = fmaf(a, t, -p);
  df_add(hi, lo, -p);
  lo -= pe;
}

// X[0:i0, :] -= R11[0:i0, i0:i0+nb] X[i0:i0+nb, :]: each thread a tile of RU rows x CV columns, one
// CV-wide shared load of X and one RU-wide 16- or 8-byte load of a column of R11 per step. Every entry
// takes the same FMAs in the same order whatever the tile shape. Only a row group reaching past i0 (the
// rows of the diagonal block, read by the vector load) masks its R11 values.
template <int RU, int CV>
__device__ __forceinline__ void solve_update(float* X, const float* __restrict__ R11, int64_t ldf, int i0, int nb) {
  constexpr int CG = TS_COLS / CV;
  const int tid = threadIdx.x;
  const int cg = CV * (tid % CG);
  const int rstep = RU * (int)(blockDim.x / CG);
  for (int j0 = RU * (tid / CG); j0 < i0; j0 += rstep) {
    float acc[RU][CV];
#pragma unroll
    for (int u = 0; u < RU; ++u)
#pragma unroll
      for (int v = 0; v < CV; ++v) acc[u][v] = j0 + u < i0 ? X[(j0 + u) * TS_COLS + cg + v] : 0.0f;
    const bool full = j0 + RU <= i0;
    for (int ii = 0; ii < nb; ++ii) {
      float t[CV], rv[RU];
      if constexpr (CV == 4) {
        const float4 t4 = *reinterpret_cast<const float4*>(&X[(i0 + ii) * TS_COLS + cg]);
        t[0] = t4.x; t[1] = t4.y; t[2] = t4.z; t[3] = t4.w;
      } else {
        const float2 t2 = *reinterpret_cast<const float2*>(&X[(i0 + ii) * TS_COLS + cg]);
        t[0] = t2.x; t[1] = t2.y;
      }
      if constexpr (RU == 4) {
        const float4 r4 = __ldg(reinterpret_cast<const float4*>(R11 + (int64_t)(i0 + ii) * ldf + j0));
        rv[0] = r4.x; rv[1] = r4.y; rv[2] = r4.z; rv[3] = r4.w;
      } else {
        const float2 r2 = __ldg(reinterpret_cast<const float2*>(R11 + (int64_t)(i0 + ii) * ldf + j0));
        rv[0] = r2.x; rv[1] = r2.y;
      }
      if (!full) {
#pragma unroll
        for (int u = 0; u < RU; ++u) rv[u] = j0 + u < i0 ? rv[u] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < RU; ++u)
#pragma unroll
        for (int v = 0; v < CV; ++v) acc[u][v] = fmaf(-rv[u], t[v], acc[u][v]);
    }
#pragma unroll
    for (int u = 0; u < RU; ++u)
      if (j0 + u < i0)
#pragma unroll
        for (int v = 0; v < CV; ++v) X[(j0 + u) * TS_COLS + cg + v] = acc[u][v];
  }
}

// Blocked back-substitution of X (r x nc, shared memory, row stride TS_COLS) with the FP32 copy of R11
// (column-major, leading dimension ldf = r rounded up to 4: exact off the diagonal, beta rounded on it);
// Rd, dinv: shared scratch of the diagonal block.
__device__ void solve_f32_block(float* X, const float* __restrict__ R11, int r, int nc, float (*Rd)[TS_NB + 1],
                                float* dinv) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t ldf = (r + 3) & ~3;
  for (int i1 = r; i1 > 0;) {
    const int i0 = max(0, i1 - TS_NB), nb = i1 - i0;
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, kk = e % nb;
      Rd[i][kk] = R11[(int64_t)(i0 + kk) * ldf + i0 + i];
    }
    __syncthreads();
    if (tid < nb) dinv[tid] = 1.0f / Rd[tid][tid];
    __syncthreads();
    for (int c = warp; c < nc; c += (int)(blockDim.x >> 5)) {
      float t = lane < nb ? X[(i0 + lane) * TS_COLS + c] : 0.0f;
      const float dl = lane < nb ? dinv[lane] : 0.0f;
      for (int ii = nb - 1; ii >= 0; --ii) {
        if (lane == ii) t *= dl;
        const float ti = __shfl_sync(0xffffffffu, t, ii);
        if (lane < ii) t = fmaf(-Rd[lane][ii], ti, t);
      }
      if (lane < nb) X[(i0 + lane) * TS_COLS + c] = t;
    }
    __syncthreads();
    // rows above the block, 16 i0 outputs: the thread's tile shrinks with i0 so that every thread has one
    if (i0 >= (int)blockDim.x) solve_update<4, 4>(X, R11, ldf, i0, nb);
    else if (2 * i0 >= (int)blockDim.x) solve_update<2, 4>(X, R11, ldf, i0, nb);
    else solve_update<2, 2>(X, R11, ldf, i0, nb);
    __syncthreads();
    i1 = i0;
  }
}

__global__ void __launch_bounds__(TR_THREADS)
trsm_refine_kernel(const TrsmItem* __restrict__ items, int n_items) {
  extern __shared__ float Tf[];   // [r][TS_COLS] T1, then [r][TS_COLS] E and dT
  __shared__ float Rd[TS_NB][TS_NB + 1];
  __shared__ float dinv[TS_NB];
  const int q = find_trsm_item(items, n_items, blockIdx.x);
  const TrsmItem it = items[q];
  const int r = *it.rank, n = it.n;
  const int c0 = (int)(blockIdx.x - it.tile_begin) * TS_COLS;
  const int nc = min(TS_COLS, n - r - c0);
  if (nc <= 0 || r <= 0) return;
  float* Ef = Tf + (size_t)r * TS_COLS;
  const float* A = reinterpret_cast<const float*>(it.A);
  const double* R11 = it.R11;   // FP64: the diagonal (beta) of the residual
  const float* R11f = it.R11f;  // FP32 copy: the solves and the off-diagonal products
  const int tid = threadIdx.x;
  // R12's tile (exact FP32), zero in the columns past nc
  for (int e = tid; e < r * TS_COLS; e += blockDim.x) {
    const int i = e / TS_COLS, c = e % TS_COLS;
    Tf[e] = c < nc ? A[i + (int64_t)it.skel_perm[r + c0 + c] * it.lda] : 0.0f;
  }
  __syncthreads();
  solve_f32_block(Tf, R11f, r, nc, Rd, dinv);
  // E = R12 - R11 T1 in tasks of 4 rows x 2 columns: the diagonal term in FP64, the rest exact products
  // summed in double-float from the diagonal outwards. A thread takes row groups g and G - 1 - g, so every
  // thread sums about r terms (the triangle's rows are long at the top and short at the bottom).
  {
    const int G = (r + 3) >> 2;
    const int cg = 2 * (tid & 7);
    const int64_t ldf = (r + 3) & ~3;
    for (int pg = tid >> 3; pg < (G + 1) >> 1; pg += (int)(blockDim.x >> 3)) {
      for (int half = 0; half < 2; ++half) {
        const int g = half == 0 ? pg : G - 1 - pg;
        if (half == 1 && g == pg) break;   // the middle group of an odd count
        const int j0 = 4 * g;
        float hi[4][2], lo[4][2];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = j0 + u;
#pragma unroll
          for (int v = 0; v < 2; ++v) {
            hi[u][v] = 0.0f;
            lo[u][v] = 0.0f;
            if (i < r && cg + v < nc) {
              const double b = (double)A[i + (int64_t)it.skel_perm[r + c0 + cg + v] * it.lda];
              const double s0 = fma(-R11[(int64_t)i * r + i], (double)Tf[i * TS_COLS + cg + v], b);
              hi[u][v] = (float)s0;
              lo[u][v] = (float)(s0 - (double)hi[u][v]);
            }
          }
        }
        // k <= j0 + 3 meets the group's diagonal (in s0) and the zeros below it: masked. Past it every
        // entry of rows j0 .. j0 + 3 is above the diagonal or a zero (lower part, padding rows), and the
        // rows >= r are never stored
        const int kp = min(j0 + 4, r);
        for (int k = j0 + 1; k < kp; ++k) {
          const float2 t2 = *reinterpret_cast<const float2*>(&Tf[k * TS_COLS + cg]);
          const float t[2] = {t2.x, t2.y};
          const float4 r4 = __ldg(reinterpret_cast<const float4*>(R11f + (int64_t)k * ldf + j0));
          const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float a = k > j0 + u ? rv[u] : 0.0f;
#pragma unroll
            for (int v = 0; v < 2; ++v) residual_term(hi[u][v], lo[u][v], a, t[v]);
          }
        }
        // the next step's loads are issued before this step's arithmetic (the last step reloads its own)
        float4 rn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float2 tn = make_float2(0.0f, 0.0f);
        if (kp < r) {
          rn = __ldg(reinterpret_cast<const float4*>(R11f + (int64_t)kp * ldf + j0));
          tn = *reinterpret_cast<const float2*>(&Tf[kp * TS_COLS + cg]);
        }
        for (int k = kp; k < r; ++k) {
          const float4 r4 = rn;
          const float2 t2 = tn;
          const int kn = min(k + 1, r - 1);
          rn = __ldg(reinterpret_cast<const float4*>(R11f + (int64_t)kn * ldf + j0));
          tn = *reinterpret_cast<const float2*>(&Tf[kn * TS_COLS + cg]);
          const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            residual_term(hi[u][0], lo[u][0], rv[u], t2.x);
            residual_term(hi[u][1], lo[u][1], rv[u], t2.y);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < r)
#pragma unroll
            for (int v = 0; v < 2; ++v) Ef[(j0 + u) * TS_COLS + cg + v] = hi[u][v] + lo[u][v];
      }
    }
  }
  __syncthreads();
  solve_f32_block(Ef, R11f, r, nc, Rd, dinv);
  const int64_t ldt = it.ldt > 0 ? it.ldt : r;
  for (int e = tid; e < r * nc; e += blockDim.x) {
    const int c = e / r, i = e % r;
    it.T[(int64_t)(c0 + c) * ldt + i] = (double)Tf[i * TS_COLS + c] + (double)Ef[i * TS_COLS + c];
  }
}

template <typename T>
ffc_status launch_trsm_t(const TrsmItem* items_dev, int n_items, int64_t total_tiles, int r_cap_max,
                         cudaStream_t st, bool refine = false) {
  if (r_cap_max > 1024) {
    set_error("trsm: rank cap %d exceeds 1024", r_cap_max);
    return FFC_E_INVALID;
  }
  finalize_kernel<T><<<n_items, 256, 0, st>>>(items_dev);
  FFC_CUDA(cudaGetLastError());
  if (total_tiles <= 0) return FFC_OK;
  const size_t smem = (size_t)std::max(r_cap_max, 1) * TS_COLS * sizeof(double);   // FP64 tile, or two FP32 ones
  if (refine) {
    FFC_CUDA(cudaFuncSetAttribute(trsm_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    trsm_refine_kernel<<<(unsigned)total_tiles, TR_THREADS, smem, st>>>(items_dev, n_items);
    FFC_CUDA(cudaGetLastError());
    return FFC_OK;
  }
  FFC_CUDA(cudaFuncSetAttribute(trsm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  trsm_kernel<T><<<(unsigned)total_tiles, 256, smem, st>>>(items_dev, n_items);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace

int64_t trsm_tiles(int64_t n) { return (n + TS_COLS - 1) / TS_COLS; }

ffc_status launch_trsm_batched(int precision, const TrsmItem* items_dev, int n_items, int64_t total_tiles,
                               int r_cap_max, cudaStream_t st, int solve) {
  if (n_items <= 0) return FFC_OK;
  if (precision == FFC_MIXED)
    return launch_trsm_t<float>(items_dev, n_items, total_tiles, r_cap_max, st, solve != FFC_SOLVE_FP64);
  return launch_trsm_t<double>(items_dev, n_items, total_tiles, r_cap_max, st);
}

}  // namespace ffc
