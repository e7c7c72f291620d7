// Full-block ID error ||K - K(:,J) P||_F / ||K||_F (§4.1.3, step 4), FP64.
//
// K_ij = K(Y[rows_i], X_j) over all m target rows is never stored: each CTA
// takes a 64-row x 64-column tile of the non-skeleton columns, accumulates
// K(rows, J) T(:, cols) over the skeleton in 16-wide chunks staged through
// shared memory (kernel values of the skeleton columns are evaluated on the
// fly), subtracts it from the directly evaluated K(rows, cols) and sums the
// squares. Skeleton columns are reproduced exactly by the ID (P contains
// I_r), so they contribute to ||K||_F only. Per-CTA partial sums are added
// on the host in a fixed order.
#include <algorithm>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int ET = 64, EK = 16, ERR_THREADS = 256;

template <typename TP, int KIND>
__device__ __forceinline__ double kval(const TP* y, const TP* x, int d, ffc_kernel kp, double ln_rmin) {
  double acc = 0.0;
  if constexpr (KIND == FFC_POLYNOMIAL) {
    for (int k = 0; k < d; ++k) acc = fma(ld_point(y + k), ld_point(x + k), acc);
    return pow(acc / kp.h + kp.c, (double)kp.p);
  } else {
    for (int k = 0; k < d; ++k) {
      double df = ld_point(y + k) - ld_point(x + k);
      acc = fma(df, df, acc);
    }
    if constexpr (KIND == FFC_GAUSSIAN) return exp(-acc / (2.0 * kp.h * kp.h));
    else return exp(-(double)(d - 2) * (0.5 * log(acc) - ln_rmin));
  }
}

template <typename TP>
__global__ void min_d2_kernel(const TP* __restrict__ Y, const int64_t* rows, int64_t m, const TP* __restrict__ X,
                              int64_t n, int d, double* out) {
  double mn = INFINITY;
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % m, j = e / m;
    const TP* y = Y + (rows ? rows[i] : i) * (int64_t)d;
    const TP* x = X + j * (int64_t)d;
    double acc = 0.0;
    for (int k = 0; k < d; ++k) {
      double df = ld_point(y + k) - ld_point(x + k);
      acc = fma(df, df, acc);
    }
    mn = fmin(mn, acc);
  }
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0 && mn < INFINITY)
    atomicMin(reinterpret_cast<unsigned long long*>(out), (unsigned long long)__double_as_longlong(mn));
}

template <typename TP, int KIND>
__global__ void __launch_bounds__(ERR_THREADS)
id_error_kernel(const TP* __restrict__ Y, const int64_t* __restrict__ rows, int64_t m,
                const TP* __restrict__ X, int64_t n, int d, ffc_kernel kp, const int32_t* __restrict__ skel,
                const double* __restrict__ T, int64_t ldt, int64_t r, const double* min_d2, double* partial) {
  __shared__ double ks[ET][EK + 1];   // K(rows tile, skeleton chunk)
  __shared__ double ts[EK][ET + 1];   // T(skeleton chunk, cols tile)
  __shared__ double red_num[ERR_THREADS / 32], red_den[ERR_THREADS / 32];
  const int64_t nr = n - r;
  const int64_t row_tiles = (m + ET - 1) / ET;
  const int64_t i0 = (blockIdx.x % row_tiles) * ET;
  const int64_t c0 = (blockIdx.x / row_tiles) * ET;
  const int tid = threadIdx.x;
  const int ti = tid % 16, tj = tid / 16;      // 4x4 outputs per thread: rows ti+16a, cols tj+16b
  const double ln_rmin = (KIND == FFC_LAPLACE) ? 0.5 * log(*min_d2) : 0.0;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  double den = 0.0, num = 0.0;
  for (int64_t k0 = 0; k0 < r; k0 += EK) {
    for (int e = tid; e < ET * EK; e += ERR_THREADS) {
      const int ii = e % ET, kk = e / ET;
      double v = 0.0;
      if (i0 + ii < m && k0 + kk < r) {
        const TP* y = Y + (rows ? rows[i0 + ii] : i0 + ii) * (int64_t)d;
        const TP* x = X + (int64_t)skel[k0 + kk] * d;
        v = kval<TP, KIND>(y, x, d, kp, ln_rmin);
        if (c0 == 0) den = fma(v, v, den);       // skeleton columns, counted once per row tile
      }
      ks[ii][kk] = v;
    }
    for (int e = tid; e < EK * ET; e += ERR_THREADS) {
      const int kk = e / ET, cc = e % ET;
      double v = 0.0;
      if (k0 + kk < r && c0 + cc < nr) v = T[(k0 + kk) + (c0 + cc) * ldt];
      ts[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < EK; ++kk) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const double kv = ks[ti + 16 * a][kk];
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(kv, ts[kk][tj + 16 * b], acc[a][b]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + ti + 16 * a;
    if (i >= m) continue;
    const TP* y = Y + (rows ? rows[i] : i) * (int64_t)d;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t c = c0 + tj + 16 * b;
      if (c >= nr) continue;
      const TP* x = X + (int64_t)skel[r + c] * d;
      const double kv = kval<TP, KIND>(y, x, d, kp, ln_rmin);
      const double e = kv - acc[a][b];
      num = fma(e, e, num);
      den = fma(kv, kv, den);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((tid & 31) == 0) { red_num[tid >> 5] = num; red_den[tid >> 5] = den; }
  __syncthreads();
  if (tid == 0) {
    double sn = 0.0, sd = 0.0;
    for (int w = 0; w < ERR_THREADS / 32; ++w) { sn += red_num[w]; sd += red_den[w]; }
    partial[2 * blockIdx.x] = sn;
    partial[2 * blockIdx.x + 1] = sd;
  }
}

template <typename TP>
ffc_status launch_err_t(ffc_kernel k, const TP* Y, const int64_t* rows, int64_t m, const TP* X, int64_t n,
                        int d, const int32_t* skel, const double* T, int64_t ldt, int64_t r, double* partial,
                        int64_t blocks, double* min_d2, cudaStream_t st) {
  if (k.kind == FFC_LAPLACE) {
    double inf = INFINITY;
    FFC_CUDA(cudaMemcpyAsync(min_d2, &inf, sizeof(double), cudaMemcpyHostToDevice, st));
    int g = (int)std::min<int64_t>((m * n + 255) / 256, (int64_t)sm_count() * 8);
    min_d2_kernel<TP><<<std::max(g, 1), 256, 0, st>>>(Y, rows, m, X, n, d, min_d2);
    id_error_kernel<TP, FFC_LAPLACE><<<(unsigned)blocks, ERR_THREADS, 0, st>>>(Y, rows, m, X, n, d, k, skel, T,
                                                                              ldt, r, min_d2, partial);
  } else if (k.kind == FFC_GAUSSIAN) {
    id_error_kernel<TP, FFC_GAUSSIAN><<<(unsigned)blocks, ERR_THREADS, 0, st>>>(Y, rows, m, X, n, d, k, skel, T,
                                                                               ldt, r, min_d2, partial);
  } else {
    id_error_kernel<TP, FFC_POLYNOMIAL><<<(unsigned)blocks, ERR_THREADS, 0, st>>>(Y, rows, m, X, n, d, k, skel,
                                                                                 T, ldt, r, min_d2, partial);
  }
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace

int64_t id_error_blocks(int64_t m, int64_t n, int64_t r) {
  int64_t nr = std::max<int64_t>(n - r, 1);
  return ((m + ET - 1) / ET) * ((nr + ET - 1) / ET);
}

ffc_status launch_id_error(ffc_kernel k, const void* Y, int dtype, const int64_t* rows, int64_t m,
                           const void* X, int64_t n, int d, const int32_t* skel, const double* T,
                           int64_t ldt, int64_t r, double* partial, int64_t n_partial, double* min_d2_dev,
                           double* out_host_num, double* out_host_den, cudaStream_t st) {
  ffc_status stt;
  if (dtype == FFC_F64)
    stt = launch_err_t<double>(k, (const double*)Y, rows, m, (const double*)X, n, d, skel, T, ldt, r, partial,
                               n_partial, min_d2_dev, st);
  else
    stt = launch_err_t<float>(k, (const float*)Y, rows, m, (const float*)X, n, d, skel, T, ldt, r, partial,
                              n_partial, min_d2_dev, st);
  (void)out_host_num;
  (void)out_host_den;
  return stt;
}

}  // namespace ffc
