// Exact statistical leverage scores of the rows of a block K (m x n, FP64,
// column-major), the training targets of the learned proposal.
//
// §3, Def. "Statistical Leverage": with K = U Sigma V^T and a rank r, the
// score of row i is l_i = ||U_r(i, :)||^2 (the paper states it for A = K^T
// and the rows of V_r). r is the epsilon-rank (§4.1.3 step 1): the number of
// singular values >= eps * sigma_1.
//
// Route: G = K^T K (FP64, row chunks summed in a fixed order), G = V Lambda V^T
// by cyclic Jacobi rotations, sigma_k = sqrt(lambda_k), and
// l_i = || K(i, :) V_r Sigma_r^-1 ||^2, since U_r = K V_r Sigma_r^-1.
//
// Accuracy: eigenvalues of G carry an absolute error of a few eps ||G||, so
// the subspace of U_r is accurate to about eps sigma_1^2 / (sigma_r^2 -
// sigma_{r+1}^2) (Davis-Kahan); singular values below about 1e-7 sigma_1 are
// not resolved. Training targets need far less.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ffc_internal.cuh"

namespace ffc {

constexpr int GT = 64;               // Gram tile
constexpr int G_ROWS = 16;           // rows staged per step
constexpr int LEV_MAX_N = 1024;
constexpr int JAC_THREADS = 1024;
constexpr int JAC_MAX_SWEEPS = 40;

struct LevJob {
  double* G;         // n x n Gram matrix, overwritten by the eigenvalues
  double* V;         // n x n eigenvectors
  double* W;         // n x r: V_r Sigma_r^-1
  int* perm;         // eigenpairs by decreasing eigenvalue
  double* sigma;     // n singular values, decreasing
  int64_t* rank;     // device
  int32_t* sweeps;   // device
  int n, pad;
};

// Gpart[c] (n x n row-major) = K(rows of chunk c, :)^T K(rows of chunk c, :),
// computed for the upper tiles (ti <= tj) and mirrored.
__global__ void __launch_bounds__(256) gram_kernel(const double* __restrict__ K, int64_t m, int n, int64_t ldk,
                                                   int64_t chunk_rows, double* __restrict__ Gpart) {
  __shared__ double As[G_ROWS][GT];
  __shared__ double Bs[G_ROWS][GT];
  const int nt = (n + GT - 1) / GT;
  // blockIdx.x enumerates upper tile pairs, blockIdx.y the row chunk
  int ti = 0, rem = blockIdx.x;
  while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
  const int tj = ti + rem;
  const int64_t r0 = (int64_t)blockIdx.y * chunk_rows;
  const int64_t r1 = std::min<int64_t>(m, r0 + chunk_rows);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int64_t rb = r0; rb < r1; rb += G_ROWS) {
    for (int e = threadIdx.x; e < G_ROWS * GT; e += blockDim.x) {
      const int rr = e % G_ROWS, cc = e / G_ROWS;
      const int64_t row = rb + rr;
      const int ca = ti * GT + cc, cb = tj * GT + cc;
      As[rr][cc] = (row < r1 && ca < n) ? K[(int64_t)ca * ldk + row] : 0.0;
      Bs[rr][cc] = (row < r1 && cb < n) ? K[(int64_t)cb * ldk + row] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < G_ROWS; ++rr) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[rr][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[rr][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
  double* G = Gpart + (int64_t)blockIdx.y * n * n;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int ca = ti * GT + tx + 16 * a, cb = tj * GT + ty + 16 * b;
      if (ca < n && cb < n) {
        G[(int64_t)ca * n + cb] = acc[a][b];
        if (ti != tj) G[(int64_t)cb * n + ca] = acc[a][b];
      }
    }
}

__global__ void gram_reduce_kernel(const double* __restrict__ Gpart, int chunks, int64_t nn, double* __restrict__ G) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += Gpart[(int64_t)c * nn + e];
  G[e] = s;
}

// Pair i of round k of the circle schedule over np (even) players.
__device__ __forceinline__ void round_pair(int np, int k, int i, int& p, int& q) {
  const int L = np - 1;
  if (i == 0) {
    p = 0;
    q = 1 + k % L;
  } else {
    p = 1 + (k + i) % L;
    q = 1 + (k - i + L) % L;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// Cyclic Jacobi on symmetric G (n x n row-major, overwritten by Lambda) with
// V = accumulated rotations. Rotation of pair (p, q) (Golub & Van Loan,
// "symSchur2"): tau = (g_qq - g_pp) / (2 g_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c, J = [c s; -s c] on (p, q);
// G <- J^T G J. A pair is skipped when |g_pq| <= 1e-15 sqrt(g_pp g_qq) or
// |g_pq| <= 1e-17 max_k g_kk (below the rounding of the Gram matrix itself).
// All pairs of a round are disjoint, so the update G'[P_i, P_k] =
// J_i^T G[P_i, P_k] J_k of every 2 x 2 block reads only that block.
__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(const LevJob* jobs) {
  const LevJob& jb = jobs[blockIdx.x];
  double* __restrict__ G = jb.G;
  double* __restrict__ V = jb.V;
  const int n = jb.n;
  int32_t* sweeps_out = jb.sweeps;
  __shared__ double cs[LEV_MAX_N / 2], sn[LEV_MAX_N / 2];
  __shared__ int pp[LEV_MAX_N / 2], qq[LEV_MAX_N / 2];
  __shared__ unsigned char act[LEV_MAX_N / 2];
  __shared__ int rotated;
  __shared__ double gmax;
  const int np = n + (n & 1);
  const int half = np / 2;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x)
    V[e] = (e / n == e % n) ? 1.0 : 0.0;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, fabs(G[(int64_t)k * n + k]));
    gmax = mx;
  }
  __syncthreads();
  const double floor_abs = 1e-17 * gmax;
  int sweep = 0;
  bool converged = (n <= 1);
  for (; sweep < JAC_MAX_SWEEPS && !converged; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int k = 0; k < np - 1; ++k) {
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        int p, q;
        round_pair(np, k, i, p, q);
        double c = 1.0, s = 0.0;
        unsigned char a = 0;
        if (q < n) {
          const double gpp = G[(int64_t)p * n + p], gqq = G[(int64_t)q * n + q], gpq = G[(int64_t)p * n + q];
          if (fabs(gpq) > floor_abs && fabs(gpq) > 1e-15 * sqrt(fabs(gpp) * fabs(gqq))) {
            const double tau = (gqq - gpp) / (2.0 * gpq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            a = 1;
            atomicAdd(&rotated, 1);
          }
        }
        cs[i] = c; sn[i] = s; pp[i] = p; qq[i] = q; act[i] = a;
      }
      __syncthreads();
      // blocks (i, j) of pairs; the dummy index n (odd n) is never touched
      const int64_t nb = (int64_t)half * half;
      for (int64_t e = threadIdx.x; e < nb; e += blockDim.x) {
        const int i = (int)(e / half), j = (int)(e % half);
        if (!act[i] && !act[j]) continue;
        const int p1 = pp[i], q1 = qq[i], p2 = pp[j], q2 = qq[j];
        const double c1 = cs[i], s1 = sn[i], c2 = cs[j], s2 = sn[j];
        const bool q1ok = q1 < n, q2ok = q2 < n;
        const double a00 = G[(int64_t)p1 * n + p2];
        const double a01 = q2ok ? G[(int64_t)p1 * n + q2] : 0.0;
        const double a10 = q1ok ? G[(int64_t)q1 * n + p2] : 0.0;
        const double a11 = (q1ok && q2ok) ? G[(int64_t)q1 * n + q2] : 0.0;
        // H = B J2: columns (p2, q2)
        const double h00 = c2 * a00 - s2 * a01, h01 = s2 * a00 + c2 * a01;
        const double h10 = c2 * a10 - s2 * a11, h11 = s2 * a10 + c2 * a11;
        // J1^T H: rows (p1, q1)
        double b00 = c1 * h00 - s1 * h10, b01 = c1 * h01 - s1 * h11;
        double b10 = s1 * h00 + c1 * h10, b11 = s1 * h01 + c1 * h11;
        if (i == j && act[i]) { b01 = 0.0; b10 = 0.0; }
        G[(int64_t)p1 * n + p2] = b00;
        if (q2ok) G[(int64_t)p1 * n + q2] = b01;
        if (q1ok) G[(int64_t)q1 * n + p2] = b10;
        if (q1ok && q2ok) G[(int64_t)q1 * n + q2] = b11;
      }
      // V <- V J
      for (int64_t e = threadIdx.x; e < (int64_t)n * half; e += blockDim.x) {
        const int row = (int)(e / half), i = (int)(e % half);
        if (!act[i]) continue;
        const int p = pp[i], q = qq[i];
        const double c = cs[i], s = sn[i];
        const double vp = V[(int64_t)row * n + p], vq = V[(int64_t)row * n + q];
        V[(int64_t)row * n + p] = c * vp - s * vq;
        V[(int64_t)row * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    converged = (rotated == 0);
    __syncthreads();
  }
  if (threadIdx.x == 0) *sweeps_out = converged ? sweep : -1;
}

// Order the eigenpairs by decreasing eigenvalue (ties: lower index first),
// sigma_out[k] = sqrt(max(lambda, 0)), rank r, and W = V_r Sigma_r^-1 (n x r).
__global__ void __launch_bounds__(1024) eig_order_kernel(const LevJob* jobs, double eps, int64_t r_fixed) {
  const LevJob& jb = jobs[blockIdx.x];
  const double* __restrict__ G = jb.G;
  const double* __restrict__ V = jb.V;
  const int n = jb.n;
  double* __restrict__ sigma = jb.sigma;
  int* __restrict__ perm = jb.perm;
  double* __restrict__ W = jb.W;
  int64_t* __restrict__ rank_out = jb.rank;
  __shared__ int r_sh;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const double la = G[(int64_t)a * n + a];
    int rk = 0;
    for (int b = 0; b < n; ++b) {
      const double lb = G[(int64_t)b * n + b];
      rk += (lb > la) || (lb == la && b < a);
    }
    perm[rk] = a;
    sigma[rk] = sqrt(fmax(la, 0.0));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    if (r_fixed > 0) {
      r = (int)std::min<int64_t>(r_fixed, n);
    } else if (n > 0 && sigma[0] > 0.0) {
      while (r < n && sigma[r] >= eps * sigma[0]) ++r;
    }
    while (r > 0 && !(sigma[r - 1] > 0.0)) --r;   // never divide by a zero singular value
    r_sh = r;
    *rank_out = r;
  }
  __syncthreads();
  const int r = r_sh;
  for (int64_t e = threadIdx.x; e < (int64_t)n * r; e += blockDim.x) {
    const int j = (int)(e / r), k = (int)(e % r);
    W[e] = V[(int64_t)j * n + perm[k]] / sigma[k];
  }
}

// lev[i] = sum_k (K(i, :) W(:, k))^2, 64 rows per CTA, W in 64-column tiles.
__global__ void __launch_bounds__(256) leverage_kernel(const double* __restrict__ K, int64_t m, int n, int64_t ldk,
                                                       const double* __restrict__ W, const int64_t* __restrict__ rank,
                                                       double* __restrict__ lev) {
  const int r = (int)*rank;
  __shared__ double Ks[G_ROWS][GT];   // [j][row]
  __shared__ double Ws[G_ROWS][GT];   // [j][col]
  __shared__ double red[GT][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * GT;
  double rowsum[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < r; k0 += GT) {
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int j0 = 0; j0 < n; j0 += G_ROWS) {
      for (int e = threadIdx.x; e < G_ROWS * GT; e += blockDim.x) {
        const int rr = e % GT, jj = e / GT;
        const int64_t row = row0 + rr;
        const int j = j0 + jj;
        Ks[jj][rr] = (row < m && j < n) ? K[(int64_t)j * ldk + row] : 0.0;
        const int col = k0 + rr;
        Ws[jj][rr] = (j < n && col < r) ? W[(int64_t)j * r + col] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int jj = 0; jj < G_ROWS; ++jj) {
        double kv[4], wv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) kv[a] = Ks[jj][ty + 16 * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) wv[b] = Ws[jj][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(kv[a], wv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) rowsum[a] += acc[a][b] * acc[a][b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) red[ty + 16 * a][tx] = rowsum[a];
  __syncthreads();
  if (threadIdx.x < GT) {
    const int64_t row = row0 + threadIdx.x;
    double s = 0.0;
    for (int c = 0; c < 16; ++c) s += red[threadIdx.x][c];
    if (row < m) lev[row] = s;
  }
}

ffc_status launch_leverage_batched(int B, const double* const* K, const int64_t* m, const int64_t* n,
                                   const int64_t* ldk, double eps, int64_t r_fixed, double* const* lev,
                                   double* const* sigma, int64_t* rank_host, int32_t* sweeps_host, cudaStream_t st) {
  FFC_REQUIRE(B >= 1, "leverage: need B >= 1");
  for (int b = 0; b < B; ++b) {
    FFC_REQUIRE(n[b] >= 1 && n[b] <= LEV_MAX_N, "leverage: need 1 <= n <= %d", LEV_MAX_N);
    FFC_REQUIRE(m[b] >= 1 && ldk[b] >= m[b], "leverage: need m >= 1 and ldk >= m");
    FFC_REQUIRE(K[b] && (!lev || lev[b]) && sigma[b], "leverage: null pointer");
  }
  // per block: G, V, W (n^2 each), perm (n), rank, sweeps; one Gram partial buffer shared in stream order
  size_t per = 0, gpart = 0;
  std::vector<size_t> off(B);
  std::vector<int64_t> chunks(B), crow(B);
  for (int b = 0; b < B; ++b) {
    const int64_t nn = n[b] * n[b];
    off[b] = per;
    per += ((3 * nn * sizeof(double) + n[b] * sizeof(int) + 64) + 255) & ~size_t(255);
    const int nt = (int)((n[b] + GT - 1) / GT);
    const int pairs = nt * (nt + 1) / 2;
    int64_t c = std::max<int64_t>(1, (4LL * sm_count()) / pairs);
    c = std::min<int64_t>(c, std::max<int64_t>(1, m[b] / 1024));
    c = std::min<int64_t>(c, 65535);
    chunks[b] = c;
    crow[b] = (m[b] + c - 1) / c;
    gpart = std::max(gpart, (size_t)(c * nn) * sizeof(double));
  }
  const size_t jobs_off = (per + gpart + 255) & ~size_t(255);
  char* ws = nullptr;
  FFC_CUDA(cudaMallocAsync((void**)&ws, jobs_off + sizeof(LevJob) * B + (size_t)B * 16, st));
  double* Gpart = reinterpret_cast<double*>(ws + per);
  LevJob* d_jobs = reinterpret_cast<LevJob*>(ws + jobs_off);
  int64_t* ranks = reinterpret_cast<int64_t*>(d_jobs + B);
  int32_t* sweeps = reinterpret_cast<int32_t*>(ranks + B);
  std::vector<LevJob> jobs(B);
  for (int b = 0; b < B; ++b) {
    const int64_t nn = n[b] * n[b];
    LevJob& j = jobs[b];
    j.G = reinterpret_cast<double*>(ws + off[b]);
    j.V = j.G + nn;
    j.W = j.V + nn;
    j.perm = reinterpret_cast<int*>(j.W + nn);
    j.n = (int)n[b];
    j.sigma = sigma[b];
    j.rank = ranks + b;
    j.sweeps = sweeps + b;
  }
  FFC_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(LevJob) * B, cudaMemcpyHostToDevice, st));
  for (int b = 0; b < B; ++b) {
    const int nt = (int)((n[b] + GT - 1) / GT);
    const int pairs = nt * (nt + 1) / 2;
    const int64_t nn = n[b] * n[b];
    gram_kernel<<<dim3(pairs, (unsigned)chunks[b]), 256, 0, st>>>(K[b], m[b], (int)n[b], ldk[b], crow[b], Gpart);
    gram_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(Gpart, (int)chunks[b], nn, jobs[b].G);
  }
  jacobi_kernel<<<B, JAC_THREADS, 0, st>>>(d_jobs);
  eig_order_kernel<<<B, 1024, 0, st>>>(d_jobs, eps, r_fixed);
  for (int b = 0; lev && b < B; ++b)
    leverage_kernel<<<(unsigned)((m[b] + GT - 1) / GT), 256, 0, st>>>(K[b], m[b], (int)n[b], ldk[b], jobs[b].W,
                                                                    jobs[b].rank, lev[b]);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { cudaFreeAsync(ws, st); return cuda_fail(e, "leverage kernels"); }
  std::vector<int32_t> sw(B);
  FFC_CUDA(cudaMemcpyAsync(rank_host, ranks, sizeof(int64_t) * B, cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaMemcpyAsync(sw.data(), sweeps, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
  FFC_CUDA(cudaFreeAsync(ws, st));
  FFC_CUDA(cudaStreamSynchronize(st));
  ffc_status rc = FFC_OK;
  for (int b = 0; b < B; ++b) {
    if (sweeps_host) sweeps_host[b] = sw[b];
    if (sw[b] < 0 && rc == FFC_OK) {
      set_error("leverage: Jacobi did not converge in %d sweeps (block %d)", JAC_MAX_SWEEPS, b);
      rc = FFC_E_TOL_NOT_REACHED;
    }
  }
  return rc;
}

}  // namespace ffc

extern "C" ffc_status ffc_spectrum(const double* K_dev, int64_t m, int64_t n, int64_t ldk, double eps, double* sigma_dev,
                                   int64_t* rank_host, void* stream) {
  FFC_REQUIRE(m >= 1 && n >= 1 && ldk >= m, "ffc_spectrum: need m, n >= 1 and ldk >= m");
  FFC_REQUIRE(n <= 1024, "ffc_spectrum: n = %lld exceeds 1024 columns", (long long)n);
  FFC_REQUIRE(K_dev && sigma_dev && rank_host && eps >= 0.0, "ffc_spectrum: null pointer or eps < 0");
  const double* Kp[1] = {K_dev};
  const int64_t mm[1] = {m}, nn[1] = {n}, ll[1] = {ldk};
  double* sp[1] = {sigma_dev};
  int32_t sweeps = 0;
  return ffc::launch_leverage_batched(1, Kp, mm, nn, ll, eps, 0, nullptr, sp, rank_host, &sweeps,
                                      ffc::as_stream(stream));
}
