// The outgoing representation and its use (§2.1.3, after the ID theorem):
// skeleton charges q~ = P q, potentials u = C q~ (C = K(:, J)) against the
// direct u = K q (§1, eq. e:sum), and the evaluation of the potential at every
// point of a compressed tree.
//
// Tree evaluation. A target y takes node b's representation when y lies in
// b's far field (outside b, at least xi rho_b from its centroid, §4.1 setup)
// and in the far field of none of b's ancestors at level >= min_level; a leaf
// reached with no far node on its path is summed directly without y's own
// point. Each CTA owns 128 consecutive targets in tree order (spatial
// neighbours, so their paths mostly agree) and walks the tree depth first
// from the min_level nodes; each thread keeps a bit per level of the current
// path telling whether its target was far there, so a target covered by an
// ancestor skips the subtree while the others descend. The source points of
// a node (its skeleton, or all of its points) are staged through shared
// memory in chunks and shared by the CTA's far targets. FP64 throughout.
#include <algorithm>
#include <cmath>

#include "ffc_internal.cuh"

namespace ffc {
const ffc_params* tree_result_params(const ffc_tree_result* r);
int64_t tree_result_first_node(const ffc_tree_result* r);
}  // namespace ffc

using namespace ffc;

namespace {

constexpr int AP_THREADS = 128;     // targets per CTA of the tree evaluation
constexpr int CH_THREADS = 256;     // charges kernel
constexpr int STACK_MAX = 96;       // DFS stack of the tree walk (min_level nodes + 2 per level)

// Kernel value K(y, x) exp(-log_scale) from the squared distance (Gaussian, Laplace) or the
// inner product (polynomial), FP64.
__device__ __forceinline__ double kval(const ffc_kernel& k, int d, double dd, double dot, double log_scale) {
  if (k.kind == FFC_GAUSSIAN) return exp(-dd / (2.0 * k.h * k.h) - log_scale);
  if (k.kind == FFC_LAPLACE) return exp(-0.5 * (double)(d - 2) * log(dd) - log_scale);
  const double b = dot / k.h + k.c;
  double v = 1.0;
  for (int e = 0; e < k.p; ++e) v *= b;
  return v * exp(-log_scale);
}

// q~ = q[skel[0:r]] + T q[skel[r:n]] for one item: T (r x (n - r)) column c at T + c ldt.
struct ChargeItem {
  const int32_t* skel;
  const double* T;
  int64_t ldt;
  int32_t r, n;
  const double* q;     // n charges (column 0; column c at q + c ldq)
  int64_t ldq;
  double* qt;          // r charges (column c at qt + c ldqt)
  int64_t ldqt;
};

// One CTA per (item, right-hand side): warps split the n - r columns of T, lanes take 32
// skeleton rows at a time, partial sums are added in a fixed order.
__device__ void charges_body(const ChargeItem& it, int rhs) {
  __shared__ double part[CH_THREADS / 32][32];
  const int r = it.r, nr = it.n - it.r;
  if (r <= 0) return;
  const double* q = it.q + (int64_t)rhs * it.ldq;
  double* qt = it.qt + (int64_t)rhs * it.ldqt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = CH_THREADS / 32;
  const int c_per = (nr + NW - 1) / NW;
  const int c0 = warp * c_per, c1 = min(nr, c0 + c_per);
  for (int k0 = 0; k0 < r; k0 += 32) {
    const int k = k0 + lane;
    double acc = 0.0;
    if (k < r) {
      for (int c = c0; c < c1; ++c) acc = fma(__ldg(it.T + (int64_t)c * it.ldt + k), __ldg(q + it.skel[r + c]), acc);
    }
    part[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && k < r) {
      double s = __ldg(q + it.skel[k]);
      for (int w = 0; w < NW; ++w) s += part[w][lane];
      qt[k] = s;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(CH_THREADS) charges_kernel(ChargeItem it) { charges_body(it, blockIdx.y); }

__device__ __forceinline__ bool usable_id(int status, int s) {
  return (status == FFC_OK || status == FFC_E_TOL_NOT_REACHED) && s > 0;
}

// The charges of the ID columns of the output nodes [o0, o1) (one level), into qc at skel_off: the
// points' charges q[begin + cols[c]], or, nested above the leaves, the children's skeleton charges (a
// child without a usable ID: its points' charges), in the order of the columns.
__global__ void gather_qcols_kernel(int64_t o0, int64_t first, int nested_parent, int64_t rcap,
                                    const int64_t* __restrict__ begin, const int64_t* __restrict__ count,
                                    const int32_t* __restrict__ rank, const int32_t* __restrict__ status,
                                    const int32_t* __restrict__ sv, const int64_t* __restrict__ skel_off,
                                    const int32_t* __restrict__ ncols, const int32_t* __restrict__ cols,
                                    const double* __restrict__ q, const double* __restrict__ qt,
                                    double* __restrict__ qc) {
  const int64_t o = o0 + blockIdx.x, b = first + o;
  double* dst = qc + skel_off[o];
  if (!nested_parent) {
    for (int c = threadIdx.x; c < ncols[o]; c += blockDim.x) dst[c] = q[begin[b] + cols[skel_off[o] + c]];
    return;
  }
  int64_t c = 0;
  for (int64_t ch = 2 * b + 1; ch <= 2 * b + 2; ++ch) {
    const int64_t oc = ch - first;
    if (usable_id(status[oc], sv[oc])) {
      for (int k = threadIdx.x; k < rank[oc]; k += blockDim.x) dst[c + k] = qt[oc * rcap + k];
      c += rank[oc];
    } else {
      for (int64_t j = threadIdx.x; j < count[ch]; j += blockDim.x) dst[c + j] = q[begin[ch] + j];
      c += count[ch];
    }
  }
}

// Output nodes [o0, o1): block i takes node o0 + i, its packed T (ld r) and its column charges (qc at
// skel_off); q~ goes to qt + o rcap.
__global__ void __launch_bounds__(CH_THREADS)
charges_tree_kernel(int64_t o0, int64_t rcap, const int32_t* __restrict__ rank, const int32_t* __restrict__ status,
                    const int32_t* __restrict__ sv, const int64_t* __restrict__ skel_off,
                    const int32_t* __restrict__ ncols, const int32_t* __restrict__ skel,
                    const int64_t* __restrict__ T_off, const double* __restrict__ T, const double* __restrict__ qc,
                    double* __restrict__ qt) {
  const int64_t i = o0 + blockIdx.x;
  if (!usable_id(status[i], sv[i])) return;   // such a node is evaluated from its sources
  const int r = rank[i];
  ChargeItem it{skel + skel_off[i], T + T_off[i], r > 0 ? r : 1, r, ncols[i], qc + skel_off[i], 0, qt + i * rcap, 0};
  charges_body(it, 0);
}

// Potential of one chunk of staged sources at one target: sum_c K(y, x_c) w_c, skipping the
// source at position `self` (a position in the chunk, or -1).
template <typename TP>
__device__ __forceinline__ double chunk_sum(const ffc_kernel& k, int d, const TP* __restrict__ y,
                                            const double* __restrict__ xs, const double* __restrict__ ws, int kp,
                                            int self, double log_scale) {
  double acc = 0.0;
  for (int c = 0; c < kp; ++c) {
    const double* x = xs + (int64_t)c * d;
    double dd = 0.0, dot = 0.0;
    if (k.kind == FFC_POLYNOMIAL) {
      for (int j = 0; j < d; ++j) dot = fma(ld_point(y + j), x[j], dot);
    } else {
      for (int j = 0; j < d; ++j) {
        const double df = ld_point(y + j) - x[j];
        dd = fma(df, df, dd);
      }
    }
    if (c != self) acc = fma(kval(k, d, dd, dot, log_scale), ws[c], acc);
  }
  return acc;
}

// ffc_potential: one thread per target row; sources (all n, or the listed columns) staged in chunks.
template <typename TP>
__global__ void __launch_bounds__(AP_THREADS)
potential_kernel(ffc_kernel k, const TP* __restrict__ Y, const int64_t* __restrict__ rows, int64_t m,
                 const TP* __restrict__ X, int d, const int32_t* __restrict__ cols, int64_t nc,
                 const double* __restrict__ w, double log_scale, int kp_max, double* __restrict__ u) {
  extern __shared__ double psm[];
  double* xs = psm;
  double* ws = psm + (int64_t)kp_max * d;
  const int64_t i = (int64_t)blockIdx.x * AP_THREADS + threadIdx.x;
  const bool live = i < m;
  const TP* y = Y + (live ? (rows ? rows[i] : i) : 0) * (int64_t)d;
  double acc = 0.0;
  for (int64_t c0 = 0; c0 < nc; c0 += kp_max) {
    const int kp = (int)std::min<int64_t>(kp_max, nc - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < kp * d; e += AP_THREADS) {
      const int c = e / d, j = e % d;
      const int64_t src = cols ? cols[c0 + c] : c0 + c;
      xs[e] = ld_point(X + src * d + j);
    }
    for (int c = threadIdx.x; c < kp; c += AP_THREADS) ws[c] = w[c0 + c];
    __syncthreads();
    if (live) acc += chunk_sum(k, d, y, xs, ws, kp, -1, log_scale);
  }
  if (live) u[i] = acc;
}

// Tree evaluation (see the file comment). node_out[b - first]: output index of heap node b.
struct TreeApplyArgs {
  ffc_kernel k;
  int d, depth, min_level, mode, near_field;
  int64_t N, first, rcap;
  double xi, log_scale;
  const int64_t* begin;
  const int64_t* count;
  const double* centroid;
  const double* radius;
  const int32_t* rank;      // per output node
  const int32_t* status;
  const int64_t* skel_off;
  const int32_t* skel;
  const int32_t* cols;      // the ID's columns (node-local points) at skel_off
  const int32_t* sv;        // rows sampled per node (0: no ID)
  const double* q;          // N charges, tree order
  const double* qt;         // skeleton charges, node i at qt + i rcap
  double* u;
};

template <typename TP>
__global__ void __launch_bounds__(AP_THREADS) tree_apply_kernel(TreeApplyArgs a, const TP* __restrict__ X,
                                                                int kp_max) {
  extern __shared__ double tsm[];
  double* xs = tsm;
  double* ws = tsm + (int64_t)kp_max * a.d;
  __shared__ int64_t stack[STACK_MAX];
  __shared__ int sp;
  const int d = a.d;
  const int64_t t = (int64_t)blockIdx.x * AP_THREADS + threadIdx.x;
  const bool live = t < a.N;
  const TP* y = X + (live ? t : 0) * (int64_t)d;
  double acc = 0.0;
  unsigned far_bits = 0u;        // bit l: the target was far at the current path's level-l node
  if (threadIdx.x == 0) {
    sp = 0;
    const int64_t lo = (1ll << a.min_level) - 1, hi = (1ll << (a.min_level + 1)) - 2;
    for (int64_t b = hi; b >= lo; --b) stack[sp++] = b;
  }
  __syncthreads();
  while (true) {
    const int top = sp;
    if (top == 0) break;
    const int64_t b = stack[top - 1];
    __syncthreads();
    if (threadIdx.x == 0) sp = top - 1;
    const int lev = 63 - __clzll((unsigned long long)(b + 1));
    const int64_t bg = a.begin[b], n = a.count[b];
    far_bits &= (1u << lev) - 1u;
    const bool covered = (far_bits >> a.min_level) != 0u;
    bool far = false;
    if (live && !covered && !(t >= bg && t < bg + n)) {
      const double* xc = a.centroid + b * d;
      double dd = 0.0;
      for (int j = 0; j < d; ++j) {
        const double df = ld_point(y + j) - __ldg(xc + j);
        dd = fma(df, df, dd);
      }
      const double thr = a.xi * a.radius[b];
      far = dd >= thr * thr;
    }
    if (far) far_bits |= 1u << lev;
    const bool leaf = lev == a.depth;
    const bool need = live && !covered && !far && !leaf;
    const bool nearl = live && !covered && !far && leaf && a.near_field;
    const int any_far = __syncthreads_or(far);
    const int any_need = __syncthreads_or(need);
    const int any_near = __syncthreads_or(nearl);
    if (any_far) {
      const int64_t o = b - a.first;
      const int st = a.status[o];
      const bool skel_ok = a.mode == FFC_APPLY_SKELETON && usable_id(st, a.sv[o]);
      const int64_t ns = skel_ok ? a.rank[o] : n;
      const int32_t* sk = a.skel + a.skel_off[o];
      const int32_t* cl = a.cols + a.skel_off[o];
      const double* w = skel_ok ? a.qt + o * a.rcap : a.q + bg;
      for (int64_t c0 = 0; c0 < ns; c0 += kp_max) {
        const int kp = (int)std::min<int64_t>(kp_max, ns - c0);
        for (int e = threadIdx.x; e < kp * d; e += AP_THREADS) {
          const int c = e / d, j = e % d;
          const int64_t src = bg + (skel_ok ? cl[sk[c0 + c]] : c0 + c);
          xs[e] = ld_point(X + src * d + j);
        }
        for (int c = threadIdx.x; c < kp; c += AP_THREADS) ws[c] = w[c0 + c];
        __syncthreads();
        if (far) acc += chunk_sum(a.k, d, y, xs, ws, kp, -1, a.log_scale);
        __syncthreads();
      }
    }
    if (any_near) {
      for (int64_t c0 = 0; c0 < n; c0 += kp_max) {
        const int kp = (int)std::min<int64_t>(kp_max, n - c0);
        for (int e = threadIdx.x; e < kp * d; e += AP_THREADS) {
          const int c = e / d, j = e % d;
          xs[e] = ld_point(X + (bg + c0 + c) * d + j);
        }
        for (int c = threadIdx.x; c < kp; c += AP_THREADS) ws[c] = a.q[bg + c0 + c];
        __syncthreads();
        if (nearl) {
          const int64_t self = t - (bg + c0);
          acc += chunk_sum(a.k, d, y, xs, ws, kp, (self >= 0 && self < kp) ? (int)self : -1, a.log_scale);
        }
        __syncthreads();
      }
    }
    if (any_need && threadIdx.x == 0 && sp + 2 <= STACK_MAX) {
      stack[sp++] = 2 * b + 2;
      stack[sp++] = 2 * b + 1;
    }
    __syncthreads();
  }
  if (live) a.u[t] = acc;
}

// coordinates staged per chunk: at most 64 points or 64 KB of doubles
int chunk_points(int d) { return std::max(1, std::min(64, 8192 / std::max(d, 1))); }

size_t chunk_smem(int d) { return (size_t)chunk_points(d) * (d + 1) * sizeof(double); }

template <typename TP>
ffc_status launch_potential_t(ffc_kernel k, const void* Y, const int64_t* rows, int64_t m, const void* X, int d,
                              const int32_t* cols, int64_t nc, const double* w, double log_scale, double* u,
                              cudaStream_t st) {
  const size_t smem = chunk_smem(d);
  FFC_CUDA(cudaFuncSetAttribute(potential_kernel<TP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  potential_kernel<TP><<<(unsigned)((m + AP_THREADS - 1) / AP_THREADS), AP_THREADS, smem, st>>>(
      k, (const TP*)Y, rows, m, (const TP*)X, d, cols, nc, w, log_scale, chunk_points(d), u);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

}  // namespace

extern "C" {

ffc_status ffc_skeleton_charges(const int32_t* skel_perm_dev, const double* T_dev, int64_t ldt, int64_t r, int64_t n,
                                const double* q_dev, int64_t ldq, int64_t nrhs, double* qt_dev, int64_t ldqt,
                                void* stream) {
  FFC_REQUIRE(n >= 0 && r >= 0 && r <= n && nrhs >= 0, "ffc_skeleton_charges: need 0 <= r <= n, nrhs >= 0");
  FFC_REQUIRE(r <= (1 << 30) && n <= (1 << 30), "ffc_skeleton_charges: sizes out of range");
  FFC_REQUIRE(ldt >= std::max<int64_t>(r, 1) && ldq >= std::max<int64_t>(n, 1) && ldqt >= std::max<int64_t>(r, 1),
              "ffc_skeleton_charges: need ldt >= r, ldq >= n, ldqt >= r");
  FFC_REQUIRE(nrhs <= 65535, "ffc_skeleton_charges: at most 65535 right-hand sides");
  if (r == 0 || nrhs == 0) return FFC_OK;
  FFC_REQUIRE(skel_perm_dev && q_dev && qt_dev && (r == n || T_dev), "ffc_skeleton_charges: null pointer");
  cudaStream_t st = as_stream(stream);
  ChargeItem it{skel_perm_dev, T_dev, ldt, (int32_t)r, (int32_t)n, q_dev, ldq, qt_dev, ldqt};
  charges_kernel<<<dim3(1, (unsigned)nrhs), CH_THREADS, 0, st>>>(it);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

ffc_status ffc_potential(ffc_kernel kernel, const void* Y_dev, int32_t dtype, const int64_t* rows_dev, int64_t m,
                         const void* X_dev, int64_t n, int32_t d, const int32_t* cols_dev, int64_t nc,
                         const double* w_dev, double log_scale, double* u_dev, void* stream) {
  FFC_REQUIRE(m >= 0 && n >= 0 && nc >= 0 && d >= 1, "ffc_potential: need m, n, nc >= 0 and d >= 1");
  FFC_REQUIRE(dtype == FFC_F64 || dtype == FFC_F32, "ffc_potential: bad dtype");
  FFC_REQUIRE(cols_dev || nc == n, "ffc_potential: without a column list nc must equal n");
  if (!kernel_ok(kernel, d)) return FFC_E_INVALID;
  if (m == 0) return FFC_OK;
  FFC_REQUIRE(Y_dev && u_dev && (nc == 0 || (X_dev && w_dev)), "ffc_potential: null pointer");
  FFC_REQUIRE(std::isfinite(log_scale), "ffc_potential: log_scale must be finite");
  cudaStream_t st = as_stream(stream);
  if (dtype == FFC_F64)
    return launch_potential_t<double>(kernel, Y_dev, rows_dev, m, X_dev, d, cols_dev, nc, w_dev, log_scale, u_dev, st);
  return launch_potential_t<float>(kernel, Y_dev, rows_dev, m, X_dev, d, cols_dev, nc, w_dev, log_scale, u_dev, st);
}

ffc_status ffc_tree_apply(const void* points_perm_dev, int32_t dtype, int64_t N, int32_t d, const ffc_tree* tree,
                          const ffc_tree_result* result, const double* q_dev, int32_t mode, int32_t near_field,
                          double log_scale, double* qt_dev, double* u_dev, void* stream) {
  FFC_REQUIRE(tree && result, "ffc_tree_apply: null tree or result");
  FFC_REQUIRE(N >= 1 && d >= 1 && (dtype == FFC_F64 || dtype == FFC_F32), "ffc_tree_apply: bad N, d or dtype");
  FFC_REQUIRE(mode == FFC_APPLY_SKELETON || mode == FFC_APPLY_DIRECT, "ffc_tree_apply: bad mode");
  FFC_REQUIRE(points_perm_dev && q_dev && u_dev && (mode == FFC_APPLY_DIRECT || qt_dev), "ffc_tree_apply: null pointer");
  FFC_REQUIRE(std::isfinite(log_scale), "ffc_tree_apply: log_scale must be finite");
  const ffc_params* P = tree_result_params(result);
  ffc_tree_view v{};
  ffc_status rc = ffc_tree_result_view(result, &v);
  if (rc != FFC_OK) return rc;
  FFC_REQUIRE(tree->depth >= P->min_level && tree->depth < 31 && tree->n_nodes == ((int64_t)1 << (tree->depth + 1)) - 1,
              "ffc_tree_apply: the tree does not match the compression");
  FFC_REQUIRE(v.n_out == tree->n_nodes - tree_result_first_node(result), "ffc_tree_apply: the tree does not match");
  FFC_REQUIRE((1 << P->min_level) + 2 * tree->depth + 2 <= STACK_MAX,
              "ffc_tree_apply: min_level %d and depth %d exceed the tree walk's stack", P->min_level, tree->depth);
  if (!kernel_ok(P->kernel, d)) return FFC_E_INVALID;
  cudaStream_t st = as_stream(stream);
  const int64_t rcap = P->s_max / 2;
  const int64_t first = tree_result_first_node(result);
  double* qc = nullptr;
  if (mode == FFC_APPLY_SKELETON) {
    // column charges (skel_off layout, total = the skeleton buffer's length) and the skeleton charges,
    // a level at a time from the deepest (a nested node's columns are its children's skeletons)
    int64_t tot = 0;
    FFC_CUDA(cudaMemcpyAsync(&tot, v.skel_off_dev + v.n_out, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    FFC_CUDA(cudaStreamSynchronize(st));
    FFC_CUDA(cudaMallocAsync((void**)&qc, sizeof(double) * std::max<int64_t>(tot, 1), st));
    for (int L = tree->depth; L >= P->min_level; --L) {
      const int64_t o0 = ((int64_t)1 << L) - 1 - first, o1 = ((int64_t)1 << (L + 1)) - 1 - first;
      const int nested_parent = P->nested && L < tree->depth;
      gather_qcols_kernel<<<(unsigned)(o1 - o0), 128, 0, st>>>(o0, first, nested_parent, rcap, tree->begin_dev,
                                                               tree->count_dev, v.rank_dev, v.status_dev, v.s_dev,
                                                               v.skel_off_dev, v.ncols_dev, v.cols_dev, q_dev,
                                                               qt_dev, qc);
      charges_tree_kernel<<<(unsigned)(o1 - o0), CH_THREADS, 0, st>>>(o0, rcap, v.rank_dev, v.status_dev, v.s_dev,
                                                                      v.skel_off_dev, v.ncols_dev, v.skel_dev,
                                                                      v.T_off_dev, v.T_dev, qc, qt_dev);
    }
    FFC_CUDA(cudaGetLastError());
  }
  TreeApplyArgs a{};
  a.k = P->kernel; a.d = d; a.depth = tree->depth; a.min_level = P->min_level; a.mode = mode;
  a.near_field = near_field ? 1 : 0; a.N = N; a.first = first; a.rcap = rcap; a.xi = P->xi;
  a.log_scale = log_scale; a.begin = tree->begin_dev; a.count = tree->count_dev; a.centroid = tree->centroid_dev;
  a.radius = tree->radius_dev; a.rank = v.rank_dev; a.status = v.status_dev; a.skel_off = v.skel_off_dev;
  a.skel = v.skel_dev; a.cols = v.cols_dev; a.sv = v.s_dev; a.q = q_dev; a.qt = qt_dev; a.u = u_dev;
  const int kp = chunk_points(d);
  const size_t smem = chunk_smem(d);
  const unsigned grid = (unsigned)((N + AP_THREADS - 1) / AP_THREADS);
  if (dtype == FFC_F64) {
    FFC_CUDA(cudaFuncSetAttribute(tree_apply_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tree_apply_kernel<double><<<grid, AP_THREADS, smem, st>>>(a, (const double*)points_perm_dev, kp);
  } else {
    FFC_CUDA(cudaFuncSetAttribute(tree_apply_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tree_apply_kernel<float><<<grid, AP_THREADS, smem, st>>>(a, (const float*)points_perm_dev, kp);
  }
  const cudaError_t e = cudaGetLastError();
  if (qc) FFC_CUDA(cudaFreeAsync(qc, st));
  if (e != cudaSuccess) return cuda_fail(e, "tree_apply_kernel");
  return FFC_OK;
}

}  // extern "C"
