// Column-pivoted Householder QR (the triangular solve T = R11^-1 R12 that follows it is in trsm.cu).
//
// Method: the ID of the sampled block comes from a rank-revealing QR
// K' Pi = Q [R11 R12; 0 R22] (§2.1.3, ID theorem; Appendix A.1): the
// skeleton is the first r pivots and P solves R11 P = R12.
//
// GPU design. A launch holds many independent blocks (work items). Each item
// gets a group of g CTAs; CTA c of the group owns the contiguous column range
// [n c / g, n (c+1) / g) (at most QR_NCOL_MAX columns) for the whole
// factorisation, with their residual norms in shared memory. Columns never
// move: a pivot is marked selected and its rows >= k are never read again,
// so R is formed in place in the original column positions. One step k:
//   1. every CTA folds its best (squared norm, column) key into the group's
//      step accumulator with a 64-bit atomicMax and its sum of squared norms,
//      as a 128-bit fixed-point number in three 40-bit limbs, with 64-bit
//      atomicAdds (all at L2; integer sums do not depend on the order), joins
//      the group barrier and reads back the winner and ||R22||^2 (step 0,
//      which fixes the fixed-point exponent, goes through per-CTA slots);
//   2. every CTA loads the pivot column (rows k..s-1) from L2 and forms the
//      LAPACK dlarfg reflector redundantly in shared memory;
//   3. each warp applies the reflector to its owned columns, two at a time:
//      one pass over rows k..s-1 for v^T a, one for a -= tau (v^T a) v;
//   4. one thread per column downdates the squared norm in FP64 (LAPACK
//      xLAQP2, written with squares) and flags unsafe downdates, which a
//      warp per flagged column recomputes.
// GB300's FP64 pipe is ~70x narrower than FP32, so FP64 instructions stay
// out of every full-warp path except the arithmetic that needs them (the
// FP64 element type's own updates): keys compare as integers, the downdate
// runs once per column, FP32 blocks use compensated FP32 sums of exact
// squares for their column norms.
// One cooperative launch per batch: CTA b walks its list of (item, rank in
// the item's group) entries in increasing item order, so the lowest
// unfinished item always has all of its CTAs and the group barriers cannot
// deadlock; a wait that runs out sets FFC_E_TIMEOUT and ends the item.
// Element type T: double (FFC_FP64) or float (FFC_MIXED: FP32 block,
// reflectors and updates; FP64 norm downdating and triangular solve).
#include <algorithm>
#include <cfloat>
#include <climits>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

// CTAs per SM the QR kernel is compiled for (register budget 65536 / (256 x this))
#ifndef FFC_QR_MIN_BLOCKS
#define FFC_QR_MIN_BLOCKS 3
#endif
constexpr int QR_THREADS = 256;
constexpr int QR_WARPS = QR_THREADS / 32;
// Columns one CTA may own: their norms and flags live in shared memory.
constexpr int QR_NCOL_MAX = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Pivot key: the top 44 bits of the (non-negative) squared norm, then
// 0xFFFFF - column, so the integer maximum picks the largest norm and, among
// norms equal to 2^-32 relative, the lowest column. 0 = nothing selectable.
__device__ __forceinline__ unsigned long long pivot_key(double nrm2, int col) {
  if (!(nrm2 > 0.0)) return 0ull;
  const unsigned long long b = (unsigned long long)__double_as_longlong(nrm2);
  return (b & ~0xFFFFFull) | (unsigned long long)(0xFFFFF - col);
}

// Thread 0 only: arrive and wait until `target` arrivals, polling at most `limit` times.
// false on timeout.
__device__ bool group_barrier(unsigned* ctr, unsigned target, long long limit) {
  __threadfence();
  atomicAdd(ctr, 1u);
  long long spins = 0;
  while (ld_acquire_u32(ctr) < target) {
    if (++spins > limit) return false;
    __nanosleep(40);
  }
  __threadfence();
  return true;
}

// Per-item, per-rank step slots, two in rotation (step k uses slots[k & 1]; a
// CTA can only overwrite them two steps later, after every CTA has read them):
// the CTA's pivot key and its sum of squared norms.
struct StepSlot {
  unsigned long long key;
  double sum;
};

// Exact, order-independent sum of non-negative doubles in integer arithmetic:
// each value m 2^(e-1075) is aligned to the largest exponent emax as a 128-bit
// fixed-point number (64 integer bits, 64 fraction bits) and added with carry.
// Deterministic for any summation order, and free of FP64 instructions.
struct Fix128 {
  unsigned long long hi, lo;
};

__device__ __forceinline__ int dbl_exponent(double x) {
  const int e = (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
  return e ? e : 1;
}

__device__ __forceinline__ void fix_add(Fix128& a, double x, int emax) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(b >> 52) & 0x7FF;
  unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e) m |= 1ull << 52;
  const int sh = emax - (e ? e : 1);
  if (m == 0ull || sh >= 117) return;
  if (sh < 0) {   // above the window: saturate (the caller sizes emax so this does not happen)
    a.hi = ~0ull;
    return;
  }
  const unsigned long long ih = sh < 64 ? (m >> sh) : 0ull;
  const unsigned long long il = sh == 0 ? 0ull : (sh < 64 ? (m << (64 - sh)) : (m >> (sh - 64)));
  a.lo += il;
  a.hi += ih + (a.lo < il ? 1ull : 0ull);
}

__device__ __forceinline__ void fix_add(Fix128& a, const Fix128& b) {
  a.lo += b.lo;
  a.hi += b.hi + (a.lo < b.lo ? 1ull : 0ull);
}

// value of a Fix128 aligned to emax (one thread; FP64 arithmetic)
__device__ __forceinline__ double fix_value(const Fix128& a, int emax) {
  return scalbn((double)a.hi, emax - 1075) + scalbn((double)a.lo, emax - 1075 - 64);
}

// Group reduction of steps k >= 1 through 64-bit atomics at L2: red[4 (k % 3)]
// holds the step's max pivot key and the 128-bit fixed-point sum as three
// 40-bit limbs, each summed in its own 64-bit word (integer adds commute, so
// the result does not depend on the arrival order, and up to 2^24 CTAs add
// without a limb overflowing). Rank 0 zeroes the buffer of step k + 2 after
// the barrier of step k, when every CTA has read step k - 1's buffer.
constexpr unsigned long long LIMB40 = (1ull << 40) - 1ull;

__device__ __forceinline__ void red_publish(unsigned long long* rb, unsigned long long key, const Fix128& f) {
  const unsigned __int128 F = ((unsigned __int128)f.hi << 64) | f.lo;
  atomicMax(rb, key);
  atomicAdd(rb + 1, (unsigned long long)(F & LIMB40));
  atomicAdd(rb + 2, (unsigned long long)((F >> 40) & LIMB40));
  atomicAdd(rb + 3, (unsigned long long)(F >> 80));
}

__device__ __forceinline__ void red_read(const unsigned long long* rb, unsigned long long& key, Fix128& f) {
  key = __ldcg(rb);
  const unsigned __int128 F = (unsigned __int128)__ldcg(rb + 1) + ((unsigned __int128)__ldcg(rb + 2) << 40) +
                              ((unsigned __int128)__ldcg(rb + 3) << 80);
  f.hi = (unsigned long long)(F >> 64);
  f.lo = (unsigned long long)F;
}

struct QrShared {
  unsigned long long kw[QR_WARPS];
  unsigned long long fh[QR_WARPS], fl[QR_WARPS];
  double psum[QR_THREADS];
  float fw[QR_WARPS];
  double dw[QR_WARPS];
  unsigned long long key;
  Fix128 fsum, thr;       // ||R22||^2 of the step and tol^2 ||K'||^2, fixed point at emax
  double sum, fro2, tau, beta;
  float tauf;
  int stop, status, n_rc, emax, apply;
};

// Exact square x*x = p + e (FMA), accumulated with a compensated sum (FP32 only).
__device__ __forceinline__ void comp_add_square(float x, float& s, float& c) {
  const float p = x * x;
  const float e = fmaf(x, x, -p);
  const float y = p - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
  c -= e;
}

// Squared norm of rows [i0, s) of a column, one warp; FP64 sums for FP64
// data, compensated FP32 sums of exact squares for FP32 data.
__device__ __forceinline__ double col_sumsq(const double* __restrict__ cj, int i0, int s, int lane) {
  double a0 = 0.0, a1 = 0.0;
  int i = i0 + lane;
  for (; i + 32 < s; i += 64) {
    const double x0 = cj[i], x1 = cj[i + 32];
    a0 = fma(x0, x0, a0);
    a1 = fma(x1, x1, a1);
  }
  if (i < s) { const double x0 = cj[i]; a0 = fma(x0, x0, a0); }
  return warp_sum(a0 + a1);   // valid in every lane
}

// lane 0 of the warp returns the FP64 value of a compensated FP32 pair sum
__device__ __forceinline__ double col_sumsq_f32(const float* __restrict__ cj, int i0, int s, int lane) {
  float sm = 0.f, cm = 0.f;
  for (int i = i0 + lane; i < s; i += 32) comp_add_square(cj[i], sm, cm);
  float hi = sm, lo = -cm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float t = hi + h2;
    const float bb = t - hi;
    const float err = (hi - (t - bb)) + (h2 - bb);
    hi = t;
    lo = lo + l2 + err;
  }
  double r = 0.0;
  if (lane == 0) r = (double)hi + (double)lo;
  return r;
}

template <typename T>
__device__ __forceinline__ double column_norm2(const T* __restrict__ cj, int i0, int s, int lane);

template <>
__device__ __forceinline__ double column_norm2<double>(const double* __restrict__ cj, int i0, int s, int lane) {
  return col_sumsq(cj, i0, s, lane);
}

template <>
__device__ __forceinline__ double column_norm2<float>(const float* __restrict__ cj, int i0, int s, int lane) {
  return col_sumsq_f32(cj, i0, s, lane);   // meaningful in lane 0
}

// Applies H = I - tau v v^T (v in shared memory, rows k..s-1) to one column;
// returns the updated entry in row k (in every lane).
template <typename T>
__device__ __forceinline__ T apply_reflector(T* __restrict__ cj, const T* __restrict__ vsh, T ttau, int k, int s,
                                             int lane) {
  T d0 = (T)0, d1 = (T)0, d2 = (T)0, d3 = (T)0;
  int i = k + lane;
  for (; i + 96 < s; i += 128) {
    const T x0 = cj[i], x1 = cj[i + 32], x2 = cj[i + 64], x3 = cj[i + 96];
    d0 = fma(vsh[i], x0, d0);
    d1 = fma(vsh[i + 32], x1, d1);
    d2 = fma(vsh[i + 64], x2, d2);
    d3 = fma(vsh[i + 96], x3, d3);
  }
  for (; i < s; i += 32) d0 = fma(vsh[i], cj[i], d0);
  const T tw = ttau * warp_sum((d0 + d1) + (d2 + d3));
  T ak = (T)0;
  int r = k + lane;
  if (r < s) {
    ak = fma(-tw, vsh[r], cj[r]);
    cj[r] = ak;
  }
  for (r += 32; r + 96 < s; r += 128) {
    const T x0 = cj[r], x1 = cj[r + 32], x2 = cj[r + 64], x3 = cj[r + 96];
    cj[r] = fma(-tw, vsh[r], x0);
    cj[r + 32] = fma(-tw, vsh[r + 32], x1);
    cj[r + 64] = fma(-tw, vsh[r + 64], x2);
    cj[r + 96] = fma(-tw, vsh[r + 96], x3);
  }
  for (; r < s; r += 32) cj[r] = fma(-tw, vsh[r], cj[r]);
  return __shfl_sync(0xffffffffu, ak, 0);
}

// The same for two columns at once, so that their loads are in flight together.
template <typename T>
__device__ __forceinline__ void apply_reflector2(T* __restrict__ ca, T* __restrict__ cb, const T* __restrict__ vsh,
                                                 T ttau, int k, int s, int lane, T& aka, T& akb) {
  // pass 1: 8 independent loads per lane per iteration keep enough of the
  // (L2-resident) columns in flight
  T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0, b0 = (T)0, b1 = (T)0, b2 = (T)0, b3 = (T)0;
  int i = k + lane;
  for (; i + 96 < s; i += 128) {
    const T xa0 = ca[i], xa1 = ca[i + 32], xa2 = ca[i + 64], xa3 = ca[i + 96];
    const T xb0 = cb[i], xb1 = cb[i + 32], xb2 = cb[i + 64], xb3 = cb[i + 96];
    const T v0 = vsh[i], v1 = vsh[i + 32], v2 = vsh[i + 64], v3 = vsh[i + 96];
    a0 = fma(v0, xa0, a0); a1 = fma(v1, xa1, a1); a2 = fma(v2, xa2, a2); a3 = fma(v3, xa3, a3);
    b0 = fma(v0, xb0, b0); b1 = fma(v1, xb1, b1); b2 = fma(v2, xb2, b2); b3 = fma(v3, xb3, b3);
  }
  for (; i < s; i += 32) {
    const T v0 = vsh[i];
    a0 = fma(v0, ca[i], a0);
    b0 = fma(v0, cb[i], b0);
  }
  const T twa = ttau * warp_sum((a0 + a1) + (a2 + a3)), twb = ttau * warp_sum((b0 + b1) + (b2 + b3));
  // pass 2: row k first (its entry feeds the norm downdate), then the rest
  // four rows per lane per iteration
  T ka = (T)0, kb = (T)0;
  int r = k + lane;
  if (r < s) {
    const T v = vsh[r];
    ka = fma(-twa, v, ca[r]);
    kb = fma(-twb, v, cb[r]);
    ca[r] = ka;
    cb[r] = kb;
  }
  for (r += 32; r + 96 < s; r += 128) {
    const T xa0 = ca[r], xa1 = ca[r + 32], xa2 = ca[r + 64], xa3 = ca[r + 96];
    const T xb0 = cb[r], xb1 = cb[r + 32], xb2 = cb[r + 64], xb3 = cb[r + 96];
    const T v0 = vsh[r], v1 = vsh[r + 32], v2 = vsh[r + 64], v3 = vsh[r + 96];
    ca[r] = fma(-twa, v0, xa0); ca[r + 32] = fma(-twa, v1, xa1);
    ca[r + 64] = fma(-twa, v2, xa2); ca[r + 96] = fma(-twa, v3, xa3);
    cb[r] = fma(-twb, v0, xb0); cb[r + 32] = fma(-twb, v1, xb1);
    cb[r + 64] = fma(-twb, v2, xb2); cb[r + 96] = fma(-twb, v3, xb3);
  }
  for (; r < s; r += 32) {
    const T v = vsh[r];
    ca[r] = fma(-twa, v, ca[r]);
    cb[r] = fma(-twb, v, cb[r]);
  }
  aka = __shfl_sync(0xffffffffu, ka, 0);
  akb = __shfl_sync(0xffffffffu, kb, 0);
}

// CTA-wide: (max key over threads, FP64 sum of per-thread partials) into sh.key, sh.sum.
__device__ void cta_reduce(unsigned long long key, double part, QrShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  key = warp_max_u64(key);
  if (lane == 0) sh.kw[warp] = key;
  sh.psum[threadIdx.x] = part;
  __syncthreads();
  if (warp == 0) {
    double v = 0.0;
    for (int t = lane; t < QR_THREADS; t += 32) v += sh.psum[t];
    v = warp_sum(v);
    unsigned long long kk = lane < QR_WARPS ? sh.kw[lane] : 0ull;
    kk = warp_max_u64(kk);
    if (lane == 0) { sh.key = kk; sh.sum = v; }
  }
  __syncthreads();
}

// FP64 norm downdate of the columns held by the lanes with `mine` set (lane
// c: column j, row-k entry akj), LAPACK xLAQP2 style; a column whose downdate
// is unsafe is recomputed by the whole warp (rare); then each lane folds its
// column into its pivot key and norm sum. Column j's data: base + (j - jb) lda.
template <typename T>
__device__ __forceinline__ void downdate_lane(bool mine, int j, double akj, const T* __restrict__ base, int64_t lda,
                                              int k, int s, int lane, double tol3z, double* __restrict__ vn1s,
                                              double* __restrict__ vn2s, int c0, unsigned long long& key,
                                              Fix128& psum, int emax, int jb) {
  int unsafe = 0;
  if (mine) {
    const double rest = fma(-akj, akj, vn1s[j]);
    if (rest <= tol3z * vn2s[j]) unsafe = 1;
    else vn1s[j] = rest;
  }
  unsigned um = __ballot_sync(0xffffffffu, unsafe);
  while (um) {
    const int src = __ffs(um) - 1;
    um &= um - 1u;
    const int jj = __shfl_sync(0xffffffffu, j, src);
    const double nr = column_norm2<T>(base + (int64_t)(jj - jb) * lda, k + 1, s, lane);
    if (lane == 0) { vn1s[jj] = nr; vn2s[jj] = nr; }
  }
  __syncwarp();
  if (mine) {
    const double v = vn1s[j];
    const unsigned long long kj = pivot_key(v, c0 + j);
    key = kj > key ? kj : key;
    fix_add(psum, v, emax);
  }
}

// CTA-wide: max key and the exact fixed-point sum of per-thread partials into sh.key, sh.fsum
// (integer operations only).
__device__ void cta_reduce_fix(unsigned long long key, Fix128 part, QrShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  key = warp_max_u64(key);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Fix128 g2;
    g2.hi = __shfl_xor_sync(0xffffffffu, part.hi, o);
    g2.lo = __shfl_xor_sync(0xffffffffu, part.lo, o);
    fix_add(part, g2);
  }
  if (lane == 0) { sh.kw[warp] = key; sh.fh[warp] = part.hi; sh.fl[warp] = part.lo; }
  __syncthreads();
  if (warp == 0) {
    unsigned long long kk = lane < QR_WARPS ? sh.kw[lane] : 0ull;
    Fix128 f = {lane < QR_WARPS ? sh.fh[lane] : 0ull, lane < QR_WARPS ? sh.fl[lane] : 0ull};
    kk = warp_max_u64(kk);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      Fix128 g2;
      g2.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
      g2.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
      fix_add(f, g2);
    }
    if (lane == 0) { sh.key = kk; sh.fsum = f; }
  }
  __syncthreads();
}

__device__ __forceinline__ bool fix_le(const Fix128& a, const Fix128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}

// One warp updates NC adjacent owned columns per pass (those not selected):
// v^T a for all of them, then a -= tau (v^T a) v, with NC loads per lane per
// row chunk in flight; lane 0 then downdates each column's squared norm in
// FP64 (the warp recomputes it when the downdate is unsafe) and folds the
// column into the thread's pivot key and norm sum.
template <typename T, int NC>
__device__ __forceinline__ void update_columns(T* __restrict__ A, int64_t lda, int c0, int ncols,
                                               const uint8_t* __restrict__ sels, const T* __restrict__ vsh, T ttau,
                                               bool apply, int k, int s, int warp, int lane, double tol3z,
                                               double* __restrict__ vn1s, double* __restrict__ vn2s,
                                               unsigned long long& key, Fix128& psum, int emax) {
  for (int j0 = warp * NC; j0 < ncols; j0 += QR_WARPS * NC) {
    bool va[NC];
    T* base = A + (int64_t)(c0 + j0) * lda;
#pragma unroll
    for (int c = 0; c < NC; ++c) va[c] = (j0 + c < ncols) && !sels[j0 + c];
    T ak[NC];
    if (apply) {
      T acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = (T)0;
#pragma unroll 2
      for (int i = k + lane; i < s; i += 32) {
        const T v = vsh[i];
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (va[c]) acc[c] = fma(v, base[(int64_t)c * lda + i], acc[c]);
      }
      T tw[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) tw[c] = ttau * warp_sum(acc[c]);
#pragma unroll
      for (int c = 0; c < NC; ++c) ak[c] = (T)0;
#pragma unroll 2
      for (int r = k + lane; r < s; r += 32) {
        const T v = vsh[r];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          if (va[c]) {
            const T x = fma(-tw[c], v, base[(int64_t)c * lda + r]);
            base[(int64_t)c * lda + r] = x;
            if (r == k) ak[c] = x;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) ak[c] = __shfl_sync(0xffffffffu, ak[c], 0);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) ak[c] = va[c] ? base[(int64_t)c * lda + k] : (T)0;
    }
    // lane c downdates column j0 + c: one FP64 instruction stream for all NC
    // columns (a warp-wide FP64 instruction costs the same for 1 or NC lanes)
    T my_ak = ak[0];
    bool mine = va[0] && lane == 0;
#pragma unroll
    for (int c = 1; c < NC; ++c)
      if (lane == c) { my_ak = ak[c]; mine = va[c]; }
    downdate_lane(mine, j0 + lane, (double)my_ak, base, lda, k, s, lane, tol3z, vn1s, vn2s, c0, key, psum, emax,
                  j0);
  }
}

// ---- vectorised column updates (16-byte loads; the column base and lda must be
// 16-byte aligned). Vector q of a lane covers rows kb + W q .. kb + W q + W - 1
// with kb = k rounded down to W; rows outside [k, s) are left unchanged.

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float vget(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ double vget(const double2& v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ void vset(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ void vset(double2& v, int e, double x) { if (e == 0) v.x = x; else v.y = x; }

// NC columns per warp pass, M vectors per lane per column, the whole
// segment [kb, s) held in registers (s - kb <= 32 W M): one round of loads
// for the dot, the axpy from registers, then the lane-parallel downdate.
template <typename T, int NC, int M>
__device__ __forceinline__ void update_columns_vec(T* __restrict__ A, int64_t lda, int c0, int ncols,
                                                   const uint8_t* __restrict__ sels, const T* __restrict__ vsh,
                                                   T ttau, bool apply, int k, int s, int warp, int lane,
                                                   double tol3z, double* __restrict__ vn1s,
                                                   double* __restrict__ vn2s, unsigned long long& key,
                                                   Fix128& psum, int emax) {
  using V4 = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  const int kb = k & ~(W - 1);
  for (int j0 = warp * NC; j0 < ncols; j0 += QR_WARPS * NC) {
    bool va[NC];
    T* base = A + (int64_t)(c0 + j0) * lda;
#pragma unroll
    for (int c = 0; c < NC; ++c) va[c] = (j0 + c < ncols) && !sels[j0 + c];
    T ak[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ak[c] = (T)0;
    if (apply) {
      V4 x[NC][M];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = kb + W * (lane + 32 * m);
          if (va[c] && r0 < s) x[c][m] = *reinterpret_cast<const V4*>(base + (int64_t)c * lda + r0);
          else x[c][m] = V4{};
        }
      T acc[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = (T)0;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int r0 = kb + W * (lane + 32 * m);
        if (r0 < s) {
          const V4 vv = *reinterpret_cast<const V4*>(vsh + r0);
#pragma unroll
          for (int e = 0; e < W; ++e) {
            const int r = r0 + e;
            const T v = (r >= k && r < s) ? vget(vv, e) : (T)0;
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fma(v, vget(x[c][m], e), acc[c]);
          }
        }
      }
      T tw[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) tw[c] = ttau * warp_sum(acc[c]);
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const int r0 = kb + W * (lane + 32 * m);
        if (r0 < s) {
          const V4 vv = *reinterpret_cast<const V4*>(vsh + r0);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            if (!va[c]) continue;
#pragma unroll
            for (int e = 0; e < W; ++e) {
              const int r = r0 + e;
              if (r >= k && r < s) vset(x[c][m], e, fma(-tw[c], vget(vv, e), vget(x[c][m], e)));
            }
            *reinterpret_cast<V4*>(base + (int64_t)c * lda + r0) = x[c][m];
          }
        }
      }
      // row k sits in lane 0's first vector, component k - kb
#pragma unroll
      for (int c = 0; c < NC; ++c) ak[c] = __shfl_sync(0xffffffffu, vget(x[c][0], k - kb), 0);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) ak[c] = va[c] ? base[(int64_t)c * lda + k] : (T)0;
    }
    T my_ak = ak[0];
    bool mine = va[0] && lane == 0;
#pragma unroll
    for (int c = 1; c < NC; ++c)
      if (lane == c) { my_ak = ak[c]; mine = va[c]; }
    downdate_lane(mine, j0 + lane, (double)my_ak, base, lda, k, s, lane, tol3z, vn1s, vn2s, c0, key, psum, emax,
                  j0);
  }
}

// One column per warp pass, rows in chunks of 32 W 8 (longer columns): the
// dot streams the chunks, the axpy reloads them (L1/L2 hits).
template <typename T>
__device__ __forceinline__ void update_column_vec_chunked(T* __restrict__ A, int64_t lda, int c0, int ncols,
                                                          const uint8_t* __restrict__ sels,
                                                          const T* __restrict__ vsh, T ttau, bool apply, int k,
                                                          int s, int warp, int lane, double tol3z,
                                                          double* __restrict__ vn1s, double* __restrict__ vn2s,
                                                          unsigned long long& key, Fix128& psum, int emax) {
  using V4 = typename Vec<T>::type;
  constexpr int W = Vec<T>::W, M = 8;
  const int kb = k & ~(W - 1);
  for (int j = warp; j < ncols; j += QR_WARPS) {
    const bool va = !sels[j];
    T* col = A + (int64_t)(c0 + j) * lda;
    T ak = (T)0;
    if (va && apply) {
      T acc = (T)0, acc2 = (T)0;
      for (int cb = kb; cb < s; cb += 32 * W * M) {
        V4 x[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = cb + W * (lane + 32 * m);
          x[m] = r0 < s ? *reinterpret_cast<const V4*>(col + r0) : V4{};
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = cb + W * (lane + 32 * m);
          if (r0 < s) {
            const V4 vv = *reinterpret_cast<const V4*>(vsh + r0);
#pragma unroll
            for (int e = 0; e < W; ++e) {
              const int r = r0 + e;
              const T v = (r >= k && r < s) ? vget(vv, e) : (T)0;
              if (e & 1) acc2 = fma(v, vget(x[m], e), acc2); else acc = fma(v, vget(x[m], e), acc);
            }
          }
        }
      }
      const T tw = ttau * warp_sum(acc + acc2);
      for (int cb = kb; cb < s; cb += 32 * W * M) {
        V4 x[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = cb + W * (lane + 32 * m);
          x[m] = r0 < s ? *reinterpret_cast<const V4*>(col + r0) : V4{};
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = cb + W * (lane + 32 * m);
          if (r0 < s) {
            const V4 vv = *reinterpret_cast<const V4*>(vsh + r0);
#pragma unroll
            for (int e = 0; e < W; ++e) {
              const int r = r0 + e;
              if (r >= k && r < s) vset(x[m], e, fma(-tw, vget(vv, e), vget(x[m], e)));
            }
            *reinterpret_cast<V4*>(col + r0) = x[m];
            if (cb == kb && m == 0) ak = vget(x[0], k - kb);
          }
        }
      }
      ak = __shfl_sync(0xffffffffu, ak, 0);
    } else if (va) {
      ak = col[k];
    }
    downdate_lane(va && lane == 0, j, (double)ak, A + (int64_t)c0 * lda, lda, k, s, lane, tol3z, vn1s, vn2s, c0,
                  key, psum, emax, 0);
  }
}

// ---- lazy form (FP32 columns of at most 128 M rows, held whole in registers) ----------------------
// Lane l, vector m of a warp holds rows 4 (l + 32 m) .. + 3 of a column, anchored at row 0, so one
// reflector's arithmetic on a column does not depend on the step it is applied in. The stored columns
// stay at the state after reflector w (the last write-back); a step re-applies reflectors w + 1 .. k
// from a ring of D slots in shared memory and writes the columns back only every D steps. Every
// reflector is applied with the same operations in the same order whatever D is, so the results do not
// depend on D; a column is then read every step but written once per D steps.
constexpr int QR_DEFER_MAX = 4;   // slots of the reflector ring

// H_i = I - tau v v^T (v: rows i .. s-1 of a ring slot, v[i] = 1) on NC register-resident columns
template <int NC, int M>
__device__ __forceinline__ void lazy_reflect(float4 (&x)[NC][M], const bool (&va)[NC], const float* __restrict__ v,
                                             float tau, int i, int s, int lane) {
  float acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int r0 = 4 * (lane + 32 * m);
    if (r0 + 3 >= i && r0 < s) {
      const float4 vv = *reinterpret_cast<const float4*>(v + r0);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + e;
        const float vr = (r >= i && r < s) ? vget(vv, e) : 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] = fmaf(vr, vget(x[c][m], e), acc[c]);
      }
    }
  }
  float tw[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) tw[c] = tau * warp_sum(acc[c]);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int r0 = 4 * (lane + 32 * m);
    if (r0 + 3 >= i && r0 < s) {
      const float4 vv = *reinterpret_cast<const float4*>(v + r0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (!va[c]) continue;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = r0 + e;
          if (r >= i && r < s) vset(x[c][m], e, fmaf(-tw[c], vget(vv, e), vget(x[c][m], e)));
        }
      }
    }
  }
}

// Rows [lo, s) of NC columns from global memory (lo a multiple of 4; rows below it are not needed)
template <int NC, int M>
__device__ __forceinline__ void lazy_load(float4 (&x)[NC][M], const bool (&va)[NC], const float* __restrict__ base,
                                          int64_t lda, int lo, int s, int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int r0 = 4 * (lane + 32 * m);
      x[c][m] = (va[c] && r0 >= lo && r0 < s) ? __ldcg(reinterpret_cast<const float4*>(base + (int64_t)c * lda + r0))
                                               : float4{0.0f, 0.0f, 0.0f, 0.0f};
    }
}

template <int NC, int M>
__device__ __forceinline__ void lazy_store(const float4 (&x)[NC][M], const bool (&va)[NC], float* __restrict__ base,
                                           int64_t lda, int lo, int s, int lane) {
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int r0 = 4 * (lane + 32 * m);
      if (va[c] && r0 >= lo && r0 < s) *reinterpret_cast<float4*>(base + (int64_t)c * lda + r0) = x[c][m];
    }
}

// Entry of row k of column c (every lane)
template <int NC, int M>
__device__ __forceinline__ float lazy_row(const float4 (&x)[NC][M], int c, int k) {
  const int mk = k >> 7, ek = k & 3, lk = (k >> 2) & 31;
  float v = 0.0f;
#pragma unroll
  for (int cc = 0; cc < NC; ++cc)
#pragma unroll
    for (int m = 0; m < M; ++m)
      if (cc == c && m == mk) v = vget(x[cc][m], ek);
  return __shfl_sync(0xffffffffu, v, lk);
}

// Squared norm of rows (k, s) of column c from the registers: compensated FP32 sums of exact squares,
// then the pairwise error-free combination of col_sumsq_f32; meaningful in lane 0
template <int NC, int M>
__device__ __forceinline__ double lazy_sumsq(const float4 (&x)[NC][M], int c, int k, int s, int lane) {
  float sm = 0.f, cm = 0.f;
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    if (cc != c) continue;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int r0 = 4 * (lane + 32 * m);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + e;
        if (r > k && r < s) comp_add_square(vget(x[cc][m], e), sm, cm);
      }
    }
  }
  float hi = sm, lo = -cm;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const float t = hi + h2;
    const float bb = t - hi;
    const float err = (hi - (t - bb)) + (h2 - bb);
    hi = t;
    lo = lo + l2 + err;
  }
  return lane == 0 ? (double)hi + (double)lo : 0.0;
}

// One step of the lazy form over the CTA's free columns: load (state after w), apply reflectors
// w + 1 .. k from the ring, downdate with row k, and store when `store` (the state after k).
template <int NC, int M>
__device__ __forceinline__ void update_columns_lazy(float* __restrict__ A, int64_t lda, int c0, int ncols,
                                                    const uint8_t* __restrict__ sels, const float* __restrict__ ring,
                                                    int ldv, const float* __restrict__ taur, int D, int w, int k,
                                                    int s, bool store, int warp, int lane, double tol3z,
                                                    double* __restrict__ vn1s, double* __restrict__ vn2s,
                                                    unsigned long long& key, Fix128& psum, int emax) {
  const int lo = (w + 1) & ~3;
  for (int j0 = warp * NC; j0 < ncols; j0 += QR_WARPS * NC) {
    bool va[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) va[c] = (j0 + c < ncols) && !sels[j0 + c];
    float* base = A + (int64_t)(c0 + j0) * lda;
    float4 x[NC][M];
    lazy_load<NC, M>(x, va, base, lda, lo, s, lane);
    for (int i = w + 1; i <= k; ++i) lazy_reflect<NC, M>(x, va, ring + (size_t)(i % D) * ldv, taur[i % D], i, s, lane);
    if (store) lazy_store<NC, M>(x, va, base, lda, lo, s, lane);
    // downdate (lane c owns column c), recomputing unsafe norms from the registers
    float my_ak = 0.0f;
    bool mine = false;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float akc = lazy_row<NC, M>(x, c, k);
      if (lane == c) { my_ak = akc; mine = va[c]; }
    }
    const int j = j0 + lane;
    int unsafe = 0;
    if (mine) {
      const double rest = fma(-(double)my_ak, (double)my_ak, vn1s[j]);
      if (rest <= tol3z * vn2s[j]) unsafe = 1;
      else vn1s[j] = rest;
    }
    unsigned um = __ballot_sync(0xffffffffu, unsafe);
    while (um) {
      const int src = __ffs(um) - 1;
      um &= um - 1u;
      const double nr = lazy_sumsq<NC, M>(x, src, k, s, lane);
      if (lane == 0) { vn1s[j0 + src] = nr; vn2s[j0 + src] = nr; }
    }
    __syncwarp();
    if (mine) {
      const double v = vn1s[j];
      const unsigned long long kj = pivot_key(v, c0 + j);
      key = kj > key ? kj : key;
      fix_add(psum, v, emax);
    }
  }
}

// The pivot column p after reflector k - 1 (one warp, the same arithmetic as the pass that last held it):
// rows [k, s) into the ring slot of reflector k; rows w + 1 .. k - 1 (now final rows of R) into keep[].
template <int M>
__device__ __forceinline__ void lazy_pivot_column(const float* __restrict__ cp, const float* __restrict__ ring,
                                                  int ldv, const float* __restrict__ taur, int D, int w, int k, int s,
                                                  float* __restrict__ slot, float* __restrict__ keep, int lane) {
  const bool va[1] = {true};
  float4 x[1][M];
  const int lo = (w + 1) & ~3;
  lazy_load<1, M>(x, va, cp, 0, lo, s, lane);
  for (int i = w + 1; i < k; ++i) lazy_reflect<1, M>(x, va, ring + (size_t)(i % D) * ldv, taur[i % D], i, s, lane);
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const int r0 = 4 * (lane + 32 * m);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int r = r0 + e;
      if (r >= k && r < s) slot[r] = vget(x[0][m], e);
      if (r > w && r < k) keep[r - w - 1] = vget(x[0][m], e);
    }
  }
}

// BIG: the launch has the register budget (2 CTAs per SM) to hold FP32 columns of up to
// 512 W rows in registers, so the longest columns (s = 2,048) are read once per step, and
// to take columns of up to 256 W rows two at a time
// LZ = M > 0 (FP32, BIG, s <= 128 M): the lazy form above with ring depth D; the pivot
// column is rebuilt by every CTA, and the group's rank-0 CTA writes its new rows of R after the next
// group barrier, when no CTA reads that column any more.
template <typename T, bool BIG, int LZ = 0>
__device__ void factor_item(const CpqrItem& it, const CtaAssign a, T* __restrict__ vsh, double* __restrict__ vn1s,
                            double* __restrict__ vn2s, T* __restrict__ aks, uint8_t* __restrict__ sels,
                            int16_t* __restrict__ rcl, QrShared& sh, long long spin_limit,
                            float* __restrict__ ring = nullptr, int ldv = 0, float* __restrict__ taur = nullptr,
                            float* __restrict__ keep = nullptr, int D = 1) {
  constexpr bool LAZY = LZ > 0;
  constexpr int LZM = LZ > 0 ? LZ : 8, LZNC = LZM >= 16 ? 1 : 2;   // lazy form: vectors per lane, columns per warp
  const int s = it.s, n = it.n;
  T* __restrict__ A = reinterpret_cast<T*>(it.A);
  const int64_t lda = it.lda;
  const int c0 = (int)((int64_t)n * a.rank / a.g), c1 = (int)((int64_t)n * (a.rank + 1) / a.g);
  const int ncols = c1 - c0;
  StepSlot* slots = reinterpret_cast<StepSlot*>(it.slots);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int kmax = min(it.r_max, min(s, n));
  // LAPACK's recompute threshold sqrt(eps) for the precision the columns are
  // stored in: the downdate subtracts a_kj^2, and a_kj is only as accurate as
  // the stored data, so FP32 columns need sqrt(2^-24), not sqrt(2^-53)
  const double TOL3Z = sizeof(T) == 4 ? 2.44140625e-04 : 1.0536712127723509e-08;
  // 16-byte vector access to the columns needs an aligned base and leading dimension
  const bool vec_ok = ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) && (((uint64_t)lda * sizeof(T)) % 16 == 0);

  // initial squared column norms, kept in shared memory for the whole factorisation
  for (int j = warp; j < ncols; j += QR_WARPS) {
    const double nr = column_norm2<T>(A + (int64_t)(c0 + j) * lda, 0, s, lane);
    if (lane == 0) { vn1s[j] = nr; vn2s[j] = nr; sels[j] = 0; }
  }
  __syncthreads();
  {
    unsigned long long key = 0ull;
    double part = 0.0;
    for (int j = tid; j < ncols; j += QR_THREADS) {
      const unsigned long long kj = pivot_key(vn1s[j], c0 + j);
      key = kj > key ? kj : key;
      part += vn1s[j];
    }
    cta_reduce(key, part, sh);
  }

  int k = 0;
  int w = -1;                             // LAZY: reflector the stored columns are up to date with
  int pend_p = -1, pend_n = 0, pend_lo = 0;   // LAZY: rows of R of the last pivot still to write
  for (;; ++k) {
    // group winner and ||R22||^2 for step k: publish, barrier, reduce the
    // group's slots (integer max of the keys, exact integer sum of the sums)
    if (tid == 0) {
      sh.stop = 0;
      if (a.g > 1) {
        if (k == 0) {   // step 0 fixes the fixed-point exponent: slots, read by warp 0 below
          StepSlot* sl = slots + a.rank;
          sl->key = sh.key;
          sl->sum = sh.sum;
        } else {
          red_publish(it.red + 4 * (k % 3), sh.key, sh.fsum);
        }
        if (!group_barrier(it.barrier, (unsigned)a.g * (unsigned)(k + 1), spin_limit)) {
          sh.stop = 1;
          sh.status = FFC_E_TIMEOUT;
        } else if (k > 0) {
          unsigned long long kk;
          Fix128 f;
          red_read(it.red + 4 * (k % 3), kk, f);
          sh.key = kk;
          sh.fsum = f;
          if (a.rank == 0) {
            unsigned long long* z = it.red + 4 * ((k + 2) % 3);
            z[0] = 0ull; z[1] = 0ull; z[2] = 0ull; z[3] = 0ull;
          }
        }
      } else if (k == 0) {   // one CTA: its own total fixes the exponent
        sh.emax = min(dbl_exponent(sh.sum) + 11, 2046);
      }
    }
    __syncthreads();
    if (LAZY && pend_p >= 0) {   // every CTA of the group is past its last read of the previous pivot column
      if (a.rank == 0)
        for (int r = tid; r < pend_n; r += QR_THREADS) A[(int64_t)pend_p * lda + pend_lo + r] = (T)keep[r];
      pend_p = -1;
    }
    if (a.g > 1 && !sh.stop && k == 0 && warp == 0) {
      const StepSlot* base = slots;
      unsigned long long kk = 0ull;
      // every later step's sums are below step 0's total, so its exponent
      // (plus one) bounds them; 128-bit fixed point keeps ~2^-116 of it
      int emax = 1;
      for (int t = lane; t < a.g; t += 32) emax = max(emax, dbl_exponent(__ldcg(&base[t].sum)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      emax = min(emax + 11, 2046);   // room for the sum of up to 2^11 slots
      if (lane == 0) sh.emax = emax;
      Fix128 f = {0ull, 0ull};
      for (int t = lane; t < a.g; t += 32) {
        const unsigned long long kt = __ldcg(&base[t].key);
        kk = kt > kk ? kt : kk;
        fix_add(f, __ldcg(&base[t].sum), emax);
      }
      kk = warp_max_u64(kk);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        Fix128 g2;
        g2.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
        g2.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
        fix_add(f, g2);
      }
      if (lane == 0) { sh.key = kk; sh.sum = fix_value(f, emax); }
    }
    __syncthreads();
    if (tid == 0) {
      if (!sh.stop) {
        // ||R22||_F <= tol ||K'||_F compared as squares; from step 1 on in the
        // exact fixed-point domain (no FP64 instruction per step)
        bool reached;
        if (k == 0) {
          sh.fro2 = sh.sum;
          Fix128 t = {0ull, 0ull};
          if (it.tol > 0.0) fix_add(t, it.tol * it.tol * sh.fro2, sh.emax);
          sh.thr = t;
          reached = it.tol > 0.0 && sh.sum <= it.tol * it.tol * sh.fro2;
        } else {
          reached = it.tol > 0.0 && fix_le(sh.fsum, sh.thr);
        }
        if (reached) {
          sh.stop = 1;
          sh.status = FFC_OK;
        } else if (k >= kmax || (sh.key >> 20) == 0ull) {
          sh.stop = 1;
          sh.status = it.tol > 0.0 ? FFC_E_TOL_NOT_REACHED : FFC_OK;
        }
      }
    }
    __syncthreads();
    if (sh.stop) break;
    const int p = 0xFFFFF - (int)(sh.key & 0xFFFFFull);

    // reflector from column p, rows k..s-1 (written by its owner before the barrier; LAZY: rebuilt here
    // from the state after reflector w, into the ring slot of reflector k)
    const T* cp = A + (int64_t)p * lda;
    T* const vk = LAZY ? reinterpret_cast<T*>(ring + (size_t)(k % D) * ldv) : vsh;
    if constexpr (LAZY) {
      if (warp == 0)
        lazy_pivot_column<LZM>(reinterpret_cast<const float*>(cp), ring, ldv, taur, D, w, k, s,
                               reinterpret_cast<float*>(vk), keep, lane);
      pend_p = p;
      pend_n = k - 1 - w;
      pend_lo = w + 1;
      __syncthreads();
    }
    T part = (T)0;
    for (int i = k + tid; i < s; i += QR_THREADS) {
      const T x = LAZY ? vk[i] : __ldcg(cp + i);
      vk[i] = x;
      if (i > k) part = fma(x, x, part);
    }
    part = warp_sum(part);
    if (lane == 0) {
      if (sizeof(T) == 8) sh.dw[warp] = (double)part; else sh.fw[warp] = (float)part;
    }
    __syncthreads();
    if (tid == 0) {
      T xn2 = (T)0;
      for (int w = 0; w < QR_WARPS; ++w) xn2 += sizeof(T) == 8 ? (T)sh.dw[w] : (T)sh.fw[w];
      const T alpha = vk[k];
      if (xn2 == (T)0) {
        sh.tau = 0.0;
        sh.tauf = 0.0f;
        sh.apply = 0;
        sh.beta = (double)alpha;
      } else {
        const T nrm = sqrt(fma(alpha, alpha, xn2));
        const T beta = alpha >= (T)0 ? -nrm : nrm;
        const T scale = (T)1 / (alpha - beta);
        const T tt = (beta - alpha) / beta;
        sh.tau = (double)tt;
        sh.tauf = (float)tt;
        sh.apply = 1;
        sh.beta = (double)beta;
        vk[k] = scale;   // read below, then replaced by 1
      }
      if (LAZY) taur[k % D] = sh.apply ? sh.tauf : 0.0f;
      if (a.rank == 0) { it.piv[k] = p; it.beta[k] = sh.beta; }
      if (p >= c0 && p < c1) sels[p - c0] = 1;
    }
    __syncthreads();
    const bool apply = sh.apply != 0;
    if (apply) {
      const T scale = vk[k];
      for (int i = k + 1 + tid; i < s; i += QR_THREADS) vk[i] = vk[i] * scale;
    }
    __syncthreads();
    if (tid == 0) vk[k] = (T)1;
    if (tid == 0) sh.n_rc = 0;
    __syncthreads();

    // apply H_k to the owned free columns: short columns NC at a time per
    // warp (many loads in flight), long ones two at a time
    const T ttau = sizeof(T) == 8 ? (T)sh.tau : (T)sh.tauf;
    const int emax = sh.emax;
    unsigned long long key = 0ull;
    Fix128 psum = {0ull, 0ull};
    constexpr int W = Vec<T>::W;
    const int vrows = s - (k & ~(W - 1));
    if constexpr (LAZY) {
      const bool store = k - w >= D;
      update_columns_lazy<LZNC, LZM>(reinterpret_cast<float*>(A), lda, c0, ncols, sels, ring, ldv, taur, D, w, k, s,
                                     store, warp, lane, TOL3Z, vn1s, vn2s, key, psum, emax);
      if (store) w = k;
    } else if (vec_ok) {
      if (vrows <= 32 * W)
        update_columns_vec<T, 8, 1>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                    key, psum, emax);
      else if (vrows <= 64 * W)
        update_columns_vec<T, 4, 2>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                    key, psum, emax);
      else if (vrows <= 128 * W)
        update_columns_vec<T, 2, 4>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                    key, psum, emax);
      else if (BIG && vrows <= 256 * W)
        update_columns_vec<T, 2, 8>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                    key, psum, emax);
      else if (vrows <= 256 * W)
        update_columns_vec<T, 1, 8>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                    key, psum, emax);
      else if (BIG && vrows <= 512 * W)
        update_columns_vec<T, 1, 16>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s,
                                     vn2s, key, psum, emax);
      else
        update_column_vec_chunked<T>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s,
                                     key, psum, emax);
    } else if (s - k <= 256) {
      update_columns<T, 8>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s, key,
                           psum, emax);
    } else if (s - k <= 1024) {
      update_columns<T, 4>(A, lda, c0, ncols, sels, vsh, ttau, apply, k, s, warp, lane, TOL3Z, vn1s, vn2s, key,
                           psum, emax);
    } else {
    for (int j0 = warp; j0 < ncols; j0 += 2 * QR_WARPS) {
      const int jb = j0 + QR_WARPS;
      const bool va = !sels[j0], vb = jb < ncols && !sels[jb];
      T ka = (T)0, kb = (T)0;
      if (apply) {
        if (va && vb) {
          apply_reflector2(A + (int64_t)(c0 + j0) * lda, A + (int64_t)(c0 + jb) * lda, vsh, ttau, k, s, lane, ka, kb);
        } else {
          if (va) ka = apply_reflector(A + (int64_t)(c0 + j0) * lda, vsh, ttau, k, s, lane);
          if (vb) kb = apply_reflector(A + (int64_t)(c0 + jb) * lda, vsh, ttau, k, s, lane);
        }
      } else {
        if (va) ka = A[(int64_t)(c0 + j0) * lda + k];
        if (vb) kb = A[(int64_t)(c0 + jb) * lda + k];
      }
      // FP64 norm downdate of the two columns by lanes 0 and 1, right behind
      // their update (its latency hides behind the other warps' passes)
      const bool mine = (lane == 0 && va) || (lane == 1 && vb);
      downdate_lane(mine, lane == 0 ? j0 : jb, (double)(lane == 0 ? ka : kb), A + (int64_t)c0 * lda, lda, k, s,
                    lane, TOL3Z, vn1s, vn2s, c0, key, psum, emax, 0);
    }
    }
    cta_reduce_fix(key, psum, sh);
  }

  if constexpr (LAZY) {
    // the free columns catch up with the reflectors since the last write-back (rows of R12); the last
    // pivot's rows of R follow (no CTA reads that column any more)
    if (w < k - 1) {
      const int lo = (w + 1) & ~3;
      float* Af = reinterpret_cast<float*>(A);
      for (int j0 = warp; j0 < ncols; j0 += QR_WARPS) {
        const bool va[1] = {!sels[j0]};
        float4 x[1][LZM];
        float* base = Af + (int64_t)(c0 + j0) * lda;
        lazy_load<1, LZM>(x, va, base, lda, lo, s, lane);
        for (int i = w + 1; i < k; ++i) lazy_reflect<1, LZM>(x, va, ring + (size_t)(i % D) * ldv, taur[i % D], i, s, lane);
        lazy_store<1, LZM>(x, va, base, lda, lo, s, lane);
      }
    }
    if (pend_p >= 0 && a.rank == 0)
      for (int r = tid; r < pend_n; r += QR_THREADS) A[(int64_t)pend_p * lda + pend_lo + r] = (T)keep[r];
  }
  // outputs; status_out starts at FFC_OK and a timeout anywhere in the group wins
  if (tid == 0) {
    if (sh.status == FFC_E_TIMEOUT) atomicExch(it.status_out, (int)FFC_E_TIMEOUT);
    if (a.rank == 0) {
      *it.rank_out = k;
      const double fin = k == 0 ? sh.sum : fix_value(sh.fsum, sh.emax);
      *it.r22_out = sh.fro2 > 0.0 ? sqrt(fin) / sqrt(sh.fro2) : 0.0;
      if (sh.status != FFC_E_TIMEOUT) atomicCAS(it.status_out, (int)FFC_OK, sh.status);
    }
  }
  // selected flags of the owned columns for the finalize step
  for (int j = tid; j < ncols; j += QR_THREADS) it.selected[c0 + j] = sels[j];
}

// Shared-memory row stride of the blocked form's V (a multiple of 8 elements, 8 spare) and its offset
// (after the unblocked form's arrays, 256-byte aligned).
__host__ __device__ constexpr int qr_ldv(int s_max) { return ((s_max + 7) & ~7) + 8; }
template <typename T>
__host__ __device__ constexpr size_t qr_blocked_off(int s_max) {
  return (QR_NCOL_MAX * (2 * sizeof(double) + sizeof(T) + sizeof(int16_t) + 1) +
          (size_t)((s_max > 1 ? s_max : 1) + 8) * sizeof(T) + 255) & ~size_t(255);
}

// ---------------------------------------------------------------------------------------------
// Blocked variant (the trailing matrix is read, not written, at every step).
//
// Within a panel of nb steps starting at step k0 the stored columns keep their
// panel-start values in rows >= the current step (rows above are R, written as
// each step's pivot row). With the panel's reflectors V (s x nb, shared memory,
// every CTA its own copy) and F (n x nb, global, F(c, t) = tau_t (current
// column c)^T v_t), the current column is A(:, c) - V F(c, :)^T, so step
// k = k0 + j needs, for every free column, one dot product with the stored
// column (read only): F(c, j) = tau (A(k:s, c)^T v - F(c, 0:j) w),
// w = V(k:s, 0:j)^T v; then the pivot row A(k, c) -= V(k, 0:j+1) F(c, 0:j+1)^T
// and the FP64 norm downdate. The pivot column itself is formed as
// A(k:s, p) - V(k:s, 0:j) F(p, 0:j)^T. At the end of a panel every CTA applies
// A(k_end:s, c) -= V F(c, :)^T to its columns once (skipped after the last
// step: the trailing rows are never read again). Pivots, stopping rule and
// outputs are those of the unblocked form (Businger-Golub order, LAPACK
// reflectors); only rounding differs.
constexpr int QR_NB_MAX = QR_F_STRIDE;   // panel width bound; F rows are padded to it
constexpr int QR_BLOCKED_MIN_S = 1024;   // smallest round (rows) the library blocks by default

// Blocked form, step k (panel step j): for NC owned columns per warp pass, the dot product of the
// stored rows [kb, s) with v (M vectors per lane held in registers: one round of loads), then lane c
// finishes column c: F(c, j) = tau (dot - F(c, 0:j) w), the pivot row A(k, c) -= V(k, 0:j+1) F(c, 0:j+1)^T,
// the FP64 norm downdate (an unsafe one recomputes the current rows k+1..s-1 from the stored column and
// the panel) and the pivot key. With CHUNK, columns longer than 32 W M rows stream in chunks.
template <typename T, int NC, int M, bool CHUNK>
__device__ __forceinline__ void blocked_columns(T* __restrict__ A, int64_t lda, T* __restrict__ F,
                                                T* __restrict__ Fs, int nb, int c0, int ncols,
                                                const uint8_t* __restrict__ sels, const T* __restrict__ vj,
                                                const T* __restrict__ Vs, int ldv, const T* __restrict__ wsh, T ttau,
                                                bool apply, int k, int j, int s, int warp, int lane, double tol3z,
                                                double* __restrict__ vn1s, double* __restrict__ vn2s,
                                                unsigned long long& key, Fix128& psum, int emax) {
  using V4 = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  const int kb = k & ~(W - 1);
  for (int jj0 = warp * NC; jj0 < ncols; jj0 += QR_WARPS * NC) {
    bool va[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) va[c] = (jj0 + c < ncols) && !sels[jj0 + c];
    T acc[NC], akr[NC];   // dot products; the stored A(k, c) from the first chunk's registers
#pragma unroll
    for (int c = 0; c < NC; ++c) { acc[c] = (T)0; akr[c] = (T)0; }
    if (apply) {
      for (int cb = kb; cb < s; cb += 32 * W * M) {
        V4 x[NC][M];
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int m = 0; m < M; ++m) {
            const int r0 = cb + W * (lane + 32 * m);
            x[c][m] = (va[c] && r0 < s) ? *reinterpret_cast<const V4*>(A + (int64_t)(c0 + jj0 + c) * lda + r0)
                                        : V4{};
          }
        if (cb == kb) {
          // row k sits in lane 0's first vector, component k - kb
#pragma unroll
          for (int c = 0; c < NC; ++c) akr[c] = __shfl_sync(0xffffffffu, vget(x[c][0], k - kb), 0);
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const int r0 = cb + W * (lane + 32 * m);
          if (r0 < s) {
            const V4 vv = *reinterpret_cast<const V4*>(vj + r0);
#pragma unroll
            for (int e = 0; e < W; ++e) {
              const T ve = r0 + e < s ? vget(vv, e) : (T)0;
#pragma unroll
              for (int c = 0; c < NC; ++c) acc[c] = fma(ve, vget(x[c][m], e), acc[c]);
            }
          }
        }
        if (!CHUNK) break;
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = warp_sum(acc[c]);
    T dotc = acc[0], akc = akr[0];
    bool mine = va[0] && lane == 0;
#pragma unroll
    for (int c = 1; c < NC; ++c)
      if (lane == c) { dotc = acc[c]; akc = akr[c]; mine = va[c]; }
    const int jc = jj0 + lane;
    int unsafe = 0;
    if (mine) {
      T* col = A + (int64_t)(c0 + jc) * lda;
      T* fs = Fs + jc * nb;
      T corr = (T)0, rowc = (T)0;
      for (int t = 0; t < j; ++t) {
        const T ft = fs[t];
        corr = fma(ft, wsh[t], corr);
        rowc = fma(Vs[(int64_t)t * ldv + k], ft, rowc);
      }
      const T fcj = apply ? ttau * (dotc - corr) : (T)0;
      fs[j] = fcj;
      F[(int64_t)(c0 + jc) * QR_F_STRIDE + j] = fcj;   // for the CTAs that take this column as a pivot
      const T ak = (apply ? akc : col[k]) - rowc - fcj;   // V(k, j) = 1 (and F(c, j) = 0 when H = I)
      col[k] = ak;
      const double akd = (double)ak;
      const double rest = fma(-akd, akd, vn1s[jc]);
      if (rest <= tol3z * vn2s[jc]) unsafe = 1;
      else vn1s[jc] = rest;
    }
    unsigned um = __ballot_sync(0xffffffffu, unsafe);
    while (um) {   // recompute the current norm of rows k+1..s-1 (rare)
      const int src = __ffs(um) - 1;
      um &= um - 1u;
      const int jr = jj0 + src;
      const T* col = A + (int64_t)(c0 + jr) * lda;
      const T* fs = Fs + jr * nb;
      double nr = 0.0;
      for (int i = k + 1 + lane; i < s; i += 32) {
        T x = col[i];
        for (int t = 0; t <= j; ++t) x = fma(-Vs[(int64_t)t * ldv + i], fs[t], x);
        nr = fma((double)x, (double)x, nr);
      }
      nr = warp_sum(nr);
      if (lane == 0) { vn1s[jr] = nr; vn2s[jr] = nr; }
    }
    __syncwarp();
    if (mine) {
      const double v = vn1s[jc];
      const unsigned long long kj = pivot_key(v, c0 + jc);
      key = kj > key ? kj : key;
      fix_add(psum, v, emax);
    }
  }
}

template <typename T, bool BIG>
__device__ void factor_item_blocked(const CpqrItem& it, const CtaAssign a, double* __restrict__ vn1s,
                                    double* __restrict__ vn2s, uint8_t* __restrict__ sels, T* __restrict__ Vs,
                                    int ldv, T* __restrict__ wsh, T* __restrict__ fsh, T* __restrict__ Fs, int nb,
                                    QrShared& sh, long long spin_limit) {
  using V4 = typename Vec<T>::type;
  constexpr int W = Vec<T>::W;
  const int s = it.s, n = it.n;
  T* __restrict__ A = reinterpret_cast<T*>(it.A);
  T* __restrict__ F = reinterpret_cast<T*>(it.F);
  const int64_t lda = it.lda;
  const int c0 = (int)((int64_t)n * a.rank / a.g), c1 = (int)((int64_t)n * (a.rank + 1) / a.g);
  const int ncols = c1 - c0;
  StepSlot* slots = reinterpret_cast<StepSlot*>(it.slots);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int kmax = min(it.r_max, min(s, n));
  const double TOL3Z = sizeof(T) == 4 ? 2.44140625e-04 : 1.0536712127723509e-08;

  for (int j = warp; j < ncols; j += QR_WARPS) {
    const double nr = column_norm2<T>(A + (int64_t)(c0 + j) * lda, 0, s, lane);
    if (lane == 0) { vn1s[j] = nr; vn2s[j] = nr; sels[j] = 0; }
  }
  __syncthreads();
  {
    unsigned long long key = 0ull;
    double part = 0.0;
    for (int j = tid; j < ncols; j += QR_THREADS) {
      const unsigned long long kj = pivot_key(vn1s[j], c0 + j);
      key = kj > key ? kj : key;
      part += vn1s[j];
    }
    cta_reduce(key, part, sh);
  }

  int k = 0, k0 = 0;
  double pn0 = 0.0;   // squared norm of the current panel's first pivot
  for (;; ++k) {
    // ---- group winner and ||R22||^2 of step k (as in the unblocked form)
    if (tid == 0) {
      sh.stop = 0;
      if (a.g > 1) {
        if (k == 0) {
          StepSlot* sl = slots + a.rank;
          sl->key = sh.key;
          sl->sum = sh.sum;
        } else {
          red_publish(it.red + 4 * (k % 3), sh.key, sh.fsum);
        }
        if (!group_barrier(it.barrier, (unsigned)a.g * (unsigned)(k + 1), spin_limit)) {
          sh.stop = 1;
          sh.status = FFC_E_TIMEOUT;
        } else if (k > 0) {
          unsigned long long kk;
          Fix128 f;
          red_read(it.red + 4 * (k % 3), kk, f);
          sh.key = kk;
          sh.fsum = f;
          if (a.rank == 0) {
            unsigned long long* z = it.red + 4 * ((k + 2) % 3);
            z[0] = 0ull; z[1] = 0ull; z[2] = 0ull; z[3] = 0ull;
          }
        }
      } else if (k == 0) {
        sh.emax = min(dbl_exponent(sh.sum) + 11, 2046);
      }
    }
    __syncthreads();
    if (a.g > 1 && !sh.stop && k == 0 && warp == 0) {
      unsigned long long kk = 0ull;
      int emax = 1;
      for (int t = lane; t < a.g; t += 32) emax = max(emax, dbl_exponent(__ldcg(&slots[t].sum)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      emax = min(emax + 11, 2046);
      if (lane == 0) sh.emax = emax;
      Fix128 f = {0ull, 0ull};
      for (int t = lane; t < a.g; t += 32) {
        const unsigned long long kt = __ldcg(&slots[t].key);
        kk = kt > kk ? kt : kk;
        fix_add(f, __ldcg(&slots[t].sum), emax);
      }
      kk = warp_max_u64(kk);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        Fix128 g2;
        g2.hi = __shfl_xor_sync(0xffffffffu, f.hi, o);
        g2.lo = __shfl_xor_sync(0xffffffffu, f.lo, o);
        fix_add(f, g2);
      }
      if (lane == 0) { sh.key = kk; sh.sum = fix_value(f, emax); }
    }
    __syncthreads();
    if (tid == 0 && !sh.stop) {
      bool reached;
      if (k == 0) {
        sh.fro2 = sh.sum;
        Fix128 t = {0ull, 0ull};
        if (it.tol > 0.0) fix_add(t, it.tol * it.tol * sh.fro2, sh.emax);
        sh.thr = t;
        reached = it.tol > 0.0 && sh.sum <= it.tol * it.tol * sh.fro2;
      } else {
        reached = it.tol > 0.0 && fix_le(sh.fsum, sh.thr);
      }
      if (reached) {
        sh.stop = 1;
        sh.status = FFC_OK;
      } else if (k >= kmax || (sh.key >> 20) == 0ull) {
        sh.stop = 1;
        sh.status = it.tol > 0.0 ? FFC_E_TOL_NOT_REACHED : FFC_OK;
      }
    }
    __syncthreads();
    if (sh.stop) break;
    const int p = 0xFFFFF - (int)(sh.key & 0xFFFFFull);
    const int j = k - k0;   // step within the panel
    T* __restrict__ vj = Vs + (int64_t)j * ldv;
    // the pivot's squared norm (the key's top bits); at a panel's first step it bounds every free column
    const double pk2 = __longlong_as_double((long long)(sh.key & ~0xFFFFFull));
    if (j == 0) pn0 = pk2;

    // ---- the pivot column's current rows k..s-1 into V(:, j): A(:, p) - V(:, 0:j) F(p, 0:j)^T
    if (tid < j) fsh[tid] = __ldcg(F + (int64_t)p * QR_NB_MAX + tid);
    __syncthreads();
    {
      const T* cp = A + (int64_t)p * lda;
      T part = (T)0;
      const int kb = k & ~(W - 1);
      const int iend = min(ldv, ((s + 7) & ~7) + 8);
      for (int i = kb + tid; i < iend; i += QR_THREADS) {
        T x = (T)0;
        if (i >= k && i < s) {
          x = __ldcg(cp + i);
          for (int t = 0; t < j; ++t) x = fma(-Vs[(int64_t)t * ldv + i], fsh[t], x);
          if (i > k) part = fma(x, x, part);
        }
        vj[i] = x;   // rows kb..k-1 and the padding past s are zero
      }
      part = warp_sum(part);
      if (lane == 0) {
        if (sizeof(T) == 8) sh.dw[warp] = (double)part; else sh.fw[warp] = (float)part;
      }
    }
    __syncthreads();
    if (tid == 0) {
      T xn2 = (T)0;
      for (int w = 0; w < QR_WARPS; ++w) xn2 += sizeof(T) == 8 ? (T)sh.dw[w] : (T)sh.fw[w];
      const T alpha = vj[k];
      if (xn2 == (T)0) {
        sh.tau = 0.0;
        sh.tauf = 0.0f;
        sh.apply = 0;
        sh.beta = (double)alpha;
        vj[k] = (T)0;   // H = I: v is not used (tau = 0), the scale below must not touch it
      } else {
        const T nrm = sqrt(fma(alpha, alpha, xn2));
        const T beta = alpha >= (T)0 ? -nrm : nrm;
        const T tt = (beta - alpha) / beta;
        sh.tau = (double)tt;
        sh.tauf = (float)tt;
        sh.apply = 1;
        sh.beta = (double)beta;
        vj[k] = (T)1 / (alpha - beta);   // the scale, read below, then replaced by 1
      }
      if (a.rank == 0) { it.piv[k] = p; it.beta[k] = sh.beta; }
      if (p >= c0 && p < c1) sels[p - c0] = 1;
    }
    __syncthreads();
    const bool apply = sh.apply != 0;
    if (apply) {
      const T scale = vj[k];
      for (int i = k + 1 + tid; i < s; i += QR_THREADS) vj[i] = vj[i] * scale;
    }
    __syncthreads();
    if (tid == 0) vj[k] = apply ? (T)1 : (T)0;
    __syncthreads();
    // w(t) = V(k:s, t)^T v_j for the panel's earlier reflectors (warp t, t + 8, ...)
    for (int t = warp; t < j; t += QR_WARPS) {
      const T* vt = Vs + (int64_t)t * ldv;
      T acc = (T)0;
      for (int i = k + lane; i < s; i += 32) acc = fma(vt[i], vj[i], acc);
      acc = warp_sum(acc);
      if (lane == 0) wsh[t] = acc;
    }
    __syncthreads();

    // ---- owned free columns: F(c, j), the pivot row, the norm downdate; 4 columns per warp pass
    const T ttau = sizeof(T) == 8 ? (T)sh.tau : (T)sh.tauf;
    const int emax = sh.emax;
    unsigned long long key = 0ull;
    Fix128 psum = {0ull, 0ull};
    const int vrows = s - (k & ~(W - 1));
#define FFC_BCOLS(NC_, M_, CH_)                                                                              \
  blocked_columns<T, NC_, M_, CH_>(A, lda, F, Fs, nb, c0, ncols, sels, vj, Vs, ldv, wsh, ttau, apply, k, j, s, \
                                   warp, lane, TOL3Z, vn1s, vn2s, key, psum, emax)
    if (vrows <= 32 * W) FFC_BCOLS(8, 1, false);
    else if (vrows <= 64 * W) FFC_BCOLS(4, 2, false);
    else if (vrows <= 128 * W) FFC_BCOLS(2, 4, false);
    else if (vrows <= 256 * W) FFC_BCOLS(1, 8, false);
    else if (BIG && vrows <= 512 * W) FFC_BCOLS(1, 16, false);
    else FFC_BCOLS(1, 8, true);
#undef FFC_BCOLS
    __syncthreads();   // every F(c, j) and pivot-row write of this CTA is done

    // ---- end of the panel: apply it to the rows below once (not after the last step). A panel also
    // ends once the pivot norm has fallen below a quarter of the panel's first: the current column is
    // formed as the panel-start column minus V F^T, whose rounding scales with the panel-start norm
    // (bounded by the first pivot's), so this keeps that error within 4x of the unblocked form's for
    // every column that competes for the next pivot. The rule reads only the group-wide pivot norms.
    const bool last = (k + 1 >= kmax);
    if ((j + 1 == nb || pk2 * 16.0 < pn0) && !last) {
      const int jn = j + 1, kend = k + 1;
      const int kbe = kend & ~(W - 1);
      for (int jc = warp; jc < ncols; jc += QR_WARPS) {
        if (sels[jc]) continue;
        T* col = A + (int64_t)(c0 + jc) * lda;
        const T* fr = Fs + jc * nb;
        for (int r0 = kbe + W * lane; r0 < s; r0 += 32 * W) {
          V4 x = *reinterpret_cast<const V4*>(col + r0);
          for (int t = 0; t < jn; ++t) {
            const V4 vt = *reinterpret_cast<const V4*>(Vs + (int64_t)t * ldv + r0);
            const T ft = fr[t];
#pragma unroll
            for (int e = 0; e < W; ++e) vset(x, e, fma(-vget(vt, e), ft, vget(x, e)));
          }
          // rows below kend only (rows kbe..kend-1 are R and stay), rows past s untouched
#pragma unroll
          for (int e = 0; e < W; ++e)
            if (r0 + e < kend || r0 + e >= s) vset(x, e, col[min(r0 + e, s - 1)]);
          if (r0 + W <= s && r0 >= kend) {
            *reinterpret_cast<V4*>(col + r0) = x;
          } else {
#pragma unroll
            for (int e = 0; e < W; ++e)
              if (r0 + e >= kend && r0 + e < s) col[r0 + e] = vget(x, e);
          }
        }
      }
      k0 = k + 1;
      __syncthreads();
    }
    cta_reduce_fix(key, psum, sh);
  }

  if (tid == 0) {
    if (sh.status == FFC_E_TIMEOUT) atomicExch(it.status_out, (int)FFC_E_TIMEOUT);
    if (a.rank == 0) {
      *it.rank_out = k;
      const double fin = k == 0 ? sh.sum : fix_value(sh.fsum, sh.emax);
      *it.r22_out = sh.fro2 > 0.0 ? sqrt(fin) / sqrt(sh.fro2) : 0.0;
      if (sh.status != FFC_E_TIMEOUT) atomicCAS(it.status_out, (int)FFC_OK, sh.status);
    }
  }
  for (int j = tid; j < ncols; j += QR_THREADS) it.selected[c0 + j] = sels[j];
}

template <typename T, bool BIG, int LZ = 0>
__global__ void __launch_bounds__(QR_THREADS, BIG ? 2 : FFC_QR_MIN_BLOCKS)
cpqr_kernel(const CpqrItem* __restrict__ items, const CtaAssign* __restrict__ entries,
            const int32_t* __restrict__ cta_off, long long spin_limit, int s_max, int nb, int defer) {
  (void)nb;
  // dynamic shared memory: vn1, vn2 (QR_NCOL_MAX doubles each), row-k entries
  // (QR_NCOL_MAX T), recompute list (QR_NCOL_MAX int16), selected flags
  // (QR_NCOL_MAX bytes), Householder vector (s_max T)
  extern __shared__ __align__(16) unsigned char qsm[];
  double* vn1s = reinterpret_cast<double*>(qsm);
  double* vn2s = vn1s + QR_NCOL_MAX;
  T* aks = reinterpret_cast<T*>(vn2s + QR_NCOL_MAX);
  int16_t* rcl = reinterpret_cast<int16_t*>(aks + QR_NCOL_MAX);
  uint8_t* sels = reinterpret_cast<uint8_t*>(rcl + QR_NCOL_MAX);
  T* vsh = reinterpret_cast<T*>(sels + QR_NCOL_MAX);
  // LAZY: the reflector ring (QR_DEFER_MAX slots of qr_ldv(s_max) floats), its taus and the pivot's rows
  const int ldv = qr_ldv(s_max);
  float* ring = reinterpret_cast<float*>(vsh + (std::max(s_max, 1) + 8));
  float* taur = ring + (size_t)QR_DEFER_MAX * ldv;
  float* keep = taur + QR_DEFER_MAX;
  __shared__ QrShared sh;
  const int e0 = cta_off ? cta_off[blockIdx.x] : (int)blockIdx.x;
  const int e1 = cta_off ? cta_off[blockIdx.x + 1] : (int)blockIdx.x + 1;
  for (int e = e0; e < e1; ++e) {
    const CtaAssign a = entries[e];
    const CpqrItem it = items[a.item];
    if (threadIdx.x == 0) sh.status = FFC_OK;
    __syncthreads();
    factor_item<T, BIG, LZ>(it, a, vsh, vn1s, vn2s, aks, sels, rcl, sh, spin_limit, ring, ldv, taur, keep, defer);
    __syncthreads();
  }
}

// The blocked form (every item has F; columns 16-byte aligned): CTA work lists as in cpqr_kernel.
template <typename T, bool BIG>
__global__ void __launch_bounds__(QR_THREADS, BIG ? 2 : FFC_QR_MIN_BLOCKS)
cpqr_blocked_kernel(const CpqrItem* __restrict__ items, const CtaAssign* __restrict__ entries,
                    const int32_t* __restrict__ cta_off, long long spin_limit, int s_max, int nb, int defer) {
  (void)defer;
  extern __shared__ __align__(16) unsigned char qsm[];
  double* vn1s = reinterpret_cast<double*>(qsm);
  double* vn2s = vn1s + QR_NCOL_MAX;
  uint8_t* sels = reinterpret_cast<uint8_t*>(vn2s + QR_NCOL_MAX);
  // the panel's reflectors V (nb x ldv), w (QR_NB_MAX) and F rows (QR_NB_MAX, then one per warp)
  const int ldv = qr_ldv(s_max);
  T* Vs = reinterpret_cast<T*>(qsm + qr_blocked_off<T>(s_max));
  T* wsh = Vs + (size_t)nb * ldv;
  T* fsh = wsh + QR_NB_MAX;
  T* Fs = fsh + QR_NB_MAX * (1 + QR_WARPS);   // F rows of the CTA's columns (QR_FS_COLS x nb)
  __shared__ QrShared sh;
  const int e0 = cta_off ? cta_off[blockIdx.x] : (int)blockIdx.x;
  const int e1 = cta_off ? cta_off[blockIdx.x + 1] : (int)blockIdx.x + 1;
  for (int e = e0; e < e1; ++e) {
    const CtaAssign a = entries[e];
    const CpqrItem it = items[a.item];
    if (threadIdx.x == 0) sh.status = FFC_OK;
    __syncthreads();
    factor_item_blocked<T, BIG>(it, a, vn1s, vn2s, sels, Vs, ldv, wsh, fsh, Fs, nb, sh, spin_limit);
    __syncthreads();
  }
}

// FP32 blocks: the register-resident variant (2 CTAs per SM) when the caller asks for it, by
// default from s = 1,024 on (measured faster there; at s = 512 the third CTA per SM is worth more)
template <typename T>
bool qr_big(int s_max, int big) {
  if (sizeof(T) != 4) return false;
  return big < 0 ? s_max >= QR_BIG_MIN_S_DEFAULT : big != 0;
}

using QrKernel = void (*)(const CpqrItem*, const CtaAssign*, const int32_t*, long long, int, int, int);

// the lazy form runs with a ring of defer >= 2 reflectors: FP32 register-resident (BIG) rounds whose columns
// fit the registers whole (s a multiple of 128, at most 2,048), unblocked
template <typename T>
bool qr_lazy(int s_max, int big, int nb, int defer) {
  return defer >= 2 && nb <= 1 && sizeof(T) == 4 && qr_big<T>(s_max, big) && s_max % 128 == 0 && s_max <= 2048;
}

template <typename T>
QrKernel qr_kernel_fn(int s_max, int big, int nb, int defer = 0) {
  const bool b = qr_big<T>(s_max, big);
  if (nb > 1) return b ? cpqr_blocked_kernel<T, true> : cpqr_blocked_kernel<T, false>;
  if constexpr (sizeof(T) == 4) {
    if (qr_lazy<T>(s_max, big, nb, defer)) return s_max > 1024 ? cpqr_kernel<T, true, 16> : cpqr_kernel<T, true, 8>;
  }
  return b ? cpqr_kernel<T, true> : cpqr_kernel<T, false>;
}

template <typename T>
size_t cpqr_smem_bytes(int s_max, int nb = 1, int defer = 0, int big = -1) {
  // the Householder vector follows the per-column arrays; 8 spare elements keep the vector loads of its
  // final (partial) 16-byte group inside the allocation; the blocked form's arrays or the lazy form's
  // ring, taus and pivot rows come after it
  const size_t base = QR_NCOL_MAX * (2 * sizeof(double) + sizeof(T) + sizeof(int16_t) + 1) +
                      (size_t)(std::max(s_max, 1) + 8) * sizeof(T);
  if (qr_lazy<T>(s_max, big, nb, defer))
    return base + ((size_t)QR_DEFER_MAX * qr_ldv(s_max) + 2 * QR_DEFER_MAX) * sizeof(float);
  if (nb <= 1) return base;
  return qr_blocked_off<T>(s_max) +
         ((size_t)nb * qr_ldv(s_max) + QR_NB_MAX * (2 + QR_WARPS) + (size_t)QR_FS_COLS * nb) * sizeof(T);
}

template <typename T>
ffc_status launch_cpqr_t(const CpqrItem* items, const CtaAssign* assign, const int32_t* cta_off, int grid,
                         int s_max, cudaStream_t st, int big, int nb, int defer) {
  if (defer < 0 || defer > QR_DEFER_MAX) {
    set_error("cpqr: deferral depth %d outside [0, %d]", defer, QR_DEFER_MAX);
    return FFC_E_INVALID;
  }
  if (s_max > 2048) {
    set_error("cpqr: s = %d exceeds the supported 2048 rows", s_max);
    return FFC_E_INVALID;
  }
  if (nb < 1 || nb > QR_PANEL_MAX) {
    set_error("cpqr: panel width %d outside [1, %d]", nb, QR_PANEL_MAX);
    return FFC_E_INVALID;
  }
  const size_t smem = cpqr_smem_bytes<T>(s_max, nb, defer, big);
  auto kfn = qr_kernel_fn<T>(s_max, big, nb, defer);
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
  FFC_CUDA(cudaLaunchKernelEx(&cfg, kfn, items, assign, cta_off, wait_limit(), s_max, nb,
                              qr_lazy<T>(s_max, big, nb, defer) ? defer : 1));
  return FFC_OK;
}

template <typename T>
int max_ctas_t(int s_max, int big, int nb, int defer) {
  int per_sm = 0;
  const size_t smem = cpqr_smem_bytes<T>(s_max, nb, defer, big);
  auto kfn = qr_kernel_fn<T>(s_max, big, nb, defer);
  cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, QR_THREADS, smem);
  return per_sm * sm_count();
}

}  // namespace

int cpqr_min_group(int64_t n) { return (int)std::max<int64_t>(1, (n + QR_NCOL_MAX - 1) / QR_NCOL_MAX); }

int cpqr_max_ctas(int precision, int s_max, int big, int nb, int defer) {
  return precision == FFC_MIXED ? max_ctas_t<float>(s_max, big, nb, defer) : max_ctas_t<double>(s_max, 0, nb, 0);
}

int qr_panel(int precision, int s_max, int big, bool blocked) {
  // The library's default is the unblocked form: on the L2-resident sub-batches the rounds run in, a
  // step is bound by its synchronisation (the blocked form halves the bytes a step moves but adds
  // serial phases between block barriers and measured slower). With `blocked`, the widest panel that
  // fits: FP32 rounds from s = 1,024 on (smaller rounds are latency bound; FP64 is FMA bound).
  if (!blocked || precision != FFC_MIXED || s_max < QR_BLOCKED_MIN_S) return 1;
  // V gets about 68 KB of shared memory with 2 CTAs per SM, 40 KB with 3; a power of two <= 32
  const size_t esz = precision == FFC_MIXED ? sizeof(float) : sizeof(double);
  const bool two = precision == FFC_MIXED && qr_big<float>(s_max, big);
  const size_t budget = two ? (68u << 10) : (40u << 10);
  // FP32 panels wider than 8 let the within-panel cancellation (panel-start column minus V F^T) move
  // the tolerance stop by several ranks; up to 8 it stays within one rank of the unblocked form
  const int nb_cap = QR_PANEL_MAX;
  int nb = 1;
  while (2 * nb <= nb_cap && (size_t)(2 * nb) * qr_ldv(s_max) * esz <= budget) nb *= 2;
  return nb;
}

ffc_status launch_cpqr(int precision, const CpqrItem* items_dev, const CtaAssign* assign_dev, int grid, int s_max,
                       cudaStream_t st, const int32_t* cta_off, int big, int nb, int defer) {
  if (grid <= 0) return FFC_OK;
  if (precision == FFC_MIXED)
    return launch_cpqr_t<float>(items_dev, assign_dev, cta_off, grid, s_max, st, big, nb, defer);
  return launch_cpqr_t<double>(items_dev, assign_dev, cta_off, grid, s_max, st, 0, nb, 0);
}

bool cpqr_lazy(int precision, int s_max, int big, int nb, int defer) {
  return precision == FFC_MIXED && qr_lazy<float>(s_max, big, nb, defer);
}

}  // namespace ffc
