// Kernel-block evaluation on the fifth-generation tensor cores (tcgen05, TMEM accumulators, TMA
// staging): mixed precision, Gaussian and polynomial kernels, K'_ij = K(Y[rows_i], X_j) from the
// inner products y_i . x_j (§2.2 block; kernels of §4.2 and §4.4).
//
// Arithmetic (the same as the mma.sync path): every FP32 coordinate a, centred at the node
// centroid for the Gaussian, is split into three BF16 parts a = a_hi + a_mid + a_lo (each the BF16
// rounding of the remainder), and the inner product keeps the six partial products of order at
// least 2^-16, accumulated in FP32 from the smallest up:
//   lo.hi + hi.lo + mid.mid + mid.hi + hi.mid + hi.hi.
// D2_ij = ||y_i||^2 + ||x_j||^2 - 2 y_i . x_j; where it cancels (D2 < (||y||^2 + ||x||^2) / 16) the
// epilogue recomputes it from direct FP32 differences.
//
// Two kernels:
// 1. prep: one warp per row writes the row's three BF16 planes (rows of d_pad = 32-multiple
//    coordinates, zero beyond d) and its FP32 squared norm into a scratch arena. Item q owns
//    rows [3 base_q, 3 (base_q + s_pad_q + n_pad_q)): the targets' planes hi/mid/lo (s_pad_q rows
//    each, a multiple of 128), then the sources' (n_pad_q rows each, a multiple of 256).
// 2. main: a persistent CTA per SM walks 128 x 256 output tiles. Warp 0 (one lane) streams the
//    planes in k-blocks of 32 coordinates with cp.async.bulk.tensor (64-byte swizzle) into a
//    3-stage ring; warp 1 (one lane) issues tcgen05.mma kind::f16 (M = 128, N = 256, K = 16, BF16
//    in, FP32 accumulate) into one of two TMEM accumulators of 256 columns; warps 2-5 read the
//    other accumulator with tcgen05.ld, apply the kernel and store the column-major block. Stage
//    and accumulator hand-offs are mbarriers; every wait is bounded (ffc_set_wait_limit) and a
//    wait that runs out stops all roles, drains the copies and products in flight, frees TMEM and
//    reports FFC_E_TIMEOUT.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "ffc_internal.cuh"

namespace ffc {

namespace {

constexpr int T5_M = 128;          // output rows per tile (targets)
constexpr int T5_THREADS = 192;    // producer, MMA, 4 epilogue warps
constexpr int T5_DPAD = 64;        // coordinates are padded to a multiple of the widest stage

// Tile variants: N sources per tile, BK coordinates per stage (rows of 2 BK bytes, swizzled on that
// width), NST stages in the ring; the two TMEM accumulators take 2 N columns.
template <int BN, int BK, int NST>
struct T5Cfg {
  static constexpr int N = BN, KB = BK, STAGES = NST;
  static constexpr int A_PLANE = T5_M * BK * 2;               // bytes of one plane's box
  static constexpr int B_PLANE = BN * BK * 2;
  static constexpr int STAGE = 3 * A_PLANE + 3 * B_PLANE;
  static constexpr int BAR_OFF = NST * STAGE;
  static constexpr int SMEM = BAR_OFF + 256 + 1024;           // + barriers, + alignment slack
  static constexpr int TMEM_COLS = 2 * BN;
  static constexpr int SW = 2 * BK;                           // swizzle span in bytes: 32, 64 or 128
  // UMMA layout type of the swizzle (32 B: 6, 64 B: 4, 128 B: 2) and the 8-row group stride
  static constexpr uint64_t LAYOUT = SW == 128 ? 2 : SW == 64 ? 4 : 6;
  static constexpr uint32_t SBO = 8 * SW;
  // instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B
  // (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(T5_M >> 4) << 24);
  static_assert(STAGE % 1024 == 0, "stages keep the 1024-byte alignment of the swizzle atoms");
  static_assert(SMEM <= 232448, "shared memory per CTA");
  static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256 && (BK == 16 || BK == 32 || BK == 64), "tile shape");
  static_assert(T5_DPAD % BK == 0, "coordinate padding");
};
using T5V0 = T5Cfg<256, 32, 3>;   // 72 KB stages
using T5V1 = T5Cfg<128, 64, 2>;   // 96 KB stages, 128-byte swizzle
using T5V2 = T5Cfg<128, 32, 4>;   // 48 KB stages
using T5V3 = T5Cfg<256, 16, 6>;   // 36 KB stages, 32-byte swizzle
using T5V4 = T5Cfg<128, 16, 8>;   // 24 KB stages
constexpr int T5_VARIANTS = 5;
__host__ __device__ constexpr int t5_bn(int v) { return (v == 0 || v == 3) ? 256 : 128; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity (polled at least once): false when the poll limit
// ran out (the abort flag is then raised) or another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit, volatile int* abort_flag) {
  for (long long t = 0;; ++t) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (t >= limit) break;
  }
  *abort_flag = 1;
  return false;
}
// Teardown wait for copies or products already issued: bounded by the default limit whatever the
// caller's (they complete in microseconds), and deaf to the abort flag.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (long long t = 0; t < SPIN_LIMIT_DEFAULT; ++t)
    if (mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile with a swizzled layout: rows of SW bytes,
// 8-row groups SBO bytes apart (stride byte offset); the leading byte offset is unused for swizzled
// K-major tiles (encoded 1); bit 46 is the descriptor version of tcgen05; bits 61-63 the layout.
template <class C>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(C::SBO >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= C::LAYOUT << 61;
  return d;
}

template <class C>
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(C::IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes (one row per thread), waited on
// in the same statement so that no use of the registers is scheduled before the load completes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int e = 0; e < 32; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ int find_item_t5(const EvalItem* items, int n_items, int64_t g) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].tile_begin <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int find_row_item_t5(const EvalItem* items, int n_items, int64_t r) {
  int lo = 0, hi = n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].tc_base <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void split3_t5(float a, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

// One coordinate, centred: FP32 points against the FP32 rounding of the centre (common to targets
// and sources, so it cancels in their differences), FP64 points in FP64 before the rounding.
template <typename TP>
__device__ __forceinline__ float centred(const TP* row, int k, const double* ctr);
template <>
__device__ __forceinline__ float centred<float>(const float* row, int k, const double* ctr) {
  const float a = __ldg(row + k);
  return ctr ? a - (float)ctr[k] : a;
}
template <>
__device__ __forceinline__ float centred<double>(const double* row, int k, const double* ctr) {
  const double a = __ldg(row + k);
  return (float)(ctr ? a - ctr[k] : a);
}

// ---------------------------------------------------------------------------------------------
// prep: one warp per arena row; lane l covers coordinates [k0 + 8 l, k0 + 8 l + 8) of each 256-wide
// chunk (16-byte stores per plane). The squared norm is the FP32 sum of the lane's squares in
// increasing k, then a fixed xor-shuffle tree.
template <typename TP, int MODE>
__global__ void __launch_bounds__(256)
tc5_prep_kernel(const TP* __restrict__ Y, const TP* __restrict__ X, int d, int d_pad,
                const EvalItem* __restrict__ items, int n_items, int64_t total_rows,
                __nv_bfloat16* __restrict__ planes, float* __restrict__ norms) {
  const int lane = threadIdx.x & 31;
  const int64_t gr = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (gr >= total_rows) return;   // uniform per warp
  const int q = find_row_item_t5(items, n_items, gr);
  const EvalItem& it = items[q];
  const int64_t local = gr - it.tc_base;
  const int64_t sp = it.tc_spad, np = it.tc_npad;
  const bool is_a = local < sp;
  const int64_t r = is_a ? local : local - sp;
  const bool valid = is_a ? r < it.s : r < it.n;
  const double* ctr = MODE == 0 ? it.center : nullptr;
  const TP* row = nullptr;
  if (valid) row = is_a ? Y + it.rows[r] * (int64_t)d : X + (it.x_begin + r) * (int64_t)d;
  const int64_t base = 3 * it.tc_base;
  const int64_t prow = is_a ? base + r : base + 3 * sp + r;   // plane 0's row; plane p adds p * (s_pad or n_pad)
  const int64_t pstep = is_a ? sp : np;
  float nrm = 0.0f;
  for (int k0 = 0; k0 < d_pad; k0 += 256) {
    const int kb = k0 + 8 * lane;
    if (kb >= d_pad) break;
    __align__(16) __nv_bfloat16 ph[8], pm[8], pl[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kb + e;
      const float a = (valid && k < d) ? centred<TP>(row, k, ctr) : 0.0f;
      nrm = fmaf(a, a, nrm);
      split3_t5(a, ph[e], pm[e], pl[e]);
    }
    *reinterpret_cast<uint4*>(planes + prow * d_pad + kb) = *reinterpret_cast<const uint4*>(ph);
    *reinterpret_cast<uint4*>(planes + (prow + pstep) * d_pad + kb) = *reinterpret_cast<const uint4*>(pm);
    *reinterpret_cast<uint4*>(planes + (prow + 2 * pstep) * d_pad + kb) = *reinterpret_cast<const uint4*>(pl);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
  if (lane == 0) norms[gr] = nrm;
}

struct T5Tile {
  int q;
  int64_t i0, j0;
  bool skip;
};

template <int BN>
__device__ __forceinline__ T5Tile tile_of(const EvalItem* items, int n_items, int64_t g) {
  T5Tile t;
  t.q = find_item_t5(items, n_items, g);
  const EvalItem& it = items[t.q];
  const int64_t rt = it.row_tiles > 0 ? it.row_tiles : 1;
  const int64_t local = g - it.tile_begin;
  t.i0 = (local % rt) * T5_M;
  t.j0 = (local / rt) * BN;
  t.skip = t.i0 >= it.s || t.j0 >= it.n;
  return t;
}

// ---------------------------------------------------------------------------------------------
// main kernel. MODE 0: Gaussian (centred distances), 2: polynomial (inner products).
template <typename TP, int MODE, class C>
__global__ void __launch_bounds__(T5_THREADS, 1)
tc5_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
           const TP* __restrict__ Y, const TP* __restrict__ X, int d, int d_pad, ffc_kernel kp,
           const EvalItem* __restrict__ items, int n_items, int64_t total_tiles, const float* __restrict__ norms,
           long long limit, int32_t* __restrict__ status) {
  extern __shared__ unsigned char t5_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(t5_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + C::BAR_OFF);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accfull = empty + C::STAGES;
  uint64_t* accempty = accfull + 2;
  uint64_t* done = accempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* fault_item = reinterpret_cast<int*>(tmem_slot + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&accfull[b], 1); mbar_init(&accempty[b], 4); }
    mbar_init(done, 1);
    *abort_flag = 0;
    *fault_item = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == 1) {   // the whole warp allocates the two accumulators (512 columns)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int KB = d_pad / C::KB;

  if (warp == 0) {
    // ---- producer ----
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      long long u = 0;
      bool ok = true;
      for (int64_t g = blockIdx.x; g < total_tiles && ok; g += gridDim.x) {
        const T5Tile t = tile_of<C::N>(items, n_items, g);
        if (t.skip) continue;
        const EvalItem& it = items[t.q];
        const int64_t base = 3 * it.tc_base;
        const int arow = (int)(base + t.i0), brow = (int)(base + 3 * it.tc_spad + t.j0);
        for (int kb = 0; kb < KB; ++kb, ++u) {
          const int st = (int)(u % C::STAGES);
          const uint32_t ph = (uint32_t)((u / C::STAGES) & 1);
          if (!mbar_wait(&empty[st], ph ^ 1u, limit, abort_flag)) { *fault_item = t.q; ok = false; break; }
          unsigned char* sa = sm + st * C::STAGE;
          unsigned char* sb = sa + 3 * C::A_PLANE;
          mbar_expect_tx(&full[st], (uint32_t)C::STAGE);
          const int x = kb * C::KB;
#pragma unroll
          for (int p = 0; p < 3; ++p) tma_load_2d(sa + p * C::A_PLANE, &tmA, &full[st], x, arow + p * (int)it.tc_spad);
#pragma unroll
          for (int p = 0; p < 3; ++p) tma_load_2d(sb + p * C::B_PLANE, &tmB, &full[st], x, brow + p * (int)it.tc_npad);
        }
      }
      // copies still in flight complete before the CTA leaves (bounded)
      for (long long v = u > C::STAGES ? u - C::STAGES : 0; v < u; ++v)
        mbar_drain(&full[v % C::STAGES], (uint32_t)((v / C::STAGES) & 1));
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      long long u = 0, tcount = 0;
      bool ok = true;
      for (int64_t g = blockIdx.x; g < total_tiles && ok; g += gridDim.x) {
        const T5Tile t = tile_of<C::N>(items, n_items, g);
        if (t.skip) continue;
        const int buf = (int)(tcount & 1);
        const uint32_t aph = (uint32_t)((tcount >> 1) & 1);
        ++tcount;
        if (!mbar_wait(&accempty[buf], aph ^ 1u, limit, abort_flag)) { *fault_item = t.q; break; }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * C::N);
        for (int kb = 0; kb < KB; ++kb, ++u) {
          const int st = (int)(u % C::STAGES);
          const uint32_t ph = (uint32_t)((u / C::STAGES) & 1);
          if (!mbar_wait(&full[st], ph, limit, abort_flag)) { *fault_item = t.q; ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(sm + st * C::STAGE);
          const uint32_t sb = sa + 3 * C::A_PLANE;
#pragma unroll
          for (int ks = 0; ks < C::KB / 16; ++ks) {
            // planes: A at sa + pa * 8 KB, B at sb + pb * 16 KB; the k-step advances 32 bytes
            const uint64_t a0 = sdesc<C>(sa + ks * 32), a1 = sdesc<C>(sa + C::A_PLANE + ks * 32),
                           a2 = sdesc<C>(sa + 2 * C::A_PLANE + ks * 32);
            const uint64_t b0 = sdesc<C>(sb + ks * 32), b1 = sdesc<C>(sb + C::B_PLANE + ks * 32),
                           b2 = sdesc<C>(sb + 2 * C::B_PLANE + ks * 32);
            const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
            umma_bf16<C>(dt, a2, b0, first);   // lo . hi
            umma_bf16<C>(dt, a0, b2, 1u);      // hi . lo
            umma_bf16<C>(dt, a1, b1, 1u);      // mid . mid
            umma_bf16<C>(dt, a1, b0, 1u);      // mid . hi
            umma_bf16<C>(dt, a0, b1, 1u);      // hi . mid
            umma_bf16<C>(dt, a0, b0, 1u);      // hi . hi
          }
          umma_commit(&empty[st]);   // the stage is free once these products have read it
        }
        if (!ok) break;
        umma_commit(&accfull[buf]);
      }
      // every product issued has completed before TMEM is released (bounded)
      umma_commit(done);
      mbar_drain(done, 0u);
    }
  } else {
    // ---- epilogue: warps 2..5 read TMEM lanes 32 (warp % 4) .. + 31 ----
    const int quarter = warp & 3;
    const int li = 32 * quarter + lane;
    const float inv2h2 = (float)(0.5 / (kp.h * kp.h));
    const float invh = (float)(1.0 / kp.h), cc = (float)kp.c;
    long long tcount = 0;
    for (int64_t g = blockIdx.x; g < total_tiles; g += gridDim.x) {
      const T5Tile t = tile_of<C::N>(items, n_items, g);
      if (t.skip) continue;
      const int buf = (int)(tcount & 1);
      const uint32_t aph = (uint32_t)((tcount >> 1) & 1);
      ++tcount;
      bool ok = mbar_wait(&accfull[buf], aph, limit, abort_flag);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) { if (lane == 0) *fault_item = t.q; break; }
      tc_fence_after();
      // the item's fields in registers (the stores below could otherwise force their reloads)
      const EvalItem* ip = items + t.q;
      const int64_t s_it = ip->s, n_it = ip->n, ldk = ip->ldk, xb = ip->x_begin, nb = ip->tc_base + ip->tc_spad;
      float* __restrict__ K = reinterpret_cast<float*>(ip->K);
      const double* ctr = MODE == 0 ? ip->center : nullptr;
      const int64_t i = t.i0 + li;
      const bool vi = i < s_it;
      float ny = 0.0f;
      int64_t yrow = 0;
      if (vi) {
        ny = norms[ip->tc_base + i];
        if (MODE == 0) yrow = ip->rows[i];
      }
      const int64_t jrem = n_it - t.j0;
      const int jn = jrem < (int64_t)C::N ? (int)jrem : C::N;
      float* __restrict__ Kcol = K + i + t.j0 * ldk;   // this thread's row, column j0 of the tile
      for (int c = 0; c < C::N / 32; ++c) {
        float v[32];
        __syncwarp();
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(buf * C::N + 32 * c), v);
        if (c == C::N / 32 - 1) {   // the accumulator is free for the next tile's products
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&accempty[buf]);
        }
        // the chunk's 32 source norms, one per lane, broadcast below
        float nxl = 0.0f;
        if (MODE == 0 && 32 * c + lane < jn) nxl = __ldg(norms + nb + t.j0 + 32 * c + lane);
        uint32_t redo = 0u;   // Gaussian entries whose D2 cancels: recomputed after the chunk
        if (MODE == 0) {
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            const float nx = __shfl_sync(0xffffffffu, nxl, e);
            const float d2 = ny + nx - 2.0f * v[e];
            if (d2 < 0.0625f * (ny + nx)) redo |= 1u << e;
            v[e] = expf(-fmaxf(d2, 0.0f) * inv2h2);
          }
        } else {
          // (x.y / h + c)^p: the power's loop outside, 32 independent products inside
          float b[32];
#pragma unroll
          for (int e = 0; e < 32; ++e) {
            b[e] = v[e] * invh + cc;
            v[e] = b[e];
          }
          for (int s2 = 1; s2 < kp.p; ++s2) {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] *= b[e];
          }
        }
#pragma unroll
        for (int e = 0; e < 32; ++e)
          if (vi && 32 * c + e < jn) Kcol[(int64_t)(32 * c + e) * ldk] = v[e];
        if (MODE == 0 && vi) {
          // cancellation: direct FP32 differences of the same centred, rounded coordinates
          redo &= jn - 32 * c >= 32 ? 0xffffffffu : (jn - 32 * c > 0 ? (1u << (jn - 32 * c)) - 1u : 0u);
          while (redo) {
            const int e = __ffs(redo) - 1;
            redo &= redo - 1u;
            const int jl = 32 * c + e;
            const TP* yr = Y + yrow * (int64_t)d;
            const TP* xr = X + (xb + t.j0 + jl) * (int64_t)d;
            float a2 = 0.0f;
            for (int k = 0; k < d; ++k) {
              const float df = centred<TP>(yr, k, ctr) - centred<TP>(xr, k, ctr);
              a2 = fmaf(df, df, a2);
            }
            Kcol[(int64_t)jl * ldk] = expf(-fmaxf(a2, 0.0f) * inv2h2);
          }
        }
      }
    }
  }
  // teardown: all roles have left their loops; the accumulators are released by the warp that took them
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)C::TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && *abort_flag && status) atomicExch(status + *fault_item, (int)FFC_E_TIMEOUT);
}

}  // namespace

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no link to the driver library).
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      (void)cudaGetLastError();
  });
  return fn;
}

size_t plane_bytes(int64_t total_rows, int d) {
  return ((size_t)3 * (size_t)total_rows * (size_t)eval_tc5_dpad(d) * 2 + 255) & ~size_t(255);
}

}  // namespace

int64_t eval_tc5_pad_s(int64_t s) { return (s + T5_M - 1) / T5_M * T5_M; }
int64_t eval_tc5_pad_n(int64_t n) { return (n + 255) / 256 * 256; }   // a multiple of every variant's N
int eval_tc5_dpad(int d) { return (d + T5_DPAD - 1) / T5_DPAD * T5_DPAD; }
int64_t eval_tc5_tiles(int64_t s, int64_t n, int v) {
  const int bn = t5_bn(v);
  return ((s + T5_M - 1) / T5_M) * ((n + bn - 1) / bn);
}
int64_t eval_tc5_row_tiles(int64_t s) { return (s + T5_M - 1) / T5_M; }
size_t eval_tc5_scratch_bytes(int64_t total_rows, int d) {
  return plane_bytes(total_rows, d) + (size_t)total_rows * sizeof(float) + 256;
}

namespace {

template <typename TP, int MODE, class C>
ffc_status launch_t5(const CUtensorMap& tmA, const CUtensorMap& tmB, const TP* Y, const TP* X, int d, int dp,
                     ffc_kernel k, const EvalItem* items_dev, int n_items, int64_t total_tiles, const float* norms,
                     int32_t* status, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>(total_tiles, (int64_t)sm_count());
  FFC_CUDA(cudaFuncSetAttribute(tc5_kernel<TP, MODE, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  tc5_kernel<TP, MODE, C><<<grid, T5_THREADS, C::SMEM, st>>>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles,
                                                            norms, wait_limit(), status);
  FFC_CUDA(cudaGetLastError());
  return FFC_OK;
}

template <typename TP, int MODE>
ffc_status launch_t5_variant(int v, const CUtensorMap& tmA, const CUtensorMap& tmB, const TP* Y, const TP* X, int d,
                             int dp, ffc_kernel k, const EvalItem* items_dev, int n_items, int64_t total_tiles,
                             const float* norms, int32_t* status, cudaStream_t st) {
  switch (v) {
    case 0: return launch_t5<TP, MODE, T5V0>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles, norms, status, st);
    case 1: return launch_t5<TP, MODE, T5V1>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles, norms, status, st);
    case 2: return launch_t5<TP, MODE, T5V2>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles, norms, status, st);
    case 3: return launch_t5<TP, MODE, T5V3>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles, norms, status, st);
    default: return launch_t5<TP, MODE, T5V4>(tmA, tmB, Y, X, d, dp, k, items_dev, n_items, total_tiles, norms, status, st);
  }
}

CUtensorMapSwizzle swizzle_of(int bk) {
  return bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
}
int bk_of(int v) { return v == 1 ? 64 : (v == 0 || v == 2) ? 32 : 16; }

}  // namespace

ffc_status launch_eval_tc5(ffc_kernel k, const void* Y, int dtype, const void* X, int d, int v,
                           const EvalItem* items_dev, int n_items, int64_t total_tiles, int64_t total_rows,
                           void* scratch, double* log_scale, int32_t* status, cudaStream_t st) {
  if (log_scale) FFC_CUDA(cudaMemsetAsync(log_scale, 0, sizeof(double) * n_items, st));
  if (total_tiles <= 0 || total_rows <= 0) return FFC_OK;
  FFC_REQUIRE(v >= 0 && v < T5_VARIANTS, "tcgen05 evaluation: tile variant %d", v);
  FFC_REQUIRE(k.kind == FFC_GAUSSIAN || k.kind == FFC_POLYNOMIAL, "tcgen05 evaluation: Gaussian or polynomial");
  FFC_REQUIRE(d >= 1, "tcgen05 evaluation: d = %d", d);
  FFC_REQUIRE(scratch && (reinterpret_cast<uintptr_t>(scratch) & 255) == 0, "tcgen05 evaluation: scratch alignment");
  FFC_REQUIRE(3 * total_rows < ((int64_t)1 << 31), "tcgen05 evaluation: %lld arena rows", (long long)total_rows);
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) {
    set_error("tcgen05 evaluation: the driver's tensor-map encoder is unavailable");
    return FFC_E_CUDA;
  }
  const int dp = eval_tc5_dpad(d);
  __nv_bfloat16* planes = reinterpret_cast<__nv_bfloat16*>(scratch);
  float* norms = reinterpret_cast<float*>(reinterpret_cast<char*>(scratch) + plane_bytes(total_rows, d));
  // tensor maps over the arena [3 total_rows][d_pad] BF16: boxes of BK coordinates (2 BK bytes, swizzled
  // on that span) by 128 target rows or N source rows
  const int bk = bk_of(v), bn = t5_bn(v);
  CUtensorMap tmA, tmB;
  const cuuint64_t gdim[2] = {(cuuint64_t)dp, (cuuint64_t)(3 * total_rows)};
  const cuuint64_t gstride[1] = {(cuuint64_t)dp * 2};
  const cuuint32_t boxA[2] = {(cuuint32_t)bk, (cuuint32_t)T5_M}, boxB[2] = {(cuuint32_t)bk, (cuuint32_t)bn};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r1 = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, planes, gdim, gstride, boxA, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(bk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  const CUresult r2 = enc(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, planes, gdim, gstride, boxB, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_of(bk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) {
    set_error("tcgen05 evaluation: tensor-map encoding failed (%d, %d)", (int)r1, (int)r2);
    return FFC_E_CUDA;
  }
  const unsigned prep_blocks = (unsigned)((total_rows + 7) / 8);
#define FFC_T5_LAUNCH(TP, MODE)                                                                                    \
  do {                                                                                                             \
    tc5_prep_kernel<TP, MODE><<<prep_blocks, 256, 0, st>>>((const TP*)Y, (const TP*)X, d, dp, items_dev, n_items,    \
                                                           total_rows, planes, norms);                             \
    FFC_CUDA(cudaGetLastError());                                                                                  \
    return launch_t5_variant<TP, MODE>(v, tmA, tmB, (const TP*)Y, (const TP*)X, d, dp, k, items_dev, n_items,       \
                                       total_tiles, norms, status, st);                                            \
  } while (0)
  if (dtype == FFC_F64) {
    if (k.kind == FFC_GAUSSIAN) FFC_T5_LAUNCH(double, 0); else FFC_T5_LAUNCH(double, 2);
  } else {
    if (k.kind == FFC_GAUSSIAN) FFC_T5_LAUNCH(float, 0); else FFC_T5_LAUNCH(float, 2);
  }
#undef FFC_T5_LAUNCH
}

}  // namespace ffc
