// Tensor-core (tcgen05 / TMEM) version of the Ozaki-split Gram G = U^T V.
//
// Same arithmetic contract as ozaki.cu (exact BF16 digit products, FP64-class
// result, no FP64 instruction on the hot path), mapped onto the sm_100-family
// tensor cores:
//
//  * one CTA owns a 128 x 144 output tile (128 columns of U = MMA M, up to 144
//    columns of V = MMA N) and a slab of rows; the contraction runs in chunks
//    of 32 rows;
//  * staging: every thread loads FP64 values of the chunk, the chunk column
//    exponents E are reduced in shared memory, and each value is cut into S
//    signed 8-bit digits d_s; plane s stores d_s * 2^(-8(s-1)) (exact BF16) in
//    the K-major, no-swizzle core-matrix layout of the UMMA shared-memory
//    descriptors (8 rows x 16 bytes per core matrix), written as 16-byte stores;
//  * one elected thread issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32)
//    into three TMEM accumulators: level 2 (digit pair (1,1)), level 3 (pairs
//    (1,2), (2,1)) and all pairs of levels 4 .. S+1.  With |d| <= 128 and 32
//    rows per chunk the first two are exact; the third holds terms below 2^-16
//    of the first, so its FP32 rounding contributes < 2^-40;
//  * completion is signalled through tcgen05.commit on an mbarrier; the wait is
//    bounded (a missed completion marks the result NaN instead of hanging);
//  * flush: each thread reads its TMEM lane (one output row) with tcgen05.ld
//    and adds the three scaled sums into a double-float (two FP32) register
//    accumulator relative to per-column reference exponents;
//  * the slab partials (hi, lo, exponent) go through ozaki_slab_reduce_kernel.
#include <algorithm>

#include "kernels.cuh"
#include "ozaki_common.cuh"

namespace lob {
namespace {

constexpr int TCM = 128;        // MMA M: columns of U per tile
constexpr int TCN = 144;        // max MMA N: columns of V per tile
constexpr int TCK = 32;         // rows per chunk
constexpr int KG = TCK / 8;     // core-matrix groups along K
constexpr int kThr = 256;
constexpr int kZero = -30000;
constexpr int kNone = -100000;
constexpr int kWindow = 40;     // reference exponent = chunk max - kWindow (lazy)
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ int eff_exp0(double x) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFLL) == 0) return kZero;
  const int be = (int)((b >> 52) & 0x7FF);
  return be == 0 ? 1 : be;
}

__device__ __forceinline__ float p2f(int k) {
  return k < -126 ? 0.0f : (k > 127 ? __int_as_float(0x7F000000) : __int_as_float((k + 127) << 23));
}

// S pre-weighted digits of x relative to 2^E (biased-exponent bound eb = E + 1022),
// as BF16 bit patterns: plane s holds d_s * 2^(-8 s) (s = 0 .. S-1).
template <int S>
__device__ __forceinline__ void split_weighted(double x, int E, uint16_t out[S]) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long mant = bits & 0x000FFFFFFFFFFFFFLL;
  if (be != 0) mant |= 0x0010000000000000LL;
  const int sh = (be == 0 ? 1 : be) - 1076 + 8 * S - E;
  long long F;
  if (mant == 0 || sh <= -64) {
    F = 0;
  } else if (sh >= 0) {
    F = mant << sh;
  } else {
    F = (mant + (1LL << (-sh - 1))) >> (-sh);
  }
  if (bits < 0) F = -F;
  int d[S];
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int v = (int)((F & 0xFF) ^ 0x80) - 0x80;
    F = (F - v) >> 8;
    d[s] = v;
  }
  d[0] = (int)F;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const float f = (__int_as_float(0x4B400000 + d[s]) - 12582912.0f) * p2f(-8 * s);
    out[s] = (uint16_t)(__float_as_uint(f) >> 16);
  }
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory descriptor: K-major, no swizzle.  lbo: byte distance of
// K-adjacent core matrices, sbo: byte distance of M/N-adjacent core matrices.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for the sm_100 family
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), FP32 accumulator.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16_tc(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcShared {
  // digit planes: [S][KG][TCM/8][8 rows][8 bf16] for A, [S][KG][TCN/8][8][8] for B
  // (sized for the largest S at run time; see tc_stage_bytes)
  int eA[TCM], eB[TCN];        // chunk exponent bound E per column
  int rA[TCM], rB[TCN];        // reference exponents
  int dA[TCM], dB[TCN];        // reference change of this chunk (<= 0)
  int emA[KG][TCM], emB[KG][TCN];
  float sB[TCN];               // per-column chunk scale 2^(eB - rB)
  SegList segU, segV;
  unsigned long long mbar;
  uint32_t tmem_base;
  int rescale;
};

template <int S>
__host__ __device__ constexpr size_t planes_bytes() {
  return (size_t)S * KG * (TCM + TCN) * 8 * 2;
}

__device__ __forceinline__ const double* seg_col(const SegList& s, int c, int64_t* ld) {
  int i = 0;
  for (int t = 1; t < s.nseg; ++t) i += (c >= s.off[t]) ? 1 : 0;
  *ld = s.ld[i];
  return s.ptr[i] + (c - s.off[i]);
}

// One core-matrix row: 8 consecutive rows (k) of one column, split into S
// planes; each plane gets one 16-byte store at dst + s * plane_stride.
template <int S>
__device__ __forceinline__ void stage_core(const double* col, int64_t ld, int64_t row0,
                                           int64_t r1, int E, uint16_t* dst,
                                           size_t plane_stride) {
  uint32_t w[S][4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = row0 + i;
    const double x = (col && row < r1) ? col[row * ld] : 0.0;
    uint16_t dg[S];
    split_weighted<S>(x, E, dg);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if (i & 1)
        w[s][i >> 1] |= (uint32_t)dg[s] << 16;
      else
        w[s][i >> 1] = dg[s];
    }
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
    *reinterpret_cast<uint4*>(dst + s * plane_stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

// Phase A (exact levels 2, 3, 4), flush of level 4, phase B (levels 5..S+1 in
// the same columns), flush of everything into (hi, lo).  The planes of the
// chunk are in shared memory and fenced.  Returns true if an MMA completion
// was not observed within the bounded wait.
template <int S>
__device__ __forceinline__ bool tc_mma_and_flush(TcShared& sh, int tid, int warp, int lane,
                                                 int my_row, int col0, uint32_t aBase,
                                                 uint32_t bBase, uint32_t idesc, uint32_t acc2,
                                                 uint32_t acc3, uint32_t accl, uint32_t& phase,
                                                 float (&hi)[72], float (&lo)[72]) {
  // phase A (one thread): exact levels 2, 3 and 4
  const uint32_t lboA = (TCM / 8) * 128, lboB = (TCN / 8) * 128, sbo = 128;
  const uint32_t planeA_bytes = KG * (TCM / 8) * 128, planeB_bytes = KG * (TCN / 8) * 128;
  auto issue = [&](uint32_t acc, int si, int ti, bool first) {
#pragma unroll
    for (int ks = 0; ks < TCK / 16; ++ks) {
      // K offset ks*16 = two core-matrix groups
      const uint64_t a = smem_desc(aBase + si * planeA_bytes + ks * 2 * lboA, lboA, sbo);
      const uint64_t b = smem_desc(bBase + ti * planeB_bytes + ks * 2 * lboB, lboB, sbo);
      mma_bf16_tc(acc, a, b, idesc, (first && ks == 0) ? 0u : 1u);
    }
  };
  auto issue_level = [&](uint32_t acc, int L, bool first) {
    for (int si = max(1, L - S); si <= min(S, L - 1); ++si) {
      issue(acc, si - 1, L - si - 1, first);
      first = false;
    }
  };
  auto commit_and_wait = [&]() -> bool {
    if (tid == 0)
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              smem_u32(&sh.mbar)));
    uint32_t done = 0;
    for (int spin = 0; spin < (1 << 22) && !done; ++spin) {
      asm volatile(
          "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
          "selp.b32 %0, 1, 0, P;\n\t}\n"
          : "=r"(done)
          : "r"(smem_u32(&sh.mbar)), "r"(phase));
    }
    phase ^= 1u;
    const bool bad = __syncthreads_or(!done);
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    return bad;
  };
  const float sa = p2f(sh.eA[my_row] - sh.rA[my_row] - 14);
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  auto flush1 = [&](uint32_t acc) {
#pragma unroll
    for (int cb = 0; cb < 72; cb += 8) {
      float v[8];
      tmem_ld8(acc + lane_off + col0 + cb, v);
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
      for (int i = 0; i < 8; ++i)
        two_sum_acc(hi[cb + i], lo[cb + i], v[i] * (sa * sh.sB[col0 + cb + i]));
    }
  };
  if (sh.rescale) {
    const float fa = p2f(max(sh.dA[my_row], -127));
#pragma unroll
    for (int j = 0; j < 72; ++j) {
      const float f = fa * p2f(max(sh.dB[min(col0 + j, TCN - 1)], -127));
      hi[j] *= f;
      lo[j] *= f;
    }
  }
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    issue_level(acc2, 2, true);
    issue_level(acc3, 3, true);
    if (S >= 3) issue_level(accl, 4, true);
  }
  if (commit_and_wait()) {
    return true;
  }
  if (S >= 3) flush1(accl);
  // further phases into the same columns: for S = 7 level 5 gets its own exact
  // phase so that the inexact tail (levels >= 6, below 2^-32 of level 2)
  // rounds below 2^-53; otherwise levels 5 .. S+1 (below 2^-24) share one.
  for (int L0 = 5; L0 <= S + 1;) {
    const int L1 = (S >= 7 && L0 == 5) ? 5 : S + 1;
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      bool first = true;
      for (int L = L0; L <= L1; ++L) {
        issue_level(accl, L, first);
        first = false;
      }
    }
    if (commit_and_wait()) return true;
    flush1(accl);
    L0 = L1 + 1;
  }
  flush1(acc2);
  flush1(acc3);
  // renormalise
#pragma unroll
  for (int j = 0; j < 72; ++j) {
    const float s2 = hi[j] + lo[j];
    lo[j] = lo[j] - (s2 - hi[j]);
    hi[j] = s2;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
    return false;
}

template <int S>
__global__ void __launch_bounds__(kThr, 1)
    ozaki_gram_tc_kernel(int64_t n, SegList U, int p, SegList V, int q, int64_t rows_per_slab,
                         float4* __restrict__ partial) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* planeA = reinterpret_cast<uint16_t*>(smem_raw);
  uint16_t* planeB = planeA + (size_t)S * KG * TCM * 8 * 8 / 8;  // S*KG*(TCM/8) core mats * 64 elems
  TcShared& sh = *reinterpret_cast<TcShared*>(smem_raw + planes_bytes<S>());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tp = blockIdx.x * TCM, tq = blockIdx.y * TCN;
  const int nq = min(TCN, q - tq);             // valid V columns of this tile
  const int Nmma = (nq + 15) / 16 * 16;        // MMA N (multiple of 16)
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_slab;
  const int64_t r1 = min(n, r0 + rows_per_slab);

  if (tid == 0) {
    sh.segU = U;
    sh.segV = V;
  }
  for (int i = tid; i < TCM; i += kThr) sh.rA[i] = kNone;
  for (int i = tid; i < TCN; i += kThr) sh.rB[i] = kNone;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sh.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = sh.tmem_base;
  const uint32_t acc2 = tmem, acc3 = tmem + TCN, accl = tmem + 2 * TCN;

  // flush ownership: warp w reads TMEM lanes 32*(w%4) .. +31 (one output row
  // per thread) and columns 72*(w/4) .. +71 of the tile
  const int my_row = 32 * (warp & 3) + lane;
  const int col0 = 72 * (warp >> 2);
  float hi[72], lo[72];
#pragma unroll
  for (int j = 0; j < 72; ++j) hi[j] = lo[j] = 0.f;

  uint32_t phase = 0;
  bool failed = false;
  const uint32_t idesc = instr_desc(TCM, Nmma);
  const uint32_t aBase = smem_u32(planeA), bBase = smem_u32(planeB);

  for (int64_t r = r0; r < r1; r += TCK) {
    // ---- 1. chunk exponents: max effective exponent per column over 32 rows
    for (int it = tid; it < KG * TCM; it += kThr) {
      const int c = it % TCM, kg = it / TCM;
      int e = kZero;
      if (tp + c < p) {
        int64_t ld;
        const double* col = seg_col(sh.segU, tp + c, &ld);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t row = r + kg * 8 + i;
          if (row < r1) e = max(e, eff_exp0(col[row * ld]));
        }
      }
      sh.emA[kg][c] = e;
    }
    for (int it = tid; it < KG * TCN; it += kThr) {
      const int c = it % TCN, kg = it / TCN;
      int e = kZero;
      if (c < nq) {
        int64_t ld;
        const double* col = seg_col(sh.segV, tq + c, &ld);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int64_t row = r + kg * 8 + i;
          if (row < r1) e = max(e, eff_exp0(col[row * ld]));
        }
      }
      sh.emB[kg][c] = e;
    }
    __syncthreads();
    if (tid == 0) sh.rescale = 0;
    __syncthreads();
    for (int c = tid; c < TCM + TCN; c += kThr) {
      if (c < TCM) {
        int e = kZero;
        for (int kg = 0; kg < KG; ++kg) e = max(e, sh.emA[kg][c]);
        const int E = e - 1022;
        const int rn = max(sh.rA[c], E - kWindow);
        sh.dA[c] = (sh.rA[c] == kNone) ? 0 : sh.rA[c] - rn;
        if (sh.dA[c] != 0) sh.rescale = 1;
        sh.rA[c] = rn;
        sh.eA[c] = E;
      } else {
        const int j = c - TCM;
        int e = kZero;
        for (int kg = 0; kg < KG; ++kg) e = max(e, sh.emB[kg][j]);
        const int E = e - 1022;
        const int rn = max(sh.rB[j], E - kWindow);
        sh.dB[j] = (sh.rB[j] == kNone) ? 0 : sh.rB[j] - rn;
        if (sh.dB[j] != 0) sh.rescale = 1;
        sh.rB[j] = rn;
        sh.eB[j] = E;
        sh.sB[j] = p2f(E - rn);
      }
    }
    __syncthreads();
    // ---- 2. split into the core-matrix planes (16-byte stores)
    for (int it = tid; it < KG * TCM; it += kThr) {
      const int c = it % TCM, kg = it / TCM;
      const int E = sh.eA[c];
      int64_t ld = 0;
      const double* col = (tp + c < p) ? seg_col(sh.segU, tp + c, &ld) : nullptr;
      stage_core<S>(col, ld, r + kg * 8, r1, E,
                    planeA + ((size_t)(kg * (TCM / 8) + (c >> 3)) * 64 + (c & 7) * 8),
                    (size_t)KG * (TCM / 8) * 64);
    }
    for (int it = tid; it < KG * TCN; it += kThr) {
      const int c = it % TCN, kg = it / TCN;
      const int E = sh.eB[c];
      int64_t ld = 0;
      const double* col = (c < nq) ? seg_col(sh.segV, tq + c, &ld) : nullptr;
      stage_core<S>(col, ld, r + kg * 8, r1, E,
                    planeB + ((size_t)(kg * (TCN / 8) + (c >> 3)) * 64 + (c & 7) * 8),
                    (size_t)KG * (TCN / 8) * 64);
    }
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (tc_mma_and_flush<S>(sh, tid, warp, lane, my_row, col0, aBase, bBase, idesc, acc2, acc3,
                            accl, phase, hi, lo)) {
      failed = true;
      break;
    }
  }
  // ---- partial result (hi, lo, exponent) of this slab
  float4* out = partial + (int64_t)blockIdx.z * p * q;
  const int gi = tp + my_row;
  if (gi < p) {
#pragma unroll
    for (int j = 0; j < 72; ++j) {
      const int c = col0 + j;
      if (c < nq) {
        float4 v;
        v.x = failed ? __int_as_float(0x7FC00000) : hi[j];
        v.y = failed ? 0.f : lo[j];
        v.z = __int_as_float(sh.rA[my_row] + sh.rB[c]);
        v.w = 0.f;
        out[(int64_t)gi * q + (tq + c)] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

// ---------------------------------------------------------------- update
// Y = beta Y0 + alpha S C on tcgen05.  A (M = 128 rows of S) x K (32 columns
// of S per chunk, row exponents per chunk, columns balanced by 2^-colexp[k]);
// B = alpha C with rows balanced by 2^colexp[k], pre-split once per call into
// the exact shared-memory plane layout [chunk][ntile][S][KG][TCN/8][8][8] by
// split_c_tc_kernel, with per-(chunk, column) exponents.

template <int S>
__global__ void split_c_tc_kernel(const double* __restrict__ C, int64_t ldc, int s, int m,
                                  int ntiles, double alpha, const int* __restrict__ colexp,
                                  uint16_t* __restrict__ Cs, int* __restrict__ Ce) {
  // one warp per (chunk, padded column); lane = k within the chunk
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nchunks = (s + TCK - 1) / TCK;
  const int ncols = ntiles * TCN;
  if (w >= nchunks * ncols) return;
  const int ch = w / ncols, jj = w % ncols;
  const int tile = jj / TCN, j = jj % TCN;
  const int k = ch * TCK + lane;
  double x = 0.0;
  if (jj < m && k < s) x = ldexp(alpha * C[k + (int64_t)jj * ldc], colexp ? colexp[k] : 0);
  int e = eff_exp0(x);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  const int E = e - 1022;
  uint16_t dg[S];
  split_weighted<S>(x, E, dg);
  const size_t base = (size_t)(ch * ntiles + tile) * S * KG * (TCN / 8) * 64;
  const int kg = lane >> 3, ng = j >> 3;
#pragma unroll
  for (int sl = 0; sl < S; ++sl)
    Cs[base + (((size_t)sl * KG + kg) * (TCN / 8) + ng) * 64 + (j & 7) * 8 + (lane & 7)] = dg[sl];
  if (lane == 0) Ce[(ch * ntiles + tile) * TCN + j] = E;
}

template <int S>
__global__ void __launch_bounds__(kThr, 1)
    ozaki_update_tc_kernel(int64_t n, SegList Sg, int s, const int* __restrict__ colexp,
                           const uint16_t* __restrict__ Cs, const int* __restrict__ Ce, int m,
                           int ntiles, double beta, SegList Y0, OutList Y) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  uint16_t* planeA = reinterpret_cast<uint16_t*>(smem_raw);
  uint16_t* planeB = planeA + (size_t)S * KG * TCM * 8;
  TcShared& sh = *reinterpret_cast<TcShared*>(smem_raw + planes_bytes<S>());
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = (int)(blockIdx.x % ntiles);
  const int64_t row0 = (int64_t)(blockIdx.x / ntiles) * TCM;
  const int tn = tile * TCN;
  const int nq = min(TCN, m - tn);
  const int Nmma = (nq + 15) / 16 * 16;
  const int nchunks = (s + TCK - 1) / TCK;

  if (tid == 0) sh.segU = Sg;
  for (int i = tid; i < TCM; i += kThr) sh.rA[i] = kNone;
  for (int i = tid; i < TCN; i += kThr) sh.rB[i] = kNone;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&sh.tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sh.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = sh.tmem_base;
  const uint32_t acc2 = tmem, acc3 = tmem + TCN, accl = tmem + 2 * TCN;
  const int my_row = 32 * (warp & 3) + lane;
  const int col0 = 72 * (warp >> 2);
  float hi[72], lo[72];
#pragma unroll
  for (int j = 0; j < 72; ++j) hi[j] = lo[j] = 0.f;
  uint32_t phase = 0;
  bool failed = false;
  const uint32_t idesc = instr_desc(TCM, Nmma);
  const uint32_t aBase = smem_u32(planeA), bBase = smem_u32(planeB);

  for (int ch = 0; ch < nchunks; ++ch) {
    const int k0 = ch * TCK;
    // ---- row exponents of the balanced S chunk (items: row x 8 consecutive k)
    for (int it = tid; it < KG * TCM; it += kThr) {
      const int rl = it % TCM, kg = it / TCM;
      const int64_t row = row0 + rl;
      int e = kZero;
      if (row < n) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = k0 + kg * 8 + i;
          if (k < s) {
            int64_t ld;
            const double* col = seg_col(sh.segU, k, &ld);
            const double x = col[row * ld];
            const int ee = eff_exp0(x);
            if (ee != kZero) e = max(e, ee - (colexp ? colexp[k] : 0));
          }
        }
      }
      sh.emA[kg][rl] = e;
    }
    // ---- B planes and exponents of this chunk / column tile (pre-split)
    {
      const uint4* src = reinterpret_cast<const uint4*>(
          Cs + (size_t)(ch * ntiles + tile) * S * KG * (TCN / 8) * 64);
      uint4* dst = reinterpret_cast<uint4*>(planeB);
      const int nvec = S * KG * (TCN / 8) * 64 / 8;
      for (int v = tid; v < nvec; v += kThr) dst[v] = src[v];
      for (int j = tid; j < TCN; j += kThr) sh.eB[j] = Ce[(ch * ntiles + tile) * TCN + j];
    }
    __syncthreads();
    if (tid == 0) sh.rescale = 0;
    __syncthreads();
    for (int c = tid; c < TCM + TCN; c += kThr) {
      if (c < TCM) {
        int e = kZero;
        for (int kg = 0; kg < KG; ++kg) e = max(e, sh.emA[kg][c]);
        const int E = e - 1022;
        const int rn = max(sh.rA[c], E - kWindow);
        sh.dA[c] = (sh.rA[c] == kNone) ? 0 : sh.rA[c] - rn;
        if (sh.dA[c] != 0) sh.rescale = 1;
        sh.rA[c] = rn;
        sh.eA[c] = E;
      } else {
        const int j = c - TCM;
        const int E = sh.eB[j];
        const int rn = max(sh.rB[j], E - kWindow);
        sh.dB[j] = (sh.rB[j] == kNone) ? 0 : sh.rB[j] - rn;
        if (sh.dB[j] != 0) sh.rescale = 1;
        sh.rB[j] = rn;
        sh.sB[j] = p2f(E - rn);
      }
    }
    __syncthreads();
    // ---- split the S chunk into the A planes
    for (int it = tid; it < KG * TCM; it += kThr) {
      const int rl = it % TCM, kg = it / TCM;
      const int64_t row = row0 + rl;
      const int E = sh.eA[rl];
      uint32_t w[S][4];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + kg * 8 + i;
        double x = 0.0;
        int cs = 0;
        if (row < n && k < s) {
          int64_t ld;
          const double* col = seg_col(sh.segU, k, &ld);
          x = col[row * ld];
          cs = colexp ? colexp[k] : 0;
        }
        uint16_t dg[S];
        split_weighted<S>(x, E + cs, dg);
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
          if (i & 1)
            w[sl][i >> 1] |= (uint32_t)dg[sl] << 16;
          else
            w[sl][i >> 1] = dg[sl];
        }
      }
      uint16_t* dst = planeA + ((size_t)(kg * (TCM / 8) + (rl >> 3)) * 64 + (rl & 7) * 8);
#pragma unroll
      for (int sl = 0; sl < S; ++sl)
        *reinterpret_cast<uint4*>(dst + (size_t)sl * KG * (TCM / 8) * 64) =
            make_uint4(w[sl][0], w[sl][1], w[sl][2], w[sl][3]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (tc_mma_and_flush<S>(sh, tid, warp, lane, my_row, col0, aBase, bBase, idesc, acc2, acc3,
                            accl, phase, hi, lo)) {
      failed = true;
      break;
    }
  }
  // ---- output rows: Y = (hi + lo) 2^(rA + rB) + beta Y0
  const int64_t row = row0 + my_row;
  if (row < n) {
#pragma unroll
    for (int j = 0; j < 72; ++j) {
      const int c = tn + col0 + j;
      if (col0 + j < nq) {
        const double y0 = beta != 0.0 ? seg_load(Y0, c, row) : 0.0;
        *out_addr(Y, c, row) =
            failed ? __longlong_as_double(0x7FF8000000000000LL)
                   : assemble_df(hi[j], lo[j], sh.rA[my_row] + sh.rB[col0 + j], y0);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

template <int S>
size_t tc_smem_bytes() {
  return planes_bytes<S>() + sizeof(TcShared) + 64;
}

void tc_plan(int64_t n, int p, int q, int* slabs, int64_t* rows_per_slab) {
  const int64_t tiles = ceil_div(p, TCM) * ceil_div(q, TCN);
  int64_t s = std::max<int64_t>(1, ceil_div(152, tiles));
  s = std::min<int64_t>(s, std::max<int64_t>(1, ceil_div(n, 8 * TCK)));
  int64_t r = round_up(ceil_div(std::max<int64_t>(n, 1), s), TCK);
  s = std::max<int64_t>(1, ceil_div(std::max<int64_t>(n, 1), r));
  *slabs = (int)s;
  *rows_per_slab = r;
}

template <int S>
int tc_launch(cudaStream_t st, int64_t n, const SegList& U, int p, const SegList& V, int q,
              int slabs, int64_t rps, float4* partial) {
  const size_t sh = tc_smem_bytes<S>();
  static bool configured = false;
  if (!configured) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_gram_tc_kernel<S>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    configured = true;
  }
  dim3 grid((unsigned)ceil_div(p, TCM), (unsigned)ceil_div(q, TCN), (unsigned)slabs);
  ozaki_gram_tc_kernel<S><<<grid, kThr, sh, st>>>(n, U, p, V, q, rps, partial);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace

int64_t gram_tc_workspace(int64_t n, int p, int q) {
  int slabs;
  int64_t r;
  tc_plan(n, p, q, &slabs, &r);
  return (int64_t)slabs * p * q * (int64_t)sizeof(float4);
}

int gram_tc(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
            int64_t ldg, int slices, void* work, int64_t work_bytes) {
  const int p = U.off[U.nseg], q = V.off[V.nseg];
  if (p <= 0 || q <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  if (n <= 0) return gram_ozaki(st, n, U, V, G, ldg, slices, work, work_bytes);
  int slabs;
  int64_t rps;
  tc_plan(n, p, q, &slabs, &rps);
  if (work_bytes < (int64_t)slabs * p * q * (int64_t)sizeof(float4)) return LOBPCG_ERR_ARG;
  float4* partial = (float4*)work;
  int rc;
  switch (slices) {
    case 3: rc = tc_launch<3>(st, n, U, p, V, q, slabs, rps, partial); break;
    case 4: rc = tc_launch<4>(st, n, U, p, V, q, slabs, rps, partial); break;
    case 5: rc = tc_launch<5>(st, n, U, p, V, q, slabs, rps, partial); break;
    case 6: rc = tc_launch<6>(st, n, U, p, V, q, slabs, rps, partial); break;
    case 7: rc = tc_launch<7>(st, n, U, p, V, q, slabs, rps, partial); break;
    default: return LOBPCG_ERR_ARG;
  }
  if (rc) return rc;
  return ozaki_slab_reduce(st, partial, slabs, p, q, G, ldg);
}

}  // namespace lob

namespace lob {

namespace {

template <int S>
int update_tc_launch(cudaStream_t st, int64_t n, const SegList& Sg, int s, const double* C,
                     int64_t ldc, int m, double alpha, double beta, const SegList& Y0,
                     const OutList& Y, const int* colexp, void* work) {
  const int ntiles = (int)ceil_div(m, TCN);
  const int nchunks = (int)ceil_div(s, TCK);
  uint16_t* Cs = (uint16_t*)work;
  const size_t cs_elems = (size_t)nchunks * ntiles * S * KG * (TCN / 8) * 64;
  int* Ce = (int*)(Cs + cs_elems);
  int* cx = Ce + (size_t)nchunks * ntiles * TCN;
  if (!colexp) {
    int rc = column_exponents(st, n, Sg, s, cx);
    if (rc) return rc;
    colexp = cx;
  }
  {
    const int64_t warps = (int64_t)nchunks * ntiles * TCN;
    split_c_tc_kernel<S><<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(
        C, ldc, s, m, ntiles, alpha, colexp, Cs, Ce);
    LOB_LAUNCHED();
  }
  const size_t sh = tc_smem_bytes<S>();
  static bool configured = false;
  if (!configured) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_update_tc_kernel<S>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    configured = true;
  }
  const int64_t blocks = ceil_div(n, TCM) * ntiles;
  ozaki_update_tc_kernel<S><<<(unsigned)blocks, kThr, sh, st>>>(n, Sg, s, colexp, Cs, Ce, m,
                                                                ntiles, beta, Y0, Y);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace

int64_t update_tc_workspace(int64_t, int s, int m, int slices) {
  if (slices == 0) slices = 6;
  const int64_t ntiles = ceil_div(std::max(m, 1), TCN);
  const int64_t nchunks = ceil_div(std::max(s, 1), TCK);
  return nchunks * ntiles * slices * KG * (TCN / 8) * 64 * 2 + nchunks * ntiles * TCN * 4 +
         (int64_t)std::max(s, 1) * 4 + 256;
}

int update_tc(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc, int m,
              double alpha, double beta, const SegList& Y0, const OutList& Y, int slices,
              void* work, int64_t work_bytes, const int* colexp) {
  const int s = S.off[S.nseg];
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  if (s == 0) return update_f64(st, n, S, C, ldc, m, alpha, beta, Y0, Y);
  if (work_bytes < update_tc_workspace(n, s, m, slices)) return LOBPCG_ERR_ARG;
  if (beta != 0.0 && beta != 1.0) return LOBPCG_ERR_ARG;
  switch (slices) {
    case 3: return update_tc_launch<3>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 4: return update_tc_launch<4>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 5: return update_tc_launch<5>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 6: return update_tc_launch<6>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 7: return update_tc_launch<7>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    default: return LOBPCG_ERR_ARG;
  }
}

}  // namespace lob
