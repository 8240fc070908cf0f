// FP64-accurate dense contractions on the BF16 tensor cores (Ozaki-style exact
// splitting: Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication", 2012).
//
// Why: on GB300 the FP64 units run at 1/64 of the FP32 rate, so the Gram
// S^T Y and the basis update S C of every LOBPCG iteration cannot use FP64
// arithmetic at all without being compute bound by two orders of magnitude.
// These kernels therefore contain NO FP64 arithmetic on the hot path:
//
//  * split: every FP64 input x of a chunk (64 contraction indices) is written
//    as a fixed-point number relative to 2^E, E the exponent bound of its
//    chunk row/column, and cut into S signed 8-bit digits:
//        x = 2^E * sum_{s=1..S} d_s 2^(1-8s),   |d_s| <= 128,
//    using integer operations on the IEEE bit pattern only.  Each digit is
//    exact in BF16.
//  * multiply: digit products of level L = s + t (pairs with L <= S + 1) are
//    accumulated by mma.sync m16n8k16 BF16 -> FP32.  Every product is an
//    integer of magnitude <= 2^14 and a level holds at most S pairs over a
//    64-long chunk, so the FP32 sums stay below 2^24 and are EXACT.
//  * flush: after each chunk, each level's exact sum is scaled by its power
//    of two (exact) and added into a double-float accumulator (hi, lo FP32
//    with an error-free two-sum), relative to a running per-row/per-column
//    reference exponent so that FP32's range is never exceeded.
//  * output: the double result is assembled from (hi, lo, exponent) with
//    int64 arithmetic.
// Accuracy (S = 6): each output's error is below ~2^-44 * n * max|u_i| max|v_j|
// per chunk-relative scale, i.e. about 1e-13 normwise: FP64-class for the
// Rayleigh-Ritz and the convergence test of Eq. (9).
#include <algorithm>

#include "kernels.cuh"
#include "ozaki_common.cuh"

namespace lob {
namespace {

constexpr int TM = 64;       // output rows per CTA (M: columns of U / rows of S)
constexpr int TN = 64;       // output columns per CTA (N: columns of V / of C)
constexpr int KC = 64;       // contraction chunk
constexpr int LDK = KC + 8;  // bf16 per staged row (padding: conflict-free fragment loads)
constexpr int LDW = LDK / 2; // 32-bit words per staged row
constexpr int kThreads = 256;
constexpr int kNoExp = -100000;

// ---- integer-only FP64 helpers ------------------------------------------

constexpr int kZeroBe = -30000;  // "biased exponent" of an exact zero (ignored by max)

// Biased exponent of x * 2^-cshift (as an unbounded int); kZeroBe for x == 0.
__device__ __forceinline__ int eff_exp(double x, int cshift) {
  const long long b = __double_as_longlong(x);
  if ((b & 0x7FFFFFFFFFFFFFFFLL) == 0) return kZeroBe;
  const int be = (int)((b >> 52) & 0x7FF);
  return (be == 0 ? 1 : be) - cshift;
}

// E such that |x * 2^-cshift| < 2^E for every x of effective exponent <= be.
__device__ __forceinline__ int exp_bound(int be) { return be - 1022; }

// x * 2^-cshift = 2^E sum_{s=1..S} d_s 2^(1-8s); digits written as BF16 bit
// patterns (dig[0] is the most significant).  Integer operations only.
template <int S>
__device__ __forceinline__ void split_digits(double x, int E, int cshift, uint32_t dig[S]) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  long long mant = bits & 0x000FFFFFFFFFFFFFLL;
  if (be != 0) mant |= 0x0010000000000000LL;
  // |x| 2^-cshift 2^(8S-1-E) = mant * 2^sh
  const int sh = (be == 0 ? 1 : be) - cshift - 1076 + 8 * S - E;
  long long F;
  if (mant == 0 || sh <= -64) {
    F = 0;
  } else if (sh >= 0) {
    F = mant << sh;  // only possible for S = 7 (sh <= 2)
  } else {
    const int r = -sh;
    F = (mant + (1LL << (r - 1))) >> r;
  }
  if (bits < 0) F = -F;
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int d = (int)(((F & 0xFF) ^ 0x80)) - 0x80;  // signed low digit in [-128, 127]
    F = (F - d) >> 8;
    // exact int -> float via the 1.5*2^23 bias; the top 16 bits are the BF16
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    dig[s] = __float_as_uint(f) >> 16;
  }
  const float f0 = __int_as_float(0x4B400000 + (int)F) - 12582912.0f;
  dig[0] = __float_as_uint(f0) >> 16;
}

__device__ __forceinline__ float pow2f(int k) {
  return k < -126 ? 0.0f : __int_as_float((k + 127) << 23);
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

// ---- the shared MMA / flush core ------------------------------------------

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Acc {
  float hi[2][2][4];
  float lo[2][2][4];
};

// Shared-memory staging of one chunk: S digit planes of A ([TM][LDK] bf16) and
// of B ([TN][LDK] bf16), plus the chunk exponents and running references.
template <int S>
struct Stage {
  uint32_t A[S][TM * LDW];
  uint32_t B[S][TN * LDW];
  int eA[TM], eB[TN];
  int rA[TM], rB[TN];
  int oA[TM], oB[TN];
  int red[4][TM];
};

// Warp layout: 8 warps = 2 (M) x 4 (N); warp tile 32 x 16 = 2 m16 x 2 n8.
template <int S>
__device__ __forceinline__ void mma_levels_and_flush(Stage<S>& sm, Acc& acc, int warp, int lane) {
  const int wm = warp & 1, wn = warp >> 1;
  const int g = lane >> 2, t = lane & 3;
  // rescale the running sums where a reference exponent moved up
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = wm * 32 + mt * 16 + g + ((e & 2) ? 8 : 0);
        const int j = wn * 16 + nt * 8 + 2 * t + (e & 1);
        const int d = (sm.oA[i] - sm.rA[i]) + (sm.oB[j] - sm.rB[j]);
        if (d != 0) {
          const float f = pow2f(max(d, -127));
          acc.hi[mt][nt][e] *= f;
          acc.lo[mt][nt][e] *= f;
        }
      }
#pragma unroll 1
  for (int L = 2; L <= S + 1; ++L) {
    float c[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[mt][nt][e] = 0.f;
    const int s_lo = max(1, L - S), s_hi = min(S, L - 1);
#pragma unroll 1
    for (int s = s_lo; s <= s_hi; ++s) {
      const uint32_t* As = sm.A[s - 1];
      const uint32_t* Bs = sm.B[L - s - 1];
#pragma unroll
      for (int ks = 0; ks < KC / 16; ++ks) {
        uint32_t a[2][4], b[2][2];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int r = wm * 32 + mt * 16 + g;
          const int kw = ks * 8 + t;  // word index of k = ks*16 + 2t
          a[mt][0] = As[r * LDW + kw];
          a[mt][1] = As[(r + 8) * LDW + kw];
          a[mt][2] = As[r * LDW + kw + 4];
          a[mt][3] = As[(r + 8) * LDW + kw + 4];
        }
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int cidx = wn * 16 + nt * 8 + g;
          const int kw = ks * 8 + t;
          b[nt][0] = Bs[cidx * LDW + kw];
          b[nt][1] = Bs[cidx * LDW + kw + 4];
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) mma_bf16(c[mt][nt], a[mt], b[nt]);
      }
    }
    // exact level sum -> double-float accumulator
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = wm * 32 + mt * 16 + g + ((e & 2) ? 8 : 0);
          const int j = wn * 16 + nt * 8 + 2 * t + (e & 1);
          const int k = (sm.eA[i] - sm.rA[i]) + (sm.eB[j] - sm.rB[j]) + 2 - 8 * L;
          two_sum_add(acc.hi[mt][nt][e], acc.lo[mt][nt][e], c[mt][nt][e] * pow2f(k));
        }
  }
  // renormalise (hi, lo)
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float s = acc.hi[mt][nt][e] + acc.lo[mt][nt][e];
        acc.lo[mt][nt][e] = acc.lo[mt][nt][e] - (s - acc.hi[mt][nt][e]);
        acc.hi[mt][nt][e] = s;
      }
}

// Update the running references after eA/eB of a chunk are known.
template <int S>
__device__ __forceinline__ void update_refs(Stage<S>& sm, int tid) {
  if (tid < TM) {
    sm.oA[tid] = sm.rA[tid];
    sm.rA[tid] = max(sm.rA[tid], sm.eA[tid]);
  } else if (tid < TM + TN) {
    const int j = tid - TM;
    sm.oB[j] = sm.rB[j];
    sm.rB[j] = max(sm.rB[j], sm.eB[j]);
  }
}

// ---- Gram: G = U^T V ------------------------------------------------------
// A(m, k) = U(k, m), B(n, k) = V(k, n); k runs over the rows of a slab.
// Thread layout for staging: column c = tid % 64, row-pair group rg = tid / 64;
// it owns rows 2*(rg + 4i) + {0, 1}, i = 0..7, of the chunk.

template <int S>
__device__ __forceinline__ void stage_cols(const SegList& X, int ncols, int c0, int64_t r,
                                           int64_t r1, uint32_t (*planes)[TM * LDW], int* eout,
                                           int (*red)[TM], int tid) {
  const int c = tid & 63, rg = tid >> 6;
  const bool colok = c0 + c < ncols;
  double v[16];
  int be = kZeroBe;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int64_t row = r + 2 * (rg + 4 * i) + b;
      const double x = (colok && row < r1) ? seg_load(X, c0 + c, row) : 0.0;
      v[2 * i + b] = x;
      be = max(be, eff_exp(x, 0));
    }
  red[rg][c] = be;
  __syncthreads();
  if (rg == 0) eout[c] = exp_bound(max(max(red[0][c], red[1][c]), max(red[2][c], red[3][c])));
  __syncthreads();
  const int E = eout[c];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    uint32_t d0[S], d1[S];
    split_digits<S>(v[2 * i], E, 0, d0);
    split_digits<S>(v[2 * i + 1], E, 0, d1);
    const int kw = rg + 4 * i;  // word index of the row pair
#pragma unroll
    for (int s = 0; s < S; ++s) planes[s][c * LDW + kw] = d0[s] | (d1[s] << 16);
  }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gram_kernel(int64_t n, SegList U, int p, SegList V, int q, int64_t rows_per_slab,
                      float4* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage<S>& sm = *reinterpret_cast<Stage<S>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tp = blockIdx.x * TM, tq = blockIdx.y * TN;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per_slab;
  const int64_t r1 = min(n, r0 + rows_per_slab);
  Acc acc;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc.hi[mt][nt][e] = acc.lo[mt][nt][e] = 0.f;
  if (tid < TM) sm.rA[tid] = kNoExp;
  if (tid < TN) sm.rB[tid] = kNoExp;
  for (int64_t r = r0; r < r1; r += KC) {
    stage_cols<S>(U, p, tp, r, r1, sm.A, sm.eA, sm.red, tid);
    stage_cols<S>(V, q, tq, r, r1, sm.B, sm.eB, sm.red, tid);
    update_refs<S>(sm, tid);
    __syncthreads();
    mma_levels_and_flush<S>(sm, acc, warp, lane);
    __syncthreads();
  }
  // partial result of this slab: (hi, lo, exponent) per output
  const int wm = warp & 1, wn = warp >> 1, g = lane >> 2, t = lane & 3;
  float4* out = partial + (int64_t)blockIdx.z * p * q;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = wm * 32 + mt * 16 + g + ((e & 2) ? 8 : 0);
        const int j = wn * 16 + nt * 8 + 2 * t + (e & 1);
        if (tp + i < p && tq + j < q) {
          float4 v;
          v.x = acc.hi[mt][nt][e];
          v.y = acc.lo[mt][nt][e];
          v.z = __int_as_float(sm.rA[i] + sm.rB[j]);
          v.w = 0.f;
          out[(int64_t)(tp + i) * q + (tq + j)] = v;
        }
      }
}

// Sum the slab partials in a fixed order (double-float, common exponent).
__global__ void ozaki_slab_reduce_kernel(const float4* __restrict__ partial, int slabs, int p,
                                         int q, double* __restrict__ G, int64_t ldg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * q) return;
  int R = -2000000;
  for (int z = 0; z < slabs; ++z) {
    const float4 v = partial[(int64_t)z * p * q + e];
    if (v.x != 0.f || v.y != 0.f) R = max(R, __float_as_int(v.z));
  }
  float hi = 0.f, lo = 0.f;
  if (R > -2000000)
    for (int z = 0; z < slabs; ++z) {
      const float4 v = partial[(int64_t)z * p * q + e];
      if (v.x == 0.f && v.y == 0.f) continue;
      const float f = pow2f(max(__float_as_int(v.z) - R, -127));
      two_sum_add(hi, lo, v.x * f);
      two_sum_add(hi, lo, v.y * f);
    }
  const int i = (int)(e / q), j = (int)(e % q);
  G[i + (int64_t)j * ldg] = (R > -2000000) ? assemble_df(hi, lo, R, 0.0) : 0.0;
}

// ---- update: Y = beta Y0 + alpha S C ---------------------------------------
// A(m, k) = S(row m, col k) with a per-row exponent per chunk; B(n, k) =
// alpha C(k, n) pre-split per chunk into global memory by split_c_kernel.

template <int S>
__global__ void split_c_kernel(const double* __restrict__ C, int64_t ldc, int s, int m,
                               int mpad, double alpha, const int* __restrict__ colexp,
                               uint32_t* __restrict__ Cs, int* __restrict__ Ce) {
  // one warp per (chunk, column); lanes cover the 64 k of the chunk in pairs.
  // Row k of C is scaled by 2^colexp[k] (the inverse of S's column scaling).
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nchunks = (s + KC - 1) / KC;
  if (w >= nchunks * mpad) return;
  const int ch = w / mpad, j = w % mpad;
  const int k0 = ch * KC + 2 * lane;
  double x0 = 0.0, x1 = 0.0;
  if (j < m) {
    if (k0 < s) x0 = ldexp(alpha * C[k0 + (int64_t)j * ldc], colexp ? colexp[k0] : 0);
    if (k0 + 1 < s) x1 = ldexp(alpha * C[k0 + 1 + (int64_t)j * ldc], colexp ? colexp[k0 + 1] : 0);
  }
  int be = max(eff_exp(x0, 0), eff_exp(x1, 0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) be = max(be, __shfl_xor_sync(0xffffffffu, be, o));
  const int E = exp_bound(be);
  uint32_t d0[S], d1[S];
  split_digits<S>(x0, E, 0, d0);
  split_digits<S>(x1, E, 0, d1);
  uint32_t* base = Cs + (int64_t)ch * S * mpad * LDW;
#pragma unroll
  for (int sl = 0; sl < S; ++sl) base[((int64_t)sl * mpad + j) * LDW + lane] = d0[sl] | (d1[sl] << 16);
  if (lane < LDW - 32) {
#pragma unroll
    for (int sl = 0; sl < S; ++sl) base[((int64_t)sl * mpad + j) * LDW + 32 + lane] = 0u;
  }
  if (lane == 0) Ce[ch * mpad + j] = E;
}

// Column exponents of an n x s block: colexp[k] = E with max_i |S(i,k)| < 2^E
// (0 for an all-zero column).  Used when the caller gives no column scaling.
__global__ void colexp_kernel(int64_t n, SegList Sg, int s, int* __restrict__ colexp) {
  __shared__ int red[256];
  const int k = blockIdx.x;
  int be = kZeroBe;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) be = max(be, eff_exp(seg_load(Sg, k, r), 0));
  red[threadIdx.x] = be;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) colexp[k] = red[0] == kZeroBe ? 0 : exp_bound(red[0]);
}

// Rows: thread owns row m = tid / 4 and the 16 contraction indices 16*(tid % 4) + 0..15.
// Column k of S is scaled by 2^-colexp[k] (exactly, in the exponent).
template <int S>
__device__ __forceinline__ void stage_rows(const SegList& Sg, int s, int k0, int64_t row0,
                                           int64_t n, const int* colexp, Stage<S>& sm, int tid) {
  const int rloc = tid >> 2, kg = tid & 3;
  const int64_t row = row0 + rloc;
  double v[16];
  int cs[16];
  int be = kZeroBe;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k = k0 + 16 * kg + i;
    const bool ok = row < n && k < s;
    const double x = ok ? seg_load(Sg, k, row) : 0.0;
    cs[i] = (ok && colexp) ? colexp[k] : 0;
    v[i] = x;
    be = max(be, eff_exp(x, cs[i]));
  }
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 1));
  be = max(be, __shfl_xor_sync(0xffffffffu, be, 2));
  const int E = exp_bound(be);
  if (kg == 0) sm.eA[rloc] = E;
#pragma unroll
  for (int i = 0; i < 16; i += 2) {
    uint32_t d0[S], d1[S];
    split_digits<S>(v[i], E, cs[i], d0);
    split_digits<S>(v[i + 1], E, cs[i + 1], d1);
    const int kw = 8 * kg + i / 2;
#pragma unroll
    for (int sl = 0; sl < S; ++sl) sm.A[sl][rloc * LDW + kw] = d0[sl] | (d1[sl] << 16);
  }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_update_kernel(int64_t n, SegList Sg, int s, const int* __restrict__ colexp,
                        const uint32_t* __restrict__ Cs, const int* __restrict__ Ce, int m,
                        int mpad, double beta, SegList Y0, OutList Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Stage<S>& sm = *reinterpret_cast<Stage<S>*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // column tiles vary fastest so the CTAs sharing a row tile of S run together
  const int ncol = mpad / TN;
  const int tn = (int)(blockIdx.x % ncol) * TN;
  const int64_t row0 = (int64_t)(blockIdx.x / ncol) * TM;
  Acc acc;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc.hi[mt][nt][e] = acc.lo[mt][nt][e] = 0.f;
  if (tid < TM) sm.rA[tid] = kNoExp;
  if (tid < TN) sm.rB[tid] = kNoExp;
  const int nchunks = (s + KC - 1) / KC;
  for (int ch = 0; ch < nchunks; ++ch) {
    stage_rows<S>(Sg, s, ch * KC, row0, n, colexp, sm, tid);
    // B planes of this chunk and column tile: S * TN rows of LDW words
    const uint4* src = reinterpret_cast<const uint4*>(Cs + (int64_t)ch * S * mpad * LDW);
    for (int idx = tid; idx < S * TN * (LDW / 4); idx += kThreads) {
      const int sl = idx / (TN * (LDW / 4));
      const int rem = idx % (TN * (LDW / 4));
      const int jj = rem / (LDW / 4), w4 = rem % (LDW / 4);
      const uint4 val = src[((int64_t)sl * mpad + tn + jj) * (LDW / 4) + w4];
      reinterpret_cast<uint4*>(sm.B[sl])[jj * (LDW / 4) + w4] = val;
    }
    if (tid < TN) sm.eB[tid] = Ce[ch * mpad + tn + tid];
    __syncthreads();
    update_refs<S>(sm, tid);
    __syncthreads();
    mma_levels_and_flush<S>(sm, acc, warp, lane);
    __syncthreads();
  }
  const int wm = warp & 1, wn = warp >> 1, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = wm * 32 + mt * 16 + g + ((e & 2) ? 8 : 0);
        const int j = wn * 16 + nt * 8 + 2 * t + (e & 1);
        const int64_t row = row0 + i;
        const int c = tn + j;
        if (row < n && c < m) {
          const double y0 = beta != 0.0 ? seg_load(Y0, c, row) : 0.0;
          *out_addr(Y, c, row) =
              assemble_df(acc.hi[mt][nt][e], acc.lo[mt][nt][e], sm.rA[i] + sm.rB[j], y0);
        }
      }
}

// ---- planning ---------------------------------------------------------------

void gram_plan(int64_t n, int p, int q, int* slabs, int64_t* rows_per_slab) {
  const int64_t tiles = ceil_div(p, TM) * ceil_div(q, TN);
  int64_t s = std::max<int64_t>(1, ceil_div(2 * 152, tiles));
  s = std::min<int64_t>(s, std::max<int64_t>(1, ceil_div(n, 4 * KC)));
  int64_t r = round_up(ceil_div(std::max<int64_t>(n, 1), s), KC);
  s = std::max<int64_t>(1, ceil_div(std::max<int64_t>(n, 1), r));
  *slabs = (int)s;
  *rows_per_slab = r;
}

template <int S>
size_t stage_bytes() {
  return sizeof(Stage<S>);
}

template <int S>
int gram_launch(cudaStream_t st, int64_t n, const SegList& U, int p, const SegList& V, int q,
                int slabs, int64_t rps, float4* partial) {
  const size_t sh = stage_bytes<S>();
  static bool configured[64] = {false};  // the attribute is per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_gram_kernel<S>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  dim3 grid((unsigned)ceil_div(p, TM), (unsigned)ceil_div(q, TN), (unsigned)slabs);
  ozaki_gram_kernel<S><<<grid, kThreads, sh, st>>>(n, U, p, V, q, rps, partial);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

template <int S>
int update_launch(cudaStream_t st, int64_t n, const SegList& Sg, int s, const double* C,
                  int64_t ldc, int m, double alpha, double beta, const SegList& Y0,
                  const OutList& Y, const int* colexp, void* work) {
  const int mpad = (int)round_up(m, TN);
  const int nchunks = (int)ceil_div(s, KC);
  uint32_t* Cs = (uint32_t*)work;
  int* Ce = (int*)(Cs + (size_t)nchunks * S * mpad * LDW);
  int* cx = Ce + (size_t)nchunks * mpad;
  if (!colexp) {
    colexp_kernel<<<s, 256, 0, st>>>(n, Sg, s, cx);
    LOB_LAUNCHED();
    colexp = cx;
  }
  {
    const int64_t warps = (int64_t)nchunks * mpad;
    split_c_kernel<S><<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(C, ldc, s, m, mpad,
                                                                          alpha, colexp, Cs, Ce);
    LOB_LAUNCHED();
  }
  const size_t sh = stage_bytes<S>();
  static bool configured[64] = {false};  // the attribute is per device
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_update_kernel<S>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const int64_t blocks = (int64_t)(mpad / TN) * ceil_div(n, TM);
  ozaki_update_kernel<S><<<(unsigned)blocks, kThreads, sh, st>>>(n, Sg, s, colexp, Cs, Ce, m,
                                                                 mpad, beta, Y0, Y);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace

int column_exponents(cudaStream_t st, int64_t n, const SegList& Sg, int s, int* out) {
  if (s <= 0) return LOBPCG_OK;
  colexp_kernel<<<s, 256, 0, st>>>(n, Sg, s, out);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int ozaki_slab_reduce(cudaStream_t st, const float4* partial, int slabs, int p, int q, double* G,
                      int64_t ldg) {
  const int64_t tot = (int64_t)p * q;
  ozaki_slab_reduce_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(partial, slabs, p, q, G,
                                                                         ldg);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int64_t gram_ozaki_workspace(int64_t n, int p, int q, int) {
  int slabs;
  int64_t r;
  gram_plan(n, p, q, &slabs, &r);
  return (int64_t)slabs * p * q * (int64_t)sizeof(float4);
}

int gram_ozaki(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
               int64_t ldg, int slices, void* work, int64_t work_bytes) {
  const int p = U.off[U.nseg], q = V.off[V.nseg];
  if (p <= 0 || q <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  int slabs;
  int64_t rps;
  gram_plan(n, p, q, &slabs, &rps);
  if (work_bytes < (int64_t)slabs * p * q * (int64_t)sizeof(float4)) return LOBPCG_ERR_ARG;
  float4* partial = (float4*)work;
  int rc;
  if (n <= 0) {
    LOB_CUDA_OK(cudaMemsetAsync(partial, 0, (size_t)p * q * sizeof(float4), st));
    slabs = 1;
    rc = LOBPCG_OK;
  } else {
    switch (slices) {
      case 3: rc = gram_launch<3>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 4: rc = gram_launch<4>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 5: rc = gram_launch<5>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 6: rc = gram_launch<6>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 7: rc = gram_launch<7>(st, n, U, p, V, q, slabs, rps, partial); break;
      default: return LOBPCG_ERR_ARG;
    }
  }
  if (rc) return rc;
  const int64_t tot = (int64_t)p * q;
  ozaki_slab_reduce_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(partial, slabs, p, q, G,
                                                                         ldg);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int64_t update_ozaki_workspace(int64_t, int s, int m, int slices) {
  if (slices == 0) slices = 6;
  const int64_t mpad = round_up(std::max(m, 1), TN);
  const int64_t nchunks = ceil_div(std::max(s, 1), KC);
  return nchunks * slices * mpad * LDW * 4 + nchunks * mpad * 4 + nchunks * KC * 4 + 256;
}

int update_ozaki(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc,
                 int m, double alpha, double beta, const SegList& Y0, const OutList& Y,
                 int slices, void* work, int64_t work_bytes, const int* colexp) {
  const int s = S.off[S.nseg];
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  if (s == 0) {
    // Y = beta Y0: reuse the FP64 kernel path (no contraction)
    return update_f64(st, n, S, C, ldc, m, alpha, beta, Y0, Y);
  }
  if (work_bytes < update_ozaki_workspace(n, s, m, slices)) return LOBPCG_ERR_ARG;
  if (beta != 0.0 && beta != 1.0) return LOBPCG_ERR_ARG;
  switch (slices) {
    case 3: return update_launch<3>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 4: return update_launch<4>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 5: return update_launch<5>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 6: return update_launch<6>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    case 7: return update_launch<7>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work);
    default: return LOBPCG_ERR_ARG;
  }
}

}  // namespace lob

namespace lob {

// Same Ozaki Gram as gram_ozaki, but with the slab count lowered until the
// slab partials fit in work_bytes (used by the allocation-free entry point,
// whose scratch has a fixed size).  Returns LOBPCG_ERR_ARG when even one slab
// (p * q partials of 16 bytes) does not fit.
int gram_ozaki_bounded(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
                       int64_t ldg, int slices, void* work, int64_t work_bytes) {
  const int p = U.off[U.nseg], q = V.off[V.nseg];
  if (p <= 0 || q <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  const int64_t per_slab = (int64_t)p * q * (int64_t)sizeof(float4);
  if (per_slab > work_bytes) return LOBPCG_ERR_ARG;
  int slabs;
  int64_t rps;
  gram_plan(n, p, q, &slabs, &rps);
  const int64_t cap = work_bytes / per_slab;
  if (slabs > cap) {
    slabs = (int)cap;
    rps = round_up(ceil_div(std::max<int64_t>(n, 1), slabs), KC);
    slabs = (int)std::max<int64_t>(1, ceil_div(std::max<int64_t>(n, 1), rps));
  }
  float4* partial = (float4*)work;
  int rc;
  if (n <= 0) {
    LOB_CUDA_OK(cudaMemsetAsync(partial, 0, (size_t)per_slab, st));
    slabs = 1;
    rc = LOBPCG_OK;
  } else {
    switch (slices) {
      case 3: rc = gram_launch<3>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 4: rc = gram_launch<4>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 5: rc = gram_launch<5>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 6: rc = gram_launch<6>(st, n, U, p, V, q, slabs, rps, partial); break;
      case 7: rc = gram_launch<7>(st, n, U, p, V, q, slabs, rps, partial); break;
      default: return LOBPCG_ERR_ARG;
    }
  }
  if (rc) return rc;
  ozaki_slab_reduce_kernel<<<(unsigned)ceil_div((int64_t)p * q, 256), 256, 0, st>>>(
      partial, slabs, p, q, G, ldg);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

}  // namespace lob
