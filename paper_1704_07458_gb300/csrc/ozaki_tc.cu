// Tensor-core (tcgen05 / TMEM) FP64 emulation of the two n-scaled
// contractions of an LOBPCG iteration (Sec. 5.2, Eqs. (10)-(14)): the Gram
// G = U^T V and the basis update Y = beta Y0 + alpha S C.
//
// Arithmetic (the contract of ozaki.cu): each FP64 operand is cut, relative to
// an exponent shared by a block of values, into S signed 8-bit digits (exact
// in BF16); digit products are exact; every level of digit pairs but the last
// is summed exactly in an FP32 TMEM accumulator; accumulators are converted
// exactly into int64 registers and the FP64 result is assembled with integer
// operations only.  No FP64 instruction runs on the hot path.
//
// GB300 mapping:
//  * one CTA per SM owns a 128 x NT output tile (Gram: 256 threads; update:
//    512 compute threads and one issuer warp),
//    NT <= 96 a multiple of 16: tcgen05.mma kind::f16, M = 128, N = NT, K = 16;
//  * the contraction runs in chunks of 16 (rows of U and V for the Gram,
//    columns of S for the update), grouped in blocks of 256 that share one
//    exponent per operand column (Gram) or row (update).  With |digit| <= 128
//    the sums of levels 0, 1, 2 (and 3 for S = 7) stay below 2^24 in their
//    units over a block, so they are exact in FP32; the deeper levels (below
//    2^-24 resp. 2^-32 of level 0) share one inexact accumulator.  4 or 5
//    accumulators x NT columns fit the 512 TMEM columns, and TMEM is read once
//    per block instead of once per chunk;
//  * the raw FP64 operands stream into three shared-memory stages by cp.async,
//    two chunks ahead of use, so that no thread waits on a global load; the
//    tensor core multiplies chunk c while the compute threads cut chunk c + 1
//    (two digit-plane stages in the Gram, three in the update); the digits of
//    the small matrix C of the update are cut once per call and arrive by
//    cp.async.bulk two chunks ahead;
//  * the shared exponents come from a streaming pre-pass at full occupancy
//    (per 256-row block and column for the Gram, per row for the update), so
//    the tensor-core kernels never wait on a global load of their own;
//  * every mbarrier wait is bounded: a wait that runs out marks the result NaN
//    (and, for the update, sets a status bit that the solver reads with its
//    per-iteration scalars) and the CTA returns instead of hanging.
#include <algorithm>

#include "kernels.cuh"
#include "ozaki_common.cuh"

namespace lob {
namespace {

constexpr int TCM = 128;            // MMA M
constexpr int TCK = 16;             // contraction length of a chunk (one MMA K)
constexpr int KG = TCK / 8;         // core-matrix groups along K in a chunk
constexpr int kChunksPerBlock = 16; // 256 rows / columns share one exponent
constexpr int kRaw = 3;             // raw FP64 stages (prefetch distance 2)
constexpr int kBlock = TCK * kChunksPerBlock;
constexpr int NTMAX = 96;           // max MMA N (output columns of a tile)
constexpr int kThr = 256;
constexpr int kFrac = 30;           // fraction bits of the int64 accumulators
constexpr int kEZero = -4000;       // exponent of an all-zero block
constexpr uint32_t kTmemCols = 512;
constexpr int kSpin = 1 << 22;      // bound of every mbarrier wait
constexpr int kMaxUpdateK = 6144;   // columns of S an update takes (3 n_x <= 6144)

template <int S>
__host__ __device__ constexpr int nacc() { return S >= 7 ? 5 : (S < 4 ? S : 4); }
// accumulator of digit level l = s + t (0-based digit indices)
template <int S>
__host__ __device__ constexpr int acc_of(int l) { return l < nacc<S>() - 1 ? l : nacc<S>() - 1; }
template <int S>
__host__ __device__ constexpr size_t planeA_bytes() { return (size_t)KG * (TCM / 8) * 128; }
__host__ __device__ inline size_t planeB_bytes(int NT) { return (size_t)KG * (NT / 8) * 128; }

// 0x80 in each of the S-1 low bytes: adding it turns the fixed-point value
// into bytes that are the balanced digits plus 128.
template <int S>
__host__ __device__ constexpr long long digit_bias() {
  long long b = 0;
  for (int i = 0; i < S - 1; ++i) b |= 0x80LL << (8 * i);
  return b;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Digits of x relative to the exponent bound E (|x| < 2^E): the fixed-point
// integer F = round(x 2^(8S-1-E)) (|F| <= 2^(8S-1)) written in balanced base
// 256, F = sum_s d_s 256^(S-1-s), |d_s| <= 128; returns the pre-weighted
// values d_s 2^(-8s), each exact in BF16.  Integer operations only.
template <int S>
__device__ __forceinline__ void digits(double x, int E, float (&d)[S]) {
  const long long bits = __double_as_longlong(x);
  const int be = (int)((bits >> 52) & 0x7FF);
  const long long mant = (bits & 0x000FFFFFFFFFFFFFLL) | ((long long)(be != 0) << 52);
  // F = round(mant 2^sh), sh = max(be, 1) - 1076 + 8S - E <= 2 whenever
  // |x| < 2^E (a zero x gives F = 0 for any sh).  Branch-free: with
  // v = mant 2^3 < 2^56 and t = 2 - sh clamped to [0, 63],
  // F = ((v >> t) + 1) >> 1 (round half up in magnitude).
  const int t = min(max(2 - (max(be, 1) - 1076 + 8 * S - E), 0), 63);
  const long long F = (((mant << 3) >> t) + 1) >> 1;
  const long long G = digit_bias<S>() + (bits < 0 ? -F : F);
  const uint32_t lo = (uint32_t)G, hi = (uint32_t)((unsigned long long)G >> 32);
#pragma unroll
  for (int s = 1; s < S; ++s) {
    const int b = S - 1 - s;  // byte of digit s
    const uint32_t w = b < 4 ? lo : hi;
    // 0x4B0000xx is 2^23 + xx; minus (2^23 + 128), scaled by 2^-8s (exact)
    const float f = __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (uint32_t)(b & 3)));
    const float sc = __uint_as_float((uint32_t)(127 - 8 * s) << 23);
    d[s] = fmaf(f, sc, -8388736.0f * sc);
  }
  d[0] = (float)(int)(G >> (8 * (S - 1)));
}

// 8 consecutive K values of one M/N index -> S planes, one 16-byte shared
// store per plane (K-major core-matrix row: 8 BF16 along K).
template <int S>
__device__ __forceinline__ void split8(const double (&x)[8], const int (&E)[8], uint32_t dst,
                                       uint32_t pstride) {
  uint32_t w[S][4];
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    float a[S], b[S];
    digits<S>(x[i], E[i], a);
    digits<S>(x[i + 1], E[i + 1], b);
#pragma unroll
    for (int s = 0; s < S; ++s)
      w[s][i >> 1] = __byte_perm(__float_as_uint(a[s]), __float_as_uint(b[s]), 0x7632);
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(dst + s * pstride),
                 "r"(w[s][0]), "r"(w[s][1]), "r"(w[s][2]), "r"(w[s][3])
                 : "memory");
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

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
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

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count));
}

// Bounded wait for the completion of the mbarrier phase with the given parity
// (at most `limit` polls); false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int limit = kSpin) {
  uint32_t done = 0;
  for (int spin = 0; spin < limit && !done; ++spin)
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
  return done != 0;
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   dst_smem),
               "r"(kTmemCols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
               "r"(kTmemCols));
}

// All digit-pair MMAs of one chunk (both K halves) into the accumulators.
// started: bit a set once accumulator a has been written in this block.
// (TCK = 16: one MMA of K = 16 per digit pair.)  The descriptors of the
// planes differ from the stage's first one only in the 14-bit start address
// field (shared addresses < 256 KB), so they are formed by addition.
template <int S>
__device__ __forceinline__ void issue_chunk(uint32_t tmem, int NT, uint32_t aStage,
                                            uint32_t bStage, uint32_t& started) {
  static_assert(TCK == 16, "one MMA per digit pair and chunk");
  const uint32_t lboA = (TCM / 8) * 128, lboB = (uint32_t)(NT / 8) * 128, sbo = 128;
  const uint64_t pa16 = planeA_bytes<S>() >> 4, pb16 = planeB_bytes(NT) >> 4;
  const uint32_t idesc = instr_desc(TCM, NT);
  const uint64_t da0 = smem_desc(aStage, lboA, sbo), db0 = smem_desc(bStage, lboB, sbo);
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int t = 0; t + s < S; ++t) {
      const int a = acc_of<S>(s + t);
      mma_bf16(tmem + (uint32_t)(a * NT), da0 + s * pa16, db0 + t * pb16, idesc,
               (started >> a) & 1u);
      started |= 1u << a;
    }
}

constexpr int kIssuer = kThr - 32;  // thread that issues MMAs and bulk copies (lightest split load)

// Exact int64 value (units 2^-kFrac of the level-0 unit) of the accumulators
// of one output: levels 0..2 (and 3 for S = 7) are exact FP32 integers in
// their units (< 2^24), the last accumulator is rounded at 2^-kFrac.
template <int S>
__device__ __forceinline__ long long acc_to_i64(const float (&v)[5]) {
  constexpr int NA = nacc<S>();
  long long T = 0;
#pragma unroll
  for (int a = 0; a < NA; ++a) {
    // level a in units 2^(-8a); scale so that the int32 conversion is exact
    // (exact levels) or rounds at 2^-kFrac (last accumulator)
    const bool last = (a == NA - 1) && (S >= 4);
    const int sc = last ? kFrac : 8 * a;
    const int i = __float2int_rn(v[a] * __uint_as_float((uint32_t)(127 + sc) << 23));
    T += last ? (long long)i : ((long long)i << (kFrac - 8 * a));
  }
  return T;
}

__device__ __forceinline__ long long shr_sat(long long v, int k) {
  return k <= 0 ? v : (k > 62 ? 0 : (v >> k));
}

// v * 2^e + y0 rounded to FP64 (error below 1 ulp), integer operations only.
__device__ __forceinline__ double assemble_i64(long long v, int e, double y0) {
  if ((__double_as_longlong(y0) << 1) == 0) return int_to_double_fast(v, e);  // y0 = +-0, no FP64 op
  long long my;
  int ey;
  double_parts(y0, my, ey);
  if (v == 0) return y0;
  const int top = max(e + bitlen(v), ey + bitlen(my));
  const int base = top - 61;
  const int kv = e - base, ky = ey - base;
  const long long a = kv >= 0 ? (v << kv) : shr_sat(v, -kv);
  const long long b = ky >= 0 ? (my << ky) : shr_sat(my, -ky);
  return int_to_double(a + b, base);
}

__device__ __forceinline__ void seg_col_ptr(const SegList& s, int c, const double** p,
                                            long long* ld) {
  int i = 0;
#pragma unroll
  for (int t = 1; t < kMaxSeg; ++t) i += (t < s.nseg && c >= s.off[t]) ? 1 : 0;
  *p = s.ptr[i] + (c - s.off[i]);
  *ld = s.ld[i];
}

// 8-byte global -> shared copy (zero fill when !valid; src must still be a
// mapped address), completion tracked by cp.async groups.
__device__ __forceinline__ void cp_async8(uint32_t dst, const double* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// wait until at most one group of this thread is pending
__device__ __forceinline__ void cp_async_wait1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait0() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void ld_shared_f64(uint32_t a, double& x) {
  asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(x) : "r"(a) : "memory");
}

// ------------------------------------------------------------------- Gram
constexpr int kGcols = TCM + NTMAX;  // column slots of a Gram tile: A columns, then B columns

struct GramShared {
  unsigned long long mdone[2];
  uint32_t tmem_base;
  int fail;
  int eCur[kGcols];   // exponent bounds E of the current block
  int R[kGcols];      // reference exponents of the int64 accumulators
  int dR[kGcols];     // reference increase at the current block
  const double* cptr[kGcols];
  long long cld[kGcols];
};

template <int S>
size_t gram_smem_bytes(int NT) {
  return 2 * (S * planeA_bytes<S>() + S * planeB_bytes(NT)) +
         (size_t)kRaw * TCK * kGcols * 8 + sizeof(GramShared) + 1024;
}

// E[b][c] = exponent bound of column c over rows [256 b, 256 b + 256): the
// biased exponent maximum (at least 1) minus 1022.  One warp per (block, 32
// columns), lanes over columns; high words only.
__global__ void block_col_exp_kernel(int64_t n, SegList L, int ncols, int64_t nblk,
                                     int* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int64_t b = (int64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int c = blockIdx.x * 32 + lane;
  if (b >= nblk || c >= ncols) return;
  const double* p;
  long long ld;
  seg_col_ptr(L, c, &p, &ld);
  const int64_t r0 = b * kBlock, r1 = min(n, r0 + kBlock);
  int e = 1;
  for (int64_t r = r0; r < r1; r += 16) {
    int hw[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int64_t row = min(r + i, r1 - 1);
      hw[i] = __ldg(reinterpret_cast<const int*>(p + row * ld) + 1);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) e = max(e, (hw[i] >> 20) & 0x7FF);
  }
  E[b * ncols + c] = e - 1022;
}

// Stage rows [r, r + TCK) of column slot c = tid into raw (row-major
// [TCK][kGcols]): lanes over consecutive columns (coalesced), rows by pointer
// increments.
__device__ __forceinline__ void gram_stage_raw(const GramShared& sh, int ncs, int64_t r,
                                               int64_t rend, uint32_t raw, int tid,
                                               const double* any) {
  if (tid >= ncs) return;
  const double* p = sh.cptr[tid];
  const long long ld = sh.cld[tid];
  const double* src = p ? p + r * ld : any;
  const int64_t left = rend - r;
  const int nv = !p ? 0 : (left >= TCK ? TCK : (left > 0 ? (int)left : 0));
#pragma unroll
  for (int i = 0; i < TCK; ++i) {
    cp_async8(raw + (uint32_t)(i * kGcols + tid) * 8, i < nv ? src : any, i < nv);
    src += ld;
  }
}

template <int S>
__global__ void __launch_bounds__(kThr, 1)
    ozaki_gram_tc_kernel(int64_t n, SegList U, int p, SegList V, int q, int NT,
                         int64_t blocks_per_slab, const int* __restrict__ EU,
                         const int* __restrict__ EV, int4* __restrict__ partial) {
  constexpr int NA = nacc<S>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const uint32_t pa = (uint32_t)planeA_bytes<S>(), pb = (uint32_t)planeB_bytes(NT);
  // stage st: A planes at aS0 + st * S * pa, B planes at bS0 + st * S * pb
  const uint32_t aS0 = smem_u32(base), bS0 = smem_u32(base) + 2 * S * pa;
  const uint32_t raw0 = smem_u32(base) + 2 * S * (pa + pb);
  constexpr uint32_t rawB = TCK * kGcols * 8;  // bytes per raw stage
  GramShared& sh = *reinterpret_cast<GramShared*>(base + 2 * S * (pa + pb) + kRaw * rawB);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tp = blockIdx.x * TCM, tq = blockIdx.y * NT;
  const int np_ = min(TCM, p - tp), nq_ = min(NT, q - tq);
  const int64_t nblk = ceil_div(n, kBlock);
  const int64_t b0 = (int64_t)blockIdx.z * blocks_per_slab;
  const int64_t b1 = min(nblk, b0 + blocks_per_slab);
  const int64_t r_begin = b0 * kBlock, r_end = min(n, b1 * kBlock);
  const int64_t nchunks = ceil_div(r_end - r_begin, TCK);
  const int ncs = TCM + NT;  // column slots: A columns, then B columns
  const double* any = U.ptr[0];

  for (int c = tid; c < kGcols; c += kThr) {
    const double* ptr = nullptr;
    long long ld = 0;
    if (c < TCM && c < np_) seg_col_ptr(U, tp + c, &ptr, &ld);
    if (c >= TCM && c - TCM < nq_) seg_col_ptr(V, tq + c - TCM, &ptr, &ld);
    sh.cptr[c] = ptr;
    sh.cld[c] = ld;
    sh.R[c] = kEZero;
  }
  if (warp == 0) tmem_alloc(smem_u32(&sh.tmem_base));
  if (tid == 0) {
    mbar_init(smem_u32(&sh.mdone[0]), 1);
    mbar_init(smem_u32(&sh.mdone[1]), 1);
    sh.fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = sh.tmem_base;

  // prologue: first two chunks in flight
  for (int g = 0; g < 2; ++g) {
    if (g < nchunks)
      gram_stage_raw(sh, ncs, r_begin + (int64_t)g * TCK, r_end, raw0 + g * rawB, tid, any);
    cp_async_commit();
  }
  cp_async_wait1();
  __syncthreads();

  // flush ownership: TMEM lane = A column my_i, B columns j0 .. j0 + NT/2 - 1
  const int my_i = 32 * (warp & 3) + lane;
  const int half = NT / 2;
  const int j0 = half * (warp >> 2);
  const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
  long long acc[NTMAX / 2];
#pragma unroll
  for (int j = 0; j < NTMAX / 2; ++j) acc[j] = 0;
  bool failed = false;
  uint32_t started = 0;
  int64_t gc = 0;  // chunk counter of the slab
  // cut items of this thread: (column slot, 8-row group), at most two
  int it_c[2], it_kg[2];
  uint32_t it_dst[2], it_ps[2];
  int nit = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int it = tid + h * kThr;
    it_c[h] = it % ncs;
    it_kg[h] = it / ncs;
    if (it < ncs * KG) nit = h + 1;
    const int c = it_c[h], kg = it_kg[h];
    it_dst[h] = c < TCM ? (uint32_t)((kg * (TCM / 8) + (c >> 3)) * 128 + (c & 7) * 16)
                        : (uint32_t)((kg * (NT / 8) + ((c - TCM) >> 3)) * 128 + ((c - TCM) & 7) * 16);
    it_ps[h] = c < TCM ? pa : pb;
  }

  for (int64_t b = b0; b < b1 && !failed; ++b) {
    // ---- block start: exponents of this block, reference update
    for (int c = tid; c < ncs; c += kThr) {
      const int E = !sh.cptr[c] ? kEZero
                    : c < TCM    ? EU[b * p + tp + c]
                                 : EV[b * q + tq + c - TCM];
      const int Rn = max(sh.R[c], E);
      sh.dR[c] = Rn - sh.R[c];
      sh.R[c] = Rn;
      sh.eCur[c] = E;
    }
    __syncthreads();
    started = 0;
    const int64_t rb = b * kBlock;
    for (int ch = 0; ch < kChunksPerBlock; ++ch) {
      const int64_t r = rb + (int64_t)ch * TCK;
      if (r >= r_end) break;
      const uint32_t st = (uint32_t)(gc & 1);
      const uint32_t raw = raw0 + (uint32_t)(gc % kRaw) * rawB;
      if (gc >= 2 && !mbar_wait(smem_u32(&sh.mdone[st]), (uint32_t)((gc >> 1) - 1) & 1))
        sh.fail = 1;
      // cut the staged chunk: items (column slot, 8-row group)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h < nit) {
          const int c = it_c[h], kg = it_kg[h];
          double x[8];
          int E[8];
          const int Ec = sh.eCur[c];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            ld_shared_f64(raw + (uint32_t)((kg * 8 + i) * kGcols + c) * 8, x[i]);
            E[i] = Ec;
          }
          const uint32_t base_st = c < TCM ? aS0 + st * S * pa : bS0 + st * S * pb;
          split8<S>(x, E, base_st + it_dst[h], it_ps[h]);
        }
      }
      // chunk gc + 2 into the stage just read by chunk gc - 1
      if (gc + 2 < nchunks)
        gram_stage_raw(sh, ncs, r_begin + (gc + 2) * TCK, r_end,
                       raw0 + (uint32_t)((gc + 2) % kRaw) * rawB, tid, any);
      cp_async_commit();
      cp_async_wait1();  // chunk gc + 1 has landed (this thread's copies)
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      if (__syncthreads_or(sh.fail)) {
        failed = true;
        break;
      }
      if (tid == kIssuer) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        issue_chunk<S>(tmem, NT, aS0 + st * S * pa, bS0 + st * S * pb, started);
        mma_commit(smem_u32(&sh.mdone[st]));
      }
      ++gc;
    }
    if (failed) break;
    // ---- block end: wait for the last chunk's MMAs, fold TMEM into int64
    if (!mbar_wait(smem_u32(&sh.mdone[(gc - 1) & 1]), (uint32_t)((gc - 1) >> 1) & 1)) sh.fail = 1;
    if (__syncthreads_or(sh.fail)) {
      failed = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    {
      const int Ei = sh.eCur[my_i], Ri = sh.R[my_i], di = sh.dR[my_i];
#pragma unroll
      for (int g = 0; g < NTMAX / 16; ++g) {
        if (8 * g < half) {
          float v[NA][8];
#pragma unroll
          for (int a = 0; a < NA; ++a) tmem_ld8(tmem + lane_off + a * NT + j0 + 8 * g, v[a]);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int cj = TCM + j0 + 8 * g + i;
            float w[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int a = 0; a < NA; ++a) w[a] = v[a][i];
            const long long T = acc_to_i64<S>(w);
            const int shift = Ri + sh.R[cj] - Ei - sh.eCur[cj];
            acc[8 * g + i] = shr_sat(acc[8 * g + i], di + sh.dR[cj]) + shr_sat(T, shift);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
  }
  cp_async_wait0();  // no copy may outlive the CTA
  // ---- slab partial: (value, exponent) = acc * 2^(R_i + R_j - 14 - kFrac)
  if (my_i < np_) {
    int4* out = partial + ((int64_t)blockIdx.z * p + tp + my_i) * q + tq;
#pragma unroll
    for (int g = 0; g < NTMAX / 16; ++g)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int j = j0 + 8 * g + i;
        if (8 * g < half && j < nq_) {
          const long long v = failed ? 0 : acc[8 * g + i];
          int4 w;
          w.x = (int)(unsigned)(unsigned long long)v;
          w.y = (int)(v >> 32);
          w.z = sh.R[my_i] + sh.R[TCM + j] - 14 - kFrac;
          w.w = failed ? 1 : 0;
          out[j] = w;
        }
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    tmem_dealloc(tmem);
  }
}

// G(i, j) = sum over slabs of the int64 partials, aligned and summed in 128-bit
// integers in slab order (deterministic), rounded once to FP64.
__global__ void gram_tc_reduce_kernel(const int4* __restrict__ partial, int slabs, int p, int q,
                                      double* __restrict__ G, int64_t ldg) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)p * q) return;
  const int i = (int)(idx / q), j = (int)(idx % q);
  int emax = -2000000000;
  bool bad = false;
  for (int s = 0; s < slabs; ++s) {
    const int4 w = partial[((int64_t)s * p + i) * q + j];
    bad |= w.w != 0;
    if (w.x != 0 || w.y != 0) emax = max(emax, w.z);
  }
  double out = 0.0;
  if (bad) {
    out = __longlong_as_double(0x7FF8000000000000LL);
  } else if (emax > -2000000000) {
    __int128 sum = 0;
    for (int s = 0; s < slabs; ++s) {
      const int4 w = partial[((int64_t)s * p + i) * q + j];
      const long long v = ((long long)w.y << 32) | (long long)(unsigned)w.x;
      if (v == 0) continue;
      const int k = emax - w.z;  // >= 0
      if (k < 100) sum += (((__int128)v) << 56) >> k;
    }
    if (sum != 0) {
      const bool neg = sum < 0;
      const unsigned __int128 a = neg ? (unsigned __int128)(-sum) : (unsigned __int128)sum;
      const unsigned long long hi = (unsigned long long)(a >> 64), lo = (unsigned long long)a;
      const int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
      const int sh = top > 62 ? top - 62 : 0;
      unsigned long long m = (unsigned long long)(a >> sh);
      if (sh > 0 && (a & ((((unsigned __int128)1) << sh) - 1)) != 0) m |= 1;  // sticky
      out = int_to_double(neg ? -(long long)m : (long long)m, emax - 56 + sh);
    }
  }
  G[i + (int64_t)j * ldg] = out;
}

void gram_tiles(int q, int* ntq, int* NT) {
  *ntq = (int)ceil_div(q, NTMAX);
  *NT = (int)round_up(ceil_div(q, *ntq), 16);
}

void gram_plan(int64_t n, int p, int q, int* slabs, int64_t* per_slab) {
  int ntq, NT;
  gram_tiles(q, &ntq, &NT);
  const int64_t tiles = ceil_div(p, TCM) * ntq;
  const int64_t nblk = std::max<int64_t>(1, ceil_div(n, kBlock));
  // one wave of CTAs; at most 64 blocks per slab keeps the int64 sums < 2^61
  int64_t s = std::max<int64_t>(ceil_div(152, tiles), ceil_div(nblk, 64));
  s = std::min(s, nblk);
  const int64_t per = ceil_div(nblk, s);
  *slabs = (int)ceil_div(nblk, per);
  *per_slab = per;
}

template <int S>
int gram_tc_launch(cudaStream_t st, int64_t n, const SegList& U, int p, const SegList& V, int q,
                   int slabs, int64_t per, const int* EU, const int* EV, int4* partial) {
  int ntq, NT;
  gram_tiles(q, &ntq, &NT);
  const size_t sh = gram_smem_bytes<S>(NTMAX);
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_gram_tc_kernel<S>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  dim3 grid((unsigned)ceil_div(p, TCM), (unsigned)ntq, (unsigned)slabs);
  ozaki_gram_tc_kernel<S><<<grid, kThr, gram_smem_bytes<S>(NT), st>>>(n, U, p, V, q, NT, per, EU,
                                                                      EV, partial);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// ----------------------------------------------------------------- update
// Y = beta Y0 + alpha S C.  A = S (M = 128 rows, K = s columns; one exponent
// per row over all columns of the balanced S(i, k) 2^-colexp[k]), B = alpha C
// with rows scaled by 2^colexp[k] (one exponent per column over all k), cut
// once per call by split_c_tc_kernel into the shared-memory plane layout
// [chunk][tile][S][KG][NT/8][8][8].  Persistent CTAs walk the (row block,
// column tile) pairs; the row exponents of a CTA's next tile are computed
// during its current tile.

template <int S>
__global__ void split_c_tc_kernel(const double* __restrict__ C, int64_t ldc, int s, int m,
                                  int ntiles, int NT, double alpha, const int* __restrict__ colexp,
                                  uint16_t* __restrict__ Cs, int* __restrict__ Ce) {
  // one warp per padded column; lanes over k
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int ncols = ntiles * NT;
  if (w >= ncols) return;
  const int tile = w / NT, j = w % NT;
  const int nch = (int)ceil_div(s, TCK);
  auto val = [&](int k) -> double {
    if (w >= m || k >= s) return 0.0;
    return ldexp(alpha * C[k + (int64_t)w * ldc], colexp ? colexp[k] : 0);
  };
  int e = 0;  // biased exponent maximum; 0 = all zero
  for (int k = lane; k < s; k += 32) {
    const double x = val(k);
    if (x != 0.0) e = max(e, max((int)((__double_as_longlong(x) >> 52) & 0x7FF), 1));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  const int E = e ? e - 1022 : kEZero;
  if (lane == 0) Ce[w] = E;
  const size_t blk = (size_t)S * KG * (NT / 8) * 64;  // bf16 per (chunk, tile)
  for (int k = lane; k < nch * TCK; k += 32) {
    float d[S];
    digits<S>(val(k), E, d);
    const int ch = k / TCK, kk = k % TCK;
    uint16_t* dst = Cs + (size_t)(ch * ntiles + tile) * blk;
#pragma unroll
    for (int sl = 0; sl < S; ++sl)
      dst[(((size_t)sl * KG + (kk >> 3)) * (NT / 8) + (j >> 3)) * 64 + (j & 7) * 8 + (kk & 7)] =
          (uint16_t)(__float_as_uint(d[sl]) >> 16);
  }
}

constexpr int kRawRow = TCK + 1;  // raw row pitch in doubles (odd: conflict-free 8-byte reads)
constexpr int kUThr = 512;        // compute threads of the update (16 warps)
constexpr int kUThrAll = kUThr + 32;  // + one issuer warp
constexpr int kUIssuer = kUThr;   // issuer thread of the update (warp 16, lane 0)
constexpr int kUStages = 3;       // digit-plane stages of A and B (chunks in flight)
constexpr int kUCols = NTMAX / 32 * 8;  // output columns of one thread (8-column groups cg + 4 i)

struct UpdShared {
  unsigned long long bfull[kUStages], mdone[kUStages];
  uint32_t tmem_base;
  int fail;
  int eA[TCM];     // row exponent bounds of the balanced S, current tile
  int eC[NTMAX];   // column exponent bounds of the balanced C, current tile
  SegList seg;
};

// ER[i] = exponent bound of row i of the balanced S(i, k) 2^-colexp[k] over all
// k (kEZero for a zero row).  One warp per row, lanes over the columns of each
// segment in turn (plain pointer arithmetic within a segment).
__global__ void row_exp_kernel(int64_t n, SegList Sg, int s, const int* __restrict__ colexp,
                               int* __restrict__ ER) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  int e = -1000000;
#pragma unroll
  for (int g = 0; g < kMaxSeg; ++g) {
    if (g >= Sg.nseg) break;
    const int c0 = Sg.off[g], w = Sg.off[g + 1] - c0;
    const double* base = Sg.ptr[g] + row * Sg.ld[g];
    for (int c = lane; c < w; c += 64) {  // two loads in flight per lane
      const bool two = c + 32 < w;
      const long long b0 = __double_as_longlong(__ldg(base + c));
      const long long b1 = two ? __double_as_longlong(__ldg(base + c + 32)) : 0LL;
      const int x0 = colexp ? __ldg(colexp + c0 + c) : 0;
      const int x1 = (colexp && two) ? __ldg(colexp + c0 + c + 32) : 0;
      if ((b0 << 1) != 0) e = max(e, max((int)((b0 >> 52) & 0x7FF), 1) - x0);
      if ((b1 << 1) != 0) e = max(e, max((int)((b1 >> 52) & 0x7FF), 1) - x1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) ER[row] = e > -1000000 ? e - 1022 : kEZero;
}

__device__ __forceinline__ void upd_k(const UpdShared& sh, int k, const double** p,
                                      long long* ld) {
  seg_col_ptr(sh.seg, k, p, ld);
}

// Stage S(rows row0 .. row0 + 127, columns kc .. kc + TCK - 1) into raw
// ([TCM][kRawRow]); zero outside the matrix.
__device__ __forceinline__ void upd_stage_raw(const UpdShared& sh, int64_t n, int s, int64_t row0,
                                              int kc, uint32_t raw, int tid) {
  // thread: column kk = tid % TCK, rows tid / TCK + 32 j (coalesced along k)
  const int kk = tid % TCK, r0 = tid / TCK;
  const int k = kc + kk;
  const double* p;
  long long ld;
  upd_k(sh, k < s ? k : 0, &p, &ld);
  const double* src = p + (row0 + r0) * ld;
  const long long step = (long long)(kUThr / TCK) * ld;
#pragma unroll
  for (int j = 0; j < TCM * TCK / kUThr; ++j) {
    const int rl = r0 + j * (kUThr / TCK);
    const bool ok = k < s && row0 + rl < n;
    cp_async8(raw + (uint32_t)(rl * kRawRow + kk) * 8, ok ? src : p, ok);
    src += step;
  }
}

// 4 consecutive K values of one M index -> S planes, one 8-byte shared store
// per plane (half a K-major core-matrix row).
template <int S>
__device__ __forceinline__ void split4(const double (&x)[4], const int (&E)[4], uint32_t dst,
                                       uint32_t pstride) {
  uint32_t w[S][2];
#pragma unroll
  for (int i = 0; i < 4; i += 2) {
    float a[S], b[S];
    digits<S>(x[i], E[i], a);
    digits<S>(x[i + 1], E[i + 1], b);
#pragma unroll
    for (int sl = 0; sl < S; ++sl)
      w[sl][i >> 1] = __byte_perm(__float_as_uint(a[sl]), __float_as_uint(b[sl]), 0x7632);
  }
#pragma unroll
  for (int sl = 0; sl < S; ++sl)
    asm volatile("st.shared.v2.b32 [%0], {%1, %2};\n" ::"r"(dst + sl * pstride), "r"(w[sl][0]),
                 "r"(w[sl][1])
                 : "memory");
}

template <int S>
__host__ __device__ inline size_t upd_regionA(int NT) {
  const size_t a = (size_t)kUStages * S * planeA_bytes<S>();
  return (a + 1023) / 1024 * 1024;
}

template <int S>
size_t upd_smem_bytes(int NT, int s) {
  return upd_regionA<S>(NT) + (size_t)kUStages * S * planeB_bytes(NT) +
         (size_t)kRaw * TCM * kRawRow * 8 + sizeof(UpdShared) +
         (size_t)round_up(std::max(s, 1), 4) * 4 + 1024;
}

// One CTA per SM: 16 compute warps cut the staged S chunks into digit planes
// and convert the TMEM accumulators; one issuer thread (warp 16) issues the
// MMAs and the bulk copies of C's digits.  Three plane stages: the issuer
// fetches C's digits of chunk g + 2 while the tensor core multiplies chunk g
// and the compute warps cut chunk g + 1.
// kOneBlock: s <= 256, a single exponent block; the TMEM accumulators go
// straight to the output (no int64 carry registers).
// 17 warps: the busiest of the four SM sub-partitions holds five, so the
// register cap is 16,384 / (5 x 32) -> 96 per thread (the multi-block
// variant spills its int64 carries a little; the s <= 256 one does not)
template <int S, bool kOneBlock>
__global__ void __launch_bounds__(kUThrAll, 1)
    ozaki_update_tc_kernel(int64_t n, SegList Sg, int s, const int* __restrict__ colexp,
                           const uint16_t* __restrict__ Cs, const int* __restrict__ Ce,
                           const int* __restrict__ ER, int m, int ntiles, int NT,
                           int64_t ntile_total, double beta, SegList Y0, OutList Y,
                           int* status) {
  constexpr int NA = nacc<S>();
  constexpr int NS = kUStages;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  const uint32_t pa = (uint32_t)planeA_bytes<S>(), pb = (uint32_t)planeB_bytes(NT);
  const size_t regA = upd_regionA<S>(NT);
  // region A: the A planes of the stages
  const uint32_t aS0 = smem_u32(base), bS0 = smem_u32(base) + (uint32_t)regA;
  const uint32_t raw0 = bS0 + NS * S * pb;
  constexpr uint32_t rawB = TCM * kRawRow * 8;
  unsigned char* after_raw = base + regA + (size_t)NS * S * pb + kRaw * rawB;
  UpdShared& sh = *reinterpret_cast<UpdShared*>(after_raw);
  int* cx = reinterpret_cast<int*>(after_raw + sizeof(UpdShared));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool compute = tid < kUThr;
  const bool has_y0 = beta != 0.0;  // the kernel's only FP64 operation
  const int nch = (int)ceil_div(s, TCK);
  const size_t cs_blk = (size_t)S * KG * (NT / 8) * 64;  // bf16 per (chunk, tile)
  const uint32_t bbytes = (uint32_t)(cs_blk * 2);

  if (warp == 0) tmem_alloc(smem_u32(&sh.tmem_base));
  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(smem_u32(&sh.bfull[i]), 1);
      mbar_init(smem_u32(&sh.mdone[i]), 1);
    }
    sh.fail = 0;
    sh.seg = Sg;
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  for (int k = tid; k < s; k += kUThrAll) cx[k] = colexp ? colexp[k] : 0;
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = sh.tmem_base;

  // digit split: row rl of the tile, columns 4 kq .. 4 kq + 3 of the chunk
  // (lane pairs share a row: a warp's 8-byte plane stores are contiguous)
  const int rl = 16 * (warp & 7) + (lane >> 1), kq = 2 * ((warp >> 3) & 1) + (lane & 1);
  const uint32_t aoff =
      (uint32_t)(((kq >> 1) * (TCM / 8) + (rl >> 3)) * 128 + (rl & 7) * 16 + (kq & 1) * 8);
  // epilogue: TMEM lane quarter q (tile rows 32 q ..), 8-column groups cg + 4 i
  const int q = warp & 3, cg = (warp >> 2) & 3;
  const int my_r = 32 * q + lane;
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  bool failed = false;
  int64_t gc = 0;  // chunk counter of this CTA over all its tiles
  const int64_t t0 = blockIdx.x, tstep = gridDim.x;
  auto tile_row0 = [&](int64_t t) { return (t / ntiles) * TCM; };
  const int64_t my_chunks = ((ntile_total - t0 + tstep - 1) / tstep) * nch;
  // chunk g of this CTA: tile t0 + (g / nch) tstep, columns (g % nch) TCK;
  // plane stage g % NS, used for the (g / NS)-th time.  Staging (every
  // compute thread) and the B copies (issuer) each walk the chunks in order,
  // so their positions advance by one chunk per call: no division by a
  // runtime value per chunk (64-bit division is a long software sequence).
  int64_t st_g = 0, st_t = t0, st_row0 = tile_row0(t0);
  int st_c = 0, st_slot = 0;
  auto stage_next = [&]() {  // raw S of chunk st_g into raw stage st_g % kRaw
    if (st_g < my_chunks)
      upd_stage_raw(sh, n, s, st_row0, st_c * TCK, raw0 + (uint32_t)st_slot * rawB, tid);
    cp_async_commit();
    ++st_g;
    st_slot = st_slot + 1 == kRaw ? 0 : st_slot + 1;
    if (++st_c == nch) {
      st_c = 0;
      st_t += tstep;
      st_row0 = tile_row0(st_t);
    }
  };
  int64_t lb_g = 0, lb_t = t0;
  int lb_c = 0, lb_tile = (int)(t0 % ntiles);
  auto load_b_next = [&]() {  // issuer: B digits of chunk lb_g into stage lb_g % NS
    const uint32_t st = (uint32_t)(lb_g % NS);
    const size_t src = ((size_t)lb_c * ntiles + (size_t)lb_tile) * cs_blk;
    ++lb_g;
    if (++lb_c == nch) {
      lb_c = 0;
      lb_t += tstep;
      lb_tile = (int)(lb_t % ntiles);
    }
    uint64_t state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;\n"
                 : "=l"(state)
                 : "r"(smem_u32(&sh.bfull[st])), "r"(bbytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];\n" ::"r"(bS0 + st * S * pb),
        "l"(Cs + src), "r"(bbytes), "r"(smem_u32(&sh.bfull[st]))
        : "memory");
  };
  auto parity = [](int64_t g) { return (uint32_t)((g / NS) & 1); };
  int64_t b_issued = -1;  // last chunk whose B copy the issuer started
  int64_t m_issued = -1;  // last chunk whose MMAs the issuer committed
  if (compute) {
    stage_next();
    stage_next();
    cp_async_wait1();
  } else if (tid == kUIssuer) {
    for (int64_t g = 0; g < 2 && g < my_chunks; ++g) {
      load_b_next();
      b_issued = g;
    }
  }
  __syncthreads();

  for (int64_t t = t0; t < ntile_total && !failed; t += tstep) {
    const int tile = (int)(t % ntiles);
    const int64_t row0 = tile_row0(t);
    const int tn = tile * NT;
    const int nq_ = min(NT, m - tn);
    for (int r = tid; r < TCM; r += kUThrAll) sh.eA[r] = row0 + r < n ? ER[row0 + r] : kEZero;
    for (int j = tid; j < NTMAX; j += kUThrAll) sh.eC[j] = j < NT ? Ce[tn + j] : kEZero;
    __syncthreads();
    long long acc[kOneBlock ? 1 : kUCols];
#pragma unroll
    for (int j = 0; j < (kOneBlock ? 1 : kUCols); ++j) acc[j] = 0;
    uint32_t started = 0;
    for (int kc = 0; kc < s && !failed; kc += kBlock) {  // blocks of 256 columns
      started = 0;
      const int kend = min(s, kc + kBlock);
      const bool last_block = kend >= s;
      for (int k1 = kc; k1 < kend; k1 += TCK) {
        const uint32_t st = (uint32_t)(gc % NS);
        if (compute) {
          const uint32_t raw = raw0 + (uint32_t)(gc % kRaw) * rawB;
          // the stage's planes are free once the MMAs of chunk gc - NS are done
          if (gc >= NS && !mbar_wait(smem_u32(&sh.mdone[st]), parity(gc - NS))) sh.fail = 1;
          {
            double x[4];
            int E[4];
            const int Er = sh.eA[rl];
            const uint32_t src = raw + (uint32_t)(rl * kRawRow + kq * 4) * 8;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              ld_shared_f64(src + 8 * i, x[i]);
              const int k = k1 + kq * 4 + i;
              E[i] = Er + (k < s ? cx[k] : 0);
            }
            split4<S>(x, E, aS0 + st * S * pa + aoff, pa);
          }
          stage_next();  // chunk gc + 2
          cp_async_wait1();
          asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        if (__syncthreads_or(sh.fail)) {
          failed = true;
          break;
        }
        if (tid == kUIssuer) {
          if (!mbar_wait(smem_u32(&sh.bfull[st]), parity(gc))) {
            sh.fail = 1;
          } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            issue_chunk<S>(tmem, NT, aS0 + st * S * pa, bS0 + st * S * pb, started);
            mma_commit(smem_u32(&sh.mdone[st]));
            m_issued = gc;
            // B of chunk gc + 2 into the stage of chunk gc - 1 once its MMAs are done
            if (gc + 2 < my_chunks) {
              if (gc >= 1 &&
                  !mbar_wait(smem_u32(&sh.mdone[(gc - 1) % NS]), parity(gc - 1))) {
                sh.fail = 1;
              } else {
                load_b_next();  // chunk gc + 2
                b_issued = gc + 2;
              }
            }
          }
        }
        ++gc;
      }
      if (failed) break;
      if (!mbar_wait(smem_u32(&sh.mdone[(gc - 1) % NS]), parity(gc - 1))) sh.fail = 1;
      if (__syncthreads_or(sh.fail)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      if (!last_block) {
        if (!kOneBlock && compute) {
#pragma unroll
          for (int i = 0; i < kUCols / 8; ++i) {
            const int g = cg + 4 * i;
            if (8 * g < NT) {
              float v[NA][8];
#pragma unroll
              for (int a = 0; a < NA; ++a) tmem_ld8(tmem + lane_off + a * NT + 8 * g, v[a]);
              asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                float w[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < NA; ++a) w[a] = v[a][c];
                if (!kOneBlock) acc[(8 * i + c) % (kOneBlock ? 1 : kUCols)] += acc_to_i64<S>(w);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
      }
    }
    // ---- output: Y = acc 2^(E_row + E_col - 14 - kFrac) + beta Y0.  All
    // sixteen compute warps convert at once: a warp owns its TMEM lane
    // quarter's 32 rows and the 8-column groups cg + 4 i, and each thread
    // stores the 8 consecutive outputs of its row per group straight to
    // global memory (no staging pass, no barrier between conversion and
    // store)
    if (compute) {
      const int64_t row = row0 + my_r;
      const bool live = row < n;
      const int Er = sh.eA[my_r];
#pragma unroll
      for (int i = 0; i < kUCols / 8; ++i) {
        const int g = cg + 4 * i;
        if (8 * g < NT) {  // warp-uniform: the TMEM loads are .sync.aligned
          float v[NA][8];
          if (!failed) {
#pragma unroll
            for (int a = 0; a < NA; ++a) tmem_ld8(tmem + lane_off + a * NT + 8 * g, v[a]);
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          }
          if (live) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const int j = 8 * g + c;
              if (j < nq_) {
                double out = __longlong_as_double(0x7FF8000000000000LL);
                if (!failed) {
                  float w[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                  for (int a = 0; a < NA; ++a) w[a] = v[a][c];
                  long long T = acc_to_i64<S>(w);
                  if (!kOneBlock) T += acc[(8 * i + c) % (kOneBlock ? 1 : kUCols)];
                  const double y0 = has_y0 ? seg_load(Y0, tn + j, row) : 0.0;
                  out = assemble_i64(T, Er + sh.eC[j] - 14 - kFrac, y0);
                }
                *out_addr(Y, tn + j, row) = out;
              }
            }
          }
        }
      }
    }
    // TMEM and the tile's exponents are reused by the next tile
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
  }
  if (compute) cp_async_wait0();  // no copy may outlive the CTA
  if (tid == 0 && failed && status) atomicOr(status, 1);
  if (tid == kUIssuer && failed) {
    // drain what is still in flight: the B copies not yet consumed and the
    // last committed MMAs (bounded waits; their outcome no longer matters)
    for (int64_t g = m_issued + 1; g <= b_issued; ++g)
      mbar_wait(smem_u32(&sh.bfull[g % NS]), parity(g));
    if (m_issued >= 0) mbar_wait(smem_u32(&sh.mdone[m_issued % NS]), parity(m_issued));
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    tmem_dealloc(tmem);
  }
}

void update_tiles(int m, int* ntiles, int* NT) {
  *ntiles = (int)ceil_div(std::max(m, 1), NTMAX);
  *NT = (int)round_up(ceil_div(std::max(m, 1), *ntiles), 16);
}

template <int S>
int update_tc_launch(cudaStream_t st, int64_t n, const SegList& Sg, int s, const double* C,
                     int64_t ldc, int m, double alpha, double beta, const SegList& Y0,
                     const OutList& Y, const int* colexp, void* work, int* status) {
  int ntiles, NT;
  update_tiles(m, &ntiles, &NT);
  const int nch = (int)ceil_div(s, TCK);
  uint16_t* Cs = (uint16_t*)work;
  const size_t cs_elems = (size_t)nch * ntiles * S * KG * (NT / 8) * 64;
  int* Ce = (int*)(Cs + cs_elems);
  int* cxw = Ce + (size_t)ntiles * NT;
  int* ER = cxw + s;
  if (!colexp) {
    int rc = column_exponents(st, n, Sg, s, cxw);
    if (rc) return rc;
    colexp = cxw;
  }
  row_exp_kernel<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(n, Sg, s, colexp, ER);
  LOB_LAUNCHED();
  {
    const int64_t warps = (int64_t)ntiles * NT;
    split_c_tc_kernel<S><<<(unsigned)ceil_div(warps * 32, 256), 256, 0, st>>>(
        C, ldc, s, m, ntiles, NT, alpha, colexp, Cs, Ce);
    LOB_LAUNCHED();
  }
  const size_t shmax = upd_smem_bytes<S>(NTMAX, kMaxUpdateK);
  // the attribute is per device: set it once on every device that launches
  static bool configured[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_update_tc_kernel<S, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmax));
    LOB_CUDA_OK(cudaFuncSetAttribute(ozaki_update_tc_kernel<S, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shmax));
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  const int64_t tiles = ceil_div(n, TCM) * ntiles;
  const int64_t grid = std::min<int64_t>(tiles, 152);
  if (s <= kBlock)
    ozaki_update_tc_kernel<S, true><<<(unsigned)grid, kUThrAll, upd_smem_bytes<S>(NT, s), st>>>(
        n, Sg, s, colexp, Cs, Ce, ER, m, ntiles, NT, tiles, beta, Y0, Y, status);
  else
    ozaki_update_tc_kernel<S, false><<<(unsigned)grid, kUThrAll, upd_smem_bytes<S>(NT, s), st>>>(
        n, Sg, s, colexp, Cs, Ce, ER, m, ntiles, NT, tiles, beta, Y0, Y, status);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

// One CTA waits on the first phase of a barrier that expects one arrival and
// gets none: the bounded wait must run out and report it in *status (bit 0),
// as the Gram and update kernels do, and the CTA must return normally.
__global__ void wait_selftest_kernel(int limit, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, limit)) atomicOr(status, 1);
}

}  // namespace

int wait_selftest(cudaStream_t st, int limit, int* status) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit, status);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int64_t gram_tc_workspace(int64_t n, int p, int q) {
  int slabs;
  int64_t per;
  gram_plan(n, p, q, &slabs, &per);
  const int64_t nblk = std::max<int64_t>(1, ceil_div(n, kBlock));
  return (int64_t)slabs * p * q * (int64_t)sizeof(int4) + nblk * (p + q) * 4;
}

int gram_tc(cudaStream_t st, int64_t n, const SegList& U, const SegList& V, double* G,
            int64_t ldg, int slices, void* work, int64_t work_bytes) {
  const int p = U.off[U.nseg], q = V.off[V.nseg];
  if (p <= 0 || q <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  if (n <= 0) return gram_ozaki(st, n, U, V, G, ldg, slices, work, work_bytes);
  int slabs;
  int64_t per;
  gram_plan(n, p, q, &slabs, &per);
  if (work_bytes < gram_tc_workspace(n, p, q)) return LOBPCG_ERR_ARG;
  if (slices < 3 || slices > 7) return LOBPCG_ERR_ARG;
  int4* partial = (int4*)work;
  const int64_t nblk = ceil_div(n, kBlock);
  int* EU = (int*)(partial + (int64_t)slabs * p * q);
  int* EV = EU + nblk * p;
  block_col_exp_kernel<<<dim3((unsigned)ceil_div(p, 32), (unsigned)ceil_div(nblk, 8)), 256, 0,
                         st>>>(n, U, p, nblk, EU);
  LOB_LAUNCHED();
  block_col_exp_kernel<<<dim3((unsigned)ceil_div(q, 32), (unsigned)ceil_div(nblk, 8)), 256, 0,
                         st>>>(n, V, q, nblk, EV);
  LOB_LAUNCHED();
  int rc;
  switch (slices) {
    case 3: rc = gram_tc_launch<3>(st, n, U, p, V, q, slabs, per, EU, EV, partial); break;
    case 4: rc = gram_tc_launch<4>(st, n, U, p, V, q, slabs, per, EU, EV, partial); break;
    case 5: rc = gram_tc_launch<5>(st, n, U, p, V, q, slabs, per, EU, EV, partial); break;
    case 6: rc = gram_tc_launch<6>(st, n, U, p, V, q, slabs, per, EU, EV, partial); break;
    default: rc = gram_tc_launch<7>(st, n, U, p, V, q, slabs, per, EU, EV, partial); break;
  }
  if (rc) return rc;
  const int64_t total = (int64_t)p * q;
  gram_tc_reduce_kernel<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>(partial, slabs, p, q, G,
                                                                         ldg);
  LOB_LAUNCHED();
  return LOBPCG_OK;
}

int64_t update_tc_workspace(int64_t n, int s, int m, int slices) {
  if (slices == 0) slices = 6;
  int ntiles, NT;
  update_tiles(m, &ntiles, &NT);
  const int64_t nch = ceil_div(std::max(s, 1), TCK);
  return nch * ntiles * slices * KG * (NT / 8) * 64 * 2 + (int64_t)ntiles * NT * 4 +
         (int64_t)std::max(s, 1) * 4 + std::max<int64_t>(n, 1) * 4 + 256;
}

int update_tc(cudaStream_t st, int64_t n, const SegList& S, const double* C, int64_t ldc, int m,
              double alpha, double beta, const SegList& Y0, const OutList& Y, int slices,
              void* work, int64_t work_bytes, const int* colexp, int* status) {
  const int s = S.off[S.nseg];
  if (n <= 0 || m <= 0) return LOBPCG_OK;
  if (slices == 0) slices = 6;
  if (s == 0) return update_f64(st, n, S, C, ldc, m, alpha, beta, Y0, Y);
  if (s > kMaxUpdateK) return LOBPCG_ERR_ARG;
  if (work_bytes < update_tc_workspace(n, s, m, slices)) return LOBPCG_ERR_ARG;
  if (beta != 0.0 && beta != 1.0) return LOBPCG_ERR_ARG;
  switch (slices) {
    case 3: return update_tc_launch<3>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work, status);
    case 4: return update_tc_launch<4>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work, status);
    case 5: return update_tc_launch<5>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work, status);
    case 6: return update_tc_launch<6>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work, status);
    case 7: return update_tc_launch<7>(st, n, S, s, C, ldc, m, alpha, beta, Y0, Y, colexp, work, status);
    default: return LOBPCG_ERR_ARG;
  }
}

}  // namespace lob
