// Rate of tcgen05.mma kind::f16 (BF16 operands, FP32 accumulator in TMEM),
// M = 128, K = 16, on one CTA per SM: 400 chunks of 21 MMAs, each chunk
// committed to an mbarrier, the MMAs of a chunk rotating over 4 (N <= 128)
// or 2 accumulators.  Operands are zero-filled shared memory (or TMEM for A);
// only the timing matters.  Two issuing threads are compared:
//   probe_unrolled  descriptors precomputed, the 21 MMAs unrolled with
//                   compile-time operands: the tensor pipe's own rate;
//   probe_runtime   descriptors built per MMA with integer modulo and a
//                   run-time layout switch: bound by the issuing thread.
// Layouts (MODE): 0 no swizzle, 8x16-byte core matrices (LBO 2048 / N*16,
// SBO 128); 2 128-byte swizzle, K-major (SBO 1024, four K = 16 slices per
// atom row selected by a 32-byte start advance); 3 A read from TMEM
// (columns after the accumulators), B as 0.  Every wait is bounded; each
// CTA frees its TMEM on every path.
// Build and run: python -m paper_1704_07458_gb300.profiling mma-rate
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

constexpr int kSpin = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count));
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  uint32_t done = 0;
  for (int spin = 0; spin < kSpin && !done; ++spin)
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
// layout: 0 none, 6 32-byte swizzle, 2 128-byte swizzle (bits 61-63)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                              uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)(layout & 7) << 61;
  return d;
}
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate));
}

constexpr uint32_t kAbytes = 32 * 1024;
constexpr uint32_t kBbytes = 64 * 1024;
constexpr size_t kSmem = kAbytes + kBbytes + 1024;

template <int MODE, int N>
__global__ void __launch_bounds__(128, 1) probe_unrolled(int chunks, int* fail, long long* cycles) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) unsigned long long bar[2];
  unsigned char* base = sm + ((1024 - (smem_u32(sm) & 1023)) & 1023);
  for (uint32_t i = threadIdx.x; i < (kAbytes + kBbytes) / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(base)[i] = 0u;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar[0]), 1);
    mbar_init(smem_u32(&bar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tbase;
  constexpr uint32_t acol = 4u * (uint32_t)N;
  if (MODE == 3) {
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (uint32_t c = 0; c < 48; c += 8)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(
              tmem + lane_base + acol + c),
          "r"(0u)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (threadIdx.x == 0) {
    const uint32_t a0 = smem_u32(base), b0 = a0 + kAbytes;
    constexpr uint32_t idesc = instr_desc(128, N);
    uint64_t ad[6], bd[6];
    uint32_t at[6], dd[4];
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      if (MODE == 0 || MODE == 3) {
        ad[p] = smem_desc(a0 + (uint32_t)p * 4096, 2048, 128, 0);
        bd[p] = smem_desc(b0 + (uint32_t)p * (uint32_t)N * 32, (uint32_t)N * 16, 128, 0);
      } else {
        ad[p] = smem_desc(a0 + (uint32_t)(p >> 2) * 16384 + (uint32_t)(p & 3) * 32, 16, 1024, 2);
        bd[p] = smem_desc(b0 + (uint32_t)(p >> 2) * 32768 + (uint32_t)(p & 3) * 32, 16, 1024, 2);
      }
      at[p] = tmem + acol + (uint32_t)p * 8;
    }
    constexpr int slots = N <= 128 ? 4 : 2;
#pragma unroll
    for (int q = 0; q < 4; ++q) dd[q] = tmem + (uint32_t)((q % slots) * N);
    long long t0 = clock64();
    bool bad = false;
    int c = 0;
    for (; c < chunks && !bad; ++c) {
      const int st = c & 1;
      if (c >= 2 && !mbar_wait(smem_u32(&bar[st]), (uint32_t)(((c >> 1) - 1) & 1))) bad = true;
      if (bad) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      const uint32_t acc = c > 0 ? 1u : 0u;
#pragma unroll
      for (int i = 0; i < 21; ++i) {
        const int pa = i % 6, pb = (i / 6 + i) % 6;
        if (MODE == 3)
          mma_ts(dd[i % 4], at[pa], bd[pb], idesc, acc);
        else
          mma_ss(dd[i % 4], ad[pa], bd[pb], idesc, acc);
      }
      mma_commit(smem_u32(&bar[st]));
    }
    for (int g = c - 2; g < c; ++g)
      if (g >= 0 && !mbar_wait(smem_u32(&bar[g & 1]), (uint32_t)((g >> 1) & 1))) bad = true;
    cycles[blockIdx.x] = clock64() - t0;
    if (bad) atomicAdd(fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
  }
}

__global__ void __launch_bounds__(128, 1) probe_runtime(int mode, int chunks, int nmma, int N, int* fail,
                                                long long* cycles) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) unsigned long long bar[2];
  unsigned char* base = sm + ((1024 - (smem_u32(sm) & 1023)) & 1023);
  for (uint32_t i = threadIdx.x; i < (kAbytes + kBbytes) / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(base)[i] = 0u;
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tbase)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar[0]), 1);
    mbar_init(smem_u32(&bar[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tbase;
  // mode 3: zero the A columns of TMEM (after 4 N-column accumulators)
  const uint32_t acol = 4u * (uint32_t)N;
  if (mode == 3) {
    const int warp = threadIdx.x >> 5;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    for (uint32_t c = 0; c < 48; c += 8)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};\n" ::"r"(
              tmem + lane_base + acol + c),
          "r"(0u)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if (threadIdx.x == 0) {
    const uint32_t a0 = smem_u32(base), b0 = a0 + kAbytes;
    const uint32_t idesc = instr_desc(128, N);
    const int slots = N <= 128 ? 4 : 2;
    long long t0 = clock64();
    bool bad = false;
    int c = 0;
    for (; c < chunks && !bad; ++c) {
      const int st = c & 1;
      if (c >= 2 && !mbar_wait(smem_u32(&bar[st]), (uint32_t)(((c >> 1) - 1) & 1))) bad = true;
      if (bad) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      for (int i = 0; i < nmma; ++i) {
        const int pa = i % 6, pb = (i / 6 + i) % 6;
        const uint32_t d = tmem + (uint32_t)((i % slots) * N);
        const uint32_t acc = c > 0 ? 1u : 0u;
        if (mode == 0) {
          mma_ss(d, smem_desc(a0 + (uint32_t)pa * 4096, 2048, 128, 0),
                 smem_desc(b0 + (uint32_t)pb * (uint32_t)N * 32, (uint32_t)N * 16, 128, 0),
                 idesc, acc);
        } else if (mode == 1) {
          mma_ss(d, smem_desc(a0 + (uint32_t)pa * 4096, 16, 256, 6),
                 smem_desc(b0 + (uint32_t)pb * (uint32_t)N * 32, 16, 256, 6), idesc, acc);
        } else if (mode == 2) {
          // plane p: atom p / 4, K slice p % 4 (32-byte start advance)
          const uint32_t aa = a0 + (uint32_t)(pa >> 2) * 16384 + (uint32_t)(pa & 3) * 32;
          const uint32_t bb = b0 + (uint32_t)(pb >> 2) * 32768 + (uint32_t)(pb & 3) * 32;
          mma_ss(d, smem_desc(aa, 16, 1024, 2), smem_desc(bb, 16, 1024, 2), idesc, acc);
        } else {
          mma_ts(d, tmem + acol + (uint32_t)pa * 8,
                 smem_desc(b0 + (uint32_t)pb * (uint32_t)N * 32, (uint32_t)N * 16, 128, 0),
                 idesc, acc);
        }
      }
      mma_commit(smem_u32(&bar[st]));
    }
    for (int g = c - 2; g < c; ++g)
      if (g >= 0 && !mbar_wait(smem_u32(&bar[g & 1]), (uint32_t)((g >> 1) & 1))) bad = true;
    cycles[blockIdx.x] = clock64() - t0;
    if (bad) atomicAdd(fail, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512));
  }
}

template <int MODE, int N>
int run(int* fail, long long* cyc) {
  const int chunks = 400;
  cudaFuncSetAttribute(probe_unrolled<MODE, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kSmem);
  cudaMemset(fail, 0, sizeof(int));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  probe_unrolled<MODE, N><<<152, 128, kSmem>>>(chunks, fail, cyc);
  cudaEventRecord(e0);
  probe_unrolled<MODE, N><<<152, 128, kSmem>>>(chunks, fail, cyc);
  cudaEventRecord(e1);
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    printf("CUDA error %s (mode %d N %d)\n", cudaGetErrorString(err), MODE, N);
    return 1;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  long long h[152];
  int f = 0;
  cudaMemcpy(h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
  cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
  double avg = 0;
  for (int i = 0; i < 152; ++i) avg += (double)h[i] / 152;
  printf("unrolled layout %d N %3d: %.3f ms, %.1f cycles/MMA, failed waits %d\n", MODE, N, ms,
         avg / chunks / 21, f);
  return f != 0;
}

int run_runtime(int N, int* fail, long long* cyc) {
  const int chunks = 400, nmma = 21;
  cudaFuncSetAttribute(probe_runtime, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  cudaMemset(fail, 0, sizeof(int));
  probe_runtime<<<152, 128, kSmem>>>(0, chunks, nmma, N, fail, cyc);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0);
  probe_runtime<<<152, 128, kSmem>>>(0, chunks, nmma, N, fail, cyc);
  cudaEventRecord(e1);
  cudaError_t err = cudaDeviceSynchronize();
  if (err != cudaSuccess) {
    printf("CUDA error %s (runtime N %d)\n", cudaGetErrorString(err), N);
    return 1;
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  long long h[152];
  int f = 0;
  cudaMemcpy(h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
  cudaMemcpy(&f, fail, sizeof(int), cudaMemcpyDeviceToHost);
  double avg = 0;
  for (int i = 0; i < 152; ++i) avg += (double)h[i] / 152;
  printf("runtime  layout 0 N %3d: %.3f ms, %.1f cycles/MMA, failed waits %d\n", N, ms,
         avg / chunks / nmma, f);
  return f != 0;
}

int main() {
  int* fail;
  long long* cyc;
  cudaMalloc(&fail, sizeof(int));
  cudaMalloc(&cyc, 152 * sizeof(long long));
  int rc = 0;
  rc |= run<0, 16>(fail, cyc);
  rc |= run<0, 32>(fail, cyc);
  rc |= run<0, 48>(fail, cyc);
  rc |= run<0, 64>(fail, cyc);
  rc |= run<0, 80>(fail, cyc);
  rc |= run<0, 96>(fail, cyc);
  rc |= run<0, 112>(fail, cyc);
  rc |= run<0, 128>(fail, cyc);
  rc |= run<0, 144>(fail, cyc);
  rc |= run<0, 160>(fail, cyc);
  rc |= run<0, 192>(fail, cyc);
  rc |= run<0, 224>(fail, cyc);
  rc |= run<0, 256>(fail, cyc);
  rc |= run<2, 80>(fail, cyc);
  rc |= run<2, 128>(fail, cyc);
  rc |= run<2, 256>(fail, cyc);
  rc |= run<3, 80>(fail, cyc);
  rc |= run<3, 96>(fail, cyc);
  rc |= run_runtime(80, fail, cyc);
  rc |= run_runtime(128, fail, cyc);
  rc |= run_runtime(256, fail, cyc);
  return rc;
}
