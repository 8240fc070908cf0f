// Shared definitions of the GB300 LOBPCG library (device and host side).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/lobpcg.h"

#define LOBPCG_EXPORT extern "C" __attribute__((visibility("default")))

namespace lob {

constexpr int kMaxSeg = 4;

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }

// A row-major block presented as up to kMaxSeg column segments, each with its
// own base pointer and leading dimension: S = [X, P, W] without copies.
struct SegList {
  const double* ptr[kMaxSeg];
  int64_t ld[kMaxSeg];
  int off[kMaxSeg + 1];  // prefix sums of segment widths; off[nseg] = total columns
  int nseg;
};

inline SegList seg1(const double* p, int64_t ld, int cols) {
  SegList s{};
  s.ptr[0] = p; s.ld[0] = ld; s.off[0] = 0; s.off[1] = cols; s.nseg = 1;
  for (int i = 2; i <= kMaxSeg; ++i) s.off[i] = cols;
  return s;
}

inline void seg_push(SegList& s, const double* p, int64_t ld, int cols) {
  if (cols <= 0) return;
  s.ptr[s.nseg] = p; s.ld[s.nseg] = ld;
  s.off[s.nseg + 1] = s.off[s.nseg] + cols;
  s.nseg++;
  for (int i = s.nseg + 1; i <= kMaxSeg; ++i) s.off[i] = s.off[s.nseg];
}

inline SegList seg_empty() {
  SegList s{};
  s.nseg = 0;
  return s;
}

__device__ __forceinline__ double seg_load(const SegList& s, int c, int64_t row) {
  int i = 0;
#pragma unroll
  for (int t = 1; t < kMaxSeg; ++t) i += (t < s.nseg && c >= s.off[t]) ? 1 : 0;
  return s.ptr[i][row * s.ld[i] + (c - s.off[i])];
}

// Output block split into up to two destinations by column (e.g. [X_new, P_new]).
struct OutList {
  double* ptr[2];
  int64_t ld[2];
  int split;  // columns < split go to ptr[0], the rest to ptr[1]
};

__device__ __forceinline__ double* out_addr(const OutList& o, int c, int64_t row) {
  return c < o.split ? o.ptr[0] + row * o.ld[0] + c : o.ptr[1] + row * o.ld[1] + (c - o.split);
}

// Kernel launch counter (host side, per process) used for the stats.
extern int64_t g_launches;

}  // namespace lob

#define LOB_CUDA_OK(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return LOBPCG_ERR_CUDA;         \
  } while (0)

#define LOB_LAUNCHED()                                     \
  do {                                                     \
    ++lob::g_launches;                                     \
    if (cudaPeekAtLastError() != cudaSuccess) return LOBPCG_ERR_CUDA; \
  } while (0)
