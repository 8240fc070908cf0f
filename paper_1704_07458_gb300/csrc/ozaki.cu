// FP64-accurate tensor-core contractions by exact BF16 splitting (Ozaki scheme).
#include "kernels.cuh"

namespace lob {

int64_t gram_ozaki_workspace(int64_t, int, int, int) { return 16; }
int gram_ozaki(cudaStream_t, int64_t, const SegList&, const SegList&, double*, int64_t, int,
               void*, int64_t) {
  return LOBPCG_ERR_ARG;
}
int64_t update_ozaki_workspace(int64_t, int, int, int) { return 0; }
int update_ozaki(cudaStream_t, int64_t, const SegList&, const double*, int64_t, int, double,
                 double, const SegList&, const OutList&, int, void*, int64_t) {
  return LOBPCG_ERR_ARG;
}

}  // namespace lob
