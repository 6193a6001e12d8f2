// repulse.cu -- exact O(n^2) repulsion of t-SNE (van der Maaten & Hinton 2008,
// Eq. 5, the q-term of the gradient):
//
//   Fr_i = sum_{j != i} w_ij^2 (y_i - y_j),   Z = sum_{i != j} w_ij,
//   w_ij = 1 / (1 + |y_i - y_j|^2)
//
// The per-item work lives in repulse_item.cuh; this file holds the one-item-
// per-CTA kernel and its launch configurations.
#include "repulse_item.cuh"

namespace tsne {

// Launch configurations.  cfg 0: large problems; cfg 1: mid-sized problems (and the
// fused kernel's direct items); cfg 2: 512-row items; cfg 3: 256-row items with
// 256-column tiles (problems of 4e7 to 4e8 pairs); cfg 4: 256-row items with
// 128-column tiles (problems below 4e7 pairs, e.g. one sample of up to ~6,000
// points: enough items to reach most SMs).
struct RepCfg {
  int threads, R, tile;
};
static const RepCfg kRepCfgs[] = {
    {256, 8, 1024}, {128, 4, 256}, {256, 4, 512}, {128, 2, 256}, {128, 2, 128}};

int rep_cfg_count() { return (int)(sizeof(kRepCfgs) / sizeof(kRepCfgs[0])); }
void rep_cfg_shape(int cfg, int* rows_per_item, int* tile_cols) {
  *rows_per_item = kRepCfgs[cfg].threads * kRepCfgs[cfg].R;
  *tile_cols = kRepCfgs[cfg].tile;
}

cudaError_t launch_repulse_direct(int cfg, const float2* Y, const SampleTable& tab, int64_t items,
                                  float2* Fpart, double* zpart, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  switch (cfg) {
    case 0:
      repulse_direct_kernel<256, 8, 1024><<<(unsigned)items, 256, 0, st>>>(Y, tab, Fpart, zpart);
      break;
    case 1:
      repulse_direct_kernel<128, 4, 256><<<(unsigned)items, 128, 0, st>>>(Y, tab, Fpart, zpart);
      break;
    case 2:
      repulse_direct_kernel<256, 4, 512><<<(unsigned)items, 256, 0, st>>>(Y, tab, Fpart, zpart);
      break;
    case 3:
      repulse_direct_kernel<128, 2, 256><<<(unsigned)items, 128, 0, st>>>(Y, tab, Fpart, zpart);
      break;
    case 4:
      repulse_direct_kernel<128, 2, 128><<<(unsigned)items, 128, 0, st>>>(Y, tab, Fpart, zpart);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsne
