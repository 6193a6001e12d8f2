// repulse.cu -- exact O(n^2) repulsion of t-SNE (van der Maaten & Hinton 2008,
// Eq. 5, the q-term of the gradient):
//
//   Fr_i = sum_{j != i} w_ij^2 (y_i - y_j),   Z = sum_{i != j} w_ij,
//   w_ij = 1 / (1 + |y_i - y_j|^2)
//
// The per-item work lives in repulse_item.cuh; this file holds the one-item-
// per-CTA kernel and its launch configurations.
#include "attract.cuh"
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

// Small problems (cfg 3 and 4): the attraction rows and the direct repulsion
// items in one launch, since at these sizes a launch costs more than its work.
// Blocks [0, att_blocks) take 2 x THREADS / 32 attraction rows each (the rows
// of the attraction kernel's blocks, in the same order and arithmetic), the
// others one repulsion item each.
template <int THREADS, int R, int TILE>
__global__ void __launch_bounds__(THREADS, 2)
forces_direct_kernel(const tsne_csr P, int64_t att_blocks, const float2* __restrict__ Y,
                     const __grid_constant__ SampleTable tab, float2* __restrict__ Fpart,
                     double* __restrict__ zpart, float2* __restrict__ Fa,
                     double2* __restrict__ klrow, int iter_arg, const WsHeader* hdr,
                     int kl_every, int force_kl, int32_t* status) {
  __shared__ float4 tile[TILE];
  __shared__ double zred[THREADS / 32];
  if ((int64_t)blockIdx.x < att_blocks) {  // the whole block
    attract_rows(blockIdx.x, THREADS / 32, P.row_ptr, P.col, P.val, P.n, P.cap, Y, Fa, klrow,
                 iter_arg, hdr, kl_every, force_kl, status);
    return;
  }
  direct_item<THREADS, R, TILE>(Y, tab, (int)((int64_t)blockIdx.x - att_blocks), Fpart, zpart,
                                tile, zred);
}

// Both force terms of a direct plan in one launch; cudaErrorNotSupported for
// the configurations that keep two launches.
cudaError_t launch_forces_direct(int cfg, const tsne_csr& P, const float2* Y,
                                 const SampleTable& tab, int64_t items, float2* Fpart,
                                 double* zpart, float2* Fa, double2* klrow, int iter_arg,
                                 const WsHeader* hdr, int kl_every, int force_kl,
                                 int32_t* status, cudaStream_t st) {
  if (cfg != 3 && cfg != 4) return cudaErrorNotSupported;
  const int64_t rows_per_block = 2 * (128 / 32);
  const int64_t att = P.n > 0 ? (P.n + rows_per_block - 1) / rows_per_block : 0;
  const int64_t grid = att + (items > 0 ? items : 0);
  if (grid <= 0) return cudaSuccess;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (cfg == 3)
    forces_direct_kernel<128, 2, 256><<<(unsigned)grid, 128, 0, st>>>(
        P, att, Y, tab, Fpart, zpart, Fa, klrow, iter_arg, hdr, kl_every, force_kl, status);
  else
    forces_direct_kernel<128, 2, 128><<<(unsigned)grid, 128, 0, st>>>(
        P, att, Y, tab, Fpart, zpart, Fa, klrow, iter_arg, hdr, kl_every, force_kl, status);
  return cudaGetLastError();
}

}  // namespace tsne
