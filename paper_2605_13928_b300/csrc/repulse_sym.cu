// repulse_sym.cu -- launcher of the symmetric (unordered-pair) repulsion kernel;
// the work of one group pair is in repulse_sym_item.cuh.
#include "repulse_sym_item.cuh"

namespace tsne {

int sym_group_size(int W) { return W * 256; }

// Tiles of the tiled fixed-point form per sample of G groups.
int64_t sym_tile_count(int64_t G) { return tile_count(G); }


// Tiled fixed-point launch (1024-point groups): one CTA per tile, then one per
// diagonal group (diag_items of them; 0 leaves the diagonal groups to the
// direct kernel).
cudaError_t launch_repulse_sym_tiled(const float2* Y, const SampleTable& tab, int64_t diag_items,
                                     double* zpart, unsigned long long* Facc, float2* Fpart,
                                     double* zdiag, int32_t* status, cudaStream_t st) {
  const int64_t blocks = tab.tile_off[tab.S] + diag_items;
  if (blocks <= 0) return cudaSuccess;
  constexpr size_t smem = sizeof(float) * sym_tile_smem_floats<4>();
  // set on every call: the attribute belongs to the current device's context
  cudaError_t e = cudaFuncSetAttribute(repulse_sym_tiled_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  repulse_sym_tiled_kernel<4><<<(unsigned)blocks, 128, smem, st>>>(Y, tab, zpart, Facc, status,
                                                                   Fpart, zdiag);
  return cudaGetLastError();
}

// Partial-buffer form: one group pair per CTA, then one CTA per diagonal group
// (diag_items of them, or 0).
cudaError_t launch_repulse_sym(int W, const float2* Y, const SampleTable& tab, int64_t items,
                               int64_t diag_items, float2* Rbuf, float2* Cbuf, double* zpart,
                               float2* Fpart, double* zdiag, cudaStream_t st) {
  const int64_t blocks = items + diag_items;
  if (blocks <= 0) return cudaSuccess;
  switch (W) {
    case 8:
      repulse_sym_kernel<8, false><<<(unsigned)blocks, 256, 0, st>>>(
          Y, tab, Rbuf, Cbuf, zpart, nullptr, nullptr, Fpart, zdiag);
      break;
    case 4:
      repulse_sym_kernel<4, false><<<(unsigned)blocks, 128, 0, st>>>(
          Y, tab, Rbuf, Cbuf, zpart, nullptr, nullptr, Fpart, zdiag);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsne
