// repulse_sym.cu -- launcher of the symmetric (unordered-pair) repulsion kernel;
// the work of one group pair is in repulse_sym_item.cuh.
#include "repulse_sym_item.cuh"

namespace tsne {

int sym_group_size(int W) { return W * 256; }

// Tiles of the tiled fixed-point form per sample of G groups.
int64_t sym_tile_count(int64_t G) { return tile_count(G); }


// Tiled fixed-point launch (1024-point groups): one CTA per tile.
cudaError_t launch_repulse_sym_tiled(const float2* Y, const SampleTable& tab, double* zpart,
                                     unsigned long long* Facc, int32_t* status,
                                     cudaStream_t st) {
  const int64_t blocks = tab.tile_off[tab.S];
  if (blocks <= 0) return cudaSuccess;
  constexpr size_t smem = sizeof(float) * sym_tile_smem_floats<4>();
  // set on every call: the attribute belongs to the current device's context
  cudaError_t e = cudaFuncSetAttribute(repulse_sym_tiled_kernel<4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  repulse_sym_tiled_kernel<4><<<(unsigned)blocks, 128, smem, st>>>(Y, tab, zpart, Facc, status);
  return cudaGetLastError();
}

// Partial-buffer form: one group pair per CTA.
cudaError_t launch_repulse_sym(int W, const float2* Y, const SampleTable& tab, int64_t items,
                               float2* Rbuf, float2* Cbuf, double* zpart, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  switch (W) {
    case 8:
      repulse_sym_kernel<8, false><<<(unsigned)items, 256, 0, st>>>(Y, tab, Rbuf, Cbuf, zpart,
                                                                     nullptr, nullptr);
      break;
    case 4:
      repulse_sym_kernel<4, false><<<(unsigned)items, 128, 0, st>>>(Y, tab, Rbuf, Cbuf, zpart,
                                                                     nullptr, nullptr);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsne
