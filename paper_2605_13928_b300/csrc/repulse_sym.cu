// repulse_sym.cu -- launcher of the symmetric (unordered-pair) repulsion kernel;
// the work of one group pair is in repulse_sym_item.cuh.
#include "repulse_sym_item.cuh"

namespace tsne {

int sym_group_size(int W) { return W * 256; }

cudaError_t launch_repulse_sym(int W, const float2* Y, const SampleTable& tab, int64_t items,
                               float2* Rbuf, float2* Cbuf, double* zpart, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  switch (W) {
    case 8:
      repulse_sym_kernel<8><<<(unsigned)items, 256, 0, st>>>(Y, tab, Rbuf, Cbuf, zpart);
      break;
    case 4:
      repulse_sym_kernel<4><<<(unsigned)items, 128, 0, st>>>(Y, tab, Rbuf, Cbuf, zpart);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsne
