// repulse_sym.cu -- launcher of the symmetric (unordered-pair) repulsion kernel;
// the work of one group pair is in repulse_sym_item.cuh.
#include "repulse_sym_item.cuh"

namespace tsne {

int sym_group_size(int W) { return W * 256; }

// fx: fixed-point accumulation into Facc (1024-point groups only) instead of
// the Rbuf / Cbuf partial buffers.
cudaError_t launch_repulse_sym(int W, bool fx, const float2* Y, const SampleTable& tab,
                               int64_t items, float2* Rbuf, float2* Cbuf, double* zpart,
                               unsigned long long* Facc, int32_t* status, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  if (fx) {
    if (W != 4) return cudaErrorInvalidValue;
    repulse_sym_kernel<4, true><<<(unsigned)items, 128, 0, st>>>(Y, tab, Rbuf, Cbuf, zpart,
                                                                  Facc, status);
    return cudaGetLastError();
  }
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
