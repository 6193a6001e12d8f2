// noalloc.cu -- tsne_kl_grad_noalloc: the exact KL gradient for callers that
// cannot allocate device memory.
//
// tsne_kl_grad needs a caller workspace (partial forces, per-item Z sums).
// Some callers cannot provide one: code embedded in a host application whose
// own allocator owns every device allocation and forbids others, or a loop
// that must not pay cudaMalloc's implicit device-wide synchronisation, and
// that cannot keep a workspace of its own alive between calls.  This entry
// point takes its scratch from a fixed array in the library's device memory
// instead, so it calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and behaviour:
//   * one sample of 2 <= n <= TSNE_NOALLOC_MAX_N points (65,536); larger n is
//     rejected with TSNE_ERR_CAPACITY before anything is enqueued;
//   * the scratch array (TSNE_NOALLOC_SCRATCH_BYTES = 6 MiB) exists on every
//     device that loads the library and stays allocated until the process
//     exits;
//   * every call shares that one array: calls whose work overlaps on the GPU
//     (different streams, or different host threads on one device) race and
//     give wrong results; order them on one stream;
//   * the array keeps the previous call's contents; every scratch value this
//     path reads is written earlier in the same call, so nothing needs
//     clearing;
//   * the first call on a device looks up the device address of the array on
//     that device (cudaGetSymbolAddress with the device current) and caches
//     it: make that first call before any stream capture begins.
// The result equals tsne_kl_grad's up to summation order (FP32 partial sums per
// tile, FP64 across tiles): the direct repulsion kernel runs with at most four
// column chunks.
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace tsne {
void rep_cfg_shape(int cfg, int* rows_per_item, int* tile_cols);
cudaError_t launch_repulse_direct(int cfg, const float2* Y, const SampleTable& tab, int64_t items,
                                  double2* Fpart, double* zpart, cudaStream_t st);
cudaError_t launch_attract(const tsne_csr& P, const float2* Y, float2* Fa, double2* klrow,
                           int iter_arg, const WsHeader* hdr, int kl_every, int force_kl,
                           int32_t* status, cudaStream_t st);
cudaError_t launch_reduce(const SampleTable& tab, const RepBufs& rb, const double2* klrow,
                          double* Zout, double* kl_out, float alpha, int iter_arg,
                          const WsHeader* hdr, int kl_every, int force_kl, int64_t kl_slots,
                          cudaStream_t st);
cudaError_t launch_grad(const SampleTable& tab, const RepBufs& rb, const float2* Fa,
                        const double* Z, float alpha, float2* grad, cudaStream_t st);
}  // namespace tsne

using namespace tsne;

namespace {

constexpr size_t kNoallocBytes = TSNE_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocCfg = 1;     // direct kernel, 128 threads x 4 rows, 256-column tiles
constexpr int kNoallocChunks = 4;  // column chunks per row tile

// The scratch.  In host code this name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSNE_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TSNE_ERR_DEVICE;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TSNE_ERR_CUDA;
    g_scratch[dev] = p;
  }
  *out = g_scratch[dev];
  return TSNE_OK;
}

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int tsne_kl_grad_noalloc(const tsne_csr* P, const float* Y, float alpha, float* grad,
                                    double* Z, double* kl, int32_t* dev_status,
                                    tsne_stream_t stream) {
  if (!P || !Y || !Z || !isfinite(alpha)) return TSNE_ERR_ARG;
  const int64_t n = P->n;
  if (n < 2 || P->cap < 0 || !P->row_ptr || (P->cap > 0 && (!P->col || !P->val)))
    return TSNE_ERR_ARG;
  if (n > TSNE_NOALLOC_MAX_N) return TSNE_ERR_CAPACITY;

  // one sample: direct kernel, row tiles of `rows`, up to kNoallocChunks chunks
  SampleTable tab;
  memset(&tab, 0, sizeof(tab));
  int rows = 0, tile = 0;
  rep_cfg_shape(kNoallocCfg, &rows, &tile);
  const int64_t ntiles = (n + tile - 1) / tile;
  const int64_t ch = ntiles < kNoallocChunks ? ntiles : kNoallocChunks;
  const int64_t rtiles = (n + rows - 1) / rows;
  tab.S = 1;
  tab.rows_per_item = rows;
  tab.tile_cols = tile;
  tab.blk_pts = 256;
  tab.max_chunks = (int)ch;
  tab.pt_off[1] = n;
  tab.fp_off[1] = ch * n;
  tab.item_off[1] = (int32_t)(rtiles * ch);
  tab.blk_off[1] = (int32_t)((n + 255) / 256);
  tab.chunks[0] = (int32_t)ch;

  // scratch layout: Fa | partial forces | per-item Z | per-row KL terms
  size_t off = 0;
  const size_t oFa = off;    off = up256(off + sizeof(float2) * (size_t)n);
  const size_t oFpart = off; off = up256(off + sizeof(double2) * (size_t)(ch * n));
  const size_t oZpart = off; off = up256(off + sizeof(double) * (size_t)(rtiles * ch));
  const size_t oKlrow = off; off = up256(off + sizeof(double2) * (size_t)n);
  if (off > kNoallocBytes) return TSNE_ERR_CAPACITY;

  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  char* b = static_cast<char*>(base);
  cudaStream_t st = (cudaStream_t)stream;
  const float2* Y2 = reinterpret_cast<const float2*>(Y);
  float2* Fa = reinterpret_cast<float2*>(b + oFa);
  double2* Fpart = reinterpret_cast<double2*>(b + oFpart);
  double* zpart = reinterpret_cast<double*>(b + oZpart);
  double2* klrow = kl ? reinterpret_cast<double2*>(b + oKlrow) : nullptr;
  // the header argument is never read when the KL value is requested explicitly
  const WsHeader* hdr = reinterpret_cast<const WsHeader*>(b);
  RepBufs rb;
  rb.Fpart = Fpart;
  rb.zpart = zpart;
  rb.Rbuf = nullptr;
  rb.Cbuf = nullptr;
  rb.Facc = nullptr;
  rb.zred_part = nullptr;  // single-stage reduction
  rb.zred_nb = 0;
  rb.zsym = nullptr;
  TSNE_CUDA_TRY(launch_attract(*P, Y2, Fa, klrow, 0, hdr, 0, kl ? 1 : 0, dev_status, st));
  TSNE_CUDA_TRY(launch_repulse_direct(kNoallocCfg, Y2, tab, rtiles * ch, Fpart, zpart, st));
  TSNE_CUDA_TRY(launch_reduce(tab, rb, klrow, Z, kl, alpha, 0, hdr, 0, kl ? 1 : 0, 1, st));
  if (grad) TSNE_CUDA_TRY(launch_grad(tab, rb, Fa, Z, alpha, reinterpret_cast<float2*>(grad), st));
  return TSNE_OK;
}
