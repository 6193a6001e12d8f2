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
//   * one sample of 2 <= n <= TSNE_NOALLOC_MAX_N points (65,536), the same
//     lower bound as tsne_kl_grad; a larger n is rejected with
//     TSNE_ERR_CAPACITY before anything is enqueued;
//   * the scratch array (TSNE_NOALLOC_SCRATCH_BYTES = 6 MiB) exists on every
//     device that loads the library and stays allocated until the process
//     exits;
//   * every call shares that one array: calls whose work overlaps on the GPU
//     (different streams, or different host threads on one device) race and
//     give wrong results; order them on one stream;
//   * the array keeps the previous call's contents; every scratch value this
//     path reads is written earlier in the same call, so nothing needs
//     clearing;
//   * the array's device address belongs to the CUDA context that loaded the
//     library's module.  The first call under a context looks that address up
//     (cudaGetSymbolAddress with the context current) and caches it under the
//     context's unique ID (cuCtxGetId, never reused in a process), so callers
//     that switch between their own driver-API contexts, or that reset the
//     device and so get a new primary context, get the address that is valid
//     where the kernels run.  Make each context's first call before any stream
//     capture begins on it.
// The result equals tsne_kl_grad's up to summation order (FP32 partial sums per
// tile, FP64 across tiles): the direct repulsion kernel runs with at most four
// column chunks.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace tsne {
void rep_cfg_shape(int cfg, int* rows_per_item, int* tile_cols);
cudaError_t launch_repulse_direct(int cfg, const float2* Y, const SampleTable& tab, int64_t items,
                                  float2* Fpart, double* zpart, cudaStream_t st);
cudaError_t launch_attract(const tsne_csr& P, const float2* Y, float2* Fa, double2* klrow,
                           int iter_arg, const WsHeader* hdr, int kl_every, int force_kl,
                           int32_t* status, cudaStream_t st);
cudaError_t launch_reduce(const SampleTable& tab, const RepBufs& rb, const double2* klrow,
                          double* Zout, double* kl_out, float alpha, int iter_arg,
                          const WsHeader* hdr, int kl_every, int force_kl, int64_t kl_slots,
                          cudaStream_t st, bool part_only = false);
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

// Addresses looked up so far, one per context (a process rarely has more
// than a few; the table is searched linearly and refilled round-robin).
constexpr int kMaxContexts = 64;
struct CtxAddr {
  unsigned long long ctx_id;  // cuCtxGetId; 0 = empty slot (IDs start at 1)
  void* addr;
};
std::mutex g_mu;
CtxAddr g_addr[kMaxContexts] = {};
int g_next = 0;

// cuCtxGetCurrent and cuCtxGetId through the runtime's driver entry point, so
// that the library needs no link-time dependency on the driver library.
struct CtxFns {
  PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  PFN_cuCtxGetId_v12000 get_id = nullptr;
};
const CtxFns& ctx_fns() {
  static CtxFns f = [] {
    CtxFns r;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      r.get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      r.get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
    cudaGetLastError();  // a failed lookup must not surface in a later call
    return r;
  }();
  return f;
}

// Unique ID of the current context (0 if none is current or the lookup fails).
unsigned long long current_ctx_id() {
  const CtxFns& f = ctx_fns();
  if (!f.get_current || !f.get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (f.get_current(&c) != CUDA_SUCCESS || !c) return 0;
  if (f.get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array in the current context.
int scratch_address(void** out) {
  unsigned long long id = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (id != 0)
    for (int k = 0; k < kMaxContexts; k++)
      if (g_addr[k].ctx_id == id) {
        *out = g_addr[k].addr;
        return TSNE_OK;
      }
  // first call under this context (or none current yet: the lookup makes the
  // device's primary context current)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();  // clear the error so no later call reports it as its own
    return TSNE_ERR_CUDA;
  }
  if (id == 0) id = current_ctx_id();
  if (id != 0) {
    g_addr[g_next] = CtxAddr{id, p};
    g_next = (g_next + 1) % kMaxContexts;
  }
  *out = p;
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

  // scratch layout: header | Fa | partial forces | per-item Z | per-row KL terms
  size_t off = 0;
  const size_t oHdr = off;   off = up256(off + sizeof(WsHeader));
  const size_t oFa = off;    off = up256(off + sizeof(float2) * (size_t)n);
  const size_t oFpart = off; off = up256(off + sizeof(float2) * (size_t)(ch * n));
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
  float2* Fpart = reinterpret_cast<float2*>(b + oFpart);
  double* zpart = reinterpret_cast<double*>(b + oZpart);
  double2* klrow = kl ? reinterpret_cast<double2*>(b + oKlrow) : nullptr;
  // a header of its own: the kernels read its iteration counter only when the
  // KL value is due by schedule, which never happens here (it is requested
  // explicitly or not at all), but no other region is aliased to it
  const WsHeader* hdr = reinterpret_cast<const WsHeader*>(b + oHdr);
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
