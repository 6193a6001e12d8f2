// api.cu -- the C ABI of libtsne.so (declared in include/tsne.h): argument
// checks, work planning, workspace layout and kernel launches.  Every step of
// the computation runs in the kernels of this library.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <memory>
#include <vector>

#include "common.cuh"

namespace tsne {
// repulse.cu
int rep_cfg_count();
void rep_cfg_shape(int cfg, int* rows_per_item, int* tile_cols);
cudaError_t launch_repulse_direct(int cfg, const float2* Y, const SampleTable& tab, int64_t items,
                                  double2* Fpart, double* zpart, cudaStream_t st);
// gradient.cu
cudaError_t launch_attract(const tsne_csr& P, const float2* Y, float2* Fa, double2* klrow,
                           int iter_arg, const WsHeader* hdr, int kl_every, int force_kl,
                           int32_t* status, cudaStream_t st);
cudaError_t launch_reduce(const SampleTable& tab, const double* zpart, const double2* klrow,
                          double* Zout, double* kl_out, float alpha, int iter_arg,
                          const WsHeader* hdr, int kl_every, int force_kl, cudaStream_t st);
cudaError_t launch_grad(const SampleTable& tab, const double2* Fpart, const float2* Fa,
                        const double* Z, float alpha, float2* grad, cudaStream_t st);
cudaError_t launch_update(const SampleTable& tab, const double2* Fpart, const float2* Fa,
                          const double* Z, const Schedule& q, int iter_arg, WsHeader* hdr,
                          float2* Y, float2* U, float2* G, int32_t* status, cudaStream_t st);
cudaError_t launch_set_iter(WsHeader* hdr, int iter, cudaStream_t st);
// plain.cu
cudaError_t launch_plain(const tsne_csr& P, const SampleTable& tab, const float2* Y, float alpha,
                         float2* grad, double* Z, float2* Fa, float2* Fr, float* Zi,
                         int64_t* seg, int32_t* sid, int32_t* status, cudaStream_t st);
}  // namespace tsne

using namespace tsne;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return 148;
  return sms;
}

// Carves consecutive 256-byte aligned regions out of a workspace.
struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  }
};

// Fills pt_off / S of a table from the batch; checks the offsets.
int table_from_batch(int64_t n, const tsne_batch* B, int64_t min_ns, SampleTable* tab) {
  memset(tab, 0, sizeof(*tab));
  if (n < 0) return TSNE_ERR_ARG;
  if (!B) {
    tab->S = 1;
    tab->pt_off[0] = 0;
    tab->pt_off[1] = n;
  } else {
    if (B->n_samples < 1 || B->n_samples > kMaxS || !B->pt_off) return TSNE_ERR_ARG;
    tab->S = B->n_samples;
    if (B->pt_off[0] != 0 || B->pt_off[B->n_samples] != n) return TSNE_ERR_ARG;
    for (int s = 0; s <= B->n_samples; s++) tab->pt_off[s] = B->pt_off[s];
  }
  for (int s = 0; s < tab->S; s++)
    if (tab->pt_off[s + 1] - tab->pt_off[s] < min_ns) return TSNE_ERR_ARG;
  return TSNE_OK;
}

// Point-wise blocks: 256 points per block, never straddling a sample.
void fill_blocks(SampleTable* tab) {
  tab->blk_pts = 256;
  int32_t b = 0;
  for (int s = 0; s < tab->S; s++) {
    tab->blk_off[s] = b;
    const int64_t ns = tab->pt_off[s + 1] - tab->pt_off[s];
    b += (int32_t)((ns + tab->blk_pts - 1) / tab->blk_pts);
  }
  tab->blk_off[tab->S] = b;
}

struct GradPlan {
  SampleTable tab;
  int cfg;
  int64_t n;
  int64_t items;
  int64_t fpart_elems;
  size_t off_hdr, off_Fa, off_Fpart, off_zpart, off_klrow, off_Z, off_kl, total;
};

int choose_cfg(const SampleTable& tab, int variant) {
  if (variant == TSNE_VARIANT_DIRECT_L) return 0;
  if (variant == TSNE_VARIANT_DIRECT_S) return 1;
  double pairs = 0.0;
  int64_t nmax = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    pairs += (double)ns * (double)ns;
    if (ns > nmax) nmax = ns;
  }
  return (nmax >= 32768 && pairs >= 4e9) ? 0 : 1;
}

// Work split of the repulsion.  Items of one sample cost rows_per_item x chunk
// width pair evaluations; the chunk width is chosen so the whole call has about
// 32 items per resident CTA slot (load balance over 148 SMs), never narrower
// than one shared-memory tile, with at most 64 chunks per sample.
int make_grad_plan(int64_t n, const tsne_batch* B, const tsne_params* prm, GradPlan* pl) {
  int rc = table_from_batch(n, B, 2, &pl->tab);
  if (rc) return rc;
  SampleTable& tab = pl->tab;
  fill_blocks(&tab);
  pl->n = n;
  pl->cfg = choose_cfg(tab, prm ? prm->variant : TSNE_VARIANT_AUTO);
  int rows = 0, tile = 0;
  rep_cfg_shape(pl->cfg, &rows, &tile);
  tab.rows_per_item = rows;
  tab.tile_cols = tile;
  double pairs = 0.0;
  for (int s = 0; s < tab.S; s++) {
    const double ns = (double)(tab.pt_off[s + 1] - tab.pt_off[s]);
    pairs += ns * ns;
  }
  const double slots = 2.0 * device_sm_count();
  const double width = fmax((double)tile, pairs / ((double)rows * 32.0 * slots));
  int64_t items = 0, fp = 0;
  int maxc = 1;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    const int64_t ntiles = (ns + tile - 1) / tile;
    int64_t ch = (int64_t)ceil((double)ns / width);
    if (ch < 1) ch = 1;
    if (ch > ntiles) ch = ntiles;
    if (ch > 64) ch = 64;
    const int64_t rt = (ns + rows - 1) / rows;
    tab.item_off[s] = (int32_t)items;
    tab.chunks[s] = (int32_t)ch;
    tab.fp_off[s] = fp;
    items += rt * ch;
    fp += ch * ns;
    if (ch > maxc) maxc = (int)ch;
    if (items > 0x7fffffffLL) return TSNE_ERR_ARG;
  }
  tab.item_off[tab.S] = (int32_t)items;
  tab.fp_off[tab.S] = fp;
  tab.max_chunks = maxc;
  pl->items = items;
  pl->fpart_elems = fp;
  Carver c;
  pl->off_hdr = c.take(sizeof(WsHeader));
  pl->off_Fa = c.take(sizeof(float2) * (size_t)n);
  pl->off_Fpart = c.take(sizeof(double2) * (size_t)fp);
  pl->off_zpart = c.take(sizeof(double) * (size_t)items);
  pl->off_klrow = c.take(sizeof(double2) * (size_t)n);
  pl->off_Z = c.take(sizeof(double) * (size_t)tab.S);
  pl->off_kl = c.take(sizeof(double) * (size_t)tab.S);
  pl->total = c.off;
  return TSNE_OK;
}

int check_ws(const void* ws, size_t ws_bytes, size_t need) {
  if (need == 0) return TSNE_OK;
  if (!ws || ((uintptr_t)ws & (kAlign - 1)) || ws_bytes < need) return TSNE_ERR_WORKSPACE;
  return TSNE_OK;
}

int check_csr(const tsne_csr* P, int64_t* n_out) {
  if (!P || P->n < 0 || P->cap < 0) return TSNE_ERR_ARG;
  if (P->n > 0 && (!P->row_ptr || (P->cap > 0 && (!P->col || !P->val)))) return TSNE_ERR_ARG;
  if (P->n >= 0x7fffffffLL) return TSNE_ERR_ARG;  // column indices are int32
  *n_out = P->n;
  return TSNE_OK;
}

Schedule schedule_from(const tsne_params* p) {
  Schedule q;
  q.n_iter = p->n_iter;
  q.ee_iters = p->ee_iters;
  q.mom_switch = p->mom_switch;
  q.kl_every = p->kl_every;
  q.ee = p->ee;
  q.mom0 = p->mom0;
  q.mom1 = p->mom1;
  q.lr = p->lr;
  q.min_gain = p->min_gain;
  return q;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

}  // namespace

extern "C" {

void tsne_params_default(tsne_params* p) {
  if (!p) return;
  p->perplexity = 30.0f;
  p->k = 90;
  p->knn_mode = TSNE_KNN_FP32;
  p->cand_mult = 2.0f;
  p->calib_tol = 1e-5f;
  p->calib_max_iter = 200;
  p->n_iter = 750;
  p->ee_iters = 250;
  p->ee = 12.0f;
  p->mom_switch = 250;
  p->mom0 = 0.5f;
  p->mom1 = 0.8f;
  p->lr = 0.0f;
  p->min_gain = 0.01f;
  p->kl_every = 50;
  p->variant = TSNE_VARIANT_AUTO;
  p->use_graph = 1;
}

const char* tsne_strerror(int code) {
  switch (code) {
    case TSNE_OK: return "ok";
    case TSNE_ERR_ARG: return "invalid argument";
    case TSNE_ERR_CAPACITY: return "output capacity too small";
    case TSNE_ERR_CUDA: return "CUDA runtime error";
    case TSNE_ERR_TIMEOUT: return "bounded device wait timed out";
    case TSNE_ERR_NOT_CONVERGED: return "perplexity calibration missed some rows";
    case TSNE_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case TSNE_ERR_DEVICE: return "unsupported device";
    case TSNE_ERR_DEVICE_STATUS: return "a kernel reported an error in the status word";
    default: return "unknown error";
  }
}

const char* tsne_version(void) { return "libtsne 0.1 (sm_103a)"; }

size_t tsne_workspace_size(int op, int64_t n, int d, int k, const tsne_batch* B,
                           const tsne_params* prm) {
  (void)d;
  (void)k;
  tsne_params def;
  if (!prm) {
    tsne_params_default(&def);
    prm = &def;
  }
  switch (op) {
    case TSNE_OP_KL_GRAD: {
      std::unique_ptr<GradPlan> pl(new GradPlan);
      if (make_grad_plan(n, B, prm, pl.get())) return 0;
      return pl->total;
    }
    case TSNE_OP_PLAIN: {
      Carver c;
      c.take(sizeof(float2) * (size_t)n);   // Fa
      c.take(sizeof(float2) * (size_t)n);   // Fr
      c.take(sizeof(float) * (size_t)n);    // Z_i
      c.take(sizeof(int64_t) * 2 * (size_t)n);  // segments
      c.take(sizeof(int32_t) * (size_t)n);  // sample ids
      return c.off;
    }
    default:
      return 0;
  }
}

int tsne_kl_grad(const tsne_csr* P, const tsne_batch* B, const float* Y, float alpha, float* grad,
                 double* Z, double* kl, const tsne_params* prm, void* ws, size_t ws_bytes,
                 int32_t* dev_status, tsne_stream_t stream) {
  int64_t n = 0;
  int rc = check_csr(P, &n);
  if (rc) return rc;
  if (!Y || !Z || !isfinite(alpha)) return TSNE_ERR_ARG;
  tsne_params def;
  if (!prm) {
    tsne_params_default(&def);
    prm = &def;
  }
  std::unique_ptr<GradPlan> pl(new GradPlan);
  rc = make_grad_plan(n, B, prm, pl.get());
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, pl->total);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* Y2 = reinterpret_cast<const float2*>(Y);
  WsHeader* hdr = at<WsHeader>(ws, pl->off_hdr);
  float2* Fa = at<float2>(ws, pl->off_Fa);
  double2* Fpart = at<double2>(ws, pl->off_Fpart);
  double* zpart = at<double>(ws, pl->off_zpart);
  double2* klrow = kl ? at<double2>(ws, pl->off_klrow) : nullptr;
  TSNE_CUDA_TRY(launch_attract(*P, Y2, Fa, klrow, 0, hdr, 0, kl ? 1 : 0, dev_status, st));
  TSNE_CUDA_TRY(launch_repulse_direct(pl->cfg, Y2, pl->tab, pl->items, Fpart, zpart, st));
  TSNE_CUDA_TRY(launch_reduce(pl->tab, zpart, klrow, Z, kl, alpha, 0, hdr, 0, kl ? 1 : 0, st));
  if (grad)
    TSNE_CUDA_TRY(launch_grad(pl->tab, Fpart, Fa, Z, alpha, reinterpret_cast<float2*>(grad), st));
  return TSNE_OK;
}

int tsne_kl_grad_plain(const tsne_csr* P, const tsne_batch* B, const float* Y, float alpha,
                       float* grad, double* Z, void* ws, size_t ws_bytes, int32_t* dev_status,
                       tsne_stream_t stream) {
  int64_t n = 0;
  int rc = check_csr(P, &n);
  if (rc) return rc;
  if (!Y || !Z) return TSNE_ERR_ARG;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  rc = table_from_batch(n, B, 2, tab.get());
  if (rc) return rc;
  Carver c;
  const size_t oFa = c.take(sizeof(float2) * (size_t)n);
  const size_t oFr = c.take(sizeof(float2) * (size_t)n);
  const size_t oZi = c.take(sizeof(float) * (size_t)n);
  const size_t oSeg = c.take(sizeof(int64_t) * 2 * (size_t)n);
  const size_t oSid = c.take(sizeof(int32_t) * (size_t)n);
  rc = check_ws(ws, ws_bytes, c.off);
  if (rc) return rc;
  if (n == 0) return TSNE_OK;
  TSNE_CUDA_TRY(launch_plain(*P, *tab, reinterpret_cast<const float2*>(Y), alpha,
                             reinterpret_cast<float2*>(grad), Z, at<float2>(ws, oFa),
                             at<float2>(ws, oFr), at<float>(ws, oZi), at<int64_t>(ws, oSeg),
                             at<int32_t>(ws, oSid), dev_status, (cudaStream_t)stream));
  return TSNE_OK;
}

int tsne_step(const tsne_csr* P, const tsne_batch* B, float* Y, float* uY, float* gains, int iter,
              const tsne_params* prm, double* Z, double* kl, void* ws, size_t ws_bytes,
              int32_t* dev_status, tsne_stream_t stream) {
  int64_t n = 0;
  int rc = check_csr(P, &n);
  if (rc) return rc;
  if (!Y || !uY || !gains || !prm || iter < -1) return TSNE_ERR_ARG;
  if (prm->kl_every < 0 || !(prm->min_gain >= 0.f)) return TSNE_ERR_ARG;
  std::unique_ptr<GradPlan> pl(new GradPlan);
  rc = make_grad_plan(n, B, prm, pl.get());
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, pl->total);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const Schedule q = schedule_from(prm);
  const float2* Y2 = reinterpret_cast<const float2*>(Y);
  WsHeader* hdr = at<WsHeader>(ws, pl->off_hdr);
  float2* Fa = at<float2>(ws, pl->off_Fa);
  double2* Fpart = at<double2>(ws, pl->off_Fpart);
  double* zpart = at<double>(ws, pl->off_zpart);
  const bool track_kl = kl && prm->kl_every > 0;
  double2* klrow = track_kl ? at<double2>(ws, pl->off_klrow) : nullptr;
  double* Zuse = Z ? Z : at<double>(ws, pl->off_Z);
  TSNE_CUDA_TRY(launch_attract(*P, Y2, Fa, klrow, iter, hdr, prm->kl_every, 0, dev_status, st));
  TSNE_CUDA_TRY(launch_repulse_direct(pl->cfg, Y2, pl->tab, pl->items, Fpart, zpart, st));
  TSNE_CUDA_TRY(launch_reduce(pl->tab, zpart, klrow, Zuse, track_kl ? kl : nullptr, 1.0f, iter,
                              hdr, prm->kl_every, 0, st));
  TSNE_CUDA_TRY(launch_update(pl->tab, Fpart, Fa, Zuse, q, iter, hdr, reinterpret_cast<float2*>(Y),
                              reinterpret_cast<float2*>(uY), reinterpret_cast<float2*>(gains),
                              dev_status, st));
  return TSNE_OK;
}

int tsne_step_reset(void* ws, size_t ws_bytes, int iter, tsne_stream_t stream) {
  if (!ws || ((uintptr_t)ws & (kAlign - 1)) || ws_bytes < sizeof(WsHeader) || iter < 0)
    return TSNE_ERR_WORKSPACE;
  TSNE_CUDA_TRY(launch_set_iter(reinterpret_cast<WsHeader*>(ws), iter, (cudaStream_t)stream));
  return TSNE_OK;
}

}  // extern "C"
