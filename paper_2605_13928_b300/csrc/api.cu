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
                                  float2* Fpart, double* zpart, cudaStream_t st);
cudaError_t launch_forces_direct(int cfg, const tsne_csr& P, const float2* Y,
                                 const SampleTable& tab, int64_t items, float2* Fpart,
                                 double* zpart, float2* Fa, double2* klrow, int iter_arg,
                                 const WsHeader* hdr, int kl_every, int force_kl,
                                 int32_t* status, cudaStream_t st);
// repulse_sym.cu
int sym_group_size(int W);
cudaError_t launch_repulse_sym(int W, const float2* Y, const SampleTable& tab, int64_t items,
                               int64_t diag_items, float2* Rbuf, float2* Cbuf, double* zpart,
                               float2* Fpart, double* zdiag, cudaStream_t st);
int64_t sym_tile_count(int64_t G);
cudaError_t launch_repulse_sym_tiled(const float2* Y, const SampleTable& tab, int64_t diag_items,
                                     double* zpart, unsigned long long* Facc, float2* Fpart,
                                     double* zdiag, int32_t* status, cudaStream_t st);
// gradient.cu
cudaError_t launch_attract(const tsne_csr& P, const float2* Y, float2* Fa, double2* klrow,
                           int iter_arg, const WsHeader* hdr, int kl_every, int force_kl,
                           int32_t* status, cudaStream_t st);
cudaError_t launch_reduce(const SampleTable& tab, const RepBufs& rb, const double2* klrow,
                          double* Zout, double* kl_out, float alpha, int iter_arg,
                          const WsHeader* hdr, int kl_every, int force_kl, int64_t kl_slots,
                          cudaStream_t st, bool part_only = false);
cudaError_t launch_grad(const SampleTable& tab, const RepBufs& rb, const float2* Fa,
                        const double* Z, float alpha, float2* grad, cudaStream_t st);
cudaError_t launch_update(const SampleTable& tab, const RepBufs& rb, const float2* Fa,
                          const double* Z, const Schedule& q, int iter_arg, WsHeader* hdr,
                          float2* Y, float2* U, float2* G, int32_t* status, double* Zout,
                          double* kl_out, int kl_every, int64_t kl_slots,
                          const double2* klrow, bool self_reduce, cudaStream_t st);
cudaError_t launch_set_iter(WsHeader* hdr, int iter, cudaStream_t st);
// fused.cu
cudaError_t launch_fused(const SampleTable& tab, const FusedArgs& a, cudaStream_t st);
int64_t fused_cnt_words(const SampleTable& tab);
void fused_plan(const SampleTable& tab, FusedArgs* a);
// plain.cu
cudaError_t launch_plain(const tsne_csr& P, const SampleTable& tab, const float2* Y, float alpha,
                         float2* grad, double* Z, float2* Fa, float2* Fr, float* Zi,
                         int64_t* seg, int32_t* sid, int32_t* status, cudaStream_t st);
cudaError_t launch_plain_step(const tsne_csr& P, const SampleTable& tab, float2* Y, float2* U,
                              float2* G, float alpha, float mu, float lr, float min_gain,
                              float2* grad, double* Z, float2* Fa, float2* Fr, float* Zi,
                              int64_t* seg, int32_t* sid, int32_t* status, cudaStream_t st);
// knn.cu
size_t knn_fp32_smem(int d, int k);
cudaError_t launch_knn_fp32(const float* X, int d, int k, const SampleTable& tab, int32_t* idx,
                            float* d2, cudaStream_t st);
// knn_tc.cu
size_t knn_tc_ws_bytes(int64_t n, int S);
int knn_tc_max_k2();
size_t pca_ws_bytes(int64_t n, int g, bool fit);
bool pca_layout_ok(const float* A, int64_t lda);
cudaError_t launch_pca_fit(const float* A, int64_t n, int g, int64_t lda, int k, int n_power,
                           const float* omega, float* scores, float* comp, double* sigma,
                           double* ev, double* mean_out, double* total_var, void* ws,
                           int32_t* status, cudaStream_t st);
cudaError_t launch_pca_transform(const float* A, int64_t n, int g, int64_t lda,
                                 const double* mean_in, const float* comp, int k, float* scores,
                                 void* ws, int32_t* status, cudaStream_t st);
cudaError_t launch_knn_tc(const float* X, int64_t n, int d, int k, int k2, const SampleTable& tab,
                          void* ws, int32_t* idx, float* d2, int32_t* status,
                          long long wait_limit, cudaStream_t st);
// affinity.cu / sort.cu
cudaError_t launch_calibrate(const float* d2, int64_t n, int k, float perp, float tol,
                             int max_iter, float* pc, float* beta, int64_t* n_bad,
                             cudaStream_t st);
struct SymWs {
  uint64_t* k0; uint64_t* k1; float* v0; float* v1;
  uint32_t* hist; uint32_t* part; uint32_t* bstart; uint32_t* row_cnt;
};
cudaError_t launch_symmetrize(const int32_t* idx, const float* pc, int64_t n, int k,
                              const SampleTable& tab, const SymWs& w, int64_t* row_ptr,
                              int32_t* col, float* val, int64_t cap, int fuzzy, int32_t* status,
                              cudaStream_t st);
cudaError_t launch_fuzzy_calibrate(const float* d2, int64_t n, int k, float tol, int max_iter,
                                   float* w, float* rho, float* sigma, int64_t* n_bad,
                                   cudaStream_t st);
int64_t radix_tiles(int64_t m);
// umap.cu
int umap_block_points();
cudaError_t launch_umap_layout(const int64_t* rp, const int32_t* col, const float* w, float2* Y,
                               float2* scratch, const SampleTable& tab, int n_epochs, int epoch0,
                               int n_run, float a, float b, float alpha0, int n_neg,
                               uint64_t seed, int32_t* status, cudaStream_t st);
size_t umap_init_ws_bytes();
cudaError_t launch_umap_init(const float* S, int64_t n, int64_t ld, float2* U, void* ws,
                             int32_t* status, cudaStream_t st);
int umap_fit_ab(double min_dist, double spread, double* a_out, double* b_out);
int64_t scan_parts_len(int64_t m);
cudaError_t launch_fill_f32(float* p, int64_t m, float v, cudaStream_t st);
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

// Point-wise blocks of `pts` points, never straddling a sample.
void fill_blocks(SampleTable* tab, int pts = 256) {
  tab->blk_pts = pts;
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
  int cfg;        // direct kernel configuration
  int sym_w;      // symmetric kernel warps per CTA (0: direct only)
  int sym_fx;     // symmetric kernel sums in fixed point (Facc) instead of partial buffers
  int fused;      // tsne_step: one persistent launch per iteration (batched samples)
  size_t off_cnt; // fused: queue head, exit count, per-sample completion counters
  int64_t n;
  int64_t items;  // direct work items
  int64_t sym_items;
  int64_t fpart_elems;
  size_t off_hdr, off_Fa, off_Fpart, off_zpart, off_Rbuf, off_Cbuf, off_Facc, off_zsym,
      off_klrow, off_Z, off_kl, off_zred, total;
  int zred_nb;    // slices per sample of the two-stage Z / KL reduction
};

int make_sym_plan(int64_t n, GradPlan* pl, int W, int fx_mode);

// Slices per sample of the two-stage Z / KL reduction (a pure function of the
// sample count, so that the summation order does not depend on the device).
int zred_slices(int S) {
  const int nb = 256 / (S > 0 ? S : 1);
  return nb < 1 ? 1 : nb > 64 ? 64 : nb;
}

// The partial buffers of the symmetric split take 16 B per point and group pair,
// i.e. O(N^2) (7.8 GB at 1M points); the tiled fixed-point form needs O(N)
// scratch and is as fast once its tiles fill the GPU many times over (1M points
// on B300: 159.8-160.0 ms per step against 160.1 ms with the buffers), so AUTO
// takes it when the call has at least kTileWaves waves of tiles (three CTAs per
// SM); with fewer, whole tiles leave SMs idle (50,000 points: 91 tiles, 1.19
// against 0.79 ms per iteration) and AUTO keeps the buffers.  SYM4 keeps the
// buffers while they fit this budget and sums in fixed point beyond it.
constexpr double kSymBufBudget = 32.0 * (1ull << 30);
constexpr int kTileWaves = 8;

bool tiles_fill_gpu(const SampleTable& tab) {
  int64_t T = 0;
  for (int s = 0; s < tab.S; s++)
    T += tsne::sym_tile_count((tab.pt_off[s + 1] - tab.pt_off[s] + 1023) / 1024);
  return T >= (int64_t)kTileWaves * 3 * device_sm_count();
}

int64_t max_sample(const SampleTable& tab) {
  int64_t nmax = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    if (ns > nmax) nmax = ns;
  }
  return nmax;
}

// The persistent one-launch iteration (fused.cu) runs when asked for
// (TSNE_VARIANT_FUSED, or the autotuner's choice); AUTO keeps the per-term
// kernels, measured faster on the 64-sample batch (0.68 against 0.76 ms per
// step on B300).
bool choose_fused(const SampleTable& tab, int variant, bool for_step) {
  (void)tab;
  return for_step && variant == TSNE_VARIANT_FUSED;
}

// The symmetric split pays off once samples span several groups; the direct
// form handles small problems (and every diagonal group).
bool choose_sym(const SampleTable& tab, int variant) {
  if (variant == TSNE_VARIANT_SYM || variant == TSNE_VARIANT_SYM4 ||
      variant == TSNE_VARIANT_SYM4_FX)
    return true;
  if (variant != TSNE_VARIANT_AUTO) return false;
  int64_t nmax = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    if (ns > nmax) nmax = ns;
  }
  return nmax >= 16384;
}

int choose_cfg(const SampleTable& tab, int variant) {
  if (variant == TSNE_VARIANT_DIRECT_L) return 0;
  if (variant == TSNE_VARIANT_DIRECT_S || variant == TSNE_VARIANT_FUSED) return 1;
  if (variant == TSNE_VARIANT_DIRECT_M) return 2;
  double pairs = 0.0;
  int64_t nmax = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    pairs += (double)ns * (double)ns;
    if (ns > nmax) nmax = ns;
  }
  // small problems need small items to spread over the SMs (B300, one graph-
  // captured step: 2,000 points 32.3 -> 20.9 us, 5,000 points 37.9 -> 29.9 us,
  // 12,000 points 73.7 -> 69.8 us against cfg 1)
  if (pairs < 4e7) return 4;
  if (pairs < 4e8) return 3;
  return (nmax >= 32768 && pairs >= 4e9) ? 0 : 1;
}

// Work split of the repulsion.  Items of one sample cost rows_per_item x chunk
// width pair evaluations; the chunk width is chosen so the whole call has about
// 32 items per resident CTA slot (load balance over 148 SMs), never narrower
// than one shared-memory tile, with at most 64 chunks per sample.
int make_grad_plan(int64_t n, const tsne_batch* B, const tsne_params* prm, GradPlan* pl,
                   bool for_step = false) {
  int rc = table_from_batch(n, B, 2, &pl->tab);
  if (rc) return rc;
  SampleTable& tab = pl->tab;
  fill_blocks(&tab);
  pl->n = n;
  const int variant = prm ? prm->variant : TSNE_VARIANT_AUTO;
  if (variant < TSNE_VARIANT_AUTO || variant > TSNE_VARIANT_SYM4_FX) return TSNE_ERR_ARG;
  pl->fused = choose_fused(tab, variant, for_step) ? 1 : 0;
  pl->off_cnt = 0;
  // the fused launch runs the symmetric split with groups of 1024 points
  if (pl->fused) return make_sym_plan(n, pl, 4, 0);
  // AUTO takes the 1024-point groups: faster than 2048 at every size measured
  // (50k to 1M points) on B300
  if (choose_sym(tab, variant)) {
    if (variant == TSNE_VARIANT_SYM) return make_sym_plan(n, pl, 8, 0);
    return make_sym_plan(n, pl, 4,
                         variant == TSNE_VARIANT_SYM4_FX ||
                                 (variant == TSNE_VARIANT_AUTO && tiles_fill_gpu(tab))
                             ? 1
                             : -1);
  }
  pl->sym_w = 0;
  pl->sym_items = 0;
  pl->cfg = choose_cfg(tab, variant);
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
  pl->off_Fpart = c.take(sizeof(float2) * (size_t)fp);
  pl->off_zpart = c.take(sizeof(double) * (size_t)items);
  pl->off_Rbuf = pl->off_Cbuf = pl->off_Facc = pl->off_zsym = 0;
  pl->sym_fx = 0;
  pl->off_klrow = c.take(sizeof(double2) * (size_t)n);
  pl->off_Z = c.take(sizeof(double) * (size_t)tab.S);
  pl->off_kl = c.take(sizeof(double) * (size_t)tab.S);
  pl->zred_nb = zred_slices(tab.S);
  pl->off_zred = c.take(3 * sizeof(double) * (size_t)tab.S * (size_t)pl->zred_nb);
  pl->total = c.off;
  return TSNE_OK;
}

// Tiled fixed-point form: the tiles of every sample (tile_off).
void plan_sym_tiles(GradPlan* pl, int64_t GS) {
  SampleTable& tab = pl->tab;
  int64_t T = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t G = (tab.pt_off[s + 1] - tab.pt_off[s] + GS - 1) / GS;
    tab.tile_off[s] = (int32_t)T;
    T += sym_tile_count(G);
  }
  tab.tile_off[tab.S] = (int32_t)T;
}

// Symmetric split: groups of GS = W x 256 points (W = 8: 2048, W = 4: 1024);
// the symmetric kernel evaluates every pair of distinct groups once and, in the
// same launch after them, every diagonal group's pairs once (one item per
// group, written like a direct-kernel item of GS rows); the fused kernel takes
// the same items from its queue.  fx_mode: 1 fixed-point sums, 0 partial
// buffers, -1 buffers within kSymBufBudget.
int make_sym_plan(int64_t n, GradPlan* pl, int W, int fx_mode) {
  SampleTable& tab = pl->tab;
  pl->cfg = W == 4 ? 2 : 0;  // GS-row items: cfg 2 for 1024, cfg 0 for 2048
  pl->sym_w = W;
  const int GS = sym_group_size(pl->sym_w);
  int rows = 0, tile = 0;
  rep_cfg_shape(pl->cfg, &rows, &tile);
  if (rows > GS || GS % rows != 0) return TSNE_ERR_ARG;
  tab.rows_per_item = rows;
  tab.tile_cols = tile;
  tab.diag = 1;
  tab.sym_gs = GS;
  int64_t items = 0, sym = 0, fp = 0;
  for (int s = 0; s < tab.S; s++) {
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    const int64_t G = (ns + GS - 1) / GS;
    tab.item_off[s] = (int32_t)items;
    tab.sym_off[s] = (int32_t)sym;
    tab.chunks[s] = 1;
    tab.fp_off[s] = fp;
    items += (ns + rows - 1) / rows;
    sym += G * (G - 1) / 2;
    fp += ns;
    if (sym > 0x7fffffffLL) return TSNE_ERR_ARG;
  }
  tab.item_off[tab.S] = (int32_t)items;
  tab.sym_off[tab.S] = (int32_t)sym;
  tab.fp_off[tab.S] = fp;
  tab.max_chunks = 1;
  pl->items = items;
  pl->sym_items = sym;
  pl->fpart_elems = fp;
  Carver c;
  pl->off_hdr = c.take(sizeof(WsHeader));
  pl->off_Fa = c.take(sizeof(float2) * (size_t)n);
  pl->off_Fpart = c.take(sizeof(float2) * (size_t)fp);
  pl->off_zpart = c.take(sizeof(double) * (size_t)items);
  const double buf_bytes = 2.0 * sizeof(float2) * (double)sym * (double)GS;
  pl->sym_fx = fx_mode > 0 || (fx_mode < 0 && buf_bytes > kSymBufBudget) ? 1 : 0;
  if (pl->sym_fx) plan_sym_tiles(pl, GS);
  pl->off_Rbuf = pl->off_Cbuf = pl->off_Facc = 0;
  if (pl->sym_fx) {
    pl->off_Facc = c.take(2 * sizeof(unsigned long long) * (size_t)n);
  } else {
    pl->off_Rbuf = c.take(sizeof(float2) * (size_t)sym * GS);
    pl->off_Cbuf = c.take(sizeof(float2) * (size_t)sym * GS);
  }
  pl->off_zsym = c.take(sizeof(double) * (size_t)sym);
  pl->off_klrow = c.take(sizeof(double2) * (size_t)n);
  pl->off_Z = c.take(sizeof(double) * (size_t)tab.S);
  pl->off_kl = c.take(sizeof(double) * (size_t)tab.S);
  if (pl->fused) pl->off_cnt = c.take(sizeof(uint32_t) * (size_t)fused_cnt_words(tab));
  pl->zred_nb = zred_slices(tab.S);
  pl->off_zred = c.take(3 * sizeof(double) * (size_t)tab.S * (size_t)pl->zred_nb);
  pl->total = c.off;
  return TSNE_OK;
}

RepBufs rep_bufs(const GradPlan& pl, void* ws) {
  RepBufs rb;
  rb.Fpart = reinterpret_cast<const float2*>(static_cast<char*>(ws) + pl.off_Fpart);
  rb.zpart = reinterpret_cast<const double*>(static_cast<char*>(ws) + pl.off_zpart);
  const bool bufs = pl.sym_w && !pl.sym_fx;
  rb.Rbuf = bufs ? reinterpret_cast<const float2*>(static_cast<char*>(ws) + pl.off_Rbuf) : nullptr;
  rb.Cbuf = bufs ? reinterpret_cast<const float2*>(static_cast<char*>(ws) + pl.off_Cbuf) : nullptr;
  rb.Facc = pl.sym_w && pl.sym_fx
                ? reinterpret_cast<const unsigned long long*>(static_cast<char*>(ws) + pl.off_Facc)
                : nullptr;
  rb.zsym = pl.sym_w ? reinterpret_cast<const double*>(static_cast<char*>(ws) + pl.off_zsym)
                     : nullptr;
  rb.zred_part = reinterpret_cast<double*>(static_cast<char*>(ws) + pl.off_zred);
  rb.zred_nb = pl.zred_nb;
  return rb;
}

// All repulsion launches of one gradient evaluation.
cudaError_t launch_repulsion(const GradPlan& pl, const float2* Y, void* ws, int32_t* status,
                             cudaStream_t st) {
  char* b = static_cast<char*>(ws);
  if (pl.sym_w && pl.sym_fx) {
    cudaError_t z = cudaMemsetAsync(b + pl.off_Facc, 0,
                                    2 * sizeof(unsigned long long) * (size_t)pl.n, st);
    if (z != cudaSuccess) return z;
  }
  float2* Fpart = reinterpret_cast<float2*>(b + pl.off_Fpart);
  double* zpart = reinterpret_cast<double*>(b + pl.off_zpart);
  if (!pl.sym_w) return launch_repulse_direct(pl.cfg, Y, pl.tab, pl.items, Fpart, zpart, st);
  // the symmetric launch runs the diagonal groups (pl.items of them) after the pairs
  const int64_t diag = pl.items;
  if (pl.sym_fx)
    return launch_repulse_sym_tiled(Y, pl.tab, diag, reinterpret_cast<double*>(b + pl.off_zsym),
                                    reinterpret_cast<unsigned long long*>(b + pl.off_Facc),
                                    Fpart, zpart, status, st);
  return launch_repulse_sym(pl.sym_w, Y, pl.tab, pl.sym_items, diag,
                            reinterpret_cast<float2*>(b + pl.off_Rbuf),
                            reinterpret_cast<float2*>(b + pl.off_Cbuf),
                            reinterpret_cast<double*>(b + pl.off_zsym), Fpart, zpart, st);
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

// Host-side fault injection for tests of the error paths: TSNE_FAULT holds
// "<entry>:<code>" pairs separated by commas, e.g. "tsne_knn:-3,tsne_step:-1";
// the named entry point then returns that code before doing anything.  Nothing
// is injected on the GPU.
int injected_fault(const char* entry) {
  const char* env = getenv("TSNE_FAULT");
  if (!env || !*env) return 0;
  const size_t len = strlen(entry);
  for (const char* p = env; (p = strstr(p, entry)) != nullptr; p += len) {
    const bool starts = p == env || p[-1] == ',';
    if (starts && p[len] == ':') return atoi(p + len + 1);
  }
  return 0;
}

// Cycles a device-side wait may spin before giving up (TSNE_WAIT_LIMIT
// overrides the default of about two seconds at 2 GHz).
long long device_wait_limit() {
  const char* env = getenv("TSNE_WAIT_LIMIT");
  if (env && *env) {
    const long long v = atoll(env);
    if (v > 0) return v;
  }
  return 4000000000ll;
}

// Workspace of the plain form: Fa, Fr, Z_i, per-point segments and sample ids
// (tsne_kl_grad_plain), then the gradient and Z_s of tsne_step_plain.
struct PlainLayout {
  size_t Fa, Fr, Zi, seg, sid, grad, Z, total;
};

PlainLayout plain_layout(int64_t n, int S) {
  PlainLayout L;
  Carver c;
  L.Fa = c.take(sizeof(float2) * (size_t)n);
  L.Fr = c.take(sizeof(float2) * (size_t)n);
  L.Zi = c.take(sizeof(float) * (size_t)n);
  L.seg = c.take(sizeof(int64_t) * 2 * (size_t)n);
  L.sid = c.take(sizeof(int32_t) * (size_t)n);
  L.grad = c.take(sizeof(float2) * (size_t)n);
  L.Z = c.take(sizeof(double) * (size_t)(S > 0 ? S : 1));
  L.total = c.off;
  return L;
}

// Workspace of tsne_affinities: conditional P, then the symmetrisation
// buffers (key/value copies for the radix sort of the transposed entries and
// the forward lists, digit histograms, scan partials, row starts of the
// transposed entries, row counts).
struct AffLayout {
  size_t pc, k0, k1, v0, v1, hist, part, bstart, row_cnt, total;
};

AffLayout aff_layout(int64_t n, int k) {
  AffLayout L;
  const int64_t m2 = n * (int64_t)k;  // transposed entries (and forward entries)
  const int64_t nt = radix_tiles(m2);
  int64_t scan_max = 256 * nt;  // the largest scan: digit histograms or rows
  if (n + 1 > scan_max) scan_max = n + 1;
  Carver c;
  L.pc = c.take(sizeof(float) * (size_t)(n * k));
  L.k0 = c.take(sizeof(uint64_t) * (size_t)(2 * m2));  // transposed keys, forward lists
  L.k1 = c.take(sizeof(uint64_t) * (size_t)m2);
  L.v0 = c.take(sizeof(float) * (size_t)(2 * m2));     // transposed values, duplicate counts
  L.v1 = c.take(sizeof(float) * (size_t)m2);
  L.hist = c.take(sizeof(uint32_t) * (size_t)(256 * nt));
  L.part = c.take(sizeof(uint32_t) * (size_t)scan_parts_len(scan_max));
  L.bstart = c.take(sizeof(uint32_t) * (size_t)(n + 1));
  L.row_cnt = c.take(sizeof(uint32_t) * (size_t)(n + 1));
  L.total = c.off;
  return L;
}

}  // namespace

extern "C" {

void tsne_params_default(tsne_params* p) {
  if (!p) return;
  p->perplexity = 30.0f;
  p->k = 90;
  p->knn_mode = TSNE_KNN_BF16_RERANK;
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
    case TSNE_OP_KL_GRAD: {  // covers both tsne_kl_grad and tsne_step
      std::unique_ptr<GradPlan> pl(new GradPlan);
      if (make_grad_plan(n, B, prm, pl.get(), false)) return 0;
      size_t need = pl->total;
      if (make_grad_plan(n, B, prm, pl.get(), true)) return 0;
      return need > pl->total ? need : pl->total;
    }
    case TSNE_OP_KNN: {
      if (prm->knn_mode != TSNE_KNN_BF16_RERANK || n <= 0) return 0;
      const int S = B ? B->n_samples : 1;
      return knn_tc_ws_bytes(n, S);
    }
    case TSNE_OP_AFFINITIES:
    case TSNE_OP_KNN_GRAPH:
      if (n < 0 || k < 1) return 0;
      return aff_layout(n, k).total;
    case TSNE_OP_PCA:
      if (n < TSNE_PCA_SKETCH + 1 || d < TSNE_PCA_SKETCH) return 0;
      return pca_ws_bytes(n, d, true);
    case TSNE_OP_PCA_TRANSFORM:
      if (n < 1 || d < 1) return 0;
      return pca_ws_bytes(n, d, false);
    case TSNE_OP_UMAP_LAYOUT:
      if (n < 1) return 0;
      return align_up(sizeof(float2) * (size_t)n);
    case TSNE_OP_UMAP_INIT:
      if (n < 1) return 0;
      return align_up(umap_init_ws_bytes());
    case TSNE_OP_PLAIN: {  // covers tsne_kl_grad_plain and tsne_step_plain
      const int S = B ? B->n_samples : 1;
      return plain_layout(n, S).total;
    }
    default:
      return 0;
  }
}

// The attraction runs on a side stream, concurrently with the repulsion: it is
// bound by the latency of its dependent loads, the repulsion by the FP32 pipe,
// and an attraction block fits beside the repulsion's CTAs on an SM.  One
// non-blocking stream and two events per host thread and device, created on
// first use and kept for the thread's lifetime; under stream capture the fork
// and the join become edges of the graph.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
constexpr int kMaxSideDevices = 64;

static cudaError_t side_stream(SideStream** out) {
  thread_local SideStream ss[kMaxSideDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxSideDevices) return cudaErrorInvalidDevice;
  SideStream& x = ss[dev];
  if (!x.join) {
    if (!x.s && (e = cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking)) != cudaSuccess)
      return e;
    if (!x.fork && (e = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming)) != cudaSuccess)
      return e;
    if ((e = cudaEventCreateWithFlags(&x.join, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *out = &x;
  return cudaSuccess;
}

// Repulsion on st and attraction on the side stream, joined back into st, when
// the plan uses the symmetric kernel (the case where an attraction block fits
// beside its CTAs); smaller plans, made of short direct-kernel launches, keep
// both on st, where a fork and a join would only add latency.
static cudaError_t launch_forces(const GradPlan& pl, const tsne_csr& P, const float2* Y,
                                 float2* Fa, double2* klrow, int iter_arg, const WsHeader* hdr,
                                 int kl_every, int force_kl, void* ws, int32_t* status,
                                 cudaStream_t st) {
  if (!pl.sym_w) {
    if (pl.cfg == 3 || pl.cfg == 4) {  // small problems: both terms in one launch
      char* b = static_cast<char*>(ws);
      return launch_forces_direct(pl.cfg, P, Y, pl.tab, pl.items,
                                  reinterpret_cast<float2*>(b + pl.off_Fpart),
                                  reinterpret_cast<double*>(b + pl.off_zpart), Fa, klrow,
                                  iter_arg, hdr, kl_every, force_kl, status, st);
    }
    const cudaError_t ea =
        launch_attract(P, Y, Fa, klrow, iter_arg, hdr, kl_every, force_kl, status, st);
    if (ea != cudaSuccess) return ea;
    return launch_repulsion(pl, Y, ws, status, st);
  }
  SideStream* ss = nullptr;
  cudaError_t e = side_stream(&ss);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventRecord(ss->fork, st)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(ss->s, ss->fork, 0)) != cudaSuccess) return e;
  const cudaError_t er = launch_repulsion(pl, Y, ws, status, st);
  const cudaError_t ea =
      launch_attract(P, Y, Fa, klrow, iter_arg, hdr, kl_every, force_kl, status, ss->s);
  // join even after a failed launch, so that no capture is left forked
  if ((e = cudaEventRecord(ss->join, ss->s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(st, ss->join, 0)) != cudaSuccess) return e;
  return er != cudaSuccess ? er : ea;
}

int tsne_kl_grad(const tsne_csr* P, const tsne_batch* B, const float* Y, float alpha, float* grad,
                 double* Z, double* kl, const tsne_params* prm, void* ws, size_t ws_bytes,
                 int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_kl_grad")) return f;
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
  const RepBufs rb = rep_bufs(*pl, ws);
  double2* klrow = kl ? at<double2>(ws, pl->off_klrow) : nullptr;
  TSNE_CUDA_TRY(launch_forces(*pl, *P, Y2, Fa, klrow, 0, hdr, 0, kl ? 1 : 0, ws, dev_status, st));
  TSNE_CUDA_TRY(launch_reduce(pl->tab, rb, klrow, Z, kl, alpha, 0, hdr, 0, kl ? 1 : 0,
                              pl->tab.S, st));
  if (grad)
    TSNE_CUDA_TRY(launch_grad(pl->tab, rb, Fa, Z, alpha, reinterpret_cast<float2*>(grad), st));
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
  const PlainLayout pl = plain_layout(n, tab->S);
  rc = check_ws(ws, ws_bytes, pl.Z);  // the regions up to the step's gradient
  if (rc) return rc;
  if (n == 0) return TSNE_OK;
  TSNE_CUDA_TRY(launch_plain(*P, *tab, reinterpret_cast<const float2*>(Y), alpha,
                             reinterpret_cast<float2*>(grad), Z, at<float2>(ws, pl.Fa),
                             at<float2>(ws, pl.Fr), at<float>(ws, pl.Zi), at<int64_t>(ws, pl.seg),
                             at<int32_t>(ws, pl.sid), dev_status, (cudaStream_t)stream));
  return TSNE_OK;
}

int tsne_step_plain(const tsne_csr* P, const tsne_batch* B, float* Y, float* uY, float* gains,
                    int iter, const tsne_params* prm, void* ws, size_t ws_bytes,
                    int32_t* dev_status, tsne_stream_t stream) {
  int64_t n = 0;
  int rc = check_csr(P, &n);
  if (rc) return rc;
  if (!Y || !uY || !gains || !prm || iter < 0 || !(prm->min_gain >= 0.f)) return TSNE_ERR_ARG;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  rc = table_from_batch(n, B, 2, tab.get());
  if (rc) return rc;
  const PlainLayout pl = plain_layout(n, tab->S);
  rc = check_ws(ws, ws_bytes, pl.total);
  if (rc) return rc;
  if (n == 0) return TSNE_OK;
  const float alpha = iter < prm->ee_iters ? prm->ee : 1.0f;
  const float mu = iter < prm->mom_switch ? prm->mom0 : prm->mom1;
  TSNE_CUDA_TRY(launch_plain_step(
      *P, *tab, reinterpret_cast<float2*>(Y), reinterpret_cast<float2*>(uY),
      reinterpret_cast<float2*>(gains), alpha, mu, prm->lr, prm->min_gain, at<float2>(ws, pl.grad),
      at<double>(ws, pl.Z), at<float2>(ws, pl.Fa), at<float2>(ws, pl.Fr), at<float>(ws, pl.Zi),
      at<int64_t>(ws, pl.seg), at<int32_t>(ws, pl.sid), dev_status, (cudaStream_t)stream));
  return TSNE_OK;
}

int tsne_step(const tsne_csr* P, const tsne_batch* B, float* Y, float* uY, float* gains, int iter,
              const tsne_params* prm, double* Z, double* kl, void* ws, size_t ws_bytes,
              int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_step")) return f;
  int64_t n = 0;
  int rc = check_csr(P, &n);
  if (rc) return rc;
  if (!Y || !uY || !gains || !prm || iter < -1) return TSNE_ERR_ARG;
  if (prm->kl_every < 0 || !(prm->min_gain >= 0.f)) return TSNE_ERR_ARG;
  std::unique_ptr<GradPlan> pl(new GradPlan);
  rc = make_grad_plan(n, B, prm, pl.get(), true);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, pl->total);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const Schedule q = schedule_from(prm);
  if (pl->fused) {
    std::unique_ptr<FusedArgs> ap(new FusedArgs);
    FusedArgs& a = *ap;
    fused_plan(pl->tab, &a);
    a.P = *P;
    a.Y = reinterpret_cast<float2*>(Y);
    a.U = reinterpret_cast<float2*>(uY);
    a.G = reinterpret_cast<float2*>(gains);
    a.Fa = at<float2>(ws, pl->off_Fa);
    a.Fpart = at<float2>(ws, pl->off_Fpart);
    a.zpart = at<double>(ws, pl->off_zpart);
    a.Rbuf = at<float2>(ws, pl->off_Rbuf);
    a.Cbuf = at<float2>(ws, pl->off_Cbuf);
    a.zsym = at<double>(ws, pl->off_zsym);
    const bool kl_on = kl && prm->kl_every > 0;
    a.klrow = kl_on ? at<double2>(ws, pl->off_klrow) : nullptr;
    a.Zout = Z ? Z : at<double>(ws, pl->off_Z);
    a.kl_out = kl_on ? kl : nullptr;
    a.kl_slots = kl_on ? (int64_t)(prm->n_iter / prm->kl_every) * pl->tab.S : 0;
    a.hdr = at<WsHeader>(ws, pl->off_hdr);
    a.cnt = at<uint32_t>(ws, pl->off_cnt);
    a.status = dev_status;
    a.wait_limit = device_wait_limit();
    a.q = q;
    a.iter_arg = iter;
    TSNE_CUDA_TRY(launch_fused(pl->tab, a, st));
    return TSNE_OK;
  }
  const float2* Y2 = reinterpret_cast<const float2*>(Y);
  WsHeader* hdr = at<WsHeader>(ws, pl->off_hdr);
  float2* Fa = at<float2>(ws, pl->off_Fa);
  const RepBufs rb = rep_bufs(*pl, ws);
  const bool track_kl = kl && prm->kl_every > 0;
  double2* klrow = track_kl ? at<double2>(ws, pl->off_klrow) : nullptr;
  double* Zuse = Z ? Z : at<double>(ws, pl->off_Z);
  TSNE_CUDA_TRY(launch_forces(*pl, *P, Y2, Fa, klrow, iter, hdr, prm->kl_every, 0, ws, dev_status,
                              st));
  const int64_t kl_slots =
      track_kl ? (int64_t)(prm->n_iter / prm->kl_every) * pl->tab.S : 0;
  // with the two-stage reduction the update kernel takes stage two (one launch
  // fewer); plans with few items per sample leave the whole reduction to it
  // (two fewer)
  bool small = true;  // at most 4096 Z partials per sample: the update kernel sums them
  for (int s = 0; small && s < pl->tab.S; s++) {
    const int64_t ni = pl->tab.item_off[s + 1] - pl->tab.item_off[s];
    const int64_t ny = pl->tab.sym_gs > 0 ? pl->tab.sym_off[s + 1] - pl->tab.sym_off[s] : 0;
    small = ni + ny <= 4096;
  }
  const bool fin = small || rb.zred_part != nullptr;
  double* kl_use = track_kl ? kl : nullptr;
  if (!small)
    TSNE_CUDA_TRY(launch_reduce(pl->tab, rb, klrow, Zuse, kl_use, 1.0f, iter, hdr,
                                prm->kl_every, 0, kl_slots, st, fin));
  TSNE_CUDA_TRY(launch_update(pl->tab, rb, Fa, Zuse, q, iter, hdr, reinterpret_cast<float2*>(Y),
                              reinterpret_cast<float2*>(uY), reinterpret_cast<float2*>(gains),
                              dev_status, fin ? Zuse : nullptr, fin ? kl_use : nullptr,
                              prm->kl_every, kl_slots, klrow, small, st));
  return TSNE_OK;
}

int tsne_step_reset(void* ws, size_t ws_bytes, int iter, tsne_stream_t stream) {
  if (!ws || ((uintptr_t)ws & (kAlign - 1)) || ws_bytes < sizeof(WsHeader) || iter < 0)
    return TSNE_ERR_WORKSPACE;
  TSNE_CUDA_TRY(launch_set_iter(reinterpret_cast<WsHeader*>(ws), iter, (cudaStream_t)stream));
  return TSNE_OK;
}

}  // extern "C"

extern "C" {

int tsne_knn(const float* X, int64_t n, int d, int k, const tsne_batch* B, int knn_mode,
             float cand_mult, int32_t* nbr_idx, float* nbr_d2, void* ws, size_t ws_bytes,
             int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_knn")) return f;
  if (n < 0 || d < 1 || k < 1 || n >= 0x7fffffffLL) return TSNE_ERR_ARG;
  if (n > 0 && (!X || !nbr_idx || !nbr_d2)) return TSNE_ERR_ARG;
  if (knn_mode != TSNE_KNN_FP32 && knn_mode != TSNE_KNN_BF16_RERANK) return TSNE_ERR_ARG;
  if (d > 64) return TSNE_ERR_ARG;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  int rc = table_from_batch(n, B, (int64_t)k + 1, tab.get());
  if (rc) return rc;
  if (n == 0) return TSNE_OK;
  fill_blocks(tab.get(), 128);
  cudaStream_t st = (cudaStream_t)stream;
  if (knn_mode == TSNE_KNN_FP32) {
    const size_t smem = knn_fp32_smem(d, k);
    if (smem == 0 || smem > 227 * 1024) return TSNE_ERR_ARG;
    TSNE_CUDA_TRY(launch_knn_fp32(X, d, k, *tab, nbr_idx, nbr_d2, st));
    return TSNE_OK;
  }
  // BF16 tensor-core distances, candidate filter, exact FP32 re-rank
  if (!(cand_mult >= 1.0f)) return TSNE_ERR_ARG;
  int k2 = (int)ceilf(cand_mult * (float)k);
  if (k2 > knn_tc_max_k2()) k2 = knn_tc_max_k2();
  if (k2 < k) return TSNE_ERR_ARG;  // k above the re-rank capacity
  rc = check_ws(ws, ws_bytes, knn_tc_ws_bytes(n, tab->S));
  if (rc) return rc;
  TSNE_CUDA_TRY(launch_knn_tc(X, n, d, k, k2, *tab, ws, nbr_idx, nbr_d2, dev_status,
                              device_wait_limit(), st));
  return TSNE_OK;
}

int tsne_affinities(const int32_t* nbr_idx, const float* nbr_d2, int64_t n, int k,
                    const tsne_batch* B, float perplexity, float tol, int max_iter, tsne_csr* P,
                    float* beta, int64_t* n_bad, void* ws, size_t ws_bytes, int32_t* dev_status,
                    tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_affinities")) return f;
  if (n < 0 || k < 1 || k > 256 || n >= 0x7fffffffLL) return TSNE_ERR_ARG;
  if (!(perplexity > 1.0f) || !(perplexity < (float)k) || !(tol > 0.f) || max_iter < 1)
    return TSNE_ERR_ARG;
  if (!P || P->n != n || (n > 0 && (!nbr_idx || !nbr_d2 || !P->row_ptr || !P->col || !P->val)))
    return TSNE_ERR_ARG;
  const int64_t m = 2 * n * (int64_t)k;
  if (m >= 0x7fffffffLL) return TSNE_ERR_ARG;
  if (P->cap < m) return TSNE_ERR_CAPACITY;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  int rc = table_from_batch(n, B, (int64_t)k + 1, tab.get());
  if (rc) return rc;
  fill_blocks(tab.get(), 128);
  const AffLayout L = aff_layout(n, k);
  rc = check_ws(ws, ws_bytes, L.total);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    TSNE_CUDA_TRY(cudaMemsetAsync(P->row_ptr, 0, sizeof(int64_t), st));
    return TSNE_OK;
  }
  float* pc = at<float>(ws, L.pc);
  TSNE_CUDA_TRY(launch_calibrate(nbr_d2, n, k, perplexity, tol, max_iter, pc, beta, n_bad, st));
  SymWs w;
  w.k0 = at<uint64_t>(ws, L.k0);
  w.k1 = at<uint64_t>(ws, L.k1);
  w.v0 = at<float>(ws, L.v0);
  w.v1 = at<float>(ws, L.v1);
  w.hist = at<uint32_t>(ws, L.hist);
  w.part = at<uint32_t>(ws, L.part);
  w.bstart = at<uint32_t>(ws, L.bstart);
  w.row_cnt = at<uint32_t>(ws, L.row_cnt);
  TSNE_CUDA_TRY(launch_symmetrize(nbr_idx, pc, n, k, *tab, w, P->row_ptr, P->col, P->val, P->cap,
                                  0, dev_status, st));
  return TSNE_OK;
}

int tsne_knn_graph(const int32_t* nbr_idx, const float* nbr_d2, int64_t n, int k,
                   const tsne_batch* B, float tol, int max_iter, tsne_csr* G, float* rho,
                   float* sigma, int64_t* n_bad, void* ws, size_t ws_bytes, int32_t* dev_status,
                   tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_knn_graph")) return f;
  if (n < 0 || k < 2 || k > 256 || n >= 0x7fffffffLL) return TSNE_ERR_ARG;
  if (!(tol > 0.f) || max_iter < 1) return TSNE_ERR_ARG;
  if (!G || G->n != n || (n > 0 && (!nbr_idx || !nbr_d2 || !G->row_ptr || !G->col || !G->val)))
    return TSNE_ERR_ARG;
  const int64_t m = 2 * n * (int64_t)k;
  if (m >= 0x7fffffffLL) return TSNE_ERR_ARG;
  if (G->cap < m) return TSNE_ERR_CAPACITY;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  int rc = table_from_batch(n, B, (int64_t)k + 1, tab.get());
  if (rc) return rc;
  fill_blocks(tab.get(), 128);
  const AffLayout L = aff_layout(n, k);
  rc = check_ws(ws, ws_bytes, L.total);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    TSNE_CUDA_TRY(cudaMemsetAsync(G->row_ptr, 0, sizeof(int64_t), st));
    return TSNE_OK;
  }
  float* wgt = at<float>(ws, L.pc);
  TSNE_CUDA_TRY(launch_fuzzy_calibrate(nbr_d2, n, k, tol, max_iter, wgt, rho, sigma, n_bad, st));
  SymWs w;
  w.k0 = at<uint64_t>(ws, L.k0);
  w.k1 = at<uint64_t>(ws, L.k1);
  w.v0 = at<float>(ws, L.v0);
  w.v1 = at<float>(ws, L.v1);
  w.hist = at<uint32_t>(ws, L.hist);
  w.part = at<uint32_t>(ws, L.part);
  w.bstart = at<uint32_t>(ws, L.bstart);
  w.row_cnt = at<uint32_t>(ws, L.row_cnt);
  TSNE_CUDA_TRY(launch_symmetrize(nbr_idx, wgt, n, k, *tab, w, G->row_ptr, G->col, G->val, G->cap,
                                  1, dev_status, st));
  return TSNE_OK;
}

int tsne_umap_layout(const tsne_csr* G, const tsne_batch* B, float* Y, int n_epochs, int epoch0,
                     int n_run, float a, float b, float alpha0, int n_neg, uint64_t seed, void* ws,
                     size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_umap_layout")) return f;
  int64_t n = 0;
  int rc = check_csr(G, &n);
  if (rc) return rc;
  if (n > 0 && !Y) return TSNE_ERR_ARG;
  if (n_epochs < 1 || n_epochs >= (1 << 24) || epoch0 < 0 || n_run < 0 ||
      (int64_t)epoch0 + n_run > n_epochs)
    return TSNE_ERR_ARG;
  if (!(a > 0.f) || !isfinite(a) || !(b > 0.f) || !isfinite(b)) return TSNE_ERR_ARG;
  if (!(alpha0 > 0.f) || !isfinite(alpha0) || n_neg < 0 || n_neg > 15) return TSNE_ERR_ARG;
  std::unique_ptr<SampleTable> tab(new SampleTable);
  rc = table_from_batch(n, B, 1, tab.get());
  if (rc) return rc;
  fill_blocks(tab.get(), umap_block_points());
  if (n == 0 || n_run == 0) return TSNE_OK;
  rc = check_ws(ws, ws_bytes, sizeof(float2) * (size_t)n);
  if (rc) return rc;
  TSNE_CUDA_TRY(launch_umap_layout(G->row_ptr, G->col, G->val, reinterpret_cast<float2*>(Y),
                                   static_cast<float2*>(ws), *tab, n_epochs, epoch0, n_run, a, b,
                                   alpha0, n_neg, seed, dev_status, (cudaStream_t)stream));
  return TSNE_OK;
}

int tsne_umap_ab(float min_dist, float spread, double* a, double* b) {
  if (const int f = injected_fault("tsne_umap_ab")) return f;
  if (!a || !b || !(min_dist >= 0.f) || !(spread > 0.f) || !isfinite(min_dist) ||
      !isfinite(spread))
    return TSNE_ERR_ARG;
  return umap_fit_ab((double)min_dist, (double)spread, a, b);
}

int tsne_umap_init(const float* scores, int64_t n, int64_t ld, float* U, void* ws,
                   size_t ws_bytes, int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_umap_init")) return f;
  if (n < 0 || ld < 2) return TSNE_ERR_ARG;
  if (n == 0) return TSNE_OK;
  if (!scores || !U) return TSNE_ERR_ARG;
  const int rc = check_ws(ws, ws_bytes, align_up(umap_init_ws_bytes()));
  if (rc) return rc;
  TSNE_CUDA_TRY(launch_umap_init(scores, n, ld, reinterpret_cast<float2*>(U), ws, dev_status,
                                 (cudaStream_t)stream));
  return TSNE_OK;
}

}  // extern "C"

namespace {

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Stream-ordered scratch of one tsne_run call, freed in reverse order.
struct RunAllocs {
  cudaStream_t st;
  std::vector<void*> ptrs;
  template <typename T>
  cudaError_t get(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, count ? count * sizeof(T) : 256, st);
    if (e == cudaSuccess) ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return e;
  }
  void release(void* p) {
    for (size_t i = 0; i < ptrs.size(); i++)
      if (ptrs[i] == p) {
        cudaFreeAsync(p, st);
        ptrs.erase(ptrs.begin() + i);
        return;
      }
  }
  ~RunAllocs() {
    for (size_t i = ptrs.size(); i-- > 0;) cudaFreeAsync(ptrs[i], st);
    cudaStreamSynchronize(st);
  }
};

#define RUN_TRY(expr)                         \
  do {                                        \
    int _rc = (expr);                         \
    if (_rc != TSNE_OK) return _rc;           \
  } while (0)

int run_impl(const float* X, int64_t n, int d, const tsne_batch* B, const tsne_params* prm,
             float* Y, double* kl_trace, int32_t* status_out, cudaStream_t st) {
  const int k = prm->k;
  const bool x_dev = is_device_ptr(X), y_dev = is_device_ptr(Y);
  RunAllocs A;
  A.st = st;
  int S = B ? B->n_samples : 1;
  const float* Xd = X;
  if (!x_dev) {
    float* t;
    TSNE_CUDA_TRY(A.get(&t, (size_t)n * d));
    TSNE_CUDA_TRY(cudaMemcpyAsync(t, X, sizeof(float) * n * d, cudaMemcpyHostToDevice, st));
    Xd = t;
  }
  float* Yd = Y;
  if (!y_dev) {
    TSNE_CUDA_TRY(A.get(&Yd, (size_t)n * 2));
    TSNE_CUDA_TRY(cudaMemcpyAsync(Yd, Y, sizeof(float) * n * 2, cudaMemcpyHostToDevice, st));
  }
  int32_t* status;
  int64_t* n_bad;
  TSNE_CUDA_TRY(A.get(&status, 1));
  TSNE_CUDA_TRY(A.get(&n_bad, 1));
  TSNE_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  TSNE_CUDA_TRY(cudaMemsetAsync(n_bad, 0, sizeof(int64_t), st));

  // kNN and affinities
  int32_t* idx;
  float* d2;
  TSNE_CUDA_TRY(A.get(&idx, (size_t)n * k));
  TSNE_CUDA_TRY(A.get(&d2, (size_t)n * k));
  {
    const size_t kwsb = tsne_workspace_size(TSNE_OP_KNN, n, d, k, B, prm);
    char* kws = nullptr;
    if (kwsb) TSNE_CUDA_TRY(A.get(&kws, kwsb));
    RUN_TRY(tsne_knn(Xd, n, d, k, B, prm->knn_mode, prm->cand_mult, idx, d2, kws, kwsb, status,
                     (tsne_stream_t)st));
    if (kws) A.release(kws);
  }
  if (!x_dev) A.release((void*)Xd);
  tsne_csr P;
  P.n = n;
  P.nnz = 0;
  P.cap = 2 * n * (int64_t)k;
  TSNE_CUDA_TRY(A.get(&P.row_ptr, (size_t)n + 1));
  TSNE_CUDA_TRY(A.get(&P.col, (size_t)P.cap));
  TSNE_CUDA_TRY(A.get(&P.val, (size_t)P.cap));
  {
    const size_t wsb = tsne_workspace_size(TSNE_OP_AFFINITIES, n, d, k, B, prm);
    char* ws;
    TSNE_CUDA_TRY(A.get(&ws, wsb));
    RUN_TRY(tsne_affinities(idx, d2, n, k, B, prm->perplexity, prm->calib_tol,
                            prm->calib_max_iter, &P, nullptr, n_bad, ws, wsb, status,
                            (tsne_stream_t)st));
    A.release(ws);
  }
  A.release(idx);
  A.release(d2);

  // optimisation
  float *U, *G;
  TSNE_CUDA_TRY(A.get(&U, (size_t)n * 2));
  TSNE_CUDA_TRY(A.get(&G, (size_t)n * 2));
  TSNE_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(float) * n * 2, st));
  TSNE_CUDA_TRY(launch_fill_f32(G, n * 2, 1.0f, st));
  const int n_kl = prm->kl_every > 0 ? prm->n_iter / prm->kl_every : 0;
  double* kl_dev = nullptr;
  if (n_kl > 0 && kl_trace) {
    TSNE_CUDA_TRY(A.get(&kl_dev, (size_t)n_kl * S));
    TSNE_CUDA_TRY(cudaMemsetAsync(kl_dev, 0, sizeof(double) * n_kl * S, st));
  }
  const size_t gwsb = tsne_workspace_size(TSNE_OP_KL_GRAD, n, d, k, B, prm);
  char* gws;
  TSNE_CUDA_TRY(A.get(&gws, gwsb));
  RUN_TRY(tsne_step_reset(gws, gwsb, 0, (tsne_stream_t)st));
  const int chunk = 25;
  int done = 0;
  if (prm->use_graph && prm->n_iter >= chunk) {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    SideStream* side = nullptr;  // created before the capture opens
    TSNE_CUDA_TRY(side_stream(&side));
    TSNE_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = TSNE_OK;
    for (int c = 0; c < chunk && rc == TSNE_OK; c++)
      rc = tsne_step(&P, B, Yd, U, G, -1, prm, nullptr, kl_dev, gws, gwsb, status,
                     (tsne_stream_t)st);
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (rc != TSNE_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    TSNE_CUDA_TRY(ce);
    ce = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    TSNE_CUDA_TRY(ce);
    for (; done + chunk <= prm->n_iter; done += chunk) {
      ce = cudaGraphLaunch(ge, st);
      if (ce != cudaSuccess) break;
    }
    cudaGraphExecDestroy(ge);
    TSNE_CUDA_TRY(ce);
  }
  for (; done < prm->n_iter; done++)
    RUN_TRY(tsne_step(&P, B, Yd, U, G, -1, prm, nullptr, kl_dev, gws, gwsb, status,
                      (tsne_stream_t)st));

  // results
  int32_t st_h = 0;
  int64_t bad_h = 0;
  if (!y_dev)
    TSNE_CUDA_TRY(cudaMemcpyAsync(Y, Yd, sizeof(float) * n * 2, cudaMemcpyDeviceToHost, st));
  if (kl_dev)
    TSNE_CUDA_TRY(cudaMemcpyAsync(kl_trace, kl_dev, sizeof(double) * n_kl * S,
                                  cudaMemcpyDeviceToHost, st));
  TSNE_CUDA_TRY(cudaMemcpyAsync(&st_h, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TSNE_CUDA_TRY(cudaMemcpyAsync(&bad_h, n_bad, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TSNE_CUDA_TRY(cudaStreamSynchronize(st));
  if (status_out) *status_out = st_h;
  if (st_h) return TSNE_ERR_DEVICE_STATUS;
  if (bad_h) return TSNE_ERR_NOT_CONVERGED;
  return TSNE_OK;
}

}  // namespace

extern "C" int tsne_run(const float* X, int64_t n, int d, const tsne_batch* B,
                        const tsne_params* prm, float* Y, double* kl_trace, int32_t* status_out,
                        tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_run")) return f;
  if (!X || !Y || !prm || n < 2 || d < 1) return TSNE_ERR_ARG;
  if (prm->n_iter < 0 || prm->k < 1) return TSNE_ERR_ARG;
  if (status_out) *status_out = 0;
  // Work on an internal non-blocking stream (capturable), ordered after the
  // caller's stream, and synchronised before returning.
  cudaStream_t cs = (cudaStream_t)stream, st = nullptr;
  cudaEvent_t ev = nullptr;
  TSNE_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  int rc = TSNE_OK;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(ev, cs) != cudaSuccess || cudaStreamWaitEvent(st, ev, 0) != cudaSuccess) {
    rc = TSNE_ERR_CUDA;
  } else {
    rc = run_impl(X, n, d, B, prm, Y, kl_trace, status_out, st);
  }
  if (ev) cudaEventDestroy(ev);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
  return rc;
}

extern "C" {

int tsne_pca(const float* A, int64_t n, int g, int64_t lda, int k, int n_power,
             const float* omega, float* scores, float* components, double* sigma,
             double* explained_var, double* mean, double* total_var, void* ws, size_t ws_bytes,
             int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_pca")) return f;
  if (n < TSNE_PCA_SKETCH + 1 || g < TSNE_PCA_SKETCH || lda < g || k < 1 ||
      k > TSNE_PCA_SKETCH || n_power < 0 || n_power > 64 || n >= 0x7fffffffLL ||
      g > (1 << 24))
    return TSNE_ERR_ARG;
  if (!A || !omega || !scores || !components || !total_var) return TSNE_ERR_ARG;
  if (!tsne::pca_layout_ok(A, lda)) return TSNE_ERR_ARG;
  const int rc = check_ws(ws, ws_bytes, tsne::pca_ws_bytes(n, g, true));
  if (rc) return rc;
  TSNE_CUDA_TRY(tsne::launch_pca_fit(A, n, g, lda, k, n_power, omega, scores, components, sigma,
                                     explained_var, mean, total_var, ws, dev_status,
                                     (cudaStream_t)stream));
  return TSNE_OK;
}

int tsne_pca_transform(const float* A, int64_t n, int g, int64_t lda, const double* mean,
                       const float* components, int k, float* scores, void* ws, size_t ws_bytes,
                       int32_t* dev_status, tsne_stream_t stream) {
  if (const int f = injected_fault("tsne_pca_transform")) return f;
  if (n < 1 || g < 1 || lda < g || k < 1 || k > TSNE_PCA_SKETCH || n >= 0x7fffffffLL ||
      g > (1 << 24))
    return TSNE_ERR_ARG;
  if (!A || !mean || !components || !scores) return TSNE_ERR_ARG;
  if (!tsne::pca_layout_ok(A, lda)) return TSNE_ERR_ARG;
  const int rc = check_ws(ws, ws_bytes, tsne::pca_ws_bytes(n, g, false));
  if (rc) return rc;
  TSNE_CUDA_TRY(tsne::launch_pca_transform(A, n, g, lda, mean, components, k, scores, ws,
                                           dev_status, (cudaStream_t)stream));
  return TSNE_OK;
}

}  // extern "C"
