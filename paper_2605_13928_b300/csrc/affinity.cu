// affinity.cu -- t-SNE input affinities on the kNN graph
// (van der Maaten & Hinton 2008, Sec. 2; sparse form of van der Maaten 2014,
// Sec. 3):
//   p_{j|i} = exp(-beta_i d2_ij) / sum_l exp(-beta_i d2_il) over the k
//   neighbours, beta_i chosen so that H_i = -sum_j p_{j|i} log p_{j|i} equals
//   log(perplexity); then P = (P_cond + P_cond^T) / (2 n_s).
#include "common.cuh"

namespace tsne {

cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t m, uint32_t* part,
                            cudaStream_t st);

// ---------------------------------------------------------------------------
// Calibration: two rows per warp (a half-warp, 16 lanes, each), KPL neighbour
// distances per lane in registers.  With s_j = d2_j - min d2 and
// S = sum exp(-beta s_j):
//   H(beta) = log S + beta sum_j exp(-beta s_j) s_j / S,
// strictly decreasing from log k (beta = 0) to log(#ties at the minimum), with
// dH/dbeta = -beta Var(s) under the row's p (the same sums and sum p s^2).
// Safeguarded Newton: start at beta = 1; each step keeps the bracket
// [lo, hi] of the root (lo = 0, hi = +inf at first) and takes the Newton step
// when it lands inside the bracket, else doubles beta (no upper end yet) or
// halves the bracket; it stops when |H - log perplexity| <= tol.  Rows with
// #ties >= perplexity cannot reach the target: they get the beta -> infinity
// limit (uniform on the tied set, beta = +inf) and count in n_bad, as do rows
// out of iterations.
// ---------------------------------------------------------------------------
// Sum over the 16 lanes of this thread's half-warp.
__device__ __forceinline__ float half_sum(float x) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int KPL>
__global__ void __launch_bounds__(256)
calibrate_kernel(const float* __restrict__ d2, int64_t n, int k, float perp, float tol,
                 int max_iter, float* __restrict__ pc, float* __restrict__ beta_out,
                 unsigned long long* __restrict__ n_bad) {
  const int hl = threadIdx.x & 15;
  const int64_t i =
      ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 2 + ((threadIdx.x >> 4) & 1);
  if (__all_sync(0xffffffffu, i >= n)) return;
  const bool row = i < n;
  float s[KPL];
  bool v[KPL];
  float dmin = INFINITY;
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    const int a = hl + 16 * m;
    v[m] = row && a < k;
    s[m] = v[m] ? d2[i * k + a] : 0.f;
    if (v[m]) dmin = fminf(dmin, s[m]);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  float ties = 0.f;
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    s[m] = v[m] ? s[m] - dmin : 0.f;
    ties += (v[m] && s[m] == 0.f) ? 1.f : 0.f;
  }
  ties = half_sum(ties);

  const float target = logf(perp);
  float beta = 1.f;
  bool bad = false;
  // act: this half-warp's row still searches; the loop runs while either does
  bool act = row;
  if (row && ties >= perp) {
    beta = INFINITY;
    bad = true;
    act = false;
  }
  bool done = false;
  float lo = 0.f, hi = INFINITY;
  for (int it = 0; it < max_iter && __any_sync(0xffffffffu, act); it++) {
    float S = 0.f, M = 0.f, Q = 0.f;
#pragma unroll
    for (int m = 0; m < KPL; m++) {
      const float w = v[m] && act ? expf(-beta * s[m]) : 0.f;
      const float ws = w * s[m];
      S += w;
      M += ws;
      Q = fmaf(ws, s[m], Q);
    }
    S = half_sum(S);
    M = half_sum(M);
    Q = half_sum(Q);
    if (act) {
      const float H = logf(S) + beta * M / S;
      if (fabsf(H - target) <= tol) {
        done = true;
        act = false;
      } else {
        if (H > target) lo = beta; else hi = beta;
        const float E = M / S;
        const float var = Q / S - E * E;
        float nb = beta + (H - target) / (beta * var);  // Newton: dH/dbeta = -beta var
        if (!(nb > lo && nb < hi)) nb = isinf(hi) ? 2.f * beta : 0.5f * (lo + hi);
        if (nb == beta) act = false;  // bracket at FP32 resolution
        else beta = nb;
      }
    }
  }
  if (row && !isinf(beta)) bad = !done;
  // conditional probabilities at the final beta
  float w[KPL];
  float S = 0.f;
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    if (isinf(beta)) w[m] = (v[m] && s[m] == 0.f) ? 1.f : 0.f;
    else w[m] = v[m] ? expf(-beta * s[m]) : 0.f;
    S += w[m];
  }
  S = half_sum(S);
  if (!row) return;
  const float inv = 1.f / S;
#pragma unroll
  for (int m = 0; m < KPL; m++)
    if (v[m]) pc[i * k + hl + 16 * m] = w[m] * inv;
  if (hl == 0) {
    if (beta_out) beta_out[i] = beta;
    if (bad && n_bad) atomicAdd(n_bad, 1ull);
  }
}

cudaError_t launch_calibrate(const float* d2, int64_t n, int k, float perp, float tol,
                             int max_iter, float* pc, float* beta, int64_t* n_bad,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 15) / 16);  // 16 rows per 256-thread block
  unsigned long long* nb = reinterpret_cast<unsigned long long*>(n_bad);
#define TSNE_CALIBRATE(KPL) \
  calibrate_kernel<KPL><<<blocks, 256, 0, st>>>(d2, n, k, perp, tol, max_iter, pc, beta, nb)
  if (k <= 16) TSNE_CALIBRATE(1);
  else if (k <= 32) TSNE_CALIBRATE(2);
  else if (k <= 64) TSNE_CALIBRATE(4);
  else if (k <= 96) TSNE_CALIBRATE(6);
  else if (k <= 128) TSNE_CALIBRATE(8);
  else if (k <= 256) TSNE_CALIBRATE(16);
  else return cudaErrorInvalidValue;
#undef TSNE_CALIBRATE
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fuzzy neighbour graph (UMAP's fuzzy simplicial set; McInnes, Healy &
// Melville 2018, Sec. 3.1), one warp per row.  With d_j = sqrt(d2_j) the
// distances to the k neighbours, rho = the smallest positive d_j (0 if none)
// and x_j = max(0, d_j - rho):
//   f(sigma) = sum_j exp(-x_j / sigma) = log2(k)
// by bisection on sigma (start 1, double while f < target, then halve the
// bracket) to |f - log2 k| <= tol; w_j = exp(-x_j / sigma).  f increases from
// #(x_j = 0) to k, so rows with #(x_j = 0) >= log2 k take the sigma -> 0
// limit (w = 1 where x_j = 0, else 0; sigma = 0) and count in n_bad, as do
// rows out of iterations.
// ---------------------------------------------------------------------------
template <int KPL>
__global__ void __launch_bounds__(256)
fuzzy_calibrate_kernel(const float* __restrict__ d2, int64_t n, int k, float tol, int max_iter,
                       float* __restrict__ w_out, float* __restrict__ rho_out,
                       float* __restrict__ sigma_out, unsigned long long* __restrict__ n_bad) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  float x[KPL];
  bool v[KPL];
  float rmin = INFINITY;
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    const int a = lane + 32 * m;
    v[m] = a < k;
    x[m] = v[m] ? sqrtf(d2[i * k + a]) : 0.f;
    if (v[m] && x[m] > 0.f) rmin = fminf(rmin, x[m]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
  const float rho = isinf(rmin) ? 0.f : rmin;
  int zeros = 0;
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    x[m] = v[m] ? fmaxf(x[m] - rho, 0.f) : 0.f;
    zeros += (v[m] && x[m] == 0.f) ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  const float target = log2f((float)k);
  float sigma = 0.f;
  bool bad = true;
  if ((float)zeros < target) {
    float s = 1.f, lo = 0.f, hi = INFINITY;
    for (int it = 0; it < max_iter; it++) {
      float f = 0.f;
#pragma unroll
      for (int m = 0; m < KPL; m++) f += v[m] ? expf(-x[m] / s) : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (fabsf(f - target) <= tol) {
        bad = false;
        break;
      }
      if (f > target) hi = s; else lo = s;
      const float ns = isinf(hi) ? 2.f * s : 0.5f * (lo + hi);
      if (ns == s) break;  // bracket at FP32 resolution
      s = ns;
    }
    sigma = s;
  }
#pragma unroll
  for (int m = 0; m < KPL; m++) {
    if (!v[m]) continue;
    const float w = sigma > 0.f ? expf(-x[m] / sigma) : (x[m] == 0.f ? 1.f : 0.f);
    w_out[i * k + lane + 32 * m] = w;
  }
  if (lane == 0) {
    if (rho_out) rho_out[i] = rho;
    if (sigma_out) sigma_out[i] = sigma;
    if (bad && n_bad) atomicAdd(n_bad, 1ull);
  }
}

cudaError_t launch_fuzzy_calibrate(const float* d2, int64_t n, int k, float tol, int max_iter,
                                   float* w, float* rho, float* sigma, int64_t* n_bad,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 7) / 8);
  unsigned long long* nb = reinterpret_cast<unsigned long long*>(n_bad);
  if (k <= 32)
    fuzzy_calibrate_kernel<1><<<blocks, 256, 0, st>>>(d2, n, k, tol, max_iter, w, rho, sigma, nb);
  else if (k <= 64)
    fuzzy_calibrate_kernel<2><<<blocks, 256, 0, st>>>(d2, n, k, tol, max_iter, w, rho, sigma, nb);
  else if (k <= 128)
    fuzzy_calibrate_kernel<4><<<blocks, 256, 0, st>>>(d2, n, k, tol, max_iter, w, rho, sigma, nb);
  else if (k <= 256)
    fuzzy_calibrate_kernel<8><<<blocks, 256, 0, st>>>(d2, n, k, tol, max_iter, w, rho, sigma, nb);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Symmetrisation.  Every conditional entry (i -> j, c) is emitted twice, as
// key (i, j) and key (j, i), with value c / (2 n_s); keys are row << bits | col,
// where 2^bits is the first power of two not below the batch's point count.
// After a stable radix sort the entries of one (row, col) are adjacent: their
// sum is p_ij (at most one copy from each direction), emitted once.  For the
// fuzzy graph the values are the membership strengths w (no scaling) and the
// two copies combine by the fuzzy union w_ij + w_ji - w_ij w_ji.
// A neighbour outside the row's sample, or the row itself, is an invalid
// index: it is flagged and emitted as the all-ones key, which sorts last and
// is dropped (a valid key cannot have its low 2 * bits bits all set, since
// that needs row = col).
// ---------------------------------------------------------------------------
constexpr uint64_t kDropKey = ~0ull;

// A warp per row (blocks of kEmitRows rows never straddle a sample): the lanes
// take the row's k entries, so the reads of idx / pc and the writes of the key
// pairs are contiguous across the warp.
constexpr int kEmitRows = 8;

__global__ void __launch_bounds__(32 * kEmitRows)
sym_emit_kernel(const int32_t* __restrict__ idx, const float* __restrict__ pc, int k, int bits,
                const __grid_constant__ SampleTable tab, int fuzzy, uint64_t* __restrict__ keys,
                float* __restrict__ vals, int32_t* status) {
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t i = p0 + (int64_t)(b - tab.blk_off[s]) * kEmitRows + (threadIdx.x >> 5);
  if (i >= p1) return;
  const float scale = fuzzy ? 1.f : 0.5f / (float)(p1 - p0);
  bool bad = false;
  for (int a = threadIdx.x & 31; a < k; a += 32) {
    const int64_t e = i * k + a;
    const int64_t j = idx[e];
    const float c = pc[e] * scale;
    if (j < p0 || j >= p1 || j == i) {
      bad = true;
      reinterpret_cast<ulonglong2*>(keys)[e] = make_ulonglong2(kDropKey, kDropKey);
      reinterpret_cast<float2*>(vals)[e] = make_float2(0.f, 0.f);
      continue;
    }
    reinterpret_cast<ulonglong2*>(keys)[e] =
        make_ulonglong2(((uint64_t)i << bits) | (uint64_t)j, ((uint64_t)j << bits) | (uint64_t)i);
    reinterpret_cast<float2*>(vals)[e] = make_float2(c, c);
  }
  if (bad) raise_status(status, TSNE_STATUS_BAD_INDEX);
}

// The sorted keys are cut into tiles of kSymTile; a head is the first key of a
// run of equal valid keys (at most two: one from each direction).
//   count:   heads per tile, and per row (one atomic add per (warp, row): the
//            keys are sorted by row, so a warp's heads mostly share one);
//   compact: with the tiles' exclusive scan, each head's output slot is its
//            tile's offset + the heads before it in the tile (warp ballots in
//            input order, warps in order); its value merges the run.
constexpr int kSymThreads = 256;
constexpr int kSymPerThread = 16;
constexpr int kSymTile = kSymThreads * kSymPerThread;
constexpr int kSymPerWarp = kSymTile / (kSymThreads / 32);  // 512 consecutive keys per warp

int64_t sym_tiles(int64_t m) { return (m + kSymTile - 1) / kSymTile; }

__device__ __forceinline__ bool sym_is_head(const uint64_t* keys, int64_t e, uint64_t key) {
  return key != kDropKey && (e == 0 || keys[e - 1] != key);
}

__global__ void __launch_bounds__(kSymThreads)
sym_count_kernel(const uint64_t* __restrict__ keys, int64_t m, int bits,
                 uint32_t* __restrict__ tile_cnt, uint32_t* __restrict__ row_cnt) {
  __shared__ uint32_t wsum[kSymThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSymTile + (int64_t)w * kSymPerWarp;
  uint32_t c = 0;
#pragma unroll 4
  for (int r = 0; r < kSymPerWarp / 32; r++) {
    const int64_t e = base + r * 32 + lane;
    bool h = false;
    uint32_t row = 0xffffffffu;
    if (e < m) {
      const uint64_t key = keys[e];
      h = sym_is_head(keys, e, key);
      if (h) row = (uint32_t)(key >> bits);
    }
    c += h ? 1u : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, row);
    if (h && lane == __ffs(peers) - 1) atomicAdd(&row_cnt[row], __popc(peers));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) wsum[w] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < kSymThreads / 32; k++) t += wsum[k];
    tile_cnt[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kSymThreads)
sym_compact_kernel(const uint64_t* __restrict__ keys, const float* __restrict__ vals, int64_t m,
                   int bits, const uint32_t* __restrict__ tile_off, int32_t* __restrict__ col,
                   float* __restrict__ val, int64_t cap, int fuzzy, int32_t* status) {
  constexpr int R = kSymPerWarp / 32;
  __shared__ uint32_t wsum[kSymThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSymTile + (int64_t)w * kSymPerWarp;
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t hmask[R];
  uint32_t c = 0;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t e = base + r * 32 + lane;
    const bool h = e < m && sym_is_head(keys, e, keys[e]);
    hmask[r] = __ballot_sync(0xffffffffu, h);
    c += __popc(hmask[r]);
  }
  if (lane == 0) wsum[w] = c;
  __syncthreads();
  uint32_t slot = tile_off[blockIdx.x];
  for (int k = 0; k < w; k++) slot += wsum[k];
  bool over = false;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t e = base + r * 32 + lane;
    if ((hmask[r] >> lane) & 1u) {
      const uint64_t key = keys[e];
      float v = vals[e];
      for (int64_t f = e + 1; f < m && keys[f] == key; f++) {
        const float u = vals[f];
        v = fuzzy ? (v + u) - v * u : v + u;  // fuzzy union a + b - ab, or the sum
      }
      const int64_t p = (int64_t)slot + __popc(hmask[r] & lt);
      if (p >= cap) {
        over = true;
      } else {
        col[p] = (int32_t)(key & ((1ull << bits) - 1ull));
        val[p] = v;
      }
    }
    slot += __popc(hmask[r]);
  }
  if (over) raise_status(status, TSNE_STATUS_CAPACITY);
}

__global__ void u32_to_i64_kernel(const uint32_t* __restrict__ in, int64_t m,
                                  int64_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) out[e] = (int64_t)in[e];
}

int64_t radix_tiles(int64_t m);
int64_t scan_parts_len(int64_t m);
cudaError_t launch_radix_sort(uint64_t* k0, float* v0, uint64_t* k1, float* v1, int64_t m,
                              const int* bit_lo, const int* bit_hi, int nranges, uint32_t* hist,
                              uint32_t* part, uint64_t** k_res, float** v_res, cudaStream_t st);

// Workspace of the symmetrisation for n points and k neighbours (m = 2nk).
struct SymWs {
  uint64_t* k0; uint64_t* k1; float* v0; float* v1;
  uint32_t* hist; uint32_t* part; uint32_t* head; uint32_t* row_cnt;
};

cudaError_t launch_symmetrize(const int32_t* idx, const float* pc, int64_t n, int k,
                              const SampleTable& tab, const SymWs& w, int64_t* row_ptr,
                              int32_t* col, float* val, int64_t cap, int fuzzy, int32_t* status,
                              cudaStream_t st) {
  const int64_t m = 2 * n * (int64_t)k;
  if (n <= 0) return cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st);
  // key = (row << bits) | column, with row and column below 2^bits
  int bits = 1;
  while ((1ll << bits) < n) bits++;
  {
    SampleTable* te = new SampleTable(tab);
    int32_t nb = 0;
    for (int s = 0; s < tab.S; s++) {
      te->blk_off[s] = nb;
      nb += (int32_t)((tab.pt_off[s + 1] - tab.pt_off[s] + kEmitRows - 1) / kEmitRows);
    }
    te->blk_off[tab.S] = nb;
    te->blk_pts = kEmitRows;
    sym_emit_kernel<<<nb, 32 * kEmitRows, 0, st>>>(idx, pc, k, bits, *te, fuzzy, w.k0, w.v0,
                                                   status);
    delete te;
  }
  // one range of 2 * bits key bits: 5 passes of 8-bit digits at 200k or 1M
  // points (two 32-bit halves of bits each would take 6)
  const int lo[1] = {0};
  const int hi[1] = {2 * bits};
  uint64_t* ks;
  float* vs;
  cudaError_t e = launch_radix_sort(w.k0, w.v0, w.k1, w.v1, m, lo, hi, 1, w.hist, w.part, &ks,
                                    &vs, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.row_cnt, 0, sizeof(uint32_t) * (size_t)(n + 1), st);
  if (e != cudaSuccess) return e;
  const int64_t ntile = sym_tiles(m);
  sym_count_kernel<<<(unsigned)ntile, kSymThreads, 0, st>>>(ks, m, bits, w.head, w.row_cnt);
  e = launch_scan_u32(w.head, w.head, ntile, w.part, st);
  if (e != cudaSuccess) return e;
  sym_compact_kernel<<<(unsigned)ntile, kSymThreads, 0, st>>>(ks, vs, m, bits, w.head, col, val,
                                                              cap, fuzzy, status);
  e = launch_scan_u32(w.row_cnt, w.row_cnt, n + 1, w.part, st);
  if (e != cudaSuccess) return e;
  u32_to_i64_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(w.row_cnt, n + 1, row_ptr);
  return cudaGetLastError();
}

}  // namespace tsne
