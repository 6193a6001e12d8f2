// umap.cu -- UMAP layout optimisation on the fuzzy neighbour graph
// (McInnes, Healy & Melville 2018, Sec. 3.2 and their embedding optimisation
// algorithm): stochastic gradient steps on the fuzzy-set cross entropy with
// edge sampling by weight and negative sampling.
//
// Low-dimensional membership Phi(d) = 1 / (1 + a d^(2b)).  Epoch e of n_epochs
// (learning rate alpha_e = alpha0 (1 - e / n_epochs)): every directed entry q =
// (i, j) of the symmetric graph, of weight p, is taken with probability p; a
// taken entry adds to point i
//   clip(-2ab d^(2b-2) / (1 + a d^(2b)) (y_i - y_j))              (0 if d = 0)
// and, for each of n_neg vertices c drawn uniformly from i's sample (c != i),
//   clip(2b / ((1e-3 + d^2) (1 + a d^(2b))) (y_i - y_c)),
// each coordinate clipped to [-4, 4].  Epochs are synchronous: the terms use
// the positions at the start of the epoch and y_i += alpha_e (their sum) at its
// end, so an epoch is a pure function of its input and needs no atomics: only
// the row's own point moves.
//
// Draws are counter-based (splitmix64, Steele, Lea & Flood 2014): for epoch e,
// entry q and draw s (0: the entry's own draw, 1..n_neg: its negatives),
// h = splitmix64((e << 40) + (q << 4) + s  xor  seed); the entry is taken when
// (h >> 40) 2^-24 < p (24-bit uniform, exact in FP32), and negative s is vertex
// p0 + ((h >> 32) n_s >> 32) of the sample [p0, p0 + n_s).
//
// d^(2b) is __powf(d^2, b), the hardware exp2(b log2 d^2), and the coefficients
// use the fast division __fdividef (2 ulp): about 1e-7 relative error per term.
//
// Layout: one warp per point i.  The row's entries are taken 32 at a time: each
// lane makes one entry's draw (coalesced CSR reads), the taken entries are
// compacted in entry order, and their terms (1 + n_neg each) are spread over
// all 32 lanes, so a warp gathers up to 32 positions at once whatever the
// sampling left.  Each lane sums its terms in FP32 in a fixed order and a fixed
// butterfly adds the lanes.  Y is double-buffered (read Y, write Yout).
#include "common.cuh"

namespace tsne {

constexpr int kUmapWarps = 8;  // points per 256-thread block

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t umap_draw(uint64_t seed, int e, int64_t q, int s) {
  const uint64_t t = ((uint64_t)e << 40) + ((uint64_t)q << 4) + (uint64_t)s;
  return splitmix64(t ^ seed);
}

__device__ __forceinline__ float clip4(float v) { return fminf(fmaxf(v, -4.f), 4.f); }

__global__ void __launch_bounds__(32 * kUmapWarps)
umap_epoch_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                  const float* __restrict__ w, const float2* __restrict__ Y,
                  float2* __restrict__ Yout, const __grid_constant__ SampleTable tab, int e,
                  float alpha, float a, float b, int n_neg, uint64_t seed, int32_t* status) {
  const int blk = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, blk);
  const int lane = threadIdx.x & 31;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1], ns = p1 - p0;
  const int64_t i = p0 + (int64_t)(blk - tab.blk_off[s]) * kUmapWarps + (threadIdx.x >> 5);
  if (i >= p1) return;  // whole warp
  const float2 yi = Y[i];
  const int64_t n = tab.pt_off[tab.S];
  const float two_ab = 2.f * a * b, two_b = 2.f * b;
  float dx = 0.f, dy = 0.f;
  bool bad = false;
  __shared__ int64_t taken_q[kUmapWarps][32];
  int64_t* tq = taken_q[threadIdx.x >> 5];
  const int per = 1 + n_neg;  // terms per taken entry
  // t / per as (t M) >> 16, M = ceil(2^16 / per): exact for t < 512 since the
  // error t (M - 2^16 / per) / 2^16 < 1/128 stays below 1/per (per <= 16)
  const uint32_t M = (65536u + (uint32_t)per - 1u) / (uint32_t)per;
  const int64_t q1 = rp[i + 1];
  for (int64_t base = rp[i]; base < q1; base += 32) {
    // the draws of up to 32 entries, then the taken ones compacted in entry order
    const int64_t q = base + lane;
    bool tk = false;
    if (q < q1) {
      const uint64_t h0 = umap_draw(seed, e, q, 0);
      tk = (float)(uint32_t)(h0 >> 40) * 0x1p-24f < w[q];
    }
    const uint32_t m = __ballot_sync(0xffffffffu, tk);
    if (tk) tq[__popc(m & ((1u << lane) - 1u))] = q;
    __syncwarp();
    // the chunk's terms (entry k, term s: s = 0 its attraction, 1..n_neg its
    // negatives) spread over the lanes: term t = k (1 + n_neg) + s goes to lane t % 32
    const int nt = __popc(m) * per;
    for (int t = lane; t < nt; t += 32) {
      const int k = (int)(((uint32_t)t * M) >> 16), sd = t - k * per;
      const int64_t qk = tq[k];
      if (sd == 0) {
        const int32_t j = col[qk];
        if (j < 0 || (int64_t)j >= n) {
          bad = true;
          continue;
        }
        const float2 yj = Y[j];
        const float ex = yi.x - yj.x, ey = yi.y - yj.y;
        const float d2 = fmaf(ex, ex, ey * ey);
        if (d2 > 0.f) {
          const float pb = __powf(d2, b);
          const float coef = -two_ab * __fdividef(pb, d2 * fmaf(a, pb, 1.f));
          dx += clip4(coef * ex);
          dy += clip4(coef * ey);
        }
      } else {
        const uint64_t h = umap_draw(seed, e, qk, sd);
        // (h >> 32) n_s >> 32 as one high-half multiply (n_s < 2^31)
        const int64_t c = p0 + (int64_t)__umulhi((uint32_t)(h >> 32), (uint32_t)ns);
        if (c == i) continue;
        const float2 yc = Y[c];
        const float ex = yi.x - yc.x, ey = yi.y - yc.y;
        const float d2 = fmaf(ex, ex, ey * ey);
        const float pb = __powf(d2, b);
        const float coef = __fdividef(two_b, (1e-3f + d2) * fmaf(a, pb, 1.f));
        dx += clip4(coef * ex);
        dy += clip4(coef * ey);
      }
    }
    __syncwarp();  // the list is read before the next chunk overwrites it
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dx += __shfl_xor_sync(0xffffffffu, dx, o);
    dy += __shfl_xor_sync(0xffffffffu, dy, o);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(status, TSNE_STATUS_BAD_INDEX);
  if (lane == 0) {
    const float2 y = make_float2(fmaf(alpha, dx, yi.x), fmaf(alpha, dy, yi.y));
    if (!(isfinite(y.x) && isfinite(y.y))) raise_status(status, TSNE_STATUS_NONFINITE);
    Yout[i] = y;
  }
}

int umap_block_points() { return kUmapWarps; }

// Epochs epoch0 .. epoch0 + n_run - 1 of an n_epochs schedule; Y in/out,
// scratch n float2.  tab: blocks of kUmapWarps points (blk_off) per sample.
cudaError_t launch_umap_layout(const int64_t* rp, const int32_t* col, const float* w, float2* Y,
                               float2* scratch, const SampleTable& tab, int n_epochs, int epoch0,
                               int n_run, float a, float b, float alpha0, int n_neg,
                               uint64_t seed, int32_t* status, cudaStream_t st) {
  const int64_t n = tab.pt_off[tab.S];
  const unsigned grid = (unsigned)tab.blk_off[tab.S];
  if (n <= 0 || n_run <= 0 || grid == 0) return cudaSuccess;
  float2* src = Y;
  float2* dst = scratch;
  for (int r = 0; r < n_run; r++) {
    const int e = epoch0 + r;
    const float alpha = (float)((double)alpha0 * (1.0 - (double)e / (double)n_epochs));
    umap_epoch_kernel<<<grid, 32 * kUmapWarps, 0, st>>>(rp, col, w, src, dst, tab, e, alpha, a,
                                                          b, n_neg, seed, status);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    float2* t = src;
    src = dst;
    dst = t;
  }
  if (src != Y) return cudaMemcpyAsync(Y, src, sizeof(float2) * (size_t)n,
                                       cudaMemcpyDeviceToDevice, st);
  return cudaSuccess;
}

}  // namespace tsne
