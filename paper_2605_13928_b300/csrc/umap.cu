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
#include <math.h>

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

// ---------------------------------------------------------------------------
// Initial layout from PCA scores: U = the first two score columns, centred
// (FP64 means) and scaled so that the larger coordinate range is [-10, 10]
// (max |U| = 10).  Fixed grid (kInitBlocks blocks, grid-stride loops) and
// fixed-order reductions, so the result does not depend on the device.
// ---------------------------------------------------------------------------
constexpr int kInitBlocks = 512;

__global__ void __launch_bounds__(256)
umap_init_sum_kernel(const float* __restrict__ S, int64_t n, int64_t ld,
                     double2* __restrict__ part) {
  __shared__ double sx[256], sy[256];
  double ax = 0.0, ay = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kInitBlocks * 256) {
    ax += (double)S[i * ld];
    ay += (double)S[i * ld + 1];
  }
  sx[threadIdx.x] = ax;
  sy[threadIdx.x] = ay;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(sx[0], sy[0]);
}

// one block: the means from the partial sums (fixed order), then, after
// umap_init_max_kernel, the scale
__global__ void __launch_bounds__(256)
umap_init_mean_kernel(const double2* __restrict__ part, int64_t n, double2* __restrict__ mean) {
  if (threadIdx.x == 0) {
    double ax = 0.0, ay = 0.0;
    for (int b = 0; b < kInitBlocks; b++) {
      ax += part[b].x;
      ay += part[b].y;
    }
    *mean = make_double2(ax / (double)n, ay / (double)n);
  }
}

__global__ void __launch_bounds__(256)
umap_init_center_kernel(const float* __restrict__ S, int64_t n, int64_t ld,
                        const double2* __restrict__ mean, float2* __restrict__ U,
                        float* __restrict__ pmax) {
  __shared__ float sm[256];
  const float mx = (float)mean->x, my = (float)mean->y;
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kInitBlocks * 256) {
    const float2 u = make_float2(S[i * ld] - mx, S[i * ld + 1] - my);
    U[i] = u;
    m = fmaxf(m, fmaxf(fabsf(u.x), fabsf(u.y)));
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sm[threadIdx.x] = fmaxf(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) pmax[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(256)
umap_init_scale_kernel(float2* __restrict__ U, int64_t n, const float* __restrict__ pmax,
                       int32_t* status) {
  __shared__ float scale;
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int b = 0; b < kInitBlocks; b++) m = fmaxf(m, pmax[b]);
    scale = 10.0f / fmaxf(m, 1e-30f);
    if (!isfinite(m)) raise_status(status, TSNE_STATUS_NONFINITE);
  }
  __syncthreads();
  const float c = scale;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)kInitBlocks * 256) {
    const float2 u = U[i];
    U[i] = make_float2(u.x * c, u.y * c);
  }
}

size_t umap_init_ws_bytes() {
  return sizeof(double2) * (kInitBlocks + 1) + sizeof(float) * kInitBlocks + 256;
}

cudaError_t launch_umap_init(const float* S, int64_t n, int64_t ld, float2* U, void* ws,
                             int32_t* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  double2* part = static_cast<double2*>(ws);
  double2* mean = part + kInitBlocks;
  float* pmax = reinterpret_cast<float*>(mean + 1);
  umap_init_sum_kernel<<<kInitBlocks, 256, 0, st>>>(S, n, ld, part);
  umap_init_mean_kernel<<<1, 32, 0, st>>>(part, n, mean);
  umap_init_center_kernel<<<kInitBlocks, 256, 0, st>>>(S, n, ld, mean, U, pmax);
  umap_init_scale_kernel<<<kInitBlocks, 256, 0, st>>>(U, n, pmax, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// (a, b) of the low-dimensional membership 1 / (1 + a d^(2b)) (McInnes, Healy &
// Melville 2018, Sec. 3.2): the least-squares fit to Psi(d) = 1 for
// d < min_dist and exp(-(d - min_dist) / spread) beyond, on 300 evenly spaced
// d in [0, 3 spread] (d = 0 contributes 1 - 1 = 0 at any (a, b) and is left
// out).  Levenberg-Marquardt in FP64 on the host from (a, b) = (1, 1): damping
// lambda diag(J^T J); a step that keeps a, b > 0 and lowers the squared
// residual is kept (lambda x 0.3), any other is rejected (lambda x 10).
// ---------------------------------------------------------------------------
int umap_fit_ab(double min_dist, double spread, double* a_out, double* b_out) {
  constexpr int M = 299;
  double x[M], t[M], lx[M];
  for (int k = 0; k < M; k++) {
    const double d = 3.0 * spread * (double)(k + 1) / 299.0;
    x[k] = d;
    lx[k] = log(d);
    t[k] = d < min_dist ? 1.0 : exp(-(d - min_dist) / spread);
  }
  // residual r = f - t and its Jacobian rows (df/da, df/db); returns sum r^2
  auto eval = [&](double a, double b, double* r, double (*J)[2]) {
    double c = 0.0;
    for (int k = 0; k < M; k++) {
      const double xb = exp(2.0 * b * lx[k]);
      const double f = 1.0 / (1.0 + a * xb);
      r[k] = f - t[k];
      J[k][0] = -xb * f * f;
      J[k][1] = -a * xb * 2.0 * lx[k] * f * f;
      c += r[k] * r[k];
    }
    return c;
  };
  static thread_local double r[M], J[M][2], r2[M], J2[M][2];
  double a = 1.0, b = 1.0, lam = 1e-3;
  double cost = eval(a, b, r, J);
  for (int iter = 0; iter < 100; iter++) {
    double A00 = 0, A01 = 0, A11 = 0, g0 = 0, g1 = 0;
    for (int k = 0; k < M; k++) {
      A00 += J[k][0] * J[k][0];
      A01 += J[k][0] * J[k][1];
      A11 += J[k][1] * J[k][1];
      g0 += J[k][0] * r[k];
      g1 += J[k][1] * r[k];
    }
    // (A + lam diag A) step = -g, by Cramer's rule
    const double B00 = A00 * (1.0 + lam), B11 = A11 * (1.0 + lam), B01 = A01;
    const double det = B00 * B11 - B01 * B01;
    bool accepted = false;
    if (det != 0.0 && isfinite(det)) {
      const double s0 = (-g0 * B11 + g1 * B01) / det;
      const double s1 = (-g1 * B00 + g0 * B01) / det;
      const double a2 = a + s0, b2 = b + s1;
      if (a2 > 0.0 && b2 > 0.0) {
        const double c2 = eval(a2, b2, r2, J2);
        if (c2 < cost) {
          a = a2;
          b = b2;
          cost = c2;
          for (int k = 0; k < M; k++) {
            r[k] = r2[k];
            J[k][0] = J2[k][0];
            J[k][1] = J2[k][1];
          }
          lam *= 0.3;
          accepted = true;
          if (fmax(fabs(s0), fabs(s1)) < 1e-12 * fmax(a, b)) break;
        }
      }
    }
    if (!accepted) {
      lam *= 10.0;
      if (lam > 1e12) break;
    }
  }
  if (!(a > 0.0) || !(b > 0.0) || !isfinite(a) || !isfinite(b)) return TSNE_ERR_NOT_CONVERGED;
  *a_out = a;
  *b_out = b;
  return TSNE_OK;
}

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
