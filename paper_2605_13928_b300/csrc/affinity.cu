// affinity.cu -- t-SNE input affinities on the kNN graph
// (van der Maaten & Hinton 2008, Sec. 2; sparse form of van der Maaten 2014,
// Sec. 3):
//   p_{j|i} = exp(-beta_i d2_ij) / sum_l exp(-beta_i d2_il) over the k
//   neighbours, beta_i chosen so that H_i = -sum_j p_{j|i} log p_{j|i} equals
//   log(perplexity); then P = (P_cond + P_cond^T) / (2 n_s) (symmetrize.cu).
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

}  // namespace tsne
