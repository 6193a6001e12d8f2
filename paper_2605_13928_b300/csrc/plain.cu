// plain.cu -- the plain GPU form of the exact t-SNE gradient, kept as the
// comparison baseline for the tiled path: one thread per row, operands read
// straight from global memory, FP32 accumulation, IEEE division, and one
// kernel per term (Z and repulsion, attraction, combination), no tiling.
//   Fr_i = sum_{j != i} w_ij^2 (y_i - y_j),  Z_i = sum_{j != i} w_ij,
//   Fa_i = sum_j p_ij w_ij (y_i - y_j),      g_i = 4 (alpha Fa_i - Fr_i / Z)
// (van der Maaten & Hinton 2008, Eq. 5).
#include "common.cuh"

namespace tsne {

__global__ void plain_repulse_kernel(const float2* __restrict__ Y, const int64_t* __restrict__ seg,
                                     int64_t n, float2* __restrict__ Fr, float* __restrict__ Zi) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j0 = seg[2 * i], j1 = seg[2 * i + 1];
  const float2 yi = Y[i];
  float fx = 0.f, fy = 0.f, z = 0.f;
  for (int64_t j = j0; j < j1; j++) {
    if (j == i) continue;
    const float2 yj = Y[j];
    const float dx = yi.x - yj.x, dy = yi.y - yj.y;
    const float w = 1.0f / (1.0f + dx * dx + dy * dy);
    z += w;
    fx += w * w * dx;
    fy += w * w * dy;
  }
  Fr[i] = make_float2(fx, fy);
  Zi[i] = z;
}

__global__ void plain_attract_kernel(const int64_t* __restrict__ row_ptr,
                                     const int32_t* __restrict__ col,
                                     const float* __restrict__ val, int64_t n, int64_t cap,
                                     const float2* __restrict__ Y, float2* __restrict__ Fa,
                                     int32_t* status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t e0 = row_ptr[i], e1 = row_ptr[i + 1];
  if (e0 < 0 || e1 < e0 || e1 > cap) {
    raise_status(status, TSNE_STATUS_BAD_INDEX);
    e0 = e1 = 0;
  }
  const float2 yi = Y[i];
  float fx = 0.f, fy = 0.f;
  for (int64_t e = e0; e < e1; e++) {
    const int32_t j = col[e];
    if ((uint64_t)(int64_t)j >= (uint64_t)n) {
      raise_status(status, TSNE_STATUS_BAD_INDEX);
      continue;
    }
    const float2 yj = Y[j];
    const float dx = yi.x - yj.x, dy = yi.y - yj.y;
    const float w = 1.0f / (1.0f + dx * dx + dy * dy);
    fx += val[e] * w * dx;
    fy += val[e] * w * dy;
  }
  Fa[i] = make_float2(fx, fy);
}

// Z_s = sum of Z_i over the sample, one CTA per sample (FP64, fixed order).
__global__ void plain_z_kernel(const float* __restrict__ Zi, const __grid_constant__ SampleTable tab,
                               double* __restrict__ Z) {
  __shared__ double sh[256];
  const int s = blockIdx.x;
  double z = 0.0;
  for (int64_t i = tab.pt_off[s] + threadIdx.x; i < tab.pt_off[s + 1]; i += blockDim.x)
    z += (double)Zi[i];
  sh[threadIdx.x] = z;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) Z[s] = sh[0];
}

__global__ void plain_grad_kernel(const float2* __restrict__ Fa, const float2* __restrict__ Fr,
                                  const double* __restrict__ Z, const int32_t* __restrict__ sid,
                                  int64_t n, float alpha, float2* __restrict__ grad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z = (float)Z[sid[i]];
  const float2 a = Fa[i], r = Fr[i];
  grad[i] = make_float2(4.f * (alpha * a.x - r.x / z), 4.f * (alpha * a.y - r.y / z));
}

// Plain optimiser update, one thread per point: the gains / momentum / position
// rule of the tiled path (van der Maaten & Hinton 2008, Sec. 3.4), reading the
// gradient written by plain_grad_kernel.
__global__ void plain_update_kernel(const float2* __restrict__ grad,
                                    const int64_t* __restrict__ seg, int64_t n, float alpha_unused,
                                    float mu, float lr, float min_gain, float2* __restrict__ Y,
                                    float2* __restrict__ U, float2* __restrict__ G,
                                    int32_t* status) {
  (void)alpha_unused;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float eta = lr > 0.f ? lr : (float)(seg[2 * i + 1] - seg[2 * i]) / 12.0f;
  const float2 g = grad[i];
  float2 u = U[i], gn = G[i], y = Y[i];
  float gx = (g.x * u.x < 0.f) ? gn.x + 0.2f : gn.x * 0.8f;
  float gy = (g.y * u.y < 0.f) ? gn.y + 0.2f : gn.y * 0.8f;
  gx = fmaxf(gx, min_gain);
  gy = fmaxf(gy, min_gain);
  u.x = mu * u.x - eta * gx * g.x;
  u.y = mu * u.y - eta * gy * g.y;
  y.x += u.x;
  y.y += u.y;
  if (!(isfinite(y.x) && isfinite(y.y))) raise_status(status, TSNE_STATUS_NONFINITE);
  U[i] = u;
  G[i] = make_float2(gx, gy);
  Y[i] = y;
}

// Per-point sample segment [j0, j1) and sample id, written once per call.
__global__ void plain_seg_kernel(const __grid_constant__ SampleTable tab, int64_t n,
                                 int64_t* __restrict__ seg, int32_t* __restrict__ sid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = tab.S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab.pt_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  seg[2 * i] = tab.pt_off[lo];
  seg[2 * i + 1] = tab.pt_off[lo + 1];
  sid[i] = lo;
}

cudaError_t launch_plain(const tsne_csr& P, const SampleTable& tab, const float2* Y, float alpha,
                         float2* grad, double* Z, float2* Fa, float2* Fr, float* Zi,
                         int64_t* seg, int32_t* sid, int32_t* status, cudaStream_t st) {
  const int64_t n = P.n;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  plain_seg_kernel<<<blocks, 256, 0, st>>>(tab, n, seg, sid);
  plain_repulse_kernel<<<blocks, 256, 0, st>>>(Y, seg, n, Fr, Zi);
  plain_attract_kernel<<<blocks, 256, 0, st>>>(P.row_ptr, P.col, P.val, n, P.cap, Y, Fa, status);
  plain_z_kernel<<<tab.S, 256, 0, st>>>(Zi, tab, Z);
  if (grad) plain_grad_kernel<<<blocks, 256, 0, st>>>(Fa, Fr, Z, sid, n, alpha, grad);
  return cudaGetLastError();
}

// One plain optimiser iteration: the plain gradient at exaggeration alpha, then
// the plain update with momentum mu.
cudaError_t launch_plain_step(const tsne_csr& P, const SampleTable& tab, float2* Y, float2* U,
                              float2* G, float alpha, float mu, float lr, float min_gain,
                              float2* grad, double* Z, float2* Fa, float2* Fr, float* Zi,
                              int64_t* seg, int32_t* sid, int32_t* status, cudaStream_t st) {
  cudaError_t e = launch_plain(P, tab, Y, alpha, grad, Z, Fa, Fr, Zi, seg, sid, status, st);
  if (e != cudaSuccess) return e;
  const int64_t n = P.n;
  plain_update_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(grad, seg, n, alpha, mu, lr,
                                                                     min_gain, Y, U, G, status);
  return cudaGetLastError();
}

}  // namespace tsne
