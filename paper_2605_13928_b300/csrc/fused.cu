// fused.cu -- one persistent launch per optimiser iteration for a batch of
// independent samples (many uneven embeddings at once).
//
// A fixed grid (resident CTAs only) pulls direct-form work items (sample, row
// tile, column chunk; repulse_item.cuh) from an atomic queue.  The first
// chunk of every row tile also computes the attraction of its rows (one warp
// per row over the CSR row of P).  When a CTA finishes an item it counts it
// for its sample; the CTA that completes a sample's last item finalises that
// sample on the spot: Z_s (FP64, fixed order over the sample's items), the KL
// value when due, and the gradient / gains / momentum / position update of
// all the sample's points.  No CTA ever waits for another: completion is
// detected by integer counters only, so the launch needs no grid barrier and
// cannot deadlock whatever the number of resident CTAs.  Results do not depend
// on which CTA processes which item (every item writes fixed locations and
// every reduction runs in a fixed order).  Data written by other CTAs in the
// same launch is read with ld.global.cg (L2, not the incoherent L1).
//
// The counters (queue head, per-sample completions, exited CTAs) are zeroed
// by a memset node before each launch; in device-counter mode the last CTA to
// exit advances the iteration counter.
#include "repulse_item.cuh"

namespace tsne {


template <int THREADS>
__device__ __forceinline__ double fused_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < THREADS / 32; k++) t += sh[k];  // every thread gets the total
  return t;
}

// Attraction Fa_i = sum_j p_ij w_ij (y_i - y_j) of rows [r0, r1), warp per row
// (same arithmetic as attract_kernel); KL row terms when due.
template <int THREADS>
__device__ __forceinline__ void fused_attract(const FusedArgs& a, int64_t r0, int64_t r1,
                                              bool kl_now) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = a.P.n;
  for (int64_t i = r0 + w; i < r1; i += THREADS / 32) {
    int64_t e0 = a.P.row_ptr[i], e1 = a.P.row_ptr[i + 1];
    if (e0 < 0 || e1 < e0 || e1 > a.P.cap) {
      if (lane == 0) raise_status(a.status, TSNE_STATUS_BAD_INDEX);
      e0 = e1 = 0;
    }
    const float2 yi = a.Y[i];
    float fx = 0.f, fy = 0.f;
    double ka = 0.0, kb = 0.0;
    bool bad = false;
    for (int64_t e = e0 + lane; e < e1; e += 32) {
      const int32_t j = a.P.col[e];
      if ((uint64_t)(int64_t)j >= (uint64_t)n) { bad = true; continue; }
      const float p = a.P.val[e];
      const float2 yj = a.Y[j];
      const float dx = yi.x - yj.x, dy = yi.y - yj.y;
      const float d2 = fmaf(dx, dx, dy * dy);
      const float wv = 1.0f / (1.0f + d2);
      const float pw = p * wv;
      fx = fmaf(pw, dx, fx);
      fy = fmaf(pw, dy, fy);
      if (kl_now && p > 0.f) {
        ka += (double)p * (double)logf(p);
        kb += (double)p * (double)log1pf(d2);
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(a.status, TSNE_STATUS_BAD_INDEX);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      fx += __shfl_down_sync(0xffffffffu, fx, o);
      fy += __shfl_down_sync(0xffffffffu, fy, o);
      ka += __shfl_down_sync(0xffffffffu, ka, o);
      kb += __shfl_down_sync(0xffffffffu, kb, o);
    }
    if (lane == 0) {
      a.Fa[i] = make_float2(fx, fy);
      if (kl_now) a.klrow[i] = make_double2(ka, kb);
    }
  }
}

// Z_s, KL_s and the update of every point of sample s (one CTA).
template <int THREADS>
__device__ void fused_finalize(const FusedArgs& a, const SampleTable& tab, int s, int it,
                               bool kl_now, double* sh) {
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1], ns = p1 - p0;
  double z = 0.0;
  for (int64_t k = tab.item_off[s] + threadIdx.x; k < tab.item_off[s + 1]; k += THREADS)
    z += __ldcg(&a.zpart[k]);
  const double Zs = fused_block_sum<THREADS>(z, sh);
  if (kl_now) {
    double ka = 0.0, kb = 0.0;
    for (int64_t i = p0 + threadIdx.x; i < p1; i += THREADS) {
      const double2 v = __ldcg(&a.klrow[i]);
      ka += v.x;
      kb += v.y;
    }
    ka = fused_block_sum<THREADS>(ka, sh);
    kb = fused_block_sum<THREADS>(kb, sh);
    const int64_t slot = (int64_t)((it + 1) / a.q.kl_every - 1) * tab.S + s;
    if (threadIdx.x == 0 && slot >= 0 && slot < a.kl_slots) a.kl_out[slot] = ka + kb + log(Zs);
  }
  if (threadIdx.x == 0 && a.Zout) a.Zout[s] = Zs;
  const float alpha = sched_alpha(a.q, it), mu = sched_mom(a.q, it);
  const float eta = a.q.lr > 0.f ? a.q.lr : (float)ns / 12.0f;
  const int ch = tab.chunks[s];
  const double inv = 1.0 / Zs;
  for (int64_t i = p0 + threadIdx.x; i < p1; i += THREADS) {
    const double2* fp = a.Fpart + tab.fp_off[s] + (i - p0);
    double rx = 0.0, ry = 0.0;
    for (int c = 0; c < ch; c++) {
      const double2 v = __ldcg(&fp[(int64_t)c * ns]);
      rx += v.x;
      ry += v.y;
    }
    const float2 fa = __ldcg(&a.Fa[i]);
    const float gxv = (float)(4.0 * ((double)alpha * (double)fa.x - rx * inv));
    const float gyv = (float)(4.0 * ((double)alpha * (double)fa.y - ry * inv));
    float2 u = a.U[i], gn = a.G[i], y = a.Y[i];
    float gx = (gxv * u.x < 0.f) ? gn.x + 0.2f : gn.x * 0.8f;
    float gy = (gyv * u.y < 0.f) ? gn.y + 0.2f : gn.y * 0.8f;
    gx = fmaxf(gx, a.q.min_gain);
    gy = fmaxf(gy, a.q.min_gain);
    u.x = mu * u.x - eta * gx * gxv;
    u.y = mu * u.y - eta * gy * gyv;
    y.x += u.x;
    y.y += u.y;
    if (!(isfinite(y.x) && isfinite(y.y))) raise_status(a.status, TSNE_STATUS_NONFINITE);
    a.U[i] = u;
    a.G[i] = make_float2(gx, gy);
    a.Y[i] = y;
  }
}

template <int THREADS, int R, int TILE>
__global__ void __launch_bounds__(THREADS, 2)
iterate_fused_kernel(const __grid_constant__ SampleTable tab, const __grid_constant__ FusedArgs a) {
  constexpr int ROWS = THREADS * R;
  __shared__ float4 tile[TILE];
  __shared__ double zred[THREADS / 32];
  __shared__ int s_item, s_last;
  const int it = a.iter_arg >= 0 ? a.iter_arg : *(volatile int32_t*)&a.hdr->iter;
  const bool kl_now = a.kl_out != nullptr && a.klrow != nullptr && a.q.kl_every > 0 &&
                      ((it + 1) % a.q.kl_every) == 0;
  const int total = tab.item_off[tab.S];
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.cnt[0], 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total) break;
    direct_item<THREADS, R, TILE>(a.Y, tab, item, a.Fpart, a.zpart, tile, zred);
    const int s = find_sample(tab.item_off, tab.S, item);
    const int local = item - tab.item_off[s];
    const int ch = tab.chunks[s];
    const int rt = local / ch, cc = local - rt * ch;
    if (cc == 0) {
      const int64_t r0 = tab.pt_off[s] + (int64_t)rt * ROWS;
      const int64_t r1 = min(r0 + (int64_t)ROWS, tab.pt_off[s + 1]);
      fused_attract<THREADS>(a, r0, r1, kl_now);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t need = (uint32_t)(tab.item_off[s + 1] - tab.item_off[s]);
      s_last = atomicAdd(&a.cnt[2 + s], 1u) == need - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      fused_finalize<THREADS>(a, tab, s, it, kl_now, zred);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && a.iter_arg < 0) {
    __threadfence();
    if (atomicAdd(&a.cnt[1], 1u) == gridDim.x - 1) {
      a.hdr->iter = it + 1;
      __threadfence();
    }
  }
}

// Launches the fused iteration with the cfg-1 tile shape (128 threads x 4
// rows, 256-column tiles).  cnt has 2 + S words and is zeroed here first.
cudaError_t launch_fused(const SampleTable& tab, const FusedArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.cnt, 0, sizeof(uint32_t) * (size_t)(2 + tab.S), st);
  if (e != cudaSuccess) return e;
  const int total = tab.item_off[tab.S];
  if (total <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_fused_kernel<128, 4, 256>, 128,
                                                  0);
    grid_cap = (sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
  }
  const int grid = total < grid_cap ? total : grid_cap;
  iterate_fused_kernel<128, 4, 256><<<grid, 128, 0, st>>>(tab, a);
  return cudaGetLastError();
}

}  // namespace tsne
