// fused.cu -- one persistent launch per optimiser iteration for a batch of
// independent samples (many uneven embeddings at once).
//
// Every sample is cut into groups of GS = 1024 points (the symmetric split of
// repulse_sym_item.cuh with 4 warps).  A fixed grid (resident CTAs only) pulls
// work items from one atomic queue: per sample, first its G diagonal-group
// items (direct form, 128 threads x 8 rows = one group against itself, self
// pair masked; the same CTA also computes the attraction of the group's rows,
// one warp per row over the CSR row of P), then its G (G - 1) / 2
// off-diagonal group pairs (each unordered pair of points once).  When a CTA
// finishes an item it counts it for its sample; the CTA that completes a
// sample's last item computes Z_s (FP64, fixed order over the sample's items)
// and the KL value when due, and appends the sample's groups to a ready list.
// Behind all compute items the queue holds one update slot per group; slot k
// waits -- bounded -- for the k-th ready-list entry and then updates that
// group's points (gradient, gains, momentum, position).  Every compute item is
// handed out before any update slot, and compute items never wait, so every
// wait ends.  No CTA ever waits for another: completion is
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
#include "repulse_sym_item.cuh"

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

// Attraction Fa_i = sum_j p_ij w_ij (y_i - y_j) of rows [r0, r1), a half-warp
// per row (the same arithmetic and summation order as attract_kernel); KL row
// terms when due.
template <int THREADS>
__device__ __forceinline__ void fused_attract(const FusedArgs& a, int64_t r0, int64_t r1,
                                              bool kl_now) {
  const int hl = threadIdx.x & 15, w = threadIdx.x >> 5, half = (threadIdx.x >> 4) & 1;
  const int64_t n = a.P.n;
  for (int64_t base = r0 + 2 * w; base < r1; base += 2 * (THREADS / 32)) {
    const int64_t i = base + half;
    int64_t e0 = 0, e1 = 0;
    bool bad = false;
    if (i < r1) {
      e0 = a.P.row_ptr[i];
      e1 = a.P.row_ptr[i + 1];
      if (e0 < 0 || e1 < e0 || e1 > a.P.cap) {
        bad = true;
        e0 = e1 = 0;
      }
    }
    const float2 yi = i < r1 ? a.Y[i] : make_float2(0.f, 0.f);
    float fx = 0.f, fy = 0.f;
    double ka = 0.0, kb = 0.0;
    // four entries per lane per step (see attract_kernel): loads in flight together
    int64_t e = e0 + hl;
    for (; e + 48 < e1; e += 64) {
      int32_t j[4];
      float p[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        j[u] = a.P.col[e + 16 * u];
        p[u] = a.P.val[e + 16 * u];
      }
      float2 yj[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const bool ok = (uint64_t)(int64_t)j[u] < (uint64_t)n;
        bad |= !ok;
        yj[u] = a.Y[ok ? j[u] : 0];
        if (!ok) p[u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const float dx = yi.x - yj[u].x, dy = yi.y - yj[u].y;
        const float d2 = fmaf(dx, dx, dy * dy);
        const float pw = p[u] * (1.0f / (1.0f + d2));
        fx = fmaf(pw, dx, fx);
        fy = fmaf(pw, dy, fy);
        if (kl_now && p[u] > 0.f) {
          ka += (double)p[u] * (double)logf(p[u]);
          kb += (double)p[u] * (double)log1pf(d2);
        }
      }
    }
    for (; e < e1; e += 16) {
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
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
      raise_status(a.status, TSNE_STATUS_BAD_INDEX);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {  // within the half-warp
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      ka += __shfl_xor_sync(0xffffffffu, ka, o);
      kb += __shfl_xor_sync(0xffffffffu, kb, o);
    }
    if (hl == 0 && i < r1) {
      a.Fa[i] = make_float2(fx, fy);
      if (kl_now) a.klrow[i] = make_double2(ka, kb);
    }
  }
}

// Z_s and KL_s of a completed sample (one CTA); published through zs[s] and
// the ready flag of the sample.
template <int THREADS>
__device__ void fused_sample_done(const FusedArgs& a, const SampleTable& tab, int s, int it,
                                  bool kl_now, double* sh) {
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  double z = 0.0;
  for (int64_t k = tab.item_off[s] + threadIdx.x; k < tab.item_off[s + 1]; k += THREADS)
    z += __ldcg(&a.zpart[k]);
  for (int64_t k = tab.sym_off[s] + threadIdx.x; k < tab.sym_off[s + 1]; k += THREADS)
    z += 2.0 * __ldcg(&a.zsym[k]);
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
  if (threadIdx.x == 0) {
    a.Zout[s] = Zs;
    __threadfence();
    // publish the sample's groups on the ready list (entries hold group + 1)
    const int64_t G = tab.item_off[s + 1] - tab.item_off[s];
    const uint32_t base = atomicAdd(&a.cnt[2], (uint32_t)G);
    volatile uint32_t* list = a.cnt + 3 + tab.S;
    for (int64_t g = 0; g < G; g++) list[base + g] = (uint32_t)(tab.item_off[s] + g) + 1u;
    __threadfence();
  }
}

// Gradient, gains, momentum and position of the points of group g of sample s.
// Partial forces: the diagonal group's direct partial plus the row partials of
// pairs (g, h > g) and the column partials of pairs (h < g, g).
template <int THREADS>
__device__ void fused_update_group(const FusedArgs& a, const SampleTable& tab, int s, int g,
                                   int it, double Zs) {
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1], ns = p1 - p0;
  const float alpha = sched_alpha(a.q, it), mu = sched_mom(a.q, it);
  const float eta = a.q.lr > 0.f ? a.q.lr : (float)ns / 12.0f;
  const float inv = (float)(1.0 / Zs);
  const int64_t GS = tab.sym_gs;
  const int64_t G = (ns + GS - 1) / GS;
  const int64_t sbase = tab.sym_off[s];
  const int64_t i1 = min(p0 + (int64_t)(g + 1) * GS, p1);
  for (int64_t i = p0 + (int64_t)g * GS + threadIdx.x; i < i1; i += THREADS) {
    const float2 d = __ldcg(&a.Fpart[tab.fp_off[s] + (i - p0)]);
    float sx = d.x, cx = 0.f, sy = d.y, cy = 0.f;
    const int64_t o = (i - p0) - (int64_t)g * GS;
    sym_partials_acc<true>(a.Rbuf, a.Cbuf, sbase, G, GS, g, o, sx, cx, sy, cy);
    const float rx = sx + cx, ry = sy + cy;
    const float2 fa = __ldcg(&a.Fa[i]);
    const float gxv = 4.0f * fmaf(alpha, fa.x, -rx * inv);
    const float gyv = 4.0f * fmaf(alpha, fa.y, -ry * inv);
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

// Sample of a combined queue position: items of sample s occupy
// [item_off[s] + sym_off[s], item_off[s + 1] + sym_off[s + 1]).
__device__ __forceinline__ int fused_sample(const SampleTable& tab, int x) {
  int lo = 0, hi = tab.S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tab.item_off[mid] + tab.sym_off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kFusedThreads = 128;  // 4 warps: symmetric groups of 1024, direct 128 x 8 rows
constexpr int kFusedW = 4;
constexpr int kFusedR = 8;
constexpr int kFusedTile = 512;

__global__ void __launch_bounds__(kFusedThreads, 3)
iterate_fused_kernel(const __grid_constant__ SampleTable tab, const __grid_constant__ FusedArgs a) {
  constexpr int GS = kFusedW * 256;
  static_assert(kFusedThreads * kFusedR == GS, "a diagonal item is one group");
  __shared__ __align__(16) float sm[4 * GS];  // symmetric columns, or the direct tile
  __shared__ double zred[kFusedThreads / 32];
  __shared__ int s_item, s_last;
  const int it = a.iter_arg >= 0 ? a.iter_arg : *(volatile int32_t*)&a.hdr->iter;
  const bool kl_now = a.kl_out != nullptr && a.klrow != nullptr && a.q.kl_every > 0 &&
                      ((it + 1) % a.q.kl_every) == 0;
  const int total = tab.item_off[tab.S] + tab.sym_off[tab.S];  // compute items
  const int total_upd = total + tab.item_off[tab.S];          // + one update item per group
  while (true) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.cnt[0], 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= total_upd) break;
    if (item >= total) {
      // update slot k takes the k-th group published on the ready list (groups
      // are published as their samples complete); the wait is bounded
      __shared__ uint32_t s_entry;
      if (threadIdx.x == 0) {
        volatile uint32_t* slot = a.cnt + 3 + tab.S + (item - total);
        const long long t0 = clock64();
        uint32_t e = *slot;
        while (e == 0u) {
          if (clock64() - t0 > a.wait_limit) {
            raise_status(a.status, TSNE_STATUS_TIMEOUT);
            break;
          }
          __nanosleep(128);
          e = *slot;
        }
        s_entry = e;
        __threadfence();
      }
      __syncthreads();
      const uint32_t e = s_entry;
      if (e != 0u) {
        const int u = (int)e - 1;
        const int s = find_sample(tab.item_off, tab.S, u);
        fused_update_group<kFusedThreads>(a, tab, s, u - tab.item_off[s], it,
                                          __ldcg(&a.Zout[s]));
      }
      __syncthreads();
      continue;
    }
    const int s = fused_sample(tab, item);
    const int local = item - tab.item_off[s] - tab.sym_off[s];
    const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
    const int G = (int)((p1 - p0 + GS - 1) / GS);
    if (local < G) {
      __syncthreads();  // the previous item's shared memory is no longer read
      direct_work<kFusedThreads, kFusedR, kFusedTile>(a.Y, tab, s, local, 0,
                                                       tab.item_off[s] + local, a.Fpart, a.zpart,
                                                       reinterpret_cast<float4*>(sm), zred);
      const int64_t r0 = p0 + (int64_t)local * GS;
      fused_attract<kFusedThreads>(a, r0, min(r0 + (int64_t)GS, p1), kl_now);
    } else {
      int g, h;
      tri_decode(local - G, G, &g, &h);
      sym_work<kFusedW>(a.Y, tab, s, g, h, tab.sym_off[s] + (local - G), a.Rbuf, a.Cbuf, a.zsym,
                        sm, zred);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t need = (uint32_t)(G + G * (G - 1) / 2);
      s_last = atomicAdd(&a.cnt[3 + s], 1u) == need - 1u;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      fused_sample_done<kFusedThreads>(a, tab, s, it, kl_now, zred);
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

int fused_group_size() { return kFusedW * 256; }

// Words of the fused counter block: queue head, exited CTAs, ready-list tail,
// per-sample completed items, ready list (one entry per group).
int64_t fused_cnt_words(const SampleTable& tab) { return 3 + tab.S + tab.item_off[tab.S]; }

// One fused iteration; the counter block is zeroed here first.
cudaError_t launch_fused(const SampleTable& tab, const FusedArgs& a, cudaStream_t st) {
  cudaError_t e =
      cudaMemsetAsync(a.cnt, 0, sizeof(uint32_t) * (size_t)fused_cnt_words(tab), st);
  if (e != cudaSuccess) return e;
  const int total = tab.item_off[tab.S] + tab.sym_off[tab.S] + tab.item_off[tab.S];
  if (total <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_fused_kernel, kFusedThreads, 0);
    grid_cap = (sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
  }
  const int grid = total < grid_cap ? total : grid_cap;
  iterate_fused_kernel<<<grid, kFusedThreads, 0, st>>>(tab, a);
  return cudaGetLastError();
}

}  // namespace tsne
