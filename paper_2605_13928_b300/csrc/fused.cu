// fused.cu -- one persistent launch per optimiser iteration for a batch of
// independent samples (many uneven embeddings at once).
//
// Every sample is cut into groups of GS = 1024 points (the symmetric split of
// repulse_sym_item.cuh with 4 warps).  A fixed grid of resident CTAs (two per
// SM) runs the whole iteration.  Each CTA has two roles, so that work bound by
// the FP32 pipe and work bound by the latency of dependent loads share every
// SM instead of taking turns:
//
//  * warps 0-3 (the compute warpgroup, its own named barrier) pull compute
//    items from one queue: per sample, its off-diagonal group pairs and its
//    diagonal groups (each unordered pair of points once: sym_diag_work);
//  * warps 4-5 (latency warps, no block barrier) pull attraction items: 64
//    rows of P, eight rows at a time per warp with four lanes per row and
//    sixteen gathers in flight per lane (KL row terms when due); the compute
//    warps join them once the compute queue has run dry.
//
// Samples are taken largest first.  The warp that completes a sample's last
// item (compute or attraction) computes Z_s in FP64 in a fixed order (and the
// KL value when due) and appends the sample's update blocks (256 points each)
// to a ready list.  Every warp whose queue has run dry takes update slots:
// slot k waits -- bounded -- for the k-th ready-list entry, then updates those
// points (gradient, gains, momentum, position).  Compute and attraction items
// never wait, so every sample completes and every wait ends; no CTA waits for
// another CTA to start, so the launch needs no grid barrier and cannot
// deadlock whatever the number of resident CTAs.  Results do not depend on
// which warp or CTA processes which item (every item writes fixed locations,
// every reduction runs in a fixed order).  Data written by other CTAs in the
// same launch is read with ld.global.cg (L2, not the incoherent L1).
//
// The counters are zeroed by a memset node before each launch; in
// device-counter mode the last CTA to exit advances the iteration counter.
#include <algorithm>
#include <numeric>
#include <vector>

#include "repulse_sym_item.cuh"

namespace tsne {

constexpr int kFzW = 4;                  // compute warps (symmetric groups of 1024)
constexpr int kFzLat = 2;                // latency warps
constexpr int kFzThreads = 32 * (kFzW + kFzLat);
constexpr int kFzAttRows = 64;           // rows per attraction item
constexpr int kFzUpdPts = 256;           // points per update slot

// counter block: [0] compute queue, [1] attraction queue, [2] update queue,
// [3] ready-list tail, [4] exited CTAs, [5 + s] finished items of sample s,
// [5 + S + k] ready list (update block + 1)
constexpr int kCntQc = 0, kCntQa = 1, kCntQu = 2, kCntTail = 3, kCntExit = 4, kCntS = 5;

__device__ __forceinline__ int fz_find(const int32_t* off, int S, int32_t x) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void fz_item_done(const FusedArgs& a, const SampleTable& tab, int s,
                                             int it, bool kl_now);

// Attraction Fa_i = sum_j p_ij w_ij (y_i - y_j) of rows [r0, r1) by one warp:
// eight rows at a time, four lanes per row, sixteen entries per lane in flight;
// each lane sums its entries in order and the row's four lanes are added by a
// fixed butterfly.  KL row terms (FP64) when due.  These warps share their
// SM's issue slots with FP32-bound compute warps, so the loop is kept lean:
// whole chunks of 16 entries per lane run without per-entry range checks, and
// w = 1 / (1 + d^2) takes the hardware reciprocal (one MUFU operation, about
// 1 ulp, as in the repulsion) instead of an IEEE division.
constexpr int kFzAttLanes = 4, kFzAttDepth = 16;

__device__ __forceinline__ void fz_att_term(float2 yi, float2 yj, float p, bool kl_now,
                                            float& fx, float& fy, double& ka, double& kb) {
  const float dx = yi.x - yj.x, dy = yi.y - yj.y;
  const float d2 = fmaf(dx, dx, dy * dy);
  const float pw = p * rcp_approx(1.0f + d2);
  fx = fmaf(pw, dx, fx);
  fy = fmaf(pw, dy, fy);
  if (kl_now && p > 0.f) {
    ka += (double)p * (double)logf(p);
    kb += (double)p * (double)log1pf(d2);
  }
}

__device__ __forceinline__ void fz_attract(const FusedArgs& a, int64_t r0, int64_t r1,
                                           bool kl_now) {
  constexpr int RPW = 32 / kFzAttLanes;              // rows per warp step
  constexpr int STEP = kFzAttLanes * kFzAttDepth;    // entries of a row per step
  const int lane = threadIdx.x & 31, sub = lane & (kFzAttLanes - 1);
  const uint32_t n = (uint32_t)a.P.n;
  for (int64_t base = r0; base < r1; base += RPW) {
    const int64_t i = base + lane / kFzAttLanes;
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
    int64_t e = e0 + sub;
    for (; e + (STEP - kFzAttLanes) < e1; e += STEP) {  // whole chunks
      int32_t j[kFzAttDepth];
      float p[kFzAttDepth];
#pragma unroll
      for (int u = 0; u < kFzAttDepth; u++) {
        j[u] = a.P.col[e + kFzAttLanes * u];
        p[u] = a.P.val[e + kFzAttLanes * u];
      }
      float2 yj[kFzAttDepth];
#pragma unroll
      for (int u = 0; u < kFzAttDepth; u++) {
        const bool ok = (uint32_t)j[u] < n;
        bad |= !ok;
        yj[u] = a.Y[ok ? j[u] : 0];
        if (!ok) p[u] = 0.f;
      }
#pragma unroll
      for (int u = 0; u < kFzAttDepth; u++) fz_att_term(yi, yj[u], p[u], kl_now, fx, fy, ka, kb);
    }
    for (; e < e1; e += kFzAttLanes) {  // the rest, one entry at a time
      const int32_t j = a.P.col[e];
      if ((uint32_t)j >= n) {
        bad = true;
        continue;
      }
      fz_att_term(yi, a.Y[j], a.P.val[e], kl_now, fx, fy, ka, kb);
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) raise_status(a.status, TSNE_STATUS_BAD_INDEX);
#pragma unroll
    for (int o = kFzAttLanes / 2; o > 0; o >>= 1) {  // within the row's lanes
      fx += __shfl_xor_sync(0xffffffffu, fx, o);
      fy += __shfl_xor_sync(0xffffffffu, fy, o);
      ka += __shfl_xor_sync(0xffffffffu, ka, o);
      kb += __shfl_xor_sync(0xffffffffu, kb, o);
    }
    if (sub == 0 && i < r1) {
      a.Fa[i] = make_float2(fx, fy);
      if (kl_now) a.klrow[i] = make_double2(ka, kb);
    }
  }
}

// Attraction items until the attraction queue runs dry, by one warp.
__device__ __forceinline__ void fz_attraction_items(const FusedArgs& a, const SampleTable& tab,
                                                    int it, bool kl_now) {
  const int32_t na = a.a_off[tab.S];
  while (true) {
    uint32_t c = 0;
    if ((threadIdx.x & 31) == 0) c = atomicAdd(&a.cnt[kCntQa], 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    if ((int32_t)c >= na) return;
    const int k = fz_find(a.a_off, tab.S, (int32_t)c);
    const int s = a.ord[k];
    const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
    const int64_t r0 = p0 + (int64_t)((int32_t)c - a.a_off[k]) * kFzAttRows;
    fz_attract(a, r0, min(r0 + (int64_t)kFzAttRows, p1), kl_now);
    fz_item_done(a, tab, s, it, kl_now);
  }
}

// Fixed-order FP64 warp sum: lane-strided partial sums, then a fixed butterfly
// (the same order whichever warp runs it).
__device__ __forceinline__ double fz_warp_total(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Z_s and KL_s of a completed sample by one warp; then the sample's update
// blocks go on the ready list.
__device__ void fz_sample_done(const FusedArgs& a, const SampleTable& tab, int s, int it,
                               bool kl_now) {
  const int lane = threadIdx.x & 31;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  double z = 0.0;
  for (int64_t k = tab.item_off[s] + lane; k < tab.item_off[s + 1]; k += 32)
    z += __ldcg(&a.zpart[k]);
  for (int64_t k = tab.sym_off[s] + lane; k < tab.sym_off[s + 1]; k += 32)
    z += 2.0 * __ldcg(&a.zsym[k]);
  const double Zs = fz_warp_total(z);
  if (kl_now) {
    double ka = 0.0, kb = 0.0;
    for (int64_t i = p0 + lane; i < p1; i += 32) {
      const double2 v = __ldcg(&a.klrow[i]);
      ka += v.x;
      kb += v.y;
    }
    ka = fz_warp_total(ka);
    kb = fz_warp_total(kb);
    const int64_t slot = (int64_t)((it + 1) / a.q.kl_every - 1) * tab.S + s;
    if (lane == 0 && slot >= 0 && slot < a.kl_slots) a.kl_out[slot] = ka + kb + log(Zs);
  }
  if (lane == 0) {
    a.Zout[s] = Zs;
    __threadfence();
    const int32_t b0 = tab.blk_off[s], nb = tab.blk_off[s + 1] - b0;
    const uint32_t base = atomicAdd(&a.cnt[kCntTail], (uint32_t)nb);
    volatile uint32_t* list = a.cnt + kCntS + tab.S;
    for (int32_t b = 0; b < nb; b++) list[base + b] = (uint32_t)(b0 + b) + 1u;
    __threadfence();
  }
  __syncwarp();
}

// Counts one finished item of sample s for the calling warp (whose threads, and
// for a compute item the whole warpgroup, have fenced their writes before); the
// warp that finishes the sample's last item runs fz_sample_done.
__device__ __forceinline__ void fz_item_done(const FusedArgs& a, const SampleTable& tab, int s,
                                             int it, bool kl_now) {
  uint32_t last = 0;
  __threadfence();
  __syncwarp();
  if ((threadIdx.x & 31) == 0)
    last = atomicAdd(&a.cnt[kCntS + s], 1u) + 1u == a.need[s] ? 1u : 0u;
  last = __shfl_sync(0xffffffffu, last, 0);
  if (last) {
    __threadfence();
    fz_sample_done(a, tab, s, it, kl_now);
  }
}

// Update slots, by one warp, until the update queue runs dry: slot k waits
// (bounded) for the k-th ready-list entry, a block of 256 points, and updates
// those points (eight per lane).
__device__ void fz_updates(const FusedArgs& a, const SampleTable& tab, int it) {
  const int lane = threadIdx.x & 31;
  const int32_t nblk = tab.blk_off[tab.S];
  while (true) {
    uint32_t k = 0;
    if (lane == 0) k = atomicAdd(&a.cnt[kCntQu], 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if ((int32_t)k >= nblk) return;
    uint32_t e = 0;
    if (lane == 0) {
      volatile uint32_t* slot = a.cnt + kCntS + tab.S + k;
      const long long t0 = clock64();
      e = *slot;
      while (e == 0u) {
        if (clock64() - t0 > a.wait_limit) {
          raise_status(a.status, TSNE_STATUS_TIMEOUT);
          break;
        }
        __nanosleep(256);
        e = *slot;
      }
      __threadfence();
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e == 0u) continue;  // gave up: the status word says so
    const int32_t b = (int32_t)e - 1;
    const int s = fz_find(tab.blk_off, tab.S, b);
    const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1], ns = p1 - p0;
    const double Zs = __ldcg(&a.Zout[s]);
    const float alpha = sched_alpha(a.q, it), mu = sched_mom(a.q, it);
    const float eta = a.q.lr > 0.f ? a.q.lr : (float)ns / 12.0f;
    const float inv = (float)(1.0 / Zs);
    const int64_t GS = tab.sym_gs, G = (ns + GS - 1) / GS;
    const int64_t i0 = p0 + (int64_t)(b - tab.blk_off[s]) * kFzUpdPts;
    for (int64_t i = i0 + lane; i < min(i0 + kFzUpdPts, p1); i += 32) {
      const float2 d = __ldcg(&a.Fpart[tab.fp_off[s] + (i - p0)]);
      float sx = d.x, cx = 0.f, sy = d.y, cy = 0.f;
      const int64_t g = (i - p0) / GS, o = (i - p0) - g * GS;
      sym_partials_acc<true>(a.Rbuf, a.Cbuf, tab.sym_off[s], G, GS, g, o, sx, cx, sy, cy);
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
}

__global__ void __launch_bounds__(kFzThreads, 2)
iterate_fused_kernel(const __grid_constant__ SampleTable tab, const __grid_constant__ FusedArgs a) {
  constexpr int GS = kFzW * 256;
  __shared__ __align__(16) float sm[4 * GS];  // a group's columns and their accumulators
  // per-warp column sums of a partial column group (sym_pass_partial)
  __shared__ __align__(16) float priv[kFzW * (kFzW - 1) * 512];
  __shared__ double zred[kFzW];
  __shared__ int s_item;
  const int it = a.iter_arg >= 0 ? a.iter_arg : *(volatile int32_t*)&a.hdr->iter;
  const bool kl_now = a.kl_out != nullptr && a.klrow != nullptr && a.q.kl_every > 0 &&
                      ((it + 1) % a.q.kl_every) == 0;
  const int warp = threadIdx.x >> 5;
  if (warp < kFzW) {
    // ---------------- compute warpgroup ----------------
    const int32_t nc = a.c_off[tab.S];
    while (true) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(&a.cnt[kCntQc], 1u);
      Wg0Bar::sync();
      const int c = s_item;
      Wg0Bar::sync();  // every thread has read s_item before it is overwritten
      if (c >= nc) break;
      const int k = fz_find(a.c_off, tab.S, c);
      const int s = a.ord[k];
      const int local = c - a.c_off[k];
      const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
      const int G = (int)((p1 - p0 + GS - 1) / GS);
      const int nsym = G * (G - 1) / 2;
      if (local < nsym) {
        int g, h;
        tri_decode(local, G, &g, &h);
        sym_work<kFzW, false, Wg0Bar>(a.Y, tab, s, g, h, tab.sym_off[s] + local, a.Rbuf, a.Cbuf,
                                      a.zsym, sm, zred, nullptr, nullptr, priv);
      } else {
        const int g = local - nsym;  // diagonal group g
        sym_diag_work<kFzW, false, Wg0Bar>(a.Y, tab, s, g, tab.item_off[s] + g, a.Fpart, a.zpart,
                                           sm, zred);
      }
      __threadfence();  // each thread's writes of the item, before it is counted
      Wg0Bar::sync();
      if (warp == 0) fz_item_done(a, tab, s, it, kl_now);
    }
  }
  // ---------------- attraction: the latency warps from the start, the compute
  // warps once the compute queue has run dry ----------------
  fz_attraction_items(a, tab, it, kl_now);
  // ---------------- every warp: update slots ----------------
  fz_updates(a, tab, it);
  __syncthreads();
  if (threadIdx.x == 0 && a.iter_arg < 0) {
    __threadfence();
    if (atomicAdd(&a.cnt[kCntExit], 1u) == gridDim.x - 1) {
      a.hdr->iter = it + 1;
      __threadfence();
    }
  }
}

int fused_group_size() { return kFzW * 256; }
int fused_update_points() { return kFzUpdPts; }

// Words of the fused counter block: five queue / list counters, per-sample
// finished items, ready list (one entry per 256-point update block).
int64_t fused_cnt_words(const SampleTable& tab) { return kCntS + tab.S + tab.blk_off[tab.S]; }

// Fills the work lists of a fused launch: samples largest first (ord), the
// compute items (symmetric pairs, then diagonal halves) and attraction items
// of each in that order (c_off, a_off), and the items each sample completes
// with (need).
void fused_plan(const SampleTable& tab, FusedArgs* a) {
  const int S = tab.S;
  std::vector<int> ord(S);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    return tab.pt_off[x + 1] - tab.pt_off[x] > tab.pt_off[y + 1] - tab.pt_off[y];
  });
  int32_t c = 0, at = 0;
  for (int k = 0; k < S; k++) {
    const int s = ord[k];
    const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
    const int64_t G = (ns + 1023) / 1024;
    const int32_t nsym = (int32_t)(G * (G - 1) / 2);
    const int32_t ndiag = tab.item_off[s + 1] - tab.item_off[s];
    const int32_t natt = (int32_t)((ns + kFzAttRows - 1) / kFzAttRows);
    a->ord[k] = s;
    a->c_off[k] = c;
    a->a_off[k] = at;
    a->need[s] = (uint32_t)(nsym + ndiag + natt);
    c += nsym + ndiag;
    at += natt;
  }
  a->c_off[S] = c;
  a->a_off[S] = at;
}

// One fused iteration; the counter block is zeroed here first.
cudaError_t launch_fused(const SampleTable& tab, const FusedArgs& a, cudaStream_t st) {
  cudaError_t e =
      cudaMemsetAsync(a.cnt, 0, sizeof(uint32_t) * (size_t)fused_cnt_words(tab), st);
  if (e != cudaSuccess) return e;
  if (tab.pt_off[tab.S] <= 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_fused_kernel,
                                                         kFzThreads, 0)) != cudaSuccess)
    return e;
  const int grid = (sms > 0 ? sms : 148) * (per_sm > 0 ? per_sm : 1);
  iterate_fused_kernel<<<grid, kFzThreads, 0, st>>>(tab, a);
  return cudaGetLastError();
}

}  // namespace tsne
