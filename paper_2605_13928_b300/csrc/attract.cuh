// attract.cuh -- the attraction term of the exact t-SNE gradient as a device
// function (the attraction kernel, and the small-problem launch that runs it
// beside the direct repulsion items, call it), and the KL schedule test.
#pragma once
#include "common.cuh"

namespace tsne {

__device__ __forceinline__ bool kl_due(int iter_arg, const WsHeader* hdr, int kl_every,
                                       int force_kl) {
  if (force_kl) return true;
  if (kl_every <= 0) return false;
  const int it = iter_arg >= 0 ? iter_arg : hdr->iter;
  return ((it + 1) % kl_every) == 0;
}

// Rows of block `blk` (wpb warps, two rows per warp) of the attraction.
__device__ __forceinline__ void attract_rows(int64_t blk, int wpb,
                                             const int64_t* __restrict__ row_ptr,
                                             const int32_t* __restrict__ col,
                                             const float* __restrict__ val, int64_t n, int64_t cap,
                                             const float2* __restrict__ Y, float2* __restrict__ Fa,
                                             double2* __restrict__ klrow, int iter_arg,
                                             const WsHeader* hdr, int kl_every, int force_kl,
                                             int32_t* status) {
  // two rows per warp, a half-warp (16 lanes) each: twice the rows in flight for
  // the same registers, since a row is bound by its chain of dependent loads
  // (row_ptr, then col / val, then the y_j gathers)
  const int hl = threadIdx.x & 15;
  const int64_t i = (blk * wpb + (threadIdx.x >> 5)) * 2 + ((threadIdx.x >> 4) & 1);
  const bool want_kl = klrow != nullptr && kl_due(iter_arg, hdr, kl_every, force_kl);
  int64_t e0 = 0, e1 = 0;
  bool bad = false;
  if (i < n) {
    e0 = row_ptr[i];
    e1 = row_ptr[i + 1];
    if (e0 < 0 || e1 < e0 || e1 > cap) {
      bad = true;
      e0 = e1 = 0;
    }
  }
  const float2 yi = i < n ? Y[i] : make_float2(0.f, 0.f);
  float fx = 0.f, fy = 0.f;
  double a = 0.0, b = 0.0;
  // four entries per lane per step: their index, value and Y gathers are all
  // in flight together
  int64_t e = e0 + hl;
  for (; e + 48 < e1; e += 64) {
    int32_t j[4];
    float p[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      j[u] = col[e + 16 * u];
      p[u] = val[e + 16 * u];
    }
    float2 yj[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const bool ok = (uint64_t)(int64_t)j[u] < (uint64_t)n;
      bad |= !ok;
      yj[u] = Y[ok ? j[u] : 0];
      if (!ok) p[u] = 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const float dx = yi.x - yj[u].x, dy = yi.y - yj[u].y;
      const float d2 = fmaf(dx, dx, dy * dy);
      const float pw = p[u] * rcp_approx(1.0f + d2);
      fx = fmaf(pw, dx, fx);
      fy = fmaf(pw, dy, fy);
      if (want_kl && p[u] > 0.f) {
        a += (double)p[u] * (double)logf(p[u]);
        b += (double)p[u] * (double)log1pf(d2);
      }
    }
  }
  if (e < e1) {  // the rest (under 64 entries): one masked chunk, its loads in flight together
    int32_t j[4];
    float p[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const int64_t q = e + 16 * u;
      j[u] = q < e1 ? col[q] : 0;
      p[u] = q < e1 ? val[q] : 0.f;
    }
    float2 yj[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const bool ok = (uint64_t)(int64_t)j[u] < (uint64_t)n;
      bad |= !ok;
      yj[u] = Y[ok ? j[u] : 0];
      if (!ok) p[u] = 0.f;
    }
    // masked entries add exactly zero (p = 0, finite y_j): the same sums, in the same order
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const float dx = yi.x - yj[u].x, dy = yi.y - yj[u].y;
      const float d2 = fmaf(dx, dx, dy * dy);
      const float pw = p[u] * rcp_approx(1.0f + d2);
      fx = fmaf(pw, dx, fx);
      fy = fmaf(pw, dy, fy);
      if (want_kl && p[u] > 0.f) {
        a += (double)p[u] * (double)logf(p[u]);
        b += (double)p[u] * (double)log1pf(d2);
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
    raise_status(status, TSNE_STATUS_BAD_INDEX);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {  // within the half-warp
    fx += __shfl_xor_sync(0xffffffffu, fx, o);
    fy += __shfl_xor_sync(0xffffffffu, fy, o);
  }
  if (want_kl) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
  if (hl == 0 && i < n) {
    Fa[i] = make_float2(fx, fy);
    if (want_kl) klrow[i] = make_double2(a, b);
  }
}

}  // namespace tsne
