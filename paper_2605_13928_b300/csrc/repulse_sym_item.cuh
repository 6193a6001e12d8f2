// repulse_sym_item.cuh -- exact repulsion over unordered pairs (each i < j once).
//
// Same quantities as the direct kernel (van der Maaten & Hinton 2008, Eq. 5,
// q-term): Fr_i = sum_{j != i} w_ij^2 (y_i - y_j), Z = sum_{i != j} w_ij.  A
// pair's term enters row i with + and row j with - (w is symmetric), so one
// evaluation serves both rows.  Per unordered pair: 10 FP32 lane-operations
// (dx, dy, 2 FMA for t, Z, q^2, 2 FMA into row i, 2 FMA into row j) and one
// MUFU reciprocal, i.e. 5 lane-ops and 0.5 reciprocals per ordered pair: the
// FP32 pipe caps the kernel at 25.6 ordered pairs per clock per SM.
//
// Work item = one off-diagonal pair (g, h) of point groups of GS = W * 256
// points of the same sample.  Warp w owns 256 rows of group g (lane l: rows
// l + 32 r, r < 8, coordinates duplicated {x, x} for the packed operands).
// Group h's 2048 columns sit in shared memory as eight blocks of 256 with
// their running force accumulators.  At step t warp w takes column block
// (w + t) mod W: each lane loads 8 consecutive columns (four packed pairs)
// with their accumulators, computes its 8 x 8 block, passes the columns and
// accumulators to the next lane by shuffle, and after 32 rotations every
// column has met the warp's 256 rows; the accumulators go back to shared
// memory for the warp that takes the block at step t + 1.  Row accumulators
// stay in registers for the whole item.
//
// Column accumulators hold G_j = sum_i q^2 (y_i - y_j) = -F_j, so the same
// packed FMA updates row and column sums.  Points past the end of the sample
// are sentinels: rows at (3e38, 3e38), columns at (1e38, 1e38).  Every pair
// involving a sentinel has t = +inf, q = +0 and contributes exactly zero;
// sentinel-sentinel pairs have dx = 2e38 (finite), so also t = +inf.
//
// Outputs (FP32, deterministic order): Rbuf[item][GS] row partials of group
// g, Cbuf[item][GS] column partials (-G) of group h, zpart[item] the item's
// sum over unordered pairs (Z counts ordered pairs: x 2 in the reduction).
// Fixed-point form (FX): the row and column partials are added to the per-point
// 64-bit accumulators Facc instead (x of all n points, then y; fx_add).
#pragma once
#include "common.cuh"

namespace tsne {

// Symmetric work on the group pair (g, h) of sample s; outputs at symmetric
// index `item` (Rbuf / Cbuf rows, or Facc when FX; zpart).  Shared memory: sm
// holds 4 * GS floats, zred W doubles.
template <int W, bool FX = false>
__device__ __forceinline__ void sym_work(const float2* __restrict__ Y, const SampleTable& tab,
                                         int s, int g, int h, int64_t item,
                                         float2* __restrict__ Rbuf, float2* __restrict__ Cbuf,
                                         double* __restrict__ zpart, float* sm, double* zred,
                                         unsigned long long* __restrict__ Facc = nullptr,
                                         int32_t* status = nullptr) {
  constexpr int R = 8, C = 8, CP = C / 2;
  constexpr int BLK = 256;  // points per warp block
  constexpr int GS = W * BLK;
  float* scx = sm;
  float* scy = sm + GS;
  float* sgx = sm + 2 * GS;
  float* sgy = sm + 3 * GS;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  // all warps are done with the previous item's shared-memory columns
  __syncthreads();
  const int64_t rbase = p0 + (int64_t)g * GS, cbase = p0 + (int64_t)h * GS;

  // column group h into shared memory (sentinels past the sample end)
  for (int c = threadIdx.x; c < GS; c += W * 32) {
    const int64_t j = cbase + c;
    const float2 v = j < p1 ? Y[j] : make_float2(1.0e38f, 1.0e38f);
    scx[c] = v.x;
    scy[c] = v.y;
    sgx[c] = 0.f;
    sgy[c] = 0.f;
  }
  // this warp's rows
  float2 xr[R], yr[R], fxr[R], fyr[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = rbase + w * BLK + r * 32 + lane;
    const float2 v = i < p1 ? Y[i] : make_float2(3.0e38f, 3.0e38f);
    xr[r] = make_float2(v.x, v.x);
    yr[r] = make_float2(v.y, v.y);
    fxr[r] = make_float2(0.f, 0.f);
    fyr[r] = make_float2(0.f, 0.f);
  }
  __syncthreads();

  const float2 NEG1 = make_float2(-1.f, -1.f);
  const float2 ONE2 = make_float2(1.f, 1.f);
  double zd = 0.0;
  const int src = (lane + 31) & 31;  // columns move from lane l - 1 to lane l

  for (int t = 0; t < W; t++) {
    const int b = (w + t) % W;
    const int c0 = b * BLK + lane * C;
    float2 xc[CP], yc[CP], gx[CP], gy[CP], zz[CP];
    {
      const float4 a0 = *reinterpret_cast<const float4*>(&scx[c0]);
      const float4 a1 = *reinterpret_cast<const float4*>(&scx[c0 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&scy[c0]);
      const float4 b1 = *reinterpret_cast<const float4*>(&scy[c0 + 4]);
      const float4 g0 = *reinterpret_cast<const float4*>(&sgx[c0]);
      const float4 g1 = *reinterpret_cast<const float4*>(&sgx[c0 + 4]);
      const float4 h0 = *reinterpret_cast<const float4*>(&sgy[c0]);
      const float4 h1 = *reinterpret_cast<const float4*>(&sgy[c0 + 4]);
      xc[0] = make_float2(a0.x, a0.y); xc[1] = make_float2(a0.z, a0.w);
      xc[2] = make_float2(a1.x, a1.y); xc[3] = make_float2(a1.z, a1.w);
      yc[0] = make_float2(b0.x, b0.y); yc[1] = make_float2(b0.z, b0.w);
      yc[2] = make_float2(b1.x, b1.y); yc[3] = make_float2(b1.z, b1.w);
      gx[0] = make_float2(g0.x, g0.y); gx[1] = make_float2(g0.z, g0.w);
      gx[2] = make_float2(g1.x, g1.y); gx[3] = make_float2(g1.z, g1.w);
      gy[0] = make_float2(h0.x, h0.y); gy[1] = make_float2(h0.z, h0.w);
      gy[2] = make_float2(h1.x, h1.y); gy[3] = make_float2(h1.z, h1.w);
    }
#pragma unroll
    for (int m = 0; m < CP; m++) zz[m] = make_float2(0.f, 0.f);

#pragma unroll(FX ? 2 : 1)
    for (int rot = 0; rot < 32; rot++) {
#pragma unroll
      for (int r = 0; r < R; r++) {
#pragma unroll
        for (int m = 0; m < CP; m++) {
          const float2 dx = __ffma2_rn(xc[m], NEG1, xr[r]);
          const float2 dy = __ffma2_rn(yc[m], NEG1, yr[r]);
          float2 tt = __ffma2_rn(dx, dx, ONE2);
          tt = __ffma2_rn(dy, dy, tt);
          const float2 q = make_float2(rcp_approx(tt.x), rcp_approx(tt.y));
          zz[m] = __fadd2_rn(zz[m], q);
          const float2 q2 = __fmul2_rn(q, q);
          fxr[r] = __ffma2_rn(q2, dx, fxr[r]);
          fyr[r] = __ffma2_rn(q2, dy, fyr[r]);
          gx[m] = __ffma2_rn(q2, dx, gx[m]);
          gy[m] = __ffma2_rn(q2, dy, gy[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < CP; m++) {
        xc[m].x = __shfl_sync(0xffffffffu, xc[m].x, src);
        xc[m].y = __shfl_sync(0xffffffffu, xc[m].y, src);
        yc[m].x = __shfl_sync(0xffffffffu, yc[m].x, src);
        yc[m].y = __shfl_sync(0xffffffffu, yc[m].y, src);
        gx[m].x = __shfl_sync(0xffffffffu, gx[m].x, src);
        gx[m].y = __shfl_sync(0xffffffffu, gx[m].y, src);
        gy[m].x = __shfl_sync(0xffffffffu, gy[m].x, src);
        gy[m].y = __shfl_sync(0xffffffffu, gy[m].y, src);
      }
    }
    // after 32 rotations every lane holds its own columns again
    *reinterpret_cast<float4*>(&sgx[c0]) = make_float4(gx[0].x, gx[0].y, gx[1].x, gx[1].y);
    *reinterpret_cast<float4*>(&sgx[c0 + 4]) = make_float4(gx[2].x, gx[2].y, gx[3].x, gx[3].y);
    *reinterpret_cast<float4*>(&sgy[c0]) = make_float4(gy[0].x, gy[0].y, gy[1].x, gy[1].y);
    *reinterpret_cast<float4*>(&sgy[c0 + 4]) = make_float4(gy[2].x, gy[2].y, gy[3].x, gy[3].y);
#pragma unroll
    for (int m = 0; m < CP; m++) zd += (double)zz[m].x + (double)zz[m].y;
    __syncthreads();
  }

  if constexpr (FX) {
    // row partials of group g and column partials of group h (F_j = -G_j) into
    // the fixed-point accumulators; a warp's adds cover 256 contiguous bytes
    const float scale = exp2f((float)fx_shift(p1 - p0));
    unsigned long long* Fy = Facc + tab.pt_off[tab.S];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = rbase + w * BLK + r * 32 + lane;
      if (i < p1) {
        fx_add(&Facc[i], fxr[r].x + fxr[r].y, scale, status);
        fx_add(&Fy[i], fyr[r].x + fyr[r].y, scale, status);
      }
    }
    for (int c = threadIdx.x; c < GS; c += W * 32) {
      const int64_t j = cbase + c;
      if (j < p1) {
        fx_add(&Facc[j], -sgx[c], scale, status);
        fx_add(&Fy[j], -sgy[c], scale, status);
      }
    }
  } else {
    // row partials of group g
    float2* rout = Rbuf + (int64_t)item * GS;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int o = w * BLK + r * 32 + lane;
      rout[o] = make_float2(fxr[r].x + fxr[r].y, fyr[r].x + fyr[r].y);
    }
    // column partials of group h: F_j = -G_j
    float2* cout = Cbuf + (int64_t)item * GS;
    for (int c = threadIdx.x; c < GS; c += W * 32) cout[c] = make_float2(-sgx[c], -sgy[c]);
  }

#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zd += __shfl_down_sync(0xffffffffu, zd, o);
  if (lane == 0) zred[w] = zd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double z = 0.0;
#pragma unroll
    for (int k = 0; k < W; k++) z += zred[k];
    zpart[item] = z;
  }
}

// FX with 1024-point groups is held to 3 CTAs per SM (its epilogue would
// otherwise take the kernel past 170 registers).
template <int W, bool FX>
__global__ void __launch_bounds__(W * 32, (W == 4 && FX) ? 3 : 2)
repulse_sym_kernel(const float2* __restrict__ Y, const __grid_constant__ SampleTable tab,
                   float2* __restrict__ Rbuf, float2* __restrict__ Cbuf,
                   double* __restrict__ zpart, unsigned long long* __restrict__ Facc,
                   int32_t* status) {
  constexpr int GS = W * 256;
  __shared__ __align__(16) float sm[4 * GS];
  __shared__ double zred[W];
  const int item = blockIdx.x;
  const int s = find_sample(tab.sym_off, tab.S, item);
  const int64_t G = (tab.pt_off[s + 1] - tab.pt_off[s] + GS - 1) / GS;
  int g, h;
  tri_decode(item - tab.sym_off[s], G, &g, &h);
  sym_work<W, FX>(Y, tab, s, g, h, item, Rbuf, Cbuf, zpart, sm, zred, Facc, status);
}

}  // namespace tsne
