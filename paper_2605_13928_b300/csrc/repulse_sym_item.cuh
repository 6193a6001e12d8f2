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
// Item = one off-diagonal pair (g, h) of point groups of GS = W * 256 points
// of the same sample.  Warp w owns 256 rows of group g (lane l: rows l + 32 r,
// r < 8, coordinates duplicated {x, x} for the packed operands).  Group h's
// columns sit in shared memory as W blocks of 256 with their force
// accumulators.  At step t warp w takes column block (w + t) mod W: each lane
// loads 8 consecutive columns (four packed pairs), computes its 8 x 8 block,
// passes the columns and their running sums to the next lane by shuffle, and
// after 32 rotations every column has met the warp's 256 rows; the visit's
// column sums (256 rows each) are then added to the accumulators in shared
// memory, which the warp that takes the block at step t + 1 extends.  Row
// accumulators stay in registers for the whole item.  Only a sample's last
// group can be partial, and it is always a column group: its blocks of
// sentinels only are skipped (sym_pass_partial, sym_blocks).
//
// A diagonal group (g = h) is an item of its own, after all group pairs of the
// launch (sym_diag_work): the triangle of each warp's block (sym_tri) and the
// block pairs, the last of them split in half between the two warps
// (sym_half_visit), so that each unordered pair is taken once.
//
// Column accumulators hold G_j = sum_i q^2 (y_i - y_j) = -F_j, so the same
// packed FMA updates row and column sums.  Points past the end of the sample
// are sentinels: rows at (3e38, 3e38), columns at (1e38, 1e38).  Every pair
// involving a sentinel has t = +inf, q = +0 and contributes exactly zero;
// sentinel-sentinel pairs have dx = 2e38 (finite), so also t = +inf.
//
// Rounding: every FP32 running sum is bounded in length before it is folded
// into longer sums (compensated FP32 or 64-bit fixed point across items): a
// row's sum over one item holds 512 terms per packed half (a tile adds its up
// to 4 item partials), a column's sum 1024 terms per item, or, in the tiled
// fixed-point form, up to 4096 (the tile's row groups, one after another).
//
// Two output forms:
//  * partial buffers (sym_work, FX = false): Rbuf[item][GS] row partials of
//    group g, Cbuf[item][GS] column partials (-G) of group h, zpart[item] the
//    item's sum over unordered pairs (Z counts ordered pairs: x 2 in the
//    reduction);
//  * fixed point (FX): the row and column partials are added to the per-point
//    64-bit accumulators Facc (x of all n points, then y; fx_add).  Large
//    the items are taken in tiles of TB x TB group pairs (sym_tile_work): the
//    rows' per-item partials are folded in shared memory and the columns'
//    accumulators of the tile's TB column groups stay in shared memory, so a
//    tile adds each of its points once instead of once per item.
#pragma once
#include "common.cuh"

namespace tsne {

// The building blocks of a warp's work on 256 rows x 256 columns.  A lane
// holds 8 rows (packed {v, v}: xr, yr, row sums fxr, fyr) and 8 consecutive
// columns as 4 packed pairs (xc, yc, column sums gx, gy, sums of w zz).

// Every pair of the lane's 8 rows and 8 columns: w into zz, w^2 (y_i - y_j)
// into the row sums and the column sums (32 packed evaluations).
__device__ __forceinline__ void sym_block(const float2 (&xr)[8], const float2 (&yr)[8],
                                          float2 (&fxr)[8], float2 (&fyr)[8],
                                          const float2 (&xc)[4], const float2 (&yc)[4],
                                          float2 (&gx)[4], float2 (&gy)[4], float2 (&zz)[4]) {
  const float2 NEG1 = make_float2(-1.f, -1.f);
  const float2 ONE2 = make_float2(1.f, 1.f);
#pragma unroll
  for (int r = 0; r < 8; r++) {
#pragma unroll
    for (int m = 0; m < 4; m++) {
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
}

// Four packed pairs from lane src.
__device__ __forceinline__ void sym_shift(float2 (&v)[4], int src) {
#pragma unroll
  for (int m = 0; m < 4; m++) {
    v[m].x = __shfl_sync(0xffffffffu, v[m].x, src);
    v[m].y = __shfl_sync(0xffffffffu, v[m].y, src);
  }
}

__device__ __forceinline__ void sym_ld8(const float* p, float2 (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  v[0] = make_float2(a.x, a.y);
  v[1] = make_float2(a.z, a.w);
  v[2] = make_float2(b.x, b.y);
  v[3] = make_float2(b.z, b.w);
}

__device__ __forceinline__ void sym_st8(float* p, const float2 (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  *reinterpret_cast<float4*>(p + 4) = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
}

__device__ __forceinline__ void sym_zd(const float2 (&zz)[4], double& zd) {
#pragma unroll
  for (int m = 0; m < 4; m++) zd += (double)zz[m].x + (double)zz[m].y;
}

// One visit: the warp's 8 rows per lane against one block of 256 columns in
// shared memory (positions bx / by, accumulators bgx / bgy; lane l takes
// columns 8l .. 8l + 7), 32 rotations: each lane computes its 8 x 8 block and
// passes the columns and their running sums to the next lane, and after 32
// rotations every lane holds its own columns' sums again and stores them.  The
// column sums continue the accumulators' values (ZERO: start from zero).  Adds
// this thread's share of the visit's sum of w (unordered pairs) to zd.
template <bool UNROLL2, bool ZERO = false>
__device__ __forceinline__ void sym_visit(const float2 (&xr)[8], const float2 (&yr)[8],
                                          float2 (&fxr)[8], float2 (&fyr)[8], const float* bx,
                                          const float* by, float* bgx, float* bgy, double& zd) {
  const int lane = threadIdx.x & 31;
  const int src = (lane + 31) & 31;  // columns move from lane l - 1 to lane l
  const int c0 = lane * 8;
  float2 xc[4], yc[4], gx[4], gy[4], zz[4];
  sym_ld8(bx + c0, xc);
  sym_ld8(by + c0, yc);
  if (ZERO) {
#pragma unroll
    for (int m = 0; m < 4; m++) gx[m] = gy[m] = make_float2(0.f, 0.f);
  } else {
    sym_ld8(bgx + c0, gx);
    sym_ld8(bgy + c0, gy);
  }
#pragma unroll
  for (int m = 0; m < 4; m++) zz[m] = make_float2(0.f, 0.f);
#pragma unroll(UNROLL2 ? 2 : 1)
  for (int rot = 0; rot < 32; rot++) {
    sym_block(xr, yr, fxr, fyr, xc, yc, gx, gy, zz);
    sym_shift(xc, src);
    sym_shift(yc, src);
    sym_shift(gx, src);
    sym_shift(gy, src);
  }
  sym_st8(bgx + c0, gx);
  sym_st8(bgy + c0, gy);
  sym_zd(zz, zd);
}

// Half a visit of a diagonal group's block pair (u, v), u != v, whose rows and
// columns share the column layout: rotations 0 .. 15 (rows of u against
// columns of v) or, shift_first, rotations 1 .. 16 (rows of v against columns
// of u).  Lane a of u meets lane b of v in the first when (a - b) mod 32 is in
// [0, 15], in the second when it is in [16, 31]: the two halves, run by the
// warps of u and of v, take every pair of the two blocks once.  The columns'
// sums, 16 lanes away from home at the end, are sent home and stored.
__device__ __forceinline__ void sym_half_visit(const float2 (&xr)[8], const float2 (&yr)[8],
                                               float2 (&fxr)[8], float2 (&fyr)[8],
                                               const float* bx, const float* by, float* bgx,
                                               float* bgy, bool shift_first, double& zd) {
  const int lane = threadIdx.x & 31;
  const int src = (lane + 31) & 31;
  const int c0 = lane * 8;
  float2 xc[4], yc[4], gx[4], gy[4], zz[4];
  sym_ld8(bx + c0, xc);
  sym_ld8(by + c0, yc);
  sym_ld8(bgx + c0, gx);
  sym_ld8(bgy + c0, gy);
#pragma unroll
  for (int m = 0; m < 4; m++) zz[m] = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int rot = 0; rot < 16; rot++) {
    if (shift_first) {
      sym_shift(xc, src);
      sym_shift(yc, src);
      sym_shift(gx, src);
      sym_shift(gy, src);
    }
    sym_block(xr, yr, fxr, fyr, xc, yc, gx, gy, zz);
    if (!shift_first) {
      sym_shift(xc, src);
      sym_shift(yc, src);
      sym_shift(gx, src);
      sym_shift(gy, src);
    }
  }
  // lane l holds the sums of lane l - 16's columns
  const int home = (lane + 16) & 31;
  sym_shift(gx, home);
  sym_shift(gy, home);
  sym_st8(bgx + c0, gx);
  sym_st8(bgy + c0, gy);
  sym_zd(zz, zd);
}

// W steps: at step t warp w visits column block (w + t) mod W of one column
// group in shared memory (positions scx / scy, accumulators sgx / sgy of GS =
// W * 256 columns).  SKIP: blocks b >= nbc hold only sentinel columns (past
// the end of the sample) and are skipped, their pairs contributing exactly
// zero.  Adds this thread's share of the group pair's sum of w (unordered
// pairs) to zd.  Ends with every warp done with shared memory.  (Folding each
// visit's column sums into the accumulators instead, to shorten the FP32
// running sums, cost 6 to 10 registers and, at three CTAs per SM, 12 % of the
// kernel's speed.)
template <int W, bool UNROLL2, class Bar = CtaBar, bool SKIP = false>
__device__ __forceinline__ void sym_pass(const float2 (&xr)[8], const float2 (&yr)[8],
                                         float2 (&fxr)[8], float2 (&fyr)[8], const float* scx,
                                         const float* scy, float* sgx, float* sgy, double& zd,
                                         int nbc = W) {
  constexpr int BLK = 256;  // points per warp block
  const int w = threadIdx.x >> 5;
  for (int t = 0; t < W; t++) {
    const int b = (w + t) % W;
    if (!SKIP || b < nbc)
      sym_visit<UNROLL2>(xr, yr, fxr, fyr, scx + b * BLK, scy + b * BLK, sgx + b * BLK,
                         sgy + b * BLK, zd);
    Bar::sync();
  }
}

// A column group with nbc < W non-empty blocks: every warp visits the nbc
// blocks, in the order (w + t) mod nbc, each visit with column sums of its own
// (priv: W x (W - 1) blocks of 2 x 256 floats), so that all warps work at
// every step; the sums then go to the accumulators sgx / sgy, added over the
// warps in warp order.  Ends with every warp done with shared memory.
template <int W, bool UNROLL2, class Bar = CtaBar>
__device__ __forceinline__ void sym_pass_partial(const float2 (&xr)[8], const float2 (&yr)[8],
                                                 float2 (&fxr)[8], float2 (&fyr)[8],
                                                 const float* scx, const float* scy, float* sgx,
                                                 float* sgy, float* priv, int nbc, double& zd) {
  constexpr int BLK = 256;
  const int w = threadIdx.x >> 5;
  for (int t = 0; t < nbc; t++) {
    const int b = (w + t) % nbc;
    float* pg = priv + (w * (W - 1) + b) * 2 * BLK;
    sym_visit<UNROLL2, true>(xr, yr, fxr, fyr, scx + b * BLK, scy + b * BLK, pg, pg + BLK, zd);
  }
  Bar::sync();
  for (int c = threadIdx.x; c < nbc * BLK; c += W * 32) {
    const int b = c / BLK, o = c - b * BLK;
    float sx = 0.f, sy = 0.f;
#pragma unroll
    for (int k = 0; k < W; k++) {
      const float* pg = priv + (k * (W - 1) + b) * 2 * BLK;
      sx += pg[o];
      sy += pg[BLK + o];
    }
    sgx[c] = sx;
    sgy[c] = sy;
  }
  Bar::sync();
}

// The triangle of one 256-point block: every unordered pair of two distinct
// points of the block once.  The warp's rows are the block's points in the
// column layout (lane l: points 8l .. 8l + 7, packed {v, v}) and the columns
// are the same points: at rotation 0 each lane pairs its own 8 points (column
// c > row r), at rotations 1 .. 15 it meets the points of lane l - rot, at
// rotation 16 lanes 0 .. 15 meet those of lane l + 16 (each lane pair at
// distance 16 once).  The columns' sums are then sent home and stored to the
// block's accumulators bgx / bgy.  Adds this thread's share of the sum of w
// over the block's unordered pairs to zd.
__device__ __forceinline__ void sym_tri(const float2 (&xr)[8], const float2 (&yr)[8],
                                        float2 (&fxr)[8], float2 (&fyr)[8], const float* bx,
                                        const float* by, float* bgx, float* bgy, double& zd) {
  const int lane = threadIdx.x & 31;
  const float2 NEG1 = make_float2(-1.f, -1.f);
  const float2 ONE2 = make_float2(1.f, 1.f);
  const int src = (lane + 31) & 31;
  const int c0 = lane * 8;
  float2 xc[4], yc[4], gx[4], gy[4], zz[4];
  sym_ld8(bx + c0, xc);
  sym_ld8(by + c0, yc);
#pragma unroll
  for (int m = 0; m < 4; m++) gx[m] = gy[m] = zz[m] = make_float2(0.f, 0.f);
  // rotation 0: row r against the lane's own columns 2m (.x) and 2m + 1 (.y),
  // only those after r
#pragma unroll
  for (int r = 0; r < 8; r++) {
#pragma unroll
    for (int m = 0; m < 4; m++) {
      if (2 * m + 1 <= r) continue;
      const float2 dx = __ffma2_rn(xc[m], NEG1, xr[r]);
      const float2 dy = __ffma2_rn(yc[m], NEG1, yr[r]);
      float2 tt = __ffma2_rn(dx, dx, ONE2);
      tt = __ffma2_rn(dy, dy, tt);
      float2 q = make_float2(rcp_approx(tt.x), rcp_approx(tt.y));
      if (2 * m == r) q.x = 0.f;  // the point itself
      zz[m] = __fadd2_rn(zz[m], q);
      const float2 q2 = __fmul2_rn(q, q);
      fxr[r] = __ffma2_rn(q2, dx, fxr[r]);
      fyr[r] = __ffma2_rn(q2, dy, fyr[r]);
      gx[m] = __ffma2_rn(q2, dx, gx[m]);
      gy[m] = __ffma2_rn(q2, dy, gy[m]);
    }
  }
#pragma unroll 1
  for (int rot = 1; rot <= 16; rot++) {
    sym_shift(xc, src);
    sym_shift(yc, src);
    sym_shift(gx, src);
    sym_shift(gy, src);
    if (rot < 16 || lane < 16) sym_block(xr, yr, fxr, fyr, xc, yc, gx, gy, zz);
  }
  const int home = (lane + 16) & 31;
  sym_shift(gx, home);
  sym_shift(gy, home);
  sym_st8(bgx + c0, gx);
  sym_st8(bgy + c0, gy);
  sym_zd(zz, zd);
}

// Non-empty 256-column blocks of the group starting at global point base of a
// sample ending at p1 (0 .. W).
template <int W>
__device__ __forceinline__ int sym_blocks(int64_t base, int64_t p1) {
  const int64_t v = p1 - base;
  const int64_t nb = v <= 0 ? 0 : (v + 255) / 256;
  return (int)(nb < W ? nb : W);
}

// Column group starting at global point cbase (points >= p1 are sentinels) into
// shared memory: positions and zeroed accumulators.
template <int W>
__device__ __forceinline__ void sym_load_cols(const float2* __restrict__ Y, int64_t cbase,
                                              int64_t p1, float* scx, float* scy, float* sgx,
                                              float* sgy) {
  constexpr int GS = W * 256;
  for (int c = threadIdx.x; c < GS; c += W * 32) {
    const int64_t j = cbase + c;
    const float2 v = j < p1 ? Y[j] : make_float2(1.0e38f, 1.0e38f);
    scx[c] = v.x;
    scy[c] = v.y;
    sgx[c] = 0.f;
    sgy[c] = 0.f;
  }
}

// This warp's 8 rows per lane of the group starting at rbase (packed {v, v}).
template <int W>
__device__ __forceinline__ void sym_load_rows(const float2* __restrict__ Y, int64_t rbase,
                                              int64_t p1, float2 (&xr)[8], float2 (&yr)[8]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < 8; r++) {
    const int64_t i = rbase + w * 256 + r * 32 + lane;
    const float2 v = i < p1 ? Y[i] : make_float2(3.0e38f, 3.0e38f);
    xr[r] = make_float2(v.x, v.x);
    yr[r] = make_float2(v.y, v.y);
  }
}

// Fixed-order block sum of the item's Z share into zpart[slot] (thread 0
// writes).  Ends with a barrier, so zred may be reused at once.
template <int W, class Bar = CtaBar>
__device__ __forceinline__ void sym_store_z(double zd, double* zred, double* zpart,
                                            int64_t slot) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zd += __shfl_down_sync(0xffffffffu, zd, o);
  if (lane == 0) zred[w] = zd;
  Bar::sync();
  if (threadIdx.x == 0) {
    double z = 0.0;
#pragma unroll
    for (int k = 0; k < W; k++) z += zred[k];
    zpart[slot] = z;
  }
  Bar::sync();
}

// Symmetric work on the group pair (g, h) of sample s; outputs at symmetric
// index `item` (Rbuf / Cbuf rows, or Facc when FX; zpart).  Shared memory: sm
// holds 4 * GS floats, zred W doubles; priv (W x (W - 1) x 512 floats, or
// null) lets a partial column group run on all warps (sym_pass_partial),
// without it its empty blocks are skipped.
template <int W, bool FX = false, class Bar = CtaBar>
__device__ __forceinline__ void sym_work(const float2* __restrict__ Y, const SampleTable& tab,
                                         int s, int g, int h, int64_t item,
                                         float2* __restrict__ Rbuf, float2* __restrict__ Cbuf,
                                         double* __restrict__ zpart, float* sm, double* zred,
                                         unsigned long long* __restrict__ Facc = nullptr,
                                         int32_t* status = nullptr, float* priv = nullptr) {
  constexpr int R = 8;
  constexpr int BLK = 256;
  constexpr int GS = W * BLK;
  float* scx = sm;
  float* scy = sm + GS;
  float* sgx = sm + 2 * GS;
  float* sgy = sm + 3 * GS;

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  // all warps are done with the previous item's shared-memory columns
  Bar::sync();
  const int64_t rbase = p0 + (int64_t)g * GS, cbase = p0 + (int64_t)h * GS;
  sym_load_cols<W>(Y, cbase, p1, scx, scy, sgx, sgy);
  float2 xr[R], yr[R], fxr[R], fyr[R];
  sym_load_rows<W>(Y, rbase, p1, xr, yr);
#pragma unroll
  for (int r = 0; r < R; r++) {
    fxr[r] = make_float2(0.f, 0.f);
    fyr[r] = make_float2(0.f, 0.f);
  }
  Bar::sync();
  // only the sample's last group can be partial, and it is always the column
  // group (h > g)
  const int nbc = sym_blocks<W>(cbase, p1);
  double zd = 0.0;
  if (nbc == W)
    sym_pass<W, FX, Bar>(xr, yr, fxr, fyr, scx, scy, sgx, sgy, zd);
  else if (priv)
    sym_pass_partial<W, FX, Bar>(xr, yr, fxr, fyr, scx, scy, sgx, sgy, priv, nbc, zd);
  else
    sym_pass<W, FX, Bar, true>(xr, yr, fxr, fyr, scx, scy, sgx, sgy, zd, nbc);

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
  sym_store_z<W, Bar>(zd, zred, zpart, item);
}

// Diagonal group g of sample s (rows and columns the same GS points): every
// unordered pair of two distinct points of the group once.  Warp w takes the
// points of block w as rows in the column layout; step 0: the triangle of block
// w; steps t = 1 .. W/2 - 1: the block pair (w, (w + t) mod W); step W/2: half
// of the block pair (w, (w + W/2) mod W), whose other half the warp of the
// other block takes (sym_half_visit), so that every warp does the same work;
// blocks of sentinels only are skipped.  Outputs are those of a direct-kernel item of the
// whole group: the points' partial forces (row sums minus column sums, one
// FP32 value per point and coordinate) to Fpart[fp_off[s] + point - p0], the
// group's sum of w over ordered pairs (twice the unordered sum) to
// zpart[item].  Shared memory: sm 4 * GS floats, zred W doubles.
template <int W, bool UNROLL2, class Bar = CtaBar>
__device__ __forceinline__ void sym_diag_work(const float2* __restrict__ Y,
                                              const SampleTable& tab, int s, int g, int64_t item,
                                              float2* __restrict__ Fpart,
                                              double* __restrict__ zpart, float* sm,
                                              double* zred) {
  constexpr int R = 8, BLK = 256, GS = W * BLK;
  float* scx = sm;
  float* scy = sm + GS;
  float* sgx = sm + 2 * GS;
  float* sgy = sm + 3 * GS;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t base = p0 + (int64_t)g * GS;
  const int nb = sym_blocks<W>(base, p1);
  Bar::sync();  // the previous work's shared memory is no longer read
  sym_load_cols<W>(Y, base, p1, scx, scy, sgx, sgy);
  Bar::sync();
  float2 xr[R], yr[R], fxr[R], fyr[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int o = w * BLK + lane * 8 + r;
    const bool in = base + o < p1;
    const float x = in ? scx[o] : 3.0e38f, y = in ? scy[o] : 3.0e38f;
    xr[r] = make_float2(x, x);
    yr[r] = make_float2(y, y);
    fxr[r] = make_float2(0.f, 0.f);
    fyr[r] = make_float2(0.f, 0.f);
  }
  double zd = 0.0;
  if (w < nb)
    sym_tri(xr, yr, fxr, fyr, scx + w * BLK, scy + w * BLK, sgx + w * BLK, sgy + w * BLK, zd);
  Bar::sync();
  for (int t = 1; t < W / 2; t++) {
    const int b = (w + t) % W;
    if (w < nb && b < nb)
      sym_visit<UNROLL2>(xr, yr, fxr, fyr, scx + b * BLK, scy + b * BLK, sgx + b * BLK,
                         sgy + b * BLK, zd);
    Bar::sync();
  }
  {
    const int b = (w + W / 2) % W;
    if (w < nb && b < nb)
      sym_half_visit(xr, yr, fxr, fyr, scx + b * BLK, scy + b * BLK, sgx + b * BLK,
                     sgy + b * BLK, w >= W / 2, zd);
    Bar::sync();
  }
  float2* out = Fpart + tab.fp_off[s] + (base - p0);
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int o = w * BLK + lane * 8 + r;
    if (base + o < p1)
      out[o] = make_float2((fxr[r].x + fxr[r].y) - sgx[o], (fyr[r].x + fyr[r].y) - sgy[o]);
  }
  sym_store_z<W, Bar>(2.0 * zd, zred, zpart, item);
}

// 1024-point groups: at most 152 registers, so that three CTAs per SM leave
// room for two 2-warp blocks of the attraction kernel (48 registers), which
// runs beside this kernel on a side stream; unbounded, the diagonal groups'
// work takes the kernel to 182 registers.  2048-point groups: 128 (two CTAs).
template <int W, bool FX>
__global__ void __maxnreg__(W == 4 ? 152 : 128)
repulse_sym_kernel(const float2* __restrict__ Y, const __grid_constant__ SampleTable tab,
                   float2* __restrict__ Rbuf, float2* __restrict__ Cbuf,
                   double* __restrict__ zpart, unsigned long long* __restrict__ Facc,
                   int32_t* status, float2* __restrict__ Fpart, double* __restrict__ zdiag) {
  constexpr int GS = W * 256;
  constexpr int NPRIV = W == 4 ? W * (W - 1) * 512 : 4;  // 2048-point groups: skip instead
  __shared__ __align__(16) float sm[4 * GS];
  __shared__ __align__(16) float priv[NPRIV];
  __shared__ double zred[W];
  const int item = blockIdx.x;
  const int nsym = tab.sym_off[tab.S];
  if (item >= nsym) {
    // diagonal groups, after every group pair (about half a pair's work each)
    const int d = item - nsym;
    const int s = find_sample(tab.item_off, tab.S, d);
    sym_diag_work<W, FX>(Y, tab, s, d - tab.item_off[s], d, Fpart, zdiag, sm, zred);
    return;
  }
  const int s = find_sample(tab.sym_off, tab.S, item);
  const int64_t G = (tab.pt_off[s + 1] - tab.pt_off[s] + GS - 1) / GS;
  int g, h;
  tri_decode(item - tab.sym_off[s], G, &g, &h);
  sym_work<W, FX>(Y, tab, s, g, h, item, Rbuf, Cbuf, zpart, sm, zred, Facc, status,
                  W == 4 ? priv : nullptr);
}

// ---------------------------------------------------------------------------
// Tiled fixed-point form.  The groups of a sample (G of them) form blocks of
// TB consecutive groups (B = ceil(G / TB) blocks, m_I groups in block I: TB
// except possibly the last).  The sample's items are ordered tile by tile:
// block-row I (every pair (g, h > g) with g in block I) holds the tiles
// J = I .. B - 1 (the pairs with h in block J), the diagonal tile J = I first,
// and within a tile the pairs in g-major order.  Block-row I starts at item
// tri_first(TB I, G) (the pairs with a smaller row group); within it tile
// J > I starts at m_I (m_I - 1) / 2 + m_I TB (J - I - 1).  Tile ids run over
// the block pairs I <= J in row-major order.
// ---------------------------------------------------------------------------
constexpr int kTB = 4;  // groups per tile side

__host__ __device__ __forceinline__ int64_t tile_blocks(int64_t G) { return (G + kTB - 1) / kTB; }
__host__ __device__ __forceinline__ int64_t tile_count(int64_t G) {
  const int64_t B = tile_blocks(G);
  return B * (B + 1) / 2;
}
__host__ __device__ __forceinline__ int tile_m(int64_t I, int64_t G) {
  const int64_t r = G - I * kTB;
  return (int)(r < kTB ? r : kTB);
}
// first tile id of block-row I (tiles (I', J) with I' < I, J >= I')
__host__ __device__ __forceinline__ int64_t tile_row_first(int64_t I, int64_t B) {
  return I * B - I * (I - 1) / 2;
}
// first item of tile (I, J), I <= J
__host__ __device__ __forceinline__ int64_t tile_item_first(int64_t I, int64_t J, int64_t G) {
  const int64_t mI = tile_m(I, G);
  int64_t v = tri_first(I * kTB, G);
  if (J > I) v += mI * (mI - 1) / 2 + mI * kTB * (J - I - 1);
  return v;
}

// Tile t of a sample in processing order, longest first: the off-diagonal
// tiles of full blocks (16 pairs each), then the diagonal tiles of full blocks
// (6 pairs), then the tiles of a partial last block (if G is not a multiple of
// TB).  The items' numbering (tile_item_first) is independent of this order.
__device__ __forceinline__ void tile_decode(int64_t t, int64_t G, int* I_out, int* J_out) {
  const int64_t Bf = G / kTB;  // full blocks
  const int64_t n1 = Bf * (Bf - 1) / 2;
  if (t < n1) {
    int I, J;
    tri_decode(t, Bf, &I, &J);
    *I_out = I;
    *J_out = J;
  } else if (t < n1 + Bf) {
    *I_out = *J_out = (int)(t - n1);
  } else {
    const int64_t t3 = t - n1 - Bf;  // (I, Bf) for I < Bf, then (Bf, Bf)
    *I_out = (int)(t3 < Bf ? t3 : Bf);
    *J_out = (int)Bf;
  }
}

// Shared memory of the tiled kernel, in floats: TB column groups (positions
// and accumulators, 4 GS each) and the rows' per-item fold (2 * 8 per thread).
template <int W>
constexpr int sym_tile_smem_floats() {
  return kTB * 4 * (W * 256) + 2 * 8 * (W * 32);
}

// All items of tile (I, J) of sample s into the fixed-point accumulators; the
// item sums of w go to zpart[sym_off[s] + item].
template <int W, class Bar = CtaBar>
__device__ __forceinline__ void sym_tile_work(const float2* __restrict__ Y,
                                              const SampleTable& tab, int s, int I, int J,
                                              double* __restrict__ zpart, float* sm,
                                              double* zred, unsigned long long* __restrict__ Facc,
                                              int32_t* status) {
  constexpr int R = 8, BLK = 256, GS = W * BLK;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t G = (p1 - p0 + GS - 1) / GS;
  const int mI = tile_m(I, G), mJ = tile_m(J, G);
  float* fold = sm + kTB * 4 * GS;  // [2][R][W * 32]: this thread's row partials
  const float scale = exp2f((float)fx_shift(p1 - p0));
  unsigned long long* Fy = Facc + tab.pt_off[tab.S];

  Bar::sync();  // the previous work's shared memory is no longer read
  for (int b = 0; b < mJ; b++) {
    float* cb = sm + b * 4 * GS;
    sym_load_cols<W>(Y, p0 + (int64_t)(J * kTB + b) * GS, p1, cb, cb + GS, cb + 2 * GS,
                     cb + 3 * GS);
  }
  int64_t item = tab.sym_off[s] + tile_item_first(I, J, G);
  for (int a = 0; a < mI; a++) {
    const int b0 = (J == I) ? a + 1 : 0;  // the diagonal tile holds h > g only
    if (b0 >= mJ) break;
    const int g = I * kTB + a;
    const int64_t rbase = p0 + (int64_t)g * GS;
    float2 xr[R], yr[R];
    sym_load_rows<W>(Y, rbase, p1, xr, yr);
#pragma unroll
    for (int r = 0; r < R; r++) {
      fold[r * W * 32 + threadIdx.x] = 0.f;
      fold[(R + r) * W * 32 + threadIdx.x] = 0.f;
    }
    Bar::sync();  // columns loaded
    for (int b = b0; b < mJ; b++) {
      float* cb = sm + b * 4 * GS;
      float2 fxr[R], fyr[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        fxr[r] = make_float2(0.f, 0.f);
        fyr[r] = make_float2(0.f, 0.f);
      }
      double zd = 0.0;
      sym_pass<W, true, Bar>(xr, yr, fxr, fyr, cb, cb + GS, cb + 2 * GS, cb + 3 * GS, zd);
#pragma unroll
      for (int r = 0; r < R; r++) {
        fold[r * W * 32 + threadIdx.x] += fxr[r].x + fxr[r].y;
        fold[(R + r) * W * 32 + threadIdx.x] += fyr[r].x + fyr[r].y;
      }
      sym_store_z<W, Bar>(zd, zred, zpart, item++);
    }
    // row partials of group g over this tile's column groups
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int64_t i = rbase + w * BLK + r * 32 + lane;
      if (i < p1) {
        fx_add(&Facc[i], fold[r * W * 32 + threadIdx.x], scale, status);
        fx_add(&Fy[i], fold[(R + r) * W * 32 + threadIdx.x], scale, status);
      }
    }
  }
  // column partials of the tile's column groups (F_j = -G_j); in the diagonal
  // tile the first group was never a column
  Bar::sync();
  for (int b = (J == I) ? 1 : 0; b < mJ; b++) {
    const float* cb = sm + b * 4 * GS;
    const int64_t cbase = p0 + (int64_t)(J * kTB + b) * GS;
    for (int c = threadIdx.x; c < GS; c += W * 32) {
      const int64_t j = cbase + c;
      if (j < p1) {
        fx_add(&Facc[j], -cb[2 * GS + c], scale, status);
        fx_add(&Fy[j], -cb[3 * GS + c], scale, status);
      }
    }
  }
}

// Tiled fixed-point launch: block b < tile_off[S] takes tile b of the global
// order (sample by sample, tile_off[s] = first tile of sample s; within a
// sample, tile_decode's longest-first order); the blocks after them take the
// diagonal groups (sym_diag_work: Fpart, zdiag).  Dynamic shared memory:
// sym_tile_smem_floats<W>() floats.
template <int W>
__global__ void __launch_bounds__(W * 32, 3)
repulse_sym_tiled_kernel(const float2* __restrict__ Y, const __grid_constant__ SampleTable tab,
                         double* __restrict__ zpart, unsigned long long* __restrict__ Facc,
                         int32_t* status, float2* __restrict__ Fpart,
                         double* __restrict__ zdiag) {
  constexpr int GS = W * 256;
  extern __shared__ __align__(16) float smt[];
  __shared__ double zred[W];
  const int32_t blk = (int32_t)blockIdx.x;
  const int32_t ntiles = tab.tile_off[tab.S];
  if (blk >= ntiles) {
    const int d = blk - ntiles;
    const int s = find_sample(tab.item_off, tab.S, d);
    sym_diag_work<W, true>(Y, tab, s, d - tab.item_off[s], d, Fpart, zdiag, smt, zred);
    return;
  }
  const int s = find_sample(tab.tile_off, tab.S, blk);
  const int64_t G = (tab.pt_off[s + 1] - tab.pt_off[s] + GS - 1) / GS;
  int I, J;
  tile_decode(blk - tab.tile_off[s], G, &I, &J);
  sym_tile_work<W>(Y, tab, s, I, J, zpart, smt, zred, Facc, status);
}

}  // namespace tsne
