// repulse_item.cuh -- the direct-form repulsion of one work item, shared by
// the per-term kernel (repulse.cu) and the fused batched iteration (fused.cu).
//
// Direct (ordered-pair) form.  One CTA processes one work item = (sample, row
// tile, column chunk).  Each thread keeps R rows in registers, packed two rows
// per float2 so that every FP32 step is one packed FFMA2/FADD2/FMUL2
// instruction for two pairs; only the reciprocal is scalar (one MUFU.RCP per
// pair).  Columns of Y stream through shared memory in tiles of TILE points
// stored as {x, x, y, y}: one broadcast 128-bit load gives both packed operands.
//
// Per ordered pair: 8 FP32 lane-operations (dx, dy, 2 FMA for t, Z add, q^2,
// 2 FMA for the force) and 1 MUFU reciprocal; the SM executes 128 FP32 lane
// operations and 16 reciprocals per clock, so both pipes cap the kernel at 16
// pairs per clock per SM.
//
// Accuracy: FP32 partial sums per shared-memory tile, folded after every tile
// into a compensated FP32 sum per row (TwoSum: the running sum plus the sum of
// its rounding errors); the chunk result is written as float2.  Only Z is
// summed in FP64.  The self
// pair (i == j) is masked out in the tiles that hold the CTA's own rows, so
// Z has no self terms to cancel.  Columns past the end of a chunk are filled
// with a far sentinel (3e38, 3e38): t overflows to +inf, rcp(+inf) = +0, so
// they add exactly zero.
#pragma once
#include "common.cuh"

namespace tsne {

// One column against RP packed row pairs.  MASK: zero q for the self pair
// (row r sits at column slot ti + r * THREADS of this tile).
template <int RP, bool MASK, int STRIDE>
__device__ __forceinline__ void pair_block(const float4 col, int c, const float2 (&ax)[RP],
                                           const float2 (&ay)[RP], int64_t ti, float2 (&fx)[RP],
                                           float2 (&fy)[RP], float2 (&zz)[RP]) {
  const float2 NEG1 = make_float2(-1.f, -1.f);
  const float2 ONE2 = make_float2(1.f, 1.f);
  const float2 xc = make_float2(col.x, col.y);
  const float2 yc = make_float2(col.z, col.w);
#pragma unroll
  for (int p = 0; p < RP; p++) {
    const float2 dx = __ffma2_rn(xc, NEG1, ax[p]);
    const float2 dy = __ffma2_rn(yc, NEG1, ay[p]);
    float2 t = __ffma2_rn(dx, dx, ONE2);
    t = __ffma2_rn(dy, dy, t);
    float2 q = make_float2(rcp_approx(t.x), rcp_approx(t.y));
    if (MASK) {
      if (ti + (int64_t)(2 * p) * STRIDE == c) q.x = 0.f;
      if (ti + (int64_t)(2 * p + 1) * STRIDE == c) q.y = 0.f;
    }
    zz[p] = __fadd2_rn(zz[p], q);
    const float2 q2 = __fmul2_rn(q, q);
    fx[p] = __ffma2_rn(q2, dx, fx[p]);
    fy[p] = __ffma2_rn(q2, dy, fy[p]);
  }
}

// One work item (sample, row tile, column chunk) by the whole CTA: partial
// forces of the tile's rows over the chunk's columns into Fpart, the item's
// sum of w into zpart[item].  `tile` holds TILE float4, `zred` THREADS / 32
// doubles of shared memory.
// Direct-form work on (sample s, row tile rt, column chunk cc); the item's sum
// of w goes to zpart[zslot].
template <int THREADS, int R, int TILE, class Bar = CtaBar>
__device__ __forceinline__ void direct_work(const float2* __restrict__ Y, const SampleTable& tab,
                                            int s, int rt, int cc, int64_t zslot,
                                            float2* __restrict__ Fpart,
                                            double* __restrict__ zpart, float4* tile,
                                            double* zred) {
  static_assert(R % 2 == 0, "rows are processed in packed pairs");
  constexpr int RP = R / 2;
  constexpr int ROWS = THREADS * R;
  const int tid = threadIdx.x;
  const int ch = tab.chunks[s];
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t ns = p1 - p0;
  const int64_t row0 = p0 + (int64_t)rt * ROWS;
  const int64_t ntiles = (ns + TILE - 1) / TILE;
  int64_t c_begin, c_end;
  if (tab.diag) {  // diagonal group of the symmetric split: columns = the tile's group
    const int64_t g0 = p0 + ((row0 - p0) / tab.sym_gs) * tab.sym_gs;
    c_begin = g0;
    c_end = min(g0 + (int64_t)tab.sym_gs, p1);
  } else {
    c_begin = p0 + (cc * ntiles / ch) * TILE;
    c_end = min(p0 + ((cc + 1) * ntiles / ch) * TILE, p1);
  }

  float2 ax[RP], ay[RP];
  bool valid[R];
#pragma unroll
  for (int p = 0; p < RP; p++) {
    const int64_t i0 = row0 + (2 * p) * THREADS + tid;
    const int64_t i1 = i0 + THREADS;
    valid[2 * p] = i0 < p1;
    valid[2 * p + 1] = i1 < p1;
    const float2 y0 = valid[2 * p] ? Y[i0] : make_float2(0.f, 0.f);
    const float2 y1 = valid[2 * p + 1] ? Y[i1] : make_float2(0.f, 0.f);
    ax[p] = make_float2(y0.x, y1.x);
    ay[p] = make_float2(y0.y, y1.y);
  }

  // compensated FP32 row sums across tiles: (s, c) pairs
  float fxs[R], fxc[R], fys[R], fyc[R];
#pragma unroll
  for (int r = 0; r < R; r++) { fxs[r] = fxc[r] = fys[r] = fyc[r] = 0.f; }
  double zd = 0.0;

  for (int64_t cb = c_begin; cb < c_end; cb += TILE) {
    Bar::sync();
    for (int c = tid; c < TILE; c += THREADS) {
      const int64_t j = cb + c;
      const float2 v = (j < c_end) ? Y[j] : make_float2(3.0e38f, 3.0e38f);
      tile[c] = make_float4(v.x, v.x, v.y, v.y);
    }
    Bar::sync();
    const int ncols = (int)((c_end - cb) < TILE ? (c_end - cb) : TILE);
    const int nc4 = (ncols + 3) & ~3;  // sentinels fill the rest of the tile

    float2 fx[RP], fy[RP], zz[RP];
#pragma unroll
    for (int p = 0; p < RP; p++) {
      fx[p] = make_float2(0.f, 0.f);
      fy[p] = make_float2(0.f, 0.f);
      zz[p] = make_float2(0.f, 0.f);
    }
    // Tiles that hold some of this CTA's own rows drop the self pair j == i
    // exactly (its q = 1 would otherwise swamp a small Z); all other tiles
    // take the unmasked loop.
    const bool overlap = cb < row0 + ROWS && row0 < cb + TILE;
    if (!overlap) {
#pragma unroll 4
      for (int c = 0; c < nc4; c++) pair_block<RP, false, THREADS>(tile[c], 0, ax, ay, 0, fx, fy, zz);
    } else {
      const int64_t ti = row0 + tid - cb;  // column slot of row r is ti + r * THREADS
      for (int c = 0; c < nc4; c++) pair_block<RP, true, THREADS>(tile[c], c, ax, ay, ti, fx, fy, zz);
    }
#pragma unroll
    for (int p = 0; p < RP; p++) {
      two_sum_acc(fxs[2 * p], fxc[2 * p], fx[p].x);
      two_sum_acc(fxs[2 * p + 1], fxc[2 * p + 1], fx[p].y);
      two_sum_acc(fys[2 * p], fyc[2 * p], fy[p].x);
      two_sum_acc(fys[2 * p + 1], fyc[2 * p + 1], fy[p].y);
      if (valid[2 * p]) zd += zz[p].x;
      if (valid[2 * p + 1]) zd += zz[p].y;
    }
  }

  float2* out = Fpart + tab.fp_off[s] + (int64_t)cc * ns;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int64_t i = row0 + r * THREADS + tid;
    if (valid[r]) out[i - p0] = make_float2(fxs[r] + fxc[r], fys[r] + fyc[r]);
  }

  // Fixed-order block reduction of Z (deterministic).
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zd += __shfl_down_sync(0xffffffffu, zd, o);
  if ((tid & 31) == 0) zred[tid >> 5] = zd;
  Bar::sync();
  if (tid == 0) {
    double z = 0.0;
#pragma unroll
    for (int w = 0; w < THREADS / 32; w++) z += zred[w];
    zpart[zslot] = z;
  }
}

// One work item (sample, row tile, column chunk) by the whole CTA: partial
// forces of the tile's rows over the chunk's columns into Fpart, the item's
// sum of w into zpart[item].  `tile` holds TILE float4, `zred` THREADS / 32
// doubles of shared memory.
template <int THREADS, int R, int TILE>
__device__ __forceinline__ void direct_item(const float2* __restrict__ Y, const SampleTable& tab,
                                            int item, float2* __restrict__ Fpart,
                                            double* __restrict__ zpart, float4* tile,
                                            double* zred) {
  const int s = find_sample(tab.item_off, tab.S, item);
  const int local = item - tab.item_off[s];
  const int ch = tab.chunks[s];
  const int rt = local / ch, cc = local - rt * ch;
  direct_work<THREADS, R, TILE>(Y, tab, s, rt, cc, item, Fpart, zpart, tile, zred);
}

template <int THREADS, int R, int TILE>
__global__ void __launch_bounds__(THREADS, 2)
repulse_direct_kernel(const float2* __restrict__ Y, const __grid_constant__ SampleTable tab,
                      float2* __restrict__ Fpart, double* __restrict__ zpart) {
  __shared__ float4 tile[TILE];
  __shared__ double zred[THREADS / 32];
  direct_item<THREADS, R, TILE>(Y, tab, blockIdx.x, Fpart, zpart, tile, zred);
}

}  // namespace tsne
