// common.cuh -- shared definitions of the libtsne CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsne.h"

#define TSNE_CUDA_TRY(expr)                          \
  do {                                               \
    cudaError_t _e = (expr);                         \
    if (_e != cudaSuccess) return TSNE_ERR_CUDA;     \
  } while (0)

namespace tsne {

constexpr int kMaxS = TSNE_MAX_SAMPLES;

// Per-call description of the samples and of the repulsion work split,
// passed by value as a __grid_constant__ kernel parameter (no device table,
// so the calls stay capturable in CUDA graphs without uploads).
//
//  pt_off[s]    first point of sample s (pt_off[S] = n)
//  item_off[s]  first repulsion work item of sample s (item_off[S] = total)
//  blk_off[s]   first point-block of sample s for point-wise kernels
//  fp_off[s]    first element of sample s in the partial-force buffer
//  chunks[s]    column chunks of sample s; item = row_tile * chunks + chunk
//
// Symmetric split (sym_gs > 0): every sample is cut into groups of sym_gs
// points; the symmetric kernel evaluates each off-diagonal group pair g < h
// once and, in the same launch, each diagonal group's own pairs once (one
// item per group, with the outputs of a direct item of the whole group: one
// partial per point at fp_off, its Z at item_off); the persistent kernel runs
// the diagonal groups as direct items (`diag` = 1: columns = the item's own
// group, one chunk).  sym_off[s] is the first symmetric item of sample s; item
// t of a sample with G groups is the t-th pair (g, h) in row-major
// upper-triangular order.
struct SampleTable {
  int S;
  int rows_per_item;  // rows handled by one direct work item
  int tile_cols;      // columns per shared-memory tile
  int blk_pts;        // points per block of the point-wise kernels
  int max_chunks;
  int diag;           // direct kernel: columns = the item's own row range
  int sym_gs;         // group size of the symmetric split (0: direct only)
  int pad_;
  int64_t pt_off[kMaxS + 1];
  int64_t fp_off[kMaxS + 1];
  int32_t item_off[kMaxS + 1];
  int32_t blk_off[kMaxS + 1];
  int32_t chunks[kMaxS];
  int32_t sym_off[kMaxS + 1];
  int32_t tile_off[kMaxS + 1];  // tiled fixed-point form: first tile of sample s
};

// Upper-triangular pair index: pairs (g, h), 0 <= g < h < G, in row-major
// order; first(g) = g G - g (g + 1) / 2.
__host__ __device__ __forceinline__ int64_t tri_first(int64_t g, int64_t G) {
  return g * G - g * (g + 1) / 2;
}
__device__ __forceinline__ void tri_decode(int64_t t, int64_t G, int* g_out, int* h_out) {
  int64_t lo = 0, hi = G - 2;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (tri_first(mid, G) <= t) lo = mid; else hi = mid - 1;
  }
  *g_out = (int)lo;
  *h_out = (int)(lo + 1 + (t - tri_first(lo, G)));
}

// Largest s with off[s] <= x, for x in [off[0], off[S]); all threads of a
// block search the same x, so the loads are broadcasts.
__device__ __forceinline__ int find_sample(const int32_t* off, int S, int32_t x) {
  int lo = 0, hi = S - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Barrier policies of the work functions shared by several kernels: the whole
// CTA, or only its first 128 threads (named barrier 1) when the CTA's other
// warps run other work at the same time (the persistent batched kernel).
struct CtaBar {
  __device__ __forceinline__ static void sync() { __syncthreads(); }
};
struct Wg0Bar {
  __device__ __forceinline__ static void sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
};

__device__ __forceinline__ void raise_status(int32_t* st, int bits) {
  if (st) atomicOr(st, bits);
}

// Hardware approximate reciprocal (one MUFU.RCP; PTX rcp.approx.ftz.f32).
// Its relative error against the exact 1/t is checked in the GPU tests.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Repulsion partial results read by the reductions.
struct RepBufs {
  const float2* Fpart;   // direct kernel: per (chunk, point) partial forces
  const double* zpart;   // direct kernel: per item sum of w over ordered pairs
  const float2* Rbuf;    // symmetric kernel: per (item, row of group g)
  const float2* Cbuf;    // symmetric kernel: per (item, column of group h)
  const unsigned long long* Facc;  // fixed-point form: x[n] then y[n] (else null)
  double* zred_part;     // two-stage reduction: per (sample, slice) sums of z and KL (or null)
  int zred_nb;           // slices per sample
  const double* zsym;    // symmetric kernel: per item sum of w over unordered pairs
};

// Error-free addition (Knuth's TwoSum): s + v = t + e exactly in FP32
// arithmetic; the running pair (s, c) keeps the sum and the sum of rounding
// errors of every addition in a fixed order.
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v) {
  const float t = s + v;
  const float bp = t - s;
  c += (s - (t - bp)) + (v - bp);
  s = t;
}

// Adds the symmetric-split partial forces of point o of group g (of G groups
// of GS points; sym_base = first symmetric item of the sample) to the
// compensated FP32 sums (sx, cx), (sy, cy): the column partials of items
// (h < g, g) and the row partials of items (g, h > g), in increasing h.  The
// buffers are read once (streaming loads, eight in flight per thread, the last
// fewer than eight as one masked batch whose empty slots add exactly +0); the
// compensated sums keep FP64-like accuracy at FP32 pipe cost.  kL2Only: the
// buffers were written by other CTAs of the same launch, so loads bypass L1.
template <bool kL2Only>
__device__ __forceinline__ float2 ld_partial(const float2* p) {
  return kL2Only ? __ldcg(p) : __ldcs(p);
}

template <bool kL2Only = false>
__device__ __forceinline__ void sym_partials_acc(const float2* __restrict__ Rbuf,
                                                 const float2* __restrict__ Cbuf,
                                                 int64_t sym_base, int64_t G, int64_t GS,
                                                 int64_t g, int64_t o, float& sx, float& cx,
                                                 float& sy, float& cy) {
  constexpr int U = 8;
  // columns: item of (h, g) is sym_base + tri_first(h, G) + (g - h - 1)
  int64_t h = 0;
  for (; h + U <= g; h += U) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      v[u] = ld_partial<kL2Only>(
          &Cbuf[(sym_base + tri_first(h + u, G) + (g - h - u - 1)) * GS + o]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      two_sum_acc(sx, cx, v[u].x);
      two_sum_acc(sy, cy, v[u].y);
    }
  }
  if (h < g) {  // the rest (under U) as one batch of loads; the masked slots add +0
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      v[u] = h + u < g ? ld_partial<kL2Only>(
                             &Cbuf[(sym_base + tri_first(h + u, G) + (g - h - u - 1)) * GS + o])
                       : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; u++) {
      two_sum_acc(sx, cx, v[u].x);
      two_sum_acc(sy, cy, v[u].y);
    }
  }
  // rows: items (g, h) for h = g + 1 .. G - 1 are consecutive
  const float2* r = Rbuf + (sym_base + tri_first(g, G)) * GS + o;
  const int64_t nr = G - g - 1;
  int64_t t = 0;
  for (; t + U <= nr; t += U) {
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; u++) v[u] = ld_partial<kL2Only>(&r[(t + u) * GS]);
#pragma unroll
    for (int u = 0; u < U; u++) {
      two_sum_acc(sx, cx, v[u].x);
      two_sum_acc(sy, cy, v[u].y);
    }
  }
  if (t < nr) {  // the rest, likewise
    float2 v[U];
#pragma unroll
    for (int u = 0; u < U; u++)
      v[u] = t + u < nr ? ld_partial<kL2Only>(&r[(t + u) * GS]) : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < U; u++) {
      two_sum_acc(sx, cx, v[u].x);
      two_sum_acc(sy, cy, v[u].y);
    }
  }
}

// Fixed-point alternative to the partial buffers (TSNE_VARIANT_SYM4_FX, and
// AUTO once the buffers, which grow as N^2, would pass their memory budget):
// every group pair adds its FP32 row and column partials, scaled by 2^S and
// rounded, into two 64-bit integer accumulators per point with atomics.
// Integer addition is associative, so the sums do not depend on the order in
// which the pairs finish and the result stays bitwise reproducible; the scratch
// is O(N).
//
// Range: |Fr_i| = |sum_j w_ij^2 (y_i - y_j)| <= (ns - 1) max_d d / (1 + d^2)^2
// = (ns - 1) 3 sqrt(3) / 16 < ns / 2 for a sample of ns points, and so is
// every partial.  With S = 62 - bitlen(ns) the scaled sums stay below 2^61.
// Error: each partial is rounded once, by at most 2^-(S+1); a point takes
// G - 1 partials (G groups), so |dFr_i| <= (G - 1) 2^-(S+1) (1.1e-10 at
// ns = 1e6, G = 977).
__host__ __device__ __forceinline__ int fx_shift(int64_t ns) {
  int b = 0;
  while (b < 63 && (ns >> b) != 0) b++;  // bit length of ns
  return 62 - b;
}

// Adds v * 2^S (scale = 2^S, exact in FP32) to a fixed-point accumulator; a
// non-finite partial (from non-finite positions) is left out and raises
// TSNE_STATUS_NONFINITE.
__device__ __forceinline__ void fx_add(unsigned long long* acc, float v, float scale,
                                       int32_t* status) {
  const float x = v * scale;
  if (isfinite(x))
    atomicAdd(acc, (unsigned long long)__float2ll_rn(x));
  else
    raise_status(status, TSNE_STATUS_NONFINITE);
}

// Force of point i from the fixed-point accumulators (x of all n points, then
// y; written by other CTAs, so read from L2), rounded once to FP32: the
// int64 -> float conversion is correctly rounded and 2^-S is exact.
__device__ __forceinline__ float2 fx_get(const unsigned long long* acc, int64_t n, int64_t i,
                                         int S) {
  const float r = exp2f((float)-S);
  return make_float2(__ll2float_rn((long long)__ldcg(&acc[i])) * r,
                     __ll2float_rn((long long)__ldcg(&acc[n + i])) * r);
}

// Schedule of the optimiser at iteration `it`.
struct Schedule {
  int n_iter, ee_iters, mom_switch, kl_every;
  float ee, mom0, mom1, lr, min_gain;
};

__device__ __forceinline__ float sched_alpha(const Schedule& q, int it) {
  return it < q.ee_iters ? q.ee : 1.0f;
}
__device__ __forceinline__ float sched_mom(const Schedule& q, int it) {
  return it < q.mom_switch ? q.mom0 : q.mom1;
}

// Workspace header (first 256 bytes of every kl_grad / step workspace).
struct WsHeader {
  int32_t iter;       // device iteration counter for tsne_step(iter = -1)
  uint32_t done;      // finished-block counter of the update kernel
  int32_t pad[62];
};

// Arguments of the fused batched iteration (fused.cu).
struct FusedArgs {
  tsne_csr P;
  float2* Y;
  float2* U;
  float2* G;
  float2* Fa;
  float2* Fpart;      // diagonal-group partial forces (one per point)
  double* zpart;      // diagonal-group items' sums of w
  float2* Rbuf;       // symmetric items' row partials
  float2* Cbuf;       // symmetric items' column partials
  double* zsym;       // symmetric items' sums of w (unordered pairs)
  double2* klrow;     // per-row KL terms (null: no KL)
  double* Zout;       // per sample
  double* kl_out;     // KL trace (null: none)
  int64_t kl_slots;
  WsHeader* hdr;
  uint32_t* cnt;      // queue heads, ready-list tail, exited CTAs, items done per
                      // sample, ready list (fused.cu)
  int32_t* status;
  long long wait_limit;  // cycles an update slot waits for its ready-list entry
  Schedule q;
  int iter_arg;       // >= 0: iteration from the host; -1: workspace counter
  // work lists (fused_plan): samples largest first, their compute and
  // attraction items in that order, and the items each sample completes with
  int32_t ord[kMaxS];
  int32_t c_off[kMaxS + 1];
  int32_t a_off[kMaxS + 1];
  uint32_t need[kMaxS];
};

}  // namespace tsne
