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
struct SampleTable {
  int S;
  int rows_per_item;  // rows handled by one repulsion work item
  int tile_cols;      // columns per shared-memory tile
  int blk_pts;        // points per block of the point-wise kernels
  int max_chunks;
  int pad_;
  int64_t pt_off[kMaxS + 1];
  int64_t fp_off[kMaxS + 1];
  int32_t item_off[kMaxS + 1];
  int32_t blk_off[kMaxS + 1];
  int32_t chunks[kMaxS];
};

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

}  // namespace tsne
