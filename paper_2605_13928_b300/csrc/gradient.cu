// gradient.cu -- attraction over the sparse P, the FP64 reductions of Z and KL,
// and the point-wise gradient / optimiser kernels of exact t-SNE
// (van der Maaten & Hinton 2008, Eq. 5 and Sec. 3.4).
#include "attract.cuh"

namespace tsne {

// ---------------------------------------------------------------------------
// Attraction  Fa_i = sum_{j in row i} p_ij w_ij (y_i - y_j), a half-warp per row.
// Lanes read consecutive CSR entries (coalesced col/val), gather y_j (Y is
// small and stays in L2), take w_ij with the hardware reciprocal (as the
// repulsion does), and the warp reduces in a fixed order.  When `kl`
// is set the row also yields sum p log p and sum p log(1 + d^2) in FP64 for
// the KL value.  Indices are checked: a column outside [0, n) or a row range
// outside [0, cap] raises TSNE_STATUS_BAD_INDEX and is skipped.
// HBM traffic per stored entry: 4 B column + 4 B value.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
attract_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
               const float* __restrict__ val, int64_t n, int64_t cap,
               const float2* __restrict__ Y, float2* __restrict__ Fa,
               double2* __restrict__ klrow, int iter_arg, const WsHeader* hdr, int kl_every,
               int force_kl, int32_t* status) {
  attract_rows(blockIdx.x, blockDim.x >> 5, row_ptr, col, val, n, cap, Y, Fa, klrow, iter_arg,
               hdr, kl_every, force_kl, status);
}

cudaError_t launch_attract(const tsne_csr& P, const float2* Y, float2* Fa, double2* klrow,
                           int iter_arg, const WsHeader* hdr, int kl_every, int force_kl,
                           int32_t* status, cudaStream_t st) {
  if (P.n <= 0) return cudaSuccess;
  // 2 warps x 2 rows: blocks of 64 threads x 48 registers, two of which fit in
  // the 7,168 registers that three CTAs of the symmetric repulsion kernel leave
  // free on an SM, so the attraction, launched on a side stream, can run in the
  // repulsion's shadow
  const int rows_per_block = 4;
  const int64_t blocks = (P.n + rows_per_block - 1) / rows_per_block;
  attract_kernel<<<(unsigned)blocks, 16 * rows_per_block, 0, st>>>(
      P.row_ptr, P.col, P.val, P.n, P.cap, Y, Fa, klrow, iter_arg, hdr, kl_every, force_kl,
      status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-sample reductions in FP64 and fixed order (one CTA per sample):
//   Z_s  = sum of the sample's repulsion work-item partials
//   KL_s = sum p log p + alpha sum p log(1 + d^2) + log Z_s   (if due)
// kl_out slot: kl_slot_base + s, where kl_slot_base is computed from the
// iteration when the step is driven by the device counter.
// ---------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < THREADS / 32; k++) t += sh[k];
  }
  return t;  // valid in thread 0
}

// Stage one of the two-stage reduction (rb.zred_part set): CTA (b, s) sums
// slice b of nb of the sample's Z partials (the direct items, then twice the
// symmetric items) and, when the KL value is due, slice b of its rows' KL
// terms, each in a fixed order; stage two (reduce_kernel) adds the nb slices
// in order.  One CTA per sample would run the FP64 adds of ~5e5 items on one
// SM (0.3 ms at 1M points).
__global__ void __launch_bounds__(256)
reduce_part_kernel(const __grid_constant__ SampleTable tab, const RepBufs rb,
                   const double2* __restrict__ klrow, int iter_arg, const WsHeader* hdr,
                   int kl_every, int force_kl, int want_kl_out) {
  __shared__ double sh[8];
  const int s = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  const int64_t i0 = tab.item_off[s], ni = tab.item_off[s + 1] - i0;
  const int64_t y0 = tab.sym_off[s], ny = tab.sym_gs > 0 ? tab.sym_off[s + 1] - y0 : 0;
  const int64_t tot = ni + ny;
  const int64_t lo = tot * b / nb, hi = tot * (b + 1) / nb;
  double z = 0.0;
  for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x)
    z += t < ni ? rb.zpart[i0 + t] : 2.0 * rb.zsym[y0 + (t - ni)];
  z = block_sum<256>(z, sh);
  double a = 0.0, c = 0.0;
  const bool want_kl = want_kl_out && klrow != nullptr && kl_due(iter_arg, hdr, kl_every, force_kl);
  if (want_kl) {
    const int64_t p0 = tab.pt_off[s], ns = tab.pt_off[s + 1] - p0;
    const int64_t r1 = p0 + ns * (b + 1) / nb;
    for (int64_t i = p0 + ns * b / nb + threadIdx.x; i < r1; i += blockDim.x) {
      const double2 v = klrow[i];
      a += v.x;
      c += v.y;
    }
    a = block_sum<256>(a, sh);
    c = block_sum<256>(c, sh);
  }
  if (threadIdx.x == 0) {
    double* o = rb.zred_part + ((int64_t)s * nb + b) * 3;
    o[0] = z;
    o[1] = a;
    o[2] = c;
  }
}

__global__ void __launch_bounds__(256)
reduce_kernel(const __grid_constant__ SampleTable tab, const RepBufs rb,
              const double2* __restrict__ klrow, double* __restrict__ Zout,
              double* __restrict__ kl_out, float alpha_arg, int iter_arg, const WsHeader* hdr,
              int kl_every, int force_kl, int stride_kl, int64_t kl_slots) {
  __shared__ double sh[8];
  const int s = blockIdx.x;
  const bool two_stage = rb.zred_part != nullptr;
  double z = 0.0;
  if (two_stage) {
    if (threadIdx.x == 0)
      for (int b = 0; b < rb.zred_nb; b++) z += rb.zred_part[((int64_t)s * rb.zred_nb + b) * 3];
  } else {
    for (int64_t it = tab.item_off[s] + threadIdx.x; it < tab.item_off[s + 1]; it += blockDim.x)
      z += rb.zpart[it];
    if (tab.sym_gs > 0)  // unordered pairs count twice in Z
      for (int64_t it = tab.sym_off[s] + threadIdx.x; it < tab.sym_off[s + 1]; it += blockDim.x)
        z += 2.0 * rb.zsym[it];
    z = block_sum<256>(z, sh);
  }
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  __shared__ double zs;
  if (threadIdx.x == 0) {
    zs = z;
    if (Zout) Zout[s] = zs;
  }
  const bool want_kl = kl_out != nullptr && klrow != nullptr &&
                       kl_due(iter_arg, hdr, kl_every, force_kl);
  if (!want_kl) return;
  double a = 0.0, b = 0.0;
  if (two_stage) {
    if (threadIdx.x == 0)
      for (int k = 0; k < rb.zred_nb; k++) {
        a += rb.zred_part[((int64_t)s * rb.zred_nb + k) * 3 + 1];
        b += rb.zred_part[((int64_t)s * rb.zred_nb + k) * 3 + 2];
      }
  } else {
    for (int64_t i = p0 + threadIdx.x; i < p1; i += blockDim.x) {
      const double2 v = klrow[i];
      a += v.x;
      b += v.y;
    }
    a = block_sum<256>(a, sh);
    b = block_sum<256>(b, sh);
  }
  if (threadIdx.x == 0) {
    // alpha: given explicitly (kl_grad), or 1 for the KL trace of tsne_step
    const double alpha = force_kl ? (double)alpha_arg : 1.0;
    int slot = s;
    if (!force_kl) {
      const int it = iter_arg >= 0 ? iter_arg : hdr->iter;
      slot = ((it + 1) / kl_every - 1) * stride_kl + s;
    }
    if (slot >= 0 && slot < kl_slots) kl_out[slot] = a + alpha * b + log(zs);
  }
}

// kl_slots: number of entries of kl_out (writes beyond it are dropped).
// part_only: run stage one alone (the update kernel finishes the reduction).
cudaError_t launch_reduce(const SampleTable& tab, const RepBufs& rb, const double2* klrow,
                          double* Zout, double* kl_out, float alpha, int iter_arg,
                          const WsHeader* hdr, int kl_every, int force_kl, int64_t kl_slots,
                          cudaStream_t st, bool part_only) {
  if (rb.zred_part) {
    reduce_part_kernel<<<dim3((unsigned)rb.zred_nb, (unsigned)tab.S), 256, 0, st>>>(
        tab, rb, klrow, iter_arg, hdr, kl_every, force_kl, kl_out != nullptr ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || part_only) return e;
  }
  reduce_kernel<<<tab.S, 256, 0, st>>>(tab, rb, klrow, Zout, kl_out, alpha, iter_arg, hdr,
                                       kl_every, force_kl, tab.S, kl_slots);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Point-wise combination.  Fr_i = the point's partial forces (direct chunks,
// then the symmetric split's group-pair partials or fixed-point sums) summed
// with compensated FP32 arithmetic in a fixed order; g_i = 4 (alpha Fa_i -
// Fr_i / Z_s) in FP32 (1 / Z_s is formed in FP64 from the FP64 Z_s and rounded
// once).  Blocks never straddle a sample (blk_off), so Z_s and the learning
// rate are uniform in a block.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 point_grad(const SampleTable& tab, int s, int64_t i,
                                             const RepBufs& rb, const float2* __restrict__ Fa,
                                             double Zs, float alpha) {
  const int64_t p0 = tab.pt_off[s], ns = tab.pt_off[s + 1] - p0;
  const float2* fp = rb.Fpart + tab.fp_off[s] + (i - p0);
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  const int ch = tab.chunks[s];
  for (int c = 0; c < ch; c++) {
    const float2 v = fp[(int64_t)c * ns];
    two_sum_acc(sx, cx, v.x);
    two_sum_acc(sy, cy, v.y);
  }
  if (tab.sym_gs > 0 && rb.Facc) {
    // symmetric split, fixed-point form: all off-diagonal group pairs
    const float2 v = fx_get(rb.Facc, tab.pt_off[tab.S], i, fx_shift(ns));
    two_sum_acc(sx, cx, v.x);
    two_sum_acc(sy, cy, v.y);
  } else if (tab.sym_gs > 0) {
    // symmetric split: row partials of items (g, h > g), column partials of (h < g, g)
    const int64_t GS = tab.sym_gs;
    const int64_t G = (ns + GS - 1) / GS;
    const int64_t g = (i - p0) / GS, o = (i - p0) - g * GS;
    sym_partials_acc(rb.Rbuf, rb.Cbuf, tab.sym_off[s], G, GS, g, o, sx, cx, sy, cy);
  }
  const float2 a = Fa[i];
  const float inv = (float)(1.0 / Zs);
  const float rx = sx + cx, ry = sy + cy;
  return make_float2(4.0f * fmaf(alpha, a.x, -rx * inv), 4.0f * fmaf(alpha, a.y, -ry * inv));
}

__global__ void __launch_bounds__(256)
grad_kernel(const __grid_constant__ SampleTable tab, const RepBufs rb,
            const float2* __restrict__ Fa, const double* __restrict__ Z, float alpha,
            float2* __restrict__ grad) {
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t i = tab.pt_off[s] + (int64_t)(b - tab.blk_off[s]) * tab.blk_pts + threadIdx.x;
  if (i >= tab.pt_off[s + 1]) return;
  grad[i] = point_grad(tab, s, i, rb, Fa, Z[s], alpha);
}

cudaError_t launch_grad(const SampleTable& tab, const RepBufs& rb, const float2* Fa,
                        const double* Z, float alpha, float2* grad, cudaStream_t st) {
  const int blocks = tab.blk_off[tab.S];
  if (blocks <= 0) return cudaSuccess;
  grad_kernel<<<blocks, tab.blk_pts, 0, st>>>(tab, rb, Fa, Z, alpha, grad);
  return cudaGetLastError();
}

// One optimiser iteration for every point (gains, momentum, position).  With
// iter_arg < 0 the iteration comes from the workspace counter, which the last
// block to finish advances (all blocks have read it by then).
// With the two-stage reduction (rb.zred_part), stage two happens here: every
// block adds its sample's Z slices in slice order (the same sum in every block,
// and the same as reduce_kernel's), and the sample's first block stores Z_s in
// Zout and, when due, the KL value in its trace slot.  With self_reduce (plans
// with few work items per sample, no reduction launch before this one) every
// block sums its sample's item partials itself (direct items, then twice the
// symmetric ones, strided over the block and added in a fixed tree), and the
// sample's first block also sums its rows' KL terms.  Otherwise Z holds Z_s.
__global__ void __launch_bounds__(256)
update_kernel(const __grid_constant__ SampleTable tab, const RepBufs rb,
              const float2* __restrict__ Fa, const double* __restrict__ Z, Schedule q,
              int iter_arg, WsHeader* hdr, float2* __restrict__ Y, float2* __restrict__ U,
              float2* __restrict__ G, int32_t* status, double* __restrict__ Zout,
              double* __restrict__ kl_out, int kl_every, int64_t kl_slots,
              const double2* __restrict__ klrow, int self_reduce) {
  __shared__ double zsh;
  __shared__ double sh[8];
  const int b = blockIdx.x;
  const int it = iter_arg >= 0 ? iter_arg : *(volatile int32_t*)&hdr->iter;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t p0 = tab.pt_off[s];
  const int64_t i = p0 + (int64_t)(b - tab.blk_off[s]) * tab.blk_pts + threadIdx.x;
  if (self_reduce) {  // block-uniform; blockDim.x == 256
    const int64_t i0 = tab.item_off[s], ni = tab.item_off[s + 1] - i0;
    const int64_t y0 = tab.sym_off[s], ny = tab.sym_gs > 0 ? tab.sym_off[s + 1] - y0 : 0;
    double z = 0.0;
    for (int64_t t = threadIdx.x; t < ni + ny; t += blockDim.x)
      z += t < ni ? rb.zpart[i0 + t] : 2.0 * rb.zsym[y0 + (t - ni)];
    z = block_sum<256>(z, sh);
    if (threadIdx.x == 0) zsh = z;
    __syncthreads();
    z = zsh;
    if (b == tab.blk_off[s]) {
      if (Zout && threadIdx.x == 0) Zout[s] = z;
      if (kl_out && klrow && kl_every > 0 && ((it + 1) % kl_every) == 0) {
        double a = 0.0, c = 0.0;
        for (int64_t r = p0 + threadIdx.x; r < tab.pt_off[s + 1]; r += blockDim.x) {
          const double2 v = klrow[r];
          a += v.x;
          c += v.y;
        }
        a = block_sum<256>(a, sh);
        c = block_sum<256>(c, sh);
        if (threadIdx.x == 0) {
          const int64_t slot = (int64_t)((it + 1) / kl_every - 1) * tab.S + s;
          if (slot >= 0 && slot < kl_slots) kl_out[slot] = a + c + log(z);
        }
      }
    }
  } else if (threadIdx.x == 0) {
    double z = 0.0;
    if (rb.zred_part) {
      const double* part = rb.zred_part + (int64_t)s * rb.zred_nb * 3;
      for (int k = 0; k < rb.zred_nb; k++) z += part[k * 3];
      if (b == tab.blk_off[s]) {
        if (Zout) Zout[s] = z;
        if (kl_out && kl_every > 0 && ((it + 1) % kl_every) == 0) {
          double a = 0.0, c = 0.0;
          for (int k = 0; k < rb.zred_nb; k++) {
            a += part[k * 3 + 1];
            c += part[k * 3 + 2];
          }
          const int64_t slot = (int64_t)((it + 1) / kl_every - 1) * tab.S + s;
          if (slot >= 0 && slot < kl_slots) kl_out[slot] = a + c + log(z);
        }
      }
    } else {
      z = Z[s];
    }
    zsh = z;
  }
  __syncthreads();
  const double Zs = zsh;
  if (i < tab.pt_off[s + 1]) {
    const float alpha = sched_alpha(q, it);
    const float mu = sched_mom(q, it);
    const float eta = q.lr > 0.f ? q.lr : (float)(tab.pt_off[s + 1] - p0) / 12.0f;
    const float2 g = point_grad(tab, s, i, rb, Fa, Zs, alpha);
    float2 u = U[i], gn = G[i], y = Y[i];
    float gx = (g.x * u.x < 0.f) ? gn.x + 0.2f : gn.x * 0.8f;
    float gy = (g.y * u.y < 0.f) ? gn.y + 0.2f : gn.y * 0.8f;
    gx = fmaxf(gx, q.min_gain);
    gy = fmaxf(gy, q.min_gain);
    u.x = mu * u.x - eta * gx * g.x;
    u.y = mu * u.y - eta * gy * g.y;
    y.x += u.x;
    y.y += u.y;
    if (!(isfinite(y.x) && isfinite(y.y))) raise_status(status, TSNE_STATUS_NONFINITE);
    U[i] = u;
    G[i] = make_float2(gx, gy);
    Y[i] = y;
  }
  if (iter_arg < 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned prev = atomicAdd(&hdr->done, 1u);
      if (prev == gridDim.x - 1) {
        hdr->done = 0;
        hdr->iter = it + 1;
        __threadfence();
      }
    }
  }
}

// With rb.zred_part set, the call also finishes the reduction (Zout, and the
// KL trace kl_out of kl_slots entries when kl_every > 0); then only
// reduce_part_kernel needs to run before it.
cudaError_t launch_update(const SampleTable& tab, const RepBufs& rb, const float2* Fa,
                          const double* Z, const Schedule& q, int iter_arg, WsHeader* hdr,
                          float2* Y, float2* U, float2* G, int32_t* status, double* Zout,
                          double* kl_out, int kl_every, int64_t kl_slots,
                          const double2* klrow, bool self_reduce, cudaStream_t st) {
  const int blocks = tab.blk_off[tab.S];
  if (blocks <= 0) return cudaSuccess;
  if (self_reduce && tab.blk_pts != 256) return cudaErrorInvalidValue;
  update_kernel<<<blocks, tab.blk_pts, 0, st>>>(tab, rb, Fa, Z, q, iter_arg, hdr, Y, U, G,
                                                status, Zout, kl_out, kl_every, kl_slots, klrow,
                                                self_reduce ? 1 : 0);
  return cudaGetLastError();
}

__global__ void fill_f32_kernel(float* __restrict__ p, int64_t m, float v) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) p[e] = v;
}

cudaError_t launch_fill_f32(float* p, int64_t m, float v, cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  fill_f32_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(p, m, v);
  return cudaGetLastError();
}

__global__ void set_iter_kernel(WsHeader* hdr, int iter) {
  hdr->iter = iter;
  hdr->done = 0;
}

cudaError_t launch_set_iter(WsHeader* hdr, int iter, cudaStream_t st) {
  set_iter_kernel<<<1, 1, 0, st>>>(hdr, iter);
  return cudaGetLastError();
}

}  // namespace tsne
