// pca.cu -- principal component analysis of an n x g FP32 matrix on B300:
// the step of the single-cell pipeline that produces the 50-D scores the
// neighbour graph and t-SNE consume (the paper's Table 1, step 5).
//
// Method: randomized subspace iteration with a Rayleigh-Ritz step (Halko,
// Martinsson & Tropp 2011, Algorithms 4.4 and 5.1) on the column-centred
// matrix Ac = A - 1 mu^T, with a sketch of L = 64 columns:
//   Y = Ac Omega;  Q = orth(Y);
//   repeat q times:  W = orth(Ac^T Q);  Q = orth(Ac W);
//   Z = Ac^T Q  (= B^T, B = Q^T Ac);  B B^T = Z^T Z = U~ diag(sigma^2) U~^T;
//   components V_c = Z u~_c / sigma_c;  scores T_c = sigma_c Q u~_c.
// With a spectral gap after the k-th singular value the result converges to
// the exact principal axes (the largest-eigenvalue eigenvectors of Ac^T Ac).
//
// B300 mapping:
// * column means: compensated FP32 sums, FP64 across row chunks.
// * the two products Ac W (M = n, K = g) and Ac^T Q (M = g, K = n, split over
//   K into chunks reduced in FP64 in a fixed order) run in one persistent
//   tcgen05 kernel that reads the caller's FP32 A once per pass: TMA streams
//   FP32 tiles of A into shared memory, converter warps centre every value,
//   split it into BF16 hi + lo (x - hi - lo is at most 2^-18 |x|) and lay
//   both out as K-major swizzled operands (transposing the tile for Ac^T Q),
//   one thread issues three M128 N64 K16 MMAs per K step (hi.hi + hi.lo +
//   lo.hi, FP32 accumulation in tensor memory, two accumulators) and four
//   epilogue warps drain tensor memory to global.  HBM-bound; no copy of A.
// * orth: CholeskyQR2 -- Gram matrix X^T X (FP32 within 256-row blocks,
//   FP64 across), FP64 Cholesky and triangular inverse in one CTA, X R^-1.
//   A non-positive pivot retries with a diagonal shift (shifted CholeskyQR).
// * Rayleigh-Ritz: FP64 cyclic Jacobi on the 64 x 64 Z^T Z in one CTA
//   (round-robin ordering, 32 disjoint rotations per round).
// Sign convention: every axis is flipped so that its largest-magnitude
// entry (lowest gene index among ties) is positive.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tsne {

constexpr int PC_L = 64;           // sketch width (= MMA N)
constexpr int PC_BM = 128;         // rows per tile (= TMEM lanes)
constexpr int PC_BK = 64;          // BF16 per K block (one 128-byte swizzled row)
constexpr int PC_A_BYTES = PC_BM * PC_BK * 2;   // 16 KB per plane
constexpr int PC_B_BYTES = PC_L * PC_BK * 2;    // 8 KB per plane
constexpr int PC_GRAM_BLOCKS = 4 * 148;  // most blocks of a Gram launch
constexpr int PC_COLSUM_CH = 512;   // row chunks of the column sums
constexpr int PC_KSEG = 32;         // K blocks per tensor-core accumulation (2048 values)

constexpr uint32_t kPcIdesc = idesc_bf16_f32(PC_BM, PC_L);

__host__ __device__ __forceinline__ int64_t round_up(int64_t x, int64_t m) {
  return (x + m - 1) / m * m;
}

// ---------------------------------------------------------------------------
// Column means: thread = column, compensated FP32 sums over a chunk of rows,
// FP64 partial per (chunk, column), then a fixed-order FP64 sum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
pca_colsum_kernel(const float* __restrict__ A, int64_t n, int g, int64_t lda,
                  double* __restrict__ part) {
  const int c = blockIdx.x * 256 + threadIdx.x;
  const int ch = blockIdx.y;
  const int64_t per = (n + PC_COLSUM_CH - 1) / PC_COLSUM_CH;
  const int64_t r0 = (int64_t)ch * per, r1 = min(n, r0 + per);
  if (c >= g) return;
  float s = 0.f, e = 0.f, q = 0.f, qe = 0.f;  // sum and sum of squares, compensated
  int64_t r = r0;
  for (; r + 8 <= r1; r += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) v[u] = __ldcs(&A[(r + u) * lda + c]);
#pragma unroll
    for (int u = 0; u < 8; u++) {
      two_sum_acc(s, e, v[u]);
      const float p = v[u] * v[u];
      two_sum_acc(q, qe, p);
      qe += fmaf(v[u], v[u], -p);  // exact rounding error of the square
    }
  }
  for (; r < r1; r++) {
    const float v = __ldcs(&A[r * lda + c]);
    two_sum_acc(s, e, v);
    const float p = v * v;
    two_sum_acc(q, qe, p);
    qe += fmaf(v, v, -p);
  }
  part[(int64_t)ch * g + c] = (double)s + (double)e;
  part[((int64_t)PC_COLSUM_CH + ch) * g + c] = (double)q + (double)qe;
}

// mean_c = S1 / n; css_c = S2 - S1^2 / n (centred sum of squares, FP64);
// the FP32 hi / lo split of the mean feeds the converters.
__global__ void pca_colmean_kernel(const double* __restrict__ part, int64_t n, int g, int gp,
                                   double* __restrict__ mean, float* __restrict__ mh,
                                   float* __restrict__ ml, double* __restrict__ css) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gp) return;
  double s1 = 0.0, s2 = 0.0;
  if (c < g)
    for (int ch = 0; ch < PC_COLSUM_CH; ch++) {
      s1 += part[(int64_t)ch * g + c];
      s2 += part[((int64_t)PC_COLSUM_CH + ch) * g + c];
    }
  const double m = c < g ? s1 / (double)n : 0.0;
  mean[c] = m;
  css[c] = c < g ? fmax(s2 - s1 * m, 0.0) : 0.0;
  const float h = (float)m;
  mh[c] = h;
  ml[c] = (float)(m - (double)h);
}

// Mean given by the caller (g values, FP64) -> padded FP32 hi/lo split.
__global__ void pca_mean_split_kernel(const double* __restrict__ mean_in, int g, int gp,
                                      float* __restrict__ mh, float* __restrict__ ml) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gp) return;
  const double m = c < g ? mean_in[c] : 0.0;
  const float h = (float)m;
  mh[c] = h;
  ml[c] = (float)(m - (double)h);
}

// x = hi + lo with hi, lo BF16 (|x - hi - lo| <= 2^-18 |x| away from underflow).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Fixed-order sum of m FP64 values into out[0] (one block of 256 threads).
__global__ void pca_sum_kernel(const double* __restrict__ x, int64_t m, double scale,
                               double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += 256) s += x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// Sketch operand: Wt[h][j][c] = split(M[c * ldm + j]) (transposed) for c < g,
// j < cols; zero elsewhere (j < 64, c < gp).  Row-major M (g x cols) when
// trans = 0; when trans = 1, M is cols x g (components, one axis per row).
__global__ void pca_sketch_split_kernel(const float* __restrict__ M, int g, int gp, int cols,
                                        int trans, __nv_bfloat16* __restrict__ Wt) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)PC_L * gp) return;
  const int j = (int)(e / gp), c = (int)(e % gp);
  float x = 0.f;
  if (j < cols && c < g) x = trans ? M[(int64_t)j * g + c] : M[(int64_t)c * cols + j];
  __nv_bfloat16 hi, lo;
  split_bf16(x, hi, lo);
  Wt[e] = hi;
  Wt[(int64_t)PC_L * gp + e] = lo;
}

// ---------------------------------------------------------------------------
// tcgen05 products with the centred matrix, straight from the caller's FP32 A.
//   rows (kTrans = 0): out[m][j] = sum_c Ac[m][c] B[j][c]      (M = cells, K = genes)
//   cols (kTrans = 1): out[kc][m][j] = sum_{cells of chunk kc} Ac[cell][m] B[j][cell]
//                                                             (M = genes, K = cells)
// B = Bhi + Blo (BF16, 64 x K, K-major, tensor maps tmBh / tmBl).
// Item t: m-tile mt = t % m_tiles, K chunk kc = t / m_tiles (K blocks
// [kc kpc, min(kb_total, (kc + 1) kpc))).
// Roles (448 threads):
//   warp 4      TMA producer: FP32 tiles of A (128-byte swizzle, 5-stage ring,
//               plus the K block's mean slices for the rows product) and the
//               B tiles (3-stage ring);
//   warps 6-13  converters: centre each value (x - mu_hi - mu_lo), split it
//               into BF16 hi + lo and store both straight into tensor memory
//               as the MMA's A operand (row m in lane m, K packed along
//               columns; two operand stages), transposing the tile for the
//               cols product;
//   warp 5      MMA issuer: Ahi.Bhi + Ahi.Blo + Alo.Bhi, M128 N64 K16, A from
//               tensor memory, B from shared memory, into a double-buffered
//               FP32 accumulator in tensor memory;
//   warps 0-3   epilogue: tensor memory -> out rows (m < rows_valid).
// Every wait is bounded.
// ---------------------------------------------------------------------------
constexpr int PF_RAW = 5;   // FP32 tiles of A (+ the K block's mean for the rows product)
constexpr int PF_OPS = 2;   // A operand stages in tensor memory
constexpr int PF_BST = 3;   // B operand tiles
constexpr int PF_CONV = 8;  // converter warps (6 .. 13)
constexpr int PF_THREADS = 32 * (6 + PF_CONV);
constexpr int PF_RAW_BYTES = 128 * 64 * 4;                      // 32 KB of FP32
constexpr int PF_RAW_STRIDE = PF_RAW_BYTES + 1024;               // + mean hi / lo (512 B)
constexpr uint32_t PF_B_BYTES = 2 * PC_B_BYTES;                  // 16 KB (B hi, B lo)
constexpr uint32_t PF_TMEM_COLS = 256;  // 2 accumulators x 64 + 2 operand stages x 64
constexpr uint32_t PF_TMEM_A0 = 2 * PC_L;  // first operand column

struct PfSmem {
  uint64_t raw_full[PF_RAW], raw_empty[PF_RAW], op_full[PF_OPS], op_empty[PF_OPS],
      b_full[PF_BST], b_empty[PF_BST], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_slot;
  int abort;
};
constexpr size_t kPfSmemBytes =
    1024 + (size_t)PF_RAW_STRIDE * PF_RAW + (size_t)PF_B_BYTES * PF_BST + sizeof(PfSmem);

// Bound of the waits that drain work already issued after an abort (copies in
// flight, committed MMAs): about 2 s at 2 GHz, far above what that work takes,
// and independent of the pipeline waits' limit.
constexpr long long kPcDrainLimit = 4000000000ll;

struct PfArgs {
  int m_tiles, nchunk, kpc, kb_total;
  int64_t n;            // cells (rows of A)
  int g;                // genes
  int64_t rows_valid;   // output rows stored
  int ldo, ncols;
  int64_t chunk_stride;
  float* out;
  const float* mh;      // mean split (gp entries, zero for padded genes)
  const float* ml;
  int32_t* status;
  long long wait_limit;
};

// x - mh - ml for a pair, then BF16 hi + lo of both (packed FP32x2 arithmetic;
// x - hi is exact as an FMA with -1).
__device__ __forceinline__ void centre_split2(float2 v, float2 nmh, float2 nml, uint32_t& hi,
                                              uint32_t& lo) {
  const float2 x = __fadd2_rn(__fadd2_rn(v, nmh), nml);
  const __nv_bfloat162 h = __float22bfloat162_rn(x);
  const float2 hf = __bfloat1622float2(h);
  const float2 r = __ffma2_rn(hf, make_float2(-1.f, -1.f), x);
  const __nv_bfloat162 l = __float22bfloat162_rn(r);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <bool kTrans>
__global__ void __launch_bounds__(PF_THREADS, 1)
pca_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                const __grid_constant__ CUtensorMap tmBl, const PfArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* raw = base;                                     // PF_RAW x 33 KB
  uint8_t* bst = base + (size_t)PF_RAW_STRIDE * PF_RAW;    // PF_BST x 16 KB
  PfSmem* S = reinterpret_cast<PfSmem*>(bst + (size_t)PF_B_BYTES * PF_BST);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int items = a.m_tiles * a.nchunk;

  if (tid == 0) {
    for (int q = 0; q < PF_RAW; q++) {
      mbar_init(&S->raw_full[q], 1);
      mbar_init(&S->raw_empty[q], 32 * PF_CONV);
    }
    for (int q = 0; q < PF_OPS; q++) {
      mbar_init(&S->op_full[q], 32 * PF_CONV);
      mbar_init(&S->op_empty[q], 1);
    }
    for (int q = 0; q < PF_BST; q++) {
      mbar_init(&S->b_full[q], 1);
      mbar_init(&S->b_empty[q], 1);
    }
    for (int q = 0; q < 2; q++) {
      mbar_init(&S->acc_full[q], 1);
      mbar_init(&S->acc_empty[q], PC_BM);
    }
    mbar_init(&S->drain, 1);
    S->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(&S->tmem_slot, PF_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->tmem_slot;

  if (warp == 4) {
    // ---------------- TMA producer: FP32 tiles of A, the mean, B tiles ----------------
    if (lane == 0) {
      long long it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < items; t += gridDim.x) {
        const int mt = t % a.m_tiles, kc = t / a.m_tiles;
        const int kb0 = kc * a.kpc, kb1 = min(a.kb_total, kb0 + a.kpc);
        for (int kb = kb0; kb < kb1; kb++, it++) {
          const int q = (int)(it % PF_RAW), qb = (int)(it % PF_BST);
          if (it >= PF_RAW &&
              (*(volatile int*)&S->abort ||
               !mbar_wait(&S->raw_empty[q], (uint32_t)((it / PF_RAW) - 1) & 1u, a.wait_limit))) {
            ok = false;
            break;
          }
          uint8_t* st = raw + (size_t)q * PF_RAW_STRIDE;
          mbar_arrive_expect_tx(&S->raw_full[q], PF_RAW_BYTES + (kTrans ? 0 : 512));
          if (!kTrans) {  // 128 cells x 64 genes: two boxes of 32 genes x 128 cells + mean
            tma_load_2d(st, &tmA, &S->raw_full[q], kb * 64, mt * PC_BM);
            tma_load_2d(st + PF_RAW_BYTES / 2, &tmA, &S->raw_full[q], kb * 64 + 32, mt * PC_BM);
            bulk_load(st + PF_RAW_BYTES, a.mh + kb * 64, 256, &S->raw_full[q]);
            bulk_load(st + PF_RAW_BYTES + 256, a.ml + kb * 64, 256, &S->raw_full[q]);
          } else {        // 64 cells x 128 genes: four boxes of 32 genes x 64 cells
#pragma unroll
            for (int bx = 0; bx < 4; bx++)
              tma_load_2d(st + bx * (PF_RAW_BYTES / 4), &tmA, &S->raw_full[q],
                          mt * PC_BM + 32 * bx, kb * 64);
          }
          if (it >= PF_BST &&
              (*(volatile int*)&S->abort ||
               !mbar_wait(&S->b_empty[qb], (uint32_t)((it / PF_BST) - 1) & 1u, a.wait_limit))) {
            ok = false;
            issued = it + 1;  // the A tile above is in flight
            break;
          }
          uint8_t* sb = bst + (size_t)qb * PF_B_BYTES;
          mbar_arrive_expect_tx(&S->b_full[qb], PF_B_BYTES);
          tma_load_2d(sb, &tmBh, &S->b_full[qb], kb * PC_BK, 0);
          tma_load_2d(sb + PC_B_BYTES, &tmBl, &S->b_full[qb], kb * PC_BK, 0);
          issued = it + 1;
        }
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(a.status, TSNE_STATUS_TIMEOUT);
        // copies already issued land before the CTA may exit; the drain has its
        // own long bound, independent of the pipeline waits' limit
        for (long long j = issued > PF_RAW ? issued - PF_RAW : 0; j < issued; j++)
          mbar_wait(&S->raw_full[j % PF_RAW], (uint32_t)(j / PF_RAW) & 1u, kPcDrainLimit);
        for (long long j = issued > PF_BST ? issued - PF_BST : 0; j < issued; j++)
          mbar_wait(&S->b_full[j % PF_BST], (uint32_t)(j / PF_BST) & 1u, kPcDrainLimit);
      }
    }
  } else if (warp >= 6) {
    // ---------------- converters: centre, split, store to tensor memory ----------------
    // lane quarter (warp % 4) = operand rows 32 (warp % 4) .. + 31 (the rule of
    // tcgen05.st); the two warps of a quarter take K halves hb = 0, 1:
    // rows product: row m = cell, genes 32 hb .. + 31 of the K block;
    // cols product: row m = gene, cells 32 hb .. + 31 of the K block.
    const int m = 32 * (warp & 3) + lane;
    const int hb = (warp - 6) >> 2;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    long long it = 0;
    bool aborted = false;
    for (int t = blockIdx.x; !aborted && t < items; t += gridDim.x) {
      const int mt = t % a.m_tiles, kc = t / a.m_tiles;
      const int kb0 = kc * a.kpc, kb1 = min(a.kb_total, kb0 + a.kpc);
      float2 tmh = make_float2(0.f, 0.f), tml = make_float2(0.f, 0.f);
      if (kTrans) {  // this row's gene (fixed over the item)
        const float mh = a.mh[mt * PC_BM + m], ml = a.ml[mt * PC_BM + m];
        tmh = make_float2(-mh, -mh);
        tml = make_float2(-ml, -ml);
      }
      const bool row_ok = kTrans || ((int64_t)mt * PC_BM + m < a.n);
      for (int kb = kb0; kb < kb1; kb++, it++) {
        const int rq = (int)(it % PF_RAW), oq = (int)(it % PF_OPS);
        bool ok = !*(volatile int*)&S->abort &&
                  mbar_wait(&S->raw_full[rq], (uint32_t)(it / PF_RAW) & 1u, a.wait_limit);
        if (ok && it >= PF_OPS)
          ok = mbar_wait(&S->op_empty[oq], (uint32_t)((it / PF_OPS) - 1) & 1u, a.wait_limit);
        // each converter warp decides for itself (no barrier across the converter
        // warps, which then drift apart by up to the rings' depth)
        if (__any_sync(0xffffffffu, !ok || *(volatile int*)&S->abort)) {
          aborted = true;
          break;
        }
        tc_fence_after();
        const uint8_t* rs = raw + (size_t)rq * PF_RAW_STRIDE;
        uint32_t hw[16], lw[16];  // 32 K values of row m as 16 packed BF16 pairs
        if (!kTrans) {
          // raw element (row r, gene c) sits in box c / 32, row r, 16-byte
          // chunk ((c % 32) / 4) ^ (r % 8); genes 32 hb + 4q .. + 3 are chunk q of box hb
          const uint32_t sw = (uint32_t)(m & 7);
          const uint8_t* rrow = rs + hb * (PF_RAW_BYTES / 2) + m * 128;
          const float4* mh4 = reinterpret_cast<const float4*>(rs + PF_RAW_BYTES) + hb * 8;
          const float4* ml4 = reinterpret_cast<const float4*>(rs + PF_RAW_BYTES + 256) + hb * 8;
#pragma unroll
          for (int q = 0; q < 8; q++) {
            float4 v = *reinterpret_cast<const float4*>(rrow + (((uint32_t)q ^ sw) << 4));
            const float4 m1 = mh4[q], m2 = ml4[q];
            centre_split2(make_float2(v.x, v.y), make_float2(-m1.x, -m1.y),
                          make_float2(-m2.x, -m2.y), hw[2 * q], lw[2 * q]);
            centre_split2(make_float2(v.z, v.w), make_float2(-m1.z, -m1.w),
                          make_float2(-m2.z, -m2.w), hw[2 * q + 1], lw[2 * q + 1]);
          }
          if (!row_ok) {
#pragma unroll
            for (int u = 0; u < 16; u++) hw[u] = lw[u] = 0u;
          }
        } else {
          // raw element (cell k, gene m) sits in box m / 32, row k, chunk
          // ((m % 32) / 4) ^ (k % 8), word m % 4
          const uint8_t* col = rs + (m >> 5) * (PF_RAW_BYTES / 4) + (((uint32_t)m & 3u) << 2);
          const uint32_t cch = ((uint32_t)m & 31u) >> 2;
          const int64_t cell0 = (int64_t)kb * 64 + 32 * hb;
#pragma unroll
          for (int u = 0; u < 16; u++) {
            const int k0 = 32 * hb + 2 * u, k1 = k0 + 1;
            float2 v = make_float2(
                *reinterpret_cast<const float*>(col + k0 * 128 + ((cch ^ ((uint32_t)k0 & 7u)) << 4)),
                *reinterpret_cast<const float*>(col + k1 * 128 + ((cch ^ ((uint32_t)k1 & 7u)) << 4)));
            centre_split2(v, tmh, tml, hw[u], lw[u]);
            // cells past the end are zero-filled by TMA but must stay zero after centring
            if (cell0 + 2 * u >= a.n) hw[u] &= 0xffff0000u, lw[u] &= 0xffff0000u;
            if (cell0 + 2 * u + 1 >= a.n) hw[u] &= 0x0000ffffu, lw[u] &= 0x0000ffffu;
          }
        }
        // operand stage oq: hi in columns A0 + 64 oq + [0, 32), lo in [32, 64)
        const uint32_t acol = tmem + PF_TMEM_A0 + 64u * (uint32_t)oq + 16u * (uint32_t)hb;
        tmem_st16(lane_base + acol, hw);
        tmem_st16(lane_base + acol + 32u, lw);
        tmem_st_wait();
        tc_fence_before();
        mbar_arrive(&S->op_full[oq]);
        mbar_arrive(&S->raw_empty[rq]);
      }
    }
    if (aborted && lane == 0) {
      raise_status(a.status, TSNE_STATUS_TIMEOUT);
      *(volatile int*)&S->abort = 1;
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long it = 0;
      int li = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < items; t += gridDim.x, li++) {
        const int kc = t / a.m_tiles;
        const int kb0 = kc * a.kpc, kb1 = min(a.kb_total, kb0 + a.kpc);
        const int bb = li & 1;
        if (li >= 2 &&
            !mbar_wait(&S->acc_empty[bb], (uint32_t)((li >> 1) - 1) & 1u, a.wait_limit)) {
          ok = false;
          break;
        }
        const uint32_t d = tmem + (uint32_t)(bb * PC_L);
        for (int kb = kb0; kb < kb1; kb++, it++) {
          const int q = (int)(it % PF_OPS), qb = (int)(it % PF_BST);
          if (*(volatile int*)&S->abort ||
              !mbar_wait(&S->op_full[q], (uint32_t)(it / PF_OPS) & 1u, a.wait_limit) ||
              !mbar_wait(&S->b_full[qb], (uint32_t)(it / PF_BST) & 1u, a.wait_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = tmem + PF_TMEM_A0 + 64u * (uint32_t)q, al = ah + 32u;
          const uint32_t sb = smem_u32(bst + (size_t)qb * PF_B_BYTES);
          const uint64_t bh = sw128_desc(sb), bl = sw128_desc(sb + PC_B_BYTES);
#pragma unroll
          for (int kk = 0; kk < PC_BK / 16; kk++) {  // K = 16: 8 operand columns, 2 desc units
            mma_bf16_ts(d, ah + 8u * kk, bh + 2 * kk, kPcIdesc, (kb > kb0 || kk > 0) ? 1u : 0u);
            mma_bf16_ts(d, ah + 8u * kk, bl + 2 * kk, kPcIdesc, 1u);
            mma_bf16_ts(d, al + 8u * kk, bh + 2 * kk, kPcIdesc, 1u);
          }
          mma_commit(&S->op_empty[q]);
          mma_commit(&S->b_empty[qb]);
        }
        if (!ok) break;
        mma_commit(&S->acc_full[bb]);
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(a.status, TSNE_STATUS_TIMEOUT);
        mma_commit(&S->drain);
        mbar_wait(&S->drain, 0, kPcDrainLimit);
      }
    }
  } else {
    // ---------------- epilogue: thread = output row ----------------
    int li = 0;
    for (int t = blockIdx.x; t < items; t += gridDim.x, li++) {
      const int mt = t % a.m_tiles, kc = t / a.m_tiles;
      const int bb = li & 1;
      const bool ok = mbar_wait(&S->acc_full[bb], (uint32_t)(li >> 1) & 1u, a.wait_limit);
      tc_fence_after();
      if (__any_sync(0xffffffffu, !ok || *(volatile int*)&S->abort)) break;
      const int64_t m = (int64_t)mt * PC_BM + tid;
      float* o = a.out + (int64_t)kc * a.chunk_stride + m * a.ldo;
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bb * PC_L);
      const bool vec = a.ncols == PC_L && (a.ldo & 3) == 0;  // whole 256-byte rows
#pragma unroll 1
      for (int ch = 0; ch < PC_L / 32; ch++) {
        uint32_t r[32];
        tmem_ld32(tl + ch * 32, r);
        if (m < a.rows_valid) {
          if (vec) {
            float4* o4 = reinterpret_cast<float4*>(o + ch * 32);
#pragma unroll
            for (int u = 0; u < 8; u++)
              __stcs(o4 + u, make_float4(__uint_as_float(r[4 * u]), __uint_as_float(r[4 * u + 1]),
                                         __uint_as_float(r[4 * u + 2]),
                                         __uint_as_float(r[4 * u + 3])));
          } else {
#pragma unroll
            for (int u = 0; u < 32; u++)
              if (ch * 32 + u < a.ncols) o[ch * 32 + u] = __uint_as_float(r[u]);
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&S->acc_empty[bb]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, PF_TMEM_COLS);
  }
}

// Fixed-order compensated sum of the K-chunk partials (rows x 64 each):
//   out[r * ldo + j] = sum_kc P[kc][r * 64 + j]   for j < ncols.
__global__ void pca_chunk_reduce_kernel(const float* __restrict__ P, int nchunk, int64_t rows,
                                        int ldo, int ncols, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * 64) return;
  const int j = (int)(e & 63);
  if (j >= ncols) return;
  const int64_t m = rows * 64;
  // compensated FP32 sum (TwoSum) in chunk order: as accurate as an FP64 sum
  // for the FP32 result, on the FP32 pipe (FP64 adds run slowly on this part)
  float s = 0.f, c = 0.f;
  int kc = 0;
  for (; kc + 4 <= nchunk; kc += 4) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; u++) v[u] = __ldcs(&P[(int64_t)(kc + u) * m + e]);
#pragma unroll
    for (int u = 0; u < 4; u++) two_sum_acc(s, c, v[u]);
  }
  for (; kc < nchunk; kc++) two_sum_acc(s, c, __ldcs(&P[(int64_t)kc * m + e]));
  out[(e >> 6) * ldo + j] = s + c;
}

// ---------------------------------------------------------------------------
// Gram matrix X^T X of a rows x 64 FP32 matrix.  Block = 4 row groups x 64
// threads; thread (grp, t) owns the 8 x 8 output tile (t / 8, t % 8) and
// accumulates it over every fourth row of the block's rpb rows (a multiple
// of 256, staged 256 rows at a time in shared memory).  kExact: each product is
// split exactly (p + e = a b by FMA) and summed with TwoSum, which keeps
// FP64-like accuracy; otherwise plain FP32 accumulation.  The four row groups
// are combined in FP64 and written as part[block][64 x 64].
// ---------------------------------------------------------------------------
template <bool kExact>
__global__ void __launch_bounds__(256)
pca_gram_kernel(const float* __restrict__ X, int64_t rows, int rpb, double* __restrict__ part) {
  extern __shared__ __align__(16) float xs[];  // 256 x 64 staged rows, then FP64 combine
  const int grp = threadIdx.x >> 6, t = threadIdx.x & 63;
  const int a0 = (t >> 3) * 8, b0 = (t & 7) * 8;
  float acc[64], cmp[kExact ? 64 : 1];
#pragma unroll
  for (int u = 0; u < 64; u++) acc[u] = 0.f;
#pragma unroll
  for (int u = 0; u < (kExact ? 64 : 1); u++) cmp[u] = 0.f;
  const int64_t r_begin = (int64_t)blockIdx.x * rpb;
  for (int sb = 0; sb < rpb / 256; sb++) {
    const int64_t rb = r_begin + sb * 256;
    if (rb >= rows) break;
    __syncthreads();
    for (int e = threadIdx.x; e < 256 * 16; e += 256) {
      const int rr = e >> 4, q = e & 15;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (rb + rr < rows) v = __ldcs(reinterpret_cast<const float4*>(X + (rb + rr) * 64) + q);
      reinterpret_cast<float4*>(xs)[e] = v;
    }
    __syncthreads();
    for (int r = grp; r < 256; r += 4) {
      const float4* xr = reinterpret_cast<const float4*>(xs + r * 64);
      const float4 p0 = xr[a0 / 4], p1 = xr[a0 / 4 + 1];
      const float4 q0 = xr[b0 / 4], q1 = xr[b0 / 4 + 1];
      const float xa[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
      const float xb[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
          if constexpr (kExact) {
            const float pr = xa[i] * xb[j];
            const float er = fmaf(xa[i], xb[j], -pr);  // exact product error
            two_sum_acc(acc[i * 8 + j], cmp[i * 8 + j], pr);
            cmp[i * 8 + j] += er;
          } else {
            acc[i * 8 + j] = fmaf(xa[i], xb[j], acc[i * 8 + j]);
          }
        }
    }
  }
  // combine the four row groups in FP64 through shared memory
  __syncthreads();
  double* red = reinterpret_cast<double*>(xs);  // 4 x 4096 doubles = 128 KB > staged area
  // two rounds of 2 groups each so that 64 KB of shared memory suffice
  double* o = part + (int64_t)blockIdx.x * 4096;
  for (int round = 0; round < 2; round++) {
    if ((grp >> 1) == round) {
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
          const int u = i * 8 + j;
          double v = (double)acc[u];
          if constexpr (kExact) v += (double)cmp[u];
          red[(grp & 1) * 4096 + (a0 + i) * 64 + b0 + j] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4096; e += 256) {
      const double v = red[e] + red[4096 + e];
      o[e] = round == 0 ? v : o[e] + v;
    }
    __syncthreads();
  }
}

__global__ void pca_gram_sum_kernel(const double* __restrict__ part, int nblk,
                                    double* __restrict__ W) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4096) return;
  double s = 0.0;
  for (int b = 0; b < nblk; b++) s += part[(int64_t)b * 4096 + e];
  W[e] = s;
}

// ---------------------------------------------------------------------------
// Cholesky W + shift I = R^T R (FP64, one block of 1024 threads, right-looking:
// column j of R, then a parallel rank-1 update of the trailing upper
// triangle, at most four entries per thread).  shift_rel > 0: shift =
// shift_rel * trace(W) (shifted CholeskyQR); a non-positive pivot retries with
// a shift growing by 1e2 from 1e-7 trace(W) (the rounding level of the
// FP32-accumulated Gram matrix).  Output: R (upper, FP32, row-major 64 x 64)
// and 1 / R_jj.  TSNE_STATUS_NONFINITE if every retry fails.
// ---------------------------------------------------------------------------
constexpr int kCholThreads = 1024;

__global__ void __launch_bounds__(kCholThreads)
pca_chol_kernel(const double* __restrict__ Wg, double shift_rel, float* __restrict__ R_out,
                float* __restrict__ rinv_out, int32_t* status) {
  __shared__ double W[64][65];
  __shared__ double piv_inv;
  __shared__ double trace;
  __shared__ int fail;
  const int tid = threadIdx.x;
  const int tc = tid & 63, tr0 = tid >> 6;  // column, first of the rows tr0 + 16 q
  if (tid < 32) {
    double t = Wg[tid * 64 + tid] + Wg[(tid + 32) * 64 + tid + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (tid == 0) trace = t;
  }
  __syncthreads();
  const double tr = trace;
  double shift = shift_rel * tr;
  for (int attempt = 0; attempt < 8; attempt++) {
    for (int e = tid; e < 4096; e += kCholThreads) {
      const int i = e >> 6, c = e & 63;
      W[i][c] = Wg[e] + (i == c ? shift : 0.0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < 64; j++) {
      if (tid == 0) {
        double d = W[j][j];
        if (!(d > 0.0)) {
          fail = 1;
          d = 1.0;
        }
        const double r = sqrt(d);
        W[j][j] = r;
        piv_inv = 1.0 / r;
      }
      __syncthreads();
      if (tid > j && tid < 64) W[j][tid] *= piv_inv;  // R[j][t]
      __syncthreads();
      // W[i][c] -= R[j][i] R[j][c] for j < i <= c
      if (tc > j) {
        const double rc = W[j][tc];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int i = tr0 + 16 * q;
          if (i > j && i <= tc) W[i][tc] -= W[j][i] * rc;
        }
      }
      __syncthreads();
    }
    if (!fail) break;
    shift = shift == 0.0 ? 1e-7 * tr : shift * 1e2;
    __syncthreads();
    if (attempt == 7 && tid == 0) raise_status(status, TSNE_STATUS_NONFINITE);
  }
  for (int e = tid; e < 4096; e += kCholThreads) {
    const int i = e >> 6, c = e & 63;
    R_out[e] = (i <= c) ? (float)W[i][c] : 0.f;
  }
  if (tid < 64) rinv_out[tid] = (float)(1.0 / W[tid][tid]);
}

// X <- X R^-1 by forward substitution per row (q R = x), optionally also
// written as the transposed BF16 split Xt[h][j][r] (r < rows_pad, zero for
// r >= rows).
__global__ void __launch_bounds__(128)
pca_apply_kernel(float* __restrict__ X, int64_t rows, int64_t rows_pad, const float* __restrict__ R,
                 const float* __restrict__ rinv, __nv_bfloat16* __restrict__ Xt) {
  __shared__ __align__(16) float Rs[64 * 64];
  __shared__ float ri[64];
  for (int e = threadIdx.x; e < 4096; e += 128) Rs[e] = R[e];
  if (threadIdx.x < 64) ri[threadIdx.x] = rinv[threadIdx.x];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (r >= rows_pad) return;
  float q[64];
  if (r < rows) {
    const float4* xr = reinterpret_cast<const float4*>(X + r * 64);
#pragma unroll
    for (int c = 0; c < 16; c++) {
      const float4 v = xr[c];
      q[4 * c] = v.x;
      q[4 * c + 1] = v.y;
      q[4 * c + 2] = v.z;
      q[4 * c + 3] = v.w;
    }
    // right-looking: once q_i is final, subtract q_i R[i][j] from every later
    // j, reading row i of R four entries at a time (entries j <= i of R are
    // zero, so only j = i itself must be left out)
#pragma unroll
    for (int i = 0; i < 64; i++) {
      const float qi = q[i] * ri[i];
#pragma unroll
      for (int j4 = (i + 1) / 4; j4 < 16; j4++) {
        const float4 rv = reinterpret_cast<const float4*>(Rs + i * 64)[j4];
        const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
        for (int u = 0; u < 4; u++)
          if (4 * j4 + u > i) q[4 * j4 + u] = fmaf(-qi, rr[u], q[4 * j4 + u]);
      }
      q[i] = qi;
    }
    float4* xw = reinterpret_cast<float4*>(X + r * 64);
#pragma unroll
    for (int c = 0; c < 16; c++)
      xw[c] = make_float4(q[4 * c], q[4 * c + 1], q[4 * c + 2], q[4 * c + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 64; j++) q[j] = 0.f;
  }
  if (Xt != nullptr) {
    const int64_t plane = (int64_t)PC_L * rows_pad;
#pragma unroll
    for (int j = 0; j < 64; j++) {
      __nv_bfloat16 hi, lo;
      split_bf16(q[j], hi, lo);
      Xt[(int64_t)j * rows_pad + r] = hi;
      Xt[plane + (int64_t)j * rows_pad + r] = lo;
    }
  }
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition of the 64 x 64 FP64 matrix G = Z^T Z.
// FP64 arithmetic is scarce on this GPU, so the O(64^3) work is FP32:
// 1. pca_eig32_kernel: cyclic Jacobi in FP32 (round-robin ordering, 32
//    disjoint rotations per round; the rotation of Golub & Van Loan's 2 x 2
//    symmetric Schur decomposition) -> V32, orthogonal to FP32 rounding.
// 2. pca_eig_refine_kernel (one block per column), FP64: W' = V32^T G V32 and
//    M = V32^T V32, both diagonal up to FP32 rounding.
// 3. pca_eig_coef_kernel: first-order solution of W' y = lambda M y around
//    the diagonal (FP64): lambda_c = W'_cc / M_cc (a Rayleigh quotient: its
//    error is second order), y_dc = (lambda_c M_dc - W'_dc) / (lambda_d -
//    lambda_c) for d != c (dropped where it exceeds 0.1, i.e. for nearly
//    equal eigenvalues, whose vectors are not determined beyond that),
//    y_cc = 1 - (M_cc - 1) / 2; descending order.
// 4. pca_eig_combine_kernel: U = V32 Y in FP64, columns in descending order;
//    pca_eig_orth_kernel: one Newton-Schulz step U (3 I - U^T U) / 2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
pca_eig32_kernel(const double* __restrict__ Gg, float* __restrict__ Vout) {
  __shared__ float W[64][65], V[64][65];
  __shared__ float cs[32][2];
  __shared__ int pp[32], qq[32];
  __shared__ float red[8];
  __shared__ int done;
  __shared__ float fro;
  const int t = threadIdx.x;
  for (int e = t; e < 4096; e += 256) {
    W[e >> 6][e & 63] = (float)Gg[e];
    V[e >> 6][e & 63] = ((e >> 6) == (e & 63)) ? 1.f : 0.f;
  }
  __syncthreads();
  {
    float f = 0.f;
    for (int e = t; e < 4096; e += 256) f += W[e >> 6][e & 63] * W[e >> 6][e & 63];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
    if ((t & 31) == 0) red[t >> 5] = f;
    __syncthreads();
    if (t == 0) {
      float s = 0.f;
      for (int w = 0; w < 8; w++) s += red[w];
      fro = s;
    }
    __syncthreads();
  }
  for (int sweep = 0; sweep < 30; sweep++) {
    for (int rnd = 0; rnd < 63; rnd++) {
      if (t < 32) {
        const int a = t == 0 ? 0 : 1 + (t - 1 + rnd) % 63;
        const int b = 1 + (62 - t + rnd) % 63;  // position 63 - t of the round-robin
        const int p = min(a, b), q = max(a, b);
        pp[t] = p;
        qq[t] = q;
        const float apq = W[p][q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) > 1e-30f * (fabsf(W[p][p]) + fabsf(W[q][q])) && apq != 0.f) {
          const float tau = (W[q][q] - W[p][p]) / (2.f * apq);
          const float tt = (tau >= 0.f ? 1.f : -1.f) / (fabsf(tau) + sqrtf(1.f + tau * tau));
          c = rsqrtf(1.f + tt * tt);
          s = tt * c;
        }
        cs[t][0] = c;
        cs[t][1] = s;
      }
      __syncthreads();
      for (int e = t; e < 32 * 64; e += 256) {  // rows: W <- J^T W
        const int k = e >> 6, j = e & 63;
        const int p = pp[k], q = qq[k];
        const float c = cs[k][0], s = cs[k][1];
        const float wp = W[p][j], wq = W[q][j];
        W[p][j] = c * wp - s * wq;
        W[q][j] = s * wp + c * wq;
      }
      __syncthreads();
      for (int e = t; e < 32 * 64; e += 256) {  // columns: W <- W J, V <- V J
        const int k = e >> 6, j = e & 63;
        const int p = pp[k], q = qq[k];
        const float c = cs[k][0], s = cs[k][1];
        const float wp = W[j][p], wq = W[j][q];
        W[j][p] = c * wp - s * wq;
        W[j][q] = s * wp + c * wq;
        const float vp = V[j][p], vq = V[j][q];
        V[j][p] = c * vp - s * vq;
        V[j][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    float off = 0.f;
    for (int e = t; e < 4096; e += 256)
      if ((e >> 6) != (e & 63)) off += W[e >> 6][e & 63] * W[e >> 6][e & 63];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_down_sync(0xffffffffu, off, o);
    if ((t & 31) == 0) red[t >> 5] = off;
    __syncthreads();
    if (t == 0) {
      float sum = 0.f;
      for (int w = 0; w < 8; w++) sum += red[w];
      done = sum <= 1e-13f * fro;  // off-diagonal norm ~ FP32 rounding of the matrix
    }
    __syncthreads();
    if (done) break;
  }
  for (int e = t; e < 4096; e += 256) Vout[e] = V[e >> 6][e & 63];
}

__global__ void __launch_bounds__(64)
pca_eig_refine_kernel(const double* __restrict__ G, const float* __restrict__ V,
                      double* __restrict__ Wp, double* __restrict__ M) {
  __shared__ double gv[64], vc[64];
  const int c = blockIdx.x, t = threadIdx.x;
  vc[t] = (double)V[t * 64 + c];
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < 64; k++) s += G[t * 64 + k] * vc[k];  // (G v_c)_t
  gv[t] = s;
  __syncthreads();
  double w = 0.0, m = 0.0;
  for (int k = 0; k < 64; k++) {
    const double vk = (double)V[k * 64 + t];  // entry k of column t
    w += vk * gv[k];
    m += vk * vc[k];
  }
  Wp[t * 64 + c] = w;  // v_t^T G v_c
  M[t * 64 + c] = m;   // v_t^T v_c
}

__global__ void __launch_bounds__(64)
pca_eig_coef_kernel(const double* __restrict__ Wp, const double* __restrict__ M,
                    double* __restrict__ lam, double* __restrict__ Y) {
  __shared__ double l[64];
  __shared__ int order[64];
  const int c = threadIdx.x;
  l[c] = Wp[c * 64 + c] / M[c * 64 + c];
  __syncthreads();
  for (int d = 0; d < 64; d++) {
    double y;
    if (d == c) {
      y = 1.0 - 0.5 * (M[c * 64 + c] - 1.0);
    } else {
      const double den = l[d] - l[c];
      const double num = l[c] * M[d * 64 + c] - Wp[d * 64 + c];
      y = (den != 0.0 && fabs(num) <= 0.1 * fabs(den)) ? num / den : 0.0;
    }
    Y[d * 64 + c] = y;
  }
  if (c == 0) {
    for (int i = 0; i < 64; i++) order[i] = i;
    for (int i = 1; i < 64; i++) {  // descending, ties keep the lower index first
      const int v = order[i];
      int j = i - 1;
      while (j >= 0 && l[order[j]] < l[v]) {
        order[j + 1] = order[j];
        j--;
      }
      order[j + 1] = v;
    }
  }
  __syncthreads();
  lam[c] = l[order[c]];
  lam[64 + c] = (double)order[c];  // source column of sorted position c
}

// U[:, c] = V32 y_src(c) in FP64, src(c) the column of the c-th largest eigenvalue.
__global__ void __launch_bounds__(64)
pca_eig_combine_kernel(const float* __restrict__ V, const double* __restrict__ Y,
                       const double* __restrict__ lam, double* __restrict__ U) {
  const int c = blockIdx.x, t = threadIdx.x;
  const int src = (int)lam[64 + c];
  double s = 0.0;
  for (int d = 0; d < 64; d++) s += (double)V[t * 64 + d] * Y[d * 64 + src];
  U[t * 64 + c] = s;
}

// One Newton-Schulz step towards the nearest orthogonal matrix:
// Uo[:, c] = 1.5 U[:, c] - 0.5 U (U^T U)[:, c].
__global__ void __launch_bounds__(64)
pca_eig_orth_kernel(const double* __restrict__ U, double* __restrict__ Uo) {
  __shared__ double m[64], uc[64];
  const int c = blockIdx.x, t = threadIdx.x;
  uc[t] = U[t * 64 + c];
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < 64; k++) s += U[k * 64 + t] * uc[k];  // (U^T U)[t][c]
  m[t] = s;
  __syncthreads();
  double v = 0.0;
  for (int d = 0; d < 64; d++) v += U[t * 64 + d] * m[d];
  Uo[t * 64 + c] = 1.5 * uc[t] - 0.5 * v;
}

// Components V[c][col] = (Z[col,:] . U[:, c]) / sigma_c for c < k, col < g:
// one thread per (col, c), FP64 arithmetic, FP32 output.
__global__ void __launch_bounds__(256)
pca_components_kernel(const float* __restrict__ Z, int g, int k, const double* __restrict__ lam,
                      const double* __restrict__ U, float* __restrict__ comp) {
  const int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (e >= (int64_t)g * k) return;
  const int col = (int)(e / k), c = (int)(e % k);
  const float4* z4 = reinterpret_cast<const float4*>(Z + (int64_t)col * 64);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 16; q++) {
    const float4 z = z4[q];
    s += (double)z.x * U[(4 * q) * 64 + c] + (double)z.y * U[(4 * q + 1) * 64 + c] +
         (double)z.z * U[(4 * q + 2) * 64 + c] + (double)z.w * U[(4 * q + 3) * 64 + c];
  }
  const double l = lam[c];
  comp[(int64_t)c * g + col] = (float)(l > 0.0 ? s / sqrt(l) : 0.0);
}

// One block per component: the entry of largest magnitude (lowest index among
// ties) decides the sign; the row is flipped in place and sign[c] recorded.
__global__ void __launch_bounds__(256)
pca_sign_kernel(float* __restrict__ comp, int g, float* __restrict__ sign) {
  __shared__ float bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  float* v = comp + (int64_t)c * g;
  float best = -1.f;
  int bidx = 0x7fffffff;
  for (int i = threadIdx.x; i < g; i += 256) {
    const float a = fabsf(v[i]);
    if (a > best) {  // increasing i: the first maximum of this thread is kept
      best = a;
      bidx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const float a = bv[threadIdx.x + o];
      const int ai = bi[threadIdx.x + o];
      if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ai < bi[threadIdx.x])) {
        bv[threadIdx.x] = a;
        bi[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const float sg = (bi[0] < g && v[bi[0]] < 0.f) ? -1.f : 1.f;
  __syncthreads();
  if (sg < 0.f)
    for (int i = threadIdx.x; i < g; i += 256) v[i] = -v[i];
  if (threadIdx.x == 0) sign[c] = sg;
}

// Scores T[r][c] = sign_c sigma_c (Q[r,:] . U[:, c]) for c < k.  A block of
// 128 threads stages 128 rows of Q in shared memory (coalesced), each thread
// forms its row's k scores with M[j][c] = sign_c sigma_c U[j][c] read four
// columns at a time, and the block writes its 128 x k scores (contiguous in
// T) back through shared memory with coalesced stores.
constexpr int SC_ROWS = 128;
constexpr int SC_LD = 68;  // shared row stride (floats): 16-byte rows, few bank conflicts
constexpr size_t kScoresSmem = (size_t)(SC_ROWS * SC_LD + 64 * 64) * sizeof(float);

// The 64 x 64 right factor of the scores, M[r][c] = U[r][c] sqrt(lam_c) sign_c
// (zero for c >= k), formed once in FP64 and rounded to FP32 (the square roots
// are FP64, which this part runs slowly: once per fit, not once per row tile).
__global__ void pca_scores_matrix_kernel(int k, const double* __restrict__ lam,
                                         const double* __restrict__ U,
                                         const float* __restrict__ sign, float* __restrict__ M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4096) return;
  const int c = e & 63;
  M[e] = c < k ? (float)(U[e] * sqrt(fmax(lam[c], 0.0))) * sign[c] : 0.f;
}

__global__ void __launch_bounds__(SC_ROWS)
pca_scores_kernel(const float* __restrict__ Q, int64_t n, int k, const float* __restrict__ Msc,
                  float* __restrict__ T) {
  extern __shared__ __align__(16) float scs[];
  float* Qs = scs;                     // [128][SC_LD], later the 128 x k output tile
  float* M = scs + SC_ROWS * SC_LD;    // [64][64]
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * SC_ROWS;
  const int rows = (int)min((int64_t)SC_ROWS, n - r0);
  for (int e = t; e < 4096; e += SC_ROWS) M[e] = Msc[e];
  const float4* q4 = reinterpret_cast<const float4*>(Q + r0 * 64);
  for (int e = t; e < rows * 16; e += SC_ROWS) {
    const int r = e >> 4, c4 = e & 15;
    *reinterpret_cast<float4*>(&Qs[r * SC_LD + 4 * c4]) = __ldcs(q4 + e);
  }
  __syncthreads();
  float acc[64];
#pragma unroll
  for (int c = 0; c < 64; c++) acc[c] = 0.f;
  if (t < rows) {
#pragma unroll
    for (int q = 0; q < 16; q++) {
      const float4 v = *reinterpret_cast<const float4*>(&Qs[t * SC_LD + 4 * q]);
      const float y[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const float4* mr = reinterpret_cast<const float4*>(M + (4 * q + u) * 64);
#pragma unroll
        for (int c4 = 0; c4 < 16; c4++) {
          const float4 m = mr[c4];
          acc[4 * c4] = fmaf(y[u], m.x, acc[4 * c4]);
          acc[4 * c4 + 1] = fmaf(y[u], m.y, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(y[u], m.z, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(y[u], m.w, acc[4 * c4 + 3]);
        }
      }
    }
  }
  __syncthreads();  // Qs is reused as the output tile
  if (t < rows) {
#pragma unroll
    for (int c = 0; c < 64; c++)
      if (c < k) Qs[t * k + c] = acc[c];
  }
  __syncthreads();
  float* out = T + r0 * k;
  for (int e = t; e < rows * k; e += SC_ROWS) __stcs(out + e, Qs[e]);
}

// sigma_c = sqrt(lam_c), explained variance lam_c / (n - 1).
__global__ void pca_sigma_kernel(const double* __restrict__ lam, int k, int64_t n,
                                 double* __restrict__ sigma, double* __restrict__ ev) {
  const int c = threadIdx.x;
  if (c >= k) return;
  const double l = fmax(lam[c], 0.0);
  if (sigma) sigma[c] = sqrt(l);
  if (ev) ev[c] = l / (double)(n - 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static size_t pal(size_t x) { return (x + 255) & ~(size_t)255; }

// Gram launch shape: at most PC_GRAM_BLOCKS blocks of rpb rows (multiple of 256).
static void gram_shape(int64_t rows, int* blocks, int* rpb) {
  const int64_t sub = (rows + 255) / 256;
  const int64_t b = sub < PC_GRAM_BLOCKS ? sub : PC_GRAM_BLOCKS;
  const int64_t per = (sub + b - 1) / b;
  *rpb = (int)(per * 256);
  *blocks = (int)((rows + *rpb - 1) / *rpb);
}

struct PcaLayout {
  int64_t n, np;
  int g, gp;
  int m_tiles_rows, m_tiles_cols, nchunk, kpc, kb_rows, kb_cols, nchunk_rows;
  size_t off_mean, off_mh, off_ml, off_colpart, off_ssq, off_Y, off_Yp, off_Qt, off_Zp, off_Z, off_Wt,
      off_gpart, off_W, off_R, off_rinv, off_V32, off_Wp, off_M, off_Yc, off_lam, off_U, off_sign,
      off_Msc,
      total;
};

static PcaLayout pca_layout(int64_t n, int g, bool with_fit) {
  PcaLayout L{};
  L.n = n;
  L.g = g;
  L.gp = (int)round_up(g, 128);
  L.np = round_up(n, 64);
  L.m_tiles_rows = (int)((n + PC_BM - 1) / PC_BM);
  L.m_tiles_cols = L.gp / PC_BM;
  L.kb_rows = L.gp / PC_BK;
  L.kb_cols = (int)(L.np / PC_BK);
  // The tensor cores' FP32 accumulation is not round-to-nearest: summed over K
  // values it drifts towards zero by about 3e-9 K relative (measured).  Every
  // accumulation therefore covers at most PC_KSEG K blocks (2048 values) and
  // the segments are summed in a fixed order with compensated (TwoSum) FP32
  // arithmetic, as accurate as FP64 for the FP32 result.
  L.kpc = PC_KSEG;
  L.nchunk = (L.kb_cols + L.kpc - 1) / L.kpc;
  L.nchunk_rows = (L.kb_rows + PC_KSEG - 1) / PC_KSEG;
  const int64_t gblk = PC_GRAM_BLOCKS;
  const size_t F = with_fit ? 1 : 0;
  size_t o = 0;
  L.off_mean = o;    o = pal(o + sizeof(double) * L.gp);
  L.off_mh = o;      o = pal(o + sizeof(float) * L.gp);
  L.off_ml = o;      o = pal(o + sizeof(float) * L.gp);
  L.off_colpart = o; o = pal(o + F * 2 * sizeof(double) * PC_COLSUM_CH * g);
  L.off_ssq = o;     o = pal(o + F * sizeof(double) * L.gp);
  L.off_Y = o;       o = pal(o + F * sizeof(float) * (size_t)L.np * PC_L);
  L.off_Yp = o;      o = pal(o + (L.nchunk_rows > 1 ? sizeof(float) * (size_t)L.nchunk_rows *
                                                         (size_t)n * PC_L : 0));
  L.off_Qt = o;      o = pal(o + F * 2 * sizeof(__nv_bfloat16) * (size_t)PC_L * L.np);
  L.off_Zp = o;      o = pal(o + F * sizeof(float) * (size_t)L.nchunk * L.gp * PC_L);
  L.off_Z = o;       o = pal(o + F * sizeof(float) * (size_t)L.gp * PC_L);
  L.off_Wt = o;      o = pal(o + 2 * sizeof(__nv_bfloat16) * (size_t)PC_L * L.gp);
  L.off_gpart = o;   o = pal(o + F * sizeof(double) * 4096 * (size_t)gblk);
  L.off_W = o;       o = pal(o + sizeof(double) * 4096);
  L.off_R = o;       o = pal(o + sizeof(float) * 4096);
  L.off_rinv = o;    o = pal(o + sizeof(float) * 64);
  L.off_V32 = o;     o = pal(o + sizeof(float) * 4096);
  L.off_Wp = o;      o = pal(o + sizeof(double) * 4096);
  L.off_M = o;       o = pal(o + sizeof(double) * 4096);
  L.off_Yc = o;      o = pal(o + sizeof(double) * 4096);
  L.off_lam = o;     o = pal(o + sizeof(double) * 128);
  L.off_U = o;       o = pal(o + sizeof(double) * 4096);
  L.off_sign = o;    o = pal(o + sizeof(float) * 64);
  L.off_Msc = o;     o = pal(o + sizeof(float) * 4096);
  L.total = o;
  return L;
}

size_t pca_ws_bytes(int64_t n, int g, bool fit) { return pca_layout(n, g, fit).total; }

// A must start on 16 bytes with a row stride of a multiple of 16 bytes (TMA).
bool pca_layout_ok(const float* A, int64_t lda) {
  return ((reinterpret_cast<uintptr_t>(A) & 15) == 0) && (lda % 4 == 0);
}

static bool encode_2d(CUtensorMap* tm, CUtensorMapDataType dt, const void* base, uint64_t inner,
                      uint64_t outer, uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

static int g_num_sms = 0;

// One product with the centred A (see pca_gemm_kernel); B: 2 planes of
// 64 x b_inner BF16.
template <bool kTrans>
static cudaError_t run_gemm(const float* A, int64_t n, int g, int64_t lda,
                            const __nv_bfloat16* B, uint64_t b_inner, int m_tiles, int nchunk,
                            int kpc, int kb_total, int64_t rows_valid, int ldo, int ncols,
                            int64_t chunk_stride, float* out, const float* mh, const float* ml,
                            int32_t* status, cudaStream_t st) {
  CUtensorMap ta, tbh, tbl;
  const uint64_t b_plane = b_inner * (uint64_t)PC_L;
  if (!encode_2d(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, A, (uint64_t)g, (uint64_t)n,
                 (uint64_t)lda * 4, 32, kTrans ? 64 : PC_BM) ||
      !encode_2d(&tbh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B, b_inner, PC_L, b_inner * 2, PC_BK,
                 PC_L) ||
      !encode_2d(&tbl, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, B + b_plane, b_inner, PC_L,
                 b_inner * 2, PC_BK, PC_L))
    return cudaErrorInvalidValue;
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  cudaError_t e = cudaFuncSetAttribute(pca_gemm_kernel<kTrans>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPfSmemBytes);
  if (e != cudaSuccess) return e;
  PfArgs ga;
  ga.m_tiles = m_tiles;
  ga.nchunk = nchunk;
  ga.kpc = kpc;
  ga.kb_total = kb_total;
  ga.n = n;
  ga.g = g;
  ga.rows_valid = rows_valid;
  ga.ldo = ldo;
  ga.ncols = ncols;
  ga.chunk_stride = chunk_stride;
  ga.out = out;
  ga.mh = mh;
  ga.ml = ml;
  ga.status = status;
  ga.wait_limit = 4000000000ll;
  const int items = m_tiles * nchunk;
  const int grid = items < g_num_sms ? items : g_num_sms;
  pca_gemm_kernel<kTrans><<<grid, PF_THREADS, kPfSmemBytes, st>>>(ta, tbh, tbl, ga);
  return cudaGetLastError();
}

// Orthonormal basis of the columns of X (rows x 64, row stride 64), in place:
// CholeskyQR passes (the first one optionally shifted by shift_rel *
// trace(X^T X); a pivot that fails retries with a growing shift).  The last
// pass also writes the transposed split Xt (64 x rows_pad) when Xt is given.
struct OrthBufs {
  double* gpart;
  double* W;
  float* R;
  float* rinv;
};

static cudaError_t orth(float* X, int64_t rows, int64_t rows_pad, __nv_bfloat16* Xt, int passes,
                        double shift_rel, const OrthBufs& b, int32_t* status, cudaStream_t st) {
  int gblk, rpb;
  gram_shape(rows, &gblk, &rpb);
  cudaError_t e = cudaFuncSetAttribute(pca_gram_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       256 * 64 * (int)sizeof(float));
  if (e != cudaSuccess) return e;
  for (int p = 0; p < passes; p++) {
    pca_gram_kernel<false><<<gblk, 256, 256 * 64 * sizeof(float), st>>>(X, rows, rpb, b.gpart);
    pca_gram_sum_kernel<<<16, 256, 0, st>>>(b.gpart, gblk, b.W);
    pca_chol_kernel<<<1, kCholThreads, 0, st>>>(b.W, p == 0 ? shift_rel : 0.0, b.R, b.rinv,
                                                status);
    const bool last = p == passes - 1;
    const int64_t r_launch = (last && Xt) ? rows_pad : rows;
    pca_apply_kernel<<<(unsigned)((r_launch + 127) / 128), 128, 0, st>>>(
        X, rows, rows_pad, b.R, b.rinv, last ? Xt : nullptr);
  }
  return cudaGetLastError();
}

// Ac W for all n rows into out (row stride ldo, first ncols columns): one
// accumulation per K segment; with several segments the partials (Yp,
// nseg x n x 64) are summed with compensated FP32 arithmetic in a fixed order.
static cudaError_t rows_gemm(const float* A, int64_t n, int g, int64_t lda,
                             const __nv_bfloat16* Wt, const PcaLayout& L, float* Yp, float* out,
                             int ldo, int ncols, const float* mh, const float* ml,
                             int32_t* status, cudaStream_t st) {
  if (L.nchunk_rows == 1)
    return run_gemm<false>(A, n, g, lda, Wt, (uint64_t)L.gp, L.m_tiles_rows, 1, L.kb_rows,
                           L.kb_rows, n, ldo, ncols, 0, out, mh, ml, status, st);
  cudaError_t r = run_gemm<false>(A, n, g, lda, Wt, (uint64_t)L.gp, L.m_tiles_rows,
                                  L.nchunk_rows, PC_KSEG, L.kb_rows, n, PC_L, PC_L,
                                  n * PC_L, Yp, mh, ml, status, st);
  if (r != cudaSuccess) return r;
  pca_chunk_reduce_kernel<<<(unsigned)((n * PC_L + 255) / 256), 256, 0, st>>>(
      Yp, L.nchunk_rows, n, ldo, ncols, out);
  return cudaGetLastError();
}

cudaError_t launch_pca_fit(const float* A, int64_t n, int g, int64_t lda, int k, int n_power,
                           const float* omega, float* scores, float* comp, double* sigma,
                           double* ev, double* mean_out, double* total_var, void* ws,
                           int32_t* status, cudaStream_t st) {
  const PcaLayout L = pca_layout(n, g, true);
  char* w = static_cast<char*>(ws);
  double* mean = reinterpret_cast<double*>(w + L.off_mean);
  float* mh = reinterpret_cast<float*>(w + L.off_mh);
  float* ml = reinterpret_cast<float*>(w + L.off_ml);
  double* colpart = reinterpret_cast<double*>(w + L.off_colpart);
  double* ssq = reinterpret_cast<double*>(w + L.off_ssq);
  float* Y = reinterpret_cast<float*>(w + L.off_Y);
  float* Yp = reinterpret_cast<float*>(w + L.off_Yp);
  __nv_bfloat16* Qt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Qt);
  float* Zp = reinterpret_cast<float*>(w + L.off_Zp);
  float* Z = reinterpret_cast<float*>(w + L.off_Z);
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Wt);
  double* gpart = reinterpret_cast<double*>(w + L.off_gpart);
  double* W = reinterpret_cast<double*>(w + L.off_W);
  OrthBufs ob;
  ob.gpart = gpart;
  ob.W = W;
  ob.R = reinterpret_cast<float*>(w + L.off_R);
  ob.rinv = reinterpret_cast<float*>(w + L.off_rinv);
  float* V32 = reinterpret_cast<float*>(w + L.off_V32);
  double* Wp = reinterpret_cast<double*>(w + L.off_Wp);
  double* Mm = reinterpret_cast<double*>(w + L.off_M);
  double* Yc = reinterpret_cast<double*>(w + L.off_Yc);
  double* lam = reinterpret_cast<double*>(w + L.off_lam);
  double* U = reinterpret_cast<double*>(w + L.off_U);
  float* sign = reinterpret_cast<float*>(w + L.off_sign);
  float* Msc = reinterpret_cast<float*>(w + L.off_Msc);

  // column means (and their FP32 hi / lo split used by the converters)
  pca_colsum_kernel<<<dim3((g + 255) / 256, PC_COLSUM_CH), 256, 0, st>>>(A, n, g, lda, colpart);
  pca_colmean_kernel<<<(L.gp + 255) / 256, 256, 0, st>>>(colpart, n, g, L.gp, mean, mh, ml,
                                                         ssq);
  pca_sum_kernel<<<1, 256, 0, st>>>(ssq, L.gp, 1.0 / (double)(n - 1), total_var);
  pca_sketch_split_kernel<<<(unsigned)((PC_L * (int64_t)L.gp + 255) / 256), 256, 0, st>>>(
      omega, g, L.gp, PC_L, 0, Wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  // CholeskyQR: a shift is added only where a pivot fails (a fixed shift
  // would damp the weak directions that later products must keep)
  const double kShift = 0.0;
  auto rows_product = [&](int passes) -> cudaError_t {  // Y = Ac W, Q = orth(Y) (+ Qt)
    cudaError_t r = rows_gemm(A, n, g, lda, Wt, L, Yp, Y, PC_L, PC_L, mh, ml, status, st);
    if (r != cudaSuccess) return r;
    return orth(Y, n, L.np, Qt, passes, kShift, ob, status, st);
  };
  auto cols_product = [&]() -> cudaError_t {  // Z = Ac^T Q (K-split, FP64 chunk sums)
    cudaError_t r = run_gemm<true>(A, n, g, lda, Qt, (uint64_t)L.np, L.m_tiles_cols, L.nchunk,
                                   L.kpc, L.kb_cols, L.gp, PC_L, PC_L, (int64_t)L.gp * PC_L, Zp,
                                   mh, ml, status, st);
    if (r != cudaSuccess) return r;
    const int64_t m = (int64_t)L.gp * PC_L;
    pca_chunk_reduce_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(Zp, L.nchunk, L.gp,
                                                                          PC_L, PC_L, Z);
    return cudaGetLastError();
  };
  // intermediate bases only need to be well conditioned (one pass); the basis
  // of the Rayleigh-Ritz step gets two
  if ((e = rows_product(n_power == 0 ? 2 : 1)) != cudaSuccess) return e;
  for (int it = 0; it < n_power; it++) {
    if ((e = cols_product()) != cudaSuccess) return e;
    if ((e = orth(Z, L.gp, L.gp, Wt, 1, kShift, ob, status, st)) != cudaSuccess) return e;
    if ((e = rows_product(it == n_power - 1 ? 2 : 1)) != cudaSuccess) return e;
  }
  if ((e = cols_product()) != cudaSuccess) return e;
  // Rayleigh-Ritz: Z^T Z = U diag(lam) U^T (compensated Gram, FP32 Jacobi,
  // FP64 first-order correction, Newton-Schulz)
  int zblk, zrpb;
  gram_shape(L.gp, &zblk, &zrpb);
  e = cudaFuncSetAttribute(pca_gram_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           256 * 64 * (int)sizeof(float));
  if (e != cudaSuccess) return e;
  pca_gram_kernel<true><<<zblk, 256, 256 * 64 * sizeof(float), st>>>(Z, L.gp, zrpb, gpart);
  pca_gram_sum_kernel<<<16, 256, 0, st>>>(gpart, zblk, W);
  pca_eig32_kernel<<<1, 256, 0, st>>>(W, V32);
  pca_eig_refine_kernel<<<64, 64, 0, st>>>(W, V32, Wp, Mm);
  pca_eig_coef_kernel<<<1, 64, 0, st>>>(Wp, Mm, lam, Yc);
  pca_eig_combine_kernel<<<64, 64, 0, st>>>(V32, Yc, lam, Mm);
  pca_eig_orth_kernel<<<64, 64, 0, st>>>(Mm, U);
  pca_components_kernel<<<(unsigned)(((int64_t)g * k + 255) / 256), 256, 0, st>>>(Z, g, k, lam, U,
                                                                                comp);
  pca_sign_kernel<<<k, 256, 0, st>>>(comp, g, sign);
  e = cudaFuncSetAttribute(pca_scores_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kScoresSmem);
  if (e != cudaSuccess) return e;
  pca_scores_matrix_kernel<<<16, 256, 0, st>>>(k, lam, U, sign, Msc);
  pca_scores_kernel<<<(unsigned)((n + SC_ROWS - 1) / SC_ROWS), SC_ROWS, kScoresSmem, st>>>(
      Y, n, k, Msc, scores);
  pca_sigma_kernel<<<1, 64, 0, st>>>(lam, k, n, sigma, ev);
  if (mean_out)
    cudaMemcpyAsync(mean_out, mean, sizeof(double) * g, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

cudaError_t launch_pca_transform(const float* A, int64_t n, int g, int64_t lda,
                                 const double* mean_in, const float* comp, int k, float* scores,
                                 void* ws, int32_t* status, cudaStream_t st) {
  const PcaLayout L = pca_layout(n, g, false);
  char* w = static_cast<char*>(ws);
  float* mh = reinterpret_cast<float*>(w + L.off_mh);
  float* ml = reinterpret_cast<float*>(w + L.off_ml);
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Wt);
  pca_mean_split_kernel<<<(L.gp + 255) / 256, 256, 0, st>>>(mean_in, g, L.gp, mh, ml);
  pca_sketch_split_kernel<<<(unsigned)((PC_L * (int64_t)L.gp + 255) / 256), 256, 0, st>>>(
      comp, g, L.gp, k, 1, Wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float* Yp = reinterpret_cast<float*>(w + L.off_Yp);
  return rows_gemm(A, n, g, lda, Wt, L, Yp, scores, k, k, mh, ml, status, st);
}

}  // namespace tsne
