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
// * prep: column means (compensated FP32 sums, FP64 across chunks), then one
//   pass that centres A, splits every value x into BF16 hi + lo (x - hi - lo
//   is at most 2^-18 |x|) and writes the split matrix row-major (n x gp) and
//   transposed (gp x np).  Both products below are then K-major for tcgen05.
// * the two products Ac W (M = n, K = g) and Ac^T Q (M = g, K = n, split over
//   K into chunks reduced in FP64 in a fixed order) run in one persistent
//   tcgen05 kernel: a TMA producer warp streams 128 x 64 BF16 tiles of the
//   hi and lo planes of A and 64 x 64 tiles of the sketch, one thread issues
//   three M128 N64 K16 MMAs per K step (hi.hi + hi.lo + lo.hi, FP32
//   accumulation in tensor memory, two accumulators), four epilogue warps
//   drain tensor memory to global.  Each pass streams the split matrix once:
//   HBM-bound, tensor pipe lightly loaded.
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
constexpr int PC_STAGES = 4;
constexpr int PC_THREADS = 192;    // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr int PC_A_BYTES = PC_BM * PC_BK * 2;   // 16 KB per plane
constexpr int PC_B_BYTES = PC_L * PC_BK * 2;    // 8 KB per plane
constexpr int PC_STAGE_BYTES = 2 * PC_A_BYTES + 2 * PC_B_BYTES;  // 48 KB
constexpr int PC_GRAM_ROWS = 2048;  // rows per Gram block (8 sub-blocks of 256)
constexpr int PC_COLSUM_CH = 256;   // row chunks of the column sums

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
  float s = 0.f, e = 0.f;
  int64_t r = r0;
  for (; r + 4 <= r1; r += 4) {
    const float v0 = __ldcs(&A[r * lda + c]), v1 = __ldcs(&A[(r + 1) * lda + c]);
    const float v2 = __ldcs(&A[(r + 2) * lda + c]), v3 = __ldcs(&A[(r + 3) * lda + c]);
    two_sum_acc(s, e, v0);
    two_sum_acc(s, e, v1);
    two_sum_acc(s, e, v2);
    two_sum_acc(s, e, v3);
  }
  for (; r < r1; r++) two_sum_acc(s, e, __ldcs(&A[r * lda + c]));
  part[(int64_t)ch * g + c] = (double)s + (double)e;
}

__global__ void pca_colmean_kernel(const double* __restrict__ part, int64_t n, int g, int gp,
                                   double* __restrict__ mean) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gp) return;
  double s = 0.0;
  if (c < g)
    for (int ch = 0; ch < PC_COLSUM_CH; ch++) s += part[(int64_t)ch * g + c];
  mean[c] = c < g ? s / (double)n : 0.0;
}

// ---------------------------------------------------------------------------
// Centre + BF16 hi/lo split.  Tile of 64 rows x 64 columns per block.
//   As[h][r][c]  (h = 0 hi, 1 lo; r < n, c < gp; zero for c >= g)
//   At[h][c][r]  (c < gp, r < np; zero for r >= n or c >= g), optional
// ssq[block] = sum of squared centred values (for the total variance).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

__global__ void __launch_bounds__(256)
pca_prep_kernel(const float* __restrict__ A, int64_t n, int g, int64_t lda, int gp, int64_t np,
                const double* __restrict__ mean, __nv_bfloat16* __restrict__ As,
                __nv_bfloat16* __restrict__ At, double* __restrict__ ssq) {
  __shared__ __nv_bfloat16 th[64][66], tl[64][66];  // [column][row], padded
  __shared__ double red[8];
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 4 rows per pass
  const int c = blockIdx.y * 64 + tx;                       // grid: x = row tile, y = column tile
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  float mh = 0.f, ml = 0.f;
  if (c < g) {
    const double m = mean[c];
    mh = (float)m;
    ml = (float)(m - (double)mh);
  }
  const int64_t plane = n * (int64_t)gp;
  float ss = 0.f, se = 0.f;
#pragma unroll 4
  for (int i = 0; i < 16; i++) {
    const int rr = ty + 4 * i;
    const int64_t r = r0 + rr;
    float x = 0.f;
    if (r < n && c < g) x = (__ldcs(&A[r * lda + c]) - mh) - ml;
    __nv_bfloat16 hi, lo;
    split_bf16(x, hi, lo);
    if (r < n && c < gp) {
      As[r * gp + c] = hi;
      As[plane + r * gp + c] = lo;
    }
    th[tx][rr] = hi;
    tl[tx][rr] = lo;
    two_sum_acc(ss, se, x * x);
  }
  if (At != nullptr) {
    __syncthreads();
    // 64 columns x 64 rows of each plane: thread writes 8 consecutive rows (16 B)
    const int64_t tplane = (int64_t)gp * np;
    for (int e = threadIdx.x; e < 2 * 64 * 8; e += 256) {
      const int h = e >> 9, col = (e >> 3) & 63, seg = e & 7;
      const int cc = blockIdx.y * 64 + col;
      const int64_t rr = r0 + seg * 8;
      if (cc < gp && rr < np) {
        const __nv_bfloat16(*t)[66] = h ? tl : th;
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = t[col][seg * 8 + u];
        *reinterpret_cast<uint4*>(&At[h * tplane + (int64_t)cc * np + rr]) =
            *reinterpret_cast<const uint4*>(v);
      }
    }
  }
  // block sum of squares (fixed order)
  double d = (double)ss + (double)se;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0 && ssq != nullptr) {
    double t = 0.0;
    for (int w = 0; w < 8; w++) t += red[w];
    ssq[(int64_t)blockIdx.x * gridDim.y + blockIdx.y] = t;
  }
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
// tcgen05 product.  Item t: m-tile mt = t % m_tiles, K chunk kc = t / m_tiles
// (k blocks [kc * kpc, min(kb_total, (kc + 1) * kpc))).
//   out[kc * chunk_stride + m * ldo + j] = sum over the chunk's K of
//       A[m, k] * B[j, k]  for m < rows_valid, j < ncols
// with A = Ahi + Alo (tensor maps tmA[2], M x K) and B = Bhi + Blo (tmB[2],
// 64 x K), computed as Ahi.Bhi + Ahi.Blo + Alo.Bhi in FP32.
// ---------------------------------------------------------------------------
struct PcSmem {
  uint64_t full[PC_STAGES], empty[PC_STAGES], acc_full[2], acc_empty[2], drain;
  uint32_t tmem_slot;
  int abort;
};
constexpr size_t kPcSmemBytes = 1024 + (size_t)PC_STAGE_BYTES * PC_STAGES + sizeof(PcSmem);

struct PcGemmArgs {
  int m_tiles, nchunk, kpc, kb_total;
  int64_t rows_valid;
  int ldo, ncols;
  int64_t chunk_stride;
  float* out;
  int32_t* status;
  long long wait_limit;
};

__device__ __forceinline__ bool pc_epi_bar_or(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q, o;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred o, 1, 128, q;\n"
      " selp.u32 %0, 1, 0, o;\n}"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(PC_THREADS, 1)
pca_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                const PcGemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  PcSmem* S = reinterpret_cast<PcSmem*>(base + (size_t)PC_STAGE_BYTES * PC_STAGES);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int items = a.m_tiles * a.nchunk;

  if (tid == 0) {
    for (int q = 0; q < PC_STAGES; q++) {
      mbar_init(&S->full[q], 1);
      mbar_init(&S->empty[q], 1);
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
  if (warp == 5) tmem_alloc(&S->tmem_slot, 2 * PC_L);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->tmem_slot;

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long it = 0, issued = 0;
      bool ok = true;
      for (int t = blockIdx.x; ok && t < items; t += gridDim.x) {
        const int mt = t % a.m_tiles, kc = t / a.m_tiles;
        const int kb0 = kc * a.kpc, kb1 = min(a.kb_total, kb0 + a.kpc);
        for (int kb = kb0; kb < kb1; kb++, it++) {
          const int q = (int)(it % PC_STAGES);
          if (it >= PC_STAGES) {
            if (*(volatile int*)&S->abort ||
                !mbar_wait(&S->empty[q], (uint32_t)((it / PC_STAGES) - 1) & 1u, a.wait_limit)) {
              ok = false;
              break;
            }
          }
          uint8_t* st = base + (size_t)q * PC_STAGE_BYTES;
          mbar_arrive_expect_tx(&S->full[q], PC_STAGE_BYTES);
          tma_load_2d(st, &tmAh, &S->full[q], kb * PC_BK, mt * PC_BM);
          tma_load_2d(st + PC_A_BYTES, &tmAl, &S->full[q], kb * PC_BK, mt * PC_BM);
          tma_load_2d(st + 2 * PC_A_BYTES, &tmBh, &S->full[q], kb * PC_BK, 0);
          tma_load_2d(st + 2 * PC_A_BYTES + PC_B_BYTES, &tmBl, &S->full[q], kb * PC_BK, 0);
          issued = it + 1;
        }
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(a.status, TSNE_STATUS_TIMEOUT);
        for (long long j = issued > PC_STAGES ? issued - PC_STAGES : 0; j < issued; j++)
          mbar_wait(&S->full[j % PC_STAGES], (uint32_t)(j / PC_STAGES) & 1u, a.wait_limit);
      }
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
          const int q = (int)(it % PC_STAGES);
          if (*(volatile int*)&S->abort ||
              !mbar_wait(&S->full[q], (uint32_t)(it / PC_STAGES) & 1u, a.wait_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + (size_t)q * PC_STAGE_BYTES);
          const uint64_t ah = sw128_desc(st), al = sw128_desc(st + PC_A_BYTES);
          const uint64_t bh = sw128_desc(st + 2 * PC_A_BYTES);
          const uint64_t bl = sw128_desc(st + 2 * PC_A_BYTES + PC_B_BYTES);
#pragma unroll
          for (int kk = 0; kk < PC_BK / 16; kk++) {  // 16 BF16 = 32 B = 2 descriptor units
            mma_bf16(d, ah + 2 * kk, bh + 2 * kk, kPcIdesc, (kb > kb0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, ah + 2 * kk, bl + 2 * kk, kPcIdesc, 1u);
            mma_bf16(d, al + 2 * kk, bh + 2 * kk, kPcIdesc, 1u);
          }
          mma_commit(&S->empty[q]);
        }
        if (!ok) break;
        mma_commit(&S->acc_full[bb]);
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(a.status, TSNE_STATUS_TIMEOUT);
        // every MMA issued so far completes before tensor memory is released
        mma_commit(&S->drain);
        mbar_wait(&S->drain, 0, a.wait_limit);
      }
    }
  } else {
    // ---------------- epilogue: thread = row ----------------
    int li = 0;
    for (int t = blockIdx.x; t < items; t += gridDim.x, li++) {
      const int mt = t % a.m_tiles, kc = t / a.m_tiles;
      const int bb = li & 1;
      const bool ok = mbar_wait(&S->acc_full[bb], (uint32_t)(li >> 1) & 1u, a.wait_limit);
      tc_fence_after();
      if (pc_epi_bar_or(!ok || *(volatile int*)&S->abort)) break;
      const int64_t m = (int64_t)mt * PC_BM + tid;
      float* o = a.out + (int64_t)kc * a.chunk_stride + m * a.ldo;
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bb * PC_L);
#pragma unroll 1
      for (int ch = 0; ch < PC_L / 32; ch++) {
        uint32_t r[32];
        tmem_ld32(tl + ch * 32, r);
        if (m < a.rows_valid) {
#pragma unroll
          for (int u = 0; u < 32; u++)
            if (ch * 32 + u < a.ncols) o[ch * 32 + u] = __uint_as_float(r[u]);
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
    tmem_dealloc(tmem, 2 * PC_L);
  }
}

// Fixed-order FP64 sum of the K-chunk partials: Z[e] = sum_kc P[kc][e].
__global__ void pca_chunk_reduce_kernel(const float* __restrict__ P, int nchunk, int64_t m,
                                        float* __restrict__ Z) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  double s = 0.0;
  for (int kc = 0; kc < nchunk; kc++) s += (double)__ldcs(&P[(int64_t)kc * m + e]);
  Z[e] = (float)s;
}

// ---------------------------------------------------------------------------
// Gram matrix of a rows x 64 FP32 matrix: FP32 within 256-row sub-blocks,
// FP64 across sub-blocks and blocks (part[block][64 x 64]).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
pca_gram_kernel(const float* __restrict__ X, int64_t rows, double* __restrict__ part) {
  extern __shared__ float xs[];  // 256 x 64
  const int a = threadIdx.x >> 2, b0 = (threadIdx.x & 3) * 16;
  double acc[16];
#pragma unroll
  for (int u = 0; u < 16; u++) acc[u] = 0.0;
  const int64_t r_begin = (int64_t)blockIdx.x * PC_GRAM_ROWS;
  for (int sb = 0; sb < PC_GRAM_ROWS / 256; sb++) {
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
    float f[16];
#pragma unroll
    for (int u = 0; u < 16; u++) f[u] = 0.f;
    for (int r = 0; r < 256; r++) {
      const float xa = xs[r * 64 + a];
      const float4* xb = reinterpret_cast<const float4*>(xs + r * 64 + b0);
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float4 v = xb[q];
        f[4 * q] = fmaf(xa, v.x, f[4 * q]);
        f[4 * q + 1] = fmaf(xa, v.y, f[4 * q + 1]);
        f[4 * q + 2] = fmaf(xa, v.z, f[4 * q + 2]);
        f[4 * q + 3] = fmaf(xa, v.w, f[4 * q + 3]);
      }
    }
#pragma unroll
    for (int u = 0; u < 16; u++) acc[u] += (double)f[u];
  }
  double* o = part + (int64_t)blockIdx.x * 4096 + a * 64 + b0;
#pragma unroll
  for (int u = 0; u < 16; u++) o[u] = acc[u];
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
// Cholesky W = R^T R (FP64, one block of 64 threads) and Rinv = R^-1 (upper).
// A pivot <= 0 restarts with W + shift I, shift growing from 1e-13 trace(W)
// by 1e3 per retry; status gets TSNE_STATUS_NONFINITE if all retries fail.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(64)
pca_chol_kernel(const double* __restrict__ Wg, float* __restrict__ Rinv_out,
                int32_t* status) {
  __shared__ double W[64][65], R[64][65], Ri[64][65];
  __shared__ int fail;
  const int t = threadIdx.x;
  double tr = 0.0;
  for (int i = 0; i < 64; i++) tr += Wg[i * 64 + i];
  double shift = 0.0;
  for (int attempt = 0; attempt < 6; attempt++) {
    for (int i = 0; i < 64; i++) {
      W[i][t] = Wg[i * 64 + t] + (i == t ? shift : 0.0);
      R[i][t] = 0.0;
    }
    if (t == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < 64; j++) {
      // column j of R: R[j][j] = sqrt(W[j][j] - sum_p R[p][j]^2),
      // R[j][i] = (W[j][i] - sum_p R[p][j] R[p][i]) / R[j][j]  (i > j)
      __shared__ double piv;
      if (t == 0) {
        double d = W[j][j];
        for (int p = 0; p < j; p++) d -= R[p][j] * R[p][j];
        if (!(d > 0.0)) {
          fail = 1;
          d = 1.0;
        }
        piv = sqrt(d);
        R[j][j] = piv;
      }
      __syncthreads();
      if (t > j) {
        double v = W[j][t];
        for (int p = 0; p < j; p++) v -= R[p][j] * R[p][t];
        R[j][t] = v / piv;
      }
      __syncthreads();
    }
    if (!fail) break;
    shift = shift == 0.0 ? 1e-13 * tr : shift * 1e3;
    __syncthreads();
    if (attempt == 5 && t == 0) raise_status(status, TSNE_STATUS_NONFINITE);
  }
  // Rinv column t by back substitution: R Ri = I
  for (int i = 0; i < 64; i++) Ri[i][t] = 0.0;
  for (int i = t; i >= 0; i--) {
    double v = (i == t) ? 1.0 : 0.0;
    for (int p = i + 1; p <= t; p++) v -= R[i][p] * Ri[p][t];
    Ri[i][t] = v / R[i][i];
  }
  __syncthreads();
  for (int i = 0; i < 64; i++) Rinv_out[i * 64 + t] = (float)Ri[i][t];
}

// X <- X Rinv (Rinv upper triangular), optionally also written as the
// transposed BF16 split Xt[h][j][r] (r < rows_pad, zero for r >= rows).
__global__ void __launch_bounds__(128)
pca_apply_kernel(float* __restrict__ X, int64_t rows, int64_t rows_pad,
                 const float* __restrict__ Rinv, __nv_bfloat16* __restrict__ Xt) {
  __shared__ float Rs[64 * 64];
  for (int e = threadIdx.x; e < 4096; e += 128) Rs[e] = Rinv[e];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (r >= rows_pad) return;
  float out[64];
  if (r < rows) {
    float y[64];
    const float4* xr = reinterpret_cast<const float4*>(X + r * 64);
#pragma unroll
    for (int q = 0; q < 16; q++) {
      const float4 v = xr[q];
      y[4 * q] = v.x;
      y[4 * q + 1] = v.y;
      y[4 * q + 2] = v.z;
      y[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < 64; j++) {
      float s = 0.f;
#pragma unroll
      for (int i = 0; i <= j; i++) s = fmaf(y[i], Rs[i * 64 + j], s);
      out[j] = s;
    }
    float4* xw = reinterpret_cast<float4*>(X + r * 64);
#pragma unroll
    for (int q = 0; q < 16; q++)
      xw[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < 64; j++) out[j] = 0.f;
  }
  if (Xt != nullptr) {
    const int64_t plane = (int64_t)PC_L * rows_pad;
#pragma unroll
    for (int j = 0; j < 64; j++) {
      __nv_bfloat16 hi, lo;
      split_bf16(out[j], hi, lo);
      Xt[(int64_t)j * rows_pad + r] = hi;
      Xt[plane + (int64_t)j * rows_pad + r] = lo;
    }
  }
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition of the 64 x 64 FP64 matrix W (cyclic Jacobi,
// round-robin ordering: 63 rounds of 32 disjoint (p, q) rotations per sweep;
// rotation from Golub & Van Loan's 2 x 2 symmetric Schur decomposition).
// Output: lam[64] descending, U[64 x 64] with eigenvector c in column c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
pca_eig_kernel(const double* __restrict__ Wg, double* __restrict__ lam,
               double* __restrict__ U) {
  __shared__ double W[64][65], V[64][65];
  __shared__ double cs[32][2];
  __shared__ int pp[32], qq[32];
  __shared__ double red[8];
  __shared__ int done;
  __shared__ int order[64];
  const int t = threadIdx.x;
  for (int e = t; e < 4096; e += 256) {
    W[e >> 6][e & 63] = Wg[e];
    V[e >> 6][e & 63] = ((e >> 6) == (e & 63)) ? 1.0 : 0.0;
  }
  __syncthreads();
  double fro = 0.0;
  for (int e = 0; e < 4096; e++) fro += W[e >> 6][e & 63] * W[e >> 6][e & 63];
  for (int sweep = 0; sweep < 40; sweep++) {
    for (int rnd = 0; rnd < 63; rnd++) {
      if (t < 32) {
        const int a = t == 0 ? 0 : 1 + (t - 1 + rnd) % 63;
        const int b = 1 + (62 - t + rnd) % 63;  // position 63 - t
        const int p = min(a, b), q = max(a, b);
        pp[t] = p;
        qq[t] = q;
        const double apq = W[p][q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (W[q][q] - W[p][p]) / (2.0 * apq);
          const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        cs[t][0] = c;
        cs[t][1] = s;
      }
      __syncthreads();
      // rows: W <- J^T W
      for (int e = t; e < 32 * 64; e += 256) {
        const int k = e >> 6, j = e & 63;
        const int p = pp[k], q = qq[k];
        const double c = cs[k][0], s = cs[k][1];
        const double wp = W[p][j], wq = W[q][j];
        W[p][j] = c * wp - s * wq;
        W[q][j] = s * wp + c * wq;
      }
      __syncthreads();
      // columns: W <- W J, V <- V J
      for (int e = t; e < 32 * 64; e += 256) {
        const int k = e >> 6, j = e & 63;
        const int p = pp[k], q = qq[k];
        const double c = cs[k][0], s = cs[k][1];
        const double wp = W[j][p], wq = W[j][q];
        W[j][p] = c * wp - s * wq;
        W[j][q] = s * wp + c * wq;
        const double vp = V[j][p], vq = V[j][q];
        V[j][p] = c * vp - s * vq;
        V[j][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    // off-diagonal mass
    double off = 0.0;
    for (int e = t; e < 4096; e += 256)
      if ((e >> 6) != (e & 63)) off += W[e >> 6][e & 63] * W[e >> 6][e & 63];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_down_sync(0xffffffffu, off, o);
    if ((t & 31) == 0) red[t >> 5] = off;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < 8; w++) s += red[w];
      done = s <= 1e-26 * fro;  // off-diagonal norm below 1e-13 of the Frobenius norm
    }
    __syncthreads();
    if (done) break;
  }
  // descending order of the eigenvalues (ties: lower index first)
  if (t == 0) {
    for (int i = 0; i < 64; i++) order[i] = i;
    for (int i = 1; i < 64; i++) {
      const int v = order[i];
      int j = i - 1;
      while (j >= 0 && W[order[j]][order[j]] < W[v][v]) {
        order[j + 1] = order[j];
        j--;
      }
      order[j + 1] = v;
    }
  }
  __syncthreads();
  if (t < 64) lam[t] = W[order[t]][order[t]];
  for (int e = t; e < 4096; e += 256) {
    const int r = e >> 6, c = e & 63;
    U[r * 64 + c] = V[r][order[c]];
  }
}

// Components V[c][col] = (Z[col,:] . U[:, c]) / sigma_c for c < k, col < g
// (FP64 arithmetic, FP32 output), then the sign convention.
__global__ void __launch_bounds__(256)
pca_components_kernel(const float* __restrict__ Z, int g, int k, const double* __restrict__ lam,
                      const double* __restrict__ U, float* __restrict__ comp) {
  __shared__ double Us[64 * 64];
  __shared__ double inv[64];
  for (int e = threadIdx.x; e < 4096; e += 256) Us[e] = U[e];
  if (threadIdx.x < 64) {
    const double l = lam[threadIdx.x];
    inv[threadIdx.x] = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
  }
  __syncthreads();
  const int col = blockIdx.x * 256 + threadIdx.x;
  if (col >= g) return;
  double z[64];
#pragma unroll
  for (int j = 0; j < 64; j++) z[j] = (double)Z[(int64_t)col * 64 + j];
  for (int c = 0; c < k; c++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 64; j++) s += z[j] * Us[j * 64 + c];
    comp[(int64_t)c * g + col] = (float)(s * inv[c]);
  }
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

// Scores T[r][c] = sign_c sigma_c (Q[r,:] . U[:, c]) for c < k.
__global__ void __launch_bounds__(128)
pca_scores_kernel(const float* __restrict__ Q, int64_t n, int k, const double* __restrict__ lam,
                  const double* __restrict__ U, const float* __restrict__ sign,
                  float* __restrict__ T) {
  __shared__ float M[64 * 64];
  for (int e = threadIdx.x; e < 4096; e += 128) {
    const int j = e >> 6, c = e & 63;
    M[e] = c < k ? (float)(U[e] * sqrt(fmax(lam[c], 0.0))) * sign[c] : 0.f;
  }
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * 128 + threadIdx.x;
  if (r >= n) return;
  float y[64];
  const float4* xr = reinterpret_cast<const float4*>(Q + r * 64);
#pragma unroll
  for (int q = 0; q < 16; q++) {
    const float4 v = xr[q];
    y[4 * q] = v.x;
    y[4 * q + 1] = v.y;
    y[4 * q + 2] = v.z;
    y[4 * q + 3] = v.w;
  }
  for (int c = 0; c < k; c++) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 64; j++) s = fmaf(y[j], M[j * 64 + c], s);
    T[r * k + c] = s;
  }
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

struct PcaLayout {
  int64_t n, np;
  int g, gp;
  int m_tiles_rows, m_tiles_cols, nchunk, kpc, kb_rows, kb_cols;
  size_t off_mean, off_colpart, off_ssq, off_As, off_At, off_Y, off_Qt, off_Zp, off_Z, off_Wt,
      off_gpart, off_W, off_Rinv, off_lam, off_U, off_sign, total;
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
  // K chunks of the transposed product: about 8 waves of 148 CTAs
  int target = (8 * 148 + L.m_tiles_cols - 1) / L.m_tiles_cols;
  if (target > L.kb_cols) target = L.kb_cols;
  L.kpc = (L.kb_cols + target - 1) / target;
  L.nchunk = (L.kb_cols + L.kpc - 1) / L.kpc;
  const int64_t nprep = (int64_t)(L.gp / 64) * (L.np / 64);
  const int64_t gblk = ((n > L.gp ? n : (int64_t)L.gp) + PC_GRAM_ROWS - 1) / PC_GRAM_ROWS;
  size_t o = 0;
  L.off_mean = o;    o = pal(o + sizeof(double) * L.gp);
  L.off_colpart = o; o = pal(o + (with_fit ? sizeof(double) * PC_COLSUM_CH * g : 0));
  L.off_ssq = o;     o = pal(o + (with_fit ? sizeof(double) * nprep : 0));
  L.off_As = o;      o = pal(o + 2 * sizeof(__nv_bfloat16) * (size_t)n * L.gp);
  L.off_At = o;      o = pal(o + (with_fit ? 2 * sizeof(__nv_bfloat16) * (size_t)L.gp * L.np : 0));
  L.off_Y = o;       o = pal(o + (with_fit ? sizeof(float) * (size_t)L.np * PC_L : 0));
  L.off_Qt = o;      o = pal(o + (with_fit ? 2 * sizeof(__nv_bfloat16) * (size_t)PC_L * L.np : 0));
  L.off_Zp = o;      o = pal(o + (with_fit ? sizeof(float) * (size_t)L.nchunk * L.gp * PC_L : 0));
  L.off_Z = o;       o = pal(o + (with_fit ? sizeof(float) * (size_t)L.gp * PC_L : 0));
  L.off_Wt = o;      o = pal(o + 2 * sizeof(__nv_bfloat16) * (size_t)PC_L * L.gp);
  L.off_gpart = o;   o = pal(o + (with_fit ? sizeof(double) * 4096 * (size_t)gblk : 0));
  L.off_W = o;       o = pal(o + sizeof(double) * 4096);
  L.off_Rinv = o;    o = pal(o + sizeof(float) * 4096);
  L.off_lam = o;     o = pal(o + sizeof(double) * 64);
  L.off_U = o;       o = pal(o + sizeof(double) * 4096);
  L.off_sign = o;    o = pal(o + sizeof(float) * 64);
  L.total = o;
  return L;
}

size_t pca_ws_bytes(int64_t n, int g, bool fit) { return pca_layout(n, g, fit).total; }

static bool encode_bf16_2d(CUtensorMap* tm, const void* base, uint64_t inner, uint64_t outer,
                           uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

static int g_num_sms = 0;

static cudaError_t run_gemm(const __nv_bfloat16* A, uint64_t a_inner, uint64_t a_outer,
                            const __nv_bfloat16* B, uint64_t b_inner, int m_tiles, int nchunk,
                            int kpc, int kb_total, int64_t rows_valid, int ldo, int ncols,
                            int64_t chunk_stride, float* out, int32_t* status, cudaStream_t st) {
  CUtensorMap tah, tal, tbh, tbl;
  const uint64_t a_plane = a_inner * a_outer, b_plane = b_inner * (uint64_t)PC_L;
  if (!encode_bf16_2d(&tah, A, a_inner, a_outer, a_inner * 2, PC_BK, PC_BM) ||
      !encode_bf16_2d(&tal, A + a_plane, a_inner, a_outer, a_inner * 2, PC_BK, PC_BM) ||
      !encode_bf16_2d(&tbh, B, b_inner, PC_L, b_inner * 2, PC_BK, PC_L) ||
      !encode_bf16_2d(&tbl, B + b_plane, b_inner, PC_L, b_inner * 2, PC_BK, PC_L))
    return cudaErrorInvalidValue;
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  cudaError_t e = cudaFuncSetAttribute(pca_gemm_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPcSmemBytes);
  if (e != cudaSuccess) return e;
  PcGemmArgs ga;
  ga.m_tiles = m_tiles;
  ga.nchunk = nchunk;
  ga.kpc = kpc;
  ga.kb_total = kb_total;
  ga.rows_valid = rows_valid;
  ga.ldo = ldo;
  ga.ncols = ncols;
  ga.chunk_stride = chunk_stride;
  ga.out = out;
  ga.status = status;
  ga.wait_limit = 4000000000ll;
  const int items = m_tiles * nchunk;
  const int grid = items < g_num_sms ? items : g_num_sms;
  pca_gemm_kernel<<<grid, PC_THREADS, kPcSmemBytes, st>>>(tah, tal, tbh, tbl, ga);
  return cudaGetLastError();
}

// CholeskyQR passes on X (rows x 64, row stride 64); the last pass also
// writes the transposed split Xt (64 x rows_pad) when Xt is given.
static cudaError_t orth(float* X, int64_t rows, int64_t rows_pad, __nv_bfloat16* Xt, int passes,
                        double* gpart, double* W, float* Rinv, int32_t* status, cudaStream_t st) {
  const int gblk = (int)((rows + PC_GRAM_ROWS - 1) / PC_GRAM_ROWS);
  cudaError_t e = cudaFuncSetAttribute(pca_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       256 * 64 * (int)sizeof(float));
  if (e != cudaSuccess) return e;
  for (int p = 0; p < passes; p++) {
    pca_gram_kernel<<<gblk, 256, 256 * 64 * sizeof(float), st>>>(X, rows, gpart);
    pca_gram_sum_kernel<<<16, 256, 0, st>>>(gpart, gblk, W);
    pca_chol_kernel<<<1, 64, 0, st>>>(W, Rinv, status);
    const bool last = p == passes - 1;
    const int64_t r_launch = (last && Xt) ? rows_pad : rows;
    pca_apply_kernel<<<(unsigned)((r_launch + 127) / 128), 128, 0, st>>>(
        X, rows, rows_pad, Rinv, last ? Xt : nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_pca_fit(const float* A, int64_t n, int g, int64_t lda, int k, int n_power,
                           const float* omega, float* scores, float* comp, double* sigma,
                           double* ev, double* mean_out, double* total_var, void* ws,
                           int32_t* status, cudaStream_t st) {
  const PcaLayout L = pca_layout(n, g, true);
  char* w = static_cast<char*>(ws);
  double* mean = reinterpret_cast<double*>(w + L.off_mean);
  double* colpart = reinterpret_cast<double*>(w + L.off_colpart);
  double* ssq = reinterpret_cast<double*>(w + L.off_ssq);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(w + L.off_As);
  __nv_bfloat16* At = reinterpret_cast<__nv_bfloat16*>(w + L.off_At);
  float* Y = reinterpret_cast<float*>(w + L.off_Y);
  __nv_bfloat16* Qt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Qt);
  float* Zp = reinterpret_cast<float*>(w + L.off_Zp);
  float* Z = reinterpret_cast<float*>(w + L.off_Z);
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Wt);
  double* gpart = reinterpret_cast<double*>(w + L.off_gpart);
  double* W = reinterpret_cast<double*>(w + L.off_W);
  float* Rinv = reinterpret_cast<float*>(w + L.off_Rinv);
  double* lam = reinterpret_cast<double*>(w + L.off_lam);
  double* U = reinterpret_cast<double*>(w + L.off_U);
  float* sign = reinterpret_cast<float*>(w + L.off_sign);

  // column means and the centred split matrix (row-major and transposed)
  pca_colsum_kernel<<<dim3((g + 255) / 256, PC_COLSUM_CH), 256, 0, st>>>(A, n, g, lda, colpart);
  pca_colmean_kernel<<<(L.gp + 255) / 256, 256, 0, st>>>(colpart, n, g, L.gp, mean);
  const dim3 pgrid((unsigned)(L.np / 64), L.gp / 64);
  pca_prep_kernel<<<pgrid, 256, 0, st>>>(A, n, g, lda, L.gp, L.np, mean, As, At, ssq);
  pca_sum_kernel<<<1, 256, 0, st>>>(ssq, (int64_t)pgrid.x * pgrid.y, 1.0 / (double)(n - 1),
                                    total_var);
  pca_sketch_split_kernel<<<(unsigned)((PC_L * (int64_t)L.gp + 255) / 256), 256, 0, st>>>(
      omega, g, L.gp, PC_L, 0, Wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;

  const int passes = 2;
  auto rows_product = [&]() -> cudaError_t {  // Y = Ac W, then Q = orth(Y) (+ Qt)
    cudaError_t r = run_gemm(As, (uint64_t)L.gp, (uint64_t)n, Wt, (uint64_t)L.gp, L.m_tiles_rows,
                             1, L.kb_rows, L.kb_rows, n, PC_L, PC_L, 0, Y, status, st);
    if (r != cudaSuccess) return r;
    return orth(Y, n, L.np, Qt, passes, gpart, W, Rinv, status, st);
  };
  auto cols_product = [&]() -> cudaError_t {  // Z = Ac^T Q (K-split, FP64 chunk sums)
    cudaError_t r = run_gemm(At, (uint64_t)L.np, (uint64_t)L.gp, Qt, (uint64_t)L.np,
                             L.m_tiles_cols, L.nchunk, L.kpc, L.kb_cols, L.gp, PC_L, PC_L,
                             (int64_t)L.gp * PC_L, Zp, status, st);
    if (r != cudaSuccess) return r;
    const int64_t m = (int64_t)L.gp * PC_L;
    pca_chunk_reduce_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(Zp, L.nchunk, m, Z);
    return cudaGetLastError();
  };
  if ((e = rows_product()) != cudaSuccess) return e;
  for (int it = 0; it < n_power; it++) {
    if ((e = cols_product()) != cudaSuccess) return e;
    if ((e = orth(Z, L.gp, L.gp, Wt, passes, gpart, W, Rinv, status, st)) != cudaSuccess) return e;
    if ((e = rows_product()) != cudaSuccess) return e;
  }
  if ((e = cols_product()) != cudaSuccess) return e;
  // Rayleigh-Ritz: Z^T Z = U diag(lam) U^T
  const int zblk = (int)((L.gp + PC_GRAM_ROWS - 1) / PC_GRAM_ROWS);
  e = cudaFuncSetAttribute(pca_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           256 * 64 * (int)sizeof(float));
  if (e != cudaSuccess) return e;
  pca_gram_kernel<<<zblk, 256, 256 * 64 * sizeof(float), st>>>(Z, L.gp, gpart);
  pca_gram_sum_kernel<<<16, 256, 0, st>>>(gpart, zblk, W);
  pca_eig_kernel<<<1, 256, 0, st>>>(W, lam, U);
  pca_components_kernel<<<(g + 255) / 256, 256, 0, st>>>(Z, g, k, lam, U, comp);
  pca_sign_kernel<<<k, 256, 0, st>>>(comp, g, sign);
  pca_scores_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(Y, n, k, lam, U, sign, scores);
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
  double* mean = reinterpret_cast<double*>(w + L.off_mean);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(w + L.off_As);
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(w + L.off_Wt);
  cudaMemsetAsync(mean, 0, sizeof(double) * L.gp, st);
  cudaMemcpyAsync(mean, mean_in, sizeof(double) * g, cudaMemcpyDeviceToDevice, st);
  const dim3 pgrid((unsigned)(L.np / 64), L.gp / 64);
  pca_prep_kernel<<<pgrid, 256, 0, st>>>(A, n, g, lda, L.gp, L.np, mean, As, nullptr, nullptr);
  pca_sketch_split_kernel<<<(unsigned)((PC_L * (int64_t)L.gp + 255) / 256), 256, 0, st>>>(
      comp, g, L.gp, k, 1, Wt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return run_gemm(As, (uint64_t)L.gp, (uint64_t)n, Wt, (uint64_t)L.gp, L.m_tiles_rows, 1,
                  L.kb_rows, L.kb_rows, n, k, k, 0, scores, status, st);
}

}  // namespace tsne
