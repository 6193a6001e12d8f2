// knn.cu -- exact FP32 brute-force k nearest neighbours (t-SNE input
// affinities are built on the k nearest neighbours, van der Maaten 2014,
// Sec. 3): for every query point i the k points j != i of its sample with the
// smallest d2_ij = sum_c (x_ic - x_jc)^2, ordered by (d2, j).
//
// One thread per query row, QB rows per CTA (CTAs never straddle a sample).
// The query coordinates sit in registers; candidate points stream through
// shared memory in tiles of CT points stored dimension-major, so one 128-bit
// broadcast load gives one coordinate of four candidates.  Distances use
// direct differences (2 FP32 lane operations per dimension and pair).  Each
// thread keeps its current k best in a shared-memory list (entry m of thread
// t at m * QB + t) and the k-th distance in a register: a candidate enters
// only if its d2 is strictly below it, and candidates are visited in
// increasing j, so equal distances keep the smaller index first.
#include "common.cuh"

namespace tsne {

template <int QB, int CT, int DMAX>
__global__ void __launch_bounds__(QB)
knn_fp32_kernel(const float* __restrict__ X, int d, int k, const __grid_constant__ SampleTable tab,
                int32_t* __restrict__ nbr_idx, float* __restrict__ nbr_d2) {
  extern __shared__ float4 smem4[];
  // layout: tile[DMAX/4 * ... ] as float (d x CT, dimension-major), then lists
  float* tile = reinterpret_cast<float*>(smem4);                  // d * CT floats
  float* ld = tile + (size_t)DMAX * CT;                             // k * QB distances
  int32_t* li = reinterpret_cast<int32_t*>(ld + (size_t)k * QB);   // k * QB indices

  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t i = p0 + (int64_t)(b - tab.blk_off[s]) * QB + tid;
  const bool active = i < p1;

  float q[DMAX];
#pragma unroll
  for (int c = 0; c < DMAX; c++) q[c] = (active && c < d) ? X[i * d + c] : 0.f;

  for (int m = 0; m < k; m++) {
    ld[m * QB + tid] = INFINITY;
    li[m * QB + tid] = -1;
  }
  // padding dimensions d..DMAX-1 stay zero in every tile
  for (int e = d * CT + tid; e < DMAX * CT; e += QB) tile[e] = 0.f;
  float kth = INFINITY;

  for (int64_t cb = p0; cb < p1; cb += CT) {
    const int nc = (int)((p1 - cb) < CT ? (p1 - cb) : CT);
    __syncthreads();
    // coalesced: consecutive threads read consecutive floats of the nc x d block
    const float* src = X + cb * d;
    for (int g = tid; g < nc * d; g += QB) {
      const int p = g / d, c = g - p * d;
      tile[c * CT + p] = src[g];
    }
    __syncthreads();
    for (int p = 0; p < nc; p += 4) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int c = 0; c < DMAX; c++) {
        const float4 v = *reinterpret_cast<const float4*>(tile + c * CT + p);
        const float t0 = q[c] - v.x, t1 = q[c] - v.y, t2 = q[c] - v.z, t3 = q[c] - v.w;
        a0 = fmaf(t0, t0, a0);
        a1 = fmaf(t1, t1, a1);
        a2 = fmaf(t2, t2, a2);
        a3 = fmaf(t3, t3, a3);
      }
      const float dd[4] = {a0, a1, a2, a3};
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const int64_t j = cb + p + u;
        if (!active || p + u >= nc || j == i || !(dd[u] < kth)) continue;
        // insert (dd[u], j) keeping ascending (d2, index) order
        int pos = k - 1;
        while (pos > 0 && ld[(pos - 1) * QB + tid] > dd[u]) {
          ld[pos * QB + tid] = ld[(pos - 1) * QB + tid];
          li[pos * QB + tid] = li[(pos - 1) * QB + tid];
          pos--;
        }
        ld[pos * QB + tid] = dd[u];
        li[pos * QB + tid] = (int32_t)j;
        kth = ld[(k - 1) * QB + tid];
      }
    }
  }
  if (!active) return;
  for (int m = 0; m < k; m++) {
    nbr_d2[i * k + m] = ld[m * QB + tid];
    nbr_idx[i * k + m] = li[m * QB + tid];
  }
}

static int knn_dmax(int d) { return d <= 64 ? ((d + 7) / 8) * 8 : 0; }

size_t knn_fp32_smem(int d, int k) {
  constexpr int QB = 128, CT = 64;
  const int dmax = knn_dmax(d);
  if (dmax == 0 || k <= 0) return 0;
  return sizeof(float) * ((size_t)dmax * CT) + (sizeof(float) + sizeof(int32_t)) * (size_t)k * QB;
}

template <int DMAX>
static cudaError_t launch_knn_d(const float* X, int d, int k, const SampleTable& tab,
                                int32_t* idx, float* d2, cudaStream_t st) {
  constexpr int QB = 128, CT = 64;
  const size_t smem = knn_fp32_smem(d, k);
  auto kern = knn_fp32_kernel<QB, CT, DMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = tab.blk_off[tab.S];
  if (blocks <= 0) return cudaSuccess;
  kern<<<blocks, QB, smem, st>>>(X, d, k, tab, idx, d2);
  return cudaGetLastError();
}

// Requires tab.blk_pts == 128 (one block = 128 query rows of one sample).
cudaError_t launch_knn_fp32(const float* X, int d, int k, const SampleTable& tab, int32_t* idx,
                            float* d2, cudaStream_t st) {
  switch (knn_dmax(d)) {
    case 8: return launch_knn_d<8>(X, d, k, tab, idx, d2, st);
    case 16: return launch_knn_d<16>(X, d, k, tab, idx, d2, st);
    case 24: return launch_knn_d<24>(X, d, k, tab, idx, d2, st);
    case 32: return launch_knn_d<32>(X, d, k, tab, idx, d2, st);
    case 40: return launch_knn_d<40>(X, d, k, tab, idx, d2, st);
    case 48: return launch_knn_d<48>(X, d, k, tab, idx, d2, st);
    case 56: return launch_knn_d<56>(X, d, k, tab, idx, d2, st);
    case 64: return launch_knn_d<64>(X, d, k, tab, idx, d2, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tsne
