// sort.cu -- device-wide primitives used to build the symmetric P:
//   * exclusive prefix sum of uint32 (three phases: chunk sums, a one-CTA
//     scan of the chunk sums, chunk scans plus offset);
//   * stable least-significant-digit radix sort of (uint64 key, float value)
//     pairs, 8-bit digits, only over the bit ranges that carry information.
// Both are deterministic: integer counts only, and every element's output
// position is a pure function of the input order (ties keep input order).
#include "common.cuh"

namespace tsne {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of v over the CTA (blockDim.x == kScanThreads); returns the
// prefix of this thread and writes the CTA total to *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* sh, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  __syncthreads();
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = lane < kScanThreads / 32 ? sh[lane] : 0u;
    x = warp_incl_scan(x);
    if (lane < kScanThreads / 32) sh[lane] = x;
  }
  __syncthreads();
  *total = sh[kScanThreads / 32 - 1];
  return inc - v + (w > 0 ? sh[w - 1] : 0u);
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce_kernel(const uint32_t* __restrict__ in, int64_t m, uint32_t* __restrict__ part) {
  __shared__ uint32_t sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk;
  uint32_t s = 0;
  for (int r = 0; r < kScanItems; r++) {
    const int64_t e = base + (int64_t)r * kScanThreads + threadIdx.x;
    if (e < m) s += in[e];
  }
  uint32_t tot;
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// One CTA: exclusive scan of part[0..np) in place; part[np] = grand total.
__global__ void __launch_bounds__(kScanThreads)
scan_parts_kernel(uint32_t* __restrict__ part, int64_t np) {
  __shared__ uint32_t sh[32];
  uint32_t carry = 0;
  for (int64_t b = 0; b < np; b += kScanThreads) {
    const int64_t e = b + threadIdx.x;
    const uint32_t v = e < np ? part[e] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, sh, &tot);
    if (e < np) part[e] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) part[np] = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_apply_kernel(const uint32_t* __restrict__ in, int64_t m, const uint32_t* __restrict__ part,
                  uint32_t* __restrict__ out) {
  __shared__ uint32_t sh[32];
  // each thread owns kScanItems consecutive elements of the chunk
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    v[r] = (base + r < m) ? in[base + r] : 0u;
    s += v[r];
  }
  uint32_t tot;
  uint32_t run = block_excl_scan(s, sh, &tot) + part[blockIdx.x];
#pragma unroll
  for (int r = 0; r < kScanItems; r++) {
    if (base + r < m) out[base + r] = run;
    run += v[r];
  }
}

int64_t scan_parts_len(int64_t m) { return (m + kScanChunk - 1) / kScanChunk + 1; }

// out[i] = sum_{j < i} in[i]; part must hold scan_parts_len(m) entries and
// receives the grand total at part[scan_parts_len(m) - 1].  in == out allowed.
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t m, uint32_t* part,
                            cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  const int64_t np = (m + kScanChunk - 1) / kScanChunk;
  scan_reduce_kernel<<<(unsigned)np, kScanThreads, 0, st>>>(in, m, part);
  scan_parts_kernel<<<1, kScanThreads, 0, st>>>(part, np);
  scan_apply_kernel<<<(unsigned)np, kScanThreads, 0, st>>>(in, m, part, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radix sort.  A CTA owns a tile of kRadixTile consecutive elements.
//   hist:    hist[digit * ntiles + tile] = count of the digit in the tile
//   scan:    exclusive scan of hist (digit-major) = first output slot of
//            (digit, tile): all smaller digits first, then earlier tiles
//   scatter: the tile is walked in rounds of 256 consecutive elements; an
//            element's slot adds the counts of equal digits before it in the
//            round (warp match + per-warp prefix), so ties keep input order;
//            the tile is ordered in shared memory first and written out run
//            by run.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;

__global__ void __launch_bounds__(kRadixThreads)
radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t m, int shift, int64_t ntiles,
                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixRounds; r++) {
    const int64_t e = base + (int64_t)r * kRadixThreads + threadIdx.x;
    if (e < m) atomicAdd(&cnt[(keys[e] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// The tile is first placed in shared memory in its sorted order (stable: rank
// within a digit in input order), then written out in that order, so that the
// threads of a warp write consecutive slots of one digit's run (coalesced)
// instead of 32 scattered 8-byte slots.  A tile's count of digit d is the gap
// between its scanned offset and the next entry of the digit-major scan.
// Warp w ranks the w-th contiguous 1/8 of the tile on its own (all of its 16
// loads in flight at once, a running count per digit in its own shared-memory
// row), so that the CTA meets at a barrier four times per tile, not per round.
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixPerWarp = kRadixTile / kRadixWarps;  // 512 elements
constexpr size_t kRadixSmem = (size_t)kRadixTile * (sizeof(uint64_t) + sizeof(float));

__global__ void __launch_bounds__(kRadixThreads)
radix_scatter_kernel(const uint64_t* __restrict__ kin, const float* __restrict__ vin, int64_t m,
                     int shift, int64_t ntiles, const uint32_t* __restrict__ off,
                     uint64_t* __restrict__ kout, float* __restrict__ vout) {
  constexpr int W = kRadixWarps;
  extern __shared__ __align__(16) uint8_t radix_smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(radix_smem);
  float* sval = reinterpret_cast<float*>(radix_smem + sizeof(uint64_t) * kRadixTile);
  __shared__ uint32_t lstart[256];   // first local slot of each digit
  __shared__ uint32_t gstart[256];   // first global slot of each digit for this tile
  __shared__ uint32_t wcnt[W][256];  // per-warp digit counts, then per-warp first local slots
  __shared__ uint32_t scan_sh[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t tbase = (int64_t)blockIdx.x * kRadixTile;
  const int tcount = (int)min((int64_t)kRadixTile, m - tbase);
  for (int q = tid; q < W * 256; q += kRadixThreads) (&wcnt[0][0])[q] = 0u;
  {
    const int64_t idx = (int64_t)tid * ntiles + blockIdx.x;
    const uint32_t g0 = off[idx];
    const uint32_t g1 = idx + 1 < 256 * ntiles ? off[idx + 1] : (uint32_t)m;
    const uint32_t c = g1 - g0;
    // exclusive scan of the 256 counts (one per thread)
    uint32_t inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) scan_sh[w] = inc;
    __syncthreads();  // also orders the clearing of wcnt before its use
    uint32_t wbase = 0;
    for (int k = 0; k < w; k++) wbase += scan_sh[k];
    lstart[tid] = wbase + inc - c;
    gstart[tid] = g0;
  }
  // this warp's elements: wb + r * 32 + lane, r = 0 .. 15, in input order
  const int wb = w * kRadixPerWarp;
  constexpr int R = kRadixPerWarp / 32;
  uint64_t key[R];
  float val[R];
  uint32_t dg[R], rank[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int q = wb + r * 32 + lane;
    const bool ok = q < tcount;
    key[r] = ok ? kin[tbase + q] : 0ull;
    val[r] = ok ? vin[tbase + q] : 0.f;
    dg[r] = ok ? (uint32_t)((key[r] >> shift) & 0xff) : 256u;  // 256: matches no digit
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint32_t* cnt = wcnt[w];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const uint32_t peers = __match_any_sync(0xffffffffu, dg[r]);
    const uint32_t before = dg[r] < 256u ? cnt[dg[r]] : 0u;
    rank[r] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (dg[r] < 256u && (peers & lt_mask) == 0u) cnt[dg[r]] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: the warps' first local slots, in warp order after the digit's start
  {
    uint32_t run = lstart[tid];
#pragma unroll
    for (int k = 0; k < W; k++) {
      const uint32_t c = wcnt[k][tid];
      wcnt[k][tid] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; r++) {
    if (dg[r] < 256u) {
      const uint32_t pos = cnt[dg[r]] + rank[r];
      skey[pos] = key[r];
      sval[pos] = val[r];
    }
  }
  __syncthreads();
  for (int r = tid; r < tcount; r += kRadixThreads) {
    const uint64_t k = skey[r];
    const uint32_t d = (uint32_t)((k >> shift) & 0xff);
    const uint32_t pos = gstart[d] + ((uint32_t)r - lstart[d]);
    kout[pos] = k;
    vout[pos] = sval[r];
  }
}

int64_t radix_tiles(int64_t m) { return (m + kRadixTile - 1) / kRadixTile; }

// Sorts (keys, vals) of length m by the bits [lo, hi) of each listed range
// (LSD order: ranges and digits from least significant).  k0/v0 hold the input;
// k1/v1 are scratch of the same size; *k_res / *v_res receive the buffers that
// hold the result.  hist: 256 * radix_tiles(m) entries; part:
// scan_parts_len(256 * radix_tiles(m)) entries.
cudaError_t launch_radix_sort(uint64_t* k0, float* v0, uint64_t* k1, float* v1, int64_t m,
                              const int* bit_lo, const int* bit_hi, int nranges, uint32_t* hist,
                              uint32_t* part, uint64_t** k_res, float** v_res, cudaStream_t st) {
  uint64_t* ka = k0;
  uint64_t* kb = k1;
  float* va = v0;
  float* vb = v1;
  const int64_t nt = radix_tiles(m);
  cudaError_t ea = cudaFuncSetAttribute(radix_scatter_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kRadixSmem);
  if (ea != cudaSuccess) return ea;
  for (int g = 0; g < nranges && m > 0; g++) {
    for (int sh = bit_lo[g]; sh < bit_hi[g]; sh += 8) {
      radix_hist_kernel<<<(unsigned)nt, kRadixThreads, 0, st>>>(ka, m, sh, nt, hist);
      cudaError_t e = launch_scan_u32(hist, hist, 256 * nt, part, st);
      if (e != cudaSuccess) return e;
      radix_scatter_kernel<<<(unsigned)nt, kRadixThreads, kRadixSmem, st>>>(ka, va, m, sh, nt,
                                                                           hist, kb, vb);
      uint64_t* tk = ka; ka = kb; kb = tk;
      float* tv = va; va = vb; vb = tv;
    }
  }
  *k_res = ka;
  *v_res = va;
  return cudaGetLastError();
}

}  // namespace tsne
