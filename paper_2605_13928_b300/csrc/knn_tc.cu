// knn_tc.cu -- k nearest neighbours with a BF16 tcgen05 distance GEMM, a
// per-row candidate filter and an exact FP32 re-rank (t-SNE input affinities
// need the k nearest neighbours; van der Maaten 2014, Sec. 3).
//
// 1. prep: every sample is centred (translation leaves distances unchanged);
//    the centred points are rounded to BF16 (h_i, padded to 64 dims) and
//    n_i = |h_i|^2 is taken of the rounded values, so that
//        d2~_ij = n_i + n_j - 2 h_i . h_j
//    is the exact squared distance of the rounded points (up to FP32
//    rounding of the dot product).  Its error against the true distance is
//    about 2 (x_i - x_j) . (e_i - e_j) with e the BF16 rounding error -- small
//    for close pairs, which are the ones that matter.
// 2. tcgen05 GEMM + filter: a CTA owns 128 query rows of one sample.  A TMA
//    producer warp streams column tiles of 128 BF16 rows (128 B each,
//    128-byte swizzle) through a 4-stage shared-memory ring; one thread issues
//    tcgen05.mma kind::f16 (M = 128, N = 128, K = 16, four per tile) into a
//    double-buffered FP32 accumulator in tensor memory; four epilogue warps
//    (thread = query row = TMEM lane) read it back with tcgen05.ld, form
//    v = n_j - 2 s (so d2~ = n_i + v) and append (d2~, j) to the row's
//    candidate buffer when d2~ is below the row's threshold.  For d <= 61 the
//    term -n_j / 2 rides in the product itself (three spare K columns: -1/2 in
//    the A row, a three-term BF16 split of n_j in the B row), so the epilogue
//    compares s' = s - n_j / 2 with -thr / 2 and loads no norms.  When a buffer
//    passes TC_CAP entries the warp prunes it cooperatively: it keeps every
//    entry up to a threshold x with at least k2 entries at or below it (early-
//    exit radix passes; at most (TC_CAP + k2) / 2 kept), and x becomes the new
//    threshold.  After the last tile the buffer is cut to exactly the k2 best
//    (ties in column order).
// 3. re-rank: one warp per row computes exact FP32 distances of its <= k2
//    candidates (same operation order as the FP32 brute-force kernel) and
//    sorts (d2, j) with a bitonic network in registers (eight keys per lane,
//    shuffles across lanes); the first k are the output.
//
// Every wait on an mbarrier is bounded: the pipeline waits by wait_limit
// cycles (TSNE_WAIT_LIMIT, default ~2 s), the drains after an abort by their
// own long bound.  A role that gives up raises TSNE_STATUS_TIMEOUT and sets a
// shared abort flag; each epilogue warp takes its abort decision with a warp
// vote so all its lanes agree; the producer waits for the copies it has issued
// and the MMA issuer for its committed MMAs before the CTA may exit, and
// tensor memory is released only after every role has stopped.  Rows of an
// aborted CTA get no candidates (re-rank output: index -1).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tcgen05.cuh"

namespace tsne {

constexpr int TC_BM = 128;       // query rows per CTA (= TMEM lanes)
constexpr int TC_BN = 128;       // columns per tile
constexpr int TC_BK = 64;        // padded dimensions (BF16)
constexpr int TC_STAGES = 4;     // B-tile ring
constexpr int TC_NACC = 2;       // accumulator buffers in tensor memory
constexpr int TC_THREADS = 192;  // warps 0-3 epilogue, 4 TMA producer, 5 MMA issuer
constexpr int TC_CAP = 448;      // prune when a row buffer holds more than this
constexpr int TC_CAPT = TC_CAP + TC_BN;   // row buffer entries (one tile of headroom)
constexpr int TC_PER_LANE = TC_CAPT / 32; // buffer entries per lane in a prune
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 2;  // 16 KB (A tile and each B tile)
constexpr int TC_KMAX2 = 256;    // largest candidate count of the re-rank sort
constexpr int TC_FOLD_COL = TC_BK - 3;  // first of the three folded-norm columns

static_assert(TC_CAPT % 32 == 0, "prune loads the buffer 32 entries at a time");
// A row holds at most TC_CAP entries when a tile starts (every tile ends with a
// prune of the rows above it) and takes at most TC_BN entries from a tile, so
// its buffer of TC_CAPT entries cannot overflow and the appends need no check.
static_assert(TC_CAPT >= TC_CAP + TC_BN, "a tile's appends fit behind TC_CAP entries");
static_assert(TC_KMAX2 < TC_CAP, "a prune during the scan keeps fewer than TC_CAP entries");

constexpr uint32_t kIdesc = idesc_bf16_f32(TC_BM, TC_BN);

// Eight consecutive floats from a 32-byte aligned global address (one 256-bit
// load, so each of a warp's scattered rows costs one full sector per load).
__device__ __forceinline__ void ld_v8(const float* p, float (&r)[8]) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]),
        "=f"(r[7])
      : "l"(p));
}

// Order-preserving map of FP32 bits to uint32 (and back).
__device__ __forceinline__ uint32_t fkey(uint32_t b) {
  return b ^ ((b & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  return __uint_as_float(k ^ ((k & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu));
}

// Largest of three (one PTX max.f32 with three sources).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One radix pass over the warp's keys (entry r * 32 + lane valid when below
// cnt): a 256-bin histogram (hist: 256 words of shared memory owned by the
// warp) of the digit (key >> shift) & 255 of the keys whose bits under `high`
// equal prefix, then the digit whose inclusive count first reaches k.  below /
// incl: the matching keys in the bins before that digit / up to and with it.
__device__ void radix_pass(const uint32_t (&key)[TC_PER_LANE], int cnt, uint32_t high,
                           uint32_t prefix, int shift, uint32_t k, uint32_t* hist,
                           uint32_t& digit, uint32_t& below, uint32_t& incl) {
  const int lane = threadIdx.x & 31;
  reinterpret_cast<uint4*>(hist)[2 * lane] = make_uint4(0u, 0u, 0u, 0u);
  reinterpret_cast<uint4*>(hist)[2 * lane + 1] = make_uint4(0u, 0u, 0u, 0u);
  __syncwarp();
#pragma unroll
  for (int r = 0; r < TC_PER_LANE; r++)
    if (r * 32 + lane < cnt && (key[r] & high) == prefix)
      atomicAdd(&hist[(key[r] >> shift) & 255u], 1u);
  __syncwarp();
  // lane l holds bins 8 l .. 8 l + 7; the first lane whose inclusive count
  // reaches k holds the digit
  const uint4 h0 = reinterpret_cast<const uint4*>(hist)[2 * lane];
  const uint4 h1 = reinterpret_cast<const uint4*>(hist)[2 * lane + 1];
  const uint32_t b[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
  uint32_t tot = 0u;
#pragma unroll
  for (int j = 0; j < 8; j++) tot += b[j];
  uint32_t inc = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  const int L = __ffs(__ballot_sync(0xffffffffu, inc >= k)) - 1;
  uint32_t dg = 0u, bl = 0u, ic = 0u;
  if (lane == L) {
    uint32_t c = inc - tot;  // keys in the bins before this lane's first
    bool found = false;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (!found && c + b[j] >= k) {
        dg = (uint32_t)(8 * L + j);
        bl = c;
        ic = c + b[j];
        found = true;
      }
      c += b[j];
    }
  }
  digit = __shfl_sync(0xffffffffu, dg, L);
  below = __shfl_sync(0xffffffffu, bl, L);
  incl = __shfl_sync(0xffffffffu, ic, L);
  __syncwarp();  // the histogram is read before the next pass clears it
}

// The keep-th smallest of the warp's keys (1 <= keep <= cnt), i.e. the
// smallest x with #(key <= x) >= keep: a radix select over the four 8-bit
// digits, most significant first.
__device__ uint32_t warp_select(const uint32_t (&key)[TC_PER_LANE], int cnt, int keep,
                                uint32_t* hist) {
  uint32_t prefix = 0u;  // digits fixed so far
  uint32_t k = (uint32_t)keep;  // rank still sought among the keys matching them
#pragma unroll 1
  for (int pass = 0; pass < 4; pass++) {
    const int shift = 24 - 8 * pass;
    const uint32_t high = pass == 0 ? 0u : 0xFFFFFFFFu << (shift + 8);
    uint32_t digit, below, incl;
    radix_pass(key, cnt, high, prefix, shift, k, hist, digit, below, incl);
    prefix |= digit << shift;
    k -= below;
  }
  return prefix;
}

// Prunes a row buffer of `cnt` entries (key = fkey(d2 bits)) in place, every
// lane of the warp taking part, and returns the largest kept key x; `kept`
// receives the number of entries kept.
//  * limit > keep (a prune while the scan goes on): any x with
//    #(key <= x) >= keep is a valid threshold -- an entry above x has keep
//    smaller ones already, so it is not among the row's keep nearest.  Radix
//    passes of 8 bits, starting under the keys' highest differing bit, narrow
//    the bin that holds the keep-th smallest key, and stop as soon as every
//    entry up to the top of that bin is at most `limit` entries; those are
//    kept, in buffer order.  (The keys of a row pile up just under its
//    threshold, so one pass seldom suffices and the exact select seldom runs.)
//  * otherwise: exactly the keep smallest (ties in buffer order).
__device__ uint32_t warp_prune(uint2* e, int cnt, int keep, int limit, uint32_t* hist,
                               int& kept) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  uint2 v[TC_PER_LANE];
  uint32_t key[TC_PER_LANE];
#pragma unroll
  for (int r = 0; r < TC_PER_LANE; r++) {
    const int q = r * 32 + lane;
    v[r] = q < cnt ? e[q] : make_uint2(0u, 0u);
    key[r] = q < cnt ? fkey(v[r].x) : 0xFFFFFFFFu;
  }
  uint32_t x = 0u;
  bool done = false;
  if (limit > keep) {
    uint32_t kmin = 0xFFFFFFFFu, kmax = 0u;
#pragma unroll
    for (int r = 0; r < TC_PER_LANE; r++) {
      if (r * 32 + lane < cnt) {
        kmin = min(kmin, key[r]);
        kmax = max(kmax, key[r]);
      }
    }
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (kmin != kmax) {
      const int hb = 31 - __clz(kmin ^ kmax);  // bits above hb are common to all keys
      uint32_t high = hb == 31 ? 0u : 0xFFFFFFFFu << (hb + 1);
      uint32_t prefix = kmin & high;
      uint32_t k = (uint32_t)keep, below_all = 0u;
#pragma unroll 1
      for (int top = hb; top >= 0; top -= 8) {
        const int shift = top >= 7 ? top - 7 : 0;
        uint32_t digit, below, incl;
        radix_pass(key, cnt, high, prefix, shift, k, hist, digit, below, incl);
        if (below_all + incl <= (uint32_t)limit) {
          // keep every key up to the top of the bin
          const uint32_t t_hi = prefix | (digit << shift) | ((1u << shift) - 1u);
#pragma unroll
          for (int r = 0; r < TC_PER_LANE; r++)
            if (r * 32 + lane < cnt && key[r] <= t_hi) x = max(x, key[r]);
          x = __reduce_max_sync(0xffffffffu, x);
          done = true;
          break;
        }
        prefix |= digit << shift;
        high |= 0xFFFFFFFFu << shift;
        below_all += below;
        k -= below;
        if (shift == 0) break;
      }
    }
  }
  if (done) {
    int out = 0;
#pragma unroll
    for (int r = 0; r < TC_PER_LANE; r++) {
      const bool kp = r * 32 + lane < cnt && key[r] <= x;
      const uint32_t km = __ballot_sync(0xffffffffu, kp);
      if (kp) e[out + __popc(km & lt)] = v[r];
      out += __popc(km);
    }
    __syncwarp();
    kept = out;
    return x;
  }
  x = warp_select(key, cnt, keep, hist);
  int below = 0;
#pragma unroll
  for (int r = 0; r < TC_PER_LANE; r++) below += (r * 32 + lane < cnt && key[r] < x) ? 1 : 0;
  below = warp_sum_i(below);
  const int ties_keep = keep - below;
  __syncwarp();
  int out = 0, ties_seen = 0;
#pragma unroll
  for (int r = 0; r < TC_PER_LANE; r++) {
    const bool valid = r * 32 + lane < cnt;
    const bool tie = valid && key[r] == x;
    const uint32_t tm = __ballot_sync(0xffffffffu, tie);
    const bool kp = valid && (key[r] < x || (tie && ties_seen + __popc(tm & lt) < ties_keep));
    const uint32_t km = __ballot_sync(0xffffffffu, kp);
    if (kp) e[out + __popc(km & lt)] = v[r];
    out += __popc(km);
    ties_seen += __popc(tm);
  }
  __syncwarp();
  kept = keep;
  return x;
}

struct TcSmem {
  uint64_t full[TC_STAGES], empty[TC_STAGES], acc_full[TC_NACC], acc_empty[TC_NACC], a_full;
  uint32_t tmem_slot;
  int abort;
  alignas(16) float norm[4][TC_NACC][TC_BN];  // per epilogue warp
  alignas(16) uint32_t hist[4][256];          // per epilogue warp: radix-select histogram
};
constexpr size_t kTcSmemBytes = 1024 + (size_t)TC_TILE_BYTES * (1 + TC_STAGES) + sizeof(TcSmem);

// Bound of the waits that drain work already issued (TMA copies in flight, the
// last committed MMAs) after an abort: about 2 s at 2 GHz, far above the
// microseconds that work takes, and independent of the pipeline waits'
// wait_limit.
constexpr long long kTcDrainLimit = 4000000000ll;

// kFold: the B rows carry -n_j / 2 in three spare K columns (see prep), so the
// accumulator holds s' = s - n_j / 2 and the filter needs no column norms.
template <bool kFold>
__global__ void __launch_bounds__(TC_THREADS, 2)
knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const float* __restrict__ norms, int k2, const __grid_constant__ SampleTable tab,
              uint2* __restrict__ cand, int32_t* __restrict__ cand_cnt, int32_t* status,
              long long wait_limit) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + TC_TILE_BYTES;
  TcSmem* S = reinterpret_cast<TcSmem*>(base + (size_t)TC_TILE_BYTES * (1 + TC_STAGES));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t row0 = p0 + (int64_t)(b - tab.blk_off[s]) * TC_BM;
  const int ntile = (int)((p1 - p0 + TC_BN - 1) / TC_BN);
  // column tiles start at the CTA's own tile and wrap around the sample: in the
  // spatial order the nearest points come first and the thresholds tighten early
  const int t_first = (int)((row0 - p0) / TC_BN);

  if (tid == 0) {
    for (int q = 0; q < TC_STAGES; q++) {
      mbar_init(&S->full[q], 1);
      mbar_init(&S->empty[q], 1);
    }
    for (int q = 0; q < TC_NACC; q++) {
      mbar_init(&S->acc_full[q], 1);
      mbar_init(&S->acc_empty[q], TC_BM);
    }
    mbar_init(&S->a_full, 1);
    S->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 5) tmem_alloc(&S->tmem_slot, TC_NACC * TC_BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->tmem_slot;

  if (warp == 4) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      mbar_arrive_expect_tx(&S->a_full, TC_TILE_BYTES);
      tma_load_2d(sA, &tmA, &S->a_full, 0, (int)row0);
      for (int t = 0; t < ntile; t++) {
        const int q = t % TC_STAGES;
        if (t >= TC_STAGES) {
          if (*(volatile int*)&S->abort ||
              !mbar_wait(&S->empty[q], (uint32_t)((t / TC_STAGES) - 1) & 1u, wait_limit)) {
            ok = false;
            break;
          }
        }
        mbar_arrive_expect_tx(&S->full[q], TC_TILE_BYTES);
        const int tt = t_first + t < ntile ? t_first + t : t_first + t - ntile;
        tma_load_2d(sB + (size_t)q * TC_TILE_BYTES, &tmB, &S->full[q], 0,
                    (int)(p0 + (int64_t)tt * TC_BN));
        issued = t + 1;
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(status, TSNE_STATUS_TIMEOUT);
        // let the copies already issued land before the CTA can exit: each wait
        // is bounded by the long drain limit, not by the pipeline's wait_limit
        // (which a caller may set short), since an issued copy always completes
        // within microseconds (earlier copies completed before their stage was
        // reused)
        mbar_wait(&S->a_full, 0, kTcDrainLimit);
        for (int t = issued > TC_STAGES ? issued - TC_STAGES : 0; t < issued; t++)
          mbar_wait(&S->full[t % TC_STAGES], (uint32_t)(t / TC_STAGES) & 1u, kTcDrainLimit);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      bool ok = mbar_wait(&S->a_full, 0, wait_limit);
      int committed = 0;
      const uint64_t adesc = sw128_desc(smem_u32(sA));
      for (int t = 0; ok && t < ntile; t++) {
        const int q = t % TC_STAGES, bb = t % TC_NACC;
        if (*(volatile int*)&S->abort) { ok = false; break; }
        if (!mbar_wait(&S->full[q], (uint32_t)(t / TC_STAGES) & 1u, wait_limit)) { ok = false; break; }
        if (t >= TC_NACC &&
            !mbar_wait(&S->acc_empty[bb], (uint32_t)((t / TC_NACC) - 1) & 1u, wait_limit)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint64_t bdesc = sw128_desc(smem_u32(sB + (size_t)q * TC_TILE_BYTES));
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; kk++)  // 16 BF16 = 32 bytes = 2 descriptor units
          mma_bf16(tmem + (uint32_t)(bb * TC_BN), adesc + 2 * kk, bdesc + 2 * kk, kIdesc,
                   kk > 0 ? 1u : 0u);
        mma_commit(&S->empty[q]);
        mma_commit(&S->acc_full[bb]);
        committed = t + 1;
      }
      if (!ok) {
        *(volatile int*)&S->abort = 1;
        raise_status(status, TSNE_STATUS_TIMEOUT);
        if (committed > 0)  // the last committed MMAs must finish before TMEM is freed
          mbar_wait(&S->acc_full[(committed - 1) % TC_NACC],
                    (uint32_t)((committed - 1) / TC_NACC) & 1u, kTcDrainLimit);
      }
    }
  } else {
    // ---------------- epilogue: thread = query row ----------------
    const int64_t i = row0 + tid;
    const bool valid = i < p1;
    const float ni = valid ? norms[i] : 0.f;
    float thr_v = valid ? INFINITY : -INFINITY;  // candidate iff n_j - 2 s < thr_v
    float tau = -0.5f * thr_v;                     // folded: candidate iff s' > tau
    int cnt = 0;
    uint2* buf = cand + (valid ? i : 0) * (int64_t)TC_CAPT;
    const int prune_limit = (TC_CAP + k2) / 2;  // k2 < TC_CAP: limit in (k2, TC_CAP)
    bool aborted = false;
    // Each warp keeps its own copy of a tile's 128 column norms (four per lane),
    // so the four epilogue warps need no barrier among themselves and drift
    // apart by up to a tile (a row prune in one warp does not hold up the
    // others).  The norms of tile t + 1 are loaded while tile t is processed.
    float* wnorm = S->norm[warp][0];
    float nrm_next[4];
    if constexpr (!kFold) {
      const int64_t j0 = p0 + (int64_t)t_first * TC_BN;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int64_t j = j0 + q * 32 + lane;
        nrm_next[q] = j < p1 ? __ldg(&norms[j]) : INFINITY;
      }
    }
    for (int t = 0; t < ntile; t++) {
      const int bb = t % TC_NACC;
      if constexpr (!kFold) {
#pragma unroll
        for (int q = 0; q < 4; q++) wnorm[bb * TC_BN + q * 32 + lane] = nrm_next[q];
      }
      const bool ok = mbar_wait(&S->acc_full[bb], (uint32_t)(t / TC_NACC) & 1u, wait_limit);
      tc_fence_after();
      const int tt = t_first + t < ntile ? t_first + t : t_first + t - ntile;
      const int64_t j0 = p0 + (int64_t)tt * TC_BN;
      if (!kFold && t + 1 < ntile) {
        const int tn = tt + 1 < ntile ? tt + 1 : 0;
        const int64_t jn = p0 + (int64_t)tn * TC_BN;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int64_t j = jn + q * 32 + lane;
          nrm_next[q] = j < p1 ? __ldg(&norms[j]) : INFINITY;
        }
      }
      if (__any_sync(0xffffffffu, !ok || *(volatile int*)&S->abort)) {
        aborted = true;
        break;
      }
      __syncwarp();  // this warp's norm copy is written
      const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bb * TC_BN);
      const float2 M2 = make_float2(-2.f, -2.f);
      // One 32-column chunk of the row's accumulator tile: filter and append.
      auto chunk = [&](const uint32_t (&r)[32], float m32, int ch) {
        if constexpr (kFold) {
          // s' per column.  m32, the largest s' of the row's 32 columns, comes
          // with the load (tcgen05.ld.red), so a chunk in which no row of the
          // warp passes tau (about 95 % of them at 1M points) costs one compare
          // and one vote.  Otherwise a group of 4 is flagged when its largest s'
          // passes tau.  Columns of another sample (or past the end) are real
          // rows of the B operand here, so a chunk that crosses the sample's end
          // also tests j < p1; the row's own point is excluded in the CTA's own
          // tile (the first one, t = 0).  Both tests are warp-uniform per chunk.
          if (__any_sync(0xffffffffu, m32 > tau)) {
            uint32_t mask = 0u;
#pragma unroll
            for (int c4 = 0; c4 < 8; c4++) {
              const float m4 =
                  fmaxf(fmax3(__uint_as_float(r[4 * c4]), __uint_as_float(r[4 * c4 + 1]),
                              __uint_as_float(r[4 * c4 + 2])),
                        __uint_as_float(r[4 * c4 + 3]));
              mask |= (m4 > tau ? 1u : 0u) << c4;
            }
            mask = __reduce_or_sync(0xffffffffu, mask);
            const int64_t jc = j0 + ch * 32;
            if (t == 0 || jc + 32 > p1) {
#pragma unroll
              for (int c4 = 0; c4 < 8; c4++) {
                if (mask & (1u << c4)) {  // warp-uniform
#pragma unroll
                  for (int u = 0; u < 4; u++) {
                    const int64_t j = jc + 4 * c4 + u;
                    const float sp = __uint_as_float(r[4 * c4 + u]);
                    if (sp > tau && j < p1 && j != i) {
                      buf[cnt] = make_uint2(__float_as_uint(fmaf(-2.f, sp, ni)), (uint32_t)j);
                      cnt++;
                    }
                  }
                }
              }
            } else {
#pragma unroll
              for (int c4 = 0; c4 < 8; c4++) {
                if (mask & (1u << c4)) {  // warp-uniform
#pragma unroll
                  for (int u = 0; u < 4; u++) {
                    const float sp = __uint_as_float(r[4 * c4 + u]);
                    if (sp > tau) {
                      buf[cnt] = make_uint2(__float_as_uint(fmaf(-2.f, sp, ni)),
                                            (uint32_t)(jc + 4 * c4 + u));
                      cnt++;
                    }
                  }
                }
              }
            }
          }
          return;
        }
        const float4* nb4 = reinterpret_cast<const float4*>(&wnorm[bb * TC_BN + ch * 32]);
        // v = n_j - 2 s (packed FFMA2) for all 32 columns first, with the minimum
        // of each group of 4 columns folded into a per-row bit mask; one warp OR of
        // the masks then names the groups in which some row of the warp has a
        // candidate (about 0.2 % of pairs pass).  The group tests carry no
        // branches, so the 8 groups' arithmetic runs back to back.
        float v[32];
        uint32_t mask = 0u;
#pragma unroll
        for (int c4 = 0; c4 < 8; c4++) {
          const float4 nb = nb4[c4];
          const float2 v01 = __ffma2_rn(
              make_float2(__uint_as_float(r[4 * c4]), __uint_as_float(r[4 * c4 + 1])), M2,
              make_float2(nb.x, nb.y));
          const float2 v23 = __ffma2_rn(
              make_float2(__uint_as_float(r[4 * c4 + 2]), __uint_as_float(r[4 * c4 + 3])), M2,
              make_float2(nb.z, nb.w));
          v[4 * c4] = v01.x;
          v[4 * c4 + 1] = v01.y;
          v[4 * c4 + 2] = v23.x;
          v[4 * c4 + 3] = v23.y;
          const float m4 = fminf(fminf(v01.x, v01.y), fminf(v23.x, v23.y));
          mask |= (m4 < thr_v ? 1u : 0u) << c4;
        }
        mask = __reduce_or_sync(0xffffffffu, mask);
        if (mask) {
          const int64_t jc = j0 + ch * 32;
#pragma unroll
          for (int c4 = 0; c4 < 8; c4++) {
            if (mask & (1u << c4)) {  // warp-uniform
#pragma unroll
              for (int u = 0; u < 4; u++) {
                const int64_t j = jc + 4 * c4 + u;
                const float vv = v[4 * c4 + u];
                if (vv < thr_v && (t != 0 || j != i)) {
                  buf[cnt] = make_uint2(__float_as_uint(ni + vv), (uint32_t)j);
                  cnt++;
                }
              }
            }
          }
        }
      };
      // The four chunks with the load of chunk c + 1 in flight while chunk c is
      // filtered (two register sets); the accumulator buffer is handed back to
      // the MMA issuer as soon as its last chunk is in registers.  The folded
      // form loads with the row maximum of each chunk (ma / mb); the other form
      // does not use it.
      static_assert(TC_BN == 128, "four 32-column chunks per tile");
      uint32_t ra[32], rb[32];
      float ma = 0.f, mb = 0.f;
      auto ld = [&](uint32_t a, uint32_t (&r)[32], float& m) {
        if constexpr (kFold) tmem_ld32_max_issue(a, r, m); else tmem_ld32_issue(a, r);
      };
      auto wt = [&](uint32_t (&r)[32], float& m) {
        if constexpr (kFold) tmem_ld_wait_m(r, m); else tmem_ld_wait(r);
      };
      ld(tl, ra, ma);
      wt(ra, ma);
      ld(tl + 32, rb, mb);
      chunk(ra, ma, 0);
      wt(rb, mb);
      ld(tl + 64, ra, ma);
      chunk(rb, mb, 1);
      wt(ra, ma);
      ld(tl + 96, rb, mb);
      chunk(ra, ma, 2);
      wt(rb, mb);
      tc_fence_before();
      mbar_arrive(&S->acc_empty[bb]);
      chunk(rb, mb, 3);
      // prune rows whose buffers passed TC_CAP (warp-cooperative, one row at a
      // time) to at most prune_limit entries, so that a buffer takes at least
      // TC_CAP - prune_limit more entries before its next prune
      uint32_t need = __ballot_sync(0xffffffffu, cnt > TC_CAP);
      while (need) {
        const int L = __ffs(need) - 1;
        need &= need - 1;
        const int64_t iL = __shfl_sync(0xffffffffu, (long long)i, L);
        const int cL = __shfl_sync(0xffffffffu, cnt, L);
        int kept;
        const uint32_t x =
            warp_prune(cand + iL * (int64_t)TC_CAPT, cL, k2, prune_limit, S->hist[warp], kept);
        if (lane == L) {
          cnt = kept;
          thr_v = fkey_inv(x) - ni;
          tau = -0.5f * thr_v;
        }
      }
    }
    if (!aborted) {
      uint32_t need = __ballot_sync(0xffffffffu, cnt > k2);
      while (need) {
        const int L = __ffs(need) - 1;
        need &= need - 1;
        const int64_t iL = __shfl_sync(0xffffffffu, (long long)i, L);
        const int cL = __shfl_sync(0xffffffffu, cnt, L);
        int kept;
        warp_prune(cand + iL * (int64_t)TC_CAPT, cL, k2, k2, S->hist[warp], kept);
        if (lane == L) cnt = kept;
      }
    }
    if (valid) cand_cnt[i] = aborted ? 0 : cnt;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, TC_NACC * TC_BN);
  }
}

// ---------------------------------------------------------------------------
// prep: per-sample mean (FP64, fixed order), BF16 rounding, norms of the
// rounded points.
// ---------------------------------------------------------------------------
// Row chunks per sample in the mean reduction: enough CTAs to fill the GPU
// for one large sample (each thread's loop is a chain of dependent loads and
// adds, so the chunk length sets the kernel's time).
constexpr int MEAN_CH = 256;

constexpr int KEY_DIMS = 3;  // coordinates of the spatial (Morton) ordering key

// Per (sample, row chunk): FP64 column sums of the chunk (4 row groups x 64
// dims), and the minimum / maximum of the first KEY_DIMS coordinates.
__global__ void __launch_bounds__(256)
mean_partial_kernel(const float* __restrict__ X, int d, const __grid_constant__ SampleTable tab,
                    double* __restrict__ part, float* __restrict__ mmpart) {
  __shared__ double sh[4][64];
  __shared__ float smin[4][64], smax[4][64];
  const int s = blockIdx.x, ch = blockIdx.y, c = threadIdx.x & 63, g = threadIdx.x >> 6;
  const int64_t p0 = tab.pt_off[s], ns = tab.pt_off[s + 1] - p0;
  const int64_t r0 = p0 + ns * ch / MEAN_CH, r1 = p0 + ns * (ch + 1) / MEAN_CH;
  double a = 0.0;
  float lo = INFINITY, hi = -INFINITY;
  if (c < d)
#pragma unroll 4
    for (int64_t i = r0 + g; i < r1; i += 4) {
      const float x = X[i * d + c];
      a += (double)x;
      lo = fminf(lo, x);
      hi = fmaxf(hi, x);
    }
  sh[g][c] = a;
  smin[g][c] = lo;
  smax[g][c] = hi;
  __syncthreads();
  if (g == 0) {
    const int64_t o = (int64_t)s * MEAN_CH + ch;
    part[o * 64 + c] = sh[0][c] + sh[1][c] + sh[2][c] + sh[3][c];
    if (c < KEY_DIMS) {
      mmpart[(o * 2 + 0) * KEY_DIMS + c] =
          fminf(fminf(smin[0][c], smin[1][c]), fminf(smin[2][c], smin[3][c]));
      mmpart[(o * 2 + 1) * KEY_DIMS + c] =
          fmaxf(fmaxf(smax[0][c], smax[1][c]), fmaxf(smax[2][c], smax[3][c]));
    }
  }
}

// Per sample: mean of each dimension from the chunk sums, in chunk order, and
// the bounding box of the first KEY_DIMS coordinates (box[s][0..2] minima,
// box[s][4..6] maxima).
__global__ void mean_final_kernel(const double* __restrict__ part,
                                  const float* __restrict__ mmpart, int d,
                                  const __grid_constant__ SampleTable tab,
                                  float* __restrict__ mean, float* __restrict__ box) {
  const int s = blockIdx.x, c = threadIdx.x;
  const int64_t ns = tab.pt_off[s + 1] - tab.pt_off[s];
  double t = 0.0;
  for (int ch = 0; ch < MEAN_CH; ch++) t += part[((int64_t)s * MEAN_CH + ch) * 64 + c];
  mean[s * 64 + c] = (c < d && ns > 0) ? (float)(t / (double)ns) : 0.f;
  if (c < KEY_DIMS) {
    float lo = INFINITY, hi = -INFINITY;
    for (int ch = 0; ch < MEAN_CH; ch++) {
      const int64_t o = (int64_t)s * MEAN_CH + ch;
      lo = fminf(lo, mmpart[(o * 2 + 0) * KEY_DIMS + c]);
      hi = fmaxf(hi, mmpart[(o * 2 + 1) * KEY_DIMS + c]);
    }
    box[s * 8 + c] = lo;
    box[s * 8 + 4 + c] = hi;
  }
}

// Spatial ordering key of every point: sample index in bits 48.., then the
// Morton interleave of its first KEY_DIMS coordinates quantised to 16 bits in
// the sample's bounding box.  Points close in the key are close in space, so
// sorting by it gathers neighbours into nearby positions.
__device__ __forceinline__ uint64_t spread3_16(uint32_t x) {
  uint64_t v = x & 0xFFFFu;
  v = (v | (v << 32)) & 0x00FF00000000FFFFull;
  v = (v | (v << 16)) & 0x00FF0000FF0000FFull;
  v = (v | (v << 8)) & 0xF00F00F00F00F00Full;
  v = (v | (v << 4)) & 0x30C30C30C30C30C3ull;
  v = (v | (v << 2)) & 0x9249249249249249ull;
  return v;
}

__global__ void __launch_bounds__(256)
spatial_key_kernel(const float* __restrict__ X, int d, const __grid_constant__ SampleTable tab,
                   const float* __restrict__ box, uint64_t* __restrict__ keys,
                   float* __restrict__ vals) {
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t i = tab.pt_off[s] + (int64_t)(b - tab.blk_off[s]) * tab.blk_pts + threadIdx.x;
  if (i >= tab.pt_off[s + 1]) return;
  uint64_t m = 0;
#pragma unroll
  for (int c = 0; c < KEY_DIMS; c++) {
    uint32_t q = 0;
    if (c < d) {
      const float lo = box[s * 8 + c], hi = box[s * 8 + 4 + c];
      const float t = hi > lo ? (X[i * d + c] - lo) / (hi - lo) : 0.f;
      q = (uint32_t)fminf(fmaxf(t * 65535.0f, 0.f), 65535.0f);
    }
    m |= spread3_16(q) << c;
  }
  keys[i] = ((uint64_t)s << 48) | m;
  vals[i] = __int_as_float((int)i);
}

// Position r of the spatial order holds point i = perm[r] (same sample).
// XN (non-null when d <= TC_FOLD_COL): the B operand of the folded filter, the
// same BF16 row with n_r split into three BF16 terms (n_r = n1 + n2 + n3 to
// about 2^-24 n_r) in columns TC_FOLD_COL..+2, where the A row (XB) holds -1/2:
// the product then accumulates h_i . h_r - n_r / 2.
__global__ void __launch_bounds__(256)
to_bf16_kernel(const float* __restrict__ X, int d, const __grid_constant__ SampleTable tab,
               const float* __restrict__ mean, const int32_t* __restrict__ perm,
               __nv_bfloat16* __restrict__ XB, float* __restrict__ norms,
               __nv_bfloat16* __restrict__ XN, float* __restrict__ XP) {
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t r = tab.pt_off[s] + (int64_t)(b - tab.blk_off[s]) * tab.blk_pts + threadIdx.x;
  if (r >= tab.pt_off[s + 1]) return;
  const int64_t i = perm[r];
  float nrm = 0.f;
  __nv_bfloat16* out = XB + r * TC_BK;
  for (int c = 0; c < TC_BK; c += 2) {
    const float x0 = c < d ? X[i * d + c] : 0.f, x1 = c + 1 < d ? X[i * d + c + 1] : 0.f;
    *reinterpret_cast<float2*>(XP + r * TC_BK + c) = make_float2(x0, x1);
    const float v0 = c < d ? x0 - mean[s * 64 + c] : 0.f;
    const float v1 = c + 1 < d ? x1 - mean[s * 64 + c + 1] : 0.f;
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v0), h1 = __float2bfloat16_rn(v1);
    const float f0 = __bfloat162float(h0), f1 = __bfloat162float(h1);
    nrm = fmaf(f0, f0, nrm);
    nrm = fmaf(f1, f1, nrm);
    __nv_bfloat162 pr;
    pr.x = h0;
    pr.y = h1;
    *reinterpret_cast<__nv_bfloat162*>(out + c) = pr;
    if (XN) *reinterpret_cast<__nv_bfloat162*>(XN + r * TC_BK + c) = pr;
  }
  norms[r] = nrm;
  if (XN) {
    const __nv_bfloat16 n1 = __float2bfloat16_rn(nrm);
    const float r1 = nrm - __bfloat162float(n1);
    const __nv_bfloat16 n2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 n3 = __float2bfloat16_rn(r1 - __bfloat162float(n2));
    const __nv_bfloat16 mh = __float2bfloat16_rn(-0.5f);
    out[TC_FOLD_COL] = mh;
    out[TC_FOLD_COL + 1] = mh;
    out[TC_FOLD_COL + 2] = mh;
    XN[r * TC_BK + TC_FOLD_COL] = n1;
    XN[r * TC_BK + TC_FOLD_COL + 1] = n2;
    XN[r * TC_BK + TC_FOLD_COL + 2] = n3;
  }
}

// ---------------------------------------------------------------------------
// Exact FP32 re-rank: one warp per row, distances of the <= k2 candidates in
// the operation order of the FP32 brute-force kernel, bitonic sort of the
// keys (d2 << 32 | j) in registers, first k written.
// ---------------------------------------------------------------------------
template <int DMAX>
__global__ void __launch_bounds__(256)
knn_rerank_kernel(const float* __restrict__ XP, int d, int k, const uint2* __restrict__ cand,
                  const int32_t* __restrict__ cand_cnt, const int32_t* __restrict__ perm,
                  int64_t n, int32_t* __restrict__ nbr_idx, float* __restrict__ nbr_d2) {
  __shared__ unsigned long long keys[8][TC_KMAX2];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + w;  // position in the spatial order
  if (r >= n) return;
  const int64_t i = perm[r];                       // the point it holds
  const int m = cand_cnt[r];
  // XP: the points in the spatial order, FP32, rows of 64 (zero past d), so the
  // candidates of a row (spatial neighbours) sit close together in memory
  float q[DMAX];
  {
    const float4* xq = reinterpret_cast<const float4*>(XP + r * TC_BK);
#pragma unroll
    for (int c4 = 0; c4 < DMAX / 4; c4++) {
      const float4 v = xq[c4];
      q[4 * c4] = v.x;
      q[4 * c4 + 1] = v.y;
      q[4 * c4 + 2] = v.z;
      q[4 * c4 + 3] = v.w;
    }
  }
  unsigned long long* kk = keys[w];
  for (int e = lane; e < TC_KMAX2; e += 32) {
    unsigned long long key = ~0ull;
    if (e < m) {
      const uint32_t jp = cand[r * (int64_t)TC_CAPT + e].y;
      const int64_t j = perm[jp];
      const float* xj = XP + (int64_t)jp * TC_BK;  // rows of 256 bytes, 256-byte aligned
      float a = 0.f;
      static_assert(DMAX % 8 == 0, "whole 32-byte loads");
#pragma unroll
      for (int c8 = 0; c8 < DMAX / 8; c8++) {
        float v[8];
        ld_v8(xj + 8 * c8, v);
#pragma unroll
        for (int u = 0; u < 8; u++) {
          const float t = q[8 * c8 + u] - v[u];
          a = fmaf(t, t, a);
        }
      }
      key = ((unsigned long long)fkey(__float_as_uint(a)) << 32) | (uint32_t)j;
    }
    kk[e] = key;
  }
  __syncwarp();
  // bitonic sort of the 256 keys in registers: lane l holds x[t] = key
  // t * 32 + l; strides of 32 and more pair registers of one lane, smaller
  // strides pair lanes (one 64-bit shuffle per key)
  static_assert(TC_KMAX2 == 256, "eight keys per lane");
  unsigned long long x[8];
#pragma unroll
  for (int t = 0; t < 8; t++) x[t] = kk[t * 32 + lane];
#pragma unroll
  for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
        const int rs = stride >> 5;
#pragma unroll
        for (int t = 0; t < 8; t++) {
          if ((t & rs) == 0) {
            const bool up = ((t * 32) & size) == 0;
            const unsigned long long a = x[t], b = x[t | rs];
            const bool sw = (a > b) == up;
            x[t] = sw ? b : a;
            x[t | rs] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < 8; t++) {
          const bool up = ((t * 32 + lane) & size) == 0;
          const bool lower = (lane & stride) == 0;
          const unsigned long long y = __shfl_xor_sync(0xffffffffu, x[t], stride);
          const unsigned long long lo = x[t] < y ? x[t] : y, hi = x[t] < y ? y : x[t];
          x[t] = (lower == up) ? lo : hi;
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; t++) kk[t * 32 + lane] = x[t];
  __syncwarp();
  for (int e = lane; e < k; e += 32) {
    const unsigned long long key = kk[e];
    nbr_idx[i * k + e] = (int32_t)(key & 0xffffffffu);
    nbr_d2[i * k + e] = fkey_inv((uint32_t)(key >> 32));
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int64_t radix_tiles(int64_t m);
int64_t scan_parts_len(int64_t m);
cudaError_t launch_radix_sort(uint64_t* k0, float* v0, uint64_t* k1, float* v1, int64_t m,
                              const int* bit_lo, const int* bit_hi, int nranges, uint32_t* hist,
                              uint32_t* part, uint64_t** k_res, float** v_res, cudaStream_t st);

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace of the BF16 path: BF16 points, norms, sample means, per-row
// candidate buffers (TC_CAPT entries of 8 bytes) and candidate counts.
size_t knn_tc_ws_bytes(int64_t n, int S) {
  size_t (*align)(size_t) = al256;
  size_t off = 0;
  off = align(off + sizeof(__nv_bfloat16) * (size_t)n * TC_BK);  // XB
  off = align(off + sizeof(__nv_bfloat16) * (size_t)n * TC_BK);  // XN (folded norms)
  off = align(off + sizeof(float) * (size_t)n * TC_BK);          // XP (FP32, spatial order)
  off = align(off + sizeof(float) * (size_t)n);                  // norms
  off = align(off + sizeof(float) * (size_t)S * 64);             // means
  off = align(off + sizeof(uint2) * (size_t)n * TC_CAPT);        // candidate buffers
  off = align(off + sizeof(int32_t) * (size_t)n);                // candidate counts
  off = align(off + sizeof(double) * (size_t)S * MEAN_CH * 64);  // mean partial sums
  off = align(off + sizeof(float) * (size_t)S * MEAN_CH * 2 * KEY_DIMS);  // min / max parts
  off = align(off + sizeof(float) * (size_t)S * 8);              // bounding boxes
  off = align(off + 2 * sizeof(uint64_t) * (size_t)n);           // sort keys (two copies)
  off = align(off + 2 * sizeof(float) * (size_t)n);              // sort values (two copies)
  const int64_t nt = radix_tiles(n);
  off = align(off + sizeof(uint32_t) * (size_t)(256 * nt));      // digit histograms
  off = align(off + sizeof(uint32_t) * (size_t)scan_parts_len(256 * nt > n ? 256 * nt : n));
  return off;
}

int knn_tc_max_k2() { return TC_KMAX2; }

// X n x d FP32; tab with blk_pts = 128 (query blocks never straddle a sample).
cudaError_t launch_knn_tc(const float* X, int64_t n, int d, int k, int k2, const SampleTable& tab,
                          void* ws, int32_t* idx, float* d2, int32_t* status,
                          long long wait_limit, cudaStream_t st) {
  size_t (*align)(size_t) = al256;
  if (d > TC_BK || k2 > TC_KMAX2 || k2 < k || n <= 0) return cudaErrorInvalidValue;
  char* w = static_cast<char*>(ws);
  size_t off = 0;
  __nv_bfloat16* XB = reinterpret_cast<__nv_bfloat16*>(w + off);
  off = align(off + sizeof(__nv_bfloat16) * (size_t)n * TC_BK);
  const bool fold = d <= TC_FOLD_COL;
  __nv_bfloat16* XN = fold ? reinterpret_cast<__nv_bfloat16*>(w + off) : nullptr;
  off = align(off + sizeof(__nv_bfloat16) * (size_t)n * TC_BK);
  float* XP = reinterpret_cast<float*>(w + off);
  off = align(off + sizeof(float) * (size_t)n * TC_BK);
  float* norms = reinterpret_cast<float*>(w + off);
  off = align(off + sizeof(float) * (size_t)n);
  float* mean = reinterpret_cast<float*>(w + off);
  off = align(off + sizeof(float) * (size_t)tab.S * 64);
  uint2* cand = reinterpret_cast<uint2*>(w + off);
  off = align(off + sizeof(uint2) * (size_t)n * TC_CAPT);
  int32_t* cnt = reinterpret_cast<int32_t*>(w + off);
  off = align(off + sizeof(int32_t) * (size_t)n);
  double* mpart = reinterpret_cast<double*>(w + off);
  off = align(off + sizeof(double) * (size_t)tab.S * MEAN_CH * 64);
  float* mmpart = reinterpret_cast<float*>(w + off);
  off = align(off + sizeof(float) * (size_t)tab.S * MEAN_CH * 2 * KEY_DIMS);
  float* box = reinterpret_cast<float*>(w + off);
  off = align(off + sizeof(float) * (size_t)tab.S * 8);
  uint64_t* k0 = reinterpret_cast<uint64_t*>(w + off);
  uint64_t* k1 = k0 + n;
  off = align(off + 2 * sizeof(uint64_t) * (size_t)n);
  float* v0 = reinterpret_cast<float*>(w + off);
  float* v1 = v0 + n;
  off = align(off + 2 * sizeof(float) * (size_t)n);
  const int64_t nt = radix_tiles(n);
  uint32_t* hist = reinterpret_cast<uint32_t*>(w + off);
  off = align(off + sizeof(uint32_t) * (size_t)(256 * nt));
  uint32_t* spart = reinterpret_cast<uint32_t*>(w + off);

  // prep (256-point blocks of the same samples)
  SampleTable* t256 = new SampleTable(tab);
  t256->blk_pts = 256;
  int32_t bsum = 0;
  for (int s = 0; s < tab.S; s++) {
    t256->blk_off[s] = bsum;
    bsum += (int32_t)((tab.pt_off[s + 1] - tab.pt_off[s] + 255) / 256);
  }
  t256->blk_off[tab.S] = bsum;
  mean_partial_kernel<<<dim3(tab.S, MEAN_CH), 256, 0, st>>>(X, d, tab, mpart, mmpart);
  mean_final_kernel<<<tab.S, 64, 0, st>>>(mpart, mmpart, d, tab, mean, box);
  // spatial order: sort points by (sample, Morton key); perm[r] = point at position r
  spatial_key_kernel<<<bsum, 256, 0, st>>>(X, d, *t256, box, k0, v0);
  int sbits = 0;
  while ((1 << sbits) < tab.S) sbits++;
  const int lo[2] = {0, 48}, hi[2] = {48, 48 + sbits};
  uint64_t* kres;
  float* vres;
  cudaError_t e0 = launch_radix_sort(k0, v0, k1, v1, n, lo, hi, 2, hist, spart, &kres, &vres, st);
  if (e0 != cudaSuccess) {
    delete t256;
    return e0;
  }
  const int32_t* perm = reinterpret_cast<const int32_t*>(vres);
  to_bf16_kernel<<<bsum, 256, 0, st>>>(X, d, *t256, mean, perm, XB, norms, XN, XP);
  delete t256;

  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tmA, tmB;
  const cuuint64_t dims[2] = {(cuuint64_t)TC_BK, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)TC_BK * sizeof(__nv_bfloat16)};
  const cuuint32_t tbox[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BN};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, XB, dims, strides, tbox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  tmB = tmA;
  if (fold && enc(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, XN, dims, strides, tbox, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;

  auto kern = fold ? knn_tc_kernel<true> : knn_tc_kernel<false>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes);
  if (e != cudaSuccess) return e;
  kern<<<tab.blk_off[tab.S], TC_THREADS, kTcSmemBytes, st>>>(tmA, tmB, norms, k2, tab, cand, cnt,
                                                             status, wait_limit);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned rb = (unsigned)((n + 7) / 8);
  switch (((d + 7) / 8) * 8) {
    case 8: knn_rerank_kernel<8><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 16: knn_rerank_kernel<16><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 24: knn_rerank_kernel<24><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 32: knn_rerank_kernel<32><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 40: knn_rerank_kernel<40><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 48: knn_rerank_kernel<48><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 56: knn_rerank_kernel<56><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    case 64: knn_rerank_kernel<64><<<rb, 256, 0, st>>>(XP, d, k, cand, cnt, perm, n, idx, d2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsne
