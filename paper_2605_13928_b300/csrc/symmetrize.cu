// symmetrize.cu -- the symmetric P of t-SNE on the kNN graph
// (van der Maaten 2014, Sec. 3): P = (P_cond + P_cond^T) / (2 n_s), on the
// union of the forward pattern (i -> j for j among i's neighbours) and its
// transpose; and, with the fuzzy union w + w' - w w' in place of the sum, the
// fuzzy graph of UMAP (McInnes, Healy & Melville 2018, Sec. 3.1).
//
// Row i of the result merges two lists sorted by column:
//   A_i: the forward entries of row i (its k neighbours), sorted in registers
//        by one warp per row;
//   B_i: the transposed entries (j -> i for every row j that lists i).  They
//        are emitted as (i << bits | j) in increasing j and sorted by i alone
//        (a stable radix sort over the row bits), so each B_i is in column
//        order without a sort over the column bits.
// A column in both lists is one entry with the two values combined (a + b, or
// the fuzzy union); its position in the row is the number of union columns
// before it: #(A < c) + #(B < c) - #(A and B < c), where the last term is a
// running count of B's columns found in A, kept per B entry.
//
// A neighbour outside the row's sample, or the row itself, is an invalid
// index: it is flagged (TSNE_STATUS_BAD_INDEX) and left out.  A column listed
// twice in one row (not produced by the kNN routines, but accepted here) is
// folded into one forward entry, in column-then-value order, before anything
// is emitted.  Everything is a function of the input alone: no atomics decide
// an order or a sum.
#include "common.cuh"

namespace tsne {

cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t m, uint32_t* part,
                            cudaStream_t st);
cudaError_t launch_radix_sort(uint64_t* k0, float* v0, uint64_t* k1, float* v1, int64_t m,
                              const int* bit_lo, const int* bit_hi, int nranges, uint32_t* hist,
                              uint32_t* part, uint64_t** k_res, float** v_res, cudaStream_t st);

// A forward entry: column in the high 32 bits, the FP32 value's bits in the
// low 32 (so that sorting the words sorts by column).  Empty slots are
// all ones, which sort last.
constexpr uint64_t kNoEntry = ~0ull;
constexpr int kSymRows = 8;   // rows (warps) per block; a block never straddles a sample
constexpr int kSymMaxK = 256; // k of at most 256: eight keys per lane

__device__ __forceinline__ uint32_t ent_col(uint64_t x) { return (uint32_t)(x >> 32); }
__device__ __forceinline__ float ent_val(uint64_t x) {
  return __uint_as_float((uint32_t)(x & 0xffffffffu));
}
__device__ __forceinline__ float combine(float a, float b, int fuzzy) {
  return fuzzy ? (a + b) - a * b : a + b;
}

// Ascending bitonic sort of the warp's 32 * KPL words, word t * 32 + lane in
// x[t] of that lane: strides of 32 and more pair registers of one lane,
// smaller strides pair lanes.
template <int KPL>
__device__ __forceinline__ void warp_sort(uint64_t (&x)[KPL]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * KPL; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
        const int rs = stride >> 5;
#pragma unroll
        for (int t = 0; t < KPL; t++) {
          if ((t & rs) == 0) {
            const bool up = ((t * 32) & size) == 0;
            const uint64_t a = x[t], b = x[t | rs];
            const bool sw = (a > b) == up;
            x[t] = sw ? b : a;
            x[t | rs] = sw ? a : b;
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < KPL; t++) {
          const bool up = ((t * 32 + lane) & size) == 0;
          const bool lower = (lane & stride) == 0;
          const uint64_t y = __shfl_xor_sync(0xffffffffu, x[t], stride);
          const uint64_t lo = x[t] < y ? x[t] : y, hi = x[t] < y ? y : x[t];
          x[t] = (lower == up) ? lo : hi;
        }
      }
    }
  }
}

// Forward lists: one warp per row i (blocks of kSymRows rows never straddle a
// sample).  The row's k entries (j, c scaled) are sorted by column; a column
// listed twice is folded; the sorted list is A_i (k words, empty slots last),
// and each of its entries is also emitted as the transposed key (j << bits | i)
// at the same slot i * k + a, so that the transposed keys come in increasing i.
template <int KPL>
__global__ void __launch_bounds__(32 * kSymRows)
sym_forward_kernel(const int32_t* __restrict__ idx, const float* __restrict__ pc, int k, int bits,
                   const __grid_constant__ SampleTable tab, int fuzzy, uint64_t* __restrict__ A,
                   uint64_t* __restrict__ bkey, float* __restrict__ bval, int32_t* status) {
  __shared__ uint64_t fold[kSymRows][32 * KPL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = blockIdx.x;
  const int s = find_sample(tab.blk_off, tab.S, b);
  const int64_t p0 = tab.pt_off[s], p1 = tab.pt_off[s + 1];
  const int64_t i = p0 + (int64_t)(b - tab.blk_off[s]) * kSymRows + w;
  if (i >= p1) return;  // the whole warp
  const float scale = fuzzy ? 1.f : 0.5f / (float)(p1 - p0);
  uint64_t x[KPL];
  bool bad = false;
#pragma unroll
  for (int t = 0; t < KPL; t++) {
    const int a = t * 32 + lane;
    x[t] = kNoEntry;
    if (a < k) {
      const int64_t e = i * k + a;
      const int64_t j = idx[e];
      if (j < p0 || j >= p1 || j == i)
        bad = true;
      else
        x[t] = ((uint64_t)(uint32_t)j << 32) | __float_as_uint(pc[e] * scale);
    }
  }
  if (bad) raise_status(status, TSNE_STATUS_BAD_INDEX);
  warp_sort<KPL>(x);
  // a column listed twice sits next to its copy now
  bool dup = false;
#pragma unroll
  for (int t = 0; t < KPL; t++) {
    uint64_t prev = __shfl_up_sync(0xffffffffu, x[t], 1);
    const uint64_t wrap = __shfl_sync(0xffffffffu, x[t > 0 ? t - 1 : 0], 31);
    if (lane == 0) prev = t > 0 ? wrap : kNoEntry;
    dup |= x[t] != kNoEntry && prev != kNoEntry && ent_col(prev) == ent_col(x[t]);
  }
  if (__any_sync(0xffffffffu, dup)) {
    uint64_t* f = fold[w];
#pragma unroll
    for (int t = 0; t < KPL; t++) f[t * 32 + lane] = x[t];
    __syncwarp();
    if (lane == 0) {  // fold each run of one column into its first entry, in order
      int o = 0;
      for (int q = 0; q < 32 * KPL && f[q] != kNoEntry; q++) {
        if (o > 0 && ent_col(f[o - 1]) == ent_col(f[q])) {
          const float v = combine(ent_val(f[o - 1]), ent_val(f[q]), fuzzy);
          f[o - 1] = ((uint64_t)ent_col(f[q]) << 32) | __float_as_uint(v);
        } else {
          f[o++] = f[q];
        }
      }
      for (int q = o; q < 32 * KPL; q++) f[q] = kNoEntry;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < KPL; t++) x[t] = f[t * 32 + lane];
  }
#pragma unroll
  for (int t = 0; t < KPL; t++) {
    const int a = t * 32 + lane;
    if (a < k) {
      const int64_t e = i * k + a;
      const bool ok = x[t] != kNoEntry;
      A[e] = x[t];
      bkey[e] = ok ? ((uint64_t)ent_col(x[t]) << bits) | (uint64_t)i : ~0ull;
      bval[e] = ok ? ent_val(x[t]) : 0.f;
    }
  }
}

// bstart[r] = first position of row r in the sorted transposed keys, for
// r = 0 .. n (bstart[n] = the count of valid keys; the dropped all-ones keys
// sort last).  Position p writes the rows after its predecessor's, up to its own.
__global__ void sym_bstart_kernel(const uint64_t* __restrict__ bkey, int64_t m2, int bits,
                                  int64_t n, uint32_t* __restrict__ bstart) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > m2) return;
  auto row_of = [&](int64_t q) -> int64_t {
    if (q >= m2) return n;
    const uint64_t r = bkey[q] >> bits;
    return r < (uint64_t)n ? (int64_t)r : n;
  };
  const int64_t r = row_of(p);
  const int64_t rp = p == 0 ? -1 : row_of(p - 1);
  for (int64_t q = rp + 1; q <= r; q++) bstart[q] = (uint32_t)p;
}

// Index of the first of the n sorted words s[0 .. n) not below c.
__device__ __forceinline__ int lower_bound_u32(const uint32_t* s, int n, uint32_t c) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s[mid] < c) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Loads A_i's columns into s (empty slots as 0xffffffff, which sort last) and
// returns the number of valid entries.
template <int KPL>
__device__ __forceinline__ int load_forward(const uint64_t* __restrict__ A, int64_t i, int k,
                                            uint32_t* s, uint64_t (&x)[KPL]) {
  const int lane = threadIdx.x & 31;
  int na = 0;
#pragma unroll
  for (int t = 0; t < KPL; t++) {
    const int a = t * 32 + lane;
    x[t] = a < k ? A[i * k + a] : kNoEntry;
    s[a] = ent_col(x[t]);
    na += x[t] != kNoEntry ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) na += __shfl_xor_sync(0xffffffffu, na, o);
  __syncwarp();
  return na;
}

// Per row i (one warp): dupc[p] = how many of B_i's entries before p have
// their column in A_i, and row_cnt[i] = |A_i| + |B_i| - |A_i and B_i|.
template <int KPL>
__global__ void __launch_bounds__(32 * kSymRows)
sym_count_kernel(const uint64_t* __restrict__ A, int k, const uint64_t* __restrict__ bkey,
                 const uint32_t* __restrict__ bstart, int64_t n, uint64_t cmask,
                 uint32_t* __restrict__ dupc, uint32_t* __restrict__ row_cnt) {
  __shared__ uint32_t sa[kSymRows][32 * KPL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kSymRows + w;
  if (i >= n) return;
  uint64_t x[KPL];
  const int na = load_forward<KPL>(A, i, k, sa[w], x);
  const int64_t b0 = bstart[i], b1 = bstart[i + 1];
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t run = 0;
  for (int64_t q = b0; q < b1; q += 32) {
    const int64_t p = q + lane;
    bool f = false;
    if (p < b1) {
      const uint32_t c = (uint32_t)(bkey[p] & cmask);
      const int at = lower_bound_u32(sa[w], na, c);
      f = at < na && sa[w][at] == c;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    if (p < b1) dupc[p] = run + __popc(bal & lt);
    run += __popc(bal);
  }
  if (lane == 0) row_cnt[i] = (uint32_t)(na + (b1 - b0)) - run;
}

// Per row i (one warp): every entry of the merged row at its slot.  An entry
// of A_i with column c lands after the union's columns below c: its index a in
// A_i, plus the B_i entries below c, less those among them also in A_i; an
// entry of B_i not in A_i likewise.  B_i's columns are searched in shared
// memory when they fit (up to 32 * KPL), else in global memory.
template <int KPL>
__global__ void __launch_bounds__(32 * kSymRows)
sym_write_kernel(const uint64_t* __restrict__ A, int k, const uint64_t* __restrict__ bkey,
                 const float* __restrict__ bval, const uint32_t* __restrict__ bstart,
                 const uint32_t* __restrict__ dupc, const uint32_t* __restrict__ row_off,
                 int64_t n, uint64_t cmask, int fuzzy, int32_t* __restrict__ col,
                 float* __restrict__ val, int64_t cap, int32_t* status) {
  __shared__ uint32_t sa[kSymRows][32 * KPL];
  __shared__ uint32_t sb[kSymRows][32 * KPL];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kSymRows + w;
  if (i >= n) return;
  uint64_t x[KPL];
  const int na = load_forward<KPL>(A, i, k, sa[w], x);
  const int64_t b0 = bstart[i], b1 = bstart[i + 1];
  const int64_t nb = b1 - b0;
  const int64_t base = row_off[i];
  const uint32_t dups = (uint32_t)(na + nb) - (row_off[i + 1] - row_off[i]);
  const bool staged = nb <= 32 * KPL;
  if (staged) {
    for (int q = lane; q < nb; q += 32) sb[w][q] = (uint32_t)(bkey[b0 + q] & cmask);
    __syncwarp();
  }
  bool over = false;
#pragma unroll
  for (int t = 0; t < KPL; t++) {
    const int a = t * 32 + lane;
    if (a < na) {
      const uint32_t c = ent_col(x[t]);
      int64_t at;  // B_i's entries below c
      if (staged) {
        at = lower_bound_u32(sb[w], (int)nb, c);
      } else {
        int64_t lo = 0, hi = nb;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if ((uint32_t)(bkey[b0 + mid] & cmask) < c) lo = mid + 1; else hi = mid;
        }
        at = lo;
      }
      const bool found = at < nb && (uint32_t)(bkey[b0 + at] & cmask) == c;
      const uint32_t dp = at < nb ? dupc[b0 + at] : dups;
      const int64_t p = base + a + at - dp;
      const float v = found ? combine(ent_val(x[t]), bval[b0 + at], fuzzy) : ent_val(x[t]);
      if (p < cap) {
        col[p] = (int32_t)c;
        val[p] = v;
      } else {
        over = true;
      }
    }
  }
  for (int64_t q = lane; q < nb; q += 32) {
    const uint32_t c = staged ? sb[w][q] : (uint32_t)(bkey[b0 + q] & cmask);
    const int at = lower_bound_u32(sa[w], na, c);
    if (at < na && sa[w][at] == c) continue;  // merged into A_i's entry
    const int64_t p = base + q + at - dupc[b0 + q];
    if (p < cap) {
      col[p] = (int32_t)c;
      val[p] = bval[b0 + q];
    } else {
      over = true;
    }
  }
  if (over) raise_status(status, TSNE_STATUS_CAPACITY);
}

__global__ void u32_to_i64_kernel(const uint32_t* __restrict__ in, int64_t m,
                                  int64_t* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) out[e] = (int64_t)in[e];
}

// Workspace of the symmetrisation for n points and k neighbours: k0 and v0
// hold 2nk words, k1 and v1 nk (the radix sort's second buffers), hist 256
// words per radix tile of nk keys, bstart and row_cnt n + 1.
struct SymWs {
  uint64_t* k0; uint64_t* k1; float* v0; float* v1;
  uint32_t* hist; uint32_t* part; uint32_t* bstart; uint32_t* row_cnt;
};

template <int KPL>
static cudaError_t symmetrize_k(const int32_t* idx, const float* pc, int64_t n, int k,
                                const SampleTable& tab, const SymWs& w, int64_t* row_ptr,
                                int32_t* col, float* val, int64_t cap, int fuzzy,
                                int32_t* status, cudaStream_t st) {
  const int64_t m2 = n * (int64_t)k;
  // keys (row << bits | col) with 2^bits > n, so the all-ones row of a dropped
  // key is above every valid row
  int bits = 1;
  while ((1ll << bits) <= n) bits++;
  const uint64_t cmask = (1ull << bits) - 1ull;
  uint64_t* A = w.k0 + m2;                               // forward lists (second half of k0)
  uint32_t* dupc = reinterpret_cast<uint32_t*>(w.v0 + m2);  // second half of v0
  {
    SampleTable* te = new SampleTable(tab);
    int32_t nblk = 0;
    for (int s = 0; s < tab.S; s++) {
      te->blk_off[s] = nblk;
      nblk += (int32_t)((tab.pt_off[s + 1] - tab.pt_off[s] + kSymRows - 1) / kSymRows);
    }
    te->blk_off[tab.S] = nblk;
    te->blk_pts = kSymRows;
    sym_forward_kernel<KPL><<<nblk, 32 * kSymRows, 0, st>>>(idx, pc, k, bits, *te, fuzzy, A, w.k0,
                                                            w.v0, status);
    delete te;
  }
  // stable sort of the transposed keys by their row bits only: columns stay in
  // increasing order within a row
  const int lo[1] = {bits};
  const int hi[1] = {2 * bits};
  uint64_t* bk;
  float* bv;
  cudaError_t e = launch_radix_sort(w.k0, w.v0, w.k1, w.v1, m2, lo, hi, 1, w.hist, w.part, &bk,
                                    &bv, st);
  if (e != cudaSuccess) return e;
  sym_bstart_kernel<<<(unsigned)((m2 + 1 + 255) / 256), 256, 0, st>>>(bk, m2, bits, n, w.bstart);
  const unsigned rb = (unsigned)((n + kSymRows - 1) / kSymRows);
  e = cudaMemsetAsync(w.row_cnt + n, 0, sizeof(uint32_t), st);
  if (e != cudaSuccess) return e;
  sym_count_kernel<KPL><<<rb, 32 * kSymRows, 0, st>>>(A, k, bk, w.bstart, n, cmask, dupc,
                                                      w.row_cnt);
  e = launch_scan_u32(w.row_cnt, w.row_cnt, n + 1, w.part, st);
  if (e != cudaSuccess) return e;
  sym_write_kernel<KPL><<<rb, 32 * kSymRows, 0, st>>>(A, k, bk, bv, w.bstart, dupc, w.row_cnt, n,
                                                      cmask, fuzzy, col, val, cap, status);
  u32_to_i64_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(w.row_cnt, n + 1, row_ptr);
  return cudaGetLastError();
}

cudaError_t launch_symmetrize(const int32_t* idx, const float* pc, int64_t n, int k,
                              const SampleTable& tab, const SymWs& w, int64_t* row_ptr,
                              int32_t* col, float* val, int64_t cap, int fuzzy, int32_t* status,
                              cudaStream_t st) {
  if (n <= 0) return cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st);
  if (k <= 32) return symmetrize_k<1>(idx, pc, n, k, tab, w, row_ptr, col, val, cap, fuzzy, status, st);
  if (k <= 64) return symmetrize_k<2>(idx, pc, n, k, tab, w, row_ptr, col, val, cap, fuzzy, status, st);
  if (k <= 128) return symmetrize_k<4>(idx, pc, n, k, tab, w, row_ptr, col, val, cap, fuzzy, status, st);
  if (k <= kSymMaxK) return symmetrize_k<8>(idx, pc, n, k, tab, w, row_ptr, col, val, cap, fuzzy, status, st);
  return cudaErrorInvalidValue;
}

}  // namespace tsne
