// k_sort.cu -- stable LSD radix sort of (u64 key, u32 value) pairs with the
// element count read from device memory, and an exclusive scan. Used by the
// cell sort (a2: key = cell << pid_bits | pid, unique, so the order is unique)
// and by the ionization resolve (events ordered by primary pid).
//
// One pass per 8-bit digit: (1) per-tile digit histograms, (2) per-digit scan of
// the tile histograms plus the digit totals, (3) stable scatter: tiles are
// processed in rounds of 256 consecutive elements; within a round the rank of an
// element among equal digits comes from __match_any_sync inside its warp and a
// prefix over the warps, so equal digits keep their input order.
#include "pic_internal.cuh"
#include "pic_kernels.cuh"

namespace pic {

constexpr int kSortBlock = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortBlock * kSortRounds;  // 4096 elements per tile
constexpr int kWarps = kSortBlock / 32;

static long long sort_blocks(long long n_max) { return (n_max + kSortTile - 1) / kSortTile > 0 ? (n_max + kSortTile - 1) / kSortTile : 1; }
long long sort_hist_entries(long long n_max) { return 256 * sort_blocks(n_max); }

__global__ void __launch_bounds__(kSortBlock) k_radix_hist(const unsigned long long* __restrict__ keys,
                                                           const unsigned long long* n_dev, long long n_max, int shift,
                                                           uint32_t* __restrict__ hist, int nblocks, const int* skip) {
  if (skip && *skip) return;
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long n = min((long long)*n_dev, n_max);
  const long long t0 = (long long)blockIdx.x * kSortTile;
  const long long t1 = min(t0 + kSortTile, n);
  for (long long i = t0 + threadIdx.x; i < t1; i += kSortBlock) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(long long)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of that digit's row over the tiles, and
// the digit total.
__global__ void __launch_bounds__(kSortBlock) k_radix_scan_rows(uint32_t* __restrict__ hist, int nblocks,
                                                                uint32_t* __restrict__ digit_tot, const int* skip) {
  if (skip && *skip) return;
  __shared__ uint32_t part[kSortBlock];
  uint32_t* row = hist + (long long)blockIdx.x * nblocks;
  const int per = (nblocks + kSortBlock - 1) / kSortBlock;
  const int b0 = threadIdx.x * per;
  uint32_t s = 0;
  for (int b = b0; b < min(b0 + per, nblocks); ++b) s += row[b];
  part[threadIdx.x] = s;
  __syncthreads();
  // inclusive scan of the partials (Hillis-Steele)
  for (int o = 1; o < kSortBlock; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int b = b0; b < min(b0 + per, nblocks); ++b) {
    const uint32_t v = row[b];
    row[b] = run;
    run += v;
  }
  if (threadIdx.x == kSortBlock - 1) digit_tot[blockIdx.x] = part[kSortBlock - 1];
}

__global__ void __launch_bounds__(kSortBlock) k_radix_scatter(const unsigned long long* __restrict__ kin,
                                                              const uint32_t* __restrict__ vin,
                                                              unsigned long long* __restrict__ kout,
                                                              uint32_t* __restrict__ vout, const unsigned long long* n_dev,
                                                              long long n_max, int shift, const uint32_t* __restrict__ hist,
                                                              int nblocks, const uint32_t* __restrict__ digit_tot,
                                                              const int* skip) {
  if (skip && *skip) return;
  __shared__ uint32_t base[256];           // global start of each digit for this tile
  __shared__ uint32_t wc[kWarps][256];     // per-warp digit counts -> offsets
  __shared__ uint32_t tot[256];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  // digit offsets: exclusive scan of the digit totals (256 entries)
  tot[t] = digit_tot[t];
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    const uint32_t v = t >= o ? tot[t - o] : 0u;
    __syncthreads();
    tot[t] += v;
    __syncthreads();
  }
  base[t] = (t ? tot[t - 1] : 0u) + hist[(long long)t * nblocks + blockIdx.x];
  for (int ww = 0; ww < kWarps; ++ww) wc[ww][t] = 0;
  __syncthreads();
  const long long n = min((long long)*n_dev, n_max);
  const long long t0 = (long long)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortRounds; ++r) {
    const long long i = t0 + (long long)r * kSortBlock + t;
    const bool valid = i < n;
    unsigned long long key = 0;
    uint32_t val = 0;
    uint32_t d = 256;
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (uint32_t)((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t lrank = __popc(peers & lt);
    if (valid && lrank == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    {
      // thread t owns digit t: turn per-warp counts into offsets, advance base
      uint32_t s = base[t];
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = wc[ww][t];
        wc[ww][t] = s;
        s += c;
      }
      base[t] = s;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = wc[w][d] + lrank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    for (int ww = 0; ww < kWarps; ++ww) wc[ww][t] = 0;
    __syncthreads();
  }
}

// Small inputs (n <= kSmallSort, the usual ionization event count): one block
// ranks every pair against all others (ties by input position, so the order is
// the stable one), writes it at its rank in the buffers the radix passes would
// end in, and sets *done so that those passes return at once.
constexpr int kSmallSort = 2048;
// In a recorded graph the radix passes sit in a conditional IF node whose
// condition this kernel sets (use_graph): they are launched only when needed.
__global__ void __launch_bounds__(1024) k_small_sort(const unsigned long long* __restrict__ kin,
                                                     const uint32_t* __restrict__ vin,
                                                     unsigned long long* __restrict__ kout,
                                                     uint32_t* __restrict__ vout, const unsigned long long* n_dev,
                                                     long long n_max, int* done, cudaGraphConditionalHandle h_radix,
                                                     int use_graph) {
  __shared__ unsigned long long sk[kSmallSort];
  const long long n = min((long long)*n_dev, n_max);
  if (use_graph && threadIdx.x == 0) cudaGraphSetConditional(h_radix, n > kSmallSort ? 1u : 0u);
  if (n > kSmallSort) {
    if (threadIdx.x == 0) *done = 0;
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = kin[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const unsigned long long k = sk[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const unsigned long long kj = sk[j];
      rank += (kj < k || (kj == k && j < i)) ? 1 : 0;
    }
    kout[rank] = k;
    vout[rank] = vin[i];
  }
  if (threadIdx.x == 0) *done = 1;
}

static int radix_passes(const SortBuffers& b, const unsigned long long* n_dev, int bit0, int bit1, cudaStream_t s,
                        const int* skip);

// When s is capturing (a step being recorded), the small path's kernel decides
// through a conditional IF node whether the radix passes run at all.
static cudaError_t radix_if_node(const SortBuffers& b, const unsigned long long* n_dev, int bit0, int bit1,
                                 cudaStream_t s) {
  cudaStreamCaptureStatus status;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &status, nullptr, &g, &deps, &edges, &ndeps);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h;
  if ((e = cudaGraphConditionalHandleCreate(&h, g, 0u, cudaGraphCondAssignDefault))) return e;
  PIC_LAUNCH(1, 1024, 0, s, k_small_sort)(b.ka, b.va, b.kb, b.vb, n_dev, b.n_max, b.small_done, h, 1);
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaStreamGetCaptureInfo(s, &status, nullptr, &g, &deps, &edges, &ndeps))) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if ((e = cudaGraphAddNode(&node, g, deps, edges, ndeps, &np))) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if ((e = cudaStreamBeginCaptureToGraph(b.aux, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) return e;
  radix_passes(b, n_dev, bit0, bit1, b.aux, nullptr);
  cudaGraph_t tmp;
  const cudaError_t e1 = cudaStreamEndCapture(b.aux, &tmp);
  if ((e = cudaGetLastError()) || (e = e1)) return e;
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

int radix_sort_pairs(const SortBuffers& b, const unsigned long long* n_dev, int bit0, int bit1, cudaStream_t s,
                     bool small_path) {
  const int passes = (bit1 - bit0 + 7) / 8;
  const int* skip = nullptr;
  // the small path writes where an odd number of passes ends (kb, vb); an even
  // number would end in the input buffers, which the ranking still reads
  if (small_path && (passes & 1)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (b.aux && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive) {
      if (radix_if_node(b, n_dev, bit0, bit1, s) != cudaSuccess) {
        // a half-built node must not be replayed: synchronising a capturing
        // stream is illegal and invalidates the capture, so the recording
        // fails and the instance steps directly from then on
        cudaStreamSynchronize(s);
        cudaGetLastError();
      }
      return 1;
    }
    const cudaGraphConditionalHandle none = 0;
    PIC_LAUNCH(1, 1024, 0, s, k_small_sort)(b.ka, b.va, b.kb, b.vb, n_dev, b.n_max, b.small_done, none, 0);
    skip = b.small_done;
  }
  return radix_passes(b, n_dev, bit0, bit1, s, skip);
}

static int radix_passes(const SortBuffers& b, const unsigned long long* n_dev, int bit0, int bit1, cudaStream_t s,
                        const int* skip) {
  const int nblocks = (int)sort_blocks(b.n_max);
  int src = 0;
  for (int shift = bit0; shift < bit1; shift += 8) {
    const unsigned long long* kin = src ? b.kb : b.ka;
    const uint32_t* vin = src ? b.vb : b.va;
    unsigned long long* kout = src ? b.ka : b.kb;
    uint32_t* vout = src ? b.va : b.vb;
    PIC_LAUNCH(nblocks, kSortBlock, 0, s, k_radix_hist)(kin, n_dev, b.n_max, shift, b.hist, nblocks, skip);
    PIC_LAUNCH(256, kSortBlock, 0, s, k_radix_scan_rows)(b.hist, nblocks, b.digit_tot, skip);
    PIC_LAUNCH(nblocks, kSortBlock, 0, s, k_radix_scatter)(kin, vin, kout, vout, n_dev, b.n_max, shift, b.hist, nblocks,
                                                   b.digit_tot, skip);
    src ^= 1;
  }
  return src;
}

// ---------------------------------------------------------------------------
// cell sort by buckets: scatter into the buckets, then sort each bucket
// ---------------------------------------------------------------------------
// words[i] = cell << 32 | slot (the bucket and the slot taken in it); the pair
// (pid << 32 | i) goes to cell_start[cell] + slot. The dead bucket is cell =
// ncell, and cell_start[ncell] is the live total. Tombstones are dropped after
// the sort, so their order is free: they take their permutation entries here,
// in slot order, and their bucket is never sorted.
__global__ void k_seg_scatter(long long ncell, long long n_max, const unsigned long long* n_dev,
                              const unsigned long long* __restrict__ words, const uint32_t* __restrict__ pids,
                              const long long* __restrict__ cs, unsigned long long* __restrict__ out,
                              uint32_t* __restrict__ perm) {
  const long long n = min((long long)*n_dev, n_max);
  for (long long i = gtid(); i < n; i += gstride()) {
    const unsigned long long w = words[i];
    const long long pos = cs[w >> 32] + (long long)(w & 0xFFFFFFFFull);
    if ((long long)(w >> 32) == ncell)
      perm[pos] = (uint32_t)i;
    else
      out[pos] = ((unsigned long long)pids[i] << 32) | (unsigned long long)i;
  }
}

// One thread per cell bucket: the rank of an entry among the bucket's
// (pid, index) values is its place. Larger buckets
// are listed for the warp-wide kernel (from the front of `big`) or the
// block-wide one (from the back; ncell + 1 entries hold both lists).
__global__ void k_seg_sort(long long ncell, const long long* __restrict__ cs, const unsigned long long* n_dev,
                           const unsigned long long* __restrict__ v, uint32_t* __restrict__ perm,
                           int32_t* __restrict__ big, SegCtl* ctl) {
  (void)n_dev;
  for (long long c = gtid(); c < ncell; c += gstride()) {
    const long long a = cs[c];
    const long long b = cs[c + 1];
    const long long m = b - a;
    if (m <= 0) continue;
    if (m == 1) {
      perm[a] = (uint32_t)v[a];
      continue;
    }
    if (m > kSegMid) {
      big[ncell - atomicAdd(&ctl->nbig, 1)] = (int32_t)c;
      continue;
    }
    if (m > kSegSmall) {
      big[atomicAdd(&ctl->nmid, 1)] = (int32_t)c;
      continue;
    }
    for (long long j = a; j < b; ++j) {
      const unsigned long long x = v[j];
      int r = 0;
      for (long long k = a; k < b; ++k) r += v[k] < x ? 1 : 0;
      perm[a + r] = (uint32_t)x;
    }
  }
}

// One warp per bucket of the front list (up to kSegMid entries, staged in the
// warp's slice of shared memory).
constexpr int kMidWarps = kSortBlock / 32;
__global__ void __launch_bounds__(kSortBlock) k_seg_sort_mid(long long ncell, const long long* __restrict__ cs,
                                                             const unsigned long long* n_dev,
                                                             const unsigned long long* __restrict__ v,
                                                             uint32_t* __restrict__ perm,
                                                             const int32_t* __restrict__ big, const SegCtl* ctl) {
  __shared__ unsigned long long sv[kMidWarps][kSegMid];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long n = (long long)*n_dev;
  const int nmid = ctl->nmid;
  for (int q = blockIdx.x * kMidWarps + w; q < nmid; q += gridDim.x * kMidWarps) {
    const long long c = big[q];
    const long long a = cs[c];
    const long long b = c < ncell ? cs[c + 1] : n;
    const int m = (int)(b - a);  // kSegSmall < m <= kSegMid
    __syncwarp();  // the previous bucket's readers are done with this slice
    for (int j = lane; j < m; j += 32) sv[w][j] = v[a + j];
    __syncwarp();
    for (int j = lane; j < m; j += 32) {
      const unsigned long long x = sv[w][j];
      int r = 0;
      for (int k = 0; k < m; ++k) r += sv[w][k] < x ? 1 : 0;
      perm[a + r] = (uint32_t)x;
    }
  }
}

// One block per bucket of the back list (up to kSegBig entries staged in
// shared memory; a larger one sets overflow and is left to the radix path).
__global__ void __launch_bounds__(kSortBlock) k_seg_sort_big(long long ncell, const long long* __restrict__ cs,
                                                             const unsigned long long* n_dev,
                                                             const unsigned long long* __restrict__ v,
                                                             uint32_t* __restrict__ perm,
                                                             const int32_t* __restrict__ big, SegCtl* ctl) {
  __shared__ unsigned long long sv[kSegBig];
  const long long n = (long long)*n_dev;
  const int nbig = ctl->nbig;
  for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
    const long long c = big[ncell - q];
    const long long a = cs[c];
    const long long b = c < ncell ? cs[c + 1] : n;
    const int m = (int)(b - a);
    if (m > kSegBig) {  // the same m in every thread: the block skips together
      if (threadIdx.x == 0) ctl->overflow = 1;
      continue;
    }
    __syncthreads();  // the previous bucket's readers are done with sv
    for (int j = threadIdx.x; j < m; j += blockDim.x) sv[j] = v[a + j];
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const unsigned long long x = sv[j];
      int r = 0;
      for (int k = 0; k < m; ++k) r += sv[k] < x ? 1 : 0;
      perm[a + r] = (uint32_t)x;
    }
  }
}

static int seg_grid(long long n) {
  const long long b = (n + kSortBlock - 1) / kSortBlock;
  const long long cap = 16LL * sm_count();
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

void launch_seg_scatter(long long ncell, long long n_max, const unsigned long long* n_dev,
                        const unsigned long long* words, const uint32_t* pids, const long long* cell_start,
                        unsigned long long* out, uint32_t* perm, cudaStream_t s) {
  PIC_LAUNCH(seg_grid(n_max), kSortBlock, 0, s, k_seg_scatter)(ncell, n_max, n_dev, words, pids, cell_start, out,
                                                               perm);
}

void launch_seg_sort(long long ncell, const long long* cell_start, const unsigned long long* n_dev,
                     const unsigned long long* vals, uint32_t* perm, int32_t* big, SegCtl* ctl, cudaStream_t s) {
  PIC_LAUNCH(seg_grid(ncell), kSortBlock, 0, s, k_seg_sort)(ncell, cell_start, n_dev, vals, perm, big, ctl);
  PIC_LAUNCH(8 * sm_count(), kSortBlock, 0, s, k_seg_sort_mid)(ncell, cell_start, n_dev, vals, perm, big, ctl);
  PIC_LAUNCH(2 * sm_count(), kSortBlock, 0, s, k_seg_sort_big)(ncell, cell_start, n_dev, vals, perm, big, ctl);
}

// ---------------------------------------------------------------------------
// exclusive scan int32 -> int64 (three kernels: tile sums, scan of sums, tiles)
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanBlock * kScanItems;

size_t scan_temp_bytes(long long n) {
  const long long tiles = (n + kScanTile - 1) / kScanTile + 1;
  return (size_t)tiles * sizeof(long long);
}

__device__ __forceinline__ long long block_incl_scan(long long v, long long* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const long long a = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
    __syncthreads();
    sm[threadIdx.x] += a;
    __syncthreads();
  }
  return sm[threadIdx.x];
}

__global__ void k_scan_tiles(const int32_t* __restrict__ c, long long n, long long* __restrict__ tile_sum) {
  __shared__ long long sm[kScanBlock];
  const long long t0 = (long long)blockIdx.x * kScanTile;
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
    if (i < n) s += c[i];
  }
  const long long inc = block_incl_scan(s, sm);
  if (threadIdx.x == kScanBlock - 1) tile_sum[blockIdx.x] = inc;
}

__global__ void k_scan_sums(long long* tile_sum, int ntiles) {
  __shared__ long long sm[kScanBlock];
  long long carry = 0;
  for (int b0 = 0; b0 < ntiles; b0 += kScanBlock) {
    const int i = b0 + threadIdx.x;
    const long long v = i < ntiles ? tile_sum[i] : 0;
    const long long inc = block_incl_scan(v, sm);
    if (i < ntiles) tile_sum[i] = carry + inc - v;  // exclusive
    __syncthreads();
    carry += sm[kScanBlock - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_sum[ntiles] = carry;
}

__global__ void k_scan_apply(const int32_t* __restrict__ c, long long n, const long long* __restrict__ tile_sum,
                             long long* __restrict__ out, int ntiles) {
  __shared__ long long sm[kScanBlock];
  const long long t0 = (long long)blockIdx.x * kScanTile;
  long long loc[kScanItems];
  long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
    loc[k] = s;
    if (i < n) s += c[i];
  }
  const long long inc = block_incl_scan(s, sm);
  const long long off = tile_sum[blockIdx.x] + inc - s;
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = t0 + (long long)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = off + loc[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tile_sum[ntiles];
}

void exclusive_scan_i32_i64(const int32_t* counts, long long n, long long* out, void* temp, cudaStream_t s) {
  const int ntiles = (int)((n + kScanTile - 1) / kScanTile);
  long long* ts = (long long*)temp;
  if (ntiles == 0) {
    cudaMemsetAsync(out, 0, sizeof(long long), s);
    return;
  }
  PIC_LAUNCH(ntiles, kScanBlock, 0, s, k_scan_tiles)(counts, n, ts);
  PIC_LAUNCH(1, kScanBlock, 0, s, k_scan_sums)(ts, ntiles);
  PIC_LAUNCH(ntiles, kScanBlock, 0, s, k_scan_apply)(counts, n, ts, out, ntiles);
}

}  // namespace pic
