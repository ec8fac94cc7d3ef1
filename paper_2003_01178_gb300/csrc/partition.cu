// Radix partitioning without stability, and the two operators built on it:
//
//  * crys_sort_msb - the most-significant-digit radix sort the paper's GPU sort number
//    comes from (Section 4.4): two 8-bit partition passes on the top digits, then every
//    bucket of the top 16 bits is sorted inside one thread block (shared memory) by the
//    low 16 bits.  Unstable, as in the paper.
//  * crys_join_partitioned - the radix-partitioned hash join Section 4.3 sets beside the
//    no-partitioning join for build sides far beyond the caches: both sides are split by
//    hash bits in two passes so that each build partition's table fits in shared memory,
//    then each partition is built and probed there.
//
// A partition pass moves (key, value) pairs by an 8-bit digit of the key inside each of
// up to 65536 segments (the buckets of the previous pass): a histogram kernel counts the
// digits of every tile, a scan kernel turns the counts into the start of every (segment,
// digit) bucket, and a scatter kernel ranks a tile's pairs by digit with per-warp
// shared-memory counters (atomic, hence unstable), reserves each digit's run of the tile
// with one global atomic per digit, sorts the tile in shared memory and stores each run
// with consecutive addresses.  No pass waits on another block, so nothing here spins.
#include "common.cuh"

namespace crys {
namespace {

constexpr int kBuckets = 256;
constexpr int kPartThreads = 256;
constexpr int kPartItems = 8;
constexpr int kPartTile = kPartThreads * kPartItems;  // rows per tile of a partition pass

// Digit of a key: ((key * mult) >> shift) & mask, then XOR flip.  Sort digits use
// mult = 1 (flip 0x80 on the top digit for signed order); join digits use the bits of
// the multiplicative hash key * 2654435769 from the top down.
struct DigitFn {
  uint32_t mult, shift, mask, flip;
  __host__ __device__ __forceinline__ uint32_t operator()(int32_t k) const {
    return (((static_cast<uint32_t>(k) * mult) >> shift) & mask) ^ flip;
  }
};

// Segments of a pass: segment s covers rows [begin[s], begin[s] + size[s]) and owns the
// tiles [tile_start[s], tile_start[s + 1]) of the pass (tile_start has count + 1 entries);
// tile_seg[b] is the segment of tile b (unused when there is one segment).
struct Segs {
  const int64_t* begin;
  const int64_t* size;
  const uint32_t* tile_start;
  const uint32_t* tile_seg;
  int32_t count;
};

// The segment and rows of tile `b` of a pass: seg = -1 past the last tile.
struct TileAt {
  int seg;
  int valid;
  int64_t row0;
};

__device__ __forceinline__ TileAt find_tile(const Segs& S, uint32_t b, int tile_rows) {
  TileAt r{-1, 0, 0};
  if (b >= S.tile_start[S.count]) return r;
  const int lo = S.count == 1 ? 0 : static_cast<int>(S.tile_seg[b]);
  const int64_t t = static_cast<int64_t>(b - S.tile_start[lo]);
  const int64_t rem = S.size[lo] - t * tile_rows;
  r.seg = lo;
  r.row0 = S.begin[lo] + t * tile_rows;
  r.valid = static_cast<int>(rem < tile_rows ? rem : tile_rows);
  return r;
}

// Block-wide exclusive scan of one value per thread (THREADS <= 1024); also returns the
// total.  `tmp` holds one word per warp.
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* tmp, uint32_t* total) {
  constexpr int WARPS = THREADS / kWarp;
  const int lane = threadIdx.x % kWarp, warp = threadIdx.x / kWarp;
  const uint32_t inc = static_cast<uint32_t>(warp_inclusive_scan(static_cast<int32_t>(x), lane));
  if (lane == kWarp - 1) tmp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < WARPS ? tmp[lane] : 0u;
    const uint32_t wi = static_cast<uint32_t>(warp_inclusive_scan(static_cast<int32_t>(w), lane));
    if (lane < WARPS) tmp[lane] = wi - w;
    if (lane == WARPS - 1) tmp[WARPS] = wi;  // the total, beside the warps' offsets
  }
  __syncthreads();
  const uint32_t r = tmp[warp] + inc - x;
  *total = tmp[WARPS];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- segment set-up

// One segment covering rows [0, n).
__global__ void seg_init_kernel(int64_t n, int tile_rows, int64_t* begin, int64_t* size, uint32_t* tile_start) {
  begin[0] = 0;
  size[0] = n;
  tile_start[0] = 0;
  tile_start[1] = static_cast<uint32_t>((n + tile_rows - 1) / tile_rows);
}

// The buckets of a pass as the segments of the next one: begin/size from the bucket
// starts and counts, their tile prefix and the segment of every tile (one block of 1024
// threads, any count).
__global__ void __launch_bounds__(1024) seg_from_buckets_kernel(const int64_t* bucket_begin, const uint32_t* bucket_count,
                                                                int n, int tile_rows, int64_t* begin, int64_t* size,
                                                                uint32_t* tile_start, uint32_t* tile_seg) {
  __shared__ uint32_t tmp[kWarp + 1];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int i = base + static_cast<int>(threadIdx.x);
    uint32_t tiles = 0;
    if (i < n) {
      begin[i] = bucket_begin[i];
      size[i] = bucket_count[i];
      tiles = (bucket_count[i] + static_cast<uint32_t>(tile_rows) - 1) / static_cast<uint32_t>(tile_rows);
    }
    uint32_t total;
    const uint32_t ex = block_exclusive_scan<1024>(tiles, tmp, &total);
    if (i < n) tile_start[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile_start[n] = carry;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += 1024)
    for (uint32_t t = tile_start[i]; t < tile_start[i + 1]; ++t) tile_seg[t] = static_cast<uint32_t>(i);
}

// ---------------------------------------------------------------- one partition pass

// Digit counts of every segment.  A persistent block takes a contiguous range of the
// pass's tiles (so it stays in one segment for many tiles), counts in shared memory and
// adds its counts to the segment's when the segment changes and at the end.
__global__ void __launch_bounds__(kPartThreads) part_hist_kernel(const int32_t* __restrict__ keys, Segs S, DigitFn f,
                                                                 uint32_t* hist) {
  constexpr int kCopies = 4;
  __shared__ uint32_t h[kCopies][kBuckets];
  const int tid = threadIdx.x;
  for (int i = tid; i < kCopies * kBuckets; i += kPartThreads) (&h[0][0])[i] = 0;
  const uint32_t total = S.tile_start[S.count];
  const uint32_t t0 = static_cast<uint32_t>((static_cast<uint64_t>(total) * blockIdx.x) / gridDim.x);
  const uint32_t t1 = static_cast<uint32_t>((static_cast<uint64_t>(total) * (blockIdx.x + 1)) / gridDim.x);
  uint32_t* mine = h[(tid / kWarp) % kCopies];
  int cur = -1;
  auto flush = [&](int seg) {
    __syncthreads();
    for (int d = tid; d < kBuckets; d += kPartThreads) {
      uint32_t c = 0;
#pragma unroll
      for (int r = 0; r < kCopies; ++r) {
        c += h[r][d];
        h[r][d] = 0;
      }
      if (c) atomicAdd(&hist[static_cast<int64_t>(seg) * kBuckets + d], c);
    }
    __syncthreads();
  };
  __syncthreads();
  for (uint32_t b = t0; b < t1; ++b) {
    const TileAt at = find_tile(S, b, kPartTile);  // every thread: the same few cached words
    if (at.seg != cur) {
      if (cur >= 0) flush(cur);
      cur = at.seg;
    }
    int32_t k[kPartItems];
#pragma unroll
    for (int i = 0; i < kPartItems; ++i) {
      const int idx = i * kPartThreads + tid;
      k[i] = idx < at.valid ? keys[at.row0 + idx] : 0;
    }
#pragma unroll
    for (int i = 0; i < kPartItems; ++i)
      if (i * kPartThreads + tid < at.valid) atomicAdd(&mine[f(k[i])], 1u);
  }
  if (cur >= 0) flush(cur);
}

// Bucket starts of every segment: begin of the segment plus the exclusive prefix of its
// digit counts.  One block of 256 threads per segment.
__global__ void __launch_bounds__(kBuckets) part_scan_kernel(const uint32_t* hist, const int64_t* seg_begin,
                                                             unsigned long long* cursor, int64_t* bucket_begin) {
  __shared__ uint32_t tmp[kWarp + 1];
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kBuckets + threadIdx.x;
  uint32_t total;
  const uint32_t ex = block_exclusive_scan<kBuckets>(hist[i], tmp, &total);
  const int64_t b = seg_begin[blockIdx.x] + ex;
  cursor[i] = static_cast<unsigned long long>(b);
  bucket_begin[i] = b;
}

constexpr long long kSkipRun = -(1ll << 62);  // a digit run that is reported and dropped
static_assert(kPartThreads == kBuckets, "one thread per digit in the scatter's bookkeeping");

struct ScatterArgs {
  const int32_t* kin;
  const int32_t* vin;
  int32_t* kout;
  int32_t* vout;
  Segs S;
  DigitFn f;
  unsigned long long* cursor;  // [segments][256] next free row of each bucket
  int32_t* err;
};

__global__ void __launch_bounds__(kPartThreads) part_scatter_kernel(const __grid_constant__ ScatterArgs a) {
  constexpr int WARPS = kPartThreads / kWarp;
  extern __shared__ __align__(16) int32_t part_smem[];
  int32_t* sk = part_smem;               // the tile's keys in bucket order
  int32_t* sv = part_smem + kPartTile;   // and values
  __shared__ uint32_t wh[WARPS][kBuckets];  // per-warp digit counts, then the warps' offsets
  __shared__ uint32_t lstart[kBuckets];     // tile-local start of each digit's run
  __shared__ long long gshift[kBuckets];    // global row minus tile-local position, or kSkipRun
  __shared__ uint32_t tmp[kWarp + 1];
  __shared__ int seg_sh;
  __shared__ long long row0_sh, seg_lo_sh, seg_hi_sh;
  __shared__ int valid_sh;
  const int tid = threadIdx.x, warp = tid / kWarp;
  for (int i = tid; i < WARPS * kBuckets; i += kPartThreads) (&wh[0][0])[i] = 0;
  if (tid == 0) {
    const TileAt at = find_tile(a.S, blockIdx.x, kPartTile);
    seg_sh = at.seg;
    row0_sh = at.row0;
    valid_sh = at.valid;
    if (at.seg >= 0) {
      seg_lo_sh = a.S.begin[at.seg];
      seg_hi_sh = a.S.begin[at.seg] + a.S.size[at.seg];
    }
  }
  __syncthreads();
  const int seg = seg_sh;
  if (seg < 0) return;
  const int64_t row0 = row0_sh;
  const int valid = valid_sh;
  int32_t k[kPartItems], v[kPartItems];
  uint32_t r[kPartItems];
#pragma unroll
  for (int i = 0; i < kPartItems; ++i) {
    const int idx = i * kPartThreads + tid;
    k[i] = idx < valid ? a.kin[row0 + idx] : 0;
    v[i] = idx < valid ? a.vin[row0 + idx] : 0;
  }
  // rank inside the warp's counters (shared-memory atomics: unstable)
#pragma unroll
  for (int i = 0; i < kPartItems; ++i)
    r[i] = (i * kPartThreads + tid < valid) ? atomicAdd(&wh[warp][a.f(k[i])], 1u) : 0u;
  __syncthreads();
  {
    const int d = tid;  // kPartThreads == kBuckets: one thread per digit
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const uint32_t c = wh[w][d];
      wh[w][d] = run;
      run += c;
    }
    uint32_t total;
    const uint32_t ls = block_exclusive_scan<kPartThreads>(run, tmp, &total);
    lstart[d] = ls;
    long long shift = 0;
    if (run) {
      const long long g = static_cast<long long>(atomicAdd(&a.cursor[static_cast<int64_t>(seg) * kBuckets + d],
                                                           static_cast<unsigned long long>(run)));
      // the run must stay inside its segment (it does whenever the counts came from
      // these keys); otherwise report and drop it rather than write out of place
      if (g < seg_lo_sh || g + run > seg_hi_sh) {
        set_error(a.err, CRYS_DEV_BOUNDS);
        shift = kSkipRun;
      } else {
        shift = g - ls;
      }
    }
    gshift[d] = shift;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kPartItems; ++i) {
    if (i * kPartThreads + tid < valid) {
      const uint32_t d = a.f(k[i]);
      const uint32_t p = lstart[d] + wh[warp][d] + r[i];
      sk[p] = k[i];
      sv[p] = v[i];
    }
  }
  __syncthreads();
  for (int j = tid; j < valid; j += kPartThreads) {
    const int32_t key = sk[j];
    const long long s = gshift[a.f(key)];
    if (s == kSkipRun) continue;
    a.kout[s + j] = key;
    a.vout[s + j] = sv[j];
  }
}

// ---------------------------------------------------------------- local sort (MSB sort)
//
// Every bucket of the top 16 key bits is sorted by the low 16 bits inside one block.  A
// bucket of at most kLocalCap rows is sorted in shared memory as (low 16 bits, row)
// words, 4 stable passes of 4 bits: each thread owns kLocalIpt consecutive words, counts
// their digits in packed 8-bit counters, a block scan over (digit, thread) gives every
// thread the first position of each digit, and the thread walks its words in order
// (stable).  The sorted rows are then gathered from the bucket in global memory (it was
// just read, so L2 serves the gather) and stored with consecutive addresses.

constexpr int kLocalThreads = 256;
constexpr int kLocalIpt = 20;
constexpr int kLocalCap = kLocalThreads * kLocalIpt;  // 5120 rows: a 13-bit row index
static_assert(kLocalCap <= 8192 && kLocalIpt <= 255, "13-bit rows, 8-bit per-thread digit counters");
constexpr int kLocalPad = kLocalIpt + 1;              // words per thread slice incl. one pad word

// Position p of the sorted order in the padded layout (one pad word per 16 words, so that
// the threads' slices start in distinct banks).
__device__ __forceinline__ int padded(int p) { return p + p / kLocalIpt; }

// One stable 4-bit pass of the words in `src` (cnt valid ones, padded layout) into
// `dst` by the digit (w >> shift) & 15.  `scan` holds 16 x kLocalThreads counters.
__device__ __forceinline__ void local_pass(const uint32_t* src, uint32_t* dst, int cnt, int shift, uint32_t* scan,
                                           uint32_t* tmp) {
  const int t = threadIdx.x;
  uint32_t w[kLocalIpt];
  uint32_t c4[4] = {0u, 0u, 0u, 0u};  // 16 digit counters of 8 bits, packed four to a word
#pragma unroll
  for (int i = 0; i < kLocalIpt; ++i) {
    const int p = t * kLocalIpt + i;
    w[i] = p < cnt ? src[t * kLocalPad + i] : 0u;
    if (p < cnt) {
      const uint32_t d = (w[i] >> shift) & 15u;
      const uint32_t inc = 1u << (8 * (d & 3u));
      c4[0] += (d >> 2) == 0 ? inc : 0u;
      c4[1] += (d >> 2) == 1 ? inc : 0u;
      c4[2] += (d >> 2) == 2 ? inc : 0u;
      c4[3] += (d >> 2) == 3 ? inc : 0u;
    }
  }
#pragma unroll
  for (int d = 0; d < 16; ++d) scan[d * kLocalThreads + t] = (c4[d >> 2] >> (8 * (d & 3))) & 0xFFu;
  __syncthreads();
  // exclusive scan of the 16 x kLocalThreads counters in (digit, thread) order: each
  // thread takes 16 consecutive counters, then one block scan of the threads' sums
  static_assert(16 * kLocalThreads % kLocalThreads == 0, "16 counters per thread");
  uint32_t loc[16];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    loc[j] = scan[t * 16 + j];
    sum += loc[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan<kLocalThreads>(sum, tmp, &total);
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const uint32_t c = loc[j];
    scan[t * 16 + j] = run;
    run += c;
  }
  __syncthreads();
  // stable placement: this thread's words in order, each at its digit's next position
#pragma unroll
  for (int i = 0; i < kLocalIpt; ++i) {
    if (t * kLocalIpt + i < cnt) {
      const uint32_t d = (w[i] >> shift) & 15u;
      uint32_t* slot = &scan[d * kLocalThreads + t];
      const uint32_t p = *slot;
      *slot = p + 1;
      dst[padded(static_cast<int>(p))] = w[i];
    }
  }
  __syncthreads();
}

struct LocalArgs {
  const int32_t* kin;  // buckets of the top 16 bits (after two partition passes)
  const int32_t* vin;
  int32_t* kout;
  int32_t* vout;
  const int64_t* bucket_begin;   // [65536]
  const uint32_t* bucket_count;  // [65536]
  int32_t* err;
};

// Rows of a bucket larger than kLocalCap: sorted by one block through global memory,
// 4 stable passes of 4 bits over chunks of kLocalCap rows (the digit starts of the whole
// bucket carried from chunk to chunk), kin -> kout -> kin -> kout -> kin, then copied
// to kout.  Correct for every input; a bucket this large means heavily repeated top bits.
__device__ void local_sort_large(const LocalArgs& a, int64_t begin, int64_t size, uint32_t* words, uint32_t* scan,
                                 uint32_t* tmp) {
  __shared__ uint32_t digit_base[16];
  const int t = threadIdx.x;
  int32_t* bufk[2] = {const_cast<int32_t*>(a.kin), a.kout};
  int32_t* bufv[2] = {const_cast<int32_t*>(a.vin), a.vout};
  uint32_t* wa = words;                          // padded word arrays of one chunk
  uint32_t* wb = words + kLocalThreads * kLocalPad;
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 4 * pass;
    const int32_t* sk = bufk[pass & 1];
    const int32_t* sv = bufv[pass & 1];
    int32_t* dk = bufk[(pass + 1) & 1];
    int32_t* dv = bufv[(pass + 1) & 1];
    // digit counts of the whole bucket, then their exclusive prefix
    if (t < 16) digit_base[t] = 0;
    __syncthreads();
    for (int64_t i = t; i < size; i += kLocalThreads)
      atomicAdd(&digit_base[(static_cast<uint32_t>(sk[begin + i]) >> shift) & 15u], 1u);
    __syncthreads();
    if (t == 0) {
      uint32_t run = 0;
      for (int d = 0; d < 16; ++d) {
        const uint32_t c = digit_base[d];
        digit_base[d] = run;
        run += c;
      }
    }
    __syncthreads();
    for (int64_t c0 = 0; c0 < size; c0 += kLocalCap) {
      const int cnt = static_cast<int>((size - c0) < kLocalCap ? (size - c0) : kLocalCap);
      // words of the chunk: (digit << 13) | row within the chunk, in chunk order
#pragma unroll
      for (int i = 0; i < kLocalIpt; ++i) {
        const int p = t * kLocalIpt + i;
        if (p < cnt) {
          const uint32_t d = (static_cast<uint32_t>(sk[begin + c0 + p]) >> shift) & 15u;
          wa[t * kLocalPad + i] = (d << 13) | static_cast<uint32_t>(p);
        }
      }
      __syncthreads();
      local_pass(wa, wb, cnt, 13, scan, tmp);
      // wb holds the chunk stably ordered by digit; a word's rank inside its digit is its
      // position minus the chunk's count of smaller digits
      __shared__ uint32_t chunk_start[16];
      __shared__ uint32_t chunk_count[16];
      if (t < 16) chunk_count[t] = 0;
      __syncthreads();
      for (int p = t; p < cnt; p += kLocalThreads) atomicAdd(&chunk_count[wb[padded(p)] >> 13], 1u);
      __syncthreads();
      if (t == 0) {
        uint32_t run = 0;
        for (int d = 0; d < 16; ++d) {
          chunk_start[d] = run;
          run += chunk_count[d];
        }
      }
      __syncthreads();
      for (int p = t; p < cnt; p += kLocalThreads) {
        const uint32_t w = wb[padded(p)];
        const uint32_t d = w >> 13, row = w & 8191u;
        const int64_t g = begin + digit_base[d] + (p - chunk_start[d]);
        dk[g] = sk[begin + c0 + row];
        dv[g] = sv[begin + c0 + row];
      }
      __syncthreads();
      if (t < 16) digit_base[t] += chunk_count[t];
      __syncthreads();
    }
    __threadfence_block();
    __syncthreads();
  }
  // four passes end in kin: copy the bucket to kout
  for (int64_t i = t; i < size; i += kLocalThreads) {
    a.kout[begin + i] = a.kin[begin + i];
    a.vout[begin + i] = a.vin[begin + i];
  }
}

__global__ void __launch_bounds__(kLocalThreads) local_sort_kernel(const __grid_constant__ LocalArgs a) {
  extern __shared__ __align__(16) uint32_t local_smem[];
  uint32_t* wa = local_smem;                                   // padded words, ping
  uint32_t* wb = local_smem + kLocalThreads * kLocalPad;      // pong
  uint32_t* scan = wb + kLocalThreads * kLocalPad;            // 16 x kLocalThreads counters
  __shared__ uint32_t tmp[kWarp + 1];
  const int t = threadIdx.x;
  const int64_t begin = a.bucket_begin[blockIdx.x];
  const int64_t size = a.bucket_count[blockIdx.x];
  if (size == 0) return;
  if (size > kLocalCap) {
    local_sort_large(a, begin, size, local_smem, scan, tmp);
    return;
  }
  const int cnt = static_cast<int>(size);
#pragma unroll
  for (int i = 0; i < kLocalIpt; ++i) {
    const int p = t * kLocalIpt + i;
    if (p < cnt) wa[t * kLocalPad + i] = ((static_cast<uint32_t>(a.kin[begin + p]) & 0xFFFFu) << 13) | static_cast<uint32_t>(p);
  }
  __syncthreads();
  local_pass(wa, wb, cnt, 13, scan, tmp);
  local_pass(wb, wa, cnt, 17, scan, tmp);
  local_pass(wa, wb, cnt, 21, scan, tmp);
  local_pass(wb, wa, cnt, 25, scan, tmp);
  for (int p = t; p < cnt; p += kLocalThreads) {
    const uint32_t row = wa[padded(p)] & 8191u;
    a.kout[begin + p] = a.kin[begin + row];
    a.vout[begin + p] = a.vin[begin + row];
  }
}

constexpr size_t kLocalSmem = (2 * kLocalThreads * kLocalPad + 16 * kLocalThreads) * sizeof(uint32_t);

// ---------------------------------------------------------------- partitioned join
//
// After both sides are partitioned by the same hash bits, build partition p's table in
// shared memory (linear probing, capacity a power of two of at least twice its rows, at
// most kJoinSlots) and probe the tiles of probe partition p against it.  Persistent
// blocks take contiguous ranges of probe tiles, so a block works through whole
// partitions in order, builds each table once, and has the copy engine bring the next
// tile's rows into L2 while it probes.  A build partition too large for shared memory
// gets a table in global scratch at 4 x its first row (its capacity is at most 4 x its
// rows, so the regions of different partitions do not overlap), built beforehand.  Each
// block adds its sum and matches with one atomic each.

constexpr int kJoinThreads = 512;
constexpr int kJoinItems = 16;
constexpr int kJoinTile = kJoinThreads * kJoinItems;  // probe rows per block
constexpr int kJoinSlots = 8192;                      // 64 KB table in shared memory

struct JoinArgs {
  const int32_t* bkey;  // build side, partitioned
  const int32_t* bval;
  const int64_t* b_begin;   // [partitions]
  const uint32_t* b_count;  // [partitions]
  const int32_t* pkey;      // probe side, partitioned
  const int32_t* ppay;
  Segs probe;               // probe partitions with their tile prefix
  uint64_t* arena;          // global tables of oversized build partitions (4 x build rows)
  unsigned long long* sum;
  unsigned long long* matches;
  int32_t* err;
};

// Slot of a key inside a partition's table: the MurmurHash3 32-bit finaliser (Appleby),
// independent of the multiplicative hash whose top bits chose the partition.
__device__ __forceinline__ uint32_t slot_hash(int32_t k) {
  uint32_t h = static_cast<uint32_t>(k);
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// The single partition of a join whose build side needs no partitioning.
__global__ void one_partition_kernel(int64_t nb, int64_t np, int tile_rows, int64_t* b_begin, uint32_t* b_count,
                                     int64_t* p_begin, int64_t* p_size, uint32_t* p_tiles) {
  b_begin[0] = 0;
  b_count[0] = static_cast<uint32_t>(nb);
  p_begin[0] = 0;
  p_size[0] = np;
  p_tiles[0] = 0;
  p_tiles[1] = static_cast<uint32_t>((np + tile_rows - 1) / tile_rows);
}

// Table capacity of a build partition: a power of two of at least twice its rows.
__device__ __forceinline__ uint32_t join_capacity(uint32_t rows) {
  uint32_t cap = 2;
  while (cap < 2u * rows) cap <<= 1;
  return cap;
}

// Inserts the rows of build partition p into `table` (cap slots, already empty).
__device__ __forceinline__ void join_insert(const JoinArgs& a, int64_t bb, uint32_t bn, uint64_t* table, uint32_t cap,
                                            int nthreads) {
  const uint32_t mask = cap - 1;
  for (uint32_t i = threadIdx.x; i < bn; i += nthreads) {
    const int32_t key = a.bkey[bb + i];
    const uint64_t packed = static_cast<uint64_t>(static_cast<uint32_t>(key)) |
                            (static_cast<uint64_t>(static_cast<uint32_t>(a.bval[bb + i])) << 32);
    uint32_t h = slot_hash(key) & mask;
    for (uint32_t step = 0; step < cap; ++step) {
      const uint64_t prev = atomicCAS(reinterpret_cast<unsigned long long*>(table + h), kEmptySlot, packed);
      if (prev == kEmptySlot) break;
      if (static_cast<uint32_t>(prev) == static_cast<uint32_t>(key)) {
        set_error(a.err, CRYS_DEV_DUP_KEY);
        break;
      }
      h = (h + 1) & mask;
    }
  }
}

// Build partitions too large for shared memory get their table in the global arena, built
// once here (one block per partition) before any probe reads it.
__global__ void __launch_bounds__(kJoinThreads) join_build_large_kernel(const __grid_constant__ JoinArgs a, int parts) {
  const int p = blockIdx.x;
  if (p >= parts) return;
  const uint32_t bn = a.b_count[p];
  const uint32_t cap = join_capacity(bn);
  if (cap <= static_cast<uint32_t>(kJoinSlots)) return;
  const int64_t bb = a.b_begin[p];
  uint64_t* table = a.arena + 4 * bb;
  for (uint32_t i = threadIdx.x; i < cap; i += kJoinThreads) table[i] = kEmptySlot;
  __syncthreads();
  join_insert(a, bb, bn, table, cap, kJoinThreads);
}

// Bulk L2 prefetch of rows [row, row + rows) of a column (whole 16-byte groups inside the
// range; a partial group at either end is left to the demand loads).
__device__ __forceinline__ void prefetch_rows(const int32_t* col, int64_t row, int64_t rows) {
  const int64_t first = (row + 3) & ~int64_t{3}, last = (row + rows) & ~int64_t{3};
  if (last > first) bulk_prefetch_l2(col + first, static_cast<uint32_t>((last - first) * 4));
}

__global__ void __launch_bounds__(kJoinThreads, 2) join_partition_kernel(const __grid_constant__ JoinArgs a) {
  extern __shared__ __align__(16) uint64_t stab[];  // kJoinSlots slots
  __shared__ uint64_t red[kJoinThreads / kWarp];
  const int tid = threadIdx.x;
  // a persistent block takes a contiguous range of the probe tiles: tiles of one partition
  // are adjacent, so a block mostly works through whole partitions in order
  const uint32_t total = a.probe.tile_start[a.probe.count];
  const uint32_t t0 = static_cast<uint32_t>((static_cast<uint64_t>(total) * blockIdx.x) / gridDim.x);
  const uint32_t t1 = static_cast<uint32_t>((static_cast<uint64_t>(total) * (blockIdx.x + 1)) / gridDim.x);
  uint64_t sum = 0, matches = 0;
  int built = -1;  // partition whose table is in shared memory
  for (uint32_t b = t0; b < t1; ++b) {
    const TileAt at = find_tile(a.probe, b, kJoinTile);
    const int p = at.seg;
    const int64_t bb = a.b_begin[p];
    const uint32_t bn = a.b_count[p];
    const uint32_t cap = join_capacity(bn);
    const bool in_smem = cap <= static_cast<uint32_t>(kJoinSlots);
    if (tid == 0 && b + 1 < t1) {  // the next tile's rows travel to L2 meanwhile
      const TileAt nx = find_tile(a.probe, b + 1, kJoinTile);
      prefetch_rows(a.pkey, nx.row0, nx.valid);
      prefetch_rows(a.ppay, nx.row0, nx.valid);
      if (nx.seg != p) {
        prefetch_rows(a.bkey, a.b_begin[nx.seg], a.b_count[nx.seg]);
        prefetch_rows(a.bval, a.b_begin[nx.seg], a.b_count[nx.seg]);
      }
    }
    const uint64_t* table = in_smem ? stab : a.arena + 4 * bb;  // the arena's table is built already
    const uint32_t mask = cap - 1;
    int32_t k[kJoinItems], pay[kJoinItems];
#pragma unroll
    for (int i = 0; i < kJoinItems; ++i) {
      const int idx = i * kJoinThreads + tid;
      k[i] = idx < at.valid ? a.pkey[at.row0 + idx] : 0;
      pay[i] = idx < at.valid ? a.ppay[at.row0 + idx] : 0;
    }
    if (in_smem && built != p) {
      __syncthreads();  // the previous partition's probes are done with the table
      for (uint32_t i = tid; i < cap; i += kJoinThreads) stab[i] = kEmptySlot;
      __syncthreads();
      join_insert(a, bb, bn, stab, cap, kJoinThreads);
      __syncthreads();
      built = p;
    }
#pragma unroll
    for (int i = 0; i < kJoinItems; ++i) {
      if (i * kJoinThreads + tid >= at.valid) continue;
      uint32_t h = slot_hash(k[i]) & mask;
      for (uint32_t step = 0; step < cap; ++step) {
        const uint64_t s = table[h];
        if (s == kEmptySlot) break;
        if (static_cast<uint32_t>(s) == static_cast<uint32_t>(k[i])) {
          sum += static_cast<uint64_t>(static_cast<int64_t>(pay[i]) * static_cast<int64_t>(static_cast<int32_t>(s >> 32)));
          matches += 1;
          break;
        }
        h = (h + 1) & mask;
      }
    }
  }
  const uint64_t bs = block_sum_u64<kJoinThreads>(sum, red);
  const uint64_t bm = block_sum_u64<kJoinThreads>(matches, red);
  if (tid == 0) {
    if (bs) atomicAdd(a.sum, static_cast<unsigned long long>(bs));
    if (a.matches && bm) atomicAdd(a.matches, static_cast<unsigned long long>(bm));
  }
}

// ---------------------------------------------------------------- host side

size_t up256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// A bump allocator over caller scratch (every region 256-byte aligned).
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(void* p) : base(static_cast<char*>(p)) {}
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += up256(count * sizeof(T));
    return p;
  }
};

// Device arrays of one partition level of one side.
struct Level {
  int64_t* seg_begin;
  int64_t* seg_size;
  uint32_t* tile_start;
  uint32_t* tile_seg;         // [tiles]
  uint32_t* hist;             // [segments][256]
  unsigned long long* cursor;  // [segments][256]
  int64_t* bucket_begin;      // [segments * 256]
};

int64_t tiles_bound(int64_t n, int segments, int tile_rows) { return (n + tile_rows - 1) / tile_rows + segments; }

Level carve_level(Carve& c, int segments, int64_t rows) {
  Level L;
  L.seg_begin = c.take<int64_t>(segments);
  L.seg_size = c.take<int64_t>(segments);
  L.tile_start = c.take<uint32_t>(segments + 1);
  L.tile_seg = c.take<uint32_t>(static_cast<size_t>(tiles_bound(rows, segments, kPartTile)));
  L.hist = c.take<uint32_t>(static_cast<size_t>(segments) * kBuckets);
  L.cursor = c.take<unsigned long long>(static_cast<size_t>(segments) * kBuckets);
  L.bucket_begin = c.take<int64_t>(static_cast<size_t>(segments) * kBuckets);
  return L;
}

// One partition pass over the segments of L (already set up): histogram, scan, scatter.
int run_pass(const Level& L, int segments, int64_t n, const int32_t* kin, const int32_t* vin, int32_t* kout,
             int32_t* vout, DigitFn f, int32_t* err, cudaStream_t s) {
  if (cudaMemsetAsync(L.hist, 0, static_cast<size_t>(segments) * kBuckets * 4, s) != cudaSuccess) return CRYS_ECUDA;
  Segs S{L.seg_begin, L.seg_size, L.tile_start, L.tile_seg, segments};
  const int64_t grid = tiles_bound(n, segments, kPartTile);
  const int64_t hist_grid = grid < static_cast<int64_t>(sm_count()) * 8 ? grid : static_cast<int64_t>(sm_count()) * 8;
  part_hist_kernel<<<static_cast<unsigned>(hist_grid), kPartThreads, 0, s>>>(kin, S, f, L.hist);
  note_launch();
  part_scan_kernel<<<static_cast<unsigned>(segments), kBuckets, 0, s>>>(L.hist, L.seg_begin, L.cursor,
                                                                        L.bucket_begin);
  note_launch();
  ScatterArgs a{kin, vin, kout, vout, S, f, L.cursor, err};
  const size_t smem = static_cast<size_t>(kPartTile) * 8;
  if (!allow_smem(part_scatter_kernel, smem)) return CRYS_ECUDA;
  part_scatter_kernel<<<static_cast<unsigned>(grid), kPartThreads, smem, s>>>(a);
  note_launch();
  return check_launch();
}

bool no_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x + na <= y || y + nb <= x;
}

// Hash bits of the join's partitioning for a build side of nb rows: partitions of about
// 2048 rows (a 4096-slot table, a quarter of the shared-memory table), at most 16 bits in
// two passes of at most 8.
int join_bits(int64_t nb) {
  int bits = 0;
  while (bits < 16 && (nb >> bits) > 2048) ++bits;
  return bits;
}

}  // namespace
}  // namespace crys

extern "C" int crys_sort_msb(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out, int32_t* vals_out,
                             int64_t n, void* d_temp, size_t* temp_bytes, crys_stream stream) {
  using namespace crys;
  if (n < 0 || n > (1ll << 31) - 1) return CRYS_EINVAL;
  // scratch: a (key, value) buffer of n rows and the two levels' arrays
  auto layout = [&](void* base, int32_t** tk, int32_t** tv, Level* A, Level* B) {
    Carve c(base);
    *tk = c.take<int32_t>(static_cast<size_t>(n));
    *tv = c.take<int32_t>(static_cast<size_t>(n));
    *A = carve_level(c, 1, n);
    *B = carve_level(c, kBuckets, n);
    return c.off;
  };
  int32_t *tk, *tv;
  Level A, B;
  const size_t need = layout(nullptr, &tk, &tv, &A, &B);
  if (!d_temp && temp_bytes) {
    *temp_bytes = need;
    return CRYS_OK;
  }
  if (n == 0) return CRYS_OK;
  if (!d_temp || !temp_bytes) return CRYS_EINVAL;
  if (*temp_bytes < need) return CRYS_ENOMEM;
  if (!keys_in || !vals_in || !keys_out || !vals_out || (reinterpret_cast<uintptr_t>(d_temp) & 255u)) return CRYS_EINVAL;
  const size_t nb = static_cast<size_t>(n) * 4;
  if (!no_overlap(keys_out, nb, keys_in, nb) || !no_overlap(keys_out, nb, vals_in, nb) ||
      !no_overlap(vals_out, nb, keys_in, nb) || !no_overlap(vals_out, nb, vals_in, nb) ||
      !no_overlap(keys_out, nb, vals_out, nb))
    return CRYS_EINVAL;
  layout(d_temp, &tk, &tv, &A, &B);
  int32_t* err = device_error_word();
  if (!err) return CRYS_ECUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // level A: the whole array by the top digit (sign bit flipped), input -> output buffers
  seg_init_kernel<<<1, 1, 0, s>>>(n, kPartTile, A.seg_begin, A.seg_size, A.tile_start);
  note_launch();
  int rc = run_pass(A, 1, n, keys_in, vals_in, keys_out, vals_out, DigitFn{1u, 24u, 0xFFu, 0x80u}, err, s);
  if (rc != CRYS_OK) return rc;
  // level B: each of the 256 buckets by the next digit, output -> scratch buffers
  seg_from_buckets_kernel<<<1, 1024, 0, s>>>(A.bucket_begin, A.hist, kBuckets, kPartTile, B.seg_begin, B.seg_size,
                                             B.tile_start, B.tile_seg);
  note_launch();
  rc = run_pass(B, kBuckets, n, keys_out, vals_out, tk, tv, DigitFn{1u, 16u, 0xFFu, 0u}, err, s);
  if (rc != CRYS_OK) return rc;
  // every bucket of the top 16 bits sorted by the low 16 bits, scratch -> output
  LocalArgs L{tk, tv, keys_out, vals_out, B.bucket_begin, B.hist, err};
  if (!allow_smem(local_sort_kernel, kLocalSmem)) return CRYS_ECUDA;
  local_sort_kernel<<<kBuckets * kBuckets, kLocalThreads, kLocalSmem, s>>>(L);
  note_launch();
  return check_launch();
}

extern "C" int crys_join_partitioned(const int32_t* bkeys, const int32_t* bvals, int64_t nb, const int32_t* fk,
                                     const int32_t* payload, int64_t np, int64_t* d_sum, int64_t* d_matches,
                                     void* d_temp, size_t* temp_bytes, crys_stream stream) {
  using namespace crys;
  if (nb < 0 || np < 0 || nb > (1ll << 30) || np > (1ll << 31) - 1) return CRYS_EINVAL;
  const int bits = join_bits(nb);
  const int b1 = (bits + 1) / 2, b2 = bits / 2;
  const int parts1 = 1 << b1;
  // partition index space: bucket d of pass-2 segment g is partition g * 256 + d (digits
  // of a narrower pass leave the upper buckets empty)
  const int parts = bits == 0 ? 1 : (b2 == 0 ? kBuckets : parts1 * kBuckets);
  struct Side {
    int32_t *k1, *v1, *k2, *v2;  // rows after pass 1 and after pass 2
    Level A, B;
  };
  struct Parts {  // the partitions the join kernel reads
    int64_t* b_begin;
    uint32_t* b_count;
    int64_t* p_begin;
    int64_t* p_size;
    uint32_t* p_tiles;
    uint32_t* p_tile_seg;
    uint64_t* arena;
  };
  auto layout = [&](void* base, Side* R, Side* P, Parts* J) {
    Carve c(base);
    for (Side* sd : {R, P}) {
      const size_t rows = static_cast<size_t>(sd == R ? nb : np);
      sd->k1 = c.take<int32_t>(rows);
      sd->v1 = c.take<int32_t>(rows);
      sd->k2 = c.take<int32_t>(rows);
      sd->v2 = c.take<int32_t>(rows);
      sd->A = carve_level(c, 1, static_cast<int64_t>(rows));
      sd->B = carve_level(c, parts1, static_cast<int64_t>(rows));
    }
    J->b_begin = c.take<int64_t>(1);
    J->b_count = c.take<uint32_t>(1);
    J->p_begin = c.take<int64_t>(static_cast<size_t>(parts));
    J->p_size = c.take<int64_t>(static_cast<size_t>(parts));
    J->p_tiles = c.take<uint32_t>(static_cast<size_t>(parts) + 1);
    J->p_tile_seg = c.take<uint32_t>(static_cast<size_t>(tiles_bound(np, parts, kJoinTile)));
    J->arena = c.take<uint64_t>(static_cast<size_t>(4) * static_cast<size_t>(nb > 0 ? nb : 1));
    return c.off;
  };
  Side R, P;
  Parts J;
  const size_t need = layout(nullptr, &R, &P, &J);
  if (!d_temp && temp_bytes) {
    *temp_bytes = need;
    return CRYS_OK;
  }
  if (!d_sum) return CRYS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_sum, 0, 8, s) != cudaSuccess) return CRYS_ECUDA;
  if (d_matches && cudaMemsetAsync(d_matches, 0, 8, s) != cudaSuccess) return CRYS_ECUDA;
  if (nb == 0 || np == 0) return CRYS_OK;
  if (!d_temp || !temp_bytes) return CRYS_EINVAL;
  if (*temp_bytes < need) return CRYS_ENOMEM;
  if (!bkeys || !bvals || !fk || !payload || (reinterpret_cast<uintptr_t>(d_temp) & 255u)) return CRYS_EINVAL;
  layout(d_temp, &R, &P, &J);
  int32_t* err = device_error_word();
  if (!err) return CRYS_ECUDA;
  // both sides partitioned by the same hash bits: pass 1 by the top b1 bits, pass 2 by
  // the next b2 bits inside each pass-1 partition
  const DigitFn f1{2654435769u, static_cast<uint32_t>(32 - b1), static_cast<uint32_t>(parts1 - 1), 0u};
  const DigitFn f2{2654435769u, static_cast<uint32_t>(32 - bits), static_cast<uint32_t>((1 << b2) - 1), 0u};
  Side* sides[2] = {&R, &P};
  const int32_t* in_k[2] = {bkeys, fk};
  const int32_t* in_v[2] = {bvals, payload};
  const int64_t rows[2] = {nb, np};
  const int32_t* fin_k[2] = {bkeys, fk};
  const int32_t* fin_v[2] = {bvals, payload};
  const int64_t* fin_begin[2] = {nullptr, nullptr};
  const uint32_t* fin_count[2] = {nullptr, nullptr};
  for (int w = 0; w < 2 && bits > 0; ++w) {
    Side& sd = *sides[w];
    seg_init_kernel<<<1, 1, 0, s>>>(rows[w], kPartTile, sd.A.seg_begin, sd.A.seg_size, sd.A.tile_start);
    note_launch();
    int rc = run_pass(sd.A, 1, rows[w], in_k[w], in_v[w], sd.k1, sd.v1, f1, err, s);
    if (rc != CRYS_OK) return rc;
    fin_k[w] = sd.k1;
    fin_v[w] = sd.v1;
    fin_begin[w] = sd.A.bucket_begin;
    fin_count[w] = sd.A.hist;
    if (b2 == 0) continue;
    seg_from_buckets_kernel<<<1, 1024, 0, s>>>(sd.A.bucket_begin, sd.A.hist, parts1, kPartTile, sd.B.seg_begin,
                                               sd.B.seg_size, sd.B.tile_start, sd.B.tile_seg);
    note_launch();
    rc = run_pass(sd.B, parts1, rows[w], sd.k1, sd.v1, sd.k2, sd.v2, f2, err, s);
    if (rc != CRYS_OK) return rc;
    fin_k[w] = sd.k2;
    fin_v[w] = sd.v2;
    fin_begin[w] = sd.B.bucket_begin;
    fin_count[w] = sd.B.hist;
  }
  const int64_t* b_begin = fin_begin[0];
  const uint32_t* b_count = fin_count[0];
  if (bits == 0) {  // one partition: the inputs as they are
    one_partition_kernel<<<1, 1, 0, s>>>(nb, np, kJoinTile, J.b_begin, J.b_count, J.p_begin, J.p_size, J.p_tiles);
    note_launch();
    b_begin = J.b_begin;
    b_count = J.b_count;
  } else {
    seg_from_buckets_kernel<<<1, 1024, 0, s>>>(fin_begin[1], fin_count[1], parts, kJoinTile, J.p_begin, J.p_size,
                                               J.p_tiles, J.p_tile_seg);
    note_launch();
  }
  JoinArgs a;
  a.bkey = fin_k[0];
  a.bval = fin_v[0];
  a.b_begin = b_begin;
  a.b_count = b_count;
  a.pkey = fin_k[1];
  a.ppay = fin_v[1];
  a.probe = Segs{J.p_begin, J.p_size, J.p_tiles, J.p_tile_seg, parts};
  a.arena = J.arena;
  a.sum = reinterpret_cast<unsigned long long*>(d_sum);
  a.matches = reinterpret_cast<unsigned long long*>(d_matches);
  a.err = err;
  join_build_large_kernel<<<static_cast<unsigned>(parts), kJoinThreads, 0, s>>>(a, parts);
  note_launch();
  const size_t smem = static_cast<size_t>(kJoinSlots) * 8;
  if (!allow_smem(join_partition_kernel, smem)) return CRYS_ECUDA;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(join_partition_kernel), kJoinThreads, smem);
  int64_t grid = tiles_bound(np, parts, kJoinTile);
  if (grid > static_cast<int64_t>(per_sm) * sm_count()) grid = static_cast<int64_t>(per_sm) * sm_count();
  join_partition_kernel<<<static_cast<unsigned>(grid), kJoinThreads, smem, s>>>(a);
  note_launch();
  return check_launch();
}
