// Least-significant-digit radix sort of (key, value) pairs (Section 4.4): 8-bit digits,
// four stable radix-partition passes from the low digit to the high digit.
//
// The paper's passes each run a histogram phase and a shuffle phase; here
//  * one up-front kernel reads the keys once and histograms all four digits (the
//    global start of every digit bucket of every pass, after a 256-wide scan), and
//  * each pass is ONE kernel: a thread block takes the next tile id from an atomic
//    counter, ranks its keys stably inside the block (per-warp multisplit with
//    ballots: keys are processed warp-striped, round by round, so rank order equals
//    input order), publishes its per-digit counts and finds the counts of all earlier tiles
//    with a decoupled look-back, then writes keys and values through shared memory in
//    sorted order so that each digit's run is stored with consecutive addresses.
// So the data crosses HBM once per pass (read 8N, write 8N) plus one 4N key read.
//
// The paper notes that its V100 kernels could partition only 7 bits per stable pass
// because each thread kept a 2^r histogram in registers; the per-warp shared-memory
// multisplit used here keeps 8-bit stable passes.  Signed order: the top digit has its
// sign bit flipped.
#include <type_traits>

#include "common.cuh"
#include "pipeline.cuh"
#include "tiles.h"

namespace crys {
namespace {

constexpr int kRadix = 256;
constexpr int kPasses = 4;
constexpr uint32_t kFlagAggregate = 1u << 30;
constexpr uint32_t kFlagInclusive = 2u << 30;
constexpr uint32_t kValueMask = (1u << 30) - 1;

__device__ __forceinline__ uint32_t digit_of(int32_t key, int pass) {
  const uint32_t d = (static_cast<uint32_t>(key) >> (8 * pass)) & 0xFFu;
  return pass == kPasses - 1 ? d ^ 0x80u : d;
}

// ---------------------------------------------------------------- histogram

constexpr int kHistThreads = 512;
constexpr int kHistCopies = 4;  // shared-memory copies of the 4x256 histogram

__global__ void __launch_bounds__(kHistThreads) sort_hist_kernel(const int32_t* __restrict__ keys,
                                                                  int64_t n, unsigned int* hist) {
  __shared__ unsigned int h[kHistCopies][kPasses * kRadix];
  for (int i = threadIdx.x; i < kHistCopies * kPasses * kRadix; i += kHistThreads)
    (&h[0][0])[i] = 0;
  __syncthreads();
  unsigned int* mine = h[(threadIdx.x / kWarp) % kHistCopies];
  const uint64_t pol = policy_evict_first();
  const int64_t nvec = n / 4;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * kHistThreads;
  for (int64_t v = static_cast<int64_t>(blockIdx.x) * kHistThreads + threadIdx.x; v < nvec; v += stride) {
    const int4 q = ld_stream_v4(keys + 4 * v, pol);
    const int32_t k4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int p = 0; p < kPasses; ++p) atomicAdd(&mine[p * kRadix + digit_of(k4[e], p)], 1u);
  }
  if (blockIdx.x == 0) {
    for (int64_t i = 4 * nvec + threadIdx.x; i < n; i += kHistThreads) {
      const int32_t k = keys[i];
#pragma unroll
      for (int p = 0; p < kPasses; ++p) atomicAdd(&mine[p * kRadix + digit_of(k, p)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPasses * kRadix; i += kHistThreads) {
    unsigned int c = 0;
#pragma unroll
    for (int r = 0; r < kHistCopies; ++r) c += h[r][i];
    if (c) atomicAdd(hist + i, c);
  }
}

// Exclusive scan of each pass's 256 digit counts: warp p scans pass p.
__global__ void sort_scan_kernel(const unsigned int* hist, unsigned int* base) {
  const int lane = threadIdx.x % kWarp, pass = threadIdx.x / kWarp;
  if (pass >= kPasses) return;
  unsigned int carry = 0;
  for (int c0 = 0; c0 < kRadix; c0 += kWarp) {
    const unsigned int x = hist[pass * kRadix + c0 + lane];
    const unsigned int inc = static_cast<unsigned int>(warp_inclusive_scan(static_cast<int32_t>(x), lane));
    base[pass * kRadix + c0 + lane] = carry + inc - x;
    carry += __shfl_sync(0xFFFFFFFFu, inc, kWarp - 1);
  }
}

// ---------------------------------------------------------------- one pass

struct PassArgs {
  const int32_t* keys_in;
  const int32_t* vals_in;
  int32_t* keys_out;
  int32_t* vals_out;
  int64_t n;
  int pass;
  const unsigned int* digit_base;  // 256 bucket starts of this pass
  uint32_t* status;                // per tile x digit look-back words
  unsigned int* tile_counter;
  unsigned int* abort_word;        // set by the first block of this sort that gives up
  uint32_t tile_base;              // first tile id handed out (0 unless a test stalls)
  uint64_t wait_ns;                // bound of a look-back wait
  int32_t* err;
};

template <int THREADS, int ITEMS, int PASS>
__global__ void __launch_bounds__(THREADS) sort_pass_kernel(PassArgs a) {
  constexpr int WARPS = THREADS / kWarp;
  constexpr int TILE = THREADS * ITEMS;
  constexpr int WSEG = kWarp * ITEMS;
  static_assert(THREADS >= kRadix, "one thread per digit");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int32_t* skeys = reinterpret_cast<int32_t*>(smem_raw);  // tile keys: input order, then sorted
  int32_t* svals = skeys + TILE;                           // tile values: input order, then sorted
  __shared__ unsigned int whist[WARPS][kRadix];  // per-warp digit counts, then offsets
  __shared__ unsigned int tile_start[kRadix];    // tile-local start of each digit run
  __shared__ int32_t out_shift[kRadix];          // global position minus local position
  __shared__ unsigned int scan_tmp[kRadix / kWarp];
  __shared__ unsigned int tile_sh;
  __shared__ __align__(8) uint64_t loaded;

  const int tid = threadIdx.x, lane = tid % kWarp, warp = tid / kWarp;
  if (tid == 0) {
    // a sort whose earlier pass gave up does no further work (tile id past the end)
    tile_sh = ld_relaxed_u32(a.abort_word) ? 0xFFFFFFFFu : a.tile_base + atomicAdd(a.tile_counter, 1u);
    mbar_init(&loaded, 1);
    fence_barrier_init();
  }
  for (int i = tid; i < WARPS * kRadix; i += THREADS) (&whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = tile_sh;
  if (tile * TILE >= a.n) return;  // nothing issued on the barrier yet
  const int64_t tile_row = tile * TILE;
  const int valid = static_cast<int>((a.n - tile_row) < TILE ? (a.n - tile_row) : TILE);
  const int bulk = valid & ~3;
  // BlockLoad: keys and values of the tile, one bulk copy each.
  if (tid == 0) {
    const uint64_t pol = policy_evict_first();
    const uint32_t bytes = static_cast<uint32_t>(bulk) * 4u;
    mbar_arrive_expect_tx(&loaded, 2 * bytes);
    if (bytes) {
      bulk_load(skeys, a.keys_in + tile_row, bytes, &loaded, pol);
      bulk_load(svals, a.vals_in + tile_row, bytes, &loaded, pol);
    }
  }
  if (bulk < valid) {  // ragged end of the last tile
    for (int i = bulk + tid; i < valid; i += THREADS) {
      skeys[i] = a.keys_in[tile_row + i];
      svals[i] = a.vals_in[tile_row + i];
    }
  }
  const bool ok = mbar_wait_bounded(&loaded, 0, a.err);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) mbar_wait_bounded(&loaded, 0, a.err);
    return;
  }

  // Stable per-warp ranking, warp-striped: item i of lane l in warp w is tile position
  // w*32*ITEMS + i*32 + l.  In round i the lanes holding the same digit are found with
  // 8 ballots (one per digit bit); each gets (keys of that digit in earlier rounds) +
  // (same-digit lanes below it).  Rows past the end take part in no group.
  const uint32_t lt_mask = (1u << lane) - 1u;
  int32_t key[ITEMS];
  uint32_t rank[ITEMS];
  // a full tile (all but possibly the last) ranks without per-item bounds predicates
  auto rank_items = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
      const int pos = warp * WSEG + i * kWarp + lane;
      const bool real = FULL || pos < valid;
      key[i] = real ? skeys[pos] : 0;
      const uint32_t d = real ? digit_of(key[i], PASS) : 0u;
      uint32_t peers = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, real);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t vote = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? vote : ~vote;
      }
      uint32_t before = 0;
      if (real) before = whist[warp][d];
      __syncwarp();
      rank[i] = before + __popc(peers & lt_mask);
      if (real && (peers & lt_mask) == 0) whist[warp][d] = before + __popc(peers);
      __syncwarp();
    }
  };
  if (valid == TILE)
    rank_items(std::true_type{});
  else
    rank_items(std::false_type{});
  __syncthreads();

  // Per digit: exclusive offsets of the warps and the tile's count.
  unsigned int count = 0;
  if (tid < kRadix) {
#pragma unroll
    for (int w = 0; w < WARPS; ++w) {
      const unsigned int c = whist[w][tid];
      whist[w][tid] = count;
      count += c;
    }
    // Tile-local exclusive scan across digits (threads 0..255 = 8 warps).
    const unsigned int inc = static_cast<unsigned int>(warp_inclusive_scan(static_cast<int32_t>(count), lane));
    if (lane == kWarp - 1) scan_tmp[warp] = inc;
    tile_start[tid] = inc - count;
  }
  __syncthreads();
  bool failed = false;
  if (tid < kRadix) {
    unsigned int wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += scan_tmp[w];
    tile_start[tid] += wbase;
    // Decoupled look-back for digit tid over the earlier tiles.
    uint32_t* st = a.status + tile * kRadix + tid;
    unsigned int excl = 0;
    if (tile == 0) {
      st_relaxed_u32(st, kFlagInclusive | count);
    } else {
      st_relaxed_u32(st, kFlagAggregate | count);
      int64_t p = tile - 1;
      uint64_t t0 = 0;
      bool timing = false;
      while (p >= 0) {
        const uint32_t w = ld_relaxed_u32(a.status + p * kRadix + tid);
        const uint32_t flag = w >> 30;
        if (flag == 0) {
          if (!timing) {
            t0 = global_timer_ns();
            timing = true;
          } else if (global_timer_ns() - t0 > a.wait_ns) {
            set_error(a.err, CRYS_DEV_TIMEOUT);
            st_relaxed_u32(a.abort_word, 1u);
            failed = true;
            break;
          }
          if (ld_relaxed_u32(a.abort_word)) {  // another block of this sort gave up
            failed = true;
            break;
          }
          continue;
        }
        timing = false;
        excl += w & kValueMask;
        if (flag == 2) break;
        --p;
      }
      if (!failed) st_relaxed_u32(st, kFlagInclusive | (excl + count));
    }
    out_shift[tid] = static_cast<int32_t>(a.digit_base[tid] + excl - tile_start[tid]);
    // the digit's run [start, start + count) of this tile must land inside the output
    const int64_t start = static_cast<int64_t>(a.digit_base[tid]) + excl;
    if (!failed && count && (start < 0 || start + count > a.n)) {
      set_error(a.err, CRYS_DEV_BOUNDS);
      failed = true;
    }
  }
  if (__syncthreads_or(failed)) return;

  // BlockShuffle in place: keys to their sorted positions (every key of the tile is in
  // some thread's registers), then values (read first, written after a barrier).
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int pos = warp * WSEG + i * kWarp + lane;
    if (pos < valid) {
      const uint32_t d = digit_of(key[i], PASS);
      rank[i] += tile_start[d] + whist[warp][d];
      skeys[rank[i]] = key[i];
    }
  }
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int pos = warp * WSEG + i * kWarp + lane;
    key[i] = pos < valid ? svals[pos] : 0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < ITEMS; ++i) {
    const int pos = warp * WSEG + i * kWarp + lane;
    if (pos < valid) svals[rank[i]] = key[i];
  }
  __syncthreads();
  // BlockStore in sorted order: each digit run is written with consecutive addresses.
  for (int i = tid; i < valid; i += THREADS) {
    const int32_t k = skeys[i];
    const int64_t g = static_cast<int64_t>(out_shift[digit_of(k, PASS)]) + i;  // checked per digit above
    a.keys_out[g] = k;
    a.vals_out[g] = svals[i];
  }
}

struct Layout {
  size_t tmp_keys, tmp_vals, hist, base, counters, status, total;
  int64_t tiles;
};

size_t up256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

int64_t min_tile() {
  int64_t m = INT64_MAX;
  for (int i = 0; i < kNumVariants[CRYS_OP_SORT]; ++i) {
    const int64_t t = static_cast<int64_t>(kTiles[CRYS_OP_SORT][i].threads) * kTiles[CRYS_OP_SORT][i].items;
    if (t < m) m = t;
  }
  return m;
}

Layout layout(int64_t n) {
  Layout L;
  L.tiles = (n + min_tile() - 1) / min_tile();
  size_t off = 0;
  L.tmp_keys = off;
  off += up256(static_cast<size_t>(n) * 4);
  L.tmp_vals = off;
  off += up256(static_cast<size_t>(n) * 4);
  L.hist = off;
  off += up256(kPasses * kRadix * 4);
  L.base = off;
  off += up256(kPasses * kRadix * 4);
  L.counters = off;
  off += 256;
  L.status = off;
  off += up256(static_cast<size_t>(L.tiles) * kRadix * 4);
  L.total = off;
  return L;
}

template <int THREADS, int ITEMS>
int run_passes(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out, int32_t* vals_out,
               int64_t n, char* temp, const Layout& L, cudaStream_t s) {
  constexpr int TILE = THREADS * ITEMS;
  const int64_t tiles = (n + TILE - 1) / TILE;
  const size_t smem = static_cast<size_t>(TILE) * 8;
  using Kernel = void (*)(PassArgs);
  const Kernel kernels[kPasses] = {sort_pass_kernel<THREADS, ITEMS, 0>, sort_pass_kernel<THREADS, ITEMS, 1>,
                                   sort_pass_kernel<THREADS, ITEMS, 2>, sort_pass_kernel<THREADS, ITEMS, 3>};
  for (int p = 0; p < kPasses; ++p)
    if (!allow_smem(kernels[p], smem)) return CRYS_ECUDA;
  int32_t* tk = reinterpret_cast<int32_t*>(temp + L.tmp_keys);
  int32_t* tv = reinterpret_cast<int32_t*>(temp + L.tmp_vals);
  const int32_t* src_k[kPasses] = {keys_in, tk, keys_out, tk};
  const int32_t* src_v[kPasses] = {vals_in, tv, vals_out, tv};
  int32_t* dst_k[kPasses] = {tk, keys_out, tk, keys_out};
  int32_t* dst_v[kPasses] = {tv, vals_out, tv, vals_out};
  PassArgs a;
  a.n = n;
  a.status = reinterpret_cast<uint32_t*>(temp + L.status);
  a.abort_word = reinterpret_cast<unsigned int*>(temp + L.counters) + kPasses;
  a.err = device_error_word();
  if (!a.err) return CRYS_ECUDA;
  uint32_t stall_base = 0;
  uint64_t stall_ns = kWaitBoundNs;
  take_stall(CRYS_OP_SORT, &stall_base, &stall_ns);  // a test's stall applies to the first pass
  for (int p = 0; p < kPasses; ++p) {
    a.tile_base = p == 0 ? stall_base : 0u;
    a.wait_ns = p == 0 ? stall_ns : kWaitBoundNs;
    a.keys_in = src_k[p];
    a.vals_in = src_v[p];
    a.keys_out = dst_k[p];
    a.vals_out = dst_v[p];
    a.pass = p;
    a.digit_base = reinterpret_cast<unsigned int*>(temp + L.base) + p * kRadix;
    a.tile_counter = reinterpret_cast<unsigned int*>(temp + L.counters) + p;
    if (cudaMemsetAsync(a.status, 0, static_cast<size_t>(tiles) * kRadix * 4, s) != cudaSuccess)
      return CRYS_ECUDA;
    kernels[p]<<<static_cast<unsigned int>(tiles), THREADS, smem, s>>>(a);
    note_launch();
    if (check_launch() != CRYS_OK) return CRYS_ECUDA;
  }
  return CRYS_OK;
}

constexpr int kOp = CRYS_OP_SORT;

}  // namespace
}  // namespace crys

extern "C" int crys_sort(const int32_t* keys_in, const int32_t* vals_in, int32_t* keys_out,
                         int32_t* vals_out, int64_t n, void* d_temp, size_t* temp_bytes,
                         crys_stream stream) {
  using namespace crys;
  if (n < 0 || n > static_cast<int64_t>(kValueMask)) return CRYS_EINVAL;
  const Layout L = layout(n);
  if (!d_temp && temp_bytes) {
    *temp_bytes = L.total;
    return CRYS_OK;
  }
  if (n == 0) return CRYS_OK;
  if (!d_temp || !temp_bytes) return CRYS_EINVAL;
  if (*temp_bytes < L.total) return CRYS_ENOMEM;
  if (!keys_in || !vals_in || !keys_out || !vals_out || !aligned16(keys_in) || !aligned16(vals_in) ||
      !aligned16(keys_out) || !aligned16(vals_out))
    return CRYS_EINVAL;
  if (reinterpret_cast<uintptr_t>(d_temp) & 255u) return CRYS_EINVAL;
  auto overlaps = [n](const void* a, const void* b) {
    const char* x = static_cast<const char*>(a);
    const char* y = static_cast<const char*>(b);
    return x < y + n * 4 && y < x + n * 4;
  };
  if (overlaps(keys_out, keys_in) || overlaps(keys_out, vals_in) || overlaps(vals_out, keys_in) ||
      overlaps(vals_out, vals_in) || overlaps(keys_out, vals_out))
    return CRYS_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* temp = static_cast<char*>(d_temp);
  if (cudaMemsetAsync(temp + L.hist, 0, L.status - L.hist, s) != cudaSuccess) return CRYS_ECUDA;
  const int hist_grid = sm_count() * 4;
  sort_hist_kernel<<<hist_grid, kHistThreads, 0, s>>>(keys_in, n, reinterpret_cast<unsigned int*>(temp + L.hist));
  note_launch();
  sort_scan_kernel<<<1, kPasses * kWarp, 0, s>>>(reinterpret_cast<unsigned int*>(temp + L.hist),
                                                 reinterpret_cast<unsigned int*>(temp + L.base));
  note_launch();
  if (check_launch() != CRYS_OK) return CRYS_ECUDA;
  switch (tile_variant(kOp)) {
    case 1: return run_passes<kTiles[kOp][1].threads, kTiles[kOp][1].items>(keys_in, vals_in, keys_out, vals_out, n, temp, L, s);
    case 2: return run_passes<kTiles[kOp][2].threads, kTiles[kOp][2].items>(keys_in, vals_in, keys_out, vals_out, n, temp, L, s);
    case 3: return run_passes<kTiles[kOp][3].threads, kTiles[kOp][3].items>(keys_in, vals_in, keys_out, vals_out, n, temp, L, s);
    default: return run_passes<kTiles[kOp][0].threads, kTiles[kOp][0].items>(keys_in, vals_in, keys_out, vals_out, n, temp, L, s);
  }
}
