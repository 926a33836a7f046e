// Binning of projected Gaussians into screen tiles (the 3D GS tile scheme the
// paper builds on, Sec. 4.1.1), with an own stable LSD radix sort.
//
// Plan (all counts stay on the device, nothing is read back):
//   1. compact the visible entries -> (depth key, entry) lists;
//   2. sort them by depth key (4 passes of 8 bits; stable, so equal depths keep
//      entry order);
//   3. exclusive scan of tiles_touched in depth order -> pair offsets and the
//      pair count (checked against the capacity);
//   4. emit one (tile, entry) pair per overlapped tile, in depth order;
//   5. stable sort of the pairs by tile id (ceil(log2 T)/8 passes): every tile's
//      list is then in (depth, entry) order, the same order as a full sort on
//      (tile, depth bits, entry) keys;
//   6. [start, end) of each tile.
// The radix sort is one-sweep: the kernel that writes the keys (compaction,
// emission) also counts the digits of every pass, then one kernel per pass
// whose blocks chain their digit offsets by decoupled look-back (bounded waits).
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ inline unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr int kMaxPasses = 4;

// Digit histograms of the radix sort's passes, accumulated by the kernel that
// writes the keys: h[pass][digit] in shared memory, then added to the global
// histograms.  Warp-collective (all 32 lanes call it).  From pass `tested` on
// (the high digits) a digit shared by all of the warp's valid keys costs one
// atomic; the lower digits are spread out and go straight to the atomics.
__device__ inline void hist_keys(uint32_t (*h)[kRadix], int passes, uint32_t key, bool valid, int tested) {
  const unsigned vm = __ballot_sync(FULL, valid);
  if (vm == 0) return;
  const int leader = __ffs(vm) - 1;
#pragma unroll
  for (int p = 0; p < kMaxPasses; ++p) {
    if (p >= passes) break;
    const int d = (int)((key >> (kRadixBits * p)) & (kRadix - 1));
    if (p < tested) {
      if (valid) atomicAdd(&h[p][d], 1u);
      continue;
    }
    const int d0 = __shfl_sync(FULL, d, leader);
    if (__all_sync(FULL, !valid || d == d0)) {
      if ((int)(threadIdx.x & 31) == leader) atomicAdd(&h[p][d0], (uint32_t)__popc(vm));
    } else if (valid) {
      atomicAdd(&h[p][d], 1u);
    }
  }
}

__device__ inline void hist_flush(uint32_t (*h)[kRadix], int passes, uint32_t* __restrict__ ghist) {
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t c = (&h[0][0])[i];
    if (c) atomicAdd(ghist + i, c);
  }
}

// Block-wide exclusive scan of one uint32 per thread (256 threads).
__device__ inline uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
    uint32_t s = t;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = s - t;
    if (lane == 31) s_warp[32] = s;
  }
  __syncthreads();
  uint32_t r = x - v + s_warp[w];
  if (total) *total = s_warp[32];
  __syncthreads();
  return r;
}

// In-block ordered scan helper: each warp owns 512 consecutive items
// (16 rounds of 32), so item order = (warp, round, lane).
struct WarpItems {
  static __device__ inline int64_t index(int64_t base, int r) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    return base + (int64_t)w * (32 * kSortItems) + r * 32 + lane;
  }
};

// ---------------------------------------------------------------------------
// Decoupled look-back.  A block publishes one 64-bit word per value: its own
// total flagged A as soon as it is known, then the inclusive prefix flagged P;
// a successor adds A words going back until it meets a P.  Blocks take their
// index from a ticket counter in the order they start, so a block only ever
// waits for blocks that are already running; every wait is bounded and sets
// GS_ERR_TIMEOUT if it runs out.
// ---------------------------------------------------------------------------
constexpr unsigned long long kFlagA = 1ull << 62, kFlagP = 2ull << 62, kFlagMask = 3ull << 62;
constexpr int kSpinLimit = 1 << 22;

__device__ inline void st_relaxed(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ inline unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The block's ticket (thread 0 draws it; every thread gets it).
__device__ inline int block_ticket(int* ticket, int* s_tk) {
  if (threadIdx.x == 0) *s_tk = atomicAdd(ticket, 1);
  __syncthreads();
  return *s_tk;
}

// Exclusive prefix over the blocks before blk of their totals (agg: this
// block's total, as seen by warp 0).  Called by every thread of the block;
// warp 0 reads the words of 32 predecessors at a time (lane l: block j - l)
// and adds them up to the nearest P.
__device__ inline unsigned long long block_lookback(unsigned long long* words, int blk, unsigned long long agg,
                                                    Header* hdr, unsigned long long* s_excl,
                                                    int spin_limit = kSpinLimit) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned long long* mine = words + blk;
    if (lane == 0) st_relaxed(mine, (blk == 0 ? kFlagP : kFlagA) | agg);
    unsigned long long excl = 0;
    int j = blk - 1, spins = 0;
    while (j >= 0) {
      const int q = j - lane;
      // before block 0: a zero inclusive prefix (never consumed: block 0 always publishes P)
      const unsigned long long f = q >= 0 ? ld_relaxed(words + q) : kFlagP;
      const unsigned long long st = f & kFlagMask;
      const unsigned pm = __ballot_sync(FULL, st == kFlagP), zm = __ballot_sync(FULL, st == 0);
      const int last = pm ? __ffs(pm) - 1 : 31;                  // lanes 0..last are needed
      const unsigned need = last == 31 ? FULL : (2u << last) - 1u;
      if (zm & need) {                                           // one of them is not published yet
        if (++spins > spin_limit) {
          if (lane == 0) set_status(hdr, GS_ERR_TIMEOUT);
          break;
        }
        continue;
      }
      unsigned long long c = lane <= last ? (f & ~kFlagMask) : 0ull;
      for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
      excl += c;
      if (pm) break;
      j -= 32;
    }
    if (lane == 0) {
      if (blk > 0) st_relaxed(mine, kFlagP | (excl + agg));
      *s_excl = excl;
    }
  }
  __syncthreads();
  return *s_excl;
}

// Test hook for the bounded waits: one block runs the look-back as block 1 of a
// scan whose block 0 never publishes its word, so the wait runs out after
// spin_limit polls, sets GS_ERR_TIMEOUT and the kernel returns.
__global__ void k_wait_timeout(unsigned long long* words, int spin_limit, Header* hdr) {
  __shared__ unsigned long long s_excl;
  if (threadIdx.x < 2) words[threadIdx.x] = 0ull;
  __syncthreads();
  block_lookback(words, 1, 1ull, hdr, &s_excl, spin_limit);
}

cudaError_t launch_wait_timeout(void* ws, const Layout& L, int spin_limit, cudaStream_t s) {
  k_wait_timeout<<<1, 32, 0, s>>>(at<unsigned long long>(ws, L.scanaux + 64), spin_limit, at<Header>(ws, L.hdr));
  return cudaGetLastError();
}

// Compaction of visible entries: (key, entry) at their rank among visible
// ones, in one pass (block offsets by look-back); the last block writes the
// visible count.  Also counts the depth keys' digits for the sort.
__global__ void __launch_bounds__(kSortThreads)
k_compact(const uint32_t* __restrict__ key, int64_t E, uint32_t* __restrict__ okey, uint32_t* __restrict__ oval,
          uint32_t* __restrict__ ghist, unsigned long long* __restrict__ words, int* ticket,
          unsigned long long* __restrict__ n_vis_out, Header* hdr) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_wtot[8];
  __shared__ uint32_t s_h[kMaxPasses][kRadix];   // the depth sort's digit histograms
  __shared__ int s_tk;
  __shared__ unsigned long long s_excl;
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  const int blk = block_ticket(ticket, &s_tk);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blk * kSortTile;
  uint32_t k[kSortItems];
  uint32_t wsum = 0;
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = WarpItems::index(base, r);
    k[r] = i < E ? key[i] : kInvalidKey;
    wsum += __popc(__ballot_sync(FULL, k[r] != kInvalidKey));
  }
  if (lane == 0) s_wtot[w] = wsum;
  __syncthreads();
  uint32_t tot = 0, before = 0;
  for (int i = 0; i < 8; ++i) {
    before += i < w ? s_wtot[i] : 0u;
    tot += s_wtot[i];
  }
  const unsigned long long excl = block_lookback(words, blk, tot, hdr, &s_excl);
  if (threadIdx.x == 0 && base + kSortTile >= E) *n_vis_out = excl + tot;   // the last block
  uint32_t off = (uint32_t)excl + before;
  for (int r = 0; r < kSortItems; ++r) {
    const bool v = k[r] != kInvalidKey;
    const unsigned bal = __ballot_sync(FULL, v);
    if (v) {
      uint32_t pos = off + __popc(bal & lanemask_lt());
      okey[pos] = k[r];
      oval[pos] = (uint32_t)WarpItems::index(base, r);
    }
    off += __popc(bal);
    hist_keys(s_h, kMaxPasses, k[r], v, kMaxPasses - 1);
  }
  hist_flush(s_h, kMaxPasses, ghist);
}

// Exclusive scan of tiles_touched in depth order, in one pass: pair_off[k] is
// the first pair of the k-th nearest visible entry.  The block holding the
// last entry writes the pair count and checks it against the capacity.
__global__ void __launch_bounds__(kSortThreads)
k_pair_offsets(const uint32_t* __restrict__ sval, const unsigned long long* n_vis_ptr, int64_t E,
               const uint32_t* __restrict__ touched, uint32_t* __restrict__ pair_off,
               uint32_t* __restrict__ chunk_first, int64_t n_chunks, unsigned long long* __restrict__ words,
               int* ticket, unsigned long long* __restrict__ n_pairs_out, int64_t cap, Header* hdr) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_wtot[8];
  __shared__ int s_tk;
  __shared__ unsigned long long s_excl;
  const int blk = block_ticket(ticket, &s_tk);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t n = clamp_count(n_vis_ptr, E);
  const int64_t base = (int64_t)blk * kSortTile;
  if (base >= n) {   // so do all later tickets: nobody waits for this block
    if (blk == 0 && threadIdx.x == 0) *n_pairs_out = 0;   // no visible entry
    return;
  }
  uint32_t cnt[kSortItems];
  uint32_t wsum = 0;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t i = WarpItems::index(base, r);
    cnt[r] = i < n ? __ldg(touched + __ldg(sval + i)) & kTouchedMask : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    uint32_t x = cnt[r];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    wsum += x;
  }
  if (lane == 0) s_wtot[w] = wsum;
  __syncthreads();
  uint32_t tot = 0, before = 0;
  for (int i = 0; i < 8; ++i) {
    before += i < w ? s_wtot[i] : 0u;
    tot += s_wtot[i];
  }
  const unsigned long long excl = block_lookback(words, blk, tot, hdr, &s_excl);
  if (threadIdx.x == 0 && base + kSortTile >= n) {   // the block holding the last entry
    *n_pairs_out = excl + tot;
    if (cap > 0 && excl + tot > (unsigned long long)cap) set_status(hdr, GS_ERR_CAPACITY);
  }
  uint32_t off = (uint32_t)excl + before;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    uint32_t x = cnt[r];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    const int64_t i = WarpItems::index(base, r);
    if (i < n) {
      const uint32_t o = off + x - cnt[r];
      pair_off[i] = o;
      // the entry that holds the first pair of every emission chunk starting in it
      const int64_t qe = ((int64_t)o + cnt[r] - 1) / kEmitChunk;
      for (int64_t q = ((int64_t)o + kEmitChunk - 1) / kEmitChunk; cnt[r] && q <= qe && q < n_chunks; ++q)
        chunk_first[q] = (uint32_t)i;
    }
    off += __shfl_sync(FULL, x, 31);
  }
}

// Last k in [0, n) with off[k] <= p (off is non-decreasing, off[0] = 0).
__device__ inline int64_t last_le(const uint32_t* off, int64_t n, uint32_t p) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Emission of (tile, entry) pairs in depth order, load-balanced over the whole
// grid: block slice c writes pairs [c * kEmitChunk, (c + 1) * kEmitChunk).  The
// pair-offset kernel records the entry holding each slice's first pair, which
// gives the slice's entry range (at most one entry per pair, so it fits in
// shared memory; only a slice cut short by the capacity searches pair_off);
// each thread then finds the entry of each of its pairs by a short search there.  Stores are contiguous
// and a splat covering hundreds of tiles is shared by many threads.

__global__ void __launch_bounds__(kSortThreads)
k_emit(const FrameDev* __restrict__ fd, const uint32_t* __restrict__ sval,
       const unsigned long long* n_vis_ptr, const unsigned long long* n_pairs_ptr, int64_t E,
       const short4* __restrict__ rect, const uint32_t* __restrict__ pair_off, int64_t cap,
       uint32_t* __restrict__ ptile, uint32_t* __restrict__ pval, const uint32_t* __restrict__ chunk_first,
       int64_t n_chunks, int tile_passes, uint32_t* __restrict__ ghist, int64_t T, Header* hdr) {
  pdl_wait();
  pdl_trigger();
  // per entry of the slice: its first pair, and (entry, first tile of its
  // rectangle, rectangle width | tile row length << 16, 1 / width)
  __shared__ uint32_t s_off[kEmitChunk + 1];
  __shared__ uint4 s_ent[kEmitChunk + 1];
  __shared__ uint4 s_idx[kEmitChunk / 8];   // per pair: its entry's slot in s_off (uint16, 8 per piece)
  __shared__ int64_t s_k[2];
  __shared__ uint32_t s_h[kMaxPasses][kRadix];   // the tile sort's digit histograms
  static_assert(kEmitChunk == 8 * kSortThreads, "one 8-pair run per thread");
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_h[0][0])[i] = 0;
  const int64_t n = clamp_count(n_vis_ptr, E);
  const int64_t P = clamp_count(n_pairs_ptr, cap);
  const int nv = fd->n_views;
  const int sx = fd->tile_shift_x, sy = fd->tile_shift_y;
  const int tiles_x0 = fd->views[0].tiles_x;
  for (int64_t p0 = (int64_t)blockIdx.x * kEmitChunk; p0 < P; p0 += (int64_t)gridDim.x * kEmitChunk) {
    const int64_t p1 = min(P, p0 + kEmitChunk);
    __syncthreads();
    if (threadIdx.x == 0) {   // entries holding pairs p0 and p1 - 1 (every entry holds >= 1 pair)
      const int64_t q = p0 / kEmitChunk;
      s_k[0] = chunk_first[q];
      if (p1 < P && q + 1 < n_chunks) {   // pair p1 exists, so its entry is in the table
        const uint32_t e1 = chunk_first[q + 1];
        s_k[1] = __ldg(pair_off + e1) == (uint32_t)p1 ? (int64_t)e1 - 1 : (int64_t)e1;
      } else {
        s_k[1] = last_le(pair_off, n, (uint32_t)(p1 - 1));
      }
    }
    __syncthreads();
    const int64_t k0 = s_k[0];
    const int m = (int)(s_k[1] - k0 + 1);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const uint32_t e = __ldg(sval + k0 + i);
      s_off[i] = __ldg(pair_off + k0 + i);
      const short4 rc = rect[e];
      int rowlen = tiles_x0, toff = 0;
      if (nv > 1) {
        const int vi = find_view(fd->entry_off, nv, (int64_t)e);
        rowlen = fd->views[vi].tiles_x;
        toff = fd->tile_off[vi];
      }
      const int tx0 = rc.x >> sx, ty0 = rc.z >> sy;
      const uint32_t nx = (uint32_t)((rc.y >> sx) - tx0 + 1);
      s_ent[i] = make_uint4(e, (uint32_t)(toff + ty0 * rowlen + tx0), nx | ((uint32_t)rowlen << 16),
                            __float_as_uint(__frcp_rn((float)nx)));
    }
    __syncthreads();
    // each thread finds the entry of its first of 8 consecutive pairs by
    // binary search and walks forward for the other 7
    {
      const uint32_t q0 = (uint32_t)(p0 + 8 * threadIdx.x);
      const int64_t left = p1 - (int64_t)q0;
      const int np = left < 8 ? (int)left : 8;
      uint32_t w[4] = {0u, 0u, 0u, 0u};
      if (np > 0) {
        int lo = 0, hi = m - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= q0) lo = mid; else hi = mid - 1;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          if (r < np) {
            while (lo + 1 < m && s_off[lo + 1] <= q0 + r) ++lo;
            w[r >> 1] |= (uint32_t)lo << (16 * (r & 1));
          }
        }
      }
      s_idx[threadIdx.x] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    const uint16_t* idx = reinterpret_cast<const uint16_t*>(s_idx);
    const int cnt = (int)(p1 - p0);
    for (int i0 = 0; i0 < cnt; i0 += blockDim.x) {   // coalesced writes; warp-uniform trip count
      const int i = i0 + threadIdx.x;
      const bool ok = i < cnt;
      uint32_t t = 0;
      if (ok) {
        const int lo = idx[i];
        const uint4 en = s_ent[lo];
        const int nx = (int)(en.z & 0xFFFFu), rowlen = (int)(en.z >> 16);
        const int local = (int)((uint32_t)(p0 + i) - s_off[lo]);
        // row and column of the pair in its rectangle: a reciprocal estimate of
        // local / nx, within one of the quotient while local < 2^23 (a view has
        // at most 2^23 tiles), then one integer correction step
        int ty = (int)(((float)local + 0.5f) * __uint_as_float(en.w));
        int tx = local - ty * nx;
        if (tx < 0) { --ty; tx += nx; } else if (tx >= nx) { ++ty; tx -= nx; }
        t = en.y + (uint32_t)(ty * rowlen + tx);
        (void)GS_IN_BOUNDS(hdr, t < T, BS_EMIT_TILE, t);
        (void)GS_IN_BOUNDS(hdr, en.x < E, BS_EMIT_ENTRY, en.x);
        ptile[p0 + i] = t;
        pval[p0 + i] = en.x;
      }
      hist_keys(s_h, tile_passes, t, ok, 1);
    }
  }
  hist_flush(s_h, tile_passes, ghist);
}

// ---------------------------------------------------------------------------
// Radix sort pass: histogram, per-digit scan over blocks, stable scatter
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_ranges(const uint32_t* __restrict__ ptile, const unsigned long long* n_pairs_ptr, int64_t cap,
         int2* __restrict__ ranges, int64_t T, Header* hdr) {
  pdl_wait();
  pdl_trigger();
  const int64_t P = clamp_count(n_pairs_ptr, cap);
  // four consecutive pairs per thread: one 16-byte load (the buffer is 16-byte
  // aligned), scalar loads for its two neighbours and for a ragged tail
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 4 * q < P;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * q;
    uint32_t t[6];
    if (i0 + 4 <= P) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(ptile) + q);
      t[1] = v.x; t[2] = v.y; t[3] = v.z; t[4] = v.w;
    } else {
      for (int k = 0; k < 4; ++k) t[1 + k] = i0 + k < P ? ptile[i0 + k] : 0xFFFFFFFFu;
    }
    t[0] = i0 > 0 ? ptile[i0 - 1] : 0xFFFFFFFFu;
    t[5] = i0 + 4 < P ? ptile[i0 + 4] : 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t i = i0 + k;
      if (i >= P) break;
      if (!GS_IN_BOUNDS(hdr, t[k + 1] < T, BS_RANGE_TILE, t[k + 1])) continue;
      if (i == 0 || t[k] != t[k + 1]) ranges[t[k + 1]].x = (int)i;
      if (i == P - 1 || t[k + 2] != t[k + 1]) ranges[t[k + 1]].y = (int)(i + 1);
    }
  }
}

// Work order of the compositing kernels: tiles by decreasing cost, so that
// the longest items start first and the persistent kernels end on short ones.
// The cost (the tile's list length unless `cost` is given) is bucketed by its
// floor(log2) and three more mantissa bits (256 buckets, heaviest first); one
// block, counting sort in shared memory.  The order inside a bucket is arbitrary: each pixel is
// computed by one warp whatever the order.
__device__ inline int cost_bucket(uint32_t c) {
  if (c < 8) return (int)c;
  const int e = 31 - __clz(c);                      // >= 3
  return ((e - 2) << 3) | (int)((c >> (e - 3)) & 7u);   // monotone in c, < 256
}

__global__ void __launch_bounds__(1024) k_tile_order(const int2* __restrict__ ranges,
                                                     const uint32_t* __restrict__ cost, int T,
                                                     int* __restrict__ order) {
  pdl_wait();
  pdl_trigger();
  __shared__ int cnt[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) cnt[b] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const uint32_t c = cost ? cost[t] : (uint32_t)max(ranges[t].y - ranges[t].x, 0);
    atomicAdd(&cnt[cost_bucket(c)], 1);
  }
  __syncthreads();
  if (threadIdx.x < 32) {   // exclusive offsets, heaviest bucket first: lane l owns buckets 255-8l .. 248-8l
    const int lane = threadIdx.x;
    int n[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) { n[i] = cnt[255 - 8 * lane - i]; sum += n[i]; }
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    int acc = incl - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) { cnt[255 - 8 * lane - i] = acc; acc += n[i]; }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const uint32_t c = cost ? cost[t] : (uint32_t)max(ranges[t].y - ranges[t].x, 0);
    order[atomicAdd(&cnt[cost_bucket(c)], 1)] = t;
  }
}

cudaError_t launch_tile_order(void* ws, const Layout& L, const uint32_t* cost, int* order, cudaStream_t s) {
  if (L.T > 0) launch_pdl(k_tile_order, 1, 1024, 0, s, at<int2>(ws, L.ranges), cost, (int)L.T, order);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-sweep LSD radix sort: the digit histograms of every pass are counted by
// the kernel that writes the keys (hist_keys); each pass is then a single kernel in which
// a block ranks its 4096 keys, publishes its per-digit counts, finds the
// counts of all blocks before it by decoupled look-back (each predecessor's
// word holds its own count, flagged A, or the inclusive prefix, flagged P) and
// scatters.  Blocks take their tile of keys in the order they start (a ticket
// counter), so a block only ever waits for blocks that are already running;
// every wait is bounded and sets GS_ERR_TIMEOUT if it runs out.
//
// kBallot finds the lanes of a warp holding the same digit (its peer mask)
// with one ballot per digit bit (the last pass's digit may have fewer than 8);
// otherwise a digit shared by the whole warp needs no matching and the others
// take `match.any`, which costs about 36 SM cycles per warp-wide call.
// A pass over a full 8-bit digit (the depth sort's four passes, the tile
// sort's first: digits spread over many values) runs two blocks per SM with
// ballots, 128 registers holding a thread's keys, values and ranks without
// spilling; the tile sort's last pass (a few high bits of the tile index,
// often shared by a whole warp) runs three blocks per SM with `match.any`.
// The look-back reads 4 predecessors' words per poll.
// ---------------------------------------------------------------------------
constexpr int kLookWindow = 4;          // predecessors' words per poll (registers bound it)
constexpr int kLookWindowBallot = 4;    // the same in the ballot passes, whose keys are placed first

// Exclusive prefix of digit d over the blocks before blk: the predecessors'
// words are read kLookWindow at a time, nearest first, and added up to the
// nearest P; a window with an unpublished word before that P is read again.
template <int kLookWindow>
__device__ inline uint32_t digit_lookback(const unsigned long long* look, int blk, int d, Header* hdr) {
  uint32_t excl = 0;
  int j = blk - 1, spins = 0;
  while (j >= 0) {
    unsigned long long f[kLookWindow];
#pragma unroll
    for (int q = 0; q < kLookWindow; ++q)   // before block 0: a zero inclusive prefix
      f[q] = j - q >= 0 ? ld_relaxed(look + (int64_t)(j - q) * kRadix + d) : kFlagP;
    int qp = kLookWindow;
#pragma unroll
    for (int q = kLookWindow - 1; q >= 0; --q)
      if ((f[q] & kFlagMask) == kFlagP) qp = q;
    bool ready = true;
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < kLookWindow; ++q)
      if (q <= qp) {
        ready = ready && (f[q] & kFlagMask) != 0;
        sum += (uint32_t)f[q];
      }
    if (!ready) {
      if (++spins > kSpinLimit) { set_status(hdr, GS_ERR_TIMEOUT); break; }
      continue;
    }
    excl += sum;
    if (qp < kLookWindow) break;
    j -= kLookWindow;
  }
  return excl;
}

template <int kMinBlocks, bool kBallot>
__global__ void __launch_bounds__(kSortThreads, kMinBlocks)
k_onesweep(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
           uint32_t* __restrict__ vout, const unsigned long long* count_ptr, int64_t cap, int pass, int dbits,
           const uint32_t* __restrict__ ghist, unsigned long long* __restrict__ look, int* ticket, Header* hdr) {
  pdl_wait();
  pdl_trigger();
  // [half][warp][digit] running digit counts of a warp's two halves of items
  // (rounds 0-7 and 8-15: two independent chains), then [0]: the warps' bases
  __shared__ uint16_t s_wc[2][8][kRadix];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_dstart[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_warp[33];
  __shared__ int s_blk;
  const int w = threadIdx.x >> 5;
  const int shift = kRadixBits * pass;
  if (threadIdx.x == 0) s_blk = atomicAdd(ticket, 1);
  for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) reinterpret_cast<uint32_t*>(&s_wc[0][0][0])[i] = 0;
  __syncthreads();
  const int blk = s_blk;
  const int64_t n = clamp_count(count_ptr, cap);
  const int64_t base = (int64_t)blk * kSortTile;
  if (base >= n) return;   // so do all blocks with later tickets: nobody waits for this one
  uint32_t k[kSortItems], v[kSortItems], rank[kSortItems];
  const unsigned lt = lanemask_lt();
  // tile-local item index of round r: w * 512 + 32 r + lane (WarpItems order)
  const int nloc = (int)min((int64_t)kSortTile, n - base);
  const int li0 = w * (32 * kSortItems) + (threadIdx.x & 31);
  const uint32_t* kb = kin + base;
  const uint32_t* vb = vin + base;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {   // all loads in flight before any ranking
    const int li = li0 + 32 * r;
    k[r] = li < nloc ? __ldg(kb + li) : 0u;
    v[r] = li < nloc ? __ldg(vb + li) : 0u;
  }
  // the peer masks of all items first (independent of one another), then the
  // warp's running digit counts item by item, rounds r and r + 8 side by side
  // in two counter sets
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const bool valid = li0 + 32 * r < nloc;
    const uint32_t d = (k[r] >> shift) & (kRadix - 1);
    const int dv = valid ? (int)d : kRadix;
    if (kBallot) {
      unsigned peers = __ballot_sync(FULL, valid);   // lanes past the end match nobody
#pragma unroll
      for (int b = 0; b < kRadixBits; ++b) {
        if (b < dbits) {
          const bool bit = (d >> b) & 1u;
          const unsigned m = __ballot_sync(FULL, bit);
          peers &= bit ? m : ~m;
        }
      }
      rank[r] = peers;
    } else {   // a digit shared by the whole warp needs no matching
      rank[r] = __all_sync(FULL, dv == __shfl_sync(FULL, dv, 0)) ? FULL : __match_any_sync(FULL, dv);
    }
  }
  constexpr int kHalf = kSortItems / 2;
#pragma unroll
  for (int r = 0; r < kHalf; ++r) {
    const int r2 = r + kHalf;
    const int dA = li0 + 32 * r < nloc ? (int)((k[r] >> shift) & (kRadix - 1)) : kRadix;
    const int dB = li0 + 32 * r2 < nloc ? (int)((k[r2] >> shift) & (kRadix - 1)) : kRadix;
    const unsigned pA = rank[r], pB = rank[r2];
    const uint32_t oA = dA < kRadix ? s_wc[0][w][dA] : 0u;
    const uint32_t oB = dB < kRadix ? s_wc[1][w][dB] : 0u;
    rank[r] = oA + __popc(pA & lt);
    rank[r2] = oB + __popc(pB & lt);
    __syncwarp();
    if (dA < kRadix && (pA & lt) == 0) s_wc[0][w][dA] = (uint16_t)(oA + __popc(pA));
    if (dB < kRadix && (pB & lt) == 0) s_wc[1][w][dB] = (uint16_t)(oB + __popc(pB));
    __syncwarp();
  }
  // the second half's items follow the first half's items of the same digit
#pragma unroll
  for (int r = kHalf; r < kSortItems; ++r) {
    const int d = li0 + 32 * r < nloc ? (int)((k[r] >> shift) & (kRadix - 1)) : kRadix;
    if (d < kRadix) rank[r] += s_wc[0][w][d];
  }
  __syncthreads();
  const int d = threadIdx.x;   // one thread per digit from here on
  uint32_t c[8], cnt = 0;
  for (int i = 0; i < 8; ++i) { c[i] = (uint32_t)s_wc[0][i][d] + s_wc[1][i][d]; cnt += c[i]; }
  unsigned long long* mine = look + (int64_t)blk * kRadix + d;
  // a digit no key holds (most of a narrow or concentrated digit's values)
  // needs neither the word nor the look-back: every block skips it alike
  const uint32_t gcnt = ghist[pass * kRadix + d];
  if (gcnt) st_relaxed(mine, (blk == 0 ? kFlagP : kFlagA) | cnt);   // successors may start looking
  // block-local exclusive scan over (digit, warp) in digit-major order, and the
  // digit's start in the whole key set (exclusive scan of the global histogram)
  const uint32_t start = block_exclusive_scan(cnt, s_warp, nullptr);
  const uint32_t dbase = block_exclusive_scan(gcnt, s_warp, nullptr);
  s_dstart[d] = start;
  uint32_t run = start;
  for (int i = 0; i < 8; ++i) { s_wc[0][i][d] = (uint16_t)run; run += c[i]; }   // bases <= 4096
  // the keys in block order of digits: with ballots (two blocks per SM) before
  // the look-back, so that their registers are free for its window
  auto place = [&]() {
    for (int r = 0; r < kSortItems; ++r) {
      if (li0 + 32 * r < nloc) {
        const int dd = (int)((k[r] >> shift) & (kRadix - 1));
        const uint32_t pos = s_wc[0][w][dd] + rank[r];
        s_keys[pos] = k[r];
        s_vals[pos] = v[r];
      }
    }
  };
  if (kBallot) {
    __syncthreads();
    place();
  }
  // decoupled look-back: keys of digit d in the blocks before this one
  uint32_t excl = 0;
  if (blk > 0 && gcnt) {
    excl = digit_lookback<kBallot ? kLookWindowBallot : kLookWindow>(look, blk, d, hdr);
    st_relaxed(mine, kFlagP | (excl + cnt));
  }
  s_gbase[d] = dbase + excl;
  __syncthreads();
  if (!kBallot) {
    place();
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nloc; i += kSortThreads) {
    const uint32_t kk = s_keys[i];
    const int dd = (int)((kk >> shift) & (kRadix - 1));
    const uint32_t dst = s_gbase[dd] + (uint32_t)i - s_dstart[dd];
    if (GS_IN_BOUNDS(hdr, dst < n, BS_SORT_DST, dst)) {
      kout[dst] = kk;
      vout[dst] = s_vals[i];
    }
  }
}

// Sorts (k0, v0) by the low `bits` bits of the keys, whose digit histograms are
// already in aux; the result ends in (k0, v0) after an even number of 8-bit
// passes, else in (k1, v1).
static cudaError_t radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                              const unsigned long long* count, int64_t cap, int nb, int bits, void* aux,
                              size_t aux_bytes, Header* hdr, cudaStream_t s) {
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  uint32_t* ghist = static_cast<uint32_t*>(aux);                       // [kMaxPasses][256]
  int* tickets = reinterpret_cast<int*>(ghist + kMaxPasses * kRadix);   // [kMaxPasses]
  unsigned long long* look = reinterpret_cast<unsigned long long*>(static_cast<char*>(aux) + 8192);
  (void)aux_bytes;   // cleared by the binning's single memset
  uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
  for (int p = 0; p < passes; ++p) {
    // keys are below 2^bits: the last pass's digit has its remaining bits only
    const int dbits = bits - kRadixBits * p < kRadixBits ? bits - kRadixBits * p : kRadixBits;
    unsigned long long* lp = look + (int64_t)p * nb * kRadix;
    if (dbits == kRadixBits)
      launch_pdl(k_onesweep<2, true>, nb, kSortThreads, 0, s, ki, vi, ko, vo, count, cap, p, dbits, ghist, lp,
                 tickets + p, hdr);
    else
      launch_pdl(k_onesweep<3, false>, nb, kSortThreads, 0, s, ki, vi, ko, vo, count, cap, p, dbits, ghist, lp,
                 tickets + p, hdr);
    uint32_t* t;
    t = ki; ki = ko; ko = t;
    t = vi; vi = vo; vo = t;
  }
  return cudaGetLastError();
}

int tile_sort_bits(int64_t n_tiles) {
  int bits = 0;
  while ((int64_t(1) << bits) < n_tiles) ++bits;
  return bits < 1 ? 1 : bits;
}

cudaError_t launch_bin(void* ws, const Layout& L, const FrameDev& hf, cudaStream_t s) {
  const FrameDev* fd = at<FrameDev>(ws, L.frame);
  Header* hdr = at<Header>(ws, L.hdr);
  uint32_t* key = at<uint32_t>(ws, L.key);
  uint32_t* touched = at<uint32_t>(ws, L.touched);
  int* scan_ticket = at<int>(ws, L.scanaux);   // [0]: compaction, [1]: pair offsets
  unsigned long long* scan_words = at<unsigned long long>(ws, L.scanaux + 64);   // [2][nb_E]
  uint32_t *vk0 = at<uint32_t>(ws, L.vkey[0]), *vk1 = at<uint32_t>(ws, L.vkey[1]);
  uint32_t *vv0 = at<uint32_t>(ws, L.vval[0]), *vv1 = at<uint32_t>(ws, L.vval[1]);
  uint32_t *pt0 = at<uint32_t>(ws, L.ptile[0]), *pt1 = at<uint32_t>(ws, L.ptile[1]);
  uint32_t *pv0 = at<uint32_t>(ws, L.pval[0]), *pv1 = at<uint32_t>(ws, L.pval[1]);
  (void)hf;
  // 0. one memset clears both sorts' and both scans' auxiliary words and the
  //    tile ranges (contiguous)
  cudaError_t e0 = cudaMemsetAsync(at<char>(ws, L.sortaux[0]), 0, L.ranges + 8 * (size_t)L.T - L.sortaux[0], s);
  if (e0 != cudaSuccess) return e0;
  // 1. compaction (also counts the depth keys' digits for the sort)
  launch_pdl(k_compact, L.nb_E, kSortThreads, 0, s, key, L.E, vk0, vv0, at<uint32_t>(ws, L.sortaux[0]), scan_words,
             scan_ticket, &hdr->n_vis, hdr);
  // 2. depth sort: 31 bits (z > 0, so the sign bit is clear)
  cudaError_t err = radix_sort(vk0, vv0, vk1, vv1, &hdr->n_vis, L.E, L.nb_E, 32, at<void>(ws, L.sortaux[0]),
                               L.sortaux_bytes[0], hdr, s);
  if (err != cudaSuccess) return err;
  // 3. pair offsets (the pair count and the capacity check)
  uint32_t* pair_off = at<uint32_t>(ws, L.pair_off);
  uint32_t* chunk_first = at<uint32_t>(ws, L.chunk_first);
  const int64_t n_chunks = (L.Pcap + kEmitChunk - 1) / kEmitChunk + 1;
  launch_pdl(k_pair_offsets, L.nb_E, kSortThreads, 0, s, vv0, &hdr->n_vis, L.E, touched, pair_off, chunk_first,
             n_chunks, scan_words + L.nb_E, scan_ticket + 1, &hdr->n_pairs, L.Pcap, hdr);
  // 4. emission
  // (the emission also counts the tile keys' digits for the sort)
  const int bits = tile_sort_bits(L.T);
  const int tile_passes = (bits + kRadixBits - 1) / kRadixBits;
  const int eg = (int)std::min<int64_t>((L.Pcap + kEmitChunk - 1) / kEmitChunk, 148 * 8);
  launch_pdl(k_emit, eg, kSortThreads, 0, s, fd, vv0, &hdr->n_vis, &hdr->n_pairs, L.E, at<short4>(ws, L.rect),
             pair_off, L.Pcap, pt0, pv0, chunk_first, n_chunks, tile_passes, at<uint32_t>(ws, L.sortaux[1]), L.T,
             hdr);
  // 5. tile sort
  err = radix_sort(pt0, pv0, pt1, pv1, &hdr->n_pairs, L.Pcap, L.nb_P, bits, at<void>(ws, L.sortaux[1]),
                   L.sortaux_bytes[1], hdr, s);
  if (err != cudaSuccess) return err;
  uint32_t* ptile = at<uint32_t>(ws, L.ptile_final);
  // 6. ranges
  int g = (int)std::max<int64_t>(1, std::min<int64_t>((L.Pcap / 4 + 255) / 256, 148 * 16));
  launch_pdl(k_ranges, g, 256, 0, s, ptile, &hdr->n_pairs, L.Pcap, at<int2>(ws, L.ranges), L.T, hdr);
  // 7. compositing work order (by list length)
  return launch_tile_order(ws, L, nullptr, at<int>(ws, L.tile_order), s);
}

}  // namespace gs
