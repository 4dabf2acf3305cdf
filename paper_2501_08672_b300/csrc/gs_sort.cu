// Tile binning: the (tile, depth) sort the 3D-GS tile rasteriser relies on
// (Sec. II-C mentions its tile-based depth sorting).
//
// A least-significant-digit radix sort of 64-bit keys (tile << 32 | depth
// bits) first sorts on the depth digits, which are identical for every pair
// a Gaussian emits.  So the depth digits are sorted once per record (M keys)
// instead of once per pair (P keys): records are put in depth order (a
// stable radix sort on the high word of their 64-bit double-float depth key,
// then runs of equal high words ordered by the low word), expanded into pairs
// in that order, and the pairs are stably radix-sorted by tile id only
// (ceil(log2 T) bits).  The result is the order of the full sort on
// (tile, 64-bit depth key) with ties broken by record index.
//
// Every kernel reads counts from device memory, so the whole binning step
// needs no host synchronisation and can be captured in a CUDA graph; the
// pair capacity is fixed by the workspace and overflow is latched.
#include "gs_internal.cuh"

namespace gsb {

namespace {

constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned long long clamp_n(unsigned long long n_host,
                                                      const unsigned long long* n_dev) {
    if (!n_dev) return n_host;
    const unsigned long long d = *n_dev;
    return d < n_host ? d : n_host;
}

// ---- LSD radix sort pass --------------------------------------------------
//
// One pass sorts on `bits` (<= 8) bits starting at `shift`.  The keys are cut
// into tiles of kRTile = 4096 consecutive keys, one tile per block:
//   upsweep:   per-tile digit histogram -> hist[digit * nblk + tile]
//   scan:      device-wide exclusive scan of hist (digit-major), so the entry
//              is the first output position of that digit from that tile
//   downsweep: the tile ranks its keys stably (each warp ranks a contiguous
//              slice with private digit counters, a scan over warps and
//              digits places the slices), stages them digit-sorted in shared
//              memory, and writes each digit run to consecutive positions.
// The key count may live in device memory (n_dev), so the grid is sized by
// the capacity and tiles past the count do nothing.

constexpr int kRItems = 16;
constexpr int kRTile = kRadixThreads * kRItems;

__device__ __forceinline__ uint32_t lane_lt_mask() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Also zeroes `nzero` 64-bit words at `zero` (block 0): the look-back flags
// and ticket of the scan that follows, without a separate memset.
template <bool MAPPED>
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const uint32_t* __restrict__ keys,
                                                                 unsigned long long n_host,
                                                                 const unsigned long long* n_dev,
                                                                 int shift, int bits,
                                                                 uint32_t* __restrict__ hist,
                                                                 unsigned long long* __restrict__ zero, int nzero,
                                                                 const unsigned long long* __restrict__ key_range) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t wh[kRadixWarps][256];
    const KeyMap km = MAPPED ? load_key_map(key_range) : KeyMap{0u, 0};
    const int t = threadIdx.x, w = t >> 5;
    if (blockIdx.x == 0)
        for (int i = t; i < nzero; i += kRadixThreads) zero[i] = 0ull;
#pragma unroll
    for (int k = 0; k < kRadixWarps; ++k) wh[k][t] = 0u;
    __syncthreads();
    const unsigned long long n = clamp_n(n_host, n_dev);
    const unsigned long long base = (unsigned long long)blockIdx.x * kRTile;
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t kk[kRItems];
#pragma unroll
    for (int k = 0; k < kRItems; ++k) {
        const unsigned long long i = base + (unsigned long long)k * kRadixThreads + t;
        kk[k] = i < n ? keys[i] : 0u;
        if (MAPPED) kk[k] = map_key(kk[k], km);
    }
#pragma unroll
    for (int k = 0; k < kRItems; ++k) {
        const unsigned long long i = base + (unsigned long long)k * kRadixThreads + t;
        if (i < n) atomicAdd(&wh[w][(kk[k] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kRadixWarps; ++k) c += wh[k][t];
    hist[(size_t)t * gridDim.x + blockIdx.x] = c;
}

// Downsweep.  Warp w owns the contiguous slice [w * 512, (w + 1) * 512) of
// the tile and ranks it in 16 rounds of 32 consecutive keys with counters
// only it touches: match.any groups equal digits of a round, the group
// leader reads the running count of its digit and adds the group size, and
// the group's lanes take consecutive ranks after it.  A scan over the warps
// per digit and over the digits then places every key stably within the
// tile, the tile is staged digit-sorted in shared memory and written out in
// runs of consecutive positions.
template <bool MAPPED>
__global__ void __launch_bounds__(kRadixThreads, 3) k_radix_downsweep(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
    uint32_t* __restrict__ vout, unsigned long long n_host, const unsigned long long* n_dev, int shift,
    int bits, const uint32_t* __restrict__ hist, const unsigned long long* __restrict__ key_range) {
    pdl_wait();
    pdl_trigger();
    constexpr int kSlice = kRTile / kRadixWarps;  // 512 keys per warp
    __shared__ uint32_t s_keys[kRTile];
    __shared__ uint32_t s_vals[kRTile];
    __shared__ uint32_t s_wc[kRadixWarps][256];
    __shared__ uint32_t s_start[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_wsum[kRadixWarps];
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const unsigned long long n = clamp_n(n_host, n_dev);
    const unsigned long long base = (unsigned long long)blockIdx.x * kRTile;
    if (base >= n) return;
    const int count = (int)(n - base < (unsigned long long)kRTile ? n - base : (unsigned long long)kRTile);
    const uint32_t mask = (1u << bits) - 1u;
    const uint32_t lt = lane_lt_mask();
    // digits of the mapped key (depth sort) or of the key itself
    const KeyMap km = MAPPED ? load_key_map(key_range) : KeyMap{0u, 0};
    auto digit = [&](uint32_t k) { return ((MAPPED ? map_key(k, km) : k) >> shift) & mask; };
#pragma unroll
    for (int ww = 0; ww < kRadixWarps; ++ww) s_wc[ww][t] = 0u;
    s_gbase[t] = hist[(size_t)t * gridDim.x + blockIdx.x];
    __syncthreads();

    uint32_t key[kRItems], val[kRItems], rank[kRItems];
#pragma unroll
    for (int k = 0; k < kRItems; ++k) {
        const int j = w * kSlice + k * 32 + lane;
        key[k] = j < count ? kin[base + j] : 0u;
        val[k] = j < count ? vin[base + j] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kRItems; ++k) {
        const bool valid = w * kSlice + k * 32 + lane < count;
        const uint32_t d = digit(key[k]);
        // lanes holding the same digit: one ballot per digit bit (an invalid
        // lane is its own group)
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
        uint32_t peers = vm;
#pragma unroll
        for (int bit = 0; bit < 8; ++bit) {
            const bool set = (d >> bit) & 1u;
            const uint32_t bm = __ballot_sync(0xffffffffu, set);
            peers &= set ? bm : ~bm;
        }
        if (!valid) peers = 1u << lane;
        const int leader = __ffs(peers) - 1;
        uint32_t before = 0;
        if (valid && lane == leader) {
            before = s_wc[w][d];
            s_wc[w][d] = before + __popc(peers);
        }
        before = __shfl_sync(0xffffffffu, before, leader);
        rank[k] = before + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit t: offsets of the warps' runs, and the tile's digit count
    uint32_t total = 0;
#pragma unroll
    for (int ww = 0; ww < kRadixWarps; ++ww) {
        const uint32_t c = s_wc[ww][t];
        s_wc[ww][t] = total;
        total += c;
    }
    {
        uint32_t x = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[w] = x;
        __syncthreads();
        uint32_t wp = 0;
        for (int ww = 0; ww < w; ++ww) wp += s_wsum[ww];
        s_start[t] = wp + x - total;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRItems; ++k) {
        if (w * kSlice + k * 32 + lane < count) {
            const uint32_t d = digit(key[k]);
            const uint32_t pos = s_start[d] + s_wc[w][d] + rank[k];
            s_keys[pos] = key[k];
            s_vals[pos] = val[k];
        }
    }
    __syncthreads();
    // consecutive threads write consecutive positions of each digit run
    for (int i = t; i < count; i += kRadixThreads) {
        const uint32_t k = s_keys[i];
        const uint32_t d = digit(k);
        const uint32_t pos = s_gbase[d] + (uint32_t)i - s_start[d];
        if (pos < n) {  // always true for a consistent histogram; guards the write
            kout[pos] = k;
            vout[pos] = s_vals[i];
        }
    }
}

constexpr int kU32ScanChunk = 4096;

// Device-wide exclusive scan of a u32 array in place in one pass (decoupled
// look-back): each block takes the next 4096-entry chunk from a ticket (so
// every chunk before it belongs to a block that has started), publishes the
// chunk's sum, and one warp walks back over the flags of the 32 chunks before
// it at a time, adding sums until it meets a published inclusive prefix.
// A flag word packs the status (bits 62-63: 0 not ready, 1 chunk sum, 2
// inclusive prefix) with the 32-bit value; the words and the ticket are
// zeroed before each scan.  Waits are bounded: after kLookbackPolls polls
// without progress the block latches GS_ERR_TIMEOUT in the status word and
// finishes with the sums it has (the result is then unusable, and the host
// learns it from gs_sync_status).
constexpr int kLookbackPolls = 1 << 20;

__global__ void __launch_bounds__(1024) k_u32_scan_lookback(uint32_t* __restrict__ a, long long n,
                                                            unsigned long long* flags, unsigned int* ticket,
                                                            unsigned int* status) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_w[32];
    __shared__ unsigned int s_chunk;
    __shared__ uint32_t s_prefix;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_chunk = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long chunk = s_chunk;
    const long long base = chunk * kU32ScanChunk + (long long)t * 4;
    uint32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? a[base + k] : 0u;
        s += v[k];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t y = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        s_w[lane] = y;
        const uint32_t agg = __shfl_sync(0xffffffffu, y, 31);
        volatile unsigned long long* vf = flags;
        if (chunk == 0) {
            if (lane == 0) {
                vf[0] = (2ull << 62) | agg;
                s_prefix = 0;
            }
        } else {
            if (lane == 0) vf[chunk] = (1ull << 62) | agg;
            uint32_t excl = 0;
            long long j = chunk - 1;  // the window is chunks j - 31 .. j
            for (;;) {
                const long long idx = j - lane;
                unsigned long long f = 2ull << 62;  // before chunk 0: a prefix of 0
                if (idx >= 0) f = vf[idx];
                int polls = 0;
                while (__any_sync(0xffffffffu, (f >> 62) == 0)) {
                    if (++polls > kLookbackPolls) {
                        if (lane == 0) atomicCAS(status, 0u, (unsigned int)(-GS_ERR_TIMEOUT));
                        f = (2ull << 62) | (f & 0xFFFFFFFFull);  // give up: treat as a prefix
                        break;
                    }
                    if ((f >> 62) == 0) f = vf[idx];
                }
                const uint32_t pre = __ballot_sync(0xffffffffu, (f >> 62) == 2);
                const int stop = pre ? __ffs(pre) - 1 : 31;  // nearest chunk holding a prefix
                uint32_t val = lane <= stop ? (uint32_t)(f & 0xFFFFFFFFull) : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                excl += val;
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) {
                vf[chunk] = (2ull << 62) | (uint32_t)(excl + agg);
                s_prefix = excl;
            }
        }
    }
    __syncthreads();
    uint32_t run = s_prefix + (w > 0 ? s_w[w - 1] : 0u) + x - s;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) {
            a[base + k] = run;
            run += v[k];
        }
}

// Exclusive scan of a u32 array in place by one block: thread t scans a
// contiguous chunk, a block scan of the chunk totals gives its offset.  For
// the digit-major histograms of tiny sorts (up to kU32SingleScanMax entries,
// e.g. the tile-order pass); beyond a few thousand entries one block is
// slower than a device-wide scan (measured: 80 us against 15 us at 100k
// entries).
constexpr long long kU32SingleScanMax = 1ll << 14;

__global__ void __launch_bounds__(1024) k_u32_scan_single(uint32_t* __restrict__ a, long long n) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_w[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const long long per = (n + 1023) / 1024;
    const long long b0 = (long long)t * per;
    const long long b1 = b0 + per < n ? b0 + per : n;
    uint32_t sum = 0;
    for (long long i = b0; i < b1; ++i) sum += a[i];
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t y = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    uint32_t run = (w > 0 ? s_w[w - 1] : 0u) + x - sum;
    for (long long i = b0; i < b1; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Depth order, second step.  The records are sorted stably by the 24-bit map
// of the high word of their 64-bit depth key (see KeyMap), so records with
// equal mapped keys sit in runs in record order; each run is put in (high
// word, low word, record) order here, which is the order of the full 64-bit
// key with ties by record index (the map is monotone).  One thread per run:
// insertion sort for short runs (the common case: a run spans 2^s key values
// at most), heapsort beyond kFixupInsertion (a long run only costs time).
// The high words move with the records.  Culled records (mapped key
// 0xFFFFFF, never listed) are left alone.
constexpr long long kFixupInsertion = 48;

struct DepthKey {
    uint32_t h;
    unsigned long long l;  // low word, record
    __device__ __forceinline__ bool operator>(const DepthKey& o) const { return h != o.h ? h > o.h : l > o.l; }
};

__device__ __forceinline__ DepthKey depth_key(const uint32_t* hi, const uint32_t* a, const uint32_t* lo, long long i) {
    const uint32_t v = a[i];
    return DepthKey{hi[i], ((unsigned long long)lo[v] << 32) | v};
}

__device__ void heap_sift(uint32_t* hi, uint32_t* a, long long root, long long n, const uint32_t* lo) {
    const uint32_t h = hi[root], v = a[root];
    const DepthKey kv = depth_key(hi, a, lo, root);
    long long i = root;
    while (true) {
        long long c = 2 * i + 1;
        if (c >= n) break;
        DepthKey kc = depth_key(hi, a, lo, c);
        if (c + 1 < n) {
            const DepthKey kr = depth_key(hi, a, lo, c + 1);
            if (kr > kc) {
                ++c;
                kc = kr;
            }
        }
        if (!(kc > kv)) break;
        hi[i] = hi[c];
        a[i] = a[c];
        i = c;
    }
    hi[i] = h;
    a[i] = v;
}

// Block 0 also zeroes `nzero` 64-bit words at `zero`: the look-back flags and
// ticket of the offsets scan that follows.
__global__ void __launch_bounds__(256) k_depth_fixup(uint32_t* __restrict__ hi, uint32_t* __restrict__ vals,
                                                     const uint32_t* __restrict__ lo, long long M,
                                                     unsigned long long* __restrict__ zero, int nzero,
                                                     const unsigned long long* __restrict__ key_range) {
    pdl_wait();
    pdl_trigger();
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0ull;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const KeyMap km = load_key_map(key_range);
    const uint32_t h = map_key(hi[j], km);
    if (h == 0xFFFFFFu) return;
    if (j > 0 && map_key(hi[j - 1], km) == h) return;      // not the first of its run
    if (j + 1 >= M || map_key(hi[j + 1], km) != h) return;  // a run of one
    long long e = j + 2;
    while (e < M && map_key(hi[e], km) == h) ++e;
    uint32_t* a = vals + j;
    uint32_t* ha = hi + j;
    const long long n = e - j;
    if (n <= kFixupInsertion) {
        for (long long i = 1; i < n; ++i) {
            const uint32_t hv = ha[i], v = a[i];
            const DepthKey kv = depth_key(ha, a, lo, i);
            long long k = i - 1;
            while (k >= 0 && depth_key(ha, a, lo, k) > kv) {
                ha[k + 1] = ha[k];
                a[k + 1] = a[k];
                --k;
            }
            ha[k + 1] = hv;
            a[k + 1] = v;
        }
        return;
    }
    for (long long r = n / 2 - 1; r >= 0; --r) heap_sift(ha, a, r, n, lo);
    for (long long end = n - 1; end > 0; --end) {
        const uint32_t th = ha[0], t = a[0];
        ha[0] = ha[end];
        a[0] = a[end];
        ha[end] = th;
        a[end] = t;
        heap_sift(ha, a, 0, end, lo);
    }
}

// ---- tiles-touched scan in depth order ------------------------------------

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total) {
    __shared__ uint32_t s_w[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t y = lane < nw ? s_w[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    total = s_w[(blockDim.x >> 5) - 1];
    const uint32_t wprefix = w > 0 ? s_w[w - 1] : 0u;
    __syncthreads();
    return wprefix + x - v;
}

// Pair offsets in one pass: the exclusive scan of tiles-touched over the
// records in depth order, by decoupled look-back over 4096-record chunks taken
// from a ticket (as k_u32_scan_lookback; flag words pack a 2-bit status with a
// 62-bit value).  The block of the last chunk knows the grand total: it
// stores the pair count and latches GS_ERR_CAPACITY when it exceeds cap.
__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(const uint32_t* __restrict__ order,
                                                               const uint32_t* __restrict__ touched, long long M,
                                                               unsigned long long* flags, int nchunks,
                                                               unsigned long long* __restrict__ offsets,
                                                               unsigned long long* __restrict__ counters, long long cap,
                                                               unsigned int* status,
                                                               unsigned long long* status_pairs) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned int s_chunk;
    __shared__ unsigned long long s_prefix;
    const int t = threadIdx.x, lane = t & 31;
    // The depth sort is done: the next projection opens a new key-range
    // generation, into cleared slots.  (A slot can start out holding a value
    // tagged with a later generation, e.g. in a workspace allocated over old
    // data; the projection's atomicMax would never replace it, and every
    // binning would fall back to the coarse key map with its long runs of
    // equal keys.  Cleared here, such a value lasts one binning at most.)
    if (blockIdx.x == 0 && t == 0) {
        counters[kCtrRangeGen] += 1ull;
        counters[kCtrRangeMax] = 0ull;
        counters[kCtrRangeMin] = 0ull;
    }
    if (t == 0) s_chunk = atomicAdd(reinterpret_cast<unsigned int*>(flags + nchunks), 1u);
    __syncthreads();
    const long long chunk = s_chunk;
    const long long base = chunk * kScanChunk + (long long)t * kScanItems;
    uint32_t v[kScanItems];
    uint32_t sum = 0;
    if (base + kScanItems <= M) {  // 16-byte aligned: base is a multiple of 4
        const uint4 o4 = *reinterpret_cast<const uint4*>(order + base);
        v[0] = touched[o4.x];
        v[1] = touched[o4.y];
        v[2] = touched[o4.z];
        v[3] = touched[o4.w];
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < M ? touched[order[base + k]] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) sum += v[k];
    uint32_t agg32;
    const uint32_t ex = block_exclusive_scan(sum, agg32);
    if (t < 32) {
        const unsigned long long agg = agg32;
        constexpr unsigned long long kVal = (1ull << 62) - 1ull;
        volatile unsigned long long* vf = flags;
        unsigned long long excl = 0;
        if (chunk == 0) {
            if (lane == 0) vf[0] = (2ull << 62) | agg;
        } else {
            if (lane == 0) vf[chunk] = (1ull << 62) | agg;
            long long j = chunk - 1;
            for (;;) {
                const long long idx = j - lane;
                unsigned long long f = 2ull << 62;  // before chunk 0: a prefix of 0
                if (idx >= 0) f = vf[idx];
                int polls = 0;
                while (__any_sync(0xffffffffu, (f >> 62) == 0)) {
                    if (++polls > kLookbackPolls) {
                        if (lane == 0) atomicCAS(status, 0u, (unsigned int)(-GS_ERR_TIMEOUT));
                        f = (2ull << 62) | (f & kVal);
                        break;
                    }
                    if ((f >> 62) == 0) f = vf[idx];
                }
                const uint32_t pre = __ballot_sync(0xffffffffu, (f >> 62) == 2);
                const int stop = pre ? __ffs(pre) - 1 : 31;
                unsigned long long val = lane <= stop ? (f & kVal) : 0ull;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                excl += val;
                if (pre) break;
                j -= 32;
            }
            if (lane == 0) vf[chunk] = (2ull << 62) | ((excl + agg) & kVal);
        }
        if (lane == 0) {
            s_prefix = excl;
            if (chunk == nchunks - 1) {
                const unsigned long long total = excl + agg;
                counters[0] = total;
                if (status_pairs) *status_pairs = total;
                if (total > (unsigned long long)cap && status) atomicCAS(status, 0u, (unsigned int)(-GS_ERR_CAPACITY));
            }
        }
    }
    __syncthreads();
    unsigned long long run = s_prefix + ex;
    if (base + kScanItems <= M) {
        ulonglong2* o2 = reinterpret_cast<ulonglong2*>(offsets + base);
        const unsigned long long r1 = run + v[0], r2 = r1 + v[1], r3 = r2 + v[2];
        o2[0] = make_ulonglong2(run, r1);
        o2[1] = make_ulonglong2(r2, r3);
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k)
            if (base + k < M) {
                offsets[base + k] = run;
                run += v[k];
            }
    }
}

// One thread per record in depth order writes its pairs (global tile id,
// record index) at its scanned offset, row-major over the tiles of its
// rectangle that its footprint reaches.  Rectangles of up to kMaskTiles
// tiles come with the mask of listed tiles from the projection.  Larger ones
// are emitted by the whole warp from the same row spans k_project counted
// with: the owner's footprint is broadcast, each lane takes one tile row,
// and a warp scan of the rows' tile counts places them in row-major order.
__device__ __forceinline__ uint32_t warp_exclusive_scan(uint32_t v, uint32_t* total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// F > 1 (bins of F x F compositing tiles, split later): each pair's key
// also carries, above its bin id (bits from 32 - F^2 up), the mask of the
// bin's tiles the record's footprint reaches, row-major: per tile row of the
// bin the columns footrows_span gives at the tile size ts / F (the binning's
// own test, so the split lists are those of binning at the tile size).
template <int F>
__device__ __forceinline__ uint32_t tile_mask(const FootRows& fr, int bx, int by, int tts) {
    uint32_t m = 0;
#pragma unroll
    for (int sy = 0; sy < F; ++sy) {
        int a, b;
        if (footrows_span(fr, by * F + sy, tts, bx * F, bx * F + F, &a, &b))
            m |= ((2u << (b - bx * F)) - (1u << (a - bx * F))) << (sy * F);
    }
    return m << (32 - F * F);
}

template <int F>
__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ order,
                                              const int4* __restrict__ rects,
                                              const float4* __restrict__ rec,
                                              const unsigned long long* __restrict__ offsets, long long M,
                                              long long cap, int ts, float log2_alpha_min,
                                              uint32_t* __restrict__ pkeys, uint32_t* __restrict__ pvals,
                                              uint32_t* __restrict__ pair_rec) {
    pdl_wait();
    pdl_trigger();
    // The pair's value: its record, or, for the deterministic backward
    // (pair_rec non-NULL), its own emission index, the record going to
    // pair_rec, so that the tile sort also yields every pair's emission index.
    auto put_val = [pvals, pair_rec](unsigned long long q, uint32_t rr) {
        if (pair_rec) {
            pvals[q] = (uint32_t)q;
            pair_rec[q] = rr;
        } else {
            pvals[q] = rr;
        }
    };
    const long long j0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = j0 < M;
    if (__all_sync(0xffffffffu, !live)) return;
    const long long j = live ? j0 : 0;
    const uint32_t r = order[j];
    // the record's rectangle, then its tile count and listed-tile mask (the
    // two halves of one 32-byte entry)
    const int4 rc = rects[2 * r];
    const int4 rm = rects[2 * r + 1];
    const uint32_t tt = live ? (uint32_t)rm.x : 0u;
    const int tx0 = rc.x & 0xFFFF, ty0 = (rc.x >> 16) & 0xFFFF;
    const int tx1 = rc.y & 0xFFFF, ty1 = (rc.y >> 16) & 0xFFFF;
    const bool test = log2_alpha_min > -3.0e38f;
    const int w = tx1 - tx0;
    const int area = w * (ty1 - ty0);
    const bool coop = tt > 0 && test && area > kMaskTiles;
    const unsigned long long o0 = offsets[j];
    const unsigned long long oend = o0 + tt;
    const unsigned long long ucap = (unsigned long long)cap;
    const int lane = threadIdx.x & 31;
    {
        // Records of the mask path (rectangles of <= 32 tiles) are written by
        // the warp together: the warp's records are consecutive in depth
        // order, so their pairs fill one contiguous range, and lane l writes
        // positions l, l + 32, ... of it.  The owner of a position is the
        // last record whose first position is at or below it (binary search
        // over the lanes' offsets), the tile its mask's j-th set bit, bits
        // in row-major order of the rectangle.
        const bool mp = tt > 0 && area <= kMaskTiles;
        const unsigned long long wbase = __shfl_sync(0xffffffffu, o0, 0);  // lane 0 is live
        const uint32_t rel = live ? (uint32_t)(o0 - wbase) : 0xFFFFFFFFu;
        const uint32_t wtotal = __reduce_max_sync(0xffffffffu, live ? rel + tt : 0u);
        const uint32_t mask = mp ? (uint32_t)rm.y : 0u;
        const uint32_t key0 = (uint32_t)rc.z + (uint32_t)ty0 * (uint32_t)rc.w + (uint32_t)tx0;
        // floor(b / w) = (b * ceil(2048 / w)) >> 11 for b < 32, w <= 32
        const uint32_t info = mp ? ((uint32_t)w | ((2048u + (uint32_t)w - 1u) / (uint32_t)w) << 8 | 0x80000000u) : 0u;
        FootRows mf{};  // the record's footprint rows, for the tile masks of F > 1
        if (F > 1 && mp) mf = make_footrows(rec[3 * r], rec[3 * r + 1], rec[3 * r + 1].z - log2_alpha_min);
        for (uint32_t p0 = 0; p0 < wtotal; p0 += 32) {
            const uint32_t pr = p0 + (uint32_t)lane;
            int e = 0;
#pragma unroll
            for (int st = 16; st >= 1; st >>= 1) {
                const uint32_t oc = __shfl_sync(0xffffffffu, rel, e + st);
                if (oc <= pr) e += st;
            }
            const uint32_t ie = __shfl_sync(0xffffffffu, info, e);
            const uint32_t me = __shfl_sync(0xffffffffu, mask, e);
            const uint32_t ke = __shfl_sync(0xffffffffu, key0, e);
            const uint32_t se = (uint32_t)__shfl_sync(0xffffffffu, rc.w, e);
            const uint32_t re = __shfl_sync(0xffffffffu, r, e);
            const uint32_t be = __shfl_sync(0xffffffffu, rel, e);
            FootRows ef{};  // the owner's footprint rows (F > 1)
            uint32_t rx = 0;
            if constexpr (F > 1) {
                ef.qx = __shfl_sync(0xffffffffu, mf.qx, e);
                ef.qy = __shfl_sync(0xffffffffu, mf.qy, e);
                ef.A = __shfl_sync(0xffffffffu, mf.A, e);
                ef.B = __shfl_sync(0xffffffffu, mf.B, e);
                ef.det = __shfl_sync(0xffffffffu, mf.det, e);
                ef.invA = __shfl_sync(0xffffffffu, mf.invA, e);
                ef.ymax = __shfl_sync(0xffffffffu, mf.ymax, e);
                ef.dyr = __shfl_sync(0xffffffffu, mf.dyr, e);
                ef.lim = __shfl_sync(0xffffffffu, mf.lim, e);
                rx = (uint32_t)__shfl_sync(0xffffffffu, rc.x, e);
            }
            const unsigned long long q = wbase + pr;
            if (pr < wtotal && (ie >> 31) && q < ucap) {
                // the (pr - be)-th set bit of the mask (0 based), by halving
                uint32_t jj = pr - be, m = me, bit = 0;
#pragma unroll
                for (int h = 16; h >= 1; h >>= 1) {
                    const uint32_t c = __popc(m & ((1u << h) - 1u));
                    if (jj >= c) {
                        jj -= c;
                        bit += (uint32_t)h;
                        m >>= h;
                    }
                }
                const bool found = (m & 1u) && jj == 0;  // else the mask holds fewer bits than counted
                const uint32_t we = ie & 0xFFu, mul = (ie >> 8) & 0xFFFu;
                const uint32_t row = (bit * mul) >> 11;
                uint32_t key = found ? ke + row * se + (bit - row * we) : 0xFFFFFFFFu;
                if (F > 1 && found)
                    key |= tile_mask<F>(ef, (int)(rx & 0xFFFFu) + (int)(bit - row * we), (int)(rx >> 16) + (int)row,
                                        ts / F);
                pkeys[q] = key;
                put_val(q, re);
            }
        }
    }
    if (tt > 0 && !coop && area > kMaskTiles) {
        // exact mode (no test): every tile of a large rectangle
        unsigned long long o = o0;
        for (int ty = ty0; ty < ty1 && o < oend; ++ty)
            for (int tx = tx0; tx < tx1 && o < oend; ++tx, ++o)
                if (o < ucap) {
                    pkeys[o] = (uint32_t)rc.z + (uint32_t)ty * (uint32_t)rc.w + (uint32_t)tx;
                    put_val(o, r);
                }
    }
    FootRows fr{};
    if (coop) fr = make_footrows(rec[3 * r], rec[3 * r + 1], rec[3 * r + 1].z - log2_alpha_min);
    for (unsigned big = __ballot_sync(0xffffffffu, coop); big; big &= big - 1) {
        const int src = __ffs(big) - 1;
        FootRows bf;
        bf.qx = __shfl_sync(0xffffffffu, fr.qx, src);
        bf.qy = __shfl_sync(0xffffffffu, fr.qy, src);
        bf.A = __shfl_sync(0xffffffffu, fr.A, src);
        bf.B = __shfl_sync(0xffffffffu, fr.B, src);
        bf.det = __shfl_sync(0xffffffffu, fr.det, src);
        bf.invA = __shfl_sync(0xffffffffu, fr.invA, src);
        bf.ymax = __shfl_sync(0xffffffffu, fr.ymax, src);
        bf.dyr = __shfl_sync(0xffffffffu, fr.dyr, src);
        bf.lim = __shfl_sync(0xffffffffu, fr.lim, src);
        const uint32_t br = __shfl_sync(0xffffffffu, r, src);
        const int rx = __shfl_sync(0xffffffffu, rc.x, src), ry = __shfl_sync(0xffffffffu, rc.y, src);
        const uint32_t bz = (uint32_t)__shfl_sync(0xffffffffu, rc.z, src);
        const uint32_t bwid = (uint32_t)__shfl_sync(0xffffffffu, rc.w, src);
        const unsigned long long bo0 = __shfl_sync(0xffffffffu, o0, src);
        const unsigned long long boend = __shfl_sync(0xffffffffu, oend, src);
        const int bx0 = rx & 0xFFFF, by0 = (rx >> 16) & 0xFFFF, bx1 = ry & 0xFFFF, by1 = (ry >> 16) & 0xFFFF;
        unsigned long long o = bo0;
        for (int row0 = by0; row0 < by1; row0 += 32) {
            // lane l finds the span of tile row row0 + l; the rows' runs then
            // fill [o, o + total) and the warp writes that range together
            // (lane l positions l, l + 32, ...), each position's row found
            // by a binary search over the lanes' run starts as in the mask path
            const int ty = row0 + lane;
            int a = 0, b = -1;
            if (ty < by1 && !footrows_span(bf, ty, ts, bx0, bx1, &a, &b)) b = -1;
            uint32_t total;
            const uint32_t cnt = (uint32_t)(b - a + 1);
            const uint32_t start = warp_exclusive_scan(cnt, &total);
            for (uint32_t p0 = 0; p0 < total; p0 += 32) {
                const uint32_t pr = p0 + (uint32_t)lane;
                int e = 0;
#pragma unroll
                for (int st = 16; st >= 1; st >>= 1) {
                    const uint32_t sc = __shfl_sync(0xffffffffu, start, e + st);
                    if (sc <= pr) e += st;
                }
                const int ae = __shfl_sync(0xffffffffu, a, e);
                const uint32_t se = __shfl_sync(0xffffffffu, start, e);
                const unsigned long long q = o + pr;
                if (pr < total && q < boend && q < ucap) {
                    uint32_t key = bz + (uint32_t)(row0 + e) * bwid + (uint32_t)ae + (pr - se);
                    if (F > 1) key |= tile_mask<F>(bf, ae + (int)(pr - se), row0 + e, ts / F);
                    pkeys[q] = key;
                    put_val(q, br);
                }
            }
            o += total;
        }
        for (unsigned long long q = o + lane; q < boend; q += 32)
            if (q < ucap) {
                pkeys[q] = 0xFFFFFFFFu;
                put_val(q, br);
            }
    }
}

// Longest-list-first tile order for the compositing launches: key = 255 -
// (a log-scale code of the list length: 16 steps per octave), one stable
// 8-bit radix pass, so CTAs of long lists are dispatched first and short ones
// fill the tail.
// When the last compositing forward keyed the same number of tiles by their
// walk depth (counters[kCtrOrderTiles]), those keys stay: the depth a tile's
// pixels reached in the last iteration predicts its work better than its list
// length.  Either way every tile gets a key and its index, so the sort yields
// a permutation of the tiles whatever the keys hold.
__global__ void k_tile_keys(const uint2* __restrict__ ranges, int n_tiles, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, const unsigned long long* __restrict__ counters) {
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tiles) return;
    if (counters[kCtrOrderTiles] != (unsigned long long)n_tiles) {
        const uint2 rg = ranges[i];
        keys[i] = tile_order_key(rg.y - rg.x);
    }
    vals[i] = (uint32_t)i;
}

// Tile ranges over the sorted pair keys: a tile's list starts where its key
// differs from the previous one and ends where it differs from the next.
// Each thread takes 4 consecutive keys in one 16-byte load (the key buffer is
// 256-byte aligned); the neighbours across threads come by warp shuffles.
__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ keys, long long cap,
                                                const unsigned long long* __restrict__ n_dev, uint32_t n_tiles,
                                                uint32_t key_bits_mask, uint2* __restrict__ ranges) {
    pdl_wait();
    pdl_trigger();
    const unsigned long long n = clamp_n((unsigned long long)cap, n_dev);
    const unsigned long long n4 = (n + 3) / 4;
    const uint4* __restrict__ k4 = reinterpret_cast<const uint4*>(keys);
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of rounds (shuffles need all 32);
    // each round takes two chunks of 32 x 4 keys, both loaded first
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x * 2 + (threadIdx.x & ~31u) * 2; base < n4;
         base += stride * 2) {
        uint32_t v[2][4];
        uint32_t pv[2], nx[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const unsigned long long g = base + 32 * c + lane;
            const unsigned long long j0 = 4 * g;
            v[c][0] = v[c][1] = v[c][2] = v[c][3] = 0xFFFFFFFFu;
            if (j0 + 3 < n) {
                const uint4 q = k4[g];
                v[c][0] = q.x & key_bits_mask; v[c][1] = q.y & key_bits_mask;
                v[c][2] = q.z & key_bits_mask; v[c][3] = q.w & key_bits_mask;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (j0 + i < n) v[c][i] = keys[j0 + i] & key_bits_mask;
            }
            pv[c] = 0xFFFFFFFFu;
            nx[c] = 0xFFFFFFFFu;
            if (lane == 0 && j0 > 0 && j0 - 1 < n) pv[c] = keys[j0 - 1] & key_bits_mask;
            if (lane == 31 && j0 + 4 < n) nx[c] = keys[j0 + 4] & key_bits_mask;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const unsigned long long g = base + 32 * c + lane;
            const unsigned long long j0 = 4 * g;
            uint32_t prev = __shfl_up_sync(0xffffffffu, v[c][3], 1);
            uint32_t next = __shfl_down_sync(0xffffffffu, v[c][0], 1);
            if (lane == 0) prev = pv[c];
            if (lane == 31) next = nx[c];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const unsigned long long j = j0 + i;
                const uint32_t k = v[c][i];
                if (j >= n || k >= n_tiles) continue;
                const uint32_t p = i > 0 ? v[c][i - 1] : prev;
                const uint32_t x = i < 3 ? v[c][i + 1] : next;
                if (j == 0 || p != k) ranges[k].x = (uint32_t)j;
                if (j + 1 == n || x != k) ranges[k].y = (uint32_t)(j + 1);
            }
        }
    }
}

// Split of the bin lists into tile lists.  A bin is an F x F block of
// compositing tiles (F = 2 or 4); its list is front to back.  First, one
// thread per sorted pair finds which of its bin's tiles the record's
// alpha >= alpha_min footprint reaches (per tile row of the bin, the columns
// footrows_span gives: the binning's own test at the tile size) and stores
// that mask over the pair's key (the bin id, no longer needed once the bin
// ranges are taken).  Then one warp per bin walks the masks in list order
// and appends each record to the lists of the tiles in its mask (ballot and
// prefix count per tile), so every tile list stays front to back and holds
// the records binning at the tile size lists.  Tile s of the bin (row-major)
// writes its list at F^2 start + s len, where [start, start + len) is the
// bin's range (room for every record of the bin), and its range goes to
// ranges[tile]; tiles past the image edge get none.
__device__ __forceinline__ int refine_view(const RefineGeom& g, int bin) {
    int lo = 0, hi = g.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.bin_off[mid] <= bin) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One block per bin, each warp taking TW of the bin's F^2 tiles.  The bin's
// list goes through shared memory in rounds of one record per thread (the
// next round's loads in flight while the current one is split); a warp reads
// the round's masks 32 at a time and appends, for each of its tiles, the
// records whose mask has the tile's bit to the tile's list, in list order
// (ballot and prefix count).  The masks sit above the bin ids in the keys.
constexpr int kSplitTilesPerWarp = 1;  // (4 per warp, one load of the masks for four tiles, measured slower)
template <int F>
__global__ void __launch_bounds__(32 * F * F / kSplitTilesPerWarp) k_refine_split(
    const __grid_constant__ RefineGeom g, const uint2* __restrict__ bin_ranges, const uint32_t* __restrict__ keys,
    const uint32_t* __restrict__ vals, long long cap, uint32_t* __restrict__ rvals, uint2* __restrict__ ranges) {
    pdl_wait();
    pdl_trigger();
    constexpr int S = F * F;
    constexpr int TW = kSplitTilesPerWarp < S ? kSplitTilesPerWarp : S;
    constexpr int NW = S / TW;
    constexpr int R = 32 * NW;  // records per round
    __shared__ uint32_t s_m[2][R], s_r[2][R];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int bin = blockIdx.x;
    const int v = refine_view(g, bin);
    const int lb = bin - g.bin_off[v];
    const int by = lb / g.bins_x[v], bx = lb - by * g.bins_x[v];
    uint2 rg = bin_ranges[bin];
    if (!(rg.x <= rg.y && (long long)rg.y <= cap)) rg.y = rg.x;
    const uint32_t len = rg.y - rg.x;
    const uint32_t* mk = keys + rg.x;
    const uint32_t* vl = vals + rg.x;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t pos[TW];
#pragma unroll
    for (int k = 0; k < TW; ++k) pos[k] = 0u;
    uint32_t nm = 0, nr = 0;  // this thread's record of the next round
    if ((uint32_t)threadIdx.x < len) {
        nm = mk[threadIdx.x];
        nr = vl[threadIdx.x];
    }
    int buf = 0;
    for (uint32_t c0 = 0; c0 < len; c0 += R, buf ^= 1) {
        s_m[buf][threadIdx.x] = nm;
        s_r[buf][threadIdx.x] = nr;
        __syncthreads();
        const uint32_t i = c0 + R + threadIdx.x;
        nm = i < len ? mk[i] : 0u;
        nr = i < len ? vl[i] : 0u;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const uint32_t m = s_m[buf][32 * j + lane] >> (32 - S + w * TW);  // 0 past the end of the list
            const uint32_t rr = s_r[buf][32 * j + lane];
#pragma unroll
            for (int k = 0; k < TW; ++k) {
                const bool h = (m >> k) & 1u;
                const uint32_t b = __ballot_sync(0xffffffffu, h);
                const int t = w * TW + k;
                if (h) rvals[rg.x * (uint32_t)S + (uint32_t)t * len + pos[k] + __popc(b & lt_mask)] = rr;
                pos[k] += __popc(b);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < TW; ++k) {
        const int t = w * TW + k;
        const int tx = bx * F + t % F, ty = by * F + t / F;
        if (lane == 0 && tx < g.tiles_x[v] && ty < g.tiles_y[v]) {  // past the image edge: no tile
            const uint32_t q0 = rg.x * (uint32_t)S + (uint32_t)t * len;
            ranges[g.tile_off[v] + ty * g.tiles_x[v] + tx] = make_uint2(q0, q0 + pos[k]);
        }
    }
}

// Deterministic backward: after the tile sort the pair values are emission
// indices.  Each place p of the tile lists gets its pair's record back, and
// pair_inv records where each emission index went (~0 for a pair listed in
// no tile), so that a record's partials can later be found in the order of
// its tiles (its pairs are contiguous in emission order).
__global__ void __launch_bounds__(256) k_pair_places(const uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                     const uint32_t* __restrict__ pair_rec,
                                                     uint32_t* __restrict__ pair_inv, long long cap,
                                                     const unsigned long long* __restrict__ n_dev,
                                                     uint32_t n_tiles) {
    pdl_wait();
    pdl_trigger();
    const unsigned long long n = clamp_n((unsigned long long)cap, n_dev);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const uint32_t e = vals[p];
        if (e >= n) continue;  // cannot happen: every emitted value is an index below n
        vals[p] = pair_rec[e];
        pair_inv[e] = keys[p] < n_tiles ? (uint32_t)p : 0xFFFFFFFFu;
    }
}

__global__ void k_set_u32(unsigned int* p, unsigned int v) {
    pdl_wait();
    pdl_trigger(); *p = v; }

}  // namespace

size_t selftest_wait_scratch_bytes() { return sizeof(uint32_t) * 2 * kU32ScanChunk + 4 * sizeof(unsigned long long); }

// The scan's bounded wait made to expire: two chunks whose ticket starts at 1,
// so the one block takes chunk 1 and waits for chunk 0's flag, which nothing
// sets; after its poll limit it latches GS_ERR_TIMEOUT and finishes.
cudaError_t launch_selftest_wait(void* scratch, unsigned int* status, cudaStream_t s) {
    uint32_t* a = static_cast<uint32_t*>(scratch);
    unsigned long long* flags = reinterpret_cast<unsigned long long*>(a + 2 * kU32ScanChunk);
    cudaError_t e = cudaMemsetAsync(scratch, 0, selftest_wait_scratch_bytes(), s);
    if (e != cudaSuccess) return e;
    pdl_launch(k_set_u32, 1, 1, 0, s, reinterpret_cast<unsigned int*>(flags + 2), 1u);
    pdl_launch(k_u32_scan_lookback, 1, 1024, 0, s, a, 2 * kU32ScanChunk, flags, reinterpret_cast<unsigned int*>(flags + 2),
                                          status);
    return cudaGetLastError();
}

namespace {

int radix_blocks(unsigned long long n_host) {
    return (int)((n_host + kRTile - 1) / kRTile);
}

// Sorts (key, value) pairs on the low key_bits bits of the keys (of their
// depth-key map when key_range is set), ping-ponging between buffer 0 and 1;
// *result_buf receives the buffer holding the result.
cudaError_t radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const WsPtrs& ws,
                       unsigned long long n_host, const unsigned long long* n_dev, int key_bits,
                       int* result_buf, unsigned int* status, cudaStream_t s, Prof& pf,
                       const unsigned long long* key_range = nullptr) {
    const int passes = key_bits <= 0 ? 0 : (key_bits + 7) / 8;
    const int dbits = passes ? (key_bits + passes - 1) / passes : 0;
    const int nblk = radix_blocks(n_host);
    const long long nh = 256ll * nblk;
    const int nparts = (int)((nh + kU32ScanChunk - 1) / kU32ScanChunk);
    uint32_t* kin = k0;
    uint32_t* vin = v0;
    uint32_t* kout = k1;
    uint32_t* vout = v1;
    for (int p = 0; p < passes && nblk > 0; ++p) {
        const int shift = p * dbits;
        const int bits = key_bits - shift < dbits ? key_bits - shift : dbits;
        // flags of the nparts chunks, then the ticket, zeroed by the upsweep for the look-back scan
        unsigned long long* flags = reinterpret_cast<unsigned long long*>(ws.hist_part);
        const bool single = nh <= kU32SingleScanMax;
        if (key_range)
            pdl_launch(k_radix_upsweep<true>, nblk, kRadixThreads, 0, s, kin, n_host, n_dev, shift, bits, ws.hist,
                       flags, single ? 0 : nparts + 1, key_range);
        else
            pdl_launch(k_radix_upsweep<false>, nblk, kRadixThreads, 0, s, kin, n_host, n_dev, shift, bits, ws.hist,
                       flags, single ? 0 : nparts + 1, key_range);
        if (single) {
            pdl_launch(k_u32_scan_single, 1, 1024, 0, s, ws.hist, nh);
            pf.count(3);
        } else {
            pf.count(3);
            pdl_launch(k_u32_scan_lookback, nparts, 1024, 0, s, ws.hist, nh, flags,
                                                        reinterpret_cast<unsigned int*>(flags + nparts), status);
        }
        if (key_range)
            pdl_launch(k_radix_downsweep<true>, nblk, kRadixThreads, 0, s, kin, vin, kout, vout, n_host, n_dev, shift,
                       bits, ws.hist, key_range);
        else
            pdl_launch(k_radix_downsweep<false>, nblk, kRadixThreads, 0, s, kin, vin, kout, vout, n_host, n_dev, shift,
                       bits, ws.hist, key_range);
        uint32_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    *result_buf = passes % 2;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_bin(const BatchParam& bp, WsPtrs& ws, unsigned int* status,
                       unsigned long long* status_pairs, cudaStream_t s, Prof& pf, const RefineGeom* geom,
                       int n_tiles) {
    const long long M = bp.total_recs;
    cudaError_t e;
    if (M <= 0) return cudaSuccess;
    // 1. front-to-back order of records by the 64-bit double-float depth key:
    //    a stable radix sort on the 24-bit map of the high word (3 passes from
    //    dhi / dvals[1], the record indices the projection wrote, to dkeys[1] /
    //    dvals[0]), then the runs of equal mapped keys by (high word, low
    //    word, record)
    int pi = pf.begin(GS_KF_DEPTH_SORT, s, 1);  // the fix-up; radix_sort counts its own launches
    int dbuf = 0;
    const unsigned long long* key_range = ws.counters;
    e = radix_sort(ws.dhi, ws.dvals[1], ws.dkeys[1], ws.dvals[0], ws, (unsigned long long)M, nullptr, 24, &dbuf,
                   status, s, pf, key_range);
    if (e != cudaSuccess) return e;
    if (dbuf != 1) return cudaErrorInvalidValue;  // three passes end in the second buffers
    const int nb = (int)((M + kScanChunk - 1) / kScanChunk);
    pdl_launch(k_depth_fixup, (unsigned)((M + 255) / 256), 256, 0, s, ws.dkeys[1], ws.dvals[0], ws.dkeys[0], M,
               ws.scan_part, nb + 1, key_range);
    pf.end(pi, s);
    const uint32_t* order = ws.dvals[0];
    // 2. exclusive scan of tiles-touched in that order (single pass; flags zeroed by the fix-up)
    pi = pf.begin(GS_KF_TILE_SCAN, s, 1);
    pdl_launch(k_scan_offsets, nb, kScanThreads, 0, s, order, ws.tiles_touched, M, ws.scan_part, nb, ws.offsets,
               ws.counters, ws.cap, status, status_pairs);
    pf.end(pi, s);
    // 3. expand records into (tile, record) pairs; with bins of F x F tiles
    //    the keys also carry the tile masks of the later split
    if (ws.refine > 1 && !geom) return cudaErrorInvalidValue;
    const int F = geom ? ws.refine : 1;
    if (F != 1 && F != 2 && F != 4) return cudaErrorInvalidValue;
    pi = pf.begin(GS_KF_EMIT, s);
    {
        const unsigned eg = (unsigned)((M + 255) / 256);
        if (F == 1)
            pdl_launch(k_emit<1>, eg, 256, 0, s, order, ws.rect, ws.rec, ws.offsets, M,
                       ws.cap, bp.tile_size, ws.log2_alpha_min, ws.pkeys[0], ws.pvals[0], ws.pair_rec);
        else if (F == 2)
            pdl_launch(k_emit<2>, eg, 256, 0, s, order, ws.rect, ws.rec, ws.offsets, M,
                       ws.cap, bp.tile_size, ws.log2_alpha_min, ws.pkeys[0], ws.pvals[0], ws.pair_rec);
        else
            pdl_launch(k_emit<4>, eg, 256, 0, s, order, ws.rect, ws.rec, ws.offsets, M,
                       ws.cap, bp.tile_size, ws.log2_alpha_min, ws.pkeys[0], ws.pvals[0], ws.pair_rec);
    }
    pf.end(pi, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // 4. stable sort of pairs by global tile id
    int tile_bits = 1;
    while ((1ll << tile_bits) < (long long)bp.total_tiles) ++tile_bits;
    int pbuf = 0;
    pi = pf.begin(GS_KF_TILE_SORT, s, 0);
    e = radix_sort(ws.pkeys[0], ws.pvals[0], ws.pkeys[1], ws.pvals[1], ws, (unsigned long long)ws.cap,
                   ws.counters, tile_bits, &pbuf, status, s, pf);
    if (e == cudaSuccess && ws.pair_rec) {
        pf.count(1);
        pdl_launch(k_pair_places, 1184, 256, 0, s, ws.pkeys[pbuf], ws.pvals[pbuf], ws.pair_rec, ws.pair_inv, ws.cap,
                   ws.counters, (uint32_t)bp.total_tiles);
    }
    pf.end(pi, s);
    if (e != cudaSuccess) return e;
    ws.sorted_buf = pbuf;
    // 5. per-bin [start, end) (the keys' bin ids below their tile masks)
    if (F == 1) n_tiles = bp.total_tiles;
    uint2* bin_ranges = F > 1 ? ws.ranges_bin : ws.ranges;
    pi = pf.begin(GS_KF_RANGES, s, 2);  // memset, ranges
    e = cudaMemsetAsync(bin_ranges, 0, sizeof(uint2) * (size_t)bp.total_tiles, s);
    if (e != cudaSuccess) return e;
    pdl_launch(k_ranges, 1184, 256, 0, s, ws.pkeys[pbuf], ws.cap, ws.counters, (uint32_t)bp.total_tiles,
               F == 1 ? 0xFFFFFFFFu : (1u << (32 - F * F)) - 1u, bin_ranges);
    pf.end(pi, s);
    // 6. bins of F x F tiles: each bin's list split into its tiles' lists
    //    (every tile's range written, so no clearing)
    if (F > 1) {
        pi = pf.begin(GS_KF_REFINE, s, 1);
        if (F == 2)
            pdl_launch(k_refine_split<2>, bp.total_tiles, 32 * 4 / kSplitTilesPerWarp, 0, s, *geom, bin_ranges, ws.pkeys[pbuf],
                       ws.pvals[pbuf], ws.cap, ws.rvals, ws.ranges);
        else
            pdl_launch(k_refine_split<4>, bp.total_tiles, 32 * 16 / kSplitTilesPerWarp, 0, s, *geom, bin_ranges, ws.pkeys[pbuf],
                       ws.pvals[pbuf], ws.cap, ws.rvals, ws.ranges);
        pf.end(pi, s);
    }
    // 7. longest-list-first order of the compositing tiles
    pi = pf.begin(GS_KF_RANGES, s, 1);  // keys; radix_sort counts its own launches
    pdl_launch(k_tile_keys, (n_tiles + 255) / 256, 256, 0, s, ws.ranges, n_tiles, ws.okeys[0], ws.ovals[0],
               ws.counters);
    int obuf = 0;
    e = radix_sort(ws.okeys[0], ws.ovals[0], ws.okeys[1], ws.ovals[1], ws, (unsigned long long)n_tiles,
                   nullptr, 8, &obuf, status, s, pf);
    pf.end(pi, s);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_tile_order(const WsPtrs& ws, int n_tiles, unsigned int* status, cudaStream_t s, Prof& pf) {
    if (n_tiles <= 0) return cudaSuccess;
    const int pi = pf.begin(GS_KF_RANGES, s, 0);  // radix_sort counts its own launches
    int obuf = 0;
    cudaError_t e = radix_sort(ws.okeys[0], ws.ovals[0], ws.okeys[1], ws.ovals[1], ws, (unsigned long long)n_tiles,
                               nullptr, 8, &obuf, status, s, pf);
    pf.end(pi, s);
    if (e == cudaSuccess && obuf != 1) return cudaErrorInvalidValue;
    return e;
}

}  // namespace gsb
