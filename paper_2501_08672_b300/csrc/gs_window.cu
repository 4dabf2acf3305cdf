// Sliding-window maintenance on the device (Sec. II-C) and the SH0
// initialisation of new Gaussians (Sec. II-B.2).
//
// Step 2 (deletion and compaction): with n_keep survivors, the k-th hole
// (deleted row below n_keep, ascending) receives the k-th survivor at or
// above n_keep counted from the rear (descending), so survivors below n_keep
// never move and the window stays contiguous in [0, n_keep).  Holes and
// movers both follow from one survivor prefix S(i) (survivors before row i):
// a hole i < n_keep has rank i - S(i), a mover i >= n_keep rank
// S(i) - S(n_keep).  S is scanned in three phases (block totals, one-block
// scan of the totals that also yields n_keep and S(n_keep), block-local
// scan), all counts in device memory.  Every mover's source row is at or
// above n_keep and every destination below it, so the row copies do not
// overlap.
//
// SH0 initialisation: the colour of a new Gaussian is the bilinear
// interpolation of the camera image at its projected mean (pixel (u, v)
// sampled at (u + 0.5, v + 0.5), the four neighbours weighted by the areas of
// the opposite sub-rectangles), and k0 = (c - 0.5) / C0 so that the degree-0
// colour reproduces it; higher orders start at 0.
#include "gs_internal.cuh"

namespace gsb {

namespace {

constexpr int kWinThreads = 1024;
constexpr int kMaxCols = 32;

// The columns, by value as a kernel parameter (no host-to-device copy).
struct ColTable {
    uint32_t* ptr[kMaxCols];
    int words[kMaxCols];
    int n;
};
constexpr int kWinItems = 4;
constexpr int kWinChunk = kWinThreads * kWinItems;

// Exclusive scan of one value per thread over the block; *total receives the block sum.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* total) {
    __shared__ unsigned s_w[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned y = lane < nw ? s_w[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    *total = s_w[(blockDim.x >> 5) - 1];
    const unsigned wprefix = w > 0 ? s_w[w - 1] : 0u;
    __syncthreads();
    return wprefix + x - v;
}

__device__ __forceinline__ unsigned keep_count(const uint8_t* keep, long long base, long long end) {
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kWinItems; ++k)
        if (base + k < end) s += keep[base + k] != 0;
    return s;
}

// Survivors per block of kWinChunk rows.
__global__ void __launch_bounds__(kWinThreads) k_win_reduce(const uint8_t* __restrict__ keep, long long n,
                                                            unsigned* __restrict__ part) {
    pdl_wait();
    pdl_trigger();
    const long long base = (long long)blockIdx.x * kWinChunk + (long long)threadIdx.x * kWinItems;
    unsigned total;
    block_exclusive_scan(keep_count(keep, base, n), &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: exclusive scan of the block survivor counts (part becomes the
// survivor prefix S at each block start), n_keep = the grand total, and
// S(n_keep), the survivors below n_keep, counted in the block holding row
// n_keep; movers = holes = n_keep - S(n_keep).
__global__ void __launch_bounds__(1024) k_win_top(const uint8_t* __restrict__ keep, long long n, unsigned* part,
                                                  int nparts, long long* n_keep_out, long long* counts) {
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s[1024];
    const int t = threadIdx.x;
    const int per = (nparts + 1023) / 1024;
    const int b0 = t * per;
    unsigned long long sum = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nparts) sum += part[b0 + k];
    s[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned long long v = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    unsigned long long run = s[t] - sum;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nparts) {
            const unsigned v = part[b0 + k];
            part[b0 + k] = (unsigned)run;
            run += v;
        }
    const long long nk = (long long)s[1023];
    __syncthreads();  // part[] rewritten before the read below
    const long long blk = nk / kWinChunk;
    unsigned below = 0;
    if (blk < nparts) below = keep_count(keep, blk * kWinChunk + (long long)t * kWinItems, nk);
    unsigned tot;
    block_exclusive_scan(below, &tot);
    if (t == 0) {
        const long long snk = (blk < nparts ? (long long)part[blk] : nk) + (blk < nparts ? (long long)tot : 0ll);
        *n_keep_out = nk;
        counts[0] = snk;       // survivors below n_keep
        counts[1] = nk - snk;  // holes = movers
    }
}

// Ranks from the survivor prefix S(i) (survivors before row i): a removed
// row i has rank i - S(i) among all removed rows (ascending), so the first
// n_movers entries of that list are the holes below n_keep; a mover
// i >= n_keep has rank S(i) - S(n_keep) among the movers (ascending);
// moved_from[r] = r for the survivors below n_keep.  leaving_rows (optional)
// receives the removed rows' list too.
__global__ void __launch_bounds__(kWinThreads) k_win_rank(const uint8_t* __restrict__ keep, long long n,
                                                          const long long* __restrict__ n_keep,
                                                          const unsigned* __restrict__ part,
                                                          const long long* __restrict__ counts,
                                                          int32_t* __restrict__ holes_list,
                                                          int32_t* __restrict__ movers_asc,
                                                          int32_t* __restrict__ moved_from,
                                                          int32_t* __restrict__ leaving_rows) {
    pdl_wait();
    pdl_trigger();
    const long long base = (long long)blockIdx.x * kWinChunk + (long long)threadIdx.x * kWinItems;
    bool f[kWinItems];
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < kWinItems; ++k) {
        f[k] = base + k < n && keep[base + k] != 0;
        c += f[k];
    }
    unsigned total;
    long long S = (long long)part[blockIdx.x] + block_exclusive_scan(c, &total);
    const long long nk = *n_keep, snk = counts[0];
#pragma unroll
    for (int k = 0; k < kWinItems; ++k) {
        const long long i = base + k;
        if (i >= n) break;
        if (!f[k]) {
            holes_list[i - S] = (int32_t)i;
            if (leaving_rows) leaving_rows[i - S] = (int32_t)i;
        } else if (i < nk) {
            if (moved_from) moved_from[i] = (int32_t)i;
        } else {
            movers_asc[S - snk] = (int32_t)i;
        }
        S += f[k];
    }
}

// Row copies by warps.  A warp holds up to 32 entries (lane e: source row
// s_row, destination row d_row, d_row < 0 = no entry) and copies every column
// of those rows word-parallel: word w of a column's chunk is word w % words of
// entry w / words, so neighbouring lanes touch neighbouring words of a row and
// the rows of neighbouring entries; eight words per lane are in flight.
constexpr int kCopyThreads = 256;
constexpr int kCopyUnroll = 8;
constexpr int kCopyBlocksPerSM = 4;

__device__ __forceinline__ void warp_copy_rows(const ColTable& from, const ColTable& to, int32_t s_row,
                                               int32_t d_row) {
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < from.n; ++c) {
        const int words = from.words[c];
        // (w + 0.5) / words is at least 1 / (2 words) from an integer and below
        // 32, so the FP32 quotient truncates to w / words exactly.
        const float inv = 1.f / (float)words;
        const int total = 32 * words;
        const uint32_t* __restrict__ f = from.ptr[c];
        uint32_t* __restrict__ t = to.ptr[c];
        if (!t) continue;  // a column the caller does not want (warp-uniform)
        for (int w0 = 0; w0 < total; w0 += 32 * kCopyUnroll) {
            uint32_t val[kCopyUnroll];
            long long dpos[kCopyUnroll];
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u) {
                const int w = w0 + u * 32 + lane;
                const int e = min(__float2int_rz(((float)w + 0.5f) * inv), 31);
                const int k = w - e * words;
                const int32_t sr = __shfl_sync(0xffffffffu, s_row, e);
                const int32_t dr = __shfl_sync(0xffffffffu, d_row, e);
                const bool ok = w < total && dr >= 0;
                dpos[u] = ok ? (long long)dr * words + k : -1ll;
                val[u] = ok ? f[(long long)sr * words + k] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kCopyUnroll; ++u)
                if (dpos[u] >= 0) t[dpos[u]] = val[u];
        }
    }
}

// Mover of ascending rank q moves into the hole of rank n_movers - 1 - q; a
// warp takes 32 consecutive ranks (grid-stride over the rank chunks).
__global__ void __launch_bounds__(kCopyThreads, kCopyBlocksPerSM) k_win_move(const ColTable cols, long long n,
                                                           const long long* __restrict__ counts,
                                                           const int32_t* __restrict__ holes_list,
                                                           const int32_t* __restrict__ movers_asc,
                                                           int32_t* __restrict__ moved_from) {
    pdl_wait();
    pdl_trigger();
    const long long n_movers = min(counts[1], n);
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * kCopyThreads + threadIdx.x) >> 5;
    const long long n_warps = (long long)gridDim.x * (kCopyThreads / 32);
    for (long long q0 = warp * 32; q0 < n_movers; q0 += n_warps * 32) {
        const long long q = q0 + lane;
        int32_t src = 0, dst = -1;
        if (q < n_movers) {
            src = movers_asc[q];
            dst = holes_list[n_movers - 1 - q];
            if (moved_from) moved_from[dst] = src;
        }
        warp_copy_rows(cols, cols, src, dst);
    }
}

// Rows idx[0..m) of each source column, gathered contiguously into dst
// (columns whose destination is NULL are skipped).  With n_keep set, m is
// n - *n_keep (the rows removed by the compaction), read on the device.
__global__ void __launch_bounds__(kCopyThreads, kCopyBlocksPerSM) k_win_gather(const ColTable src, const ColTable dst,
                                                             const int32_t* __restrict__ idx, long long m,
                                                             long long n, const long long* __restrict__ n_keep) {
    pdl_wait();
    pdl_trigger();
    if (n_keep) m = min(max(n - *n_keep, 0ll), m);
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * kCopyThreads + threadIdx.x) >> 5;
    const long long n_warps = (long long)gridDim.x * (kCopyThreads / 32);
    for (long long j0 = warp * 32; j0 < m; j0 += n_warps * 32) {
        const long long j = j0 + lane;
        int32_t r = 0, d = -1;
        if (j < m) {
            r = idx[j];
            // validated on the host for host-known indices; guards the read
            if (r >= 0 && r < n) d = (int32_t)j;
            else r = 0;
        }
        warp_copy_rows(src, dst, r, d);
    }
}

// Rows [a, b) of every column set to zero (contiguous words per column).
__global__ void __launch_bounds__(kCopyThreads) k_win_clear(const ColTable cols, long long a, long long b) {
    pdl_wait();
    pdl_trigger();
    const long long t0 = (long long)blockIdx.x * kCopyThreads + threadIdx.x;
    const long long stride = (long long)gridDim.x * kCopyThreads;
    for (int c = 0; c < cols.n; ++c) {
        const int words = cols.words[c];
        uint32_t* p = cols.ptr[c] + a * words;
        const long long cnt = (b - a) * words;
        for (long long i = t0; i < cnt; i += stride) p[i] = 0u;
    }
}

// One thread per new Gaussian for the colour; the warp's 32 rows of SH
// coefficients are one contiguous range, written by the whole warp in
// coalesced stores (lane l takes positions l, l + 32, ...; the k0 values
// come from their rows' lanes by shuffles).
template <int D>
__global__ void __launch_bounds__(256) k_sh_init(const ViewParam V, const float* __restrict__ means,
                                                 const float* __restrict__ image, long long begin, long long end,
                                                 float z_near, float* __restrict__ sh) {
    pdl_wait();
    pdl_trigger();
    constexpr int K3 = 3 * (D + 1) * (D + 1);  // floats per row
    const long long i0 = begin + (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    if (i0 >= end) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    const long long i = i0 + lane;
    const bool live = i < end;
    const long long ii = live ? i : i0;
    const float mx = means[3 * ii], my = means[3 * ii + 1], mz = means[3 * ii + 2];
    const float x = V.R[0] * mx + V.R[1] * my + V.R[2] * mz + V.t[0];
    const float y = V.R[3] * mx + V.R[4] * my + V.R[5] * mz + V.t[1];
    const float z = V.R[6] * mx + V.R[7] * my + V.R[8] * mz + V.t[2];
    float c[3] = {0.5f, 0.5f, 0.5f};
    if (z > z_near) {
        const float u = V.fx * x / z + V.cx - 0.5f;  // continuous pixel coordinate of pixel centres
        const float v = V.fy * y / z + V.cy - 0.5f;
        if (u > -0.5f && v > -0.5f && u < (float)V.W - 0.5f && v < (float)V.H - 0.5f) {
            const float uc = fminf(fmaxf(u, 0.f), (float)(V.W - 1));
            const float vc = fminf(fmaxf(v, 0.f), (float)(V.H - 1));
            const int u0 = min((int)floorf(uc), V.W - 1), v0 = min((int)floorf(vc), V.H - 1);
            const int u1 = min(u0 + 1, V.W - 1), v1 = min(v0 + 1, V.H - 1);
            const float a = uc - (float)u0, b = vc - (float)v0;
            const long long hw = (long long)V.W * V.H;
            for (int ch = 0; ch < 3; ++ch) {
                const float* im = image + ch * hw;
                const float c00 = im[(long long)v0 * V.W + u0], c01 = im[(long long)v0 * V.W + u1];
                const float c10 = im[(long long)v1 * V.W + u0], c11 = im[(long long)v1 * V.W + u1];
                c[ch] = (1.f - a) * (1.f - b) * c00 + a * (1.f - b) * c01 + (1.f - a) * b * c10 + a * b * c11;
            }
        }
    }
    constexpr float kInvShC0 = 3.5449077018110318f;  // 2 sqrt(pi) = 1 / C0
    const float k0[3] = {(c[0] - 0.5f) * kInvShC0, (c[1] - 0.5f) * kInvShC0, (c[2] - 0.5f) * kInvShC0};
    const long long rows = end - i0 < 32 ? end - i0 : 32;
    float* o = sh + (size_t)i0 * K3;
#pragma unroll
    for (int e0 = 0; e0 < 32 * K3; e0 += 32) {
        const int e = e0 + lane;
        const int row = e / K3, ch = e - row * K3;
        const float v0 = __shfl_sync(0xffffffffu, k0[0], row);
        const float v1 = __shfl_sync(0xffffffffu, k0[1], row);
        const float v2 = __shfl_sync(0xffffffffu, k0[2], row);
        if (row < rows) o[e] = ch == 0 ? v0 : ch == 1 ? v1 : ch == 2 ? v2 : 0.f;
    }
}

ColTable col_table(const gs_window_column* cols, int n_cols) {
    ColTable t{};
    t.n = n_cols;
    for (int c = 0; c < n_cols; ++c) {
        t.ptr[c] = static_cast<uint32_t*>(cols[c].ptr);
        t.words[c] = cols[c].bytes_per_gaussian / 4;
    }
    return t;
}

}  // namespace

int window_max_columns() { return kMaxCols; }

size_t window_scratch_bytes(long long n) {
    const long long nblk = (n + kWinChunk - 1) / kWinChunk;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    return al(sizeof(long long) * 2) + al(sizeof(unsigned) * (size_t)(nblk > 0 ? nblk : 1)) +
           al(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)) * 2;
}

// Grid of the row-copy kernels: one chunk of 32 rows per warp, at most the
// blocks one SM holds at once (up to 64 registers a thread) times the SMs,
// grid-stride beyond that.
unsigned copy_grid(long long rows, int sm_count) {
    const long long chunks = (rows + 31) / 32;
    const long long blocks = (chunks + kCopyThreads / 32 - 1) / (kCopyThreads / 32);
    const long long cap = (long long)(sm_count > 0 ? sm_count : 148) * kCopyBlocksPerSM;
    return (unsigned)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

cudaError_t launch_window_compact(const gs_window_column* cols_host, const gs_window_column* leave_dst, int n_cols,
                                  long long n, const uint8_t* keep, long long* n_keep_dev, int32_t* moved_from,
                                  int32_t* leaving_rows, void* scratch, int sm_count, cudaStream_t s, Prof& pf) {
    const long long nblk = (n + kWinChunk - 1) / kWinChunk;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char* p = static_cast<char*>(scratch);
    long long* counts = reinterpret_cast<long long*>(p);
    p += al(sizeof(long long) * 2);
    unsigned* part = reinterpret_cast<unsigned*>(p);
    p += al(sizeof(unsigned) * (size_t)(nblk > 0 ? nblk : 1));
    int32_t* holes_list = reinterpret_cast<int32_t*>(p);
    p += al(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* movers_asc = reinterpret_cast<int32_t*>(p);
    const ColTable cols = col_table(cols_host, n_cols);
    const int pi = pf.begin(GS_KF_WINDOW, s, leave_dst ? 5 : 4);
    pdl_launch(k_win_reduce, (unsigned)nblk, kWinThreads, 0, s, keep, n, part);
    pdl_launch(k_win_top, 1, 1024, 0, s, keep, n, part, (int)nblk, n_keep_dev, counts);
    pdl_launch(k_win_rank, (unsigned)nblk, kWinThreads, 0, s, keep, n, n_keep_dev, part, counts, holes_list, movers_asc,
                                                       moved_from, leaving_rows);
    if (leave_dst)  // Step 1 before the moves overwrite the holes
        pdl_launch(k_win_gather, copy_grid(n, sm_count), kCopyThreads, 0, s, cols, col_table(leave_dst, n_cols), holes_list,
                                                                      n, n, n_keep_dev);
    pdl_launch(k_win_move, copy_grid(n / 2, sm_count), kCopyThreads, 0, s, cols, n, counts, holes_list, movers_asc,
                                                                  moved_from);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_window_gather(const gs_window_column* src_host, const gs_window_column* dst_host, int n_cols,
                                 const int32_t* idx, long long m, long long n, int sm_count, cudaStream_t s,
                                 Prof& pf) {
    const int pi = pf.begin(GS_KF_WINDOW, s);
    if (m > 0)
        pdl_launch(k_win_gather, copy_grid(m, sm_count), kCopyThreads, 0, s, col_table(src_host, n_cols),
                                                                      col_table(dst_host, n_cols), idx, m, n, nullptr);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_window_clear(const gs_window_column* cols_host, int n_cols, long long begin, long long end,
                                int sm_count, cudaStream_t s, Prof& pf) {
    if (end <= begin) return cudaSuccess;
    const int pi = pf.begin(GS_KF_WINDOW, s);
    const ColTable cols = col_table(cols_host, n_cols);
    long long words = 0;
    for (int c = 0; c < n_cols; ++c) words += cols.words[c];
    pdl_launch(k_win_clear, copy_grid((end - begin) * words / 32, sm_count), kCopyThreads, 0, s, cols, begin, end);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_sh_init(const ViewParam& V, const float* means, const float* image, long long begin,
                           long long end, int sh_degree, float z_near, float* sh, cudaStream_t s, Prof& pf) {
    if (end <= begin) return cudaSuccess;
    const int pi = pf.begin(GS_KF_WINDOW, s);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    const unsigned grid = (unsigned)((end - begin + 255) / 256);
    switch (K) {
        case 1: pdl_launch(k_sh_init<0>, grid, 256, 0, s, V, means, image, begin, end, z_near, sh); break;
        case 4: pdl_launch(k_sh_init<1>, grid, 256, 0, s, V, means, image, begin, end, z_near, sh); break;
        case 9: pdl_launch(k_sh_init<2>, grid, 256, 0, s, V, means, image, begin, end, z_near, sh); break;
        default: pdl_launch(k_sh_init<3>, grid, 256, 0, s, V, means, image, begin, end, z_near, sh); break;
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
