// Sliding-window maintenance on the device (Sec. II-C) and the SH0
// initialisation of new Gaussians (Sec. II-B.2).
//
// Step 2 (deletion and compaction): with n_keep survivors, the k-th hole
// (deleted row below n_keep, ascending) receives the k-th survivor at or
// above n_keep counted from the rear (descending), so survivors below n_keep
// never move and the window stays contiguous in [0, n_keep).  Holes and
// movers are counted together: both exclusive prefix counts are packed in
// one 64-bit word (holes low, movers high) and scanned in three phases
// (block totals, one-block scan of the totals, block-local scan), all counts
// in device memory.  Every mover's source row is at or above n_keep and
// every destination below it, so the row copies do not overlap.
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

__device__ __forceinline__ unsigned long long block_exclusive_scan_u64(unsigned long long v,
                                                                       unsigned long long* total) {
    __shared__ unsigned long long s_w[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long y = lane < nw ? s_w[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        s_w[lane] = y;
    }
    __syncthreads();
    *total = s_w[(blockDim.x >> 5) - 1];
    const unsigned long long wprefix = w > 0 ? s_w[w - 1] : 0ull;
    __syncthreads();
    return wprefix + x - v;
}

// Per-row flags: survivors (phase "keep"), or hole | mover << 32 once n_keep is known.
__device__ __forceinline__ unsigned long long row_flags(const uint8_t* keep, long long i, long long n,
                                                        const long long* n_keep) {
    if (i >= n) return 0ull;
    const bool k = keep[i] != 0;
    if (!n_keep) return k ? 1ull : 0ull;
    const long long nk = *n_keep;
    if (!k && i < nk) return 1ull;               // hole
    if (k && i >= nk) return 1ull << 32;         // mover
    return 0ull;
}

__global__ void __launch_bounds__(kWinThreads) k_win_reduce(const uint8_t* __restrict__ keep, long long n,
                                                            const long long* n_keep,
                                                            unsigned long long* __restrict__ part) {
    const long long base = (long long)blockIdx.x * kWinChunk + (long long)threadIdx.x * kWinItems;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kWinItems; ++k) s += row_flags(keep, base + k, n, n_keep);
    unsigned long long total;
    block_exclusive_scan_u64(s, &total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Exclusive scan of the block totals by one block; with keep_total set, the
// grand total (the survivors) is written there.
__global__ void __launch_bounds__(1024) k_win_top(unsigned long long* part, int nparts, long long* keep_total,
                                                  unsigned long long* grand) {
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
            const unsigned long long v = part[b0 + k];
            part[b0 + k] = run;
            run += v;
        }
    if (t == 1023) {
        if (keep_total) *keep_total = (long long)s[1023];
        if (grand) *grand = s[1023];
    }
}

// Ranks: holes_list[hole rank] = row, movers_asc[mover rank] = row, and
// moved_from[r] = r for the survivors below n_keep.
__global__ void __launch_bounds__(kWinThreads) k_win_rank(const uint8_t* __restrict__ keep, long long n,
                                                          const long long* __restrict__ n_keep,
                                                          const unsigned long long* __restrict__ part,
                                                          int32_t* __restrict__ holes_list,
                                                          int32_t* __restrict__ movers_asc,
                                                          int32_t* __restrict__ moved_from) {
    const long long base = (long long)blockIdx.x * kWinChunk + (long long)threadIdx.x * kWinItems;
    unsigned long long f[kWinItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kWinItems; ++k) {
        f[k] = row_flags(keep, base + k, n, n_keep);
        s += f[k];
    }
    unsigned long long total;
    unsigned long long run = part[blockIdx.x] + block_exclusive_scan_u64(s, &total);
    const long long nk = *n_keep;
#pragma unroll
    for (int k = 0; k < kWinItems; ++k) {
        const long long i = base + k;
        if (i >= n) break;
        if (f[k] & 0xFFFFFFFFull) holes_list[run & 0xFFFFFFFFull] = (int32_t)i;
        if (f[k] >> 32) movers_asc[run >> 32] = (int32_t)i;
        if (moved_from && i < nk && keep[i]) moved_from[i] = (int32_t)i;
        run += f[k];
    }
}

// One thread per mover (ascending rank q): its row moves into the hole of
// rank n_movers - 1 - q.
__global__ void __launch_bounds__(256) k_win_move(const ColTable cols, long long n,
                                                  const unsigned long long* __restrict__ grand,
                                                  const int32_t* __restrict__ holes_list,
                                                  const int32_t* __restrict__ movers_asc,
                                                  int32_t* __restrict__ moved_from) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n_movers = (long long)(*grand >> 32);
    if (q >= n_movers || q >= n) return;
    const int32_t src = movers_asc[q];
    const int32_t dst = holes_list[n_movers - 1 - q];
    for (int c = 0; c < cols.n; ++c) {
        const int words = cols.words[c];
        const uint32_t* from = cols.ptr[c] + (size_t)src * words;
        uint32_t* to = cols.ptr[c] + (size_t)dst * words;
        for (int k = 0; k < words; ++k) to[k] = from[k];
    }
    if (moved_from) moved_from[dst] = src;
}

// Rows idx[0..m) of each source column, gathered contiguously into dst.
__global__ void __launch_bounds__(256) k_win_gather(const ColTable src, const ColTable dst,
                                                    const int32_t* __restrict__ idx, long long m, long long n) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int32_t r = idx[j];
    if (r < 0 || r >= n) return;  // validated on the host for host-known indices; guards the read
    for (int c = 0; c < src.n; ++c) {
        const int words = src.words[c];
        const uint32_t* from = src.ptr[c] + (size_t)r * words;
        uint32_t* to = dst.ptr[c] + (size_t)j * words;
        for (int k = 0; k < words; ++k) to[k] = from[k];
    }
}

__global__ void __launch_bounds__(256) k_sh_init(const ViewParam V, const float* __restrict__ means,
                                                 const float* __restrict__ image, long long begin, long long end,
                                                 int K, float z_near, float* __restrict__ sh) {
    const long long i = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= end) return;
    const float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
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
    float* o = sh + (size_t)i * K * 3;
    for (int ch = 0; ch < 3; ++ch) o[ch] = (c[ch] - 0.5f) * kInvShC0;
    for (int e = 3; e < K * 3; ++e) o[e] = 0.f;
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
    return al(sizeof(unsigned long long) * (size_t)(2 * nblk + 2)) + al(sizeof(int32_t) * (size_t)(n > 0 ? n : 1)) * 2;
}

cudaError_t launch_window_compact(const gs_window_column* cols_host, int n_cols, long long n, const uint8_t* keep,
                                  long long* n_keep_dev, int32_t* moved_from, void* scratch, cudaStream_t s,
                                  Prof& pf) {
    const long long nblk = (n + kWinChunk - 1) / kWinChunk;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    char* p = static_cast<char*>(scratch);
    unsigned long long* part = reinterpret_cast<unsigned long long*>(p);
    unsigned long long* grand = part + nblk;
    p += al(sizeof(unsigned long long) * (size_t)(2 * nblk + 2));
    int32_t* holes_list = reinterpret_cast<int32_t*>(p);
    p += al(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t* movers_asc = reinterpret_cast<int32_t*>(p);
    const ColTable cols = col_table(cols_host, n_cols);
    const int pi = pf.begin(GS_KF_WINDOW, s, 6);
    // survivors -> n_keep
    k_win_reduce<<<(unsigned)nblk, kWinThreads, 0, s>>>(keep, n, nullptr, part);
    k_win_top<<<1, 1024, 0, s>>>(part, (int)nblk, n_keep_dev, nullptr);
    // holes and movers
    k_win_reduce<<<(unsigned)nblk, kWinThreads, 0, s>>>(keep, n, n_keep_dev, part);
    k_win_top<<<1, 1024, 0, s>>>(part, (int)nblk, nullptr, grand);
    k_win_rank<<<(unsigned)nblk, kWinThreads, 0, s>>>(keep, n, n_keep_dev, part, holes_list, movers_asc,
                                                       moved_from);
    k_win_move<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cols, n, grand, holes_list, movers_asc, moved_from);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_window_gather(const gs_window_column* src_host, const gs_window_column* dst_host, int n_cols,
                                 const int32_t* idx, long long m, long long n, cudaStream_t s, Prof& pf) {
    const int pi = pf.begin(GS_KF_WINDOW, s);
    if (m > 0)
        k_win_gather<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(col_table(src_host, n_cols),
                                                                  col_table(dst_host, n_cols), idx, m, n);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_sh_init(const ViewParam& V, const float* means, const float* image, long long begin,
                           long long end, int sh_degree, float z_near, float* sh, cudaStream_t s, Prof& pf) {
    if (end <= begin) return cudaSuccess;
    const int pi = pf.begin(GS_KF_WINDOW, s);
    const int K = (sh_degree + 1) * (sh_degree + 1);
    k_sh_init<<<(unsigned)((end - begin + 255) / 256), 256, 0, s>>>(V, means, image, begin, end, K, z_near, sh);
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
