// Photometric loss with a structural term: L = (1/V) sum_v [(1 - lambda)
// mean |x - y| + lambda (1 - mean SSIM(x, y))], x the rendered image, y the
// target, SSIM of Wang et al. (2004) per channel with an 11 x 11 Gaussian
// window (sigma 1.5) and zero padding:
//   s = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)),
// mu, s^2 = E[x^2] - mu^2 and s_xy = E[xy] - mu_x mu_y the windowed moments.
// The paper's loss (Eq. gaussian_optimization) is the L1 norm; this is the
// structural variant common in 3D-GS training.
//
// Two passes over 32 x 32 output tiles of one (view, channel) plane, 256
// threads as 32 columns x 8:
//   k_ssim_fwd: the tile and a 5-pixel halo of x and y staged in shared
//     memory; the five moments by a separable window, rows first (a thread
//     slides the 11 taps over 4 neighbouring columns of one staged row, from
//     14 values held in registers), then columns (a thread slides over 4
//     rows of one column); s and its partial derivatives with respect to
//     mu_x, E[x^2] and E[xy] written per pixel as three planes, block sums of
//     s and |x - y|;
//   k_ssim_bwd: the three derivative planes staged the same way and averaged
//     by the same (symmetric) window, which is the adjoint of the moment
//     windows: ds_total/dx(p) = G*(ds/dmu_x) + 2 x G*(ds/dE_xx) + y G*(ds/dE_xy).
// Shared rows are padded so that the row pass (4 rows x 8 column groups per
// warp) and the column pass (32 consecutive columns per warp) are free of
// bank conflicts.
#include "gs_internal.cuh"

namespace gsb {

namespace {

constexpr int kTX = 32, kTY = 32;        // output tile
constexpr int kR = kSsimRadius;          // window radius (11 taps)
constexpr int kTaps = 2 * kR + 1;
constexpr int kSX = kTX + 2 * kR;        // staged tile width (42)
constexpr int kSY = kTY + 2 * kR;        // staged tile height (42)
constexpr int kRun = 4;                  // outputs per thread along a row or a column
constexpr int kGroups = kTX / kRun;      // column groups of a row (8)
constexpr int kSsimThreads = 256;        // 32 x 8
constexpr int kRows = kSsimThreads / kTX;  // 8

// Asynchronous 4-byte copy global -> shared (cp.async); with valid false no
// byte is read and the shared word is zero-filled (the image's zero padding).
__device__ __forceinline__ void stage4(float* dst, const float* src, bool valid) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Stages NP planes' (kSY x kSX) windows at (x0 - kR, y0 - kR) of a W x H image.
template <int NP>
__device__ __forceinline__ void stage_tile(float (*dst)[kSY][kSX + 1], const float* const* planes, int W, int H,
                                           int x0, int y0) {
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    for (int r = ty; r < kSY; r += kRows) {
        const int gy = y0 - kR + r;
        for (int c = tx; c < kSX; c += kTX) {
            const int gx = x0 - kR + c;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const long long o = in ? (long long)gy * W + gx : 0;
#pragma unroll
            for (int i = 0; i < NP; ++i) stage4(&dst[i][r][c], planes[i] + o, in);
        }
    }
    stage_wait();
}

// Row pass: out[q][r][4g + j] = sum_k g[k] map_q(in[.][r][4g + j + k]) for
// NM maps of NI staged planes; each thread loads its 14 staged values of
// every plane once.
template <int NI, int NM, class Map>
__device__ __forceinline__ void row_pass(const SsimParam& sp, const float (*in)[kSY][kSX + 1],
                                         float (*out)[kSY][kTX + 1], Map map) {
    constexpr int kSpan = kRun + kTaps - 1;
    for (int t = threadIdx.x; t < kSY * kGroups; t += kSsimThreads) {
        const int r = t / kGroups, c0 = (t % kGroups) * kRun;
        float v[NI][kSpan];
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int m = 0; m < kSpan; ++m) v[i][m] = in[i][r][c0 + m];
#pragma unroll
        for (int q = 0; q < NM; ++q) {
            float w[kSpan];
#pragma unroll
            for (int m = 0; m < kSpan; ++m) w[m] = map(q, v, m);
#pragma unroll
            for (int j = 0; j < kRun; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kTaps; ++k) acc = fmaf(sp.g[k], w[j + k], acc);
                out[q][r][c0 + j] = acc;
            }
        }
    }
}

// Column pass of one map for this thread's column c and rows r0..r0+3.
__device__ __forceinline__ void col_pass(const SsimParam& sp, const float (*in)[kTX + 1], int r0, int c,
                                         float* res) {
    float v[kRun + kTaps - 1];
#pragma unroll
    for (int m = 0; m < kRun + kTaps - 1; ++m) v[m] = in[r0 + m][c];
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kTaps; ++k) acc = fmaf(sp.g[k], v[j + k], acc);
        res[j] = acc;
    }
}

__global__ void __launch_bounds__(kSsimThreads) k_ssim_fwd(const __grid_constant__ BatchParam bp, SsimParam sp,
                                                           const float* __restrict__ rgb,
                                                           const float* __restrict__ target,
                                                           float* __restrict__ dmaps, long long plane_stride,
                                                           float* __restrict__ partials) {
    pdl_wait();
    pdl_trigger();
    const int view = blockIdx.z / 3, ch = blockIdx.z - 3 * view;
    const ViewParam& V = bp.v[view];
    const int W = V.W, H = V.H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    const long long part = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (x0 >= W || y0 >= H) {  // a smaller view than the grid
        if (threadIdx.x == 0) partials[part] = 0.f;
        return;
    }
    const long long plane_off = 3 * V.pix_off + (long long)ch * W * H;
    __shared__ float st[2][kSY][kSX + 1];  // staged x, y
    __shared__ float hm[5][kSY][kTX + 1];  // row-averaged x, y, x^2, y^2, xy
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    {
        const float* planes[2] = {rgb + plane_off, target + plane_off};
        stage_tile<2>(st, planes, W, H, x0, y0);
    }
    __syncthreads();
    row_pass<2, 5>(sp, st, hm, [](int q, const float (*v)[kRun + kTaps - 1], int m) {
        const float u = v[0][m], w = v[1][m];
        return q == 0 ? u : q == 1 ? w : q == 2 ? u * u : q == 3 ? w * w : u * w;
    });
    __syncthreads();
    const long long npx = (long long)W * H;
    const int r0 = ty * kRun;
    float m[5][kRun];
#pragma unroll
    for (int q = 0; q < 5; ++q) col_pass(sp, hm[q], r0, tx, m[q]);
    float s_sum = 0.f, l1_sum = 0.f;
    const int gx = x0 + tx;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        const int gy = y0 + r0 + j;
        if (gx >= W || gy >= H) continue;
        const float mx = m[0][j], my = m[1][j];
        const float a1 = fmaf(2.f * mx, my, sp.C1);
        const float a2 = fmaf(2.f, m[4][j] - mx * my, sp.C2);
        const float b1 = fmaf(mx, mx, fmaf(my, my, sp.C1));
        const float b2 = (m[2][j] - mx * mx) + (m[3][j] - my * my) + sp.C2;
        // approximate reciprocals (at most 2 ulp; b1, b2 >= C1, C2 > 0)
        const float ib1 = __fdividef(1.f, b1), ib2 = __fdividef(1.f, b2);
        const float ib = ib1 * ib2;
        const float s = a1 * a2 * ib;
        const long long o = plane_off + (long long)gy * W + gx;
        dmaps[o] = 2.f * my * (a2 - a1) * ib - 2.f * mx * s * (ib1 - ib2);
        dmaps[plane_stride + o] = -s * ib2;
        dmaps[2 * plane_stride + o] = 2.f * a1 * ib;
        s_sum += s;
        l1_sum += fabsf(st[0][r0 + j + kR][tx + kR] - st[1][r0 + j + kR][tx + kR]);
    }
    // block sum of ((1 - lambda) |x - y| - lambda s) / (3 H W V)
    float v = ((1.f - sp.lambda) * l1_sum - sp.lambda * s_sum) / ((float)(3 * npx) * (float)bp.n_views);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float sw[kSsimThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kSsimThreads / 32; ++w) t += sw[w];
        partials[part] = t;
    }
}

__global__ void __launch_bounds__(kSsimThreads) k_ssim_bwd(const __grid_constant__ BatchParam bp, SsimParam sp,
                                                           const float* __restrict__ rgb,
                                                           const float* __restrict__ target,
                                                           const float* __restrict__ dmaps, long long plane_stride,
                                                           float* __restrict__ dL_drgb) {
    pdl_wait();
    pdl_trigger();
    const int view = blockIdx.z / 3, ch = blockIdx.z - 3 * view;
    const ViewParam& V = bp.v[view];
    const int W = V.W, H = V.H;
    const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
    if (x0 >= W || y0 >= H) return;
    const long long plane_off = 3 * V.pix_off + (long long)ch * W * H;
    __shared__ float ds[3][kSY][kSX + 1];
    __shared__ float hm[3][kSY][kTX + 1];
    const int tx = threadIdx.x % kTX, ty = threadIdx.x / kTX;
    {
        const float* planes[3] = {dmaps + plane_off, dmaps + plane_stride + plane_off,
                                  dmaps + 2 * plane_stride + plane_off};
        stage_tile<3>(ds, planes, W, H, x0, y0);
    }
    __syncthreads();
    row_pass<3, 3>(sp, ds, hm, [](int q, const float (*v)[kRun + kTaps - 1], int m) { return v[q][m]; });
    __syncthreads();
    const int r0 = ty * kRun;
    float m[3][kRun];
#pragma unroll
    for (int q = 0; q < 3; ++q) col_pass(sp, hm[q], r0, tx, m[q]);
    const float scale = 1.f / ((float)(3ll * W * H) * (float)bp.n_views);
    const int gx = x0 + tx;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        const int gy = y0 + r0 + j;
        if (gx >= W || gy >= H) continue;
        const long long o = plane_off + (long long)gy * W + gx;
        const float x = rgb[o], y = target[o];
        const float dsdx = m[0][j] + 2.f * x * m[1][j] + y * m[2][j];
        const float diff = x - y;
        const float sg = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        dL_drgb[o] = scale * ((1.f - sp.lambda) * sg - sp.lambda * dsdx);
    }
}

__global__ void k_ssim_finish(const float* __restrict__ partials, long long n, float lambda,
                              float* __restrict__ loss) {
    pdl_wait();
    pdl_trigger();
    __shared__ float sw[32];
    float s = 0.f;
    const long long nb = blockDim.x;
    long long i = threadIdx.x;
    for (; i + 7 * nb < n; i += 8 * nb) {  // eight loads in flight per thread
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = partials[i + u * nb];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; i < n; i += nb) s += partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sw[w];
        *loss = lambda + t;  // the lambda * 1 of each view's (1 - mean s), averaged over views
    }
}

dim3 ssim_grid(const BatchParam& bp) {
    int mw = 0, mh = 0;
    for (int v = 0; v < bp.n_views; ++v) {
        mw = bp.v[v].W > mw ? bp.v[v].W : mw;
        mh = bp.v[v].H > mh ? bp.v[v].H : mh;
    }
    return dim3((unsigned)((mw + kTX - 1) / kTX), (unsigned)((mh + kTY - 1) / kTY), (unsigned)(3 * bp.n_views));
}

}  // namespace

size_t ssim_scratch_floats(const BatchParam& bp) {
    const dim3 g = ssim_grid(bp);
    return (size_t)3 * 3 * (size_t)bp.total_px + (size_t)g.x * g.y * g.z;
}

cudaError_t launch_ssim(const BatchParam& bp, const SsimParam& sp, const float* rgb, const float* target,
                        float* scratch, float* dL_drgb, float* loss, cudaStream_t s, Prof& pf) {
    const dim3 grid = ssim_grid(bp);
    float* dmaps = scratch;  // three planes of 3 * total_px
    const long long plane = 3 * bp.total_px;
    float* partials = scratch + (size_t)3 * (size_t)plane;
    const int pi = pf.begin(GS_KF_SSIM, s, loss ? 3 : 2);
    pdl_launch(k_ssim_fwd, grid, kSsimThreads, 0, s, bp, sp, rgb, target, dmaps, plane, partials);
    pdl_launch(k_ssim_bwd, grid, kSsimThreads, 0, s, bp, sp, rgb, target, dmaps, plane, dL_drgb);
    if (loss) pdl_launch(k_ssim_finish, 1, 1024, 0, s, partials, (long long)grid.x * grid.y * grid.z, sp.lambda, loss);
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
