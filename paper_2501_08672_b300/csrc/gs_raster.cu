// Per-tile compositing (Eq. raster), its backward pass, and the L1
// photometric loss (Eq. gaussian_optimization).
//
// One CTA per screen tile of TS x TS pixels, one pixel per thread.  The
// tile's depth-sorted Gaussian list is staged through shared memory in
// batches of TS*TS records (every thread loads one record, every thread
// reads all of them: broadcast reads, no bank conflicts).
//
// The fragment test is done in the log2 domain: with the record holding
// A' = -A/2 log2(e), B' = -B log2(e), C' = -C/2 log2(e) and l = log2(sigma),
//   p = A' dx^2 + B' dx dy + C' dy^2 + l  =  log2(sigma G(x)),
// so alpha_raw = 2^p (one ex2) and alpha < alpha_min is p < log2(alpha_min).
// Forward and backward evaluate p and alpha with the same function, so both
// passes make identical decisions.
//
// Unit of work: the visited fragment (pixel, Gaussian) pair.  These kernels
// are bound by FP32/MUFU issue, not by HBM.
#include "gs_internal.cuh"

namespace gsb {

namespace {

__device__ __forceinline__ float frag_log2_alpha(const float4 a, const float4 b, float fx, float fy,
                                                 float& dx, float& dy) {
    dx = fx - a.x;
    dy = fy - a.y;
    return fmaf(fmaf(a.z, dx, a.w * dy), dx, fmaf(b.x * dy, dy, b.y));
}

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_render_fwd(const __grid_constant__ BatchParam bp,
                                                        RenderConst rc,
                                                        const float4* __restrict__ rec,
                                                        const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ svals,
                                                        float* __restrict__ rgb,
                                                        float* __restrict__ T_final,
                                                        uint32_t* __restrict__ n_contrib) {
    constexpr int NT = TS * TS;
    __shared__ float4 s_a[NT];
    __shared__ float4 s_b[NT];
    __shared__ float s_c[NT];
    const int t = threadIdx.x;
    const int tile = blockIdx.x;
    const ViewParam& V = bp.v[find_view_by_tile(bp, tile)];
    const int lt = tile - V.tile_off;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    const int px = tx * TS + (t % TS), py = ty * TS + (t / TS);
    const bool inside = px < V.W && py < V.H;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const uint2 rg = ranges[tile];

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0;
    bool done = !inside;
    for (uint32_t start = rg.x; start < rg.y; start += NT) {
        if (__syncthreads_count(done) == NT) break;
        const uint32_t idx = start + t;
        if (idx < rg.y) {
            const uint32_t r = svals[idx];
            s_a[t] = rec[3 * r];
            s_b[t] = rec[3 * r + 1];
            s_c[t] = rec[3 * r + 2].x;
        }
        __syncthreads();
        const int cnt = min((uint32_t)NT, rg.y - start);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                float dx, dy;
                const float p = frag_log2_alpha(a, b, fx, fy, dx, dy);
                if (p < rc.log2_alpha_min) continue;
                const float alpha = fminf(rc.alpha_max, ex2_approx(p));
                const float Tn = T * (1.f - alpha);
                if (Tn < rc.T_min) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(b.z, w, C0);
                C1 = fmaf(b.w, w, C1);
                C2 = fmaf(s_c[j], w, C2);
                T = Tn;
                last = start - rg.x + j + 1;
            }
        }
    }
    if (inside) {
        const long long hw = (long long)V.W * V.H;
        const long long pl = (long long)py * V.W + px;
        float* out = rgb + 3 * V.pix_off;
        out[pl] = C0 + T * rc.bg[0];
        out[hw + pl] = C1 + T * rc.bg[1];
        out[2 * hw + pl] = C2 + T * rc.bg[2];
        T_final[V.pix_off + pl] = T;
        n_contrib[V.pix_off + pl] = last;
    }
}

// Backward of the compositing.  Walks the tile's list back to front from
// the largest n_contrib in the tile.  With T the transmittance behind
// fragment j and R the light composited behind it (normalised by T),
//   T_j = T_{j+1} / (1 - alpha_j),   dL/dc_j = alpha_j T_j g,
//   dL/dalpha_j = T_j g . (c_j - R_j),  R_{j-1} = R_j + alpha_j (c_j - R_j),
// with R = bg behind the last contributor.  Per-record accumulators (9
// floats, see grad2d in gs.h) are reduced over the warp and added with one
// atomic per warp and component; the factor ln 2 and the conversion to the
// natural conic happen in the projection backward.
template <int TS>
__global__ void __launch_bounds__(TS * TS) k_render_bwd(const __grid_constant__ BatchParam bp,
                                                        RenderConst rc,
                                                        const float4* __restrict__ rec,
                                                        const uint2* __restrict__ ranges,
                                                        const uint32_t* __restrict__ svals,
                                                        const float* __restrict__ T_final,
                                                        const uint32_t* __restrict__ n_contrib,
                                                        const float* __restrict__ dL_drgb,
                                                        float* __restrict__ grad2d) {
    constexpr int NT = TS * TS;
    __shared__ float4 s_a[NT];
    __shared__ float4 s_b[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_r[NT];
    __shared__ uint32_t s_maxnc;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int tile = blockIdx.x;
    const ViewParam& V = bp.v[find_view_by_tile(bp, tile)];
    const int lt = tile - V.tile_off;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    const int px = tx * TS + (t % TS), py = ty * TS + (t / TS);
    const bool inside = px < V.W && py < V.H;
    const float fx = px + 0.5f, fy = py + 0.5f;
    const uint2 rg = ranges[tile];

    const long long hw = (long long)V.W * V.H;
    const long long pl = (long long)py * V.W + px;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t nc = 0;
    if (inside) {
        T = T_final[V.pix_off + pl];
        nc = n_contrib[V.pix_off + pl];
        const float* gp = dL_drgb + 3 * V.pix_off;
        g0 = gp[pl];
        g1 = gp[hw + pl];
        g2 = gp[2 * hw + pl];
    }
    float R0 = rc.bg[0], R1 = rc.bg[1], R2 = rc.bg[2];
    if (t == 0) s_maxnc = 0;
    __syncthreads();
    if (nc) atomicMax(&s_maxnc, nc);
    __syncthreads();
    // n_contrib never exceeds the tile's list length when it comes from the
    // forward pass over the same bins; clamp so other inputs cannot read
    // past the list.
    const int maxnc = min((int)s_maxnc, (int)(rg.y - rg.x));

    for (int hi = maxnc; hi > 0; hi -= NT) {
        const int lo = hi - NT > 0 ? hi - NT : 0;
        const int cnt = hi - lo;
        __syncthreads();
        if (t < cnt) {
            const uint32_t r = svals[rg.x + hi - 1 - t];
            s_r[t] = r;
            s_a[t] = rec[3 * r];
            s_b[t] = rec[3 * r + 1];
            s_c[t] = rec[3 * r + 2].x;
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const int rel = hi - 1 - j;
            const float4 a = s_a[j];
            const float4 b = s_b[j];
            float dx, dy;
            const float p = frag_log2_alpha(a, b, fx, fy, dx, dy);
            const bool act = rel < (int)nc && p >= rc.log2_alpha_min;
            float v[kGrad2D];
#pragma unroll
            for (int k = 0; k < kGrad2D; ++k) v[k] = 0.f;
            if (act) {
                const float araw = ex2_approx(p);
                const float alpha = fminf(rc.alpha_max, araw);
                T = __fdividef(T, 1.f - alpha);
                const float w = alpha * T;
                const float c2 = s_c[j];
                v[6] = w * g0;
                v[7] = w * g1;
                v[8] = w * g2;
                const float d0 = b.z - R0, d1 = b.w - R1, d2 = c2 - R2;
                const float dalpha = T * (g0 * d0 + g1 * d1 + g2 * d2);
                R0 = fmaf(alpha, d0, R0);
                R1 = fmaf(alpha, d1, R1);
                R2 = fmaf(alpha, d2, R2);
                const float ga = araw < rc.alpha_max ? dalpha * araw : 0.f;
                v[0] = -ga * fmaf(2.f * a.z, dx, a.w * dy);
                v[1] = -ga * fmaf(a.w, dx, 2.f * b.x * dy);
                const float gdx = ga * dx;
                v[2] = gdx * dx;
                v[3] = gdx * dy;
                v[4] = ga * dy * dy;
                v[5] = ga;
            }
            if (__any_sync(0xffffffffu, act)) {
#pragma unroll
                for (int k = 0; k < kGrad2D; ++k) {
                    float x = v[k];
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    v[k] = x;
                }
                if (lane == 0) {
                    float* dst = grad2d + (size_t)s_r[j] * kGrad2D;
#pragma unroll
                    for (int k = 0; k < kGrad2D; ++k)
                        if (v[k] != 0.f) atomicAdd(dst + k, v[k]);
                }
            }
        }
    }
}

constexpr int kL1Threads = 256;
constexpr int kL1Items = 4;

// L1 loss and its gradient; grid.y is the view.
__global__ void __launch_bounds__(kL1Threads) k_l1(const __grid_constant__ BatchParam bp,
                                                   const float* __restrict__ rgb,
                                                   const float* __restrict__ target,
                                                   float* __restrict__ dL_drgb,
                                                   float* __restrict__ partials) {
    const ViewParam& V = bp.v[blockIdx.y];
    const long long n = 3ll * V.W * V.H;
    const float scale = 1.f / ((float)n * (float)bp.n_views);
    const long long off = 3 * V.pix_off;
    float s = 0.f;
    const long long base = (long long)blockIdx.x * kL1Threads * kL1Items + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kL1Items; ++k) {
        const long long e = base + (long long)k * kL1Threads;
        if (e < n) {
            const float d = rgb[off + e] - target[off + e];
            s += fabsf(d);
            dL_drgb[off + e] = d > 0.f ? scale : (d < 0.f ? -scale : 0.f);
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float sw[kL1Threads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tsum = 0.f;
        for (int w = 0; w < kL1Threads / 32; ++w) tsum += sw[w];
        partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tsum * scale;
    }
}

__global__ void k_l1_finish(const float* __restrict__ partials, int n, float* __restrict__ loss) {
    __shared__ float sw[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tsum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += sw[w];
        *loss = tsum;
    }
}

}  // namespace

cudaError_t launch_render_fwd(const BatchParam& bp, const RenderConst& rc, const WsPtrs& ws,
                              float* rgb, float* T_final, uint32_t* n_contrib, cudaStream_t s,
                              Prof& pf) {
    if (bp.total_tiles <= 0) return cudaSuccess;
    const uint32_t* svals = ws.pvals[ws.sorted_buf];
    const int pi = pf.begin(GS_KF_RASTER_FWD, s);
    switch (bp.tile_size) {
        case 8:
            k_render_fwd<8><<<bp.total_tiles, 64, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, rgb, T_final, n_contrib);
            break;
        case 16:
            k_render_fwd<16><<<bp.total_tiles, 256, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, rgb, T_final, n_contrib);
            break;
        case 32:
            k_render_fwd<32><<<bp.total_tiles, 1024, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, rgb, T_final, n_contrib);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const BatchParam& bp, const RenderConst& rc, const WsPtrs& ws,
                              const float* T_final, const uint32_t* n_contrib,
                              const float* dL_drgb, cudaStream_t s, Prof& pf) {
    pf.count(1);
    cudaError_t e = cudaMemsetAsync(ws.grad2d, 0, sizeof(float) * kGrad2D * (size_t)bp.total_recs, s);
    if (e != cudaSuccess || bp.total_tiles <= 0) return e;
    const uint32_t* svals = ws.pvals[ws.sorted_buf];
    const int pi = pf.begin(GS_KF_RASTER_BWD, s);
    switch (bp.tile_size) {
        case 8:
            k_render_bwd<8><<<bp.total_tiles, 64, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, T_final, n_contrib, dL_drgb, ws.grad2d);
            break;
        case 16:
            k_render_bwd<16><<<bp.total_tiles, 256, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, T_final, n_contrib, dL_drgb, ws.grad2d);
            break;
        case 32:
            k_render_bwd<32><<<bp.total_tiles, 1024, 0, s>>>(bp, rc, ws.rec, ws.ranges, svals, T_final, n_contrib, dL_drgb, ws.grad2d);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

int l1_grid_x(long long max_px) {
    return (int)((3 * max_px + kL1Threads * kL1Items - 1) / (kL1Threads * kL1Items));
}

cudaError_t launch_l1(const BatchParam& bp, const WsPtrs& ws, const float* rgb, const float* target,
                      float* dL_drgb, float* loss, cudaStream_t s, Prof& pf) {
    long long max_px = 0;
    for (int v = 0; v < bp.n_views; ++v) {
        const long long px = (long long)bp.v[v].W * bp.v[v].H;
        if (px > max_px) max_px = px;
    }
    const int gx = l1_grid_x(max_px);
    dim3 grid(gx, bp.n_views);
    const int pi = pf.begin(GS_KF_L1, s, loss ? 2 : 1);
    k_l1<<<grid, kL1Threads, 0, s>>>(bp, rgb, target, dL_drgb, ws.partials);
    if (loss) k_l1_finish<<<1, 1024, 0, s>>>(ws.partials, gx * bp.n_views, loss);
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
