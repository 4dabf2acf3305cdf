// Per-tile compositing (Eq. raster), its backward pass, and the L1
// photometric loss (Eq. gaussian_optimization).
//
// One CTA per screen tile of TS x TS pixels, PPT pixels per thread; the
// CTAs are dispatched longest tile list first.  Each warp walks the tile's
// depth-sorted list on its own: per step its lanes fetch 32 (or 64)
// records, keep those whose footprint box reaches the warp's pixels
// (ballot-compacted, in list order, into the warp's shared slots), and the
// warp then composites only those (every lane reads every slot: broadcast
// reads).  There is no block-wide barrier.
//
// The fragment test is done in the log2 domain: with the record holding the
// scaled principal axes v1, v2 of the footprint (v_k = e_k sqrt(log2(e) /
// (2 lambda_k)), e_k, lambda_k the eigenpairs of Sigma2) and l = log2(sigma),
//   p = l - (d.v1)^2 - (d.v2)^2  =  log2(sigma G(x)),   d = x - q,
// so alpha_raw = 2^p (one ex2) and alpha < alpha_min is p < log2(alpha_min).
// Record layout (3 x float4): (qx, qy, v1x, v1y), (v2x, v2y, l, r), (g, b,
// depth, ext) with ext the footprint box's half-extents as two FP16.
// Forward and backward evaluate p and alpha with the same operations in the
// same order, so both passes make identical decisions.
//
// Unit of work: the visited fragment (pixel, Gaussian) pair.  These kernels
// are bound by FP32/MUFU issue, not by HBM.
#include <mutex>

#include <cuda.h>

#include "gs_internal.cuh"

namespace gsb {

namespace {

// Thread layout: a TS x TS tile is covered by TS*TS/PPT threads.  A warp
// covers a block of WW columns x RPW*PPT pixel rows (RPW = 32/WW thread
// rows); lane l owns column l % WW and, for its k-th pixel, row
// k*RPW + l/WW of the warp's block.  The k-th pixels of a warp thus form a
// compact WW x RPW block, so a footprint edge crossing the warp's block
// leaves few k with only a handful of active lanes.  WW = TS, except for
// 16 x 16 tiles at 2 pixels per thread, whose four warps take 8 x 8 blocks
// (squarer blocks are reached by fewer records than 16 x 4 strips), and at
// 4 pixels per thread (QUAD), whose two warps take 16 x 8 blocks, the k-th
// pixels of a warp being the k-th 8 x 4 quadrant of its block: the same
// 8 x 4 groups of pixels per body as at 2 pixels per thread, with half as
// many warps staging and reducing each record.
template <int TS, int PPT>
struct PixelMap {
    static_assert(TS <= 32 && 32 % TS == 0 && (TS * TS / PPT) % 32 == 0, "unsupported launch shape");
    static constexpr bool QUAD = TS == 16 && PPT == 4;
    static constexpr int WW = (TS == 16 && (PPT == 2 || QUAD)) ? 8 : TS;
    static constexpr int RPW = 32 / WW;
    static constexpr int WCOLS = QUAD ? 1 : TS / WW;
    int px, py;  // column, row of pixel 0
    __device__ __forceinline__ PixelMap(int tx, int ty, int t) {
        const int w = t >> 5, l = t & 31;
        px = tx * TS + (w % WCOLS) * WW + (l % WW);
        py = ty * TS + (w / WCOLS) * RPW * (QUAD ? 2 : PPT) + l / WW;
    }
    __device__ __forceinline__ int row(int k) const { return py + (QUAD ? (k >> 1) : k) * RPW; }
    __device__ __forceinline__ int col(int k) const { return QUAD ? px + (k & 1) * 8 : px; }
    // distinct columns of a thread's pixels; pixel k is in column k % NCOL
    static constexpr int NCOL = QUAD ? 2 : 1;
};

// Pixel-centre box of the pixels a warp owns.  A record whose footprint box
// (centre q, half-extents packed as two FP16 values rounded up) misses it
// has alpha < alpha_min at every pixel of the warp, so the warp skips it.
struct WarpBox {
    float cx, cy, hx, hy;
    __device__ __forceinline__ bool reaches(float qx, float qy, float ext) const {
        const __half2 e = *reinterpret_cast<const __half2*>(&ext);
        return fabsf(qx - cx) <= __low2float(e) + hx && fabsf(qy - cy) <= __high2float(e) + hy;
    }
};

// The exact test behind the box test: does the record's alpha >= alpha_min
// ellipse reach a pixel centre of the warp's block (the test the binning uses
// for tiles, with the same margin)?  Only meaningful when alpha_min > 0.
__device__ __forceinline__ bool ellipse_reaches(const WarpBox& wb, float4 r0, float4 r1, float log2_alpha_min) {
    const Footprint fp = make_footprint(r0, r1, r1.z - log2_alpha_min);
    return footprint_hits_rect(fp, wb.cx - wb.hx, wb.cx + wb.hx, wb.cy - wb.hy, wb.cy + wb.hy);
}

__device__ __forceinline__ WarpBox warp_box(int px_first, int px_last, int py_first, int py_last) {
    const int x0 = __reduce_min_sync(0xffffffffu, px_first), x1 = __reduce_max_sync(0xffffffffu, px_last);
    const int y0 = __reduce_min_sync(0xffffffffu, py_first), y1 = __reduce_max_sync(0xffffffffu, py_last);
    WarpBox b;
    b.cx = 0.5f * (float)(x0 + x1 + 1);
    b.cy = 0.5f * (float)(y0 + y1 + 1);
    b.hx = 0.5f * (float)(x1 - x0);
    b.hy = 0.5f * (float)(y1 - y0);
    return b;
}
constexpr int kGroup = 4;  // Gaussians per warp reduction in the backward

// Register budget of the forward: the compiler's choice (0 = no minimum of
// resident blocks; capping the 16 x 16 tile at 4 pixels per thread to 64
// registers for 32 warps spilled and was slower).
template <int NT, int PPT>
constexpr int fwd_min_blocks() { return 0; }

// CNT: also count each pixel's contributors into n_used (a statistic for the
// fragment model; the plain forward does without the counter).
template <int TS, int PPT, int BATCH, bool CNT>
__global__ void __launch_bounds__(TS * TS / PPT, fwd_min_blocks<TS * TS / PPT, PPT>()) k_render_fwd(const __grid_constant__ BatchParam bp,
                                                              RenderConst rc,
                                                              const float4* __restrict__ rec,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ tile_order,
                                                              const uint32_t* __restrict__ svals,
                                                              float* __restrict__ rgb,
                                                              float* __restrict__ T_final,
                                                              uint32_t* __restrict__ n_contrib,
                                                              uint32_t* __restrict__ n_used,
                                                              const float* __restrict__ target,
                                                              float* __restrict__ dL_drgb,
                                                              float* __restrict__ partials,
                                                              uint32_t* __restrict__ order_keys,
                                                              uint32_t* __restrict__ order_vals,
                                                              unsigned long long* __restrict__ counters) {
    pdl_wait();
    pdl_trigger();
    // Each warp walks the tile's list on its own: per step every lane fetches
    // Q records, the records whose footprint box reaches the warp's pixels
    // are compacted (in list order) into the warp's shared slots, and the
    // warp composites only those.  No block barrier: a warp whose pixels
    // are all saturated stops without waiting for the others.
    constexpr int NT = TS * TS / PPT;
    constexpr int NW = NT / 32;
    constexpr int Q = BATCH >= 256 ? 2 : 1;
    constexpr int WB = 32 * Q;
    __shared__ float4 s_a[NW][WB];
    __shared__ float4 s_b[NW][WB];
    __shared__ float4 s_c[NW][WB];  // colour 1, 2; list position + 1 (bits)
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int w = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int tile = (int)tile_order[blockIdx.x];  // longest lists first
    const ViewParam& V = bp.v[find_view_by_tile(bp, tile)];
    const int lt = tile - V.tile_off;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    const PixelMap<TS, PPT> pm(tx, ty, t);
    // thr[k]: the exponent a fragment must reach at pixel k; +inf once the
    // pixel is saturated (or outside the image), so one compare both skips
    // faint fragments and finished pixels
    constexpr int NCOL = PixelMap<TS, PPT>::NCOL;
    float fx[NCOL], fy[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT], thr[PPT];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) fx[c] = pm.col(c) + 0.5f;
    uint32_t last[PPT], used[PPT];
    const float kDone = __int_as_float(0x7f800000);
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        fy[k] = pm.row(k) + 0.5f;
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        used[k] = 0;
        thr[k] = (pm.col(k) < V.W && pm.row(k) < V.H) ? rc.log2_alpha_min : kDone;
    }
    uint2 rg = ranges[tile];
    if (!gs_checked(rg.x <= rg.y && (long long)rg.y <= rc.cap, rc)) rg.y = rg.x;

    for (uint32_t start = rg.x; start < rg.y; start += WB) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) all = all && thr[k] == kDone;
        if (__all_sync(0xffffffffu, all)) break;
        // Box of the warp's pixels still taking contributions: a finished
        // pixel skips every fragment, so a record reaching none of the live
        // pixels is not staged.  Past the last contributor of most pixels
        // (tiles with a few pixels that never saturate walk their whole list)
        // this box is far smaller than the warp's.
        WarpBox wb;
        {
            int x0 = 1 << 20, x1 = -(1 << 20), y0 = 1 << 20, y1 = -(1 << 20);
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (thr[k] != kDone) {
                    x0 = min(x0, pm.col(k));
                    x1 = max(x1, pm.col(k));
                    y0 = min(y0, pm.row(k));
                    y1 = max(y1, pm.row(k));
                }
            wb = warp_box(x0, x1, y0, y1);
        }
        int n = 0;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const uint32_t idx = start + q * 32 + lane;
            bool reach = false;
            uint32_t r = 0;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
            if (idx < rg.y) {
                r = svals[idx];
                if (gs_checked(r < (uint32_t)bp.total_recs, rc)) {
                    a = rec[3 * r];
                    c = rec[3 * r + 2];
                    reach = wb.reaches(a.x, a.y, c.w);
                    if (reach) b = rec[3 * r + 1];
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, reach);
            if (reach) {
                const int pos = n + __popc(m & lt_mask);
                s_a[w][pos] = a;
                s_b[w][pos] = b;
                s_c[w][pos] = make_float4(c.x, c.y, __uint_as_float(idx - rg.x + 1), 0.f);
            }
            n += __popc(m);
        }
        __syncwarp();
        if (!all) {
            for (int j = 0; j < n; ++j) {
                const float4 a = s_a[w][j];
                const float4 b = s_b[w][j];
                const float4 c = s_c[w][j];
                const uint32_t pos1 = __float_as_uint(c.z);
                float dxc[NCOL], u1c[NCOL], u2c[NCOL];
#pragma unroll
                for (int c = 0; c < NCOL; ++c) {
                    dxc[c] = fx[c] - a.x;
                    u1c[c] = dxc[c] * a.z;
                    u2c[c] = dxc[c] * b.x;
                }
#pragma unroll
                for (int k = 0; k < PPT; ++k) {
                    const float dx = dxc[k % NCOL], u1 = u1c[k % NCOL], u2 = u2c[k % NCOL];
                    const float dy = fy[k] - a.y;
                    const float t1 = fmaf(dy, a.w, u1);
                    const float t2 = fmaf(dy, b.y, u2);
                    const float p = fmaf(-t1, t1, fmaf(-t2, t2, b.z));
                    if (p < thr[k]) continue;  // faint fragment, or pixel finished
                    const float alpha = fminf(rc.alpha_max, ex2_approx(p));
                    // w = alpha T and T (1 - alpha) = T - w
                    const float wgt = alpha * T[k];
                    const float Tn = T[k] - wgt;
                    if (Tn < rc.T_min) {
                        thr[k] = kDone;
                        continue;
                    }
                    C0[k] = fmaf(b.w, wgt, C0[k]);
                    C1[k] = fmaf(c.x, wgt, C1[k]);
                    C2[k] = fmaf(c.y, wgt, C2[k]);
                    T[k] = Tn;
                    last[k] = pos1;
                    if (CNT) ++used[k];
                }
            }
        }
        __syncwarp();
    }
    const long long hw = (long long)V.W * V.H;
    // With a target the L1 loss is folded in here (Eq. gaussian_optimization):
    // a pixel's gradient sign(C - target) / (3 H W V) needs only its own
    // colour, and the tile's sum of |C - target| goes to partials[tile].
    const float scale = 1.f / ((float)(3 * hw) * (float)bp.n_views);
    float lsum = 0.f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (pm.col(k) < V.W && pm.row(k) < V.H) {
            const long long pl = (long long)pm.row(k) * V.W + pm.col(k);
            const float o0 = C0[k] + T[k] * rc.bg[0];
            const float o1 = C1[k] + T[k] * rc.bg[1];
            const float o2 = C2[k] + T[k] * rc.bg[2];
            if (rgb) {
                float* out = rgb + 3 * V.pix_off;
                out[pl] = o0;
                out[hw + pl] = o1;
                out[2 * hw + pl] = o2;
            }
            T_final[V.pix_off + pl] = T[k];
            n_contrib[V.pix_off + pl] = last[k];
            if (CNT) n_used[V.pix_off + pl] = used[k];
            if (target) {
                const float* y = target + 3 * V.pix_off;
                float* g = dL_drgb + 3 * V.pix_off;
                const float d0 = o0 - y[pl], d1 = o1 - y[hw + pl], d2 = o2 - y[2 * hw + pl];
                lsum += fabsf(d0) + fabsf(d1) + fabsf(d2);
                g[pl] = d0 > 0.f ? scale : (d0 < 0.f ? -scale : 0.f);
                g[hw + pl] = d1 > 0.f ? scale : (d1 < 0.f ? -scale : 0.f);
                g[2 * hw + pl] = d2 > 0.f ? scale : (d2 < 0.f ? -scale : 0.f);
            }
        }
    }
    // The backward walks each tile back from its deepest contributor: that
    // depth, the tile's largest n_contrib, keys the tile in the dispatch order
    // of the backward (heaviest first; sorted after this launch).
    uint32_t deep = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) deep = max(deep, last[k]);
    deep = __reduce_max_sync(0xffffffffu, deep);
    if (target) {
        // per-tile partial, summed in a fixed order (indexed by tile, not by
        // launch order, so the loss does not depend on the dispatch order)
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    }
    __shared__ float s_l[NW];
    __shared__ uint32_t s_deep[NW];
    if (NW > 1) {
        if (lane == 0) {
            s_l[w] = lsum;
            s_deep[w] = deep;
        }
        __syncthreads();
    }
    if (t == 0) {
        float tsum = lsum;
        for (int i = 1; i < NW; ++i) {
            tsum += s_l[i];
            deep = max(deep, s_deep[i]);
        }
        if (target) partials[tile] = tsum * scale;
        order_keys[tile] = tile_order_key(deep);
        order_vals[tile] = (uint32_t)tile;
        if (blockIdx.x == 0) counters[kCtrOrderTiles] = (unsigned long long)bp.total_tiles;
    }
}

// Backward of the compositing.  Walks the tile's list back to front from
// the largest n_contrib of each warp's pixels.  With T the transmittance behind
// fragment j and R the light composited behind it (normalised by T),
//   T_j = T_{j+1} / (1 - alpha_j),   dL/dc_j = alpha_j T_j g,
//   dL/dalpha_j = T_j g . (c_j - R_j),  R_{j-1} = R_j + alpha_j (c_j - R_j),
// with R = bg behind the last contributor; only the scalar g . R is carried
// (g . R_{j-1} = g . R_j + alpha_j (g . c_j - g . R_j)).  With ga = dL/dalpha * 2^p where
// alpha is not clamped (dL/dp up to the factor ln 2), the 9 per-record
// accumulators are
//   sum ga (d.v1), sum ga (d.v2), sum ga dx^2, sum ga dx dy, sum ga dy^2,
//   sum ga, sum w g_r, sum w g_g, sum w g_b      (w = alpha T),
// summed over the thread's PPT pixels, reduced over the warp, and added
// with one atomic per (warp, record, component); the factor ln 2, the
// principal axes and the conversion to the natural conic are applied in
// the projection backward.
// Register budget of the backward: enough blocks for 28 resident warps per
// SM (72 registers; the kernel is issue-bound and its warps stall on short
// dependency chains and on the shared-memory reduction, so occupancy buys
// issue slots): 0.964 ms against 0.970 at 24 warps.
// (From 4 pixels per thread on, the cap would spill: no target there, except
// the 16 x 16 tile's two 16 x 8 warp blocks (QUAD), held to 80 registers
// for 24 resident warps: 0.977 ms against 0.992 at 96 registers, at the
// headline workload.  A 64-register cap for 32 warps at 2 pixels per thread
// spills a little and is slower, 0.993 against 0.970 ms.)
template <int NT, int PPT>
constexpr int bwd_min_blocks() {
    return (NT == 64 && PPT == 4) ? 12 : (PPT >= 4 ? 1 : (896 / NT > 32 ? 32 : 896 / NT));
}

// DET: the deterministic form.  All warps of the tile walk the list from the
// tile's deepest contributor in windows of kDetWindow records (several
// staging batches, so warps drift within a window and meet at its end); each
// warp leaves its per-record totals in shared memory, the block adds them in
// warp order and writes one 9-float partial per listed record at its place in
// the tile list (pair_grad), zeros where no pixel of the tile contributes; no
// atomics.
constexpr int kDetWindow = 64;
template <int TS, int PPT, int BATCH, bool DET>
__global__ void __launch_bounds__(TS * TS / PPT, bwd_min_blocks<TS * TS / PPT, PPT>()) k_render_bwd(const __grid_constant__ BatchParam bp,
                                                              RenderConst rc,
                                                              const float4* __restrict__ rec,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ tile_order,
                                                              const uint32_t* __restrict__ svals,
                                                              const float* __restrict__ T_final,
                                                              const uint32_t* __restrict__ n_contrib,
                                                              const float* __restrict__ dL_drgb,
                                                              float* __restrict__ grad2d,
                                                              float* __restrict__ pair_grad) {
    pdl_wait();
    pdl_trigger();
    // Each warp walks the list on its own, back to front from its deepest
    // contributor, fetching Q records per lane per step and compacting the
    // ones whose footprint box reaches its pixels (as in the forward).  No
    // block barrier: the warps of a tile finish independently.
    constexpr int NT = TS * TS / PPT;
    constexpr int NW = NT / 32;
    constexpr int Q = BATCH >= 256 ? 2 : 1;
    constexpr int WB = 32 * Q;
    __shared__ float4 s_a[NW][WB];
    __shared__ float4 s_b[NW][WB];
    __shared__ float4 s_c[NW][WB];  // colour 1, 2; position in the list (bits); record (bits)
    // per-warp transposition matrix of the warp reduction (where it fits the
    // 48 KB of static shared memory with the staging above)
    // records per deterministic window (a multiple of the staging batch)
    constexpr int DW = DET ? (kDetWindow > WB ? kDetWindow : WB) : 1;
    constexpr bool kSmemRed = NW * 32 * 144 + 3 * NW * WB * 16 + (DET ? NW * DW * kGrad2D * 4 : 0) <= 44 * 1024;
    __shared__ float4 s_red[kSmemRed ? NW : 1][32][9];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int tile = (int)tile_order[blockIdx.x];  // longest lists first
    const ViewParam& V = bp.v[find_view_by_tile(bp, tile)];
    const int lt = tile - V.tile_off;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    const PixelMap<TS, PPT> pm(tx, ty, t);
    uint2 rg = ranges[tile];
    if (!gs_checked(rg.x <= rg.y && (long long)rg.y <= rc.cap, rc)) rg.y = rg.x;
    const long long hw = (long long)V.W * V.H;
    const float* gimg = dL_drgb + 3 * V.pix_off;

    constexpr int NCOL = PixelMap<TS, PPT>::NCOL;
    float fx[NCOL], fy[PPT], T[PPT], g0[PPT], g1[PPT], g2[PPT], gR[PPT];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) fx[c] = pm.col(c) + 0.5f;
    int nc[PPT];
    uint32_t mine = 0;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        fy[k] = pm.row(k) + 0.5f;
        T[k] = 1.f;
        g0[k] = g1[k] = g2[k] = 0.f;
        nc[k] = 0;
        if (pm.col(k) < V.W && pm.row(k) < V.H) {
            const long long pl = (long long)pm.row(k) * V.W + pm.col(k);
            T[k] = T_final[V.pix_off + pl];
            nc[k] = (int)n_contrib[V.pix_off + pl];
            g0[k] = gimg[pl];
            g1[k] = gimg[hw + pl];
            g2[k] = gimg[2 * hw + pl];
        }
        gR[k] = g0[k] * rc.bg[0] + g1[k] * rc.bg[1] + g2[k] * rc.bg[2];
        mine = max(mine, (uint32_t)nc[k]);
    }
    const int wmax = min((int)__reduce_max_sync(0xffffffffu, mine), (int)(rg.y - rg.x));
    // deterministic form: per-warp totals of the batch's records, and the
    // tile's deepest contributor
    __shared__ float s_acc[DET ? NW : 1][DW][kGrad2D];
    __shared__ int s_wmax[DET ? NW : 1];
    int walk = wmax;
    if constexpr (DET) {
        if (lane == 0) s_wmax[warp] = wmax;
        __syncthreads();
        walk = 0;
#pragma unroll
        for (int i = 0; i < NW; ++i) walk = max(walk, s_wmax[i]);
    }

    for (int hi = walk; hi > 0; hi -= WB) {
        int n = 0;
        // deterministic form: top of the current window and its last batch
        const int wtop = walk - ((walk - hi) / DW) * DW;
        const bool wlast = hi <= WB || wtop - (hi - WB) >= DW;
        if constexpr (DET) {
            if (hi == wtop)
                for (int i = lane; i < DW * kGrad2D; i += 32) (&s_acc[warp][0][0])[i] = 0.f;
        }
        // a warp whose pixels all stop before this batch stages nothing
        const bool act = !DET || hi - WB < wmax;
        // Box of the warp's pixels that can take a contribution from this
        // batch (n_contrib above its first place): a record reaching no such
        // pixel adds nothing, and deep in the list, where most of the tile's
        // pixels are already saturated, this box is much smaller than the
        // warp's (empty, hence reached by nothing, when no pixel is live).
        WarpBox wb;
        {
            int x0 = 1 << 20, x1 = -(1 << 20), y0 = 1 << 20, y1 = -(1 << 20);
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (nc[k] > hi - WB) {
                    x0 = min(x0, pm.col(k));
                    x1 = max(x1, pm.col(k));
                    y0 = min(y0, pm.row(k));
                    y1 = max(y1, pm.row(k));
                }
            wb = warp_box(x0, x1, y0, y1);
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (!act) break;
            const int rel = hi - 1 - (q * 32 + lane);
            bool reach = false;
            uint32_t r = 0;
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
            if (rel >= 0 && gs_checked((r = svals[rg.x + rel]) < (uint32_t)bp.total_recs, rc)) {
                a = rec[3 * r];
                c = rec[3 * r + 2];
                reach = wb.reaches(a.x, a.y, c.w);
                if (reach) {
                    b = rec[3 * r + 1];
                    // a warp smaller than the tile also drops records whose
                    // ellipse misses its block (the bins only test the tile)
                    if (NW > 1 && rc.alpha_min > 0.f) reach = ellipse_reaches(wb, a, b, rc.log2_alpha_min);
                }
            }
            const uint32_t m = __ballot_sync(0xffffffffu, reach);
            if (reach) {
                const int pos = n + __popc(m & lt_mask);
                s_a[warp][pos] = a;
                s_b[warp][pos] = b;
                s_c[warp][pos] = make_float4(c.x, c.y, __int_as_float(rel), __uint_as_float(r));
            }
            n += __popc(m);
        }
        __syncwarp();
        for (int j0 = 0; j0 < n; j0 += kGroup) {
            // contributions of kGroup consecutive listed Gaussians, summed over
            // this thread's pixels (9 accumulators each).  With the reduction
            // through shared memory each Gaussian's first 8 go to this lane's
            // row as soon as they are complete (one set of accumulators in
            // registers, component 8 kept in y); else all kGroup sets stay in
            // registers for the butterfly.
            constexpr int NV = kSmemRed ? 1 : kGroup;
            float v[NV][kGrad2D];
            float y[kGroup];
            if constexpr (!kSmemRed) {
#pragma unroll
                for (int g = 0; g < kGroup; ++g)
#pragma unroll
                    for (int e = 0; e < kGrad2D; ++e) v[g][e] = 0.f;
            }
            bool any = false;
#pragma unroll
            for (int g = 0; g < kGroup; ++g) {
                const int j = j0 + g;
                float* vg = v[kSmemRed ? 0 : g];
                if constexpr (kSmemRed) {
#pragma unroll
                    for (int e = 0; e < kGrad2D; ++e) vg[e] = 0.f;
                }
                if (j < n) {

                    const float4 a = s_a[warp][j];
                    const float4 b = s_b[warp][j];
                    const float4 c = s_c[warp][j];
                    const int rel = __float_as_int(c.z);
                    float dxc[NCOL], u1c[NCOL], u2c[NCOL];
#pragma unroll
                    for (int c = 0; c < NCOL; ++c) {
                        dxc[c] = fx[c] - a.x;
                        u1c[c] = dxc[c] * a.z;
                        u2c[c] = dxc[c] * b.x;
                    }
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const float dx = dxc[k % NCOL], u1 = u1c[k % NCOL], u2 = u2c[k % NCOL];
                        const float dy = fy[k] - a.y;
                        const float t1 = fmaf(dy, a.w, u1);
                        const float t2 = fmaf(dy, b.y, u2);
                        const float p = fmaf(-t1, t1, fmaf(-t2, t2, b.z));
                        // behind the pixel's last contributor, or a faint fragment
                        if (rel >= nc[k] || p < rc.log2_alpha_min) continue;
                        any = true;
                        const float araw = ex2_approx(p);
                        const float alpha = fminf(rc.alpha_max, araw);
                        T[k] = __fdividef(T[k], 1.f - alpha);
                        const float w = alpha * T[k];
                        vg[6] = fmaf(w, g0[k], vg[6]);
                        vg[7] = fmaf(w, g1[k], vg[7]);
                        vg[8] = fmaf(w, g2[k], vg[8]);
                        const float gd = fmaf(g0[k], b.w, fmaf(g1[k], c.x, fmaf(g2[k], c.y, -gR[k])));
                        const float dalpha = T[k] * gd;
                        gR[k] = fmaf(alpha, gd, gR[k]);
                        const float ga = araw < rc.alpha_max ? dalpha * araw : 0.f;
                        // dp/dq = 2 ((d.v1) v1 + (d.v2) v2) with v1, v2 fixed per
                        // record: only ga (d.v1), ga (d.v2) are summed here
                        vg[0] = fmaf(ga, t1, vg[0]);
                        vg[1] = fmaf(ga, t2, vg[1]);
                        const float gdx = ga * dx;
                        vg[2] = fmaf(gdx, dx, vg[2]);
                        vg[3] = fmaf(gdx, dy, vg[3]);
                        vg[4] = fmaf(ga * dy, dy, vg[4]);
                        vg[5] += ga;
                    }
                }
                if constexpr (kSmemRed) {
                    float4* row = s_red[warp][lane];
                    row[2 * g] = make_float4(vg[0], vg[1], vg[2], vg[3]);
                    row[2 * g + 1] = make_float4(vg[4], vg[5], vg[6], vg[7]);
                    y[g] = vg[8];
                }
            }
            if (__any_sync(0xffffffffu, any)) {
                // Warp totals of the 32 values v[g][e], e < 8.  Each lane ends
                // with the total of one value: index vi, component vi & 7 of
                // Gaussian vi >> 3.
                float tot;
                int vi;
                if constexpr (kSmemRed) {
                    // Through shared memory: each lane has stored its values as
                    // 8 float4 words in its row (rows 144 bytes apart, so the
                    // stores of 8 lanes fall into distinct banks); lane l adds
                    // chunk c = l & 7 (values 4c..4c+3) over the 8 rows of its
                    // lane group (l & 24), conflict-free too; two halving levels
                    // over the 4 groups leave it value 4c + 2 ((l >> 4) & 1) +
                    // ((l >> 3) & 1).  Half the instructions of the butterfly
                    // below (no selects for 28 of its 31 levels' values).
                    __syncwarp();
                    const int c = lane & 7, r0 = lane & 24;
                    float4 acc = s_red[warp][r0][c];
#pragma unroll
                    for (int j = 1; j < 8; ++j) {
                        const float4 q = s_red[warp][r0 + j][c];
                        acc.x += q.x;
                        acc.y += q.y;
                        acc.z += q.z;
                        acc.w += q.w;
                    }
                    __syncwarp();
                    const bool u16 = (lane & 16) != 0, u8 = (lane & 8) != 0;
                    const float h0 = (u16 ? acc.z : acc.x) + __shfl_xor_sync(0xffffffffu, u16 ? acc.x : acc.z, 16);
                    const float h1 = (u16 ? acc.w : acc.y) + __shfl_xor_sync(0xffffffffu, u16 ? acc.y : acc.w, 16);
                    tot = (u8 ? h1 : h0) + __shfl_xor_sync(0xffffffffu, u8 ? h0 : h1, 8);
                    vi = 4 * c + 2 * (int)u16 + (int)u8;
                } else {
                    // Reduce-scatter by butterfly: the 32 values are halved at
                    // each level (a lane keeps the half selected by its lane bit
                    // and receives its partner's copy of it), leaving lane l
                    // with the warp total of value l.
                    float x[32];
#pragma unroll
                    for (int g = 0; g < kGroup; ++g)
#pragma unroll
                        for (int e = 0; e < 8; ++e) x[g * 8 + e] = v[g][e];
#pragma unroll
                    for (int o = 16, len = 32; o > 0; o >>= 1, len >>= 1) {
                        const bool upper = (lane & o) != 0;
#pragma unroll
                        for (int i = 0; i < len / 2; ++i) {
                            const float send = upper ? x[i] : x[i + len / 2];
                            const float keep = upper ? x[i + len / 2] : x[i];
                            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                        }
                    }
                    tot = x[0];
                    vi = lane;
                }
                // component 8 of the 4 Gaussians: two halving levels leave
                // lane l with Gaussian l >> 3, then a sum over its 8 lanes
                if constexpr (!kSmemRed) {
#pragma unroll
                    for (int g = 0; g < kGroup; ++g) y[g] = v[g][8];
                }
#pragma unroll
                for (int o = 16, len = kGroup; o >= 8; o >>= 1, len >>= 1) {
                    const bool upper = (lane & o) != 0;
#pragma unroll
                    for (int i = 0; i < len / 2; ++i) {
                        const float send = upper ? y[i] : y[i + len / 2];
                        const float keep = upper ? y[i + len / 2] : y[i];
                        y[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                    }
                }
                float yb = y[0];
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) yb += __shfl_xor_sync(0xffffffffu, yb, o);
                const int gm = vi >> 3, em = vi & 7;  // this lane's main value
                const int gl = lane >> 3, el = lane & 7;  // component 8 of Gaussian gl at el == 0
                if constexpr (DET) {
                    if (j0 + gm < n) s_acc[warp][wtop - 1 - __float_as_int(s_c[warp][j0 + gm].z)][em] = tot;
                    if (el == 0 && j0 + gl < n) s_acc[warp][wtop - 1 - __float_as_int(s_c[warp][j0 + gl].z)][8] = yb;
                } else {
                    if (j0 + gm < n && tot != 0.f)
                        atomicAdd(grad2d + (size_t)__float_as_uint(s_c[warp][j0 + gm].w) * kGrad2D + em, tot);
                    if (el == 0 && j0 + gl < n && yb != 0.f)
                        atomicAdd(grad2d + (size_t)__float_as_uint(s_c[warp][j0 + gl].w) * kGrad2D + 8, yb);
                }
            }
        }
        __syncwarp();
        if constexpr (DET) {
            if (wlast) {
                // the tile's partial of each record of the window: warp totals
                // added in warp order
                __syncthreads();
                for (int i = t; i < DW * kGrad2D; i += NT) {
                    const int slot = i / kGrad2D, c = i - slot * kGrad2D;
                    const int rel = wtop - 1 - slot;
                    if (rel < 0) continue;
                    float v = 0.f;
#pragma unroll
                    for (int w2 = 0; w2 < NW; ++w2) v += s_acc[w2][slot][c];
                    pair_grad[(size_t)(rg.x + (uint32_t)rel) * kPairGradStride + c] = v;
                }
                __syncthreads();
            }
        }
    }
    if constexpr (DET) {
        // records beyond every pixel's last contributor
        const size_t end = (size_t)rg.y * kPairGradStride;
        for (size_t i = (size_t)(rg.x + (uint32_t)walk) * kPairGradStride + t; i < end; i += NT) pair_grad[i] = 0.f;
    }
}

// Deterministic backward: a record's 2D gradient is the sum of its pairs'
// partials.  Its pairs are contiguous in emission order (records in depth
// order, k-th record at offsets[k]), and pair_inv gives each one's place in
// the tile lists.  A warp takes 32 consecutive records; their pairs are one
// contiguous emission range, which its lanes walk 32 positions at a time
// (coalesced place reads, one partial row of three 16-byte words per lane),
// each position's record found by a binary search over the lanes' offsets.
// A segmented scan across the lanes (a fixed pattern of shuffles) sums each
// record's positions within the 32, a carry takes a record across rounds,
// and the lane at a record's last position writes it: the same order on
// every run.  Records without pairs are written as zero.
__global__ void __launch_bounds__(256) k_pair_grad_reduce(const uint32_t* __restrict__ order,
                                                          const unsigned long long* __restrict__ offsets,
                                                          const uint32_t* __restrict__ touched,
                                                          const uint32_t* __restrict__ pair_inv,
                                                          const float* __restrict__ pair_grad, long long M,
                                                          long long cap, const unsigned long long* __restrict__ n_dev,
                                                          float* __restrict__ grad2d) {
    pdl_wait();
    pdl_trigger();
    const long long k0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll;
    if (k0 >= M) return;  // whole warps: M is the same for all lanes
    const int lane = threadIdx.x & 31;
    const long long k = k0 + lane;
    const bool live = k < M;
    unsigned long long n = n_dev[0];
    if (n > (unsigned long long)cap) n = (unsigned long long)cap;
    const uint32_t r = live ? order[k] : 0u;
    const uint32_t cnt = live ? touched[r] : 0u;
    const unsigned long long e0 = live ? offsets[k] : 0ull;
    const unsigned long long wbase = __shfl_sync(0xffffffffu, e0, 0);
    const uint32_t rel = live ? (uint32_t)(e0 - wbase) : 0xFFFFFFFFu;
    const uint32_t wtotal = __reduce_max_sync(0xffffffffu, live ? rel + cnt : 0u);
    if (live && cnt == 0)
        for (int c = 0; c < kGrad2D; ++c) grad2d[(size_t)r * kGrad2D + c] = 0.f;
    float carry[kGrad2D];
#pragma unroll
    for (int c = 0; c < kGrad2D; ++c) carry[c] = 0.f;
    int carry_owner = -1;
    for (uint32_t p0 = 0; p0 < wtotal; p0 += 32) {
        const uint32_t pr = p0 + (uint32_t)lane;
        // owner: the last lane whose first position is at or below pr
        int o = 0;
#pragma unroll
        for (int st = 16; st >= 1; st >>= 1) {
            const uint32_t oc = __shfl_sync(0xffffffffu, rel, o + st);
            if (oc <= pr) o += st;
        }
        const bool in = pr < wtotal;
        float v[kGrad2D];
#pragma unroll
        for (int c = 0; c < kGrad2D; ++c) v[c] = 0.f;
        const unsigned long long e = wbase + pr;
        if (in && e < n) {
            const uint32_t p = pair_inv[e];
            if (p != 0xFFFFFFFFu) {
                const float4* row = reinterpret_cast<const float4*>(pair_grad + (size_t)p * kPairGradStride);
                const float4 x = row[0], y = row[1], z = row[2];
                v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
                v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
                v[8] = z.x;
            }
        }
        // segmented inclusive scan over the lanes, segments = owners
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int od = __shfl_up_sync(0xffffffffu, o, d);
            const bool same = lane >= d && od == o;
#pragma unroll
            for (int c = 0; c < kGrad2D; ++c) {
                const float u = __shfl_up_sync(0xffffffffu, v[c], d);
                if (same) v[c] += u;
            }
        }
        if (o == carry_owner) {
#pragma unroll
            for (int c = 0; c < kGrad2D; ++c) v[c] += carry[c];
        }
        // the record of the round's last lane continues into the next round
        const int last_owner = __shfl_sync(0xffffffffu, o, 31);
#pragma unroll
        for (int c = 0; c < kGrad2D; ++c) carry[c] = __shfl_sync(0xffffffffu, v[c], 31);
        carry_owner = last_owner;
        const uint32_t ro = __shfl_sync(0xffffffffu, r, o);
        const uint32_t rel_o = __shfl_sync(0xffffffffu, rel, o);
        const uint32_t cnt_o = __shfl_sync(0xffffffffu, cnt, o);
        if (in && pr == rel_o + cnt_o - 1u) {
#pragma unroll
            for (int c = 0; c < kGrad2D; ++c) grad2d[(size_t)ro * kGrad2D + c] = v[c];
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
    pdl_wait();
    pdl_trigger();
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
    pdl_wait();
    pdl_trigger();
    __shared__ float sw[32];
    float s = 0.f;
    int i = threadIdx.x;
    const int nb = (int)blockDim.x;
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
        float tsum = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += sw[w];
        *loss = tsum;
    }
}

// ---- pose normal equations (Sec. II-D) -------------------------------------
//
// Forward-mode compositing: per pixel, the colour C, transmittance T and their
// derivatives dC (3 x 6), dT (6) with respect to the pose perturbation xi, over
// the same fragments and with the same decisions as k_render_fwd.  With
// m = (d.v1) v1 + (d.v2) v2 = M d (M = log2(e)/2 Sigma2^-1), the exponent
// p = l - d^T M d moves by
//   dp = 2 m . dq + 2 ln2 m^T dSigma2 m
// (d = x - q; dM = -M dSigma2 M / (log2(e)/2)), alpha = 2^p by
// dalpha = alpha ln2 dp unless clamped, and
//   dC += dc w + c (dalpha T + alpha dT),  dT <- dT (1 - alpha) - T dalpha.
// Each pixel then adds H H^T, H r and r^2 (H_ch = dC_ch + bg_ch dT,
// r = target - (C + T bg)) to its thread's 28 sums; the tile sums them over
// its warps and writes one FP32 partial per tile.  Each warp walks the list
// on its own, kPNBatch records per step, compacted by footprint box as in the
// forward.
constexpr int kPNBatch = 16;

template <int TS>
__global__ void __launch_bounds__(TS * TS) k_render_pose_normal(const __grid_constant__ BatchParam bp,
                                                                RenderConst rc,
                                                                const float4* __restrict__ rec,
                                                                const uint2* __restrict__ ranges,
                                                                const uint32_t* __restrict__ tile_order,
                                                                const uint32_t* __restrict__ svals,
                                                                const float4* __restrict__ tan,
                                                                const float* __restrict__ target,
                                                                float* __restrict__ partials,
                                                                float* __restrict__ H_pix,
                                                                uint32_t* __restrict__ order_keys,
                                                                uint32_t* __restrict__ order_vals,
                                                                unsigned long long* __restrict__ counters) {
    pdl_wait();
    pdl_trigger();
    constexpr int NT = TS * TS;
    constexpr int NW = NT / 32;
    __shared__ float4 s_a[NW][kPNBatch];
    __shared__ float4 s_b[NW][kPNBatch];
    __shared__ float2 s_c[NW][kPNBatch];
    __shared__ float4 s_t[NW][kPNBatch][kPoseTan4];
    __shared__ float s_red[NW][kNormalVals];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int w = t >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int tile = (int)tile_order[blockIdx.x];
    const ViewParam& V = bp.v[find_view_by_tile(bp, tile)];
    const int lt = tile - V.tile_off;
    const int ty = lt / V.tiles_x, tx = lt - ty * V.tiles_x;
    const PixelMap<TS, 1> pm(tx, ty, t);
    const int px = pm.px, py = pm.row(0);
    const float fx = px + 0.5f, fy = py + 0.5f;
    const WarpBox wb = warp_box(px, px, py, py);
    const bool inside = px < V.W && py < V.H;
    bool done = !inside;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    float dT[6], dC[3][6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        dT[k] = 0.f;
        dC[0][k] = dC[1][k] = dC[2][k] = 0.f;
    }
    uint2 rg = ranges[tile];
    if (!gs_checked(rg.x <= rg.y && (long long)rg.y <= rc.cap, rc)) rg.y = rg.x;
    uint32_t walked = 0;  // list entries this warp fetched (its walk depth)
    for (uint32_t start = rg.x; start < rg.y; start += kPNBatch) {
        if (__all_sync(0xffffffffu, done)) break;
        walked = min(start + kPNBatch, rg.y) - rg.x;
        const uint32_t idx = start + lane;
        bool reach = false;
        uint32_t r = 0;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
        float4 b = a;
        if (lane < kPNBatch && idx < rg.y && gs_checked((r = svals[idx]) < (uint32_t)bp.total_recs, rc)) {
            a = rec[3 * r];
            c = rec[3 * r + 2];
            reach = wb.reaches(a.x, a.y, c.w);
            if (reach) b = rec[3 * r + 1];
        }
        const uint32_t m = __ballot_sync(0xffffffffu, reach);
        if (reach) {
            const int pos = __popc(m & lt_mask);
            s_a[w][pos] = a;
            s_b[w][pos] = b;
            s_c[w][pos] = make_float2(c.x, c.y);
#pragma unroll
            for (int q = 0; q < kPoseTan4; ++q) s_t[w][pos][q] = tan[(size_t)kPoseTan4 * r + q];
        }
        const int n = __popc(m);
        __syncwarp();
        if (!done) {
            for (int j = 0; j < n; ++j) {
                const float4 ra = s_a[w][j];
                const float4 rb = s_b[w][j];
                const float2 rc2 = s_c[w][j];
                const float dx = fx - ra.x;
                const float dy = fy - ra.y;
                const float t1 = fmaf(dy, ra.w, dx * ra.z);
                const float t2 = fmaf(dy, rb.y, dx * rb.x);
                const float p = fmaf(-t1, t1, fmaf(-t2, t2, rb.z));
                if (p < rc.log2_alpha_min) continue;
                const float araw = ex2_approx(p);
                const float alpha = fminf(rc.alpha_max, araw);
                const float wgt = alpha * T;
                const float Tn = T - wgt;  // as k_render_fwd
                if (Tn < rc.T_min) {
                    done = true;
                    break;
                }
                const float mx = fmaf(t1, ra.z, t2 * rb.x);
                const float my = fmaf(t1, ra.w, t2 * rb.y);
                const float sc = araw < rc.alpha_max ? alpha * kLn2 : 0.f;
                const float k2 = 2.f * kLn2;
                const float mm0 = k2 * mx * mx, mm1 = 2.f * k2 * mx * my, mm2 = k2 * my * my;
                const float m2x = 2.f * mx, m2y = 2.f * my;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    const float4 ta = s_t[w][j][2 * k];
                    const float4 tb = s_t[w][j][2 * k + 1];
                    const float dp = fmaf(m2x, ta.x, fmaf(m2y, ta.y, fmaf(mm0, ta.z, fmaf(mm1, ta.w, mm2 * tb.x))));
                    const float da = sc * dp;
                    const float dw = fmaf(da, T, alpha * dT[k]);
                    dC[0][k] = fmaf(tb.y, wgt, fmaf(rb.w, dw, dC[0][k]));
                    dC[1][k] = fmaf(tb.z, wgt, fmaf(rc2.x, dw, dC[1][k]));
                    dC[2][k] = fmaf(tb.w, wgt, fmaf(rc2.y, dw, dC[2][k]));
                    dT[k] = fmaf(dT[k], 1.f - alpha, -T * da);
                }
                C0 = fmaf(rb.w, wgt, C0);
                C1 = fmaf(rc2.x, wgt, C1);
                C2 = fmaf(rc2.y, wgt, C2);
                T = Tn;
            }
        }
        __syncwarp();
    }
    // this pixel's terms of the normal equations
    float acc[kNormalVals];
#pragma unroll
    for (int e = 0; e < kNormalVals; ++e) acc[e] = 0.f;
    if (inside) {
        const long long hw = (long long)V.W * V.H;
        const long long pl = (long long)py * V.W + px;
        const float* tg = target + 3 * V.pix_off;
        const float Cc[3] = {C0, C1, C2};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float Hc[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) Hc[k] = fmaf(rc.bg[ch], dT[k], dC[ch][k]);
            const float res = tg[ch * hw + pl] - fmaf(T, rc.bg[ch], Cc[ch]);
            int e = 0;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int k = i; k < 6; ++k) {
                    acc[e] = fmaf(Hc[i], Hc[k], acc[e]);
                    ++e;
                }
#pragma unroll
            for (int k = 0; k < 6; ++k) acc[21 + k] = fmaf(Hc[k], res, acc[21 + k]);
            acc[27] = fmaf(res, res, acc[27]);
            if (H_pix) {
                float* hp = H_pix + 18 * (V.pix_off + pl) + 6 * ch;
#pragma unroll
                for (int k = 0; k < 6; ++k) hp[k] = Hc[k];
            }
        }
    }
#pragma unroll
    for (int e = 0; e < kNormalVals; ++e) {
        float v = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[w][e] = v;
    }
    __shared__ uint32_t s_walk[NW];
    if (lane == 0) s_walk[w] = walked;
    __syncthreads();
    if (t == 0) {
        // the tile's walk depth keys it in the next iteration's dispatch
        // order (binning keeps these keys while the tile count matches)
        uint32_t deep = 0;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) deep = max(deep, s_walk[ww]);
        order_keys[tile] = tile_order_key(deep);
        order_vals[tile] = (uint32_t)tile;
        if (blockIdx.x == 0) counters[kCtrOrderTiles] = (unsigned long long)bp.total_tiles;
    }
    if (t < kNormalVals) {
        float v = 0.f;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) v += s_red[ww][t];
        partials[(size_t)tile * kNormalVals + t] = v;
    }
}

// Per view: the FP64 sum of its tiles' partials.  grid.x is the view.
// Per-view totals of the per-tile partials in FP64, in two fixed-order
// stages: kPNChunks blocks per view each sum a contiguous run of the view's
// tiles (warp w of a block takes tiles w, w + 8, ..., lane e value e), then
// one warp per view adds the chunk sums.  The FP64 rate of one SM is a few
// operations per clock, so the sums are spread over many SMs.
constexpr int kPNChunks = 64;
constexpr int kPNChunkWarps = 8;

__global__ void __launch_bounds__(32 * kPNChunkWarps) k_pose_normal_chunks(const __grid_constant__ BatchParam bp,
                                                                         const float* __restrict__ partials,
                                                                         double* __restrict__ chunk_sums) {
    pdl_wait();
    pdl_trigger();
    __shared__ double s_sum[kPNChunkWarps][32];
    const ViewParam& V = bp.v[blockIdx.y];
    const int e = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int ntiles = V.tiles_x * ((V.H + bp.tile_size - 1) / bp.tile_size);
    const int t0 = (int)((long long)ntiles * blockIdx.x / kPNChunks);
    const int t1 = (int)((long long)ntiles * (blockIdx.x + 1) / kPNChunks);
    const float* src = partials + (size_t)V.tile_off * kNormalVals + e;
    double acc = 0.0;
    if (e < kNormalVals)
        for (int tl = t0 + w; tl < t1; tl += kPNChunkWarps) acc += (double)src[(size_t)tl * kNormalVals];
    s_sum[w][e] = acc;
    __syncthreads();
    if (threadIdx.x < kNormalVals) {
        double v = 0.0;
#pragma unroll
        for (int g = 0; g < kPNChunkWarps; ++g) v += s_sum[g][threadIdx.x];
        chunk_sums[((size_t)blockIdx.y * kPNChunks + blockIdx.x) * kNormalVals + threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(32) k_pose_normal_finish(const double* __restrict__ chunk_sums,
                                                           double* __restrict__ normal) {
    pdl_wait();
    pdl_trigger();
    const int e = threadIdx.x;
    if (e >= kNormalVals) return;
    const double* src = chunk_sums + (size_t)blockIdx.x * kPNChunks * kNormalVals + e;
    double v = 0.0;
    for (int c = 0; c < kPNChunks; ++c) v += src[(size_t)c * kNormalVals];
    normal[(size_t)blockIdx.x * kNormalVals + e] = v;
}

}  // namespace

// Compiled raster variants: (tile size, pixels per thread, staging depth).
// Threads per CTA = TS * TS / PPT (a multiple of 32); BATCH is a multiple of it.
#define GS_RASTER_VARIANTS(X) \
    X(8, 1, 128) X(8, 1, 256) X(8, 2, 128) X(8, 2, 256) \
    X(16, 1, 256) X(16, 2, 128) X(16, 2, 256) X(16, 4, 128) X(16, 4, 256) X(16, 8, 128) X(16, 8, 256) \
    X(32, 4, 256) X(32, 8, 128) X(32, 8, 256)

bool raster_variant_exists(int ts, int ppt, int batch) {
#define GS_X(T, P, B) if (ts == T && ppt == P && batch == B) return true;
    GS_RASTER_VARIANTS(GS_X)
#undef GS_X
    return false;
}

cudaError_t launch_render_fwd(const BatchParam& bp, const RenderConst& rc_in, const WsPtrs& ws,
                              float* rgb, float* T_final, uint32_t* n_contrib, uint32_t* n_used,
                              const float* target, float* dL_drgb, float* loss, cudaStream_t s, Prof& pf) {
    RenderConst rc = rc_in;
    rc.cap = tile_list_cap(ws);
    if (bp.total_tiles <= 0) {
        // no pixels: the loss is 0 (the caller's views are all non-empty, so
        // this is unreachable through the C ABI; kept for safety)
        if (target && loss) return cudaMemsetAsync(loss, 0, sizeof(float), s);
        return cudaSuccess;
    }
    const uint32_t* svals = tile_list_vals(ws);
    float* partials = target ? ws.partials : nullptr;
    const int pi = pf.begin(GS_KF_RASTER_FWD, s);
    bool done = false;
#define GS_X(T, P, B)                                                                                  \
    if (!done && bp.tile_size == T && bp.ppt == P && bp.batch == B) {                                  \
        if (n_used)                                                                                    \
            pdl_launch(k_render_fwd<T, P, B, true>, bp.total_tiles, T * T / P, 0, s, bp, rc, ws.rec, ws.ranges, \
                       ws.ovals[1], svals, rgb, T_final, n_contrib, n_used, target, dL_drgb, partials,        \
                       ws.okeys[0], ws.ovals[0], ws.counters);                                            \
        else                                                                                           \
            pdl_launch(k_render_fwd<T, P, B, false>, bp.total_tiles, T * T / P, 0, s, bp, rc, ws.rec, ws.ranges, \
                       ws.ovals[1], svals, rgb, T_final, n_contrib, n_used, target, dL_drgb, partials,        \
                       ws.okeys[0], ws.ovals[0], ws.counters);                                            \
        done = true;                                                                                   \
    }
    GS_RASTER_VARIANTS(GS_X)
#undef GS_X
    pf.end(pi, s);
    if (!done) return cudaErrorInvalidValue;
    if (target && loss) {
        const int pl = pf.begin(GS_KF_L1, s);
        pdl_launch(k_l1_finish, 1, 1024, 0, s, partials, bp.total_tiles, loss);
        pf.end(pl, s);
    }
    // the dispatch order of the next compositing launches (the backward):
    // deepest walk first; not worth its launches when every tile's block is
    // resident at once (at most 16 per SM)
    if (rc.sm_count <= 0 || bp.total_tiles > 16 * rc.sm_count) {
        cudaError_t e = launch_tile_order(ws, bp.total_tiles, rc.status, s, pf);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_render_bwd(const BatchParam& bp, const RenderConst& rc_in, const WsPtrs& ws,
                              const float* T_final, const uint32_t* n_contrib,
                              const float* dL_drgb, cudaStream_t s, Prof& pf) {
    RenderConst rc = rc_in;
    rc.cap = tile_list_cap(ws);
    // deterministic form: per-pair partials, then a fixed-order sum per record
    // (which writes every record, so no clearing)
    const bool det = ws.pair_grad != nullptr;
    cudaError_t e = cudaSuccess;
    if (!det) {
        pf.count(1);
        e = cudaMemsetAsync(ws.grad2d, 0, sizeof(float) * kGrad2D * (size_t)bp.total_recs, s);
    }
    if (e != cudaSuccess || bp.total_tiles <= 0) return e;
    const uint32_t* svals = tile_list_vals(ws);
    const int pi = pf.begin(GS_KF_RASTER_BWD, s, det ? 2 : 1);
    bool done = false;
#define GS_X(T, P, B)                                                                                      \
    if (!done && bp.tile_size == T && bp.ppt == P && bp.batch == B) {                                      \
        if (det)                                                                                           \
            pdl_launch(k_render_bwd<T, P, B, true>, bp.total_tiles, T * T / P, 0, s, bp, rc, ws.rec, ws.ranges, \
                       ws.ovals[1], svals, T_final, n_contrib, dL_drgb, ws.grad2d, ws.pair_grad);         \
        else                                                                                               \
            pdl_launch(k_render_bwd<T, P, B, false>, bp.total_tiles, T * T / P, 0, s, bp, rc, ws.rec, ws.ranges, \
                       ws.ovals[1], svals, T_final, n_contrib, dL_drgb, ws.grad2d, ws.pair_grad);         \
        done = true;                                                                                       \
    }
    GS_RASTER_VARIANTS(GS_X)
#undef GS_X
    if (done && det) {
        // the binning's depth order: its 4-pass radix sort of the 32-bit high
        // words ends in buffer 0, which the tie fix-up reorders in place
        const long long M = bp.total_recs;
        pdl_launch(k_pair_grad_reduce, (unsigned)((M + 255) / 256), 256, 0, s, ws.dvals[0], ws.offsets,
                   ws.tiles_touched, ws.pair_inv, ws.pair_grad, M, ws.cap, ws.counters, ws.grad2d);
    }
    pf.end(pi, s);
    if (!done) return cudaErrorInvalidValue;
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
    pdl_launch(k_l1, grid, kL1Threads, 0, s, bp, rgb, target, dL_drgb, ws.partials);
    if (loss) pdl_launch(k_l1_finish, 1, 1024, 0, s, ws.partials, gx * bp.n_views, loss);
    pf.end(pi, s);
    return cudaGetLastError();
}

// ---- L1 loss without any allocation --------------------------------------
//
// For callers that cannot allocate device memory: its block partial sums live
// in a fixed array in the library's own device memory instead of a caller
// workspace.  The array is loaded with the library on every GPU that uses it
// and kept until the process exits.  Every call on a device shares it, so
// calls whose launches overlap on that device race; each call writes every
// slot it later reads, so nothing has to be cleared between calls.

constexpr long long kL1ScratchFloats = 1ll << 18;  // 1 MiB of FP32 partial sums
constexpr int kL1ScratchDevices = 64;

static __device__ __align__(256) float g_l1_scratch[kL1ScratchFloats];

namespace {
// Device address of g_l1_scratch per device, with the unique id of the CUDA
// context it was looked up in.  Host code only knows a stand-in for the
// array; its device address belongs to the context that loaded the module,
// so a new context on the device (after cudaDeviceReset, for instance) needs
// a new lookup.
struct L1ScratchAddr {
    unsigned long long ctx_id;
    void* ptr;
};
std::mutex g_l1_scratch_mu;
L1ScratchAddr g_l1_scratch_addr[kL1ScratchDevices] = {};

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
bool g_ctx_entry_points_tried = false;

// Unique id of the current CUDA context (false when no context is current or
// the driver lacks the entry points).  Called with g_l1_scratch_mu held.
bool current_context_id(unsigned long long* id) {
    if (!g_ctx_entry_points_tried) {
        g_ctx_entry_points_tried = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&g_ctx_get_current),
                                             12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            g_ctx_get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&g_ctx_get_id), 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            g_ctx_get_id = nullptr;
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return false;
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS || !c) return false;
    return g_ctx_get_id(c, id) == CUDA_SUCCESS;
}
}  // namespace

long long l1_partials_needed(const BatchParam& bp) {
    long long max_px = 0;
    for (int v = 0; v < bp.n_views; ++v) {
        const long long px = (long long)bp.v[v].W * bp.v[v].H;
        if (px > max_px) max_px = px;
    }
    return (long long)l1_grid_x(max_px) * bp.n_views;
}

long long l1_scratch_capacity() { return kL1ScratchFloats; }

cudaError_t launch_l1_static(const BatchParam& bp, const float* rgb, const float* target, float* dL_drgb,
                             float* loss, cudaStream_t s) {
    const long long need = l1_partials_needed(bp);
    if (need > kL1ScratchFloats) return cudaErrorInvalidValue;  // the caller checks this first
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kL1ScratchDevices) return cudaErrorInvalidDevice;
    void* ptr = nullptr;
    {
        // The first call in each context on this device (which is current)
        // looks up the array's device address; later calls in the same
        // context reuse it.
        std::lock_guard<std::mutex> lock(g_l1_scratch_mu);
        L1ScratchAddr& a = g_l1_scratch_addr[dev];
        unsigned long long id = 0;
        const bool have_id = current_context_id(&id);
        if (a.ptr && have_id && a.ctx_id == id) {
            ptr = a.ptr;
        } else {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            e = cudaStreamIsCapturing(s, &cs);
            if (e != cudaSuccess) return e;
            if (cs != cudaStreamCaptureStatusNone) {
                // no lookup while capturing: without a context id to compare,
                // the address of the last lookup is the best there is
                if (!have_id && a.ptr) ptr = a.ptr;
                else return cudaErrorStreamCaptureUnsupported;
            } else {
                e = cudaGetSymbolAddress(&ptr, g_l1_scratch);
                if (e != cudaSuccess) return e;
                unsigned long long id2 = 0;
                a.ptr = ptr;
                a.ctx_id = current_context_id(&id2) ? id2 : 0;
            }
        }
    }
    float* partials = static_cast<float*>(ptr);
    const int gx = (int)(need / bp.n_views);
    dim3 grid(gx, bp.n_views);
    pdl_launch(k_l1, grid, kL1Threads, 0, s, bp, rgb, target, dL_drgb, partials);
    if (loss) pdl_launch(k_l1_finish, 1, 1024, 0, s, partials, (int)need, loss);
    return cudaGetLastError();
}

bool pose_normal_supported(int ts) { return ts == 8 || ts == 16; }

size_t pose_normal_partials_floats(long long n_tiles) {
    return ((size_t)kNormalVals * (size_t)n_tiles + 1) & ~(size_t)1;  // even: the FP64 chunk sums follow
}

size_t pose_normal_chunk_floats(int n_views) { return (size_t)2 * kPNChunks * kNormalVals * (size_t)n_views; }

cudaError_t launch_pose_normal(const BatchParam& bp, const RenderConst& rc_in, const WsPtrs& ws,
                               const float4* tangents, const float* target, float* partials, double* normal,
                               float* H_pix, cudaStream_t s, Prof& pf) {
    RenderConst rc = rc_in;
    rc.cap = tile_list_cap(ws);
    if (bp.total_tiles <= 0) return cudaSuccess;
    const uint32_t* svals = tile_list_vals(ws);
    const int pi = pf.begin(GS_KF_POSE_NORMAL, s, 3);
    if (bp.tile_size == 8)
        pdl_launch(k_render_pose_normal<8>, bp.total_tiles, 64, 0, s, bp, rc, ws.rec, ws.ranges, ws.ovals[1], svals,
                                                               tangents, target, partials, H_pix, ws.okeys[0], ws.ovals[0], ws.counters);
    else if (bp.tile_size == 16)
        pdl_launch(k_render_pose_normal<16>, bp.total_tiles, 256, 0, s, bp, rc, ws.rec, ws.ranges, ws.ovals[1], svals,
                                                                 tangents, target, partials, H_pix, ws.okeys[0], ws.ovals[0], ws.counters);
    else
        return cudaErrorInvalidValue;
    // the chunk sums follow the per-tile partials in the scratch (8-byte aligned)
    double* chunk_sums = reinterpret_cast<double*>(partials + pose_normal_partials_floats(bp.total_tiles));
    pdl_launch(k_pose_normal_chunks, dim3(kPNChunks, bp.n_views), 32 * kPNChunkWarps, 0, s, bp, partials, chunk_sums);
    pdl_launch(k_pose_normal_finish, bp.n_views, 32, 0, s, chunk_sums, normal);
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb

