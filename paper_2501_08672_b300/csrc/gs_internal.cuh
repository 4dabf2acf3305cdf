// Internal declarations shared by the CUDA translation units of libgs_b300.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gs.h"

#include <utility>

namespace gsb {

constexpr int kMaxViews = GS_MAX_VIEWS;
constexpr int kRecFloats = 12;   // projected record: 3 x float4
constexpr int kGrad2D = 9;       // per-record 2D gradient
// Row stride of the deterministic backward's per-pair partials: 9 values
// padded to three 16-byte words.
constexpr int kPairGradStride = 12;
constexpr int kSsimRadius = 5;    // 11-tap SSIM window
constexpr int kPoseTan4 = 12;     // per-record pose tangents: 12 x float4 (see k_pose_tangents)
constexpr int kNormalVals = 28;   // per-view normal equations: 21 + 6 + 1
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Per-view data passed by value to kernels (kernel parameter space).
struct ViewParam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float campos[3];
    int W, H;
    int tiles_x, tiles_y;
    int tile_off;        // first global tile id of the view
    int pad_;
    long long g_begin, g_end;
    long long rec_off;   // first record of the view
    long long pix_off;   // first pixel of the view
};

struct BatchParam {
    int n_views;
    int total_tiles;
    long long total_recs;
    long long total_px;
    int max_count;       // largest g_end - g_begin over views
    int tile_size;
    int ppt;             // pixels per thread of the raster kernels
    int batch;           // records staged per shared-memory batch
    ViewParam v[kMaxViews];
};

// SSIM window taps (normalised Gaussian, sigma 1.5), constants and the
// weight of the structural term.
struct SsimParam {
    float g[2 * kSsimRadius + 1];
    float C1, C2, lambda;
};

struct RenderConst {
    float alpha_min, alpha_max, T_min, blur, z_near;
    float log2_alpha_min;   // -inf when alpha_min == 0
    float bg[3];
    unsigned int* status;   // the context's latched status word
    long long cap;          // pair capacity of the workspace (set by the compositing launches)
    int sm_count;           // SMs of the device (0: unknown)
};

// Bounds checks of the checked build (compiled with -DGS_CHECKED): the
// compositing kernels test every index they read from device memory (a
// tile's pair range against the capacity, a pair's record against the
// record count) before using it.  A failed test latches GS_ERR_BOUNDS in the
// status word (read by gs_sync_status) and the caller skips the access.  In
// the normal build the test is constant true and compiles away.
__device__ __forceinline__ bool gs_checked(bool ok, const RenderConst& rc) {
#ifdef GS_CHECKED
    if (!ok && rc.status) atomicCAS(rc.status, 0u, (unsigned int)(-GS_ERR_BOUNDS));
    return ok;
#else
    (void)ok;
    (void)rc;
    return true;
#endif
}

struct GaussPtrs {
    const float* means;
    const void* log_scales;
    const void* quats;
    const void* opacity;
    const void* sh;
    int scale_dtype, rot_dtype, opacity_dtype, sh_dtype;
    int sh_degree;
    long long n;
};

struct GradPtrs {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity;
    float* sh;
};

// Device-side pointers into the caller's workspace.
struct WsPtrs {
    float4* rec;             // [M][3]
    int4* rect;              // [2M]: per record (x0|y0<<16, x1|y1<<16, first tile id of the view, tiles_x),
                             // (tiles touched, listed-tile mask, 0, 0); 32 bytes, one sector per gather
    uint32_t* tiles_touched; // [M]
    uint32_t* dkeys[2];      // [M] low depth-key words, then scratch
    uint32_t* dvals[2];      // [M]
    uint32_t* dhi;           // [M] high depth-key words
    unsigned long long* offsets; // [M]
    unsigned long long* scan_part; // [scan blocks]
    uint32_t* pkeys[2];      // [cap]
    uint32_t* pvals[2];      // [cap]
    uint32_t* hist;          // [256 * radix tiles]
    uint32_t* hist_part;     // look-back scan: [radix scan chunks + 1] 64-bit flags, then the ticket
    uint2* ranges;           // [T] per compositing tile, into tile_list_vals()
    uint2* ranges_bin;       // [bins] per bin, into pvals[sorted_buf] (== ranges when refine == 1)
    uint32_t* rvals;         // [refine^2 cap] per-tile lists split from the bin lists (refine > 1)
    uint32_t* okeys[2];      // [T] tile-order keys
    uint32_t* ovals[2];      // [T] tiles, longest list first (buffer 1 after the sort)
    float* grad2d;           // [M][9]
    unsigned long long* counters; // [8]: [0] pairs needed, [1..3] depth-key range (kCtrRange*), [4] kCtrOrderTiles
    float* partials;         // reduction scratch
    // deterministic backward only (nullptr otherwise):
    uint32_t* pair_rec;      // [cap] record of each pair at its emission index
    uint32_t* pair_inv;      // [cap] emission index -> place in the tile lists (~0: listed in no tile)
    float* pair_grad;        // [cap][kPairGradStride] per-(tile, record) 2D gradient partials (9 used), at the place in the tile lists
    long long cap;
    int scan_blocks;
    float log2_alpha_min;    // -inf in exact mode (every tile of the box is reached)
    int sorted_buf;          // which pvals buffer holds the sorted pairs
    int refine;              // bin side / tile side: 1 (bins are the tiles), 2 or 4
};

// The records of every compositing tile's list: the sorted pairs, or with
// bins of refine x refine tiles the per-tile lists split from them.
inline const uint32_t* tile_list_vals(const WsPtrs& ws) {
    return ws.refine > 1 ? ws.rvals : ws.pvals[ws.sorted_buf];
}
// Entries of that buffer (the tile ranges stay below it).
inline long long tile_list_cap(const WsPtrs& ws) { return ws.cap * ws.refine * ws.refine; }

// Geometry of the split of bin lists into tile lists: per view, its first
// bin and bins per row, and its first tile and tiles per row and column.
struct RefineGeom {
    int n_views, ts;
    int bin_off[kMaxViews], bins_x[kMaxViews];
    int tile_off[kMaxViews], tiles_x[kMaxViews], tiles_y[kMaxViews];
};

// ---- depth-key range ------------------------------------------------------
//
// The projection records the range [kmin, kmax] of the valid high depth-key
// words (culled records carry 0xFFFFFFFF) in counters[kCtrRangeMax] and
// counters[kCtrRangeMin] by 64-bit atomicMax, with the projection's
// generation counters[kCtrRangeGen] in the high word (kmax, and ~kmin, in the
// low word), so no reset is needed: a value of an older generation loses to
// any of the current one.  Binning advances the generation once its depth
// sort is done.  The depth sort orders records by the 24-bit map of a key,
// (key - kmin) >> s with the least s that keeps the range below 0xFFFFFF, and
// culled keys at 0xFFFFFF; the map is monotone, so equal mapped keys form
// runs that the fix-up orders by the full key.  When the slots do not carry
// the current generation (binning again without a new projection, or a
// workspace never projected into) the map falls back to key >> 8: still
// monotone, with longer runs.
constexpr int kCtrRangeMax = 1;
constexpr int kCtrRangeMin = 2;
constexpr int kCtrRangeGen = 3;
// counters[kCtrOrderTiles]: the tile count the dispatch keys in okeys[0] were
// written for by the last compositing forward (each tile keyed by its walk
// depth); binning orders the next forward by them when it matches.
constexpr int kCtrOrderTiles = 4;

struct KeyMap {
    uint32_t kmin;
    int s;
};

__device__ __forceinline__ KeyMap load_key_map(const unsigned long long* counters) {
    const unsigned long long hi = counters[kCtrRangeMax], lo = counters[kCtrRangeMin];
    const uint32_t gen = (uint32_t)counters[kCtrRangeGen];
    KeyMap m{0u, 8};
    if ((uint32_t)(hi >> 32) == gen && (uint32_t)(lo >> 32) == gen) {
        const uint32_t kmax = (uint32_t)hi, kmin = ~(uint32_t)lo;
        const uint32_t r = kmax >= kmin ? kmax - kmin : 0u;
        int s = 0;
        while ((r >> s) > 0xFFFFFEu) ++s;
        m.kmin = kmin;
        m.s = s;
    }
    return m;
}

__device__ __forceinline__ uint32_t map_key(uint32_t k, const KeyMap& m) {
    return k == 0xFFFFFFFFu ? 0xFFFFFFu : (k - m.kmin) >> m.s;
}

// ---- small device helpers --------------------------------------------------

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float load_as_float(const void* p, int dtype, long long i) {
    if (dtype == GS_F32) return static_cast<const float*>(p)[i];
    if (dtype == GS_F16) return __half2float(static_cast<const __half*>(p)[i]);
    return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

__device__ __forceinline__ int find_view_by_tile(const BatchParam& bp, int tile) {
    int lo = 0, hi = bp.n_views - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (bp.v[mid].tile_off <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Whether a record's footprint {d : (d.v1)^2 + (d.v2)^2 <= L}, centred at q,
// reaches the rectangle [x0, x1] x [y0, y1] (pixel centres of a tile): the
// minimum of the convex quadratic A dx^2 + 2 B dx dy + C dy^2 over the
// rectangle is 0 when q lies inside, else it lies on one of the four edges,
// where it is a clamped 1D minimum.  The small relative margin only adds
// tiles.  Written with explicitly rounded operations so that every caller
// gets bit-identical answers (the pair count and the pair emission must agree).
// For footprint rectangles of up to kMaskTiles tiles the projection stores
// which tiles it listed (a row-major bit mask), so the emission does not
// test them again; larger rectangles are emitted by a whole warp.
constexpr int kMaskTiles = 32;

struct Footprint {
    float qx, qy, A, B, C, nBoA, nBoC, lim;  // nBoA = -B/A, nBoC = -B/C
};

__device__ __forceinline__ Footprint make_footprint(float4 r0, float4 r1, float L) {
    Footprint f;
    f.qx = r0.x;
    f.qy = r0.y;
    f.A = __fmaf_rn(r0.z, r0.z, __fmul_rn(r1.x, r1.x));
    f.B = __fmaf_rn(r0.z, r0.w, __fmul_rn(r1.x, r1.y));
    f.C = __fmaf_rn(r0.w, r0.w, __fmul_rn(r1.y, r1.y));
    f.nBoA = __fdiv_rn(-f.B, f.A);
    f.nBoC = __fdiv_rn(-f.B, f.C);
    f.lim = __fmaf_rn(L, 1.001f, 1e-3f);
    return f;
}

__device__ __forceinline__ bool footprint_hits_rect(const Footprint& f, float x0, float x1, float y0, float y1) {
    const float ax = __fadd_rn(x0, -f.qx), bx = __fadd_rn(x1, -f.qx);
    const float ay = __fadd_rn(y0, -f.qy), by = __fadd_rn(y1, -f.qy);
    if (ax <= 0.f && bx >= 0.f && ay <= 0.f && by >= 0.f) return true;
    auto q2 = [&](float dx, float dy) {
        return __fmaf_rn(__fmul_rn(f.A, dx), dx,
                         __fmaf_rn(__fmul_rn(2.f, __fmul_rn(f.B, dx)), dy, __fmul_rn(__fmul_rn(f.C, dy), dy)));
    };
    // horizontal edges (dy fixed): minimiser dx = -B dy / A; vertical: dy = -B dx / C
    float best = q2(fminf(fmaxf(__fmul_rn(f.nBoA, ay), ax), bx), ay);
    best = fminf(best, q2(fminf(fmaxf(__fmul_rn(f.nBoA, by), ax), bx), by));
    best = fminf(best, q2(ax, fminf(fmaxf(__fmul_rn(f.nBoC, ax), ay), by)));
    best = fminf(best, q2(bx, fminf(fmaxf(__fmul_rn(f.nBoC, bx), ay), by)));
    return best <= f.lim;
}

// Row spans of the same ellipse q(d) <= lim (q = A dx^2 + 2B dx dy + C dy^2,
// d = pixel centre - q), for counting and emitting the tiles it reaches one
// tile row at a time: within a row's band of pixel-centre rows the ellipse's
// x-extent is an interval, and the tiles whose pixel-centre columns meet it
// are a contiguous run.  This lists exactly the tiles footprint_hits_rect
// accepts, up to rounding far inside the margin of lim.  det = AC - B^2 is
// formed as (v1x v2y - v2x v1y)^2 (Lagrange's identity), so thin footprints
// keep it accurate; rightmost point of the ellipse at dy = dyr, leftmost at
// -dyr; |dy| <= ymax on the ellipse.
struct FootRows {
    float qx, qy, A, B, det, invA, ymax, dyr, lim;
};

__device__ __forceinline__ FootRows make_footrows(float4 r0, float4 r1, float L) {
    FootRows f;
    f.qx = r0.x;
    f.qy = r0.y;
    f.A = __fmaf_rn(r0.z, r0.z, __fmul_rn(r1.x, r1.x));
    f.B = __fmaf_rn(r0.z, r0.w, __fmul_rn(r1.x, r1.y));
    const float C = __fmaf_rn(r0.w, r0.w, __fmul_rn(r1.y, r1.y));
    const float dv = __fmaf_rn(r0.z, r1.y, -__fmul_rn(r1.x, r0.w));
    f.det = __fmul_rn(dv, dv);
    f.lim = __fmaf_rn(L, 1.001f, 1e-3f);
    f.invA = __frcp_rn(f.A);
    f.ymax = __fsqrt_rn(__fdiv_rn(__fmul_rn(f.A, f.lim), f.det));
    const float xmax = __fsqrt_rn(__fdiv_rn(__fmul_rn(C, f.lim), f.det));
    f.dyr = __fdiv_rn(__fmul_rn(-f.B, xmax), C);
    return f;
}

// Square root by the hardware's approximate instruction (relative error about
// 2^-22); the row spans below take their x-extents from it, far inside the
// 0.1 % margin on lim, and the projection and the emission share the code.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Tile columns [*a, *b] of tile row ty (clipped to [tx0, tx1)) that the
// ellipse reaches; false when none.
__device__ __forceinline__ bool footrows_span(const FootRows& f, int ty, int ts, int tx0, int tx1, int* a,
                                              int* b) {
    const float ya = __fadd_rn((float)(ty * ts) + 0.5f, -f.qy);
    const float yb = __fadd_rn((float)(ty * ts + ts) - 0.5f, -f.qy);
    const float lo = fmaxf(ya, -f.ymax), hi = fminf(yb, f.ymax);
    if (!(lo <= hi)) return false;
    const float dR = fminf(fmaxf(f.dyr, lo), hi);
    const float dL = fminf(fmaxf(-f.dyr, lo), hi);
    const float sR = sqrt_approx(fmaxf(__fmaf_rn(-f.det, __fmul_rn(dR, dR), __fmul_rn(f.A, f.lim)), 0.f));
    const float sL = sqrt_approx(fmaxf(__fmaf_rn(-f.det, __fmul_rn(dL, dL), __fmul_rn(f.A, f.lim)), 0.f));
    const float xr = __fmul_rn(__fadd_rn(__fmul_rn(-f.B, dR), sR), f.invA);
    const float xl = __fmul_rn(__fadd_rn(__fmul_rn(-f.B, dL), -sL), f.invA);
    // tile tx is reached when tx ts + 0.5 <= qx + xr and tx ts + ts - 0.5 >= qx + xl
    const float inv_ts = __int_as_float((128 - __ffs(ts)) << 23);  // 1 / ts, exact (ts a power of two)
    const int ta = max(tx0, (int)ceilf(__fmul_rn(__fadd_rn(__fadd_rn(f.qx, xl), 0.5f), inv_ts) - 1.f));
    const int tb = min(tx1 - 1, (int)floorf(__fmul_rn(__fadd_rn(__fadd_rn(f.qx, xr), -0.5f), inv_ts)));
    if (ta > tb) return false;
    *a = ta;
    *b = tb;
    return true;
}

// Dispatch key of a tile in the longest-first order of the compositing
// launches: 255 - a log-scale code of its work (16 steps per octave), so one
// stable 8-bit radix pass puts the heaviest tiles first.
__device__ __forceinline__ uint32_t tile_order_key(uint32_t len) {
    uint32_t code = 0;
    if (len) {
        const int e = 31 - __clz(len);
        const uint32_t m = e >= 4 ? (len >> (e - 4)) & 15u : (len << (4 - e)) & 15u;
        code = min(255u, (uint32_t)e * 16u + m);
    }
    return 255u - code;
}

// ---- programmatic dependent launch ----------------------------------------
//
// Every kernel of the library starts with pdl_wait() and pdl_trigger() and is
// launched by pdl_launch with programmatic stream serialization, so in a
// stream (and in a captured graph) the next kernel is launched while this
// one drains and its blocks wait in pdl_wait() until this grid has completed
// and its memory is visible.  The wait comes first, before any early return:
// a kernel's completion then implies the completion of everything before it
// in the stream.  Without a programmatic dependency both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);  // errors surface via cudaGetLastError
}

// ---- host-side launch accounting and optional event timing ---------------

struct Prof {
    uint32_t mask = 0;
    long long launches = 0;
    struct Rec {
        int fam;
        cudaEvent_t a, b;
    };
    Rec* recs = nullptr;     // pending timed launches
    int n_recs = 0, cap_recs = 0;
    cudaEvent_t* pool = nullptr;
    int pool_size = 0, pool_used = 0;

    // Counts `n` launches of family `fam`; returns a record index when the
    // family is timed (the start event is recorded on `s`), else -1.
    int begin(int fam, cudaStream_t s, int n = 1);
    void count(int n) { launches += n; }
    void end(int idx, cudaStream_t s);
    void release();
};

// ---- launch wrappers (host), one per kernel family ------------------------

cudaError_t launch_project(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                           const WsPtrs& ws, cudaStream_t s, Prof& pf);
// bp: the batch at the bin size; with ws.refine > 1, geom and n_tiles give
// the compositing tiles the bin lists are split into.
// Reorders the compositing tiles (ws.ovals[1]) by the keys in ws.okeys[0] /
// ws.ovals[0] (one stable 8-bit radix pass over n_tiles).
cudaError_t launch_tile_order(const WsPtrs& ws, int n_tiles, unsigned int* status, cudaStream_t s, Prof& pf);
cudaError_t launch_bin(const BatchParam& bp, WsPtrs& ws, unsigned int* status,
                       unsigned long long* status_pairs, cudaStream_t s, Prof& pf,
                       const RefineGeom* geom = nullptr, int n_tiles = 0);
bool raster_variant_exists(int ts, int ppt, int batch);
cudaError_t measure_alu(int sm_count, float* sink, cudaStream_t s, double* ffma_tflops, double* ex2_gops);
size_t selftest_wait_scratch_bytes();
cudaError_t launch_selftest_wait(void* scratch, unsigned int* status, cudaStream_t s);
size_t ssim_scratch_floats(const BatchParam& bp);
cudaError_t launch_ssim(const BatchParam& bp, const SsimParam& sp, const float* rgb, const float* target,
                        float* scratch, float* dL_drgb, float* loss, cudaStream_t s, Prof& pf);
int window_max_columns();
size_t window_scratch_bytes(long long n);
cudaError_t launch_window_compact(const gs_window_column* cols, const gs_window_column* leave_dst, int n_cols,
                                  long long n, const uint8_t* keep, long long* n_keep_dev, int32_t* moved_from,
                                  int32_t* leaving_rows, void* scratch, int sm_count, cudaStream_t s, Prof& pf);
cudaError_t launch_window_gather(const gs_window_column* src, const gs_window_column* dst, int n_cols,
                                 const int32_t* idx, long long m, long long n, int sm_count, cudaStream_t s,
                                 Prof& pf);
cudaError_t launch_window_clear(const gs_window_column* cols, int n_cols, long long begin, long long end,
                                int sm_count, cudaStream_t s, Prof& pf);
cudaError_t launch_sh_init(const ViewParam& V, const float* means, const float* image, long long begin,
                           long long end, int sh_degree, float z_near, float* sh, cudaStream_t s, Prof& pf);
cudaError_t launch_pose_tangents(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                                 const WsPtrs& ws, float4* tangents, cudaStream_t s, Prof& pf);
bool pose_normal_supported(int ts);
// Scratch of the pose normal equations after the per-record tangents: the
// per-tile partials (an even number of floats), then the FP64 chunk sums.
size_t pose_normal_partials_floats(long long n_tiles);
size_t pose_normal_chunk_floats(int n_views);
cudaError_t launch_pose_normal(const BatchParam& bp, const RenderConst& rc, const WsPtrs& ws,
                               const float4* tangents, const float* target, float* partials, double* normal,
                               float* H_pix, cudaStream_t s, Prof& pf);
// target non-null: also the L1 loss (dL_drgb, and loss when non-null) from
// per-tile partials in ws.partials (one per tile); rgb may then be null.
cudaError_t launch_render_fwd(const BatchParam& bp, const RenderConst& rc, const WsPtrs& ws,
                              float* rgb, float* T_final, uint32_t* n_contrib, uint32_t* n_used,
                              const float* target, float* dL_drgb, float* loss, cudaStream_t s, Prof& pf);
cudaError_t launch_render_bwd(const BatchParam& bp, const RenderConst& rc, const WsPtrs& ws,
                              const float* T_final, const uint32_t* n_contrib,
                              const float* dL_drgb, cudaStream_t s, Prof& pf);
cudaError_t launch_project_bwd(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                               const WsPtrs& ws, const GradPtrs* grads, float* dL_dpose,
                               cudaStream_t s, Prof& pf, bool accumulate = false);
cudaError_t launch_l1(const BatchParam& bp, const WsPtrs& ws, const float* rgb,
                      const float* target, float* dL_drgb, float* loss, cudaStream_t s, Prof& pf);
long long l1_partials_needed(const BatchParam& bp);
long long l1_scratch_capacity();
cudaError_t launch_l1_static(const BatchParam& bp, const float* rgb, const float* target, float* dL_drgb,
                             float* loss, cudaStream_t s);
cudaError_t launch_adam_ranges(float* p, const float* g, float* m, float* v, const gs_range* ranges, int n_ranges,
                               float b1, float b2, float eps, float step_size, float inv_sqrt_bc2,
                               const gs_lowp_segment* segs, int n_segs, cudaStream_t s, Prof& pf,
                               long long* step_dev, float lr, float2* coef, int sm_count);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n,
                        float b1, float b2, float eps, float step_size, float inv_sqrt_bc2,
                        const gs_lowp_segment* segs, int n_segs, cudaStream_t s, Prof& pf,
                        long long* step_dev = nullptr, float lr = 0.f, float2* coef = nullptr);

}  // namespace gsb
