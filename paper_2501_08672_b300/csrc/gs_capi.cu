// C ABI of libgs_b300: argument validation, workspace layout, view tables and
// kernel orchestration.  Every entry point validates on the host, launches on
// the caller's stream and returns a gs_status; nothing here synchronises or
// allocates except context creation/destruction and gs_sync_status (and
// gs_bin when the caller asks for the pair count).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "gs_internal.cuh"

struct gs_ctx {
    int device;
    gs_config cfg;
    int sm_count;
    gsb::Prof prof;
    unsigned int* d_status;           // [0] latched status (negated gs_status), [2..3] pair count
    unsigned long long* d_pairs;      // points into d_status
    float2* d_adam_coef;              // points into d_status (bytes 64..71)
    char err[512];
};

namespace gsb {

int Prof::begin(int fam, cudaStream_t s, int n) {
    launches += n;
    if (!(mask & (1u << fam))) return -1;
    if (pool_used + 2 > pool_size) {
        const int grow = pool_size ? pool_size : 256;
        cudaEvent_t* np = static_cast<cudaEvent_t*>(realloc(pool, sizeof(cudaEvent_t) * (pool_size + grow)));
        if (!np) return -1;
        pool = np;
        for (int k = 0; k < grow; ++k)
            if (cudaEventCreate(&pool[pool_size + k]) != cudaSuccess) {
                cudaGetLastError();
                return -1;
            }
        pool_size += grow;
    }
    if (n_recs == cap_recs) {
        const int nc = cap_recs ? 2 * cap_recs : 128;
        Rec* nr = static_cast<Rec*>(realloc(recs, sizeof(Rec) * nc));
        if (!nr) return -1;
        recs = nr;
        cap_recs = nc;
    }
    Rec& r = recs[n_recs];
    r.fam = fam;
    r.a = pool[pool_used++];
    r.b = pool[pool_used++];
    cudaEventRecord(r.a, s);
    return n_recs++;
}

void Prof::end(int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(recs[idx].b, s);
}

void Prof::release() {
    for (int k = 0; k < pool_size; ++k) cudaEventDestroy(pool[k]);
    free(pool);
    free(recs);
    pool = nullptr;
    recs = nullptr;
    pool_size = pool_used = n_recs = cap_recs = 0;
}

}  // namespace gsb

namespace {

using namespace gsb;

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int fail(gs_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

// Error text into a caller-supplied buffer (for entry points without a context).
int fail_msg(char* msg, size_t len, int code, const char* fmt, ...) {
    if (msg && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, len, fmt, ap);
        va_end(ap);
    }
    return code;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int tile_key_bits(int total_tiles) {
    int b = 1;
    while ((1ll << b) < (long long)total_tiles) ++b;
    return b;
}

int sorted_buffer(int total_tiles) {
    const int bits = tile_key_bits(total_tiles);
    const int passes = (bits + 7) / 8;
    return passes % 2;
}

struct Layout {
    gs_ws_layout pub;
    size_t scan_part, dkeys1, dvals1, pkeys1, pvals1, hist, hist_part, partials, okeys0, okeys1, ovals0, ovals1;
    size_t pair_rec, pair_inv, pair_grad;  // deterministic backward (0 when off)
    size_t rvals;                          // per-tile lists split from the bins (0 when the bins are the tiles)
    int scan_blocks;
    int bin_tiles;                         // bins (== tiles when refine == 1)
    int refine;                            // bin side / tile side
    long long max_g_end;
};

// The binning's tile size: gs_config.bin_tile_size where it applies
// (truncated mode, not deterministic), else the compositing tile size.
int bin_size_of(const gs_config& c) {
    if (c.bin_tile_size == 0 || c.bin_tile_size == c.tile_size || c.deterministic || !(c.alpha_min > 0.f))
        return c.tile_size;
    return c.bin_tile_size;
}

int l1_blocks_x(long long max_px) { return (int)((3 * max_px + 1023) / 1024); }

// Validates the views (host) and computes the workspace layout.
int make_layout(gs_ctx* ctx, const gs_config& cfg, const gs_view* views, int n_views,
                int64_t max_pairs, Layout& L) {
    if (!views) return fail(ctx, GS_ERR_INVALID_ARG, "views is NULL");
    if (n_views < 1 || n_views > GS_MAX_VIEWS)
        return fail(ctx, GS_ERR_INVALID_ARG, "n_views=%d outside [1, %d]", n_views, GS_MAX_VIEWS);
    if (max_pairs < 0 || max_pairs > 0x7FFFFFFFll)
        return fail(ctx, GS_ERR_INVALID_ARG, "max_pairs=%lld outside [0, 2^31)", (long long)max_pairs);
    const int ts = cfg.tile_size;
    int bs = bin_size_of(cfg);
    long long M = 0, P = 0, T = 0, Tb = 0, max_px = 0, max_g_end = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_view& V = views[v];
        if (V.width <= 0 || V.height <= 0 || V.width > 32768 || V.height > 32768)
            return fail(ctx, GS_ERR_INVALID_ARG, "view %d: size %dx%d outside [1, 32768]", v, V.width, V.height);
        if (V.g_begin < 0 || V.g_end <= V.g_begin)
            return fail(ctx, GS_ERR_INVALID_ARG, "view %d: empty or negative Gaussian range [%lld, %lld)", v,
                        (long long)V.g_begin, (long long)V.g_end);
        for (int k = 0; k < 9; ++k)
            if (!isfinite(V.R_cw[k])) return fail(ctx, GS_ERR_NONFINITE, "view %d: R_cw not finite", v);
        for (int k = 0; k < 3; ++k)
            if (!isfinite(V.t_cw[k])) return fail(ctx, GS_ERR_NONFINITE, "view %d: t_cw not finite", v);
        if (!isfinite(V.fx) || !isfinite(V.fy) || !isfinite(V.cx) || !isfinite(V.cy))
            return fail(ctx, GS_ERR_NONFINITE, "view %d: intrinsics not finite", v);
        if (!(V.fx > 0.f) || !(V.fy > 0.f))
            return fail(ctx, GS_ERR_INVALID_ARG, "view %d: focal lengths must be positive", v);
        M += V.g_end - V.g_begin;
        const long long tx = (V.width + ts - 1) / ts, ty = (V.height + ts - 1) / ts;
        T += tx * ty;
        Tb += (long long)((V.width + bs - 1) / bs) * ((V.height + bs - 1) / bs);
        P += (long long)V.width * V.height;
        if ((long long)V.width * V.height > max_px) max_px = (long long)V.width * V.height;
        if (V.g_end > max_g_end) max_g_end = V.g_end;
    }
    if (M >= 0xFFFFFFFFll) return fail(ctx, GS_ERR_INVALID_ARG, "too many (view, Gaussian) records: %lld", M);
    if (T >= 0x7FFFFFFFll) return fail(ctx, GS_ERR_INVALID_ARG, "too many tiles: %lld", T);

    // the pair keys hold a bin id below the F^2-bit tile mask, and the id
    // 2^(32 - F^2) - 1 marks unlisted pairs: with more bins, bin at the tile size
    if (bs != ts && Tb >= (1ll << (32 - (bs / ts) * (bs / ts))) - 1) {
        bs = ts;
        Tb = T;
    }
    const long long cap = max_pairs;
    L.refine = bs / ts;
    L.bin_tiles = (int)Tb;
    if ((long long)L.refine * L.refine * cap >= 0xFFFFFFFFll)
        return fail(ctx, GS_ERR_INVALID_ARG, "max_pairs=%lld: %d^2 max_pairs must stay below 2^32 with bins of %d",
                    (long long)max_pairs, L.refine, bs);
    long long big = M > cap ? M : cap;
    if (T > big) big = T;
    if (Tb > big) big = Tb;
    const long long radix_tiles = (big + 4095) / 4096;      // tiles of the radix sort passes
    const long long hist_parts = (256 * radix_tiles + 4095) / 4096;
    L.scan_blocks = (int)((M + 4095) / 4096);
    L.max_g_end = max_g_end;
    const long long pose_blocks = (max_g_end + 255) / 256;
    long long partials = (long long)n_views * pose_blocks * 6;
    const long long l1 = (long long)n_views * l1_blocks_x(max_px);
    if (l1 > partials) partials = l1;
    if (T > partials) partials = T;  // the L1 loss folded into the forward: one partial per tile

    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off = align_up(off + bytes); return o; };
    gs_ws_layout& W = L.pub;
    memset(&W, 0, sizeof(W));
    W.records = take(sizeof(float) * kRecFloats * (size_t)M);
    W.rects = take(2 * sizeof(int4) * (size_t)M);
    W.tiles_touched = take(sizeof(uint32_t) * (size_t)M);
    W.depth_keys = take(sizeof(uint32_t) * (size_t)M);
    L.dkeys1 = take(sizeof(uint32_t) * (size_t)M);
    W.depth_hi = take(sizeof(uint32_t) * (size_t)M);
    W.depth_vals = take(sizeof(uint32_t) * (size_t)M);
    L.dvals1 = take(sizeof(uint32_t) * (size_t)M);
    W.pair_offsets = take(sizeof(unsigned long long) * (size_t)M);
    L.scan_part = take(sizeof(unsigned long long) * (size_t)(L.scan_blocks + 1));
    W.pair_keys = take(sizeof(uint32_t) * (size_t)cap);
    L.pkeys1 = take(sizeof(uint32_t) * (size_t)cap);
    W.pair_vals = take(sizeof(uint32_t) * (size_t)cap);
    L.pvals1 = take(sizeof(uint32_t) * (size_t)cap);
    L.hist = take(sizeof(uint32_t) * 256 * (size_t)(radix_tiles > 0 ? radix_tiles : 1));
    L.hist_part = take(sizeof(unsigned long long) * (size_t)(hist_parts + 2));  // look-back flags + ticket
    W.tile_ranges = take(sizeof(uint2) * (size_t)T);
    W.bin_ranges = L.refine > 1 ? take(sizeof(uint2) * (size_t)Tb) : W.tile_ranges;
    L.rvals = L.refine > 1 ? take(sizeof(uint32_t) * (size_t)(L.refine * L.refine) * (size_t)cap) : 0;
    L.okeys0 = take(sizeof(uint32_t) * (size_t)T);
    L.okeys1 = take(sizeof(uint32_t) * (size_t)T);
    L.ovals0 = take(sizeof(uint32_t) * (size_t)T);
    L.ovals1 = take(sizeof(uint32_t) * (size_t)T);
    W.grad2d = take(sizeof(float) * kGrad2D * (size_t)M);
    W.counters = take(sizeof(unsigned long long) * 8);
    L.partials = take(sizeof(float) * (size_t)partials);
    L.pair_rec = L.pair_inv = L.pair_grad = 0;
    if (cfg.deterministic) {
        L.pair_rec = take(sizeof(uint32_t) * (size_t)cap);
        L.pair_inv = take(sizeof(uint32_t) * (size_t)cap);
        L.pair_grad = take(sizeof(float) * kPairGradStride * (size_t)cap);
    }
    W.total = off;
    W.bin_keys = sorted_buffer((int)Tb) ? L.pkeys1 : W.pair_keys;
    W.bin_vals = sorted_buffer((int)Tb) ? L.pvals1 : W.pair_vals;
    W.sorted_vals = L.refine > 1 ? L.rvals : W.bin_vals;
    W.n_records = M;
    W.n_tiles = (int32_t)T;
    W.n_pixels = P;
    W.n_bins = (int32_t)Tb;
    W.bin_size = bs;
    return GS_OK;
}

int check_ws(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws, Layout& L) {
    if (!ws || !ws->ptr) return fail(ctx, GS_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws->ptr) % kAlign)
        return fail(ctx, GS_ERR_INVALID_ARG, "workspace base is not 256-byte aligned");
    int rc = make_layout(ctx, ctx->cfg, views, n_views, ws->max_pairs, L);
    if (rc) return rc;
    if (ws->bytes < L.pub.total)
        return fail(ctx, GS_ERR_INVALID_ARG, "workspace has %zu bytes, needs %zu", ws->bytes, L.pub.total);
    return GS_OK;
}

WsPtrs ws_ptrs(const gs_workspace* ws, const Layout& L) {
    char* b = static_cast<char*>(ws->ptr);
    WsPtrs p{};
    p.rec = reinterpret_cast<float4*>(b + L.pub.records);
    p.rect = reinterpret_cast<int4*>(b + L.pub.rects);
    p.tiles_touched = reinterpret_cast<uint32_t*>(b + L.pub.tiles_touched);
    p.dkeys[0] = reinterpret_cast<uint32_t*>(b + L.pub.depth_keys);
    p.dkeys[1] = reinterpret_cast<uint32_t*>(b + L.dkeys1);
    p.dvals[0] = reinterpret_cast<uint32_t*>(b + L.pub.depth_vals);
    p.dvals[1] = reinterpret_cast<uint32_t*>(b + L.dvals1);
    p.dhi = reinterpret_cast<uint32_t*>(b + L.pub.depth_hi);
    p.offsets = reinterpret_cast<unsigned long long*>(b + L.pub.pair_offsets);
    p.scan_part = reinterpret_cast<unsigned long long*>(b + L.scan_part);
    p.pkeys[0] = reinterpret_cast<uint32_t*>(b + L.pub.pair_keys);
    p.pkeys[1] = reinterpret_cast<uint32_t*>(b + L.pkeys1);
    p.pvals[0] = reinterpret_cast<uint32_t*>(b + L.pub.pair_vals);
    p.pvals[1] = reinterpret_cast<uint32_t*>(b + L.pvals1);
    p.hist = reinterpret_cast<uint32_t*>(b + L.hist);
    p.hist_part = reinterpret_cast<uint32_t*>(b + L.hist_part);
    p.ranges = reinterpret_cast<uint2*>(b + L.pub.tile_ranges);
    p.ranges_bin = reinterpret_cast<uint2*>(b + L.pub.bin_ranges);
    p.rvals = L.rvals ? reinterpret_cast<uint32_t*>(b + L.rvals) : nullptr;
    p.refine = L.refine;
    p.okeys[0] = reinterpret_cast<uint32_t*>(b + L.okeys0);
    p.okeys[1] = reinterpret_cast<uint32_t*>(b + L.okeys1);
    p.ovals[0] = reinterpret_cast<uint32_t*>(b + L.ovals0);
    p.ovals[1] = reinterpret_cast<uint32_t*>(b + L.ovals1);
    p.grad2d = reinterpret_cast<float*>(b + L.pub.grad2d);
    p.counters = reinterpret_cast<unsigned long long*>(b + L.pub.counters);
    p.partials = reinterpret_cast<float*>(b + L.partials);
    p.pair_rec = L.pair_rec ? reinterpret_cast<uint32_t*>(b + L.pair_rec) : nullptr;
    p.pair_inv = L.pair_inv ? reinterpret_cast<uint32_t*>(b + L.pair_inv) : nullptr;
    p.pair_grad = L.pair_grad ? reinterpret_cast<float*>(b + L.pair_grad) : nullptr;
    p.cap = ws->max_pairs;
    p.scan_blocks = L.scan_blocks;
    p.sorted_buf = sorted_buffer(L.bin_tiles);
    p.log2_alpha_min = -INFINITY;
    return p;
}

// Default launch shape: the fastest measured at the headline workload for
// each tile size (16 x 16 tiles at 2 pixels per thread and 128-record batches
// win by 5 % and more over the other shapes).
int default_ppt(int ts) { return ts == 32 ? 4 : 2; }
int default_batch(int ts, int ppt) { return ts * ts / ppt <= 128 ? 128 : 256; }

// The batch with tiles of cfg.tile_size pixels, or of ts pixels (the bins)
// when ts is nonzero.
void make_batch(const gs_config& cfg, const gs_view* views, int n_views, BatchParam& bp, int ts = 0) {
    memset(&bp, 0, sizeof(bp));
    if (ts == 0) ts = cfg.tile_size;
    bp.n_views = n_views;
    bp.tile_size = ts;
    bp.ppt = cfg.pixels_per_thread ? cfg.pixels_per_thread : default_ppt(cfg.tile_size);
    bp.batch = cfg.batch ? cfg.batch : default_batch(cfg.tile_size, bp.ppt);
    long long rec = 0, pix = 0;
    int tiles = 0, maxc = 0;
    for (int v = 0; v < n_views; ++v) {
        const gs_view& S = views[v];
        ViewParam& V = bp.v[v];
        memcpy(V.R, S.R_cw, sizeof(V.R));
        memcpy(V.t, S.t_cw, sizeof(V.t));
        V.fx = S.fx; V.fy = S.fy; V.cx = S.cx; V.cy = S.cy;
        for (int k = 0; k < 3; ++k) {  // camera centre -R^T t
            const double c = -((double)S.R_cw[k] * S.t_cw[0] + (double)S.R_cw[3 + k] * S.t_cw[1] +
                               (double)S.R_cw[6 + k] * S.t_cw[2]);
            V.campos[k] = (float)c;
        }
        V.W = S.width; V.H = S.height;
        V.tiles_x = (S.width + ts - 1) / ts;
        V.tiles_y = (S.height + ts - 1) / ts;
        V.tile_off = tiles;
        V.g_begin = S.g_begin; V.g_end = S.g_end;
        V.rec_off = rec;
        V.pix_off = pix;
        tiles += V.tiles_x * V.tiles_y;
        rec += S.g_end - S.g_begin;
        pix += (long long)S.width * S.height;
        if (S.g_end - S.g_begin > maxc) maxc = (int)(S.g_end - S.g_begin);
    }
    bp.total_tiles = tiles;
    bp.total_recs = rec;
    bp.total_px = pix;
    bp.max_count = maxc;
}

RenderConst make_rc(const gs_config& c) {
    RenderConst r;
    r.alpha_min = c.alpha_min;
    r.alpha_max = c.alpha_max;
    r.T_min = c.T_min;
    r.blur = c.blur;
    r.z_near = c.z_near;
    r.log2_alpha_min = c.alpha_min > 0.f ? log2f(c.alpha_min) : -INFINITY;
    for (int k = 0; k < 3; ++k) r.bg[k] = c.bg[k];
    r.status = nullptr;
    r.cap = 0;
    r.sm_count = 0;
    return r;
}

// The context's render constants: its configuration and its status word.
RenderConst ctx_rc(const gs_ctx* ctx) {
    RenderConst r = make_rc(ctx->cfg);
    r.status = ctx->d_status;
    r.sm_count = ctx->sm_count;
    return r;
}

int check_gaussians(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views, GaussPtrs& out) {
    if (!g) return fail(ctx, GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (!g->means || !g->log_scales || !g->quats || !g->opacity || !g->sh)
        return fail(ctx, GS_ERR_INVALID_ARG, "a Gaussian attribute pointer is NULL");
    if (g->n <= 0) return fail(ctx, GS_ERR_INVALID_ARG, "n=%lld must be positive", (long long)g->n);
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(ctx, GS_ERR_INVALID_ARG, "sh_degree=%d not in [0, 3]", g->sh_degree);
    const int dts[4] = {g->scale_dtype, g->rot_dtype, g->opacity_dtype, g->sh_dtype};
    for (int k = 0; k < 4; ++k)
        if (dts[k] < GS_F32 || dts[k] > GS_BF16) return fail(ctx, GS_ERR_INVALID_ARG, "bad dtype %d", dts[k]);
    for (int v = 0; v < n_views; ++v)
        if (views[v].g_end > g->n)
            return fail(ctx, GS_ERR_INVALID_ARG, "view %d: g_end=%lld exceeds n=%lld", v,
                        (long long)views[v].g_end, (long long)g->n);
    out.means = g->means;
    out.log_scales = g->log_scales;
    out.quats = g->quats;
    out.opacity = g->opacity;
    out.sh = g->sh;
    out.scale_dtype = g->scale_dtype;
    out.rot_dtype = g->rot_dtype;
    out.opacity_dtype = g->opacity_dtype;
    out.sh_dtype = g->sh_dtype;
    out.sh_degree = g->sh_degree;
    out.n = g->n;
    return GS_OK;
}

int cuda_fail(gs_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, GS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

int check_config(const gs_config& c, char* msg, size_t n) {
    if (c.tile_size != 8 && c.tile_size != 16 && c.tile_size != 32) {
        snprintf(msg, n, "tile_size=%d not in {8, 16, 32}", c.tile_size);
        return GS_ERR_INVALID_ARG;
    }
    const int ppt = c.pixels_per_thread ? c.pixels_per_thread : default_ppt(c.tile_size);
    const int batch = c.batch ? c.batch : default_batch(c.tile_size, ppt);
    if (!raster_variant_exists(c.tile_size, ppt, batch)) {
        snprintf(msg, n, "no compositing kernel for tile %d, %d pixels per thread, batch %d", c.tile_size, ppt, batch);
        return GS_ERR_INVALID_ARG;
    }
    if (!(c.alpha_min >= 0.f) || !(c.alpha_max > c.alpha_min) || !(c.alpha_max <= 1.f) || !(c.T_min >= 0.f) ||
        !(c.T_min < 1.f) || !(c.blur >= 0.f) || !(c.z_near > 0.f)) {
        snprintf(msg, n, "config constants out of range");
        return GS_ERR_INVALID_ARG;
    }
    for (int k = 0; k < 3; ++k)
        if (!isfinite(c.bg[k])) {
            snprintf(msg, n, "background not finite");
            return GS_ERR_INVALID_ARG;
        }
    if (c.deterministic != 0 && c.deterministic != 1) {
        snprintf(msg, n, "deterministic=%d not in {0, 1}", c.deterministic);
        return GS_ERR_INVALID_ARG;
    }
    if (c.bin_tile_size != 0 && c.bin_tile_size != c.tile_size && c.bin_tile_size != 2 * c.tile_size &&
        c.bin_tile_size != 4 * c.tile_size) {
        snprintf(msg, n, "bin_tile_size=%d is not 0 or 1, 2 or 4 times tile_size=%d", c.bin_tile_size, c.tile_size);
        return GS_ERR_INVALID_ARG;
    }
    if (c.bin_tile_size > 32) {
        snprintf(msg, n, "bin_tile_size=%d above 32", c.bin_tile_size);
        return GS_ERR_INVALID_ARG;
    }
    return GS_OK;
}

}  // namespace

extern "C" {

void gs_config_default(gs_config* cfg) {
    if (!cfg) return;
    cfg->tile_size = 16;
    cfg->alpha_min = 1.0f / 255.0f;
    cfg->alpha_max = 0.99f;
    cfg->T_min = 1e-4f;
    cfg->blur = 0.3f;
    cfg->z_near = 0.2f;
    cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.f;
    cfg->pixels_per_thread = 0;
    cfg->batch = 0;
    cfg->deterministic = 0;
    cfg->bin_tile_size = 0;
}

const char* gs_version(void) { return "gs_b300 0.1 (sm_103a)"; }

int gs_context_create(gs_ctx** out, int device, const gs_config* cfg) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_config c;
    gs_config_default(&c);
    if (cfg) c = *cfg;
    char msg[256];
    if (check_config(c, msg, sizeof(msg)) != GS_OK) return GS_ERR_INVALID_ARG;
    gs_ctx* ctx = new (std::nothrow) gs_ctx();
    if (!ctx) return GS_ERR_OOM;
    ctx->device = device;
    ctx->cfg = c;
    ctx->err[0] = 0;
    DeviceGuard dg(device);
    if (!dg.ok) { delete ctx; return GS_ERR_CUDA; }
    if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete ctx;
        return GS_ERR_CUDA;
    }
    if (cudaMalloc(&ctx->d_status, 256) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GS_ERR_OOM;
    }
    ctx->d_pairs = reinterpret_cast<unsigned long long*>(ctx->d_status + 2);
    ctx->d_adam_coef = reinterpret_cast<float2*>(ctx->d_status + 16);
    if (cudaMemset(ctx->d_status, 0, 256) != cudaSuccess) {
        cudaFree(ctx->d_status);
        delete ctx;
        return GS_ERR_CUDA;
    }
    *out = ctx;
    return GS_OK;
}

int gs_context_destroy(gs_ctx* ctx) {
    if (!ctx) return GS_OK;
    {
        DeviceGuard dg(ctx->device);
        if (ctx->d_status) cudaFree(ctx->d_status);
        ctx->prof.release();
    }
    delete ctx;
    return GS_OK;
}

int gs_calibrate_alu(gs_ctx* ctx, gs_stream stream, double* ffma_tflops, double* ex2_gops) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!ffma_tflops || !ex2_gops) return fail(ctx, GS_ERR_INVALID_ARG, "output pointer is NULL");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, GS_ERR_CUDA, "cudaSetDevice(%d) failed", ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the never-taken stores of the microbenchmarks point at a spare word of the status block
    cudaError_t e = measure_alu(ctx->sm_count, reinterpret_cast<float*>(ctx->d_status + 48), s, ffma_tflops,
                                ex2_gops);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_calibrate_alu");
    return GS_OK;
}

const char* gs_last_error(const gs_ctx* ctx) { return ctx ? ctx->err : "context is NULL"; }

int gs_get_config(const gs_ctx* ctx, gs_config* cfg) {
    if (!ctx || !cfg) return GS_ERR_INVALID_ARG;
    *cfg = ctx->cfg;
    return GS_OK;
}

int gs_workspace_query(const gs_ctx* ctx, const gs_view* views, int n_views, int64_t max_pairs,
                       size_t* bytes) {
    if (!ctx || !bytes) return GS_ERR_INVALID_ARG;
    Layout L;
    const int rc = make_layout(const_cast<gs_ctx*>(ctx), ctx->cfg, views, n_views, max_pairs, L);
    if (rc) return rc;
    *bytes = L.pub.total;
    return GS_OK;
}

int gs_workspace_layout(const gs_ctx* ctx, const gs_view* views, int n_views, int64_t max_pairs,
                        gs_ws_layout* out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    Layout L;
    const int rc = make_layout(const_cast<gs_ctx*>(ctx), ctx->cfg, views, n_views, max_pairs, L);
    if (rc) return rc;
    *out = L.pub;
    return GS_OK;
}

int gs_project(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
               const gs_workspace* ws, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    GaussPtrs gp;
    if ((rc = check_gaussians(ctx, g, views, n_views, gp))) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;  // records are listed per bin
    make_batch(ctx->cfg, views, n_views, bp, L.pub.bin_size);
    const WsPtrs wp = ws_ptrs(ws, L);
    cudaError_t e = launch_project(bp, gp, ctx_rc(ctx), wp, reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_project");
}

int gs_bin(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws,
           uint64_t* pairs_needed, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;  // at the bin size
    make_batch(ctx->cfg, views, n_views, bp, L.pub.bin_size);
    WsPtrs wp = ws_ptrs(ws, L);
    wp.log2_alpha_min = ctx_rc(ctx).log2_alpha_min;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RefineGeom geom;
    int n_tiles = bp.total_tiles;
    if (wp.refine > 1) {
        BatchParam bt;  // the compositing tiles
        make_batch(ctx->cfg, views, n_views, bt);
        memset(&geom, 0, sizeof(geom));
        geom.n_views = n_views;
        geom.ts = bt.tile_size;
        for (int v = 0; v < n_views; ++v) {
            geom.bin_off[v] = bp.v[v].tile_off;
            geom.bins_x[v] = bp.v[v].tiles_x;
            geom.tile_off[v] = bt.v[v].tile_off;
            geom.tiles_x[v] = bt.v[v].tiles_x;
            geom.tiles_y[v] = bt.v[v].tiles_y;
        }
        n_tiles = bt.total_tiles;
    }
    cudaError_t e = launch_bin(bp, wp, ctx->d_status, ctx->d_pairs, s, ctx->prof, wp.refine > 1 ? &geom : nullptr,
                               n_tiles);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_bin");
    if (wp.sorted_buf != sorted_buffer(bp.total_tiles))
        return fail(ctx, GS_ERR_CUDA, "gs_bin: sorted buffer parity mismatch");
    if (pairs_needed) {
        unsigned long long n = 0;
        if ((e = cudaMemcpyAsync(&n, wp.counters, sizeof(n), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return cuda_fail(ctx, e, "gs_bin (pair count)");
        *pairs_needed = n;
        if ((long long)n > ws->max_pairs)
            return fail(ctx, GS_ERR_CAPACITY, "gs_bin: %llu pairs exceed the capacity %lld", n,
                        (long long)ws->max_pairs);
    }
    return GS_OK;
}

int gs_render_fwd(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws, float* rgb,
                  float* T_final, uint32_t* n_contrib, uint32_t* n_used, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!rgb || !T_final || !n_contrib) return fail(ctx, GS_ERR_INVALID_ARG, "an output pointer is NULL");
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    const WsPtrs wp = ws_ptrs(ws, L);
    cudaError_t e = launch_render_fwd(bp, ctx_rc(ctx), wp, rgb, T_final, n_contrib, n_used, nullptr, nullptr,
                                      nullptr, reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_render_fwd");
}

int gs_render_fwd_l1(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws, const float* target,
                     float* rgb, float* T_final, uint32_t* n_contrib, uint32_t* n_used, float* dL_drgb,
                     float* loss_dev, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!target || !T_final || !n_contrib || !dL_drgb)
        return fail(ctx, GS_ERR_INVALID_ARG, "target, T_final, n_contrib or dL_drgb is NULL");
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    const WsPtrs wp = ws_ptrs(ws, L);
    cudaError_t e = launch_render_fwd(bp, ctx_rc(ctx), wp, rgb, T_final, n_contrib, n_used, target, dL_drgb,
                                      loss_dev, reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_render_fwd_l1");
}

int gs_l1_loss(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws, const float* rgb,
               const float* target, float* dL_drgb, float* loss_dev, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!rgb || !target || !dL_drgb) return fail(ctx, GS_ERR_INVALID_ARG, "an image pointer is NULL");
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    const WsPtrs wp = ws_ptrs(ws, L);
    cudaError_t e = launch_l1(bp, wp, rgb, target, dL_drgb, loss_dev, reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_l1_loss");
}

int gs_l1_loss_noalloc(const gs_view* views, int n_views, const float* rgb, const float* target, float* dL_drgb,
                       float* loss_dev, gs_stream stream, char* msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = 0;
    if (!rgb || !target || !dL_drgb) return fail_msg(msg, msg_len, GS_ERR_INVALID_ARG, "an image pointer is NULL");
    if (!views || n_views < 1 || n_views > GS_MAX_VIEWS)
        return fail_msg(msg, msg_len, GS_ERR_INVALID_ARG, "n_views=%d outside [1, %d] or views is NULL", n_views,
                        GS_MAX_VIEWS);
    for (int v = 0; v < n_views; ++v)
        if (views[v].width <= 0 || views[v].height <= 0 || views[v].width > 32768 || views[v].height > 32768)
            return fail_msg(msg, msg_len, GS_ERR_INVALID_ARG, "view %d: size %dx%d outside [1, 32768]", v,
                            views[v].width, views[v].height);
    gs_config cfg;
    gs_config_default(&cfg);
    BatchParam bp;
    make_batch(cfg, views, n_views, bp);
    const long long need = l1_partials_needed(bp);
    if (need > l1_scratch_capacity())
        return fail_msg(msg, msg_len, GS_ERR_CAPACITY,
                        "gs_l1_loss_noalloc: the batch needs %lld partial sums, the fixed scratch holds %lld", need,
                        l1_scratch_capacity());
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int cur = -1, sdev = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e == cudaSuccess) e = cudaStreamGetDevice(s, &sdev);
    if (e != cudaSuccess)
        return fail_msg(msg, msg_len, GS_ERR_CUDA, "gs_l1_loss_noalloc: %s", cudaGetErrorString(e));
    if (sdev != cur)
        return fail_msg(msg, msg_len, GS_ERR_INVALID_ARG,
                        "gs_l1_loss_noalloc: the stream belongs to device %d, the current device is %d", sdev, cur);
    e = launch_l1_static(bp, rgb, target, dL_drgb, loss_dev, s);
    if (e == cudaErrorStreamCaptureUnsupported)
        return fail_msg(msg, msg_len, GS_ERR_INVALID_ARG,
                        "gs_l1_loss_noalloc: the first call in a CUDA context looks up the scratch address and "
                        "must not be captured");
    if (e != cudaSuccess)
        return fail_msg(msg, msg_len, GS_ERR_CUDA, "gs_l1_loss_noalloc: %s", cudaGetErrorString(e));
    return GS_OK;
}

namespace {
bool image_views_ok(const gs_view* views, int n_views) {
    if (!views || n_views < 1 || n_views > GS_MAX_VIEWS) return false;
    for (int v = 0; v < n_views; ++v)
        if (views[v].width <= 0 || views[v].height <= 0 || views[v].width > 32768 || views[v].height > 32768)
            return false;
    return true;
}
}  // namespace

size_t gs_dssim_scratch_floats(const gs_view* views, int n_views) {
    if (!image_views_ok(views, n_views)) return 0;
    gs_config cfg;
    gs_config_default(&cfg);
    BatchParam bp;
    make_batch(cfg, views, n_views, bp);
    return ssim_scratch_floats(bp);
}

int gs_dssim_loss(gs_ctx* ctx, const gs_view* views, int n_views, const float* rgb, const float* target,
                  float lambda, float* scratch, float* dL_drgb, float* loss_dev, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!rgb || !target || !dL_drgb || !scratch)
        return fail(ctx, GS_ERR_INVALID_ARG, "an image or scratch pointer is NULL");
    if (!image_views_ok(views, n_views))
        return fail(ctx, GS_ERR_INVALID_ARG, "views NULL, n_views=%d outside [1, %d] or a size outside [1, 32768]",
                    n_views, GS_MAX_VIEWS);
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(ctx, GS_ERR_INVALID_ARG, "lambda=%g outside [0, 1]", lambda);
    if (reinterpret_cast<uintptr_t>(scratch) % 16) return fail(ctx, GS_ERR_INVALID_ARG, "scratch is not 16-byte aligned");
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    SsimParam sp;
    double g[2 * kSsimRadius + 1], sum = 0.0;
    for (int k = 0; k <= 2 * kSsimRadius; ++k) {
        const double d = (double)(k - kSsimRadius);
        g[k] = exp(-d * d / (2.0 * 1.5 * 1.5));
        sum += g[k];
    }
    for (int k = 0; k <= 2 * kSsimRadius; ++k) sp.g[k] = (float)(g[k] / sum);
    sp.C1 = 0.01f * 0.01f;
    sp.C2 = 0.03f * 0.03f;
    sp.lambda = lambda;
    const cudaError_t e = launch_ssim(bp, sp, rgb, target, scratch, dL_drgb, loss_dev,
                                      reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_dssim_loss");
}

namespace {
int render_bwd_impl(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views, const gs_workspace* ws,
                    const float* T_final, const uint32_t* n_contrib, const float* dL_drgb, const gs_grads* grads,
                    float* dL_dpose_dev, gs_stream stream, bool accumulate) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!T_final || !n_contrib || !dL_drgb) return fail(ctx, GS_ERR_INVALID_ARG, "an image pointer is NULL");
    if (!grads && !dL_dpose_dev) return fail(ctx, GS_ERR_INVALID_ARG, "grads and dL_dpose are both NULL");
    if (grads && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity || !grads->sh))
        return fail(ctx, GS_ERR_INVALID_ARG, "a gradient pointer is NULL");
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    GaussPtrs gp;
    if ((rc = check_gaussians(ctx, g, views, n_views, gp))) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    const WsPtrs wp = ws_ptrs(ws, L);
    const RenderConst rcst = ctx_rc(ctx);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_render_bwd(bp, rcst, wp, T_final, n_contrib, dL_drgb, s, ctx->prof);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_render_bwd (raster)");
    GradPtrs gr;
    if (grads) {
        gr.means = grads->means;
        gr.log_scales = grads->log_scales;
        gr.quats = grads->quats;
        gr.opacity = grads->opacity;
        gr.sh = grads->sh;
    }
    e = launch_project_bwd(bp, gp, rcst, wp, grads ? &gr : nullptr, dL_dpose_dev, s, ctx->prof, accumulate);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_render_bwd (projection)");
}
}  // namespace

int gs_render_bwd(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views, const gs_workspace* ws,
                  const float* T_final, const uint32_t* n_contrib, const float* dL_drgb, const gs_grads* grads,
                  float* dL_dpose_dev, gs_stream stream) {
    return render_bwd_impl(ctx, g, views, n_views, ws, T_final, n_contrib, dL_drgb, grads, dL_dpose_dev, stream,
                           false);
}

int gs_render_bwd_accumulate(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
                             const gs_workspace* ws, const float* T_final, const uint32_t* n_contrib,
                             const float* dL_drgb, const gs_grads* grads, float* dL_dpose_dev, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!grads) return fail(ctx, GS_ERR_INVALID_ARG, "grads is NULL");
    return render_bwd_impl(ctx, g, views, n_views, ws, T_final, n_contrib, dL_drgb, grads, dL_dpose_dev, stream,
                           true);
}

int gs_pose_grad(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views, const gs_workspace* ws,
                 const float* T_final, const uint32_t* n_contrib, const float* dL_drgb, float* dL_dpose_dev,
                 gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!dL_dpose_dev) return fail(ctx, GS_ERR_INVALID_ARG, "dL_dpose is NULL");
    return render_bwd_impl(ctx, g, views, n_views, ws, T_final, n_contrib, dL_drgb, nullptr, dL_dpose_dev, stream,
                           false);
}

namespace {
int check_columns(gs_ctx* ctx, const gs_window_column* cols, int n_cols, const char* what) {
    if (!cols) return fail(ctx, GS_ERR_INVALID_ARG, "%s columns are NULL", what);
    if (n_cols < 1 || n_cols > window_max_columns())
        return fail(ctx, GS_ERR_INVALID_ARG, "n_cols=%d outside [1, %d]", n_cols, window_max_columns());
    for (int c = 0; c < n_cols; ++c) {
        if (!cols[c].ptr) return fail(ctx, GS_ERR_INVALID_ARG, "%s column %d is NULL", what, c);
        if (cols[c].bytes_per_gaussian <= 0 || cols[c].bytes_per_gaussian % 4 ||
            cols[c].bytes_per_gaussian > GS_WINDOW_MAX_COLUMN_BYTES)
            return fail(ctx, GS_ERR_INVALID_ARG,
                        "%s column %d: bytes_per_gaussian=%d is not a positive multiple of 4 up to %d", what, c,
                        cols[c].bytes_per_gaussian, GS_WINDOW_MAX_COLUMN_BYTES);
        if (reinterpret_cast<uintptr_t>(cols[c].ptr) % 4)
            return fail(ctx, GS_ERR_INVALID_ARG, "%s column %d is not 4-byte aligned", what, c);
    }
    return GS_OK;
}
}  // namespace

size_t gs_window_scratch_bytes(int64_t n) { return window_scratch_bytes(n < 0 ? 0 : (long long)n); }

namespace {
int window_remove_impl(gs_ctx* ctx, const gs_window_column* cols, const gs_window_column* leave_dst, int n_cols,
                       int64_t n, const uint8_t* keep, int64_t* n_keep_dev, int32_t* moved_from,
                       int32_t* leaving_rows, void* scratch, gs_stream stream, const char* what) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_columns(ctx, cols, n_cols, "window");
    if (rc) return rc;
    if (leave_dst) {
        for (int c = 0; c < n_cols; ++c) {
            if (!leave_dst[c].ptr) continue;  // column not gathered
            if (leave_dst[c].bytes_per_gaussian != cols[c].bytes_per_gaussian)
                return fail(ctx, GS_ERR_INVALID_ARG, "column %d: leave_dst width differs from the window's", c);
            if (reinterpret_cast<uintptr_t>(leave_dst[c].ptr) % 4)
                return fail(ctx, GS_ERR_INVALID_ARG, "leave_dst column %d is not 4-byte aligned", c);
        }
    }
    if (n < 0 || n > 0x7FFFFFFFll) return fail(ctx, GS_ERR_INVALID_ARG, "n=%lld outside [0, 2^31)", (long long)n);
    if (!keep || !n_keep_dev || !scratch) return fail(ctx, GS_ERR_INVALID_ARG, "keep, n_keep or scratch is NULL");
    if (reinterpret_cast<uintptr_t>(scratch) % 256)
        return fail(ctx, GS_ERR_INVALID_ARG, "scratch is not 256-byte aligned");
    DeviceGuard dg(ctx->device);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) {
        const cudaError_t e = cudaMemsetAsync(n_keep_dev, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, what);
    }
    const cudaError_t e = launch_window_compact(cols, leave_dst, n_cols, (long long)n, keep,
                                                reinterpret_cast<long long*>(n_keep_dev), moved_from, leaving_rows,
                                                scratch, ctx->sm_count, s, ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, what);
}
}  // namespace

int gs_window_compact(gs_ctx* ctx, const gs_window_column* cols, int n_cols, int64_t n, const uint8_t* keep,
                      int64_t* n_keep_dev, int32_t* moved_from, void* scratch, gs_stream stream) {
    return window_remove_impl(ctx, cols, nullptr, n_cols, n, keep, n_keep_dev, moved_from, nullptr, scratch, stream,
                              "gs_window_compact");
}

int gs_window_remove(gs_ctx* ctx, const gs_window_column* cols, const gs_window_column* leave_dst, int n_cols,
                     int64_t n, const uint8_t* keep, int64_t* n_keep_dev, int32_t* moved_from, int32_t* leaving_rows,
                     void* scratch, gs_stream stream) {
    return window_remove_impl(ctx, cols, leave_dst, n_cols, n, keep, n_keep_dev, moved_from, leaving_rows, scratch,
                              stream, "gs_window_remove");
}

int gs_window_gather(gs_ctx* ctx, const gs_window_column* src, const gs_window_column* dst, int n_cols, int64_t n,
                     const int32_t* idx, int64_t m, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_columns(ctx, src, n_cols, "source");
    if (rc) return rc;
    if ((rc = check_columns(ctx, dst, n_cols, "destination"))) return rc;
    for (int c = 0; c < n_cols; ++c)
        if (src[c].bytes_per_gaussian != dst[c].bytes_per_gaussian)
            return fail(ctx, GS_ERR_INVALID_ARG, "column %d: source and destination widths differ", c);
    if (n < 0 || m < 0 || (m > 0 && !idx)) return fail(ctx, GS_ERR_INVALID_ARG, "bad n, m or idx");
    DeviceGuard dg(ctx->device);
    const cudaError_t e = launch_window_gather(src, dst, n_cols, idx, (long long)m, (long long)n, ctx->sm_count,
                                               reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_window_gather");
}

int gs_window_clear(gs_ctx* ctx, const gs_window_column* cols, int n_cols, int64_t begin, int64_t end,
                    gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_columns(ctx, cols, n_cols, "window");
    if (rc) return rc;
    if (begin < 0 || end < begin || end > 0x7FFFFFFFll)
        return fail(ctx, GS_ERR_INVALID_ARG, "rows [%lld, %lld) outside [0, 2^31)", (long long)begin, (long long)end);
    DeviceGuard dg(ctx->device);
    const cudaError_t e = launch_window_clear(cols, n_cols, (long long)begin, (long long)end, ctx->sm_count,
                                              reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_window_clear");
}

int gs_sh_init_bilinear(gs_ctx* ctx, const gs_gaussians* g, const gs_view* view, const float* image, int64_t begin,
                        int64_t end, float* sh_out, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!g || !g->means || !view || !image || !sh_out)
        return fail(ctx, GS_ERR_INVALID_ARG, "gaussians, means, view, image or sh_out is NULL");
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(ctx, GS_ERR_INVALID_ARG, "sh_degree=%d not in [0, 3]", g->sh_degree);
    if (begin < 0 || end < begin || end > g->n)
        return fail(ctx, GS_ERR_INVALID_ARG, "range [%lld, %lld) outside [0, %lld]", (long long)begin,
                    (long long)end, (long long)g->n);
    if (view->width <= 0 || view->height <= 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "view size %dx%d", view->width, view->height);
    for (int k = 0; k < 9; ++k)
        if (!isfinite(view->R_cw[k])) return fail(ctx, GS_ERR_NONFINITE, "R_cw not finite");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(view->t_cw[k])) return fail(ctx, GS_ERR_NONFINITE, "t_cw not finite");
    if (!(view->fx > 0.f) || !(view->fy > 0.f) || !isfinite(view->cx) || !isfinite(view->cy))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad intrinsics");
    DeviceGuard dg(ctx->device);
    gs_view v1 = *view;
    v1.g_begin = 0;
    v1.g_end = g->n > 0 ? g->n : 1;
    BatchParam bp;
    make_batch(ctx->cfg, &v1, 1, bp);
    const cudaError_t e = launch_sh_init(bp.v[0], g->means, image, (long long)begin, (long long)end, g->sh_degree,
                                         ctx->cfg.z_near, sh_out, reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_sh_init_bilinear");
}

int gs_pose_normal_scratch(gs_ctx* ctx, const gs_view* views, int n_views, size_t* floats) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!floats) return fail(ctx, GS_ERR_INVALID_ARG, "floats is NULL");
    Layout L;
    int rc = make_layout(ctx, ctx->cfg, views, n_views, 0, L);
    if (rc) return rc;
    *floats = (size_t)4 * kPoseTan4 * (size_t)L.pub.n_records + pose_normal_partials_floats(L.pub.n_tiles) +
              pose_normal_chunk_floats(n_views);
    return GS_OK;
}

int gs_pose_normal(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views, const gs_workspace* ws,
                   const float* target, float* scratch, double* normal, float* H_pix, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!target || !scratch || !normal) return fail(ctx, GS_ERR_INVALID_ARG, "target, scratch or normal is NULL");
    if (reinterpret_cast<uintptr_t>(scratch) % 16)
        return fail(ctx, GS_ERR_INVALID_ARG, "scratch is not 16-byte aligned");
    if (!pose_normal_supported(ctx->cfg.tile_size))
        return fail(ctx, GS_ERR_UNSUPPORTED, "pose normal equations need a tile size of 8 or 16 (config has %d)",
                    ctx->cfg.tile_size);
    Layout L;
    int rc = check_ws(ctx, views, n_views, ws, L);
    if (rc) return rc;
    GaussPtrs gp;
    if ((rc = check_gaussians(ctx, g, views, n_views, gp))) return rc;
    DeviceGuard dg(ctx->device);
    BatchParam bp;
    make_batch(ctx->cfg, views, n_views, bp);
    const WsPtrs wp = ws_ptrs(ws, L);
    const RenderConst rcst = ctx_rc(ctx);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4* tangents = reinterpret_cast<float4*>(scratch);
    float* partials = scratch + (size_t)4 * kPoseTan4 * (size_t)L.pub.n_records;
    cudaError_t e = launch_pose_tangents(bp, gp, rcst, wp, tangents, s, ctx->prof);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_pose_normal (tangents)");
    e = launch_pose_normal(bp, rcst, wp, tangents, target, partials, normal, H_pix, s, ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_pose_normal (compositing)");
}

namespace {
int check_adam(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n, float lr, float b1,
               float b2, float eps, const gs_lowp_segment* segs, int n_segs) {
    if (!param || !grad || !m || !v) return fail(ctx, GS_ERR_INVALID_ARG, "an Adam buffer is NULL");
    if (n < 0) return fail(ctx, GS_ERR_INVALID_ARG, "n=%lld is negative", (long long)n);
    if (!(lr >= 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return fail(ctx, GS_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
    if (n_segs < 0 || n_segs > 8 || (n_segs > 0 && !segs))
        return fail(ctx, GS_ERR_INVALID_ARG, "n_segs=%d outside [0, 8]", n_segs);
    for (int k = 0; k < n_segs; ++k) {
        if (!segs[k].dst || segs[k].begin < 0 || segs[k].end > n || segs[k].end < segs[k].begin ||
            (segs[k].dtype != GS_F16 && segs[k].dtype != GS_BF16))
            return fail(ctx, GS_ERR_INVALID_ARG, "low-precision segment %d is invalid", k);
    }
    return GS_OK;
}
}  // namespace

int gs_adam_step(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n, float lr, float b1,
                 float b2, float eps, int64_t step, const gs_lowp_segment* segs, int n_segs, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_adam(ctx, param, grad, m, v, n, lr, b1, b2, eps, segs, n_segs);
    if (rc) return rc;
    if (step < 1) return fail(ctx, GS_ERR_INVALID_ARG, "step=%lld must be >= 1", (long long)step);
    if (n == 0) return GS_OK;
    DeviceGuard dg(ctx->device);
    const double bc1 = 1.0 - pow((double)b1, (double)step);
    const double bc2 = 1.0 - pow((double)b2, (double)step);
    const float step_size = (float)(lr / bc1);
    const float inv_sqrt_bc2 = (float)(1.0 / sqrt(bc2));
    cudaError_t e = launch_adam(param, grad, m, v, n, b1, b2, eps, step_size, inv_sqrt_bc2, segs, n_segs,
                                reinterpret_cast<cudaStream_t>(stream), ctx->prof);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_adam_step");
}

int gs_adam_step_dev(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n, float lr,
                     float b1, float b2, float eps, int64_t* step_dev, const gs_lowp_segment* segs, int n_segs,
                     gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_adam(ctx, param, grad, m, v, n, lr, b1, b2, eps, segs, n_segs);
    if (rc) return rc;
    if (!step_dev) return fail(ctx, GS_ERR_INVALID_ARG, "step_dev is NULL");
    if (n == 0) return GS_OK;
    DeviceGuard dg(ctx->device);
    cudaError_t e = launch_adam(param, grad, m, v, n, b1, b2, eps, 0.f, 0.f, segs, n_segs,
                                reinterpret_cast<cudaStream_t>(stream), ctx->prof,
                                reinterpret_cast<long long*>(step_dev), lr, ctx->d_adam_coef);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_adam_step_dev");
}

int gs_adam_step_ranges(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n,
                        const gs_range* ranges, int n_ranges, float lr, float b1, float b2, float eps, int64_t step,
                        int64_t* step_dev, const gs_lowp_segment* segs, int n_segs, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    int rc = check_adam(ctx, param, grad, m, v, n, lr, b1, b2, eps, segs, n_segs);
    if (rc) return rc;
    if (!step_dev && step < 1) return fail(ctx, GS_ERR_INVALID_ARG, "step=%lld must be >= 1", (long long)step);
    if (!ranges || n_ranges < 1 || n_ranges > 8)
        return fail(ctx, GS_ERR_INVALID_ARG, "n_ranges=%d outside [1, 8] or ranges is NULL", n_ranges);
    if (((reinterpret_cast<uintptr_t>(param) | reinterpret_cast<uintptr_t>(grad) | reinterpret_cast<uintptr_t>(m) |
          reinterpret_cast<uintptr_t>(v)) & 15) != 0)
        return fail(ctx, GS_ERR_INVALID_ARG, "Adam buffers must be 16-byte aligned");
    for (int k = 0; k < n_ranges; ++k) {
        if (ranges[k].begin < 0 || ranges[k].end < ranges[k].begin || ranges[k].end > n || ranges[k].begin % 4)
            return fail(ctx, GS_ERR_INVALID_ARG, "range %d [%lld, %lld) invalid (begin a multiple of 4, end <= n)", k,
                        (long long)ranges[k].begin, (long long)ranges[k].end);
        for (int j = 0; j < k; ++j)
            if (ranges[k].begin < ranges[j].end && ranges[j].begin < ranges[k].end)
                return fail(ctx, GS_ERR_INVALID_ARG, "ranges %d and %d overlap", j, k);
    }
    DeviceGuard dg(ctx->device);
    float step_size = 0.f, inv_sqrt_bc2 = 0.f;
    if (!step_dev) {
        step_size = (float)(lr / (1.0 - pow((double)b1, (double)step)));
        inv_sqrt_bc2 = (float)(1.0 / sqrt(1.0 - pow((double)b2, (double)step)));
    }
    cudaError_t e = launch_adam_ranges(param, grad, m, v, ranges, n_ranges, b1, b2, eps, step_size, inv_sqrt_bc2,
                                       segs, n_segs, reinterpret_cast<cudaStream_t>(stream), ctx->prof,
                                       reinterpret_cast<long long*>(step_dev), lr, ctx->d_adam_coef, ctx->sm_count);
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_adam_step_ranges");
}

size_t gs_selftest_wait_scratch_bytes(void) { return selftest_wait_scratch_bytes(); }

int gs_selftest_bounded_wait(gs_ctx* ctx, void* scratch, gs_stream stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!scratch || reinterpret_cast<uintptr_t>(scratch) % 256)
        return fail(ctx, GS_ERR_INVALID_ARG, "scratch is NULL or not 256-byte aligned");
    DeviceGuard dg(ctx->device);
    const cudaError_t e = launch_selftest_wait(scratch, ctx->d_status, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? GS_OK : cuda_fail(ctx, e, "gs_selftest_bounded_wait");
}

int gs_sync_status(gs_ctx* ctx, gs_stream stream, uint64_t* pairs_needed) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned int host[16];
    cudaError_t e = cudaMemcpyAsync(host, ctx->d_status, 64, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_sync_status");
    unsigned long long pairs;
    memcpy(&pairs, host + 2, sizeof(pairs));
    if (pairs_needed) *pairs_needed = pairs;
    const unsigned int code = host[0];
    if (code) {
        e = cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_sync_status (clear)");
        return fail(ctx, -(int)code, "device status %d (pairs needed %llu)", -(int)code, pairs);
    }
    return GS_OK;
}

int gs_profile_enable(gs_ctx* ctx, uint32_t family_mask) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (family_mask >> GS_KF_COUNT) return fail(ctx, GS_ERR_INVALID_ARG, "family mask 0x%x has unknown bits", family_mask);
    ctx->prof.mask = family_mask;
    return GS_OK;
}

int gs_profile_collect(gs_ctx* ctx, gs_stream stream, gs_profile_entry* out, int max_entries, int* n_out) {
    if (!ctx || (max_entries > 0 && !out) || max_entries < 0) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    Prof& pf = ctx->prof;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gs_profile_collect");
    double ms[GS_KF_COUNT] = {0};
    int cnt[GS_KF_COUNT] = {0};
    for (int k = 0; k < pf.n_recs; ++k) {
        float t = 0.f;
        if ((e = cudaEventSynchronize(pf.recs[k].b)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&t, pf.recs[k].a, pf.recs[k].b)) != cudaSuccess)
            return cuda_fail(ctx, e, "gs_profile_collect (event)");
        ms[pf.recs[k].fam] += t;
        cnt[pf.recs[k].fam] += 1;
    }
    pf.n_recs = 0;
    pf.pool_used = 0;
    int n = 0;
    for (int f = 0; f < GS_KF_COUNT; ++f) {
        if (!cnt[f]) continue;
        if (n < max_entries) {
            out[n].family = f;
            out[n].launches = cnt[f];
            out[n].total_ms = ms[f];
        }
        ++n;
    }
    if (n_out) *n_out = n < max_entries ? n : max_entries;
    return GS_OK;
}

int64_t gs_launch_count(const gs_ctx* ctx) { return ctx ? (int64_t)ctx->prof.launches : -1; }

int32_t gs_checked_build(void) {
#ifdef GS_CHECKED
    return 1;
#else
    return 0;
#endif
}

}  // extern "C"
