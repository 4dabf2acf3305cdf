// EWA projection of (view, Gaussian) pairs and its backward pass.
//
// Forward (Sec. II-B.1): Sigma3 = (R S)(R S)^T (Eq. 3dgs), q = pi(T_CW p_W)
// (Eq. q), Sigma2 = (J W) Sigma3 (J W)^T + blur I (Eq. spat), opacity
// sigmoid(logit), colour from real SH of degree 0/1.  One thread per
// (view, Gaussian); grid.y is the view so all view parameters are uniform in
// a block.  HBM-bound: ~92 B read per Gaussian per view (FP32, degree 1),
// 48 B record + 16 B rectangle + 12 B keys written.
//
// Backward: one thread per Gaussian walks the views that contain it,
// rebuilds the forward quantities, chains the per-record 2D gradients
// (written by the compositing backward) to the parameters, and (optionally)
// reduces the pose gradient of the left perturbation T_CW <- Exp(dphi, dt)
// T_CW (Appendix A) per block into a partials buffer.
#include <math.h>

#include "gs_internal.cuh"

namespace gsb {

namespace {

// Real spherical harmonics of degree D <= 3 with the Condon-Shortley phase,
// index k = l^2 + l + m (m = -l..l), as homogeneous polynomials of the unit
// view direction (x, y, z).  The normalisation of (l, m) is
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0, folded with
// the Legendre factor of each polynomial:
constexpr float kShC0 = 0.28209479177387814f;  // 1/2 sqrt(1/pi)
constexpr float kShC1 = 0.48860251190291990f;  // 1/2 sqrt(3/pi): y, z, x
constexpr float kShA2 = 1.0925484305920792f;   // 1/2 sqrt(15/pi): xy, yz, xz
constexpr float kShB2 = 0.31539156525252005f;  // 1/4 sqrt(5/pi): 2z^2 - x^2 - y^2
constexpr float kShC2 = 0.54627421529603960f;  // 1/4 sqrt(15/pi): x^2 - y^2
constexpr float kShE3 = 0.59004358992664350f;  // 1/4 sqrt(35/(2 pi)): y (3x^2 - y^2), x (x^2 - 3y^2)
constexpr float kShF3 = 2.8906114426405540f;   // 1/2 sqrt(105/pi): xyz
constexpr float kShG3 = 0.45704579946446580f;  // 1/4 sqrt(21/(2 pi)): y, x times (4z^2 - x^2 - y^2)
constexpr float kShH3 = 0.37317633259011540f;  // 1/4 sqrt(7/pi): z (2z^2 - 3x^2 - 3y^2)
constexpr float kShJ3 = 1.4453057213202770f;   // 1/4 sqrt(105/pi): z (x^2 - y^2)

template <int D>
__device__ __forceinline__ void sh_basis(const float* d, float* Y) {
    const float x = d[0], y = d[1], z = d[2];
    Y[0] = kShC0;
    if (D >= 1) {
        Y[1] = -kShC1 * y;
        Y[2] = kShC1 * z;
        Y[3] = -kShC1 * x;
    }
    if (D >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = kShA2 * x * y;
        Y[5] = -kShA2 * y * z;
        Y[6] = kShB2 * (2.f * zz - xx - yy);
        Y[7] = -kShA2 * x * z;
        Y[8] = kShC2 * (xx - yy);
        if (D >= 3) {
            Y[9] = -kShE3 * y * (3.f * xx - yy);
            Y[10] = kShF3 * x * y * z;
            Y[11] = -kShG3 * y * (4.f * zz - xx - yy);
            Y[12] = kShH3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
            Y[13] = -kShG3 * x * (4.f * zz - xx - yy);
            Y[14] = kShJ3 * z * (xx - yy);
            Y[15] = -kShE3 * x * (xx - 3.f * yy);
        }
    }
}

// Derivative of every basis polynomial along v: T[k] = grad Y_k(d) . v.
template <int D>
__device__ __forceinline__ void sh_basis_along(const float* d, const float* v, float* T) {
    const float x = d[0], y = d[1], z = d[2], vx = v[0], vy = v[1], vz = v[2];
    T[0] = 0.f;
    if (D >= 1) {
        T[1] = -kShC1 * vy;
        T[2] = kShC1 * vz;
        T[3] = -kShC1 * vx;
    }
    if (D >= 2) {
        T[4] = kShA2 * (vx * y + x * vy);
        T[5] = -kShA2 * (vy * z + y * vz);
        T[6] = 2.f * kShB2 * (2.f * z * vz - x * vx - y * vy);
        T[7] = -kShA2 * (vx * z + x * vz);
        T[8] = 2.f * kShC2 * (x * vx - y * vy);
        if (D >= 3) {
            const float xx = x * x, yy = y * y, zz = z * z;
            T[9] = -kShE3 * (6.f * x * y * vx + 3.f * (xx - yy) * vy);
            T[10] = kShF3 * (y * z * vx + x * z * vy + x * y * vz);
            T[11] = -kShG3 * (-2.f * x * y * vx + (4.f * zz - xx - 3.f * yy) * vy + 8.f * y * z * vz);
            T[12] = kShH3 * (-6.f * x * z * vx - 6.f * y * z * vy + (6.f * zz - 3.f * xx - 3.f * yy) * vz);
            T[13] = -kShG3 * ((4.f * zz - 3.f * xx - yy) * vx - 2.f * x * y * vy + 8.f * x * z * vz);
            T[14] = kShJ3 * (2.f * x * z * vx - 2.f * y * z * vy + (xx - yy) * vz);
            T[15] = -kShE3 * (3.f * (xx - yy) * vx - 6.f * x * y * vy);
        }
    }
}

struct Proj {
    float qh[4];     // unit quaternion
    float inv_qn;    // 1 / |quat|
    float R[9];
    float s[3];      // exp(log-scale)
    float M[9];      // R S, so Sigma3 = M M^T
    float pc[3];
    float Tm[6];     // J W, row-major 2x3
    float U[6];      // T M, row-major 2x3, so Sigma2 = U U^T + blur I
    float a, b, c;   // Sigma2 with blur
    float det;
    float A, B, C;   // conic
    float sigma;
    float dir[3];
    float inv_len;
    float raw[3];
};

__device__ __forceinline__ void quat_rot(const float* q, float* R) {
    const float w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Loads Gaussian i and computes the view-independent part (Sigma3).
__device__ __forceinline__ void load_gaussian(const GaussPtrs& g, long long i, float* mu, Proj& P,
                                              float& ologit) {
    mu[0] = g.means[3 * i + 0];
    mu[1] = g.means[3 * i + 1];
    mu[2] = g.means[3 * i + 2];
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = load_as_float(g.quats, g.rot_dtype, 4 * i + k);
    const float qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    P.inv_qn = 1.f / sqrtf(qn2);
    for (int k = 0; k < 4; ++k) P.qh[k] = q[k] * P.inv_qn;
    quat_rot(P.qh, P.R);
    for (int k = 0; k < 3; ++k) P.s[k] = expf(load_as_float(g.log_scales, g.scale_dtype, 3 * i + k));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) P.M[3 * a + b] = P.R[3 * a + b] * P.s[b];
    ologit = load_as_float(g.opacity, g.opacity_dtype, i);
}

// View-dependent part.  Returns false when culled (z <= z_near or a
// degenerate Sigma2).  Sigma2 is formed from U = J W R S as U U^T + blur I
// (entries a and c are sums of squares) and its determinant by the
// Cauchy-Binet sum of squared 2x2 minors of U plus the blur terms: every term
// is non-negative, so the determinant keeps full FP32 relative accuracy even
// for long thin footprints, where a c - b^2 would cancel.
__device__ __forceinline__ bool project_view(const ViewParam& V, const RenderConst& rc,
                                             const float* mu, Proj& P) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        P.pc[r] = V.R[3 * r] * mu[0] + V.R[3 * r + 1] * mu[1] + V.R[3 * r + 2] * mu[2] + V.t[r];
    const float x = P.pc[0], y = P.pc[1], z = P.pc[2];
    if (!(z > rc.z_near)) return false;
    const float iz = 1.f / z;
    const float j00 = V.fx * iz, j02 = -V.fx * x * iz * iz;
    const float j11 = V.fy * iz, j12 = -V.fy * y * iz * iz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        P.Tm[c] = j00 * V.R[c] + j02 * V.R[6 + c];
        P.Tm[3 + c] = j11 * V.R[3 + c] + j12 * V.R[6 + c];
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P.U[k] = P.Tm[0] * P.M[k] + P.Tm[1] * P.M[3 + k] + P.Tm[2] * P.M[6 + k];
        P.U[3 + k] = P.Tm[3] * P.M[k] + P.Tm[4] * P.M[3 + k] + P.Tm[5] * P.M[6 + k];
    }
    const float* u0 = P.U;
    const float* u1 = P.U + 3;
    const float a0 = u0[0] * u0[0] + u0[1] * u0[1] + u0[2] * u0[2];
    const float c0 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
    P.a = a0 + rc.blur;
    P.b = u0[0] * u1[0] + u0[1] * u1[1] + u0[2] * u1[2];
    P.c = c0 + rc.blur;
    const float m01 = fmaf(u0[0], u1[1], -u0[1] * u1[0]);
    const float m02 = fmaf(u0[0], u1[2], -u0[2] * u1[0]);
    const float m12 = fmaf(u0[1], u1[2], -u0[2] * u1[1]);
    P.det = (m01 * m01 + m02 * m02 + m12 * m12) + rc.blur * (a0 + c0) + rc.blur * rc.blur;
    if (!(P.det > 0.f) || !(P.det < 3.0e38f)) return false;
    const float idet = 1.f / P.det;
    P.A = P.c * idet;
    P.B = -P.b * idet;
    P.C = P.a * idet;
    return true;
}

template <int D>
__device__ __forceinline__ void view_colour(const ViewParam& V, const GaussPtrs& g, long long i,
                                            const float* mu, Proj& P, float* col) {
    constexpr int K = (D + 1) * (D + 1);
    float d[3] = {mu[0] - V.campos[0], mu[1] - V.campos[1], mu[2] - V.campos[2]};
    P.inv_len = 1.f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int k = 0; k < 3; ++k) P.dir[k] = d[k] * P.inv_len;
    float Y[K];
    sh_basis<D>(P.dir, Y);
    const long long base = i * K * 3;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float v = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) v = fmaf(Y[k], load_as_float(g.sh, g.sh_dtype, base + 3 * k + ch), v);
        P.raw[ch] = v;
        col[ch] = fmaxf(v, 0.f);
    }
}

// Camera depth R_CW[2] . p_W + t_CW[2] as an unevaluated sum hi + lo of two
// floats (the compensated dot product "Dot2" of Ogita, Rump and Oishi, 2005,
// built from the error-free transformations TwoProduct (via fma) and TwoSum):
// as accurate as a dot product evaluated in twice the FP32 precision.  The
// 64-bit key (bits(hi) << 32 | ordered(lo)) orders records by this value, so
// nearly coplanar Gaussians are ordered as in exact arithmetic.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void depth_dot2(const ViewParam& V, const float* mu, float& hi, float& lo) {
    float p = V.R[6] * mu[0];
    float s = fmaf(V.R[6], mu[0], -p);
    float h, r, q;
    h = V.R[7] * mu[1];
    r = fmaf(V.R[7], mu[1], -h);
    two_sum(p, h, p, q);
    s = s + (q + r);
    h = V.R[8] * mu[2];
    r = fmaf(V.R[8], mu[2], -h);
    two_sum(p, h, p, q);
    s = s + (q + r);
    two_sum(p, V.t[2], p, q);
    s = s + q;
    hi = p + s;                // renormalise (|s| is far below |p| here)
    lo = s - (hi - p);
    lo = lo + 0.0f;            // -0 -> +0 so equal values give equal keys
}

__device__ __forceinline__ uint32_t ordered_bits(float x) {
    const uint32_t u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

template <int D>
__global__ void __launch_bounds__(256) k_project(const __grid_constant__ BatchParam bp, GaussPtrs g,
                                                 RenderConst rc, WsPtrs ws) {
    pdl_wait();
    pdl_trigger();
    // the block's range of valid high depth-key words, and its warps done
    __shared__ uint32_t s_kmin, s_kmax, s_warps;
    if (threadIdx.x == 0) {
        s_kmin = 0xFFFFFFFFu;
        s_kmax = 0u;
        s_warps = 0u;
    }
    __syncthreads();
    const ViewParam& V = bp.v[blockIdx.y];
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = V.g_end - V.g_begin;
    if (k >= cnt) return;
    const long long i = V.g_begin + k;
    const long long r = V.rec_off + k;
    uint32_t mask = 0;  // listed tiles (row-major bits) when the rectangle has <= kMaskTiles

    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0;
    int4 rect = make_int4(0, 0, V.tile_off, V.tiles_x);
    uint32_t touched = 0;
    uint32_t key_hi = 0xFFFFFFFFu, key_lo = 0xFFFFFFFFu;

    Proj P;
    float mu[3], ologit;
    load_gaussian(g, i, mu, P, ologit);
    bool ok = project_view(V, rc, mu, P);
    float sigma = 0.f;
    if (ok) {
        sigma = 1.f / (1.f + expf(-ologit));
        ok = sigma > rc.alpha_min;
    }
    if (ok) {
        const float iz = 1.f / P.pc[2];
        const float qx = V.fx * P.pc[0] * iz + V.cx;
        const float qy = V.fy * P.pc[1] * iz + V.cy;
        float col[3];
        view_colour<D>(V, g, i, mu, P, col);
        // Pixel box containing every pixel centre where sigma G >= alpha_min:
        // the ellipse d^T Sigma2^-1 d <= 2 ln(sigma / alpha_min) has half-widths
        // sqrt(r2 Sigma2_xx), sqrt(r2 Sigma2_yy).  The small margin only adds
        // pixels where alpha < alpha_min.
        float lo_x = 0.f, hi_x = (float)(V.W - 1), lo_y = 0.f, hi_y = (float)(V.H - 1);
        float ex = 65504.f, ey = 65504.f;  // half-widths of the box (exact mode: unbounded)
        if (rc.alpha_min > 0.f) {
            const float r2 = 2.f * logf(sigma / rc.alpha_min) * 1.001f;
            ex = sqrtf(r2 * P.a);
            ey = sqrtf(r2 * P.c);
            lo_x = fmaxf(ceilf(qx - ex - 0.5f), 0.f);
            hi_x = fminf(floorf(qx + ex - 0.5f), (float)(V.W - 1));
            lo_y = fmaxf(ceilf(qy - ey - 0.5f), 0.f);
            hi_y = fminf(floorf(qy + ey - 0.5f), (float)(V.H - 1));
        }
        // Exponent in eigen form: log2(sigma G) = l - (d.v1)^2 - (d.v2)^2 with
        // v_k = e_k sqrt(log2(e) / (2 lambda_k)); its FP32 error grows with the
        // square root of the footprint's condition number instead of linearly
        // as for A dx^2 + 2B dx dy + C dy^2.
        const float hsum = 0.5f * (P.a + P.c);
        const float hdif = 0.5f * (P.a - P.c);
        const float l1 = hsum + sqrtf(hdif * hdif + P.b * P.b);
        const float l2 = P.det / l1;
        float ex0, ex1;  // major eigenvector
        if (P.a >= P.c) { ex0 = l1 - P.c; ex1 = P.b; } else { ex0 = P.b; ex1 = l1 - P.a; }
        const float en = sqrtf(ex0 * ex0 + ex1 * ex1);
        if (en > 0.f) { ex0 /= en; ex1 /= en; } else { ex0 = 1.f; ex1 = 0.f; }
        const float s1 = sqrtf(0.5f * kLog2e / l1), s2 = sqrtf(0.5f * kLog2e / l2);
        r0 = make_float4(qx, qy, ex0 * s1, ex1 * s1);
        r1 = make_float4(-ex1 * s2, ex0 * s2, log2f(sigma), col[0]);
        // half-extents of the footprint's bounding box, rounded up to FP16, for
        // the raster kernels' per-warp culling (full image in exact mode)
        const float hx = fminf(ex + 0.5f, 65504.f), hy = fminf(ey + 0.5f, 65504.f);
        const __half2 ext = __halves2half2(__float2half_ru(hx), __float2half_ru(hy));
        r2 = make_float4(col[1], col[2], P.pc[2], *reinterpret_cast<const float*>(&ext));
        if (lo_x <= hi_x && lo_y <= hi_y) {
            const int ts = bp.tile_size;
            const int tx0 = (int)lo_x / ts, tx1 = (int)hi_x / ts + 1;
            const int ty0 = (int)lo_y / ts, ty1 = (int)hi_y / ts + 1;
            rect.x = tx0 | (ty0 << 16);
            rect.y = tx1 | (ty1 << 16);
            // count only the tiles the footprint reaches, one tile row at a
            // time (the spans k_emit writes)
            uint32_t hits = 0;
            const int w = tx1 - tx0;
            const int area = w * (ty1 - ty0);
            if (rc.alpha_min > 0.f) {
                const FootRows fr = make_footrows(r0, r1, r1.z - rc.log2_alpha_min);
                for (int ty = ty0; ty < ty1; ++ty) {
                    int a, b;
                    if (!footrows_span(fr, ty, ts, tx0, tx1, &a, &b)) continue;
                    hits += (uint32_t)(b - a + 1);
                    if (area <= kMaskTiles)  // bits a..b of the row, row-major
                        mask |= ((2u << (b - tx0)) - (1u << (a - tx0))) << ((ty - ty0) * w);
                }
            } else {
                hits = (uint32_t)area;
                mask = area >= 32 ? 0xFFFFFFFFu : (1u << area) - 1u;
            }
            touched = hits;
            float zhi, zlo;
            depth_dot2(V, mu, zhi, zlo);
            key_hi = ordered_bits(zhi);
            key_lo = ordered_bits(zlo);
            if (hits == 0) key_hi = key_lo = 0xFFFFFFFFu;
        }
    }
    ws.rec[3 * r + 0] = r0;
    ws.rec[3 * r + 1] = r1;
    ws.rec[3 * r + 2] = r2;
    // the rectangle with its tile count and mask in one 32-byte entry: the
    // emission gathers it in depth order, one sector per record
    ws.rect[2 * r] = rect;
    ws.rect[2 * r + 1] = make_int4((int)touched, (int)mask, 0, 0);
    ws.tiles_touched[r] = touched;
    ws.dkeys[0][r] = key_lo;
    ws.dhi[r] = key_hi;
    ws.dvals[1][r] = (uint32_t)r;  // the depth sort's input values

    // Range of the valid keys: warp minimum and maximum over the warp's live
    // lanes (those with k < cnt, all of which reach this point), block-wide by
    // shared atomics; the block's last live warp publishes it with the
    // current generation (see kCtrRangeGen).
    const long long wbase = k - (threadIdx.x & 31);
    const long long nl = cnt - wbase;
    const uint32_t live = nl >= 32 ? 0xFFFFFFFFu : (1u << nl) - 1u;
    const bool valid = key_hi != 0xFFFFFFFFu;
    const uint32_t wmin = __reduce_min_sync(live, valid ? key_hi : 0xFFFFFFFFu);
    const uint32_t wmax = __reduce_max_sync(live, valid ? key_hi : 0u);
    if ((threadIdx.x & 31) == 0) {
        if (wmin <= wmax) {
            atomicMin(&s_kmin, wmin);
            atomicMax(&s_kmax, wmax);
        }
        __threadfence_block();
        const long long bl = cnt - (long long)blockIdx.x * blockDim.x;  // live threads of the block
        const uint32_t nw = (uint32_t)((bl >= (long long)blockDim.x ? (long long)blockDim.x : bl) + 31) / 32;
        if (atomicAdd(&s_warps, 1u) + 1u == nw) {
            __threadfence_block();
            const uint32_t bmin = atomicOr(&s_kmin, 0u), bmax = atomicOr(&s_kmax, 0u);
            if (bmin <= bmax) {
                // the slots only grow, so a block whose values do not exceed
                // what it reads now can skip its atomic
                const unsigned long long gen = (unsigned long long)(uint32_t)ws.counters[kCtrRangeGen] << 32;
                const unsigned long long vmax = gen | bmax, vmin = gen | (unsigned long long)(~bmin);
                volatile const unsigned long long* c = ws.counters;
                if (c[kCtrRangeMax] < vmax) atomicMax(&ws.counters[kCtrRangeMax], vmax);
                if (c[kCtrRangeMin] < vmin) atomicMax(&ws.counters[kCtrRangeMin], vmin);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Backward

template <int D>
__global__ void __launch_bounds__(256, 3) k_project_bwd(const __grid_constant__ BatchParam bp,
                                                     GaussPtrs g, RenderConst rc, WsPtrs ws,
                                                     GradPtrs gr, int want_params, int want_pose,
                                                     int pose_blocks) {
    pdl_wait();
    pdl_trigger();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < g.n;
    constexpr int K = (D + 1) * (D + 1);

    Proj P;
    float mu[3] = {0.f, 0.f, 0.f}, ologit = 0.f;
    if (live) load_gaussian(g, i, mu, P, ologit);

    float gmu[3] = {0.f, 0.f, 0.f};
    float gM[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dL/d(R S)
    float gop = 0.f;
    float gsh[K * 3];
#pragma unroll
    for (int e = 0; e < K * 3; ++e) gsh[e] = 0.f;

    __shared__ float s_red[8][6];

    for (int vi = 0; vi < bp.n_views; ++vi) {
        const ViewParam& V = bp.v[vi];
        float pose[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool inview = live && i >= V.g_begin && i < V.g_end;
        const long long r = V.rec_off + (i - V.g_begin);
        float acc[kGrad2D];
        if (inview) {
            bool any = false;
            for (int e = 0; e < kGrad2D; ++e) {
                acc[e] = ws.grad2d[r * kGrad2D + e];
                any |= acc[e] != 0.f;
            }
            inview = any && project_view(V, rc, mu, P);
        }
        if (inview) {
            const float sigma = 1.f / (1.f + expf(-ologit));
            // record-space gradients -> natural parameters (see k_render_bwd):
            // acc[0..1] hold sum ga (d.v1), sum ga (d.v2); dp/dq = 2 ((d.v1) v1 + (d.v2) v2)
            const float4 ra = ws.rec[3 * r], rb = ws.rec[3 * r + 1];
            const float gqx = 2.f * kLn2 * fmaf(ra.z, acc[0], rb.x * acc[1]);
            const float gqy = 2.f * kLn2 * fmaf(ra.w, acc[0], rb.y * acc[1]);
            const float gA = -0.5f * acc[2], gB = -acc[3], gC = -0.5f * acc[4];
            const float gsig = acc[5] / sigma;
            float col[3];
            view_colour<D>(V, g, i, mu, P, col);
            // colour -> SH (+ view direction): dL/dk_k = Y_k graw, and the
            // direction gradient sum_k w_k grad Y_k with w_k = sum_ch k_k,ch graw_ch
            float gd[3] = {0.f, 0.f, 0.f};
            {
                float graw[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) graw[ch] = P.raw[ch] > 0.f ? acc[6 + ch] : 0.f;
                float Y[K];
                sh_basis<D>(P.dir, Y);
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) gsh[3 * k + ch] = fmaf(Y[k], graw[ch], gsh[3 * k + ch]);
                if (D >= 1) {
                    const long long base = i * K * 3;
                    float w[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        w[k] = 0.f;
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch)
                            w[k] = fmaf(load_as_float(g.sh, g.sh_dtype, base + 3 * k + ch), graw[ch], w[k]);
                    }
                    float gdir[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float e[3] = {c == 0 ? 1.f : 0.f, c == 1 ? 1.f : 0.f, c == 2 ? 1.f : 0.f};
                        float T[K];
                        sh_basis_along<D>(P.dir, e, T);
                        gdir[c] = 0.f;
#pragma unroll
                        for (int k = 1; k < K; ++k) gdir[c] = fmaf(w[k], T[k], gdir[c]);
                    }
                    // dir = d / |d|: dL/dd = (gdir - dir (dir . gdir)) / |d|
                    const float dd = P.dir[0] * gdir[0] + P.dir[1] * gdir[1] + P.dir[2] * gdir[2];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        gd[k] = (gdir[k] - P.dir[k] * dd) * P.inv_len;
                        gmu[k] += gd[k];
                    }
                }
            }
            gop += gsig * sigma * (1.f - sigma);

            // conic Q = Sigma2^-1, dL/dSigma2 = -Q G Q with G = [[gA, gB/2], [gB/2, gC]]
            const float hB = 0.5f * gB;
            const float m00 = P.A * gA + P.B * hB, m01 = P.A * hB + P.B * gC;
            const float m10 = P.B * gA + P.C * hB, m11 = P.B * hB + P.C * gC;
            const float G00 = -(m00 * P.A + m01 * P.B);
            const float G01 = -(m00 * P.B + m01 * P.C);
            const float G11 = -(m10 * P.B + m11 * P.C);
            // Sigma2 = U U^T + blur I with U = T M: dL/dU = 2 G2 U, dL/dT = dL/dU M^T,
            // dL/dM += T^T dL/dU (accumulated over views).
            float gU0[3], gU1[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gU0[k] = 2.f * (G00 * P.U[k] + G01 * P.U[3 + k]);
                gU1[k] = 2.f * (G01 * P.U[k] + G11 * P.U[3 + k]);
            }
            float gT0[3], gT1[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                gT0[j] = gU0[0] * P.M[3 * j] + gU0[1] * P.M[3 * j + 1] + gU0[2] * P.M[3 * j + 2];
                gT1[j] = gU1[0] * P.M[3 * j] + gU1[1] * P.M[3 * j + 1] + gU1[2] * P.M[3 * j + 2];
            }
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) gM[3 * j + k] += P.Tm[j] * gU0[k] + P.Tm[3 + j] * gU1[k];
            // T = J W: dL/dJ = dL/dT W^T (only J00, J02, J11, J12 are non-zero)
            const float gJ00 = gT0[0] * V.R[0] + gT0[1] * V.R[1] + gT0[2] * V.R[2];
            const float gJ02 = gT0[0] * V.R[6] + gT0[1] * V.R[7] + gT0[2] * V.R[8];
            const float gJ11 = gT1[0] * V.R[3] + gT1[1] * V.R[4] + gT1[2] * V.R[5];
            const float gJ12 = gT1[0] * V.R[6] + gT1[1] * V.R[7] + gT1[2] * V.R[8];
            const float x = P.pc[0], y = P.pc[1], z = P.pc[2];
            const float iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
            float gp[3];
            gp[0] = gJ02 * (-V.fx * iz2) + gqx * V.fx * iz;
            gp[1] = gJ12 * (-V.fy * iz2) + gqy * V.fy * iz;
            gp[2] = gJ00 * (-V.fx * iz2) + gJ02 * (2.f * V.fx * x * iz3) + gJ11 * (-V.fy * iz2) +
                    gJ12 * (2.f * V.fy * y * iz3) - (gqx * V.fx * x + gqy * V.fy * y) * iz2;
            // p_C = W mu + t
            for (int k = 0; k < 3; ++k)
                gmu[k] += V.R[k] * gp[0] + V.R[3 + k] * gp[1] + V.R[6 + k] * gp[2];
            if (want_pose) {
                // dL/dW (through T = J W) = J^T dL/dT; J rows: (j00, 0, j02), (0, j11, j12)
                const float j00 = V.fx * iz, j02 = -V.fx * x * iz2;
                const float j11 = V.fy * iz, j12 = -V.fy * y * iz2;
                float gW[9];
                for (int b = 0; b < 3; ++b) {
                    gW[b] = j00 * gT0[b];
                    gW[3 + b] = j11 * gT1[b];
                    gW[6 + b] = j02 * gT0[b] + j12 * gT1[b];
                }
                // M = gW W^T ; dphi += vee-like terms (M21 - M12, M02 - M20, M10 - M01)
                float Mw[9];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        Mw[3 * a + b] = gW[3 * a] * V.R[3 * b] + gW[3 * a + 1] * V.R[3 * b + 1] +
                                        gW[3 * a + 2] * V.R[3 * b + 2];
                pose[0] = (y * gp[2] - z * gp[1]) + (Mw[7] - Mw[5]);
                pose[1] = (z * gp[0] - x * gp[2]) + (Mw[2] - Mw[6]);
                pose[2] = (x * gp[1] - y * gp[0]) + (Mw[3] - Mw[1]);
                for (int k = 0; k < 3; ++k)
                    pose[3 + k] = gp[k] + V.R[3 * k] * gd[0] + V.R[3 * k + 1] * gd[1] + V.R[3 * k + 2] * gd[2];
            }
        }
        if (want_pose) {
            // Block reduction of the 6 pose components for this view.
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                float v = pose[k];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                pose[k] = v;
            }
            const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
            if (lane == 0)
                for (int k = 0; k < 6; ++k) s_red[w][k] = pose[k];
            __syncthreads();
            if (threadIdx.x < 6 && (int)blockIdx.x < pose_blocks) {
                float v = 0.f;
                for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) v += s_red[ww][threadIdx.x];
                ws.partials[((long long)vi * pose_blocks + blockIdx.x) * 6 + threadIdx.x] = v;
            }
            __syncthreads();
        }
    }

    if (!live || !want_params) return;
    // want_params 2: add to the gradients already there (several batches of
    // views summed before one optimiser step)
    const bool acc = want_params == 2;
    auto put = [acc](float* dst, float v) { *dst = acc ? *dst + v : v; };
    float gR[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) gR[3 * a + b] = gM[3 * a + b] * P.s[b];
    for (int b = 0; b < 3; ++b)
        put(gr.log_scales + 3 * i + b, (gM[b] * P.R[b] + gM[3 + b] * P.R[3 + b] + gM[6 + b] * P.R[6 + b]) * P.s[b]);
    const float w = P.qh[0], x = P.qh[1], y = P.qh[2], z = P.qh[3];
    float gq[4];
    gq[0] = 2.f * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2.f * (y * gR[1] + z * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] + z * gR[6] + w * gR[7] -
                   2.f * x * gR[8]);
    gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7] -
                   2.f * y * gR[8]);
    gq[3] = 2.f * (-2.f * z * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * z * gR[4] + y * gR[5] +
                   x * gR[6] + y * gR[7]);
    const float dq = gq[0] * P.qh[0] + gq[1] * P.qh[1] + gq[2] * P.qh[2] + gq[3] * P.qh[3];
    for (int k = 0; k < 4; ++k) put(gr.quats + 4 * i + k, (gq[k] - P.qh[k] * dq) * P.inv_qn);
    for (int k = 0; k < 3; ++k) put(gr.means + 3 * i + k, gmu[k]);
    put(gr.opacity + i, gop);
#pragma unroll
    for (int e = 0; e < K * 3; ++e) put(gr.sh + i * K * 3 + e, gsh[e]);
}

__global__ void k_pose_finish(const float* partials, int nblocks, int n_views, float* dL_dpose) {
    pdl_wait();
    pdl_trigger();
    // one warp per (view, component): fixed-order sum for determinism
    const int item = blockIdx.x;
    if (item >= n_views * 6) return;
    const int vi = item / 6, k = item % 6;
    float s = 0.f;
    for (int b = threadIdx.x; b < nblocks; b += 32) s += partials[((long long)vi * nblocks + b) * 6 + k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) dL_dpose[vi * 6 + k] = s;
}

// Pose tangents of one record (view, Gaussian): derivatives of its projected
// mean q, of Sigma2 and of its colour with respect to the left perturbation
// xi = [dphi; dt] of the camera, T_CW <- Exp(xi) T_CW (Appendix A), for the
// forward-mode compositing of the pose normal equations.  With p_C the
// camera-frame mean, J the projection Jacobian and Mc = R_CW R S:
//   dp_C/ddphi_k = e_k x p_C,  dp_C/ddt_k = e_k,  dR_CW/ddphi_k = [e_k]x R_CW,
//   dq = J dp_C,  U = J Mc:  dU = dJ Mc + J [e_k]x Mc,
//   dSigma2 = dU U^T + U dU^T,
//   dcolour = d SH(dir) with dir = (mu - campos)/|mu - campos| and
//   dcampos/ddt_k = -(row k of R_CW)^T (0 where the colour is clamped).
// Layout per record, k = 0..5: tan[12 r + 2k] = (dq_x, dq_y, dS_a, dS_b),
// tan[12 r + 2k + 1] = (dS_c, dc_r, dc_g, dc_b), with Sigma2 = [[a, b], [b, c]].
// Records with no listed tile are skipped (never read).
template <int D>
__global__ void __launch_bounds__(256) k_pose_tangents(const __grid_constant__ BatchParam bp, GaussPtrs g,
                                                       RenderConst rc, WsPtrs ws, float4* __restrict__ tan) {
    pdl_wait();
    pdl_trigger();
    const ViewParam& V = bp.v[blockIdx.y];
    const long long k0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cnt = V.g_end - V.g_begin;
    if (k0 >= cnt) return;
    const long long i = V.g_begin + k0;
    const long long r = V.rec_off + k0;
    if (ws.tiles_touched[r] == 0) return;
    Proj P;
    float mu[3], ologit;
    load_gaussian(g, i, mu, P, ologit);
    if (!project_view(V, rc, mu, P)) return;
    float col[3];
    view_colour<D>(V, g, i, mu, P, col);
    float Mc[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
            Mc[3 * a + b] = V.R[3 * a] * P.M[b] + V.R[3 * a + 1] * P.M[3 + b] + V.R[3 * a + 2] * P.M[6 + b];
    const float x = P.pc[0], y = P.pc[1], z = P.pc[2];
    const float iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
    const float j00 = V.fx * iz, j02 = -V.fx * x * iz2;
    const float j11 = V.fy * iz, j12 = -V.fy * y * iz2;
    constexpr int K = (D + 1) * (D + 1);
    float4* out = tan + (size_t)kPoseTan4 * r;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        float dp[3] = {0.f, 0.f, 0.f};
        if (k == 0) { dp[1] = -z; dp[2] = y; }
        if (k == 1) { dp[0] = z; dp[2] = -x; }
        if (k == 2) { dp[0] = -y; dp[1] = x; }
        if (k >= 3) dp[k - 3] = 1.f;
        const float dj00 = -V.fx * dp[2] * iz2;
        const float dj02 = -V.fx * dp[0] * iz2 + 2.f * V.fx * x * dp[2] * iz3;
        const float dj11 = -V.fy * dp[2] * iz2;
        const float dj12 = -V.fy * dp[1] * iz2 + 2.f * V.fy * y * dp[2] * iz3;
        const float dqx = j00 * dp[0] + j02 * dp[2];
        const float dqy = j11 * dp[1] + j12 * dp[2];
        float dU0[3], dU1[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const float m0 = Mc[b], m1 = Mc[3 + b], m2 = Mc[6 + b];
            // [e_k]x Mc, column b
            float X0 = 0.f, X1 = 0.f, X2 = 0.f;
            if (k == 0) { X1 = -m2; X2 = m1; }
            if (k == 1) { X0 = m2; X2 = -m0; }
            if (k == 2) { X0 = -m1; X1 = m0; }
            dU0[b] = dj00 * m0 + dj02 * m2 + j00 * X0 + j02 * X2;
            dU1[b] = dj11 * m1 + dj12 * m2 + j11 * X1 + j12 * X2;
        }
        const float* U0 = P.U;
        const float* U1 = P.U + 3;
        const float dSa = 2.f * (dU0[0] * U0[0] + dU0[1] * U0[1] + dU0[2] * U0[2]);
        const float dSb = dU0[0] * U1[0] + dU0[1] * U1[1] + dU0[2] * U1[2] + U0[0] * dU1[0] + U0[1] * dU1[1] +
                          U0[2] * dU1[2];
        const float dSc = 2.f * (dU1[0] * U1[0] + dU1[1] * U1[1] + dU1[2] * U1[2]);
        float dc[3] = {0.f, 0.f, 0.f};
        if (k >= 3 && D >= 1) {
            // a camera translation moves the centre: d(dir) = (W^T e - dir (dir . W^T e)) / |d|
            const float dv0 = V.R[3 * (k - 3)], dv1 = V.R[3 * (k - 3) + 1], dv2 = V.R[3 * (k - 3) + 2];
            const float dd = P.dir[0] * dv0 + P.dir[1] * dv1 + P.dir[2] * dv2;
            const float ddir[3] = {(dv0 - P.dir[0] * dd) * P.inv_len, (dv1 - P.dir[1] * dd) * P.inv_len,
                                   (dv2 - P.dir[2] * dd) * P.inv_len};
            float T[K];
            sh_basis_along<D>(P.dir, ddir, T);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float draw = 0.f;
#pragma unroll
                for (int m = 1; m < K; ++m)
                    draw = fmaf(T[m], load_as_float(g.sh, g.sh_dtype, i * K * 3 + 3 * m + ch), draw);
                dc[ch] = P.raw[ch] > 0.f ? draw : 0.f;
            }
        }
        out[2 * k] = make_float4(dqx, dqy, dSa, dSb);
        out[2 * k + 1] = make_float4(dSc, dc[0], dc[1], dc[2]);
    }
}

}  // namespace

cudaError_t launch_project(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                           const WsPtrs& ws, cudaStream_t s, Prof& pf) {
    if (bp.max_count <= 0) return cudaSuccess;
    dim3 grid((unsigned)((bp.max_count + 255) / 256), (unsigned)bp.n_views);
    const int pi = pf.begin(GS_KF_PROJECT, s);
    switch (g.sh_degree) {
        case 0: pdl_launch(k_project<0>, grid, 256, 0, s, bp, g, rc, ws); break;
        case 1: pdl_launch(k_project<1>, grid, 256, 0, s, bp, g, rc, ws); break;
        case 2: pdl_launch(k_project<2>, grid, 256, 0, s, bp, g, rc, ws); break;
        default: pdl_launch(k_project<3>, grid, 256, 0, s, bp, g, rc, ws); break;
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_project_bwd(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                               const WsPtrs& ws, const GradPtrs* grads, float* dL_dpose,
                               cudaStream_t s, Prof& pf, bool accumulate) {
    if (g.n <= 0) return cudaSuccess;
    const int nblk = (int)((g.n + 255) / 256);
    long long max_g_end = 0;
    for (int v = 0; v < bp.n_views; ++v)
        if (bp.v[v].g_end > max_g_end) max_g_end = bp.v[v].g_end;
    // Blocks past the last Gaussian any view renders contribute no pose
    // gradient; the partials buffer is sized for the others.
    const int pose_blocks = (int)((max_g_end + 255) / 256);
    GradPtrs gr = grads ? *grads : GradPtrs{nullptr, nullptr, nullptr, nullptr, nullptr};
    const int pi = pf.begin(GS_KF_PROJECT_BWD, s, dL_dpose ? 2 : 1);
    const int wp = grads == nullptr ? 0 : (accumulate ? 2 : 1), wq = dL_dpose != nullptr;
    switch (g.sh_degree) {
        case 0: pdl_launch(k_project_bwd<0>, nblk, 256, 0, s, bp, g, rc, ws, gr, wp, wq, pose_blocks); break;
        case 1: pdl_launch(k_project_bwd<1>, nblk, 256, 0, s, bp, g, rc, ws, gr, wp, wq, pose_blocks); break;
        case 2: pdl_launch(k_project_bwd<2>, nblk, 256, 0, s, bp, g, rc, ws, gr, wp, wq, pose_blocks); break;
        default: pdl_launch(k_project_bwd<3>, nblk, 256, 0, s, bp, g, rc, ws, gr, wp, wq, pose_blocks); break;
    }
    if (dL_dpose) pdl_launch(k_pose_finish, bp.n_views * 6, 32, 0, s, ws.partials, pose_blocks, bp.n_views, dL_dpose);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_pose_tangents(const BatchParam& bp, const GaussPtrs& g, const RenderConst& rc,
                                 const WsPtrs& ws, float4* tangents, cudaStream_t s, Prof& pf) {
    if (bp.max_count <= 0) return cudaSuccess;
    dim3 grid((unsigned)((bp.max_count + 255) / 256), (unsigned)bp.n_views);
    const int pi = pf.begin(GS_KF_POSE_NORMAL, s);
    switch (g.sh_degree) {
        case 0: pdl_launch(k_pose_tangents<0>, grid, 256, 0, s, bp, g, rc, ws, tangents); break;
        case 1: pdl_launch(k_pose_tangents<1>, grid, 256, 0, s, bp, g, rc, ws, tangents); break;
        case 2: pdl_launch(k_pose_tangents<2>, grid, 256, 0, s, bp, g, rc, ws, tangents); break;
        default: pdl_launch(k_pose_tangents<3>, grid, 256, 0, s, bp, g, rc, ws, tangents); break;
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
