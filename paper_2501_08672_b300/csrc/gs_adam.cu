// Adam step over the flat FP32 parameter vector of the window (Sec. II-B.2,
// "Adam optimizer"; Kingma & Ba with bias correction as in torch.optim.Adam).
// HBM-bound: reads p, g, m, v and writes p, m, v (28 B per parameter), plus
// 2 B per parameter for an optional FP16/BF16 render copy.
#include "gs_internal.cuh"

namespace gsb {

namespace {

struct SegTable {
    long long begin[8], end[8];
    void* dst[8];
    int dtype[8];
    int n;
};

__device__ __forceinline__ void store_lowp(const SegTable& st, long long i, float x) {
    for (int s = 0; s < st.n; ++s) {
        if (i >= st.begin[s] && i < st.end[s]) {
            const long long o = i - st.begin[s];
            if (st.dtype[s] == GS_F16)
                static_cast<__half*>(st.dst[s])[o] = __float2half_rn(x);
            else
                static_cast<__nv_bfloat16*>(st.dst[s])[o] = __float2bfloat16_rn(x);
        }
    }
}

__device__ __forceinline__ float adam1(float& p, float g, float& m, float& v, float b1, float b2,
                                       float eps, float step_size, float inv_sqrt_bc2) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    const float denom = sqrtf(v) * inv_sqrt_bc2 + eps;
    p = p - step_size * (m / denom);
    return p;
}

// Step counter kept on the device (graph replays advance it): increments the
// count and stores lr / (1 - b1^t) and 1 / sqrt(1 - b2^t) for the Adam launch.
__global__ void k_adam_coef(long long* step, float lr, float b1, float b2, float2* coef) {
    pdl_wait();
    pdl_trigger();
    const long long t = ++(*step);
    const double bc1 = 1.0 - pow((double)b1, (double)t);
    const double bc2 = 1.0 - pow((double)b2, (double)t);
    *coef = make_float2((float)(lr / bc1), (float)(1.0 / sqrt(bc2)));
}

__global__ void __launch_bounds__(256) k_adam4(float4* __restrict__ p, const float4* __restrict__ g,
                                               float4* __restrict__ m, float4* __restrict__ v,
                                               long long n4, float b1, float b2, float eps,
                                               float step_size, float inv_sqrt_bc2, SegTable st,
                                               const float2* __restrict__ coef) {
    pdl_wait();
    pdl_trigger();
    if (coef) {
        const float2 c = *coef;
        step_size = c.x;
        inv_sqrt_bc2 = c.y;
    }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 pp = p[i], gg = g[i], mm = m[i], vv = v[i];
        adam1(pp.x, gg.x, mm.x, vv.x, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.y, gg.y, mm.y, vv.y, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.z, gg.z, mm.z, vv.z, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.w, gg.w, mm.w, vv.w, b1, b2, eps, step_size, inv_sqrt_bc2);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
        if (st.n) {
            store_lowp(st, 4 * i + 0, pp.x);
            store_lowp(st, 4 * i + 1, pp.y);
            store_lowp(st, 4 * i + 2, pp.z);
            store_lowp(st, 4 * i + 3, pp.w);
        }
    }
}

__global__ void k_adam_tail(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long start, long long n, float b1, float b2,
                            float eps, float step_size, float inv_sqrt_bc2, SegTable st,
                            const float2* __restrict__ coef) {
    pdl_wait();
    pdl_trigger();
    if (coef) {
        const float2 c = *coef;
        step_size = c.x;
        inv_sqrt_bc2 = c.y;
    }
    for (long long i = start + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float pp = p[i], mm = m[i], vv = v[i];
        adam1(pp, g[i], mm, vv, b1, b2, eps, step_size, inv_sqrt_bc2);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
        if (st.n) store_lowp(st, i, pp);
    }
}

// Adam over the union of up to 8 element ranges (the active rows of each
// parameter group): float4 work over the ranges' aligned parts concatenated
// (range r covers virtual float4 indices [pre4[r], pre4[r + 1])), and the
// ranges' last 0-3 elements by the first threads.
struct RangeTable {
    long long begin4[8];    // first float4 of the range (its begin / 4)
    long long pre4[9];      // prefix of the ranges' float4 counts
    long long tail0[8];     // first element of the range's scalar tail
    int tail_len[8];        // 0..3
    int n;
};

__global__ void __launch_bounds__(256) k_adam_ranges(float* __restrict__ p, const float* __restrict__ g,
                                                     float* __restrict__ m, float* __restrict__ v, RangeTable rt,
                                                     float b1, float b2, float eps, float step_size,
                                                     float inv_sqrt_bc2, SegTable st,
                                                     const float2* __restrict__ coef) {
    pdl_wait();
    pdl_trigger();
    if (coef) {
        const float2 c = *coef;
        step_size = c.x;
        inv_sqrt_bc2 = c.y;
    }
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n4 = rt.pre4[rt.n];
    int r = 0;
    for (long long i = tid; i < n4; i += stride) {
        while (i >= rt.pre4[r + 1]) ++r;  // i only grows, so r does too
        const long long q = rt.begin4[r] + (i - rt.pre4[r]);
        float4 pp = reinterpret_cast<float4*>(p)[q], gg = reinterpret_cast<const float4*>(g)[q];
        float4 mm = reinterpret_cast<float4*>(m)[q], vv = reinterpret_cast<float4*>(v)[q];
        adam1(pp.x, gg.x, mm.x, vv.x, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.y, gg.y, mm.y, vv.y, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.z, gg.z, mm.z, vv.z, b1, b2, eps, step_size, inv_sqrt_bc2);
        adam1(pp.w, gg.w, mm.w, vv.w, b1, b2, eps, step_size, inv_sqrt_bc2);
        reinterpret_cast<float4*>(p)[q] = pp;
        reinterpret_cast<float4*>(m)[q] = mm;
        reinterpret_cast<float4*>(v)[q] = vv;
        if (st.n) {
            store_lowp(st, 4 * q + 0, pp.x);
            store_lowp(st, 4 * q + 1, pp.y);
            store_lowp(st, 4 * q + 2, pp.z);
            store_lowp(st, 4 * q + 3, pp.w);
        }
    }
    if (tid < 4 * rt.n) {  // range tid / 4, tail element tid % 4
        const int rr = (int)(tid / 4), e = (int)(tid % 4);
        if (e < rt.tail_len[rr]) {
            const long long i = rt.tail0[rr] + e;
            float pp = p[i], mm = m[i], vv = v[i];
            adam1(pp, g[i], mm, vv, b1, b2, eps, step_size, inv_sqrt_bc2);
            p[i] = pp;
            m[i] = mm;
            v[i] = vv;
            if (st.n) store_lowp(st, i, pp);
        }
    }
}

}  // namespace

cudaError_t launch_adam_ranges(float* p, const float* g, float* m, float* v, const gs_range* ranges, int n_ranges,
                               float b1, float b2, float eps, float step_size, float inv_sqrt_bc2,
                               const gs_lowp_segment* segs, int n_segs, cudaStream_t s, Prof& pf,
                               long long* step_dev, float lr, float2* coef, int sm_count) {
    SegTable st{};
    st.n = n_segs;
    for (int k = 0; k < n_segs && k < 8; ++k) {
        st.begin[k] = segs[k].begin;
        st.end[k] = segs[k].end;
        st.dst[k] = segs[k].dst;
        st.dtype[k] = segs[k].dtype;
    }
    RangeTable rt{};
    rt.n = n_ranges;
    rt.pre4[0] = 0;
    for (int k = 0; k < n_ranges; ++k) {
        const long long len = ranges[k].end - ranges[k].begin;
        rt.begin4[k] = ranges[k].begin / 4;
        rt.pre4[k + 1] = rt.pre4[k] + len / 4;
        rt.tail0[k] = ranges[k].begin + 4 * (len / 4);
        rt.tail_len[k] = (int)(len % 4);
    }
    const int pi = pf.begin(GS_KF_ADAM, s, 1 + (step_dev != nullptr));
    if (step_dev) pdl_launch(k_adam_coef, 1, 1, 0, s, step_dev, lr, b1, b2, coef);
    const long long n4 = rt.pre4[n_ranges];
    long long blocks = (n4 + 255) / 256;
    const long long cap = (long long)(sm_count > 0 ? sm_count : 148) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;  // the tails need one block
    pdl_launch(k_adam_ranges, (unsigned)blocks, 256, 0, s, p, g, m, v, rt, b1, b2, eps, step_size, inv_sqrt_bc2, st,
                                                   step_dev ? coef : nullptr);
    pf.end(pi, s);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n,
                        float b1, float b2, float eps, float step_size, float inv_sqrt_bc2,
                        const gs_lowp_segment* segs, int n_segs, cudaStream_t s, Prof& pf,
                        long long* step_dev, float lr, float2* coef) {
    SegTable st{};
    st.n = n_segs;
    for (int k = 0; k < n_segs && k < 8; ++k) {
        st.begin[k] = segs[k].begin;
        st.end[k] = segs[k].end;
        st.dst[k] = segs[k].dst;
        st.dtype[k] = segs[k].dtype;
    }
    const bool aligned = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(g) |
                           reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    long long n4 = aligned ? n / 4 : 0;
    const int pi = pf.begin(GS_KF_ADAM, s, (n4 > 0) + (4 * n4 < n) + (step_dev != nullptr));
    if (step_dev) pdl_launch(k_adam_coef, 1, 1, 0, s, step_dev, lr, b1, b2, coef);
    const float2* cf = step_dev ? coef : nullptr;
    if (n4 > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        long long blocks = (n4 + 255) / 256;
        const long long cap = (long long)sms * 8;
        if (blocks > cap) blocks = cap;
        pdl_launch(k_adam4, (unsigned)blocks, 256, 0, s, reinterpret_cast<float4*>(p), reinterpret_cast<const float4*>(g),
                                                 reinterpret_cast<float4*>(m), reinterpret_cast<float4*>(v), n4, b1,
                                                 b2, eps, step_size, inv_sqrt_bc2, st, cf);
    }
    if (4 * n4 < n) {
        const long long rest = n - 4 * n4;
        const long long blocks = rest < 256 * 1184 ? (rest + 255) / 256 : 1184;
        pdl_launch(k_adam_tail, (unsigned)blocks, 256, 0, s, p, g, m, v, 4 * n4, n, b1, b2, eps, step_size,
                                                     inv_sqrt_bc2, st, cf);
    }
    pf.end(pi, s);
    return cudaGetLastError();
}

}  // namespace gsb
