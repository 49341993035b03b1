// Dynamic adjustment: log compression with dynamic-range clipping (paper
// the last block of Fig. 2; Sec. III clips the displayed range).
//
//   out = clamp(20 log10(max(env, 1e-30 ref) / ref), lo, hi)
//
// ref is the caller's per-frame reference, or the frame's largest non-NaN
// envelope value.  The frame maximum is a whole-frame dependency; without a
// caller reference one thread-block cluster per frame (8 CTAs) reduces it in
// distributed shared memory and then writes the frame, so no global scratch
// and no second launch are needed.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace wf {

__global__ void logclip_ref_kernel(const float* __restrict__ env, const float* __restrict__ ref,
                                   long long frame, float lo, float hi, float* __restrict__ out) {
    const int b = blockIdx.y;
    const float r = __ldg(ref + b);
    const float* src = env + (long long)b * frame;
    float* dst = out + (long long)b * frame;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < frame;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = db_value(src[i], r, lo, hi);
}

constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 1024;

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
logclip_cluster_kernel(const float* env, long long frame, float lo, float hi, float* out) {
    __shared__ float warp_max[kClusterThreads / 32];
    __shared__ float cta_max;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.y;
    const float* src = env + (long long)b * frame;
    float* dst = out + (long long)b * frame;
    const long long stride = (long long)kClusterCtas * kClusterThreads;
    const long long first = (long long)rank * kClusterThreads + threadIdx.x;

    float m = 0.0f;
    for (long long i = first; i < frame; i += stride) {
        const float v = src[i];
        if (v == v) m = fmaxf(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = warp_max[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) cta_max = v;
    }
    cluster.sync();
    float ref = 0.0f;
#pragma unroll
    for (int r = 0; r < kClusterCtas; ++r) ref = fmaxf(ref, *cluster.map_shared_rank(&cta_max, r));
    cluster.sync();  // peers' shared memory stays alive until every CTA has read it
    for (long long i = first; i < frame; i += stride) dst[i] = db_value(src[i], ref, lo, hi);
}

// Reverse mode.  Where the value is strictly inside (lo, hi) and env >
// 1e-30 ref (same FP32 decision as the forward), d out / d env = 20 / (ln 10
// env) and d out / d ref = -20 / (ln 10 ref); clipped, floored or NaN pixels
// pass nothing.  When ref is the frame maximum (no caller reference, or the
// caller says its reference is that maximum) the reference's cotangent goes to
// the first pixel attaining it.  One 8-CTA cluster per frame: maximum (if
// needed), then the reference cotangent and the first maximal pixel, reduced
// in distributed shared memory in a fixed order, then the write pass.
constexpr float kDbPerLn = 8.685889638065037f;   // 20 / ln 10

__device__ __forceinline__ bool db_inside(float e, float ref, float lo, float hi) {
    if (e != e || !(ref > 0.0f) || !(e > 1e-30f * ref)) return false;
    const float db = 20.0f * log10f(fmaxf(e, 1e-30f * ref) / ref);
    return db > lo && db < hi;
}

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads)
logclip_backward_kernel(const float* env, const float* ref_in, int route, long long frame, float lo,
                        float hi, const float* g_db, float* g_env) {
    __shared__ float red_f[kClusterThreads / 32];
    __shared__ long long red_i[kClusterThreads / 32];
    __shared__ float cta_f;
    __shared__ long long cta_i;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int b = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float* src = env + (long long)b * frame;
    const float* gsrc = g_db + (long long)b * frame;
    float* dst = g_env + (long long)b * frame;
    const long long stride = (long long)kClusterCtas * kClusterThreads;
    const long long first = (long long)rank * kClusterThreads + threadIdx.x;

    float ref;
    if (ref_in) {
        ref = __ldg(ref_in + b);
    } else {
        float m = 0.0f;
        for (long long i = first; i < frame; i += stride) {
            const float v = src[i];
            if (v == v) m = fmaxf(m, v);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) red_f[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            float v = 0.0f;
            for (int w = 0; w < kClusterThreads / 32; ++w) v = fmaxf(v, red_f[w]);
            cta_f = v;
        }
        cluster.sync();
        ref = 0.0f;
        for (int r = 0; r < kClusterCtas; ++r) ref = fmaxf(ref, *cluster.map_shared_rank(&cta_f, r));
        cluster.sync();
    }
    const float dref = -kDbPerLn / ref;
    float s = 0.0f;
    long long arg = frame;
    if (route) {
        for (long long i = first; i < frame; i += stride) {
            const float e = src[i];
            if (e == ref && i < arg) arg = i;
            if (db_inside(e, ref, lo, hi)) s = fmaf(gsrc[i], dref, s);
        }
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            arg = min(arg, (long long)__shfl_xor_sync(0xffffffffu, arg, o));
        }
        if (lane == 0) {
            red_f[warp] = s;
            red_i[warp] = arg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float v = 0.0f;
            long long a = frame;
            for (int w = 0; w < kClusterThreads / 32; ++w) {
                v += red_f[w];
                a = min(a, red_i[w]);
            }
            cta_f = v;
            cta_i = a;
        }
        cluster.sync();
        s = 0.0f;
        arg = frame;
        for (int r = 0; r < kClusterCtas; ++r) {
            s += *cluster.map_shared_rank(&cta_f, r);
            arg = min(arg, *cluster.map_shared_rank(&cta_i, r));
        }
        cluster.sync();
    }
    for (long long i = first; i < frame; i += stride) {
        const float e = src[i];
        float g = db_inside(e, ref, lo, hi) ? gsrc[i] * (kDbPerLn / e) : 0.0f;
        if (i == arg) g += s;
        dst[i] = g;
    }
}

}  // namespace wf

using namespace wf;

extern "C" wf_status wf_logclip(const float* env, int32_t batch, int32_t nz, int32_t nx,
                                const float* ref, float db_min, float db_max, float* out_db,
                                wf_stream stream) {
    if (!env || !out_db || batch < 1 || batch > 65535 || nz < 1 || nx < 1) return WF_ERR_INVALID_ARG;
    if (!(db_min <= db_max)) return WF_ERR_INVALID_ARG;
    const long long frame = (long long)nz * nx;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (ref) {
        long long blocks = (frame + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        logclip_ref_kernel<<<dim3((unsigned)blocks, batch), 256, 0, st>>>(env, ref, frame, db_min,
                                                                         db_max, out_db);
    } else {
        logclip_cluster_kernel<<<dim3(kClusterCtas, batch), kClusterThreads, 0, st>>>(
            env, frame, db_min, db_max, out_db);
    }
    return last_launch_status();
}

extern "C" wf_status wf_logclip_backward(const float* env, int32_t batch, int32_t nz, int32_t nx,
                                         const float* ref, int32_t ref_is_frame_max, float db_min,
                                         float db_max, const float* grad_db, float* grad_env,
                                         wf_stream stream) {
    if (!env || !grad_db || !grad_env || batch < 1 || batch > 65535 || nz < 1 || nx < 1)
        return WF_ERR_INVALID_ARG;
    if (!(db_min <= db_max)) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)env & 3u) || ((uintptr_t)grad_db & 3u) || ((uintptr_t)grad_env & 3u) ||
        ((uintptr_t)ref & 3u))
        return WF_ERR_INVALID_ARG;
    if (grad_env == env) return WF_ERR_INVALID_ARG;
    const long long frame = (long long)nz * nx;
    const int route = (!ref || ref_is_frame_max) ? 1 : 0;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    logclip_backward_kernel<<<dim3(kClusterCtas, batch), kClusterThreads, 0, st>>>(
        env, ref, route, frame, db_min, db_max, grad_db, grad_env);
    return last_launch_status();
}
