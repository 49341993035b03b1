// Dynamic adjustment: log compression with dynamic-range clipping (paper
// Fig. 2 "Dynamic Adjustment"; Sec. III clips the displayed range).
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

__device__ __forceinline__ float db_value(float e, float ref, float lo, float hi) {
    if (e != e) return e;
    if (!(ref > 0.0f)) return lo;
    const float v = fmaxf(e, 1e-30f * ref);
    const float db = 20.0f * log10f(v / ref);
    return fminf(fmaxf(db, lo), hi);
}

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
