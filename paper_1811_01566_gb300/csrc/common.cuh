// Internal helpers shared by the CUDA translation units of libwf (not part of the ABI).
#pragma once

#include <cuda.h>            // CUtensorMap (the descriptor type only; no driver API is linked)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "wf.h"

namespace wf {

// ---------------------------------------------------------------------------
// Host-side status plumbing.
// ---------------------------------------------------------------------------
inline wf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? WF_OK : WF_ERR_CUDA; }

// Raise a kernel's dynamic shared-memory limit to `bytes` once per device.
// Done outside stream capture on the first call for a device (the attribute
// is not a stream operation), so later calls can be captured in CUDA graphs.
template <typename K>
inline wf_status ensure_smem_limit(K kernel, size_t bytes, unsigned long long& done_mask) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WF_ERR_CUDA;
    const unsigned long long bit = 1ull << (dev & 63);
    if (__atomic_load_n(&done_mask, __ATOMIC_ACQUIRE) & bit) return WF_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess)
        return WF_ERR_CUDA;
    __atomic_fetch_or(&done_mask, bit, __ATOMIC_ACQ_REL);
    return WF_OK;
}

inline wf_status last_launch_status() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? WF_OK : WF_ERR_CUDA;
}

// Log compression with dynamic-range clipping of one envelope value against its frame's
// reference (the last block of Fig. 2): clamp(20 log10(max(e, 1e-30 ref) / ref), lo, hi);
// NaN stays NaN, a reference that is not positive gives lo.  Shared by the log-clip kernels
// and the envelope kernel's fused epilogue, so both give the same bits.
__device__ __forceinline__ float db_value(float e, float ref, float lo, float hi) {
    if (e != e) return e;
    if (!(ref > 0.0f)) return lo;
    const float v = fmaxf(e, 1e-30f * ref);
    const float db = 20.0f * log10f(v / ref);
    return fminf(fmaxf(db, lo), hi);
}

// Status block at the head of every DAS workspace (device side).
struct WsHeader {
    unsigned int flags;   // bit 0: staging window overflow, bit 1: gather index out of window
    unsigned int first_bad[3];
    unsigned int pad[60];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");
constexpr size_t kWsHeaderBytes = 256;

// ---------------------------------------------------------------------------
// Geometry in sample units.  The host converts every physical length to
// samples (multiplying by fs / c) in double and rounds once to float, so a
// distance d in samples is directly a delay.
// ---------------------------------------------------------------------------
struct Geom {
    float gx0, gdx;     // pixel x: gx0 + ix * gdx (samples)
    float gz0, gdz;     // pixel z: gz0 + iz * gdz (samples)
    float xe0, pitch;   // element x: xe0 + e * pitch (samples)
    float two_f;        // 2 F: aperture scale, u = (x_e - x) * 2F / z
    int apod;           // wf_apod
    int n_elements;
    int nz, nx;
    const float* elem_weight;  // device [E] or nullptr
};

__device__ __forceinline__ float pixel_x(const Geom& g, int ix) { return fmaf((float)ix, g.gdx, g.gx0); }
__device__ __forceinline__ float pixel_z(const Geom& g, int iz) { return fmaf((float)iz, g.gdz, g.gz0); }
__device__ __forceinline__ float elem_x(const Geom& g, int e) { return fmaf((float)e, g.pitch, g.xe0); }

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers (about 48 significant bits).  Built from the error-free transforms
// TwoSum (Knuth) and TwoProd (one FMA), so reference geometry keeps FP64-like
// accuracy without FP64 instructions.  Requires IEEE round-to-nearest FP32
// and no reassociation (the library is compiled without fast-math).
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__host__ __device__ inline DF df_from_double(double v) {
    DF r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return quick_two_sum(p, e + fmaf(a.hi, b.lo, a.lo * b.hi));
}

// a + k b for a small integer k (exact as a float).
__device__ __forceinline__ DF df_axpk(DF a, int k, DF b) {
    return df_add(a, df_mul(DF{(float)k, 0.0f}, b));
}

// Square root of a non-negative double-float: FP32 root plus one Newton step.
__device__ __forceinline__ DF df_sqrt(DF a) {
    if (!(a.hi > 0.0f)) return DF{0.0f, 0.0f};
    const float r = sqrtf(a.hi);
    const float rr = r * r;
    const float rre = fmaf(r, r, -rr);               // r^2 = rr + rre exactly
    const float corr = (((a.hi - rr) - rre) + a.lo) * (0.5f / r);
    return quick_two_sum(r, corr);
}

// Inverse half-aperture 2F / z of a pixel (0 when z <= 0: no aperture).
__device__ __forceinline__ float aperture_kappa(const Geom& g, float pz) {
    return pz > 0.0f ? g.two_f / pz : 0.0f;
}

}  // namespace wf
