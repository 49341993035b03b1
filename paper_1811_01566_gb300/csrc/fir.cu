// Pre-processing of RF traces (paper Sec. II-B, signal processing operators:
// FIR filter as the pre-processing op): FIR filtering and IQ demodulation.
//
//   FIR:  y[n] = sum_{k<L} h[k] x[n + (L-1)/2 - k]          (odd L, x = 0 outside)
//   IQ:   iq[m] = sum_{k<L} h[k] x[i] exp(-2 pi i f0 i / fs),  i = m D + (L-1)/2 - k
//
// Both are HBM-streaming kernels: a CTA stages its input span (converted to
// FP32, times the int16 scale) in shared memory once and every output reads
// it from there.  FIR: each thread produces 4 consecutive outputs with a
// register window over 16-byte shared loads (4 outputs x 4 taps per load).
// IQ: the mixing phase is reduced to turns in double-float before sincospif,
// so it stays exact to ~1e-7 turns at any sample index.
#include <cmath>

#include "common.cuh"

namespace wf {

constexpr int kFirThreads = 256;
constexpr int kFirOut = 4;                               // consecutive outputs per thread
constexpr int kFirBlock = kFirThreads * kFirOut;         // outputs per CTA
constexpr int kMaxTapsPad = ((WF_MAX_TAPS + 3) / 4) * 4;

struct FirArgs {
    float hr[kMaxTapsPad];   // reversed taps hr[u] = h[L-1-u], zero-padded to a multiple of 4
    int n_pad;               // padded tap count
    int n_taps;
    int ns;
    int decim;
    long long n_traces;
    float scale;
    DF turns;                // f0 / fs (IQ)
};

template <typename T> __device__ __forceinline__ float load_sample(const T* p);
template <> __device__ __forceinline__ float load_sample<float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_sample<__half>(const __half* p) {
    return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ float load_sample<int16_t>(const int16_t* p) {
    return (float)__ldg(p);
}

// y[n0 + j] = sum_u hr[u] xs[j + u], xs[i] = x[n0 - c + i].
template <typename T>
__global__ void __launch_bounds__(kFirThreads) fir_kernel(const __grid_constant__ FirArgs a,
                                                          const T* __restrict__ x, float* __restrict__ y) {
    extern __shared__ __align__(16) float xs[];          // [kFirBlock + n_pad + 4]
    const int c = (a.n_taps - 1) / 2;
    const int n0 = blockIdx.x * kFirBlock;
    const int span = kFirBlock + a.n_pad + 4;
    for (long long tr = blockIdx.y; tr < a.n_traces; tr += gridDim.y) {
        const T* src = x + tr * a.ns;
        for (int i = threadIdx.x; i < span; i += kFirThreads) {
            const int n = n0 - c + i;
            xs[i] = (n >= 0 && n < a.ns) ? load_sample<T>(src + n) * a.scale : 0.0f;
        }
        __syncthreads();
        const int b = kFirOut * threadIdx.x;
        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
        float4 lo = *reinterpret_cast<const float4*>(xs + b);
        for (int u = 0; u < a.n_pad; u += 4) {
            const float4 hi = *reinterpret_cast<const float4*>(xs + b + u + 4);
            const float w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float h = a.hr[u + q];
                acc0 = fmaf(h, w[q], acc0);
                acc1 = fmaf(h, w[q + 1], acc1);
                acc2 = fmaf(h, w[q + 2], acc2);
                acc3 = fmaf(h, w[q + 3], acc3);
            }
            lo = hi;
        }
        float* dst = y + tr * a.ns + n0 + b;
        const int left = a.ns - (n0 + b);
        if (left >= 4 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
            *reinterpret_cast<float4*>(dst) = make_float4(acc0, acc1, acc2, acc3);
        } else {
            if (left > 0) dst[0] = acc0;
            if (left > 1) dst[1] = acc1;
            if (left > 2) dst[2] = acc2;
            if (left > 3) dst[3] = acc3;
        }
        __syncthreads();
    }
}

constexpr int kIqThreads = 256;   // one output per thread
constexpr int kMaxDecim = 16;

// Phase of sample i in turns, f0 i / fs mod 1, from the double-float ratio
// (the product r_hi i is split exactly with an FMA).
__device__ __forceinline__ float mix_turns(DF r, int i) {
    const float fi = (float)i;                // exact: i < 2^24
    const float p = r.hi * fi;
    const float e = fmaf(r.hi, fi, -p);       // r_hi i = p + e exactly
    const float fp = p - floorf(p);           // exact for p < 2^23
    float t = fp + fmaf(r.lo, fi, e);
    return t - floorf(t);
}

template <typename T>
__global__ void __launch_bounds__(kIqThreads) iq_kernel(const __grid_constant__ FirArgs a,
                                                        const T* __restrict__ x, float2* __restrict__ iq,
                                                        int n_out) {
    // The mixed input span, stored by decimation phase: xm[p * plen + jj] = span sample
    // jj D + p.  Output t of the block sums taps u = v D + p over phase p at position t + v,
    // so adjacent threads read adjacent words (a plain span read at stride D conflicts on the
    // shared-memory banks for every D > 1).
    extern __shared__ __align__(16) float2 xm[];
    const int c = (a.n_taps - 1) / 2;
    const int D = a.decim;
    const int m0 = blockIdx.x * kIqThreads;
    const int i0 = m0 * D + c - (a.n_taps - 1);          // first input index of the span
    const int span = (kIqThreads - 1) * D + a.n_taps;
    const int plen = (span + D - 1) / D;                 // span samples per phase
    // j / D = (j * ceil(2^20 / D)) >> 20, exact for D <= 16 and j < 4400 (span <= 4335)
    const unsigned mdiv = ((1u << 20) + (unsigned)D - 1u) / (unsigned)D;
    for (long long tr = blockIdx.y; tr < a.n_traces; tr += gridDim.y) {
        const T* src = x + tr * a.ns;
        for (int j = threadIdx.x; j < span; j += kIqThreads) {
            const int i = i0 + j;
            float2 v = make_float2(0.0f, 0.0f);
            if (i >= 0 && i < a.ns) {
                const float s = load_sample<T>(src + i) * a.scale;
                float sn, cs;
                sincospif(2.0f * mix_turns(a.turns, i), &sn, &cs);
                v = make_float2(s * cs, -s * sn);
            }
            const int jj = (int)(((unsigned)j * mdiv) >> 20);
            xm[(j - jj * D) * plen + jj] = v;
        }
        __syncthreads();
        const int m = m0 + threadIdx.x;
        if (m < n_out) {
            // iq[m] = sum_k h[k] x[m D + c - k] = sum_u hr[u] span[t D + u], t = m - m0; with
            // u = v D + p that is phase p at position t + v
            float re = 0.0f, im = 0.0f;
            for (int p = 0; p < D && p < a.n_taps; ++p) {
                const float2* w = xm + p * plen + threadIdx.x;
                for (int u = p, v = 0; u < a.n_taps; u += D, ++v) {
                    const float h = a.hr[u];
                    const float2 x2 = w[v];
                    re = fmaf(h, x2.x, re);
                    im = fmaf(h, x2.y, im);
                }
            }
            iq[tr * n_out + m] = make_float2(re, im);
        }
        __syncthreads();
    }
}

bool fill_taps(FirArgs& a, const float* taps, int n_taps) {
    if (!taps || n_taps < 1 || n_taps > WF_MAX_TAPS || !(n_taps & 1)) return false;
    a.n_taps = n_taps;
    a.n_pad = ((n_taps + 3) / 4) * 4;
    for (int u = 0; u < kMaxTapsPad; ++u) a.hr[u] = u < n_taps ? taps[n_taps - 1 - u] : 0.0f;
    for (int k = 0; k < n_taps; ++k)
        if (!std::isfinite(taps[k])) return false;
    return true;
}

}  // namespace wf

using namespace wf;

extern "C" wf_status wf_fir(const void* rf, wf_dtype dtype, float rf_scale, int64_t n_traces,
                            int32_t n_samples, const float* taps, int32_t n_taps, float* out,
                            wf_stream stream) {
    if (!rf || !out || n_traces < 1 || n_samples < 1 || n_samples > WF_MAX_SAMPLES)
        return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (dtype == WF_I16 && !std::isfinite(rf_scale)) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)rf & 3u) || ((uintptr_t)out & 3u) || (const void*)out == rf) return WF_ERR_INVALID_ARG;
    thread_local FirArgs a;
    if (!fill_taps(a, taps, n_taps)) return WF_ERR_INVALID_ARG;
    a.ns = n_samples;
    a.n_traces = n_traces;
    a.decim = 1;
    a.scale = dtype == WF_I16 ? rf_scale : 1.0f;
    const size_t smem = sizeof(float) * (kFirBlock + a.n_pad + 4);
    dim3 grid((n_samples + kFirBlock - 1) / kFirBlock, (unsigned)std::min<int64_t>(n_traces, 65535));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    switch (dtype) {
        case WF_F32: fir_kernel<float><<<grid, kFirThreads, smem, st>>>(a, static_cast<const float*>(rf), out); break;
        case WF_F16: fir_kernel<__half><<<grid, kFirThreads, smem, st>>>(a, static_cast<const __half*>(rf), out); break;
        case WF_I16: fir_kernel<int16_t><<<grid, kFirThreads, smem, st>>>(a, static_cast<const int16_t*>(rf), out); break;
    }
    return last_launch_status();
}

extern "C" wf_status wf_iq_demod(const void* rf, wf_dtype dtype, float rf_scale, int64_t n_traces,
                                 int32_t n_samples, double f0, double fs, const float* taps,
                                 int32_t n_taps, int32_t decim, float* out_iq, wf_stream stream) {
    if (!rf || !out_iq || n_traces < 1 || n_samples < 1 || n_samples > WF_MAX_SAMPLES)
        return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (dtype == WF_I16 && !std::isfinite(rf_scale)) return WF_ERR_INVALID_ARG;
    if (decim < 1 || decim > kMaxDecim) return WF_ERR_INVALID_ARG;
    if (!std::isfinite(f0) || !(fs > 0.0) || !std::isfinite(fs)) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)rf & 3u) || ((uintptr_t)out_iq & 7u)) return WF_ERR_INVALID_ARG;
    thread_local FirArgs a;
    if (!fill_taps(a, taps, n_taps)) return WF_ERR_INVALID_ARG;
    a.ns = n_samples;
    a.n_traces = n_traces;
    a.decim = decim;
    a.scale = dtype == WF_I16 ? rf_scale : 1.0f;
    double r = std::fmod(f0 / fs, 1.0);
    if (r < 0.0) r += 1.0;
    a.turns = df_from_double(r);
    const int n_out = (n_samples + decim - 1) / decim;
    const size_t smem = sizeof(float2) * ((kIqThreads - 1) * (size_t)decim + n_taps + decim);   // phases padded
    dim3 grid((n_out + kIqThreads - 1) / kIqThreads, (unsigned)std::min<int64_t>(n_traces, 65535));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float2* o = reinterpret_cast<float2*>(out_iq);
    switch (dtype) {
        case WF_F32: iq_kernel<float><<<grid, kIqThreads, smem, st>>>(a, static_cast<const float*>(rf), o, n_out); break;
        case WF_F16: iq_kernel<__half><<<grid, kIqThreads, smem, st>>>(a, static_cast<const __half*>(rf), o, n_out); break;
        case WF_I16: iq_kernel<int16_t><<<grid, kIqThreads, smem, st>>>(a, static_cast<const int16_t*>(rf), o, n_out); break;
    }
    return last_launch_status();
}

// Windowed-sinc band-pass design (Hamming window), a host utility for wf_fir:
// h[n] = (2 f_hi sinc(2 f_hi (n - c)) - 2 f_lo sinc(2 f_lo (n - c))) w[n] with
// frequencies in cycles per sample; f_lo = 0 gives a low-pass.
extern "C" wf_status wf_fir_bandpass(double f_lo, double f_hi, double fs, int32_t n_taps,
                                     float* taps_out) {
    if (!taps_out || n_taps < 1 || n_taps > WF_MAX_TAPS || !(n_taps & 1)) return WF_ERR_INVALID_ARG;
    if (!(fs > 0.0) || !(f_lo >= 0.0) || !(f_hi > f_lo) || !(f_hi <= 0.5 * fs)) return WF_ERR_INVALID_ARG;
    const double a = f_lo / fs, b = f_hi / fs, c = 0.5 * (n_taps - 1);
    auto sinc = [](double v) { return v == 0.0 ? 1.0 : std::sin(M_PI * v) / (M_PI * v); };
    for (int n = 0; n < n_taps; ++n) {
        const double t = n - c;
        const double w = n_taps > 1 ? 0.54 - 0.46 * std::cos(2.0 * M_PI * n / (n_taps - 1)) : 1.0;
        taps_out[n] = (float)((2.0 * b * sinc(2.0 * b * t) - 2.0 * a * sinc(2.0 * a * t)) * w);
    }
    return WF_OK;
}
