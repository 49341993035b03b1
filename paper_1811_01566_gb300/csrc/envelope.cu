// Envelope detection: |analytic signal| along depth (paper Fig. 2: analytic signal,
// then absolute value; Sec. II-B builds the Hilbert transform on the FFT).
//
// For a real column b of length N the analytic signal is b + i h with h the
// discrete Hilbert transform, h = IDFT(-i sgn(k) DFT(b)) (sgn = 0 at k = 0 and
// k = N/2).  This equals IDFT(H . DFT(b)) with H = 1, 2, ..., 2, 1, 0, ..., 0
// because H = 1 + sgn and IDFT(sgn . DFT(b)) = i h for real b.  Two real
// columns a, b travel through one complex FFT pair: with Y = DFT(a + i b),
// IDFT(-i sgn . Y) = h_a + i h_b (both transforms are real), so one forward and
// one inverse complex FFT of length N give the envelopes of two columns:
// env_a = sqrt(a^2 + h_a^2), env_b = sqrt(b^2 + h_b^2).
//
// Each CTA transforms kPairs column pairs with a radix-2 Stockham FFT in
// shared memory (twiddles from sincospif of exact arguments 2m/N); the
// epilogue fuses the magnitude and the per-frame maximum.
#include <cmath>

#include "common.cuh"

namespace wf {

constexpr int kEnvThreads = 256;

// One radix-2 Stockham pass over `cnt` independent length-N sequences laid
// out back to back (stride N): span ns, twiddle step N / (2 ns).
__device__ __forceinline__ void stockham_pass(const float2* __restrict__ in, float2* __restrict__ out,
                                              const float2* __restrict__ tw, int n, int log2n, int ns,
                                              int cnt, bool inverse) {
    const int half = n >> 1;
    const int total = half * cnt;
    const int tw_step = half / ns;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int seq = q >> (log2n - 1);
        const int j = q & (half - 1);
        const float2* src = in + seq * n;
        float2* dst = out + seq * n;
        const int k = j & (ns - 1);
        float2 w = tw[k * tw_step];
        if (inverse) w.y = -w.y;
        const float2 v0 = src[j];
        const float2 u = src[j + half];
        const float2 v1 = make_float2(u.x * w.x - u.y * w.y, u.x * w.y + u.y * w.x);
        const int d = ((j - k) << 1) + k;
        dst[d] = make_float2(v0.x + v1.x, v0.y + v1.y);
        dst[d + ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
}

__device__ __forceinline__ unsigned nonneg_bits(float v) {
    return (v == v && v > 0.0f) ? __float_as_uint(v) : 0u;  // NaN and zero contribute nothing
}

template <int PAIRS>
__global__ void __launch_bounds__(kEnvThreads) envelope_kernel(const float* __restrict__ bf,
                                                               float* __restrict__ env,
                                                               float* __restrict__ frame_max,
                                                               int nz, int log2n, int nx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = nz;
    float2* A = reinterpret_cast<float2*>(smem_raw);     // [PAIRS][n]
    float2* B = A + PAIRS * n;                            // [PAIRS][n]
    float2* tw = B + PAIRS * n;                           // [n/2]
    const int b = blockIdx.y;
    const int x0 = blockIdx.x * (2 * PAIRS);
    const float* src = bf + (long long)b * nz * nx;
    float* dst = env + (long long)b * nz * nx;

    for (int m = threadIdx.x; m < (n >> 1); m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)n, &s, &c);
        tw[m] = make_float2(c, -s);  // exp(-2 pi i m / n)
    }
    // Load: pair q holds columns x0 + 2q (real part) and x0 + 2q + 1 (imaginary part).
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int pr = q / n, z = q - pr * n;
        const int xa = x0 + 2 * pr;
        const float va = xa < nx ? src[(long long)z * nx + xa] : 0.0f;
        const float vb = xa + 1 < nx ? src[(long long)z * nx + xa + 1] : 0.0f;
        A[q] = make_float2(va, vb);
    }
    __syncthreads();

    float2* in = A;
    float2* out = B;
    for (int ns = 1; ns < n; ns <<= 1) {
        stockham_pass(in, out, tw, n, log2n, ns, PAIRS, false);
        __syncthreads();
        float2* t = in; in = out; out = t;
    }
    // Y = DFT(a + i b) is in `in`; form G = -i sgn(k) Y.
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int k = q & (n - 1);
        const float2 y = in[q];
        float2 gv;
        if (k == 0 || 2 * k == n) gv = make_float2(0.0f, 0.0f);
        else if (2 * k < n) gv = make_float2(y.y, -y.x);   // -i y
        else gv = make_float2(-y.y, y.x);                  // +i y
        in[q] = gv;
    }
    __syncthreads();
    for (int ns = 1; ns < n; ns <<= 1) {
        stockham_pass(in, out, tw, n, log2n, ns, PAIRS, true);
        __syncthreads();
        float2* t = in; in = out; out = t;
    }
    // in = n * (h_a + i h_b); magnitude epilogue with the original columns.
    const float inv_n = 1.0f / (float)n;
    unsigned mx = 0u;
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int pr = q / n, z = q - pr * n;
        const int xa = x0 + 2 * pr;
        const float2 h = in[q];
        if (xa < nx) {
            const float va = src[(long long)z * nx + xa];
            const float ha = h.x * inv_n;
            const float e = __fsqrt_rn(fmaf(va, va, ha * ha));
            dst[(long long)z * nx + xa] = e;
            mx = max(mx, nonneg_bits(e));
        }
        if (xa + 1 < nx) {
            const float vb = src[(long long)z * nx + xa + 1];
            const float hb = h.y * inv_n;
            const float e = __fsqrt_rn(fmaf(vb, vb, hb * hb));
            dst[(long long)z * nx + xa + 1] = e;
            mx = max(mx, nonneg_bits(e));
        }
    }
    if (frame_max) {
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0 && mx) atomicMax(reinterpret_cast<unsigned*>(frame_max + b), mx);
    }
}

// Reverse mode.  The analytic-signal map A = F^-1 diag(H) F is Hermitian (H is
// real), and for a real column Re(A r) = r and Im(A r) = Hilbert(r).  For a
// cotangent g_env of env = |z|, z = b + i Hilbert(b), the cotangent of z is
// g = g_env z / |z| (0 where |z| = 0) and that of the real column b is
// Re(A^H g) = Re(A g) = Re(g) - Hilbert(Im g).  Per column pair: one paired
// Hilbert transform rebuilds z, a second one transforms the imaginary parts.
template <int PAIRS>
__global__ void __launch_bounds__(kEnvThreads) envelope_backward_kernel(
    const float* bf, const float* grad_env, float* grad_bf, int nz, int log2n, int nx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = nz;
    float2* A = reinterpret_cast<float2*>(smem_raw);     // [PAIRS][n]
    float2* B = A + PAIRS * n;                            // [PAIRS][n]
    float2* R = B + PAIRS * n;                            // [PAIRS][n] real parts of g
    float2* tw = R + PAIRS * n;                           // [n/2]
    const int b = blockIdx.y;
    const int x0 = blockIdx.x * (2 * PAIRS);
    const long long fo = (long long)b * nz * nx;
    const float* src = bf + fo;

    for (int m = threadIdx.x; m < (n >> 1); m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)n, &s, &c);
        tw[m] = make_float2(c, -s);
    }
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int pr = q / n, z = q - pr * n;
        const int xa = x0 + 2 * pr;
        const float va = xa < nx ? src[(long long)z * nx + xa] : 0.0f;
        const float vb = xa + 1 < nx ? src[(long long)z * nx + xa + 1] : 0.0f;
        A[q] = make_float2(va, vb);
    }
    __syncthreads();
    // Paired Hilbert transform of the sequences in `buf` (result n * (h_a + i h_b) in the
    // returned buffer).
    auto hilbert = [&](float2* in, float2* out) {
        for (int ns = 1; ns < n; ns <<= 1) {
            stockham_pass(in, out, tw, n, log2n, ns, PAIRS, false);
            __syncthreads();
            float2* t = in; in = out; out = t;
        }
        for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
            const int k = q & (n - 1);
            const float2 y = in[q];
            float2 gv;
            if (k == 0 || 2 * k == n) gv = make_float2(0.0f, 0.0f);
            else if (2 * k < n) gv = make_float2(y.y, -y.x);
            else gv = make_float2(-y.y, y.x);
            in[q] = gv;
        }
        __syncthreads();
        for (int ns = 1; ns < n; ns <<= 1) {
            stockham_pass(in, out, tw, n, log2n, ns, PAIRS, true);
            __syncthreads();
            float2* t = in; in = out; out = t;
        }
        return in;
    };
    float2* h = hilbert(A, B);
    float2* other = h == A ? B : A;
    const float inv_n = 1.0f / (float)n;
    // g = g_env z / |z|: real parts to R, imaginary parts (the next transform's input) to `other`.
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int pr = q / n, z = q - pr * n;
        const int xa = x0 + 2 * pr;
        float2 re = make_float2(0.0f, 0.0f), im = make_float2(0.0f, 0.0f);
        const float2 hv = h[q];
        if (xa < nx) {
            const float va = src[(long long)z * nx + xa], ha = hv.x * inv_n;
            const float e = __fsqrt_rn(fmaf(va, va, ha * ha));
            const float g = grad_env[fo + (long long)z * nx + xa];
            if (e > 0.0f) {
                const float ge = g / e;
                re.x = ge * va;
                im.x = ge * ha;
            }
        }
        if (xa + 1 < nx) {
            const float vb = src[(long long)z * nx + xa + 1], hb = hv.y * inv_n;
            const float e = __fsqrt_rn(fmaf(vb, vb, hb * hb));
            const float g = grad_env[fo + (long long)z * nx + xa + 1];
            if (e > 0.0f) {
                const float ge = g / e;
                re.y = ge * vb;
                im.y = ge * hb;
            }
        }
        R[q] = re;
        other[q] = im;
    }
    __syncthreads();
    h = hilbert(other, h);
    for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
        const int pr = q / n, z = q - pr * n;
        const int xa = x0 + 2 * pr;
        const float2 hv = h[q], re = R[q];
        if (xa < nx) grad_bf[fo + (long long)z * nx + xa] = re.x - hv.x * inv_n;
        if (xa + 1 < nx) grad_bf[fo + (long long)z * nx + xa + 1] = re.y - hv.y * inv_n;
    }
}

}  // namespace wf

using namespace wf;

extern "C" wf_status wf_envelope(const float* bf, int32_t batch, int32_t nz, int32_t nx, float* env,
                                 float* frame_max, wf_stream stream) {
    if (!bf || !env || batch < 1 || batch > 65535 || nx < 1 || nz < 2 || nz > 4096)
        return WF_ERR_INVALID_ARG;
    if (nz & (nz - 1)) return WF_ERR_INVALID_ARG;
    if (bf == env) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)bf & 3u) || ((uintptr_t)env & 3u) || ((uintptr_t)frame_max & 3u))
        return WF_ERR_INVALID_ARG;
    int log2n = 0;
    while ((1 << log2n) < nz) ++log2n;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (frame_max) {
        wf_status s = cuda_status(cudaMemsetAsync(frame_max, 0, sizeof(float) * batch, st));
        if (s != WF_OK) return s;
    }
    constexpr int kPairs = 1;
    const size_t smem = sizeof(float2) * (2 * kPairs * (size_t)nz + nz / 2);
    static unsigned long long smem_set = 0ull;
    const size_t smem_max = sizeof(float2) * (2 * kPairs * 4096 + 2048);
    wf_status s = ensure_smem_limit(envelope_kernel<kPairs>, smem_max, smem_set);
    if (s != WF_OK) return s;
    dim3 grid((nx + 2 * kPairs - 1) / (2 * kPairs), batch);
    envelope_kernel<kPairs><<<grid, kEnvThreads, smem, st>>>(bf, env, frame_max, nz, log2n, nx);
    return last_launch_status();
}

extern "C" wf_status wf_envelope_backward(const float* bf, int32_t batch, int32_t nz, int32_t nx,
                                          const float* grad_env, float* grad_bf, wf_stream stream) {
    if (!bf || !grad_env || !grad_bf || batch < 1 || batch > 65535 || nx < 1 || nz < 2 || nz > 4096)
        return WF_ERR_INVALID_ARG;
    if (nz & (nz - 1)) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)bf & 3u) || ((uintptr_t)grad_env & 3u) || ((uintptr_t)grad_bf & 3u))
        return WF_ERR_INVALID_ARG;
    int log2n = 0;
    while ((1 << log2n) < nz) ++log2n;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    constexpr int kPairs = 1;
    const size_t smem = sizeof(float2) * (3 * kPairs * (size_t)nz + nz / 2);
    static unsigned long long smem_set = 0ull;
    const size_t smem_max = sizeof(float2) * (3 * kPairs * 4096 + 2048);
    wf_status s = ensure_smem_limit(envelope_backward_kernel<kPairs>, smem_max, smem_set);
    if (s != WF_OK) return s;
    dim3 grid((nx + 2 * kPairs - 1) / (2 * kPairs), batch);
    envelope_backward_kernel<kPairs><<<grid, kEnvThreads, smem, st>>>(bf, grad_env, grad_bf, nz, log2n, nx);
    return last_launch_status();
}
