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
// The forward kernel transforms one to four column pairs per CTA (four pairs:
// eight adjacent columns, each row of the block one 32-byte sector) with radix-4
// Stockham passes in shared memory (one radix-2 pass first when log2 N is odd;
// the formulation of Govindaraju et al., "High performance discrete Fourier
// transforms on graphics processors", SC 2008); twiddles from sincospif of
// exact arguments 2m/N; the epilogue fuses the magnitude and the per-frame
// maximum.  The reverse kernel takes one column pair per CTA with the same passes.
#include <algorithm>
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

// One radix-4 Stockham pass over `cnt` length-N sequences back to back (stride
// N): span ns, twiddles tw[m] = exp(-2 pi i m / N) for m < 3N/4, conjugated for
// the inverse.  Input j + r N/4 (r = 0..3) of a sequence is multiplied by
// w^r, w = exp(-+2 pi i (j mod ns) / (4 ns)), the four go through a DFT of
// length 4 and land at 4 (j - j mod ns) + (j mod ns) + r ns.
__device__ __forceinline__ void stockham_pass4(const float2* __restrict__ in, float2* __restrict__ out,
                                               const float2* __restrict__ tw, int n, int log2n, int ns,
                                               int cnt, bool inverse) {
    const int quarter = n >> 2;
    const int total = quarter * cnt;
    const int tw_step = quarter / ns;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int seq = q >> (log2n - 2);
        const int j = q & (quarter - 1);
        const float2* src = in + seq * n;
        float2* dst = out + seq * n;
        const int k = j & (ns - 1);
        const int m = k * tw_step;
        float2 w1 = tw[m], w2 = tw[2 * m], w3 = tw[3 * m];
        if (inverse) {
            w1.y = -w1.y;
            w2.y = -w2.y;
            w3.y = -w3.y;
        }
        const float2 v0 = src[j];
        const float2 u1 = src[j + quarter], u2 = src[j + 2 * quarter], u3 = src[j + 3 * quarter];
        const float2 v1 = make_float2(u1.x * w1.x - u1.y * w1.y, u1.x * w1.y + u1.y * w1.x);
        const float2 v2 = make_float2(u2.x * w2.x - u2.y * w2.y, u2.x * w2.y + u2.y * w2.x);
        const float2 v3 = make_float2(u3.x * w3.x - u3.y * w3.y, u3.x * w3.y + u3.y * w3.x);
        const float2 a0 = make_float2(v0.x + v2.x, v0.y + v2.y), a1 = make_float2(v0.x - v2.x, v0.y - v2.y);
        const float2 a2 = make_float2(v1.x + v3.x, v1.y + v3.y), a3 = make_float2(v1.x - v3.x, v1.y - v3.y);
        // -i a3 (forward) or +i a3 (inverse)
        const float2 ja3 = inverse ? make_float2(-a3.y, a3.x) : make_float2(a3.y, -a3.x);
        const int d = ((j - k) << 2) + k;
        dst[d] = make_float2(a0.x + a2.x, a0.y + a2.y);
        dst[d + ns] = make_float2(a1.x + ja3.x, a1.y + ja3.y);
        dst[d + 2 * ns] = make_float2(a0.x - a2.x, a0.y - a2.y);
        dst[d + 3 * ns] = make_float2(a1.x - ja3.x, a1.y - ja3.y);
    }
}

// Full Stockham FFT of `cnt` sequences: a radix-2 pass when log2 n is odd, then radix-4
// passes.  Returns the buffer holding the result (in or out).
__device__ __forceinline__ float2* stockham_fft(float2* in, float2* out, const float2* tw, int n,
                                                int log2n, int cnt, bool inverse) {
    int ns = 1;
    if (log2n & 1) {
        stockham_pass(in, out, tw, n, log2n, ns, cnt, inverse);
        __syncthreads();
        float2* t = in; in = out; out = t;
        ns = 2;
    }
    for (; ns < n; ns <<= 2) {
        stockham_pass4(in, out, tw, n, log2n, ns, cnt, inverse);
        __syncthreads();
        float2* t = in; in = out; out = t;
    }
    return in;
}

__device__ __forceinline__ unsigned nonneg_bits(float v) {
    return (v == v && v > 0.0f) ? __float_as_uint(v) : 0u;  // NaN and zero contribute nothing
}

constexpr int kEnvFwdThreads = 512;
constexpr int kEnvUnroll = 4;

// Forward envelope of `pairs` column pairs (2 * pairs adjacent columns) per CTA.  With `db`
// set the epilogue also writes the log-clipped value against the caller's reference ref[b]
// (env may then be null).
__global__ void __launch_bounds__(kEnvFwdThreads) envelope_kernel(const float* __restrict__ bf,
                                                                  float* __restrict__ env,
                                                                  float* __restrict__ frame_max, int nz,
                                                                  int log2n, int nx, int pairs,
                                                                  const float* __restrict__ ref, float lo,
                                                                  float hi, float* __restrict__ db) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = nz;
    float2* A = reinterpret_cast<float2*>(smem_raw);     // [pairs][n]
    float2* B = A + pairs * n;                            // [pairs][n]
    float2* tw = B + pairs * n;                           // [3n/4] (n/2 for n = 2)
    const int b = blockIdx.y;
    const int cols = 2 * pairs, lc = 31 - __clz(cols);    // columns per CTA (a power of two)
    const int x0 = blockIdx.x * cols;
    const float* src = bf + (long long)b * nz * nx;
    float* dst = env ? env + (long long)b * nz * nx : nullptr;
    float* dbo = db ? db + (long long)b * nz * nx : nullptr;
    const float rb = db ? __ldg(ref + b) : 0.0f;

    const int ntw = n >= 4 ? 3 * (n >> 2) : (n >> 1);
    for (int m = threadIdx.x; m < ntw; m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)n, &s, &c);
        tw[m] = make_float2(c, -s);  // exp(-2 pi i m / n)
    }
    // Load: element q is row z = q / cols, column x0 + (q mod cols): adjacent threads read adjacent
    // columns of a row.  Pair p holds columns x0 + 2p (real part) and x0 + 2p + 1 (imaginary part).
    // kEnvUnroll loads per thread are issued before any is stored, so a small CTA keeps
    // several global reads in flight instead of waiting out each one in turn.
    float* Af = reinterpret_cast<float*>(A);
    const int total = cols * n;
    for (int q0 = threadIdx.x; q0 < total; q0 += kEnvUnroll * blockDim.x) {
        float v[kEnvUnroll];
#pragma unroll
        for (int u = 0; u < kEnvUnroll; ++u) {
            const int q = q0 + u * blockDim.x;
            const int z = q >> lc, x = x0 + (q & (cols - 1));
            v[u] = (q < total && x < nx) ? src[(long long)z * nx + x] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kEnvUnroll; ++u) {
            const int q = q0 + u * blockDim.x;
            const int z = q >> lc, c = q & (cols - 1);
            if (q < total) Af[2 * ((c >> 1) * n + z) + (c & 1)] = v[u];
        }
    }
    __syncthreads();
    float2* y = stockham_fft(A, B, tw, n, log2n, pairs, false);
    float2* other = y == A ? B : A;
    // Y = DFT(a + i b); form G = -i sgn(k) Y.
    for (int q = threadIdx.x; q < pairs * n; q += blockDim.x) {
        const int k = q & (n - 1);
        const float2 v = y[q];
        float2 gv;
        if (k == 0 || 2 * k == n) gv = make_float2(0.0f, 0.0f);
        else if (2 * k < n) gv = make_float2(v.y, -v.x);   // -i y
        else gv = make_float2(-v.y, v.x);                  // +i y
        y[q] = gv;
    }
    __syncthreads();
    const float2* h = stockham_fft(y, other, tw, n, log2n, pairs, true);
    // h = n (h_a + i h_b); magnitude epilogue with the original columns, row-major as the load.
    const float inv_n = 1.0f / (float)n;
    const float* hf = reinterpret_cast<const float*>(h);
    unsigned mx = 0u;
    for (int q0 = threadIdx.x; q0 < total; q0 += kEnvUnroll * blockDim.x) {
        float v[kEnvUnroll];
#pragma unroll
        for (int u = 0; u < kEnvUnroll; ++u) {
            const int q = q0 + u * blockDim.x;
            const int z = q >> lc, x = x0 + (q & (cols - 1));
            v[u] = (q < total && x < nx) ? src[(long long)z * nx + x] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kEnvUnroll; ++u) {
            const int q = q0 + u * blockDim.x;
            const int z = q >> lc, c = q & (cols - 1);
            const int x = x0 + c;
            if (q < total && x < nx) {
                const float hv = hf[2 * ((c >> 1) * n + z) + (c & 1)] * inv_n;
                const float e = __fsqrt_rn(fmaf(v[u], v[u], hv * hv));
                if (dst) dst[(long long)z * nx + x] = e;
                if (dbo) dbo[(long long)z * nx + x] = db_value(e, rb, lo, hi);
                mx = max(mx, nonneg_bits(e));
            }
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
    float2* tw = R + PAIRS * n;                           // [3n/4] (n/2 for n = 2)
    const int b = blockIdx.y;
    const int x0 = blockIdx.x * (2 * PAIRS);
    const long long fo = (long long)b * nz * nx;
    const float* src = bf + fo;

    const int ntw = n >= 4 ? 3 * (n >> 2) : (n >> 1);
    for (int m = threadIdx.x; m < ntw; m += blockDim.x) {
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
        float2* y = stockham_fft(in, out, tw, n, log2n, PAIRS, false);
        float2* o = y == in ? out : in;
        for (int q = threadIdx.x; q < PAIRS * n; q += blockDim.x) {
            const int k = q & (n - 1);
            const float2 v = y[q];
            float2 gv;
            if (k == 0 || 2 * k == n) gv = make_float2(0.0f, 0.0f);
            else if (2 * k < n) gv = make_float2(v.y, -v.x);
            else gv = make_float2(-v.y, v.x);
            y[q] = gv;
        }
        __syncthreads();
        return stockham_fft(y, o, tw, n, log2n, PAIRS, true);
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

namespace {

// Forward launch shared by wf_envelope and wf_envelope_logclip (db set: fused log-clip).
wf_status envelope_forward(const float* bf, int32_t batch, int32_t nz, int32_t nx, float* env,
                           float* frame_max, const float* ref, float lo, float hi, float* db,
                           wf_stream stream) {
    if (!bf || !(env || db) || batch < 1 || batch > 65535 || nx < 1 || nz < 2 || nz > 4096)
        return WF_ERR_INVALID_ARG;
    if (nz & (nz - 1)) return WF_ERR_INVALID_ARG;
    if (bf == env || bf == db) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)bf & 3u) || ((uintptr_t)env & 3u) || ((uintptr_t)frame_max & 3u) || ((uintptr_t)db & 3u))
        return WF_ERR_INVALID_ARG;
    int log2n = 0;
    while ((1 << log2n) < nz) ++log2n;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (frame_max) {
        wf_status s = cuda_status(cudaMemsetAsync(frame_max, 0, sizeof(float) * batch, st));
        if (s != WF_OK) return s;
    }
    // Column pairs per CTA: as many as keep at least ~600 CTAs in flight (four SM-fulls of
    // 152 SMs), up to four (eight adjacent columns: one 32-byte sector per row), two at
    // nz = 4096 (shared memory); one thread per radix-4 butterfly of a pass, at least 256
    // threads (the loads and the epilogue run on all of them).
    const long long col_pairs = (long long)batch * ((nx + 1) / 2);
    int pairs = 1;
    while (pairs < (nz <= 2048 ? 4 : 2) && col_pairs / (2 * pairs) >= 600) pairs *= 2;
    const int threads = (int)std::min<long long>(kEnvFwdThreads, std::max<long long>(256, (long long)pairs * nz / 4));
    const size_t smem = sizeof(float2) * (2 * (size_t)pairs * nz + (nz >= 4 ? 3 * (nz / 4) : nz / 2));
    static unsigned long long smem_set = 0ull;
    const size_t smem_max = sizeof(float2) * (2 * 2 * 4096 + 3 * 1024);
    wf_status s = ensure_smem_limit(envelope_kernel, smem_max, smem_set);
    if (s != WF_OK) return s;
    dim3 grid((nx + 2 * pairs - 1) / (2 * pairs), batch);
    envelope_kernel<<<grid, threads, smem, st>>>(bf, env, frame_max, nz, log2n, nx, pairs, ref, lo, hi, db);
    return last_launch_status();
}

}  // namespace

extern "C" wf_status wf_envelope(const float* bf, int32_t batch, int32_t nz, int32_t nx, float* env,
                                 float* frame_max, wf_stream stream) {
    if (!env) return WF_ERR_INVALID_ARG;
    return envelope_forward(bf, batch, nz, nx, env, frame_max, nullptr, 0.0f, 0.0f, nullptr, stream);
}

extern "C" wf_status wf_envelope_logclip(const float* bf, int32_t batch, int32_t nz, int32_t nx,
                                         const float* ref, float db_min, float db_max, float* env,
                                         float* out_db, float* frame_max, wf_stream stream) {
    if (!ref || !out_db || !(db_min <= db_max)) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)ref & 3u) || (env && env == out_db)) return WF_ERR_INVALID_ARG;
    return envelope_forward(bf, batch, nz, nx, env, frame_max, ref, db_min, db_max, out_db, stream);
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
    const size_t smem = sizeof(float2) * (3 * kPairs * (size_t)nz + (nz >= 4 ? 3 * (nz / 4) : nz / 2));
    static unsigned long long smem_set = 0ull;
    const size_t smem_max = sizeof(float2) * (3 * kPairs * 4096 + 3 * 1024);
    wf_status s = ensure_smem_limit(envelope_backward_kernel<kPairs>, smem_max, smem_set);
    if (s != WF_OK) return s;
    dim3 grid((nx + 2 * kPairs - 1) / (2 * kPairs), batch);
    envelope_backward_kernel<kPairs><<<grid, kEnvThreads, smem, st>>>(bf, grad_env, grad_bf, nz, log2n, nx);
    return last_launch_status();
}
