// Delay-and-sum beamforming for STAI and PWI (paper Sec. II-B, Fig. 2 "Beamforming").
//
// b(p) = sum_t Wt(p,t) sum_r Wr(p,r) lerp(rf[t][r], Dt(p,t) + Dr(p,r))
//   STAI: Dt = |p - x_{e_t}| - t_start fs,   Wt = apod(p, e_t) g_{e_t}
//   PWI:  Dt = x sin th + z cos th - t0 fs,   Wt = 1
//   both: Dr = |p - x_r|,                     Wr = apod(p, r) g_r
// (all lengths in samples).  DAS is a gather-sum, not a contraction: no
// tensor cores.  Design (GB300):
//  * a CTA owns a 16 (z) x 32 (x) pixel tile and one slice of transmits; the
//    tile's aperture gives the range of elements that can contribute;
//  * receive elements are processed in chunks of 8 whose geometry (distance,
//    weight) lives in registers, transmit geometry of the slice sits in a
//    thread-private shared table; both are computed on the fly, never read
//    from global memory;
//  * for every (transmit, receive chunk) the sample window the tile can
//    touch is staged into shared memory as FP32 pairs (x[i], x[i+1]-x[i]),
//    so one 8-byte shared load and one FMA interpolate a sample;
//  * the floor of the fractional delay is taken with a round-down add of
//    1.5 * 2^23 (exact for |s| < 2^22), avoiding slow float->int converts;
//  * partial images of the transmit slices go to the workspace and a second
//    kernel sums them in slice order (deterministic; fills the GPU when the
//    frame has few tiles).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace wf {

constexpr int kTZ = 16;                 // tile rows (z)
constexpr int kTX = 32;                 // tile columns (x) = lanes
constexpr int kThreads = 256;           // 8 warps
constexpr int kP = kTZ / (kThreads / 32);  // pixels (rows) per thread
constexpr int kTilePix = kTZ * kTX;
constexpr int kC = 8;                   // receive elements per chunk
constexpr int kTS = 8;                  // transmits per slice
constexpr int kMaxWindow = 2048;        // staged positions per trace
constexpr float kMagic = 12582912.0f;   // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

struct TxInfo {
    float a, b, c;  // STAI: c = -t_start fs.  PWI: a = sin th, b = cos th, c = -t0 fs
    int e;          // STAI: element fired
};

struct DasArgs {
    Geom g;
    int n_tx, ns;
    int tiles_x, n_slices, n_items;  // items per frame = tiles * slices
    int W;                           // staged positions per trace (shared stride)
    const void* rf;
    float rf_scale;
    long long frame_elems;           // n_tx * E * ns
    float* part;                     // [batch][n_items][kTilePix]
    float* out;                      // direct kernel only
    WsHeader* hdr;
    TxInfo tx[WF_MAX_TX];
};

template <typename T> struct RF;
template <> struct RF<float> {
    static __device__ __forceinline__ float2 pair(const float* p, float) {
        float a = __ldg(p), b = __ldg(p + 1);
        return make_float2(a, b - a);
    }
    static __device__ __forceinline__ float one(const float* p, float) { return __ldg(p); }
};
template <> struct RF<__half> {
    static __device__ __forceinline__ float2 pair(const __half* p, float) {
        float a = __half2float(p[0]), b = __half2float(p[1]);
        return make_float2(a, b - a);
    }
    static __device__ __forceinline__ float one(const __half* p, float) { return __half2float(*p); }
};
template <> struct RF<int16_t> {
    static __device__ __forceinline__ float2 pair(const int16_t* p, float s) {
        int a = __ldg(p), b = __ldg(p + 1);
        return make_float2((float)a * s, (float)(b - a) * s);
    }
    static __device__ __forceinline__ float one(const int16_t* p, float s) { return (float)__ldg(p) * s; }
};

// Transmit-side delay and weight for a pixel.
template <int MODE>
__device__ __forceinline__ float2 tx_term(const Geom& g, const TxInfo& ti, float px, float pz,
                                          float z2, float kap) {
    if (MODE == 0) {
        float xe = elem_x(g, ti.e);
        float w = apod_weight(g.apod, xe, px, kap);
        if (g.elem_weight) w *= __ldg(g.elem_weight + ti.e);
        return make_float2(elem_dist(xe, px, z2) + ti.c, w);
    }
    return make_float2(fmaf(px, ti.a, fmaf(pz, ti.b, ti.c)), 1.0f);
}

// Receive-side weight (0 outside [0, E)).
__device__ __forceinline__ float rx_weight(const Geom& g, int r, float xe, float px, float kap) {
    if (r < 0 || r >= g.n_elements) return 0.0f;
    float w = apod_weight(g.apod, xe, px, kap);
    if (g.elem_weight) w *= __ldg(g.elem_weight + r);
    return w;
}

// Range [min, max] of the transmit term over the tile rectangle.
template <int MODE>
__device__ __forceinline__ float2 tx_bounds(const Geom& g, const TxInfo& ti, float xlo, float xhi,
                                            float zlo, float zhi) {
    if (MODE == 0) {
        float xe = elem_x(g, ti.e);
        float dxm = fmaxf(0.0f, fmaxf(xlo - xe, xe - xhi));
        float dfar = fmaxf(fabsf(xe - xlo), fabsf(xe - xhi));
        return make_float2(__fsqrt_rn(fmaf(dxm, dxm, zlo * zlo)) + ti.c,
                           __fsqrt_rn(fmaf(dfar, dfar, zhi * zhi)) + ti.c);
    }
    float v0 = fmaf(xlo, ti.a, fmaf(zlo, ti.b, ti.c));
    float v1 = fmaf(xhi, ti.a, fmaf(zlo, ti.b, ti.c));
    float v2 = fmaf(xlo, ti.a, fmaf(zhi, ti.b, ti.c));
    float v3 = fmaf(xhi, ti.a, fmaf(zhi, ti.b, ti.c));
    return make_float2(fminf(fminf(v0, v1), fminf(v2, v3)), fmaxf(fmaxf(v0, v1), fmaxf(v2, v3)));
}

// Range of the receive distance over the tile rectangle and elements [r0, r1].
__device__ __forceinline__ float2 rx_bounds(const Geom& g, int r0, int r1, float xlo, float xhi,
                                            float zlo, float zhi) {
    float xa = elem_x(g, r0), xb = elem_x(g, r1);
    float dxm = fmaxf(0.0f, fmaxf(xlo - xb, xa - xhi));
    float dfar = fmaxf(xb - xlo, xhi - xa);
    return make_float2(__fsqrt_rn(fmaf(dxm, dxm, zlo * zlo)), __fsqrt_rn(fmaf(dfar, dfar, zhi * zhi)));
}

__device__ __forceinline__ void flag(WsHeader* h, unsigned bit, unsigned a, unsigned b, unsigned c) {
    if (atomicOr(&h->flags, bit) == 0u) {
        h->first_bad[0] = a;
        h->first_bad[1] = b;
        h->first_bad[2] = c;
    }
}

// Element range that can be inside the aperture of some pixel of the tile.
__device__ __forceinline__ int2 tile_elements(const Geom& g, float xlo, float xhi, float zhi) {
    if (g.apod == WF_APOD_NONE) return make_int2(0, g.n_elements - 1);
    if (!(zhi > 0.0f)) return make_int2(1, 0);
    float half = zhi / g.two_f;
    int lo = (int)floorf((xlo - half - g.xe0) / g.pitch) - 1;
    int hi = (int)ceilf((xhi + half - g.xe0) / g.pitch) + 1;
    return make_int2(max(lo, 0), min(hi, g.n_elements - 1));
}

template <int MODE, typename T, bool CHECK>
__global__ void __launch_bounds__(kThreads, 2) das_tiled_kernel(const __grid_constant__ DasArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);                      // [kC][W]
    float2* ttab = buf + kC * a.W;                                           // [kTS][kP][kThreads]
    float2* tb = ttab + kTS * kP * kThreads;                                 // [kTS] tx bounds
    int* tlist = reinterpret_cast<int*>(tb + kTS);                           // [kTS]
    __shared__ int s_nact;

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.x, b = blockIdx.y;
    const int slice = item % a.n_slices, tile = item / a.n_slices;
    const int ix0 = (tile % a.tiles_x) * kTX, iz0 = (tile / a.tiles_x) * kTZ;
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;

    const float px = pixel_x(g, ix0 + lane);
    float pz[kP], z2[kP], kap[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        pz[p] = pixel_z(g, iz0 + warp * kP + p);
        z2[p] = pz[p] * pz[p];
        kap[p] = aperture_kappa(g, pz[p]);
    }
    const float xlo = pixel_x(g, ix0), xhi = pixel_x(g, ix0 + kTX - 1);
    const float zlo = pixel_z(g, iz0), zhi = pixel_z(g, iz0 + kTZ - 1);
    const int2 er = tile_elements(g, xlo, xhi, zhi);

    const int t_begin = slice * kTS, t_end = min(a.n_tx, t_begin + kTS);
    if (tid == 0) {
        int n = 0;
        for (int t = t_begin; t < t_end; ++t) {
            if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
            tlist[n++] = t;
        }
        s_nact = er.x <= er.y ? n : 0;
    }
    __syncthreads();
    const int n_act = s_nact;

    // Transmit geometry of the slice: per-thread table + per-transmit bounds.
    for (int j = 0; j < n_act; ++j) {
        const TxInfo ti = a.tx[tlist[j]];
#pragma unroll
        for (int p = 0; p < kP; ++p) ttab[(j * kP + p) * kThreads + tid] = tx_term<MODE>(g, ti, px, pz[p], z2[p], kap[p]);
        if (tid == j) tb[j] = tx_bounds<MODE>(g, ti, xlo, xhi, zlo, zhi);
    }
    __syncthreads();

    float acc[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) acc[p] = 0.0f;
    const int n_chunks = n_act > 0 ? (er.y - er.x + kC) / kC : 0;

    for (int k = 0; k < n_chunks; ++k) {
        const int r0 = er.x + k * kC;
        float Dr[kC][kP], Wr[kC][kP];
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            const float xe = elem_x(g, r0 + c);
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                Dr[c][p] = elem_dist(xe, px, z2[p]);
                Wr[c][p] = (r0 + c <= er.y) ? rx_weight(g, r0 + c, xe, px, kap[p]) : 0.0f;
            }
        }
        const float2 rb = rx_bounds(g, r0, min(r0 + kC - 1, g.n_elements - 1), xlo, xhi, zlo, zhi);

        for (int j = 0; j < n_act; ++j) {
            const int t = tlist[j];
            const float2 tbj = tb[j];
            const int lo = (int)floorf(tbj.x + rb.x) - 2;
            int len = (int)ceilf(tbj.y + rb.y) + 2 - lo + 1;
            if (lo + len <= 0 || lo > a.ns - 2) continue;  // window outside the record: adds 0
            if (len > a.W) {
                if (tid == 0) flag(a.hdr, 1u, (unsigned)blockIdx.x, (unsigned)len, (unsigned)a.W);
                len = a.W;
            }
            // Stage the window of the kC traces (t, r0..r0+kC-1) as FP32 pairs.
#pragma unroll 1
            for (int c = 0; c < kC; ++c) {
                const int r = r0 + c;
                float2* dst = buf + c * a.W;
                const T* tr = rf + ((long long)t * g.n_elements + r) * a.ns;
                const bool ok_r = r < g.n_elements;
                for (int q = tid; q < len; q += kThreads) {
                    const int n = lo + q;
                    float2 v = make_float2(0.0f, 0.0f);
                    if (ok_r && n >= 0 && n <= a.ns - 2) v = RF<T>::pair(tr + n, a.rf_scale);
                    dst[q] = v;
                }
            }
            __syncthreads();

            float2 tw[kP];
            float acct[kP];
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                tw[p] = ttab[(j * kP + p) * kThreads + tid];
                acct[p] = 0.0f;
            }
            const int base = kMagicBits + lo;
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                const float2* bc = buf + c * a.W;
#pragma unroll
                for (int p = 0; p < kP; ++p) {
                    const float s = tw[p].x + Dr[c][p];
                    const float m = __fadd_rd(s, kMagic);
                    const float f = s - (m - kMagic);
                    int idx = __float_as_int(m) - base;
                    if (CHECK && (idx < 0 || idx >= len)) {
                        flag(a.hdr, 2u, (unsigned)blockIdx.x, (unsigned)idx, (unsigned)len);
                        idx = 0;
                    }
                    const float2 ab = bc[idx];
                    acct[p] = fmaf(Wr[c][p], fmaf(f, ab.y, ab.x), acct[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < kP; ++p) acc[p] = fmaf(tw[p].y, acct[p], acc[p]);
            __syncthreads();
        }
    }

    float* dst = a.part + ((long long)b * a.n_items + item) * kTilePix;
#pragma unroll
    for (int p = 0; p < kP; ++p) dst[(warp * kP + p) * kTX + lane] = acc[p];
}

// Sum the transmit-slice partials of every pixel in slice order.
__global__ void das_reduce_kernel(const float* __restrict__ part, float* __restrict__ out, int nz,
                                  int nx, int tiles_x, int n_slices, int n_items) {
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= nx) return;
    const int tile = (iz / kTZ) * tiles_x + ix / kTX;
    const int local = (iz % kTZ) * kTX + (ix % kTX);
    const float* p = part + ((long long)b * n_items + (long long)tile * n_slices) * kTilePix + local;
    float s = 0.0f;
    for (int k = 0; k < n_slices; ++k) s += p[(long long)k * kTilePix];
    out[((long long)b * nz + iz) * nx + ix] = s;
}

// Direct per-pixel gather for geometries whose staging windows do not fit in
// shared memory (very coarse grids): same arithmetic, RF read through L1.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) das_direct_kernel(const __grid_constant__ DasArgs a) {
    const Geom& g = a.g;
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iz = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int b = blockIdx.z;
    if (ix >= g.nx || iz >= g.nz) return;
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;
    const float px = pixel_x(g, ix), pz = pixel_z(g, iz), z2 = pz * pz, kap = aperture_kappa(g, pz);
    const int2 er = tile_elements(g, px, px, pz);
    float acc = 0.0f;
    for (int t = 0; t < a.n_tx; ++t) {
        const float2 tw = tx_term<MODE>(g, a.tx[t], px, pz, z2, kap);
        if (tw.y == 0.0f) continue;
        float inner = 0.0f;
        for (int r = er.x; r <= er.y; ++r) {
            const float xe = elem_x(g, r);
            const float w = rx_weight(g, r, xe, px, kap);
            if (w == 0.0f) continue;
            const float s = tw.x + elem_dist(xe, px, z2);
            const float m = __fadd_rd(s, kMagic);
            const float f = s - (m - kMagic);
            const int i = __float_as_int(m) - kMagicBits;
            if (i < 0 || i > a.ns - 2) continue;
            const float2 ab = RF<T>::pair(rf + ((long long)t * g.n_elements + r) * a.ns + i, a.rf_scale);
            inner = fmaf(w, fmaf(f, ab.y, ab.x), inner);
        }
        acc = fmaf(tw.y, inner, acc);
    }
    a.out[((long long)b * g.nz + iz) * g.nx + ix] = acc;
}

// FP32 delays exactly as the DAS kernels form them (Dt + Dr).
template <int MODE>
__global__ void das_delays_kernel(const __grid_constant__ DasArgs a, const int32_t* __restrict__ pix,
                                  int n_pix, float* __restrict__ out) {
    const Geom& g = a.g;
    const long long n = (long long)n_pix * a.n_tx * g.n_elements;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i % g.n_elements);
        const int t = (int)((i / g.n_elements) % a.n_tx);
        const int q = (int)(i / ((long long)g.n_elements * a.n_tx));
        const int lin = pix[q];
        const float px = pixel_x(g, lin % g.nx), pz = pixel_z(g, lin / g.nx);
        const float z2 = pz * pz, kap = aperture_kappa(g, pz);
        const float2 tw = tx_term<MODE>(g, a.tx[t], px, pz, z2, kap);
        out[i] = tw.x + elem_dist(elem_x(g, r), px, z2);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

wf_status check_probe_grid(const wf_probe* p, const wf_grid* g) {
    if (!p || !g) return WF_ERR_INVALID_ARG;
    if (p->n_elements < 1 || p->n_elements > WF_MAX_ELEMENTS) return WF_ERR_INVALID_ARG;
    if (!finite_pos(p->pitch) || !finite_pos(p->fs) || !finite_pos(p->c)) return WF_ERR_INVALID_ARG;
    if (p->apod != WF_APOD_HANN && p->apod != WF_APOD_RECT && p->apod != WF_APOD_NONE)
        return WF_ERR_INVALID_ARG;
    if (p->apod != WF_APOD_NONE && !finite_pos(p->f_number)) return WF_ERR_INVALID_ARG;
    if (g->nz < 1 || g->nx < 1 || g->nz > 65535 || g->nx > (1 << 24)) return WF_ERR_INVALID_ARG;
    if (!std::isfinite(g->x_min) || !std::isfinite(g->x_max) || !std::isfinite(g->z_min) ||
        !std::isfinite(g->z_max))
        return WF_ERR_INVALID_ARG;
    if (g->x_max < g->x_min || g->z_max < g->z_min || g->z_min < 0.0) return WF_ERR_INVALID_ARG;
    return WF_OK;
}

Geom make_geom(const wf_probe* p, const wf_grid* g) {
    const double sc = p->fs / p->c;  // samples per metre
    Geom G;
    G.gx0 = (float)(g->x_min * sc);
    G.gdx = (float)(g->nx > 1 ? (g->x_max - g->x_min) / (g->nx - 1) * sc : 0.0);
    G.gz0 = (float)(g->z_min * sc);
    G.gdz = (float)(g->nz > 1 ? (g->z_max - g->z_min) / (g->nz - 1) * sc : 0.0);
    G.xe0 = (float)(-0.5 * (p->n_elements - 1) * p->pitch * sc);
    G.pitch = (float)(p->pitch * sc);
    G.two_f = (float)(2.0 * (p->apod == WF_APOD_NONE ? 1.0 : p->f_number));
    G.apod = p->apod;
    G.n_elements = p->n_elements;
    G.nz = g->nz;
    G.nx = g->nx;
    G.elem_weight = p->elem_weight;
    return G;
}

// Largest |delay| (samples) any pixel/element pair can produce, for the
// 2^22 range of the round-down floor.
double max_delay(const wf_probe* p, const wf_grid* g, double tx_extra) {
    const double sc = p->fs / p->c;
    const double half = 0.5 * (p->n_elements - 1) * p->pitch;
    const double dx = std::max(std::fabs(g->x_min), std::fabs(g->x_max)) + half;
    const double dz = std::max(std::fabs(g->z_min), std::fabs(g->z_max));
    return std::sqrt(dx * dx + dz * dz) * sc + tx_extra;
}

struct Plan {
    int tiles_x, tiles_z, n_slices, n_items;
    int W;
    bool tiled;
    size_t smem;
    size_t ws_bytes;
};

Plan make_plan(const wf_probe* p, const wf_grid* g, int batch, int n_tx) {
    const Geom G = make_geom(p, g);
    Plan P;
    P.tiles_x = (g->nx + kTX - 1) / kTX;
    P.tiles_z = (g->nz + kTZ - 1) / kTZ;
    P.n_slices = (n_tx + kTS - 1) / kTS;
    P.n_items = P.tiles_x * P.tiles_z * P.n_slices;
    // Lipschitz bound on one staging window: both distance terms move by at
    // most the tile diagonal, the receive term by (kC-1) pitches across the
    // chunk; plus floor/ceil and the +-2 margins.
    const double ex = (double)(kTX - 1) * G.gdx, ez = (double)(kTZ - 1) * G.gdz;
    const double diam = std::sqrt(ex * ex + ez * ez);
    const double w = 2.0 * diam + (kC - 1) * (double)G.pitch + 16.0;
    P.W = (int)std::ceil(w / 4.0) * 4;
    P.tiled = P.W <= kMaxWindow;
    P.smem = (size_t)kC * P.W * sizeof(float2) + (size_t)kTS * kP * kThreads * sizeof(float2) +
             kTS * sizeof(float2) + kTS * sizeof(int);
    P.ws_bytes = kWsHeaderBytes +
                 (P.tiled ? (size_t)batch * P.n_items * kTilePix * sizeof(float) : 0);
    return P;
}

constexpr size_t kMaxTiledSmem = (size_t)kC * kMaxWindow * sizeof(float2) +
                                  (size_t)kTS * kP * kThreads * sizeof(float2) +
                                  kTS * sizeof(float2) + kTS * sizeof(int);

bool check_bounds_mode() {
    const char* v = std::getenv("WF_CHECK_BOUNDS");
    return v && v[0] && v[0] != '0';
}

template <int MODE, typename T>
wf_status launch_das(DasArgs& A, const Plan& P, int batch, cudaStream_t st) {
    if (!P.tiled) {
        dim3 grid((A.g.nx + 31) / 32, (A.g.nz + 7) / 8, batch);
        das_direct_kernel<MODE, T><<<grid, 256, 0, st>>>(A);
        return last_launch_status();
    }
    static unsigned long long smem_set[2] = {0ull, 0ull};
    const bool chk = check_bounds_mode();
    auto kern = chk ? das_tiled_kernel<MODE, T, true> : das_tiled_kernel<MODE, T, false>;
    wf_status s = ensure_smem_limit(kern, kMaxTiledSmem, smem_set[chk ? 1 : 0]);
    if (s != WF_OK) return s;
    kern<<<dim3(P.n_items, batch), kThreads, P.smem, st>>>(A);
    if ((s = last_launch_status()) != WF_OK) return s;
    dim3 rg((A.g.nx + 127) / 128, A.g.nz, batch);
    das_reduce_kernel<<<rg, 128, 0, st>>>(A.part, A.out, A.g.nz, A.g.nx, P.tiles_x, P.n_slices,
                                          P.n_items);
    return last_launch_status();
}

template <int MODE>
wf_status dispatch(DasArgs& A, const Plan& P, int batch, wf_dtype dt, cudaStream_t st) {
    switch (dt) {
        case WF_F32: return launch_das<MODE, float>(A, P, batch, st);
        case WF_F16: return launch_das<MODE, __half>(A, P, batch, st);
        case WF_I16: return launch_das<MODE, int16_t>(A, P, batch, st);
    }
    return WF_ERR_INVALID_ARG;
}

wf_status das_common(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch,
                     int32_t n_tx, int32_t n_rx, int32_t n_samples, wf_dtype dtype,
                     const void* rf, float rf_scale, float* out, void* ws, size_t ws_bytes,
                     wf_stream stream, DasArgs& A) {
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (batch < 1 || batch > 65535) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    if (n_rx != probe->n_elements) return WF_ERR_INVALID_ARG;
    if (n_samples < 1 || n_samples > WF_MAX_SAMPLES) return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (dtype == WF_I16 && !std::isfinite(rf_scale)) return WF_ERR_INVALID_ARG;
    if (!rf || !out) return WF_ERR_INVALID_ARG;
    if (((uintptr_t)rf & 15u) || ((uintptr_t)out & 3u)) return WF_ERR_INVALID_ARG;
    const Plan P = make_plan(probe, grid, batch, n_tx);
    if ((long long)P.n_items > 0x7fffffffLL) return WF_ERR_UNSUPPORTED;
    if (!ws || ((uintptr_t)ws & 15u)) return WF_ERR_WORKSPACE;
    if (ws_bytes < P.ws_bytes) return WF_ERR_WORKSPACE;
    A.g = make_geom(probe, grid);
    A.n_tx = n_tx;
    A.ns = n_samples;
    A.tiles_x = P.tiles_x;
    A.n_slices = P.n_slices;
    A.n_items = P.n_items;
    A.W = P.W;
    A.rf = rf;
    A.rf_scale = dtype == WF_I16 ? rf_scale : 1.0f;
    A.frame_elems = (long long)n_tx * probe->n_elements * n_samples;
    A.hdr = static_cast<WsHeader*>(ws);
    A.part = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeaderBytes);
    A.out = out;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((s = cuda_status(cudaMemsetAsync(ws, 0, kWsHeaderBytes, st))) != WF_OK) return s;
    return mode == 0 ? dispatch<0>(A, P, batch, dtype, st) : dispatch<1>(A, P, batch, dtype, st);
}

}  // namespace
}  // namespace wf

using namespace wf;

extern "C" size_t wf_das_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                         int32_t n_tx) {
    if (check_probe_grid(probe, grid) != WF_OK || batch < 1 || n_tx < 1 || n_tx > WF_MAX_TX) return 0;
    return make_plan(probe, grid, batch, n_tx).ws_bytes;
}

extern "C" wf_status wf_das_stai(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                 int32_t n_tx, const int32_t* tx_elem, int32_t n_rx,
                                 int32_t n_samples, double t_start, wf_dtype dtype, const void* rf,
                                 float rf_scale, float* out, void* ws, size_t ws_bytes,
                                 wf_stream stream) {
    thread_local DasArgs local;  // ~4 KB parameter block, copied into the launch
    DasArgs& a = local;
    if (!probe || !std::isfinite(t_start)) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    const double t0 = t_start * probe->fs;
    for (int t = 0; t < n_tx; ++t) {
        const int e = tx_elem ? tx_elem[t] : t;
        if (e < 0 || e >= probe->n_elements) return WF_ERR_INVALID_ARG;
        a.tx[t] = TxInfo{0.0f, 0.0f, (float)(-t0), e};
    }
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (2.0 * max_delay(probe, grid, 0.0) + std::fabs(t0) >= 4194304.0) return WF_ERR_UNSUPPORTED;
    return das_common(0, probe, grid, batch, n_tx, n_rx, n_samples, dtype, rf, rf_scale, out, ws,
                      ws_bytes, stream, a);
}

extern "C" wf_status wf_das_pwi(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                int32_t n_angles, const double* angles_rad, const double* t_start,
                                int32_t n_rx, int32_t n_samples, wf_dtype dtype, const void* rf,
                                float rf_scale, float* out, void* ws, size_t ws_bytes,
                                wf_stream stream) {
    thread_local DasArgs local;
    DasArgs& a = local;
    if (!probe || !angles_rad) return WF_ERR_INVALID_ARG;
    if (n_angles < 1 || n_angles > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    double extra = 0.0;
    for (int k = 0; k < n_angles; ++k) {
        const double th = angles_rad[k], t0 = t_start ? t_start[k] : 0.0;
        if (!std::isfinite(th) || !std::isfinite(t0)) return WF_ERR_INVALID_ARG;
        a.tx[k] = TxInfo{(float)std::sin(th), (float)std::cos(th), (float)(-t0 * probe->fs), 0};
        extra = std::max(extra, std::fabs(t0 * probe->fs));
    }
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (2.0 * max_delay(probe, grid, 0.0) + extra >= 4194304.0) return WF_ERR_UNSUPPORTED;
    return das_common(1, probe, grid, batch, n_angles, n_rx, n_samples, dtype, rf, rf_scale, out,
                      ws, ws_bytes, stream, a);
}

extern "C" wf_status wf_das_delays(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                   int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                                   const double* t_start, int32_t n_pix, const int32_t* pix,
                                   float* out, wf_stream stream) {
    thread_local DasArgs local;
    DasArgs& a = local;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (mode != 0 && mode != 1) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX || n_pix < 0 || (n_pix > 0 && (!pix || !out)))
        return WF_ERR_INVALID_ARG;
    for (int t = 0; t < n_tx; ++t) {
        if (mode == 0) {
            const int e = tx_elem ? tx_elem[t] : t;
            if (e < 0 || e >= probe->n_elements) return WF_ERR_INVALID_ARG;
            const double t0 = t_start ? t_start[0] : 0.0;
            a.tx[t] = TxInfo{0.0f, 0.0f, (float)(-t0 * probe->fs), e};
        } else {
            if (!angles_rad) return WF_ERR_INVALID_ARG;
            const double th = angles_rad[t], t0 = t_start ? t_start[t] : 0.0;
            a.tx[t] = TxInfo{(float)std::sin(th), (float)std::cos(th), (float)(-t0 * probe->fs), 0};
        }
    }
    if (n_pix == 0) return WF_OK;
    a.g = make_geom(probe, grid);
    a.n_tx = n_tx;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (mode == 0) das_delays_kernel<0><<<304, 256, 0, st>>>(a, pix, n_pix, out);
    else das_delays_kernel<1><<<304, 256, 0, st>>>(a, pix, n_pix, out);
    return last_launch_status();
}

extern "C" wf_status wf_workspace_check(const void* ws, size_t ws_bytes, wf_stream stream) {
    if (!ws || ws_bytes < kWsHeaderBytes) return WF_ERR_WORKSPACE;
    WsHeader h;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return WF_ERR_CUDA;
    if (cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return WF_ERR_CUDA;
    return h.flags ? WF_ERR_INTERNAL : WF_OK;
}
