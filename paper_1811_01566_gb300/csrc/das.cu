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
//  * geometry is tile-relative: each CTA takes its tile origin c as reference
//    and, per element, the exact distance R_e = |c - x_e| in FP64; a pixel at
//    c + u then needs only the small FP32 correction
//      delta = |c + u - x_e| - R_e = N / (R_e + |c + u - x_e|),
//      N = u_x (2 (c_x - x_e) + u_x) + u_z (2 c_z + u_z),
//    and every fractional delay is formed relative to its staging window, so
//    FP32 carries a few hundred samples of range instead of thousands (delay
//    error ~3e-5 samples instead of ~2e-4);
//  * receive elements are processed in chunks of 8 whose corrections and
//    weights live in registers; transmit corrections of the slice sit in a
//    thread-private shared table; nothing geometric is read from global memory;
//  * for every (transmit, receive chunk) the sample window the tile can touch
//    is staged into shared memory as FP32 pairs (x[i], x[i+1]-x[i]), so one
//    8-byte shared load and one FMA interpolate a sample;
//  * the floor of the window-relative delay is a round-down add of 1.5 * 2^23;
//  * partial images of the transmit slices go to the workspace and a second
//    kernel sums them in slice order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "common.cuh"

namespace wf {

constexpr int kTZ = 16;                    // tile rows (z)
constexpr int kTX = 32;                    // tile columns (x) = lanes
constexpr int kThreads = 256;              // 8 warps
constexpr int kP = kTZ / (kThreads / 32);  // pixels (rows) per thread
constexpr int kTilePix = kTZ * kTX;
constexpr int kC = 8;                      // receive elements per chunk
constexpr int kTS = 8;                     // transmits per slice
constexpr int kMaxWindow = 2048;           // staged positions per trace
constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

struct TxInfo {
    double sin_d, cos_d, t0_d;  // PWI: steering; both: t0 = time of sample 0 times fs
    float sin_f, cos_f;
    int e;                      // STAI: element fired
    int pad;
};

// Sample-unit geometry in double (reference terms) next to the float copy in Geom.
struct GeomD {
    double gx0, gdx, gz0, gdz, xe0, pitch;
};

struct DasArgs {
    Geom g;
    GeomD gd;
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
};
template <> struct RF<__half> {
    static __device__ __forceinline__ float2 pair(const __half* p, float) {
        float a = __half2float(p[0]), b = __half2float(p[1]);
        return make_float2(a, b - a);
    }
};
template <> struct RF<int16_t> {
    static __device__ __forceinline__ float2 pair(const int16_t* p, float s) {
        int a = __ldg(p), b = __ldg(p + 1);
        return make_float2((float)a * s, (float)(b - a) * s);
    }
};

// Hann window 0.5 (1 + cos(pi u)) for |u| < 1, as the Taylor series of the
// cosine in v = u^2 through u^18 (truncation < 2e-9 on |u| <= 1).
__device__ __forceinline__ float hann_poly(float u) {
    const float v = u * u;
    float w = -6.93947623110688e-08f;
    w = fmaf(w, v, 2.151534793516472e-06f);
    w = fmaf(w, v, -5.2319052462422825e-05f);
    w = fmaf(w, v, 0.000964787154701961f);
    w = fmaf(w, v, -0.012903445695007025f);
    w = fmaf(w, v, 0.11766531517944656f);
    w = fmaf(w, v, -0.6676313844272946f);
    w = fmaf(w, v, 2.029356063208384f);
    w = fmaf(w, v, -2.4674011002723395f);
    return fmaf(w, v, 1.0f);
}

// Apodization weight given the lateral offset xe - x and kap = 2F / z.
__device__ __forceinline__ float apod_w(int apod, float dxe, float kap) {
    if (apod == WF_APOD_NONE) return 1.0f;
    const float u = dxe * kap;
    if (!(kap > 0.0f) || !(fabsf(u) < 1.0f)) return 0.0f;
    return apod == WF_APOD_RECT ? 1.0f : hann_poly(u);
}

// Per-element reference data of a tile (shared memory).
struct Elem {
    double R;   // |c - x_e|, samples, FP64
    float ax;   // c_x - x_e
    float Rf;   // (float) R
    float g;    // per-element weight
    float pad;
};

// Exact-to-FP64 distance from the reference point to element e.
__device__ __forceinline__ Elem make_elem(const DasArgs& a, double cx, double cz, int e) {
    const double xe = fma((double)e, a.gd.pitch, a.gd.xe0);
    const double ax = cx - xe;
    const double r2 = fma(ax, ax, cz * cz);
    const float rf = sqrtf((float)r2);
    // one Newton step on top of the FP32 root: error ~1e-14 relative
    const double R = (double)rf + (double)((float)fma(-(double)rf, (double)rf, r2) * (0.5f / rf));
    Elem el;
    el.R = r2 > 0.0 ? R : 0.0;
    el.ax = (float)ax;
    el.Rf = (float)el.R;
    el.g = a.g.elem_weight ? __ldg(a.g.elem_weight + e) : 1.0f;
    el.pad = 0.0f;
    return el;
}

// FP32 correction |c + u - x_e| - R_e for a pixel at offset (ux, uz); kz = uz (2 cz + uz).
__device__ __forceinline__ float dist_delta(const Elem& el, float ux, float kz) {
    const float n = fmaf(ux, 2.0f * el.ax + ux, kz);
    const float t = fmaf(el.Rf, el.Rf, n);
    const float d = t > 0.0f ? t * rsqrtf(t) : 0.0f;
    const float den = el.Rf + d;
    return den > 0.0f ? __fdividef(n, den) : 0.0f;
}

// Element range that can be inside the aperture of some pixel of the tile.
__device__ __forceinline__ int2 tile_elements(const Geom& g, float xlo, float xhi, float zhi) {
    if (g.apod == WF_APOD_NONE) return make_int2(0, g.n_elements - 1);
    if (!(zhi > 0.0f)) return make_int2(1, 0);
    const float half = zhi / g.two_f;
    const int lo = (int)floorf((xlo - half - g.xe0) / g.pitch) - 1;
    const int hi = (int)ceilf((xhi + half - g.xe0) / g.pitch) + 1;
    return make_int2(max(lo, 0), min(hi, g.n_elements - 1));
}

// Range [min, max] of the transmit term over the tile rectangle (FP32, for windows).
template <int MODE>
__device__ __forceinline__ float2 tx_bounds(const Geom& g, const TxInfo& ti, float xlo, float xhi,
                                            float zlo, float zhi) {
    const float c = (float)(-ti.t0_d);
    if (MODE == 0) {
        const float xe = elem_x(g, ti.e);
        const float dxm = fmaxf(0.0f, fmaxf(xlo - xe, xe - xhi));
        const float dfar = fmaxf(fabsf(xe - xlo), fabsf(xe - xhi));
        return make_float2(__fsqrt_rn(fmaf(dxm, dxm, zlo * zlo)) + c,
                           __fsqrt_rn(fmaf(dfar, dfar, zhi * zhi)) + c);
    }
    const float v0 = fmaf(xlo, ti.sin_f, fmaf(zlo, ti.cos_f, c));
    const float v1 = fmaf(xhi, ti.sin_f, fmaf(zlo, ti.cos_f, c));
    const float v2 = fmaf(xlo, ti.sin_f, fmaf(zhi, ti.cos_f, c));
    const float v3 = fmaf(xhi, ti.sin_f, fmaf(zhi, ti.cos_f, c));
    return make_float2(fminf(fminf(v0, v1), fminf(v2, v3)), fmaxf(fmaxf(v0, v1), fmaxf(v2, v3)));
}

// Range of the receive distance over the tile rectangle and elements [r0, r1].
__device__ __forceinline__ float2 rx_bounds(const Geom& g, int r0, int r1, float xlo, float xhi,
                                            float zlo, float zhi) {
    const float xa = elem_x(g, r0), xb = elem_x(g, r1);
    const float dxm = fmaxf(0.0f, fmaxf(xlo - xb, xa - xhi));
    const float dfar = fmaxf(xb - xlo, xhi - xa);
    return make_float2(__fsqrt_rn(fmaf(dxm, dxm, zlo * zlo)), __fsqrt_rn(fmaf(dfar, dfar, zhi * zhi)));
}

// Transmit reference term (FP64).
template <int MODE>
__device__ __forceinline__ double tx_ref(const TxInfo& ti, double cx, double cz, double R_et) {
    if (MODE == 0) return R_et - ti.t0_d;
    return fma(cx, ti.sin_d, fma(cz, ti.cos_d, -ti.t0_d));
}

__device__ __forceinline__ void flag(WsHeader* h, unsigned bit, unsigned a, unsigned b, unsigned c) {
    if (atomicOr(&h->flags, bit) == 0u) {
        h->first_bad[0] = a;
        h->first_bad[1] = b;
        h->first_bad[2] = c;
    }
}

// Tile geometry shared by the DAS kernel and the delay probe.
struct TileGeo {
    int ix0, iz0;
    double cx, cz;            // reference point = tile origin pixel (FP64 samples)
    float xlo, xhi, zlo, zhi; // tile rectangle (FP32 samples)
    int2 er;                  // element range
};

__device__ __forceinline__ TileGeo tile_geo(const DasArgs& a, int ix0, int iz0) {
    const Geom& g = a.g;
    TileGeo t;
    t.ix0 = ix0;
    t.iz0 = iz0;
    t.cx = fma((double)ix0, a.gd.gdx, a.gd.gx0);
    t.cz = fma((double)iz0, a.gd.gdz, a.gd.gz0);
    t.xlo = pixel_x(g, ix0);
    t.xhi = pixel_x(g, ix0 + kTX - 1);
    t.zlo = pixel_z(g, iz0);
    t.zhi = pixel_z(g, iz0 + kTZ - 1);
    t.er = tile_elements(g, t.xlo, t.xhi, t.zhi);
    return t;
}

// Staging window of (transmit term bounds tb, chunk starting at r0): lo, len
// and the FP32 window-relative base B = tx_ref + R_{r0} - lo.
struct StageInfo {
    int lo, len, skip, pad;
    float B;
    float pad2[3];
};

__device__ __forceinline__ StageInfo stage_info(const DasArgs& a, const TileGeo& tg, float2 tb,
                                                double txref, int r0, int r_last, double R_r0) {
    const float2 rb = rx_bounds(a.g, r0, r_last, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
    StageInfo si;
    si.lo = (int)floorf(tb.x + rb.x) - 2;
    si.len = (int)ceilf(tb.y + rb.y) + 2 - si.lo + 1;
    si.skip = (si.lo + si.len <= 0 || si.lo > a.ns - 2) ? 1 : 0;
    si.B = (float)(txref + R_r0 - (double)si.lo);
    si.pad = 0;
    return si;
}

template <int MODE, typename T, bool CHECK>
__global__ void __launch_bounds__(kThreads, 2) das_tiled_kernel(const __grid_constant__ DasArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* buf = reinterpret_cast<float2*>(smem_raw);                  // [kC][W]
    float2* ttab = buf + kC * a.W;                                       // [kTS][kP][kThreads]
    Elem* el = reinterpret_cast<Elem*>(ttab + kTS * kP * kThreads);      // [E]
    __shared__ float2 s_tb[kTS];
    __shared__ double s_txref[kTS];
    __shared__ int s_tlist[kTS];
    __shared__ int s_nact;
    __shared__ StageInfo s_si[2];

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.x, b = blockIdx.y;
    const int slice = item % a.n_slices, tile = item / a.n_slices;
    const TileGeo tg = tile_geo(a, (tile % a.tiles_x) * kTX, (tile / a.tiles_x) * kTZ);
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;

    // Pixel offsets from the reference point; FP32 depths for the aperture.
    const float ux = (float)lane * g.gdx;
    float uz[kP], kz[kP], kap[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        uz[p] = (float)(warp * kP + p) * g.gdz;
        kz[p] = uz[p] * fmaf(2.0f, (float)tg.cz, uz[p]);
        kap[p] = aperture_kappa(g, (float)tg.cz + uz[p]);
    }

    const int t_begin = slice * kTS, t_end = min(a.n_tx, t_begin + kTS);
    const int2 er = tg.er;
    for (int e = er.x + tid; e <= er.y; e += kThreads) el[e - er.x] = make_elem(a, tg.cx, tg.cz, e);
    if (tid == 0) {
        int n = 0;
        for (int t = t_begin; t < t_end; ++t) {
            if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
            s_tlist[n++] = t;
        }
        s_nact = er.x <= er.y ? n : 0;
    }
    __syncthreads();
    const int n_act = s_nact;

    // Transmit terms of the slice: FP64 reference, FP32 per-pixel correction + weight.
    for (int j = 0; j < n_act; ++j) {
        const TxInfo& ti = a.tx[s_tlist[j]];
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            float2 v;
            if (MODE == 0) {
                const Elem et = el[ti.e - er.x];
                v.x = dist_delta(et, ux, kz[p]);
                v.y = apod_w(g.apod, -(et.ax + ux), kap[p]) * et.g;
            } else {
                v.x = fmaf(ux, ti.sin_f, uz[p] * ti.cos_f);
                v.y = 1.0f;
            }
            ttab[(j * kP + p) * kThreads + tid] = v;
        }
        if (tid == j) {
            s_tb[j] = tx_bounds<MODE>(g, ti, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
            s_txref[j] = tx_ref<MODE>(ti, tg.cx, tg.cz, MODE == 0 ? el[ti.e - er.x].R : 0.0);
        }
    }
    const int n_chunks = n_act > 0 ? (er.y - er.x + kC) / kC : 0;
    const int n_stages = n_chunks * n_act;
    __syncthreads();
    if (tid == 0 && n_stages > 0) {
        const int r_last = min(er.x + kC - 1, er.y);
        s_si[0] = stage_info(a, tg, s_tb[0], s_txref[0], er.x, r_last, el[0].R);
    }

    float acc[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) acc[p] = 0.0f;
    float Dr[kC][kP], Wr[kC][kP];
    __syncthreads();

    for (int q = 0; q < n_stages; ++q) {
        const int k = q / n_act, j = q - k * n_act;
        const int r0 = er.x + k * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        if (j == 0) {
            // Receive chunk: window-relative distances C_c + delta and weights in registers.
            const double R0 = el[r0 - er.x].R;
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                const int re = min(r0 + c, r_last);  // padding reuses the last element, weight 0
                const Elem ee = el[re - er.x];
                const float cc = (float)(ee.R - R0);
#pragma unroll
                for (int p = 0; p < kP; ++p) {
                    Dr[c][p] = cc + dist_delta(ee, ux, kz[p]);
                    Wr[c][p] = (r0 + c <= r_last) ? apod_w(g.apod, -(ee.ax + ux), kap[p]) * ee.g
                                                  : 0.0f;
                }
            }
        }
        const StageInfo si = s_si[q & 1];
        const int t = s_tlist[j];
        int len = si.len;
        if (!si.skip) {
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
                const bool ok_r = r <= r_last;
                for (int qq = tid; qq < len; qq += kThreads) {
                    const int n = si.lo + qq;
                    float2 v = make_float2(0.0f, 0.0f);
                    if (ok_r && n >= 0 && n <= a.ns - 2) v = RF<T>::pair(tr + n, a.rf_scale);
                    dst[qq] = v;
                }
            }
        }
        if (tid == 0 && q + 1 < n_stages) {
            const int k1 = (q + 1) / n_act, j1 = (q + 1) - k1 * n_act;
            const int r01 = er.x + k1 * kC;
            s_si[(q + 1) & 1] = stage_info(a, tg, s_tb[j1], s_txref[j1], r01,
                                           min(r01 + kC - 1, er.y), el[r01 - er.x].R);
        }
        __syncthreads();
        if (!si.skip) {
            float tw[kP], wt[kP], acct[kP];
#pragma unroll
            for (int p = 0; p < kP; ++p) {
                const float2 v = ttab[(j * kP + p) * kThreads + tid];
                tw[p] = si.B + v.x;
                wt[p] = v.y;
                acct[p] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                const float2* bc = buf + c * a.W;
#pragma unroll
                for (int p = 0; p < kP; ++p) {
                    const float s = tw[p] + Dr[c][p];
                    const float m = __fadd_rd(s, kMagic);
                    const float f = s - (m - kMagic);
                    int idx = __float_as_int(m) - kMagicBits;
                    if (CHECK && (idx < 0 || idx >= len)) {
                        flag(a.hdr, 2u, (unsigned)blockIdx.x, (unsigned)idx, (unsigned)len);
                        idx = 0;
                    }
                    const float2 ab = bc[idx];
                    acct[p] = fmaf(Wr[c][p], fmaf(f, ab.y, ab.x), acct[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < kP; ++p) acc[p] = fmaf(wt[p], acct[p], acc[p]);
        }
        __syncthreads();
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
// shared memory (very coarse grids).  Delays in FP64 (this path is rare and
// has no tile-relative reference), interpolation and sums in FP32.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) das_direct_kernel(const __grid_constant__ DasArgs a) {
    const Geom& g = a.g;
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iz = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int b = blockIdx.z;
    if (ix >= g.nx || iz >= g.nz) return;
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;
    const double pxd = fma((double)ix, a.gd.gdx, a.gd.gx0);
    const double pzd = fma((double)iz, a.gd.gdz, a.gd.gz0);
    const float px = (float)pxd, pz = (float)pzd, kap = aperture_kappa(g, pz);
    const int2 er = tile_elements(g, px, px, pz);
    float acc = 0.0f;
    for (int t = 0; t < a.n_tx; ++t) {
        const TxInfo& ti = a.tx[t];
        double dt;
        float wt;
        if (MODE == 0) {
            const double xe = fma((double)ti.e, a.gd.pitch, a.gd.xe0);
            dt = sqrt((pxd - xe) * (pxd - xe) + pzd * pzd) - ti.t0_d;
            wt = apod_w(g.apod, (float)(xe - pxd), kap);
            if (g.elem_weight) wt *= __ldg(g.elem_weight + ti.e);
        } else {
            dt = fma(pxd, ti.sin_d, fma(pzd, ti.cos_d, -ti.t0_d));
            wt = 1.0f;
        }
        if (wt == 0.0f) continue;
        float inner = 0.0f;
        for (int r = er.x; r <= er.y; ++r) {
            const double xe = fma((double)r, a.gd.pitch, a.gd.xe0);
            float w = apod_w(g.apod, (float)(xe - pxd), kap);
            if (g.elem_weight) w *= __ldg(g.elem_weight + r);
            if (w == 0.0f) continue;
            const double s = dt + sqrt((pxd - xe) * (pxd - xe) + pzd * pzd);
            const double fl = floor(s);
            if (!(fl >= 0.0) || !(fl <= (double)(a.ns - 2))) continue;
            const int i = (int)fl;
            const float f = (float)(s - fl);
            const float2 ab = RF<T>::pair(rf + ((long long)t * g.n_elements + r) * a.ns + i, a.rf_scale);
            inner = fmaf(w, fmaf(f, ab.y, ab.x), inner);
        }
        acc = fmaf(wt, inner, acc);
    }
    a.out[((long long)b * g.nz + iz) * g.nx + ix] = acc;
}

// Delays (samples) exactly as the tiled kernel forms them: the window start lo
// plus the FP32 window-relative value, for (pixel, transmit, element) triples.
// Triples the kernel never evaluates (element outside the tile's aperture
// range, inactive transmit) are NaN.
template <int MODE>
__global__ void das_delays_kernel(const __grid_constant__ DasArgs a, const int32_t* __restrict__ pix,
                                  int n_pix, double* __restrict__ out) {
    const Geom& g = a.g;
    const long long n = (long long)n_pix * a.n_tx * g.n_elements;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i % g.n_elements);
        const int t = (int)((i / g.n_elements) % a.n_tx);
        const int q = (int)(i / ((long long)g.n_elements * a.n_tx));
        const int lin = pix[q];
        const int ix = lin % g.nx, iz = lin / g.nx;
        const TileGeo tg = tile_geo(a, (ix / kTX) * kTX, (iz / kTZ) * kTZ);
        const TxInfo& ti = a.tx[t];
        const int2 er = tg.er;
        if (r < er.x || r > er.y || (MODE == 0 && (ti.e < er.x || ti.e > er.y))) {
            out[i] = __longlong_as_double(0x7ff8000000000000LL);
            continue;
        }
        const float ux = (float)(ix - tg.ix0) * g.gdx;
        const float uz = (float)(iz - tg.iz0) * g.gdz;
        const float kz = uz * fmaf(2.0f, (float)tg.cz, uz);
        const int r0 = er.x + ((r - er.x) / kC) * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        const Elem e0 = make_elem(a, tg.cx, tg.cz, r0);
        const Elem erl = make_elem(a, tg.cx, tg.cz, r);
        double R_et = 0.0;
        float dtx;
        if (MODE == 0) {
            const Elem et = make_elem(a, tg.cx, tg.cz, ti.e);
            R_et = et.R;
            dtx = dist_delta(et, ux, kz);
        } else {
            dtx = fmaf(ux, ti.sin_f, uz * ti.cos_f);
        }
        const float2 tb = tx_bounds<MODE>(g, ti, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
        const StageInfo si = stage_info(a, tg, tb, tx_ref<MODE>(ti, tg.cx, tg.cz, R_et), r0, r_last,
                                        e0.R);
        const float dr = (float)(erl.R - e0.R) + dist_delta(erl, ux, kz);
        const float s = (si.B + dtx) + dr;
        out[i] = (double)si.lo + (double)s;
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

void make_geom(const wf_probe* p, const wf_grid* g, Geom& G, GeomD& D) {
    const double sc = p->fs / p->c;  // samples per metre
    D.gx0 = g->x_min * sc;
    D.gdx = g->nx > 1 ? (g->x_max - g->x_min) / (g->nx - 1) * sc : 0.0;
    D.gz0 = g->z_min * sc;
    D.gdz = g->nz > 1 ? (g->z_max - g->z_min) / (g->nz - 1) * sc : 0.0;
    D.xe0 = -0.5 * (p->n_elements - 1) * p->pitch * sc;
    D.pitch = p->pitch * sc;
    G.gx0 = (float)D.gx0;
    G.gdx = (float)D.gdx;
    G.gz0 = (float)D.gz0;
    G.gdz = (float)D.gdz;
    G.xe0 = (float)D.xe0;
    G.pitch = (float)D.pitch;
    G.two_f = (float)(2.0 * (p->apod == WF_APOD_NONE ? 1.0 : p->f_number));
    G.apod = p->apod;
    G.n_elements = p->n_elements;
    G.nz = g->nz;
    G.nx = g->nx;
    G.elem_weight = p->elem_weight;
}

// Largest |delay| (samples) any pixel/element pair can produce, for the
// 2^22 range of the round-down floor.
double max_delay(const wf_probe* p, const wf_grid* g) {
    const double sc = p->fs / p->c;
    const double half = 0.5 * (p->n_elements - 1) * p->pitch;
    const double dx = std::max(std::fabs(g->x_min), std::fabs(g->x_max)) + half;
    const double dz = std::max(std::fabs(g->z_min), std::fabs(g->z_max));
    return std::sqrt(dx * dx + dz * dz) * sc;
}

struct Plan {
    int tiles_x, tiles_z, n_slices, n_items;
    int W;
    bool tiled;
    size_t smem;
    size_t ws_bytes;
};

Plan make_plan(const wf_probe* p, const wf_grid* g, int batch, int n_tx) {
    Geom G;
    GeomD D;
    make_geom(p, g, G, D);
    Plan P;
    P.tiles_x = (g->nx + kTX - 1) / kTX;
    P.tiles_z = (g->nz + kTZ - 1) / kTZ;
    P.n_slices = (n_tx + kTS - 1) / kTS;
    P.n_items = P.tiles_x * P.tiles_z * P.n_slices;
    // Lipschitz bound on one staging window: both distance terms move by at
    // most the tile diagonal, the receive term by (kC-1) pitches across the
    // chunk; plus floor/ceil and the +-2 margins.
    const double ex = (double)(kTX - 1) * D.gdx, ez = (double)(kTZ - 1) * D.gdz;
    const double diam = std::sqrt(ex * ex + ez * ez);
    const double w = 2.0 * diam + (kC - 1) * D.pitch + 16.0;
    P.W = (int)std::ceil(w / 4.0) * 4;
    P.tiled = P.W <= kMaxWindow;
    P.smem = (size_t)kC * P.W * sizeof(float2) + (size_t)kTS * kP * kThreads * sizeof(float2) +
             (size_t)p->n_elements * sizeof(Elem);
    P.ws_bytes = kWsHeaderBytes +
                 (P.tiled ? (size_t)batch * P.n_items * kTilePix * sizeof(float) : 0);
    return P;
}

constexpr size_t kMaxTiledSmem = (size_t)kC * kMaxWindow * sizeof(float2) +
                                  (size_t)kTS * kP * kThreads * sizeof(float2) +
                                  (size_t)WF_MAX_ELEMENTS * sizeof(Elem);

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
                     wf_stream stream, DasArgs& A, double tx_extra) {
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
    if (2.0 * max_delay(probe, grid) + tx_extra >= 4194304.0) return WF_ERR_UNSUPPORTED;
    const Plan P = make_plan(probe, grid, batch, n_tx);
    if (!ws || ((uintptr_t)ws & 15u)) return WF_ERR_WORKSPACE;
    if (ws_bytes < P.ws_bytes) return WF_ERR_WORKSPACE;
    make_geom(probe, grid, A.g, A.gd);
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

// Fill the transmit table; returns the largest |t0 fs| (samples) or -1 on bad input.
double fill_tx(DasArgs& a, const wf_probe* probe, int mode, int n_tx, const int32_t* tx_elem,
               const double* angles, const double* t_start, bool per_tx_start) {
    double extra = 0.0;
    for (int t = 0; t < n_tx; ++t) {
        TxInfo ti{};
        const double t0 = t_start ? t_start[per_tx_start ? t : 0] : 0.0;
        if (!std::isfinite(t0)) return -1.0;
        ti.t0_d = t0 * probe->fs;
        if (mode == 0) {
            const int e = tx_elem ? tx_elem[t] : t;
            if (e < 0 || e >= probe->n_elements) return -1.0;
            ti.e = e;
        } else {
            const double th = angles[t];
            if (!std::isfinite(th)) return -1.0;
            ti.sin_d = std::sin(th);
            ti.cos_d = std::cos(th);
            ti.sin_f = (float)ti.sin_d;
            ti.cos_f = (float)ti.cos_d;
        }
        a.tx[t] = ti;
        extra = std::max(extra, std::fabs(ti.t0_d));
    }
    return extra;
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
    thread_local DasArgs local;  // ~10 KB parameter block, copied into the launch
    DasArgs& a = local;
    if (!probe || !std::isfinite(t_start)) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    if (check_probe_grid(probe, grid) != WF_OK) return WF_ERR_INVALID_ARG;
    const double extra = fill_tx(a, probe, 0, n_tx, tx_elem, nullptr, &t_start, false);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    return das_common(0, probe, grid, batch, n_tx, n_rx, n_samples, dtype, rf, rf_scale, out, ws,
                      ws_bytes, stream, a, extra);
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
    if (check_probe_grid(probe, grid) != WF_OK) return WF_ERR_INVALID_ARG;
    const double extra = fill_tx(a, probe, 1, n_angles, nullptr, angles_rad, t_start, true);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    return das_common(1, probe, grid, batch, n_angles, n_rx, n_samples, dtype, rf, rf_scale, out,
                      ws, ws_bytes, stream, a, extra);
}

extern "C" wf_status wf_das_delays(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                   int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                                   const double* t_start, int32_t n_pix, const int32_t* pix,
                                   double* out, wf_stream stream) {
    thread_local DasArgs local;
    DasArgs& a = local;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (mode != 0 && mode != 1) return WF_ERR_INVALID_ARG;
    if (mode == 1 && !angles_rad) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX || n_pix < 0 || (n_pix > 0 && (!pix || !out)))
        return WF_ERR_INVALID_ARG;
    const double extra = fill_tx(a, probe, mode, n_tx, tx_elem, angles_rad, t_start, mode == 1);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    if (n_pix == 0) return WF_OK;
    make_geom(probe, grid, a.g, a.gd);
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
