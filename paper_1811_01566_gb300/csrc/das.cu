// Delay-and-sum beamforming for STAI and PWI (paper Sec. II-B, Fig. 2 "Beamforming").
//
// b(p) = sum_t Wt(p,t) sum_r Wr(p,r) lerp(rf[t][r], Dt(p,t) + Dr(p,r))
//   STAI: Dt = |p - x_{e_t}| - t_start fs,   Wt = apod(p, e_t) g_{e_t}
//   PWI:  Dt = x sin th + z cos th - t0 fs,   Wt = 1
//   both: Dr = |p - x_r|,                     Wr = apod(p, r) g_r
// (all lengths in samples).  DAS is a gather-sum, not a contraction: no
// tensor cores.  Design (GB300):
//  * a CTA (8 warps) owns a pixel tile and one slice of transmits.  A warp
//    covers WCOL columns; its lanes (and P pixels per lane) run down the rows.
//    STAI uses one column per warp (tile 8 x 64): a transmit/receive pair is
//    live for whole columns, so all warps of a tile share the same aperture.
//    PWI uses 4 columns per warp (tile 32 x 32): its plane-wave delays vary
//    slowly across x, so wide tiles reuse each staged sample more.
//  * geometry is tile-relative: the tile origin c is the reference point and
//    R_e = |c - x_e| is exact (FP64, stored as a float hi/lo pair); a pixel at
//    c + u needs only the small FP32 correction
//      delta = |c + u - x_e| - R_e = N / (R_e + |c + u - x_e|),
//      N = u_x (2 (c_x - x_e) + u_x) + u_z (2 c_z + u_z),
//    and every fractional delay is formed relative to its staging window, so
//    FP32 carries a few hundred samples of range instead of thousands (delay
//    error ~3e-5 samples instead of ~2e-4);
//  * receive elements are processed in chunks of 8: corrections and weights in
//    registers, computed only by warps with an element of the chunk in their
//    aperture; STAI transmit corrections of the slice sit in a thread-private
//    shared table; nothing geometric is read from global memory;
//  * for every (transmit, receive chunk) the sample window the tile can touch
//    (exact convex bounds of the delay over the tile) is staged into shared
//    memory as FP32 pairs (x[i], x[i+1]-x[i]): one 8-byte shared load and one
//    FMA interpolate a sample.  Raw samples are loaded 16 bytes at a time one
//    stage ahead; the int16 scale is folded into the receive weights;
//  * warps skip stages whose transmit or receive chunk lies outside their
//    aperture or whose delays all fall outside the record;
//  * the floor of the window-relative delay is a round-down add of 1.5 * 2^23;
//  * partial images of the transmit slices go to the workspace and a second
//    kernel sums them in slice order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace wf {

constexpr int kThreads = 256;              // 8 warps
constexpr int kC = 8;                      // receive elements per chunk
constexpr int kTS = 16;                    // transmits (or angles) per slice
constexpr int kMaxWindow = 512;            // staged positions per trace: 64 segments of 8
constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

struct TxInfo {
    DF sin, cos, t0;   // PWI steering (double-float); both: t0 = time of sample 0 times fs
    float sin_f, cos_f;
    int e;             // STAI: element fired
    int pad;
};

// Sample-unit geometry as double-floats (reference terms) next to the float copy in Geom.
struct GeomDF {
    DF gx0, gdx, gz0, gdz, xe0, pitch;
};

struct DasArgs {
    Geom g;
    GeomDF gd;
    int n_tx, ns;
    int tiles_x, n_slices, n_items;  // items per frame = tiles * slices
    int W;                           // staged positions per trace (shared stride)
    int ring;                        // TMA raw-sample ring depth
    const void* rf;
    float rf_scale;
    long long frame_elems;           // n_tx * E * ns
    float* part;                     // [batch][n_items][256 * P] slice partials
    float* out;
    WsHeader* hdr;
    TxInfo tx[WF_MAX_TX];
};

// Tile shape of a kernel configuration.
template <int WCOL, int P>
struct Shape {
    static constexpr int kLR = 32 / WCOL;     // lane rows per warp
    static constexpr int kCols = 8 * WCOL;    // tile columns
    static constexpr int kRows = kLR * P;     // tile rows
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

// Per-element reference data of a tile (shared memory): R_e = Rhi + Rlo exactly
// enough (FP64 split into two floats), c_x - x_e and the element weight.
struct Elem {
    float Rhi, Rlo, ax, g;
};

__device__ __forceinline__ DF elem_R(const Elem& e) { return DF{e.Rhi, e.Rlo}; }

// Distance from the reference point (cx, cz) to element e, in double-float
// (relative error ~1e-13, far below the FP32 corrections added to it).
__device__ __forceinline__ Elem make_elem(const DasArgs& a, DF cx, DF cz, int e) {
    const DF xe = df_axpk(a.gd.xe0, e, a.gd.pitch);
    const DF ax = df_add(cx, df_neg(xe));
    const DF R = df_sqrt(df_add(df_mul(ax, ax), df_mul(cz, cz)));
    Elem el;
    el.Rhi = R.hi;
    el.Rlo = R.lo;
    el.ax = ax.hi;
    el.g = a.g.elem_weight ? __ldg(a.g.elem_weight + e) : 1.0f;
    return el;
}

// FP32 correction |c + u - x_e| - R_e for a pixel at offset (ux, uz); kz = uz (2 cz + uz).
__device__ __forceinline__ float dist_delta(const Elem& el, float ux, float kz) {
    const float n = fmaf(ux, 2.0f * el.ax + ux, kz);
    const float t = fmaf(el.Rhi, el.Rhi, n);
    const float d = t > 0.0f ? t * rsqrtf(t) : 0.0f;
    const float den = el.Rhi + d;
    return den > 0.0f ? __fdividef(n, den) : 0.0f;
}

// R_e - R_ref of two elements of the same tile, in FP32 (the hi parts differ exactly).
__device__ __forceinline__ float elem_rel(const Elem& e, const Elem& ref) {
    return (e.Rhi - ref.Rhi) + (e.Rlo - ref.Rlo);
}

// Element range that can be inside the aperture of some pixel of [xlo, xhi] x [.., zhi].
__device__ __forceinline__ int2 tile_elements(const Geom& g, float xlo, float xhi, float zhi) {
    if (g.apod == WF_APOD_NONE) return make_int2(0, g.n_elements - 1);
    if (!(zhi > 0.0f)) return make_int2(1, 0);
    const float half = zhi / g.two_f;
    const int lo = (int)floorf((xlo - half - g.xe0) / g.pitch) - 1;
    const int hi = (int)ceilf((xhi + half - g.xe0) / g.pitch) + 1;
    return make_int2(max(lo, 0), min(hi, g.n_elements - 1));
}

// Exact range over the rectangle [xlo, xhi] x [zlo, zhi] of the delay of one
// (transmit, receive element) pair, FP32.  Both delay forms are convex in x
// and increase with z >= 0, so the maximum sits on a bottom corner and the
// minimum on the top edge at the clamped stationary point: the midpoint of
// the two elements for STAI, x_r - z tan(th) for PWI.
template <int MODE>
__device__ __forceinline__ float2 pair_bounds(const Geom& g, const TxInfo& ti, int r, float xlo,
                                              float xhi, float zlo, float zhi) {
    const float xr = elem_x(g, r);
    const float c = -ti.t0.hi;
    if (MODE == 0) {
        const float xt = elem_x(g, ti.e);
        const float xm = fminf(fmaxf(0.5f * (xt + xr), xlo), xhi);
        const float a0 = xm - xt, b0 = xm - xr;
        const float mn = sqrtf(fmaf(a0, a0, zlo * zlo)) + sqrtf(fmaf(b0, b0, zlo * zlo));
        const float a1 = xlo - xt, b1 = xlo - xr, a2 = xhi - xt, b2 = xhi - xr;
        const float z2 = zhi * zhi;
        const float mx = fmaxf(sqrtf(fmaf(a1, a1, z2)) + sqrtf(fmaf(b1, b1, z2)),
                               sqrtf(fmaf(a2, a2, z2)) + sqrtf(fmaf(b2, b2, z2)));
        return make_float2(mn + c, mx + c);
    }
    const float xm = fminf(fmaxf(xr - zlo * (ti.sin_f / ti.cos_f), xlo), xhi);
    const float b0 = xm - xr;
    const float mn = fmaf(xm, ti.sin_f, zlo * ti.cos_f) + sqrtf(fmaf(b0, b0, zlo * zlo));
    const float b1 = xlo - xr, b2 = xhi - xr, z2 = zhi * zhi;
    const float mx = fmaxf(fmaf(xlo, ti.sin_f, zhi * ti.cos_f) + sqrtf(fmaf(b1, b1, z2)),
                           fmaf(xhi, ti.sin_f, zhi * ti.cos_f) + sqrtf(fmaf(b2, b2, z2)));
    return make_float2(mn + c, mx + c);
}

// Transmit reference term at the reference point (double-float).
template <int MODE>
__device__ __forceinline__ DF tx_ref(const TxInfo& ti, DF cx, DF cz, DF R_et) {
    if (MODE == 0) return df_add(R_et, df_neg(ti.t0));
    return df_add(df_add(df_mul(cx, ti.sin), df_mul(cz, ti.cos)), df_neg(ti.t0));
}

__device__ __forceinline__ void flag(WsHeader* h, unsigned bit, unsigned a, unsigned b, unsigned c) {
    if (atomicOr(&h->flags, bit) == 0u) {
        h->first_bad[0] = a;
        h->first_bad[1] = b;
        h->first_bad[2] = c;
    }
}

// Tile geometry shared by the DAS kernel and the delay probe; the origin pixel
// of the tile is the FP64 reference point.
struct TileGeo {
    int ix0, iz0;
    DF cx, cz;
    float xlo, xhi, zlo, zhi;
    int2 er;
};

template <int COLS, int ROWS>
__device__ __forceinline__ TileGeo tile_geo(const DasArgs& a, int ix0, int iz0) {
    const Geom& g = a.g;
    TileGeo t;
    t.ix0 = ix0;
    t.iz0 = iz0;
    t.cx = df_axpk(a.gd.gx0, ix0, a.gd.gdx);
    t.cz = df_axpk(a.gd.gz0, iz0, a.gd.gdz);
    t.xlo = pixel_x(g, ix0);
    t.xhi = pixel_x(g, ix0 + COLS - 1);
    t.zlo = pixel_z(g, iz0);
    t.zhi = pixel_z(g, iz0 + ROWS - 1);
    t.er = tile_elements(g, t.xlo, t.xhi, t.zhi);
    return t;
}

// Staging window of one (transmit, receive chunk) stage: the first staged
// sample lo (multiple of 8), the staged length (multiple of 8, <= W), the FP32
// window-relative base B = tx_ref + R_{r0} - lo, and flags (bit 0: no sample of
// the window is inside the record; bits 1..: clamped over-long window length).
struct StageInfo {
    int lo, len;
    float B;
    int flags;
    __device__ __forceinline__ bool skip() const { return flags & 1; }
    __device__ __forceinline__ int over() const { return flags >> 1; }
};

__device__ __forceinline__ StageInfo make_stage(const DasArgs& a, float mn, float mx, DF txref,
                                                DF R_r0) {
    StageInfo si;
    si.lo = ((int)floorf(mn) - 2) & ~7;
    si.len = (((int)ceilf(mx) + 2 - si.lo + 1) + 7) & ~7;
    const int skip = (si.lo + si.len <= 0 || si.lo > a.ns - 2) ? 1 : 0;
    const DF x = df_add(txref, R_r0);
    si.B = (x.hi - (float)si.lo) + x.lo;   // x.hi - lo is exact: lo is an integer near x.hi
    const int over = si.len > a.W ? si.len : 0;
    if (over) si.len = a.W;
    si.flags = skip | (over << 1);
    return si;
}

// ---------------------------------------------------------------------------
// TMA staging: bulk asynchronous copies (cp.async.bulk) of raw trace windows
// into a shared-memory ring, completion tracked by mbarriers.  Every wait is
// bounded: on timeout the kernel records a flag in the workspace header and
// carries on (its result is then unspecified, the call reports WF_ERR_INTERNAL
// through wf_workspace_check) instead of spinning forever.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr unsigned kWaitLimit = 1u << 22;   // try_wait rounds before a wait is declared stuck

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
    for (unsigned i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i >= 16) __nanosleep(64);
    }
    return false;
}

// Raw samples of one staging segment (8 consecutive samples + the next one)
// held in registers between the prefetch and the conversion.
template <typename T> struct Seg;
template <> struct Seg<int16_t> {
    uint4 v;
    int nxt;
    __device__ __forceinline__ float at(int k) const {
        const unsigned w = (k >> 1) == 0 ? v.x : (k >> 1) == 1 ? v.y : (k >> 1) == 2 ? v.z : v.w;
        return (float)((k & 1) ? ((int)w >> 16) : (int)(short)(w & 0xffffu));
    }
};
template <> struct Seg<__half> {
    uint4 v;
    int nxt;
    __device__ __forceinline__ float at(int k) const {
        const unsigned w = (k >> 1) == 0 ? v.x : (k >> 1) == 1 ? v.y : (k >> 1) == 2 ? v.z : v.w;
        return __half2float(__ushort_as_half((unsigned short)((k & 1) ? (w >> 16) : (w & 0xffffu))));
    }
};
template <> struct Seg<float> {
    float4 v0, v1;
    int nxt;
    __device__ __forceinline__ float at(int k) const {
        switch (k) {
            case 0: return v0.x; case 1: return v0.y; case 2: return v0.z; case 3: return v0.w;
            case 4: return v1.x; case 5: return v1.y; case 6: return v1.z; default: return v1.w;
        }
    }
};

template <typename T> __device__ __forceinline__ float raw_one(int bits);
template <> __device__ __forceinline__ float raw_one<int16_t>(int bits) { return (float)(short)bits; }
template <> __device__ __forceinline__ float raw_one<__half>(int bits) {
    return __half2float(__ushort_as_half((unsigned short)bits));
}
template <> __device__ __forceinline__ float raw_one<float>(int bits) { return __int_as_float(bits); }

template <typename T> __device__ __forceinline__ int raw_bits(const T* p);
template <> __device__ __forceinline__ int raw_bits<int16_t>(const int16_t* p) {
    return (int)(unsigned short)__ldg(p);
}
template <> __device__ __forceinline__ int raw_bits<__half>(const __half* p) {
    return (int)__ldg(reinterpret_cast<const unsigned short*>(p));
}
template <> __device__ __forceinline__ int raw_bits<float>(const float* p) { return __float_as_int(__ldg(p)); }

// Load samples [n0, n0 + 8) of a trace and sample n0 + 8 (zero outside [0, ns)).
template <typename T>
__device__ __forceinline__ void seg_load(Seg<T>& sg, const T* tr, int n0, int ns, bool vec_ok) {
    if (vec_ok && n0 >= 0 && n0 + 8 <= ns) {
        if constexpr (sizeof(T) == 2) {
            sg.v = __ldg(reinterpret_cast<const uint4*>(tr + n0));
        } else {
            sg.v0 = __ldg(reinterpret_cast<const float4*>(tr + n0));
            sg.v1 = __ldg(reinterpret_cast<const float4*>(tr + n0 + 4));
        }
    } else {
        int b[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) b[k] = (n0 + k >= 0 && n0 + k < ns) ? raw_bits<T>(tr + n0 + k) : 0;
        if constexpr (sizeof(T) == 2) {
            sg.v = make_uint4((unsigned)(b[0] & 0xffff) | ((unsigned)b[1] << 16),
                              (unsigned)(b[2] & 0xffff) | ((unsigned)b[3] << 16),
                              (unsigned)(b[4] & 0xffff) | ((unsigned)b[5] << 16),
                              (unsigned)(b[6] & 0xffff) | ((unsigned)b[7] << 16));
        } else {
            sg.v0 = make_float4(__int_as_float(b[0]), __int_as_float(b[1]), __int_as_float(b[2]),
                                __int_as_float(b[3]));
            sg.v1 = make_float4(__int_as_float(b[4]), __int_as_float(b[5]), __int_as_float(b[6]),
                                __int_as_float(b[7]));
        }
    }
    sg.nxt = (n0 + 8 >= 0 && n0 + 8 < ns) ? raw_bits<T>(tr + n0 + 8) : 0;
}

// Load samples [8k, 8k + 9) of a raw shared-memory row (16-byte aligned).
template <typename T>
__device__ __forceinline__ void seg_load_smem(Seg<T>& sg, const T* row, int k) {
    if constexpr (sizeof(T) == 2) {
        sg.v = *reinterpret_cast<const uint4*>(row + 8 * k);
        sg.nxt = (int)*reinterpret_cast<const unsigned short*>(row + 8 * k + 8);
    } else {
        sg.v0 = *reinterpret_cast<const float4*>(row + 8 * k);
        sg.v1 = *reinterpret_cast<const float4*>(row + 8 * k + 4);
        sg.nxt = __float_as_int(row[8 * k + 8]);
    }
}

// Convert a segment to 8 FP32 pairs (x[n], x[n+1] - x[n]) in raw units; pairs
// whose n is outside [0, ns - 2] are zero (no recorded neighbour).
template <typename T>
__device__ __forceinline__ void seg_store(const Seg<T>& sg, float2* dst, int n0, int ns) {
    float v[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = sg.at(k);
    v[8] = raw_one<T>(sg.nxt);
    const bool full = n0 >= 0 && n0 + 9 <= ns;
    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
        float2 p0 = make_float2(v[k], v[k + 1] - v[k]);
        float2 p1 = make_float2(v[k + 1], v[k + 2] - v[k + 1]);
        if (!full) {
            if (!(n0 + k >= 0 && n0 + k <= ns - 2)) p0 = make_float2(0.0f, 0.0f);
            if (!(n0 + k + 1 >= 0 && n0 + k + 1 <= ns - 2)) p1 = make_float2(0.0f, 0.0f);
        }
        d4[k >> 1] = make_float4(p0.x, p0.y, p1.x, p1.y);
    }
}

// Segment g = 64 c + k (c: trace of the chunk, k: 8-sample block) of a stage;
// thread tid handles segments tid and tid + 256.
template <typename T>
__device__ __forceinline__ void stage_prefetch(Seg<T> (&sg)[2], const DasArgs& a, const T* rf,
                                               const StageInfo& si, int t, int r0, int r_last,
                                               bool vec_ok) {
    const int nseg = si.len >> 3;
    const int k = threadIdx.x & 63;
    const T* base = rf + ((long long)t * a.g.n_elements + r0) * a.ns;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int c = (threadIdx.x >> 6) + 4 * i;
        if (k < nseg && r0 + c <= r_last) seg_load<T>(sg[i], base + (long long)c * a.ns, si.lo + 8 * k, a.ns, vec_ok);
    }
}

template <typename T>
__device__ __forceinline__ void stage_store(const Seg<T> (&sg)[2], float2* buf, const DasArgs& a,
                                            const StageInfo& si, int r0, int r_last) {
    const int nseg = si.len >> 3;
    const int k = threadIdx.x & 63;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int c = (threadIdx.x >> 6) + 4 * i;
        if (k < nseg) {
            float2* dst = buf + c * a.W + 8 * k;
            if (r0 + c <= r_last) {
                seg_store<T>(sg[i], dst, si.lo + 8 * k, a.ns);
            } else {
                float4* d4 = reinterpret_cast<float4*>(dst);
                const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                d4[0] = z; d4[1] = z; d4[2] = z; d4[3] = z;
            }
        }
    }
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Transmits per slice: STAI keeps a per-pixel transmit table in shared memory,
// so wide-P tiles take fewer transmits per slice.
template <int MODE, int P>
struct Slice {
    static constexpr int kTx = (MODE == 0 && P > 2) ? 8 : kTS;
};
constexpr int kTableStages = 256;  // stage-window ring in shared memory
constexpr int kTableBatch = 128;   // windows computed per refill (one per thread)
constexpr int kMaxRing = 3;        // TMA raw-sample ring depth

// Shared-memory layout of the tiled kernel (byte offsets, all 16-byte aligned).
struct SmemLayout {
    size_t pairs, ttab, table, elems, raw, total;
};

__host__ __device__ inline SmemLayout smem_layout(int mode, int P, int ts, int W, int n_elements,
                                                  bool db, bool tma, int ring, int rf_bytes) {
    SmemLayout L;
    size_t off = 0;
    L.pairs = off;
    off += (size_t)(db ? 2 : 1) * kC * W * sizeof(float2);
    L.ttab = off;
    off += mode == 0 ? (size_t)ts * P * kThreads * sizeof(float2) : 0;
    L.table = off;
    off += (size_t)kTableStages * sizeof(StageInfo);
    L.elems = off;
    off += (((size_t)n_elements * sizeof(Elem)) + 15) & ~(size_t)15;
    L.raw = off;
    off += tma ? (size_t)ring * kC * (W + 8) * rf_bytes : 0;
    L.total = off;
    return L;
}

template <int MODE, typename T, int WCOL, int P, bool DB, bool TMA, bool CHECK>
__global__ void __launch_bounds__(kThreads, 2) das_tiled_kernel(const __grid_constant__ DasArgs a) {
    using S = Shape<WCOL, P>;
    constexpr int TS = Slice<MODE, P>::kTx;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(MODE, P, TS, a.W, a.g.n_elements, DB, TMA, a.ring, (int)sizeof(T));
    float2* buf0 = reinterpret_cast<float2*>(smem_raw + L.pairs);   // [DB+1][kC][W] pairs
    float2* ttab = reinterpret_cast<float2*>(smem_raw + L.ttab);    // [TS][P][256] (STAI)
    StageInfo* st = reinterpret_cast<StageInfo*>(smem_raw + L.table);
    Elem* el = reinterpret_cast<Elem*>(smem_raw + L.elems);         // [E range]
    T* raw = reinterpret_cast<T*>(smem_raw + L.raw);                // [ring][kC][W + 8]
    __shared__ __align__(8) unsigned long long s_bar[kMaxRing];
    __shared__ DF s_txref[TS];
    __shared__ float2 s_dtw[TS][kThreads / 32];   // STAI: per-warp range of the transmit correction
    __shared__ int s_tlist[TS];
    __shared__ int s_nact;

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = lane % WCOL, lz = lane / WCOL;
    const int item = blockIdx.x, b = blockIdx.y;
    const int slice = item % a.n_slices, tile = item / a.n_slices;
    const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, (tile % a.tiles_x) * S::kCols,
                                                    (tile / a.tiles_x) * S::kRows);
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;
    const bool vec_ok = (a.ns & 7) == 0;
    const int RW = a.W + 8;           // raw row stride (samples)
    const int ring = TMA ? a.ring : 1;

    // Pixel offsets from the reference point: column WCOL warp + lx, rows lz + kLR p.
    const int col = WCOL * warp + lx;
    const float ux = (float)col * g.gdx;
    float kz[P], kap[P], uz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        uz[p] = (float)(lz + S::kLR * p) * g.gdz;
        kz[p] = uz[p] * fmaf(2.0f, tg.cz.hi, uz[p]);
        kap[p] = aperture_kappa(g, tg.cz.hi + uz[p]);
    }
    // Elements that can weigh on this warp's columns (all rows of the tile).
    const int2 wr = tile_elements(g, pixel_x(g, tg.ix0 + WCOL * warp),
                                  pixel_x(g, tg.ix0 + WCOL * warp + WCOL - 1), tg.zhi);

    const int t_begin = slice * TS, t_end = min(a.n_tx, t_begin + TS);
    const int2 er = tg.er;
    for (int e = er.x + tid; e <= er.y; e += kThreads) el[e - er.x] = make_elem(a, tg.cx, tg.cz, e);
    if (tid == 0) {
        int n = 0;
        for (int t = t_begin; t < t_end; ++t) {
            if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
            s_tlist[n++] = t;
        }
        s_nact = er.x <= er.y ? n : 0;
        if (TMA) {
            for (int i = 0; i < ring; ++i) mbar_init(&s_bar[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();
    const int n_act = s_nact;

    for (int j = 0; j < n_act; ++j) {
        const TxInfo& ti = a.tx[s_tlist[j]];
        if (MODE == 0) {
            // STAI transmit terms: FP32 correction + weight per pixel, per-warp range.
            const Elem et = el[ti.e - er.x];
            float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                const float2 v = make_float2(dist_delta(et, ux, kz[p]),
                                             apod_w(g.apod, -(et.ax + ux), kap[p]) * et.g);
                mn = fminf(mn, v.x);
                mx = fmaxf(mx, v.x);
                ttab[(j * P + p) * kThreads + tid] = v;
            }
            mn = warp_min(mn);
            mx = warp_max(mx);
            if (lane == 0) s_dtw[j][warp] = make_float2(mn, mx);
        }
        if (tid == j) s_txref[j] = tx_ref<MODE>(ti, tg.cx, tg.cz, MODE == 0 ? elem_R(el[ti.e - er.x]) : DF{0.0f, 0.0f});
    }
    const int n_chunks = n_act > 0 ? (er.y - er.x + kC) / kC : 0;
    const int n_stages = n_chunks * n_act;
    __syncthreads();

    // Stage windows, kTableBatch at a time into a ring of kTableStages: stage q
    // is (slice transmit q mod n_act, receive chunk q / n_act).
    auto fill_table = [&](int base) {
        const int q = base + tid;
        if (tid < kTableBatch && q < n_stages) {
            const int k = q / n_act, jj = q - k * n_act;
            const int rr0 = er.x + k * kC, rrl = min(rr0 + kC - 1, er.y);
            const TxInfo& ti = a.tx[s_tlist[jj]];
            float mn = 3.0e38f, mx = -3.0e38f;
            for (int rr = rr0; rr <= rrl; ++rr) {
                const float2 bd = pair_bounds<MODE>(g, ti, rr, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
                mn = fminf(mn, bd.x);
                mx = fmaxf(mx, bd.y);
            }
            st[q & (kTableStages - 1)] = make_stage(a, mn, mx, s_txref[jj], elem_R(el[rr0 - er.x]));
        }
    };
    // TMA producer (thread 0): raw windows of stage qq into ring slot qq % ring.
    auto issue = [&](int qq) {
        const StageInfo si = st[qq & (kTableStages - 1)];
        unsigned long long* bar = &s_bar[qq % ring];
        const int k = qq / n_act, jj = qq - k * n_act;
        const int rr0 = er.x + k * kC, rrl = min(rr0 + kC - 1, er.y);
        const int na = max(si.lo, 0), nb = min(si.lo + si.len + 8, a.ns);
        if (si.skip() || nb <= na) {
            mbar_arrive_expect(bar, 0u);
            return;
        }
        const unsigned bytes = (unsigned)((nb - na) * (int)sizeof(T));
        fence_async_shared();
        mbar_arrive_expect(bar, bytes * (unsigned)(rrl - rr0 + 1));
        T* slot = raw + (size_t)(qq % ring) * kC * RW;
        const T* src = rf + ((long long)s_tlist[jj] * g.n_elements + rr0) * a.ns + na;
        for (int c = 0; c <= rrl - rr0; ++c)
            bulk_copy_g2s(slot + c * RW + (na - si.lo), src + (long long)c * a.ns, bytes, bar);
    };
    const int ahead = TMA ? ring - 1 : 1;   // stages in flight ahead of the one being converted
    fill_table(0);

    // PWI: range of the transmit correction ux sin + uz cos over this warp's pixels.
    const float wux0 = (float)(WCOL * warp) * g.gdx, wux1 = (float)(WCOL * warp + WCOL - 1) * g.gdx;
    const float wuz1 = (float)(S::kRows - 1) * g.gdz;

    float acc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = 0.0f;
    float Dr[kC][P], Wr[kC][P];
    float dr_min = 0.0f, dr_max = 0.0f;
    unsigned cmask = 0u;
    Seg<T> sg[2];

    int j = 0, r0 = er.x;           // stage q = (chunk starting at r0, slice transmit j)
    int j1 = 0, r01 = er.x;         // stage q + 1 (register path)
    auto advance = [&](int& jj, int& rr) {
        if (++jj == n_act) { jj = 0; rr += kC; }
    };
    __syncthreads();
    if (n_stages > 0) {
        advance(j1, r01);
        if (TMA) {
            if (tid == 0)
                for (int qq = 0; qq < min(ahead, n_stages); ++qq) issue(qq);
        } else {
            const StageInfo s0 = st[0];
            if (!s0.skip()) stage_prefetch<T>(sg, a, rf, s0, s_tlist[0], er.x, min(er.x + kC - 1, er.y), vec_ok);
        }
    }

    for (int q = 0; q < n_stages; ++q) {
        const int r_last = min(r0 + kC - 1, er.y);
        const StageInfo si = st[q & (kTableStages - 1)];
        const int t = s_tlist[j];
        float2* buf = buf0 + (DB ? (q & 1) * kC * a.W : 0);
        if (si.over() && tid == 0) flag(a.hdr, 1u, (unsigned)blockIdx.x, (unsigned)si.over(), (unsigned)a.W);
        if (TMA) {
            if (!mbar_wait_bounded(&s_bar[q % ring], (unsigned)((q / ring) & 1))) {
                if (tid == 0) flag(a.hdr, 4u, (unsigned)blockIdx.x, (unsigned)q, 0u);
            }
            if (!si.skip()) {
                // raw slot -> FP32 pairs, segment (trace c, block k) = (tid >> 6 [+4], tid & 63)
                const T* slot = raw + (size_t)(q % ring) * kC * RW;
                const int nseg = si.len >> 3, k = tid & 63;
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int c = (tid >> 6) + 4 * i;
                    if (k < nseg) {
                        float2* dst = buf + c * a.W + 8 * k;
                        if (r0 + c <= r_last) {
                            Seg<T> sv;
                            seg_load_smem<T>(sv, slot + c * RW, k);
                            seg_store<T>(sv, dst, si.lo + 8 * k, a.ns);
                        } else {
                            float4* d4 = reinterpret_cast<float4*>(dst);
                            const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            d4[0] = z; d4[1] = z; d4[2] = z; d4[3] = z;
                        }
                    }
                }
            }
        } else if (!si.skip()) {
            stage_store<T>(sg, buf, a, si, r0, r_last);
        }
        __syncthreads();   // pairs of stage q visible; raw slot of stage q - 1 and (double-buffered) pairs of q - 1 free
        if (q + ahead < n_stages) {
            if (((q + ahead) & (kTableBatch - 1)) == 0) {
                fill_table(q + ahead);
                __syncthreads();
            }
            if (TMA) {
                if (tid == 0) issue(q + ahead);
            } else {
                const StageInfo s1 = st[(q + 1) & (kTableStages - 1)];
                if (!s1.skip()) stage_prefetch<T>(sg, a, rf, s1, s_tlist[j1], r01, min(r01 + kC - 1, er.y), vec_ok);
            }
        }
        if (j == 0) {
            // New receive chunk: which elements weigh on this warp, and (only for those)
            // window-relative distances C_c + delta and weights (times the int16 scale).
            cmask = 0u;
#pragma unroll
            for (int c = 0; c < kC; ++c)
                if (r0 + c <= r_last && r0 + c >= wr.x && r0 + c <= wr.y) cmask |= 1u << c;
            if (cmask) {
                const Elem e0 = el[r0 - er.x];
                float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
                for (int c = 0; c < kC; ++c) {
                    const bool on = (cmask >> c) & 1u;
                    const Elem ee = el[(on ? r0 + c : r0) - er.x];
                    const float cc = elem_rel(ee, e0);
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        Dr[c][p] = on ? cc + dist_delta(ee, ux, kz[p]) : 0.0f;
                        Wr[c][p] = on ? apod_w(g.apod, -(ee.ax + ux), kap[p]) * (ee.g * a.rf_scale) : 0.0f;
                        if (on) {
                            mn = fminf(mn, Dr[c][p]);
                            mx = fmaxf(mx, Dr[c][p]);
                        }
                    }
                }
                dr_min = warp_min(mn);
                dr_max = warp_max(mx);
            }
        }
        // Warp-level skip: transmit or chunk outside this warp's aperture, or every
        // delay of the warp outside the record.
        bool live = !si.skip() && cmask != 0u;
        float2 dtw;
        if (MODE == 0) {
            live = live && a.tx[t].e >= wr.x && a.tx[t].e <= wr.y;
            dtw = s_dtw[j][warp];
        } else {
            const float sn = a.tx[t].sin_f, cs = a.tx[t].cos_f;
            const float v0 = wux0 * sn, v1 = wux1 * sn, z1 = wuz1 * cs;
            dtw = make_float2(fminf(v0, v1) + fminf(0.0f, z1), fmaxf(v0, v1) + fmaxf(0.0f, z1));
        }
        if (live) {
            const float lo_f = (float)si.lo + si.B;
            live = (lo_f + dtw.x + dr_min <= (float)(a.ns - 1) + 0.5f) && (lo_f + dtw.y + dr_max >= -0.5f);
        }
        if (live) {
            float tw[P], wt[P], acct[P];
            const float sn = a.tx[t].sin_f, cs = a.tx[t].cos_f;
#pragma unroll
            for (int p = 0; p < P; ++p) {
                if (MODE == 0) {
                    const float2 v = ttab[(j * P + p) * kThreads + tid];
                    tw[p] = si.B + v.x;
                    wt[p] = v.y;
                } else {
                    tw[p] = si.B + fmaf(ux, sn, uz[p] * cs);
                    wt[p] = 1.0f;
                }
                acct[p] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                if (!((cmask >> c) & 1u)) continue;
                const float2* bc = buf + c * a.W;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const float s = tw[p] + Dr[c][p];
                    const float m = __fadd_rd(s, kMagic);
                    const float f = s - (m - kMagic);
                    int idx = __float_as_int(m) - kMagicBits;
                    if (CHECK && (idx < 0 || idx >= si.len)) {
                        flag(a.hdr, 2u, (unsigned)blockIdx.x, (unsigned)idx, (unsigned)si.len);
                        idx = 0;
                    }
                    const float2 ab = bc[idx];
                    acct[p] = fmaf(Wr[c][p], fmaf(f, ab.y, ab.x), acct[p]);
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) acc[p] = MODE == 0 ? fmaf(wt[p], acct[p], acc[p]) : acc[p] + acct[p];
        }
        if (!DB) __syncthreads();   // single buffer: compute of stage q done before stage q + 1 lands
        j = j1; r0 = r01;
        advance(j1, r01);
    }

    // Partial tile in thread order: [p][tid].
    float* dst = a.part + ((long long)b * a.n_items + item) * (kThreads * P);
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p * kThreads + tid] = acc[p];
}

// Sum the transmit-slice partials of every pixel in slice order.
template <int WCOL, int P>
__global__ void das_reduce_kernel(const float* __restrict__ part, float* __restrict__ out, int nz,
                                  int nx, int tiles_x, int n_slices, int n_items) {
    using S = Shape<WCOL, P>;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= nx) return;
    const int tile = (iz / S::kRows) * tiles_x + ix / S::kCols;
    const int cl = ix % S::kCols, rl = iz % S::kRows;
    const int tid = (cl / WCOL) * 32 + (rl % S::kLR) * WCOL + (cl % WCOL);
    const int local = (rl / S::kLR) * kThreads + tid;
    const float* p = part + ((long long)b * n_items + (long long)tile * n_slices) * (kThreads * P) + local;
    float s = 0.0f;
    for (int k = 0; k < n_slices; ++k) s += p[(long long)k * (kThreads * P)];
    out[((long long)b * nz + iz) * nx + ix] = s;
}

// Direct per-pixel gather for geometries whose staging windows do not fit in
// shared memory (very coarse grids).  Each pixel is its own reference point:
// delays in double-float, interpolation and sums in FP32.
template <int MODE, typename T>
__global__ void __launch_bounds__(256) das_direct_kernel(const __grid_constant__ DasArgs a) {
    const Geom& g = a.g;
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iz = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int b = blockIdx.z;
    if (ix >= g.nx || iz >= g.nz) return;
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;
    const DF px = df_axpk(a.gd.gx0, ix, a.gd.gdx), pz = df_axpk(a.gd.gz0, iz, a.gd.gdz);
    const DF pz2 = df_mul(pz, pz);
    const float kap = aperture_kappa(g, pz.hi);
    const int2 er = tile_elements(g, px.hi, px.hi, pz.hi);
    auto dist = [&](int e, float& dxe) {
        const DF d = df_add(df_axpk(a.gd.xe0, e, a.gd.pitch), df_neg(px));
        dxe = d.hi;
        return df_sqrt(df_add(df_mul(d, d), pz2));
    };
    float acc = 0.0f;
    for (int t = 0; t < a.n_tx; ++t) {
        const TxInfo& ti = a.tx[t];
        DF dt;
        float wt;
        if (MODE == 0) {
            float dxe;
            dt = df_add(dist(ti.e, dxe), df_neg(ti.t0));
            wt = apod_w(g.apod, dxe, kap);
            if (g.elem_weight) wt *= __ldg(g.elem_weight + ti.e);
        } else {
            dt = df_add(df_add(df_mul(px, ti.sin), df_mul(pz, ti.cos)), df_neg(ti.t0));
            wt = 1.0f;
        }
        if (wt == 0.0f) continue;
        float inner = 0.0f;
        for (int r = er.x; r <= er.y; ++r) {
            float dxe;
            const DF dr = dist(r, dxe);
            float w = apod_w(g.apod, dxe, kap);
            if (g.elem_weight) w *= __ldg(g.elem_weight + r);
            if (w == 0.0f) continue;
            const DF sd = df_add(dt, dr);
            float fl = floorf(sd.hi);
            float f = (sd.hi - fl) + sd.lo;
            if (f < 0.0f) { fl -= 1.0f; f += 1.0f; }
            if (f >= 1.0f) { fl += 1.0f; f -= 1.0f; }
            if (!(fl >= 0.0f) || !(fl <= (float)(a.ns - 2))) continue;
            const T* tr = rf + ((long long)t * g.n_elements + r) * a.ns + (int)fl;
            const float x0 = raw_one<T>(raw_bits<T>(tr)), x1 = raw_one<T>(raw_bits<T>(tr + 1));
            inner = fmaf(w, fmaf(f, x1 - x0, x0), inner);
        }
        acc = fmaf(wt, inner, acc);
    }
    a.out[((long long)b * g.nz + iz) * g.nx + ix] = acc * a.rf_scale;
}

// Delays (samples) exactly as the tiled kernel forms them: the window start lo
// plus the FP32 window-relative value, for (pixel, transmit, element) triples.
// Triples the kernel never evaluates (element outside the tile's aperture
// range, inactive transmit) are NaN.
template <int MODE, int WCOL, int P>
__global__ void das_delays_kernel(const __grid_constant__ DasArgs a, const int32_t* __restrict__ pix,
                                  int n_pix, int32_t* __restrict__ out_lo, float* __restrict__ out_rel) {
    using S = Shape<WCOL, P>;
    const Geom& g = a.g;
    const long long n = (long long)n_pix * a.n_tx * g.n_elements;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i % g.n_elements);
        const int t = (int)((i / g.n_elements) % a.n_tx);
        const int q = (int)(i / ((long long)g.n_elements * a.n_tx));
        const int lin = pix[q];
        const int ix = lin % g.nx, iz = lin / g.nx;
        const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, (ix / S::kCols) * S::kCols,
                                                        (iz / S::kRows) * S::kRows);
        const TxInfo& ti = a.tx[t];
        const int2 er = tg.er;
        if (r < er.x || r > er.y || (MODE == 0 && (ti.e < er.x || ti.e > er.y))) {
            out_lo[i] = 0;
            out_rel[i] = __int_as_float(0x7fc00000);
            continue;
        }
        const float ux = (float)(ix - tg.ix0) * g.gdx;
        const float uz = (float)(iz - tg.iz0) * g.gdz;
        const float kz = uz * fmaf(2.0f, tg.cz.hi, uz);
        const int r0 = er.x + ((r - er.x) / kC) * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        const Elem e0 = make_elem(a, tg.cx, tg.cz, r0);
        const Elem erl = make_elem(a, tg.cx, tg.cz, r);
        DF R_et{0.0f, 0.0f};
        float dtx;
        if (MODE == 0) {
            const Elem et = make_elem(a, tg.cx, tg.cz, ti.e);
            R_et = elem_R(et);
            dtx = dist_delta(et, ux, kz);
        } else {
            dtx = fmaf(ux, ti.sin_f, uz * ti.cos_f);
        }
        float mn = 3.0e38f, mx = -3.0e38f;
        for (int rr = r0; rr <= r_last; ++rr) {
            const float2 bd = pair_bounds<MODE>(g, ti, rr, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
            mn = fminf(mn, bd.x);
            mx = fmaxf(mx, bd.y);
        }
        const StageInfo si = make_stage(a, mn, mx, tx_ref<MODE>(ti, tg.cx, tg.cz, R_et), elem_R(e0));
        const float dr = elem_rel(erl, e0) + dist_delta(erl, ux, kz);
        const float s = (si.B + dtx) + dr;
        out_lo[i] = si.lo;
        out_rel[i] = s;
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

// Sample-unit geometry in host double precision.
struct GeomD {
    double gx0, gdx, gz0, gdz, xe0, pitch;
};

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

void make_geom(const wf_probe* p, const wf_grid* g, Geom& G, GeomDF& F) {
    GeomD D;
    make_geom(p, g, G, D);
    F.gx0 = df_from_double(D.gx0);
    F.gdx = df_from_double(D.gdx);
    F.gz0 = df_from_double(D.gz0);
    F.gdz = df_from_double(D.gdz);
    F.xe0 = df_from_double(D.xe0);
    F.pitch = df_from_double(D.pitch);
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

// Kernel configurations in order of preference: columns per warp and pixels per lane.
struct Cfg {
    int wcol, p;
};
constexpr Cfg kStaiCfgs[] = {{4, 4}, {4, 2}};
constexpr Cfg kPwiCfgs[] = {{4, 4}, {4, 2}};
constexpr size_t kSmemBudget = 113 * 1024;   // two CTAs per SM
constexpr size_t kMaxTiledSmem = 220 * 1024;  // one CTA per SM

struct Plan {
    Cfg cfg;
    int cols, rows, ts;
    int tiles_x, tiles_z, n_slices, n_items;
    int W, ring;
    bool tiled, db, tma;
    size_t smem;
    size_t ws_bytes;
};

// Upper bound on one staging window for a cols x rows tile: both distance
// terms move by at most the tile diagonal, the receive term by (kC - 1)
// pitches across the chunk; plus floor/ceil, the +-2 margins and the
// 8-sample alignment of both ends.
int window_bound(const GeomD& D, int cols, int rows) {
    const double ex = (double)(cols - 1) * D.gdx, ez = (double)(rows - 1) * D.gdz;
    const double diam = std::sqrt(ex * ex + ez * ez);
    const double w = 2.0 * diam + (kC - 1) * D.pitch + 24.0;
    return (int)std::ceil(w / 8.0) * 8;
}

// Optional tuning override "wcol,p" (WF_DAS_TILE); ignored unless it names a
// configuration of this mode that fits.
bool tile_override(int mode, Cfg& out) {
    const char* v = std::getenv("WF_DAS_TILE");
    int w = 0, p = 0;
    if (!v || std::sscanf(v, "%d,%d", &w, &p) != 2) return false;
    const Cfg* cfgs = mode == 0 ? kStaiCfgs : kPwiCfgs;
    for (int i = 0; i < 2; ++i)
        if (cfgs[i].wcol == w && cfgs[i].p == p) {
            out = cfgs[i];
            return true;
        }
    return false;
}

Plan plan_for(int mode, const Cfg& cfg, const GeomD& D, const wf_probe* p, const wf_grid* g,
              int batch, int n_tx, int ns, int rf_bytes) {
    Plan P{};
    P.cfg = cfg;
    P.cols = 8 * cfg.wcol;
    P.rows = (32 / cfg.wcol) * cfg.p;
    P.ts = (mode == 0 && cfg.p > 2) ? 8 : kTS;
    P.W = window_bound(D, P.cols, P.rows);
    P.tiled = P.W <= kMaxWindow;
    P.tiles_x = (g->nx + P.cols - 1) / P.cols;
    P.tiles_z = (g->nz + P.rows - 1) / P.rows;
    P.n_slices = (n_tx + P.ts - 1) / P.ts;
    P.n_items = P.tiles_x * P.tiles_z * P.n_slices;
    // TMA bulk copies need 16-byte aligned trace windows: samples per trace a multiple of 8.
    // WF_DAS_NO_TMA=1 selects the register-staged path instead (tuning and testing).
    const char* no_tma = std::getenv("WF_DAS_NO_TMA");
    P.tma = ns % 8 == 0 && !(no_tma && no_tma[0] && no_tma[0] != '0');
    bool found = false;
    const int rings[2] = {P.tma ? 3 : 1, P.tma ? 2 : 1};
    for (int ri = 0; ri < 2 && !found; ++ri)
        for (int dbi = 0; dbi < 2 && !found; ++dbi) {
            const bool db = dbi == 0 && P.tma;
            const SmemLayout L = smem_layout(mode, cfg.p, P.ts, P.W, p->n_elements, db, P.tma, rings[ri], rf_bytes);
            if (L.total <= kSmemBudget) {
                P.ring = rings[ri];
                P.db = db;
                P.smem = L.total;
                found = true;
            }
        }
    if (!found) {
        P.ring = P.tma ? 2 : 1;
        P.db = false;
        P.smem = smem_layout(mode, cfg.p, P.ts, P.W, p->n_elements, false, P.tma, P.ring, rf_bytes).total;
        if (P.smem > kMaxTiledSmem) P.tiled = false;
    }
    P.ws_bytes = kWsHeaderBytes +
                 (P.tiled ? (size_t)batch * P.n_items * kThreads * cfg.p * sizeof(float) : 0);
    return P;
}

Plan make_plan(int mode, const wf_probe* p, const wf_grid* g, int batch, int n_tx, int ns = 8,
               int rf_bytes = 4) {
    Geom G;
    GeomD D;
    make_geom(p, g, G, D);
    Cfg forced;
    if (tile_override(mode, forced)) {
        const Plan P = plan_for(mode, forced, D, p, g, batch, n_tx, ns, rf_bytes);
        if (P.tiled) return P;
    }
    const Cfg* cfgs = mode == 0 ? kStaiCfgs : kPwiCfgs;
    const int n = mode == 0 ? 2 : 2;
    Plan P{};
    for (int i = 0; i < n; ++i) {
        P = plan_for(mode, cfgs[i], D, p, g, batch, n_tx, ns, rf_bytes);
        if (P.tiled) return P;
    }
    return P;
}

bool check_bounds_mode() {
    const char* v = std::getenv("WF_CHECK_BOUNDS");
    return v && v[0] && v[0] != '0';
}

template <int MODE, typename T, int WCOL, int P, bool DB, bool TMA>
wf_status launch_tiled_v(DasArgs& A, const Plan& PL, int batch, cudaStream_t st) {
    static unsigned long long smem_set[2] = {0ull, 0ull};
    const bool chk = check_bounds_mode();
    auto kern = chk ? das_tiled_kernel<MODE, T, WCOL, P, DB, TMA, true>
                    : das_tiled_kernel<MODE, T, WCOL, P, DB, TMA, false>;
    wf_status s = ensure_smem_limit(kern, kMaxTiledSmem, smem_set[chk ? 1 : 0]);
    if (s != WF_OK) return s;
    kern<<<dim3(PL.n_items, batch), kThreads, PL.smem, st>>>(A);
    if ((s = last_launch_status()) != WF_OK) return s;
    dim3 rg((A.g.nx + 127) / 128, A.g.nz, batch);
    das_reduce_kernel<WCOL, P><<<rg, 128, 0, st>>>(A.part, A.out, A.g.nz, A.g.nx, PL.tiles_x,
                                                   PL.n_slices, PL.n_items);
    return last_launch_status();
}

template <int MODE, typename T, int WCOL, int P>
wf_status launch_tiled(DasArgs& A, const Plan& PL, int batch, cudaStream_t st) {
    if (!PL.tma) return launch_tiled_v<MODE, T, WCOL, P, false, false>(A, PL, batch, st);
    return PL.db ? launch_tiled_v<MODE, T, WCOL, P, true, true>(A, PL, batch, st)
                 : launch_tiled_v<MODE, T, WCOL, P, false, true>(A, PL, batch, st);
}

template <int MODE, typename T>
wf_status launch_das(DasArgs& A, const Plan& P, int batch, cudaStream_t st) {
    if (!P.tiled) {
        dim3 grid((A.g.nx + 31) / 32, (A.g.nz + 7) / 8, batch);
        das_direct_kernel<MODE, T><<<grid, 256, 0, st>>>(A);
        return last_launch_status();
    }
    return P.cfg.p == 4 ? launch_tiled<MODE, T, 4, 4>(A, P, batch, st)
                        : launch_tiled<MODE, T, 4, 2>(A, P, batch, st);
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
    const Plan P = make_plan(mode, probe, grid, batch, n_tx, n_samples, dtype == WF_F32 ? 4 : 2);
    if (!ws || ((uintptr_t)ws & 15u)) return WF_ERR_WORKSPACE;
    if (ws_bytes < P.ws_bytes) return WF_ERR_WORKSPACE;
    make_geom(probe, grid, A.g, A.gd);
    A.n_tx = n_tx;
    A.ns = n_samples;
    A.tiles_x = P.tiles_x;
    A.n_slices = P.n_slices;
    A.n_items = P.n_items;
    A.W = P.W;
    A.ring = P.ring;
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
        ti.t0 = df_from_double(t0 * probe->fs);
        if (mode == 0) {
            const int e = tx_elem ? tx_elem[t] : t;
            if (e < 0 || e >= probe->n_elements) return -1.0;
            ti.e = e;
        } else {
            const double th = angles[t];
            // steering beyond +-89 degrees has no plane wave travelling into the medium
            if (!std::isfinite(th) || std::fabs(th) > 1.5533430342749532) return -1.0;
            ti.sin = df_from_double(std::sin(th));
            ti.cos = df_from_double(std::cos(th));
            ti.sin_f = ti.sin.hi;
            ti.cos_f = ti.cos.hi;
        }
        a.tx[t] = ti;
        extra = std::max(extra, std::fabs(t0 * probe->fs));
    }
    return extra;
}

}  // namespace
}  // namespace wf

using namespace wf;

extern "C" size_t wf_das_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                         int32_t n_tx) {
    if (check_probe_grid(probe, grid) != WF_OK || batch < 1 || n_tx < 1 || n_tx > WF_MAX_TX) return 0;
    // Enough for every configuration either transmit scheme may pick.
    Geom G;
    GeomD D;
    make_geom(probe, grid, G, D);
    size_t need = kWsHeaderBytes;
    for (const Cfg& c : kStaiCfgs) need = std::max(need, plan_for(0, c, D, probe, grid, batch, n_tx, 8, 4).ws_bytes);
    for (const Cfg& c : kPwiCfgs) need = std::max(need, plan_for(1, c, D, probe, grid, batch, n_tx, 8, 4).ws_bytes);
    return need;
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
                                   int32_t* out_lo, float* out_rel, wf_stream stream) {
    thread_local DasArgs local;
    DasArgs& a = local;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (mode != 0 && mode != 1) return WF_ERR_INVALID_ARG;
    if (mode == 1 && !angles_rad) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX || n_pix < 0 || (n_pix > 0 && (!pix || !out_lo || !out_rel)))
        return WF_ERR_INVALID_ARG;
    const double extra = fill_tx(a, probe, mode, n_tx, tx_elem, angles_rad, t_start, mode == 1);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    if (n_pix == 0) return WF_OK;
    make_geom(probe, grid, a.g, a.gd);
    a.n_tx = n_tx;
    a.ns = 1 << 30;  // the probe reports delays regardless of the record length
    const Plan P = make_plan(mode, probe, grid, 1, n_tx);
    a.W = 1 << 30;   // and never clamps a window
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (mode == 0) {
        if (P.cfg.p == 4) das_delays_kernel<0, 4, 4><<<304, 256, 0, st>>>(a, pix, n_pix, out_lo, out_rel);
        else das_delays_kernel<0, 4, 2><<<304, 256, 0, st>>>(a, pix, n_pix, out_lo, out_rel);
    } else {
        if (P.cfg.p == 4) das_delays_kernel<1, 4, 4><<<304, 256, 0, st>>>(a, pix, n_pix, out_lo, out_rel);
        else das_delays_kernel<1, 4, 2><<<304, 256, 0, st>>>(a, pix, n_pix, out_lo, out_rel);
    }
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

// ---------------------------------------------------------------------------
// Fixed-scratch STAI entry point: the workspace is a file-scope device array
// instead of caller memory.  The paper has no counterpart; it serves callers
// that cannot allocate device memory themselves.
// ---------------------------------------------------------------------------
namespace wf {
namespace {

constexpr size_t kFixedScratchBytes = (size_t)WF_FIXED_SCRATCH_BYTES;

// Shared by every call on a device and held by each device that loads the library.
static __device__ __align__(256) unsigned char g_fixed_scratch[kFixedScratchBytes];

// Device address of g_fixed_scratch, looked up once per device with that device
// current (in host code the symbol is only a host-side stand-in).
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
int g_scratch_ready[kMaxDevices] = {};

wf_status fixed_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WF_ERR_UNSUPPORTED;
    if (__atomic_load_n(&g_scratch_ready[dev], __ATOMIC_ACQUIRE)) {
        *out = g_scratch_ptr[dev];
        return WF_OK;
    }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fixed_scratch) != cudaSuccess || !p) return WF_ERR_CUDA;
    g_scratch_ptr[dev] = p;
    __atomic_store_n(&g_scratch_ready[dev], 1, __ATOMIC_RELEASE);
    *out = p;
    return WF_OK;
}

}  // namespace
}  // namespace wf

extern "C" wf_status wf_das_stai_fixed_scratch(const wf_probe* probe, const wf_grid* grid,
                                               int32_t batch, int32_t n_tx, const int32_t* tx_elem,
                                               int32_t n_rx, int32_t n_samples, double t_start,
                                               wf_dtype dtype, const void* rf, float rf_scale,
                                               float* out, wf_stream stream) {
    if (check_probe_grid(probe, grid) != WF_OK || batch < 1 || n_tx < 1 || n_tx > WF_MAX_TX)
        return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (n_samples < 1 || n_samples > WF_MAX_SAMPLES) return WF_ERR_INVALID_ARG;
    const Plan P = make_plan(0, probe, grid, batch, n_tx, n_samples, dtype == WF_F32 ? 4 : 2);
    if (P.ws_bytes > kFixedScratchBytes) return WF_ERR_WORKSPACE;
    void* ws = nullptr;
    const wf_status s = fixed_scratch(&ws);
    if (s != WF_OK) return s;
    return wf_das_stai(probe, grid, batch, n_tx, tx_elem, n_rx, n_samples, t_start, dtype, rf,
                       rf_scale, out, ws, kFixedScratchBytes, stream);
}

extern "C" size_t wf_fixed_scratch_bytes(void) { return kFixedScratchBytes; }
