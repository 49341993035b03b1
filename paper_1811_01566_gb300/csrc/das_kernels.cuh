// Delay-and-sum beamforming kernels for STAI and PWI (paper Sec. II-B; the beamforming block of Fig. 2).
//
// b(p) = sum_t Wt(p,t) sum_r Wr(p,r) lerp(rf[t][r], Dt(p,t) + Dr(p,r))
//   STAI: Dt = |p - x_{e_t}| - t_start fs,   Wt = apod(p, e_t) g_{e_t}
//   PWI:  Dt = x sin th + z cos th - t0 fs,   Wt = 1
//   both: Dr = |p - x_r|,                     Wr = apod(p, r) g_r
// (all lengths in samples).  DAS is a gather-sum, not a contraction: no
// tensor cores.  Design (GB300):
//  * a CTA (8 warps) owns a pixel tile and one group of receive chunks, and
//    loops over every transmit for them, chunk-outer.  A warp covers WCOL
//    columns; its lanes (and P pixels per lane) run down the rows (tile 32 x 32
//    for P = 4).  Receive distances and weights of a chunk of 8 elements are
//    computed once per tile in registers and reused by every transmit; the
//    transmit term of a stage is recomputed per pixel (one distance and one
//    weight for STAI, one FMA for PWI).  Tiles are launched deepest row first:
//    the deep tiles have the widest apertures and carry most of the work.
//  * reciprocity (STAI with every element firing once, in element order): the
//    pairs (t, r) and (r, t) have the same delay and weights, so only t <= r is
//    evaluated, on the staged sum rf[t][r] + rf[r][t] (rf[t][t] alone on the
//    diagonal).  Linear interpolation is linear in the samples, so this is the
//    same sum with half the gathers.
//  * geometry is tile-relative: the tile origin c is the reference point and
//    R_e = |c - x_e| is formed in double-float arithmetic (two FP32 words); a
//    pixel at c + u needs only the small FP32 correction
//      delta = |c + u - x_e| - R_e = N / (R_e + |c + u - x_e|),
//      N = u_x (2 (c_x - x_e) + u_x) + u_z (2 c_z + u_z),
//    and every fractional delay is formed relative to its staging window, so
//    FP32 carries a few hundred samples of range instead of thousands;
//  * for every (transmit, receive chunk) the sample window the tile can touch
//    (exact convex bounds of the delay over the tile) is copied by TMA bulk
//    copies into a shared-memory ring and converted to FP32 pairs
//    (x[i], x[i+1]-x[i]): one 8-byte shared load and one FMA interpolate a
//    sample.  The int16 scale is folded into the receive weights;
//  * warps skip stages whose transmit or receive chunk lies outside their
//    aperture or whose delays all fall outside the record;
//  * the floor of the window-relative delay is a round-down add of 1.5 * 2^23;
//  * partial images of the chunk groups go to the workspace and a second
//    kernel sums them in group order (deterministic).
#pragma once

#include <cuda_fp16.h>

#include "common.cuh"

namespace wf {

constexpr int kThreads = 256;              // 8 warps
constexpr int kC = 8;                      // receive elements per chunk
constexpr int kMaxWindow = 512;            // staged positions per trace: 64 segments of 8
constexpr int kMaxGroups = 64;             // stage-range groups per tile
constexpr int kMaxItems = 2048;            // CTAs per frame of a work-proportional schedule
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
    // TMA descriptors of the RF array viewed as [frames * n_tx][E][ns / 8][8] (dimensions
    // listed slowest first): boxes of (W + 8) samples of 8 receive rows of one transmit
    // (tm_rows) and of one receive column of 8 transmits (tm_cols, the mirrored rows of
    // reciprocal STAI).  Filled per call when use_tmap is set.
    CUtensorMap tm_rows;
    CUtensorMap tm_cols;
    int use_tmap;
    Geom g;
    GeomDF gd;
    int n_tx, ns;
    int tiles_x, tiles_z;
    int n_groups, n_items;           // items per frame = tiles * groups
    int W;                           // staged positions per trace (shared stride)
    int ring;                        // TMA raw-sample ring depth
    int sym;                         // delay probe: reciprocal STAI pairing in use
    const void* rf;
    float rf_scale;
    long long frame_elems;           // n_tx * E * ns
    float* part;                     // [batch][n_items][256 * P] group partials
    float* out;
    WsHeader* hdr;
    // work-proportional schedule: item i is tile items[i] & 0xffff, group (items[i] >> 16) & 0xff
    // of items[i] >> 24; each tile's first CTA records (first item + 1) | groups << 24 in
    // tile_info for the reduction (0: the tile has no CTA and its pixels are 0)
    int use_table;
    unsigned* tile_info;
    unsigned items[kMaxItems];
    // reverse mode (wf_das_backward) only
    const float* grad_out;           // [batch][nz][nx] cotangent of the image
    float* grad_rf;                  // [batch][n_tx][E][ns] or null
    float* grad_w;                   // [E] or null
    float* grad_c;                   // [1] or null
    float neg_inv_c;                 // -1 / c (s per m/s of sound speed)
    // IQ data (wf_das_stai_iq / wf_das_pwi_iq): remodulation rate, cycles per baseband sample
    DF iq_k;
    TxInfo tx[WF_MAX_TX];
};

// Tile shape of a kernel configuration.
template <int WCOL, int P>
struct Shape {
    static constexpr int kLR = 32 / WCOL;     // lane rows per warp
    static constexpr int kCols = 8 * WCOL;    // tile columns
    static constexpr int kRows = kLR * P;     // tile rows
};

// Apodization weight given the lateral offset xe - x and kap = 2F / z.
// Hann 0.5 (1 + cos(pi u)) is evaluated as cos^2(pi u / 2) with the fast
// cosine (absolute error < 4e-7 on |pi u / 2| < pi / 2).
__device__ __forceinline__ float apod_w(int apod, float dxe, float kap) {
    if (apod == WF_APOD_NONE) return 1.0f;
    const float u = dxe * kap;
    if (!(kap > 0.0f) || !(fabsf(u) < 1.0f)) return 0.0f;
    if (apod == WF_APOD_RECT) return 1.0f;
    const float c = __cosf(u * 1.5707963267948966f);
    return c * c;
}

// Per-element reference data of a tile (shared memory): R_e = Rhi + Rlo,
// c_x - x_e and the element weight.
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
// of the tile is the reference point.
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

// Launch rank of a tile: deepest tile row first.
__host__ __device__ inline int tile_rank(int tz, int tx, int tiles_z, int tiles_x) {
    return (tiles_z - 1 - tz) * tiles_x + tx;
}

// Staging window of one (transmit, receive chunk) stage: the first staged
// sample lo (multiple of 8), the staged length (multiple of 8, <= W), the FP32
// window-relative base B = tx_ref + R_{r0} - lo, and flags (bit 0: no sample of
// the window is inside the record; bit 1: the window crosses an end of the
// record; bits 2..: clamped over-long window length).
struct StageInfo {
    int lo, len;
    float B;
    int flags;
    __device__ __forceinline__ bool skip() const { return flags & 1; }
    __device__ __forceinline__ bool edge() const { return (flags >> 1) & 1; }
    __device__ __forceinline__ int over() const { return flags >> 2; }
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
    const int edge = (si.lo >= 0 && si.lo + si.len <= a.ns - 1) ? 0 : 1;
    si.flags = skip | (edge << 1) | (over << 2);
    return si;
}

// A stage of a CTA's compacted list (only windows that reach the record): its
// window and its place in the (receive chunk k, transmit slot j) order.
struct Stage {
    int lo, len;
    float B;
    int meta;   // bit 0: window crosses an end of the record; bit 1: clamped over-long
                // window; bits 2..11: receive chunk k; bits 12..31: transmit slot j
    __device__ __forceinline__ bool edge() const { return meta & 1; }
    __device__ __forceinline__ bool over() const { return (meta >> 1) & 1; }
    __device__ __forceinline__ int k() const { return (meta >> 2) & 1023; }
    __device__ __forceinline__ int j() const { return (int)((unsigned)meta >> 12); }
};

__device__ __forceinline__ Stage pack_stage(const StageInfo& si, int k, int j) {
    return Stage{si.lo, si.len, si.B,
                 (si.edge() ? 1 : 0) | (si.over() ? 2 : 0) | (k << 2) | (j << 12)};
}

// Reciprocal STAI stage bookkeeping.  With n_e elements in the tile's range
// and nc = ceil(n_e / 8) receive chunks, chunk k pairs with the transmits
// er.x .. er.x + min(8 (k + 1), n_e) - 1 (those not after its last element).
// Stages before chunk k:
__host__ __device__ inline int sym_prefix(int k, int nc, int n_e) {
    return k < nc ? 4 * k * (k + 1) : 4 * (nc - 1) * nc + n_e;
}
// Chunk of the stage with global index qg (0 <= qg < sym_prefix(nc, nc, n_e)).
__device__ __forceinline__ int sym_chunk(int qg, int nc) {
    int k = (int)((sqrtf(1.0f + (float)qg) - 1.0f) * 0.5f);
    k = max(0, min(k, nc - 1));
    while (k < nc - 1 && 4 * (k + 1) * (k + 2) <= qg) ++k;
    while (k > 0 && 4 * k * (k + 1) > qg) --k;
    return k;
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
// 4-D tensor copy (TMA) of one box of the descriptor at coordinates {c0, c1, c2, c3}
// (fastest first) into shared memory, completion counted on the mbarrier.
__device__ __forceinline__ void tensor_copy_4d(void* dst, const CUtensorMap* map, int c0, int c1,
                                               int c2, int c3, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_u32(bar))
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
// held in registers between the load and the conversion.
template <typename T> struct Seg;
template <> struct Seg<int16_t> {
    uint4 v;
    int nxt;
    __device__ __forceinline__ float at(int k) const {
        const unsigned w = (k >> 1) == 0 ? v.x : (k >> 1) == 1 ? v.y : (k >> 1) == 2 ? v.z : v.w;
        // exact int16 -> float without a conversion instruction: 1.5 * 2^23 + v has v in its
        // low mantissa bits (|v| < 2^15), so subtracting 1.5 * 2^23 leaves exactly v
        const int iv = (k & 1) ? ((int)w >> 16) : ((int)(w << 16) >> 16);
        return __int_as_float(kMagicBits + iv) - kMagic;
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
template <> __device__ __forceinline__ float raw_one<int16_t>(int bits) {
    return __int_as_float(kMagicBits + (int)(short)bits) - kMagic;   // exact, as Seg<int16_t>::at
}
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

// Store 8 FP32 pairs (x[n], x[n+1] - x[n]) for n = n0 .. n0 + 7 from 9
// consecutive samples; pairs whose n is outside [0, ns - 2] are zero (no
// recorded neighbour).
__device__ __forceinline__ void pairs_store(const float (&v)[9], float2* dst, int n0, int ns) {
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

template <typename T>
__device__ __forceinline__ void seg_store(const Seg<T>& sg, float2* dst, int n0, int ns) {
    float v[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = sg.at(k);
    v[8] = raw_one<T>(sg.nxt);
    pairs_store(v, dst, n0, ns);
}

// Pairs of the sum of two traces (reciprocal STAI: rf[t][r] + rf[r][t]).
template <typename T>
__device__ __forceinline__ void seg_store_sum(const Seg<T>& sa, const Seg<T>& sb, float2* dst, int n0,
                                              int ns) {
    float v[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = sa.at(k) + sb.at(k);
    v[8] = raw_one<T>(sa.nxt) + raw_one<T>(sb.nxt);
    pairs_store(v, dst, n0, ns);
}

__device__ __forceinline__ void zero_segment(float2* dst) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    d4[0] = z; d4[1] = z; d4[2] = z; d4[3] = z;
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

// Packed pairs of FP32 values for Blackwell's f32x2 arithmetic: two of a
// thread's pixels go through one instruction, each lane rounded exactly as the
// scalar operation would be.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 x2_pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 x2_add_rm(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

constexpr int kTableStages = 256;  // stage-window ring in shared memory
constexpr int kIssueWarp = 7;      // warp whose lanes issue the staging copies
constexpr int kTableBatch = 128;   // windows computed per refill (one per thread)
constexpr int kMaxRing = 4;        // deepest TMA raw-sample ring

// Shared-memory layout of the tiled kernel (byte offsets, all 16-byte aligned).
struct SmemLayout {
    size_t pairs, table, elems, raw, total;
};

__host__ __device__ inline SmemLayout smem_layout(int W, int n_elements, bool db, bool tma, bool sym,
                                                  int ring, int rf_bytes) {
    SmemLayout L;
    size_t off = 0;
    L.pairs = off;
    off += (size_t)(db ? 2 : 1) * kC * W * sizeof(float2);
    L.table = off;
    off += (size_t)kTableStages * sizeof(Stage);
    L.elems = off;
    off += (((size_t)n_elements * sizeof(Elem)) + 15) & ~(size_t)15;
    off = (off + 127) & ~(size_t)127;   // tensor copies land on 128-byte boundaries
    L.raw = off;
    off += tma ? (size_t)ring * (sym ? 2 : 1) * kC * (W + 8) * rf_bytes : 0;
    L.total = off + 128;                 // slack: the kernel aligns the dynamic base itself
    return L;
}

// Segment (trace row c, block k) = (tid >> 6 [+ 4], tid & 63) of a stage, register path:
// samples of trace rows A (rf[t][r0 + c]) and, reciprocal, B (rf[r0 + c][t]).
template <typename T, bool SYM>
struct RegStage {
    Seg<T> a[2], b[2];
};

template <typename T, bool SYM>
__device__ __forceinline__ void stage_prefetch(RegStage<T, SYM>& rs, const DasArgs& a, const T* rf,
                                               const Stage& si, int t, int r0, int r_last,
                                               bool vec_ok) {
    const int nseg = si.len >> 3;
    const int k = threadIdx.x & 63;
    const long long E = a.g.n_elements;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int c = (threadIdx.x >> 6) + 4 * i;
        if (k >= nseg || r0 + c > r_last) continue;
        if (SYM && r0 + c < t) continue;
        seg_load<T>(rs.a[i], rf + ((long long)t * E + r0 + c) * a.ns, si.lo + 8 * k, a.ns, vec_ok);
        if (SYM && r0 + c > t)
            seg_load<T>(rs.b[i], rf + ((long long)(r0 + c) * E + t) * a.ns, si.lo + 8 * k, a.ns, vec_ok);
    }
}

template <typename T, bool SYM>
__device__ __forceinline__ void stage_store(const RegStage<T, SYM>& rs, float2* buf, const DasArgs& a,
                                            const Stage& si, int t, int r0, int r_last) {
    const int nseg = si.len >> 3;
    const int k = threadIdx.x & 63;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int c = (threadIdx.x >> 6) + 4 * i;
        if (k >= nseg) continue;
        float2* dst = buf + c * a.W + 8 * k;
        const bool on = r0 + c <= r_last && (!SYM || r0 + c >= t);
        if (!on) zero_segment(dst);
        else if (SYM && r0 + c > t) seg_store_sum<T>(rs.a[i], rs.b[i], dst, si.lo + 8 * k, a.ns);
        else seg_store<T>(rs.a[i], dst, si.lo + 8 * k, a.ns);
    }
}

// A CTA's stage space: raw stages [q0, q0 + n_stages) of its tile's list,
// which runs over the receive chunks of the element range er, chunk-outer, with
// every active transmit per chunk (reciprocal STAI: transmits up to the
// chunk's last element).  Raw stage q maps to (chunk k, transmit slot j); slot
// j is transmit tlist[j], or er.x + j when reciprocal.
struct StageSpace {
    int2 er;
    int n_e, nc, n_act, q0, n_stages;
    const int* tlist;
};

template <bool SYM>
__device__ __forceinline__ void locate_stage(const StageSpace& sp, int q, int& k, int& j) {
    if (SYM) {
        const int qg = sp.q0 + q;
        k = sym_chunk(qg, sp.nc);
        j = qg - 4 * k * (k + 1);
    } else {
        const int qg = sp.q0 + q;
        k = qg / sp.n_act;
        j = qg - k * sp.n_act;
    }
}

template <bool SYM>
__device__ __forceinline__ int stage_tx(const StageSpace& sp, int j) {
    return SYM ? sp.er.x + j : sp.tlist[j];
}

// Scan raw stages [base, base + kTableBatch) of the stage space: the windows
// that reach the record are appended in order to the ring `st` at position
// `live`.  Called by every thread of the CTA (two barriers); returns the number
// appended (block-uniform).  s_cnt: kTableBatch / 32 ints of shared scratch.
template <int MODE, bool SYM>
__device__ __forceinline__ int fill_stages(const DasArgs& a, const TileGeo& tg, const Elem* el,
                                           const StageSpace& sp, Stage* st, int* s_cnt, int base,
                                           int live) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = base + tid;
    bool keep = false;
    Stage e{};
    if (tid < kTableBatch && q < sp.n_stages) {
        int k, j;
        locate_stage<SYM>(sp, q, k, j);
        const int t = stage_tx<SYM>(sp, j);
        const int rr0 = sp.er.x + k * kC, rrl = min(rr0 + kC - 1, sp.er.y);
        const TxInfo& ti = a.tx[t];
        float mn = 3.0e38f, mx = -3.0e38f;
        for (int rr = SYM ? max(rr0, t) : rr0; rr <= rrl; ++rr) {
            const float2 bd = pair_bounds<MODE>(a.g, ti, rr, tg.xlo, tg.xhi, tg.zlo, tg.zhi);
            mn = fminf(mn, bd.x);
            mx = fmaxf(mx, bd.y);
        }
        const DF txref = tx_ref<MODE>(ti, tg.cx, tg.cz,
                                      MODE == 0 ? elem_R(el[ti.e - sp.er.x]) : DF{0.0f, 0.0f});
        const StageInfo si = make_stage(a, mn, mx, txref, elem_R(el[rr0 - sp.er.x]));
        keep = !si.skip();
        e = pack_stage(si, k, j);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0 && warp < kTableBatch / 32) s_cnt[warp] = __popc(bal);
    __syncthreads();
    int off = __popc(bal & ((1u << lane) - 1u)), total = 0;
#pragma unroll
    for (int w = 0; w < kTableBatch / 32; ++w) {
        if (w < warp) off += s_cnt[w];
        total += s_cnt[w];
    }
    if (keep) st[(live + off) & (kTableStages - 1)] = e;
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// Stage staging shared by the forward and reverse tiled kernels: the raw windows of
// a stage (transmit t, receive chunk r0 .. r_last) go into a ring slot laid out
// [rows][W + 8] (rows = 8, or 16 with the mirrored traces of reciprocal STAI) and
// are then converted to FP32 pairs (x[n], x[n+1] - x[n]).
// ---------------------------------------------------------------------------

// Issue the copies of one stage into `slot`, completion on `bar`; called by every lane of
// one warp.  Tensor maps: one box per direction, by lane 0 (samples outside the record and
// rows outside the array arrive as zeros).  Otherwise one bulk copy per trace row (lanes
// 0..7, mirrored rows lanes 8..15), of the part inside the record.
template <typename T, bool SYM>
__device__ __forceinline__ void stage_issue(const DasArgs& a, const T* rf_frame, T* slot, const Stage& si,
                                            int t, int r0, int r_last, int frame,
                                            unsigned long long* bar, int lane) {
    const int BL = a.W + 8;   // raw row stride (samples)
    if (a.use_tmap) {
        if (lane == 0) {
            const int fr = frame * a.n_tx;
            const unsigned box = (unsigned)(kC * BL) * (unsigned)sizeof(T);
            // the slot's previous contents were read by every thread before a CTA barrier;
            // a tensor copy's writes need no proxy fence after generic reads
            mbar_arrive_expect(bar, SYM ? 2u * box : box);
            tensor_copy_4d(slot, &a.tm_rows, 0, si.lo >> 3, r0, fr + t, bar);
            if (SYM) tensor_copy_4d(slot + kC * BL, &a.tm_cols, 0, si.lo >> 3, t, fr + r0, bar);
        }
        __syncwarp();
        return;
    }
    const int nrow = r_last - r0 + 1;
    const int na = max(si.lo, 0), nb = min(si.lo + si.len + 8, a.ns);
    const int ca = SYM ? max(t - r0, 0) : 0;        // first chunk row paired with t
    const int cb = SYM ? max(t - r0 + 1, 0) : nrow;  // first row with a mirrored trace
    const unsigned bytes = nb > na ? (unsigned)((nb - na) * (int)sizeof(T)) : 0u;
    if (lane == 0) mbar_arrive_expect(bar, bytes * (unsigned)((nrow - ca) + (nrow - cb)));
    __syncwarp();
    if (bytes == 0u) return;
    const long long E = a.g.n_elements;
    const int c = lane & (kC - 1);
    if (lane < kC && c >= ca && c < nrow) {
        fence_async_shared();
        bulk_copy_g2s(slot + c * BL + (na - si.lo), rf_frame + ((long long)t * E + r0 + c) * a.ns + na,
                      bytes, bar);
    } else if (SYM && lane >= kC && lane < 2 * kC && c >= cb && c < nrow) {
        fence_async_shared();
        bulk_copy_g2s(slot + (kC + c) * BL + (na - si.lo), rf_frame + ((long long)(r0 + c) * E + t) * a.ns + na,
                      bytes, bar);
    }
}

// floor(i / n) = (i * ceil(2^16 / n)) >> 16 for every segment count n in 1..64 (a window
// holds at most kMaxWindow / 8 segments) and every i < 8 n + 256 (checked exhaustively): an
// integer multiply and shift instead of a reciprocal and two conversions per segment.
struct RowDiv {
    unsigned m[kMaxWindow / 8 + 1];
    constexpr RowDiv() : m{} {
        for (int n = 1; n <= kMaxWindow / 8; ++n) m[n] = (unsigned)((65536 + n - 1) / n);
    }
};
__constant__ constexpr RowDiv kRowDiv{};

// Convert the raw windows of a stage in `slot` into FP32 pairs in `buf` ([kC][W]); called by
// every thread of the CTA (kThreads).  One 8-sample segment per thread and round.
// Reciprocal STAI (two traces per row): row c = warp, segment kk = lane [+ 32].  Otherwise
// the (row, segment) pairs are numbered row-major and thread tid takes number tid [+ 256]:
// a window of up to 32 segments costs each thread at most one segment (plane-wave windows
// have at most ~21).  Rows outside the chunk, or below the diagonal of a reciprocal pair,
// are zero.
template <typename T, bool SYM>
__device__ __forceinline__ void stage_convert(const DasArgs& a, const T* slot, float2* buf, const Stage& si,
                                              int t, int r0, int r_last) {
    static_assert(kThreads / 32 == kC, "one staged trace row per warp");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BL = a.W + 8;   // raw row stride (samples)
    const int nseg = si.len >> 3;
    const unsigned mdiv = kRowDiv.m[nseg];   // row = floor(idx / nseg) = (idx mdiv) >> 16
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        int c, kk;
        if (SYM) {
            c = warp;
            kk = lane + 32 * i;
            if (kk >= nseg) continue;
        } else {
            const int idx = tid + kThreads * i;
            if (idx >= kC * nseg) continue;
            c = (int)(((unsigned)idx * mdiv) >> 16);
            kk = idx - c * nseg;
        }
        float2* dst = buf + c * a.W + 8 * kk;
        const bool on = r0 + c <= r_last && (!SYM || r0 + c >= t);
        if (!on) {
            zero_segment(dst);
        } else {
            Seg<T> sa;
            seg_load_smem<T>(sa, slot + c * BL, kk);
            if (SYM && r0 + c > t) {
                Seg<T> sb;
                seg_load_smem<T>(sb, slot + (kC + c) * BL, kk);
                seg_store_sum<T>(sa, sb, dst, si.lo + 8 * kk, a.ns);
            } else {
                seg_store<T>(sa, dst, si.lo + 8 * kk, a.ns);
            }
        }
    }
}

template <int MODE, typename T, int WCOL, int P, bool DB, bool TMA, bool CHECK, bool SYM>
__global__ void __launch_bounds__(kThreads, 2) das_tiled_kernel(const __grid_constant__ DasArgs a) {
    static_assert(!SYM || MODE == 0, "reciprocal pairing is an STAI property");
    using S = Shape<WCOL, P>;
    constexpr int kRawRows = SYM ? 2 * kC : kC;   // raw trace rows per ring slot
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SmemLayout L = smem_layout(a.W, a.g.n_elements, DB, TMA, SYM, a.ring, (int)sizeof(T));
    float2* buf0 = reinterpret_cast<float2*>(smem_raw + L.pairs);   // [DB+1][kC][W] pairs
    Stage* st = reinterpret_cast<Stage*>(smem_raw + L.table);        // ring of compacted stages
    Elem* el = reinterpret_cast<Elem*>(smem_raw + L.elems);         // [E range]
    // [ring][kRawRows][W + 8] raw samples, 128-byte aligned for the tensor copies
    const unsigned raw_pad = (128u - (smem_u32(smem_raw) & 127u)) & 127u;   // L.total keeps 128 B slack
    T* raw = reinterpret_cast<T*>(smem_raw + raw_pad + L.raw);
    __shared__ __align__(8) unsigned long long s_bar[kMaxRing];
    __shared__ int s_tlist[WF_MAX_TX];
    __shared__ int s_info[4];
    __shared__ int s_cnt[kTableBatch / 32];

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = lane % WCOL, lz = lane / WCOL;
    const int item = blockIdx.x, b = blockIdx.y;
    int group, n_grp, tzi, txi;
    if (a.use_table) {
        const unsigned code = a.items[item];
        const int tile = (int)(code & 0xffffu);
        group = (int)((code >> 16) & 0xffu);
        n_grp = (int)(code >> 24);
        tzi = tile / a.tiles_x;
        txi = tile - tzi * a.tiles_x;
        if (b == 0 && tid == 0 && group == 0) a.tile_info[tile] = (unsigned)(item + 1) | ((unsigned)n_grp << 24);
    } else {
        group = item % a.n_groups;
        n_grp = a.n_groups;
        const int rank = item / a.n_groups;
        tzi = a.tiles_z - 1 - rank / a.tiles_x;
        txi = rank % a.tiles_x;
    }
    const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, txi * S::kCols, tzi * S::kRows);
    const T* rf = reinterpret_cast<const T*>(a.rf) + (long long)b * a.frame_elems;
    const bool vec_ok = (a.ns & 7) == 0;
    const int SLOT = kRawRows * (a.W + 8);          // samples per ring slot: [kRawRows][W + 8]
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

    const int2 er = tg.er;
    const int n_e = er.y >= er.x ? er.y - er.x + 1 : 0;
    const int nc = (n_e + kC - 1) / kC;
    for (int e = er.x + tid; e <= er.y; e += kThreads) el[e - er.x] = make_elem(a, tg.cx, tg.cz, e);
    if (tid == 0) {
        int n = 0;
        if (!SYM && n_e > 0)
            for (int t = 0; t < a.n_tx; ++t) {
                if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
                s_tlist[n++] = t;
            }
        // This group's share of the tile's raw stage list (chunk-major, every transmit
        // per chunk): equal raw-stage ranges, so a heavy chunk can span several groups.
        const long long G = n_grp;
        const long long n_raw = n_e == 0 ? 0 : SYM ? sym_prefix(nc, nc, n_e) : (long long)nc * n;
        const int qa = (int)((long long)group * n_raw / G), qb = (int)((long long)(group + 1) * n_raw / G);
        s_info[0] = n;
        s_info[1] = qa;
        s_info[2] = qb;
        if (TMA) {
            for (int i = 0; i < ring; ++i) mbar_init(&s_bar[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            if (a.use_tmap) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&a.tm_rows))
                             : "memory");
                if (SYM)
                    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(&a.tm_cols))
                                 : "memory");
            }
        }
    }
    __syncthreads();
    const int n_act = s_info[0], q0 = s_info[1], n_stages = s_info[2] - s_info[1];

    const StageSpace sp{er, n_e, nc, n_act, q0, n_stages, s_tlist};
    auto tx_of = [&](int j) { return stage_tx<SYM>(sp, j); };
    int n_live = 0, raw_next = 0;
    // Make entry `upto` of the compacted list exist while raw stages are left (all threads).
    auto need = [&](int upto) {
        while (n_live <= upto && raw_next < n_stages) {
            n_live += fill_stages<MODE, SYM>(a, tg, el, sp, st, s_cnt, raw_next, n_live);
            raw_next += kTableBatch;
        }
    };
    // TMA producer (warp kIssueWarp): raw windows of entry qq into ring slot qq % ring (slot).
    auto issue = [&](int qq, int slot) {
        const Stage si = st[qq & (kTableStages - 1)];
        const int t = tx_of(si.j());
        const int rr0 = er.x + si.k() * kC;
        stage_issue<T, SYM>(a, rf, raw + (size_t)slot * SLOT, si, t, rr0, min(rr0 + kC - 1, er.y),
                            b, &s_bar[slot], lane);
    };
    const int ahead = TMA ? ring - 1 : 1;   // stages in flight ahead of the one being converted
    need(ahead - 1);

    // PWI: range of the transmit correction ux sin + uz cos over this warp's pixels.
    const float wux0 = (float)(WCOL * warp) * g.gdx, wux1 = (float)(WCOL * warp + WCOL - 1) * g.gdx;
    const float wuz1 = (float)(S::kRows - 1) * g.gdz;

    static_assert(P % 2 == 0, "pixels per lane are processed in packed pairs");
    constexpr int H = P / 2;
    float acc[P];
#pragma unroll
    for (int p = 0; p < P; ++p) acc[p] = 0.0f;
    f32x2 Dr2[kC][H], Wr2[kC][H];   // receive distances / weights of pixel pairs (2h, 2h + 1)
    float dr_min = 0.0f, dr_max = 0.0f;
    unsigned cmask = 0u;
    RegStage<T, SYM> rs;
    const f32x2 kMagic2 = x2_pack(kMagic, kMagic);

    if (TMA) {
        if (warp == kIssueWarp)
            for (int qq = 0; qq < min(ahead, n_live); ++qq) issue(qq, qq);   // ahead < ring
    } else if (n_live > 0) {
        const Stage s0 = st[0];
        const int rr0 = er.x + s0.k() * kC;
        stage_prefetch<T, SYM>(rs, a, rf, s0, tx_of(s0.j()), rr0, min(rr0 + kC - 1, er.y), vec_ok);
    }

    int k_cur = -1;
    // Ring slot q % ring and mbarrier phase (q / ring) & 1 of stage q, advanced per stage: the
    // ring depth is a run-time value, and a division by it in every thread and stage cost 4 %
    // of full PWI.
    int slot_n = 0;
    unsigned phase_n = 0u;
    for (int q = 0; q < n_live; ++q) {
        const int slot_q = slot_n;
        const unsigned phase_q = phase_n;
        if (++slot_n == ring) {
            slot_n = 0;
            phase_n ^= 1u;
        }
        if (TMA) {
            // Stage q + ahead goes to ring slot (q - 1) % ring, whose raw samples every thread
            // converted before the previous barrier.  Issued by warp kIssueWarp before the
            // conversion of stage q: the last warp has no conversion work for windows of at
            // most 28 segments (every plane-wave window), so the copy issue leaves the stage's
            // critical path.
            need(q + ahead);
            if (warp == kIssueWarp && q + ahead < n_live)
                issue(q + ahead, slot_q + ahead < ring ? slot_q + ahead : slot_q + ahead - ring);
        }
        const Stage si = st[q & (kTableStages - 1)];
        const int k = si.k();
        const int r0 = er.x + k * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        const int t = tx_of(si.j());
        float2* buf = buf0 + (DB ? (q & 1) * kC * a.W : 0);
        if (si.over() && tid == 0) flag(a.hdr, 1u, (unsigned)blockIdx.x, (unsigned)si.len, (unsigned)a.W);
        bool stuck = false;
        if (TMA) {
            stuck = !mbar_wait_bounded(&s_bar[slot_q], phase_q);
            if (!stuck) {
                stage_convert<T, SYM>(a, raw + (size_t)slot_q * SLOT, buf, si, t, r0, r_last);
            }
        } else {
            stage_store<T, SYM>(rs, buf, a, si, t, r0, r_last);
        }
        // pairs of stage q visible; raw slot of stage q - 1 and (double-buffered) pairs of q - 1 free
        if (__syncthreads_or(stuck)) {
            // A copy never completed: record it, let the copies still in flight land
            // (bounded), and leave the stage loop together.
            if (tid == 0) {
                flag(a.hdr, 4u, (unsigned)blockIdx.x, (unsigned)q, 0u);
                for (int qq = q + 1; qq < min(q + ahead + 1, n_live); ++qq)   // issued up to q + ahead
                    mbar_wait_bounded(&s_bar[qq % ring], (unsigned)((qq / ring) & 1));
            }
            break;
        }
        if (!TMA) {
            need(q + ahead);
            if (q + ahead < n_live) {
                const Stage s1 = st[(q + 1) & (kTableStages - 1)];
                const int rr0 = er.x + s1.k() * kC;
                stage_prefetch<T, SYM>(rs, a, rf, s1, tx_of(s1.j()), rr0, min(rr0 + kC - 1, er.y), vec_ok);
            }
        }
        if (k != k_cur) {
            k_cur = k;
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
                    float d[P], w[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        d[p] = on ? cc + dist_delta(ee, ux, kz[p]) : 0.0f;
                        w[p] = on ? apod_w(g.apod, -(ee.ax + ux), kap[p]) * (ee.g * a.rf_scale) : 0.0f;
                        if (on) {
                            mn = fminf(mn, d[p]);
                            mx = fmaxf(mx, d[p]);
                        }
                    }
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        Dr2[c][h] = x2_pack(d[2 * h], d[2 * h + 1]);
                        Wr2[c][h] = x2_pack(w[2 * h], w[2 * h + 1]);
                    }
                }
                dr_min = warp_min(mn);
                dr_max = warp_max(mx);
            }
        }
        // Warp-level skip: transmit or chunk outside this warp's aperture, or every
        // delay of the warp outside the record (tested only for windows that cross
        // an end of the record).
        unsigned cm = cmask;
        if (SYM && t > r0) cm &= ~((1u << (t - r0)) - 1u);   // pairs below the diagonal
        bool live = cm != 0u;
        if (MODE == 0) live = live && a.tx[t].e >= wr.x && a.tx[t].e <= wr.y;
        float tw[P], wt[P];
        if (live) {
            if (MODE == 0) {
                const Elem et = el[a.tx[t].e - er.x];
                float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tw[p] = si.B + dist_delta(et, ux, kz[p]);
                    wt[p] = apod_w(g.apod, -(et.ax + ux), kap[p]) * et.g;
                    mn = fminf(mn, tw[p]);
                    mx = fmaxf(mx, tw[p]);
                }
                if (si.edge()) {
                    mn = warp_min(mn);
                    mx = warp_max(mx);
                    live = ((float)si.lo + mn + dr_min <= (float)(a.ns - 1) + 0.5f) &&
                           ((float)si.lo + mx + dr_max >= -0.5f);
                }
            } else {
                const float sn = a.tx[t].sin_f, cs = a.tx[t].cos_f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tw[p] = si.B + fmaf(ux, sn, uz[p] * cs);
                    wt[p] = 1.0f;
                }
                if (si.edge()) {
                    const float v0 = wux0 * sn, v1 = wux1 * sn, z1 = wuz1 * cs;
                    const float lo_f = (float)si.lo + si.B;
                    live = (lo_f + fminf(v0, v1) + fminf(0.0f, z1) + dr_min <= (float)(a.ns - 1) + 0.5f) &&
                           (lo_f + fmaxf(v0, v1) + fmaxf(0.0f, z1) + dr_max >= -0.5f);
                }
            }
        }
        if (live) {
            // Per pixel: s = tw + Dr, i = floor(s) by the round-down add of 1.5 * 2^23,
            // f = s - i, v = x[i] + f (x[i+1] - x[i]), acc += Wr v -- the delay, floor
            // and fraction two pixels per packed instruction; the interpolation and the
            // weighted sum in scalar FMAs, which read the gathered pairs where they landed.
            f32x2 tw2[H];
            float accs[P];   // this stage's sums per pixel
#pragma unroll
            for (int h = 0; h < H; ++h) {
                tw2[h] = x2_pack(tw[2 * h], tw[2 * h + 1]);
                accs[2 * h] = 0.0f;
                accs[2 * h + 1] = 0.0f;
            }
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                if (!((cm >> c) & 1u)) continue;
                const float2* bc = buf + c * a.W;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const f32x2 s2 = x2_add(tw2[h], Dr2[c][h]);
                    const f32x2 m2 = x2_add_rm(s2, kMagic2);
                    const f32x2 f2 = x2_sub(s2, x2_sub(m2, kMagic2));
                    float m0, m1;
                    x2_unpack(m2, m0, m1);
                    int i0 = __float_as_int(m0) - kMagicBits, i1 = __float_as_int(m1) - kMagicBits;
                    if (CHECK && (i0 < 0 || i0 >= si.len || i1 < 0 || i1 >= si.len)) {
                        flag(a.hdr, 2u, (unsigned)blockIdx.x, (unsigned)min(i0, i1), (unsigned)si.len);
                        i0 = 0;
                        i1 = 0;
                    }
                    const float2 a0 = bc[i0], a1 = bc[i1];
                    float f0, f1;
                    x2_unpack(f2, f0, f1);
                    // weight and sum per pixel in scalar FMAs (the same rounding as a packed
                    // FMA, without re-pairing the two interpolated values into one register pair)
                    float w0, w1;
                    x2_unpack(Wr2[c][h], w0, w1);
                    accs[2 * h] = fmaf(w0, fmaf(f0, a0.y, a0.x), accs[2 * h]);
                    accs[2 * h + 1] = fmaf(w1, fmaf(f1, a1.y, a1.x), accs[2 * h + 1]);
                }
            }
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float t0 = accs[2 * h], t1 = accs[2 * h + 1];
                acc[2 * h] = MODE == 0 ? fmaf(wt[2 * h], t0, acc[2 * h]) : acc[2 * h] + t0;
                acc[2 * h + 1] = MODE == 0 ? fmaf(wt[2 * h + 1], t1, acc[2 * h + 1]) : acc[2 * h + 1] + t1;
            }
        }
        if (!DB) __syncthreads();   // single buffer: compute of stage q done before stage q + 1 lands
    }

    // Partial tile in thread order: [p][tid].
    float* dst = a.part + ((long long)b * a.n_items + item) * (kThreads * P);
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p * kThreads + tid] = acc[p];
}

// Sum the chunk-group partials of every pixel in group order.  With a
// work-proportional schedule (tile_info != null) a tile's groups are the items
// recorded in tile_info; a tile without items has no stage inside the record.
template <int WCOL, int P>
__global__ void das_reduce_kernel(const float* __restrict__ part, const unsigned* __restrict__ tile_info,
                                  float* __restrict__ out, int nz, int nx, int tiles_x, int tiles_z,
                                  int n_groups, int n_items) {
    using S = Shape<WCOL, P>;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= nx) return;
    int first, groups;
    if (tile_info) {
        const unsigned info = tile_info[(iz / S::kRows) * tiles_x + ix / S::kCols];
        first = (int)(info & 0xffffffu) - 1;
        groups = (int)(info >> 24);
        if (info == 0u) groups = 0;
    } else {
        first = tile_rank(iz / S::kRows, ix / S::kCols, tiles_z, tiles_x) * n_groups;
        groups = n_groups;
    }
    const int cl = ix % S::kCols, rl = iz % S::kRows;
    const int tid = (cl / WCOL) * 32 + (rl % S::kLR) * WCOL + (cl % WCOL);
    const int local = (rl / S::kLR) * kThreads + tid;
    float s = 0.0f;
    if (groups > 0) {
        const float* p = part + ((long long)b * n_items + first) * (kThreads * P) + local;
        for (int k = 0; k < groups; ++k) s += p[(long long)k * (kThreads * P)];
    }
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

// ---------------------------------------------------------------------------
// Host-side launch plan and launchers (instantiated per mode and bounds-check
// variant in their own translation units).
// ---------------------------------------------------------------------------
struct Cfg {
    int wcol, p;
};

struct Plan {
    Cfg cfg;
    int cols, rows;
    int tiles_x, tiles_z, n_groups, n_items;   // n_items: uniform groups, or the schedule's count
    int W, ring;
    bool tiled, db, tma, sym;
    bool table;          // a work-proportional schedule fits (budget + tiles <= kMaxItems)
    int budget;          // CTAs per frame the schedule aims for
    size_t info_bytes;   // tile table in the workspace (after the status block)
    size_t smem;
    size_t ws_bytes;
};

constexpr size_t kMaxTiledSmem = 220 * 1024;  // one CTA per SM

template <int MODE, typename T, int WCOL, int P, bool DB, bool TMA, bool CHECK, bool SYM>
wf_status launch_tiled_v(DasArgs& A, const Plan& PL, int batch, cudaStream_t st) {
    static unsigned long long smem_set = 0ull;
    auto kern = das_tiled_kernel<MODE, T, WCOL, P, DB, TMA, CHECK, SYM>;
    wf_status s = ensure_smem_limit(kern, kMaxTiledSmem, smem_set);
    if (s != WF_OK) return s;
    if (A.n_items > 0) {
        kern<<<dim3(A.n_items, batch), kThreads, PL.smem, st>>>(A);
        if ((s = last_launch_status()) != WF_OK) return s;
    }
    dim3 rg((A.g.nx + 127) / 128, A.g.nz, batch);
    das_reduce_kernel<WCOL, P><<<rg, 128, 0, st>>>(A.part, A.use_table ? A.tile_info : nullptr, A.out,
                                                   A.g.nz, A.g.nx, PL.tiles_x, PL.tiles_z, A.n_groups,
                                                   A.n_items);
    return last_launch_status();
}

template <int MODE, typename T, int WCOL, int P, bool CHECK, bool SYM>
wf_status launch_tiled(DasArgs& A, const Plan& PL, int batch, cudaStream_t st) {
    if (!PL.tma) return launch_tiled_v<MODE, T, WCOL, P, false, false, CHECK, SYM>(A, PL, batch, st);
    return PL.db ? launch_tiled_v<MODE, T, WCOL, P, true, true, CHECK, SYM>(A, PL, batch, st)
                 : launch_tiled_v<MODE, T, WCOL, P, false, true, CHECK, SYM>(A, PL, batch, st);
}

template <int MODE, typename T, bool CHECK, bool SYM>
wf_status launch_tiled_cfg(DasArgs& A, const Plan& P, int batch, cudaStream_t st) {
    return P.cfg.p == 4 ? launch_tiled<MODE, T, 4, 4, CHECK, SYM>(A, P, batch, st)
                        : launch_tiled<MODE, T, 4, 2, CHECK, SYM>(A, P, batch, st);
}

// Reverse-mode launcher (das_grad.cu): derivatives of <grad_out, DAS(rf)> with
// respect to the RF, the element weights and the sound speed.
template <int MODE>
wf_status launch_das_backward(DasArgs& A, const Plan& P, int batch, bool need_rf, bool need_par,
                              cudaStream_t st);

// Delay-and-sum of IQ data (das_iq.cu): shared-memory layout, launch (tiled kernel and
// the group reduction into the complex image out [batch][nz][nx][2]) and |B| with frame maxima.
struct IqSmem {
    size_t pairs, rot, table, elems, raw, total;
};
size_t iq_smem_bytes(int W, int n_elements);
template <int MODE>
wf_status launch_das_iq(DasArgs& A, int batch, float* out, cudaStream_t st);
wf_status launch_iq_envelope(const float* img, int batch, long long n_frame, float* env, float* frame_max,
                             cudaStream_t st);

// Whether the reverse-mode launcher takes the tiled kernel for this plan (das_grad.cu).
bool backward_is_tiled(const Plan& P, int n_elements, bool need_rf);

// Tiled launch of one mode and bounds-check variant, every RF type.
template <int MODE, bool CHECK>
wf_status launch_das_tiled(DasArgs& A, const Plan& P, int batch, wf_dtype dt, cudaStream_t st) {
    switch (dt) {
        case WF_F32:
            return P.sym ? launch_tiled_cfg<MODE, float, CHECK, MODE == 0>(A, P, batch, st)
                         : launch_tiled_cfg<MODE, float, CHECK, false>(A, P, batch, st);
        case WF_F16:
            return P.sym ? launch_tiled_cfg<MODE, __half, CHECK, MODE == 0>(A, P, batch, st)
                         : launch_tiled_cfg<MODE, __half, CHECK, false>(A, P, batch, st);
        case WF_I16:
            return P.sym ? launch_tiled_cfg<MODE, int16_t, CHECK, MODE == 0>(A, P, batch, st)
                         : launch_tiled_cfg<MODE, int16_t, CHECK, false>(A, P, batch, st);
    }
    return WF_ERR_INVALID_ARG;
}

}  // namespace wf
