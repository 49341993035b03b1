// Reverse-mode delay-and-sum: derivatives of L = <y, b> for a cotangent y of
// the beamformed image b = DAS(rf; g, c) (a differentiable beamformer, the use
// the paper motivates for learned pipelines, Sec. I and Sec. IV).
//
// For every term (pixel p, transmit t, receive r) of the forward sum, with
// weight W = w_t w_r (STAI; w_e = a_e g_e, a the aperture window) or W = w_r
// (PWI), delay s, floor i, fraction f and 0 <= i <= ns - 2:
//   dL/d rf[t][r][i] += y W (1 - f),   dL/d rf[t][r][i+1] += y W f
//   dL/d g_e        += y (dW/dg_e) lerp          (STAI: e_t and r; PWI: r)
//   dL/d c          += y W (rf[i+1] - rf[i]) ds/dc,  ds/dc = -(s + t0 fs) / c
// (the windows depend on the geometry only, not on c).
//
// GB300 layout: the forward kernel's tiling (tile = reference point of the
// tile-relative geometry, receive chunks of 8, one group of chunks per CTA,
// every transmit per chunk, reciprocal STAI pairs when every element fires in
// order).  Per stage the RF window is staged as FP32 (value, slope) pairs (the
// slope is dlerp/ds); the interpolation transpose is accumulated with
// shared-memory atomics into a window of the same shape and flushed once per
// stage with global atomics (to both traces of a reciprocal pair).  Weight and
// sound-speed sums are reduced per warp, per CTA and then globally.  Global
// float atomics make the summation order (and so the last bits) run-dependent.
#include <type_traits>

#include "das_kernels.cuh"

namespace wf {

__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

constexpr int kBwdWCOL = 4;
constexpr int kBwdP = 2;   // tile 32 x 16 pixels: three weight sets per chunk stay in registers

constexpr int kBwdRing = 3;   // tensor-copy ring depth of the reverse kernel

struct BwdSmem {
    size_t pairs, gwin, table, elems, ge, raw, total;
};

// Shared-memory layout of the reverse kernel; with `ring` > 0 a raw ring of that many
// stage slots ([rows][W + 8] float samples, 128-byte aligned) follows.
__host__ __device__ inline BwdSmem bwd_smem_layout(int W, int n_elements, bool need_rf, int ring = 0,
                                                   bool sym = false) {
    BwdSmem L;
    size_t off = 0;
    L.pairs = off;
    off += (size_t)kC * W * sizeof(float2);
    L.gwin = off;
    off += need_rf ? (size_t)kC * (W + 8) * sizeof(float) : 0;
    L.table = off;
    off += (size_t)kTableStages * sizeof(Stage);
    L.elems = off;
    off += (((size_t)n_elements * sizeof(Elem)) + 15) & ~(size_t)15;
    L.ge = off;
    off += (((size_t)n_elements * sizeof(float)) + 15) & ~(size_t)15;
    off = (off + 127) & ~(size_t)127;
    L.raw = off;
    if (ring > 0) off += (size_t)ring * (sym ? 2 : 1) * kC * (W + 8) * sizeof(float) + 128;   // + align slack
    L.total = off;
    return L;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int MODE, bool SYM, bool NEED_RF, bool NEED_PAR, bool TMA>
__global__ void __launch_bounds__(kThreads, 2) das_backward_kernel(const __grid_constant__ DasArgs a) {
    static_assert(!SYM || MODE == 0, "reciprocal pairing is an STAI property");
    constexpr int WCOL = kBwdWCOL, P = kBwdP;
    constexpr int kRawRows = SYM ? 2 * kC : kC;
    using S = Shape<WCOL, P>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BwdSmem L = bwd_smem_layout(a.W, a.g.n_elements, NEED_RF, TMA ? kBwdRing : 0, SYM);
    // tensor-copy ring: [kBwdRing][kRawRows][W + 8] raw samples, 128-byte aligned
    const unsigned raw_pad = (128u - (smem_u32(smem_raw + L.raw) & 127u)) & 127u;
    float* raw = reinterpret_cast<float*>(smem_raw + L.raw + raw_pad);
    const int SLOT = kRawRows * (a.W + 8);
    __shared__ __align__(8) unsigned long long s_bar[kBwdRing];
    float2* buf = reinterpret_cast<float2*>(smem_raw + L.pairs);   // [kC][W] (value, slope)
    int* gw = reinterpret_cast<int*>(smem_raw + L.gwin);           // [kC][W + 8] RF cotangent window (fixed point)
    Stage* st = reinterpret_cast<Stage*>(smem_raw + L.table);      // ring of compacted stages
    Elem* el = reinterpret_cast<Elem*>(smem_raw + L.elems);        // [E range]
    float* ge = reinterpret_cast<float*>(smem_raw + L.ge);         // [E range] weight-gradient partials
    __shared__ int s_tlist[WF_MAX_TX];
    __shared__ int s_info[4];
    __shared__ float s_red[kThreads / 32];
    __shared__ float s_gm[kThreads / 32];
    __shared__ int s_cnt[kTableBatch / 32];

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = lane % WCOL, lz = lane / WCOL;
    const int item = blockIdx.x, b = blockIdx.y;
    const int group = item % a.n_groups, rank = item / a.n_groups;
    const int tzi = a.tiles_z - 1 - rank / a.tiles_x, txi = rank % a.tiles_x;
    const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, txi * S::kCols, tzi * S::kRows);
    const float* rf = reinterpret_cast<const float*>(a.rf) + (long long)b * a.frame_elems;
    float* grf = NEED_RF ? a.grad_rf + (long long)b * a.frame_elems : nullptr;
    const bool vec_ok = (a.ns & 7) == 0;
    const int GW = a.W + 8;   // cotangent window row stride (a multiple of 8 floats)
    const bool vec4 = NEED_RF && (a.ns & 3) == 0 && ((uintptr_t)a.grad_rf & 15u) == 0;
    const long long E = g.n_elements;

    const int col = WCOL * warp + lx;
    const float ux = (float)col * g.gdx;
    float kz[P], kap[P], uz[P], y[P];
    const float* yb = a.grad_out + (long long)b * g.nz * g.nx;
#pragma unroll
    for (int p = 0; p < P; ++p) {
        uz[p] = (float)(lz + S::kLR * p) * g.gdz;
        kz[p] = uz[p] * fmaf(2.0f, tg.cz.hi, uz[p]);
        kap[p] = aperture_kappa(g, tg.cz.hi + uz[p]);
        const int ix = tg.ix0 + col, iz = tg.iz0 + lz + S::kLR * p;
        y[p] = (ix < g.nx && iz < g.nz) ? __ldg(yb + (long long)iz * g.nx + ix) : 0.0f;
    }
    const int2 wr = tile_elements(g, pixel_x(g, tg.ix0 + WCOL * warp),
                                  pixel_x(g, tg.ix0 + WCOL * warp + WCOL - 1), tg.zhi);
    const int2 er = tg.er;
    const int n_e = er.y >= er.x ? er.y - er.x + 1 : 0;
    const int nc = (n_e + kC - 1) / kC;
    float gmax = 0.0f;
    for (int e = er.x + tid; e <= er.y; e += kThreads) {
        el[e - er.x] = make_elem(a, tg.cx, tg.cz, e);
        ge[e - er.x] = 0.0f;
        gmax = fmaxf(gmax, fabsf(el[e - er.x].g));
    }
    if (NEED_RF)
        for (int i = tid; i < kC * GW; i += kThreads) gw[i] = 0;
    // Fixed-point scale of the RF cotangent window.  A contribution is y W times
    // (1 - f) or f, |y W| <= ymax wmax (windows <= 1), and one window position
    // collects at most one unit-weight share per pixel of the tile, so with
    // scale = 2^21 / (ymax wmax) every contribution rounds exactly through the
    // 1.5 * 2^23 add and no 32-bit sum can overflow (256 P pixels <= 2^9).
    // Shared-memory integer atomics run about three times the rate of float ones.
    float scale = 0.0f, inv_scale = 0.0f;
    if (NEED_RF) {
        float ym = 0.0f;
#pragma unroll
        for (int p = 0; p < P; ++p) ym = fmaxf(ym, fabsf(y[p]));
        ym = warp_max(ym);
        const float gm = warp_max(gmax);
        if (lane == 0) {
            s_red[warp] = ym;
            s_gm[warp] = gm;
        }
        __syncthreads();
        float ymax = 0.0f, wmax = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) {
            ymax = fmaxf(ymax, s_red[w]);
            wmax = fmaxf(wmax, s_gm[w]);
        }
        if (MODE == 0) wmax *= wmax;   // transmit and receive weights
        const float m = ymax * wmax;
        if (m > 0.0f && m < 3.0e38f) {
            scale = 2097152.0f / m;
            inv_scale = m * (1.0f / 2097152.0f);
        }
        static_assert(kThreads * P <= 512, "fixed-point headroom assumes at most 512 pixels per tile");
    }
    if (tid == 0) {
        int n = 0;
        if (!SYM && n_e > 0)
            for (int t = 0; t < a.n_tx; ++t) {
                if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
                s_tlist[n++] = t;
            }
        // This group's share of the tile's raw stage list (chunk-major, every transmit
        // per chunk): equal raw-stage ranges, so a heavy chunk can span several groups.
        const long long G = a.n_groups;
        const long long n_raw = n_e == 0 ? 0 : SYM ? sym_prefix(nc, nc, n_e) : (long long)nc * n;
        const int qa = (int)((long long)group * n_raw / G), qb = (int)((long long)(group + 1) * n_raw / G);
        s_info[0] = n;
        s_info[1] = qa;
        s_info[2] = qb;
        if (TMA) {
            for (int i = 0; i < kBwdRing; ++i) mbar_init(&s_bar[i], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();
    const int n_act = s_info[0], q0 = s_info[1], n_stages = s_info[2] - s_info[1];

    const StageSpace sp{er, n_e, nc, n_act, q0, n_stages, s_tlist};
    auto tx_of = [&](int j) { return stage_tx<SYM>(sp, j); };
    int n_live = 0, raw_next = 0;
    auto need = [&](int upto) {   // make entry `upto` exist while raw stages are left
        while (n_live <= upto && raw_next < n_stages) {
            n_live += fill_stages<MODE, SYM>(a, tg, el, sp, st, s_cnt, raw_next, n_live);
            raw_next += kTableBatch;
        }
    };
    constexpr int ahead = TMA ? kBwdRing - 1 : 1;   // stages in flight ahead of the one converted
    need(ahead - 1);
    // Copies of stage qq into ring slot qq % kBwdRing (warp kIssueWarp).
    auto issue = [&](int qq) {
        const Stage s1 = st[qq & (kTableStages - 1)];
        const int t1 = tx_of(s1.j()), rr0 = er.x + s1.k() * kC;
        stage_issue<float, SYM>(a, rf, raw + (size_t)(qq % kBwdRing) * SLOT, s1, t1, rr0,
                                min(rr0 + kC - 1, er.y), b, &s_bar[qq % kBwdRing], lane);
    };

    // Per receive row c of the chunk, packed pixel pairs (2h, 2h + 1): distance Dr,
    // weight Wr = a_r g_r and window Ar = a_r (PWI: both times the cotangent y, which
    // does not depend on the transmit), and the weight-gradient partial gR.
    static_assert(P % 2 == 0, "pixels per lane are processed in packed pairs");
    constexpr int H = P / 2;
    f32x2 Dr2[kC][H], Wr2[kC][H], Ar2[kC][H];
    float gR[kC];
    float dr_min = 0.0f, dr_max = 0.0f, accC = 0.0f;
    unsigned cmask = 0u;
    RegStage<float, SYM> rs;
    const f32x2 kMagic2 = x2_pack(kMagic, kMagic), scale2 = x2_pack(scale, scale);
    // Weight-gradient partials of the current chunk -> shared per-element sums.
    auto flush_chunk = [&](int r0c) {
        if (!NEED_PAR || cmask == 0u) return;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
            if (!((cmask >> c) & 1u)) continue;
            const float v = warp_sum(gR[c]);
            if (lane == 0 && v != 0.0f) atomicAdd(&ge[r0c + c - er.x], v);
        }
    };

    if (TMA) {
        if (warp == kIssueWarp)
            for (int qq = 0; qq < min(ahead, n_live); ++qq) issue(qq);
    } else if (n_live > 0) {
        const Stage s0 = st[0];
        const int rr0 = er.x + s0.k() * kC;
        stage_prefetch<float, SYM>(rs, a, rf, s0, tx_of(s0.j()), rr0, min(rr0 + kC - 1, er.y), vec_ok);
    }
    int k_cur = -1;
    for (int q = 0; q < n_live; ++q) {
        if (TMA) {
            // stage q + ahead goes to ring slot (q - 1) % kBwdRing, converted before the
            // barriers of stage q - 1
            need(q + ahead);
            if (warp == kIssueWarp && q + ahead < n_live) issue(q + ahead);
        }
        const Stage si = st[q & (kTableStages - 1)];
        const int k = si.k();
        const int r0 = er.x + k * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        const int t = tx_of(si.j());
        bool stuck = false;
        if (TMA) {
            stuck = !mbar_wait_bounded(&s_bar[q % kBwdRing], (unsigned)((q / kBwdRing) & 1));
            if (!stuck) stage_convert<float, SYM>(a, raw + (size_t)(q % kBwdRing) * SLOT, buf, si, t, r0, r_last);
        } else {
            stage_store<float, SYM>(rs, buf, a, si, t, r0, r_last);
        }
        // pairs of stage q visible; cotangent window zero
        if (__syncthreads_or(stuck)) {
            // A copy never completed: let the copies still in flight land (bounded) and leave
            // the stage loop together; the gradients are then incomplete (the call's result is
            // unspecified, as for the forward kernels' timeouts).
            if (tid == 0)
                for (int qq = q + 1; qq < min(q + ahead + 1, n_live); ++qq)
                    mbar_wait_bounded(&s_bar[qq % kBwdRing], (unsigned)((qq / kBwdRing) & 1));
            break;
        }
        if (!TMA) {
            need(q + 1);
            if (q + 1 < n_live) {
                const Stage s1 = st[(q + 1) & (kTableStages - 1)];
                const int rr0 = er.x + s1.k() * kC;
                stage_prefetch<float, SYM>(rs, a, rf, s1, tx_of(s1.j()), rr0, min(rr0 + kC - 1, er.y), vec_ok);
            }
        }
        if (k != k_cur) {
            if (k_cur >= 0) flush_chunk(er.x + k_cur * kC);
            k_cur = k;
            cmask = 0u;
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                gR[c] = 0.0f;
                if (r0 + c <= r_last && r0 + c >= wr.x && r0 + c <= wr.y) cmask |= 1u << c;
            }
            if (cmask) {
                const Elem e0 = el[r0 - er.x];
                float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
                for (int c = 0; c < kC; ++c) {
                    const bool on = (cmask >> c) & 1u;
                    const Elem ee = el[(on ? r0 + c : r0) - er.x];
                    const float cc = elem_rel(ee, e0);
                    float d[P], ar[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        d[p] = on ? cc + dist_delta(ee, ux, kz[p]) : 0.0f;
                        ar[p] = on ? apod_w(g.apod, -(ee.ax + ux), kap[p]) : 0.0f;
                        if (on) {
                            mn = fminf(mn, d[p]);
                            mx = fmaxf(mx, d[p]);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        if (MODE == 1) ar[p] *= y[p];
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        Dr2[c][h] = x2_pack(d[2 * h], d[2 * h + 1]);
                        Ar2[c][h] = x2_pack(ar[2 * h], ar[2 * h + 1]);
                        Wr2[c][h] = x2_pack(ar[2 * h] * ee.g, ar[2 * h + 1] * ee.g);
                    }
                }
                dr_min = warp_min(mn);
                dr_max = warp_max(mx);
            }
        }
        unsigned cm = cmask;
        if (SYM && t > r0) cm &= ~((1u << (t - r0)) - 1u);
        bool live = cm != 0u;
        if (MODE == 0) live = live && a.tx[t].e >= wr.x && a.tx[t].e <= wr.y;
        float tw[P], yt[P], ya[P];
        if (live) {
            if (MODE == 0) {
                const Elem et = el[a.tx[t].e - er.x];
                float mn = 3.0e38f, mx = -3.0e38f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tw[p] = si.B + dist_delta(et, ux, kz[p]);
                    const float at = apod_w(g.apod, -(et.ax + ux), kap[p]);
                    ya[p] = y[p] * at;          // y a_t: transmit-weight gradient
                    yt[p] = ya[p] * et.g;       // y w_t
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
                    yt[p] = y[p];
                    ya[p] = 0.0f;
                }
            }
        }
        if (live) {
            const TxInfo& ti = a.tx[t];
            const float base_c = (float)si.lo + (ti.t0.hi + ti.t0.lo);   // s + base_c = path in samples
            const f32x2 base2 = x2_pack(base_c, base_c);
            f32x2 tw2[H], yt2[H], ya2[H], gT2 = 0ull;
#pragma unroll
            for (int h = 0; h < H; ++h) {
                tw2[h] = x2_pack(tw[2 * h], tw[2 * h + 1]);
                yt2[h] = MODE == 0 ? x2_pack(yt[2 * h], yt[2 * h + 1]) : 0ull;
                ya2[h] = MODE == 0 ? x2_pack(ya[2 * h], ya[2 * h + 1]) : 0ull;
            }
            // Per pixel pair and receive row: s = tw + Dr, i = floor(s), f = s - i,
            // v = x[i] + f x'[i]; the RF cotangent y W (1 - f), y W f goes to window
            // positions i, i + 1 in fixed point.  EDGE: the window crosses an end of
            // the record, and terms without two recorded samples drop out (elsewhere
            // every staged pair is inside the record).
            auto terms = [&](auto edge_tag) {
                constexpr bool EDGE = decltype(edge_tag)::value;
                const unsigned lim = (unsigned)(a.ns - 2);
#pragma unroll
                for (int c = 0; c < kC; ++c) {
                    if (!((cm >> c) & 1u)) continue;
                    const float2* bc = buf + c * a.W;
                    int* gc = gw + c * GW;
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        const f32x2 s2 = x2_add(tw2[h], Dr2[c][h]);
                        const f32x2 m2 = x2_add_rm(s2, kMagic2);
                        const f32x2 f2 = x2_sub(s2, x2_sub(m2, kMagic2));
                        float m0, m1;
                        x2_unpack(m2, m0, m1);
                        const int i0 = __float_as_int(m0) - kMagicBits, i1 = __float_as_int(m1) - kMagicBits;
                        const float2 a0 = bc[i0], a1 = bc[i1];
                        float f0, f1;
                        x2_unpack(f2, f0, f1);
                        const float v0 = fmaf(f0, a0.y, a0.x), v1 = fmaf(f1, a1.y, a1.x);
                        f32x2 yW2 = MODE == 0 ? x2_mul(yt2[h], Wr2[c][h]) : Wr2[c][h];
                        if (EDGE) {
                            float y0, y1;
                            x2_unpack(yW2, y0, y1);
                            if ((unsigned)(si.lo + i0) > lim) y0 = 0.0f;
                            if ((unsigned)(si.lo + i1) > lim) y1 = 0.0f;
                            yW2 = x2_pack(y0, y1);
                        }
                        if (NEED_RF) {
                            const f32x2 w12 = x2_mul(yW2, f2);
                            float q0, q1, q2, q3;
                            x2_unpack(x2_fma(x2_sub(yW2, w12), scale2, kMagic2), q0, q1);
                            x2_unpack(x2_fma(w12, scale2, kMagic2), q2, q3);
                            atomicAdd(gc + i0, __float_as_int(q0) - kMagicBits);
                            atomicAdd(gc + i0 + 1, __float_as_int(q2) - kMagicBits);
                            atomicAdd(gc + i1, __float_as_int(q1) - kMagicBits);
                            atomicAdd(gc + i1 + 1, __float_as_int(q3) - kMagicBits);
                        }
                        if (NEED_PAR) {
                            // sound speed: y W x'[i] (s + base); receive weights: y w_t a_r v;
                            // transmit weight (STAI): y a_t W_r v
                            float p0, p1, g0, g1;
                            x2_unpack(x2_mul(yW2, x2_add(base2, s2)), p0, p1);
                            accC = fmaf(p0, a0.y, fmaf(p1, a1.y, accC));
                            x2_unpack(MODE == 0 ? x2_mul(yt2[h], Ar2[c][h]) : Ar2[c][h], g0, g1);
                            gR[c] = fmaf(g0, v0, fmaf(g1, v1, gR[c]));
                            if (MODE == 0) gT2 = x2_fma(x2_mul(ya2[h], Wr2[c][h]), x2_pack(v0, v1), gT2);
                        }
                    }
                }
            };
            if (si.edge()) terms(std::true_type{});
            else terms(std::false_type{});
            if (NEED_PAR && MODE == 0) {
                float g0, g1;
                x2_unpack(gT2, g0, g1);
                const float gT = warp_sum(g0 + g1);
                if (lane == 0 && gT != 0.0f) atomicAdd(&ge[a.tx[t].e - er.x], gT);
            }
        }
        if (NEED_RF) {
            __syncthreads();   // every contribution of stage q is in the window; pairs no longer read
            {
                // window positions n = 4 m .. 4 m + 3 cover samples lo + n (lo is a multiple of
                // 8, contributions reach n <= len); rows paired with t.  Whole groups inside
                // the record go out as one 16-byte atomic add, edge groups sample by sample.
                const int span4 = (si.len + 4) >> 2, nrow = r_last - r0 + 1;
                // c = i / span4 by one multiply-shift per cell (exact for span4 <= 139 and
                // i < 8 span4 + 8; span4 <= 129 here) and one division per stage
                const unsigned mspan = ((1u << 20) + (unsigned)span4 - 1u) / (unsigned)span4;
                for (int i = tid; i < nrow * span4; i += kThreads) {
                    const int c = (int)(((unsigned)i * mspan) >> 20), m = i - c * span4;
                    int4* cell = reinterpret_cast<int4*>(gw + c * GW + 4 * m);
                    const int4 qv = *cell;
                    if ((qv.x | qv.y | qv.z | qv.w) == 0) continue;
                    *cell = make_int4(0, 0, 0, 0);
                    const float4 v = make_float4((float)qv.x * inv_scale, (float)qv.y * inv_scale,
                                                 (float)qv.z * inv_scale, (float)qv.w * inv_scale);
                    const int smp = si.lo + 4 * m;
                    const bool mirror = SYM && r0 + c > t;
                    float* d0 = grf + ((long long)t * E + r0 + c) * a.ns + smp;
                    float* d1 = mirror ? grf + ((long long)(r0 + c) * E + t) * a.ns + smp : d0;
                    if (vec4 && smp >= 0 && smp + 4 <= a.ns) {
                        atomicAdd(reinterpret_cast<float4*>(d0), v);
                        if (mirror) atomicAdd(reinterpret_cast<float4*>(d1), v);
                    } else {
                        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (vv[u] == 0.0f || smp + u < 0 || smp + u >= a.ns) continue;
                            atomicAdd(d0 + u, vv[u]);
                            if (mirror) atomicAdd(d1 + u, vv[u]);
                        }
                    }
                }
            }
        } else {
            __syncthreads();   // pairs no longer read
        }
    }
    if (NEED_PAR) {
        if (k_cur >= 0) flush_chunk(er.x + k_cur * kC);   // the CTA's last chunk
        const float sc = warp_sum(accC);
        if (lane == 0) s_red[warp] = sc;
        __syncthreads();
        if (tid == 0) {
            float tot = 0.0f;
            for (int w = 0; w < kThreads / 32; ++w) tot += s_red[w];
            if (tot != 0.0f && a.grad_c) atomicAdd(a.grad_c, tot * a.neg_inv_c);
        }
        if (a.grad_w)
            for (int e = er.x + tid; e <= er.y; e += kThreads) {
                const float v = ge[e - er.x];
                if (v != 0.0f) atomicAdd(a.grad_w + e, v);
            }
    }
}

// Per-pixel reverse mode for grids so coarse that a tile's staging window does
// not fit in shared memory (the forward's direct path): delays in
// double-float, every contribution straight to global memory with atomics.
template <int MODE>
__global__ void __launch_bounds__(256) das_backward_direct_kernel(const __grid_constant__ DasArgs a) {
    const Geom& g = a.g;
    const int ix = blockIdx.x * 32 + (threadIdx.x & 31);
    const int iz = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int b = blockIdx.z;
    float accC = 0.0f;
    if (ix < g.nx && iz < g.nz) {
        const float y = __ldg(a.grad_out + ((long long)b * g.nz + iz) * g.nx + ix);
        const float* rf = reinterpret_cast<const float*>(a.rf) + (long long)b * a.frame_elems;
        float* grf = a.grad_rf ? a.grad_rf + (long long)b * a.frame_elems : nullptr;
        const DF px = df_axpk(a.gd.gx0, ix, a.gd.gdx), pz = df_axpk(a.gd.gz0, iz, a.gd.gdz);
        const DF pz2 = df_mul(pz, pz);
        const float kap = aperture_kappa(g, pz.hi);
        const int2 er = tile_elements(g, px.hi, px.hi, pz.hi);
        auto dist = [&](int e, float& dxe) {
            const DF d = df_add(df_axpk(a.gd.xe0, e, a.gd.pitch), df_neg(px));
            dxe = d.hi;
            return df_sqrt(df_add(df_mul(d, d), pz2));
        };
        auto weight = [&](int e) { return g.elem_weight ? __ldg(g.elem_weight + e) : 1.0f; };
        for (int t = 0; t < a.n_tx && y != 0.0f; ++t) {
            const TxInfo& ti = a.tx[t];
            DF dt;
            float at = 1.0f, gt = 1.0f;
            if (MODE == 0) {
                float dxe;
                dt = df_add(dist(ti.e, dxe), df_neg(ti.t0));
                at = apod_w(g.apod, dxe, kap);
                gt = weight(ti.e);
            } else {
                dt = df_add(df_add(df_mul(px, ti.sin), df_mul(pz, ti.cos)), df_neg(ti.t0));
            }
            if (at == 0.0f) continue;
            const float t0 = ti.t0.hi + ti.t0.lo;
            float gT = 0.0f;
            for (int r = er.x; r <= er.y; ++r) {
                float dxe;
                const DF dr = dist(r, dxe);
                const float ar = apod_w(g.apod, dxe, kap);
                if (ar == 0.0f) continue;
                const DF sd = df_add(dt, dr);
                float fl = floorf(sd.hi);
                float f = (sd.hi - fl) + sd.lo;
                if (f < 0.0f) { fl -= 1.0f; f += 1.0f; }
                if (f >= 1.0f) { fl += 1.0f; f -= 1.0f; }
                if (!(fl >= 0.0f) || !(fl <= (float)(a.ns - 2))) continue;
                const long long off = ((long long)t * g.n_elements + r) * a.ns + (int)fl;
                const float x0 = __ldg(rf + off), x1 = __ldg(rf + off + 1);
                const float v = fmaf(f, x1 - x0, x0);
                const float gr = weight(r);
                const float yW = y * (gt * at) * (gr * ar);
                if (grf) {
                    atomicAdd(grf + off, yW - yW * f);
                    atomicAdd(grf + off + 1, yW * f);
                }
                accC = fmaf(yW * (x1 - x0), (fl + f) + t0, accC);
                if (a.grad_w) {
                    atomicAdd(a.grad_w + r, y * (gt * at) * ar * v);
                    if (MODE == 0) gT = fmaf(y * at * (gr * ar), v, gT);
                }
            }
            if (MODE == 0 && a.grad_w && gT != 0.0f) atomicAdd(a.grad_w + ti.e, gT);
        }
    }
    accC = warp_sum(accC);
    if ((threadIdx.x & 31) == 0 && accC != 0.0f && a.grad_c) atomicAdd(a.grad_c, accC * a.neg_inv_c);
}

template <int MODE, bool SYM, bool NEED_RF, bool NEED_PAR, bool TMA>
wf_status launch_bwd_v(DasArgs& A, const Plan& P, int batch, cudaStream_t st) {
    static unsigned long long smem_set = 0ull;
    auto kern = das_backward_kernel<MODE, SYM, NEED_RF, NEED_PAR, TMA>;
    wf_status s = ensure_smem_limit(kern, kMaxTiledSmem, smem_set);
    if (s != WF_OK) return s;
    const size_t smem = bwd_smem_layout(A.W, A.g.n_elements, NEED_RF, TMA ? kBwdRing : 0, SYM).total;
    kern<<<dim3(P.n_items, batch), kThreads, smem, st>>>(A);
    return last_launch_status();
}

template <int MODE, bool SYM, bool TMA>
wf_status launch_bwd_need(DasArgs& A, const Plan& P, int batch, bool need_rf, bool need_par,
                          cudaStream_t st) {
    if (need_rf && need_par) return launch_bwd_v<MODE, SYM, true, true, TMA>(A, P, batch, st);
    if (need_rf) return launch_bwd_v<MODE, SYM, true, false, TMA>(A, P, batch, st);
    return launch_bwd_v<MODE, SYM, false, true, TMA>(A, P, batch, st);
}

// Whether the tensor-copy staging applies: descriptors made for this call (use_tmap) and
// the raw ring fits beside the rest of the reverse kernel's shared memory.
bool backward_tma_fits(const DasArgs& A, bool need_rf, bool sym) {
    return A.use_tmap &&
           bwd_smem_layout(A.W, A.g.n_elements, need_rf, kBwdRing, sym).total <= 113 * 1024;
}

bool backward_is_tiled(const Plan& P, int n_elements, bool need_rf) {
    return P.tiled && bwd_smem_layout(P.W, n_elements, need_rf).total <= kMaxTiledSmem;
}

template <int MODE>
wf_status launch_das_backward(DasArgs& A, const Plan& P, int batch, bool need_rf, bool need_par,
                              cudaStream_t st) {
    if (P.cfg.wcol != kBwdWCOL || P.cfg.p != kBwdP) return WF_ERR_UNSUPPORTED;
    if (!need_rf && !need_par) return WF_OK;
    if (!backward_is_tiled(P, A.g.n_elements, need_rf)) {
        dim3 grid((A.g.nx + 31) / 32, (A.g.nz + 7) / 8, batch);
        das_backward_direct_kernel<MODE><<<grid, 256, 0, st>>>(A);
        return last_launch_status();
    }
    if (MODE == 0 && P.sym)
        return backward_tma_fits(A, need_rf, true)
                   ? launch_bwd_need<MODE, MODE == 0, true>(A, P, batch, need_rf, need_par, st)
                   : launch_bwd_need<MODE, MODE == 0, false>(A, P, batch, need_rf, need_par, st);
    return backward_tma_fits(A, need_rf, false)
               ? launch_bwd_need<MODE, false, true>(A, P, batch, need_rf, need_par, st)
               : launch_bwd_need<MODE, false, false>(A, P, batch, need_rf, need_par, st);
}

template wf_status launch_das_backward<0>(DasArgs&, const Plan&, int, bool, bool, cudaStream_t);
template wf_status launch_das_backward<1>(DasArgs&, const Plan&, int, bool, bool, cudaStream_t);

}  // namespace wf
