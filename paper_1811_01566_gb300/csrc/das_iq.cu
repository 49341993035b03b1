// Delay-and-sum of complex baseband (IQ) traces, STAI and PWI: beamforming after
// IQ demodulation (wf_iq_demod), the pre-processing variant of the paper's
// operator list (Sec. II-B: FIR filtering before the beamformer).
//
//   B(p) = sum_t w_t sum_r w_r lerp(iq[t][r], u) exp(2 pi i k u),
//   u = s / D (baseband samples), k = f0 D / fs (cycles per baseband sample),
//
// with the delays, apodization and tiles of the RF kernels, the geometry
// expressed in baseband samples (fs / D).  Per stage (transmit, chunk of 8
// receive elements) the window positions n = lo + i of the 8 traces are staged
// as y = iq[n] e^{2 pi i k n} and d = iq[n+1] e^{2 pi i k n} - y, so that a term
// at u = n + f is e^{2 pi i k f} (y + f d): the rotation e^{2 pi i k n} is shared
// by the rows (one table per stage, double-float phase reduction), and each term
// rotates by the fractional phase 2 pi k f only (|k f| < k).  A CTA owns a
// 32 x 16 pixel tile and one group of its stage list; group partials are summed
// in group order by a second kernel (deterministic).
#include "das_kernels.cuh"

namespace wf {

constexpr int kIqWcol = 4, kIqP = 2;   // 32 x 16 tiles, two pixels per lane

__host__ __device__ inline IqSmem iq_smem_layout(int W, int n_elements) {
    IqSmem L;
    size_t off = 0;
    L.pairs = off;
    off += (size_t)kC * W * sizeof(float4);
    L.rot = off;
    off += (size_t)(W + 8) * sizeof(float2);
    L.table = off;
    off += (size_t)kTableStages * sizeof(Stage);
    L.elems = off;
    off += (((size_t)n_elements * sizeof(Elem)) + 15) & ~(size_t)15;
    L.raw = off;   // [kC][W + 8] complex samples of the next stage, copied during this one
    off += (size_t)kC * (W + 8) * sizeof(float2);
    L.total = off;
    return L;
}

// 8-byte asynchronous copy global -> shared; src_bytes 0 writes zeros without reading.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(smem_dst)), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) das_iq_kernel(const __grid_constant__ DasArgs a) {
    using S = Shape<kIqWcol, kIqP>;
    constexpr int P = kIqP, H = P / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const IqSmem L = iq_smem_layout(a.W, a.g.n_elements);
    float4* buf = reinterpret_cast<float4*>(smem_raw + L.pairs);   // [kC][W] (y, d)
    float2* rot = reinterpret_cast<float2*>(smem_raw + L.rot);     // [W + 8] e^{2 pi i k n}
    Stage* st = reinterpret_cast<Stage*>(smem_raw + L.table);
    Elem* el = reinterpret_cast<Elem*>(smem_raw + L.elems);
    float2* raw = reinterpret_cast<float2*>(smem_raw + L.raw);      // [kC][W + 8] complex samples
    __shared__ int s_tlist[WF_MAX_TX];
    __shared__ int s_info[4];
    __shared__ int s_cnt[kTableBatch / 32];

    const Geom& g = a.g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lx = lane % kIqWcol, lz = lane / kIqWcol;
    const int item = blockIdx.x, b = blockIdx.y;
    const int group = item % a.n_groups, rank = item / a.n_groups;
    const int tzi = a.tiles_z - 1 - rank / a.tiles_x, txi = rank % a.tiles_x;
    const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, txi * S::kCols, tzi * S::kRows);
    const float2* iq = reinterpret_cast<const float2*>(a.rf) + (long long)b * a.frame_elems;
    const long long E = g.n_elements;

    const int col = kIqWcol * warp + lx;
    const float ux = (float)col * g.gdx;
    float kz[P], kap[P], uz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
        uz[p] = (float)(lz + S::kLR * p) * g.gdz;
        kz[p] = uz[p] * fmaf(2.0f, tg.cz.hi, uz[p]);
        kap[p] = aperture_kappa(g, tg.cz.hi + uz[p]);
    }
    const int2 wr = tile_elements(g, pixel_x(g, tg.ix0 + kIqWcol * warp),
                                  pixel_x(g, tg.ix0 + kIqWcol * warp + kIqWcol - 1), tg.zhi);
    const int2 er = tg.er;
    const int n_e = er.y >= er.x ? er.y - er.x + 1 : 0;
    const int nc = (n_e + kC - 1) / kC;
    for (int e = er.x + tid; e <= er.y; e += kThreads) el[e - er.x] = make_elem(a, tg.cx, tg.cz, e);
    if (tid == 0) {
        int n = 0;
        if (n_e > 0)
            for (int t = 0; t < a.n_tx; ++t) {
                if (MODE == 0 && (a.tx[t].e < er.x || a.tx[t].e > er.y)) continue;
                s_tlist[n++] = t;
            }
        const long long G = a.n_groups;
        const long long n_raw = (long long)nc * n;
        s_info[0] = n;
        s_info[1] = (int)((long long)group * n_raw / G);
        s_info[2] = (int)((long long)(group + 1) * n_raw / G);
    }
    __syncthreads();
    const int n_act = s_info[0], q0 = s_info[1], n_stages = s_info[2] - s_info[1];
    const StageSpace sp{er, n_e, nc, n_act, q0, n_stages, s_tlist};
    int n_live = 0, raw_next = 0;
    auto need = [&](int upto) {
        while (n_live <= upto && raw_next < n_stages) {
            n_live += fill_stages<MODE, false>(a, tg, el, sp, st, s_cnt, raw_next, n_live);
            raw_next += kTableBatch;
        }
    };
    need(0);
    // Samples lo .. lo + len of the chunk's rows of entry qq into `raw` by asynchronous copies
    // (row c = warp, positions 32 apart per lane; zeros outside the record and the chunk),
    // issued one stage ahead so the global latency runs under the previous stage's work.
    auto issue_raw = [&](int qq) {
        const Stage s = st[qq & (kTableStages - 1)];
        const int rr0 = er.x + s.k() * kC, rlast = min(rr0 + kC - 1, er.y);
        const bool row_on = rr0 + warp <= rlast;
        const float2* tr = iq + ((long long)stage_tx<false>(sp, s.j()) * E + rr0 + (row_on ? warp : 0)) * a.ns;
        float2* dst = raw + warp * (a.W + 8);
        for (int i = lane; i <= s.len; i += 32) {
            const int n = s.lo + i;
            const bool in = row_on && n >= 0 && n < a.ns;
            cp_async8(dst + i, tr + (in ? n : 0), in ? 8u : 0u);
        }
        cp_async_commit();
    };
    // Rotation e^{2 pi i k n} of the window positions n = lo + i, i = 0 .. len, of a stage.
    auto make_rot = [&](const Stage& s) {
        // position lane * 8 + warp: a window of a few dozen positions spreads over all warps
        for (int i = lane * (kThreads / 32) + warp; i <= s.len; i += kThreads) {
            const DF ph = df_mul(a.iq_k, DF{(float)(s.lo + i), 0.0f});   // cycles, |lo + i| < 2^22
            const float fr = (ph.hi - rintf(ph.hi)) + ph.lo;
            float sn, cs;
            sincospif(2.0f * fr, &sn, &cs);
            rot[i] = make_float2(cs, sn);
        }
    };
    if (n_live > 0) {
        issue_raw(0);
        make_rot(st[0]);
    }

    float acc_re[P], acc_im[P];
#pragma unroll
    for (int p = 0; p < P; ++p) acc_re[p] = acc_im[p] = 0.0f;
    f32x2 Dr2[kC][H], Wr2[kC][H];
    unsigned cmask = 0u;
    const float two_pi_k = 6.283185307179586f * a.iq_k.hi;
    int k_cur = -1;
    for (int q = 0; q < n_live; ++q) {
        const Stage si = st[q & (kTableStages - 1)];
        const int k = si.k();
        const int r0 = er.x + k * kC;
        const int r_last = min(r0 + kC - 1, er.y);
        const int t = stage_tx<false>(sp, si.j());
        cp_async_wait_all();   // this thread's copies of stage q
        // every copy and the rotations of stage q visible; every warp done with stage q - 1's
        // pairs (its compute precedes this barrier), so they may be overwritten
        __syncthreads();
        // staged pairs (y, d) of the chunk's rows; zero where n or n + 1 is outside the record
        const int len = si.len;
        {
            static_assert(kThreads / 32 == kC, "one trace row per warp");
            const int c = warp;   // one trace row per warp, lanes along the window: equal shares
            for (int i = lane; i < len; i += 32) {
                const int n = si.lo + i;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (r0 + c <= r_last && n >= 0 && n + 1 <= a.ns - 1) {
                    const float2 x0 = raw[c * (a.W + 8) + i], x1 = raw[c * (a.W + 8) + i + 1], e = rot[i];
                    const float yr = x0.x * e.x - x0.y * e.y, yi = x0.x * e.y + x0.y * e.x;
                    const float zr = x1.x * e.x - x1.y * e.y, zi = x1.x * e.y + x1.y * e.x;
                    v = make_float4(yr, yi, zr - yr, zi - yi);
                }
                buf[c * a.W + i] = v;
            }
        }
        __syncthreads();   // pairs visible; raw and the rotation table free
        need(q + 1);
        if (q + 1 < n_live) {   // stage q + 1's samples and rotations, under stage q's compute
            issue_raw(q + 1);
            make_rot(st[(q + 1) & (kTableStages - 1)]);
        }
        if (k != k_cur) {
            k_cur = k;
            cmask = 0u;
#pragma unroll
            for (int c = 0; c < kC; ++c)
                if (r0 + c <= r_last && r0 + c >= wr.x && r0 + c <= wr.y) cmask |= 1u << c;
            if (cmask) {
                const Elem e0 = el[r0 - er.x];
#pragma unroll
                for (int c = 0; c < kC; ++c) {
                    const bool on = (cmask >> c) & 1u;
                    const Elem ee = el[(on ? r0 + c : r0) - er.x];
                    const float cc = elem_rel(ee, e0);
                    float d[P], w[P];
#pragma unroll
                    for (int p = 0; p < P; ++p) {
                        d[p] = on ? cc + dist_delta(ee, ux, kz[p]) : 0.0f;
                        w[p] = on ? apod_w(g.apod, -(ee.ax + ux), kap[p]) * ee.g : 0.0f;
                    }
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        Dr2[c][h] = x2_pack(d[2 * h], d[2 * h + 1]);
                        Wr2[c][h] = x2_pack(w[2 * h], w[2 * h + 1]);
                    }
                }
            }
        }
        bool live = cmask != 0u;
        if (MODE == 0) live = live && a.tx[t].e >= wr.x && a.tx[t].e <= wr.y;
        if (live) {
            float tw[P], wt[P];
            if (MODE == 0) {
                const Elem et = el[a.tx[t].e - er.x];
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tw[p] = si.B + dist_delta(et, ux, kz[p]);
                    wt[p] = apod_w(g.apod, -(et.ax + ux), kap[p]) * et.g;
                }
            } else {
                const float sn = a.tx[t].sin_f, cs = a.tx[t].cos_f;
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    tw[p] = si.B + fmaf(ux, sn, uz[p] * cs);
                    wt[p] = 1.0f;
                }
            }
            const f32x2 kMagic2 = x2_pack(kMagic, kMagic);
            float sr[P], si_[P];
#pragma unroll
            for (int p = 0; p < P; ++p) sr[p] = si_[p] = 0.0f;
#pragma unroll
            for (int c = 0; c < kC; ++c) {
                if (!((cmask >> c) & 1u)) continue;
                const float4* bc = buf + c * a.W;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    const f32x2 s2 = x2_add(x2_pack(tw[2 * h], tw[2 * h + 1]), Dr2[c][h]);
                    const f32x2 m2 = x2_add_rm(s2, kMagic2);
                    const f32x2 f2 = x2_sub(s2, x2_sub(m2, kMagic2));
                    float m[2], f[2], w[2];
                    x2_unpack(m2, m[0], m[1]);
                    x2_unpack(f2, f[0], f[1]);
                    x2_unpack(Wr2[c][h], w[0], w[1]);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        int i = __float_as_int(m[u]) - kMagicBits;
                        i = min(max(i, 0), si.len - 1);   // stays inside the staged window
                        const float4 pv = bc[i];
                        const float vr = fmaf(f[u], pv.z, pv.x), vi = fmaf(f[u], pv.w, pv.y);
                        float sn, cs;
                        __sincosf(two_pi_k * f[u], &sn, &cs);
                        const int p = 2 * h + u;
                        sr[p] = fmaf(w[u], fmaf(vr, cs, -vi * sn), sr[p]);
                        si_[p] = fmaf(w[u], fmaf(vr, sn, vi * cs), si_[p]);
                    }
                }
            }
#pragma unroll
            for (int p = 0; p < P; ++p) {
                acc_re[p] = fmaf(wt[p], sr[p], acc_re[p]);
                acc_im[p] = fmaf(wt[p], si_[p], acc_im[p]);
            }
        }
    }
    float2* dst = reinterpret_cast<float2*>(a.part) + ((long long)b * a.n_items + item) * (kThreads * P);
#pragma unroll
    for (int p = 0; p < P; ++p) dst[p * kThreads + tid] = make_float2(acc_re[p], acc_im[p]);
}

// Sum the group partials of every pixel in group order (complex).
__global__ void das_iq_reduce_kernel(const float2* __restrict__ part, float2* __restrict__ out, int nz,
                                     int nx, int tiles_x, int tiles_z, int n_groups, int n_items) {
    using S = Shape<kIqWcol, kIqP>;
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iz = blockIdx.y;
    const int b = blockIdx.z;
    if (ix >= nx) return;
    const int first = tile_rank(iz / S::kRows, ix / S::kCols, tiles_z, tiles_x) * n_groups;
    const int cl = ix % S::kCols, rl = iz % S::kRows;
    const int tid = (cl / kIqWcol) * 32 + (rl % S::kLR) * kIqWcol + (cl % kIqWcol);
    const int local = (rl / S::kLR) * kThreads + tid;
    const float2* p = part + ((long long)b * n_items + first) * (kThreads * kIqP) + local;
    float2 s = make_float2(0.0f, 0.0f);
    for (int k = 0; k < n_groups; ++k) {
        const float2 v = p[(long long)k * (kThreads * kIqP)];
        s.x += v.x;
        s.y += v.y;
    }
    out[((long long)b * nz + iz) * nx + ix] = s;
}

size_t iq_smem_bytes(int W, int n_elements) { return iq_smem_layout(W, n_elements).total; }

template <int MODE>
wf_status launch_das_iq(DasArgs& A, int batch, float* out, cudaStream_t st) {
    static unsigned long long smem_set = 0ull;
    auto kern = das_iq_kernel<MODE>;
    wf_status s = ensure_smem_limit(kern, kMaxTiledSmem, smem_set);
    if (s != WF_OK) return s;
    const size_t smem = iq_smem_layout(A.W, A.g.n_elements).total;
    kern<<<dim3(A.n_items, batch), kThreads, smem, st>>>(A);
    if ((s = last_launch_status()) != WF_OK) return s;
    dim3 rg((A.g.nx + 127) / 128, A.g.nz, batch);
    das_iq_reduce_kernel<<<rg, 128, 0, st>>>(reinterpret_cast<const float2*>(A.part),
                                             reinterpret_cast<float2*>(out), A.g.nz, A.g.nx,
                                             A.tiles_x, A.tiles_z, A.n_groups, A.n_items);
    return last_launch_status();
}

template wf_status launch_das_iq<0>(DasArgs&, int, float*, cudaStream_t);
template wf_status launch_das_iq<1>(DasArgs&, int, float*, cudaStream_t);

// |B| of a complex image and, optionally, each frame's largest value (non-NaN).
__global__ void iq_envelope_kernel(const float2* __restrict__ img, long long n_frame, float* __restrict__ env,
                                   float* __restrict__ frame_max) {
    const int b = blockIdx.y;
    const float2* src = img + (long long)b * n_frame;
    float* dst = env + (long long)b * n_frame;
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_frame;
         i += (long long)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        const float e = sqrtf(fmaf(v.x, v.x, v.y * v.y));
        dst[i] = e;
        if (e > m) m = e;   // false for NaN
    }
    if (frame_max) {
        m = warp_max(m);
        if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(reinterpret_cast<unsigned*>(frame_max + b), __float_as_uint(m));
    }
}

wf_status launch_iq_envelope(const float* img, int batch, long long n_frame, float* env, float* frame_max,
                             cudaStream_t st) {
    wf_status s;
    if (frame_max && (s = cuda_status(cudaMemsetAsync(frame_max, 0, (size_t)batch * sizeof(float), st))) != WF_OK)
        return s;
    const int blocks = (int)std::min<long long>(1216, (n_frame + 255) / 256);
    iq_envelope_kernel<<<dim3(blocks, batch), 256, 0, st>>>(reinterpret_cast<const float2*>(img), n_frame, env,
                                                           frame_max);
    return last_launch_status();
}

}  // namespace wf
