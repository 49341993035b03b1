// Delay-and-sum beamforming (paper Sec. II-B, beamforming block of Fig. 2): host
// planning, argument checks and the C entry points of include/wf.h.  The
// kernels and their design are in das_kernels.cuh; the tiled launchers are
// instantiated per mode in das_stai.cu / das_pwi.cu (fast) and
// das_check.cu (bounds-checked variants).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <list>
#include <memory>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "das_kernels.cuh"

namespace wf {

extern template wf_status launch_das_tiled<0, false>(DasArgs&, const Plan&, int, wf_dtype, cudaStream_t);
extern template wf_status launch_das_tiled<1, false>(DasArgs&, const Plan&, int, wf_dtype, cudaStream_t);
extern template wf_status launch_das_tiled<0, true>(DasArgs&, const Plan&, int, wf_dtype, cudaStream_t);
extern template wf_status launch_das_tiled<1, true>(DasArgs&, const Plan&, int, wf_dtype, cudaStream_t);

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
        const int r_in = (int)(i % g.n_elements);
        const int t = (int)((i / g.n_elements) % a.n_tx);
        const int q = (int)(i / ((long long)g.n_elements * a.n_tx));
        const int lin = pix[q];
        const int ix = lin % g.nx, iz = lin / g.nx;
        const TileGeo tg = tile_geo<S::kCols, S::kRows>(a, (ix / S::kCols) * S::kCols,
                                                        (iz / S::kRows) * S::kRows);
        // Reciprocal STAI evaluates the pair (t, r) with t > r as transmit r, receive t.
        int tt = t, r = r_in;
        if (MODE == 0 && a.sym && t > r_in) {
            tt = r_in;
            r = t;
        }
        const TxInfo& ti = a.tx[tt];
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
        for (int rr = (MODE == 0 && a.sym) ? max(r0, tt) : r0; rr <= r_last; ++rr) {
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

// Tuning switches from the environment (WF_DAS_NO_SYM, WF_DAS_NO_TMA, WF_DAS_NO_TMAP, WF_DAS_TILE,
// WF_DAS_GROUPS, WF_DAS_BUDGET, WF_DAS_RING, WF_CHECK_BOUNDS), read on the first DAS
// call and again only on wf_das_reload_tuning(); `gen` counts the reloads, so plans
// cached under older switches are never reused.
struct Tuning {
    bool no_sym = false, no_tma = false, check_bounds = false;
    bool no_tmap = false;         // per-trace bulk copies instead of tensor-map boxes
    int tile_w = 0, tile_p = 0;   // 0: no tile override
    int groups = 0;               // > 0: uniform groups instead of the schedule
    int budget = 0;               // > 0: CTAs per frame of the schedule
    int ring = 0;                 // > 0: TMA ring depth cap
    unsigned gen = 0;
};

std::mutex g_tuning_mu;
Tuning g_tuning;
bool g_tuning_read = false;

bool env_flag(const char* name) {
    const char* v = std::getenv(name);
    return v && v[0] && v[0] != '0';
}

void read_tuning_locked() {
    Tuning t;
    t.gen = g_tuning.gen + 1;
    t.no_sym = env_flag("WF_DAS_NO_SYM");
    t.no_tma = env_flag("WF_DAS_NO_TMA");
    t.no_tmap = env_flag("WF_DAS_NO_TMAP");
    t.check_bounds = env_flag("WF_CHECK_BOUNDS");
    if (const char* v = std::getenv("WF_DAS_TILE"))
        if (std::sscanf(v, "%d,%d", &t.tile_w, &t.tile_p) != 2) t.tile_w = t.tile_p = 0;
    if (const char* v = std::getenv("WF_DAS_GROUPS")) t.groups = std::max(0, std::atoi(v));
    if (const char* v = std::getenv("WF_DAS_BUDGET")) t.budget = std::max(0, std::atoi(v));
    if (const char* v = std::getenv("WF_DAS_RING")) t.ring = std::max(0, std::atoi(v));
    g_tuning = t;
    g_tuning_read = true;
}

Tuning tuning() {
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    if (!g_tuning_read) read_tuning_locked();
    return g_tuning;
}

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
constexpr Cfg kStaiCfgs[] = {{4, 4}, {4, 2}};
constexpr Cfg kPwiCfgs[] = {{4, 4}, {4, 2}};
constexpr size_t kSmemBudget = 113 * 1024;   // two CTAs per SM
constexpr int kTargetItems = 1536;            // CTAs per frame the groups aim for (~5 waves)
constexpr int kTargetItemsStai = 768;

// Reciprocal STAI pairing applies when every element fires once, in element
// order (transmit t fires element t), so rf[t][r] and rf[r][t] share delay and
// weights.  WF_DAS_NO_SYM=1 turns it off (testing the general path).
bool use_sym(int mode, int n_tx, int n_elements, const int32_t* tx_elem) {
    if (mode != 0 || n_tx != n_elements) return false;
    if (tuning().no_sym) return false;
    if (tx_elem)
        for (int t = 0; t < n_tx; ++t)
            if (tx_elem[t] != t) return false;
    return true;
}

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
    const Tuning tu = tuning();
    const int w = tu.tile_w, p = tu.tile_p;
    if (w == 0) return false;
    const Cfg* cfgs = mode == 0 ? kStaiCfgs : kPwiCfgs;
    for (int i = 0; i < 2; ++i)
        if (cfgs[i].wcol == w && cfgs[i].p == p) {
            out = cfgs[i];
            return true;
        }
    return false;
}

Plan plan_for(int mode, const Cfg& cfg, const GeomD& D, const wf_probe* p, const wf_grid* g,
              int batch, int n_tx, int ns, int rf_bytes, bool sym) {
    const Tuning tu = tuning();
    Plan P{};
    P.cfg = cfg;
    P.cols = 8 * cfg.wcol;
    P.rows = (32 / cfg.wcol) * cfg.p;
    P.W = window_bound(D, P.cols, P.rows);
    P.tiled = P.W <= kMaxWindow;
    P.tiles_x = (g->nx + P.cols - 1) / P.cols;
    P.tiles_z = (g->nz + P.rows - 1) / P.rows;
    const long long tiles = (long long)P.tiles_x * P.tiles_z * batch;
    P.n_groups = (int)std::min<long long>(kMaxGroups, std::max<long long>(1, (kTargetItems + tiles - 1) / tiles));
    if (tu.groups > 0) P.n_groups = std::min(kMaxGroups, tu.groups);   // tuning override
    P.n_items = P.tiles_x * P.tiles_z * P.n_groups;
    // Work-proportional schedule (built per call from the scan geometry): budget CTAs per
    // frame plus at most one extra per tile from rounding.
    // CTAs per frame: reciprocal STAI tiles carry more start-up per stage (window
    // bounds of pair sums, two traces per row), so they take fewer, longer CTAs.
    long long target_items = mode == 0 ? kTargetItemsStai : kTargetItems;
    if (tu.budget > 0) target_items = tu.budget;   // tuning
    P.budget = (int)std::max<long long>(1, (target_items + batch - 1) / batch);
    P.table = (long long)P.budget + P.tiles_x * P.tiles_z <= kMaxItems && tu.groups == 0;
    P.info_bytes = (((size_t)P.tiles_x * P.tiles_z * sizeof(unsigned)) + 255) & ~(size_t)255;
    P.sym = sym && mode == 0;
    // TMA bulk copies need 16-byte aligned trace windows: samples per trace a multiple of 8.
    // WF_DAS_NO_TMA=1 selects the register-staged path instead (tuning and testing).
    P.tma = ns % 8 == 0 && !tu.no_tma;
    // Deepest TMA ring (stages in flight) that fits two CTAs per SM, double-buffered pairs
    // preferred; WF_DAS_RING=n caps the depth (tuning).
    bool found = false;
    int max_ring = kMaxRing;
    if (tu.ring > 0) max_ring = std::max(2, std::min(kMaxRing, tu.ring));
    struct Cand { bool db; int ring; };
    Cand cands[2 * kMaxRing + 2];
    int nc = 0;
    if (P.tma) {
        for (int r = max_ring; r >= 3; --r) cands[nc++] = {true, r};
        for (int r = max_ring; r >= 3; --r) cands[nc++] = {false, r};
        cands[nc++] = {true, 2};
        cands[nc++] = {false, 2};
    } else {
        cands[nc++] = {false, 1};
    }
    for (int i = 0; i < nc && !found; ++i) {
        const SmemLayout L = smem_layout(P.W, p->n_elements, cands[i].db, P.tma, P.sym, cands[i].ring, rf_bytes);
        if (L.total <= kSmemBudget) {
            P.ring = cands[i].ring;
            P.db = cands[i].db;
            P.smem = L.total;
            found = true;
        }
    }
    if (!found) {
        P.ring = P.tma ? 2 : 1;
        P.db = false;
        P.smem = smem_layout(P.W, p->n_elements, false, P.tma, P.sym, P.ring, rf_bytes).total;
        if (P.smem > kMaxTiledSmem) P.tiled = false;
    }
    const long long item_bound = P.table ? (long long)P.budget + P.tiles_x * P.tiles_z : P.n_items;
    P.ws_bytes = kWsHeaderBytes + P.info_bytes +
                 (P.tiled ? (size_t)batch * item_bound * kThreads * cfg.p * sizeof(float) : 0);
    return P;
}

Plan make_plan(int mode, const wf_probe* p, const wf_grid* g, int batch, int n_tx, int ns = 8,
               int rf_bytes = 4, bool sym = false) {
    Geom G;
    GeomD D;
    make_geom(p, g, G, D);
    Cfg forced;
    if (tile_override(mode, forced)) {
        const Plan P = plan_for(mode, forced, D, p, g, batch, n_tx, ns, rf_bytes, sym);
        if (P.tiled) return P;
    }
    const Cfg* cfgs = mode == 0 ? kStaiCfgs : kPwiCfgs;
    Plan P{};
    for (int i = 0; i < 2; ++i) {
        P = plan_for(mode, cfgs[i], D, p, g, batch, n_tx, ns, rf_bytes, sym);
        if (P.tiled) return P;
    }
    return P;
}

bool check_bounds_mode() { return tuning().check_bounds; }

template <int MODE>
wf_status dispatch(DasArgs& A, const Plan& P, int batch, wf_dtype dt, cudaStream_t st) {
    if (!P.tiled) {
        dim3 grid((A.g.nx + 31) / 32, (A.g.nz + 7) / 8, batch);
        switch (dt) {
            case WF_F32: das_direct_kernel<MODE, float><<<grid, 256, 0, st>>>(A); break;
            case WF_F16: das_direct_kernel<MODE, __half><<<grid, 256, 0, st>>>(A); break;
            case WF_I16: das_direct_kernel<MODE, int16_t><<<grid, 256, 0, st>>>(A); break;
        }
        return last_launch_status();
    }
    return check_bounds_mode() ? launch_das_tiled<MODE, true>(A, P, batch, dt, st)
                               : launch_das_tiled<MODE, false>(A, P, batch, dt, st);
}

// Schedule of a frame's CTAs.  For every tile, an upper estimate of the
// (transmit, receive) pairs whose delay can reach the record (0 only when the
// smallest possible delay of every pair lies beyond the record: the tile's
// image is exactly 0 and it gets no CTA).  Every other tile gets the same
// number of groups (equal ranges of its stage list), budget / live tiles, and
// tiles are launched heaviest first.  (Groups in proportion to each tile's work
// were measured slower: they cut the heavy tiles into CTAs too short to amortise
// a CTA's start-up.)  Returns the number of items.
int build_schedule(int mode, const wf_probe* p, const wf_grid* g, const Plan& P, DasArgs& A) {
    Geom G;
    GeomD D;
    make_geom(p, g, G, D);
    const int E = p->n_elements, tiles = P.tiles_x * P.tiles_z;
    const double L = (double)A.ns + 16.0;                 // beyond this a window misses the record
    std::vector<double> work(tiles, 0.0), dmin(E), d;
    for (int tz = 0; tz < P.tiles_z; ++tz)
        for (int tx = 0; tx < P.tiles_x; ++tx) {
            const int ix0 = tx * P.cols, iz0 = tz * P.rows;
            const double xlo = D.gx0 + ix0 * D.gdx, xhi = D.gx0 + (ix0 + P.cols - 1) * D.gdx;
            const double zlo = D.gz0 + iz0 * D.gdz, zhi = D.gz0 + (iz0 + P.rows - 1) * D.gdz;
            int lo = 0, hi = E - 1;
            if (p->apod != WF_APOD_NONE) {
                if (!(zhi > 0.0)) continue;                    // no aperture anywhere in the tile
                const double half = zhi / (2.0 * p->f_number);
                lo = std::max(0, (int)std::floor((xlo - half - D.xe0) / D.pitch) - 2);
                hi = std::min(E - 1, (int)std::ceil((xhi + half - D.xe0) / D.pitch) + 2);
                if (lo > hi) continue;
            }
            // smallest distance from each element to the tile (its top edge)
            for (int e = 0; e < E; ++e) {
                const double xe = D.xe0 + e * D.pitch;
                const double dx = xe < xlo ? xlo - xe : (xe > xhi ? xe - xhi : 0.0);
                dmin[e] = std::sqrt(dx * dx + zlo * zlo);
            }
            d.assign(dmin.begin() + lo, dmin.begin() + hi + 1);
            std::sort(d.begin(), d.end());
            double cnt = 0.0;
            auto upto = [&](double v) { return (double)(std::upper_bound(d.begin(), d.end(), v) - d.begin()); };
            if (mode == 0) {
                if (P.sym) {   // pairs t <= r of the element range
                    const double lim = L + A.tx[0].t0.hi;
                    for (size_t i = 0; i < d.size(); ++i) cnt += std::max(0.0, upto(lim - d[i]) - (double)i);
                } else {
                    for (int t = 0; t < A.n_tx; ++t) {
                        const int e = A.tx[t].e;
                        if (e < lo || e > hi) continue;
                        cnt += upto(L + A.tx[t].t0.hi - dmin[e]);
                    }
                }
            } else {
                for (int t = 0; t < A.n_tx; ++t) {
                    const double sn = (double)A.tx[t].sin.hi + A.tx[t].sin.lo;
                    const double cs = (double)A.tx[t].cos.hi + A.tx[t].cos.lo;
                    const double c0 = std::min(xlo * sn, xhi * sn) + zlo * cs - A.tx[t].t0.hi;
                    cnt += upto(L - c0);
                }
            }
            work[tz * P.tiles_x + tx] = cnt;
        }
    const double total = std::accumulate(work.begin(), work.end(), 0.0);
    if (!(total > 0.0)) return 0;
    std::vector<int> order(tiles);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    int live_tiles = 0;
    for (int t = 0; t < tiles; ++t) live_tiles += work[t] > 0.0;
    const int grp = std::max(1, std::min(kMaxGroups, (P.budget + live_tiles / 2) / live_tiles));
    int n = 0;
    for (int tile : order) {
        if (!(work[tile] > 0.0)) break;
        for (int k = 0; k < grp && n < kMaxItems; ++k)
            A.items[n++] = (unsigned)tile | ((unsigned)k << 16) | ((unsigned)grp << 24);
    }
    return n;
}

double fill_tx(DasArgs& a, const wf_probe* probe, int mode, int n_tx, const int32_t* tx_elem,
               const double* angles, const double* t_start, bool per_tx_start);

// ---------------------------------------------------------------------------
// TMA descriptors of the RF array.  cuTensorMapEncodeTiled is reached through the
// runtime's driver entry point, so the library links no driver API.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Descriptors of rf as [frames * n_tx][E][ns / 8][8] for boxes of (W + 8) samples of 8
// receive rows (tm_rows) and of 8 transmit rows (tm_cols); false when they cannot be made
// (the call then takes the per-trace bulk copies).  Requires ns % 8 == 0 and a 16-byte
// aligned rf: every stride is then a multiple of 16 bytes and every box row 16 bytes long.
// (The 8-sample groups of a box row are contiguous in memory.  Splitting the row into boxes
// of up to 256 samples instead measured 5 % slower on the full PWI workload.)
bool encode_rf_maps(DasArgs& A, const void* rf, wf_dtype dt, long long frames_tx, int E, int ns,
                    int W, bool sym) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || ns % 8 != 0 || ((uintptr_t)rf & 15u) || (W + 8) / 8 > 256) return false;
    const cuuint64_t eb = dt == WF_F32 ? 4 : 2;
    const CUtensorMapDataType ty = dt == WF_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == WF_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                  : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[4] = {8, (cuuint64_t)ns / 8, (cuuint64_t)E, (cuuint64_t)frames_tx};
    const cuuint64_t strides[3] = {8 * eb, (cuuint64_t)ns * eb, (cuuint64_t)E * ns * eb};
    const cuuint32_t g = (cuuint32_t)(W + 8) / 8;
    const cuuint32_t box_rows[4] = {8, g, (cuuint32_t)kC, 1};
    const cuuint32_t box_cols[4] = {8, g, 1, (cuuint32_t)kC};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    void* base = const_cast<void*>(rf);
    if (fn(&A.tm_rows, ty, 4, base, dims, strides, box_rows, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (sym && fn(&A.tm_cols, ty, 4, base, dims, strides, box_cols, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return true;
}

// ---------------------------------------------------------------------------
// Plan cache.  A DAS call's plan (tile configuration, staging, workspace layout),
// its transmit table and its CTA schedule depend only on the probe, grid, scan,
// batch, RF shape and type and the tuning switches, so they are built once per
// such key and kept, with the packed kernel arguments, in a small LRU cache: a
// repeated call copies the cached argument block, sets its pointers and
// launches.  Element weights are device data and not part of the key.
// ---------------------------------------------------------------------------
struct CachedPlan {
    Plan P;
    std::unique_ptr<DasArgs> A;   // everything but the per-call pointers and rf_scale
};

class PlanCache {
  public:
    std::shared_ptr<const CachedPlan> get(const std::string& key) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = map_.find(key);
        if (it == map_.end()) return nullptr;
        lru_.splice(lru_.begin(), lru_, it->second.first);
        return it->second.second;
    }
    void put(const std::string& key, std::shared_ptr<const CachedPlan> v) {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = map_.find(key);
        if (it != map_.end()) {
            lru_.erase(it->second.first);
            map_.erase(it);
        }
        lru_.push_front(key);
        map_.emplace(key, std::make_pair(lru_.begin(), std::move(v)));
        while (map_.size() > kCapacity) {
            map_.erase(lru_.back());
            lru_.pop_back();
        }
    }
    void clear() {
        std::lock_guard<std::mutex> lk(mu_);
        map_.clear();
        lru_.clear();
    }

  private:
    static constexpr size_t kCapacity = 64;
    std::mutex mu_;
    std::list<std::string> lru_;   // most recent first
    std::unordered_map<std::string,
                       std::pair<std::list<std::string>::iterator, std::shared_ptr<const CachedPlan>>>
        map_;
};

PlanCache g_plans;

struct KeyBuf {
    std::string s;
    template <typename T>
    void add(const T& v) { s.append(reinterpret_cast<const char*>(&v), sizeof(T)); }
    void add_bytes(const void* p, size_t n) { s.append(static_cast<const char*>(p), n); }
};

// Everything a plan depends on, field by field (no struct padding in the key).
std::string plan_key(int mode, const wf_probe* p, const wf_grid* g, int batch, int n_tx,
                     const int32_t* tx_elem, const double* angles, const double* t_start, int ns,
                     wf_dtype dtype, unsigned gen) {
    KeyBuf k;
    k.s.reserve(128 + (size_t)n_tx * 16);
    k.add(mode); k.add(gen); k.add(batch); k.add(n_tx); k.add(ns); k.add((int)dtype);
    k.add(p->n_elements); k.add(p->pitch); k.add(p->fs); k.add(p->c); k.add(p->f_number);
    k.add(p->apod);
    k.add(g->nz); k.add(g->nx); k.add(g->x_min); k.add(g->x_max); k.add(g->z_min); k.add(g->z_max);
    if (mode == 0) {
        k.add((int)(tx_elem != nullptr));
        if (tx_elem) k.add_bytes(tx_elem, (size_t)n_tx * sizeof(int32_t));
        k.add(t_start[0]);
    } else {
        k.add_bytes(angles, (size_t)n_tx * sizeof(double));
        k.add((int)(t_start != nullptr));
        if (t_start) k.add_bytes(t_start, (size_t)n_tx * sizeof(double));
    }
    return k.s;
}

wf_status get_plan(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch, int32_t n_tx,
                   const int32_t* tx_elem, const double* angles, const double* t_start,
                   int32_t n_samples, wf_dtype dtype, std::shared_ptr<const CachedPlan>& out);

// The delay-and-sum call of both transmit schemes: host checks, cached plan, launch.
// STAI passes tx_elem and t_start[0]; PWI passes angles and t_start[n_tx] (or NULL).
wf_status das_run(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch,
                  int32_t n_tx, const int32_t* tx_elem, const double* angles,
                  const double* t_start, int32_t n_rx, int32_t n_samples, wf_dtype dtype,
                  const void* rf, float rf_scale, float* out, void* ws, size_t ws_bytes,
                  wf_stream stream) {
    thread_local DasArgs A;  // ~18 KB parameter block, copied into the launch
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
    std::shared_ptr<const CachedPlan> e;
    if ((s = get_plan(mode, probe, grid, batch, n_tx, tx_elem, angles, t_start, n_samples, dtype, e)) !=
        WF_OK)
        return s;
    const Plan& P = e->P;
    if (!ws || ((uintptr_t)ws & 15u)) return WF_ERR_WORKSPACE;
    if (ws_bytes < P.ws_bytes) return WF_ERR_WORKSPACE;
    A = *e->A;
    A.g.elem_weight = probe->elem_weight;
    A.rf = rf;
    A.rf_scale = dtype == WF_I16 ? rf_scale : 1.0f;
    A.hdr = static_cast<WsHeader*>(ws);
    A.tile_info = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + kWsHeaderBytes);
    A.part = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeaderBytes + P.info_bytes);
    A.out = out;
    A.use_tmap = P.tiled && P.tma && !tuning().no_tmap &&
                 encode_rf_maps(A, rf, dtype, (long long)batch * n_tx, probe->n_elements, n_samples,
                                P.W, P.sym);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((s = cuda_status(cudaMemsetAsync(ws, 0, kWsHeaderBytes + P.info_bytes, st))) != WF_OK) return s;
    return mode == 0 ? dispatch<0>(A, P, batch, dtype, st) : dispatch<1>(A, P, batch, dtype, st);
}

// The cached plan of a call (built on a miss); arguments as das_run, already range-checked.
wf_status get_plan(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch, int32_t n_tx,
                   const int32_t* tx_elem, const double* angles, const double* t_start,
                   int32_t n_samples, wf_dtype dtype, std::shared_ptr<const CachedPlan>& out) {
    const Tuning tu = tuning();
    const std::string key =
        plan_key(mode, probe, grid, batch, n_tx, tx_elem, angles, t_start, n_samples, dtype, tu.gen);
    std::shared_ptr<const CachedPlan> e = g_plans.get(key);
    if (!e) {
        auto ne = std::make_shared<CachedPlan>();
        ne->A = std::make_unique<DasArgs>();
        DasArgs& T = *ne->A;
        std::memset(&T, 0, sizeof(T));
        const double extra = fill_tx(T, probe, mode, n_tx, tx_elem, angles, t_start, mode == 1);
        if (extra < 0.0) return WF_ERR_INVALID_ARG;
        if (2.0 * max_delay(probe, grid) + extra >= 4194304.0) return WF_ERR_UNSUPPORTED;
        const bool sym = use_sym(mode, n_tx, probe->n_elements, tx_elem);
        const Plan P = make_plan(mode, probe, grid, batch, n_tx, n_samples, dtype == WF_F32 ? 4 : 2, sym);
        ne->P = P;
        make_geom(probe, grid, T.g, T.gd);
        T.g.elem_weight = nullptr;
        T.n_tx = n_tx;
        T.ns = n_samples;
        T.tiles_x = P.tiles_x;
        T.tiles_z = P.tiles_z;
        T.n_groups = P.n_groups;
        T.n_items = P.n_items;
        T.sym = P.sym ? 1 : 0;
        T.W = P.W;
        T.ring = P.ring;
        T.frame_elems = (long long)n_tx * probe->n_elements * n_samples;
        T.use_table = 0;
        if (P.tiled && P.table) {
            T.use_table = 1;
            T.n_items = build_schedule(mode, probe, grid, P, T);
        }
        g_plans.put(key, ne);
        e = ne;
    }
    out = e;
    return WF_OK;
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

// Bounds over the tile rectangle [xlo, xhi] x [zlo, zhi] (samples) of the path of one
// (transmit, receive element) pair before the transmit offset, in double: the same
// convex-bound argument as the kernels' window planning (maximum on a bottom corner,
// minimum on the top edge at the clamped stationary point).
void pair_bounds_d(int mode, const GeomD& D, const TxInfo& ti, int e_t, int r, double xlo,
                   double xhi, double zlo, double zhi, double& mn, double& mx) {
    const double xr = D.xe0 + r * D.pitch;
    if (mode == 0) {
        const double xt = D.xe0 + e_t * D.pitch;
        const double xm = std::min(std::max(0.5 * (xt + xr), xlo), xhi);
        mn = std::hypot(xm - xt, zlo) + std::hypot(xm - xr, zlo);
        mx = std::max(std::hypot(xlo - xt, zhi) + std::hypot(xlo - xr, zhi),
                      std::hypot(xhi - xt, zhi) + std::hypot(xhi - xr, zhi));
        return;
    }
    const double sn = (double)ti.sin.hi + ti.sin.lo, cs = (double)ti.cos.hi + ti.cos.lo;
    const double xm = std::min(std::max(xr - zlo * sn / cs, xlo), xhi);
    mn = xm * sn + zlo * cs + std::hypot(xm - xr, zlo);
    mx = std::max(xlo * sn + zhi * cs + std::hypot(xlo - xr, zhi),
                  xhi * sn + zhi * cs + std::hypot(xhi - xr, zhi));
}

// Hull [lo, hi) over the whole frame of the samples the DAS kernels may stage
// from each trace [t][r] (lo >= hi: none), for every tile configuration, staging
// path and pairing a call with these arguments can select.  A superset by
// construction: element ranges one element wider than the kernels', every
// receive-chunk mate within 7 elements (for STAI also on the transmit side, which
// the reciprocal pairing stages from either end), and 24 / 32 samples of slack
// below / above the double-precision bounds for the kernels' FP32 bounds, their
// +-2 margins, 8-sample alignment and trailing neighbour segment.  A grid that
// sends a call to the per-pixel fallback needs whole traces.
void staged_hulls(int mode, const wf_probe* p, const wf_grid* g, const DasArgs& a, int n_tx,
                  const int32_t* tx_elem, int ns, int rf_bytes, std::vector<int>& lo,
                  std::vector<int>& hi) {
    const int E = p->n_elements;
    lo.assign((size_t)n_tx * E, ns);
    hi.assign((size_t)n_tx * E, 0);
    Geom G;
    GeomD D;
    make_geom(p, g, G, D);
    bool sym_possible = mode == 0 && n_tx == E;   // reciprocal pairing: every element fires, in order
    for (int t = 0; sym_possible && t < n_tx; ++t) sym_possible = (tx_elem ? tx_elem[t] : t) == t;
    const Cfg* cfgs = mode == 0 ? kStaiCfgs : kPwiCfgs;
    std::vector<Cfg> tiled;
    for (int sym = 0; sym <= (sym_possible ? 1 : 0); ++sym) {
        bool any = false;
        for (int i = 0; i < 2; ++i)
            if (plan_for(mode, cfgs[i], D, p, g, 1, n_tx, ns, rf_bytes, sym == 1).tiled) {
                any = true;
                if (std::find_if(tiled.begin(), tiled.end(), [&](const Cfg& c) {
                        return c.wcol == cfgs[i].wcol && c.p == cfgs[i].p; }) == tiled.end())
                    tiled.push_back(cfgs[i]);
            }
        if (!any) {   // the per-pixel fallback may read any sample
            std::fill(lo.begin(), lo.end(), 0);
            std::fill(hi.begin(), hi.end(), ns);
            return;
        }
    }
    // A tiling whose tiles split another's (same columns, rows a divisor) stages
    // subsets of the other's windows: its tiles are sub-rectangles with element
    // ranges no wider, so only the coarsest of such tilings is scanned.
    auto cols_of = [](const Cfg& c) { return 8 * c.wcol; };
    auto rows_of = [](const Cfg& c) { return (32 / c.wcol) * c.p; };
    std::sort(tiled.begin(), tiled.end(), [&](const Cfg& x, const Cfg& y) { return rows_of(x) > rows_of(y); });
    std::vector<Cfg> scan;
    for (const Cfg& c : tiled) {
        bool covered = false;
        for (const Cfg& o : scan)
            covered = covered || (cols_of(o) == cols_of(c) && rows_of(o) % rows_of(c) == 0);
        if (!covered) scan.push_back(c);
    }
    const double two_f = 2.0 * (p->apod == WF_APOD_NONE ? 1.0 : p->f_number);
    constexpr int kMate = kC - 1;
    std::vector<double> bmn, bmx, rmn, rmx;
    for (const Cfg& cfg : scan) {
        const int cols = cols_of(cfg), rows = rows_of(cfg);
        const int tiles_x = (g->nx + cols - 1) / cols, tiles_z = (g->nz + rows - 1) / rows;
        for (int tz = 0; tz < tiles_z; ++tz)
            for (int tx = 0; tx < tiles_x; ++tx) {
                const double xlo = D.gx0 + (double)(tx * cols) * D.gdx;
                const double xhi = D.gx0 + (double)(tx * cols + cols - 1) * D.gdx;
                const double zlo = D.gz0 + (double)(tz * rows) * D.gdz;
                const double zhi = D.gz0 + (double)(tz * rows + rows - 1) * D.gdz;
                int elo = 0, ehi = E - 1;
                if (p->apod != WF_APOD_NONE) {
                    if (!(zhi > 0.0)) continue;
                    const double half = zhi / two_f;
                    elo = std::max(0, (int)std::floor((xlo - half - D.xe0) / D.pitch) - 2);
                    ehi = std::min(E - 1, (int)std::ceil((xhi + half - D.xe0) / D.pitch) + 2);
                    if (elo > ehi) continue;
                }
                const int n_e = ehi - elo + 1;
                // transmit sides: elements (STAI, [n_e]) or angles (PWI, [n_tx]); bounds [side][receive]
                const int n_side = mode == 0 ? n_e : n_tx;
                bmn.assign((size_t)n_side * n_e, 0.0);
                bmx.assign((size_t)n_side * n_e, 0.0);
                for (int u = 0; u < n_side; ++u)
                    for (int r = 0; r < n_e; ++r)
                        pair_bounds_d(mode, D, a.tx[mode == 0 ? 0 : u], elo + u, elo + r, xlo, xhi, zlo,
                                      zhi, bmn[(size_t)u * n_e + r], bmx[(size_t)u * n_e + r]);
                // receive-chunk mates within kMate elements
                rmn.assign(bmn.size(), 0.0);
                rmx.assign(bmx.size(), 0.0);
                for (int u = 0; u < n_side; ++u)
                    for (int r = 0; r < n_e; ++r) {
                        double m0 = 1e300, m1 = -1e300;
                        for (int q = std::max(0, r - kMate); q <= std::min(n_e - 1, r + kMate); ++q) {
                            m0 = std::min(m0, bmn[(size_t)u * n_e + q]);
                            m1 = std::max(m1, bmx[(size_t)u * n_e + q]);
                        }
                        rmn[(size_t)u * n_e + r] = m0;
                        rmx[(size_t)u * n_e + r] = m1;
                    }
                for (int t = 0; t < n_tx; ++t) {
                    const int e_t = mode == 0 ? (tx_elem ? tx_elem[t] : t) : -1;
                    if (mode == 0 && (e_t < elo || e_t > ehi)) continue;
                    const double t0 = (double)a.tx[t].t0.hi + a.tx[t].t0.lo;
                    // STAI: transmit-side mates too when the reciprocal pairing can apply
                    const int u0 = mode == 0 ? (sym_possible ? std::max(0, e_t - elo - kMate) : e_t - elo) : t;
                    const int u1 = mode == 0 ? (sym_possible ? std::min(n_e - 1, e_t - elo + kMate) : e_t - elo) : t;
                    for (int r = 0; r < n_e; ++r) {
                        double m0 = 1e300, m1 = -1e300;
                        for (int u = u0; u <= u1; ++u) {
                            m0 = std::min(m0, rmn[(size_t)u * n_e + r]);
                            m1 = std::max(m1, rmx[(size_t)u * n_e + r]);
                        }
                        const double a0 = std::floor(m0 - t0) - 24.0, a1 = std::ceil(m1 - t0) + 32.0;
                        const int s0 = (int)std::max(0.0, std::min((double)ns, a0));
                        const int s1 = (int)std::max(0.0, std::min((double)ns, a1));
                        if (s0 >= s1) continue;
                        const size_t k = (size_t)t * E + elo + r;
                        lo[k] = std::min(lo[k], s0);
                        hi[k] = std::max(hi[k], s1);
                    }
                }
            }
    }
}

}  // namespace
}  // namespace wf

using namespace wf;

extern "C" wf_status wf_das_rf_boxes(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                     int32_t n_tx, const int32_t* tx_elem, const double* angles_rad,
                                     const double* t_start, int32_t n_rx, int32_t n_samples,
                                     wf_dtype dtype, int32_t group, wf_rf_box* boxes,
                                     int32_t max_boxes, int32_t* n_boxes) {
    thread_local DasArgs local;
    DasArgs& a = local;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (mode != 0 && mode != 1) return WF_ERR_INVALID_ARG;
    if (mode == 1 && !angles_rad) return WF_ERR_INVALID_ARG;
    if (n_tx < 1 || n_tx > WF_MAX_TX || n_rx != probe->n_elements) return WF_ERR_INVALID_ARG;
    if (n_samples < 1 || n_samples > WF_MAX_SAMPLES || group < 1 || !n_boxes) return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (max_boxes < 0 || (max_boxes > 0 && !boxes)) return WF_ERR_INVALID_ARG;
    if (fill_tx(a, probe, mode, n_tx, tx_elem, angles_rad, t_start, mode == 1) < 0.0) return WF_ERR_INVALID_ARG;
    std::vector<int> lo, hi;
    staged_hulls(mode, probe, grid, a, n_tx, tx_elem, n_samples, dtype == WF_F32 ? 4 : 2, lo, hi);
    const int E = probe->n_elements;
    int n = 0;
    for (int t0 = 0; t0 < n_tx; t0 += group) {
        const int t1 = std::min(n_tx, t0 + group);
        int r0 = E, r1 = -1, s0 = n_samples, s1 = 0;
        for (int t = t0; t < t1; ++t)
            for (int r = 0; r < E; ++r) {
                const size_t k = (size_t)t * E + r;
                if (lo[k] >= hi[k]) continue;
                r0 = std::min(r0, r);
                r1 = std::max(r1, r);
                s0 = std::min(s0, lo[k]);
                s1 = std::max(s1, hi[k]);
            }
        if (r1 < r0) continue;
        s0 &= ~7;                                        // 8-sample (16-byte for 16-bit RF) ends
        s1 = std::min(n_samples, (s1 + 7) & ~7);
        if (n < max_boxes) boxes[n] = wf_rf_box{t0, t1, r0, r1 + 1, s0, s1};
        ++n;
    }
    *n_boxes = n;
    return n > max_boxes && max_boxes > 0 ? WF_ERR_INVALID_ARG : WF_OK;
}

extern "C" wf_status wf_copy_rf_boxes(const void* src, void* dst, int32_t n_tx, int32_t n_rx,
                                      int32_t n_samples, int32_t elem_bytes, const wf_rf_box* boxes,
                                      int32_t n_boxes, wf_stream stream) {
    if (!src || !dst || n_tx < 1 || n_rx < 1 || n_samples < 1 || n_boxes < 0 || (n_boxes > 0 && !boxes))
        return WF_ERR_INVALID_ARG;
    if (elem_bytes != 2 && elem_bytes != 4) return WF_ERR_INVALID_ARG;
    for (int i = 0; i < n_boxes; ++i) {
        const wf_rf_box& b = boxes[i];
        if (b.t0 < 0 || b.t1 > n_tx || b.t0 >= b.t1 || b.r0 < 0 || b.r1 > n_rx || b.r0 >= b.r1 ||
            b.s0 < 0 || b.s1 > n_samples || b.s0 >= b.s1)
            return WF_ERR_INVALID_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t pitch = (size_t)n_samples * elem_bytes;
    for (int i = 0; i < n_boxes; ++i) {
        const wf_rf_box& b = boxes[i];
        cudaMemcpy3DParms P{};
        P.srcPtr = make_cudaPitchedPtr(const_cast<void*>(src), pitch, pitch, (size_t)n_rx);
        P.dstPtr = make_cudaPitchedPtr(dst, pitch, pitch, (size_t)n_rx);
        P.srcPos = make_cudaPos((size_t)b.s0 * elem_bytes, (size_t)b.r0, (size_t)b.t0);
        P.dstPos = P.srcPos;
        P.extent = make_cudaExtent((size_t)(b.s1 - b.s0) * elem_bytes, (size_t)(b.r1 - b.r0),
                                   (size_t)(b.t1 - b.t0));
        P.kind = cudaMemcpyDefault;
        const wf_status s = cuda_status(cudaMemcpy3DAsync(&P, st));
        if (s != WF_OK) return s;
    }
    return WF_OK;
}

extern "C" size_t wf_das_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                         int32_t n_tx) {
    if (check_probe_grid(probe, grid) != WF_OK || batch < 1 || n_tx < 1 || n_tx > WF_MAX_TX) return 0;
    // Enough for every configuration either transmit scheme may pick.
    Geom G;
    GeomD D;
    make_geom(probe, grid, G, D);
    size_t need = kWsHeaderBytes;
    for (const Cfg& c : kStaiCfgs)
        need = std::max(need, plan_for(0, c, D, probe, grid, batch, n_tx, 8, 4, false).ws_bytes);
    for (const Cfg& c : kPwiCfgs)
        need = std::max(need, plan_for(1, c, D, probe, grid, batch, n_tx, 8, 4, false).ws_bytes);
    return need;
}

extern "C" wf_status wf_das_stai(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                 int32_t n_tx, const int32_t* tx_elem, int32_t n_rx,
                                 int32_t n_samples, double t_start, wf_dtype dtype, const void* rf,
                                 float rf_scale, float* out, void* ws, size_t ws_bytes,
                                 wf_stream stream) {
    if (!probe || !std::isfinite(t_start)) return WF_ERR_INVALID_ARG;
    return das_run(0, probe, grid, batch, n_tx, tx_elem, nullptr, &t_start, n_rx, n_samples, dtype,
                   rf, rf_scale, out, ws, ws_bytes, stream);
}

extern "C" wf_status wf_das_pwi(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                int32_t n_angles, const double* angles_rad, const double* t_start,
                                int32_t n_rx, int32_t n_samples, wf_dtype dtype, const void* rf,
                                float rf_scale, float* out, void* ws, size_t ws_bytes,
                                wf_stream stream) {
    if (!probe || !angles_rad) return WF_ERR_INVALID_ARG;
    return das_run(1, probe, grid, batch, n_angles, nullptr, angles_rad, t_start, n_rx, n_samples,
                   dtype, rf, rf_scale, out, ws, ws_bytes, stream);
}

extern "C" wf_status wf_das_plan(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                 int32_t reverse, int32_t batch, int32_t n_tx, const int32_t* tx_elem,
                                 const double* angles_rad, const double* t_start, int32_t n_samples,
                                 wf_dtype dtype, wf_das_plan_info* info) {
    if (!info || (mode != 0 && mode != 1) || (mode == 1 && !angles_rad)) return WF_ERR_INVALID_ARG;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (batch < 1 || batch > 65535 || n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    if (n_samples < 1 || n_samples > WF_MAX_SAMPLES) return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    const double t0 = 0.0;
    const double* ts = mode == 0 ? (t_start ? t_start : &t0) : t_start;
    std::memset(info, 0, sizeof(*info));
    if (reverse) {
        thread_local DasArgs a;
        const double extra = fill_tx(a, probe, mode, n_tx, tx_elem, angles_rad, ts, mode == 1);
        if (extra < 0.0) return WF_ERR_INVALID_ARG;
        GeomD D;
        make_geom(probe, grid, a.g, D);
        const bool sym = use_sym(mode, n_tx, probe->n_elements, tx_elem);
        const Plan P = plan_for(mode, Cfg{4, 2}, D, probe, grid, batch, n_tx, n_samples, 4, sym);
        info->tiled = backward_is_tiled(P, probe->n_elements, true) ? 1 : 0;
        info->tile_cols = P.cols;
        info->tile_rows = P.rows;
        info->window = P.W;
        info->reciprocal = P.sym ? 1 : 0;
        info->ctas_per_frame = info->tiled ? P.n_items : 0;
        return WF_OK;
    }
    std::shared_ptr<const CachedPlan> e;
    if ((s = get_plan(mode, probe, grid, batch, n_tx, tx_elem, angles_rad, ts, n_samples, dtype, e)) !=
        WF_OK)
        return s;
    const Plan& P = e->P;
    info->tiled = P.tiled ? 1 : 0;
    info->tile_cols = P.cols;
    info->tile_rows = P.rows;
    info->window = P.W;
    info->ring = P.tiled && P.tma ? P.ring : 0;
    info->reciprocal = P.sym ? 1 : 0;
    info->ctas_per_frame = P.tiled ? e->A->n_items : 0;
    info->smem_bytes = P.tiled ? (int32_t)P.smem : 0;
    info->workspace_bytes = (int64_t)P.ws_bytes;
    return WF_OK;
}

// ---------------------------------------------------------------------------
// Delay-and-sum of IQ data: the RF path's geometry and tiles in baseband samples
// (fs / D), kernels in das_iq.cu.
// ---------------------------------------------------------------------------
namespace wf {
namespace {

wf_status das_iq_prepare(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch,
                         int32_t n_tx, const int32_t* tx_elem, const double* angles,
                         const double* t_start, int32_t n_rx, int32_t m_samples, int32_t decim,
                         double f0, DasArgs& A, size_t& ws_need) {
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (batch < 1 || batch > 65535 || n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    if (n_rx != probe->n_elements || m_samples < 2 || m_samples > WF_MAX_SAMPLES) return WF_ERR_INVALID_ARG;
    if (decim < 1 || decim > 64 || !std::isfinite(f0)) return WF_ERR_INVALID_ARG;
    if (mode == 1 && !angles) return WF_ERR_INVALID_ARG;
    wf_probe pb = *probe;
    pb.fs = probe->fs / decim;                       // baseband samples
    std::memset(&A, 0, offsetof(DasArgs, tx));
    const double extra = fill_tx(A, &pb, mode, n_tx, tx_elem, angles, t_start, mode == 1);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    if (2.0 * max_delay(&pb, grid) + extra >= 4194304.0) return WF_ERR_UNSUPPORTED;
    GeomD D;
    make_geom(&pb, grid, A.g, D);
    make_geom(&pb, grid, A.g, A.gd);
    const Plan P = plan_for(mode, Cfg{4, 2}, D, &pb, grid, batch, n_tx, m_samples, 8, false);
    if (!P.tiled || iq_smem_bytes(P.W, probe->n_elements) > kMaxTiledSmem) return WF_ERR_UNSUPPORTED;
    A.n_tx = n_tx;
    A.ns = m_samples;
    A.tiles_x = P.tiles_x;
    A.tiles_z = P.tiles_z;
    A.n_groups = std::max(1, std::min(kMaxGroups, P.n_groups));
    A.n_items = P.tiles_x * P.tiles_z * A.n_groups;
    A.W = P.W;
    A.sym = 0;
    A.use_table = 0;
    A.use_tmap = 0;
    A.frame_elems = (long long)n_tx * probe->n_elements * m_samples;
    A.iq_k = df_from_double(f0 * decim / probe->fs);
    ws_need = kWsHeaderBytes + (size_t)batch * A.n_items * kThreads * 2 * 2 * sizeof(float);
    return WF_OK;
}

wf_status das_iq_run(int mode, const wf_probe* probe, const wf_grid* grid, int32_t batch,
                     int32_t n_tx, const int32_t* tx_elem, const double* angles,
                     const double* t_start, int32_t n_rx, int32_t m_samples, int32_t decim,
                     double f0, const float* iq, float* out, void* ws, size_t ws_bytes,
                     wf_stream stream) {
    thread_local DasArgs A;
    size_t need = 0;
    wf_status s = das_iq_prepare(mode, probe, grid, batch, n_tx, tx_elem, angles, t_start, n_rx,
                                 m_samples, decim, f0, A, need);
    if (s != WF_OK) return s;
    if (!iq || !out || ((uintptr_t)iq & 7u) || ((uintptr_t)out & 7u)) return WF_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws & 15u) || ws_bytes < need) return WF_ERR_WORKSPACE;
    A.g.elem_weight = probe->elem_weight;
    A.rf = iq;
    A.rf_scale = 1.0f;
    A.hdr = static_cast<WsHeader*>(ws);
    A.part = reinterpret_cast<float*>(static_cast<char*>(ws) + kWsHeaderBytes);
    A.out = out;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((s = cuda_status(cudaMemsetAsync(ws, 0, kWsHeaderBytes, st))) != WF_OK) return s;
    return mode == 0 ? launch_das_iq<0>(A, batch, out, st) : launch_das_iq<1>(A, batch, out, st);
}

}  // namespace
}  // namespace wf

extern "C" size_t wf_das_iq_workspace_bytes(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                            int32_t batch, int32_t n_tx, int32_t m_samples,
                                            int32_t decim) {
    thread_local DasArgs A;
    if ((mode != 0 && mode != 1) || n_tx < 1 || n_tx > WF_MAX_TX) return 0;
    std::vector<double> ang(n_tx, 0.0);
    const double t0 = 0.0;   // STAI: one start time; plane waves: NULL, every angle at 0
    size_t need = 0;
    if (das_iq_prepare(mode, probe, grid, batch, n_tx, nullptr, ang.data(), mode == 0 ? &t0 : nullptr,
                       probe ? probe->n_elements : 0, m_samples, decim, 0.0, A, need) != WF_OK)
        return 0;
    return need;
}

extern "C" wf_status wf_das_stai_iq(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                    int32_t n_tx, const int32_t* tx_elem, int32_t n_rx,
                                    int32_t m_samples, int32_t decim, double f0, double t_start,
                                    const float* iq, float* out, void* ws, size_t ws_bytes,
                                    wf_stream stream) {
    if (!probe || !std::isfinite(t_start)) return WF_ERR_INVALID_ARG;
    return das_iq_run(0, probe, grid, batch, n_tx, tx_elem, nullptr, &t_start, n_rx, m_samples,
                      decim, f0, iq, out, ws, ws_bytes, stream);
}

extern "C" wf_status wf_das_pwi_iq(const wf_probe* probe, const wf_grid* grid, int32_t batch,
                                   int32_t n_angles, const double* angles_rad, const double* t_start,
                                   int32_t n_rx, int32_t m_samples, int32_t decim, double f0,
                                   const float* iq, float* out, void* ws, size_t ws_bytes,
                                   wf_stream stream) {
    if (!probe || !angles_rad) return WF_ERR_INVALID_ARG;
    return das_iq_run(1, probe, grid, batch, n_angles, nullptr, angles_rad, t_start, n_rx,
                      m_samples, decim, f0, iq, out, ws, ws_bytes, stream);
}

extern "C" wf_status wf_iq_envelope(const float* img, int32_t batch, int32_t nz, int32_t nx,
                                    float* env, float* frame_max, wf_stream stream) {
    if (!img || !env || batch < 1 || nz < 1 || nx < 1 || ((uintptr_t)img & 7u) || ((uintptr_t)env & 3u))
        return WF_ERR_INVALID_ARG;
    if (frame_max && ((uintptr_t)frame_max & 3u)) return WF_ERR_INVALID_ARG;
    return launch_iq_envelope(img, batch, (long long)nz * nx, env, frame_max,
                              reinterpret_cast<cudaStream_t>(stream));
}

extern "C" wf_status wf_das_reload_tuning(void) {
    {
        std::lock_guard<std::mutex> lk(g_tuning_mu);
        read_tuning_locked();
    }
    g_plans.clear();
    return WF_OK;
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
    a.sym = use_sym(mode, n_tx, probe->n_elements, tx_elem) ? 1 : 0;
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

extern "C" wf_status wf_das_backward(const wf_probe* probe, const wf_grid* grid, int32_t mode,
                                    int32_t batch, int32_t n_tx, const int32_t* tx_elem,
                                    const double* angles_rad, const double* t_start, int32_t n_rx,
                                    int32_t n_samples, const float* rf, const float* grad_out,
                                    float* grad_rf, float* grad_weight, float* grad_c,
                                    wf_stream stream) {
    thread_local DasArgs local;
    DasArgs& a = local;
    wf_status s = check_probe_grid(probe, grid);
    if (s != WF_OK) return s;
    if (mode != 0 && mode != 1) return WF_ERR_INVALID_ARG;
    if (mode == 1 && !angles_rad) return WF_ERR_INVALID_ARG;
    if (batch < 1 || batch > 65535 || n_tx < 1 || n_tx > WF_MAX_TX) return WF_ERR_INVALID_ARG;
    if (n_rx != probe->n_elements || n_samples < 1 || n_samples > WF_MAX_SAMPLES)
        return WF_ERR_INVALID_ARG;
    if (!rf || !grad_out || ((uintptr_t)rf & 15u) || ((uintptr_t)grad_out & 3u))
        return WF_ERR_INVALID_ARG;
    if (((uintptr_t)grad_rf & 3u) || ((uintptr_t)grad_weight & 3u) || ((uintptr_t)grad_c & 3u))
        return WF_ERR_INVALID_ARG;
    const double extra = fill_tx(a, probe, mode, n_tx, tx_elem, angles_rad, t_start, mode == 1);
    if (extra < 0.0) return WF_ERR_INVALID_ARG;
    if (2.0 * max_delay(probe, grid) + extra >= 4194304.0) return WF_ERR_UNSUPPORTED;
    const bool sym = use_sym(mode, n_tx, probe->n_elements, tx_elem);
    GeomD D;
    make_geom(probe, grid, a.g, D);
    make_geom(probe, grid, a.g, a.gd);
    const Plan P = plan_for(mode, Cfg{4, 2}, D, probe, grid, batch, n_tx, n_samples, 4, sym);
    a.n_tx = n_tx;
    a.ns = n_samples;
    a.tiles_x = P.tiles_x;
    a.tiles_z = P.tiles_z;
    a.n_groups = P.n_groups;
    a.n_items = P.n_items;
    a.W = P.W;
    a.ring = 1;
    a.sym = P.sym ? 1 : 0;
    a.rf = rf;
    a.rf_scale = 1.0f;
    a.frame_elems = (long long)n_tx * probe->n_elements * n_samples;
    a.part = nullptr;
    a.out = nullptr;
    a.hdr = nullptr;
    a.use_table = 0;
    a.tile_info = nullptr;
    a.grad_out = grad_out;
    a.grad_rf = grad_rf;
    a.grad_w = grad_weight;
    a.grad_c = grad_c;
    a.neg_inv_c = (float)(-1.0 / probe->c);
    a.use_tmap = P.tiled && n_samples % 8 == 0 && !tuning().no_tmap &&
                 encode_rf_maps(a, rf, WF_F32, (long long)batch * n_tx, probe->n_elements, n_samples,
                                P.W, P.sym);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (grad_rf &&
        (s = cuda_status(cudaMemsetAsync(grad_rf, 0, (size_t)batch * a.frame_elems * sizeof(float), st))) != WF_OK)
        return s;
    if (grad_weight &&
        (s = cuda_status(cudaMemsetAsync(grad_weight, 0, (size_t)probe->n_elements * sizeof(float), st))) != WF_OK)
        return s;
    if (grad_c && (s = cuda_status(cudaMemsetAsync(grad_c, 0, sizeof(float), st))) != WF_OK) return s;
    const bool need_par = grad_weight || grad_c;
    return mode == 0 ? launch_das_backward<0>(a, P, batch, grad_rf != nullptr, need_par, st)
                     : launch_das_backward<1>(a, P, batch, grad_rf != nullptr, need_par, st);
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
// current (in host code the symbol is only a host-side stand-in).  The pointer is
// published with an atomic store and read with an atomic load, so two host threads
// making their first call on one device at once never race on it.
constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};

wf_status fixed_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WF_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return WF_ERR_UNSUPPORTED;
    void* p = __atomic_load_n(&g_scratch_ptr[dev], __ATOMIC_ACQUIRE);
    if (!p) {
        if (cudaGetSymbolAddress(&p, g_fixed_scratch) != cudaSuccess || !p) return WF_ERR_CUDA;
        __atomic_store_n(&g_scratch_ptr[dev], p, __ATOMIC_RELEASE);
    }
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
    // The checks of wf_das_stai that need no pointer come first, so a bad size, count
    // or value returns WF_ERR_INVALID_ARG exactly as there; the size refusal follows
    // and precedes the pointer checks (an oversized call never looks at rf or out).
    if (!probe || !std::isfinite(t_start)) return WF_ERR_INVALID_ARG;
    if (check_probe_grid(probe, grid) != WF_OK || batch < 1 || batch > 65535 || n_tx < 1 ||
        n_tx > WF_MAX_TX)
        return WF_ERR_INVALID_ARG;
    if (n_rx != probe->n_elements || n_samples < 1 || n_samples > WF_MAX_SAMPLES)
        return WF_ERR_INVALID_ARG;
    if (dtype != WF_F32 && dtype != WF_F16 && dtype != WF_I16) return WF_ERR_INVALID_ARG;
    if (dtype == WF_I16 && !std::isfinite(rf_scale)) return WF_ERR_INVALID_ARG;
    if (tx_elem)
        for (int t = 0; t < n_tx; ++t)
            if (tx_elem[t] < 0 || tx_elem[t] >= probe->n_elements) return WF_ERR_INVALID_ARG;
    const Plan P = make_plan(0, probe, grid, batch, n_tx, n_samples, dtype == WF_F32 ? 4 : 2,
                             use_sym(0, n_tx, probe->n_elements, tx_elem));
    if (P.ws_bytes > kFixedScratchBytes) return WF_ERR_WORKSPACE;
    void* ws = nullptr;
    const wf_status s = fixed_scratch(&ws);
    if (s != WF_OK) return s;
    return wf_das_stai(probe, grid, batch, n_tx, tx_elem, n_rx, n_samples, t_start, dtype, rf,
                       rf_scale, out, ws, kFixedScratchBytes, stream);
}

extern "C" size_t wf_fixed_scratch_bytes(void) { return kFixedScratchBytes; }

extern "C" wf_status wf_fixed_scratch_check(wf_stream stream) {
    void* ws = nullptr;
    const wf_status s = fixed_scratch(&ws);
    if (s != WF_OK) return s;
    const wf_status r = wf_workspace_check(ws, kFixedScratchBytes, stream);
    if (r == WF_ERR_CUDA) return r;
    // clear the status block so the next check reports only what follows it
    if (cudaMemset(ws, 0, kWsHeaderBytes) != cudaSuccess) return WF_ERR_CUDA;
    return r;
}
