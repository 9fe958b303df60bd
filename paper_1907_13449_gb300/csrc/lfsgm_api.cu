// lfsgm_api.cu -- the C ABI declared in include/lfsgm.h: handle, configuration checks,
// host-built shift tables, workspace, launch accounting and the stage entry points.
//
// Host arithmetic that decides integers (shift tables, label grids) is done in double
// precision with FMA contraction disabled (-ffp-contract=off), so the tables are the same
// on x86 and Arm hosts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <string>

#include "../../include/lfsgm.h"
#include "lfsgm_internal.cuh"

using namespace lfsgm;

namespace {

struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Windowed rows (cost, agg, grad_cost) are read and written as 16-byte vectors: their base must be
// 16-byte aligned, or the off[p] multiple-of-4 rows would not be.
bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

// ---- shift split of a*d (see lfsgm.h): snap 2s to an integer within 2e-9, then floor / round-half-up
void shift_split(int a, double d, int &o, double &f, int &n) {
    double s = (double)a * d;
    const double t = 2.0 * s;
    const double r = std::nearbyint(t);
    if (std::fabs(t - r) <= 2e-9) s = 0.5 * r;
    const double fl = std::floor(s);
    o = (int)fl;
    f = s - fl;
    n = (int)std::floor(s + 0.5);
}

double grid_disp(double dmin, double dmax, int L, int k) {
    const double step = (dmax - dmin) / (double)(L - 1);
    return dmin + (double)k * step;
}

}  // namespace

struct lfsgm_ctx {
    lfsgm_config cfg{};
    cudaStream_t stream = nullptr;
    int N = 0, nviews = 0, ref = 0, nbits = 0, Lcd = 0;
    int C = 1;                            // colour channels; images are planes view * C + c
    ArmList arms{};
    // tuning knobs (lfsgm_set_tuning): label span of the row kernel's ranges, list-kernel CTAs per SM
    int row_kw = 36, list_ctas = 0, sgm_warps = 4;
    // scanlines that cross at least this many windows wider than 32 labels run split across a CTA's
    // warps (lfsgm_set_sgm_split; 0: none)
    int sgm_split = 0;
    std::vector<FineTap> h_fine;          // host copy of the shift table (row descriptors are rebuilt from it)
    // device tables
    FineTap *d_fine = nullptr;
    unsigned char *d_rowdesc = nullptr;   // row-kernel descriptors per (view, g0)
    int *d_order = nullptr;               // SGM scanlines, longest first
    int4 *d_ltab = nullptr;               // taps as linear offsets in the padded images (list kernel)
    int *d_otab = nullptr;       // coarse census offsets per (arm view, label), see CoarseArms
    CoarseArms ca{};
    int *d_armviews = nullptr;   // [4][kMaxArmViews]
    int *d_sel_cross = nullptr;  // the reference and the arm views
    int n_sel_cross = 0;
    int *d_sel_all = nullptr;    // every view
    int *d_sel_rest = nullptr;   // the views that are not in d_sel_cross
    int n_sel_rest = 0;
    // workspace
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = false;
    void *ccost = nullptr;                // coarse arm costs, uint8 when they fit a byte (cost8), else uint16
    bool cost8 = false;
    uint16_t *csum = nullptr;
    int *maps = nullptr, *F0 = nullptr, *F1 = nullptr, *cntpad = nullptr;
    int2 *wide_list = nullptr;         // (pixel, 32-label chunk) items for the list kernel
    int *wide_count = nullptr;
    RowPlanHost rows{};                // row-sweep cost kernel plan + tensor maps
    bool rows_maps = false;            // tensor maps encoded for the bound workspace
    float *views_pad = nullptr;        // edge-replicated padded copies (workspace)
    uint64_t *cen_pad = nullptr;
    unsigned long long *armsum = nullptr;
    int *cpen = nullptr;
    float *fpen = nullptr;
    double *partial = nullptr;
    unsigned *ticket = nullptr;           // last-block counter of the penalty mean (zero between launches)
    long long *tsum = nullptr;
    int *split = nullptr;                 // SGM scanlines split across a CTA (sgm_split_ints)
    int *status = nullptr;
    // buffers of the whole-method entry points (owned, allocated on first use)
    int *o_lo = nullptr, *o_cnt = nullptr, *o_label = nullptr;
    long long *o_off = nullptr;
    float *o_cost = nullptr, *o_agg = nullptr, *o_disp = nullptr, *o_views = nullptr;
    cudaStream_t up = nullptr;            // upload stream of lfsgm_depth_host (the non-cross views)
    cudaEvent_t up_done = nullptr;
    // backward scratch (allocated on the first lfsgm_backward): aggregate, dLoss/dC_s, branch codes
    // of the 8 or 16 directions, argmin slots, penalty gradients
    float *b_agg = nullptr, *b_gcs = nullptr, *b_gp = nullptr;
    unsigned char *b_codes = nullptr;
    int *b_amin = nullptr;
    // what the branch codes and argmin slots were recorded from (lfsgm_sgm_aggregate_record)
    struct {
        bool valid = false;
        const float *cost = nullptr, *agg = nullptr;
        const int32_t *lo = nullptr, *cnt = nullptr;
        const int64_t *off = nullptr;
        float P1 = 0.f, P2 = 0.f;
    } rec;
    // accounting
    long long launches = 0;
    bool profiling = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> pool;
    std::string err;
};

namespace {

thread_local std::string g_create_err;  // error text of a failed lfsgm_create

lfsgm_status fail(lfsgm_ctx *h, lfsgm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return st;
}

lfsgm_status cuda_fail(lfsgm_ctx *h, cudaError_t e, const char *what) {
    return fail(h, LFSGM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaEvent_t get_event(lfsgm_ctx *h) {
    if (!h->pool.empty()) {
        cudaEvent_t e = h->pool.back();
        h->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run one launcher: count it and, when profiling, bracket it with events.
template <class F>
lfsgm_status run(lfsgm_ctx *h, const char *name, F &&launch) {
    ProfRec rec{name, nullptr, nullptr};
    if (h->profiling) {
        rec.a = get_event(h);
        rec.b = get_event(h);
        cudaEventRecord(rec.a, h->stream);
    }
    const cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(h, e, name);
    h->launches++;
    if (h->profiling) {
        cudaEventRecord(rec.b, h->stream);
        h->prof.push_back(rec);
    }
    return LFSGM_OK;
}

#define LFSGM_TRY(x)                          \
    do {                                      \
        const lfsgm_status _st = (x);         \
        if (_st != LFSGM_OK) return _st;      \
    } while (0)

lfsgm_status validate(const lfsgm_config &c, char *why, size_t n) {
#define BAD(...) do { snprintf(why, n, __VA_ARGS__); return LFSGM_ERR_INVALID_ARG; } while (0)
    if (c.U < 1 || c.V < 1 || c.U * c.V < 2) BAD("need at least 2 views (U=%d V=%d)", c.U, c.V);
    if (c.U > 64 || c.V > 64) BAD("at most 64 x 64 views");
    if (c.H < 1 || c.W < 1 || (long long)c.H * c.W > (1LL << 28)) BAD("bad image size %dx%d", c.H, c.W);
    if (c.uc < 0 || c.uc >= c.U || c.vc < 0 || c.vc >= c.V) BAD("reference view out of range");
    if (c.census_w != 5 && c.census_w != 7) BAD("census_w must be 5 or 7");
    if (!(c.dmax > c.dmin) || !std::isfinite(c.dmin) || !std::isfinite(c.dmax)) BAD("need dmin < dmax");
    if (c.coarse_labels < 2 || c.coarse_labels > 256) BAD("coarse_labels must be in [2, 256]");
    if (c.fine_labels < 2 || c.fine_labels > 4096) BAD("fine_labels must be in [2, 4096]");
    if (c.fine_radius < 0) BAD("fine_radius must be >= 0");
    if (!(c.phi > 0.0)) BAD("phi must be > 0");
    if (c.fill_passes < 0 || c.fill_passes > 8) BAD("fill_passes must be in [0, 8]");
    if (!(c.w_l2 >= 0.f) || !(c.w_census >= 0.f) || !std::isfinite(c.w_l2) || !std::isfinite(c.w_census))
        BAD("cost weights must be finite and >= 0");
    if (!(c.p1_frac >= 0.0) || !(c.p2_frac >= c.p1_frac)) BAD("need 0 <= p1_frac <= p2_frac");
    if (c.subpixel < 0 || c.subpixel > 2) BAD("subpixel must be 0, 1 or 2");
    if (!(c.softmin_tau > 0.f)) BAD("softmin_tau must be > 0");
    if (c.paths != 0 && c.paths != 8 && c.paths != 16) BAD("paths must be 8 or 16");
    if (c.channels != 0 && c.channels != 1 && c.channels != 3) BAD("channels must be 1 or 3");
    if (c.boundless != 0 && c.boundless != 1) BAD("boundless must be 0 or 1");
    if (!(c.edge_threshold >= 0.f) || !std::isfinite(c.edge_threshold)) BAD("edge_threshold must be finite and >= 0");
    const double md = std::fmax(std::fabs(c.dmin), std::fabs(c.dmax));
    if (md * (std::max(c.U, c.V)) > 30000.0) BAD("shifts exceed the 16-bit table range");
    return LFSGM_OK;
#undef BAD
}

void build_arms(lfsgm_ctx *h) {
    const lfsgm_config &c = h->cfg;
    ArmList &A = h->arms;
    A.n_arms = 0;
    for (int arm = 0; arm < 4; arm++) {
        int n = 0;
        int *out = A.views[A.n_arms];
        auto add = [&](int u, int v) { out[n++] = v * c.U + u; };
        if (arm == 0) {
            for (int v = c.vc - 1; v >= 0; v--) if (c.init_views || v == 0) add(c.uc, v);
        } else if (arm == 1) {
            for (int v = c.vc + 1; v < c.V; v++) if (c.init_views || v == c.V - 1) add(c.uc, v);
        } else if (arm == 2) {
            for (int u = c.uc - 1; u >= 0; u--) if (c.init_views || u == 0) add(u, c.vc);
        } else {
            for (int u = c.uc + 1; u < c.U; u++) if (c.init_views || u == c.U - 1) add(u, c.vc);
        }
        if (n > 0) {
            A.arm_id[A.n_arms] = arm;
            A.nv[A.n_arms] = n;
            A.n_arms++;
        }
    }
}

lfsgm_status bind_workspace(lfsgm_ctx *h, void *dptr, size_t bytes, bool owned);

lfsgm_status ensure_workspace(lfsgm_ctx *h) {
    if (h->ws) return LFSGM_OK;
    size_t bytes = 0;
    lfsgm_workspace_size(h, &bytes);
    void *p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(h, LFSGM_ERR_NO_MEMORY, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    return bind_workspace(h, p, bytes, true);
}

int max_arm_views(const lfsgm_ctx *h) {
    int m = 0;
    for (int a = 0; a < h->arms.n_arms; a++) m = std::max(m, h->arms.nv[a]);
    return m;
}

}  // namespace


namespace {
lfsgm_status bind_workspace(lfsgm_ctx *h, void *dptr, size_t bytes, bool owned) {
    size_t need = 0;
    lfsgm_workspace_size(h, &need);
    if (bytes < need || ((uintptr_t)dptr & 255))
        return fail(h, LFSGM_ERR_WORKSPACE, "workspace needs %zu bytes, 256-byte aligned", need);
    if (h->ws && h->ws_owned && h->ws != dptr) cudaFree(h->ws);
    h->ws = dptr;
    h->ws_bytes = bytes;
    h->ws_owned = owned;
    const size_t N = (size_t)h->N, A = (size_t)std::max(h->arms.n_arms, 1);
    char *p = (char *)dptr;
    auto take = [&](size_t n) { char *q = p; p += align256(n); return (void *)q; };
    // the status word and the penalty-mean ticket come first, so handles that share one workspace (a
    // batch branch) share them: every layout agrees on these two words (the ticket is zero between
    // launches, and another handle's layout may overlay anything after them)
    h->status = (int *)take(4);
    h->ticket = (unsigned *)take(4);
    const size_t HWp = (size_t)h->rows.Hp * h->rows.Wp;
    h->cen_pad = (uint64_t *)take((size_t)h->nviews * h->C * HWp * 8);
    h->views_pad = (float *)take((size_t)h->nviews * HWp * (h->C > 1 ? 16 : 4));   // colour: float4 per pixel
    h->rows_maps = h->rows.ok && encode_fine_rows_maps(&h->rows, h->views_pad, h->cen_pad, h->nviews);
    h->ccost = take(A * N * h->Lcd * (h->cost8 ? 1 : 2));
    h->csum = (uint16_t *)take(A * N * h->Lcd * 2);
    h->maps = (int *)take(4 * N * 4);
    h->F0 = (int *)take(N * 4);
    h->F1 = (int *)take(N * 4);
    h->cntpad = (int *)take(N * 4);
    h->wide_list = (int2 *)take(N * (size_t)((h->cfg.fine_labels + 31) / 32) * 8);
    h->wide_count = (int *)take(4);
    h->armsum = (unsigned long long *)take(4 * 8);
    h->cpen = (int *)take(8 * 4);
    h->fpen = (float *)take(2 * 4);
    h->partial = (double *)take(2 * kPartialBlocks * 8);
    h->tsum = (long long *)take((size_t)scan_tiles(h->N) * 8);
    h->split = (int *)take((size_t)sgm_split_ints(h->cfg.H, h->cfg.W, h->cfg.paths) * 4);
    cudaError_t e = cudaMemsetAsync(h->status, 0, 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ticket, 0, 4, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "status clear");
    return LFSGM_OK;
}

// The host-side part of handle creation: defaults, validation and every size the workspace layout
// depends on (no device memory, no tables).  lfsgm_create continues from here; the batch workspace
// query uses it alone.
lfsgm_status plan_handle(const lfsgm_config &cin, lfsgm_ctx *h) {
    lfsgm_config c = cin;
    if (c.paths == 0) c.paths = 8;
    if (c.channels == 0) c.channels = 1;
    if (c.uc < 0) c.uc = (c.U - 1) / 2;
    if (c.vc < 0) c.vc = (c.V - 1) / 2;
    char why[256];
    if (validate(c, why, sizeof why) != LFSGM_OK) {
        g_create_err = why;
        return LFSGM_ERR_INVALID_ARG;
    }
    h->cfg = c;
    h->N = c.H * c.W;
    h->nviews = c.U * c.V;
    h->C = c.channels;
    h->ref = c.vc * c.U + c.uc;
    h->nbits = c.census_w * c.census_w - 1;
    h->Lcd = coarse_stride(c.coarse_labels);
    plan_fine_rows(c.U, c.V, c.uc, c.vc, c.H, c.W, c.fine_labels, c.dmin, c.dmax, h->row_kw, h->C, &h->rows);
    build_arms(h);
    // the packed coarse sums hold (paths) x (C + P2) per 16-bit half
    const long long cmax = (long long)max_arm_views(h) * h->nbits * h->C;
    h->cost8 = cmax <= 255;
    const long long p2max = (long long)std::floor(c.p2_frac * (double)cmax + 0.5);
    if (!c.boundless && (long long)c.paths * (cmax + std::max(p2max, 1LL)) >= 65536) {
        g_create_err = "coarse path sums would overflow 16 bits (too many arm views x census bits)";
        return LFSGM_ERR_UNSUPPORTED;
    }
    return LFSGM_OK;
}
}  // namespace

extern "C" {

lfsgm_status lfsgm_create(const lfsgm_config *cfg, void *stream, lfsgm_handle *out) {
    if (!cfg || !out) return LFSGM_ERR_INVALID_ARG;
    *out = nullptr;
    lfsgm_ctx *h = new lfsgm_ctx();
    {
        const lfsgm_status st = plan_handle(*cfg, h);
        if (st != LFSGM_OK) {
            delete h;
            return st;
        }
    }
    const lfsgm_config &c = h->cfg;
    h->stream = (cudaStream_t)stream;
    // shift tables in double precision
    std::vector<FineTap> fine((size_t)h->nviews * c.fine_labels);
    std::vector<short2> coarse((size_t)h->nviews * c.coarse_labels);
    for (int v = 0; v < c.V; v++)
        for (int u = 0; u < c.U; u++) {
            const int view = v * c.U + u;
            for (int g = 0; g < c.fine_labels; g++) {
                const double d = grid_disp(c.dmin, c.dmax, c.fine_labels, g);
                int ox, oy, nx, ny;
                double fx, fy;
                shift_split(u - c.uc, d, ox, fx, nx);
                shift_split(v - c.vc, d, oy, fy, ny);
                FineTap t;
                t.ox = (int16_t)ox; t.oy = (int16_t)oy; t.nx = (int16_t)nx; t.ny = (int16_t)ny;
                t.fx = (float)fx; t.fy = (float)fy;
                fine[(size_t)view * c.fine_labels + g] = t;
            }
            for (int k = 0; k < c.coarse_labels; k++) {
                const double d = grid_disp(c.dmin, c.dmax, c.coarse_labels, k);
                int ox, oy, nx, ny;
                double fx, fy;
                shift_split(u - c.uc, d, ox, fx, nx);
                shift_split(v - c.vc, d, oy, fy, ny);
                coarse[(size_t)view * c.coarse_labels + k] = make_short2((short)nx, (short)ny);
            }
        }
    std::vector<int> armviews(4 * kMaxArmViews, 0), sel_cross, sel_all;
    sel_cross.push_back(h->ref);
    for (int a = 0; a < h->arms.n_arms; a++)
        for (int i = 0; i < h->arms.nv[a]; i++) {
            armviews[a * kMaxArmViews + i] = h->arms.views[a][i];
            sel_cross.push_back(h->arms.views[a][i]);
        }
    for (int i = 0; i < h->nviews; i++) sel_all.push_back(i);
    // the complement of the initial pass's planes (reference and arm views; with the paper's four
    // extreme views the inner cross views are not among them)
    std::vector<char> in_cross(h->nviews, 0);
    in_cross[h->ref] = 1;
    for (int a = 0; a < h->arms.n_arms; a++)
        for (int i = 0; i < h->arms.nv[a]; i++) in_cross[h->arms.views[a][i]] = 1;
    std::vector<int> sel_rest;
    for (int i = 0; i < h->nviews; i++)
        if (!in_cross[i]) sel_rest.push_back(i);
    h->n_sel_rest = (int)sel_rest.size();
    if (sel_rest.empty()) sel_rest.push_back(0);          // (never launched: n_sel_rest = 0)
    // per arm: [nv][Lcd] linear offsets ny * Wp + nx of the nearest coarse shifts (0 = padding)
    std::vector<int> otab;
    h->ca.n_arms = h->arms.n_arms;
    for (int a = 0; a < h->arms.n_arms; a++) {
        h->ca.nv[a] = h->arms.nv[a];
        h->ca.tab_off[a] = (int)otab.size();
        for (int i = 0; i < h->arms.nv[a]; i++) {
            const int view = h->arms.views[a][i];
            for (int k = 0; k < h->Lcd; k++) {
                const short2 n = k < c.coarse_labels ? coarse[(size_t)view * c.coarse_labels + k] : make_short2(0, 0);
                otab.push_back((int)n.y * h->rows.Wp + (int)n.x);
            }
        }
    }
    if (otab.empty()) otab.push_back(0);
    h->n_sel_cross = (int)sel_cross.size();
    cudaError_t e;
#define ALLOC_COPY(dst, vec)                                                                  \
    e = cudaMalloc((void **)&dst, vec.size() * sizeof(vec[0]));                              \
    if (e == cudaSuccess) e = cudaMemcpy(dst, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice); \
    if (e != cudaSuccess) { g_create_err = cudaGetErrorString(e); lfsgm_destroy(h); return LFSGM_ERR_CUDA; }
    ALLOC_COPY(h->d_fine, fine);
    {
        std::vector<int> order;
        build_scan_order(c.H, c.W, c.paths, order);
        ALLOC_COPY(h->d_order, order);
    }
    {
        // (oy Wp + ox, ny Wp + nx, fx, fy) per (view, fine label), for the padded row stride Wp
        std::vector<int4> ltab(fine.size());
        for (size_t i = 0; i < fine.size(); i++) {
            const FineTap &t = fine[i];
            int4 e;
            e.x = (int)t.oy * h->rows.Wp + (int)t.ox;
            e.y = (int)t.ny * h->rows.Wp + (int)t.nx;
            memcpy(&e.z, &t.fx, 4);
            memcpy(&e.w, &t.fy, 4);
            ltab[i] = e;
        }
        ALLOC_COPY(h->d_ltab, ltab);
    }
    if (h->rows.ok) {
        std::vector<unsigned char> desc;
        const float fstep = (float)((c.dmax - c.dmin) / (double)(c.fine_labels - 1));
        if (build_fine_rows_desc(&h->rows, fine.data(), c.U, c.V, c.uc, c.vc, c.fine_labels, (float)c.dmin, fstep,
                                 desc)) {
            ALLOC_COPY(h->d_rowdesc, desc);
        } else {
            h->rows.ok = false;      // every window then goes through the list kernel
        }
    }
    h->h_fine = std::move(fine);
    ALLOC_COPY(h->d_otab, otab);
    ALLOC_COPY(h->d_armviews, armviews);
    ALLOC_COPY(h->d_sel_cross, sel_cross);
    ALLOC_COPY(h->d_sel_all, sel_all);
    ALLOC_COPY(h->d_sel_rest, sel_rest);
#undef ALLOC_COPY
    *out = h;
    return LFSGM_OK;
}

lfsgm_status lfsgm_destroy(lfsgm_handle h) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    cudaFree(h->d_fine);
    cudaFree(h->d_rowdesc);
    cudaFree(h->d_order);
    cudaFree(h->d_ltab);
    cudaFree(h->d_otab);
    cudaFree(h->d_armviews);
    cudaFree(h->d_sel_cross);
    cudaFree(h->d_sel_all);
    cudaFree(h->d_sel_rest);
    if (h->ws_owned) cudaFree(h->ws);
    cudaFree(h->o_lo); cudaFree(h->o_cnt); cudaFree(h->o_label); cudaFree(h->o_off);
    cudaFree(h->o_cost); cudaFree(h->o_agg); cudaFree(h->o_disp); cudaFree(h->o_views);
    if (h->up_done) cudaEventDestroy(h->up_done);
    if (h->up) cudaStreamDestroy(h->up);
    cudaFree(h->b_agg); cudaFree(h->b_gcs); cudaFree(h->b_gp); cudaFree(h->b_codes); cudaFree(h->b_amin);
    for (auto &r : h->prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h->pool) cudaEventDestroy(e);
    delete h;
    return LFSGM_OK;
}

lfsgm_status lfsgm_workspace_size(lfsgm_handle h, size_t *bytes) {
    if (!h || !bytes) return LFSGM_ERR_INVALID_ARG;
    const size_t N = (size_t)h->N, A = (size_t)std::max(h->arms.n_arms, 1);
    size_t b = 0;
    const size_t HWp = (size_t)h->rows.Hp * h->rows.Wp;
    b += align256((size_t)h->nviews * h->C * HWp * 8);   // census words per plane, edge-replicated padding
    b += align256((size_t)h->nviews * HWp * (h->C > 1 ? 16 : 4));   // views, edge-replicated padding
    b += align256(A * N * h->Lcd * (h->cost8 ? 1 : 2));   // coarse cost (bytes when they fit)
    b += align256(A * N * h->Lcd * 2);              // coarse path sums
    b += align256(4 * N * 4);                       // maps
    b += 3 * align256(N * 4);                       // F0, F1, padded counts
    b += align256(N * (size_t)((h->cfg.fine_labels + 31) / 32) * 8);   // (pixel, chunk) list
    b += align256(4);                               // wide-pixel count
    b += align256(4 * 8) + align256(8 * 4) + align256(2 * 4);
    b += align256(2 * kPartialBlocks * 8) + 2 * align256(4);   // partials; status word and ticket
    b += align256((size_t)scan_tiles(h->N) * 8);    // offset-scan tile sums
    b += align256((size_t)sgm_split_ints(h->cfg.H, h->cfg.W, h->cfg.paths) * 4);   // SGM scanlines to split
    *bytes = b;
    return LFSGM_OK;
}

lfsgm_status lfsgm_set_workspace(lfsgm_handle h, void *dptr, size_t bytes) {
    if (!h || !dptr) return LFSGM_ERR_INVALID_ARG;
    return bind_workspace(h, dptr, bytes, false);
}

lfsgm_status lfsgm_set_tuning(lfsgm_handle h, int32_t row_kw, int32_t list_ctas_per_sm) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if ((row_kw != 0 && row_kw != 36 && row_kw != 44) || list_ctas_per_sm < 0 || list_ctas_per_sm > 64)
        return fail(h, LFSGM_ERR_INVALID_ARG, "tuning: row_kw must be 0, 36 or 44, list_ctas_per_sm in [0, 64]");
    h->list_ctas = list_ctas_per_sm;
    const int kw = row_kw == 0 ? 36 : row_kw;
    if (kw == h->row_kw) return LFSGM_OK;
    const lfsgm_config &c = h->cfg;
    // new plan and descriptors for the new label span; the padding and the workspace layout do not
    // depend on it, so a bound workspace keeps its buffers and only the tensor maps are re-encoded
    RowPlanHost rows{};
    plan_fine_rows(c.U, c.V, c.uc, c.vc, c.H, c.W, c.fine_labels, c.dmin, c.dmax, kw, h->C, &rows);
    std::vector<unsigned char> desc;
    const float fstep = (float)((c.dmax - c.dmin) / (double)(c.fine_labels - 1));
    bool ok = rows.ok &&
              build_fine_rows_desc(&rows, h->h_fine.data(), c.U, c.V, c.uc, c.vc, c.fine_labels, (float)c.dmin, fstep,
                                   desc);
    unsigned char *d = nullptr;
    if (ok) {
        cudaError_t e = cudaMalloc(&d, desc.size());
        if (e == cudaSuccess) e = cudaMemcpy(d, desc.data(), desc.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(h, e, "row descriptors");
        }
    }
    if (h->stream) cudaStreamSynchronize(h->stream);     // no launch of the old plan is in flight
    cudaFree(h->d_rowdesc);
    h->d_rowdesc = d;
    rows.ok = ok;
    h->rows = rows;
    h->row_kw = kw;
    h->rows_maps = h->ws && h->rows.ok && encode_fine_rows_maps(&h->rows, h->views_pad, h->cen_pad, h->nviews);
    return LFSGM_OK;
}

lfsgm_status lfsgm_set_sgm_warps(lfsgm_handle h, int32_t warps_per_cta) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (warps_per_cta != 0 && warps_per_cta != 2 && warps_per_cta != 4 && warps_per_cta != 8)
        return fail(h, LFSGM_ERR_INVALID_ARG, "tuning: warps_per_cta must be 0, 2, 4 or 8");
    h->sgm_warps = warps_per_cta == 0 ? 4 : warps_per_cta;
    return LFSGM_OK;
}

lfsgm_status lfsgm_set_sgm_split(lfsgm_handle h, int32_t min_wide) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (min_wide < 0) return fail(h, LFSGM_ERR_INVALID_ARG, "tuning: min_wide must be >= 0");
    h->sgm_split = min_wide;
    return LFSGM_OK;
}

lfsgm_status lfsgm_get_sgm_split(lfsgm_handle h, int32_t *min_wide) {
    if (!h || !min_wide) return LFSGM_ERR_INVALID_ARG;
    *min_wide = h->sgm_split;
    return LFSGM_OK;
}

lfsgm_status lfsgm_get_tuning(lfsgm_handle h, int32_t *row_kw, int32_t *list_ctas_per_sm, int32_t *sgm_warps) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (row_kw) *row_kw = h->row_kw;
    if (list_ctas_per_sm) *list_ctas_per_sm = h->list_ctas;
    if (sgm_warps) *sgm_warps = h->sgm_warps;
    return LFSGM_OK;
}

lfsgm_status lfsgm_max_nnz(lfsgm_handle h, int64_t *nnz) {
    if (!h || !nnz) return LFSGM_ERR_INVALID_ARG;
    *nnz = (int64_t)h->N * ((h->cfg.fine_labels + 3) & ~3);
    return LFSGM_OK;
}

lfsgm_status lfsgm_initial_disparity(lfsgm_handle h, const float *views, int32_t Pc1, int32_t Pc2, int32_t *lo,
                                     int32_t *cnt, int64_t *off, float *dinit, int32_t *maps,
                                     int64_t *nnz_host) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!views || !lo || !cnt || !off) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (Pc1 > 0 && Pc2 < Pc1) return fail(h, LFSGM_ERR_INVALID_ARG, "need P2 >= P1 (Eq. 8)");
    if (Pc1 > 0 && (long long)h->cfg.paths * ((long long)max_arm_views(h) * h->nbits * h->C + Pc2) >= 65536)
        return fail(h, LFSGM_ERR_UNSUPPORTED, "coarse P2 too large for 16-bit path sums");
    LFSGM_TRY(ensure_workspace(h));
    const lfsgm_config &c = h->cfg;
    cudaStream_t s = h->stream;
    const int N = h->N, A = h->arms.n_arms;
    int *fin = h->F0, *fout = h->F1;
    cudaError_t e = cudaSuccess;
    if (!c.boundless) {   // boundary-less: no initial map, the windows kernel writes whole-range windows
        LFSGM_TRY(run(h, "census_cross", [&] {
            return launch_census_pad(s, views, c.H, c.W, c.census_w, h->rows.P, h->rows.Wp, h->rows.Hp, h->C,
                                     h->d_sel_cross, h->n_sel_cross, h->cen_pad, h->views_pad);
        }));
        e = cudaMemsetAsync(h->armsum, 0, 4 * 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->csum, 0, (size_t)A * N * h->Lcd * 2, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        LFSGM_TRY(run(h, "coarse_cost", [&] {
            return launch_coarse_cost(s, h->cen_pad, h->rows.P, h->rows.Wp, h->rows.Hp, c.H, c.W, h->ref, h->C,
                                      h->d_armviews, h->d_otab, h->ca, c.coarse_labels, h->ccost, h->cost8,
                                      h->armsum);
        }));
        LFSGM_TRY(run(h, "coarse_penalties", [&] {
            return launch_coarse_penalties(s, h->armsum, A, (long long)N * c.coarse_labels, c.p1_frac, c.p2_frac,
                                           Pc1, Pc2, h->cpen);
        }));
        LFSGM_TRY(run(h, "coarse_sgm", [&] {
            return launch_coarse_sgm(s, h->ccost, h->cost8, A, c.H, c.W, c.coarse_labels, h->cpen, h->csum, h->d_order,
                                     c.paths);
        }));
        LFSGM_TRY(run(h, "coarse_wta", [&] {
            return launch_coarse_wta(s, h->csum, A, N, c.coarse_labels, h->maps, maps);
        }));
        LFSGM_TRY(run(h, "fuse", [&] { return launch_fuse(s, h->maps, A, N, c.phi, h->F0); }));
        for (int it = 0; it < c.fill_passes; it++) {
            LFSGM_TRY(run(h, "hole_fill", [&] { return launch_fill(s, fin, fout, c.H, c.W); }));
            std::swap(fin, fout);
        }
    }
    LFSGM_TRY(run(h, "windows", [&] {
        return launch_windows(s, fin, N, c.fine_labels, c.coarse_labels, c.fine_radius, lo, cnt, dinit, h->cntpad,
                              h->views_pad + (size_t)h->ref * h->rows.Hp * h->rows.Wp * (h->C > 1 ? 4 : 1), h->C,
                              h->rows.P, h->rows.Wp, c.W, c.edge_threshold, c.fine_radius_far, c.boundless);
    }));
    LFSGM_TRY(run(h, "scan_sums", [&] { return launch_scan_sums(s, h->cntpad, N, h->tsum); }));
    LFSGM_TRY(run(h, "scan_top", [&] { return launch_scan_top(s, h->tsum, N); }));
    LFSGM_TRY(run(h, "scan_apply", [&] { return launch_scan_apply(s, h->cntpad, N, h->tsum, (long long *)off); }));
    if (nnz_host) {
        e = cudaMemcpyAsync(nnz_host, off + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "nnz readback");
    }
    return LFSGM_OK;
}

}  // extern "C"

namespace {
// The cost stage; `cross_done`: the padded census and views of the cross views already hold these
// views (the whole-method chain, right after its initial pass), so only the others are transformed.
lfsgm_status cost_volume_impl(lfsgm_handle h, const float *views, const int32_t *lo, const int32_t *cnt,
                              const int64_t *off, float *cost, bool cross_done) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!views || !lo || !cnt || !off || !cost) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(cost)) return fail(h, LFSGM_ERR_INVALID_ARG, "cost must be 16-byte aligned");
    LFSGM_TRY(ensure_workspace(h));
    const lfsgm_config &c = h->cfg;
    cudaStream_t s = h->stream;
    if (!cross_done) {
        LFSGM_TRY(run(h, "census_all", [&] {
            return launch_census_pad(s, views, c.H, c.W, c.census_w, h->rows.P, h->rows.Wp, h->rows.Hp, h->C,
                                     h->d_sel_all, h->nviews, h->cen_pad, h->views_pad);
        }));
    } else if (h->n_sel_rest > 0) {
        LFSGM_TRY(run(h, "census_rest", [&] {
            return launch_census_pad(s, views, c.H, c.W, c.census_w, h->rows.P, h->rows.Wp, h->rows.Hp, h->C,
                                     h->d_sel_rest, h->n_sel_rest, h->cen_pad, h->views_pad);
        }));
    }
    const cudaError_t e = cudaMemsetAsync(h->wide_count, 0, 4, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    const float fstep = (float)((c.dmax - c.dmin) / (double)(c.fine_labels - 1));
    if (h->rows_maps) {
        LFSGM_TRY(run(h, "fine_cost", [&] {
            return launch_fine_cost_rows(s, &h->rows, h->views_pad, h->cen_pad, h->d_rowdesc, c.fine_labels, c.U,
                                         c.V, c.H, c.W, h->ref, lo, cnt, (const long long *)off, c.w_l2, c.w_census,
                                         fstep, cost, h->status, h->wide_list, h->wide_count);
        }));
    } else {
        // shapes whose row tiles do not fit the TMA boxes: every pixel through the list kernel
        LFSGM_TRY(run(h, "fine_cost_all_list", [&] {
            return launch_list_all(s, lo, cnt, (const long long *)off, c.fine_labels, h->wide_list, h->wide_count,
                                   h->N, h->status);
        }));
    }
    LFSGM_TRY(run(h, "fine_cost_wide", [&] {
        return launch_fine_cost_list(s, h->views_pad, h->cen_pad, h->rows.P, h->rows.Wp, h->rows.Hp, h->d_ltab,
                                     c.fine_labels, h->nviews, h->C, c.W, h->ref, lo, cnt, (const long long *)off,
                                     c.w_l2, c.w_census, cost, h->wide_list, h->wide_count, h->list_ctas);
    }));
    return LFSGM_OK;
}
}  // namespace

extern "C" {

lfsgm_status lfsgm_cost_volume(lfsgm_handle h, const float *views, const int32_t *lo, const int32_t *cnt,
                               const int64_t *off, float *cost) {
    return cost_volume_impl(h, views, lo, cnt, off, cost, false);
}

}  // extern "C"

namespace {
// The aggregate's rows (and the first nz ints of the SGM's split table) to zero.
__global__ void zero_csr_kernel(float *a, const long long *off, int N, int *z, int nz) {
    const long long n = off[N];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nz; i += gridDim.x * blockDim.x) z[i] = 0;
}

// Zero the aggregate, then (with the split knob on, and `list`) list the SGM scanlines to split.
lfsgm_status sgm_prologue(lfsgm_ctx *h, float *agg, const int32_t *cnt, const long long *o, bool list) {
    cudaStream_t s = h->stream;
    const lfsgm_config &c = h->cfg;
    const int nz = h->sgm_split > 0 ? 1 : 0;      // the split table's list count
    LFSGM_TRY(run(h, "zero_agg", [&] {
        zero_csr_kernel<<<1216, 256, 0, s>>>(agg, o, h->N, h->split, nz);
        return cudaGetLastError();
    }));
    if (nz == 0 || !list) return LFSGM_OK;
    return run(h, "sgm_split", [&] { return launch_sgm_split(s, cnt, c.H, c.W, c.paths, h->sgm_split, h->split); });
}
__global__ void set_pen_kernel(float *pen, float P1, float P2) {
    pen[0] = P1;
    pen[1] = P2;
}
}  // namespace

extern "C" {

lfsgm_status lfsgm_sgm_aggregate(lfsgm_handle h, const float *cost, const int32_t *lo, const int32_t *cnt,
                                 const int64_t *off, float P1, float P2, float *agg) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!cost || !lo || !cnt || !off || !agg) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(cost) || !aligned16(agg)) return fail(h, LFSGM_ERR_INVALID_ARG, "cost and agg must be 16-byte aligned");
    const bool derived = P1 < 0.f;
    if (!derived && !(P1 >= 0.f && P2 >= P1 && std::isfinite(P2)))
        return fail(h, LFSGM_ERR_INVALID_ARG, "need 0 <= P1 <= P2 (Eq. 8), got %g %g", P1, P2);
    LFSGM_TRY(ensure_workspace(h));
    const lfsgm_config &c = h->cfg;
    cudaStream_t s = h->stream;
    const long long *o = (const long long *)off;
    if (derived) {
        // zero agg (and the split list's count), then the penalty mean, whose launch also lists the
        // scanlines to split
        LFSGM_TRY(sgm_prologue(h, agg, cnt, o, false));
        LFSGM_TRY(run(h, "cost_partial_sums", [&] {
            return launch_cost_partial_sums(s, cost, cnt, o, h->N, c.fine_labels, h->partial, kPartialBlocks,
                                            c.p1_frac, c.p2_frac, h->fpen, h->ticket, h->status, c.H, c.W,
                                            c.paths, h->sgm_split, h->sgm_split > 0 ? h->split : nullptr);
        }));
    } else {
        LFSGM_TRY(run(h, "set_penalties", [&] {
            set_pen_kernel<<<1, 1, 0, s>>>(h->fpen, P1, P2);
            return cudaGetLastError();
        }));
        LFSGM_TRY(sgm_prologue(h, agg, cnt, o, true));
    }
    LFSGM_TRY(run(h, "fine_sgm", [&] {
        return launch_fine_sgm(s, cost, lo, cnt, o, c.H, c.W, c.fine_labels, h->fpen, agg, h->status, h->d_order,
                               c.paths, nullptr, nullptr, 0, h->sgm_warps, h->sgm_split > 0 ? h->split : nullptr);
    }));
    return LFSGM_OK;
}

lfsgm_status lfsgm_wta_subpixel(lfsgm_handle h, const float *agg, const int32_t *lo, const int32_t *cnt,
                                const int64_t *off, int32_t *label, float *disp) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!agg || !lo || !cnt || !off || (!label && !disp)) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(agg)) return fail(h, LFSGM_ERR_INVALID_ARG, "agg must be 16-byte aligned");
    LFSGM_TRY(ensure_workspace(h));
    const lfsgm_config &c = h->cfg;
    const double step = (c.dmax - c.dmin) / (double)(c.fine_labels - 1);
    return run(h, "wta_subpixel", [&] {
        return launch_wta(h->stream, agg, lo, cnt, (const long long *)off, h->N, c.fine_labels, c.dmin, step,
                          c.subpixel, c.softmin_tau, label, disp, h->status);
    });
}

lfsgm_status lfsgm_median_filter(lfsgm_handle h, const float *disp, float *out) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!disp || !out) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (disp == out) return fail(h, LFSGM_ERR_INVALID_ARG, "the median filter needs distinct input and output");
    return run(h, "median_filter", [&] { return launch_median3(h->stream, disp, out, h->cfg.H, h->cfg.W); });
}

static lfsgm_status backward_scratch(lfsgm_handle h) {
    if (h->b_agg) return LFSGM_OK;
    int64_t cap = 0;
    lfsgm_max_nnz(h, &cap);
    cudaError_t e = cudaMalloc((void **)&h->b_agg, (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->b_gcs, (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->b_codes, (size_t)cap * h->cfg.paths);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->b_amin, (size_t)h->N * h->cfg.paths * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&h->b_gp, 2 * 4);
    if (e != cudaSuccess) return fail(h, LFSGM_ERR_NO_MEMORY, "backward scratch: %s", cudaGetErrorString(e));
    return LFSGM_OK;
}

// The SGM of Eq. 8-9 on explicit penalties into agg, recording each cell's winning branch and each
// pixel's argmin slot per direction into the handle's backward scratch.
static lfsgm_status aggregate_recording(lfsgm_handle h, const float *cost, const int32_t *lo, const int32_t *cnt,
                                        const int64_t *off, float P1, float P2, float *agg) {
    const lfsgm_config &c = h->cfg;
    cudaStream_t s = h->stream;
    const long long *o = (const long long *)off;
    int64_t cap = 0;
    lfsgm_max_nnz(h, &cap);
    h->rec.valid = false;
    LFSGM_TRY(run(h, "set_penalties", [&] {
        set_pen_kernel<<<1, 1, 0, s>>>(h->fpen, P1, P2);
        return cudaGetLastError();
    }));
    LFSGM_TRY(sgm_prologue(h, agg, cnt, o, true));
    return run(h, "fine_sgm_record", [&] {
        return launch_fine_sgm(s, cost, lo, cnt, o, c.H, c.W, c.fine_labels, h->fpen, agg, h->status, h->d_order,
                               c.paths, h->b_codes, h->b_amin, (size_t)cap, h->sgm_warps,
                               h->sgm_split > 0 ? h->split : nullptr);
    });
}

// soft-argmin adjoint, SGM adjoint on the recorded branches, l2 term -> views
static lfsgm_status backward_from_record(lfsgm_handle h, const float *views, const float *cost, const float *agg,
                                         const int32_t *lo, const int32_t *cnt, const int64_t *off, float P1,
                                         float P2, const float *grad_disp, float *grad_cost, float *grad_P1,
                                         float *grad_P2, float *grad_views) {
    const lfsgm_config &c = h->cfg;
    cudaStream_t s = h->stream;
    const size_t N = (size_t)h->N;
    int64_t cap = 0;
    lfsgm_max_nnz(h, &cap);
    const long long *o = (const long long *)off;
    const double step = (c.dmax - c.dmin) / (double)(c.fine_labels - 1);
    LFSGM_TRY(run(h, "softargmin_backward", [&] {
        return launch_softargmin_backward(s, agg, lo, cnt, o, h->N, c.fine_labels, c.dmin, step, c.softmin_tau,
                                          grad_disp, h->b_gcs, grad_cost, h->status);
    }));
    cudaError_t e = cudaMemsetAsync(h->b_gp, 0, 8, s);
    if (e == cudaSuccess && grad_views) e = cudaMemsetAsync(grad_views, 0, (size_t)h->nviews * h->C * N * 4, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    LFSGM_TRY(run(h, "sgm_backward", [&] {
        return launch_sgm_backward(s, cost, lo, cnt, o, c.H, c.W, c.fine_labels, P1, P2, h->b_gcs, h->b_codes,
                                   h->b_amin, (size_t)cap, grad_cost, h->b_gp, h->status, h->d_order, c.paths,
                                   false);
    }));
    if (grad_views) {
        // the (pixel, 32-label chunk) items of windows wider than 32 labels; narrower ones by rows,
        // which add the windows outside their row's label range to the items
        e = cudaMemsetAsync(h->wide_count, 0, 4, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "memset");
        LFSGM_TRY(run(h, "list_all", [&] {
            return launch_list_all(s, lo, cnt, o, c.fine_labels, h->wide_list, h->wide_count, h->N, h->status, 32);
        }));
        LFSGM_TRY(run(h, "views_backward", [&] {
            return launch_views_backward(s, views, h->d_fine, c.fine_labels, c.U, c.V, h->C, c.H, c.W, h->ref, lo,
                                         cnt, o, c.w_l2, (float)step, grad_cost, grad_views, h->wide_list,
                                         h->wide_count);
        }));
        LFSGM_TRY(run(h, "views_backward_list", [&] {
            return launch_views_backward_list(s, views, h->d_fine, c.fine_labels, h->nviews, h->C, c.H, c.W, h->ref,
                                              lo, cnt, o, c.w_l2, grad_cost, grad_views, h->wide_list, h->wide_count);
        }));
    }
    e = cudaMemcpyAsync(grad_P1, h->b_gp, 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(grad_P2, h->b_gp + 1, 4, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "penalty gradients");
    return LFSGM_OK;
}

static bool penalties_ok(float P1, float P2) { return P1 >= 0.f && P2 >= P1 && std::isfinite(P2); }

lfsgm_status lfsgm_sgm_aggregate_record(lfsgm_handle h, const float *cost, const int32_t *lo, const int32_t *cnt,
                                        const int64_t *off, float P1, float P2, float *agg) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!cost || !lo || !cnt || !off || !agg) return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(cost) || !aligned16(agg)) return fail(h, LFSGM_ERR_INVALID_ARG, "cost and agg must be 16-byte aligned");
    if (!penalties_ok(P1, P2))
        return fail(h, LFSGM_ERR_INVALID_ARG, "recording needs explicit penalties 0 <= P1 <= P2, got %g %g", P1, P2);
    LFSGM_TRY(ensure_workspace(h));
    LFSGM_TRY(backward_scratch(h));
    LFSGM_TRY(aggregate_recording(h, cost, lo, cnt, off, P1, P2, agg));
    h->rec.valid = true;
    h->rec.cost = cost;
    h->rec.agg = agg;
    h->rec.lo = lo;
    h->rec.cnt = cnt;
    h->rec.off = off;
    h->rec.P1 = P1;
    h->rec.P2 = P2;
    return LFSGM_OK;
}

lfsgm_status lfsgm_backward(lfsgm_handle h, const float *views, const float *cost, const int32_t *lo,
                            const int32_t *cnt, const int64_t *off, float P1, float P2, const float *grad_disp,
                            float *grad_cost, float *grad_P1, float *grad_P2, float *grad_views) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!cost || !lo || !cnt || !off || !grad_disp || !grad_cost || !grad_P1 || !grad_P2 || (grad_views && !views))
        return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(cost) || !aligned16(grad_cost))
        return fail(h, LFSGM_ERR_INVALID_ARG, "cost and grad_cost must be 16-byte aligned");
    if (!penalties_ok(P1, P2))
        return fail(h, LFSGM_ERR_INVALID_ARG, "backward needs explicit penalties 0 <= P1 <= P2, got %g %g", P1, P2);
    LFSGM_TRY(ensure_workspace(h));
    LFSGM_TRY(backward_scratch(h));
    // the forward of the SGM recomputed into the handle's own aggregate, with its record
    LFSGM_TRY(aggregate_recording(h, cost, lo, cnt, off, P1, P2, h->b_agg));
    return backward_from_record(h, views, cost, h->b_agg, lo, cnt, off, P1, P2, grad_disp, grad_cost, grad_P1,
                                grad_P2, grad_views);
}

lfsgm_status lfsgm_backward_recorded(lfsgm_handle h, const float *views, const float *cost, const float *agg,
                                     const int32_t *lo, const int32_t *cnt, const int64_t *off, float P1, float P2,
                                     const float *grad_disp, float *grad_cost, float *grad_P1, float *grad_P2,
                                     float *grad_views) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!cost || !agg || !lo || !cnt || !off || !grad_disp || !grad_cost || !grad_P1 || !grad_P2 ||
        (grad_views && !views))
        return fail(h, LFSGM_ERR_INVALID_ARG, "null buffer");
    if (!aligned16(cost) || !aligned16(grad_cost))
        return fail(h, LFSGM_ERR_INVALID_ARG, "cost and grad_cost must be 16-byte aligned");
    const auto &r = h->rec;
    if (!r.valid || r.cost != cost || r.agg != agg || r.lo != lo || r.cnt != cnt || r.off != off || r.P1 != P1 ||
        r.P2 != P2)
        return fail(h, LFSGM_ERR_INVALID_ARG,
                    "no record of lfsgm_sgm_aggregate_record on these cost, agg, window buffers and penalties");
    LFSGM_TRY(ensure_workspace(h));
    return backward_from_record(h, views, cost, agg, lo, cnt, off, P1, P2, grad_disp, grad_cost, grad_P1, grad_P2,
                                grad_views);
}

lfsgm_status lfsgm_sync(lfsgm_handle h) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    cudaError_t e = h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    if (!h->status) return LFSGM_OK;
    int st = 0;
    e = cudaMemcpy(&st, h->status, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "status readback");
    if (st != 0) {
        cudaMemset(h->status, 0, 4);
        return fail(h, (lfsgm_status)st, "device-side status %d", st);
    }
    return LFSGM_OK;
}

const char *lfsgm_last_error(lfsgm_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

int64_t lfsgm_launch_count(lfsgm_handle h) { return h ? h->launches : -1; }

lfsgm_status lfsgm_set_profiling(lfsgm_handle h, int32_t enable) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    h->profiling = enable != 0;
    return LFSGM_OK;
}

lfsgm_status lfsgm_kernel_times(lfsgm_handle h, const char **names, float *ms, int32_t cap, int32_t *n_out) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    cudaError_t e = h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "sync");
    int n = 0;
    for (auto &r : h->prof) {
        if (n < cap) {
            float t = 0.f;
            cudaEventElapsedTime(&t, r.a, r.b);
            if (names) names[n] = r.name;
            if (ms) ms[n] = t;
            n++;
        }
        h->pool.push_back(r.a);
        h->pool.push_back(r.b);
    }
    h->prof.clear();
    if (n_out) *n_out = n;
    return LFSGM_OK;
}

}  // extern "C"

namespace {
// The whole method on device views; `wait` (nullable) is an event the cost stage waits for (views
// that only the cost stage reads may still be arriving while the initial pass runs).
lfsgm_status depth_buffers(lfsgm_handle h) {
    const size_t N = (size_t)h->N;
    int64_t maxnnz = 0;
    lfsgm_max_nnz(h, &maxnnz);
    if (!h->o_lo) {
        cudaError_t e = cudaMalloc((void **)&h->o_lo, N * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_cnt, N * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_label, N * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_disp, N * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_off, (N + 1) * 8);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_cost, (size_t)maxnnz * 4);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->o_agg, (size_t)maxnnz * 4);
        if (e != cudaSuccess) return fail(h, LFSGM_ERR_NO_MEMORY, "depth buffers: %s", cudaGetErrorString(e));
    }
    return LFSGM_OK;
}

// The speed knobs of one handle: with the windows of one initial pass of `views` in (lo, cnt, off),
// time the cost stage (best of two after a warm-up) for the row kernel's label span 36 and 44 and
// then, with the better span, for the list kernel's CTAs per SM 8, 12, 24 against the default;
// keep the fastest; then the SGM's warps per CTA and split threshold the same way.  kw, lc: the
// cost knobs chosen.
lfsgm_status tune_handle(lfsgm_handle h, const float *views, int32_t *lo, int32_t *cnt, int64_t *off, float *cost,
                         float *agg, int &kw_out, int &lc_out) {
    LFSGM_TRY(lfsgm_initial_disparity(h, views, 0, 0, lo, cnt, off, nullptr, nullptr, nullptr));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(h, LFSGM_ERR_CUDA, "tuning events");
    }
    auto time_cost = [&](int kw, int lc, float &ms) -> lfsgm_status {
        lfsgm_status st = lfsgm_set_tuning(h, kw, lc);
        float best = 1e30f;
        for (int r = 0; r < 3 && st == LFSGM_OK; r++) {
            cudaEventRecord(e0, h->stream);
            st = cost_volume_impl(h, views, lo, cnt, off, cost, !h->cfg.boundless);
            cudaEventRecord(e1, h->stream);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (r > 0) best = std::min(best, t);
        }
        ms = best;
        return st;
    };
    int best_kw = 36, best_lc = 0;
    float best_ms = 1e30f;
    lfsgm_status st = LFSGM_OK;
    for (int kw : {36, 44}) {
        float ms = 0.f;
        st = time_cost(kw, 0, ms);
        if (st != LFSGM_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_kw = kw;
        }
    }
    for (int lc : {8, 12, 24}) {
        if (st != LFSGM_OK) break;
        float ms = 0.f;
        st = time_cost(best_kw, lc, ms);
        if (st == LFSGM_OK && ms < best_ms) {
            best_ms = ms;
            best_lc = lc;
        }
    }
    if (st == LFSGM_OK) st = lfsgm_set_tuning(h, best_kw, best_lc);
    // the SGM's warps (scanlines) per CTA, on the cost volume of the chosen knobs (derived penalties)
    if (st == LFSGM_OK) st = cost_volume_impl(h, views, lo, cnt, off, cost, !h->cfg.boundless);
    // and whether scanlines that cross many wide windows run split across a CTA (off or threshold 24)
    int best_w = 4, best_sp = 0;
    float best_sgm = 1e30f;
    for (int w : {4, 8, 2})
        for (int sp : {0, 24}) {
            if (st != LFSGM_OK) break;
            st = lfsgm_set_sgm_warps(h, w);
            if (st == LFSGM_OK) st = lfsgm_set_sgm_split(h, sp);
            float best = 1e30f;
            for (int r = 0; r < 3 && st == LFSGM_OK; r++) {
                cudaEventRecord(e0, h->stream);
                st = lfsgm_sgm_aggregate(h, cost, lo, cnt, off, -1.f, -1.f, agg);
                cudaEventRecord(e1, h->stream);
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (r > 0) best = std::min(best, t);
            }
            if (st == LFSGM_OK && best < best_sgm) {
                best_sgm = best;
                best_w = w;
                best_sp = sp;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == LFSGM_OK) st = lfsgm_set_sgm_warps(h, best_w);
    if (st == LFSGM_OK) st = lfsgm_set_sgm_split(h, best_sp);
    kw_out = best_kw;
    lc_out = best_lc;
    return st;
}

lfsgm_status depth_chain(lfsgm_handle h, const float *views, float *disp, int32_t *label, cudaEvent_t wait) {
    LFSGM_TRY(depth_buffers(h));
    int64_t *off = (int64_t *)h->o_off;
    LFSGM_TRY(lfsgm_initial_disparity(h, views, 0, 0, h->o_lo, h->o_cnt, off, nullptr, nullptr, nullptr));
    if (wait) {
        const cudaError_t e = cudaStreamWaitEvent(h->stream, wait, 0);
        if (e != cudaSuccess) return cuda_fail(h, e, "upload wait");
    }
    LFSGM_TRY(cost_volume_impl(h, views, h->o_lo, h->o_cnt, off, h->o_cost, !h->cfg.boundless));
    LFSGM_TRY(lfsgm_sgm_aggregate(h, h->o_cost, h->o_lo, h->o_cnt, off, -1.f, -1.f, h->o_agg));
    return lfsgm_wta_subpixel(h, h->o_agg, h->o_lo, h->o_cnt, off, label ? label : h->o_label,
                              disp ? disp : h->o_disp);
}
}  // namespace

extern "C" {

lfsgm_status lfsgm_depth(lfsgm_handle h, const float *views, float *disp, int32_t *label) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!views) return fail(h, LFSGM_ERR_INVALID_ARG, "null views");
    return depth_chain(h, views, disp, label, nullptr);
}

lfsgm_status lfsgm_autotune(lfsgm_handle h, const float *views, int32_t *row_kw, int32_t *list_ctas_per_sm) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!views) return fail(h, LFSGM_ERR_INVALID_ARG, "null views");
    LFSGM_TRY(depth_buffers(h));
    int kw = 36, lc = 0;
    LFSGM_TRY(tune_handle(h, views, h->o_lo, h->o_cnt, (int64_t *)h->o_off, h->o_cost, h->o_agg, kw, lc));
    if (row_kw) *row_kw = kw;
    if (list_ctas_per_sm) *list_ctas_per_sm = lc;
    return LFSGM_OK;
}

lfsgm_status lfsgm_depth_host(lfsgm_handle h, const float *views_host, float *disp_host, int32_t *label_host) {
    if (!h) return LFSGM_ERR_INVALID_ARG;
    if (!views_host || !disp_host) return fail(h, LFSGM_ERR_INVALID_ARG, "null host buffer");
    const lfsgm_config &c = h->cfg;
    const size_t N = (size_t)h->N, vv = (size_t)h->C * N * 4, vbytes = (size_t)h->nviews * vv;
    if (!h->o_views) {
        cudaError_t e = cudaMalloc((void **)&h->o_views, vbytes);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->up_done, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(h, LFSGM_ERR_NO_MEMORY, "views buffer: %s", cudaGetErrorString(e));
    }
    cudaStream_t s = h->stream;
    char *dv = (char *)h->o_views;
    const char *hv = (const char *)views_host;
    cudaError_t e = cudaSuccess;
    cudaEvent_t wait = nullptr;
    if (c.boundless) {
        e = cudaMemcpyAsync(dv, hv, vbytes, cudaMemcpyHostToDevice, s);
    } else {
        // The initial pass reads the cross views only (row vc and column uc): they go first on the
        // handle's stream; the other views go on the upload stream meanwhile, as four rectangles of
        // the [V][U] view grid, and the cost stage waits for them.
        const size_t pitch = (size_t)c.U * vv;
        e = cudaMemcpyAsync(dv + c.vc * pitch, hv + c.vc * pitch, pitch, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(dv + c.uc * vv, pitch, hv + c.uc * vv, pitch, vv, c.V, cudaMemcpyHostToDevice, s);
        // the upload stream starts after the work already queued on the handle's stream, so that a
        // previous light field's kernels are done with the buffer
        if (e == cudaSuccess) e = cudaEventRecord(h->up_done, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->up, h->up_done, 0);
        const int rows[2][2] = {{0, c.vc}, {c.vc + 1, c.V}};
        const int cols[2][2] = {{0, c.uc}, {c.uc + 1, c.U}};
        for (int r = 0; r < 2 && e == cudaSuccess; r++)
            for (int q = 0; q < 2 && e == cudaSuccess; q++) {
                const int v0 = rows[r][0], nvr = rows[r][1] - rows[r][0];
                const int u0 = cols[q][0], nuc = cols[q][1] - cols[q][0];
                if (nvr <= 0 || nuc <= 0) continue;
                const size_t o = (size_t)v0 * pitch + (size_t)u0 * vv;
                e = cudaMemcpy2DAsync(dv + o, pitch, hv + o, pitch, (size_t)nuc * vv, nvr, cudaMemcpyHostToDevice, h->up);
            }
        if (e == cudaSuccess) e = cudaEventRecord(h->up_done, h->up);
        wait = h->up_done;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "views upload");
    LFSGM_TRY(depth_chain(h, h->o_views, nullptr, nullptr, wait));
    e = cudaMemcpyAsync(disp_host, h->o_disp, N * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && label_host) e = cudaMemcpyAsync(label_host, h->o_label, N * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "result download");
    return LFSGM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Batches (not in the paper): many light fields of mixed shape in one CUDA-graph launch.
//
// One handle per light field (its own tables and configuration).  The light fields are split
// over K branches (streams forked from the caller's stream); within a branch they run one after
// another and share one set of scratch buffers sized for the branch's largest member.  The whole
// batch -- every stage of every light field plus a %globaltimer stamp before and after each light
// field -- is captured once into a CUDA graph, so a batch is one graph launch.  Branch count and
// assignment come from a small autotuner: longest-job-first assignment for each candidate K in
// {1, 2, 4, 8, 16} (each branch then runs its light fields shortest first), each timed on the
// device, the fastest kept (or K given by the caller).

namespace {

__global__ void stamp_kernel(unsigned long long *t) {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

struct BranchBufs {
    void *ws = nullptr;
    size_t ws_bytes = 0;
    int *lo = nullptr, *cnt = nullptr, *label = nullptr;
    long long *off = nullptr;
    float *cost = nullptr, *agg = nullptr;
};

// Longest-job-first assignment of work items to K branches (each to the least-loaded branch), then
// each branch's items shortest first: the branch's total time is the same, and more light fields
// complete early (lower median completion time).
std::vector<std::vector<int>> batch_assign(const std::vector<double> &work, int K) {
    const int n = (int)work.size();
    std::vector<std::vector<int>> plan(K);
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return work[a] > work[c]; });
    std::vector<double> load(K, 0.0);
    for (int i : idx) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        plan[k].push_back(i);
        load[k] += work[i];
    }
    for (auto &pl : plan) std::stable_sort(pl.begin(), pl.end(), [&](int a, int c) { return work[a] < work[c]; });
    return plan;
}

// Sizes that the scratch of a batch branch depends on, per light field.
struct LfSizes {
    size_t ws = 0, N = 0;
    int64_t nnz = 0;
    double work = 0.0;
};

LfSizes lf_sizes(lfsgm_ctx *h) {
    LfSizes z;
    lfsgm_workspace_size(h, &z.ws);
    lfsgm_max_nnz(h, &z.nnz);
    z.N = (size_t)h->N;
    const lfsgm_config &c = h->cfg;
    z.work = (double)h->N * ((double)h->nviews * h->C * (2 * c.fine_radius + 1) + 4.0 * c.coarse_labels);
    return z;
}

// Bytes of one branch's scratch (workspace, window map, labels, cost and aggregate), and of the
// %globaltimer stamps of n light fields; every piece starts on a 256-byte boundary.
size_t branch_bytes(size_t ws, size_t N, int64_t nnz) {
    return align256(ws) + 3 * align256(N * 4) + align256((N + 1) * 8) + 2 * align256((size_t)nnz * 4);
}
size_t stamp_bytes(int n) { return align256((1 + 2 * (size_t)n) * 8); }

size_t batch_bytes(const std::vector<LfSizes> &z, const std::vector<std::vector<int>> &plan) {
    size_t total = stamp_bytes((int)z.size());
    for (const auto &pl : plan) {
        size_t ws = 0, N = 0;
        int64_t nnz = 0;
        for (int i : pl) {
            ws = std::max(ws, z[i].ws);
            N = std::max(N, z[i].N);
            nnz = std::max(nnz, z[i].nnz);
        }
        if (!pl.empty()) total += branch_bytes(ws, N, nnz);
    }
    return total;
}

}  // namespace

struct lfsgm_batch_ctx {
    int n = 0;
    std::vector<lfsgm_ctx *> h;
    std::vector<const float *> views;
    std::vector<float *> disp;
    std::vector<double> work;           // work estimate per light field (scheduling)
    std::vector<LfSizes> sizes;         // scratch sizes per light field
    void *ext = nullptr;                // caller-owned scratch (lfsgm_batch_create_ws), else null
    size_t ext_bytes = 0;
    void *own = nullptr;                // the library's allocation of the branches' scratch
    cudaStream_t main = nullptr;       // the caller's stream: graph launches go here
    cudaStream_t cap = nullptr;        // private stream the graph is captured from
    int branches = 0;
    std::vector<std::vector<int>> plan;  // light fields of each branch, in order
    std::vector<cudaStream_t> bs;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    std::vector<BranchBufs> bb;
    unsigned long long *stamps = nullptr;   // [1 + 2n]: batch start, then (start, end) per light field
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernel_nodes = 0;
    std::string err;
};

namespace {

lfsgm_status bfail(lfsgm_batch_ctx *b, lfsgm_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return st;
}

void batch_release_plan(lfsgm_batch_ctx *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->own) cudaFree(b->own);
    b->own = nullptr;
    b->bb.clear();
    for (auto s : b->bs) cudaStreamDestroy(s);
    for (auto e : b->join) cudaEventDestroy(e);
    b->bs.clear();
    b->join.clear();
    for (auto *h : b->h) {          // the handles no longer own or see any workspace
        h->ws = nullptr;
        h->ws_owned = false;
    }
}

// Assignment of the light fields to K branches, then buffers (caller-owned or one allocation),
// streams and graph.
lfsgm_status batch_build(lfsgm_batch_ctx *b, int K) {
    batch_release_plan(b);
    b->branches = K;
    b->plan = batch_assign(b->work, K);
    const size_t total = batch_bytes(b->sizes, b->plan);
    char *base = nullptr;
    if (b->ext) {
        if (total > b->ext_bytes)
            return bfail(b, LFSGM_ERR_WORKSPACE, "batch workspace of %zu bytes is too small: %d branches need %zu",
                         b->ext_bytes, K, total);
        base = (char *)b->ext + stamp_bytes(b->n);      // the stamps sit at the start
    } else {
        const cudaError_t e = cudaMalloc(&b->own, total - stamp_bytes(b->n));
        if (e != cudaSuccess) return bfail(b, LFSGM_ERR_NO_MEMORY, "batch buffers: %s", cudaGetErrorString(e));
        base = (char *)b->own;
    }
    auto take = [&](size_t n) { char *q = base; base += align256(n); return (void *)q; };
    b->bb.assign(K, BranchBufs());
    b->bs.assign(K, nullptr);
    b->join.assign(K, nullptr);
    for (int k = 0; k < K; k++) {
        size_t ws = 0, N = 0;
        int64_t nnz = 0;
        for (int i : b->plan[k]) {
            ws = std::max(ws, b->sizes[i].ws);
            N = std::max(N, b->sizes[i].N);
            nnz = std::max(nnz, b->sizes[i].nnz);
        }
        BranchBufs &x = b->bb[k];
        cudaError_t e = cudaStreamCreateWithFlags(&b->bs[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "batch streams: %s", cudaGetErrorString(e));
        if (b->plan[k].empty()) continue;
        x.ws = take(ws);
        x.lo = (int *)take(N * 4);
        x.cnt = (int *)take(N * 4);
        x.label = (int *)take(N * 4);
        x.off = (long long *)take((N + 1) * 8);
        x.cost = (float *)take((size_t)nnz * 4);
        x.agg = (float *)take((size_t)nnz * 4);
        x.ws_bytes = ws;
        for (int i : b->plan[k]) {
            b->h[i]->stream = b->bs[k];
            const lfsgm_status st = bind_workspace(b->h[i], x.ws, x.ws_bytes, false);
            if (st != LFSGM_OK) return bfail(b, st, "workspace of light field %d: %s", i, b->h[i]->err.c_str());
        }
    }
    // capture
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    lfsgm_status st = LFSGM_OK;
    stamp_kernel<<<1, 1, 0, b->cap>>>(b->stamps);
    cudaEventRecord(b->fork, b->cap);
    for (int k = 0; k < K && st == LFSGM_OK; k++) {
        cudaStreamWaitEvent(b->bs[k], b->fork, 0);
        BranchBufs &x = b->bb[k];
        for (int i : b->plan[k]) {
            lfsgm_ctx *h = b->h[i];
            stamp_kernel<<<1, 1, 0, b->bs[k]>>>(b->stamps + 1 + 2 * i);
            int64_t *off = (int64_t *)x.off;
            st = lfsgm_initial_disparity(h, b->views[i], 0, 0, x.lo, x.cnt, off, nullptr, nullptr, nullptr);
            if (st == LFSGM_OK) st = cost_volume_impl(h, b->views[i], x.lo, x.cnt, off, x.cost, !h->cfg.boundless);
            if (st == LFSGM_OK) st = lfsgm_sgm_aggregate(h, x.cost, x.lo, x.cnt, off, -1.f, -1.f, x.agg);
            if (st == LFSGM_OK) st = lfsgm_wta_subpixel(h, x.agg, x.lo, x.cnt, off, x.label, b->disp[i]);
            if (st != LFSGM_OK) {
                bfail(b, st, "light field %d: %s", i, h->err.c_str());
                break;
            }
            stamp_kernel<<<1, 1, 0, b->bs[k]>>>(b->stamps + 2 + 2 * i);
        }
        cudaEventRecord(b->join[k], b->bs[k]);
        cudaStreamWaitEvent(b->cap, b->join[k], 0);
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (st != LFSGM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    b->kernel_nodes = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) b->kernel_nodes++;
    }
    return LFSGM_OK;
}

// Speed knobs per shape class (light fields with the same configuration), on the buffers of a
// one-branch plan: the first member is tuned (tune_handle) and every member gets its setting.
lfsgm_status batch_tune_knobs(lfsgm_batch_ctx *b) {
    if (b->branches != 1 || b->bb.empty()) return LFSGM_OK;
    BranchBufs &x = b->bb[0];
    std::vector<int> done(b->n, 0);
    for (int i = 0; i < b->n; i++) {
        if (done[i]) continue;
        lfsgm_ctx *h = b->h[i];
        int kw = 36, lc = 0;
        lfsgm_status st = tune_handle(h, b->views[i], x.lo, x.cnt, (int64_t *)x.off, x.cost, x.agg, kw, lc);
        for (int j = i; j < b->n && st == LFSGM_OK; j++)
            if (!done[j] && memcmp(&b->h[j]->cfg, &h->cfg, sizeof(lfsgm_config)) == 0) {
                st = lfsgm_set_tuning(b->h[j], kw, lc);
                if (st == LFSGM_OK) st = lfsgm_set_sgm_warps(b->h[j], h->sgm_warps);
                if (st == LFSGM_OK) st = lfsgm_set_sgm_split(b->h[j], h->sgm_split);
                done[j] = 1;
            }
        if (st != LFSGM_OK) return bfail(b, st, "tuning light field %d: %s", i, h->err.c_str());
    }
    return LFSGM_OK;
}

float batch_time_ms(lfsgm_batch_ctx *b, int reps) {
    cudaEvent_t a, c;
    cudaEventCreate(&a);
    cudaEventCreate(&c);
    float best = 1e30f;
    for (int r = 0; r < reps; r++) {
        cudaEventRecord(a, b->main);
        cudaGraphLaunch(b->exec, b->main);
        cudaEventRecord(c, b->main);
        cudaEventSynchronize(c);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, c);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(c);
    return best;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

const int kBatchK[] = {1, 2, 4, 8, 16};

lfsgm_status batch_create(int32_t n, const lfsgm_config *cfgs, const float *const *views, float *const *disp,
                          void *stream, int32_t branches, void *ws, size_t ws_bytes, lfsgm_batch *out) {
    if (!out) return LFSGM_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || !cfgs || !views || !disp) return LFSGM_ERR_INVALID_ARG;
    if (ws && ((uintptr_t)ws & 255)) {
        g_create_err = "batch workspace must be 256-byte aligned";
        return LFSGM_ERR_WORKSPACE;
    }
    lfsgm_batch_ctx *b = new lfsgm_batch_ctx();
    b->n = n;
    b->main = (cudaStream_t)stream;
    b->ext = ws;
    b->ext_bytes = ws ? ws_bytes : 0;
    for (int i = 0; i < n; i++) {
        if (!views[i] || !disp[i]) {
            g_create_err = "null views or disp pointer";
            lfsgm_batch_destroy(b);
            return LFSGM_ERR_INVALID_ARG;
        }
        lfsgm_handle h = nullptr;
        const lfsgm_status st = lfsgm_create(&cfgs[i], stream, &h);
        if (st != LFSGM_OK) {
            g_create_err = "light field " + std::to_string(i) + ": " + g_create_err;
            lfsgm_batch_destroy(b);
            return st;
        }
        b->h.push_back(h);
        b->views.push_back(views[i]);
        b->disp.push_back(disp[i]);
        b->sizes.push_back(lf_sizes(h));
        b->work.push_back(b->sizes.back().work);
    }
    cudaError_t e = cudaSuccess;
    if (b->ext) b->stamps = (unsigned long long *)b->ext;
    else e = cudaMalloc((void **)&b->stamps, stamp_bytes(n));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemset(b->stamps, 0, (1 + 2 * (size_t)n) * 8);
    if (e != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        lfsgm_batch_destroy(b);
        return LFSGM_ERR_CUDA;
    }
    lfsgm_status st = LFSGM_OK;
    if (branches > 0) {
        st = batch_build(b, std::min(branches, n));
    } else {
        // speed knobs per shape class on a one-branch plan, then the branch count K (with a caller
        // workspace: the K whose scratch fits it)
        if (!b->ext || batch_bytes(b->sizes, batch_assign(b->work, 1)) <= b->ext_bytes) {
            st = batch_build(b, 1);
            if (st == LFSGM_OK) st = batch_tune_knobs(b);
        }
        int bestK = 0;
        float best = 1e30f;
        for (int K : kBatchK) {
            if (st != LFSGM_OK) break;
            if (K > n) break;
            if (b->ext && batch_bytes(b->sizes, batch_assign(b->work, K)) > b->ext_bytes) continue;
            st = batch_build(b, K);
            if (st != LFSGM_OK) break;
            batch_time_ms(b, 1);                      // warm-up
            const float ms = batch_time_ms(b, 2);
            if (ms < best) {
                best = ms;
                bestK = K;
            }
        }
        if (st == LFSGM_OK && bestK == 0)
            st = bfail(b, LFSGM_ERR_WORKSPACE, "batch workspace of %zu bytes is too small for one branch",
                       b->ext_bytes);
        if (st == LFSGM_OK) st = batch_build(b, bestK);
    }
    if (st != LFSGM_OK) {
        g_create_err = b->err;
        lfsgm_batch_destroy(b);
        return st;
    }
    *out = b;
    return LFSGM_OK;
}

}  // namespace

extern "C" {

lfsgm_status lfsgm_batch_create(int32_t n, const lfsgm_config *cfgs, const float *const *views, float *const *disp,
                                void *stream, int32_t branches, lfsgm_batch *out) {
    return batch_create(n, cfgs, views, disp, stream, branches, nullptr, 0, out);
}

lfsgm_status lfsgm_batch_workspace_size(int32_t n, const lfsgm_config *cfgs, int32_t branches, size_t *bytes) {
    if (!bytes || n < 1 || !cfgs) return LFSGM_ERR_INVALID_ARG;
    std::vector<LfSizes> z;
    std::vector<double> work;
    for (int i = 0; i < n; i++) {
        lfsgm_ctx tmp;
        const lfsgm_status st = plan_handle(cfgs[i], &tmp);
        if (st != LFSGM_OK) {
            g_create_err = "light field " + std::to_string(i) + ": " + g_create_err;
            return st;
        }
        z.push_back(lf_sizes(&tmp));
        work.push_back(z.back().work);
    }
    size_t need = 0;
    if (branches > 0) {
        need = batch_bytes(z, batch_assign(work, std::min((int)branches, (int)n)));
    } else {
        for (int K : kBatchK)
            if (K <= n) need = std::max(need, batch_bytes(z, batch_assign(work, K)));
    }
    *bytes = need;
    return LFSGM_OK;
}

lfsgm_status lfsgm_batch_create_ws(int32_t n, const lfsgm_config *cfgs, const float *const *views,
                                   float *const *disp, void *stream, int32_t branches, void *ws, size_t ws_bytes,
                                   lfsgm_batch *out) {
    if (!ws) {
        if (out) *out = nullptr;
        g_create_err = "null batch workspace";
        return LFSGM_ERR_INVALID_ARG;
    }
    return batch_create(n, cfgs, views, disp, stream, branches, ws, ws_bytes, out);
}

lfsgm_status lfsgm_batch_run(lfsgm_batch b) {
    if (!b || !b->exec) return LFSGM_ERR_INVALID_ARG;
    const cudaError_t e = cudaGraphLaunch(b->exec, b->main);
    if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "graph launch: %s", cudaGetErrorString(e));
    return LFSGM_OK;
}

lfsgm_status lfsgm_batch_knobs(lfsgm_batch b, int32_t *row_kw, int32_t *list_ctas_per_sm) {
    if (!b) return LFSGM_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; i++) {
        if (row_kw) row_kw[i] = b->h[i]->row_kw;
        if (list_ctas_per_sm) list_ctas_per_sm[i] = b->h[i]->list_ctas;
    }
    return LFSGM_OK;
}

lfsgm_status lfsgm_batch_sgm_warps(lfsgm_batch b, int32_t *warps_per_cta) {
    if (!b || !warps_per_cta) return LFSGM_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; i++) warps_per_cta[i] = b->h[i]->sgm_warps;
    return LFSGM_OK;
}

lfsgm_status lfsgm_batch_sgm_split(lfsgm_batch b, int32_t *min_wide) {
    if (!b || !min_wide) return LFSGM_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; i++) min_wide[i] = b->h[i]->sgm_split;
    return LFSGM_OK;
}

lfsgm_status lfsgm_batch_times(lfsgm_batch b, double *start_ms, double *end_ms, int32_t *branches) {
    if (!b) return LFSGM_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->main);
    std::vector<unsigned long long> t(1 + 2 * (size_t)b->n);
    if (e == cudaSuccess) e = cudaMemcpy(t.data(), b->stamps, t.size() * 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, LFSGM_ERR_CUDA, "stamps: %s", cudaGetErrorString(e));
    for (int i = 0; i < b->n; i++) {
        if (start_ms) start_ms[i] = (double)(long long)(t[1 + 2 * i] - t[0]) * 1e-6;
        if (end_ms) end_ms[i] = (double)(long long)(t[2 + 2 * i] - t[0]) * 1e-6;
    }
    if (branches) *branches = b->branches;
    for (auto *h : b->h) {
        const lfsgm_status st = lfsgm_sync(h);
        if (st != LFSGM_OK) return bfail(b, st, "%s", h->err.c_str());
    }
    return LFSGM_OK;
}

int64_t lfsgm_batch_kernel_nodes(lfsgm_batch b) { return b ? b->kernel_nodes : -1; }

const char *lfsgm_batch_last_error(lfsgm_batch b) { return b ? b->err.c_str() : g_create_err.c_str(); }

lfsgm_status lfsgm_batch_destroy(lfsgm_batch b) {
    if (!b) return LFSGM_ERR_INVALID_ARG;
    if (!b->h.empty() || b->stamps) cudaDeviceSynchronize();
    batch_release_plan(b);
    for (auto *h : b->h) lfsgm_destroy(h);
    if (!b->ext) cudaFree(b->stamps);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return LFSGM_OK;
}

}  // extern "C"
