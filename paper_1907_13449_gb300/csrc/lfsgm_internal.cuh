// lfsgm_internal.cuh -- internal declarations shared by the library's kernels and its
// C-ABI layer.  Not installed, not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <vector>

namespace lfsgm {

// Per (view, fine label) shift split of (u-uc, v-vc) * d_g, built on the host in
// double precision (see lfsgm.h, "Shift split"); fractions rounded to float once.
struct FineTap {
    int16_t ox, oy;   // floor of the x / y shift (bilinear taps)
    int16_t nx, ny;   // nearest integer x / y shift (census position)
    float fx, fy;     // fractional parts in [0, 1)
};
static_assert(sizeof(FineTap) == 16, "FineTap must be 16 bytes");

#ifdef __CUDACC__
// A window must satisfy 0 <= lo, 1 <= cnt, lo + cnt <= G and fit its row
// (off[p+1] - off[p] >= cnt).  Kernels skip a pixel whose window does not and latch
// LFSGM_ERR_DEVICE_CHECK (7) in the handle's status word.
__device__ __forceinline__ bool window_ok(int l, int n, int G, long long row, int *status) {
    const bool ok = l >= 0 && n >= 1 && l + n <= G && (long long)n <= row;
    if (!ok && status) atomicExch(status, 7);
    return ok;
}

// A windowed row read as 16-byte vectors must start on a multiple of 4 slots (the layout's rule).
__device__ __forceinline__ bool row_aligned(long long o, int *status) {
    const bool ok = (o & 3) == 0;
    if (!ok && status) atomicExch(status, 7);
    return ok;
}

// The KW-label range [g0, g0 + KW) that holds the most windows of at most 32 labels (nar) of a
// warp's 32 pixels (ties: the lowest start; candidates are the lanes' own window starts, in lane
// order).  Returns the number of windows it holds (-1 when no lane has a narrow window).
template <int KW>
__device__ __forceinline__ int row_range(int l, int n, bool nar, int &g0) {
    int best = -1;
    g0 = 0;
    for (int c = 0; c < 32; c++) {
        const int cl = __shfl_sync(0xffffffffu, l, c);
        if (!__shfl_sync(0xffffffffu, nar, c)) continue;
        const int fit = __popc(__ballot_sync(0xffffffffu, nar && l >= cl && l + n <= cl + KW));
        if (fit > best || (fit == best && cl < g0)) {
            best = fit;
            g0 = cl;
        }
    }
    return best;
}

// Append (pixel, chunk of 32 labels) work items for a window of n labels.
__device__ __forceinline__ void push_chunks(int2 *list, int *count, int p, int n) {
    const int nch = (n + 31) >> 5;
    const int k = atomicAdd(count, nch);
    for (int c = 0; c < nch; c++) list[k + c] = make_int2(p, c);
}

// One 16-byte read-only load of a table entry.
__device__ __forceinline__ FineTap load_tap(const FineTap *t) {
    const int4 w = __ldg(reinterpret_cast<const int4 *>(t));
    FineTap r;
    r.ox = (int16_t)(w.x & 0xffff);
    r.oy = (int16_t)(w.x >> 16);
    r.nx = (int16_t)(w.y & 0xffff);
    r.ny = (int16_t)(w.y >> 16);
    r.fx = __int_as_float(w.z);
    r.fy = __int_as_float(w.w);
    return r;
}
#endif

// The SGM directions r = (dx, dy); the predecessor of p is p - r.  Same order as the oracle:
// (1,0) (-1,0) (0,1) (0,-1) (1,1) (-1,-1) (1,-1) (-1,1), then the paper's other eight of its 16
// (Sec. IV-C), of slopes 1/2 and 2: (2,1) (-2,-1) (2,-1) (-2,1) (1,2) (-1,-2) (1,-2) (-1,2).
constexpr int kMaxPaths = 16;
__host__ __device__ inline int dir_dx(int r) {
    const int t[16] = {1, -1, 0, 0, 1, -1, 1, -1, 2, -2, 2, -2, 1, -1, 1, -1};
    return t[r];
}
__host__ __device__ inline int dir_dy(int r) {
    const int t[16] = {0, 0, 1, -1, 1, -1, -1, 1, 1, -1, -1, 1, 2, -2, -2, 2};
    return t[r];
}
// Scanlines of direction r start at the pixels p whose p - r leaves the image: the first
// by = min(|dy|, H) rows on the side p - r leaves through (all W columns), then the first
// bx = min(|dx|, W) columns on the other side, without those rows.  Every pixel lies on
// exactly one scanline (walk back from it until p - r leaves the image).
__host__ __device__ inline int n_scanlines(int r, int H, int W) {
    const int ax = abs(dir_dx(r)), ay = abs(dir_dy(r));
    const int bx = ax < W ? ax : W, by = ay < H ? ay : H;
    return by * W + bx * (H - by);
}
// The same table as bit fields of two constants, for kernels that index it with a run-time r and
// would otherwise copy it to the stack: direction pair k = r >> 1 is (bx_k, by_k - 2) (x in 2-bit
// fields, y in 3-bit fields), negated for odd r.
__host__ __device__ inline void dir_of(int r, int &dx, int &dy) {
    const int k = r >> 1, sg = (r & 1) ? -1 : 1;
    dx = sg * (int)((0x5A51u >> (2 * k)) & 3u);
    dy = sg * ((int)((0x10B2DAu >> (3 * k)) & 7u) - 2);
}
// Start pixel of scanline s of the direction (dx, dy).
__host__ __device__ inline void scan_start_d(int dx, int dy, int s, int H, int W, int &x, int &y) {
    const int ay = abs(dy);
    const int by = ay < H ? ay : H;
    if (s < by * W) {
        const int i = s / W;
        x = s - i * W;
        y = dy > 0 ? i : H - 1 - i;
    } else {
        const int t = s - by * W, rows = H - by;
        const int j = t / rows;
        const int k = t - j * rows;
        x = dx > 0 ? j : W - 1 - j;
        y = dy > 0 ? by + k : (dy < 0 ? H - 1 - by - k : k);
    }
}
// Start pixel of scanline s of direction r.
__host__ __device__ inline void scan_start(int r, int s, int H, int W, int &x, int &y) {
    scan_start_d(dir_dx(r), dir_dy(r), s, H, W, x, y);
}
// The scanline of direction r through pixel (x, y): walk back to its start pixel (the last one
// before p - r leaves the image), then invert scan_start.
__host__ __device__ inline int scan_index(int r, int x, int y, int H, int W) {
    const int dx = dir_dx(r), dy = dir_dy(r);
    const int tx = dx > 0 ? x / dx : (dx < 0 ? (W - 1 - x) / (-dx) : 0x7fffffff);
    const int ty = dy > 0 ? y / dy : (dy < 0 ? (H - 1 - y) / (-dy) : 0x7fffffff);
    const int t = tx < ty ? tx : ty;
    const int xs = x - t * dx, ys = y - t * dy;
    const int ay = abs(dy), by = ay < H ? ay : H;
    if (dy > 0 && ys < by) return ys * W + xs;
    if (dy < 0 && H - 1 - ys < by) return (H - 1 - ys) * W + xs;
    const int j = dx > 0 ? xs : W - 1 - xs;
    const int k = dy > 0 ? ys - by : (dy < 0 ? H - 1 - by - ys : ys);
    return by * W + j * (H - by) + k;
}

// Cumulative scanline counts of the first `paths` directions (cum[paths] = total).
struct ScanTable {
    int cum[kMaxPaths + 1];
    int paths;
};
inline ScanTable make_scan_table(int H, int W, int paths) {
    ScanTable t;
    t.paths = paths;
    t.cum[0] = 0;
    for (int r = 0; r < kMaxPaths; r++) t.cum[r + 1] = t.cum[r] + (r < paths ? n_scanlines(r, H, W) : 0);
    return t;
}

// Steps of the scanline starting at (x0, y0) in direction (dx, dy).
__host__ __device__ inline int scan_steps(int x0, int y0, int dx, int dy, int H, int W) {
    const int lx = dx > 0 ? (W - 1 - x0) / dx + 1 : (dx < 0 ? x0 / (-dx) + 1 : 0x7fffffff);
    const int ly = dy > 0 ? (H - 1 - y0) / dy + 1 : (dy < 0 ? y0 / (-dy) + 1 : 0x7fffffff);
    return lx < ly ? lx : ly;
}
// Length of scanline s of direction r.
__host__ __device__ inline int scan_len(int r, int s, int H, int W) {
    int x, y;
    scan_start(r, s, H, W, x, y);
    return scan_steps(x, y, dir_dx(r), dir_dy(r), H, W);
}
// Every (direction r < paths, scanline s) as (s << 4 | r), longest scanline first (ties: r, then
// s): the SGM kernels take warps in this order, so the short lines fill in behind the long ones
// instead of forming a tail.
void build_scan_order(int H, int W, int paths, std::vector<int> &order);

constexpr int kMaxArmViews = 64;

struct ArmList {
    int n_arms;               // non-empty arms, in the order up, down, left, right
    int arm_id[4];            // 0 up, 1 down, 2 left, 3 right
    int nv[4];                // views per arm
    int views[4][kMaxArmViews];
};

// ----------------------------------------------------------------- launchers
// Each launcher issues exactly one kernel on `s` and returns cudaGetLastError().
cudaError_t launch_census(cudaStream_t s, const float *views, int H, int W, int census_w,
                          const int *d_sel, int nsel, uint64_t *cen);

// Coarse arms as the cost kernel sees them: views per arm and the start of each arm's
// [nv][Lcd] table of linear census offsets (ny * Wp + nx) in the offset table.
struct CoarseArms {
    int n_arms;
    int nv[4];
    int tab_off[4];
};
int coarse_lpt(int Lc);       // labels per lane: 2, 4, 8 for Lc <= 64, 128, 256
int coarse_stride(int Lc);    // Lcd: label stride of the coarse cost and sums
// Images are planes view * C + c of H x W (padded: Hp x Wp); `ref` and `armviews` count views.
cudaError_t launch_coarse_cost(cudaStream_t s, const uint64_t *cen_pad, int P, int Wp, int Hp, int H, int W, int ref,
                               int C, const int *armviews, const int *otab, const CoarseArms &ca, int Lc,
                               void *out, bool out8, unsigned long long *armsum);
cudaError_t launch_coarse_penalties(cudaStream_t s, const unsigned long long *sums, int narms,
                                    long long count, double p1f, double p2f, int P1, int P2,
                                    int *pen);
cudaError_t launch_coarse_sgm(cudaStream_t s, const void *cost, bool cost8, int narms, int H, int W, int Lc,
                              const int *pen, uint16_t *sum, const int *order, int paths);
cudaError_t launch_coarse_wta(cudaStream_t s, const uint16_t *sum, int narms, int N, int Lc, int *maps,
                              int *maps_out);

cudaError_t launch_fuse(cudaStream_t s, const int *maps, int narms, int N, double phi, int *F);
cudaError_t launch_fill(cudaStream_t s, const int *Fin, int *Fout, int H, int W);
cudaError_t launch_windows(cudaStream_t s, const int *F, int N, int G, int Lc, int R, int *lo,
                           int *cnt, float *dinit, int *cntpad, const float *ref_pad, int C, int P,
                           int Wp, int W, float edge_t, int Rfar, int boundless);
int scan_tiles(int N);   // tiles of the offset scan (tile sums buffer length)
cudaError_t launch_scan_sums(cudaStream_t s, const int *cntpad, int N, long long *tsum);
cudaError_t launch_scan_top(cudaStream_t s, long long *tsum, int N);
cudaError_t launch_scan_apply(cudaStream_t s, const int *cntpad, int N, const long long *tsum, long long *off);

cudaError_t launch_fine_cost(cudaStream_t s, const float *views, const uint64_t *cen,
                             const FineTap *tab, int G, int nviews, int H, int W, int ref,
                             const int *lo, const int *cnt, const long long *off, float wl2,
                             float wc, float *cost, int *status);

// Row-sweep cost volume (regular windows, TMA-staged from padded copies of the views and census
// words) + per-pixel list kernel (windows that do not fit a row's label range).
struct RowPlanHost {
    alignas(64) unsigned char tm_v[128];   // CUtensorMap of the padded views
    alignas(64) unsigned char tm_c[128];   // CUtensorMap of the padded census words
    unsigned char raw[128];                // kernel-side plan
    bool ok;
    int P, Wp, Hp;                         // padding and padded sizes
};
// kw: the label span of a row's range, 36 or 44 (two instantiations of the row kernel); C: channels
// (colour: span 36 only; any other span leaves the plan not ok, and every window to the list kernel).
bool plan_fine_rows(int U, int V, int uc, int vc, int H, int W, int G, double dmin, double dmax, int kw, int C,
                    RowPlanHost *out);
bool encode_fine_rows_maps(RowPlanHost *ph, const float *views_pad, const uint64_t *cen_pad, int nviews);
// Census words (planes view * C + c) and the edge-padded views (C = 1: float planes; C = 3: one
// float4 per pixel, channels interleaved) of the views listed in d_sel.
cudaError_t launch_census_pad(cudaStream_t s, const float *views, int H, int W, int census_w, int P, int Wp,
                              int Hp, int C, const int *d_sel, int nsel, uint64_t *cen_pad, float *views_pad);
bool build_fine_rows_desc(const RowPlanHost *ph, const FineTap *tab, int U, int V, int uc, int vc, int G,
                          float dmin, float fstep, std::vector<unsigned char> &out);
cudaError_t launch_fine_cost_rows(cudaStream_t s, const RowPlanHost *ph, const float *views_pad,
                                  const uint64_t *cen_pad, const unsigned char *desc, int G, int U, int V, int H,
                                  int W, int ref, const int *lo, const int *cnt, const long long *off, float wl2,
                                  float wc, float fstep, float *cost, int *status, int2 *list, int *list_count);
cudaError_t launch_list_all(cudaStream_t s, const int *lo, const int *cnt, const long long *off, int G,
                            int2 *list, int *count, int N, int *status, int min_cnt = 0);
cudaError_t launch_fine_cost_list(cudaStream_t s, const float *views_pad, const uint64_t *cen_pad, int P, int Wp,
                                  int Hp, const int4 *ltab, int G, int nviews, int C, int W, int ref,
                                  const int *lo, const int *cnt, const long long *off, float wl2, float wc,
                                  float *cost, const int2 *list, const int *count,
                                  int ctas_per_sm = 0);

// Mean cost over the active slots and the derived penalties pen = (p1f, p2f) x mean, in one launch:
// partial holds nblocks sums followed by nblocks counts; ticket (zero between launches) picks the
// block that adds them up.
// With split (not null, its first int zeroed before), the same launch also lists the SGM
// scanlines to split, as launch_sgm_split does, in extra blocks.
cudaError_t launch_cost_partial_sums(cudaStream_t s, const float *cost, const int *cnt,
                                     const long long *off, int N, int G, double *partial, int nblocks,
                                     double p1f, double p2f, float *pen, unsigned *ticket, int *status,
                                     int H, int W, int paths, int min_wide, int *split);
// split (may be null): the scanlines that launch_sgm_split listed run split across a CTA's warps
// (the same values, faster when a few scanlines cross many wide windows).
cudaError_t launch_fine_sgm(cudaStream_t s, const float *cost, const int *lo, const int *cnt,
                            const long long *off, int H, int W, int G, const float *pen, float *agg,
                            int *status, const int *order, int paths,
                            unsigned char *codes = nullptr, int *amin = nullptr, size_t nnz_cap = 0,
                            int warps_per_cta = 4, const int *split = nullptr);
// Ints of the split table of launch_fine_sgm for an H x W image and `paths` directions; its first
// int must be zero before launch_sgm_split, which lists the scanlines that cross at least min_wide
// windows wider than 32 labels.
int sgm_split_ints(int H, int W, int paths);
cudaError_t launch_sgm_split(cudaStream_t s, const int *cnt, int H, int W, int paths, int min_wide, int *split);

cudaError_t launch_median3(cudaStream_t s, const float *in, float *out, int H, int W);
cudaError_t launch_wta(cudaStream_t s, const float *agg, const int *lo, const int *cnt,
                       const long long *off, int N, int G, double dmin, double step, int mode,
                       float tau, int *label, float *disp, int *status);

cudaError_t launch_softargmin_backward(cudaStream_t s, const float *agg, const int *lo, const int *cnt,
                                       const long long *off, int N, int G, double dmin, double step, float tau,
                                       const float *gdisp, float *gCs, float *gcost, int *status);
cudaError_t launch_sgm_backward(cudaStream_t s, const float *cost, const int *lo, const int *cnt,
                                const long long *off, int H, int W, int G, float P1, float P2, const float *gCs,
                                unsigned char *codes, int *amin, size_t nnz_cap, float *gcost, float *gP,
                                int *status, const int *order, int paths,
                                bool recompute = true);
cudaError_t launch_views_backward(cudaStream_t s, const float *views, const FineTap *tab, int G, int U, int V, int C,
                                  int H, int W, int ref, const int *lo, const int *cnt, const long long *off,
                                  float wl2, float fstep, const float *gcost, float *gviews, int2 *list, int *count);
// Grey: the items of the list (wide windows, and narrow ones the row kernel left) after launch_views_backward.
cudaError_t launch_views_backward_list(cudaStream_t s, const float *views, const FineTap *tab, int G, int nviews,
                                       int C, int H, int W, int ref, const int *lo, const int *cnt,
                                       const long long *off, float wl2, const float *gcost, float *gviews,
                                       const int2 *list, const int *count);

constexpr int kPartialBlocks = 1024;

}  // namespace lfsgm
