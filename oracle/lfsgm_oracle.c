/*
 * lfsgm_oracle.c -- plain, slow FP64 CPU reference ("oracle") of the light-field
 * depth method of Anisimov, Wasenmueller and Stricker, "Rapid Light Field Depth
 * Estimation with Semi-Global Matching" (ICCP 2019).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call it.  The CUDA library
 * never includes, links or calls it, and it shares no header, table or helper
 * with the CUDA library: every step below is written out from the paper's
 * equations in the paper's order, with plain loops, in double precision.
 *
 * Conventions (the paper's symbols in brackets):
 *   views[v][u][c][y][x]  float32 input, (x,y) spatial [(u,v) in the paper],
 *                      (u,v) angular [(s,t) in the paper]; reference (uc,vc);
 *                      c the colour channel (C = 1 grey, C = 3 RGB).
 *   a view (u,v) is sampled for pixel (x,y) and disparity d at
 *        (x + (u-uc)*d, y + (v-vc)*d)                     (Eq. 1, sign flipped:
 *   the paper writes (s^-s)*d; we measure d with the opposite sign so that a
 *   larger d is a nearer plane).
 *   Disparity grids have inclusive end points:
 *        d_k = dmin + k * ((dmax-dmin)/(L-1)),  k = 0..L-1.
 *   Shift rule (the paper is silent on how fractional shifts are split):
 *        s = a*d in double; if 2s is within 2e-9 of an integer, s is snapped to
 *        that half-integer; ox = floor(s), fx = s - ox, nx = floor(s + 0.5).
 *   Image borders (the paper is silent): every tap index is clamped to the image.
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC (oracle/__init__.py).
 * OpenMP only splits loops whose iterations are independent (rows, or the pixels of a
 * row whose predecessors are final); every value is computed by the same expression in
 * the same order as the serial loop, so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t U, V, H, W;   /* angular and spatial sizes                                */
    int32_t uc, vc;       /* reference view                                           */
    int32_t census_w;     /* census window side (odd); dense window minus the centre  */
    double dmin, dmax;    /* disparity range T (Sec. III-D)                            */
    int32_t Lc;           /* coarse labels on [dmin,dmax], inclusive                  */
    int32_t init_views;   /* 0: one extreme view per arm (Sec. III-D); 1: whole arms  */
    double phi;           /* fusion threshold, coarse-label units (Sec. IV params: 3)  */
    int32_t fill_passes;  /* median hole-filling passes (Sec. III-D: one or two)       */
    int32_t G;            /* fine labels on [dmin,dmax], inclusive                    */
    int32_t R;            /* border threshold lambda in fine labels (Eq. 11)           */
    double w_l2, w_census;/* weights of Eq. 12 (l2) and Eq. 15 (census) terms          */
    int32_t paths;        /* SGM directions: 8, or the paper's 16 (Sec. IV-C)           */
    float edge_threshold; /* Sobel edge exclusion (Sec. III-D): 0 = off                 */
    int32_t channels;     /* colour channels C: 1 or 3 (0 means 1)                      */
    int32_t boundless;    /* 1: every window is the whole range, no initial map (Sec. IV-E) */
    int32_t R_far;        /* > 0: border threshold at d = dmin (depth-dependent lambda)     */
} or_cfg;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }
static int nchan(const or_cfg *c) { return c->channels > 1 ? c->channels : 1; }

/* Disparity of label k on an inclusive grid of L labels over [dmin,dmax]. */
double or_label_disp(double dmin, double dmax, int L, int k)
{
    double step = (dmax - dmin) / (double)(L - 1);
    return dmin + (double)k * step;
}

/* Split the shift a*d into integer + fraction (bilinear taps) and nearest integer
 * (census position).  See the shift rule in the file header. */
void or_shift(int a, double d, int *o, double *f, int *n)
{
    double s = (double)a * d;
    double t = 2.0 * s;
    double r = nearbyint(t);
    if (fabs(t - r) <= 2e-9) s = 0.5 * r;
    double fl = floor(s);
    *o = (int)fl;
    *f = s - fl;
    *n = (int)floor(s + 0.5);
}

/* ---------------------------------------------------------------- Census (Eq. 2-3)
 * Bit k of the word of pixel (x,y) is xi(I(x,y), I(x+dx,y+dy)) for the k-th offset of
 * the w x w window without its centre, offsets in row-major order (dy outer, dx inner),
 * bit 0 first; xi(p1,p2) = 1 iff p1 > p2 (Eq. 3).  Neighbours are clamped. */
void or_census(const double *img, int H, int W, int w, uint64_t *out)
{
    int h = w / 2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double c = (double)img[(size_t)y * W + x];
            uint64_t word = 0;
            int bit = 0;
            for (int dy = -h; dy <= h; dy++)
                for (int dx = -h; dx <= h; dx++) {
                    if (dx == 0 && dy == 0) continue;
                    int yy = clampi(y + dy, 0, H - 1), xx = clampi(x + dx, 0, W - 1);
                    double nb = (double)img[(size_t)yy * W + xx];
                    if (c > nb) word |= (uint64_t)1 << bit;
                    bit++;
                }
            out[(size_t)y * W + x] = word;
        }
}

/* Hamming distance (Eq. 5): number of positions where the two bit strings differ. */
int or_hamming(uint64_t a, uint64_t b)
{
    int n = 0;
    for (int k = 0; k < 64; k++)
        if (((a >> k) & 1u) != ((b >> k) & 1u)) n++;
    return n;
}

/* Census words of every view and channel, each channel on its own (Sec. III-B):
 * out[((v*U+u)*C + ch)*H*W + y*W + x]. */
void or_census_all(const or_cfg *c, const double *views, uint64_t *out)
{
    size_t HW = (size_t)c->H * c->W;
    size_t planes = (size_t)c->V * c->U * nchan(c);
    for (size_t q = 0; q < planes; q++)
        or_census(views + q * HW, c->H, c->W, c->census_w, out + q * HW);
}

/* ------------------------------------------------------ Initial views (Sec. III-D)
 * The paper's set V lists, in this order, the views (s^,0), (s^,t_max), (0,t^),
 * (s_max,t^): up, down, left, right of the reference.  With init_views = 1 each of
 * these becomes an arm holding every view between the reference and the extreme
 * view.  Returns the number of views of arm `arm` and writes them as (u,v) pairs. */
int or_arm_views(const or_cfg *c, int arm, int *uv)
{
    int n = 0;
    if (arm == 0) {        /* up:    (uc, v < vc) */
        for (int v = c->vc - 1; v >= 0; v--)
            if (c->init_views || v == 0) { uv[2 * n] = c->uc; uv[2 * n + 1] = v; n++; }
    } else if (arm == 1) { /* down:  (uc, v > vc) */
        for (int v = c->vc + 1; v < c->V; v++)
            if (c->init_views || v == c->V - 1) { uv[2 * n] = c->uc; uv[2 * n + 1] = v; n++; }
    } else if (arm == 2) { /* left:  (u < uc, vc) */
        for (int u = c->uc - 1; u >= 0; u--)
            if (c->init_views || u == 0) { uv[2 * n] = u; uv[2 * n + 1] = c->vc; n++; }
    } else {               /* right: (u > uc, vc) */
        for (int u = c->uc + 1; u < c->U; u++)
            if (c->init_views || u == c->U - 1) { uv[2 * n] = u; uv[2 * n + 1] = c->vc; n++; }
    }
    return n;
}

/* Coarse census cost of one arm (Eq. 7, summed over the arm's views as in Eq. 15):
 *   C_a(p,k) = sum_{(u,v) in arm} sum_ch HD(cen_ref,ch(p), cen_uv,ch(p + nearest shift at d_k)),
 * the Hamming distances of the channels summed (Sec. III-B).
 * cen: census words of all views (or_census_all).  out: [H*W][Lc] int64.
 * Returns the number of views in the arm (0 = empty arm, out untouched). */
int or_coarse_cost(const or_cfg *c, const uint64_t *cen, int arm, int64_t *out)
{
    int uv[2 * 512];
    int nv = or_arm_views(c, arm, uv);
    if (nv == 0) return 0;
    size_t HW = (size_t)c->H * c->W;
    const int Ch = nchan(c);
    const uint64_t *cref = cen + ((size_t)c->vc * c->U + c->uc) * Ch * HW;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < c->H; y++)
        for (int x = 0; x < c->W; x++)
            for (int k = 0; k < c->Lc; k++) {
                double d = or_label_disp(c->dmin, c->dmax, c->Lc, k);
                int64_t sum = 0;
                for (int i = 0; i < nv; i++) {
                    int u = uv[2 * i], v = uv[2 * i + 1];
                    int ox, oy, nx, ny;
                    double fx, fy;
                    or_shift(u - c->uc, d, &ox, &fx, &nx);
                    or_shift(v - c->vc, d, &oy, &fy, &ny);
                    int xx = clampi(x + nx, 0, c->W - 1), yy = clampi(y + ny, 0, c->H - 1);
                    const uint64_t *cv = cen + ((size_t)v * c->U + u) * Ch * HW;
                    for (int ch = 0; ch < Ch; ch++)
                        sum += or_hamming(cref[ch * HW + (size_t)y * c->W + x], cv[ch * HW + (size_t)yy * c->W + xx]);
                }
                out[((size_t)y * c->W + x) * c->Lc + k] = sum;
            }
    return nv;
}

/* Penalties derived from the mean cost (P1 = p1f * mean, P2 = p2f * mean) for the
 * integer coarse pass: rounded half up, P1 >= 1, P2 >= P1 (Eq. 8 needs P2 >= P1). */
void or_int_penalties(int64_t sum, int64_t count, double p1f, double p2f, int64_t *P1, int64_t *P2)
{
    double mean = (double)sum / (double)count;
    int64_t a = (int64_t)floor(p1f * mean + 0.5);
    int64_t b = (int64_t)floor(p2f * mean + 0.5);
    if (a < 1) a = 1;
    if (b < a) b = a;
    *P1 = a;
    *P2 = b;
}

/* --------------------------------------------------------------- SGM (Eq. 8-9)
 * The directions r = (dx,dy); the predecessor of p is p - r.  The first 8 are the horizontal,
 * vertical and diagonal ones; the paper's 16 (Sec. IV-C) add the eight of slopes 1/2 and 2. */
static const int DIRS[16][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1},
                                {2, 1}, {-2, -1}, {2, -1}, {-2, 1}, {1, 2}, {-1, -2}, {1, -2}, {-1, 2}};

/* Visit order for direction r: rows and columns are walked so that p - r is always
 * visited before p. */
static int order_y(int i, int H, int dy) { return dy >= 0 ? i : H - 1 - i; }
static int order_x(int i, int W, int dx) { return dx >= 0 ? i : W - 1 - i; }

/* Integer SGM over the full label range for one direction (Eq. 8, normalised form
 * of Hirschmueller: the minimum m of the predecessor's costs is subtracted, which
 * shifts L_r(p,.) by a constant and leaves every argmin unchanged):
 *   L(p,d) = C(p,d) + (min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m+P2) - m)
 * with L'(.) = L(p-r,.) and L(p,.) = C(p,.) where p-r is outside the image. */
static void sgm_int_step(int H, int W, int L, const int64_t *C, int64_t P1, int64_t P2, int dx, int dy,
                         int x, int y, int64_t *Lr)
{
    int qx = x - dx, qy = y - dy;
    const int64_t *c = C + ((size_t)y * W + x) * L;
    int64_t *l = Lr + ((size_t)y * W + x) * L;
    if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
        for (int d = 0; d < L; d++) l[d] = c[d];
        return;
    }
    const int64_t *lp = Lr + ((size_t)qy * W + qx) * L;
    int64_t m = lp[0];
    for (int d = 1; d < L; d++) if (lp[d] < m) m = lp[d];
    for (int d = 0; d < L; d++) {
        int64_t t = m + P2;
        if (lp[d] < t) t = lp[d];
        if (d > 0 && lp[d - 1] + P1 < t) t = lp[d - 1] + P1;
        if (d < L - 1 && lp[d + 1] + P1 < t) t = lp[d + 1] + P1;
        l[d] = c[d] + (t - m);
    }
}

/* Integer SGM over the full label range for one direction (Eq. 8, normalised form
 * of Hirschmueller: the minimum m of the predecessor's costs is subtracted, which
 * shifts L_r(p,.) by a constant and leaves every argmin unchanged):
 *   L(p,d) = C(p,d) + (min(L'(d), L'(d-1)+P1, L'(d+1)+P1, m+P2) - m)
 * with L'(.) = L(p-r,.) and L(p,.) = C(p,.) where p-r is outside the image.
 * Pixels whose predecessors are already final are processed in parallel: whole rows
 * for horizontal paths, the pixels of one row otherwise (every other direction has
 * dy != 0, so p - r lies in an earlier row). */
void or_sgm_int_path(int H, int W, int L, const int64_t *C, int64_t P1, int64_t P2, int dir, int64_t *Lr)
{
    int dx = DIRS[dir][0], dy = DIRS[dir][1];
    if (dy == 0) {
#pragma omp parallel for schedule(static)
        for (int iy = 0; iy < H; iy++)
            for (int ix = 0; ix < W; ix++)
                sgm_int_step(H, W, L, C, P1, P2, dx, dy, order_x(ix, W, dx), order_y(iy, H, dy), Lr);
    } else {
        for (int iy = 0; iy < H; iy++) {
#pragma omp parallel for schedule(static)
            for (int ix = 0; ix < W; ix++)
                sgm_int_step(H, W, L, C, P1, P2, dx, dy, order_x(ix, W, dx), order_y(iy, H, dy), Lr);
        }
    }
}

/* Sum over the 8 or 16 directions (Eq. 9). */
void or_sgm_int(int H, int W, int L, const int64_t *C, int64_t P1, int64_t P2, int paths, int64_t *Cs)
{
    size_t n = (size_t)H * W * L;
    int64_t *Lr = (int64_t *)malloc(n * sizeof(int64_t));
    memset(Cs, 0, n * sizeof(int64_t));
    for (int r = 0; r < paths; r++) {
        or_sgm_int_path(H, W, L, C, P1, P2, r, Lr);
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < n; i++) Cs[i] += Lr[i];
    }
    free(Lr);
}

/* Winner-takes-all (Eq. 10); ties go to the lowest label. */
void or_wta_int(size_t N, int L, const int64_t *Cs, int32_t *D)
{
    for (size_t p = 0; p < N; p++) {
        const int64_t *c = Cs + p * L;
        int best = 0;
        for (int d = 1; d < L; d++) if (c[d] < c[best]) best = d;
        D[p] = best;
    }
}

/* ------------------------------------------------------ Fusion (Sec. III-D)
 * D_init = D_1; then for each further map D_i in order: if |D_init - D_i| < phi the
 * new value is the average of the two, otherwise the pixel is discarded (and stays
 * discarded).  Values are coarse-label indices; NaN marks a discarded pixel. */
void or_fuse(size_t N, int nmaps, const int32_t *D, double phi, double *dinit)
{
    for (size_t p = 0; p < N; p++) {
        double v = (double)D[p];
        int ok = 1;
        for (int i = 1; i < nmaps && ok; i++) {
            double di = (double)D[(size_t)i * N + p];
            if (fabs(v - di) < phi) v = (v + di) / 2.0;
            else ok = 0;
        }
        dinit[p] = ok ? v : NAN;
    }
}

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Median hole filling (Sec. III-D, window 3 from Sec. IV params): in each pass every
 * discarded pixel takes the median of the valid values among its 8 neighbours in the
 * previous pass's map (lower middle for an even count); with no valid neighbour it
 * stays discarded. */
void or_hole_fill(int H, int W, int passes, double *dinit)
{
    size_t N = (size_t)H * W;
    double *prev = (double *)malloc(N * sizeof(double));
    for (int it = 0; it < passes; it++) {
        memcpy(prev, dinit, N * sizeof(double));
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                if (!isnan(prev[(size_t)y * W + x])) continue;
                double vals[8];
                int n = 0;
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        if (dx == 0 && dy == 0) continue;
                        int xx = x + dx, yy = y + dy;
                        if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
                        double q = prev[(size_t)yy * W + xx];
                        if (!isnan(q)) vals[n++] = q;
                    }
                if (n > 0) {
                    qsort(vals, (size_t)n, sizeof(double), cmp_double);
                    dinit[(size_t)y * W + x] = vals[(n - 1) / 2];
                }
            }
    }
    free(prev);
}

/* Borders (Eq. 11) on the fine grid.  D_init (coarse units, a multiple of 1/8) is
 * moved to the nearest fine label gc (exact rational arithmetic, ties upward), the
 * window is [gc - R, gc + R] saturated to [0, G-1]; a discarded pixel searches the
 * whole range T.  (lo, cnt) give the window as first fine label and label count. */
/* Edges of the reference view for the border exclusion (Sec. III-D): the 3 x 3 Sobel gradient
 * with the neighbours clamped to the image,
 *   gx = ((p2 + 2 p5) + p8) - ((p0 + 2 p3) + p6),  gy = ((p6 + 2 p7) + p8) - ((p0 + 2 p1) + p2)
 * (p0..p8 the window row-major), and a pixel is an edge iff gx^2 + gy^2 > t^2.  The paper gives
 * no threshold.  The sums, squares and the comparison are IEEE FP32 in exactly this order, so the
 * integer decision is the same in any implementation that follows it. */
void or_sobel_edges(int H, int W, const float *I, float t, uint8_t *edge)
{
    const float t2 = t * t;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            float q[9];
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++)
                    q[(dy + 1) * 3 + dx + 1] = I[(size_t)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];
            volatile float a, b, gx, gy, m;
            a = q[2] + 2.0f * q[5]; a = a + q[8];
            b = q[0] + 2.0f * q[3]; b = b + q[6];
            gx = a - b;
            a = q[6] + 2.0f * q[7]; a = a + q[8];
            b = q[0] + 2.0f * q[1]; b = b + q[2];
            gy = a - b;
            a = gx * gx;
            b = gy * gy;
            m = a + b;
            edge[(size_t)y * W + x] = m > t2;
        }
}

/* floor(a / b) for b > 0 */
static int64_t floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

/* Border threshold lambda for a window centred on fine label gc.  Constant R (Eq. 11) unless
 * R_far > 0: then lambda moves linearly from R_far at the far end of the range (gc = 0, d = dmin)
 * to R at the near end (gc = G-1), rounded half up in exact integer arithmetic:
 *   lambda(gc) = R + floor((2 (R_far - R)(G-1-gc) + (G-1)) / (2 (G-1))).
 * The paper proposes a larger threshold for small disparities (Sec. IV-F) without a formula. */
int or_radius(const or_cfg *c, int64_t gc)
{
    if (c->R_far <= 0) return c->R;
    int64_t den = (int64_t)c->G - 1;
    int64_t num = ((int64_t)c->R_far - c->R) * (den - gc);
    return c->R + (int)floordiv(2 * num + den, 2 * den);
}

/* Borders (Eq. 11); `edge` (nullable): pixels excluded from the borders search the whole range;
 * in the boundary-less mode (Sec. IV-E) every pixel does. */
void or_windows(const or_cfg *c, size_t N, const double *dinit, const uint8_t *edge, int32_t *lo, int32_t *cnt)
{
    for (size_t p = 0; p < N; p++) {
        if (c->boundless || isnan(dinit[p]) || (edge && edge[p])) { lo[p] = 0; cnt[p] = c->G; continue; }
        int64_t m = (int64_t)(dinit[p] * 8.0);           /* exact: dinit is k/8 */
        int64_t num = m * (int64_t)(c->G - 1);
        int64_t den = 8 * (int64_t)(c->Lc - 1);
        int64_t gc = (2 * num + den) / (2 * den);
        int64_t R = or_radius(c, gc);
        int64_t a = gc - R, b = gc + R;
        if (a < 0) a = 0;
        if (b > c->G - 1) b = c->G - 1;
        lo[p] = (int32_t)a;
        cnt[p] = (int32_t)(b - a + 1);
    }
}

/* ----------------------------------------------- Fine cost volume (Eq. 12 + Eq. 15)
 * For every pixel p and fine label g in its window, over every view (u,v) except the
 * reference:
 *   S_l2 += || I_ref(p) - bilinear(I_uv, p + (u-uc, v-vc) * d_g) ||  (Eq. 6, Eq. 12:
 *           the Euclidean norm over the channels, sqrt(sum_ch delta_ch^2); for one
 *           channel it is written as the absolute value of the difference)
 *   S_c  += sum_ch HD(cen_ref,ch(p), cen_uv,ch(p + nearest shift))   (Eq. 4, Eq. 15;
 *           the channels' Hamming distances summed, Sec. III-B)
 *   C(p,g) = w_l2 * S_l2 + w_census * S_c.
 * Bilinear: (1-fy)[(1-fx) I(x0,y0) + fx I(x0+1,y0)] + fy[(1-fx) I(x0,y0+1) + fx I(x0+1,y0+1)]
 * with every tap index clamped.  Output: cost[off[p] + j] for slot j = g - lo[p]. */
void or_cost_volume(const or_cfg *c, const double *views, const uint64_t *cen,
                    const int32_t *lo, const int32_t *cnt, const int64_t *off, double *cost)
{
    size_t HW = (size_t)c->H * c->W;
    const int Ch = nchan(c);
    const double *Iref = views + ((size_t)c->vc * c->U + c->uc) * Ch * HW;
    const uint64_t *cref = cen + ((size_t)c->vc * c->U + c->uc) * Ch * HW;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < c->H; y++)
        for (int x = 0; x < c->W; x++) {
            size_t p = (size_t)y * c->W + x;
            for (int j = 0; j < cnt[p]; j++) {
                int g = lo[p] + j;
                double d = or_label_disp(c->dmin, c->dmax, c->G, g);
                double sl2 = 0.0, sc = 0.0;
                for (int v = 0; v < c->V; v++)
                    for (int u = 0; u < c->U; u++) {
                        if (u == c->uc && v == c->vc) continue;
                        int ox, oy, nx, ny;
                        double fx, fy;
                        or_shift(u - c->uc, d, &ox, &fx, &nx);
                        or_shift(v - c->vc, d, &oy, &fy, &ny);
                        int x0 = clampi(x + ox, 0, c->W - 1), x1 = clampi(x + ox + 1, 0, c->W - 1);
                        int y0 = clampi(y + oy, 0, c->H - 1), y1 = clampi(y + oy + 1, 0, c->H - 1);
                        int xn = clampi(x + nx, 0, c->W - 1), yn = clampi(y + ny, 0, c->H - 1);
                        double sq = 0.0;
                        for (int ch = 0; ch < Ch; ch++) {
                            const double *I = views + (((size_t)v * c->U + u) * Ch + ch) * HW;
                            double i00 = I[(size_t)y0 * c->W + x0], i10 = I[(size_t)y0 * c->W + x1];
                            double i01 = I[(size_t)y1 * c->W + x0], i11 = I[(size_t)y1 * c->W + x1];
                            double smp = (1.0 - fy) * ((1.0 - fx) * i00 + fx * i10)
                                       + fy * ((1.0 - fx) * i01 + fx * i11);
                            double delta = Iref[ch * HW + p] - smp;
                            if (Ch == 1) sl2 += fabs(delta);
                            else sq += delta * delta;
                            sc += (double)or_hamming(cref[ch * HW + p],
                                                     cen[(((size_t)v * c->U + u) * Ch + ch) * HW + (size_t)yn * c->W + xn]);
                        }
                        if (Ch > 1) sl2 += sqrt(sq);
                    }
                cost[off[p] + j] = c->w_l2 * sl2 + c->w_census * sc;
            }
        }
}

static void sgm_bounded_step(int H, int W, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                             const double *C, double P1, double P2, int dx, int dy, int x, int y,
                             int normalised, double *Lr)
{
    size_t p = (size_t)y * W + x;
    int qx = x - dx, qy = y - dy;
    if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
        for (int j = 0; j < cnt[p]; j++) Lr[off[p] + j] = C[off[p] + j];
        return;
    }
    size_t q = (size_t)qy * W + qx;
    const double *lp = Lr + off[q];
    double m = lp[0];
    for (int i = 1; i < cnt[q]; i++) if (lp[i] < m) m = lp[i];
    for (int j = 0; j < cnt[p]; j++) {
        int i = lo[p] + j - lo[q];          /* slot of the same label in q */
        double t = m + P2;
        if (i >= 0 && i < cnt[q] && lp[i] < t) t = lp[i];
        if (i - 1 >= 0 && i - 1 < cnt[q] && lp[i - 1] + P1 < t) t = lp[i - 1] + P1;
        if (i + 1 >= 0 && i + 1 < cnt[q] && lp[i + 1] + P1 < t) t = lp[i + 1] + P1;
        Lr[off[p] + j] = normalised ? C[off[p] + j] + (t - m) : C[off[p] + j] + t;
    }
}

/* ------------------------------------------- Bounded SGM (Sec. III-E, Eq. 8-9)
 * Eq. 8 on the windowed cost: terms that refer to labels outside the predecessor's
 * window are absent, and m is the minimum over the predecessor's window.
 * normalised = 1: L = C + (min(...) - m)   (the form used for the depth map)
 * normalised = 0: L = C + min(...)          (Eq. 8 as printed; used by the pins). */
void or_sgm_bounded_path(int H, int W, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                         const double *C, double P1, double P2, int dir, int normalised, double *Lr)
{
    int dx = DIRS[dir][0], dy = DIRS[dir][1];
    if (dy == 0) {
#pragma omp parallel for schedule(static)
        for (int iy = 0; iy < H; iy++)
            for (int ix = 0; ix < W; ix++)
                sgm_bounded_step(H, W, lo, cnt, off, C, P1, P2, dx, dy, order_x(ix, W, dx),
                                 order_y(iy, H, dy), normalised, Lr);
    } else {
        for (int iy = 0; iy < H; iy++) {
#pragma omp parallel for schedule(static)
            for (int ix = 0; ix < W; ix++)
                sgm_bounded_step(H, W, lo, cnt, off, C, P1, P2, dx, dy, order_x(ix, W, dx),
                                 order_y(iy, H, dy), normalised, Lr);
        }
    }
}

/* C_s = sum over the 8 or 16 directions (Eq. 9), added as a balanced tree
 * ((L0+L1)+(L2+L3)) + ((L4+L5)+(L6+L7)) per group of 8, and the two groups' sums added. */
void or_sgm_bounded(int H, int W, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                    const double *C, double P1, double P2, int paths, double *Cs)
{
    size_t N = (size_t)H * W;
    size_t nnz = (size_t)off[N];
    double *Lr[16];
    for (int r = 0; r < paths; r++) {
        Lr[r] = (double *)malloc(nnz * sizeof(double));
        or_sgm_bounded_path(H, W, lo, cnt, off, C, P1, P2, r, 1, Lr[r]);
    }
    for (size_t i = 0; i < nnz; i++) {
        double t = ((Lr[0][i] + Lr[1][i]) + (Lr[2][i] + Lr[3][i])) + ((Lr[4][i] + Lr[5][i]) + (Lr[6][i] + Lr[7][i]));
        if (paths == 16)
            t += ((Lr[8][i] + Lr[9][i]) + (Lr[10][i] + Lr[11][i])) + ((Lr[12][i] + Lr[13][i]) + (Lr[14][i] + Lr[15][i]));
        Cs[i] = t;
    }
    for (int r = 0; r < paths; r++) free(Lr[r]);
}

/* ----------------------------------- WTA (Eq. 10) and sub-pixel refinement (Eq. 13)
 * label = the fine label of the smallest C_s in the window (lowest label on ties);
 * gap = second smallest - smallest (+inf for a one-label window; a certificate of how
 * close the decision was).  Sub-pixel (mode 1): if the winner is strictly inside the
 * window, i.e. in [D_L+1, D_H-1], and that interval holds at least 3 labels (cnt >= 5),
 * the vertex of the parabola through the three costs around the winner is added:
 *   delta = (C(g-1) - C(g+1)) / (2 (C(g-1) - 2 C(g) + C(g+1)))
 * (Eq. 13 prints the denominator with the opposite sign, which would move the estimate
 * away from the lower neighbour; the vertex formula is the parabola's own); a
 * non-positive denominator gives delta = 0.  Mode 0: delta = 0.
 * Mode 2 (soft-argmin, not in the paper): disp = sum_g softmax(-C_s/tau)_g d_g.
 * disp is in pixels: dmin + (label + delta) * fine step. */
void or_wta_subpixel(const or_cfg *c, size_t N, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                     const double *Cs, int mode, double tau, int32_t *label, double *disp, double *gap)
{
    double step = (c->dmax - c->dmin) / (double)(c->G - 1);
    for (size_t p = 0; p < N; p++) {
        const double *s = Cs + off[p];
        int n = cnt[p];
        int b = 0;
        for (int j = 1; j < n; j++) if (s[j] < s[b]) b = j;
        double second = INFINITY;
        for (int j = 0; j < n; j++) if (j != b && s[j] < second) second = s[j];
        gap[p] = second - s[b];
        label[p] = lo[p] + b;
        if (mode == 2) {
            double num = 0.0, den = 0.0;
            for (int j = 0; j < n; j++) {
                double w = exp(-(s[j] - s[b]) / tau);
                num += w * (c->dmin + (double)(lo[p] + j) * step);
                den += w;
            }
            disp[p] = num / den;
            continue;
        }
        double delta = 0.0;
        if (mode == 1 && n >= 5 && b >= 1 && b <= n - 2) {
            double cm = s[b - 1], c0 = s[b], cp = s[b + 1];
            double den = cm - 2.0 * c0 + cp;
            if (den > 0.0) delta = (cm - cp) / (2.0 * den);
        }
        disp[p] = c->dmin + ((double)(lo[p] + b) + delta) * step;
    }
}

/* ------------------------------------------------ adjoint (not in the paper)
 * Gradients of Loss = sum_p gd(p) * dhat(p), dhat the soft-argmin of the aggregated cost,
 * with respect to the cost volume, P1, P2 and the view intensities. */

/* Soft-argmin: dhat = sum_j w_j d_j, w = softmax(-Cs/tau) over the window, so
 * d dhat / d Cs_j = -(1/tau) w_j (d_j - dhat). */
void or_softargmin_backward(const or_cfg *c, size_t N, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                            const double *Cs, const double *gd, double tau, double *gCs)
{
    double step = (c->dmax - c->dmin) / (double)(c->G - 1);
    for (size_t p = 0; p < N; p++) {
        const double *s = Cs + off[p];
        int n = cnt[p];
        double mn = s[0];
        for (int j = 1; j < n; j++) if (s[j] < mn) mn = s[j];
        double z = 0.0, num = 0.0;
        for (int j = 0; j < n; j++) {
            double w = exp(-(s[j] - mn) / tau);
            z += w;
            num += w * (c->dmin + (double)(lo[p] + j) * step);
        }
        double dh = num / z;
        for (int j = 0; j < n; j++) {
            double w = exp(-(s[j] - mn) / tau) / z;
            double d = c->dmin + (double)(lo[p] + j) * step;
            gCs[off[p] + j] = gd[p] * (-1.0 / tau) * w * (d - dh);
        }
    }
}

/* Adjoint of one direction of the bounded, normalised recurrence (Eq. 8):
 *   L(p,g) = C(p,g) + t(p,g) - m,  t = min over the branches {L'(g), L'(g-1)+P1, L'(g+1)+P1, m+P2},
 *   m = min L'.
 * The forward pass is recomputed recording the winning branch of every cell (ties: P2 first, then
 * same, g-1, g+1, as the minimum is taken in that order with strict comparisons) and the argmin
 * slot of every pixel; the reverse pass routes lambda = dLoss/dL along the winning branches, adds
 * -sum lambda (the -m term) plus the P2-branch lambdas to the predecessor's argmin slot, and sums
 * the branch lambdas into dP1 / dP2.  gLr: dLoss/dL_r (= dLoss/dC_s), gC accumulates dLoss/dC. */
void or_sgm_bounded_path_backward(int H, int W, const int32_t *lo, const int32_t *cnt, const int64_t *off,
                                  const double *C, double P1, double P2, int dir, const double *gLr,
                                  double *gC, double *gP1, double *gP2)
{
    int dx = DIRS[dir][0], dy = DIRS[dir][1];
    size_t N = (size_t)H * W, nnz = (size_t)off[N];
    double *L = (double *)malloc(nnz * sizeof(double));
    unsigned char *code = (unsigned char *)malloc(nnz);
    int32_t *amin = (int32_t *)malloc(N * sizeof(int32_t));
    double *inc = (double *)calloc(nnz, sizeof(double));
    /* forward, in the visiting order of or_sgm_bounded_path */
    for (int iy = 0; iy < H; iy++)
        for (int ix = 0; ix < W; ix++) {
            int y = order_y(iy, H, dy), x = order_x(ix, W, dx);
            size_t p = (size_t)y * W + x;
            int qx = x - dx, qy = y - dy;
            if (qx < 0 || qx >= W || qy < 0 || qy >= H) {
                for (int j = 0; j < cnt[p]; j++) { L[off[p] + j] = C[off[p] + j]; code[off[p] + j] = 4; }
            } else {
                size_t q = (size_t)qy * W + qx;
                const double *lp = L + off[q];
                double m = lp[amin[q]];
                for (int j = 0; j < cnt[p]; j++) {
                    int i = lo[p] + j - lo[q];
                    double t = m + P2;
                    unsigned char cd = 3;
                    if (i >= 0 && i < cnt[q] && lp[i] < t) { t = lp[i]; cd = 0; }
                    if (i - 1 >= 0 && i - 1 < cnt[q] && lp[i - 1] + P1 < t) { t = lp[i - 1] + P1; cd = 1; }
                    if (i + 1 >= 0 && i + 1 < cnt[q] && lp[i + 1] + P1 < t) { t = lp[i + 1] + P1; cd = 2; }
                    L[off[p] + j] = C[off[p] + j] + (t - m);
                    code[off[p] + j] = cd;
                }
            }
            int b = 0;
            for (int j = 1; j < cnt[p]; j++) if (L[off[p] + j] < L[off[p] + b]) b = j;
            amin[p] = b;
        }
    /* reverse: successors before predecessors */
    for (int iy = H - 1; iy >= 0; iy--)
        for (int ix = W - 1; ix >= 0; ix--) {
            int y = order_y(iy, H, dy), x = order_x(ix, W, dx);
            size_t p = (size_t)y * W + x;
            int qx = x - dx, qy = y - dy;
            int has_q = !(qx < 0 || qx >= W || qy < 0 || qy >= H);
            size_t q = has_q ? (size_t)qy * W + qx : 0;
            double dm = 0.0;
            for (int j = 0; j < cnt[p]; j++) {
                double lam = gLr[off[p] + j] + inc[off[p] + j];
                gC[off[p] + j] += lam;
                if (!has_q) continue;
                int i = lo[p] + j - lo[q];
                switch (code[off[p] + j]) {
                case 0: inc[off[q] + i] += lam; break;
                case 1: inc[off[q] + i - 1] += lam; *gP1 += lam; break;
                case 2: inc[off[q] + i + 1] += lam; *gP1 += lam; break;
                default: dm += lam; *gP2 += lam; break;
                }
                dm -= lam;
            }
            if (has_q) inc[off[q] + amin[q]] += dm;
        }
    free(L);
    free(code);
    free(amin);
    free(inc);
}

/* Adjoint of the cost volume w.r.t. the views through the l2 term (Eq. 6, Eq. 12):
 *   d C / d I_ref,ch(p) = w_l2 sum_v e_ch,  d C / d I_v,ch(tap) = -w_l2 e_ch w_tap,
 * with e = delta / ||delta|| the unit colour difference (delta = I_ref(p) - B_v over the
 * channels; e = 0 where delta = 0), which for one channel is sign(delta); taps clamped as in
 * the forward; the census term is piecewise constant (no gradient). */
void or_cost_backward_views(const or_cfg *c, const double *views, const int32_t *lo, const int32_t *cnt,
                            const int64_t *off, const double *gcost, double *gviews)
{
    size_t HW = (size_t)c->H * c->W;
    const int Ch = nchan(c);
    const double *Iref = views + ((size_t)c->vc * c->U + c->uc) * Ch * HW;
    double *gref = gviews + ((size_t)c->vc * c->U + c->uc) * Ch * HW;
    for (int y = 0; y < c->H; y++)
        for (int x = 0; x < c->W; x++) {
            size_t p = (size_t)y * c->W + x;
            for (int j = 0; j < cnt[p]; j++) {
                double gcv = gcost[off[p] + j];
                if (gcv == 0.0) continue;
                double d = or_label_disp(c->dmin, c->dmax, c->G, lo[p] + j);
                for (int v = 0; v < c->V; v++)
                    for (int u = 0; u < c->U; u++) {
                        if (u == c->uc && v == c->vc) continue;
                        int ox, oy, nx, ny;
                        double fx, fy;
                        or_shift(u - c->uc, d, &ox, &fx, &nx);
                        or_shift(v - c->vc, d, &oy, &fy, &ny);
                        int x0 = clampi(x + ox, 0, c->W - 1), x1 = clampi(x + ox + 1, 0, c->W - 1);
                        int y0 = clampi(y + oy, 0, c->H - 1), y1 = clampi(y + oy + 1, 0, c->H - 1);
                        double delta[4] = {0.0, 0.0, 0.0, 0.0}, sq = 0.0;
                        for (int ch = 0; ch < Ch; ch++) {
                            const double *I = views + (((size_t)v * c->U + u) * Ch + ch) * HW;
                            double smp = (1.0 - fy) * ((1.0 - fx) * I[(size_t)y0 * c->W + x0] + fx * I[(size_t)y0 * c->W + x1])
                                       + fy * ((1.0 - fx) * I[(size_t)y1 * c->W + x0] + fx * I[(size_t)y1 * c->W + x1]);
                            delta[ch] = Iref[ch * HW + p] - smp;
                            sq += delta[ch] * delta[ch];
                        }
                        double norm = sqrt(sq);
                        for (int ch = 0; ch < Ch; ch++) {
                            double e;
                            if (Ch == 1) e = delta[0] > 0.0 ? 1.0 : (delta[0] < 0.0 ? -1.0 : 0.0);
                            else e = norm > 0.0 ? delta[ch] / norm : 0.0;
                            double g = gcv * c->w_l2 * e;
                            double *gI = gviews + (((size_t)v * c->U + u) * Ch + ch) * HW;
                            gref[ch * HW + p] += g;
                            gI[(size_t)y0 * c->W + x0] -= g * (1.0 - fy) * (1.0 - fx);
                            gI[(size_t)y0 * c->W + x1] -= g * (1.0 - fy) * fx;
                            gI[(size_t)y1 * c->W + x0] -= g * fy * (1.0 - fx);
                            gI[(size_t)y1 * c->W + x1] -= g * fy * fx;
                        }
                    }
            }
        }
}

/* Threads of the parallel row loops (the results do not depend on it); returns the count in use. */
int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Post-processing (Sec. III-F, window size 3 from Sec. IV-C): 3 x 3 median of the sub-pixel
 * disparity map.  Reading: the window is clamped to the image (border pixels repeat), so every
 * output is the 5th smallest of 9 values. */
void or_median3(int H, int W, const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double v[9];
            int n = 0;
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const int yy = clampi(y + dy, 0, H - 1), xx = clampi(x + dx, 0, W - 1);
                    double q = in[(size_t)yy * W + xx];
                    int j = n++;
                    while (j > 0 && v[j - 1] > q) { v[j] = v[j - 1]; j--; }
                    v[j] = q;
                }
            out[(size_t)y * W + x] = v[4];
        }
}
