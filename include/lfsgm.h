/*
 * lfsgm.h -- C ABI of the GB300 light-field depth library (semi-global matching on
 * a bounded light-field cost volume), after Anisimov, Wasenmueller and Stricker,
 * "Rapid Light Field Depth Estimation with Semi-Global Matching", ICCP 2019.
 *
 * Plain C: pointers and sizes only.  Every array argument is a DEVICE pointer owned
 * by the caller unless its comment says "host".  Calls are asynchronous on the
 * stream given to lfsgm_create, except where a comment says they synchronise.
 * Argument errors are returned at once; errors detected inside kernels are latched
 * in a device status word and returned by lfsgm_sync.  Nothing traps or aborts.
 *
 * Notation.  views[v][u][c][y][x] float32, contiguous: (x,y) spatial position in a view
 * (the paper's (u,v)), (u,v) angular position of the view (the paper's (s,t)), c the colour
 * channel (cfg.channels = C: 1 grey, then views[v][u][y][x]; or 3 RGB), reference view
 * (uc,vc).  A view (u,v) is sampled for pixel (x,y) and disparity d at
 *     (x + (u-uc) d, y + (v-vc) d)                      (Sec. III-A, Eq. 1)
 * (the paper writes (s^-s) d: our d has the opposite sign, larger d = nearer).
 * Labels: coarse k in [0,Lc) and fine g in [0,G) on inclusive grids over [dmin,dmax]:
 *     d_k = dmin + k*((dmax-dmin)/(Lc-1)),   d_g = dmin + g*((dmax-dmin)/(G-1)).
 * Shift split (the paper is silent): s = a*d in double; when 2s is within 2e-9 of an
 * integer, s is snapped to that half-integer; ox = floor(s), fx = s-ox (bilinear
 * taps), nx = floor(s+0.5) (census position).  Tap indices are clamped to the image.
 *
 * Windowed cost layout ("CSR", part of this ABI): pixel p = y*W + x has the fine
 * labels lo[p] .. lo[p]+cnt[p]-1; slot j of pixel p is at cost[off[p] + j].
 * off[p] is a multiple of 4 for every p in [0, N], off[N] included (16-byte aligned rows
 * whose lengths are whole 4-slot groups), and off[p+1] - off[p] >= cnt[p]; the padding
 * slots are written with 0 and never read.  off has N+1 entries.  A kernel that meets a
 * row breaking these rules skips that pixel and latches LFSGM_ERR_DEVICE_CHECK.
 * Rows are read and written as 16-byte vectors, so the cost, agg and grad_cost buffers
 * must start on a 16-byte boundary (LFSGM_ERR_INVALID_ARG otherwise, before any launch).
 */
#ifndef LFSGM_H
#define LFSGM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LFSGM_OK = 0,
    LFSGM_ERR_INVALID_ARG = 1,   /* bad config value, null pointer, P2 < P1, ...        */
    LFSGM_ERR_NO_MEMORY = 2,     /* device allocation failed                            */
    LFSGM_ERR_WORKSPACE = 3,     /* caller workspace too small or misaligned            */
    LFSGM_ERR_CUDA = 4,          /* a CUDA runtime call failed (see lfsgm_last_error)   */
    LFSGM_ERR_UNSUPPORTED = 5,   /* sizes outside what the kernels support              */
    LFSGM_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up                  */
    LFSGM_ERR_DEVICE_CHECK = 7   /* a kernel-side consistency check failed              */
} lfsgm_status;

typedef struct lfsgm_ctx *lfsgm_handle;

/* Method parameters.  The paper's values (Sec. IV "Algorithm parameters") are phi = 3,
 * lambda = 2, median window 3, P1/P2 = 21/45 and 17/35; the synthetic workloads use
 * penalties proportional to the mean cost instead (p1_frac, p2_frac). */
typedef struct {
    int32_t U, V, H, W;        /* angular (U x V views) and spatial (H x W) sizes          */
    int32_t uc, vc;            /* reference view; -1 -> (U-1)/2, (V-1)/2                    */
    int32_t census_w;          /* census window side: 5 (24 bits) or 7 (48 bits)           */
    double  dmin, dmax;        /* disparity range T (Sec. III-D), px per angular step       */
    int32_t coarse_labels;     /* Lc, 2..256                                                */
    int32_t init_views;        /* 1: whole cross arms; 0: the paper's 4 extreme views       */
    double  phi;               /* fusion threshold in coarse labels (Sec. III-D)            */
    int32_t fill_passes;       /* median hole-filling passes, 0..4 (Sec. III-D: 1 or 2)     */
    int32_t fine_labels;       /* G, 2..4096                                                */
    int32_t fine_radius;       /* R: window = nearest fine label to D_init +- R (Eq. 11)    */
    float   w_l2;              /* weight of the l2 term (Eq. 12)                             */
    float   w_census;          /* weight of the census term (Eq. 15)                         */
    double  p1_frac, p2_frac;  /* derived penalties: P = frac * mean cost                   */
    int32_t subpixel;          /* 0 none, 1 parabola (Eq. 13), 2 soft-argmin                */
    float   softmin_tau;       /* soft-argmin temperature                                   */
    int32_t paths;             /* SGM directions: 8, or the paper's 16 (Sec. IV-C) adding the
                                  slopes 1/2 and 2; 0 is read as 8                            */
    float   edge_threshold;    /* Sobel edge exclusion from the borders (Sec. III-D): pixels of
                                  the reference view with gx^2 + gy^2 > t^2 (FP32, 3 x 3 Sobel,
                                  clamped) search the whole range; 0 = off.  Colour: a pixel is
                                  an edge when it is one in any channel                       */
    int32_t channels;          /* colour channels C: 1 (grey) or 3 (RGB, Sec. III-B/C: census per
                                  channel with the Hamming distances summed, l2 the Euclidean
                                  norm of the colour difference); 0 is read as 1              */
    int32_t boundless;         /* 1: boundary-less search (Sec. IV-E): no initial map, every
                                  window is the whole range T; 0: bounded (Eq. 11)            */
    int32_t fine_radius_far;   /* > 0: depth-dependent border threshold (Sec. IV-F proposes a
                                  larger one for small disparities): lambda moves linearly from
                                  fine_radius_far at d = dmin to fine_radius at d = dmax,
                                  lambda(gc) = R + floor((2 (Rfar-R)(G-1-gc) + G-1) / (2 (G-1)))
                                  for the window centre gc; <= 0: constant fine_radius         */
} lfsgm_config;

/* Create a handle for one light-field shape.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream).  Builds the shift tables in double precision on the host
 * and uploads them.  Returns LFSGM_ERR_INVALID_ARG for an inconsistent config. */
lfsgm_status lfsgm_create(const lfsgm_config *cfg, void *stream, lfsgm_handle *out);
lfsgm_status lfsgm_destroy(lfsgm_handle h);

/* Scratch the handle needs (census words, coarse volume and sums, maps, partial sums).
 * Without lfsgm_set_workspace the handle allocates it itself on first use; with it, the
 * caller's buffer (device, 256-byte aligned, >= *bytes) is used and never freed here. */
lfsgm_status lfsgm_workspace_size(lfsgm_handle h, size_t *bytes);
lfsgm_status lfsgm_set_workspace(lfsgm_handle h, void *dptr, size_t bytes);

/* Speed knobs (not in the paper): the label span of the row cost kernel's ranges (row_kw 36 or
 * 44; 0 = 36; colour light fields run span 36 only, and with 44 send every window to the list
 * kernel), and the CTAs per SM of the (pixel, chunk) list kernel (list_ctas_per_sm 1..64; 0 = the
 * default: the CTAs resident at once, one wave; grey light fields run a 32-register form of the
 * kernel for the default and 16 or more, a 40-register one below 16).  A wider span sends fewer
 * windows to the list kernel and computes more labels per row.  Changing the span rebuilds the
 * row descriptors on the host
 * and synchronises the handle's stream; results change only in the last bits (a window moves
 * between the row and the list kernel, which add the views in different FP32 orders).  The
 * batch autotuner sets these per shape class.  Errors: LFSGM_ERR_INVALID_ARG for other values. */
lfsgm_status lfsgm_set_tuning(lfsgm_handle h, int32_t row_kw, int32_t list_ctas_per_sm);

/* Speed knob of the fine SGM (not in the paper): the warps, one scanline each, of a CTA of the
 * bounded SGM kernel, 2, 4 or 8 (0 = 4).  The aggregate is the same bit for bit for every value
 * (the direction sum is order-independent); only the time changes, with the light field's shape
 * (the bench light field runs best with 8, whole-range Middlebury-shaped windows with 4).
 * lfsgm_get_tuning reads the handle's three knobs (NULL outputs are skipped).  lfsgm_autotune
 * also picks this one, after the cost knobs, by timing lfsgm_sgm_aggregate with derived
 * penalties.  Errors: LFSGM_ERR_INVALID_ARG for other values. */
lfsgm_status lfsgm_set_sgm_warps(lfsgm_handle h, int32_t warps_per_cta);
lfsgm_status lfsgm_get_tuning(lfsgm_handle h, int32_t *row_kw, int32_t *list_ctas_per_sm,
                              int32_t *sgm_warps);

/* Speed knob of the fine SGM (not in the paper): a scanline that crosses at least min_wide
 * windows wider than 32 labels (0 = none, the default; lfsgm_autotune tries 24) runs on all the
 * warps of one CTA, which share each wide step's 32-label chunks, instead of on one warp.  Such
 * scanlines (along image borders, where the initial pass leaves whole-range windows) otherwise
 * outlast all others; the CTA's other warps wait while its first runs the narrow steps, so the
 * split pays only where a few scanlines are much longer than the rest.  Each
 * lfsgm_sgm_aggregate then first lists them (one small kernel after zeroing agg); when more than
 * 256 qualify (most windows wide), none is split.  The aggregate is the same bit for bit with any
 * value.  lfsgm_get_sgm_split reads it back.  Errors: LFSGM_ERR_INVALID_ARG for a negative value. */
lfsgm_status lfsgm_set_sgm_split(lfsgm_handle h, int32_t min_wide);
lfsgm_status lfsgm_get_sgm_split(lfsgm_handle h, int32_t *min_wide);

/* Picks the speed knobs for this handle's shape on a representative light field (views: device,
 * as for lfsgm_depth): one initial pass, then the cost stage is timed with the row kernel's label
 * span 36 and 44 and, with the better one, with the list kernel's CTAs per SM 8, 12 and 24
 * against the default; the fastest setting is kept (lfsgm_set_tuning) and returned in row_kw and
 * list_ctas_per_sm (host, nullable).  Then lfsgm_sgm_aggregate (derived penalties) is timed with
 * 4, 8 and 2 SGM warps per CTA, each with the split off and at threshold 24 (lfsgm_set_sgm_split), and
 * the fastest pair kept (lfsgm_set_sgm_warps; read the warps back with lfsgm_get_tuning).
 * Synchronous; uses the buffers of lfsgm_depth. */
lfsgm_status lfsgm_autotune(lfsgm_handle h, const float *views, int32_t *row_kw, int32_t *list_ctas_per_sm);

/* Upper bound of off[N] for this config (every pixel with a whole-range window). */
lfsgm_status lfsgm_max_nnz(lfsgm_handle h, int64_t *nnz);

/* Initial disparity map and fine search windows (Sec. III-D, Eq. 7-11):
 * census of the cross views (Eq. 2-3), per-arm census cost over the coarse labels
 * (Eq. 7 summed over the arm's views), integer SGM per arm over cfg.paths paths (Eq. 8-9),
 * WTA per arm (Eq. 10), sequential fusion with threshold phi, median hole filling,
 * borders D_init +- lambda saturated to T (Eq. 11; discarded pixels: whole range).
 * Boundary-less mode (cfg.boundless): only the windows are written (lo = 0, cnt = G), dinit is
 * NaN everywhere and maps is left untouched; no census or coarse work is done.
 *   views  [V][U][C][H][W] float32
 *   Pc1, Pc2  integer coarse penalties; Pc1 <= 0 -> per arm round(p*_frac * mean arm
 *             cost) with P1 >= 1, P2 >= P1.
 *   lo, cnt   [H*W] int32 out: window first fine label and label count
 *   off       [H*W+1] int64 out: padded row offsets (see layout above)
 *   dinit     [H*W] float32 out (nullable): fused, filled map in coarse-label units
 *             (multiples of 1/8), NaN where discarded
 *   maps      [4][H*W] int32 out (nullable): per-arm WTA labels (up, down, left, right;
 *             empty arms are skipped, so only the first n_arms rows are written)
 *   nnz_host  host int64 out (nullable): off[N]; when given the call synchronises. */
lfsgm_status lfsgm_initial_disparity(lfsgm_handle h, const float *views, int32_t Pc1, int32_t Pc2,
                                     int32_t *lo, int32_t *cnt, int64_t *off, float *dinit,
                                     int32_t *maps, int64_t *nnz_host);

/* Bounded fine cost volume (Sec. III-E, Eq. 12 and Eq. 15) over every view but the
 * reference, for the labels of each pixel's window:
 *   C(p,g) = w_l2 * sum || I_ref(p) - bilinear(I_uv, p + (u-uc, v-vc) d_g) ||
 *          + w_census * sum sum_c HD(census_ref,c(p), census_uv,c(p + nearest shift)),
 * the norm over the C channels (for C = 1 the absolute difference).
 *   views [V][U][C][H][W] float32; lo, cnt, off as produced above; cost [off[N]] float32 out. */
lfsgm_status lfsgm_cost_volume(lfsgm_handle h, const float *views, const int32_t *lo,
                               const int32_t *cnt, const int64_t *off, float *cost);

/* Bounded SGM over cfg.paths (8 or 16) paths (Sec. III-E with Eq. 8-9), normalised recurrence
 *   L_r(p,g) = C(p,g) + (min(L'(g), L'(g-1)+P1, L'(g+1)+P1, m+P2) - m),
 * L' = L_r(p-r,.) over the predecessor's window, m its minimum, absent labels left out,
 * L_r = C at path starts; agg = sum over the directions.  P1 < 0 -> P1 = p1_frac *
 * mean(cost over active slots), P2 = p2_frac * mean (computed on the device).
 * Requires 0 <= P1 <= P2 otherwise.  agg [off[N]] float32 out. */
lfsgm_status lfsgm_sgm_aggregate(lfsgm_handle h, const float *cost, const int32_t *lo,
                                 const int32_t *cnt, const int64_t *off, float P1, float P2,
                                 float *agg);

/* Winner-takes-all (Eq. 10, lowest label on ties) and sub-pixel refinement:
 * mode 1 parabola vertex (Eq. 13 with the vertex's sign) when the winner lies in
 * [lo+1, lo+cnt-2] and cnt >= 5; mode 2 soft-argmin sum softmax(-agg/tau) d_g.
 *   label [H*W] int32 out (fine label), disp [H*W] float32 out (pixels). */
lfsgm_status lfsgm_wta_subpixel(lfsgm_handle h, const float *agg, const int32_t *lo,
                                const int32_t *cnt, const int64_t *off, int32_t *label, float *disp);

/* Post-processing median filter (Sec. III-F; window size 3, Sec. IV-C): out(p) = median of the
 * 3 x 3 neighbourhood of p in disp, the window clamped to the image (border values repeat), i.e.
 * the 5th smallest of 9 values.  disp, out: [H*W] float32, device, distinct buffers.  NaN inputs
 * (invalid windows) give an unspecified selection.  Asynchronous on the handle's stream. */
lfsgm_status lfsgm_median_filter(lfsgm_handle h, const float *disp, float *out);

/* Adjoint of cost volume -> SGM -> soft-argmin (not in the paper).  Given grad_disp
 * = dLoss/d disp of the soft-argmin output, returns dLoss/d cost (grad_cost, CSR like
 * cost), dLoss/dP1 and dLoss/dP2 (device scalars) and dLoss/d views through the l2 term
 * and its bilinear weights (grad_views [V][U][C][H][W]; the census term has no gradient; for C > 1
 * the l2 term's gradient is w_l2 times the unit colour difference, 0 where the colours agree).
 * Path costs are recomputed per direction; subgradients follow the recorded argmin.
 * grad_views may be NULL (then only grad_cost and the penalty gradients are formed). */
lfsgm_status lfsgm_backward(lfsgm_handle h, const float *views, const float *cost,
                            const int32_t *lo, const int32_t *cnt, const int64_t *off,
                            float P1, float P2, const float *grad_disp, float *grad_cost,
                            float *grad_P1, float *grad_P2, float *grad_views);

/* Training form of the two calls above (not in the paper): lfsgm_sgm_aggregate_record is
 * lfsgm_sgm_aggregate on explicit penalties 0 <= P1 <= P2 (agg bit-identical to it) that also
 * records, in the handle's backward scratch, each cell's winning branch of Eq. 9 and each pixel's
 * argmin slot per direction; lfsgm_backward_recorded is lfsgm_backward on that record and on the
 * recorded aggregate, so the SGM is not run again.  The record is the handle's last one: it
 * belongs to the cost, agg, lo, cnt and off pointers and the penalties of the recording call, and
 * lfsgm_backward_recorded returns LFSGM_ERR_INVALID_ARG (nothing launched) when any of them
 * differs, or when another lfsgm_sgm_aggregate_record or lfsgm_backward has run on the handle
 * since.  The caller keeps those buffers unchanged in between (the handle checks the pointers,
 * not the contents).  Asynchronous on the handle's stream; the backward scratch is allocated on
 * first use, as by lfsgm_backward. */
lfsgm_status lfsgm_sgm_aggregate_record(lfsgm_handle h, const float *cost, const int32_t *lo,
                                        const int32_t *cnt, const int64_t *off, float P1, float P2,
                                        float *agg);
lfsgm_status lfsgm_backward_recorded(lfsgm_handle h, const float *views, const float *cost,
                                     const float *agg, const int32_t *lo, const int32_t *cnt,
                                     const int64_t *off, float P1, float P2,
                                     const float *grad_disp, float *grad_cost, float *grad_P1,
                                     float *grad_P2, float *grad_views);

/* Waits for the handle's stream and returns the latched device status (then clears it). */
lfsgm_status lfsgm_sync(lfsgm_handle h);

/* Human-readable text of the last error on this handle (static storage of the handle). */
const char *lfsgm_last_error(lfsgm_handle h);

/* Kernel launches issued through this handle since creation (for accounting). */
int64_t lfsgm_launch_count(lfsgm_handle h);

/* Per-kernel timing: with `enable` != 0 every launch is bracketed by CUDA events on the
 * handle's stream.  lfsgm_kernel_times fills up to `cap` (name, milliseconds) records of
 * the launches since the last call (names are static strings); synchronises. */
lfsgm_status lfsgm_set_profiling(lfsgm_handle h, int32_t enable);
lfsgm_status lfsgm_kernel_times(lfsgm_handle h, const char **names, float *ms, int32_t cap,
                                int32_t *n_out);

/* Whole method from HOST memory (end-to-end form): copies the views host->device,
 * runs initial disparity, cost volume, SGM (derived penalties) and WTA/sub-pixel,
 * copies disp (and label when non-NULL) device->host, and synchronises.  Device
 * buffers are owned by the handle and allocated on first use.
 *   views_host [V][U][C][H][W] float32 (pinned memory gives full copy speed)
 *   disp_host [H*W] float32, label_host [H*W] int32 (nullable). */
lfsgm_status lfsgm_depth_host(lfsgm_handle h, const float *views_host, float *disp_host,
                              int32_t *label_host);

/* Whole method on device buffers owned by the handle (views stay caller-owned):
 * the same chain as lfsgm_depth_host without the copies. disp, label: device, nullable. */
lfsgm_status lfsgm_depth(lfsgm_handle h, const float *views, float *disp, int32_t *label);

/* Batches (not in the paper): n light fields of mixed shape run as ONE CUDA-graph launch.
 * Each light field i has its own configuration cfgs[i], views[i] ([V][U][C][H][W] float32, device)
 * and output disp[i] ([H*W] float32, device); the pointers are baked into the graph at creation.
 * The pipeline of lfsgm_depth (derived penalties) runs for every light field; light fields are
 * spread over `branches` concurrent streams forked from `stream` (balanced by longest work first;
 * each branch then runs its light fields shortest first), branches
 * <= 0 lets an autotuner pick the speed knobs per shape class (lfsgm_batch_knobs), then time K in
 * {1,2,4,8,16} and keep the fastest.  Scratch is allocated at
 * creation (per branch, sized for its largest member).  lfsgm_batch_run enqueues one graph launch;
 * lfsgm_batch_times synchronises and returns, per light field, the start and end of its pipeline
 * in ms after the batch started (%globaltimer stamps inside the graph), and the branch count.
 * The light fields of one branch share one device status word (offset 0 of the branch's
 * workspace): a device-side check that fails in any of them is reported by lfsgm_batch_times
 * and stays latched for later runs of the batch. */
typedef struct lfsgm_batch_ctx *lfsgm_batch;
lfsgm_status lfsgm_batch_create(int32_t n, const lfsgm_config *cfgs, const float *const *views,
                                float *const *disp, void *stream, int32_t branches, lfsgm_batch *out);
lfsgm_status lfsgm_batch_run(lfsgm_batch b);
lfsgm_status lfsgm_batch_times(lfsgm_batch b, double *start_ms, double *end_ms, int32_t *branches);
/* The speed knobs (see lfsgm_set_tuning, lfsgm_set_sgm_warps, lfsgm_set_sgm_split) each light
 * field of the batch runs with: the autotuner (branches <= 0 at creation) tunes one member of each
 * shape class as lfsgm_autotune does and sets its knobs on every member.  row_kw,
 * list_ctas_per_sm, warps_per_cta, min_wide: host int32 [n] (nullable in lfsgm_batch_knobs). */
lfsgm_status lfsgm_batch_knobs(lfsgm_batch b, int32_t *row_kw, int32_t *list_ctas_per_sm);
lfsgm_status lfsgm_batch_sgm_warps(lfsgm_batch b, int32_t *warps_per_cta);
lfsgm_status lfsgm_batch_sgm_split(lfsgm_batch b, int32_t *min_wide);
int64_t lfsgm_batch_kernel_nodes(lfsgm_batch b);    /* kernel nodes in the batch's graph */
const char *lfsgm_batch_last_error(lfsgm_batch b);  /* NULL: error of the last failed create */
lfsgm_status lfsgm_batch_destroy(lfsgm_batch b);

/* A batch whose scratch lives in caller memory (not in the paper): for a serving process that
 * keeps its device memory in its own pool.  lfsgm_batch_workspace_size returns, from the
 * configurations alone (no device work), the bytes a batch of these light fields needs with
 * `branches` branches (branches <= 0: the most any autotuned branch count needs).
 * lfsgm_batch_create_ws is lfsgm_batch_create with that scratch taken from ws (device memory,
 * 256-byte aligned, ws_bytes long, caller-owned, valid until lfsgm_batch_destroy): the branches'
 * workspaces, window maps, labels, cost volumes and aggregates, and the timing stamps.  With
 * branches <= 0 the autotuner tries only the branch counts whose scratch fits ws_bytes.  The
 * per-light-field tables (shift tables, row descriptors) stay library-owned, as for a handle given
 * a workspace with lfsgm_set_workspace.  Errors: LFSGM_ERR_WORKSPACE if ws is misaligned or
 * too small (lfsgm_batch_last_error(NULL) gives the size needed), otherwise as lfsgm_batch_create. */
lfsgm_status lfsgm_batch_workspace_size(int32_t n, const lfsgm_config *cfgs, int32_t branches, size_t *bytes);
lfsgm_status lfsgm_batch_create_ws(int32_t n, const lfsgm_config *cfgs, const float *const *views,
                                   float *const *disp, void *stream, int32_t branches, void *ws, size_t ws_bytes,
                                   lfsgm_batch *out);

/* The bounded cost volume (same result as lfsgm_cost_volume) for callers that may not
 * allocate device memory.  The paper has no counterpart: this is a deployment variant.
 * Real-time loops and plug-ins that live inside a host application's own memory pool run
 * under a fixed device-memory budget and must not call cudaMalloc while running (it can
 * block, fail under memory pressure, or bypass the host's accounting); they cannot create
 * a handle, which allocates.  This entry point takes the configuration directly and
 * allocates nothing: its scratch (shift table, census words of every view, status word)
 * is one static device array of 32 MiB that every GPU loading this library holds until
 * the process exits.  It serves light fields with
 *     256 + round256(4 U V) + round256(16 U V G) + 8 U V H W <= 32 MiB
 * (e.g. 5x5 views of 64x64 .. 256x256) and returns LFSGM_ERR_UNSUPPORTED beyond that and
 * for colour light fields (channels > 1).
 * The first call on each device resolves the array's device address (cudaGetSymbolAddress,
 * with that device current): make that first call before any stream capture.  All calls
 * share the array, so calls that overlap on the GPU (two streams, or two host threads at
 * once) race; the status word is cleared at the start of every call and windows that break
 * the layout rules are skipped (their slots are left unwritten).
 *   cfg: as for lfsgm_create; stream: cudaStream_t; the rest as for lfsgm_cost_volume. */
lfsgm_status lfsgm_cost_volume_noalloc(const lfsgm_config *cfg, void *stream, const float *views,
                                       const int32_t *lo, const int32_t *cnt, const int64_t *off,
                                       float *cost);

#ifdef __cplusplus
}
#endif
#endif /* LFSGM_H */
