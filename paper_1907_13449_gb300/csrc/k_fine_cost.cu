// k_fine_cost.cu -- bounded fine cost volume (Sec. III-E, Eq. 12 with the census term of
// Eq. 15):
//   C(p,g) = w_l2 * sum_views |I_ref(p) - bilinear(I_uv, p + (u-uc, v-vc) d_g)|
//          + w_c  * sum_views HD(census_ref(p), census_uv(p + nearest shift)),
// over every view but the reference, for the labels g of p's window only.
//
// Generic form: one warp per pixel, lane j owns window slot j (label lo + j; wide windows
// loop in chunks of 32), and walks the views in the order v-major, u-minor.  The shift
// split of every (view, label) comes from the host-built FineTap table; taps and census
// words are read through the read-only cache.  Output rows are written coalesced,
// padding slots with 0.
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

__global__ void __launch_bounds__(256) fine_cost_generic(const float *__restrict__ views,
                                                         const uint64_t *__restrict__ cen,
                                                         const FineTap *__restrict__ tab, int G,
                                                         int nviews, int H, int W, int ref,
                                                         const int *__restrict__ lo,
                                                         const int *__restrict__ cnt,
                                                         const long long *__restrict__ off, float wl2,
                                                         float wc, float *__restrict__ cost,
                                                         int *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const size_t N = (size_t)H * W;
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < (int)N; p += warps) {
        const int x = p % W, y = p / W;
        const int l0 = __ldg(lo + p), n = __ldg(cnt + p);
        const long long o = __ldg(off + p), row = __ldg(off + p + 1) - o;
        if (!window_ok(l0, n, G, row, status)) continue;
        const float Iref = __ldg(views + (size_t)ref * N + p);
        const uint64_t cr = __ldg(cen + (size_t)ref * N + p);
        const int npad = (int)min((long long)((n + 3) & ~3), row);
        for (int j = lane; j < npad; j += 32) {
            float acc = 0.f;
            if (j < n) {
                const int g = l0 + j;
                float sl2 = 0.f;
                int sc = 0;
                for (int view = 0; view < nviews; view++) {
                    if (view == ref) continue;
                    const FineTap t = load_tap(tab + (size_t)view * G + g);
                    const float *I = views + (size_t)view * N;
                    const int x0 = min(max(x + t.ox, 0), W - 1), x1 = min(max(x + t.ox + 1, 0), W - 1);
                    const int y0 = min(max(y + t.oy, 0), H - 1), y1 = min(max(y + t.oy + 1, 0), H - 1);
                    const float i00 = __ldg(I + (size_t)y0 * W + x0), i10 = __ldg(I + (size_t)y0 * W + x1);
                    const float i01 = __ldg(I + (size_t)y1 * W + x0), i11 = __ldg(I + (size_t)y1 * W + x1);
                    const float top = (1.f - t.fx) * i00 + t.fx * i10;
                    const float bot = (1.f - t.fx) * i01 + t.fx * i11;
                    const float smp = (1.f - t.fy) * top + t.fy * bot;
                    sl2 += fabsf(Iref - smp);
                    const int xn = min(max(x + t.nx, 0), W - 1), yn = min(max(y + t.ny, 0), H - 1);
                    sc += __popcll(cr ^ __ldg(cen + (size_t)view * N + (size_t)yn * W + xn));
                }
                acc = wl2 * sl2 + wc * (float)sc;
            }
            cost[o + j] = acc;
        }
    }
}


// ---------------------------------------------------------------------------------------
// Row form for the regular (narrow) windows.
//
// For a fixed view and fine label the shift (u-uc, v-vc) d_g is the same for every pixel, so
// a warp that owns a row segment of 32 pixels sweeps one label range [g0, g0+KW) with a
// warp-uniform label index.  g0 is chosen so that as many of the 32 windows as possible lie
// inside the range; the others (and the whole-range windows of discarded pixels) go to a
// list that fine_cost_list handles pixel by pixel.
//
// Per view the warp stages the table entries of its KW labels, the view region its samples
// can touch and the census words there in its slice of shared memory.  The range splits into
// segments at the labels where the bilinear cell (integer shift) or the nearest census
// position changes.  Inside a segment the fractional shift grows linearly with the label
// (a*d is linear in d), so the bilinear sample is a quadratic polynomial in the label index i,
// s(i) = A + i (B + i C), and the census term is a constant.  A short loop over the segments
// writes each lane's (A, B, C, w_census * HD) to shared memory; the label loop is then
// branch-free: per label one broadcast load of the segment offset, one 16-byte load of the
// lane's coefficients, two FMAs for the sample and two for |I_ref - s| and the sum.
template <int KW>
__global__ void __launch_bounds__(256, 2) fine_cost_rows(const float *__restrict__ views,
                                                         const uint64_t *__restrict__ cen,
                                                         const FineTap *__restrict__ tab, int G, int U, int V,
                                                         int H, int W, int ref, const int *__restrict__ lo,
                                                         const int *__restrict__ cnt,
                                                         const long long *__restrict__ off, float wl2, float wc,
                                                         float fstep, float *__restrict__ cost,
                                                         int *__restrict__ status, int *__restrict__ list,
                                                         int *__restrict__ list_count, int rf_cap, int rc_cap,
                                                         int seg_cap) {
    static_assert(KW > 32 && KW <= 64, "two 32-bit masks cover the label range");
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const size_t warp_bytes = (size_t)seg_cap * 512 + (size_t)KW * 128 + (size_t)KW * 20 + (size_t)rc_cap * 8 +
                              (size_t)rf_cap * 4;
    unsigned char *wbase = smem + wib * warp_bytes;
    float4 *coef = (float4 *)wbase;                                             // [seg_cap][32]
    int *cdiff = (int *)(wbase + (size_t)seg_cap * 512);                        // [KW][32] census steps
    FineTap *ts = (FineTap *)(wbase + (size_t)seg_cap * 512 + (size_t)KW * 128); // [KW]
    int *segoff = (int *)((unsigned char *)ts + (size_t)KW * 16);                // [KW]
    uint64_t *rc = (uint64_t *)((unsigned char *)segoff + (size_t)KW * 4);
    float *rf = (float *)((unsigned char *)rc + (size_t)rc_cap * 8);
    const size_t N = (size_t)H * W;
    const int nviews = U * V, uc = ref % U, vc = ref / U;
    const int tiles_x = (W + 31) >> 5;
    const int task = blockIdx.x * wpb + wib;
    if (task >= tiles_x * H) return;
    const int y = task / tiles_x, x0 = (task - y * tiles_x) << 5, x = x0 + lane;
    int l = 0, n = 0;
    long long o = 0, row = 0;
    bool nar = false;
    if (x < W) {
        const int p = y * W + x;
        l = __ldg(lo + p);
        n = __ldg(cnt + p);
        o = __ldg(off + p);
        row = __ldg(off + p + 1) - o;
        if (window_ok(l, n, G, row, status)) {
            if (n <= 32) nar = true;
            else list[atomicAdd(list_count, 1)] = p;
        }
    }
    float Iref = 0.f;
    uint64_t cr = 0;
    if (nar) {
        const int p = y * W + x;
        Iref = __ldg(views + (size_t)ref * N + p);
        cr = __ldg(cen + (size_t)ref * N + p);
        const int npad = (int)min((long long)((n + 3) & ~3), row);
        for (int j = n; j < npad; j++) cost[o + j] = 0.f;
    }
    // the label range covering the most windows (ties: the lowest start); the others go to the list
    int g0 = 0, best_fit = -1;
    for (int c = 0; c < 32; c++) {
        const int cl = __shfl_sync(0xffffffffu, l, c);
        if (!__shfl_sync(0xffffffffu, nar, c)) continue;
        const int fit = __popc(__ballot_sync(0xffffffffu, nar && l >= cl && l + n <= cl + KW));
        if (fit > best_fit || (fit == best_fit && cl < g0)) {
            best_fit = fit;
            g0 = cl;
        }
    }
    if (best_fit <= 0) return;
    {
        const bool fits = nar && l >= g0 && l + n <= g0 + KW;
        if (nar && !fits) list[atomicAdd(list_count, 1)] = y * W + x;
        float acc[KW];
#pragma unroll
        for (int i = 0; i < KW; i++) {
            acc[i] = 0.f;
            cdiff[i * 32 + lane] = 0;
        }
        for (int view = 0; view < nviews; view++) {
            if (view == ref) continue;
            const FineTap *tv = tab + (size_t)view * G;
            // table entries of the range (labels past G - 1 repeat the last one and are never stored)
            for (int i = lane; i < KW; i += 32)
                reinterpret_cast<int4 *>(ts)[i] = __ldg(reinterpret_cast<const int4 *>(tv + min(g0 + i, G - 1)));
            __syncwarp();
            const FineTap ta = ts[0], tb = ts[KW - 1];
            const int oxlo = min(ta.ox, tb.ox), oxhi = max(ta.ox, tb.ox);
            const int oylo = min(ta.oy, tb.oy), oyhi = max(ta.oy, tb.oy);
            const int nxlo = min(ta.nx, tb.nx), nxhi = max(ta.nx, tb.nx);
            const int nylo = min(ta.ny, tb.ny), nyhi = max(ta.ny, tb.ny);
            const int rw = 33 + oxhi - oxlo, rh = 2 + oyhi - oylo;
            const int cw = 32 + nxhi - nxlo, ch = 1 + nyhi - nylo;
            // breakpoints: where the bilinear cell changes (segments) and where the census position changes
            const int4 *t4 = reinterpret_cast<const int4 *>(ts);
            const int i1 = min(lane + 32, KW - 1);
            const int4 e0 = t4[lane], p0 = t4[lane > 0 ? lane - 1 : 0];
            const int4 e1 = t4[i1], p1 = t4[i1 - 1];
            const unsigned sm0 = __ballot_sync(0xffffffffu, lane == 0 || e0.x != p0.x);
            const unsigned sm1 = __ballot_sync(0xffffffffu, lane + 32 < KW && e1.x != p1.x);
            const unsigned cm0 = __ballot_sync(0xffffffffu, lane == 0 || e0.y != p0.y);
            const unsigned cm1 = __ballot_sync(0xffffffffu, lane + 32 < KW && e1.y != p1.y);
            const int nseg = __popc(sm0) + __popc(sm1);
            if (rw * rh > rf_cap || cw * ch > rc_cap || nseg > seg_cap) {   // cannot happen with host-sized caps
                if (lane == 0) atomicExch(status, 7);
                __syncwarp();
                continue;
            }
            segoff[lane] = (__popc(sm0 & (0xffffffffu >> (31 - lane))) - 1) * 32;
            if (lane + 32 < KW)
                segoff[lane + 32] = (__popc(sm0) + __popc(sm1 & (0xffffffffu >> (31 - lane))) - 1) * 32;
            const float *img = views + (size_t)view * N;
            const uint64_t *cimg = cen + (size_t)view * N;
            for (int yy = 0; yy < rh; yy++) {
                const float *src = img + (size_t)min(max(y + oylo + yy, 0), H - 1) * W;
                float *dst = rf + yy * rw;
                for (int xx = lane; xx < rw; xx += 32) dst[xx] = __ldg(src + min(max(x0 + oxlo + xx, 0), W - 1));
            }
            for (int yy = 0; yy < ch; yy++) {
                const uint64_t *src = cimg + (size_t)min(max(y + nylo + yy, 0), H - 1) * W;
                uint64_t *dst = rc + yy * cw;
                for (int xx = lane; xx < cw; xx += 32) dst[xx] = __ldg(src + min(max(x0 + nxlo + xx, 0), W - 1));
            }
            __syncwarp();
            // census: a step function of the label, added as integer differences at its breakpoints
            {
                unsigned m0 = cm0, m1 = cm1;
                int prev = 0;
                while (m0 | m1) {
                    int i;
                    if (m0) {
                        i = __ffs(m0) - 1;
                        m0 &= m0 - 1;
                    } else {
                        i = 32 + __ffs(m1) - 1;
                        m1 &= m1 - 1;
                    }
                    const int wy = t4[i].y;
                    const int tnx = (int16_t)(wy & 0xffff), tny = wy >> 16;
                    const int h = __popcll(cr ^ rc[(tny - nylo) * cw + (lane + tnx - nxlo)]);
                    cdiff[i * 32 + lane] += h - prev;
                    prev = h;
                }
            }
            // l2 term: per cell segment this lane's sample polynomial in the absolute label index
            const float ax = (float)(view % U - uc) * fstep, ay = (float)(view / U - vc) * fstep;
            {
                unsigned m0 = sm0, m1 = sm1;
                for (int sgi = 0; sgi < nseg; sgi++) {
                    int i;
                    if (m0) {
                        i = __ffs(m0) - 1;
                        m0 &= m0 - 1;
                    } else {
                        i = 32 + __ffs(m1) - 1;
                        m1 &= m1 - 1;
                    }
                    const int4 w = t4[i];
                    const int tox = (int16_t)(w.x & 0xffff), toy = w.x >> 16;
                    const float tfx = __int_as_float(w.z), tfy = __int_as_float(w.w);
                    const float *q = rf + (toy - oylo) * rw + (lane + tox - oxlo);
                    const float i00 = q[0], i10 = q[1], i01 = q[rw], i11 = q[rw + 1];
                    const float c1 = i10 - i00, c2 = i01 - i00, c3 = (i11 - i01) - c1;
                    // s(t) = c0 + c1 fx + c2 fy + c3 fx fy, fx = fx0 + ax t, fy = fy0 + ay t, t = i' - i
                    const float a0 = fmaf(c3 * tfx, tfy, fmaf(c2, tfy, fmaf(c1, tfx, i00)));
                    const float b0 = fmaf(c3, fmaf(tfx, ay, tfy * ax), fmaf(c2, ay, c1 * ax));
                    const float Cq = c3 * ax * ay;
                    const float fi = (float)i;
                    coef[sgi * 32 + lane] = make_float4(fmaf(fi, fmaf(fi, Cq, -b0), a0), fmaf(-2.f * fi, Cq, b0), Cq, 0.f);
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < KW; i++) {
                const float4 k = coef[segoff[i] + lane];
                const float fi = (float)i;
                const float smp = fmaf(fi, fmaf(fi, k.z, k.y), k.x);
                acc[i] = fmaf(wl2, fabsf(Iref - smp), acc[i]);
            }
            __syncwarp();
        }
        if (fits) {
            int run = 0;
#pragma unroll
            for (int i = 0; i < KW; i++) {
                run += cdiff[i * 32 + lane];
                const int g = g0 + i;
                if (g >= l && g < l + n) cost[o + (g - l)] = fmaf(wc, (float)run, acc[i]);
            }
        }
    }
}

// The per-pixel form over a list of pixels (the whole-range windows left by fine_cost_rows):
// one warp per (pixel, chunk of 32 labels), lane = label, the view loop unrolled so that
// several independent table -> tap load chains are in flight.
__global__ void __launch_bounds__(256) fine_cost_list(const float *__restrict__ views,
                                                      const uint64_t *__restrict__ cen,
                                                      const FineTap *__restrict__ tab, int G, int nviews,
                                                      int H, int W, int ref, const int *__restrict__ lo,
                                                      const int *__restrict__ cnt,
                                                      const long long *__restrict__ off, float wl2, float wc,
                                                      float *__restrict__ cost, const int *__restrict__ list,
                                                      const int *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const size_t N = (size_t)H * W;
    const int chunks = (G + 31) >> 5;
    const long long total = (long long)(*count) * chunks;
    for (long long t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += warps) {
        const int p = list[t / chunks];
        const int chunk = (int)(t % chunks);
        const int l0 = __ldg(lo + p), n = __ldg(cnt + p);
        const long long o = __ldg(off + p), row = __ldg(off + p + 1) - o;
        const int npad = (int)min((long long)((n + 3) & ~3), row);
        const int j = chunk * 32 + lane;
        if (chunk * 32 >= npad) continue;
        const int x = p % W, y = p / W;
        const float Iref = __ldg(views + (size_t)ref * N + p);
        const uint64_t cr = __ldg(cen + (size_t)ref * N + p);
        float sl2 = 0.f;
        int sc = 0;
        if (j < n) {
            const int g = l0 + j;
#pragma unroll 4
            for (int vi = 0; vi < nviews - 1; vi++) {
                const int view = vi + (vi >= ref);
                const FineTap t = load_tap(tab + (size_t)view * G + g);
                const float *I = views + (size_t)view * N;
                const int x0 = min(max(x + t.ox, 0), W - 1), x1 = min(max(x + t.ox + 1, 0), W - 1);
                const int y0 = min(max(y + t.oy, 0), H - 1), y1 = min(max(y + t.oy + 1, 0), H - 1);
                const float i00 = __ldg(I + (size_t)y0 * W + x0), i10 = __ldg(I + (size_t)y0 * W + x1);
                const float i01 = __ldg(I + (size_t)y1 * W + x0), i11 = __ldg(I + (size_t)y1 * W + x1);
                const float top = (1.f - t.fx) * i00 + t.fx * i10;
                const float bot = (1.f - t.fx) * i01 + t.fx * i11;
                const float smp = (1.f - t.fy) * top + t.fy * bot;
                sl2 += fabsf(Iref - smp);
                const int xn = min(max(x + t.nx, 0), W - 1), yn = min(max(y + t.ny, 0), H - 1);
                sc += __popcll(cr ^ __ldg(cen + (size_t)view * N + (size_t)yn * W + xn));
            }
        }
        if (j < npad) cost[o + j] = (j < n) ? wl2 * sl2 + wc * (float)sc : 0.f;
    }
}

constexpr int kRowKW = 36;

}  // namespace

int fine_cost_tiled_caps(int U, int V, int uc, int vc, int G, double dmin, double dmax, int *rf_cap, int *rc_cap,
                         int *seg_cap) {
    // the largest integer-shift span of KW consecutive labels, per axis, and the most segments
    // (every integer and half-integer crossing of either shift starts one)
    const double step = (dmax - dmin) / (double)(G - 1);
    const int ax = (uc > U - 1 - uc ? uc : U - 1 - uc), ay = (vc > V - 1 - vc ? vc : V - 1 - vc);
    const double spx = ax * step * (kRowKW - 1), spy = ay * step * (kRowKW - 1);
    const int sx = (int)ceil(spx) + 2, sy = (int)ceil(spy) + 2;
    *rf_cap = ((33 + sx) * (2 + sy) + 3) & ~3;
    *rc_cap = (32 + sx) * (1 + sy);
    *seg_cap = 1 + ((int)ceil(spx) + 1) + ((int)ceil(spy) + 1);
    if (*seg_cap > kRowKW) *seg_cap = kRowKW;
    return (int)((size_t)*seg_cap * 512 + (size_t)kRowKW * 148 + (size_t)*rc_cap * 8 + (size_t)*rf_cap * 4);
}

cudaError_t launch_fine_cost_tiled(cudaStream_t s, const float *views, const uint64_t *cen, const FineTap *tab,
                                   int G, int U, int V, int H, int W, int ref, const int *lo, const int *cnt,
                                   const long long *off, float wl2, float wc, float *cost, int *status,
                                   int *wide_list, int *wide_count, int rf_cap, int rc_cap, int seg_cap,
                                   float fstep) {
    const int wpb = 8;
    const size_t smem = (size_t)wpb * ((size_t)seg_cap * 512 + (size_t)kRowKW * 148 + (size_t)rc_cap * 8 +
                                       (size_t)rf_cap * 4);
    cudaError_t e = cudaFuncSetAttribute(fine_cost_rows<kRowKW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long tasks = (long long)((W + 31) / 32) * H;
    const unsigned grid = (unsigned)((tasks + wpb - 1) / wpb);
    fine_cost_rows<kRowKW><<<grid, 32 * wpb, smem, s>>>(views, cen, tab, G, U, V, H, W, ref, lo, cnt, off, wl2, wc,
                                                        fstep, cost, status, wide_list, wide_count, rf_cap, rc_cap,
                                                        seg_cap);
    return cudaGetLastError();
}

cudaError_t launch_fine_cost_list(cudaStream_t s, const float *views, const uint64_t *cen, const FineTap *tab,
                                  int G, int nviews, int H, int W, int ref, const int *lo, const int *cnt,
                                  const long long *off, float wl2, float wc, float *cost, const int *list,
                                  const int *count) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    fine_cost_list<<<sms * 8, 256, 0, s>>>(views, cen, tab, G, nviews, H, W, ref, lo, cnt, off, wl2, wc, cost,
                                           list, count);
    return cudaGetLastError();
}

cudaError_t launch_fine_cost(cudaStream_t s, const float *views, const uint64_t *cen, const FineTap *tab,
                             int G, int nviews, int H, int W, int ref, const int *lo, const int *cnt,
                             const long long *off, float wl2, float wc, float *cost, int *status) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int block = 256;
    const long long want = ((long long)H * W * 32 + block - 1) / block;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    fine_cost_generic<<<grid, block, 0, s>>>(views, cen, tab, G, nviews, H, W, ref, lo, cnt, off, wl2,
                                             wc, cost, status);
    return cudaGetLastError();
}

}  // namespace lfsgm
