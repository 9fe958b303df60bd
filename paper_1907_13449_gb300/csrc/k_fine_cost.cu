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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>

#include "lfsgm_internal.cuh"

#include <algorithm>
#include <vector>

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
// Staging.  The views and census words are read from edge-replicated padded copies (a read at
// a padded position equals the clamped read), so every tile a warp needs lies inside the padded
// image.  Per view, one lane issues a TMA tile load of the view values around the row segment
// (x rounded down to the 16-byte boundary) and a bulk copy of the range's descriptor on one
// mbarrier, two stages deep, so view v+1 streams in while view v is computed; the census words
// around the segment come as a third tile on a second mbarrier, into one buffer that is refilled
// for view v+1 as soon as view v's census breakpoints have been read.  Waits are bounded: on
// expiry LFSGM_ERR_TIMEOUT is latched.
//
// Compute.  The range splits into segments at the labels where the bilinear cell (integer shift)
// changes.  Inside a segment the fractional shift grows linearly with the label (a*d is linear in
// d), so the bilinear sample minus I_ref(p) is a quadratic polynomial in the label index i,
// s(i) = A + i (B + i C).  A short loop over the segments writes each lane's (A, B, C) to shared
// memory; everything about a segment that is the same for all lanes (its fractions, their
// products with the view's shift factors, its first label) comes precomputed with the
// descriptor.  The label loop runs in blocks of four labels: a block in which no segment starts
// (the common case: segments span 8-36 labels) evaluates its labels with the coefficients in
// registers, two FMAs and one |.|-add per label; a block with a segment start reloads the lane's
// coefficients from shared memory at that label.  The l2 weight multiplies the sums once at the
// end.  The census term is a step function of the label: its Hamming distances are added as
// integer differences at the census breakpoints (a shared-memory atomic into per-lane words that
// hold two labels' 16-bit differences) and prefix-summed once at the end.
//
// Colour (C = 3, Sec. III-B/C).  The view tile is the padded float4 pixels (channels interleaved,
// a 4-D tensor map) and the census tile the view's three census planes (box depth 3).  The channels
// go one after another through the same segment and label loops: a channel's sample differences
// e_c(i) are squared into per-label sums, and the label's l2 term is the square root of the sum
// over the channels (the Euclidean norm of the colour difference); the census steps add the three
// channels' Hamming distances.
struct RowPlan {
    int P, Wp, Hp;                    // padding and padded sizes
    int bwf, bhf, bwc, bhc;           // TMA boxes (elements): view values, census words
    int seg_cap;                      // most segments (and census breakpoints) in one label range
    int ds_stride;                    // bytes of one (view, g0) descriptor slot
    int o_rf, o_ds, stage;            // view tile and descriptor of stage 0 in a warp's slice; stage 1 at +stage
    int o_rc;                         // census tile (one buffer: refilled once its breakpoints are read)
    int o_cab, o_cc, o_cdiff, o_mbar, warp_bytes;
    int kw;                           // label span of a row's range (a kernel instantiation)
    int C;                            // channels: 1, or 3 (float4 view tiles, three census planes)
};

// Descriptor of the label range [g0, g0+KW) of one view (built on the host, see
// build_fine_rows_desc): everything about the range that does not depend on the row segment.
//   bytes  0..7   int16 xf, yf, xc, yc: tile origins relative to (x0, y)
//   bytes  8..11  uint8 nseg, ncen; uint16 nbytes (bytes of this descriptor, a multiple of 16)
//   bytes 12..15  float ax * ay
//   bytes 16..23  uint64 smask: bit i set where label i starts a segment (bit 0 always)
//   bytes 24..31  float ax, ay: the view's (u-uc) * step and (v-vc) * step
//   bytes 32..    per segment 32 bytes: int tile offset of the (0,0) tap for lane 0, float first
//                 label fi, fx, fy; float fx*fy, fx*ay + fy*ax, -2 fi, 0
//   then          per census breakpoint 16 bytes: int tile offset of its word for lane 0, byte
//                 offset of its 32-bit difference word (label / 2) * 128, shift 16 * (label & 1), 0
constexpr int kDsMask = 16, kDsAxy = 24, kDsSegs = 32, kDsSegBytes = 32, kDsCenBytes = 16;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Bounded wait on an mbarrier phase: each try_wait may suspend the thread for up to 200 ns (a hint;
// it returns as soon as the phase completes), so a wait polls a few times instead of spinning, and
// 2^20 tries bound it to about 0.2 s.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
    for (int it = 0; it < (1 << 20); it++) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(mbar), "r"(parity), "n"(200) : "memory");
        if (done) return true;
    }
    return false;
}

template <int KW, int C>
__global__ void __launch_bounds__(128, C == 1 ? 5 : 2) fine_cost_rows(const __grid_constant__ CUtensorMap tm_v,
                                                         const __grid_constant__ CUtensorMap tm_c,
                                                         const unsigned char *__restrict__ desc, int G, int U, int V,
                                                         int H, int W, int ref, const int *__restrict__ lo,
                                                         const int *__restrict__ cnt,
                                                         const long long *__restrict__ off,
                                                         const float *__restrict__ views_pad,
                                                         const uint64_t *__restrict__ cen_pad, float wl2, float wc,
                                                         float *__restrict__ cost,
                                                         int *__restrict__ status, int2 *__restrict__ list,
                                                         int *__restrict__ list_count, RowPlan pl) {
    static_assert(KW > 32 && KW <= 64 && KW % 4 == 0, "two 32-bit masks cover the label range, blocks of 4");
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    unsigned char *wb = smem + (size_t)wib * pl.warp_bytes;
    float2 *cab = (float2 *)(wb + pl.o_cab) + lane;         // (A, B) [seg_cap][32]
    float *ccq = (float *)(wb + pl.o_cc) + lane;            // C [seg_cap][32]
    int *cdw = (int *)(wb + pl.o_cdiff) + lane;             // [KW / 2][32] two labels' census steps
    const unsigned mbar0 = smem_u32(wb + pl.o_mbar);        // stages 0, 1 at +0, +8; census tile at +16
    const int nviews = U * V;
    const size_t HWp = (size_t)pl.Hp * pl.Wp;
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
            else push_chunks(list, list_count, p, n);
        }
    }
    // the label range covering the most windows (ties: the lowest start); the others go to the list
    int g0;
    const int best_fit = row_range<KW>(l, n, nar, g0);
    if (best_fit <= 0) return;
    const bool fits = nar && l >= g0 && l + n <= g0 + KW;
    if (nar && !fits) push_chunks(list, list_count, y * W + x, n);
    float Iref = 0.f, Iref1 = 0.f, Iref2 = 0.f;           // the reference pixel (channels 1, 2: colour)
    uint64_t cr[C];
#pragma unroll
    for (int ch = 0; ch < C; ch++) cr[ch] = 0;
    if (fits) {
        const size_t pp = (size_t)(y + pl.P) * pl.Wp + (x + pl.P);
        if constexpr (C == 1) {
            Iref = __ldg(views_pad + (size_t)ref * HWp + pp);
        } else {
            const float4 iv = __ldg(reinterpret_cast<const float4 *>(views_pad) + (size_t)ref * HWp + pp);
            Iref = iv.x;
            Iref1 = iv.y;
            Iref2 = iv.z;
        }
#pragma unroll
        for (int ch = 0; ch < C; ch++) cr[ch] = __ldg(cen_pad + ((size_t)ref * C + ch) * HWp + pp);
        const int npad = (int)min((long long)((n + 3) & ~3), row);
        for (int j = n; j < npad; j++) cost[o + j] = 0.f;
    }
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 16));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const unsigned tile_bytes = (unsigned)(pl.bwf * pl.bhf * 4 * (C == 1 ? 1 : 4));
    const unsigned cen_bytes = (unsigned)(pl.bwc * pl.bhc * 8 * C);
    auto dsc_of = [&](int view) { return desc + ((size_t)view * G + g0) * pl.ds_stride; };
    // the first 16 bytes of the next views' descriptors (tile origins, counts, size), read one
    // view ahead of their issue
    auto head = [&](int view) { return __ldg(reinterpret_cast<const int4 *>(dsc_of(view))); };
    auto issue = [&](int view, int4 hd, int st) {
        if (lane != 0) return;
        const int xf = x0 + (int)(short)(hd.x & 0xffff), yf = y + (hd.x >> 16);
        const unsigned nb = min((unsigned)hd.z >> 16, (unsigned)pl.ds_stride) & ~15u;
        const unsigned mb = mbar0 + 8 * st;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(tile_bytes + nb) : "memory");
        if constexpr (C == 1)
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                         ::"r"(smem_u32(wb + pl.o_rf + st * pl.stage)), "l"((unsigned long long)&tm_v), "r"(xf), "r"(yf), "r"(view), "r"(mb)
                         : "memory");
        else                                       // {channel, x, y, view} of the float4 pixels
            asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                         ::"r"(smem_u32(wb + pl.o_rf + st * pl.stage)), "l"((unsigned long long)&tm_v), "r"(0), "r"(xf), "r"(yf), "r"(view), "r"(mb)
                         : "memory");
        if (nb > 0)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                         ::"r"(smem_u32(wb + pl.o_ds + st * pl.stage)), "l"(dsc_of(view)), "r"(nb), "r"(mb)
                         : "memory");
    };
    auto issue_cen = [&](int view, int4 hd) {
        if (lane != 0) return;
        const int xc = x0 + (int)(short)(hd.y & 0xffff), yc = y + (hd.y >> 16);
        const unsigned mb = mbar0 + 16;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(cen_bytes) : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(smem_u32(wb + pl.o_rc)), "l"((unsigned long long)&tm_c), "r"(xc), "r"(yc), "r"(view * C), "r"(mb)
                     : "memory");
    };
    float acc[KW];
#pragma unroll
    for (int i = 0; i < KW; i++) acc[i] = 0.f;
#pragma unroll
    for (int i = 0; i < KW / 2; i++) cdw[32 * i] = 0;
    const int nv = nviews - 1;                      // every view but the reference
    auto view_of = [&](int vi) { return vi + (vi >= ref); };
    {
        const int4 h0 = head(view_of(0));
        issue(view_of(0), h0, 0);
        issue_cen(view_of(0), h0);
    }
    int4 hd_next = nv > 1 ? head(view_of(1)) : make_int4(0, 0, 0, 0);
    bool ok = true;
    for (int vi = 0; vi < nv; vi++) {
        const int st = vi & 1;
        if (vi + 1 < nv) issue(view_of(vi + 1), hd_next, st ^ 1);
        if (!mbar_wait(mbar0 + 8 * st, (unsigned)(vi >> 1) & 1u) || !mbar_wait(mbar0 + 16, (unsigned)vi & 1u)) {
            if (lane == 0) atomicExch(status, 6);
            // let the copies still in flight land (bounded) before the warp's shared memory is released
            mbar_wait(mbar0 + 8 * st, (unsigned)(vi >> 1) & 1u);
            mbar_wait(mbar0 + 16, (unsigned)vi & 1u);
            if (vi + 1 < nv) mbar_wait(mbar0 + 8 * (st ^ 1), (unsigned)((vi + 1) >> 1) & 1u);
            ok = false;
            break;
        }
        const float *rf = (const float *)(wb + pl.o_rf + st * pl.stage);
        const uint64_t *rc = (const uint64_t *)(wb + pl.o_rc);
        const unsigned char *ds = wb + pl.o_ds + st * pl.stage;
        const int4 hdr = *(const int4 *)ds;
        const int nseg = hdr.z & 0xff, ncen = (hdr.z >> 8) & 0xff;
        const bool good = nseg >= 1 && nseg <= pl.seg_cap && ncen <= pl.seg_cap &&
                          kDsSegs + nseg * kDsSegBytes + ncen * kDsCenBytes <= ((hdr.z >> 16) & 0xffff);
        // census: integer steps at the census breakpoints
        if (good) {
            const int4 *ce = (const int4 *)(ds + kDsSegs + nseg * kDsSegBytes);
            int prev = 0;
            for (int b = 0; b < ncen; b++) {
                const int4 e = ce[b];
                int h = 0;
#pragma unroll
                for (int ch = 0; ch < C; ch++) h += __popcll(cr[ch] ^ rc[ch * pl.bwc * pl.bhc + e.x + lane]);
                atomicAdd((int *)((char *)cdw + e.y), (int)((unsigned)(h - prev) << e.z));
                prev = h;
            }
        }
        __syncwarp();                                  // every lane has read the census tile
        if (vi + 1 < nv) {
            issue_cen(view_of(vi + 1), hd_next);
            if (vi + 2 < nv) hd_next = head(view_of(vi + 2));
        }
        if (!good) {
            if (lane == 0) atomicExch(status, 7);      // cannot happen: the host checked every descriptor
            __syncwarp();
            continue;
        }
        // l2 term: per cell segment this lane's sample polynomial (minus I_ref) in the label index
        const float2 axy = *(const float2 *)(ds + kDsAxy);
        const float axay = __int_as_float(hdr.w);
        const float4 *sg = (const float4 *)(ds + kDsSegs);
        const uint2 smask = *(const uint2 *)(ds + kDsMask);
        // one channel (tile values rfc[tstride * pixel]): the segments' coefficients, then the label
        // loop, which hands each label's sample difference e to op(label, e)
        auto channel = [&](const float *rfc, int tstride, float Ic, auto &&op) {
            for (int sgi = 0; sgi < nseg; sgi++) {
                const float4 d0 = sg[2 * sgi], d1 = sg[2 * sgi + 1];
                const float *q = rfc + tstride * (__float_as_int(d0.x) + lane);
                const float i00 = q[0], i10 = q[tstride], i01 = q[tstride * pl.bwf], i11 = q[tstride * (pl.bwf + 1)];
                const float c1 = i10 - i00, c2 = i01 - i00, c3 = (i11 - i01) - c1;
                // s(t) - I_ref = (c0 - I_ref) + c1 fx + c2 fy + c3 fx fy, fx = fx0 + ax t, fy = fy0 + ay t,
                // t = i - fi: value a0, slope b0 and curvature Cq at t = 0, then in powers of i
                const float a0 = fmaf(c3, d1.x, fmaf(c2, d0.w, fmaf(c1, d0.z, i00 - Ic)));
                const float b0 = fmaf(c3, d1.y, fmaf(c2, axy.y, c1 * axy.x));
                const float Cq = c3 * axay;
                const float fi = d0.y;
                cab[32 * sgi] = make_float2(fmaf(fi, fmaf(fi, Cq, -b0), a0), fmaf(d1.z, Cq, b0));
                ccq[32 * sgi] = Cq;
            }
            // (each lane reads back only its own coefficients: no warp synchronisation needed)
            unsigned cpab = smem_u32(cab) - 256u, cpc = smem_u32(ccq) - 128u;
            float4 cf = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < KW / 4; k++) {
                const unsigned bits = (k < 8 ? smask.x >> (4 * k) : smask.y >> (4 * k - 32)) & 0xfu;
                if (bits == 0) {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const float fi = (float)(4 * k + e);
                        op(4 * k + e, fmaf(fi, fmaf(fi, cf.z, cf.y), cf.x));
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        // a segment starts at this label: step to its coefficients (predicated, no branch)
                        asm volatile("{\n .reg .pred p;\n .reg .b32 t;\n and.b32 t, %5, %6;\n setp.ne.u32 p, t, 0;\n"
                                     " @p add.u32 %3, %3, 256;\n @p add.u32 %4, %4, 128;\n"
                                     " @p ld.shared.v2.f32 {%0, %1}, [%3];\n @p ld.shared.f32 %2, [%4];\n}"
                                     : "+f"(cf.x), "+f"(cf.y), "+f"(cf.z), "+r"(cpab), "+r"(cpc)
                                     : "r"(bits), "r"(1u << e));
                        const float fi = (float)(4 * k + e);
                        op(4 * k + e, fmaf(fi, fmaf(fi, cf.z, cf.y), cf.x));
                    }
                }
            }
            __syncwarp();      // the next channel's coefficients overwrite these (a memory barrier)
        };
        if constexpr (C == 1) {
            channel(rf, 1, Iref, [&](int i, float e) { acc[i] += fabsf(e); });
        } else {
            // squared colour differences per label, then their norm
            float sq[KW];
            channel(rf, 4, Iref, [&](int i, float e) { sq[i] = e * e; });
            channel(rf + 1, 4, Iref1, [&](int i, float e) { sq[i] = fmaf(e, e, sq[i]); });
            channel(rf + 2, 4, Iref2, [&](int i, float e) { sq[i] = fmaf(e, e, sq[i]); });
#pragma unroll
            for (int i = 0; i < KW; i++) acc[i] += sqrtf(sq[i]);
        }
        __syncwarp();
    }
    if (!ok) return;
    __syncwarp();
    if (fits) {
        int run = 0;
#pragma unroll
        for (int i = 0; i < KW; i += 2) {
            // the word holds d(i) + d(i+1) 2^16 (two's complement, |d| < 2^15): split it exactly
            const int w = cdw[16 * i];
            const int d0 = (int)(short)(w & 0xffff), d1 = (w - d0) >> 16;
            run += d0;
            const int g = g0 + i;
            if (g >= l && g < l + n) cost[o + (g - l)] = fmaf(wc, (float)run, wl2 * acc[i]);
            run += d1;
            if (g + 1 >= l && g + 1 < l + n) cost[o + (g + 1 - l)] = fmaf(wc, (float)run, wl2 * acc[i + 1]);
        }
    }
}

// The per-pixel form over a list of (pixel, chunk) items (the windows left by fine_cost_rows):
// one warp per item, lane = label of the chunk, taps read from the padded views and census words
// (no clamping needed) at linear offsets (oy Wp + ox, ny Wp + nx).  Each lane reads its label's
// table entry of a view with one coalesced 16-byte load (the warp's 32 entries are contiguous);
// two views per unrolled step keep their loads in flight together.  Colour (C > 1): the padded
// views hold one float4 per pixel (channels interleaved), so a bilinear tap of all channels is
// four 16-byte loads, and the census words are planes view * C + c; the l2 term is the Euclidean
// norm of the colour difference and the census term sums the channels' Hamming distances
// (Sec. III-B/C).
constexpr int kListWarps = 4;

// LEAN (grey): 32 registers for 16 CTAs of 128 threads per SM (a few spilled bytes); the grey
// list is latency-bound, and the extra warps took the bench light field's list from 0.241 to
// 0.193 ms, while the all-wide Middlebury-shaped list runs best with 40 registers and 12 CTAs
// (0.697 vs 0.722 ms): the speed knob picks.  Colour: 12 CTAs per SM (0.42 -> 0.37 ms against 9).
template <int C, bool LEAN>
__global__ void __launch_bounds__(32 * kListWarps, C == 3 ? 12 : (LEAN ? 16 : 12)) fine_cost_list(const float *__restrict__ views_pad,
                                                      const uint64_t *__restrict__ cen_pad, int P, int Wp, int Hp,
                                                      const int4 *__restrict__ ltab, int G, int nviews,
                                                      int W, int ref, const int *__restrict__ lo,
                                                      const int *__restrict__ cnt,
                                                      const long long *__restrict__ off, float wl2, float wc,
                                                      float *__restrict__ cost, const int2 *__restrict__ list,
                                                      const int *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const size_t HWp = (size_t)Hp * Wp;
    const int total = *count;
    const int nv1 = nviews - 1;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += warps) {
        const int2 item = list[t];
        const int p = item.x, chunk = item.y;
        const int l0 = __ldg(lo + p), n = __ldg(cnt + p);
        const long long o = __ldg(off + p), row = __ldg(off + p + 1) - o;
        if (!window_ok(l0, n, G, row, nullptr)) continue;      // items are pushed for valid windows only
        const int npad = (int)min((long long)((n + 3) & ~3), row);
        const int j = chunk * 32 + lane;
        const int x = p % W, y = p / W;
        const size_t base = (size_t)(y + P) * Wp + (x + P);
        float sl2 = 0.f;
        int sc = 0;
        if (j < n) {
            uint64_t cr[C];
#pragma unroll
            for (int ch = 0; ch < C; ch++) cr[ch] = __ldg(cen_pad + ((size_t)ref * C + ch) * HWp + base);
            const int4 *tg = ltab + l0 + j;
            if constexpr (C == 1) {
                const float Iref = __ldg(views_pad + (size_t)ref * HWp + base);
#pragma unroll 2
                for (int vi = 0; vi < nv1; vi++) {
                    const int view = vi + (vi >= ref);
                    const int4 tw = __ldg(tg + (size_t)view * G);     // linear tap offsets (x + Wp y), fx, fy
                    const size_t vb = (size_t)view * HWp + base;
                    const float tfx = __int_as_float(tw.z), tfy = __int_as_float(tw.w);
                    const float *q = views_pad + vb + tw.x;
                    const float i00 = __ldg(q), i10 = __ldg(q + 1), i01 = __ldg(q + Wp), i11 = __ldg(q + Wp + 1);
                    const float top = (1.f - tfx) * i00 + tfx * i10;
                    const float bot = (1.f - tfx) * i01 + tfx * i11;
                    sl2 += fabsf(Iref - ((1.f - tfy) * top + tfy * bot));
                    sc += __popcll(cr[0] ^ __ldg(cen_pad + vb + tw.y));
                }
            } else {
                const float4 *v4 = reinterpret_cast<const float4 *>(views_pad);
                const float4 Iref = __ldg(v4 + (size_t)ref * HWp + base);
#pragma unroll 2
                for (int vi = 0; vi < nv1; vi++) {
                    const int view = vi + (vi >= ref);
                    const int4 tw = __ldg(tg + (size_t)view * G);
                    const size_t pb = (size_t)view * HWp + base;
                    const float tfx = __int_as_float(tw.z), tfy = __int_as_float(tw.w);
                    const float4 *q = v4 + pb + tw.x;
                    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + Wp), d = __ldg(q + Wp + 1);
                    auto sample = [&](float i00, float i10, float i01, float i11) {
                        const float top = (1.f - tfx) * i00 + tfx * i10;
                        const float bot = (1.f - tfx) * i01 + tfx * i11;
                        return (1.f - tfy) * top + tfy * bot;
                    };
                    const float d0 = Iref.x - sample(a.x, b.x, c.x, d.x);
                    const float d1 = Iref.y - sample(a.y, b.y, c.y, d.y);
                    const float d2 = Iref.z - sample(a.z, b.z, c.z, d.z);
                    sl2 += sqrtf(fmaf(d2, d2, fmaf(d1, d1, d0 * d0)));
#pragma unroll
                    for (int ch = 0; ch < C; ch++)
                        sc += __popcll(cr[ch] ^ __ldg(cen_pad + ((size_t)view * C + ch) * HWp + base + tw.y));
                }
            }
        }
        if (j < npad) cost[o + j] = (j < n) ? wl2 * sl2 + wc * (float)sc : 0.f;
    }
}


__global__ void list_all_kernel(const int *__restrict__ lo, const int *__restrict__ cnt,
                                const long long *__restrict__ off, int G, int2 *list, int *count, int N,
                                int *status, int min_cnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < N && cnt[p] > min_cnt && window_ok(lo[p], cnt[p], G, off[p + 1] - off[p], status))
        push_chunks(list, count, p, cnt[p]);
}

int r128(int x) { return (x + 127) & ~127; }

}  // namespace

// Padding, TMA boxes and the per-warp shared-memory layout of the row kernel for one config.
bool plan_fine_rows(int U, int V, int uc, int vc, int H, int W, int G, double dmin, double dmax, int kw, int C,
                    RowPlanHost *out) {
    RowPlan pl{};
    const int kRowKW = kw == 44 ? 44 : 36;
    pl.kw = kRowKW;
    pl.C = C;
    const double md = fmax(fabs(dmin), fabs(dmax));
    const int amax = max(max(uc, U - 1 - uc), max(vc, V - 1 - vc));
    pl.P = (int)ceil(amax * md) + 3;
    pl.Wp = (W + 2 * pl.P + 3) & ~3;
    pl.Hp = H + 2 * pl.P;
    const double step = (dmax - dmin) / (double)(G - 1);
    const int ax = max(uc, U - 1 - uc), ay = max(vc, V - 1 - vc);
    const int spx = (int)ceil(ax * step * (kRowKW - 1)), spy = (int)ceil(ay * step * (kRowKW - 1));
    // taps: columns x0+oxlo .. x0+32+oxhi, rows y+oylo .. y+oyhi+1, with oxhi-oxlo <= spx, one label of
    // slack below the FP32 origin estimate and up to 3 (floats) / 1 (words) columns of 16-byte rounding
    pl.bwf = (spx + 38 + 3) & ~3;
    pl.bhf = spy + 4;
    pl.bwc = (spx + 35 + 1) & ~1;
    pl.bhc = spy + 3;
    pl.seg_cap = min(kRowKW, spx + spy + 3);
    pl.ds_stride = (kDsSegs + pl.seg_cap * (kDsSegBytes + kDsCenBytes) + 15) & ~15;
    int o = 0;
    pl.o_rf = o;
    pl.o_ds = pl.o_rf + r128(pl.bwf * pl.bhf * 4 * (C == 1 ? 1 : 4));     // colour: float4 pixels
    pl.stage = r128(pl.o_ds + pl.ds_stride - pl.o_rf);
    o = pl.o_rf + 2 * pl.stage;
    pl.o_rc = o;
    o += r128(pl.bwc * pl.bhc * 8 * C);                                       // one plane per channel
    pl.o_cab = o;
    o += pl.seg_cap * 256;
    pl.o_cc = o;
    o += pl.seg_cap * 128;
    pl.o_cdiff = o;
    o += kRowKW / 2 * 128;
    pl.o_mbar = o;
    o += 32;
    o = r128(o);
    pl.warp_bytes = o;
    // the census steps of one label, summed over the views and channels, must fit 16 bits (at most 48
    // bits a word); colour runs the 36-label span only
    out->ok = pl.bwf <= 256 && pl.bwc <= 256 && pl.bhf <= 256 && pl.bhc <= 256 && pl.warp_bytes <= 48 * 1024 &&
              (U * V - 1) * 48 * C < 32768 && pl.ds_stride < 65536 && (C == 1 || (C == 3 && kRowKW == 36));
    static_assert(sizeof(RowPlan) <= sizeof(out->raw), "plan storage");
    memcpy(out->raw, &pl, sizeof(pl));
    out->P = pl.P;
    out->Wp = pl.Wp;
    out->Hp = pl.Hp;
    return out->ok;
}

// Descriptors of every (view, g0) label range for the row kernel, from the host copy of the
// tap table.  The tile origins repeat the kernel's former FP32 estimate (one label of slack around
// the range's shifts, x rounded down to 16 bytes); every tap and census word of the range is
// checked to lie inside the tile boxes here, so the kernel needs no bounds test.  Returns false
// (the caller then sends every window to the list kernel) if any range does not fit.
bool build_fine_rows_desc(const RowPlanHost *ph, const FineTap *tab, int U, int V, int uc, int vc, int G, float dmin,
                          float fstep, std::vector<unsigned char> &out) {
    RowPlan pl;
    memcpy(&pl, ph->raw, sizeof(pl));
    const int kRowKW = pl.kw;
    const int nviews = U * V;
    const size_t bytes = (size_t)nviews * G * pl.ds_stride;
    if (bytes > ((size_t)512 << 20)) return false;
    out.assign(bytes, 0);
    std::vector<int> segstart, censtart;
    for (int view = 0; view < nviews; view++) {
        const float a = (float)(view % U - uc), b = (float)(view / U - vc);
        for (int g0 = 0; g0 < G; g0++) {
            unsigned char *d = out.data() + ((size_t)view * G + g0) * pl.ds_stride;
            const int nvalid = std::min(kRowKW, G - g0);
            const float d0 = std::fmaf((float)g0, fstep, dmin), d1 = std::fmaf((float)(g0 + nvalid - 1), fstep, dmin);
            const float sx0 = a * d0, sx1 = a * d1, sy0 = b * d0, sy1 = b * d1;
            const int xf = ((int)std::floor(std::fmin(sx0, sx1)) - 1 + pl.P) & ~3;
            const int yf = (int)std::floor(std::fmin(sy0, sy1)) - 1 + pl.P;
            const int xc = ((int)std::floor(std::fmin(sx0, sx1) + 0.5f) - 1 + pl.P) & ~1;
            const int yc = (int)std::floor(std::fmin(sy0, sy1) + 0.5f) - 1 + pl.P;
            const int bxf = pl.P - xf, byf = pl.P - yf, bxc = pl.P - xc, byc = pl.P - yc;
            const FineTap *t = tab + (size_t)view * G + g0;
            segstart.clear();
            censtart.clear();
            int oxlo = 1 << 30, oxhi = -(1 << 30), oylo = 1 << 30, oyhi = -(1 << 30);
            int nxlo = 1 << 30, nxhi = -(1 << 30), nylo = 1 << 30, nyhi = -(1 << 30);
            for (int i = 0; i < nvalid; i++) {
                if (i == 0 || t[i].ox != t[i - 1].ox || t[i].oy != t[i - 1].oy) segstart.push_back(i);
                if (i == 0 || t[i].nx != t[i - 1].nx || t[i].ny != t[i - 1].ny) censtart.push_back(i);
                oxlo = std::min(oxlo, (int)t[i].ox);
                oxhi = std::max(oxhi, (int)t[i].ox);
                oylo = std::min(oylo, (int)t[i].oy);
                oyhi = std::max(oyhi, (int)t[i].oy);
                nxlo = std::min(nxlo, (int)t[i].nx);
                nxhi = std::max(nxhi, (int)t[i].nx);
                nylo = std::min(nylo, (int)t[i].ny);
                nyhi = std::max(nyhi, (int)t[i].ny);
            }
            if (bxf + oxlo < 0 || bxf + 32 + oxhi >= pl.bwf || byf + oylo < 0 || byf + oyhi + 1 >= pl.bhf ||
                bxc + nxlo < 0 || bxc + 31 + nxhi >= pl.bwc || byc + nylo < 0 || byc + nyhi >= pl.bhc ||
                (int)segstart.size() > pl.seg_cap || (int)censtart.size() > pl.seg_cap)
                return false;
            const int16_t org[4] = {(int16_t)xf, (int16_t)(yf), (int16_t)xc, (int16_t)yc};
            memcpy(d, org, 8);
            const int nseg = (int)segstart.size(), ncen = (int)censtart.size();
            d[8] = (unsigned char)nseg;
            d[9] = (unsigned char)ncen;
            const uint16_t nbytes = (uint16_t)((kDsSegs + nseg * kDsSegBytes + ncen * kDsCenBytes + 15) & ~15);
            memcpy(d + 10, &nbytes, 2);
            // the view's disparity-to-shift factors (u-uc) * step, (v-vc) * step and their product
            const float ax = a * fstep, ay = b * fstep, axay = ax * ay;
            memcpy(d + 12, &axay, 4);
            uint64_t smask = 0;
            for (int i : segstart) smask |= 1ull << i;
            memcpy(d + kDsMask, &smask, 8);
            const float axy[2] = {ax, ay};
            memcpy(d + kDsAxy, axy, 8);
            for (int k = 0; k < nseg; k++) {
                const FineTap &w = t[segstart[k]];
                unsigned char *e = d + kDsSegs + k * kDsSegBytes;
                const int32_t toff = (byf + w.oy) * pl.bwf + (bxf + w.ox);
                const float f[7] = {(float)segstart[k], w.fx, w.fy, w.fx * w.fy, std::fmaf(w.fx, ay, w.fy * ax),
                                    -2.f * (float)segstart[k], 0.f};
                memcpy(e, &toff, 4);
                memcpy(e + 4, f, 28);
            }
            for (int k = 0; k < ncen; k++) {
                const FineTap &w = t[censtart[k]];
                const int32_t e4[4] = {(byc + w.ny) * pl.bwc + (bxc + w.nx), (censtart[k] >> 1) * 128,
                                       16 * (censtart[k] & 1), 0};
                memcpy(d + kDsSegs + nseg * kDsSegBytes + k * kDsCenBytes, e4, 16);
            }
        }
    }
    return true;
}

// Tensor maps of the padded views (float) and census words (uint64), 3-D [view][Hp][Wp].
bool encode_fine_rows_maps(RowPlanHost *ph, const float *views_pad, const uint64_t *cen_pad, int nviews) {
    RowPlan pl;
    memcpy(&pl, ph->raw, sizeof(pl));
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (pl.C == 3) {
        // float4 pixels (the fourth float is padding): {channel, x, y, view}
        const cuuint64_t dims[4] = {4, (cuuint64_t)pl.Wp, (cuuint64_t)pl.Hp, (cuuint64_t)nviews};
        const cuuint64_t strides[3] = {16, (cuuint64_t)pl.Wp * 16, (cuuint64_t)pl.Wp * pl.Hp * 16};
        const cuuint32_t box[4] = {4, (cuuint32_t)pl.bwf, (cuuint32_t)pl.bhf, 1};
        if (encode((CUtensorMap *)ph->tm_v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)views_pad, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    } else {
        const cuuint64_t dims[3] = {(cuuint64_t)pl.Wp, (cuuint64_t)pl.Hp, (cuuint64_t)nviews};
        const cuuint64_t strides[2] = {(cuuint64_t)pl.Wp * 4, (cuuint64_t)pl.Wp * pl.Hp * 4};
        const cuuint32_t box[3] = {(cuuint32_t)pl.bwf, (cuuint32_t)pl.bhf, 1};
        if (encode((CUtensorMap *)ph->tm_v, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)views_pad, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    {
        // census planes view * C + c: a view's C planes are one box of depth C
        const cuuint64_t dims[3] = {(cuuint64_t)pl.Wp, (cuuint64_t)pl.Hp, (cuuint64_t)nviews * pl.C};
        const cuuint64_t strides[2] = {(cuuint64_t)pl.Wp * 8, (cuuint64_t)pl.Wp * pl.Hp * 8};
        const cuuint32_t box[3] = {(cuuint32_t)pl.bwc, (cuuint32_t)pl.bhc, (cuuint32_t)pl.C};
        if (encode((CUtensorMap *)ph->tm_c, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, (void *)cen_pad, dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

cudaError_t launch_fine_cost_rows(cudaStream_t s, const RowPlanHost *ph, const float *views_pad,
                                  const uint64_t *cen_pad, const unsigned char *desc, int G, int U, int V, int H, int W,
                                  int ref, const int *lo, const int *cnt, const long long *off, float wl2, float wc,
                                  float fstep, float *cost, int *status, int2 *list, int *list_count) {
    RowPlan pl;
    memcpy(&pl, ph->raw, sizeof(pl));
    // warps (row segments) per CTA: colour 2 (22 KB of shared memory per warp: five CTAs, ten warps
    // per SM; four warps per CTA fit two CTAs, eight warps, and ran 12 % slower)
    const int wpb = pl.C == 3 ? 2 : 4;
    const size_t smem = (size_t)wpb * pl.warp_bytes;
    auto kern = pl.C == 3 ? fine_cost_rows<36, 3> : (pl.kw == 44 ? fine_cost_rows<44, 1> : fine_cost_rows<36, 1>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tasks = (long long)((W + 31) / 32) * H;
    const unsigned grid = (unsigned)((tasks + wpb - 1) / wpb);
    (void)fstep;
    kern<<<grid, 32 * wpb, smem, s>>>(*(const CUtensorMap *)ph->tm_v, *(const CUtensorMap *)ph->tm_c, desc, G, U, V, H,
                                      W, ref, lo, cnt, off, views_pad, cen_pad, wl2, wc, cost, status, list, list_count,
                                      pl);
    return cudaGetLastError();
}

cudaError_t launch_list_all(cudaStream_t s, const int *lo, const int *cnt, const long long *off, int G, int2 *list,
                            int *count, int N, int *status, int min_cnt) {
    list_all_kernel<<<(N + 255) / 256, 256, 0, s>>>(lo, cnt, off, G, list, count, N, status, min_cnt);
    return cudaGetLastError();
}

cudaError_t launch_fine_cost_list(cudaStream_t s, const float *views_pad, const uint64_t *cen_pad, int P, int Wp,
                                  int Hp, const int4 *ltab, int G, int nviews, int C, int W, int ref,
                                  const int *lo, const int *cnt, const long long *off, float wl2, float wc,
                                  float *cost, const int2 *list, const int *count, int ctas_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // grid-stride over the items, by default with exactly the CTAs that are resident at once: the
    // warps then sweep the list (pixel order) once, together, and the views around the rows in
    // flight stay in L2; a second wave would sweep the whole image again (colour: 9 resident CTAs
    // per SM, 4.35 ms, against 4.92 ms with 24 and 6.48 ms with 12)
    // grey: the lean instantiation by default and for 16 or more CTAs per SM, the other one below
    const bool lean = C == 1 && (ctas_per_sm <= 0 || ctas_per_sm >= 16);
    auto kern = C == 3 ? fine_cost_list<3, false> : (lean ? fine_cost_list<1, true> : fine_cost_list<1, false>);
    int k = ctas_per_sm;
    if (k <= 0) {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, kern, 32 * kListWarps, 0);
        if (e != cudaSuccess) return e;
        k = max(k, 1);
    }
    kern<<<sms * k, 32 * kListWarps, 0, s>>>(views_pad, cen_pad, P, Wp, Hp, ltab, G, nviews, W, ref, lo, cnt, off, wl2,
                                             wc, cost, list, count);
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
