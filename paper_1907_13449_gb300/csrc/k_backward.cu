// k_backward.cu -- adjoint of cost volume -> bounded SGM (8 or 16 paths) -> soft-argmin (not in the paper).
//
// Loss gradients arrive as grad_disp = dLoss/d dhat(p) for the soft-argmin disparity
// dhat = sum_g softmax(-C_s/tau)_g d_g.  Three kernels:
//  * softargmin_backward: dLoss/dC_s(p,g) = grad_disp(p) (-1/tau) w_g (d_g - dhat).
//  * sgm_backward: one warp per (direction, scanline).  The path is recomputed forward, recording
//    for every cell the winning branch of the normalised recurrence (P2 first, then same, g-1,
//    g+1, taken with strict comparisons in that order) and for every pixel the slot of its
//    minimum; the reverse sweep carries lambda = dLoss/dL_r along the path: it adds lambda into
//    dLoss/dC, gathers the predecessor's incoming adjoint from the three slots whose branch points
//    at it, routes (P2-branch lambdas - all lambdas) to the predecessor's minimum (the -m term),
//    and sums the branch lambdas into dLoss/dP1, dLoss/dP2.  Path costs are recomputed per
//    direction instead of being stored for all 8.
//  * views_backward: one warp per (pixel, 32-label chunk); dC/dI_ref = w_l2 sum sign(I_ref - B),
//    dC/dI_v(tap) = -w_l2 sign(.) w_tap (taps clamped as in the forward); lanes of one bilinear
//    cell are summed by a segmented shuffle and added to the view with four atomics per cell.
//    The census term is piecewise constant and has no gradient.
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

constexpr int kBwdWarps = 4;

// gc with its sign flipped where e > 0 (the sign bit of e is clear): gc * sign(-e) for e != 0.
__device__ __forceinline__ float sign_of_neg(float gc, float e) {
    return __int_as_float(__float_as_int(gc) ^ (~__float_as_int(e) & 0x80000000));
}

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per pixel, lane j on window slot j (wider windows in 32-slot chunks): the minimum by
// redux.sync, the softmax normaliser z and sum_j w_j j by warp sums, both rows written coalesced.
__global__ void __launch_bounds__(256) softargmin_backward_kernel(const float *__restrict__ agg,
                                                                  const int *__restrict__ lo,
                                                                  const int *__restrict__ cnt,
                                                                  const long long *__restrict__ off, int N, int G,
                                                                  double dmin, double step, float tau,
                                                                  const float *__restrict__ gdisp,
                                                                  float *__restrict__ gCs, float *__restrict__ gcost,
                                                                  int *__restrict__ status) {
    const int lane = threadIdx.x & 31;
    const long long p = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (p >= N) return;
    const long long o = off[p];
    const int n = cnt[p], l = lo[p];
    if (!window_ok(l, n, G, off[p + 1] - o, lane == 0 ? status : nullptr)) return;   // uniform per warp
    const int npad = (int)min((long long)((n + 3) & ~3), off[p + 1] - o);
    const float *s = agg + o;
    const float it = 1.f / tau;
    const float INF = __int_as_float(0x7f800000);
    float mn = INF;
    for (int j = lane; j < n; j += 32) mn = fminf(mn, __ldg(s + j));
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(mn) : "f"(mn));
    // FP32 weights after subtracting the minimum; d_g - dhat = (j - jbar) * step
    float z = 0.f, num = 0.f;
    for (int j = lane; j < n; j += 32) {
        const float w = expf((mn - __ldg(s + j)) * it);
        z += w;
        num = fmaf(w, (float)j, num);
    }
    z = warp_sum(z);
    num = warp_sum(num);
    const float jbar = num / z;
    const float k = gdisp[p] * (-it) * (float)step / z;
    for (int j = lane; j < npad; j += 32) {
        const float g = j < n ? k * expf((mn - __ldg(s + j)) * it) * ((float)j - jbar) : 0.f;
        gCs[o + j] = g;
        gcost[o + j] = 0.f;
    }
}

// Branch codes: 0 same label, 1 label-1 (+P1), 2 label+1 (+P1), 3 m+P2, 4 path start.
__global__ void __launch_bounds__(32 * kBwdWarps) sgm_backward_kernel(
    const float *__restrict__ cost, const int *__restrict__ lo, const int *__restrict__ cnt,
    const long long *__restrict__ off, int H, int W, int G, int Gs, float P1, float P2, ScanTable st,
    const float *__restrict__ gCs, unsigned char *__restrict__ codes, int *__restrict__ amin, size_t nnz_cap,
    float *__restrict__ gcost, float *__restrict__ gP, int *__restrict__ status,
    const int *__restrict__ order, int recompute) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kBwdWarps + wib;
    if (gw >= st.cum[st.paths]) return;
    const int rs = __ldg(order + gw);            // longest scanlines first
    const int r = rs & 15, s = rs >> 4;
    const int dx = dir_dx(r), dy = dir_dy(r);
    int x0, y0;
    scan_start(r, s, H, W, x0, y0);
    const int len = scan_steps(x0, y0, dx, dy, H, W);
    unsigned char *code = codes + (size_t)r * nnz_cap;
    int *am = amin + (size_t)r * H * W;
    float *bufA = sm + (size_t)wib * 4 * Gs;   // forward: predecessor's L;  reverse: incoming adjoint of p
    float *bufB = bufA + Gs;                   // forward: this pixel's L;    reverse: incoming adjoint of q
    float *lam = bufB + Gs;                    // reverse: lambda of p by slot
    unsigned char *cds = (unsigned char *)(lam + Gs);
    const float INF = __int_as_float(0x7f800000);

    // window metadata of 32 steps per lane: (lo | cnt << 16), 0 for an invalid window, and the
    // row offset in units of 4 slots; the next block is fetched one block ahead
    const long long p0 = (long long)y0 * W + x0, dpix = (long long)dy * W + dx;
    auto fetch = [&](int kb, int &mw, int &mo, int *st_) {
        const int k = kb + lane;
        mw = 0;
        mo = 0;
        if (k >= 0 && k < len) {
            const long long p = p0 + (long long)k * dpix;
            const int l_ = __ldg(lo + p), n_ = __ldg(cnt + p);
            const long long o_ = __ldg(off + p);
            if (window_ok(l_, n_, G, __ldg(off + p + 1) - o_, st_) && (o_ & 3) == 0 && (o_ >> 2) < 0x7fffffff) {
                mw = l_ | (n_ << 16);
                mo = (int)(o_ >> 2);
            }
        }
    };

    // forward recompute: branch codes and argmin slots (recompute = 1; the library passes 0, as the
    // forward SGM's recording form writes them.  The path is kept: without it the compiler
    // allocates the reverse sweep differently and it ran 4 % slower, 0.708 vs 0.681 ms.)  Narrow
    // steps (this window and the predecessor's at most 32 labels) keep the predecessor row in
    // registers, one slot per lane, and take its neighbours by shuffles; wider ones use the rows in
    // shared memory.
    int plo = 0, pn = 0;
    float m = 0.f;
    bool first = true;
    float prev = INF;                          // predecessor row by slot (narrow form)
    bool in_smem = false;                      // the predecessor row is in bufA (general form)
    int cw, co, nw = 0, no = 0;
    fetch(0, cw, co, status);
    if (len > 32) fetch(32, nw, no, status);
    for (int k = 0; k < (recompute ? len : 0); k++) {
        const int kk = k & 31;
        if (kk == 0 && k > 0) {
            cw = nw;
            co = no;
            if (k + 32 < len) fetch(k + 32, nw, no, status);
        }
        const int win = __shfl_sync(0xffffffffu, cw, kk), ofs = __shfl_sync(0xffffffffu, co, kk);
        const int p = (int)(p0 + (long long)k * dpix);
        const int l = win & 0xffff, n = win >> 16;
        const long long o = 4ll * ofs;
        if (n == 0) {
            first = true;
            continue;
        }
        if (n <= 32 && (first || pn <= 32)) {
            if (!first && in_smem) prev = lane < pn ? bufA[lane] : INF;
            const float c = lane < n ? __ldg(cost + o + lane) : 0.f;
            float Lv = c;
            unsigned cd = 4;
            if (!first) {
                // the same candidates in the same order as the general form: P2, same, g-1, g+1
                const int i = lane + (l - plo);
                const float v0 = __shfl_sync(0xffffffffu, prev, i & 31);
                const float vm = __shfl_sync(0xffffffffu, prev, (i - 1) & 31);
                const float vp = __shfl_sync(0xffffffffu, prev, (i + 1) & 31);
                float t = m + P2;
                cd = 3;
                if ((unsigned)i < (unsigned)pn && v0 < t) { t = v0; cd = 0; }
                if ((unsigned)(i - 1) < (unsigned)pn && vm + P1 < t) { t = vm + P1; cd = 1; }
                if ((unsigned)(i + 1) < (unsigned)pn && vp + P1 < t) { t = vp + P1; cd = 2; }
                Lv = c + (t - m);
            }
            if (lane < n) code[o + lane] = (unsigned char)cd;
            const float bv = lane < n ? Lv : INF;
            float mv;
            asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(mv) : "f"(bv));
            const int slot = __reduce_min_sync(0xffffffffu, bv == mv ? (unsigned)lane : 0x7fffffffu);
            if (lane == 0) am[p] = slot;
            m = mv;
            prev = bv;
            in_smem = false;
            plo = l;
            pn = n;
            first = false;
            continue;
        }
        if (!first && !in_smem) {
            if (lane < pn) bufA[lane] = prev;
            __syncwarp();
        }
        float bv = INF;
        int bj = 0x7fffffff;
        // eight 32-label chunks per round: their cost loads are in flight together
        for (int j0 = lane; j0 < n; j0 += 256) {
        float cv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) cv[u] = j0 + 32 * u < n ? __ldg(cost + o + j0 + 32 * u) : 0.f;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int j = j0 + 32 * u;
            if (j >= n) break;
            const float c = cv[u];
            float Lv;
            unsigned char cd = 4;
            if (first) {
                Lv = c;
            } else {
                const int i = l + j - plo;
                float t = m + P2;
                cd = 3;
                if ((unsigned)i < (unsigned)pn && bufA[i] < t) { t = bufA[i]; cd = 0; }
                if ((unsigned)(i - 1) < (unsigned)pn && bufA[i - 1] + P1 < t) { t = bufA[i - 1] + P1; cd = 1; }
                if ((unsigned)(i + 1) < (unsigned)pn && bufA[i + 1] + P1 < t) { t = bufA[i + 1] + P1; cd = 2; }
                Lv = c + (t - m);
            }
            bufB[j] = Lv;
            code[o + j] = cd;
            if (Lv < bv) { bv = Lv; bj = j; }
        }
        }
        // minimum and its lowest slot
        float mv;
        asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(mv) : "f"(bv));
        const int cand = (bv == mv) ? bj : 0x7fffffff;
        const int slot = __reduce_min_sync(0xffffffffu, (unsigned)cand);
        if (lane == 0) am[p] = slot;
        m = mv;
        __syncwarp();
        float *tmp = bufA;
        bufA = bufB;
        bufB = tmp;
        in_smem = true;
        plo = l;
        pn = n;
        first = false;
    }
    __syncwarp();

    // reverse sweep (blocks of metadata in descending order; step k-1 is in this block or the one below)
    float gp1 = 0.f, gp2 = 0.f;
    bool have_inc = false;       // the current pixel has an incoming adjoint (from its successor)
    bool inc_smem = false;       // ... held in bufA by slot (general form), else in inc, one slot per lane
    float inc = 0.f;
    // the argmin slot of each step of a block, fetched with its metadata (written above by this warp)
    auto fetch_am = [&](int kb) {
        const int kq = kb + lane;
        return (kq >= 0 && kq < len) ? am[(int)(p0 + (long long)kq * dpix)] : 0;
    };
    int ca = 0, na = 0;
    {
        const int kb0 = (len - 1) & ~31;
        fetch(kb0, cw, co, nullptr);
        ca = fetch_am(kb0);
        if (kb0 >= 32) {
            fetch(kb0 - 32, nw, no, nullptr);
            na = fetch_am(kb0 - 32);
        }
    }
    // the dLoss/dC_s row and branch codes of narrow windows, loaded two steps ahead: pf1 for step
    // k - 1, pf2 for step k - 2
    bool pf1_ok = false, pf2_ok = false;
    float pf1_g = 0.f, pf2_g = 0.f;
    unsigned pf1_c = 4u, pf2_c = 4u;
    for (int k = len - 1; k >= 0; k--) {
        const int kb = k & ~31, kk = k & 31;
        if (kk == 31 && k < len - 1) {       // entered a lower block
            cw = nw;
            co = no;
            ca = na;
            if (kb >= 32) {
                fetch(kb - 32, nw, no, nullptr);
                na = fetch_am(kb - 32);
            }
        }
        const bool have_pf = pf1_ok;
        const float pre_g = pf1_g;
        const unsigned pre_c = pf1_c;
        pf1_ok = pf2_ok;
        pf1_g = pf2_g;
        pf1_c = pf2_c;
        pf2_ok = false;
        if (k >= 2) {
            // step k - 2: this block, or lane 30 / 31 of the block below
            const int w2 = __shfl_sync(0xffffffffu, kk >= 2 ? cw : nw, (kk + 30) & 31);
            const int o2 = __shfl_sync(0xffffffffu, kk >= 2 ? co : no, (kk + 30) & 31);
            const int n2 = w2 >> 16;
            if (n2 > 0 && n2 <= 32) {
                pf2_g = lane < n2 ? __ldg(gCs + 4ll * o2 + lane) : 0.f;
                pf2_c = lane < n2 ? (unsigned)__ldg(code + 4ll * o2 + lane) : 4u;
                pf2_ok = true;
            }
        }
        const int win = __shfl_sync(0xffffffffu, cw, kk), ofs = __shfl_sync(0xffffffffu, co, kk);
        // predecessor on the path: step k - 1 (this block, or lane 31 of the block below)
        const int wq = __shfl_sync(0xffffffffu, kk > 0 ? cw : nw, (kk + 31) & 31);
        const int l = win & 0xffff, n = win >> 16;
        const long long o = 4ll * ofs;
        if (n == 0) {
            have_inc = false;
            continue;
        }
        int q = -1, ql = 0, qn = 0;
        if (k > 0 && (wq >> 16) != 0) {
            q = (int)(p0 + (long long)(k - 1) * dpix);
            ql = wq & 0xffff;
            qn = wq >> 16;
        }
        if (n <= 32 && qn <= 32) {
            // narrow: lambda and the branch code of slot j on lane j; q's incoming adjoint by shuffles
            const bool act = lane < n;
            float in_v = 0.f;
            if (have_inc) in_v = inc_smem ? (act ? bufA[lane] : 0.f) : inc;
            const float gv = have_pf ? pre_g : (act ? __ldg(gCs + o + lane) : 0.f);
            const unsigned cd = have_pf ? pre_c : (act ? (unsigned)code[o + lane] : 4u);
            const float lv = act ? gv + in_v : 0.f;
            if (act) atomicAdd(gcost + o + lane, lv);
            if (cd == 1 || cd == 2) gp1 += lv;
            if (cd == 3) gp2 += lv;
            const float dm = warp_sum((cd == 3 ? lv : 0.f) - lv);
            if (q >= 0) {
                const int qa = __shfl_sync(0xffffffffu, kk > 0 ? ca : na, (kk + 31) & 31);
                const int j0 = lane + (ql - l), j1 = j0 + 1, j2 = j0 - 1;
                const float l0 = __shfl_sync(0xffffffffu, lv, j0 & 31), l1 = __shfl_sync(0xffffffffu, lv, j1 & 31);
                const float l2 = __shfl_sync(0xffffffffu, lv, j2 & 31);
                const unsigned c0 = __shfl_sync(0xffffffffu, cd, j0 & 31), c1 = __shfl_sync(0xffffffffu, cd, j1 & 31);
                const unsigned c2 = __shfl_sync(0xffffffffu, cd, j2 & 31);
                float v = 0.f;
                if ((unsigned)j0 < (unsigned)n && c0 == 0) v += l0;
                if ((unsigned)j1 < (unsigned)n && c1 == 1) v += l1;
                if ((unsigned)j2 < (unsigned)n && c2 == 2) v += l2;
                if (lane == qa) v += dm;
                inc = lane < qn ? v : 0.f;
                inc_smem = false;
                have_inc = true;
            } else {
                have_inc = false;
            }
            continue;
        }
        if (have_inc && !inc_smem) {
            if (lane < n) bufA[lane] = inc;
            __syncwarp();
        }
        float dm = 0.f;
        for (int j0 = lane; j0 < n; j0 += 256) {
        float gv[8];
        unsigned char cv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const bool in = j0 + 32 * u < n;
            gv[u] = in ? __ldg(gCs + o + j0 + 32 * u) : 0.f;
            cv[u] = in ? code[o + j0 + 32 * u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int j = j0 + 32 * u;
            if (j >= n) break;
            const float lv = gv[u] + (have_inc ? bufA[j] : 0.f);
            atomicAdd(gcost + o + j, lv);
            const unsigned char cd = cv[u];
            lam[j] = lv;
            cds[j] = cd;
            if (cd == 1 || cd == 2) gp1 += lv;
            if (cd == 3) {
                gp2 += lv;
                dm += lv;
            }
            dm -= lv;
        }
        }
        dm = warp_sum(dm);
        __syncwarp();
        if (q >= 0) {
            // gather q's incoming adjoint: label h receives from p's labels h (same), h+1 (-1 branch), h-1 (+1 branch)
            const int qa = am[q];
            for (int i = lane; i < qn; i += 32) {
                const int h = ql + i;
                float v = 0.f;
                const int j0 = h - l, j1 = h + 1 - l, j2 = h - 1 - l;
                if ((unsigned)j0 < (unsigned)n && cds[j0] == 0) v += lam[j0];
                if ((unsigned)j1 < (unsigned)n && cds[j1] == 1) v += lam[j1];
                if ((unsigned)j2 < (unsigned)n && cds[j2] == 2) v += lam[j2];
                if (i == qa) v += dm;
                bufB[i] = v;
            }
            __syncwarp();
            float *tmp = bufA;
            bufA = bufB;
            bufB = tmp;
            have_inc = true;
            inc_smem = true;
        } else {
            have_inc = false;
        }
        __syncwarp();
    }
    gp1 = warp_sum(gp1);
    gp2 = warp_sum(gp2);
    if (lane == 0) {
        if (gp1 != 0.f) atomicAdd(gP, gp1);
        if (gp2 != 0.f) atomicAdd(gP + 1, gp2);
    }
}

// One warp per (pixel, 32-label chunk) item, lane = label: the lane's tap and bilinear sample are
// recomputed as in the forward (clamped taps), g = dLoss/dC * w_l2 * sign(I_ref - B) goes to the
// reference pixel and -g * (bilinear weight) to the four taps.  Lanes whose labels share a
// bilinear cell form contiguous runs (the integer shift is monotone in the label), so a segmented
// shuffle sum leaves each run's total in its first lane, which issues the four atomics.
// Colour (C > 1; images are planes view * C + c): the l2 term is the Euclidean norm of the colour
// difference delta, so channel c takes g_c = dLoss/dC * w_l2 * delta_c / ||delta|| (0 where
// delta = 0), and each channel's four taps are summed over the run the same way.
template <int C>
__global__ void __launch_bounds__(256) views_backward_kernel(const float *__restrict__ views,
                                                             const FineTap *__restrict__ tab, int G, int nviews,
                                                             int H, int W, int ref, const int *__restrict__ lo,
                                                             const int *__restrict__ cnt,
                                                             const long long *__restrict__ off, float wl2,
                                                             const float *__restrict__ gcost,
                                                             float *__restrict__ gviews, const int2 *__restrict__ list,
                                                             const int *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const size_t N = (size_t)H * W;
    const int total = *count;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < total; it += warps) {
        const int2 item = list[it];
        const int p = item.x, chunk = item.y;
        const int l0 = __ldg(lo + p), n = __ldg(cnt + p);
        const long long o = __ldg(off + p);
        if (!window_ok(l0, n, G, __ldg(off + p + 1) - o, nullptr)) continue;   // uniform per item
        const int j = chunk * 32 + lane;
        const bool act = j < n;
        const int x = p % W, y = p / W;
        float Iref[C], gref[C];
#pragma unroll
        for (int ch = 0; ch < C; ch++) {
            Iref[ch] = __ldg(views + ((size_t)ref * C + ch) * N + p);
            gref[ch] = 0.f;
        }
        const float gc = act ? wl2 * __ldg(gcost + o + j) : 0.f;
        for (int vi = 0; vi < nviews - 1; vi++) {
            const int view = vi + (vi >= ref);
            FineTap t;
            t.ox = t.oy = 0;
            t.fx = t.fy = 0.f;
            if (act) t = load_tap(tab + (size_t)view * G + l0 + j);
            const int x0 = min(max(x + t.ox, 0), W - 1), x1 = min(max(x + t.ox + 1, 0), W - 1);
            const int y0 = min(max(y + t.oy, 0), H - 1), y1 = min(max(y + t.oy + 1, 0), H - 1);
            float g[C];
#pragma unroll
            for (int ch = 0; ch < C; ch++) g[ch] = 0.f;
            if (act && gc != 0.f) {
                float dl[C], sq = 0.f;
#pragma unroll
                for (int ch = 0; ch < C; ch++) {
                    const float *I = views + ((size_t)view * C + ch) * N;
                    const float top = (1.f - t.fx) * __ldg(I + y0 * W + x0) + t.fx * __ldg(I + y0 * W + x1);
                    const float bot = (1.f - t.fx) * __ldg(I + y1 * W + x0) + t.fx * __ldg(I + y1 * W + x1);
                    dl[ch] = Iref[ch] - ((1.f - t.fy) * top + t.fy * bot);
                    sq = fmaf(dl[ch], dl[ch], sq);
                }
                if (C == 1) {
                    g[0] = dl[0] > 0.f ? gc : (dl[0] < 0.f ? -gc : 0.f);
                } else if (sq > 0.f) {
                    const float nrm = sqrtf(sq);
#pragma unroll
                    for (int ch = 0; ch < C; ch++) g[ch] = gc * (dl[ch] / nrm);
                }
            }
            // runs of equal bilinear cells; inactive lanes (the chunk's tail) form their own run
            const int key = act ? (((int)t.oy << 16) ^ ((int)t.ox & 0xffff)) : 0x7fffffff;
            const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
            const bool head = lane == 0 || key != kprev;
            const unsigned heads = __ballot_sync(0xffffffffu, head);
            const unsigned later = lane == 31 ? 0u : (heads & (0xfffffffeu << lane));
            const int end = later ? __ffs(later) - 2 : 31;
#pragma unroll
            for (int ch = 0; ch < C; ch++) {
                gref[ch] += g[ch];
                float a00 = -g[ch] * (1.f - t.fy) * (1.f - t.fx), a10 = -g[ch] * (1.f - t.fy) * t.fx;
                float a01 = -g[ch] * t.fy * (1.f - t.fx), a11 = -g[ch] * t.fy * t.fx;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const float b00 = __shfl_down_sync(0xffffffffu, a00, d);
                    const float b10 = __shfl_down_sync(0xffffffffu, a10, d);
                    const float b01 = __shfl_down_sync(0xffffffffu, a01, d);
                    const float b11 = __shfl_down_sync(0xffffffffu, a11, d);
                    if (lane + d <= end) {
                        a00 += b00;
                        a10 += b10;
                        a01 += b01;
                        a11 += b11;
                    }
                }
                if (head && act) {
                    float *gI = gviews + ((size_t)view * C + ch) * N;
                    if (a00 != 0.f) atomicAdd(gI + y0 * W + x0, a00);
                    if (a10 != 0.f) atomicAdd(gI + y0 * W + x1, a10);
                    if (a01 != 0.f) atomicAdd(gI + y1 * W + x0, a01);
                    if (a11 != 0.f) atomicAdd(gI + y1 * W + x1, a11);
                }
            }
        }
#pragma unroll
        for (int ch = 0; ch < C; ch++) {
            const float gr = warp_sum(gref[ch]);
            if (lane == 0 && gr != 0.f) atomicAdd(gviews + ((size_t)ref * C + ch) * N + p, gr);
        }
    }
}

// Narrow windows by rows, as the forward's row kernel: a CTA of kVrWarps warps covers kVrWarps
// consecutive rows of one 32-pixel column, a warp one row (lane = pixel) and the KVR-label range
// [g0, g0 + KVR) that holds the most of its windows; the windows outside it go to the item list.
// For a view, the range splits into segments where the bilinear cell (integer shift) changes;
// inside a segment of labels t = 0, 1, ... the fractional shift is fx + ax t, fy + ay t, so
//   - the sample minus I_ref is the quadratic a0 + b0 t + Cq t^2 (from the cell's four taps), and
//     its sign gives g(t) = dLoss/dC * w_l2 * sign(I_ref - sample) for the reference pixel;
//   - a corner's tap gradient -sum_t g(t) w_corner(t) is a combination of the moments sum g,
//     sum g t, sum g t^2 (the corner weights are products of fx + ax t and fy + ay t),
// so a lane adds three moments per label and converts them into four tap gradients once per
// segment.  The tap gradients of the CTA go into one shared-memory box over its tap footprint,
// added to the view with one global atomic per non-zero element once the view is done.  Taps
// outside the box (clamped at the image border, or a label range too wide for it) go to global
// memory directly.
constexpr int kVrWarps = 8, KVR = 36, kVrBoxW = 96, kVrBoxH = 24;

__global__ void __launch_bounds__(32 * kVrWarps) views_backward_rows_kernel(
    const float *__restrict__ views, const FineTap *__restrict__ tab, int G, int U, int V, int H, int W, int ref,
    const int *__restrict__ lo, const int *__restrict__ cnt, const long long *__restrict__ off, float wl2,
    float fstep, const float *__restrict__ gcost, float *__restrict__ gviews, int2 *__restrict__ list,
    int *__restrict__ list_count) {
    __shared__ float box[kVrBoxH * kVrBoxW];
    __shared__ float gcs[kVrWarps][KVR][32];       // [row][label of the range][lane]
    __shared__ int red[2][kVrWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 32, ty0 = blockIdx.y * kVrWarps;
    const int x = x0 + lane, y = ty0 + w;
    const size_t N = (size_t)H * W;
    const int nviews = U * V;
    int l = 0, n = 0;
    long long o = 0;
    bool nar = false;
    if (x < W && y < H) {
        const size_t p = (size_t)y * W + x;
        l = __ldg(lo + p);
        n = __ldg(cnt + p);
        o = __ldg(off + p);
        nar = n <= 32 && window_ok(l, n, G, __ldg(off + p + 1) - o, nullptr);
    }
    int g0;
    const int best = row_range<KVR>(l, n, nar, g0);  // warp-uniform (rows past H: no window, -1)
    const bool fits = best > 0 && nar && l >= g0 && l + n <= g0 + KVR;
    if (nar && !fits) push_chunks(list, list_count, y * W + x, n);
#pragma unroll 4
    for (int j = 0; j < KVR; j++) {
        const int k = g0 + j - l;
        gcs[w][j][lane] = (fits && k >= 0 && k < n) ? wl2 * __ldg(gcost + o + k) : 0.f;
    }
    if (lane == 0) {
        red[0][w] = best > 0 ? g0 : 0x7fffffff;
        red[1][w] = best > 0 ? min(g0 + KVR - 1, G - 1) : -1;
    }
    for (int e = threadIdx.x; e < kVrBoxH * kVrBoxW; e += blockDim.x) box[e] = 0.f;
    __syncthreads();
    int gmn = red[0][0], gmx = red[1][0];
    for (int k = 1; k < kVrWarps; k++) {
        gmn = min(gmn, red[0][k]);
        gmx = max(gmx, red[1][k]);
    }
    if (gmx < 0) return;                               // no range in the CTA (uniform)
    const bool any = best > 0;                         // warp-uniform
    const float Iref = fits ? __ldg(views + (size_t)ref * N + (size_t)y * W + x) : 0.f;
    float gref = 0.f;
    for (int view = 0; view < nviews; view++) {
        if (view == ref) continue;
        const float ax = (float)(view % U - (ref % U)) * fstep, ay = (float)(view / U - (ref / U)) * fstep;
        const FineTap ta = load_tap(tab + (size_t)view * G + gmn), tb = load_tap(tab + (size_t)view * G + gmx);
        const int bx0 = x0 + min(ta.ox, tb.ox), by0 = ty0 + min(ta.oy, tb.oy);
        const int bw = 32 + abs(tb.ox - ta.ox) + 1, bh = kVrWarps + abs(tb.oy - ta.oy) + 1;
        const bool use_box = bw <= kVrBoxW && bh <= kVrBoxH;
        const float *I = views + (size_t)view * N;
        float *gI = gviews + (size_t)view * N;
        auto add = [&](int xc, int yc, float v) {
            if (v == 0.f) return;
            const int bx = xc - bx0, by = yc - by0;
            if (use_box && (unsigned)bx < (unsigned)bw && (unsigned)by < (unsigned)bh)
                atomicAdd(&box[by * kVrBoxW + bx], v);
            else
                atomicAdd(gI + (size_t)yc * W + xc, v);
        };
        if (any) {
            // the range's labels: lane j holds label g0 + j, lanes 0 .. KVR-33 also label g0 + 32 + lane
            const FineTap t0 = load_tap(tab + (size_t)view * G + min(g0 + lane, G - 1));
            FineTap t1 = t0;
            if (lane < KVR - 32) t1 = load_tap(tab + (size_t)view * G + min(g0 + 32 + lane, G - 1));
            const int c0 = (int)t0.ox * 65536 + (int)t0.oy, c1 = (int)t1.ox * 65536 + (int)t1.oy;
            const int p0 = __shfl_up_sync(0xffffffffu, c0, 1), p1 = __shfl_up_sync(0xffffffffu, c1, 1);
            const int c31 = __shfl_sync(0xffffffffu, c0, 31);
            const unsigned m0 = __ballot_sync(0xffffffffu, lane == 0 || c0 != p0);
            const unsigned m1 = __ballot_sync(0xffffffffu, lane < KVR - 32 && (lane == 0 ? c1 != c31 : c1 != p1));
            // segments of the range in label order
            int js = 0;
            while (js < KVR) {
                const int nx = js + 1;
                const unsigned r0 = nx < 32 ? (m0 & (0xffffffffu << nx)) : 0u;
                const unsigned r1 = nx < 32 ? m1 : (m1 & (0xffffffffu << (nx - 32)));
                const int je = r0 ? __ffs(r0) - 1 : (r1 ? 32 + __ffs(r1) - 1 : KVR);
                // the segment's cell and fractions (label js, from the lane that holds it)
                const int src = js & 31;
                const bool hi = js >= 32;
                const int ox = __shfl_sync(0xffffffffu, hi ? t1.ox : t0.ox, src);
                const int oy = __shfl_sync(0xffffffffu, hi ? t1.oy : t0.oy, src);
                const float fx = __shfl_sync(0xffffffffu, hi ? t1.fx : t0.fx, src);
                const float fy = __shfl_sync(0xffffffffu, hi ? t1.fy : t0.fy, src);
                const int xa = min(max(x + ox, 0), W - 1), xb = min(max(x + ox + 1, 0), W - 1);
                const int ya = min(max(y + oy, 0), H - 1), yb = min(max(y + oy + 1, 0), H - 1);
                float S0 = 0.f, S1 = 0.f, S2 = 0.f;
                if (fits) {
                    const float i00 = __ldg(I + (size_t)ya * W + xa), i10 = __ldg(I + (size_t)ya * W + xb);
                    const float i01 = __ldg(I + (size_t)yb * W + xa), i11 = __ldg(I + (size_t)yb * W + xb);
                    const float cx = i10 - i00, cy = i01 - i00, cxy = (i11 - i01) - cx;
                    const float a0 = fmaf(cxy * fx, fy, fmaf(cy, fy, fmaf(cx, fx, i00 - Iref)));
                    const float b0 = fmaf(cxy, fmaf(fx, ay, fy * ax), fmaf(cy, ay, cx * ax));
                    const float cq = cxy * ax * ay;
                    // two interleaved sets of moments (even and odd labels) for instruction-level parallelism
                    float T0 = 0.f, T1 = 0.f, T2 = 0.f;
                    float t = 0.f;
                    int j = js;
                    for (; j + 1 < je; j += 2, t += 2.f) {
                        const float gc0 = gcs[w][j][lane], gc1 = gcs[w][j + 1][lane];
                        const float t1 = t + 1.f;
                        const float e0 = fmaf(t, fmaf(t, cq, b0), a0), e1 = fmaf(t1, fmaf(t1, cq, b0), a0);
                        const float g0 = e0 != 0.f ? sign_of_neg(gc0, e0) : 0.f;
                        const float g1 = e1 != 0.f ? sign_of_neg(gc1, e1) : 0.f;
                        const float gt0 = g0 * t, gt1 = g1 * t1;
                        S0 += g0;
                        S1 += gt0;
                        S2 = fmaf(gt0, t, S2);
                        T0 += g1;
                        T1 += gt1;
                        T2 = fmaf(gt1, t1, T2);
                    }
                    if (j < je) {
                        const float gc = gcs[w][j][lane];
                        const float e = fmaf(t, fmaf(t, cq, b0), a0);        // sample - I_ref
                        const float g = e != 0.f ? sign_of_neg(gc, e) : 0.f;
                        const float gt = g * t;
                        S0 += g;
                        S1 += gt;
                        S2 = fmaf(gt, t, S2);
                    }
                    S0 += T0;
                    S1 += T1;
                    S2 += T2;
                    gref += S0;
                    if (S0 != 0.f || S1 != 0.f || S2 != 0.f) {
                        // -sum g w for the corners: w11 = XY, w10 = X (1 - Y), w01 = (1 - X) Y, w00 = (1 - X)(1 - Y)
                        const float GX = fmaf(ax, S1, fx * S0), GY = fmaf(ay, S1, fy * S0);
                        const float GXY = fmaf(ax * ay, S2, fmaf(fmaf(fx, ay, fy * ax), S1, fx * fy * S0));
                        const float v00 = -(S0 - GX - GY + GXY), v10 = -(GX - GXY), v01 = -(GY - GXY), v11 = -GXY;
                        const int bxa = xa - bx0, bya = ya - by0;
                        if (use_box && (unsigned)bxa < (unsigned)bw && (unsigned)(xb - bx0) < (unsigned)bw &&
                            (unsigned)bya < (unsigned)bh && (unsigned)(yb - by0) < (unsigned)bh) {
                            // the whole cell in the box: four shared-memory adds
                            float *c00 = box + bya * kVrBoxW + bxa;
                            const int dxb = xb - xa, dyb = (yb - ya) * kVrBoxW;
                            atomicAdd(c00, v00);
                            atomicAdd(c00 + dxb, v10);
                            atomicAdd(c00 + dyb, v01);
                            atomicAdd(c00 + dyb + dxb, v11);
                        } else {
                            add(xa, ya, v00);
                            add(xb, ya, v10);
                            add(xa, yb, v01);
                            add(xb, yb, v11);
                        }
                    }
                }
                js = je;
            }
        }
        __syncthreads();
        if (use_box) {
            // a warp per box row, lanes along it
            for (int by = w; by < bh; by += kVrWarps) {
                float *brow = box + by * kVrBoxW;
                float *grow = gI + (size_t)(by0 + by) * W + bx0;
                for (int bx = lane; bx < bw; bx += 32) {
                    const float v = brow[bx];
                    if (v != 0.f) {
                        atomicAdd(grow + bx, v);
                        brow[bx] = 0.f;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (fits && gref != 0.f) atomicAdd(gviews + (size_t)ref * N + (size_t)y * W + x, gref);
}

// Colour form of the rows kernel (C = 3, planar views [view * 3 + c]).  The l2 term is the norm of
// the colour difference, so label t gives channel c the gradient g_c = dLoss/dC * w_l2 * Delta_c /
// |Delta| (0 where the colours agree), Delta_c = I_ref,c - sample_c = -e_c(t) with e_c the
// channel's sample-minus-reference quadratic; each channel keeps its own three moments and its own
// shared-memory box.  Four warps (rows) per CTA, so that the three boxes and the labels' dLoss/dC
// fit the 48 KB of static shared memory.
constexpr int kVrWarpsRgb = 4;

__global__ void __launch_bounds__(32 * kVrWarpsRgb) views_backward_rows_rgb_kernel(
    const float *__restrict__ views, const FineTap *__restrict__ tab, int G, int U, int V, int H, int W, int ref,
    const int *__restrict__ lo, const int *__restrict__ cnt, const long long *__restrict__ off, float wl2,
    float fstep, const float *__restrict__ gcost, float *__restrict__ gviews, int2 *__restrict__ list,
    int *__restrict__ list_count) {
    constexpr int C = 3, NW = kVrWarpsRgb;
    __shared__ float box[C][kVrBoxH * kVrBoxW];
    __shared__ float gcs[NW][KVR][32];             // [row][label of the range][lane]
    __shared__ int red[2][NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x0 = blockIdx.x * 32, ty0 = blockIdx.y * NW;
    const int x = x0 + lane, y = ty0 + w;
    const size_t N = (size_t)H * W;
    const int nviews = U * V;
    int l = 0, n = 0;
    long long o = 0;
    bool nar = false;
    if (x < W && y < H) {
        const size_t p = (size_t)y * W + x;
        l = __ldg(lo + p);
        n = __ldg(cnt + p);
        o = __ldg(off + p);
        nar = n <= 32 && window_ok(l, n, G, __ldg(off + p + 1) - o, nullptr);
    }
    int g0;
    const int best = row_range<KVR>(l, n, nar, g0);  // warp-uniform (rows past H: no window, -1)
    const bool fits = best > 0 && nar && l >= g0 && l + n <= g0 + KVR;
    if (nar && !fits) push_chunks(list, list_count, y * W + x, n);
#pragma unroll 4
    for (int j = 0; j < KVR; j++) {
        const int k = g0 + j - l;
        gcs[w][j][lane] = (fits && k >= 0 && k < n) ? wl2 * __ldg(gcost + o + k) : 0.f;
    }
    if (lane == 0) {
        red[0][w] = best > 0 ? g0 : 0x7fffffff;
        red[1][w] = best > 0 ? min(g0 + KVR - 1, G - 1) : -1;
    }
    for (int e = threadIdx.x; e < C * kVrBoxH * kVrBoxW; e += blockDim.x) (&box[0][0])[e] = 0.f;
    __syncthreads();
    int gmn = red[0][0], gmx = red[1][0];
    for (int k = 1; k < NW; k++) {
        gmn = min(gmn, red[0][k]);
        gmx = max(gmx, red[1][k]);
    }
    if (gmx < 0) return;                               // no range in the CTA (uniform)
    const bool any = best > 0;                         // warp-uniform
    float Iref[C], gref[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        Iref[c] = fits ? __ldg(views + ((size_t)ref * C + c) * N + (size_t)y * W + x) : 0.f;
        gref[c] = 0.f;
    }
    for (int view = 0; view < nviews; view++) {
        if (view == ref) continue;
        const float ax = (float)(view % U - (ref % U)) * fstep, ay = (float)(view / U - (ref / U)) * fstep;
        const FineTap ta = load_tap(tab + (size_t)view * G + gmn), tb = load_tap(tab + (size_t)view * G + gmx);
        const int bx0 = x0 + min(ta.ox, tb.ox), by0 = ty0 + min(ta.oy, tb.oy);
        const int bw = 32 + abs(tb.ox - ta.ox) + 1, bh = NW + abs(tb.oy - ta.oy) + 1;
        const bool use_box = bw <= kVrBoxW && bh <= kVrBoxH;
        const float *I = views + (size_t)view * C * N;             // channel c at + c N
        float *gI = gviews + (size_t)view * C * N;
        if (any) {
            // the range's labels: lane j holds label g0 + j, lanes 0 .. KVR-33 also label g0 + 32 + lane
            const FineTap t0 = load_tap(tab + (size_t)view * G + min(g0 + lane, G - 1));
            FineTap t1 = t0;
            if (lane < KVR - 32) t1 = load_tap(tab + (size_t)view * G + min(g0 + 32 + lane, G - 1));
            const int c0 = (int)t0.ox * 65536 + (int)t0.oy, c1 = (int)t1.ox * 65536 + (int)t1.oy;
            const int p0 = __shfl_up_sync(0xffffffffu, c0, 1), p1 = __shfl_up_sync(0xffffffffu, c1, 1);
            const int c31 = __shfl_sync(0xffffffffu, c0, 31);
            const unsigned m0 = __ballot_sync(0xffffffffu, lane == 0 || c0 != p0);
            const unsigned m1 = __ballot_sync(0xffffffffu, lane < KVR - 32 && (lane == 0 ? c1 != c31 : c1 != p1));
            int js = 0;
            while (js < KVR) {
                const int nx = js + 1;
                const unsigned r0 = nx < 32 ? (m0 & (0xffffffffu << nx)) : 0u;
                const unsigned r1 = nx < 32 ? m1 : (m1 & (0xffffffffu << (nx - 32)));
                const int je = r0 ? __ffs(r0) - 1 : (r1 ? 32 + __ffs(r1) - 1 : KVR);
                const int src = js & 31;
                const bool hi = js >= 32;
                const int ox = __shfl_sync(0xffffffffu, hi ? t1.ox : t0.ox, src);
                const int oy = __shfl_sync(0xffffffffu, hi ? t1.oy : t0.oy, src);
                const float fx = __shfl_sync(0xffffffffu, hi ? t1.fx : t0.fx, src);
                const float fy = __shfl_sync(0xffffffffu, hi ? t1.fy : t0.fy, src);
                const int xa = min(max(x + ox, 0), W - 1), xb = min(max(x + ox + 1, 0), W - 1);
                const int ya = min(max(y + oy, 0), H - 1), yb = min(max(y + oy + 1, 0), H - 1);
                if (fits) {
                    float a0[C], b0[C], cq[C], S0[C], S1[C], S2[C];
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        const float *Ic = I + (size_t)c * N;
                        const float i00 = __ldg(Ic + (size_t)ya * W + xa), i10 = __ldg(Ic + (size_t)ya * W + xb);
                        const float i01 = __ldg(Ic + (size_t)yb * W + xa), i11 = __ldg(Ic + (size_t)yb * W + xb);
                        const float cx = i10 - i00, cy = i01 - i00, cxy = (i11 - i01) - cx;
                        a0[c] = fmaf(cxy * fx, fy, fmaf(cy, fy, fmaf(cx, fx, i00 - Iref[c])));
                        b0[c] = fmaf(cxy, fmaf(fx, ay, fy * ax), fmaf(cy, ay, cx * ax));
                        cq[c] = cxy * ax * ay;
                        S0[c] = S1[c] = S2[c] = 0.f;
                    }
                    float t = 0.f;
                    for (int j = js; j < je; j++, t += 1.f) {
                        const float gc = gcs[w][j][lane];
                        float e[C], sq = 0.f;
#pragma unroll
                        for (int c = 0; c < C; c++) {
                            e[c] = fmaf(t, fmaf(t, cq[c], b0[c]), a0[c]);      // sample - I_ref
                            sq = fmaf(e[c], e[c], sq);
                        }
                        const float sc = sq > 0.f ? -gc * rsqrtf(sq) : 0.f;    // g_c = sc e_c
#pragma unroll
                        for (int c = 0; c < C; c++) {
                            const float g = sc * e[c], gt = g * t;
                            S0[c] += g;
                            S1[c] += gt;
                            S2[c] = fmaf(gt, t, S2[c]);
                        }
                    }
                    const int bxa = xa - bx0, bya = ya - by0;
                    const bool inbox = use_box && (unsigned)bxa < (unsigned)bw && (unsigned)(xb - bx0) < (unsigned)bw &&
                                       (unsigned)bya < (unsigned)bh && (unsigned)(yb - by0) < (unsigned)bh;
#pragma unroll
                    for (int c = 0; c < C; c++) {
                        gref[c] += S0[c];
                        if (S0[c] == 0.f && S1[c] == 0.f && S2[c] == 0.f) continue;
                        // -sum g w for the corners: w11 = XY, w10 = X (1 - Y), w01 = (1 - X) Y, w00 = (1 - X)(1 - Y)
                        const float GX = fmaf(ax, S1[c], fx * S0[c]), GY = fmaf(ay, S1[c], fy * S0[c]);
                        const float GXY = fmaf(ax * ay, S2[c], fmaf(fmaf(fx, ay, fy * ax), S1[c], fx * fy * S0[c]));
                        const float v00 = -(S0[c] - GX - GY + GXY), v10 = -(GX - GXY), v01 = -(GY - GXY), v11 = -GXY;
                        if (inbox) {
                            float *c00 = box[c] + bya * kVrBoxW + bxa;
                            const int dxb = xb - xa, dyb = (yb - ya) * kVrBoxW;
                            atomicAdd(c00, v00);
                            atomicAdd(c00 + dxb, v10);
                            atomicAdd(c00 + dyb, v01);
                            atomicAdd(c00 + dyb + dxb, v11);
                        } else {
                            float *g = gI + (size_t)c * N;
                            if (v00 != 0.f) atomicAdd(g + (size_t)ya * W + xa, v00);
                            if (v10 != 0.f) atomicAdd(g + (size_t)ya * W + xb, v10);
                            if (v01 != 0.f) atomicAdd(g + (size_t)yb * W + xa, v01);
                            if (v11 != 0.f) atomicAdd(g + (size_t)yb * W + xb, v11);
                        }
                    }
                }
                js = je;
            }
        }
        __syncthreads();
        if (use_box) {
            // a warp per box row (of each channel), lanes along it
            for (int r = w; r < C * bh; r += NW) {
                const int c = r / bh, by = r - c * bh;
                float *brow = box[c] + by * kVrBoxW;
                float *grow = gI + (size_t)c * N + (size_t)(by0 + by) * W + bx0;
                for (int bx = lane; bx < bw; bx += 32) {
                    const float v = brow[bx];
                    if (v != 0.f) {
                        atomicAdd(grow + bx, v);
                        brow[bx] = 0.f;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (fits) {
#pragma unroll
        for (int c = 0; c < C; c++)
            if (gref[c] != 0.f) atomicAdd(gviews + ((size_t)ref * C + c) * N + (size_t)y * W + x, gref[c]);
    }
}

}  // namespace

cudaError_t launch_softargmin_backward(cudaStream_t s, const float *agg, const int *lo, const int *cnt,
                                       const long long *off, int N, int G, double dmin, double step, float tau,
                                       const float *gdisp, float *gCs, float *gcost, int *status) {
    softargmin_backward_kernel<<<(unsigned)(((long long)N * 32 + 255) / 256), 256, 0, s>>>(
        agg, lo, cnt, off, N, G, dmin, step, tau, gdisp, gCs, gcost, status);
    return cudaGetLastError();
}

cudaError_t launch_sgm_backward(cudaStream_t s, const float *cost, const int *lo, const int *cnt, const long long *off,
                                int H, int W, int G, float P1, float P2, const float *gCs, unsigned char *codes,
                                int *amin, size_t nnz_cap, float *gcost, float *gP, int *status, const int *order, int paths,
                                bool recompute) {
    const ScanTable st = make_scan_table(H, W, paths);
    const int Gs = (G + 31) & ~31;
    const size_t smem = (size_t)kBwdWarps * 4 * Gs * sizeof(float);   // bufA, bufB, lambda, codes per warp
    const unsigned grid = (unsigned)((st.cum[paths] + kBwdWarps - 1) / kBwdWarps);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(sgm_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    sgm_backward_kernel<<<grid, 32 * kBwdWarps, smem, s>>>(cost, lo, cnt, off, H, W, G, Gs, P1, P2, st, gCs, codes,
                                                           amin, nnz_cap, gcost, gP, status, order, recompute ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_views_backward(cudaStream_t s, const float *views, const FineTap *tab, int G, int U, int V, int C,
                                  int H, int W, int ref, const int *lo, const int *cnt, const long long *off,
                                  float wl2, float fstep, const float *gcost, float *gviews, int2 *list, int *count) {
    const int nviews = U * V;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (C == 3) {
        dim3 grid((W + 31) / 32, (H + kVrWarpsRgb - 1) / kVrWarpsRgb);
        views_backward_rows_rgb_kernel<<<grid, 32 * kVrWarpsRgb, 0, s>>>(views, tab, G, U, V, H, W, ref, lo, cnt, off,
                                                                        wl2, fstep, gcost, gviews, list, count);
        return cudaGetLastError();
    }
    dim3 grid((W + 31) / 32, (H + kVrWarps - 1) / kVrWarps);
    views_backward_rows_kernel<<<grid, 32 * kVrWarps, 0, s>>>(views, tab, G, U, V, H, W, ref, lo, cnt, off, wl2,
                                                              fstep, gcost, gviews, list, count);
    return cudaGetLastError();
}

cudaError_t launch_views_backward_list(cudaStream_t s, const float *views, const FineTap *tab, int G, int nviews,
                                       int C, int H, int W, int ref, const int *lo, const int *cnt,
                                       const long long *off, float wl2, const float *gcost, float *gviews,
                                       const int2 *list, const int *count) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // windows wider than 32 labels and narrow ones outside their row's range (the list holds their chunks)
    if (C == 3)
        views_backward_kernel<3><<<sms * 8, 256, 0, s>>>(views, tab, G, nviews, H, W, ref, lo, cnt, off, wl2, gcost,
                                                         gviews, list, count);
    else
        views_backward_kernel<1><<<sms * 8, 256, 0, s>>>(views, tab, G, nviews, H, W, ref, lo, cnt, off, wl2, gcost,
                                                         gviews, list, count);
    return cudaGetLastError();
}

}  // namespace lfsgm
