// k_sgm.cu -- bounded SGM over 8 or 16 paths on the windowed fine cost (Sec. III-E with Eq. 8-9).
//
// One warp per (direction, scanline).  Lane j owns slot j of the current pixel's window.
// When this window and the predecessor's are both at most 32 labels wide (the regular case),
// the predecessor's path costs L' stay in registers, one slot per lane, and the ragged-window
// alignment (slot i = lo(p) + j - lo(p-r)) is three shuffles with bounds checks: labels outside
// the predecessor's window are absent from the minimum (Sec. III-E).  Wider windows take the
// general form with L' in a per-warp shared-memory row (chunks of 32 slots).  Window metadata
// is fetched 32 pixels at a time (one per lane, the next block one block ahead) and also kept in a
// per-warp ring of 64 steps in shared memory; a ballot over a block finds the steps that need the
// general form, and the narrow steps between them run in a tight loop that reads the metadata of
// the step after next from the ring (one broadcast load) and loads cost rows two steps ahead.
// The step is the normalised recurrence
//   L(p,g) = C(p,g) + (min(L'(g), L'(g-1)+P1, L'(g+1)+P1, m+P2) - m),   m = min L',
// and the predecessor minimum m is one redux.sync.min.f32 per pixel.  The 8 or 16 directions run
// concurrently and add into agg (zeroed by the caller) with float atomics.  Optionally the few
// scanlines that cross many wide windows (a speed knob) run on all the warps of a CTA each, which
// share the wide steps' chunks (sgm_scanline SPLIT); a small kernel lists them first.
//
// Reproducible sum over the directions.  The aggregate C_s(p,g) = sum_r L_r(p,g) must not depend on
// the order in which the directions' atomics arrive.  Every exact L_r(p,g) lies in [0, B] with
// B = C(p,g) + P2 (the bracket is at most P2 above m), and B depends only on the cell.  Each
// direction clamps its FP32 L_r to B (removing rounding beyond the exact bound) and rounds it to a
// multiple of q = 2^(floor(log2 B) + 1 + log2(paths) - 24) before adding it.  Then every partial sum
// is a multiple of q no larger than paths x 2^(floor(log2 B) + 1) = 2^24 q, so it is exactly
// representable: each addition is exact, and the sum is the same in any order.  The rounding moves
// an addend by at most q / 2 <= 2^-21 B (8 paths) or 2^-20 B (16 paths).
//
// Derived penalties: per-block partial sums (double) of the active slots, then one block
// adds the partials in a fixed order, so the mean is deterministic.
#include "lfsgm_internal.cuh"

#include <algorithm>

namespace lfsgm {
namespace {

constexpr int kSgmWarps = 4;      // default warps (scanlines) per CTA; 2, 4 or 8 (a speed knob)
constexpr int kSplitCap = 256;    // most scanlines split across a CTA's warps (more qualify: none is)

// L rounded to a multiple of q (see above); B = C + P2 of the cell.  With M = 1.5 x 2^(floor(log2 B)
// + 23 - qsh), qsh = 23 - log2(paths), every x in [0, B] gives x + M in M's binade, whose spacing
// is q: fl(x + M) - M is x rounded to a multiple of q (half to even), and the subtraction is exact.
// mk = (23 - qsh) << 23 | 1 << 22 puts M's exponent and its leading fraction bit in place.
__device__ __forceinline__ float det_addend(float L, float B, int mk) {
    const float M = __int_as_float((__float_as_int(B) & 0x7f800000) + mk);
    return __fsub_rn(__fadd_rn(fminf(L, B), M), M);
}

__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// One scanline of direction r = rs & 15, number s = rs >> 4.  NW = 1: one warp, its own rows by
// slot (bufA, bufB) and metadata ring.  SPLIT (NW = the CTA's warps): the CTA's warps share the
// rows; warp 0 alone runs the narrow steps (the predecessor row in its registers), and every
// general step (a window or predecessor wider than 32 labels, or an invalid window) is spread over
// the warps by 32-slot chunk (warp w takes chunks w, w + NW, ...), the predecessor minimum taken
// over the warps' minima through xm ([2][NW] minima, [2][NW] slots for REC, then the minimum that
// warp 0 hands over after narrow steps), with one CTA barrier per general step (two after narrow
// steps).  Every cell gets the same value either way.
// REC: also record, for the adjoint, each cell's winning branch (0 same label, 1 label-1, 2 label+1,
// 3 m+P2, 4 path start; the first of P2, same, g-1, g+1 that equals the minimum, as the adjoint's
// own recurrence decides it) in codes[r * nnz_cap + slot] and each pixel's lowest minimising slot
// in amin[r * N + p].
template <bool REC, bool SPLIT, int NW>
__device__ __forceinline__ void sgm_scanline(const float *__restrict__ cost, const int *__restrict__ lo,
                                             const int *__restrict__ cnt, const long long *__restrict__ off,
                                             int H, int W, float P1, float P2, int G, float *__restrict__ agg,
                                             int *__restrict__ status, int rs, int mk,
                                             unsigned char *__restrict__ codes, int *__restrict__ amin,
                                             size_t nnz_cap, float *bufA, float *bufB, int2 *meta, float *xm,
                                             int wib) {
    const int lane = threadIdx.x & 31;
    const int r = rs & 15, s = rs >> 4;
    const int dx = dir_dx(r), dy = dir_dy(r);
    int x0, y0;
    scan_start(r, s, H, W, x0, y0);
    const int len = scan_steps(x0, y0, dx, dy, H, W);
    unsigned char *code = REC ? codes + (size_t)r * nnz_cap : nullptr;
    int *am = REC ? amin + (size_t)r * H * W : nullptr;
    const float INF = __int_as_float(0x7f800000);
    const bool lead = !SPLIT || wib == 0;        // the warp that runs the narrow steps
    if (SPLIT ? threadIdx.x == 0 : lane == 0) {
        bufA[-1] = INF;
        bufB[-1] = INF;
    }
    const long long p0 = (long long)y0 * W + x0, dpix = (long long)dy * W + dx;
    // window metadata of the 32 steps starting at kb, one step per lane: (lo | cnt << 16) with
    // cnt = 0 for an invalid window, and the row offset in units of 4 slots
    auto fetch = [&](int kb, int &mw, int &mo) {
        const int k = kb + lane;
        mw = 0;
        mo = 0;
        if (k < len) {
            const long long p = p0 + (long long)k * dpix;
            const int l_ = __ldg(lo + p), n_ = __ldg(cnt + p);
            const long long o_ = __ldg(off + p);
            if (window_ok(l_, n_, G, __ldg(off + p + 1) - o_, status) && (o_ & 3) == 0 && (o_ >> 2) < 0x7fffffff) {
                mw = l_ | (n_ << 16);
                mo = (int)(o_ >> 2);
            } else if ((o_ & 3) != 0 && status) {
                atomicExch(status, 7);
            }
        }
    };
    int cw, co, nw = 0, no = 0;                // this block's and the next block's metadata
    fetch(0, cw, co);
    if (len > 32) fetch(32, nw, no);
    meta[lane] = make_int2(cw, co);
    meta[32 + lane] = make_int2(nw, no);
    if (SPLIT) __syncthreads();                // the sentinels
    else __syncwarp();
    int plo = 0, pn = 0;                       // predecessor window; pn = 0: the path (re)starts
    float prev = INF, m = 0.f;                 // predecessor row (one slot per lane) and its minimum
    bool in_smem = false;                      // the predecessor row is in bufA (after a general step)
    int gpar = 0;                              // SPLIT: which half of xm this general step uses
    int k = 0;
    while (k < len) {
        const int kb = k & ~31;
        const int kbend = min(kb + 32, len);
        // steps of this block that need the general form: invalid or wider than 32 labels
        const int wn = cw >> 16;
        const unsigned bad = __ballot_sync(0xffffffffu, kb + lane < len && (wn == 0 || wn > 32));
        const unsigned ahead = bad & (0xffffffffu << (k - kb));
        int kend = ahead ? kb + __ffs(ahead) - 1 : kbend;
        if (pn > 32) kend = k;                 // a wide predecessor: the general form takes this step
        if (k < kend && !lead) {
            // SPLIT: the other warps skip to the next general step, knowing only the last narrow
            // step's window
            const int wl = __shfl_sync(0xffffffffu, cw, kend - 1 - kb);
            plo = wl & 0xffff;
            pn = wl >> 16;
            k = kend;
            in_smem = false;
        }
        if (k < kend) {
            // narrow steps: the predecessor row in registers, cost rows two steps ahead
            int ofs = __shfl_sync(0xffffffffu, co, k - kb);
            const int win = __shfl_sync(0xffffffffu, cw, k - kb);
            int l = win & 0xffff, n = win >> 16;
            float c = lane < n ? __ldg(cost + 4ll * ofs + lane) : 0.f;
            int2 mt1 = meta[(k + 1) & 63];
            float c1 = lane < (mt1.x >> 16) ? __ldg(cost + 4ll * mt1.y + lane) : 0.f;
            for (; k < kend; k++) {
                // the metadata of the step after next (from the ring; past the end of the scanline
                // it is zero: no window) and its cost row (a wide row has more than 32 slots, so its
                // first 32 are in bounds too): cost rows two steps ahead
                const int2 mt2 = meta[(k + 2) & 63];
                float c2 = 0.f;
                if (lane < (mt2.x >> 16)) c2 = __ldg(cost + 4ll * mt2.y + lane);
                const int win1 = mt1.x, ofs1 = mt1.y;
                const int n1 = win1 >> 16;
                float Lv = c;
                unsigned cd = 4;
                if (pn != 0) {
                    const int s0 = lane + (l - plo);     // slot of this label in the predecessor
                    const float v0 = __shfl_sync(0xffffffffu, prev, s0 & 31);
                    const float vm = __shfl_sync(0xffffffffu, prev, (s0 - 1) & 31);
                    const float vp = __shfl_sync(0xffffffffu, prev, (s0 + 1) & 31);
                    // min(L'(g-1) + P1, L'(g+1) + P1) = min(L'(g-1), L'(g+1)) + P1 exactly (rounding
                    // is monotone); an absent neighbour is +inf
                    const float a = (unsigned)(s0 - 1) < (unsigned)pn ? vm : INF;
                    const float b = (unsigned)(s0 + 1) < (unsigned)pn ? vp : INF;
                    const float v = (unsigned)s0 < (unsigned)pn ? v0 : INF;
                    float t = fminf(m + P2, fminf(a, b) + P1);
                    t = fminf(t, v);
                    if (REC) cd = t == m + P2 ? 3u : (t == v ? 0u : (t == a + P1 ? 1u : 2u));
                    Lv = c + (t - m);
                }
                const bool act = lane < n;
                if (act) atomicAdd(agg + 4ll * ofs + lane, det_addend(Lv, c + P2, mk));
                prev = act ? Lv : INF;
                m = warp_min(prev);
                if (REC) {
                    if (act) code[4ll * ofs + lane] = (unsigned char)cd;
                    const int slot = (int)__reduce_min_sync(0xffffffffu, prev == m ? (unsigned)lane : 0x7fffffffu);
                    if (lane == 0) am[p0 + (long long)k * dpix] = slot;
                }
                plo = l;
                pn = n;
                l = win1 & 0xffff;
                n = n1;
                ofs = ofs1;
                c = c1;
                c1 = c2;
                mt1 = mt2;
            }
            in_smem = false;
        }
        if (k < kbend) {
            // one general step: an invalid window restarts the path; a window wider than 32 labels
            // (this one or the predecessor's) works on rows by slot in shared memory
            const int win = __shfl_sync(0xffffffffu, cw, k - kb), ofs = __shfl_sync(0xffffffffu, co, k - kb);
            const int l = win & 0xffff, n = win >> 16;
            if (n == 0) {
                pn = 0;
            } else {
                if (pn != 0 && !in_smem) {
                    // the narrow steps' last row (and, SPLIT, its minimum) to shared memory
                    if (lead) {
                        if (lane < pn) bufA[lane] = prev;
                        if (lane == 0) {
                            bufA[pn] = INF;
                            if (SPLIT) xm[4 * NW] = m;
                        }
                    }
                    if (SPLIT) {
                        __syncthreads();
                        m = xm[4 * NW];
                    } else {
                        __syncwarp();
                    }
                }
                const long long o = 4ll * ofs;
                float lmin = INF;
                int lslot = 0x7fffffff;
                // sixteen of this warp's 32-label chunks per round: their cost loads are in flight
                // together, and every chunk reads the predecessor row before any chunk stores its own
                // (the compiler cannot tell bufA from bufB, so a store between them would order the
                // chunks one after another)
                constexpr int CS = 32 * NW;            // slot stride between a warp's chunks
                for (int j0 = 32 * (SPLIT ? wib : 0) + lane; j0 < n; j0 += 16 * CS) {
                    float cc[16];
#pragma unroll
                    for (int u = 0; u < 16; u++) cc[u] = j0 + CS * u < n ? __ldg(cost + o + j0 + CS * u) : 0.f;
                    if (pn != 0) {
                        // predecessor slot s read at row[s + 1] with s + 1 clamped (unsigned) to
                        // pn + 1: any slot outside [0, pn) lands on a sentinel (+inf), so an absent
                        // label drops out of the minimum (labels j >= n read in-bounds slots too)
                        const unsigned top = (unsigned)pn + 1u;
                        const float *row = bufA - 1;
                        auto step = [&](int u, float v0, float vm, float vp) {
                            const float t = fminf(fminf(m + P2, v0), fminf(vm, vp) + P1);
                            if (REC)
                                code[o + j0 + CS * u] = t == m + P2 ? 3 : (t == v0 ? 0 : (t == vm + P1 ? 1 : 2));
                            const float Ln = cc[u] + (t - m);
                            // the cell's cost cc[u] bounds its path costs (the global atomic does
                            // not order the shared-memory reads of the other chunks)
                            atomicAdd(agg + o + j0 + CS * u, det_addend(Ln, cc[u] + P2, mk));
                            cc[u] = Ln;
                        };
                        if (l == plo && n == pn) {
                            // the same window as the predecessor (a run of whole-range windows):
                            // slot j's neighbours are slots j - 1 and j + 1, and the sentinels at
                            // slots -1 and pn stand in for the absent ones
                            const float *q = bufA + j0;
#pragma unroll
                            for (int u = 0; u < 16; u++) {
                                if (j0 + CS * u >= n) break;
                                step(u, q[CS * u], q[CS * u - 1], q[CS * u + 1]);
                            }
                        } else {
#pragma unroll
                            for (int u = 0; u < 16; u++) {
                                if (j0 + CS * u >= n) break;
                                const unsigned k1 = (unsigned)(l + j0 + CS * u - plo + 1);
                                step(u, row[min(k1, top)], row[min(k1 - 1u, top)], row[min(k1 + 1u, top)]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; u++) {
                            if (j0 + CS * u >= n) break;
                            atomicAdd(agg + o + j0 + CS * u, det_addend(cc[u], cc[u] + P2, mk));
                            if (REC) code[o + j0 + CS * u] = 4;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const int j = j0 + CS * u;
                        if (j >= n) break;
                        bufB[j] = cc[u];
                        if (REC && cc[u] < lmin) lslot = j;      // a lane's slots ascend: its first minimum
                        lmin = fminf(lmin, cc[u]);
                    }
                }
                if (SPLIT) {
                    // the warps' minima (and lowest minimising slots) through xm, then the minimum
                    const float wm = warp_min(lmin);
                    int ws = 0;
                    if (REC) ws = (int)__reduce_min_sync(0xffffffffu, lmin == wm ? (unsigned)lslot : 0x7fffffffu);
                    if (lane == 0) {
                        xm[gpar * NW + wib] = wm;
                        if (REC) reinterpret_cast<int *>(xm)[2 * NW + gpar * NW + wib] = ws;
                        if (wib == 0) bufB[n] = INF;
                    }
                    __syncthreads();
                    const float mv = lane < NW ? xm[gpar * NW + lane] : INF;
                    m = warp_min(mv);
                    if (REC) {
                        const unsigned sv = lane < NW && mv == m
                                                ? (unsigned)reinterpret_cast<const int *>(xm)[2 * NW + gpar * NW + lane]
                                                : 0x7fffffffu;
                        const int slot = (int)__reduce_min_sync(0xffffffffu, sv);
                        if (wib == 0 && lane == 0) am[p0 + (long long)k * dpix] = slot;
                    }
                    gpar ^= 1;
                } else {
                    m = warp_min(lmin);
                    if (REC) {
                        const int slot = (int)__reduce_min_sync(0xffffffffu, lmin == m ? (unsigned)lslot : 0x7fffffffu);
                        if (lane == 0) am[p0 + (long long)k * dpix] = slot;
                    }
                    if (lane == 0) bufB[n] = INF;
                    __syncwarp();
                }
                float *tmp = bufA;
                bufA = bufB;
                bufB = tmp;
                if (lead) prev = lane < n ? bufA[lane] : INF;   // for a following narrow step
                in_smem = true;
                plo = l;
                pn = n;
                __syncwarp();
            }
            k++;
        }
        if ((k & 31) == 0 && k < len) {       // next block of metadata
            cw = nw;
            co = no;
            if (k + 32 < len) {
                fetch(k + 32, nw, no);
            } else {
                nw = 0;
                no = 0;
            }
            meta[(k + 32 + lane) & 63] = make_int2(nw, no);   // the slots of the block just finished
            __syncwarp();
        }
    }
}

// One warp per scanline, WPC warps per CTA; with split (not null), the first scap CTAs take one
// listed scanline each with all their warps (sgm_scanline SPLIT), and the other warps skip the
// listed ones.  split: [0] scanlines listed, [1 .. scap] the list (rs), then a mark per scanline
// (sgm_split_kernel); more than scap listed: none is split.
// Resident CTAs per SM that the register budget must allow: what the one-warp path reaches on its
// own (72 registers without the record, 96 with it; 8 warps: 80 and 128), so that the split path
// (more registers) does not lower the occupancy of every CTA.
__host__ __device__ constexpr int sgm_min_ctas(bool rec, int wpc) {
    return rec ? (wpc == 2 ? 10 : wpc == 4 ? 5 : 2) : (wpc == 2 ? 14 : wpc == 4 ? 7 : 3);
}

template <bool REC, int WPC>
__global__ void __launch_bounds__(32 * WPC, sgm_min_ctas(REC, WPC)) fine_sgm_kernel(const float *__restrict__ cost,
                                                                  const int *__restrict__ lo,
                                                                  const int *__restrict__ cnt,
                                                                  const long long *__restrict__ off,
                                                                  int H, int W, int Gs,
                                                                  const float *__restrict__ pen,
                                                                  int G, ScanTable st, float *__restrict__ agg,
                                                                  int *__restrict__ status,
                                                                  const int *__restrict__ order, int mk,
                                                                  unsigned char *__restrict__ codes,
                                                                  int *__restrict__ amin, size_t nnz_cap,
                                                                  const int *__restrict__ split, int scap) {
    extern __shared__ float sm[];
    const int wib = threadIdx.x >> 5;
    // rows by slot with one sentinel slot on each side (slot -1 and slot n hold +inf), Gs + 2 floats,
    // two per warp; then per warp a ring of the metadata of this block of 32 steps and the next one,
    // by step mod 64 (read by the narrow steps with one broadcast load); then xm (SPLIT)
    int2 *meta = reinterpret_cast<int2 *>(sm + (size_t)WPC * 2 * (Gs + 2)) + wib * 64;
    float *xm = sm + (size_t)WPC * 2 * (Gs + 2) + WPC * 128;
    const float P1 = __ldg(pen), P2 = __ldg(pen + 1);
    const int total = st.cum[st.paths];
    const int nsplit = split ? __ldg(split) : 0;
    const bool on = split && nsplit <= scap;
    if ((int)blockIdx.x < scap) {
        if (!on || (int)blockIdx.x >= nsplit) return;
        float *bufA = sm + 1;
        sgm_scanline<REC, true, WPC>(cost, lo, cnt, off, H, W, P1, P2, G, agg, status, __ldg(split + 1 + blockIdx.x),
                                     mk, codes, amin, nnz_cap, bufA, bufA + (Gs + 2), meta, xm, wib);
        return;
    }
    const int gw = ((int)blockIdx.x - scap) * WPC + wib;
    if (gw >= total) return;
    const int rs = __ldg(order + gw);            // longest scanlines first
    if (on && __ldg(split + 1 + scap + st.cum[rs & 15] + (rs >> 4))) return;
    float *bufA = sm + (size_t)wib * 2 * (Gs + 2) + 1;
    sgm_scanline<REC, false, 1>(cost, lo, cnt, off, H, W, P1, P2, G, agg, status, rs, mk, codes, amin, nnz_cap,
                                bufA, bufA + (Gs + 2), meta, xm, wib);
}

// The scanlines to split: one warp per scanline counts the windows wider than 32 labels on it
// (128 steps per round, their loads issued together) and marks it (mark[id] = 1 when listed, 0
// otherwise, for every scanline); one that reaches min_wide is listed (split[0] zeroed before,
// up to scap of them: the list's order does not matter, every scanline's values are its own).
// Warp w0 of nwarps (every lane of the warp calls it).
__device__ __forceinline__ void split_list(const int *__restrict__ cnt, int H, int W, const ScanTable &st,
                                           int min_wide, int scap, int *__restrict__ split, int w0, int nwarps) {
    const int lane = threadIdx.x & 31;
    const int total = st.cum[st.paths];
    int *mark = split + 1 + scap;
    for (int id = w0; id < total; id += nwarps) {
        // the direction: unrolled compares with the table (a run-time index would copy it to the stack)
        int r = 0, base = 0;
#pragma unroll
        for (int q = 1; q < kMaxPaths; q++)
            if (q < st.paths && id >= st.cum[q]) {
                r = q;
                base = st.cum[q];
            }
        const int s = id - base;
        int dx, dy;
        dir_of(r, dx, dy);
        int x0, y0;
        scan_start_d(dx, dy, s, H, W, x0, y0);
        const int len = scan_steps(x0, y0, dx, dy, H, W);
        const long long p0 = (long long)y0 * W + x0, dp = (long long)dy * W + dx;
        int c = 0;
        for (int k0 = 0; k0 < len; k0 += 128) {
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int k = k0 + 32 * u + lane;
                v[u] = k < len ? __ldg(cnt + p0 + k * dp) : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) c += v[u] > 32;
        }
        c = (int)__reduce_add_sync(0xffffffffu, (unsigned)c);
        if (lane == 0) {
            int listed = 0;
            if (c >= min_wide) {
                const int pos = atomicAdd(split, 1);
                if (pos < scap) {
                    split[1 + pos] = (s << 4) | r;
                    listed = 1;
                }
            }
            mark[id] = listed;
        }
    }
}

__global__ void sgm_split_kernel(const int *__restrict__ cnt, int H, int W, ScanTable st, int min_wide, int scap,
                                 int *__restrict__ split) {
    split_list(cnt, H, W, st, min_wide, scap, split, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
               (gridDim.x * blockDim.x) >> 5);
}

// Per-block sums of the active costs and slot counts (rows are 16-byte aligned, read as float4;
// slots past cnt are masked, so padding is never read into the sum).  The warps take 32
// consecutive pixels at a time, a lane its pixel: a lane sums its row's first 32 slots (8 vector
// loads issued together), and the slots past 32 of a few wide rows in the warp are then summed by
// the whole warp, one row after another (a lane a vector, the lanes' parts added in a fixed
// order), so that one wide row does not hold its warp for a dependent load per 32 slots.  Each
// lane adds its pixels in a fixed order, the block adds its warps in a fixed order, and the last
// block to finish (ticket counter) adds the block partials in block order and writes the
// penalties: the mean is deterministic.  The first nb blocks do this; blocks past them (split not
// null) list the SGM scanlines to split (split_list, split[0] zeroed before), beside them.
__global__ void __launch_bounds__(256) cost_partial_kernel(const float *__restrict__ cost,
                                                           const int *__restrict__ cnt,
                                                           const long long *__restrict__ off, int N, int G,
                                                           double *__restrict__ partial, int nb, double p1f,
                                                           double p2f, float *__restrict__ pen,
                                                           unsigned *__restrict__ ticket, int *__restrict__ status,
                                                           int H, int W, ScanTable st, int min_wide, int scap,
                                                           int *__restrict__ split) {
    if ((int)blockIdx.x >= nb) {
        split_list(cnt, H, W, st, min_wide, scap, split, (((int)blockIdx.x - nb) * blockDim.x + threadIdx.x) >> 5,
                   (((int)gridDim.x - nb) * blockDim.x) >> 5);
        return;
    }
    double s = 0.0, c = 0.0;
    const int lane0 = threadIdx.x & 31;
    const int wstride = nb * blockDim.x;
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < N; base += wstride) {
        const int p = base + lane0;
        long long o = 0;
        int n = 0;
        if (p < N) {
            o = off[p];
            n = cnt[p];
            if (!window_ok(0, n, G, off[p + 1] - o, status) || !row_aligned(o, status) ||
                !row_aligned(off[p + 1], status))
                n = 0;
        }
        const float4 *r = reinterpret_cast<const float4 *>(cost + o);
        float4 v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = 4 * q < n ? __ldg(r + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        float ps = 0.f;
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int j = 4 * q;
            ps += (j < n ? v[q].x : 0.f) + (j + 1 < n ? v[q].y : 0.f) + (j + 2 < n ? v[q].z : 0.f) +
                  (j + 3 < n ? v[q].w : 0.f);
        }
        // the slots past 32 of this warp's wide rows: a few are summed by the whole warp, one row at
        // a time; when most rows are wide (whole-range searches) each lane sums its own in 32-slot
        // chunks of 8 vector loads issued together
        unsigned wide = __ballot_sync(0xffffffffu, n > 32);
        if (__popc(wide) > 4) {
            for (int j0 = 32; j0 < n; j0 += 32) {
#pragma unroll
                for (int q = 0; q < 8; q++)
                    v[q] = j0 + 4 * q < n ? __ldg(r + (j0 >> 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const int j = j0 + 4 * q;
                    if (j < n)
                        ps += v[q].x + (j + 1 < n ? v[q].y : 0.f) + (j + 2 < n ? v[q].z : 0.f) +
                              (j + 3 < n ? v[q].w : 0.f);
                }
            }
            wide = 0u;
        }
        while (wide) {
            const int src = __ffs(wide) - 1;
            wide &= wide - 1;
            const long long ow = __shfl_sync(0xffffffffu, o, src);
            const int nw = __shfl_sync(0xffffffffu, n, src);
            const float4 *rw = reinterpret_cast<const float4 *>(cost + ow);
            float t = 0.f;
            for (int j = 32 + 4 * lane0; j < nw; j += 128) {
                const float4 a = __ldg(rw + (j >> 2));
                t += a.x + (j + 1 < nw ? a.y : 0.f) + (j + 2 < nw ? a.z : 0.f) + (j + 3 < nw ? a.w : 0.f);
            }
#pragma unroll
            for (int k = 16; k > 0; k >>= 1) t += __shfl_xor_sync(0xffffffffu, t, k);
            if (lane0 == src) ps += t;
        }
        s += (double)ps;
        c += n;
    }
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, k);
        c += __shfl_down_sync(0xffffffffu, c, k);
    }
    __shared__ double ws[32], wc[32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ws[wid] = s;
        wc[wid] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0, bc = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
            b += ws[i];
            bc += wc[i];
        }
        partial[blockIdx.x] = b;
        partial[nb + blockIdx.x] = bc;
        __threadfence();                                   // partials visible before the ticket
        last = atomicAdd(ticket, 1u) == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!last || wid != 0) return;
    // the last block: all partials are written; add them in block order (a lane every 32nd, eight
    // of them loaded together: one L2 round trip per 256 partials instead of one per 32)
    s = 0.0;
    c = 0.0;
    for (int i0 = lane; i0 < nb; i0 += 256) {
        double sv[8], cv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int i = i0 + 32 * u;
            sv[u] = i < nb ? __ldcg(partial + i) : 0.0;
            cv[u] = i < nb ? __ldcg(partial + nb + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; u++) {
            s += sv[u];
            c += cv[u];
        }
    }
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, k);
        c += __shfl_down_sync(0xffffffffu, c, k);
    }
    if (lane == 0) {
        const double mean = c > 0.0 ? s / c : 0.0;
        pen[0] = (float)(p1f * mean);
        pen[1] = (float)(p2f * mean);
        *ticket = 0u;                                      // ready for the next launch
    }
}

}  // namespace

cudaError_t launch_cost_partial_sums(cudaStream_t s, const float *cost, const int *cnt, const long long *off,
                                     int N, int G, double *partial, int nblocks, double p1f, double p2f,
                                     float *pen, unsigned *ticket, int *status, int H, int W, int paths,
                                     int min_wide, int *split) {
    const ScanTable st = make_scan_table(H, W, paths);
    int extra = 0;
    if (split) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        extra = std::min((st.cum[paths] + 7) / 8, sms * 8);      // a warp per scanline
    }
    cost_partial_kernel<<<nblocks + extra, 256, 0, s>>>(cost, cnt, off, N, G, partial, nblocks, p1f, p2f, pen, ticket,
                                                        status, H, W, st, min_wide, kSplitCap, split);
    return cudaGetLastError();
}

void build_scan_order(int H, int W, int paths, std::vector<int> &order) {
    order.clear();
    for (int r = 0; r < paths; r++)
        for (int s = 0; s < n_scanlines(r, H, W); s++) order.push_back((s << 4) | r);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return scan_len(a & 15, a >> 4, H, W) > scan_len(b & 15, b >> 4, H, W);
    });
}

int sgm_split_ints(int H, int W, int paths) {
    return 1 + kSplitCap + make_scan_table(H, W, paths).cum[paths];
}

cudaError_t launch_sgm_split(cudaStream_t s, const int *cnt, int H, int W, int paths, int min_wide, int *split) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const ScanTable st = make_scan_table(H, W, paths);
    const int want = (st.cum[paths] + 7) / 8;                 // a warp per scanline
    sgm_split_kernel<<<min(want, sms * 8), 256, 0, s>>>(cnt, H, W, st, min_wide, kSplitCap, split);
    return cudaGetLastError();
}

cudaError_t launch_fine_sgm(cudaStream_t s, const float *cost, const int *lo, const int *cnt,
                            const long long *off, int H, int W, int G, const float *pen, float *agg,
                            int *status, const int *order, int paths, unsigned char *codes, int *amin,
                            size_t nnz_cap, int warps_per_cta, const int *split) {
    const int wpc = warps_per_cta == 2 || warps_per_cta == 8 ? warps_per_cta : kSgmWarps;
    const ScanTable st = make_scan_table(H, W, paths);
    const int Gs = (G + 31) & ~31;
    const size_t smem = (size_t)wpc * (2 * (Gs + 2) * sizeof(float) + 64 * sizeof(int2)) + (size_t)(4 * wpc + 4) * 4;
    const int scap = split ? kSplitCap : 0;
    const unsigned grid = (unsigned)(scap + (st.cum[paths] + wpc - 1) / wpc);
    // one instantiation per CTA size, each with its own register budget (launch bounds)
    auto kern = codes ? (wpc == 2 ? fine_sgm_kernel<true, 2> : wpc == 8 ? fine_sgm_kernel<true, 8> : fine_sgm_kernel<true, 4>)
                      : (wpc == 2 ? fine_sgm_kernel<false, 2> : wpc == 8 ? fine_sgm_kernel<false, 8> : fine_sgm_kernel<false, 4>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int lp = 0;
    while ((1 << lp) < paths) lp++;
    const int mk = (lp << 23) | (1 << 22);       // (23 - qsh) << 23 with qsh = 23 - log2(paths)
    kern<<<grid, 32 * wpc, smem, s>>>(cost, lo, cnt, off, H, W, Gs, pen, G, st, agg, status, order, mk, codes,
                                      amin, nnz_cap, split, scap);
    return cudaGetLastError();
}

}  // namespace lfsgm
