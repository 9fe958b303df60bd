// k_coarse.cu -- the initial (coarse) pass of Sec. III-D: per-arm census cost (Eq. 7),
// penalties, integer 8-path SGM (Eq. 8-9) and WTA (Eq. 10).
//
// Layout: the arm cost and the 8-path sums are uint16 [arm][pixel][Lcd], the label dimension
// padded only to Lcd = round_up(Lc, max(4, LPT)) (LPT = labels per lane: 2, 4 or 8 for
// Lc <= 64, 128, 256), so a lane's LPT labels are one aligned 4/8/16-byte word.
//  - cost: one warp per run of 16 pixels of a row and one arm; lanes hold LPT labels each and
//    read the census words at the labels' nearest shifts from the edge-padded census (no
//    clamping needed), the shifts coming as linear offsets from a per-arm table.
//  - SGM: one warp per (arm, direction, scanline); the lane's labels stay in registers, the
//    d-1 / d+1 neighbours across lanes come by one shuffle each way, the predecessor minimum by
//    one redux.sync; the next 4 cost rows are prefetched; the 8 directions add into the sums
//    with one packed 32/64-bit reduction per lane and step (the host checks that a label's sum
//    over the 8 paths stays below 2^16, so the 16-bit fields never carry into each other).
//  - WTA: one warp per (arm, pixel), argmin by one redux.sync over (sum << 8 | label).
#include "lfsgm_internal.cuh"

#include <algorithm>

namespace lfsgm {
namespace {

constexpr int kBig = 1 << 28;   // an absent label (outside [0, Lc))
constexpr int kCoarseRun = 16;  // pixels of a row per warp in the cost kernel

template <int LPT>
struct CVec;
template <>
struct CVec<2> {
    using T = uint32_t;
    __device__ static void unpack(T w, int *c) {
        c[0] = w & 0xffff;
        c[1] = w >> 16;
    }
    __device__ static T pack(const int *c) { return (uint32_t)c[0] | ((uint32_t)c[1] << 16); }
};
template <>
struct CVec<4> {
    using T = uint2;
    __device__ static void unpack(T w, int *c) {
        c[0] = w.x & 0xffff;
        c[1] = w.x >> 16;
        c[2] = w.y & 0xffff;
        c[3] = w.y >> 16;
    }
    __device__ static T pack(const int *c) {
        return make_uint2((uint32_t)c[0] | ((uint32_t)c[1] << 16), (uint32_t)c[2] | ((uint32_t)c[3] << 16));
    }
};
template <>
struct CVec<8> {
    using T = uint4;
    __device__ static void unpack(T w, int *c) {
        c[0] = w.x & 0xffff;
        c[1] = w.x >> 16;
        c[2] = w.y & 0xffff;
        c[3] = w.y >> 16;
        c[4] = w.z & 0xffff;
        c[5] = w.z >> 16;
        c[6] = w.w & 0xffff;
        c[7] = w.w >> 16;
    }
    __device__ static T pack(const int *c) {
        return make_uint4((uint32_t)c[0] | ((uint32_t)c[1] << 16), (uint32_t)c[2] | ((uint32_t)c[3] << 16),
                          (uint32_t)c[4] | ((uint32_t)c[5] << 16), (uint32_t)c[6] | ((uint32_t)c[7] << 16));
    }
};

template <int LPT>
__device__ __forceinline__ void load_offsets(const int *p, int *o) {
    if constexpr (LPT == 2) {
        const int2 v = __ldg(reinterpret_cast<const int2 *>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < LPT; j += 4) {
            const int4 v = __ldg(reinterpret_cast<const int4 *>(p + j));
            o[j] = v.x; o[j + 1] = v.y; o[j + 2] = v.z; o[j + 3] = v.w;
        }
    }
}

// Eq. 7 per arm: C_a(p, k) = sum over the arm's views of the Hamming distance between the
// reference census word at p and the view's word at p + n(view, k) (nearest shift, clamped --
// the padded census repeats the border words, so the linear offset needs no clamping).
template <int LPT>
__global__ void __launch_bounds__(128) coarse_cost_kernel(const uint64_t *__restrict__ cen_pad, size_t HWp, int Wp,
                                                          int P, int H, int W, int ref,
                                                          const int *__restrict__ armviews,
                                                          const int *__restrict__ otab, CoarseArms ca, int Lc,
                                                          int Lcd, uint16_t *__restrict__ out,
                                                          unsigned long long *__restrict__ armsum) {
    using V = CVec<LPT>;
    const int a = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int runs_x = (W + kCoarseRun - 1) / kCoarseRun;
    const int task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (task >= runs_x * H) return;
    const int y = task / runs_x, xs = (task - y * runs_x) * kCoarseRun, xe = min(xs + kCoarseRun, W);
    const int k0 = lane * LPT;
    const bool act = k0 < Lcd;
    const int nv = ca.nv[a];
    const int *views = armviews + a * kMaxArmViews;
    const int *ot = otab + ca.tab_off[a] + k0;
    const size_t N = (size_t)H * W;
    uint16_t *O = out + (size_t)a * N * Lcd + k0;
    const size_t rowoff = (size_t)(y + P) * Wp + P;
    const uint64_t *refrow = cen_pad + (size_t)ref * HWp + rowoff;
    unsigned long long total = 0;
    for (int x = xs; x < xe; x++) {
        if (!act) continue;
        const uint64_t r = __ldg(refrow + x);
        int c[LPT];
#pragma unroll
        for (int j = 0; j < LPT; j++) c[j] = 0;
        for (int i = 0; i < nv; i++) {
            const uint64_t *base = cen_pad + (size_t)__ldg(views + i) * HWp + rowoff + x;
            int o[LPT];
            load_offsets<LPT>(ot + i * Lcd, o);
#pragma unroll
            for (int j = 0; j < LPT; j++) c[j] += __popcll(r ^ __ldg(base + o[j]));
        }
#pragma unroll
        for (int j = 0; j < LPT; j++) {
            if (k0 + j >= Lc) c[j] = 0;
            total += (unsigned)c[j];
        }
        *reinterpret_cast<typename V::T *>(O + ((size_t)y * W + x) * Lcd) = V::pack(c);
    }
    for (int o = 16; o > 0; o >>= 1) total += __shfl_down_sync(0xffffffffu, total, o);
    if (lane == 0 && total) atomicAdd(armsum + a, total);
}

// P = floor(frac * mean + 0.5) with P1 >= 1 and P2 >= P1; the mean is the exact integer sum
// over the arm's cells divided by the cell count (IEEE double, round to nearest).
__global__ void coarse_penalty_kernel(const unsigned long long *sums, int narms, long long count,
                                      double p1f, double p2f, int P1, int P2, int *pen) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int a = 0; a < narms; a++) {
        long long q1, q2;
        if (P1 > 0) {
            q1 = P1;
            q2 = P2;
        } else {
            const double mean = __ddiv_rn((double)sums[a], (double)count);
            q1 = (long long)floor(__dadd_rn(__dmul_rn(p1f, mean), 0.5));
            q2 = (long long)floor(__dadd_rn(__dmul_rn(p2f, mean), 0.5));
            if (q1 < 1) q1 = 1;
            if (q2 < q1) q2 = q1;
        }
        pen[2 * a] = (int)q1;
        pen[2 * a + 1] = (int)q2;
    }
}

template <int LPT>
__device__ __forceinline__ void red_packed(uint16_t *dst, const int *v) {
    if constexpr (LPT == 2) {
        atomicAdd(reinterpret_cast<unsigned int *>(dst), (unsigned)v[0] | ((unsigned)v[1] << 16));
    } else {
#pragma unroll
        for (int j = 0; j < LPT; j += 4) {
            const unsigned long long w = (unsigned long long)v[j] | ((unsigned long long)v[j + 1] << 16) |
                                         ((unsigned long long)v[j + 2] << 32) | ((unsigned long long)v[j + 3] << 48);
            atomicAdd(reinterpret_cast<unsigned long long *>(dst + j), w);
        }
    }
}

// One warp per (arm, direction, scanline): Eq. 8 in the normalised form
//   L(p,k) = C(p,k) + (min(L'(k), L'(k-1)+P1, L'(k+1)+P1, m+P2) - m),  m = min_k L'(k),
// L = C where the predecessor is outside the image; sum over directions (Eq. 9).
template <int LPT>
__global__ void __launch_bounds__(128) coarse_sgm_kernel(const uint16_t *__restrict__ cost, int H, int W, int Lc,
                                                         int Lcd, const int *__restrict__ pen, ScanTable st,
                                                         int narms, uint16_t *__restrict__ sum) {
    using V = CVec<LPT>;
    using T = typename V::T;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int per_arm = st.cum[8];
    if (gw >= per_arm * narms) return;
    const int arm = gw / per_arm;
    const int w = gw - arm * per_arm;
    int r = 0;
    while (w >= st.cum[r + 1]) r++;
    const int s = w - st.cum[r];
    const int dx = dir_dx(r), dy = dir_dy(r);
    int x, y;
    scan_start(r, s, H, W, x, y);
    int steps = 1 << 30;
    if (dx > 0) steps = min(steps, W - x);
    if (dx < 0) steps = min(steps, x + 1);
    if (dy > 0) steps = min(steps, H - y);
    if (dy < 0) steps = min(steps, y + 1);
    const size_t N = (size_t)H * W;
    const int k0 = lane * LPT;
    const bool act = k0 < Lcd;
    const uint16_t *C = cost + (size_t)arm * N * Lcd + k0;
    uint16_t *S = sum + (size_t)arm * N * Lcd + k0;
    const int P1 = __ldg(pen + 2 * arm), P2 = __ldg(pen + 2 * arm + 1);
    const long long dp = (long long)dy * W + dx;
    long long p = (long long)y * W + x;
    auto ld = [&](long long q) {
        T v{};
        if (act) v = __ldg(reinterpret_cast<const T *>(C + q * Lcd));
        return v;
    };
    // the next four cost rows are in flight while a step is computed
    T r0 = ld(p), r1{}, r2{}, r3{};
    if (steps > 1) r1 = ld(p + dp);
    if (steps > 2) r2 = ld(p + 2 * dp);
    if (steps > 3) r3 = ld(p + 3 * dp);
    int L[LPT];
    int m = 0;
    for (int t = 0; t < steps; t++, p += dp) {
        const T cur = r0;
        r0 = r1;
        r1 = r2;
        r2 = r3;
        if (t + 4 < steps) r3 = ld(p + 4 * dp);
        int c[LPT];
        V::unpack(cur, c);
        int Ln[LPT];
        if (t == 0) {
#pragma unroll
            for (int i = 0; i < LPT; i++) Ln[i] = (k0 + i < Lc) ? c[i] : kBig;
        } else {
            int left = __shfl_up_sync(0xffffffffu, L[LPT - 1], 1);
            int right = __shfl_down_sync(0xffffffffu, L[0], 1);
            if (lane == 0) left = kBig;
            if (lane == 31) right = kBig;
            const int mp2 = m + P2;
#pragma unroll
            for (int i = 0; i < LPT; i++) {
                const int lm = (i == 0) ? left : L[i - 1];
                const int rp = (i == LPT - 1) ? right : L[i + 1];
                int u = min(L[i], min(lm, rp) + P1);
                u = min(u, mp2);
                Ln[i] = (k0 + i < Lc) ? c[i] + (u - m) : kBig;
            }
        }
        int lmin = Ln[0];
#pragma unroll
        for (int i = 1; i < LPT; i++) lmin = min(lmin, Ln[i]);
        m = __reduce_min_sync(0xffffffffu, lmin);
        if (act) {
            int v[LPT];
#pragma unroll
            for (int i = 0; i < LPT; i++) v[i] = (k0 + i < Lc) ? Ln[i] : 0;
            red_packed<LPT>(S + p * Lcd, v);
        }
#pragma unroll
        for (int i = 0; i < LPT; i++) L[i] = Ln[i];
    }
}

// WTA over the 8-path sums (Eq. 10): lowest label on ties (the key is sum << 8 | label).
template <int LPT>
__global__ void __launch_bounds__(128) coarse_wta_kernel(const uint16_t *__restrict__ sum, int narms, int N, int Lc,
                                                         int Lcd, int *__restrict__ maps, int *__restrict__ maps_out) {
    using V = CVec<LPT>;
    const int lane = threadIdx.x & 31;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= (long long)narms * N) return;
    const int k0 = lane * LPT;
    unsigned key = 0xffffffffu;
    if (k0 < Lcd) {
        int c[LPT];
        V::unpack(__ldg(reinterpret_cast<const typename V::T *>(sum + gw * Lcd + k0)), c);
#pragma unroll
        for (int j = 0; j < LPT; j++)
            if (k0 + j < Lc) key = min(key, ((unsigned)c[j] << 8) | (unsigned)(k0 + j));
    }
    key = __reduce_min_sync(0xffffffffu, key);
    if (lane == 0) {
        maps[gw] = (int)(key & 0xffu);
        if (maps_out) maps_out[gw] = (int)(key & 0xffu);
    }
}

}  // namespace

int coarse_lpt(int Lc) { return Lc <= 64 ? 2 : (Lc <= 128 ? 4 : 8); }
int coarse_stride(int Lc) {
    const int q = std::max(4, coarse_lpt(Lc));
    return (Lc + q - 1) / q * q;
}

cudaError_t launch_coarse_cost(cudaStream_t s, const uint64_t *cen_pad, int P, int Wp, int Hp, int H, int W, int ref,
                               const int *armviews, const int *otab, const CoarseArms &ca, int Lc,
                               uint16_t *out, unsigned long long *armsum) {
    const int Lcd = coarse_stride(Lc);
    const size_t HWp = (size_t)Hp * Wp;
    const long long tasks = (long long)((W + kCoarseRun - 1) / kCoarseRun) * H;
    dim3 grid((unsigned)((tasks + 3) / 4), (unsigned)ca.n_arms);
    switch (coarse_lpt(Lc)) {
    case 2: coarse_cost_kernel<2><<<grid, 128, 0, s>>>(cen_pad, HWp, Wp, P, H, W, ref, armviews, otab, ca, Lc, Lcd, out, armsum); break;
    case 4: coarse_cost_kernel<4><<<grid, 128, 0, s>>>(cen_pad, HWp, Wp, P, H, W, ref, armviews, otab, ca, Lc, Lcd, out, armsum); break;
    default: coarse_cost_kernel<8><<<grid, 128, 0, s>>>(cen_pad, HWp, Wp, P, H, W, ref, armviews, otab, ca, Lc, Lcd, out, armsum); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_penalties(cudaStream_t s, const unsigned long long *sums, int narms,
                                    long long count, double p1f, double p2f, int P1, int P2, int *pen) {
    coarse_penalty_kernel<<<1, 32, 0, s>>>(sums, narms, count, p1f, p2f, P1, P2, pen);
    return cudaGetLastError();
}

cudaError_t launch_coarse_sgm(cudaStream_t s, const uint16_t *cost, int narms, int H, int W, int Lc,
                              const int *pen, uint16_t *sum) {
    const ScanTable st = make_scan_table(H, W);
    const int Lcd = coarse_stride(Lc);
    const long long warps = (long long)st.cum[8] * narms;
    const int block = 128;
    const unsigned grid = (unsigned)((warps * 32 + block - 1) / block);
    switch (coarse_lpt(Lc)) {
    case 2: coarse_sgm_kernel<2><<<grid, block, 0, s>>>(cost, H, W, Lc, Lcd, pen, st, narms, sum); break;
    case 4: coarse_sgm_kernel<4><<<grid, block, 0, s>>>(cost, H, W, Lc, Lcd, pen, st, narms, sum); break;
    default: coarse_sgm_kernel<8><<<grid, block, 0, s>>>(cost, H, W, Lc, Lcd, pen, st, narms, sum); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_wta(cudaStream_t s, const uint16_t *sum, int narms, int N, int Lc, int *maps,
                              int *maps_out) {
    const int Lcd = coarse_stride(Lc);
    const long long warps = (long long)narms * N;
    const unsigned grid = (unsigned)((warps * 32 + 127) / 128);
    switch (coarse_lpt(Lc)) {
    case 2: coarse_wta_kernel<2><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    case 4: coarse_wta_kernel<4><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    default: coarse_wta_kernel<8><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    }
    return cudaGetLastError();
}

}  // namespace lfsgm
