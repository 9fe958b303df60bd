// k_coarse.cu -- the initial (coarse) pass of Sec. III-D: per-arm census cost (Eq. 7),
// penalties, integer SGM over 8 or 16 paths (Eq. 8-9) and WTA (Eq. 10).
//
// Layout: the arm cost and the path sums are uint16 [arm][pixel][Lcd], the label dimension
// padded only to Lcd = round_up(Lc, max(4, LPT)) (LPT = labels per lane: 2, 4 or 8 for
// Lc <= 64, 128, 256), so a lane's LPT labels are one aligned 4/8/16-byte word; padding labels
// hold the absent-label cost (see the SGM).
//  - cost: one warp per run of 32 pixels of a row and one arm, lanes = pixels; the census words
//    at the labels' nearest shifts come from the edge-padded census (no clamping needed), the
//    shifts as linear offsets from a per-arm table.
//  - SGM: one warp per (arm, direction, scanline); the lane's labels stay in registers, the
//    d-1 / d+1 neighbours across lanes come by one shuffle each way, the predecessor minimum by
//    one redux.sync; the next 4 cost rows are prefetched; the directions add into the sums
//    with one packed 32/64-bit reduction per lane and step (the host checks that a label's sum
//    over the paths stays below 2^16, so the 16-bit fields never carry into each other).
//  - WTA: one warp per 8 (arm, pixel) rows, argmin by one redux.sync over (sum << 8 | label).
#include "lfsgm_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace lfsgm {
namespace {


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
    __device__ static T fill(uint32_t w) { return w; }
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
    __device__ static T fill(uint32_t w) { return make_uint2(w, w); }
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
    __device__ static T fill(uint32_t w) { return make_uint4(w, w, w, w); }
};

// Eq. 7 per arm: C_a(p, k) = sum over the arm's views of the Hamming distance between the
// reference census word at p and the view's word at p + n(view, k) (nearest shift, clamped --
// the padded census repeats the border words, so the linear offset needs no clamping), summed
// over the C colour channels (census planes view * C + c; Sec. III-B).
// Cost of an absent (padding) label, k >= Lc.  The host bounds paths x (C + P2) below 2^16, so a
// present label's path cost (at most C + P2) stays below 2^13 = kAbsent for 8 and 16 paths.
constexpr int kAbsent = 0x2000;

// One warp per run of 32 pixels of a row and one arm, lane = pixel.  A label's shift is the same
// for every pixel, and a view's nearest shift changes only every few labels (a view at distance d
// has about 2 d |dmax - dmin| + 1 distinct shifts over the labels), so a view's Hamming distance
// is a step function of the label: the warp finds the steps of a view 32 labels at a time (lane =
// label, a ballot of the labels whose offset differs from the previous one) and, for each step,
// reads the 32 pixels' words at the new offset (one coalesced 256-byte access), and adds the
// change of each pixel's distance to that label's entry of the lane's own difference column in
// shared memory (two labels' 16-bit differences a word).  A prefix sum over the labels then gives
// each pixel's costs, stored 4 labels a word (staging them in shared memory to write the warp's
// contiguous rows coalesced took a third of the CTAs per SM and was slower: 0.31 vs 0.24 ms).
// Lanes past the end of the row repeat the last pixel and are not stored.  OT = uint8_t when every cost fits a byte (arm views x census bits x
// channels <= 255): half the bytes for the eight sweeps of the SGM to read; padding labels then
// hold 0 and the SGM marks them absent itself.
template <int C, typename OT>
__global__ void __launch_bounds__(128) coarse_cost_kernel(const uint64_t *__restrict__ cen_pad, size_t HWp, int Wp,
                                                          int P, int H, int W, int ref,
                                                          const int *__restrict__ armviews,
                                                          const int *__restrict__ otab, CoarseArms ca, int Lc,
                                                          int Lcd, OT *__restrict__ out,
                                                          unsigned long long *__restrict__ armsum) {
    extern __shared__ int cdiff[];                 // [warp][Lcd / 2][32]
    const int a = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int runs_x = (W + 31) >> 5;
    const int task = blockIdx.x * 4 + w;
    if (task >= runs_x * H) return;
    const int y = task / runs_x, x0 = (task - y * runs_x) * 32;
    const size_t base = (size_t)(y + P) * Wp + P + min(x0 + lane, W - 1);
    const int nv = ca.nv[a];
    const int *views = armviews + a * kMaxArmViews;
    const int *ot = otab + ca.tab_off[a];
    int *cd = cdiff + (size_t)w * (Lcd / 2) * 32 + lane;
    for (int i = 0; i < Lcd / 2; i++) cd[32 * i] = 0;
    uint64_t r[C];
#pragma unroll
    for (int ch = 0; ch < C; ch++) r[ch] = __ldg(cen_pad + ((size_t)ref * C + ch) * HWp + base);
    for (int v = 0; v < nv; v++) {
        const size_t vb = (size_t)__ldg(views + v) * C;
        int hp = 0, oprev = 0;
        for (int k0 = 0; k0 < Lc; k0 += 32) {
            const int k = k0 + lane;
            const int o = k < Lc ? __ldg(ot + v * Lcd + k) : 0;
            const int up = __shfl_up_sync(0xffffffffu, o, 1);
            const int before = lane == 0 ? oprev : up;
            unsigned steps = __ballot_sync(0xffffffffu, k < Lc && (k == 0 || o != before));
            oprev = __shfl_sync(0xffffffffu, o, 31);
            // the steps four at a time: their word loads are issued together, then their distances
            while (steps) {
                int bs[4];
                uint64_t wv[4][C];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    bs[u] = steps ? __ffs(steps) - 1 : -1;          // warp-uniform
                    steps &= steps - 1;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int off = __shfl_sync(0xffffffffu, o, bs[u] & 31);
#pragma unroll
                    for (int ch = 0; ch < C; ch++)
                        wv[u][ch] = bs[u] >= 0 ? __ldg(cen_pad + (vb + ch) * HWp + base + off) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    if (bs[u] < 0) break;
                    int h = 0;
#pragma unroll
                    for (int ch = 0; ch < C; ch++) h += __popcll(r[ch] ^ wv[u][ch]);
                    const int kb = k0 + bs[u];
                    cd[32 * (kb >> 1)] += (int)((unsigned)(h - hp) << (16 * (kb & 1)));
                    hp = h;
                }
            }
        }
    }
    OT *O = out + ((size_t)a * H * W + (size_t)y * W + min(x0 + lane, W - 1)) * Lcd;
    const bool store = x0 + lane < W;
    unsigned long long total = 0;
    int run = 0;
    for (int k0 = 0; k0 < Lcd; k0 += 4) {
        int c[4];
#pragma unroll
        for (int q = 0; q < 2; q++) {
            // the word holds d(k) + d(k+1) 2^16 (two's complement, |d| < 2^15): split it exactly
            const int wd = cd[32 * ((k0 >> 1) + q)];
            const int d0 = (int)(short)(wd & 0xffff), d1 = (wd - d0) >> 16;
            run += d0;
            c[2 * q] = run;
            run += d1;
            c[2 * q + 1] = run;
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (k0 + q >= Lc) c[q] = 0;
        if (store) total += (unsigned)(c[0] + c[1] + c[2] + c[3]);
        if constexpr (sizeof(OT) == 1) {
            if (store)
                *reinterpret_cast<uint32_t *>(O + k0) =
                    (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) | ((uint32_t)c[3] << 24);
        } else {
            // padding labels (k >= Lc) hold kAbsent, above every path cost of a present label
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (k0 + q >= Lc) c[q] = kAbsent;
            if (store)
                *reinterpret_cast<uint2 *>(O + k0) = make_uint2((uint32_t)c[0] | ((uint32_t)c[1] << 16),
                                                                (uint32_t)c[2] | ((uint32_t)c[3] << 16));
        }
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
__device__ __forceinline__ void words_of(const typename CVec<LPT>::T &w, uint32_t *c) {
    if constexpr (LPT == 2) {
        c[0] = w;
    } else if constexpr (LPT == 4) {
        c[0] = w.x;
        c[1] = w.y;
    } else {
        c[0] = w.x;
        c[1] = w.y;
        c[2] = w.z;
        c[3] = w.w;
    }
}

template <int LPT>
__device__ __forceinline__ void red_words(uint16_t *dst, const uint32_t *v) {
    if constexpr (LPT == 2) {
        atomicAdd(reinterpret_cast<unsigned int *>(dst), v[0]);
    } else {
#pragma unroll
        for (int j = 0; j < LPT / 2; j += 2)
            atomicAdd(reinterpret_cast<unsigned long long *>(dst + 2 * j),
                      (unsigned long long)v[j] | ((unsigned long long)v[j + 1] << 32));
    }
}

// One warp per (arm, direction, scanline): Eq. 8 in the normalised form
//   L(p,k) = C(p,k) + (min(L'(k), L'(k-1)+P1, L'(k+1)+P1, m+P2) - m),  m = min_k L'(k),
// L = C where the predecessor is outside the image; sum over directions (Eq. 9).
// A lane's labels are held as 16-bit pairs in 32-bit words: the minima are per-halfword
// (DPX __vimin3_u16x2 / __viaddmin_u16x2) and the additions and the subtraction of m are plain 32-bit operations, exact
// because every present value stays below 2^13 (the host bounds paths (C + P2) < 2^16) and is at
// least m, so no halfword carries or borrows.  Absent labels need no masks: their cost is
// kAbsent = 2^13 (padding labels, and lanes past Lcd read it too), so their path cost stays in
// [2^13, 2^13 + P2], above every present value (never a minimum, never a chosen neighbour) and
// below 2^14; labels below 0 read 0x7fff.  The absent labels' sums overflow their halfwords,
// but a carry only runs into higher, also absent, labels or out of the reduced word, and the
// WTA reads labels below Lc only.
// Byte costs (C8): a lane's LPT bytes are one 2/4/8-byte load, widened to halfword pairs by one
// byte permute per pair that also puts kAbsent into the absent labels' halves.
template <int LPT>
struct BVec;
template <>
struct BVec<2> {
    using T = uint16_t;
    __device__ static void words(T v, uint32_t *w) { w[0] = (uint32_t)v; }
};
template <>
struct BVec<4> {
    using T = uint32_t;
    __device__ static void words(T v, uint32_t *w) { w[0] = v; }
};
template <>
struct BVec<8> {
    using T = uint2;
    __device__ static void words(T v, uint32_t *w) {
        w[0] = v.x;
        w[1] = v.y;
    }
};

template <int LPT, bool C8>
__global__ void __launch_bounds__(128) coarse_sgm_kernel(const void *__restrict__ cost_v, int H, int W, int Lc,
                                                         int Lcd, const int *__restrict__ pen, int per_arm,
                                                         int narms, uint16_t *__restrict__ sum,
    const int *__restrict__ order) {
    using CT = typename std::conditional<C8, uint8_t, uint16_t>::type;
    using T = typename std::conditional<C8, typename BVec<LPT>::T, typename CVec<LPT>::T>::type;
    const CT *cost = reinterpret_cast<const CT *>(cost_v);
    constexpr int NP = LPT / 2;
    constexpr uint32_t SENT = 0x7fff7fffu;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw >= per_arm * narms) return;
    const int arm = gw / per_arm;
    const int w = gw - arm * per_arm;
    const int rs = __ldg(order + w);             // longest scanlines first (within the arm)
    const int r = rs & 15, s = rs >> 4;
    const int dx = dir_dx(r), dy = dir_dy(r);
    int x, y;
    scan_start(r, s, H, W, x, y);
    const int steps = scan_steps(x, y, dx, dy, H, W);
    const size_t N = (size_t)H * W;
    const int k0 = lane * LPT;
    const bool act = k0 < Lcd;
    const CT *C = cost + (size_t)arm * N * Lcd + k0;
    uint16_t *S = sum + (size_t)arm * N * Lcd + k0;
    const uint32_t P1 = (uint32_t)__ldg(pen + 2 * arm), P2 = (uint32_t)__ldg(pen + 2 * arm + 1);
    const uint32_t P1P1 = P1 * 0x10001u;
    constexpr uint32_t ABS2 = (uint32_t)kAbsent * 0x10001u;
    // byte costs: one byte permute per label pair widens two bytes to halfwords and puts kAbsent
    // (= 0x2000: bytes 0x00, 0x20 of the constant operand, selectors 4 and 5) into the halves of
    // labels >= Lc (all of them on lanes past Lcd)
    uint32_t bsel[NP];
#pragma unroll
    for (int j = 0; j < NP; j++) {
        const int b = (2 * j) & 3;                                   // byte of label 2j in its word
        const uint32_t lo = (k0 + 2 * j < Lc && act) ? (uint32_t)b | (4u << 4) : 0x54u;
        const uint32_t hi = (k0 + 2 * j + 1 < Lc && act) ? (uint32_t)(b + 1) | (4u << 4) : 0x54u;
        bsel[j] = lo | (hi << 8);
    }
    // cost and sum pointers step along the scanline; the cost rows of the next four steps are in
    // flight (a ring of four registers, indexed statically by unrolling the steps by four)
    const long long dstep = ((long long)dy * W + dx) * Lcd;
    const CT *pc = C + ((long long)y * W + x) * Lcd;
    uint16_t *ps = S + ((long long)y * W + x) * Lcd;
    auto ld = [&](int t) {
        T v;
        if constexpr (C8) v = T{};
        else v = CVec<LPT>::fill(ABS2);
        if (act && t < steps) v = __ldg(reinterpret_cast<const T *>(pc + (long long)t * dstep));
        return v;
    };
    auto words = [&](const T &v, uint32_t *c) {
        if constexpr (C8) {
            uint32_t src[(NP + 1) / 2];
            BVec<LPT>::words(v, src);
#pragma unroll
            for (int j = 0; j < NP; j++) c[j] = __byte_perm(src[j / 2], (uint32_t)kAbsent, bsel[j]);
        } else {
            words_of<LPT>(v, c);
        }
    };
    T ring[4] = {ld(0), ld(1), ld(2), ld(3)};
    uint32_t L[NP];
    uint32_t m;
    auto finish = [&](const uint32_t *Ln) {       // warp minimum, packed reduction, carry the row
        uint32_t q = Ln[0];
#pragma unroll
        for (int j = 1; j < NP; j++) q = __vimin3_u16x2(q, Ln[j], Ln[j]);
        m = __reduce_min_sync(0xffffffffu, min(q & 0xffffu, q >> 16));
        if (act) red_words<LPT>(ps, Ln);
        ps += dstep;
#pragma unroll
        for (int j = 0; j < NP; j++) L[j] = Ln[j];
    };
    {   // path start: L = C
        uint32_t Ln[NP];
        words(ring[0], Ln);
        ring[0] = ld(4);
        finish(Ln);
    }
    for (int t0 = 1; t0 < steps; t0 += 4) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int t = t0 + k;
            if (t >= steps) break;
            const int slot = (1 + k) & 3;          // step t's row sits in ring[t % 4]
            uint32_t c[NP];
            words(ring[slot], c);
            ring[slot] = ld(t + 4);
            uint32_t left = __shfl_up_sync(0xffffffffu, L[NP - 1], 1);
            uint32_t right = __shfl_down_sync(0xffffffffu, L[0], 1);
            if (lane == 0) left = SENT;
            if (lane == 31) right = SENT;
            // min(L'(k), L'(k-1)+P1, L'(k+1)+P1, m+P2) = min(L'(k), min(L'(k-1), L'(k+1), m+P2-P1) + P1):
            // one 3-way and one add-then-min per halfword pair (DPX)
            const uint32_t mm = __byte_perm(m, 0, 0x1010), mq = __byte_perm(m + P2 - P1, 0, 0x1010);
            uint32_t Ln[NP];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const uint32_t pw = (j == 0) ? left : L[j - 1];
                const uint32_t nw = (j == NP - 1) ? right : L[j + 1];
                const uint32_t lm = __byte_perm(pw, L[j], 0x5432);    // labels 2j-1, 2j
                const uint32_t rp = __byte_perm(L[j], nw, 0x5432);    // labels 2j+1, 2j+2
                const uint32_t u = __viaddmin_u16x2(__vimin3_u16x2(lm, rp, mq), P1P1, L[j]);
                Ln[j] = c[j] + (u - mm);
            }
            finish(Ln);
        }
    }
}

// WTA over the path sums (Eq. 10): lowest label on ties (the key is sum << 8 | label).
// One warp per 8 consecutive (arm, pixel) rows: the 8 rows' loads are issued before the first
// reduction, so a warp waits for memory once instead of once per pixel.
constexpr int kWtaRows = 8;
template <int LPT>
__global__ void __launch_bounds__(128) coarse_wta_kernel(const uint16_t *__restrict__ sum, int narms, int N, int Lc,
                                                         int Lcd, int *__restrict__ maps, int *__restrict__ maps_out) {
    using V = CVec<LPT>;
    const int lane = threadIdx.x & 31;
    const long long g0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kWtaRows;
    const long long total = (long long)narms * N;
    if (g0 >= total) return;
    const int k0 = lane * LPT;
    typename V::T w[kWtaRows];
#pragma unroll
    for (int i = 0; i < kWtaRows; i++) {
        w[i] = typename V::T{};
        if (k0 < Lcd && g0 + i < total) w[i] = __ldg(reinterpret_cast<const typename V::T *>(sum + (g0 + i) * Lcd + k0));
    }
#pragma unroll
    for (int i = 0; i < kWtaRows; i++) {
        if (g0 + i >= total) break;                       // warp-uniform
        unsigned key = 0xffffffffu;
        int c[LPT];
        V::unpack(w[i], c);
#pragma unroll
        for (int j = 0; j < LPT; j++)
            if (k0 + j < Lc) key = min(key, ((unsigned)c[j] << 8) | (unsigned)(k0 + j));
        key = __reduce_min_sync(0xffffffffu, key);
        if (lane == 0) {
            maps[g0 + i] = (int)(key & 0xffu);
            if (maps_out) maps_out[g0 + i] = (int)(key & 0xffu);
        }
    }
}

}  // namespace

int coarse_lpt(int Lc) { return Lc <= 64 ? 2 : (Lc <= 128 ? 4 : 8); }
int coarse_stride(int Lc) {
    const int q = std::max(4, coarse_lpt(Lc));
    return (Lc + q - 1) / q * q;
}

cudaError_t launch_coarse_cost(cudaStream_t s, const uint64_t *cen_pad, int P, int Wp, int Hp, int H, int W, int ref, int C,
                               const int *armviews, const int *otab, const CoarseArms &ca, int Lc,
                               void *out, bool out8, unsigned long long *armsum) {
    const int Lcd = coarse_stride(Lc);
    const size_t HWp = (size_t)Hp * Wp;
    const long long tasks = (long long)((W + 31) / 32) * H;
    dim3 grid((unsigned)((tasks + 3) / 4), (unsigned)ca.n_arms);
    // the warps' label-difference columns (Lcd is a multiple of 4)
    const size_t smem = (size_t)4 * (Lcd / 2) * 32 * sizeof(int);
    if (out8) {
        auto kern = C == 3 ? coarse_cost_kernel<3, uint8_t> : coarse_cost_kernel<1, uint8_t>;
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, 128, smem, s>>>(cen_pad, HWp, Wp, P, H, W, ref, armviews, otab, ca, Lc, Lcd, (uint8_t *)out,
                                     armsum);
    } else {
        auto kern = C == 3 ? coarse_cost_kernel<3, uint16_t> : coarse_cost_kernel<1, uint16_t>;
        if (smem > 48 * 1024) {
            const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        kern<<<grid, 128, smem, s>>>(cen_pad, HWp, Wp, P, H, W, ref, armviews, otab, ca, Lc, Lcd, (uint16_t *)out,
                                     armsum);
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_penalties(cudaStream_t s, const unsigned long long *sums, int narms,
                                    long long count, double p1f, double p2f, int P1, int P2, int *pen) {
    coarse_penalty_kernel<<<1, 32, 0, s>>>(sums, narms, count, p1f, p2f, P1, P2, pen);
    return cudaGetLastError();
}

cudaError_t launch_coarse_sgm(cudaStream_t s, const void *cost, bool cost8, int narms, int H, int W, int Lc,
                              const int *pen, uint16_t *sum, const int *order, int paths) {
    const ScanTable st = make_scan_table(H, W, paths);
    const int Lcd = coarse_stride(Lc);
    const long long warps = (long long)st.cum[paths] * narms;
    const int block = 128;
    const unsigned grid = (unsigned)((warps * 32 + block - 1) / block);
#define LFSGM_SGM(LPT, B) coarse_sgm_kernel<LPT, B><<<grid, block, 0, s>>>(cost, H, W, Lc, Lcd, pen, st.cum[paths], narms, sum, order)
    switch (coarse_lpt(Lc)) {
    case 2: if (cost8) LFSGM_SGM(2, true); else LFSGM_SGM(2, false); break;
    case 4: if (cost8) LFSGM_SGM(4, true); else LFSGM_SGM(4, false); break;
    default: if (cost8) LFSGM_SGM(8, true); else LFSGM_SGM(8, false); break;
    }
#undef LFSGM_SGM
    return cudaGetLastError();
}

cudaError_t launch_coarse_wta(cudaStream_t s, const uint16_t *sum, int narms, int N, int Lc, int *maps,
                              int *maps_out) {
    const int Lcd = coarse_stride(Lc);
    const long long warps = ((long long)narms * N + kWtaRows - 1) / kWtaRows;
    const unsigned grid = (unsigned)((warps * 32 + 127) / 128);
    switch (coarse_lpt(Lc)) {
    case 2: coarse_wta_kernel<2><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    case 4: coarse_wta_kernel<4><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    default: coarse_wta_kernel<8><<<grid, 128, 0, s>>>(sum, narms, N, Lc, Lcd, maps, maps_out); break;
    }
    return cudaGetLastError();
}

}  // namespace lfsgm
