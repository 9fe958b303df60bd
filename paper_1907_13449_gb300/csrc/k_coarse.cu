// k_coarse.cu -- the initial (coarse) pass of Sec. III-D: per-arm census cost (Eq. 7),
// penalties, integer 8-path SGM (Eq. 8-9) and WTA (Eq. 10).
//
// Layout: the arm cost is uint16 [arm][pixel][Lcs] with the label dimension padded to
// Lcs = 32 * LPT (LPT = labels per lane in the SGM).  The SGM runs one warp per
// (arm, direction, scanline); lane l owns the LPT consecutive labels l*LPT .. l*LPT+LPT-1
// in registers, so the d-1 / d+1 neighbours are in-register except across lanes (one
// shuffle each way per step), and the predecessor's minimum is one redux.sync.  The 8
// directions run concurrently and accumulate into an exact integer sum with 32-bit
// atomics that carry two 16-bit label sums each (the host checks that a label's sum
// over the 8 paths stays below 2^16, so the halves never carry into each other).
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

constexpr int kBig = 1 << 28;   // an absent label (outside [0, Lc))

__global__ void coarse_cost_kernel(const uint64_t *__restrict__ cen_pad, int P, int Wp, int Hp, int H, int W, int ref,
                                   const int *__restrict__ views, int nv,
                                   const short2 *__restrict__ ctab, int Lc, int lcs_log2,
                                   uint16_t *__restrict__ out, unsigned long long *__restrict__ sum) {
    const size_t N = (size_t)H * W;
    const size_t total = N << lcs_log2;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned v = 0;
    if (t < total) {
        const int p = (int)(t >> lcs_log2);
        const int k = (int)(t & ((1u << lcs_log2) - 1));
        if (k < Lc) {
            const int x = p % W, y = p / W;
            const size_t HWp = (size_t)Hp * Wp;
            const uint64_t r = __ldg(cen_pad + (size_t)ref * HWp + (size_t)(y + P) * Wp + (x + P));
            for (int i = 0; i < nv; i++) {
                const int view = __ldg(views + i);
                const short2 n = __ldg(ctab + (size_t)view * Lc + k);
                const int xx = min(max(x + n.x, 0), W - 1), yy = min(max(y + n.y, 0), H - 1);
                v += __popcll(r ^ __ldg(cen_pad + (size_t)view * HWp + (size_t)(yy + P) * Wp + (xx + P)));
            }
        }
        out[t] = (uint16_t)v;
    }
    // exact integer sum of the arm's cost (for the derived penalties)
    unsigned long long w = v;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    __shared__ unsigned long long part[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = w;
    __syncthreads();
    if (wid == 0) {
        w = lane < (int)(blockDim.x >> 5) ? part[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
        if (lane == 0 && w) atomicAdd(sum, w);
    }
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
struct Vec;
template <>
struct Vec<2> {
    __device__ static void load(const uint16_t *p, int *c) {
        const uint32_t w = __ldg(reinterpret_cast<const uint32_t *>(p));
        c[0] = w & 0xffff;
        c[1] = w >> 16;
    }
};
template <>
struct Vec<4> {
    __device__ static void load(const uint16_t *p, int *c) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        c[0] = w.x & 0xffff;
        c[1] = w.x >> 16;
        c[2] = w.y & 0xffff;
        c[3] = w.y >> 16;
    }
};
template <>
struct Vec<8> {
    __device__ static void load(const uint16_t *p, int *c) {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
        c[0] = w.x & 0xffff;
        c[1] = w.x >> 16;
        c[2] = w.y & 0xffff;
        c[3] = w.y >> 16;
        c[4] = w.z & 0xffff;
        c[5] = w.z >> 16;
        c[6] = w.w & 0xffff;
        c[7] = w.w >> 16;
    }
};

// One warp per (arm, direction, scanline): Eq. 8 in the normalised form
//   L(p,k) = C(p,k) + (min(L'(k), L'(k-1)+P1, L'(k+1)+P1, m+P2) - m),  m = min_k L'(k),
// L = C where the predecessor is outside the image; sum over directions (Eq. 9).
template <int LPT>
__global__ void __launch_bounds__(128) coarse_sgm_kernel(const uint16_t *__restrict__ cost, int H, int W,
                                                         int Lc, const int *__restrict__ pen,
                                                         ScanTable st, int narms,
                                                         uint32_t *__restrict__ sum) {
    constexpr int Lcs = 32 * LPT;
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
    const size_t N = (size_t)H * W;
    const uint16_t *C = cost + (size_t)arm * N * Lcs;
    uint32_t *S = sum + (size_t)arm * N * (Lcs / 2);
    const int P1 = __ldg(pen + 2 * arm), P2 = __ldg(pen + 2 * arm + 1);
    const int k0 = lane * LPT;
    int L[LPT];
    int m = 0;
    bool first = true;
    while (x >= 0 && x < W && y >= 0 && y < H) {
        const size_t p = (size_t)y * W + x;
        int c[LPT];
        Vec<LPT>::load(C + p * Lcs + k0, c);
        int Ln[LPT];
        if (first) {
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
                int t = min(L[i], min(lm, rp) + P1);
                t = min(t, mp2);
                Ln[i] = (k0 + i < Lc) ? c[i] + (t - m) : kBig;
            }
        }
        int lmin = Ln[0];
#pragma unroll
        for (int i = 1; i < LPT; i++) lmin = min(lmin, Ln[i]);
        m = __reduce_min_sync(0xffffffffu, lmin);
#pragma unroll
        for (int i = 0; i < LPT; i += 2) {
            if (k0 + i < Lc) {
                const uint32_t lo16 = (uint32_t)Ln[i];
                const uint32_t hi16 = (k0 + i + 1 < Lc) ? (uint32_t)Ln[i + 1] : 0u;
                atomicAdd(S + p * (Lcs / 2) + (k0 + i) / 2, lo16 | (hi16 << 16));
            }
        }
#pragma unroll
        for (int i = 0; i < LPT; i++) L[i] = Ln[i];
        first = false;
        x += dx;
        y += dy;
    }
}

// WTA over the packed sums (Eq. 10): lowest label on ties.
__global__ void coarse_wta_kernel(const uint32_t *__restrict__ sum, int narms, int N, int Lc, int Lcs,
                                  int *__restrict__ maps, int *__restrict__ maps_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= narms * N) return;
    const uint32_t *s = sum + (size_t)t * (Lcs / 2);
    int best = 0;
    uint32_t bv = 0xffffffffu;
    for (int k2 = 0; k2 < (Lc + 1) / 2; k2++) {
        const uint32_t w = __ldg(s + k2);
        const uint32_t a = w & 0xffff, b = w >> 16;
        if (a < bv) { bv = a; best = 2 * k2; }
        if (2 * k2 + 1 < Lc && b < bv) { bv = b; best = 2 * k2 + 1; }
    }
    maps[t] = best;
    if (maps_out) maps_out[t] = best;
}

}  // namespace

cudaError_t launch_coarse_cost(cudaStream_t s, const uint64_t *cen_pad, int P, int Wp, int Hp, int H, int W, int ref,
                               const int *d_views, int nv, const short2 *ctab, int Lc, int Lcs,
                               uint16_t *out, unsigned long long *sum) {
    int lg = 0;
    while ((1 << lg) < Lcs) lg++;
    const size_t total = ((size_t)H * W) << lg;
    const int block = 256;
    const unsigned grid = (unsigned)((total + block - 1) / block);
    coarse_cost_kernel<<<grid, block, 0, s>>>(cen_pad, P, Wp, Hp, H, W, ref, d_views, nv, ctab, Lc, lg, out, sum);
    return cudaGetLastError();
}

cudaError_t launch_coarse_penalties(cudaStream_t s, const unsigned long long *sums, int narms,
                                    long long count, double p1f, double p2f, int P1, int P2, int *pen) {
    coarse_penalty_kernel<<<1, 32, 0, s>>>(sums, narms, count, p1f, p2f, P1, P2, pen);
    return cudaGetLastError();
}

cudaError_t launch_coarse_sgm(cudaStream_t s, const uint16_t *cost, int narms, int H, int W, int Lc,
                              int Lcs, const int *pen, uint32_t *sum) {
    const ScanTable st = make_scan_table(H, W);
    const long long warps = (long long)st.cum[8] * narms;
    const int block = 128;
    const unsigned grid = (unsigned)((warps * 32 + block - 1) / block);
    switch (Lcs) {
    case 64: coarse_sgm_kernel<2><<<grid, block, 0, s>>>(cost, H, W, Lc, pen, st, narms, sum); break;
    case 128: coarse_sgm_kernel<4><<<grid, block, 0, s>>>(cost, H, W, Lc, pen, st, narms, sum); break;
    case 256: coarse_sgm_kernel<8><<<grid, block, 0, s>>>(cost, H, W, Lc, pen, st, narms, sum); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_coarse_wta(cudaStream_t s, const uint32_t *sum, int narms, int N, int Lc, int Lcs,
                              int *maps, int *maps_out) {
    const int block = 256;
    const unsigned grid = (unsigned)(((long long)narms * N + block - 1) / block);
    coarse_wta_kernel<<<grid, block, 0, s>>>(sum, narms, N, Lc, Lcs, maps, maps_out);
    return cudaGetLastError();
}

}  // namespace lfsgm
