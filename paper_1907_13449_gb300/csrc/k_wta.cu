// k_wta.cu -- winner-takes-all (Eq. 10) and sub-pixel refinement (Sec. III-F, Eq. 13).
//
// One thread per pixel walks its window: the smallest aggregated cost wins, the lowest
// label on ties.  Mode 1 adds the vertex of the parabola through the winner and its two
// neighbours, delta = (C(g-1) - C(g+1)) / (2 (C(g-1) - 2 C(g) + C(g+1))), when the winner
// lies in [lo+1, lo+cnt-2] and that interval holds at least 3 labels (cnt >= 5); Eq. 13
// prints the denominator with the opposite sign, which would move away from the lower
// neighbour.  Mode 2 is the soft-argmin sum_g softmax(-C/tau)_g d_g (FP32 weights).
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

__global__ void wta_kernel(const float *__restrict__ agg, const int *__restrict__ lo,
                           const int *__restrict__ cnt, const long long *__restrict__ off, int N, int G,
                           double dmin, double step, int mode, float tau, int *__restrict__ label,
                           float *__restrict__ disp, int *__restrict__ status) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const float *s = agg + off[p];
    const int n = cnt[p], l = lo[p];
    // both ends of the row on a 4-slot boundary: the row then holds round4(n) slots, which the
    // vector loads below read
    if (!window_ok(l, n, G, off[p + 1] - off[p], status) || !row_aligned(off[p], status) ||
        !row_aligned(off[p + 1], status)) {
        if (label) label[p] = -1;
        if (disp) disp[p] = __int_as_float(0x7fc00000);
        return;
    }
    int b = 0;
    float bv = s[0];
    const float it = 1.f / tau;
    float num = 0.f, den = 0.f;
    if (n <= 32) {
        // the whole window in registers: its (16-byte aligned) row as 8 vector loads issued together
        float v[32];
        const float4 *r = reinterpret_cast<const float4 *>(s);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 w = 4 * q < n ? __ldg(r + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[4 * q] = w.x;
            v[4 * q + 1] = w.y;
            v[4 * q + 2] = w.z;
            v[4 * q + 3] = w.w;
        }
        bv = v[0];
#pragma unroll
        for (int j = 1; j < 32; j++)
            if (j < n && v[j] < bv) { bv = v[j]; b = j; }
        if (mode == 2 && disp) {
#pragma unroll
            for (int j = 0; j < 32; j++)
                if (j < n) {
                    const float w = expf((bv - v[j]) * it);
                    num = fmaf(w, (float)j, num);
                    den += w;
                }
        }
    } else {
        // 32-slot chunks of the row as 8 vector loads issued together, used in slot order (slot 0
        // compares equal to bv and changes nothing)
        const float4 *r = reinterpret_cast<const float4 *>(s);
        for (int j0 = 0; j0 < n; j0 += 32) {
            float4 w[8];
#pragma unroll
            for (int q = 0; q < 8; q++) w[q] = j0 + 4 * q < n ? __ldg(r + (j0 >> 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const float c4[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int j = j0 + 4 * q + e;
                    if (j < n && c4[e] < bv) { bv = c4[e]; b = j; }
                }
            }
        }
        if (mode == 2 && disp) {
            for (int j0 = 0; j0 < n; j0 += 32) {
                float4 w[8];
#pragma unroll
                for (int q = 0; q < 8; q++) w[q] = j0 + 4 * q < n ? __ldg(r + (j0 >> 2) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    const float c4[4] = {w[q].x, w[q].y, w[q].z, w[q].w};
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int j = j0 + 4 * q + e;
                        if (j < n) {
                            const float wt = expf((bv - c4[e]) * it);
                            num = fmaf(wt, (float)j, num);
                            den += wt;
                        }
                    }
                }
            }
        }
    }
    if (label) label[p] = l + b;
    if (!disp) return;
    if (mode == 2) {
        // FP32 weights after subtracting the minimum (every exponent <= 0), summed in slot order;
        // the mean slot is mapped to a disparity in double
        disp[p] = (float)(dmin + ((double)l + (double)(num / den)) * step);
        return;
    }
    double delta = 0.0;
    if (mode == 1 && n >= 5 && b >= 1 && b <= n - 2) {
        const float cm = s[b - 1], cp = s[b + 1];
        const float den = (cm - bv) + (cp - bv);
        if (den > 0.f) delta = (double)((cm - cp) / (2.f * den));
    }
    disp[p] = (float)(dmin + ((double)(l + b) + delta) * step);
}

// 3 x 3 median (Sec. III-F): thread per pixel, the window clamped to the image; the median of
// the 9 values by a fixed min/max exchange network (19 exchanges), exact: it selects one input.
__device__ __forceinline__ void cswap(float &a, float &b) {
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

__global__ void median3_kernel(const float *__restrict__ in, float *__restrict__ out, int H, int W) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W) return;
    const int xm = max(x - 1, 0), xp = min(x + 1, W - 1);
    const int ym = max(y - 1, 0), yp = min(y + 1, H - 1);
    const float *r0 = in + (size_t)ym * W, *r1 = in + (size_t)y * W, *r2 = in + (size_t)yp * W;
    float p0 = __ldg(r0 + xm), p1 = __ldg(r0 + x), p2 = __ldg(r0 + xp);
    float p3 = __ldg(r1 + xm), p4 = __ldg(r1 + x), p5 = __ldg(r1 + xp);
    float p6 = __ldg(r2 + xm), p7 = __ldg(r2 + x), p8 = __ldg(r2 + xp);
    // the classic 19-exchange median-of-9 selection network
    cswap(p1, p2); cswap(p4, p5); cswap(p7, p8);
    cswap(p0, p1); cswap(p3, p4); cswap(p6, p7);
    cswap(p1, p2); cswap(p4, p5); cswap(p7, p8);
    cswap(p0, p3); cswap(p5, p8); cswap(p4, p7);
    cswap(p3, p6); cswap(p1, p4); cswap(p2, p5);
    cswap(p4, p7); cswap(p4, p2); cswap(p6, p4);
    cswap(p4, p2);
    out[(size_t)y * W + x] = p4;
}

}  // namespace

cudaError_t launch_median3(cudaStream_t s, const float *in, float *out, int H, int W) {
    dim3 block(128), grid((W + 127) / 128, H);
    median3_kernel<<<grid, block, 0, s>>>(in, out, H, W);
    return cudaGetLastError();
}

cudaError_t launch_wta(cudaStream_t s, const float *agg, const int *lo, const int *cnt, const long long *off,
                       int N, int G, double dmin, double step, int mode, float tau, int *label, float *disp,
                       int *status) {
    wta_kernel<<<(N + 255) / 256, 256, 0, s>>>(agg, lo, cnt, off, N, G, dmin, step, mode, tau, label, disp,
                                               status);
    return cudaGetLastError();
}

}  // namespace lfsgm
