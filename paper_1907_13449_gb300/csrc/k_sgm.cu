// k_sgm.cu -- bounded 8-path SGM on the windowed fine cost (Sec. III-E with Eq. 8-9).
//
// One warp per (direction, scanline).  Lane j owns slot j of the current pixel's window
// (chunks of 32 for wide windows).  The predecessor's path costs L' sit in a per-warp
// shared-memory buffer indexed by the predecessor's slot, so the ragged-window alignment
// (slot i = lo(p) + j - lo(p-r)) is a plain indexed read with bounds checks: labels outside
// the predecessor's window are absent from the minimum (Sec. III-E).  The step is the
// normalised recurrence
//   L(p,g) = C(p,g) + (min(L'(g), L'(g-1)+P1, L'(g+1)+P1, m+P2) - m),   m = min L',
// and the predecessor minimum m is one redux.sync.min.f32 per pixel.  The 8 directions run
// concurrently and add into agg (zeroed by the caller) with float atomics.
//
// Derived penalties: per-block partial sums (double) of the active slots, then one block
// adds the partials in a fixed order, so the mean is deterministic.
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

constexpr int kSgmWarps = 4;

__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__global__ void __launch_bounds__(32 * kSgmWarps) fine_sgm_kernel(const float *__restrict__ cost,
                                                                  const int *__restrict__ lo,
                                                                  const int *__restrict__ cnt,
                                                                  const long long *__restrict__ off,
                                                                  int H, int W, int Gs,
                                                                  const float *__restrict__ pen,
                                                                  int G, ScanTable st, float *__restrict__ agg,
                                                                  int *__restrict__ status) {
    extern __shared__ float sm[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kSgmWarps + wib;
    if (gw >= st.cum[8]) return;
    int r = 0;
    while (gw >= st.cum[r + 1]) r++;
    const int s = gw - st.cum[r];
    const int dx = dir_dx(r), dy = dir_dy(r);
    int x, y;
    scan_start(r, s, H, W, x, y);
    float *bufA = sm + (size_t)wib * 2 * Gs;
    float *bufB = bufA + Gs;
    const float P1 = __ldg(pen), P2 = __ldg(pen + 1);
    int plo = 0, pcnt = 0;
    float m = 0.f;
    bool first = true;
    while (x >= 0 && x < W && y >= 0 && y < H) {
        const int p = y * W + x;
        int l = __ldg(lo + p), n = __ldg(cnt + p);
        const long long o = __ldg(off + p);
        if (!window_ok(l, n, G, __ldg(off + p + 1) - o, status)) {
            l = 0;      // an invalid window takes no part: the path restarts after it
            n = 0;
            first = true;
        }
        float lmin = __int_as_float(0x7f800000);
        for (int j = lane; j < n; j += 32) {
            const float c = __ldg(cost + o + j);
            float Lv;
            if (first) {
                Lv = c;
            } else {
                const int i = l + j - plo;
                float t = m + P2;
                if (i >= 0 && i < pcnt) t = fminf(t, bufA[i]);
                if (i >= 1 && i - 1 < pcnt) t = fminf(t, bufA[i - 1] + P1);
                if (i + 1 >= 0 && i + 1 < pcnt) t = fminf(t, bufA[i + 1] + P1);
                Lv = c + (t - m);
            }
            bufB[j] = Lv;
            lmin = fminf(lmin, Lv);
            atomicAdd(agg + o + j, Lv);
        }
        m = warp_min(lmin);
        __syncwarp();
        if (n == 0) {
            x += dx;
            y += dy;
            continue;
        }
        float *tmp = bufA;
        bufA = bufB;
        bufB = tmp;
        plo = l;
        pcnt = n;
        first = false;
        x += dx;
        y += dy;
    }
}

// Per-block sums of the active costs and slot counts (rows are 16-byte aligned, read as float4;
// slots past cnt are masked).  Each thread adds its pixels in a fixed order, the block adds its
// warps in a fixed order: the partials, and hence the mean, are deterministic.
__global__ void cost_partial_kernel(const float *__restrict__ cost, const int *__restrict__ cnt,
                                    const long long *__restrict__ off, int N, int G,
                                    double *__restrict__ partial, int *__restrict__ status) {
    double s = 0.0, c = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        const long long o = off[p];
        const int n = cnt[p];
        if (!window_ok(0, n, G, off[p + 1] - o, status)) continue;
        const float4 *r = reinterpret_cast<const float4 *>(cost + o);
        float ps = 0.f;
        for (int j = 0; j < n; j += 4) {
            const float4 v = __ldg(r + (j >> 2));
            ps += v.x + (j + 1 < n ? v.y : 0.f) + (j + 2 < n ? v.z : 0.f) + (j + 3 < n ? v.w : 0.f);
        }
        s += (double)ps;
        c += n;
    }
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, k);
        c += __shfl_down_sync(0xffffffffu, c, k);
    }
    __shared__ double ws[32], wc[32];
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
        partial[gridDim.x + blockIdx.x] = bc;
    }
}

// Mean over the active slots: one warp adds the partials (lane-strided, then a fixed
// shuffle tree), so the result does not depend on timing.
__global__ void fine_penalty_kernel(const double *__restrict__ partial, int nblocks, double p1f, double p2f,
                                    float *__restrict__ pen) {
    double s = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += 32) {
        s += partial[i];
        c += partial[nblocks + i];
    }
    for (int k = 16; k > 0; k >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, k);
        c += __shfl_down_sync(0xffffffffu, c, k);
    }
    if (threadIdx.x == 0) {
        const double mean = c > 0.0 ? s / c : 0.0;
        pen[0] = (float)(p1f * mean);
        pen[1] = (float)(p2f * mean);
    }
}

}  // namespace

cudaError_t launch_cost_partial_sums(cudaStream_t s, const float *cost, const int *cnt, const long long *off,
                                     int N, int G, double *partial, int nblocks, int *status) {
    cost_partial_kernel<<<nblocks, 256, 0, s>>>(cost, cnt, off, N, G, partial, status);
    return cudaGetLastError();
}

cudaError_t launch_fine_penalties(cudaStream_t s, const double *partial, int nblocks, double p1f, double p2f,
                                  float *pen) {
    fine_penalty_kernel<<<1, 32, 0, s>>>(partial, nblocks, p1f, p2f, pen);
    return cudaGetLastError();
}

cudaError_t launch_fine_sgm(cudaStream_t s, const float *cost, const int *lo, const int *cnt,
                            const long long *off, int H, int W, int G, const float *pen, float *agg,
                            int *status) {
    const ScanTable st = make_scan_table(H, W);
    const int Gs = (G + 31) & ~31;
    const size_t smem = (size_t)kSgmWarps * 2 * Gs * sizeof(float);
    const unsigned grid = (unsigned)((st.cum[8] + kSgmWarps - 1) / kSgmWarps);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fine_sgm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    fine_sgm_kernel<<<grid, 32 * kSgmWarps, smem, s>>>(cost, lo, cnt, off, H, W, Gs, pen, G, st, agg, status);
    return cudaGetLastError();
}

}  // namespace lfsgm
