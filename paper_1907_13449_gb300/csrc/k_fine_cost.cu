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

}  // namespace

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
