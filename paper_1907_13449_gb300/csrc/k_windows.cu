// k_windows.cu -- from the per-arm maps to the fine search windows (Sec. III-D, Eq. 11):
// sequential fusion with threshold phi, median hole filling (Jacobi passes), borders on
// the fine grid and the exclusive scan giving the padded row offsets.
//
// D_init is kept in fixed point, in units of 1/8 coarse label: with at most four maps the
// running pairwise average m <- (m + 8 k_i) / 2 stays an exact integer (8k1, 4(k1+k2), ...),
// and -1 marks a discarded pixel.
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

__global__ void fuse_kernel(const int *__restrict__ maps, int narms, int N, double phi, int *__restrict__ F) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    int m = 8 * maps[p];
    bool ok = true;
    for (int i = 1; i < narms && ok; i++) {
        const int mi = 8 * maps[(size_t)i * N + p];
        if ((double)abs(m - mi) < 8.0 * phi) m = (m + mi) / 2;
        else ok = false;
    }
    F[p] = ok ? m : -1;
}

// One Jacobi pass: a discarded pixel takes the median (lower middle) of the valid values
// among its 8 neighbours in the input map; without valid neighbours it stays discarded.
__global__ void fill_kernel(const int *__restrict__ Fin, int *__restrict__ Fout, int H, int W) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const int v = Fin[p];
    if (v >= 0) { Fout[p] = v; return; }
    const int x = p % W, y = p / W;
    int vals[8];
    int n = 0;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            if (dx == 0 && dy == 0) continue;
            const int xx = x + dx, yy = y + dy;
            if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
            const int q = Fin[yy * W + xx];
            if (q >= 0) {
                int j = n++;
                while (j > 0 && vals[j - 1] > q) { vals[j] = vals[j - 1]; j--; }
                vals[j] = q;
            }
        }
    Fout[p] = n > 0 ? vals[(n - 1) / 2] : -1;
}

// Borders (Eq. 11): nearest fine label gc = round_half_up(m (G-1) / (8 (Lc-1))), window
// [gc - R, gc + R] saturated to [0, G-1]; a discarded pixel gets the whole range, and so does
// every pixel in the boundary-less mode (Sec. IV-E; F is not read).  Rfar > 0 makes the
// threshold depth-dependent (Sec. IV-F proposes a larger one for small disparities): linear from
// Rfar at gc = 0 to R at gc = G-1, R(gc) = R + floor((2 (Rfar - R)(G-1-gc) + G-1) / (2 (G-1))).
// Edge test of the border exclusion (Sec. III-D) on the edge-padded reference view (a padded read
// is the clamped read): the 3 x 3 Sobel sums, their squares and the comparison in FP32 with
// explicit rounding, in the order the oracle uses, so both take the same decision.
__device__ __forceinline__ bool sobel_edge(const float *I, int sx, int sy, float t) {
    const float q0 = I[-sy - sx], q1 = I[-sy], q2 = I[-sy + sx];
    const float q3 = I[-sx], q5 = I[sx];
    const float q6 = I[sy - sx], q7 = I[sy], q8 = I[sy + sx];
    const float gx = __fsub_rn(__fadd_rn(__fadd_rn(q2, __fmul_rn(2.0f, q5)), q8),
                               __fadd_rn(__fadd_rn(q0, __fmul_rn(2.0f, q3)), q6));
    const float gy = __fsub_rn(__fadd_rn(__fadd_rn(q6, __fmul_rn(2.0f, q7)), q8),
                               __fadd_rn(__fadd_rn(q0, __fmul_rn(2.0f, q1)), q2));
    return __fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)) > __fmul_rn(t, t);
}

__global__ void windows_kernel(const int *__restrict__ F, int N, int G, int Lc, int R, int *__restrict__ lo,
                               int *__restrict__ cnt, float *__restrict__ dinit, int *__restrict__ cntpad,
                               const float *__restrict__ ref_pad, int C, int P, int Wp, int W,
                               float edge_t, int Rfar, int boundless) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int v = boundless ? -1 : F[p];
    // an edge in any channel of the padded reference view (colour: one float4 per pixel, the
    // channels interleaved)
    bool edge = false;
    if (edge_t > 0.f && !boundless) {
        const int sx = C == 1 ? 1 : 4;
        const float *q = ref_pad + ((size_t)(p / W + P) * Wp + (p % W + P)) * sx;
        for (int ch = 0; ch < C && !edge; ch++) edge = sobel_edge(q + ch, sx, sx * Wp, edge_t);
    }
    int a, n;
    if (v < 0 || edge) {
        a = 0;
        n = G;
        if (dinit) dinit[p] = v < 0 ? __int_as_float(0x7fc00000) : 0.125f * (float)v;
    } else {
        const long long num = (long long)v * (G - 1);
        const long long den = 8LL * (Lc - 1);
        const long long gc = (2 * num + den) / (2 * den);
        long long r = R;
        if (Rfar > 0) {
            const long long dg = G - 1, t = 2 * (long long)(Rfar - R) * (dg - gc) + dg;
            long long q = t / (2 * dg);
            if (t % (2 * dg) != 0 && t < 0) q--;          // floor division
            r = R + q;
        }
        long long lo_ = gc - r, hi_ = gc + r;
        if (lo_ < 0) lo_ = 0;
        if (hi_ > G - 1) hi_ = G - 1;
        a = (int)lo_;
        n = (int)(hi_ - lo_ + 1);
        if (dinit) dinit[p] = 0.125f * (float)v;
    }
    lo[p] = a;
    cnt[p] = n;
    cntpad[p] = (n + 3) & ~3;
}

// Exclusive scan of the padded counts in three phases over tiles of 1024 entries:
// per-tile sums, a scan of the tile sums (one CTA), then per-tile scans plus the tile offset.
constexpr int kScanTile = 1024;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *wsum, long long *total) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    const long long ex = inc - v + (wid > 0 ? wsum[wid - 1] : 0);
    if (total) *total = wsum[(blockDim.x >> 5) - 1];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(kScanTile) scan_tile_sums(const int *__restrict__ cntpad, int N, long long *__restrict__ tsum) {
    __shared__ long long wsum[32];
    const int i = blockIdx.x * kScanTile + threadIdx.x;
    long long v = i < N ? cntpad[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < kScanTile / 32; w++) s += wsum[w];
        tsum[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kScanTile) scan_tile_offsets(long long *__restrict__ tsum, int ntiles) {
    __shared__ long long wsum[32];
    long long carry = 0;
    for (int base = 0; base < ntiles; base += kScanTile) {
        const int i = base + threadIdx.x;
        const long long v = i < ntiles ? tsum[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, wsum, &total);
        if (i < ntiles) tsum[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanTile) scan_apply(const int *__restrict__ cntpad, int N, const long long *__restrict__ toff,
                                                        long long *__restrict__ off) {
    __shared__ long long wsum[32];
    const int i = blockIdx.x * kScanTile + threadIdx.x;
    const long long v = i < N ? cntpad[i] : 0;
    const long long ex = block_exclusive_scan(v, wsum, nullptr);
    const long long o = toff[blockIdx.x] + ex;
    if (i < N) off[i] = o;
    if (i == N - 1) off[N] = o + v;
}

}  // namespace

cudaError_t launch_fuse(cudaStream_t s, const int *maps, int narms, int N, double phi, int *F) {
    fuse_kernel<<<(N + 255) / 256, 256, 0, s>>>(maps, narms, N, phi, F);
    return cudaGetLastError();
}
cudaError_t launch_fill(cudaStream_t s, const int *Fin, int *Fout, int H, int W) {
    fill_kernel<<<(H * W + 255) / 256, 256, 0, s>>>(Fin, Fout, H, W);
    return cudaGetLastError();
}
cudaError_t launch_windows(cudaStream_t s, const int *F, int N, int G, int Lc, int R, int *lo, int *cnt,
                           float *dinit, int *cntpad, const float *ref_pad, int C, int P, int Wp,
                           int W, float edge_t, int Rfar, int boundless) {
    windows_kernel<<<(N + 255) / 256, 256, 0, s>>>(F, N, G, Lc, R, lo, cnt, dinit, cntpad, ref_pad, C, P, Wp,
                                                   W, edge_t, Rfar, boundless);
    return cudaGetLastError();
}
int scan_tiles(int N) { return (N + kScanTile - 1) / kScanTile; }

cudaError_t launch_scan_sums(cudaStream_t s, const int *cntpad, int N, long long *tsum) {
    scan_tile_sums<<<scan_tiles(N), kScanTile, 0, s>>>(cntpad, N, tsum);
    return cudaGetLastError();
}
cudaError_t launch_scan_top(cudaStream_t s, long long *tsum, int N) {
    scan_tile_offsets<<<1, kScanTile, 0, s>>>(tsum, scan_tiles(N));
    return cudaGetLastError();
}
cudaError_t launch_scan_apply(cudaStream_t s, const int *cntpad, int N, const long long *tsum, long long *off) {
    scan_apply<<<scan_tiles(N), kScanTile, 0, s>>>(cntpad, N, tsum, off);
    return cudaGetLastError();
}

}  // namespace lfsgm
