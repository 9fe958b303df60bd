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
// [gc - R, gc + R] saturated to [0, G-1]; a discarded pixel gets the whole range.
__global__ void windows_kernel(const int *__restrict__ F, int N, int G, int Lc, int R, int *__restrict__ lo,
                               int *__restrict__ cnt, float *__restrict__ dinit, int *__restrict__ cntpad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const int v = F[p];
    int a, n;
    if (v < 0) {
        a = 0;
        n = G;
        if (dinit) dinit[p] = __int_as_float(0x7fc00000);
    } else {
        const long long num = (long long)v * (G - 1);
        const long long den = 8LL * (Lc - 1);
        const long long gc = (2 * num + den) / (2 * den);
        long long lo_ = gc - R, hi_ = gc + R;
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

// Exclusive scan of the padded counts (one CTA of 1024 threads, contiguous chunks).
__global__ void __launch_bounds__(1024) scan_kernel(const int *__restrict__ cntpad, int N, long long *__restrict__ off) {
    __shared__ long long wsum[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int chunk = (N + 1023) / 1024;
    const int b = min(N, t * chunk), e = min(N, b + chunk);
    long long s = 0;
    for (int i = b; i < e; i++) s += cntpad[i];
    // inclusive warp scan
    long long inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    long long run = inc - s + (wid > 0 ? wsum[wid - 1] : 0);
    for (int i = b; i < e; i++) {
        off[i] = run;
        run += cntpad[i];
    }
    if (t == 1023) off[N] = wsum[31];
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
                           float *dinit, int *cntpad) {
    windows_kernel<<<(N + 255) / 256, 256, 0, s>>>(F, N, G, Lc, R, lo, cnt, dinit, cntpad);
    return cudaGetLastError();
}
cudaError_t launch_scan(cudaStream_t s, const int *cntpad, int N, long long *off) {
    scan_kernel<<<1, 1024, 0, s>>>(cntpad, N, off);
    return cudaGetLastError();
}

}  // namespace lfsgm
