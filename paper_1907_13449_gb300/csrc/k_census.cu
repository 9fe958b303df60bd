// k_census.cu -- Census transform (Sec. III-B, Eq. 2-3) of selected views.
//
// Bit k of the word of pixel (x,y) is 1 iff I(x,y) > I(x+dx,y+dy) for the k-th offset of
// the w x w window without its centre, offsets row-major (dy outer, dx inner), bit 0
// first; neighbour coordinates are clamped to the image.  One 32x8 CTA per tile and
// view; the tile plus its halo is staged in shared memory with clamped loads, so every
// neighbour read is a shared-memory read.  Output: one 64-bit word per pixel per view,
// census[view][y][x] (24 bits for 5x5, 48 bits for 7x7).
#include "lfsgm_internal.cuh"

namespace lfsgm {
namespace {

constexpr int TX = 32, TY = 8;

// Census word of the pixel whose (2 HALF + 1)^2 window starts at t (row stride ld, centre value c):
// bit k = [c > neighbour k], neighbours row-major without the centre, bit 0 first.  c > nb holds
// exactly when nb - c is negative (the difference of two distinct finite floats never rounds to
// zero, x - x = +0, and the tile holds no -0: values are staged as x + 0, which maps -0 to +0),
// so each bit is the sign of one FP32 subtraction, shifted into the word
// by a funnel shift; neighbours are visited last to first so that neighbour 0 ends in bit 0.
template <int HALF>
__device__ __forceinline__ uint64_t census_word(const float *t, int ld, float c) {
    constexpr int WN = 2 * HALF + 1, NB = WN * WN - 1, CEN = HALF * WN + HALF;
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int k = NB - 1; k >= 0; k--) {
        const int q = k < CEN ? k : k + 1;                 // window position of neighbour k
        const float d = t[(q / WN) * ld + (q % WN)] - c;
        if (k >= 32) hi = __funnelshift_l(__float_as_uint(d), hi, 1);
        else lo = __funnelshift_l(__float_as_uint(d), lo, 1);
    }
    return ((uint64_t)hi << 32) | lo;
}

template <int HALF>
__global__ void __launch_bounds__(TX *TY) census_kernel(const float *__restrict__ views, int H, int W,
                                                        const int *__restrict__ sel,
                                                        uint64_t *__restrict__ cen) {
    constexpr int SW = TX + 2 * HALF, SH = TY + 2 * HALF;
    __shared__ float tile[SH][SW + 1];
    const size_t HW = (size_t)H * W;
    const int view = sel[blockIdx.z];
    const float *img = views + (size_t)view * HW;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.y * TX + threadIdx.x;
    for (int i = tid; i < SH * SW; i += TX * TY) {
        int ty = i / SW, tx = i - ty * SW;
        int gy = min(max(y0 + ty - HALF, 0), H - 1);
        int gx = min(max(x0 + tx - HALF, 0), W - 1);
        tile[ty][tx] = __ldg(img + (size_t)gy * W + gx) + 0.0f;   // -0 becomes +0 (see census_word)
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= W || y >= H) return;
    const float c = tile[threadIdx.y + HALF][threadIdx.x + HALF];
    cen[(size_t)view * HW + (size_t)y * W + x] = census_word<HALF>(&tile[threadIdx.y][threadIdx.x], SW + 1, c);
}

// (v - c0, v - c1) as one packed FP32 subtraction (sm_100+): each half is rounded exactly as the
// scalar subtraction would be, so the signs are the same.
__device__ __forceinline__ void sub_pair(float v, float c0, float c1, uint32_t &d0, uint32_t &d1) {
    unsigned long long r;
    asm("{\n .reg .b64 va, vc;\n mov.b64 va, {%1, %1};\n mov.b64 vc, {%2, %3};\n sub.rn.f32x2 %0, va, vc;\n}"
        : "=l"(r) : "f"(v), "f"(c0), "f"(c1));
    d0 = (uint32_t)r;
    d1 = (uint32_t)(r >> 32);
}

// Census words of PPT vertically adjacent pixels whose windows start at t, t + ld, ...: every tile
// value of the union of their windows is read once, and each word takes its own neighbours in
// descending order (rows bottom-up, columns right to left), as census_word does.  Where a tile
// value is a neighbour of both pixels of a pair (0, 1), (2, 3), ..., the two differences are one
// packed subtraction.
template <int HALF, int PPT>
__device__ __forceinline__ void census_words(const float *t, int ld, const float (&c)[PPT], uint64_t (&w)[PPT]) {
    static_assert(PPT % 2 == 0, "pixels in pairs");
    constexpr int WN = 2 * HALF + 1, CEN = HALF * WN + HALF;
    uint32_t lo[PPT], hi[PPT];
#pragma unroll
    for (int i = 0; i < PPT; i++) lo[i] = hi[i] = 0;
#pragma unroll
    for (int ry = WN + PPT - 2; ry >= 0; ry--) {       // union row: window row ry - i of pixel i
#pragma unroll
        for (int rx = WN - 1; rx >= 0; rx--) {
            const float v = t[ry * ld + rx];
#pragma unroll
            for (int i = 0; i < PPT; i += 2) {
                const int r0 = ry - i, r1 = ry - i - 1;
                const int q0 = r0 * WN + rx, q1 = r1 * WN + rx;
                const bool use0 = r0 >= 0 && r0 < WN && q0 != CEN, use1 = r1 >= 0 && r1 < WN && q1 != CEN;
                uint32_t d0 = 0, d1 = 0;
                if (use0 && use1) sub_pair(v, c[i], c[i + 1], d0, d1);
                else if (use0) d0 = __float_as_uint(v - c[i]);
                else if (use1) d1 = __float_as_uint(v - c[i + 1]);
                if (use0) {
                    const int k = q0 < CEN ? q0 : q0 - 1;
                    if (k >= 32) hi[i] = __funnelshift_l(d0, hi[i], 1);
                    else lo[i] = __funnelshift_l(d0, lo[i], 1);
                }
                if (use1) {
                    const int k = q1 < CEN ? q1 : q1 - 1;
                    if (k >= 32) hi[i + 1] = __funnelshift_l(d1, hi[i + 1], 1);
                    else lo[i + 1] = __funnelshift_l(d1, lo[i + 1], 1);
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PPT; i++) w[i] = ((uint64_t)hi[i] << 32) | lo[i];
}

// Same transform, written into edge-replicated padded images: word and value of pixel (x,y) go to
// (x+P, y+P), and border pixels also fill the padding rows/columns next to them, so that a read
// at any padded position (xp, yp) returns the word/value of pixel (clamp(xp-P), clamp(yp-P)) --
// exactly the clamped read of the unpadded image.  Padded row stride Wp, Hp rows per view.
// A 32 x 4 thread block covers a 32 x 4 PPT tile: each thread takes PPT vertically adjacent pixels
// (grey 4: the tile's halo rows and the union windows are shared by more pixels; colour 2).
// Colour (C = 3): one block per view transforms the C channel planes in turn (census words go to
// the planes view * C + c), and the padded view is written interleaved, one float4 (the C
// channels and a zero) per pixel, so that a bilinear tap of all channels is one 16-byte load.
template <int HALF, int C, int PPT>
__device__ __forceinline__ void census_pad_body(const float *__restrict__ views, int H, int W, int P, int Wp, int Hp,
                                                const int *__restrict__ sel, uint64_t *__restrict__ cen_pad,
                                                float *__restrict__ views_pad) {
    constexpr int BY = 4, TYB = BY * PPT;              // thread rows, tile rows
    constexpr int SW = TX + 2 * HALF, SH = TYB + 2 * HALF;
    __shared__ float tile[SH][SW + 1];
    const size_t HW = (size_t)H * W, HWp = (size_t)Hp * Wp;
    const int view = sel[blockIdx.z];
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TYB;
    const int x = x0 + threadIdx.x, ty0 = PPT * threadIdx.y, y = y0 + ty0;
    const bool inb = x < W && y < H;
    const int xa = x == 0 ? 0 : x + P, xb = x == W - 1 ? Wp - 1 : x + P;
    // tile fill: thread (tx, ty) loads column tx of tile rows ty, ty + 4, ..., and the first 2 HALF
    // lanes also load the halo columns 32 .. SW-1 (clamped coordinates)
    const int gx0 = min(max(x0 + (int)threadIdx.x - HALF, 0), W - 1);
    const int gx1 = min(max(x0 + TX + (int)threadIdx.x - HALF, 0), W - 1);
    const bool halo = threadIdx.x < 2 * HALF;
    float cv[PPT][C] = {};
#pragma unroll
    for (int ch = 0; ch < C; ch++) {
        const float *img = views + ((size_t)view * C + ch) * HW;
        if (ch) __syncthreads();                                   // the previous channel's tile is used up
#pragma unroll
        for (int ty = threadIdx.y; ty < SH; ty += BY) {
            const float *src = img + (size_t)min(max(y0 + ty - HALF, 0), H - 1) * W;
            tile[ty][threadIdx.x] = __ldg(src + gx0) + 0.0f;       // -0 becomes +0 (see census_word)
            if (halo) tile[ty][TX + threadIdx.x] = __ldg(src + gx1) + 0.0f;
        }
        __syncthreads();
        uint64_t w[PPT];
#pragma unroll
        for (int i = 0; i < PPT; i++) w[i] = 0ull;
        if (inb) {
            float c[PPT];
#pragma unroll
            for (int i = 0; i < PPT; i++) {
                c[i] = tile[ty0 + i + HALF][threadIdx.x + HALF];
                cv[i][ch] = c[i];
            }
            census_words<HALF, PPT>(&tile[ty0][threadIdx.x], SW + 1, c, w);
        }
        // the census words of this channel, and with the last channel the padded view
        auto put = [&](uint64_t *cp, size_t q, uint64_t word, const float *val) {
            cp[q] = word;
            if (ch == C - 1) {
                if constexpr (C == 1)
                    views_pad[(size_t)view * HWp + q] = val[0];
                else
                    reinterpret_cast<float4 *>(views_pad)[(size_t)view * HWp + q] =
                        make_float4(val[0], val[1], val[2], 0.f);
            }
        };
        if constexpr (C == 1) {
            // A warp is one thread row, so y and yr are the same on all its lanes.  A pixel that is
            // not on the left or right border writes one padded column (one position inside, the
            // padding rows above or below it on the top and bottom rows), its lanes side by side;
            // the rectangle of a left or right border pixel is written by the whole warp, lanes
            // along x (a lane alone would write (P+1)^2 positions at a corner).
            if (y < H) {
                uint64_t *cp = cen_pad + (size_t)view * HWp;
                const bool xedge = inb && (x == 0 || x == W - 1);
#pragma unroll
                for (int r = 0; r < PPT; r++) {
                    const int yr = y + r;
                    if (yr >= H) break;
                    const int ya = yr == 0 ? 0 : yr + P, yb = yr == H - 1 ? Hp - 1 : yr + P;
                    if (inb && !xedge)
                        for (int yy = ya; yy <= yb; yy++) put(cp, (size_t)yy * Wp + xa, w[r], cv[r]);
                    unsigned m = __ballot_sync(0xffffffffu, xedge);
                    while (m) {
                        const int src = __ffs(m) - 1;
                        m &= m - 1;
                        const uint64_t ws = __shfl_sync(0xffffffffu, w[r], src);
                        const int sa = __shfl_sync(0xffffffffu, xa, src), sb = __shfl_sync(0xffffffffu, xb, src);
                        const float vs = __shfl_sync(0xffffffffu, cv[r][0], src);
                        for (int yy = ya; yy <= yb; yy++)
                            for (int xx = sa + (int)threadIdx.x; xx <= sb; xx += 32)
                                put(cp, (size_t)yy * Wp + xx, ws, &vs);
                    }
                }
            }
        } else if (inb) {
            // colour: each lane writes its own pixel's rectangle (measured faster here than the
            // warp-wide border writes, which raise the register count of the three-channel kernel)
            uint64_t *cp = cen_pad + ((size_t)view * C + ch) * HWp;
#pragma unroll
            for (int r = 0; r < PPT; r++) {
                const int yr = y + r;
                if (yr >= H) break;
                if (xa == xb && yr != 0 && yr != H - 1) {             // interior: one padded position
                    put(cp, (size_t)(yr + P) * Wp + xa, w[r], cv[r]);
                    continue;
                }
                const int ya = yr == 0 ? 0 : yr + P, yb = yr == H - 1 ? Hp - 1 : yr + P;
                for (int yy = ya; yy <= yb; yy++)
                    for (int xx = xa; xx <= xb; xx++) put(cp, (size_t)yy * Wp + xx, w[r], cv[r]);
            }
        }
    }
}

// Grey: 4 pixels per thread, 12 CTAs of 128 threads per SM.  Colour: 2 pixels per thread, the
// compiler's own register count.
constexpr int kPptGrey = 4, kPptRgb = 2;
template <int HALF>
__global__ void __launch_bounds__(TX * 4, 12) census_pad_kernel(const float *__restrict__ views, int H, int W,
                                                                    int P, int Wp, int Hp,
                                                                    const int *__restrict__ sel,
                                                                    uint64_t *__restrict__ cen_pad,
                                                                    float *__restrict__ views_pad) {
    census_pad_body<HALF, 1, kPptGrey>(views, H, W, P, Wp, Hp, sel, cen_pad, views_pad);
}

template <int HALF>
__global__ void __launch_bounds__(TX * 4) census_pad_rgb_kernel(const float *__restrict__ views, int H, int W,
                                                                    int P, int Wp, int Hp,
                                                                    const int *__restrict__ sel,
                                                                    uint64_t *__restrict__ cen_pad,
                                                                    float *__restrict__ views_pad) {
    census_pad_body<HALF, 3, kPptRgb>(views, H, W, P, Wp, Hp, sel, cen_pad, views_pad);
}

}  // namespace

cudaError_t launch_census_pad(cudaStream_t s, const float *views, int H, int W, int census_w, int P, int Wp, int Hp,
                              int C, const int *d_sel, int nsel, uint64_t *cen_pad, float *views_pad) {
    const int rows = 4 * (C == 3 ? kPptRgb : kPptGrey);
    dim3 block(TX, 4), grid((W + TX - 1) / TX, (H + rows - 1) / rows, nsel);
    if (C == 3) {
        if (census_w == 5) census_pad_rgb_kernel<2><<<grid, block, 0, s>>>(views, H, W, P, Wp, Hp, d_sel, cen_pad, views_pad);
        else census_pad_rgb_kernel<3><<<grid, block, 0, s>>>(views, H, W, P, Wp, Hp, d_sel, cen_pad, views_pad);
    } else {
        if (census_w == 5) census_pad_kernel<2><<<grid, block, 0, s>>>(views, H, W, P, Wp, Hp, d_sel, cen_pad, views_pad);
        else census_pad_kernel<3><<<grid, block, 0, s>>>(views, H, W, P, Wp, Hp, d_sel, cen_pad, views_pad);
    }
    return cudaGetLastError();
}

cudaError_t launch_census(cudaStream_t s, const float *views, int H, int W, int census_w,
                          const int *d_sel, int nsel, uint64_t *cen) {
    dim3 block(TX, TY), grid((W + TX - 1) / TX, (H + TY - 1) / TY, nsel);
    if (census_w == 5) census_kernel<2><<<grid, block, 0, s>>>(views, H, W, d_sel, cen);
    else census_kernel<3><<<grid, block, 0, s>>>(views, H, W, d_sel, cen);
    return cudaGetLastError();
}

}  // namespace lfsgm
