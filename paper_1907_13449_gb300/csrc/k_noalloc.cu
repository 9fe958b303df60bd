// k_noalloc.cu -- lfsgm_cost_volume_noalloc: the bounded cost volume for callers that must
// not allocate device memory.
//
// Who needs it: code that runs under a fixed device-memory budget and is not allowed to call
// cudaMalloc once it is running -- a real-time loop that must never block on an allocation
// or fail half-way under memory pressure, or a plug-in inside a host application whose own
// allocator owns all device memory and whose accounting a raw cudaMalloc would bypass.  Such
// a caller cannot create a handle (lfsgm_create allocates the shift tables and the
// workspace), so this entry point takes the configuration directly and keeps its scratch --
// the shift table, the census words of every view and a status word -- in one file-scope
// device array of fixed size.
//
// The array is part of the library image: every GPU that loads this library holds its
// kNoAllocBytes until the process exits.  Host code cannot use the array's name as a device
// address (there it is only a host-side stand-in), so the first call on each device asks the
// runtime for the real address with cudaGetSymbolAddress, with that device current, and
// caches it.  Every call reuses the same array and leaves its contents behind; the kernels
// overwrite everything they read, and the status word is cleared at the start of each call.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lfsgm.h"
#include "lfsgm_internal.cuh"

using namespace lfsgm;

namespace {

constexpr size_t kNoAllocBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (resolved once per device).
lfsgm_status noalloc_scratch(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LFSGM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return LFSGM_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LFSGM_OK;
}

// The per (view, fine label) shift table, built on the device with the same IEEE double
// operations, in the same order, as the handle's host-side builder (so the two tables are
// identical), plus the list of all views for the census launcher.
__device__ void split_shift(int a, double d, int &o, double &f, int &n) {
    double s = __dmul_rn((double)a, d);
    const double t = __dmul_rn(2.0, s);
    const double r = rint(t);
    if (fabs(__dsub_rn(t, r)) <= 2e-9) s = __dmul_rn(0.5, r);
    const double fl = floor(s);
    o = (int)fl;
    f = __dsub_rn(s, fl);
    n = (int)floor(__dadd_rn(s, 0.5));
}

__global__ void noalloc_tables_kernel(FineTap *tab, int *sel, int U, int V, int uc, int vc, int G,
                                      double dmin, double dmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nviews = U * V;
    if (i < nviews) sel[i] = i;
    if (i >= nviews * G) return;
    const int view = i / G, g = i - view * G;
    const int u = view % U, v = view / U;
    const double step = __ddiv_rn(__dsub_rn(dmax, dmin), (double)(G - 1));
    const double d = __dadd_rn(dmin, __dmul_rn((double)g, step));
    int ox, oy, nx, ny;
    double fx, fy;
    split_shift(u - uc, d, ox, fx, nx);
    split_shift(v - vc, d, oy, fy, ny);
    FineTap t;
    t.ox = (int16_t)ox;
    t.oy = (int16_t)oy;
    t.nx = (int16_t)nx;
    t.ny = (int16_t)ny;
    t.fx = (float)fx;
    t.fy = (float)fy;
    tab[i] = t;
}

}  // namespace

extern "C" lfsgm_status lfsgm_cost_volume_noalloc(const lfsgm_config *cfg, void *stream, const float *views,
                                                  const int32_t *lo, const int32_t *cnt, const int64_t *off,
                                                  float *cost) {
    if (!cfg || !views || !lo || !cnt || !off || !cost || ((uintptr_t)cost & 15) != 0) return LFSGM_ERR_INVALID_ARG;
    const lfsgm_config &c = *cfg;
    const int uc = c.uc < 0 ? (c.U - 1) / 2 : c.uc, vc = c.vc < 0 ? (c.V - 1) / 2 : c.vc;
    if (c.U < 1 || c.V < 1 || c.U * c.V < 2 || c.U > 64 || c.V > 64 || c.H < 1 || c.W < 1 ||
        uc >= c.U || vc >= c.V || (c.census_w != 5 && c.census_w != 7) || !(c.dmax > c.dmin) ||
        c.fine_labels < 2 || c.fine_labels > 4096 || !(c.w_l2 >= 0.f) || !(c.w_census >= 0.f) ||
        !std::isfinite(c.w_l2) || !std::isfinite(c.w_census) ||
        std::fmax(std::fabs(c.dmin), std::fabs(c.dmax)) * (c.U > c.V ? c.U : c.V) > 30000.0)
        return LFSGM_ERR_INVALID_ARG;
    if (c.channels != 0 && c.channels != 1) return c.channels == 3 ? LFSGM_ERR_UNSUPPORTED : LFSGM_ERR_INVALID_ARG;
    const size_t nviews = (size_t)c.U * c.V, N = (size_t)c.H * c.W, G = (size_t)c.fine_labels;
    // scratch layout: status word | view list | shift table | census words of every view
    const size_t o_sel = 256, o_tab = o_sel + round256(nviews * 4), o_cen = o_tab + round256(nviews * G * 16);
    const size_t need = o_cen + nviews * N * 8;
    if (need > kNoAllocBytes) return LFSGM_ERR_UNSUPPORTED;
    void *base = nullptr;
    const lfsgm_status st = noalloc_scratch(&base);
    if (st != LFSGM_OK) return st;
    unsigned char *b = (unsigned char *)base;
    int *status = (int *)b;
    int *sel = (int *)(b + o_sel);
    FineTap *tab = (FineTap *)(b + o_tab);
    uint64_t *cen = (uint64_t *)(b + o_cen);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return LFSGM_ERR_CUDA;
    const int n_tab = (int)(nviews * G);
    noalloc_tables_kernel<<<(n_tab + 255) / 256, 256, 0, s>>>(tab, sel, c.U, c.V, uc, vc, c.fine_labels, c.dmin,
                                                              c.dmax);
    if (cudaGetLastError() != cudaSuccess) return LFSGM_ERR_CUDA;
    if (launch_census(s, views, c.H, c.W, c.census_w, sel, (int)nviews, cen) != cudaSuccess) return LFSGM_ERR_CUDA;
    if (launch_fine_cost(s, views, cen, tab, c.fine_labels, (int)nviews, c.H, c.W, vc * c.U + uc, lo, cnt,
                         (const long long *)off, c.w_l2, c.w_census, cost, status) != cudaSuccess)
        return LFSGM_ERR_CUDA;
    return LFSGM_OK;
}
