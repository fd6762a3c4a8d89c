// tp_domain.cu -- the device side of the spatial decomposition of one box over
// several GPUs (Sec. II): particle ownership under a 3-D multi-section
// geometry, the ghost sets (particles within r_cut of another domain's box,
// the analogue of the paper's exchange of tree data between processes), and
// the row gathers and scatter-adds that pack and unpack the exchange buffers.
//
// Geometry: nx slabs along x cut at xc[0..nx]; slab i is cut into ny columns
// along y at yc[i][0..ny]; column (i, j) into nz cells along z at
// zc[i][j][0..nz].  Domain d = (i ny + j) nz + k is the half-open box
// [xc[i], xc[i+1]) x [yc[i][j], yc[i][j+1]) x [zc[i][j][k], zc[i][j][k+1]).
// First cuts 0, last cuts 1, each list non-decreasing: the domains tile the
// unit box.
//
// Selection output: the indices of the selected particles grouped by
// destination domain (domain 0 first) and ascending within each destination,
// so the lists do not depend on thread timing.  A count pass fills per-block
// counts per destination, an exclusive scan turns them into offsets, and a
// write pass ranks each block's particles per destination with warp ballots.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tp_common.cuh"

namespace tp {
size_t scan_tmp_bytes();
void scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n_host, const int64_t *d_n,
                     int64_t *total, void *tmp, cudaStream_t s);
}  // namespace tp

namespace {

constexpr int kHaloBlock = 256;
constexpr int kHaloWarps = kHaloBlock / 32;

struct HaloGeom {
    int32_t nx, ny, nz, ndom;
    const double *xc, *yc, *zc;       // cuts, as described above
    const double *lo, *hi;            // [ndom][3] domain boxes (from the cuts)
};

__device__ __forceinline__ double halo_wrap(double x)
{
    const double w = __dsub_rn(x, floor(x));
    return w >= 1.0 ? 0.0 : w;
}

// Largest i in [0, m-1] with c[i] <= v (c[0] <= v holds for wrapped v).
__device__ __forceinline__ int halo_slot(const double *c, int m, double v)
{
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int halo_owner(const HaloGeom &g, double x, double y, double z)
{
    const int i = halo_slot(g.xc, g.nx, x);
    const int j = halo_slot(g.yc + (int64_t)i * (g.ny + 1), g.ny, y);
    const int k = halo_slot(g.zc + ((int64_t)i * g.ny + j) * (g.nz + 1), g.nz, z);
    return (i * g.ny + j) * g.nz + k;
}

// Periodic distance along one axis from p in [0,1) to the box [lo, hi) within
// [0,1]: 0 inside; else the shorter way round, each difference rounded once.
__device__ __forceinline__ double halo_gap(double p, double lo, double hi)
{
    if (p < lo) return fmin(__dsub_rn(lo, p), __dsub_rn(__dadd_rn(p, 1.0), hi));
    if (p >= hi) return fmin(__dsub_rn(p, hi), __dsub_rn(__dadd_rn(lo, 1.0), p));
    return 0.0;
}

__device__ __forceinline__ bool halo_near(const HaloGeom &g, int d, double x, double y, double z, double rc2)
{
    const double *lo = g.lo + 3 * (int64_t)d, *hi = g.hi + 3 * (int64_t)d;
    const double gx = halo_gap(x, lo[0], hi[0]), gy = halo_gap(y, lo[1], hi[1]), gz = halo_gap(z, lo[2], hi[2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
    return d2 < rc2;
}

// Does particle (x,y,z) go to domain d?  mode 0: d owns it; mode 1: d is not
// `self` and its box lies within r_cut of the particle.
__device__ __forceinline__ bool halo_goes(const HaloGeom &g, int mode, int self, int owner, int d, double x,
                                          double y, double z, double rc2)
{
    if (mode == 0) return d == owner;
    return d != self && halo_near(g, d, x, y, z, rc2);
}

__global__ void k_halo_boxes(HaloGeom g, double *lo, double *hi)
{
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < g.ndom; d += gridDim.x * blockDim.x) {
        const int k = d % g.nz, j = (d / g.nz) % g.ny, i = d / (g.nz * g.ny);
        const double *yc = g.yc + (int64_t)i * (g.ny + 1);
        const double *zc = g.zc + ((int64_t)i * g.ny + j) * (g.nz + 1);
        lo[3 * d] = g.xc[i]; hi[3 * d] = g.xc[i + 1];
        lo[3 * d + 1] = yc[j]; hi[3 * d + 1] = yc[j + 1];
        lo[3 * d + 2] = zc[k]; hi[3 * d + 2] = zc[k + 1];
    }
}

// Per-block counts per destination: bc[d * nblk + b].
__global__ void __launch_bounds__(kHaloBlock) k_halo_count(HaloGeom g, const double *pos, int64_t n, int mode,
                                                           int self, double rc2, int32_t *bc, int64_t nblk,
                                                           int32_t *status)
{
    extern __shared__ int32_t cnt[];
    for (int d = threadIdx.x; d < g.ndom; d += blockDim.x) cnt[d] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)kHaloBlock + threadIdx.x;
    if (i < n) {
        const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) {
            atomicCAS(status, 0, (int32_t)TP_ERR_NONFINITE);
        } else {
            const double x = halo_wrap(px), y = halo_wrap(py), z = halo_wrap(pz);
            const int owner = halo_owner(g, x, y, z);
            if (mode == 0) {
                atomicAdd(&cnt[owner], 1);
            } else {
                for (int d = 0; d < g.ndom; d++)
                    if (halo_goes(g, mode, self, owner, d, x, y, z, rc2)) atomicAdd(&cnt[d], 1);
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < g.ndom; d += blockDim.x) bc[(int64_t)d * nblk + blockIdx.x] = cnt[d];
}

// Writes each selected index at off[d * nblk + b] + its rank among the block's
// particles bound for d (ascending index).
__global__ void __launch_bounds__(kHaloBlock) k_halo_write(HaloGeom g, const double *pos, int64_t n, int mode,
                                                           int self, double rc2, const int64_t *off, int64_t nblk,
                                                           int32_t *idx, int64_t cap)
{
    __shared__ int32_t wc[kHaloWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)kHaloBlock + threadIdx.x;
    bool ok = i < n;
    double x = 0.0, y = 0.0, z = 0.0;
    int owner = -1;
    if (ok) {
        const double px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
        ok = isfinite(px) && isfinite(py) && isfinite(pz);
        if (ok) {
            x = halo_wrap(px); y = halo_wrap(py); z = halo_wrap(pz);
            owner = halo_owner(g, x, y, z);
        }
    }
    const unsigned lt = (1u << lane) - 1u;
    for (int d = 0; d < g.ndom; d++) {
        const bool go = ok && halo_goes(g, mode, self, owner, d, x, y, z, rc2);
        const unsigned b = __ballot_sync(0xffffffffu, go);
        if (lane == 0) wc[warp] = __popc(b);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; w++) before += wc[w];
        if (go) {
            const int64_t at = off[(int64_t)d * nblk + blockIdx.x] + before + __popc(b & lt);
            if (at < cap) idx[at] = (int32_t)i;
        }
        __syncthreads();
    }
}

template <int WORDS>
__global__ void k_gather_rows_w(const uint32_t *src, const int32_t *idx, int64_t m, uint32_t *dst)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx[r];
#pragma unroll
        for (int w = 0; w < WORDS; w++) dst[WORDS * r + w] = src[WORDS * s + w];
    }
}

__global__ void k_gather_rows(const uint32_t *src, int words, const int32_t *idx, int64_t m, uint32_t *dst)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * words;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / words, w = t % words;
        dst[t] = src[(int64_t)idx[r] * words + w];
    }
}

__global__ void k_scatter_add_rows(double *dst, int width, const int32_t *idx, const double *src, int64_t m)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m * width;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / width, w = t % width;
        atomicAdd(dst + (int64_t)idx[r] * width + w, src[t]);
    }
}

bool halo_is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

tp_status halo_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return TP_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
}

}  // namespace

struct tp_halo {
    int32_t nx = 0, ny = 0, nz = 0, ndom = 0;
    bool has_cuts = false;
    double *cuts = nullptr;           // device: xc, yc, zc back to back
    double *boxes = nullptr;          // device: lo [ndom][3], hi [ndom][3]
    int32_t *status = nullptr;        // device: non-finite positions
    // count-pass scratch, grown on demand
    int64_t cap_blk = 0;
    int32_t *bc = nullptr;
    int64_t *off = nullptr;
    void *scan_tmp = nullptr;
    int64_t *d_total = nullptr;
    HaloGeom geom() const
    {
        HaloGeom g;
        g.nx = nx; g.ny = ny; g.nz = nz; g.ndom = ndom;
        g.xc = cuts;
        g.yc = cuts + (nx + 1);
        g.zc = g.yc + (int64_t)nx * (ny + 1);
        g.lo = boxes;
        g.hi = boxes + 3 * (int64_t)ndom;
        return g;
    }
};

extern "C" {

tp_status tp_halo_create(int32_t nx, int32_t ny, int32_t nz, tp_halo **out)
{
    if (!out) return TP_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz > TP_MAX_DOMAINS) return TP_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return TP_ERR_NO_DEVICE;
    }
    tp_halo *h = new tp_halo();
    h->nx = nx; h->ny = ny; h->nz = nz; h->ndom = nx * ny * nz;
    const size_t ncut = (size_t)(nx + 1) + (size_t)nx * (ny + 1) + (size_t)nx * ny * (nz + 1);
    cudaError_t e = cudaMalloc(&h->cuts, sizeof(double) * ncut);
    if (e == cudaSuccess) e = cudaMalloc(&h->boxes, sizeof(double) * 6 * (size_t)h->ndom);
    if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->d_total, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->scan_tmp, tp::scan_tmp_bytes());
    if (e != cudaSuccess) {
        tp_halo_free(h);
        return halo_cuda(e);
    }
    *out = h;
    return TP_OK;
}

tp_status tp_halo_set_cuts(tp_halo *h, const double *xc, const double *yc, const double *zc)
{
    if (!h || !xc || !yc || !zc) return TP_ERR_INVALID_ARG;
    const int nx = h->nx, ny = h->ny, nz = h->nz;
    auto check = [](const double *c, int m) {
        if (!(c[0] == 0.0) || !(c[m] == 1.0)) return false;
        for (int i = 0; i < m; i++)
            if (!(c[i] <= c[i + 1])) return false;
        return true;
    };
    if (!check(xc, nx)) return TP_ERR_INVALID_ARG;
    for (int i = 0; i < nx; i++) {
        if (!check(yc + (int64_t)i * (ny + 1), ny)) return TP_ERR_INVALID_ARG;
        for (int j = 0; j < ny; j++)
            if (!check(zc + ((int64_t)i * ny + j) * (nz + 1), nz)) return TP_ERR_INVALID_ARG;
    }
    std::vector<double> all;
    all.insert(all.end(), xc, xc + nx + 1);
    all.insert(all.end(), yc, yc + (size_t)nx * (ny + 1));
    all.insert(all.end(), zc, zc + (size_t)nx * ny * (nz + 1));
    tp_status st = halo_cuda(cudaMemcpy(h->cuts, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice));
    if (st != TP_OK) return st;
    const HaloGeom g = h->geom();
    TP_LAUNCH(k_halo_boxes, (h->ndom + 127) / 128, 128, 0, (cudaStream_t)0, g, h->boxes,
              h->boxes + 3 * (int64_t)h->ndom);
    st = halo_cuda(cudaDeviceSynchronize());
    if (st == TP_OK) h->has_cuts = true;
    return st;
}

tp_status tp_halo_select(tp_halo *h, const double *pos, int64_t n, int32_t mode, int32_t self, double r_cut,
                         int32_t *idx, int64_t cap, int64_t *counts, void *stream)
{
    if (!h || !h->has_cuts || !counts || n < 0 || n >= (1ll << 31) - 1 || cap < 0) return TP_ERR_INVALID_ARG;
    if (mode != TP_HALO_OWNER && mode != TP_HALO_GHOSTS) return TP_ERR_INVALID_ARG;
    if (mode == TP_HALO_GHOSTS && (!(r_cut > 0.0 && r_cut < 0.5) || self < 0 || self >= h->ndom))
        return TP_ERR_INVALID_ARG;
    for (int d = 0; d < h->ndom; d++) counts[d] = 0;
    if (n == 0) return TP_OK;
    if (!halo_is_device_ptr(pos) || (cap > 0 && !halo_is_device_ptr(idx))) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nblk = (n + kHaloBlock - 1) / kHaloBlock;
    if (nblk > h->cap_blk) {
        cudaFree(h->bc);
        cudaFree(h->off);
        h->bc = nullptr;
        h->off = nullptr;
        h->cap_blk = 0;
        cudaError_t e = cudaMalloc(&h->bc, sizeof(int32_t) * (size_t)(nblk * h->ndom));
        if (e == cudaSuccess) e = cudaMalloc(&h->off, sizeof(int64_t) * (size_t)(nblk * h->ndom));
        if (e != cudaSuccess) return halo_cuda(e);
        h->cap_blk = nblk;
    }
    const HaloGeom g = h->geom();
    const double rc2 = r_cut * r_cut;
    cudaMemsetAsync(h->status, 0, sizeof(int32_t), s);
    TP_LAUNCH(k_halo_count, (int)nblk, kHaloBlock, sizeof(int32_t) * h->ndom, s, g, pos, n, mode, self, rc2,
              h->bc, nblk, h->status);
    tp::scan_i32_to_i64(h->bc, h->off, nblk * h->ndom, nullptr, h->d_total, h->scan_tmp, s);
    if (cap > 0)
        TP_LAUNCH(k_halo_write, (int)nblk, kHaloBlock, 0, s, g, pos, n, mode, self, rc2, h->off, nblk, idx, cap);
    // per-destination totals: the offsets at each destination's first block
    std::vector<int64_t> first((size_t)h->ndom);
    int64_t total = 0;
    int32_t status = 0;
    for (int d = 0; d < h->ndom; d++)
        cudaMemcpyAsync(&first[d], h->off + (int64_t)d * nblk, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&total, h->d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&status, h->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    tp_status st = halo_cuda(cudaStreamSynchronize(s));
    if (st != TP_OK) return st;
    if (status != 0) return (tp_status)status;
    for (int d = 0; d < h->ndom; d++) counts[d] = (d + 1 < h->ndom ? first[d + 1] : total) - first[d];
    return total > cap ? TP_ERR_LIST_OVERFLOW : TP_OK;
}

tp_status tp_halo_free(tp_halo *h)
{
    if (!h) return TP_OK;
    cudaDeviceSynchronize();
    cudaFree(h->cuts);
    cudaFree(h->boxes);
    cudaFree(h->status);
    cudaFree(h->d_total);
    cudaFree(h->scan_tmp);
    cudaFree(h->bc);
    cudaFree(h->off);
    delete h;
    cudaGetLastError();
    return TP_OK;
}

tp_status tp_gather_rows(const void *src, int32_t words, const int32_t *idx, int64_t m, void *dst, void *stream)
{
    if (words < 1 || m < 0) return TP_ERR_INVALID_ARG;
    if (m == 0) return TP_OK;
    if (!halo_is_device_ptr(src) || !halo_is_device_ptr(idx) || !halo_is_device_ptr(dst)) return TP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t *a = static_cast<const uint32_t *>(src);
    uint32_t *b = static_cast<uint32_t *>(dst);
    const int grid = (int)std::min<int64_t>((m + 255) / 256, 152 * 32);
    switch (words) {
    case 1: TP_LAUNCH(k_gather_rows_w<1>, grid, 256, 0, s, a, idx, m, b); break;
    case 2: TP_LAUNCH(k_gather_rows_w<2>, grid, 256, 0, s, a, idx, m, b); break;
    case 3: TP_LAUNCH(k_gather_rows_w<3>, grid, 256, 0, s, a, idx, m, b); break;
    case 6: TP_LAUNCH(k_gather_rows_w<6>, grid, 256, 0, s, a, idx, m, b); break;
    default: {
        const int g2 = (int)std::min<int64_t>((m * words + 255) / 256, 152 * 32);
        TP_LAUNCH(k_gather_rows, g2, 256, 0, s, a, words, idx, m, b);
    }
    }
    return halo_cuda(cudaGetLastError());
}

tp_status tp_scatter_add_rows(double *dst, int32_t width, const int32_t *idx, const double *src, int64_t m,
                              void *stream)
{
    if (width < 1 || m < 0) return TP_ERR_INVALID_ARG;
    if (m == 0) return TP_OK;
    if (!halo_is_device_ptr(src) || !halo_is_device_ptr(idx) || !halo_is_device_ptr(dst)) return TP_ERR_INVALID_ARG;
    const int grid = (int)std::min<int64_t>((m * width + 255) / 256, 152 * 32);
    TP_LAUNCH(k_scatter_add_rows, grid, 256, 0, (cudaStream_t)stream, dst, width, idx, src, m);
    return halo_cuda(cudaGetLastError());
}

}  // extern "C"
