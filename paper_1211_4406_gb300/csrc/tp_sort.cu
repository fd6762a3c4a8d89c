// tp_sort.cu -- device-wide exclusive scans and the stable LSD radix sort of
// (Morton key, input index) pairs (the sort step of the tree build).
#include <cstdio>

#include "tp_common.cuh"

namespace {

constexpr int kScanBlocks = 512;
constexpr int kScanThreads = 256;
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 4096
constexpr int kRadixWarps = kRadixThreads / 32;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <class Tin, class Tout>
__global__ void k_scan_reduce(const Tin *in, int64_t n_host, const int64_t *d_n, Tout *partial)
{
    const int64_t n = d_n ? *d_n : n_host;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    Tout s = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += (Tout)in[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ Tout ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        Tout t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

// Each block first sums the partials of the blocks before it (its carry; the
// last block also writes the grand total), then scans its own chunk.  Integer
// sums, so the order of the additions does not change the result.
template <class Tin, class Tout>
__global__ void k_scan_apply(const Tin *in, Tout *out, int64_t n_host, const int64_t *d_n,
                             const Tout *partial, int64_t *total)
{
    __shared__ Tout warp_tot[32];
    const int64_t n = d_n ? *d_n : n_host;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk;
    const int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    Tout c = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += blockDim.x) c += partial[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) warp_tot[warp] = c;
    __syncthreads();
    Tout carry = 0;
    for (int w = 0; w < nw; w++) carry += warp_tot[w];
    __syncthreads();
    if (total && threadIdx.x == 0 && blockIdx.x == gridDim.x - 1)
        *total = (int64_t)(carry + partial[blockIdx.x]);
    for (int64_t base = b0; base < b1; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        Tout v = i < b1 ? (Tout)in[i] : Tout(0);
        Tout inc = warp_incl_scan(v);
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            Tout w = lane < nw ? warp_tot[lane] : Tout(0);
            Tout wi = warp_incl_scan(w);
            if (lane < nw) warp_tot[lane] = wi;  // inclusive over warps
        }
        __syncthreads();
        Tout before = warp == 0 ? Tout(0) : warp_tot[warp - 1];
        if (i < b1) out[i] = carry + before + inc - v;
        carry += warp_tot[nw - 1];
        __syncthreads();
    }
}

template <class Tin, class Tout>
void scan_impl(const Tin *in, Tout *out, int64_t n_host, const int64_t *d_n, int64_t *total,
               void *tmp, cudaStream_t s)
{
    Tout *partial = reinterpret_cast<Tout *>(tmp);
    auto reduce = k_scan_reduce<Tin, Tout>;
    auto apply = k_scan_apply<Tin, Tout>;
    TP_LAUNCH(reduce, kScanBlocks, kScanThreads, 0, s, in, n_host, d_n, partial);
    TP_LAUNCH(apply, kScanBlocks, kScanThreads, 0, s, in, out, n_host, d_n, (const Tout *)partial, total);
}

// ------------------------------------------------------------------------
// Radix sort: 8-bit digits, tiles of 4096 items, per-warp stable ranking with
// __match_any_sync, prefix over (digit, tile) by the device-wide scan, and
// stores staged through shared memory in output order.
// ------------------------------------------------------------------------
__device__ __forceinline__ uint32_t radix_digit(uint64_t key, uint32_t val, int shift, int mode,
                                                const int64_t *box_off, int32_t nbox)
{
    if (mode == 0) return (uint32_t)(key >> shift) & 255u;
    return ((uint32_t)tp_box_of(box_off, nbox, (int64_t)val) >> shift) & 255u;
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_hist(const uint64_t *key, const uint32_t *val, int64_t n, int shift, int mode,
             const int64_t *box_off, int32_t nbox, uint32_t *counts, int64_t nblocks)
{
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    uint32_t d[kRadixItems];               // all loads first, so that they are in flight together
#pragma unroll
    for (int r = 0; r < kRadixItems; r++) {
        const int64_t i = base + (int64_t)r * kRadixThreads + threadIdx.x;
        d[r] = i < n ? radix_digit(key[i], mode ? val[i] : 0u, shift, mode, box_off, nbox) : 256u;
    }
#pragma unroll
    for (int r = 0; r < kRadixItems; r++)
        if (d[r] < 256u) atomicAdd(&hist[d[r]], 1u);
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = hist[threadIdx.x];
}

// The scatter ranks the tile's items stably by digit (per warp with
// __match_any_sync, then across warps), stages them in shared memory in that
// order, and writes each digit's run of the tile with consecutive threads on
// consecutive addresses, so that the stores coalesce instead of landing in up
// to 32 digit buckets per warp instruction.
__global__ void __launch_bounds__(kRadixThreads)
k_radix_scatter(const uint64_t *key, const uint32_t *val, uint64_t *key2, uint32_t *val2,
                int64_t n, int shift, int mode, const int64_t *box_off, int32_t nbox,
                const uint32_t *offsets, int64_t nblocks)
{
    union Stage {
        uint32_t whist[kRadixWarps][256];   // per-warp digit counts, then their prefix over warps
        uint64_t key[kRadixTile];           // the tile's keys in output order, then
        uint32_t val[kRadixTile];           // its values
    };
    __shared__ Stage S;
    __shared__ uint8_t sdig[kRadixTile];
    __shared__ uint32_t gofs[256], tstart[256], wsum[kRadixWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = threadIdx.x; d < kRadixWarps * 256; d += kRadixThreads) S.whist[d >> 8][d & 255] = 0;
    gofs[threadIdx.x] = offsets[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kRadixTile;
    const int ntile = n - tile0 < kRadixTile ? (int)(n - tile0) : kRadixTile;
    const int64_t base = tile0 + (int64_t)warp * (32 * kRadixItems);
    const unsigned lt = (1u << lane) - 1u;
    uint64_t k[kRadixItems];
    uint32_t v[kRadixItems], dg[kRadixItems], rk[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; r++) {     // all loads first, so that they are in flight together
        const int64_t i = base + r * 32 + lane;
        const bool ok = i < n;
        k[r] = ok ? key[i] : 0ull;
        v[r] = ok ? val[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRadixItems; r++) {
        const bool ok = base + r * 32 + lane < n;
        const uint32_t d = ok ? radix_digit(k[r], v[r], shift, mode, box_off, nbox) : 256u;
        dg[r] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = d < 256u ? S.whist[warp][d] : 0u;
        __syncwarp();
        if (d < 256u && (peers & lt) == 0u) S.whist[warp][d] = before + __popc(peers);
        __syncwarp();
        rk[r] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        // digit d: prefix over the warps, then the tile's exclusive scan over digits
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < kRadixWarps; w++) {
            const uint32_t c = S.whist[w][d];
            S.whist[w][d] = run;
            run += c;
        }
        uint32_t inc = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; w++) before += wsum[w];
        tstart[d] = before + inc - run;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; r++)          // position in the tile's output order
        if (dg[r] < 256u) rk[r] += tstart[dg[r]] + S.whist[warp][dg[r]];
    __syncthreads();                               // the counts are read: the stage takes the keys
#pragma unroll
    for (int r = 0; r < kRadixItems; r++)
        if (dg[r] < 256u) {
            S.key[rk[r]] = k[r];
            sdig[rk[r]] = (uint8_t)dg[r];
        }
    __syncthreads();
    for (int i = threadIdx.x; i < ntile; i += kRadixThreads) {
        const uint32_t d = sdig[i];
        key2[gofs[d] + (uint32_t)i - tstart[d]] = S.key[i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; r++)
        if (dg[r] < 256u) S.val[rk[r]] = v[r];
    __syncthreads();
    for (int i = threadIdx.x; i < ntile; i += kRadixThreads) {
        const uint32_t d = sdig[i];
        val2[gofs[d] + (uint32_t)i - tstart[d]] = S.val[i];
    }
}

}  // namespace

namespace tp {

int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

size_t scan_tmp_bytes() { return sizeof(int64_t) * kScanBlocks; }

void scan_u32(const uint32_t *in, uint32_t *out, int64_t n_host, const int64_t *d_n,
              int64_t *total, void *tmp, cudaStream_t s)
{
    scan_impl<uint32_t, uint32_t>(in, out, n_host, d_n, total, tmp, s);
}

void scan_i64(const int64_t *in, int64_t *out, int64_t n_host, const int64_t *d_n,
              int64_t *total, void *tmp, cudaStream_t s)
{
    scan_impl<int64_t, int64_t>(in, out, n_host, d_n, total, tmp, s);
}

void scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n_host, const int64_t *d_n,
                     int64_t *total, void *tmp, cudaStream_t s)
{
    scan_impl<int32_t, int64_t>(in, out, n_host, d_n, total, tmp, s);
}

size_t radix_tmp_bytes(int64_t n)
{
    const int64_t nblocks = (n + kRadixTile - 1) / kRadixTile;
    return sizeof(uint32_t) * (size_t)(256 * (nblocks > 0 ? nblocks : 1)) + 256 + scan_tmp_bytes();
}

void radix_sort(uint64_t *key, uint32_t *val, uint64_t *key2, uint32_t *val2, int64_t n,
                int bits, const int64_t *box_off, int32_t nbox, void *tmp, cudaStream_t s)
{
    if (n <= 0) return;
    const int64_t nblocks = (n + kRadixTile - 1) / kRadixTile;
    uint32_t *counts = reinterpret_cast<uint32_t *>(tmp);
    void *scan_tmp = reinterpret_cast<char *>(tmp) +
                     ((sizeof(uint32_t) * (size_t)(256 * nblocks) + 255) & ~size_t(255));
    uint64_t *ka = key, *kb = key2;
    uint32_t *va = val, *vb = val2;
    int passes = 0;
    auto pass = [&](int shift, int mode) {
        TP_LAUNCH(k_radix_hist, (int)nblocks, kRadixThreads, 0, s, ka, va, n, shift, mode, box_off,
                  nbox, counts, nblocks);
        scan_u32(counts, counts, 256 * nblocks, nullptr, nullptr, scan_tmp, s);
        TP_LAUNCH(k_radix_scatter, (int)nblocks, kRadixThreads, 0, s, ka, va, kb, vb, n, shift, mode,
                  box_off, nbox, counts, nblocks);
        uint64_t *kt = ka; ka = kb; kb = kt;
        uint32_t *vt = va; va = vb; vb = vt;
        passes++;
    };
    for (int shift = 0; shift < bits; shift += 8) pass(shift, 0);
    if (nbox > 1)
        for (int shift = 0; shift < 32 && ((uint32_t)(nbox - 1) >> shift) != 0u; shift += 8) pass(shift, 1);
    if (passes & 1) {
        cudaMemcpyAsync(key, ka, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(val, va, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s);
    }
}

}  // namespace tp
