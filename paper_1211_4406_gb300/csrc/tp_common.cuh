// tp_common.cuh -- internal data layout and helpers of libtreepm_sr.
//
// Layout in HBM (SoA; "sorted" = Morton key order, boxes back to back):
//   particles  key u64, perm u32, x/y/z/m f64, X/Y/Z u64 fixed-point images
//   nodes      breadth-first; first/count/child/nchild/parent/skip/box i32,
//              level u8, M/S/com/lo/hi/cen/half f64, COM fixed-point u64,
//              and a 48-byte WNode record the walk streams through
//   groups     first/count/box i32, centre/half f64, u32 and u64 images
//   lists      offsets i64 [G+1], entries i32, entry records float4 (group-
//              relative scaled offset and mass, written by the walk)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/treepm_sr.h"

#define TP_MAX_LEVEL 21
#define TP_NLEVELS 22
#define TP_FILTER_SLACK 8.0   // walk-filter error bound, units of 2^-32

// Fixed-point image of a coordinate in [0,1): floor(x * 2^64).  Differences of
// two images, read as int64, are exact minimum-image offsets in units 2^-64.
__device__ __forceinline__ uint64_t tp_fixed64(double x)
{
    return __double2ull_rz(x * 18446744073709551616.0);
}

// Per-box constants, device resident.
struct BoxPrm {
    double G, eps, rcut, theta;
    double rc2, eps2, th2;            // FP64 products, formed as the oracle does
    float eps2s;                      // (k eps)^2, k = 2 / r_cut (scaled units)
    float scale;                      // k * 2^-64: fixed-point offset -> scaled FP32
    double gk2;                       // G k^2: scaled FP32 sum -> acceleration
    double scale_d;                   // 2^-64 for the FP64 path
    uint64_t T_lo, T_hi;              // cutoff thresholds on squared u32-grid gaps
    uint64_t TB_lo[TP_NLEVELS];       // opening thresholds per level
    uint64_t TB_hi[TP_NLEVELS];
    int32_t n_crit, n_leaf;
    int64_t first, count;             // particle range of the box
    double inv_n;                     // default mass
};

// The 48-byte record the walk loads per visited node.
struct __align__(16) WNode {
    uint32_t cx, cy, cz;              // floor(centre * 2^32)
    uint32_t hx, hy, hz;              // floor(half * 2^32)
    int32_t child;                    // first child, -1 for a leaf
    int32_t skip;                     // next node after this subtree, -1 = end
    int32_t first, count;             // particle range
    int32_t level, pad;
};

// The 32-byte record an interaction-list entry is made from: the source's
// fixed-point image and its mass, rounded to FP32 once per source (the entry
// records are FP32), one aligned sector per gather (particles and node
// monopoles alike).
struct __align__(32) SrcRec {
    uint64_t X, Y, Z;
    float m, pad;
};

// The FP32 value of the fixed-point offset a - b (two 64-bit images; their
// wrap-around difference read as signed is the exact minimum-image offset in
// units of 2^-64) times sc, from its two 32-bit halves: on GB300 a conversion
// of a 64-bit integer runs on the FP64 unit (1/64 of the FP32 rate), a 32-bit
// one does not.  Within one rounding step of the correctly rounded value.
// Every FP32 offset of a pair (entry records, group particles) comes from
// here, so equal images give equal offsets and a particle's own entry an
// exact zero difference.
__device__ __forceinline__ float tp_offset_f32(uint64_t a, uint64_t b, float sc)
{
    const long long d = (long long)(a - b);
    const float hi = (float)(int)(d >> 32);
    const float lo = (float)(unsigned)(d & 0xffffffffll);
    return __fmul_rn(__fmaf_rn(hi, 4294967296.0f, lo), sc);
}

struct TreeDev {
    int64_t n;
    int32_t nbox;
    int32_t xi_soft;                  // cutoff argument from the softened distance (all boxes)
    int32_t rsq_refined;              // packed FP32 kernels: the paper's refined 1/s (all boxes)
    int64_t walk_budget;              // node visits per walk; 0: n_nodes + 1 (the proof bound)
    int64_t cap_nodes, cap_groups, cap_entries;
    const BoxPrm *box;
    const int64_t *box_off;           // [nbox+1]
    // particles
    uint64_t *key;
    uint32_t *perm;
    double *x, *y, *z, *m;
    uint64_t *X, *Y, *Z;
    uint4 *P32;                       // {X, Y, Z} >> 32 per particle: the walk's 2^-32 grid
    double *rx, *ry, *rz;             // sorted positions of the last build (refit reference)
    SrcRec *psrc;                     // {X, Y, Z, m} per particle
    // nodes
    int32_t *first, *count, *child, *nchild, *parent, *skip, *nbx;
    uint8_t *level;
    double *M, *Sx, *Sy, *Sz;
    double *comx, *comy, *comz;
    double *lox, *loy, *loz, *hix, *hiy, *hiz;
    double *cenx, *ceny, *cenz, *hfx, *hfy, *hfz;
    uint64_t *cX, *cY, *cZ;           // COM fixed-point images
    SrcRec *nsrc;                     // {cX, cY, cZ, M} per node
    WNode *wn;
    int64_t *lstart, *lcount;         // [TP_NLEVELS + 1] each, device
    int64_t *n_nodes;                 // device scalar
    // groups
    int64_t *n_groups;                // device scalar
    int32_t *gfirst, *gcount, *gbox;
    double *gcx, *gcy, *gcz, *ghx, *ghy, *ghz;
    uint32_t *gux, *guy, *guz, *ghux, *ghuy, *ghuz;
    uint64_t *gX, *gY, *gZ;
    int32_t *gpad;                    // [cap_groups] padded slots the group's walk needs (count pass)
    // walk items: subtree tasks and top-level monopoles, group-major, DFS order
    int64_t cap_items;
    int32_t *icnt;                    // [cap_groups] items per group
    int32_t *iscr;                    // [cap_groups x kscr] each group's first items (count pass)
    int32_t kscr;                     // items kept per group in iscr
    int64_t *ioff;                    // [cap_groups] first item of each group
    int64_t *n_items;                 // device scalar
    int32_t *item, *igrp, *icnt2;     // [cap_items] item, its group, its entry count
    int64_t *ipos;                    // [cap_items] first entry of each item
    int64_t *ibpos;                   // [cap_items] first slot of each item in the padded buffer
    int32_t *ibound;                  // [cap_items] slot count: the task node's particle count
    int64_t cap_pad;
    int32_t *pent;                    // [cap_pad] entries of each item before compaction
    int64_t *n_pad;                   // device scalar
    // lists
    int64_t *loff;                    // [cap_groups + 1]
    int32_t *lcnt;                    // [cap_groups]
    int32_t *ent;
    float4 *rec;                      // [cap_entries] per entry: offset from the group centre
                                      // scaled by 2/r_cut (FP32 x, y, z) and mass (w)
    int64_t *n_entries;               // device scalar
    unsigned long long *n_ambig;      // device scalar
    unsigned long long *n_general;    // device scalar: groups the general FP32 pair kernels take
    // work items of the pair kernels beyond each group's first kWorkChunk
    // particles: {group, chunk} of the further chunks of larger groups
    int64_t cap_xitems;
    int2 *xitem;                      // [cap_xitems]
    int64_t *n_xitems;                // device scalar
    int32_t *status;                  // first latched error
};

// Particles per work item of the pair kernels: a group of more particles is
// taken as several items (its chunks of kWorkChunk), so that no single item
// outlasts the others in the persistent queue.
constexpr int kWorkChunk = 128;

// Items of a group's top walk kept by the count pass, so that the write pass
// copies them instead of walking again (groups with more walk again): up to
// kTopScratch per group, within kTopScratchTotal items for the whole tree.
constexpr int kTopScratch = 1024;
constexpr int64_t kTopScratchTotal = 1ll << 28;

__device__ __forceinline__ void tp_latch(int32_t *status, int32_t code)
{
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ int32_t tp_box_of(const int64_t *box_off, int32_t nbox, int64_t i)
{
    int32_t lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (box_off[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Host-side launch bookkeeping (every kernel launch goes through TP_LAUNCH).
extern "C" void tp_count_launch(void);
#define TP_LAUNCH(kernel, grid, block, smem, stream, ...)                         \
    do {                                                                          \
        tp_count_launch();                                                        \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);               \
    } while (0)

// Launch helpers implemented in the .cu files.
namespace tp {
int num_sms();   // SMs of the current device, queried once per process
void build_moments(TreeDev &T, cudaStream_t s);
void refit_gather(TreeDev &T, const double *pos, const double *mass, cudaStream_t s);
void refit_records(TreeDev &T, cudaStream_t s);
// Resident blocks per SM of `kernel` at `block` threads (at least 1).
template <class K>
int occupancy(K kernel, int block)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, block, 0) != cudaSuccess) {
        cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}
int grid_for(int64_t n, int block);
// Exclusive scans (device-wide).  Exactly one of n_host / d_n gives the
// length: d_n != nullptr reads it from the device (graph friendly).
// total (device, may be null) receives the sum.  tmp must hold scan_tmp_bytes().
size_t scan_tmp_bytes();
void scan_u32(const uint32_t *in, uint32_t *out, int64_t n_host, const int64_t *d_n,
              int64_t *total, void *tmp, cudaStream_t s);
void scan_i64(const int64_t *in, int64_t *out, int64_t n_host, const int64_t *d_n,
              int64_t *total, void *tmp, cudaStream_t s);
void scan_i32_to_i64(const int32_t *in, int64_t *out, int64_t n_host, const int64_t *d_n,
                     int64_t *total, void *tmp, cudaStream_t s);
// Stable LSD radix sort of (key, val) by the low `bits` of key; when nbox > 1
// a final pass orders by the box of each value (val = input index).
size_t radix_tmp_bytes(int64_t n);
void radix_sort(uint64_t *key, uint32_t *val, uint64_t *key2, uint32_t *val2, int64_t n,
                int bits, const int64_t *box_off, int32_t nbox, void *tmp, cudaStream_t s);
}  // namespace tp
