// tp_build.cu -- tree construction on the GPU: Morton keys of the wrapped
// positions, key-order gather, breadth-first octree topology, node monopoles
// and particle groups (the "tree construction" phase of Table I; the tree
// algorithm of Sec. I and Barnes' grouping of Sec. II).
//
// Every FP64 operation that decides a result the CPU oracle must reproduce bit
// for bit is written with explicit round-to-nearest intrinsics, so that no
// multiply-add is contracted into an FMA.
#include "tp_common.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kLevelGrid = 152 * 4;   // fixed grid: node counts live on the device
static_assert(kLevelGrid <= 1024, "the block-sum scratch of the topology passes holds 1024 sums");
constexpr int kMomBatch = 2;          // particles or children loaded together by k_boxes / k_masses

// x in [+0, 1): read as unsigned integers, the bits of such doubles (and of
// no others) lie below those of 1.0.
__device__ __forceinline__ bool unit_interval(double x)
{
    return (uint64_t)__double_as_longlong(x) < 0x3ff0000000000000ull;
}

// x - floor(x), with 1 -> 0 where the difference rounds up to 1.  For x in
// [+0, 1) floor(x) = +0 and the difference is x itself, which the common case
// returns without an FP64 operation (GB300 issues those at a small fraction
// of its integer rate).
__device__ __forceinline__ double wrap01(double x)
{
    if (unit_interval(x)) return x;
    double w = __dsub_rn(x, floor(x));
    return w >= 1.0 ? 0.0 : w;
}

// tp_fixed64 (x 2^64 truncated to 64 bits) from the IEEE-754 fields when x is
// in [+0, 1): a normal x is m 2^(e - 1075) with the 53-bit significand m and
// biased exponent e <= 1022, so x 2^64 = m 2^(e - 1011), a left shift of at
// most 11 bits or a right shift that truncates; subnormals and shifts of 64
// bits or more give 0.  Other x take the FP64 conversion.
__device__ __forceinline__ uint64_t fixed64(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    if (b >= 0x3ff0000000000000ull) return tp_fixed64(x);
    const int e = (int)(b >> 52);
    if (e == 0) return 0ull;
    const uint64_t m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int sh = e - 1011;
    return sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ull);
}

// 21 bits -> every third bit of 63 (bit b lands on 3b).
__device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ uint32_t quantise(double w)
{
    // floor(w 2^21) = floor(floor(w 2^64) / 2^43) for w in [0, 1), below 2^21
    if (unit_interval(w)) return (uint32_t)(fixed64(w) >> 43);
    double q = floor(w * 2097152.0);
    if (q > 2097151.0) q = 2097151.0;
    if (q < 0.0) q = 0.0;
    return (uint32_t)q;
}

// a1: wrap, quantise to 21 bits per axis, interleave (x bit highest).
__global__ void k_keys(const double *pos, int64_t n, uint64_t *key, uint32_t *perm, int32_t *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
            tp_latch(status, TP_ERR_NONFINITE);
            key[i] = 0;
        } else {
            key[i] = (spread3(quantise(wrap01(x))) << 2) | (spread3(quantise(wrap01(y))) << 1) |
                     spread3(quantise(wrap01(z)));
        }
        perm[i] = (uint32_t)i;
    }
}

// a3: sorted FP64 SoA (wrapped), masses, 64-bit fixed-point images.
__global__ void k_gather(const double *pos, const double *mass, TreeDev T)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < T.n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = T.perm[s];
        const double x = wrap01(pos[3 * i]), y = wrap01(pos[3 * i + 1]), z = wrap01(pos[3 * i + 2]);
        T.x[s] = x; T.y[s] = y; T.z[s] = z;
        const uint64_t X = fixed64(x), Y = fixed64(y), Z = fixed64(z);
        T.X[s] = X; T.Y[s] = Y; T.Z[s] = Z;
        T.P32[s] = make_uint4((uint32_t)(X >> 32), (uint32_t)(Y >> 32), (uint32_t)(Z >> 32), 0u);
        const double m = mass ? mass[i] : T.box[tp_box_of(T.box_off, T.nbox, i)].inv_n;
        T.m[s] = m;
        T.psrc[s] = SrcRec{X, Y, Z, (float)m, 0.f};
    }
}

// Refit: each particle keeps its sorted slot and takes the periodic image of
// its new position nearest to the position of the last build (so a node's
// members stay together when one crosses the box boundary); masses are
// replaced only when given.
__global__ void k_refit_gather(const double *pos, const double *mass, TreeDev T)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < T.n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = T.perm[s];
        const double r[3] = {T.rx[s], T.ry[s], T.rz[s]};
        double x[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const double d = __dsub_rn(pos[3 * i + c], r[c]);
            x[c] = __dadd_rn(r[c], __dsub_rn(d, rint(d)));
        }
        T.x[s] = x[0]; T.y[s] = x[1]; T.z[s] = x[2];
        const uint64_t X = fixed64(wrap01(x[0])), Y = fixed64(wrap01(x[1])), Z = fixed64(wrap01(x[2]));
        T.X[s] = X; T.Y[s] = Y; T.Z[s] = Z;
        T.P32[s] = make_uint4((uint32_t)(X >> 32), (uint32_t)(Y >> 32), (uint32_t)(Z >> 32), 0u);
        double m = T.m[s];
        if (mass) {
            m = mass[i];
            T.m[s] = m;
        }
        T.psrc[s] = SrcRec{X, Y, Z, (float)m, 0.f};
    }
}

__global__ void k_init_roots(TreeDev T)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0) {
        T.lstart[0] = 0;
        T.lcount[0] = T.nbox;
        for (int L = 1; L <= TP_NLEVELS; L++) { T.lstart[L] = T.nbox; T.lcount[L] = 0; }
        *T.n_nodes = T.nbox;
    }
    if (b < T.nbox) {
        T.first[b] = (int32_t)T.box_off[b];
        T.count[b] = (int32_t)(T.box_off[b + 1] - T.box_off[b]);
        T.level[b] = 0;
        T.parent[b] = -1;
        T.skip[b] = -1;
        T.child[b] = -1;
        T.nchild[b] = 0;
        T.nbx[b] = b;
    }
}

// Child bounds of node i at level L: b[0] = first, b[8] = first + count and
// b[o] = the first index of the range whose octant digit (at the level's
// shift) is >= o.  The digits are non-decreasing over the node's range (the
// keys are sorted and share the node's prefix), so the seven boundaries are
// independent lower-bound searches; they advance in lockstep, seven key loads
// in flight per step.  Returns the number of non-empty children (0 for a
// leaf).
__device__ __forceinline__ int child_bounds(const TreeDev &T, int32_t i, int L, int32_t *b)
{
    const int32_t f = T.first[i], c = T.count[i];
    if (L >= TP_MAX_LEVEL || c <= T.box[T.nbx[i]].n_leaf) return 0;
    const int shift = 3 * (TP_MAX_LEVEL - 1 - L);
    int32_t lo[8], hi[8];
#pragma unroll
    for (int o = 1; o < 8; o++) { lo[o] = f; hi[o] = f + c; }
    for (int it = 0; it < 32; it++) {                 // ceil(log2(count + 1)) <= 31 steps
        uint64_t kv[8];
#pragma unroll
        for (int o = 1; o < 8; o++) kv[o] = lo[o] < hi[o] ? T.key[(lo[o] + hi[o]) >> 1] : 0;
        bool more = false;
#pragma unroll
        for (int o = 1; o < 8; o++) {
            if (lo[o] < hi[o]) {
                const int32_t mid = (lo[o] + hi[o]) >> 1;
                if (((uint32_t)(kv[o] >> shift) & 7u) < (uint32_t)o) lo[o] = mid + 1; else hi[o] = mid;
                more |= lo[o] < hi[o];
            }
        }
        if (!more) break;
    }
    b[0] = f;
    b[8] = f + c;
#pragma unroll
    for (int o = 1; o < 8; o++) b[o] = lo[o];
    int k = 0;
    for (int o = 0; o < 8; o++) k += b[o + 1] > b[o];
    return k;
}

// The contiguous chunk [c0, c1) of a level's nl nodes taken by this block of
// the level grid.  The count and write passes cut every level the same way,
// so that the write pass forms the prefix of the child counts from the count
// pass's block sums (no separate scan).
__device__ __forceinline__ void level_chunk(int64_t nl, int64_t &c0, int64_t &c1)
{
    const int64_t chunk = (nl + gridDim.x - 1) / gridDim.x;
    c0 = (int64_t)blockIdx.x * chunk;
    c1 = c0 + chunk < nl ? c0 + chunk : nl;
    if (c0 > nl) c0 = nl;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// a4 (count): number of non-empty children of every node of level L (their
// inner bounds b[1..7] are kept for the write pass), and the sum over this
// block's chunk of the level in part[blockIdx.x].
__global__ void __launch_bounds__(kBlock) k_split_count(TreeDev T, int L, uint32_t *nch, int32_t *cb,
                                                        uint32_t *part)
{
    __shared__ uint32_t ws[kBlock / 32];
    const int64_t nl = T.lcount[L], s0 = T.lstart[L];
    int64_t c0, c1;
    level_chunk(nl, c0, c1);
    uint32_t sum = 0;
    for (int64_t t = c0 + threadIdx.x; t < c1; t += blockDim.x) {
        int32_t b[9];
        const int k = child_bounds(T, (int32_t)(s0 + t), L, b);
        nch[t] = (uint32_t)k;
        sum += (uint32_t)k;
        if (k > 0)
            for (int o = 1; o < 8; o++) cb[7 * t + o - 1] = b[o];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < kBlock / 32; w++) tot += ws[w];
        part[blockIdx.x] = tot;
    }
}

// The children of level-L node i (t-th of its level) at c0 onwards, in octant
// order; skip pointers make the breadth-first array walkable depth first
// without a stack (next sibling, else the parent's skip).
__device__ __forceinline__ void write_children(TreeDev &T, int L, int32_t i, int64_t t, int k, int64_t base,
                                               int64_t end, const int32_t *cb)
{
    if (k == 0 || base + k > end) {     // a leaf, or truncated by an overflow
        T.child[i] = -1;
        T.nchild[i] = 0;
        return;
    }
    int32_t b[9];
    b[0] = T.first[i];
    b[8] = b[0] + T.count[i];
    for (int o = 1; o < 8; o++) b[o] = cb[7 * t + o - 1];
    int j = 0;
    for (int o = 0; o < 8; o++) {
        if (b[o + 1] <= b[o]) continue;
        const int32_t c = (int32_t)(base + j);
        T.first[c] = b[o];
        T.count[c] = b[o + 1] - b[o];
        T.level[c] = (uint8_t)(L + 1);
        T.parent[c] = i;
        T.nbx[c] = T.nbx[i];
        T.child[c] = -1;
        T.nchild[c] = 0;
        T.skip[c] = (j == k - 1) ? T.skip[i] : c + 1;
        j++;
    }
    T.child[i] = (int32_t)base;
    T.nchild[i] = k;
}

// a4 (write): children of level-L nodes at lstart[L+1] + their exclusive
// prefix of child counts: the block sums of the chunks before this block's
// (part, from the count pass) plus a scan within the chunk.  Level L+1 starts
// right after level L; a level that would pass cap_nodes is dropped whole
// (status TP_ERR_LIST_OVERFLOW).  Every block derives the level's total
// itself; block 0 stores the next level's start and count and the node count.
__global__ void __launch_bounds__(kBlock) k_split_write(TreeDev T, int L, const uint32_t *nch,
                                                        const uint32_t *part, const int32_t *cb)
{
    constexpr int nw = kBlock / 32;
    __shared__ uint32_t warp_tot[nw], s_red[2][nw];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nl = T.lcount[L], s0 = T.lstart[L];
    uint32_t before_blk = 0, total = 0;
    for (int j = threadIdx.x; j < (int)gridDim.x; j += blockDim.x) {
        const uint32_t v = part[j];
        total += v;
        if (j < (int)blockIdx.x) before_blk += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        total += __shfl_xor_sync(0xffffffffu, total, o);
        before_blk += __shfl_xor_sync(0xffffffffu, before_blk, o);
    }
    if (lane == 0) { s_red[0][warp] = total; s_red[1][warp] = before_blk; }
    __syncthreads();
    total = before_blk = 0;
    for (int w = 0; w < nw; w++) { total += s_red[0][w]; before_blk += s_red[1][w]; }
    const int64_t base0 = s0 + nl;
    const bool overflow = base0 + (int64_t)total > T.cap_nodes;
    const int64_t nnext = overflow ? 0 : (int64_t)total;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        T.lstart[L + 1] = base0;
        T.lcount[L + 1] = nnext;
        if (overflow) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
        *T.n_nodes = base0 + nnext;
    }
    int64_t c0, c1;
    level_chunk(nl, c0, c1);
    uint32_t carry = before_blk;
    for (int64_t tb = c0; tb < c1; tb += blockDim.x) {
        const int64_t t = tb + threadIdx.x;
        const uint32_t v = t < c1 ? nch[t] : 0u;
        const uint32_t inc = warp_incl_scan_u32(v);
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < nw ? warp_tot[lane] : 0u;
            const uint32_t wi = warp_incl_scan_u32(w);
            if (lane < nw) warp_tot[lane] = wi;
        }
        __syncthreads();
        const uint32_t pre = carry + (warp == 0 ? 0u : warp_tot[warp - 1]) + inc - v;
        if (t < c1)
            write_children(T, L, (int32_t)(s0 + t), t, nnext == 0 ? 0 : (int)v, base0 + pre, base0 + nnext, cb);
        carry += warp_tot[nw - 1];
        __syncthreads();
    }
}

// Order-preserving keys of finite doubles (negative values: all bits flipped;
// others: the sign bit set), so that the tight boxes' min/max run as exact
// integer comparisons instead of on the FP64 pipe.  They order -0.0 below
// +0.0, but wrapped coordinates are never -0.0 (x - floor(x) rounds an exact
// zero to +0.0), so the result is the comparison min/max bit for bit.
__device__ __forceinline__ uint64_t ord_key(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_value(uint64_t k)
{
    const uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// a5, in two passes per level, bottom up.  k_boxes: tight boxes (leaf: the
// particles; internal: the children), their centres and half-widths and the
// walk record, which is all the walk reads.  k_masses: monopoles in canonical
// order (leaf: particles in key order; internal: children in octant order),
// centres of mass and their fixed-point images (the source records of
// monopole entries), needed from the compaction on; the build runs them
// beside the walk.  Loads take two particles (children) at a time, so that
// their latencies overlap; an index past the end repeats the last one, which
// leaves a min/max unchanged, and the sums take only the real ones, in order.
// The box of node i from the min/max keys of its particles or children: its
// bounds, centre, half-widths and walk record.
__device__ __forceinline__ void write_box(TreeDev &T, int32_t i, uint64_t klx, uint64_t kly, uint64_t klz,
                                          uint64_t khx, uint64_t khy, uint64_t khz)
{
    double lx = ord_value(klx), ly = ord_value(kly), lz = ord_value(klz);
    double hx = ord_value(khx), hy = ord_value(khy), hz = ord_value(khz);
    const int32_t cnt = T.count[i];
    if (cnt == 0) { lx = ly = lz = hx = hy = hz = 0.0; }
    T.lox[i] = lx; T.loy[i] = ly; T.loz[i] = lz;
    T.hix[i] = hx; T.hiy[i] = hy; T.hiz[i] = hz;
    const double cx = __dmul_rn(__dadd_rn(lx, hx), 0.5), cy = __dmul_rn(__dadd_rn(ly, hy), 0.5),
                 cz = __dmul_rn(__dadd_rn(lz, hz), 0.5);
    const double fx = __dmul_rn(__dsub_rn(hx, lx), 0.5), fy = __dmul_rn(__dsub_rn(hy, ly), 0.5),
                 fz = __dmul_rn(__dsub_rn(hz, lz), 0.5);
    T.cenx[i] = cx; T.ceny[i] = cy; T.cenz[i] = cz;
    T.hfx[i] = fx; T.hfy[i] = fy; T.hfz[i] = fz;
    WNode w;
    w.cx = (uint32_t)(fixed64(wrap01(cx)) >> 32);
    w.cy = (uint32_t)(fixed64(wrap01(cy)) >> 32);
    w.cz = (uint32_t)(fixed64(wrap01(cz)) >> 32);
    w.hx = (uint32_t)(fixed64(fx) >> 32);
    w.hy = (uint32_t)(fixed64(fy) >> 32);
    w.hz = (uint32_t)(fixed64(fz) >> 32);
    const int32_t nc = T.nchild[i];
    w.child = nc ? T.child[i] : -1;
    w.skip = T.skip[i];
    w.first = T.first[i];
    w.count = cnt;
    w.level = T.level[i];
    w.pad = 0;
    T.wn[i] = w;
}

__global__ void __launch_bounds__(kBlock) k_boxes(TreeDev T, int L)
{
    const int64_t nl = T.lcount[L], s0 = T.lstart[L];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nl;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(s0 + t);
        uint64_t klx = ~0ull, kly = ~0ull, klz = ~0ull, khx = 0ull, khy = 0ull, khz = 0ull;
        auto minmax = [&](uint64_t ax, uint64_t ay, uint64_t az, uint64_t bx, uint64_t by, uint64_t bz) {
            klx = ax < klx ? ax : klx; kly = ay < kly ? ay : kly; klz = az < klz ? az : klz;
            khx = bx > khx ? bx : khx; khy = by > khy ? by : khy; khz = bz > khz ? bz : khz;
        };
        const int32_t nc = T.nchild[i];
        if (nc == 0) {
            const int32_t f = T.first[i], e = f + T.count[i];
            for (int32_t p0 = f; p0 < e; p0 += kMomBatch) {
                double xp[kMomBatch], yp[kMomBatch], zp[kMomBatch];
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    const int32_t p = p0 + k < e ? p0 + k : e - 1;
                    xp[k] = T.x[p]; yp[k] = T.y[p]; zp[k] = T.z[p];
                }
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    const uint64_t kx = ord_key(xp[k]), ky = ord_key(yp[k]), kz = ord_key(zp[k]);
                    minmax(kx, ky, kz, kx, ky, kz);
                }
            }
        } else {
            const int32_t c0 = T.child[i];
            for (int32_t c = c0; c < c0 + nc; c++)
                minmax(ord_key(T.lox[c]), ord_key(T.loy[c]), ord_key(T.loz[c]), ord_key(T.hix[c]),
                       ord_key(T.hiy[c]), ord_key(T.hiz[c]));
        }
        write_box(T, i, klx, kly, klz, khx, khy, khz);
    }
}

__global__ void __launch_bounds__(kBlock) k_masses(TreeDev T, int L)
{
    const int64_t nl = T.lcount[L], s0 = T.lstart[L];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nl;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)(s0 + t);
        double M = 0.0, Sx = 0.0, Sy = 0.0, Sz = 0.0;
        const int32_t nc = T.nchild[i];
        if (nc == 0) {
            const int32_t f = T.first[i], e = f + T.count[i];
            for (int32_t p0 = f; p0 < e; p0 += kMomBatch) {
                double mp[kMomBatch], xp[kMomBatch], yp[kMomBatch], zp[kMomBatch];
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    const int32_t p = p0 + k < e ? p0 + k : e - 1;
                    mp[k] = T.m[p]; xp[k] = T.x[p]; yp[k] = T.y[p]; zp[k] = T.z[p];
                }
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    if (p0 + k < e) {
                        M = __dadd_rn(M, mp[k]);
                        Sx = __dadd_rn(Sx, __dmul_rn(mp[k], xp[k]));
                        Sy = __dadd_rn(Sy, __dmul_rn(mp[k], yp[k]));
                        Sz = __dadd_rn(Sz, __dmul_rn(mp[k], zp[k]));
                    }
                }
            }
        } else {
            const int32_t c0 = T.child[i], c1 = c0 + nc;
            for (int32_t b0 = c0; b0 < c1; b0 += kMomBatch) {
                double cm[kMomBatch], cx[kMomBatch], cy[kMomBatch], cz[kMomBatch];
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    const int32_t c = b0 + k < c1 ? b0 + k : c1 - 1;
                    cm[k] = T.M[c]; cx[k] = T.Sx[c]; cy[k] = T.Sy[c]; cz[k] = T.Sz[c];
                }
#pragma unroll
                for (int k = 0; k < kMomBatch; k++) {
                    if (b0 + k < c1) {
                        M = __dadd_rn(M, cm[k]);
                        Sx = __dadd_rn(Sx, cx[k]);
                        Sy = __dadd_rn(Sy, cy[k]);
                        Sz = __dadd_rn(Sz, cz[k]);
                    }
                }
            }
        }
        T.M[i] = M; T.Sx[i] = Sx; T.Sy[i] = Sy; T.Sz[i] = Sz;
        // an empty node's centre of mass is its box centre (k_boxes ran first)
        const double mx = M > 0.0 ? __ddiv_rn(Sx, M) : T.cenx[i];
        const double my = M > 0.0 ? __ddiv_rn(Sy, M) : T.ceny[i];
        const double mz = M > 0.0 ? __ddiv_rn(Sz, M) : T.cenz[i];
        T.comx[i] = mx; T.comy[i] = my; T.comz[i] = mz;
        // images of the centres (in [0,1) after a build; after a refit they
        // may lie just outside, hence the wrap)
        const uint64_t CX = fixed64(wrap01(mx)), CY = fixed64(wrap01(my)), CZ = fixed64(wrap01(mz));
        T.cX[i] = CX; T.cY[i] = CY; T.cZ[i] = CZ;
        T.nsrc[i] = SrcRec{CX, CY, CZ, (float)M, 0.f};
    }
}

// a6: group starts.  Under every node holding more than n_crit particles each
// maximal run of consecutive small children is cut into k = ceil(S/n_crit)
// balanced groups; a big leaf is a group by itself; a small root is one group.
__global__ void k_group_flags(TreeDev T, uint32_t *flag)
{
    const int64_t nn = *T.n_nodes;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nn;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = (int32_t)t;
        const int32_t c = T.count[i];
        const int32_t nc = T.box[T.nbx[i]].n_crit;
        const bool leaf = T.nchild[i] == 0;
        if (T.level[i] == 0 && c > 0 && (c <= nc || leaf)) flag[T.first[i]] = 1u;
        if (c <= nc || leaf) continue;
        const int32_t c0 = T.child[i], c1 = c0 + T.nchild[i];
        int32_t run0 = c0;          // first child of the current run
        for (int32_t k = c0; k <= c1; k++) {
            const bool big = k < c1 && T.count[k] > nc;
            if (k == c1 || big) {
                // flush the run [run0, k)
                int64_t S = 0;
                for (int32_t r = run0; r < k; r++) S += T.count[r];
                if (S > 0) {
                    const int64_t kg = (S + nc - 1) / nc;
                    const int64_t target = (S + kg - 1) / kg;
                    int64_t cur = 0;
                    for (int32_t r = run0; r < k; r++) {
                        const int64_t cr = T.count[r];
                        if (cur > 0 && (cur + cr > nc || cur >= target)) cur = 0;
                        if (cur == 0) flag[T.first[r]] = 1u;
                        cur += cr;
                    }
                }
                if (big && T.nchild[k] == 0) flag[T.first[k]] = 1u;
                run0 = k + 1;
            }
        }
    }
}

__global__ void k_group_fill(TreeDev T, const uint32_t *flag, const uint32_t *gofs)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < T.n;
         p += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[p]) continue;
        const uint32_t g = gofs[p];
        if ((int64_t)g >= T.cap_groups) { tp_latch(T.status, TP_ERR_LIST_OVERFLOW); continue; }
        T.gfirst[g] = (int32_t)p;
        T.gbox[g] = tp_box_of(T.box_off, T.nbox, p);
    }
}

// Group counts and tight boxes: one warp per group; min/max on the IEEE bit
// patterns (positions are >= +0, where the bit order is the numeric order).
__global__ void k_group_bbox(TreeDev T)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < G; g += nw) {
        const int32_t f = T.gfirst[g];
        const int32_t e = (g + 1 < G) ? T.gfirst[g + 1] : (int32_t)T.n;
        unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
        for (int32_t p = f + lane; p < e; p += 32) {
            const unsigned long long a = __double_as_longlong(T.x[p]), b = __double_as_longlong(T.y[p]),
                                     c = __double_as_longlong(T.z[p]);
            lo[0] = min(lo[0], a); lo[1] = min(lo[1], b); lo[2] = min(lo[2], c);
            hi[0] = max(hi[0], a); hi[1] = max(hi[1], b); hi[2] = max(hi[2], c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0) T.gcount[g] = e - f;
        if (lane < 3) {                    // one axis per lane: three FP64 chains side by side
            const unsigned long long lk = lane == 0 ? lo[0] : (lane == 1 ? lo[1] : lo[2]);
            const unsigned long long hk = lane == 0 ? hi[0] : (lane == 1 ? hi[1] : hi[2]);
            const double l = __longlong_as_double(lk), u = __longlong_as_double(hk);
            const double c = __dmul_rn(__dadd_rn(l, u), 0.5), h = __dmul_rn(__dsub_rn(u, l), 0.5);
            const uint64_t X = fixed64(c);
            (lane == 0 ? T.gcx : (lane == 1 ? T.gcy : T.gcz))[g] = c;
            (lane == 0 ? T.ghx : (lane == 1 ? T.ghy : T.ghz))[g] = h;
            (lane == 0 ? T.gX : (lane == 1 ? T.gY : T.gZ))[g] = X;
            (lane == 0 ? T.gux : (lane == 1 ? T.guy : T.guz))[g] = (uint32_t)(X >> 32);
            (lane == 0 ? T.ghux : (lane == 1 ? T.ghuy : T.ghuz))[g] = (uint32_t)(fixed64(h) >> 32);
        }
    }
}

}  // namespace

namespace tp {

void build_keys_sort_gather(TreeDev &T, const double *pos, const double *mass, uint64_t *key2,
                            uint32_t *perm2, void *radix_tmp, cudaStream_t s)
{
    if (T.n == 0) return;
    TP_LAUNCH(k_keys, grid_for(T.n, kBlock), kBlock, 0, s, pos, T.n, T.key, T.perm, T.status);
    radix_sort(T.key, T.perm, key2, perm2, T.n, 63, T.box_off, T.nbox, radix_tmp, s);
    TP_LAUNCH(k_gather, grid_for(T.n, kBlock), kBlock, 0, s, pos, mass, T);
}

// Topology (boxes and monopoles follow in build_boxes, build_masses).  nch:
// scratch of cap_nodes u32; ofs: at least kLevelGrid u32 (the count pass's
// block sums).
void build_topology(TreeDev &T, uint32_t *nch, uint32_t *ofs, int32_t *cb, void *scan_tmp, cudaStream_t s)
{
    TP_LAUNCH(k_init_roots, (T.nbox + 127) / 128, 128, 0, s, T);
    for (int L = 0; L < TP_MAX_LEVEL; L++) {       // ofs holds the count pass's block sums
        TP_LAUNCH(k_split_count, kLevelGrid, kBlock, 0, s, T, L, nch, cb, ofs);
        TP_LAUNCH(k_split_write, kLevelGrid, kBlock, 0, s, T, L, nch, (const uint32_t *)ofs, cb);
    }
}

// Boxes and walk records of every node, bottom-up by level.
void build_boxes(TreeDev &T, cudaStream_t s)
{
    for (int L = TP_MAX_LEVEL; L >= 0; L--) TP_LAUNCH(k_boxes, kLevelGrid, kBlock, 0, s, T, L);
}

// Monopoles of every node, bottom-up by level (after build_boxes).
void build_masses(TreeDev &T, cudaStream_t s)
{
    for (int L = TP_MAX_LEVEL; L >= 0; L--) TP_LAUNCH(k_masses, kLevelGrid, kBlock, 0, s, T, L);
}

void build_moments(TreeDev &T, cudaStream_t s)
{
    build_boxes(T, s);
    build_masses(T, s);
}

// New positions for a refit (same particles, same sorted order).
void refit_gather(TreeDev &T, const double *pos, const double *mass, cudaStream_t s)
{
    if (T.n == 0) return;
    TP_LAUNCH(k_refit_gather, grid_for(T.n, kBlock), kBlock, 0, s, pos, mass, T);
}

// Group starts and their count (into *T.n_groups).  flag/gofs: [n] u32.
void build_group_starts(TreeDev &T, uint32_t *flag, uint32_t *gofs, void *scan_tmp, cudaStream_t s)
{
    if (T.n == 0) {
        cudaMemsetAsync(T.n_groups, 0, sizeof(int64_t), s);
        return;
    }
    cudaMemsetAsync(flag, 0, sizeof(uint32_t) * (size_t)T.n, s);
    TP_LAUNCH(k_group_flags, kLevelGrid, kBlock, 0, s, T, flag);
    scan_u32(flag, gofs, T.n, nullptr, T.n_groups, scan_tmp, s);
}

void build_groups(TreeDev &T, const uint32_t *flag, const uint32_t *gofs, cudaStream_t s)
{
    if (T.n == 0) return;
    TP_LAUNCH(k_group_fill, grid_for(T.n, kBlock), kBlock, 0, s, T, flag, gofs);
    TP_LAUNCH(k_group_bbox, kLevelGrid, kBlock, 0, s, T);
}

}  // namespace tp
