// tp_walk.cu -- per-group interaction lists (Barnes' modified algorithm,
// Sec. II; the "tree traversal" row of Table I).
//
// The walk visits a group's tree depth first (top stage: one thread per group,
// stackless by the skip pointers of the breadth-first node array; task stage:
// one warp per subtree, one lane per particle).  At every node it decides
//   prune   periodic box-to-box gap d >= r_cut,
//   accept  no overlap with the group, largest box-to-box distance < r_cut and
//           l^2 < theta^2 d^2 (l = 2^-level): the node enters as a monopole,
//   open    otherwise (at a leaf: keep particles with point-to-box gap < r_cut).
// The decisions must equal the FP64 ones of the reference definition bit for
// bit.  GB300 runs FP64 at a small fraction of its FP32/integer rate, so each
// one is first taken on a 2^-32 integer grid: positions, centres and half-widths
// are truncated to 32-bit fixed point, wrap-around subtraction gives the
// periodic minimum image for free, and the squared gaps are exact 64-bit
// integers.  Truncation moves every gap by less than TP_FILTER_SLACK grid
// units, so comparing with thresholds widened by that slack either settles the
// decision for certain or, in a band of a few 1e-9 of the box, falls back to the
// same FP64 expression evaluated with round-to-nearest intrinsics.
#include "tp_common.cuh"

namespace {

constexpr int kBlock = 128;
constexpr int32_t kBigTask = 256;   // particles of a walk task taken in the first sweep

__device__ __forceinline__ uint32_t absdiff32(uint32_t a, uint32_t b)
{
    const int32_t t = (int32_t)(a - b);
    return t < 0 ? (uint32_t)(-(int64_t)t) : (uint32_t)t;
}

__device__ __forceinline__ double dminimg(double t) { return __dsub_rn(t, rint(t)); }

// v^2 for a grid gap v < 2^32, as one 32 x 32 -> 64-bit multiply (a 64-bit
// product would take several).  Every gap the walk squares is at most 2^31
// (wrap-around differences of 32-bit coordinates, less the half-widths), so
// a sum of three squares stays below 2^64.
__device__ __forceinline__ uint64_t sq32(uint64_t v)
{
    const uint32_t u = (uint32_t)v;
    return (uint64_t)u * u;
}

// Reference FP64 box distances: per axis t = |minimg(a - c)|, s = h + hg,
// gap = max(0, t - s), far = t + s; sums (x^2 + y^2) + z^2.
__device__ __forceinline__ double exact_dist2(double ax, double ay, double az, double hx, double hy,
                                              double hz, double cx, double cy, double cz, double gx,
                                              double gy, double gz, double *far2)
{
    const double a[3] = {ax, ay, az}, h[3] = {hx, hy, hz}, c[3] = {cx, cy, cz}, g[3] = {gx, gy, gz};
    double gp[3], fr[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double tt = fabs(dminimg(__dsub_rn(a[k], c[k])));
        const double s = __dadd_rn(h[k], g[k]);
        const double e = __dsub_rn(tt, s);
        gp[k] = e > 0.0 ? e : 0.0;
        fr[k] = __dadd_rn(tt, s);
    }
    *far2 = __dadd_rn(__dadd_rn(__dmul_rn(fr[0], fr[0]), __dmul_rn(fr[1], fr[1])), __dmul_rn(fr[2], fr[2]));
    return __dadd_rn(__dadd_rn(__dmul_rn(gp[0], gp[0]), __dmul_rn(gp[1], gp[1])), __dmul_rn(gp[2], gp[2]));
}

// The walk runs in two stages.  Top: one thread per group walks from the box
// root; an opened node holding at most `split` particles (or a leaf) is not
// descended but emitted as a task item (its node id), an accepted monopole as a
// final item -(id+1).  Task: each task expands to the list entries of its
// subtree.  The items of all groups, concatenated in group order and in
// depth-first order within a group, expand to exactly the depth-first lists of
// the reference definition.

struct WalkGroup {
    uint32_t gx, gy, gz, hx, hy, hz;
    int32_t g0, g1;
    int64_t g;
    const BoxPrm *P;
};

// An entry's record for the pair kernels: its offset from the group centre
// (wrap-around difference of the 64-bit images, the exact minimum image)
// scaled by k = 2/r_cut and converted to FP32 by tp_offset_f32, and its mass.
__device__ __forceinline__ float4 entry_record(const TreeDev &T, uint64_t GX, uint64_t GY, uint64_t GZ, float sc,
                                              int32_t e)
{
    const SrcRec q = e >= 0 ? T.psrc[e] : T.nsrc[-e - 1];
    return make_float4(tp_offset_f32(q.X, GX, sc), tp_offset_f32(q.Y, GY, sc), tp_offset_f32(q.Z, GZ, sc), q.m);
}

__device__ __forceinline__ WalkGroup load_walk_group(const TreeDev &T, int64_t g)
{
    WalkGroup W;
    W.g = g;
    W.gx = T.gux[g]; W.gy = T.guy[g]; W.gz = T.guz[g];
    W.hx = T.ghux[g]; W.hy = T.ghuy[g]; W.hz = T.ghuz[g];
    W.g0 = T.gfirst[g];
    W.g1 = W.g0 + T.gcount[g];
    W.P = &T.box[T.gbox[g]];
    return W;
}

enum { kPrune = 0, kAccept = 1, kOpen = 2 };

// The decision at node nd (w = its walk record) for group W; namb counts the
// decisions that needed the exact FP64 test.  allin reports, for an opened
// node, that its box lies wholly within r_cut of the group box for certain:
// the largest box-to-box distance on the integer grid is below the lower
// threshold.  Every particle of the node lies in its tight box [lo, hi], and
// the per-axis centre and half-width taken from it in FP64 cover that box to
// within an ulp, so each particle's point-to-box gap is at most that distance
// plus ~1e-15; the grid distance is within 3 sqrt(3) units of 2^-32 of the
// distance from the FP64 centres and half-widths (three truncations per
// axis), and the lower threshold lies TP_FILTER_SLACK = 8 units inside r_cut.
// The reference test of every such particle (FP64 gap < r_cut) therefore
// keeps it, and the walk may take the particles of an opened leaf with allin
// set without testing them.
__device__ __forceinline__ int decide_node(const TreeDev &T, const WalkGroup &W, int32_t nd, const WNode &w,
                                           int &namb, bool &allin)
{
    const uint64_t T_lo = W.P->T_lo, T_hi = W.P->T_hi;
    const uint32_t ax = absdiff32(w.cx, W.gx), ay = absdiff32(w.cy, W.gy), az = absdiff32(w.cz, W.gz);
    const uint64_t sx = (uint64_t)w.hx + W.hx, sy = (uint64_t)w.hy + W.hy, sz = (uint64_t)w.hz + W.hz;
    const uint64_t dx = ax > sx ? ax - sx : 0, dy = ay > sy ? ay - sy : 0, dz = az > sz ? az - sz : 0;
    const uint64_t gap2 = sq32(dx) + sq32(dy) + sq32(dz);
    bool exact = false;
    double gap2d = 0.0, far2d = 0.0;
    allin = false;
    if (gap2 >= T_hi) return kPrune;
    if (gap2 >= T_lo) {
        exact = true;
        namb++;
        gap2d = exact_dist2(T.cenx[nd], T.ceny[nd], T.cenz[nd], T.hfx[nd], T.hfy[nd], T.hfz[nd], T.gcx[W.g],
                            T.gcy[W.g], T.gcz[W.g], T.ghx[W.g], T.ghy[W.g], T.ghz[W.g], &far2d);
        if (gap2d >= W.P->rc2) return kPrune;
    }
    const uint64_t fx = ax + sx, fy = ay + sy, fz = az + sz;
    const uint64_t far2 = ((fx | fy | fz) >> 31) ? ~0ull : sq32(fx) + sq32(fy) + sq32(fz);
    allin = !exact && far2 < T_lo;
    const bool overlap = w.first < W.g1 && W.g0 < w.first + w.count;
    if (overlap) return kOpen;
    if (!exact) {
        const int A = far2 < T_lo ? 1 : (far2 >= T_hi ? 0 : -1);
        const int B = gap2 >= W.P->TB_hi[w.level] ? 1 : (gap2 < W.P->TB_lo[w.level] ? 0 : -1);
        if (A == 0 || B == 0) return kOpen;
        if (A == 1 && B == 1) return kAccept;
        namb++;
        gap2d = exact_dist2(T.cenx[nd], T.ceny[nd], T.cenz[nd], T.hfx[nd], T.hfy[nd], T.hfz[nd], T.gcx[W.g],
                            T.gcy[W.g], T.gcz[W.g], T.ghx[W.g], T.ghy[W.g], T.ghz[W.g], &far2d);
    }
    const double l = ldexp(1.0, -w.level);
    return far2d < W.P->rc2 && __dmul_rn(l, l) < __dmul_rn(W.P->th2, gap2d) ? kAccept : kOpen;
}

// Whether particle p of an opened leaf enters the list: point-to-box gap < r_cut.
__device__ __forceinline__ bool keep_particle(const TreeDev &T, const WalkGroup &W, int32_t p, int &namb)
{
    const uint4 q = T.P32[p];
    const uint32_t qx = absdiff32(q.x, W.gx), qy = absdiff32(q.y, W.gy), qz = absdiff32(q.z, W.gz);
    const uint64_t ex = qx > W.hx ? qx - W.hx : 0, ey = qy > W.hy ? qy - W.hy : 0, ez = qz > W.hz ? qz - W.hz : 0;
    const uint64_t p2 = sq32(ex) + sq32(ey) + sq32(ez);
    if (p2 >= W.P->T_hi) return false;
    if (p2 < W.P->T_lo) return true;
    namb++;
    double f2;
    return exact_dist2(T.x[p], T.y[p], T.z[p], 0.0, 0.0, 0.0, T.gcx[W.g], T.gcy[W.g], T.gcz[W.g], T.ghx[W.g],
                       T.ghy[W.g], T.ghz[W.g], &f2) < W.P->rc2;
}

// Top walk of one group, depth first from the box root without a stack (skip
// pointers).  Returns the number of items; with out != nullptr writes them to
// out[0 .. out_n).
__device__ int32_t walk_top(const TreeDev &T, const WalkGroup &W, int32_t start, int32_t split, int32_t *out,
                            int64_t out_n, unsigned long long &ambig, int64_t *slots = nullptr)
{
    int32_t cnt = 0;
    int32_t nd = start;
    // a preorder walk visits each node at most once
    int64_t budget = T.walk_budget > 0 ? T.walk_budget : *T.n_nodes + 1;
    while (nd >= 0) {
        if (--budget < 0 || nd >= T.cap_nodes) {
            tp_latch(T.status, TP_ERR_TIMEOUT);
            break;
        }
        const WNode w = T.wn[nd];
        int namb = 0;
        bool allin;
        const int d = decide_node(T, W, nd, w, namb, allin);
        ambig += namb;
        if (d == kPrune) {
            nd = w.skip;
        } else if (d == kAccept) {
            if (out && cnt < out_n) out[cnt] = -(nd + 1);
            cnt++;
            if (slots) *slots += 1;
            nd = w.skip;
        } else if (w.child < 0 || w.count <= split) {
            if (out && cnt < out_n) out[cnt] = nd;       // a task: expand its subtree later
            cnt++;
            if (slots) *slots += w.count;
            nd = w.skip;
        } else {
            nd = w.child;
        }
    }
    return cnt;
}

// Top walk of every group: item counts, and the first kscr items in the
// group's scratch (WRITE = false); or the items at their offsets (WRITE =
// true), copied from the scratch when it holds them all, else walked again.
template <bool WRITE>
__global__ void __launch_bounds__(kBlock) k_walk_top(TreeDev T, int32_t split)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    if (WRITE && *T.status == TP_ERR_LIST_OVERFLOW) return;
    unsigned long long ambig = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        if (!WRITE) {
            const WalkGroup W = load_walk_group(T, g);
            int64_t slots = 0;
            T.icnt[g] = walk_top(T, W, T.gbox[g], split, T.iscr + g * T.kscr, T.kscr, ambig, &slots);
            T.gpad[g] = slots < 0x7fffffff ? (int32_t)slots : 0x7fffffff;
        } else {
            const int64_t o = T.ioff[g];
            const int64_t n = T.icnt[g];
            if (o + n > T.cap_items) continue;
            if (n <= T.kscr) {                      // the count pass kept them all
                const int32_t *src = T.iscr + g * T.kscr;
                for (int64_t k = 0; k < n; k++) T.item[o + k] = src[k];
            } else {
                walk_top(T, load_walk_group(T, g), T.gbox[g], split, T.item + o, n, ambig);
            }
            for (int64_t k = 0; k < n; k++) T.igrp[o + k] = (int32_t)g;
        }
    }
    if (!WRITE && ambig) atomicAdd(T.n_ambig, ambig);
}

// Slots per item: a task expands to at most one entry per particle of its
// subtree (every entry covers at least one distinct particle), a monopole item
// to one entry.
__global__ void k_item_bounds(TreeDev T)
{
    const int64_t NI = *T.n_items < T.cap_items ? *T.n_items : T.cap_items;
    for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < NI;
         it += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = T.item[it];
        T.ibound[it] = v < 0 ? 1 : T.wn[v].count;
    }
}

// Expansion of every item into its padded slots; records the entry count.
// Each lane expands one item at a time by a stackless depth-first walk of the
// task's subtree and takes its next item from a global counter as soon as it
// is done, so lanes with short tasks do not wait for the warp's longest one.
// Every loop iteration makes one node decision per lane; the particles of the
// leaves opened in it are then tested by the whole warp, 32 per round (see
// below), so particle tests do not wait on the lanes that own them.  Each
// lane's group record sits in shared memory, where the testing lanes read
// their owner's, the ambiguous-decision count is a block counter and the
// item and budget are 32-bit: the kernel fits 56 registers, nine blocks per
// SM (measured 5 % faster than 72 registers and seven blocks; 12 bytes spill).
__global__ void __launch_bounds__(kBlock, 9) k_walk_task(TreeDev T, unsigned long long *counter)
{
    const int64_t NI = *T.n_items < T.cap_items ? *T.n_items : T.cap_items;
    if (*T.n_pad > T.cap_pad || *T.status == TP_ERR_LIST_OVERFLOW) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    __shared__ unsigned long long s_ambig;  // decisions that took the FP64 test, for the block
    if (threadIdx.x == 0) s_ambig = 0;
    __syncthreads();
    int32_t it = -1;                       // the lane's item (item counts fit 31 bits); -1 none
    bool exhausted = false;
    __shared__ WalkGroup sW[kBlock];       // each lane's group, read by the lanes testing its particles
    int32_t *out = nullptr;
    int32_t nd = -1, end = -1, pcur = 0, pend = 0, cnt = 0, bound = 0;
    bool pall = false;                     // the pending particles need no test
    int32_t budget = 0;                    // node visits left (the bound below 2^31)
    for (;;) {
        __syncwarp();                      // the last round's reads of sW before new items overwrite it
        const unsigned nm = __ballot_sync(full, it < 0 && !exhausted);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(nm));
            base = __shfl_sync(full, base, leader);
            if (it < 0 && !exhausted) {
                // two sweeps over the items: tasks of more than kBigTask
                // particles first, then the rest, so that no long task starts
                // near the end of the launch
                const int64_t cand = (int64_t)base + __popc(nm & below);
                const int64_t c = cand < NI ? cand : cand - NI;
                if (cand < 2 * NI && (cand < NI) != (T.ibound[c] > kBigTask)) {
                    // this sweep leaves the item to the other one
                } else if (cand < 2 * NI) {
                    it = (int32_t)c;
                    const int32_t v = T.item[it];
                    out = T.pent + T.ibpos[it];
                    if (v < 0) {                       // an accepted monopole
                        out[0] = v;
                        T.icnt2[it] = 1;
                        it = -1;
                    } else {
                        sW[threadIdx.x] = load_walk_group(T, T.igrp[it]);
                        nd = v;
                        end = T.wn[v].skip;
                        pcur = pend = 0;
                        cnt = 0;
                        bound = T.ibound[it];
                        const int64_t b64 = T.walk_budget > 0 ? T.walk_budget : *T.n_nodes + 1;
                        budget = b64 < 0x7fffffff ? (int32_t)b64 : 0x7fffffff;
                    }
                } else {
                    exhausted = true;
                }
            }
        }
        if (__all_sync(full, exhausted)) break;
        if (it >= 0) {
            if (nd == end || nd < 0 || --budget < 0 || nd >= T.cap_nodes) {
                if (budget < 0 || (nd != end && nd >= T.cap_nodes)) tp_latch(T.status, TP_ERR_TIMEOUT);
                if (cnt > bound) tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
                T.icnt2[it] = cnt;
                it = -1;
            } else {                                   // one node decision
                const WNode w = T.wn[nd];
                int namb = 0;
                bool allin;
                const int d = decide_node(T, sW[threadIdx.x], nd, w, namb, allin);
                if (namb) atomicAdd(&s_ambig, (unsigned long long)namb);
                if (d == kPrune) {
                    nd = w.skip;
                } else if (d == kAccept) {
                    if (cnt < bound) out[cnt] = -(nd + 1);
                    cnt++;
                    nd = w.skip;
                } else if (w.child < 0) {              // an opened leaf: its particles enter below,
                    pcur = w.first;                    // untested when it lies wholly within r_cut
                    pend = w.first + w.count;
                    pall = allin;
                    nd = w.skip;
                } else {
                    nd = w.child;
                }
            }
        }
        // The particles of the leaves opened above, tested by the whole warp,
        // 32 at a time: lane k takes the k-th pending particle in lane order
        // and its owner's group from shared memory; a ballot ranks the kept ones
        // within each owner, which writes them in particle order after its
        // entries so far (the list order of a lane-by-lane walk).  The
        // particles of a leaf wholly within r_cut are kept without a test, in
        // the same rounds, so that no lane writes a leaf alone.
        for (;;) {
            const bool has = it >= 0 && pcur < pend;
            if (!__ballot_sync(full, has)) break;
            const int32_t mine = has ? pend - pcur : 0;
            int32_t incl = mine;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += y;
            }
            const int32_t start = incl - mine;
            const int32_t total = __shfl_sync(full, incl, 31);
            int j = 0;                                 // owner of slot `lane`: first lane with incl > lane
            for (int st = 16; st > 0; st >>= 1)
                if (__shfl_sync(full, incl, j + st - 1) <= lane) j += st;
            j &= 31;
            __syncwarp();
            const WalkGroup &Wj = sW[(threadIdx.x & ~31u) + j];
            const int32_t sj = __shfl_sync(full, start, j), pj = __shfl_sync(full, pcur, j);
            const int32_t cj = __shfl_sync(full, cnt, j), bj = __shfl_sync(full, bound, j);
            int32_t *oj = reinterpret_cast<int32_t *>(
                __shfl_sync(full, reinterpret_cast<unsigned long long>(out), j));
            const bool tester = lane < total, aj = __shfl_sync(full, pall, j);
            const int32_t p = pj + (lane - sj);
            int namb = 0;
            const bool keep = tester && (aj || keep_particle(T, Wj, p, namb));
            if (namb) atomicAdd(&s_ambig, (unsigned long long)namb);
            const unsigned kept = __ballot_sync(full, keep);
            if (keep) {
                const unsigned lo = sj > 0 ? ~((1u << sj) - 1u) : full;
                const int32_t pos = cj + __popc(kept & lo & below);
                if (pos < bj) oj[pos] = p;
            }
            if (has && start < 32) {                   // this lane's share of the round
                const int32_t e = incl < 32 ? incl : 32;
                const unsigned hi = e >= 32 ? full : ((1u << e) - 1u);
                const unsigned lo = ~((1u << start) - 1u);
                cnt += __popc(kept & hi & lo);
                pcur += e - start;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_ambig) atomicAdd(T.n_ambig, s_ambig);
}

// Compaction of the padded slots into the lists: one warp per item.
// Compaction of the padded slots into the lists, with each entry's record.
// A warp takes 32 consecutive items (lane l holds item base + l); their
// entries are contiguous in the output, so the warp writes them as one run and
// finds each entry's item by a binary search over the lanes' running counts.
// The kernel waits on its gathers; capped at 40 registers it holds six
// blocks per SM instead of five (measured 0.1 ms faster at 2M).
__global__ void __launch_bounds__(256, 6) k_compact(TreeDev T)
{
    const int64_t NI = *T.n_items < T.cap_items ? *T.n_items : T.cap_items;
    if (*T.n_entries > T.cap_entries || *T.status == TP_ERR_LIST_OVERFLOW) return;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = 32 * w0; base < NI; base += 32 * nw) {
        const int64_t it = base + lane;
        const bool v = it < NI;
        const int32_t cnt = v ? T.icnt2[it] : 0;
        int32_t incl = cnt;                           // inclusive running count over the lanes
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        const int32_t total = __shfl_sync(full, incl, 31);
        const int64_t out0 = __shfl_sync(full, v ? T.ipos[it] : 0, 0);
        const int64_t sbase = v ? T.ibpos[it] - (incl - cnt) : 0;
        const int32_t g = v ? T.igrp[it] : 0;
        const float sc = v ? T.box[T.gbox[g]].scale : 0.f;
        // two entries per lane and round (k and k + 32), so that two chains of
        // dependent loads (slot, then source record) are in flight at once
        for (int32_t k0 = 0; k0 < total; k0 += 64) {
            const int32_t ka = k0 + lane, kb = ka + 32;
            int ja = 0, jb = 0;                       // lanes whose running count is <= k
            for (int st = 16; st > 0; st >>= 1) {
                const int32_t ya = __shfl_sync(full, incl, ja + st - 1);
                const int32_t yb = __shfl_sync(full, incl, jb + st - 1);
                if (ya <= ka) ja += st;
                if (yb <= kb) jb += st;
            }
            jb &= 31;
            const int64_t sba = __shfl_sync(full, sbase, ja), sbb = __shfl_sync(full, sbase, jb);
            const int32_t ga = __shfl_sync(full, g, ja), gb = __shfl_sync(full, g, jb);
            const float sca = __shfl_sync(full, sc, ja), scb = __shfl_sync(full, sc, jb);
            const bool va = ka < total, vb = kb < total;
            const int32_t ea = va ? T.pent[sba + ka] : 0;
            const int32_t eb = vb ? T.pent[sbb + kb] : 0;
            if (va) {
                T.ent[out0 + ka] = ea;
                T.rec[out0 + ka] = entry_record(T, T.gX[ga], T.gY[ga], T.gZ[ga], sca, ea);
            }
            if (vb) {
                T.ent[out0 + kb] = eb;
                T.rec[out0 + kb] = entry_record(T, T.gX[gb], T.gY[gb], T.gZ[gb], scb, eb);
            }
        }
    }
}

// Refit: the records of the kept lists from the new particle images and
// node centres of mass, against the same group centres (a warp per group).
__global__ void k_refit_records(TreeDev T)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    if (*T.n_entries > T.cap_entries) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = w0; g < G; g += nw) {
        const int64_t e0 = T.loff[g];
        const int32_t ne = T.lcnt[g];
        const uint64_t GX = T.gX[g], GY = T.gY[g], GZ = T.gZ[g];
        const float sc = T.box[T.gbox[g]].scale;
        for (int32_t k = lane; k < ne; k += 32) T.rec[e0 + k] = entry_record(T, GX, GY, GZ, sc, T.ent[e0 + k]);
    }
}

// The sort key of a work item of pair count c: the upper 16 bits of the FP32
// value of c (exponent and 7 mantissa bits; monotone in c), complemented, so
// that a two-pass sort puts the items in descending order of c to within 1 %,
// which is all the queue's balance needs.  Keys lie in [0x3000, 0x7fff];
// padding takes 0x8000 (unused groups) or 0xffff (unused extra slots).
__device__ __forceinline__ uint64_t lpt_key(uint64_t c)
{
    return (uint64_t)(0x7fffu - (__float_as_uint((float)c) >> 16));
}

// LPT keys for the persistent work queue: work items in descending order of
// their pair count n_i * n_j (ties by slot, the sort is stable).  A group's
// first kWorkChunk particles are the item in its own slot g; each further
// chunk of a larger group takes a slot past cap_groups and a {group, chunk}
// entry of the table T.xitem (slots handed out by an atomic counter: the
// order of equal keys there varies, the items' results do not).  The extra
// slots beyond the counter keep the padding key their memset gave them.
__global__ void k_lpt_keys(TreeDev T, uint64_t *key, uint32_t *val)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < T.cap_groups;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ni = g < G ? T.gcount[g] : 0;
        const uint64_t cost = g < G ? (uint64_t)(ni < kWorkChunk ? ni : kWorkChunk) * (uint64_t)T.lcnt[g] : 0;
        key[g] = g < G ? lpt_key(cost) : 0x8000ull;                   // padding sorts last
        val[g] = (uint32_t)g;
        if (g < G) {
            for (int c = 1; c * kWorkChunk < ni; c++) {
                const unsigned long long k = atomicAdd(reinterpret_cast<unsigned long long *>(T.n_xitems), 1ull);
                if ((int64_t)k >= T.cap_xitems) {               // cannot happen: cap_xitems >= n / kWorkChunk
                    tp_latch(T.status, TP_ERR_LIST_OVERFLOW);
                    break;
                }
                const int32_t nc = ni - c * kWorkChunk < kWorkChunk ? ni - c * kWorkChunk : kWorkChunk;
                key[T.cap_groups + k] = lpt_key((uint64_t)nc * (uint64_t)T.lcnt[g]);
                val[T.cap_groups + k] = (uint32_t)(T.cap_groups + k);
                T.xitem[k] = make_int2((int)g, c);
            }
            // groups whose pairs the packed FP32 kernels leave to the general ones:
            // offsets that may need the minimum image per pair, or eps = 0
            const BoxPrm &P = T.box[T.gbox[g]];
            const double hm = fmax(T.ghx[g], fmax(T.ghy[g], T.ghz[g]));
            if (2.0 * hm + P.rcut >= 0.5 - 1e-9 || !(P.eps2s > 0.f)) atomicAdd(T.n_general, 1ull);
        }
    }
}

// Per-group list offsets and counts from the item positions.
__global__ void k_list_offsets(TreeDev T)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    const int64_t NI = *T.n_items < T.cap_items ? *T.n_items : T.cap_items;
    const int64_t E = *T.n_entries;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = T.ioff[g];
        const int64_t i1 = g + 1 < G ? T.ioff[g + 1] : NI;
        const int64_t e0 = i0 < NI ? T.ipos[i0] : E;
        const int64_t e1 = i1 < NI ? T.ipos[i1] : E;
        T.loff[g] = e0;
        T.lcnt[g] = (int32_t)(e1 - e0);
    }
}

__global__ void k_list_stats(TreeDev T, unsigned long long *inter, int32_t *max_nj)
{
    const int64_t G = *T.n_groups < T.cap_groups ? *T.n_groups : T.cap_groups;
    unsigned long long s = 0;
    int32_t mx = 0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < G;
         g += (int64_t)gridDim.x * blockDim.x) {
        s += (unsigned long long)T.gcount[g] * (unsigned long long)T.lcnt[g];
        mx = max(mx, T.lcnt[g]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(inter, s);
        atomicMax(max_nj, mx);
    }
}

}  // namespace

namespace tp {

// Item counts per group -> T.ioff (scan) -> *T.n_items.
void walk_top_count(TreeDev &T, int32_t split, void *scan_tmp, cudaStream_t s)
{
    if (T.cap_groups <= 0) return;
    TP_LAUNCH(k_walk_top<false>, grid_for(T.cap_groups, kBlock), kBlock, 0, s, T, split);
    scan_i32_to_i64(T.icnt, T.ioff, 0, T.n_groups, T.n_items, scan_tmp, s);
}

// Item offsets of the groups from their counts (already in T.icnt).
void walk_top_scan(TreeDev &T, void *scan_tmp, cudaStream_t s)
{
    if (T.cap_groups <= 0) return;
    scan_i32_to_i64(T.icnt, T.ioff, 0, T.n_groups, T.n_items, scan_tmp, s);
}

// Items and their padded slot positions (scan) -> *T.n_pad.
void walk_items(TreeDev &T, int32_t split, void *scan_tmp, cudaStream_t s)
{
    if (T.cap_groups <= 0 || T.cap_items <= 0) return;
    TP_LAUNCH(k_walk_top<true>, grid_for(T.cap_groups, kBlock), kBlock, 0, s, T, split);
    TP_LAUNCH(k_item_bounds, grid_for(T.cap_items, 256), 256, 0, s, T);
    scan_i32_to_i64(T.ibound, T.ibpos, 0, T.n_items, T.n_pad, scan_tmp, s);
}

// Task expansion into the padded slots, entry positions (scan) -> *T.n_entries.
void walk_expand(TreeDev &T, unsigned long long *counter, void *scan_tmp, cudaStream_t s)
{
    if (T.cap_items <= 0) return;
    static const int bps = occupancy(k_walk_task, kBlock);   // once per process, never inside a capture
    cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    TP_LAUNCH(k_walk_task, num_sms() * bps, kBlock, 0, s, T, counter);
    scan_i32_to_i64(T.icnt2, T.ipos, 0, T.n_items, T.n_entries, scan_tmp, s);
    TP_LAUNCH(k_list_offsets, grid_for(T.cap_groups, 256), 256, 0, s, T);
}

void refit_records(TreeDev &T, cudaStream_t s)
{
    if (T.cap_groups <= 0) return;
    TP_LAUNCH(k_refit_records, grid_for(32 * T.cap_groups, 256), 256, 0, s, T);
}

void walk_write(TreeDev &T, cudaStream_t s)
{
    if (T.cap_items <= 0) return;
    TP_LAUNCH(k_compact, grid_for(T.cap_items, 256), 256, 0, s, T);
}

// order[] = work items by descending cost; key/val/key2/val2 hold
// cap_groups + cap_xitems each.
void lpt_order(TreeDev &T, uint64_t *key, uint32_t *val, uint64_t *key2, uint32_t *val2,
               void *radix_tmp, cudaStream_t s)
{
    if (T.cap_groups <= 0) return;
    cudaMemsetAsync(T.n_general, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(T.n_xitems, 0, sizeof(int64_t), s);
    if (T.cap_xitems > 0) cudaMemsetAsync(key + T.cap_groups, 0xff, sizeof(uint64_t) * (size_t)T.cap_xitems, s);
    TP_LAUNCH(k_lpt_keys, grid_for(T.cap_groups, 256), 256, 0, s, T, key, val);
    radix_sort(key, val, key2, val2, T.cap_groups + T.cap_xitems, 16, nullptr, 1, radix_tmp, s);
}

void list_stats(TreeDev &T, unsigned long long *inter, int32_t *max_nj, cudaStream_t s)
{
    TP_LAUNCH(k_list_stats, 152 * 2, 256, 0, s, T, inter, max_nj);
}

}  // namespace tp
